"""The C-ABI library builds for sm_103a, loads, exports every entry point
that include/ttnn.h declares, and rejects invalid plans before touching a GPU."""
import os
import re

import pytest

from paper_2412_06111_gb300 import _native, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ttnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:ttnn|sttnn)_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ["ttnn_plan_create", "ttnn_update_dense", "ttnn_recover", "sttnn_run", "ttnn_round",
              "ttnn_philox_gaussian", "ttnn_update_cp", "ttnn_update_ttn"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) <= set(__import__("paper_2412_06111_gb300._sigs", fromlist=["SIGS"]).SIGS)


def test_status_strings():
    lib = _native.load()
    assert lib.ttnn_status_string(0) == b"ok"
    assert lib.ttnn_status_string(1) == b"invalid argument"


@pytest.mark.parametrize("parent,leaf_modes,ident,dims,msg", [
    ([-1, 0, 0], [[], [0, 2], [1]], None, [3, 3, 3], "contiguous"),
    ([-1, 0], [[], [0, 1]], None, [3, 3], "2 children"),
    ([-1, -1, 0], [[], [0], [1]], None, [3, 3], "root"),
    ([-1, 0, 0], [[], [0], [0]], None, [3, 3], "partition"),
    ([-1, 0, 0], [[], [0], [1]], [1, 0, 0], [3, 3], "identity"),
    ([-1, 0, 0], [[], [0], [1]], None, [3, 0], "mode size"),
])
def test_invalid_trees_rejected_on_host(parent, leaf_modes, ident, dims, msg):
    with pytest.raises(api.TtnnError, match=msg) as ei:
        api.ttnn_plan_create((parent, leaf_modes, ident), dims,
                             [2] * len(parent), [1] * len(parent), 1, stream=0)
    assert ei.value.status == 1


def test_bad_ranks_rejected_on_host():
    with pytest.raises(api.TtnnError) as ei:
        api.ttnn_plan_create(([-1, 0, 0], [[], [0], [1]], None), [4, 4], [0, 0, 2], [1, 1, 1], 1,
                             stream=0)
    assert ei.value.status == 1
