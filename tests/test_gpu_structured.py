"""Structured updates on the GPU against the oracle: a CP term's sketches
(ttnn_update_cp) equal the oracle's sketches of the dense CP tensor, taken
with the plan's stored DRM factors and exact Khatri-Rao products (no second
rounding of pass-side blocks, Sec. 7).  All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

FMT = {api.F64: "f64", api.F32: "f32", api.BF16: "bf16"}
# binary64 state: summation order only; binary32 state: one rounding per entry
TOL = {api.F64: 1e-12, api.F32: 2e-6, api.BF16: 2e-6}

CASES = {
    "binary4": (W.balanced_binary(4), [7, 5, 6, 4], 3, 2),
    "toy6": (W.toy_tree(), [3, 4, 3, 5, 4, 3], 2, 2),
    "tt5": (W.tensor_train(5), [4, 3, 5, 3, 4], 2, 1),
    "tucker4": (W.tucker(4), [5, 4, 6, 3], 2, 2),
    "binary5": (W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2),
}


def _otree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def _oracle_sketch(tr, dims, r, p, seed, fmt, T):
    t = _otree(tr, dims, r, p)
    return O.sketch_ttnn(T, t, O.Drm(t, seed, fmt, "round"))


def _compare(run, want, tol):
    Om, Ps, Pr = run.sketches()
    WOm, WPs, WPr = want
    for v in WOm:
        assert rel(Om[v], WOm[v]) <= tol, ("Omega", v, rel(Om[v], WOm[v]))
        assert rel(Ps[v], WPs[v]) <= tol, ("Psi", v, rel(Ps[v], WPs[v]))
    assert rel(Pr, WPr) <= tol, ("Psi_root", rel(Pr, WPr))


@pytest.mark.parametrize("dtype", [api.F64, api.F32, api.BF16])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cp_update_matches_oracle(case, dtype):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    rng = np.random.default_rng(11)
    w, f = W.cp_term(dims, 3, rng)
    w = np.array([1.5, -0.5, 2.0])
    run = Run(tr, dims, [r] * n, [p] * n, 99, dtype=dtype)
    try:
        fd = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]
        api.ttnn_update_cp(run.state, list(w), fd, lam=0.75)
        want = _oracle_sketch(tr, dims, r, p, 99, FMT[dtype], 0.75 * W.cp_dense(w, f))
        _compare(run, want, TOL[dtype])
    finally:
        run.close()


def test_cp_update_many_ranks_and_accumulation():
    # rank 37 spans three rank chunks; two updates accumulate (linearity)
    tr, dims, r, p = CASES["toy6"]
    n = len(tr[0])
    rng = np.random.default_rng(5)
    w1, f1 = W.cp_term(dims, 37, rng)
    w1 = rng.standard_normal(37)
    w2, f2 = W.cp_term(dims, 2, rng)
    run = Run(tr, dims, [r] * n, [p] * n, 3, dtype=api.F64)
    try:
        for w, f, lam in ((w1, f1, 1.0), (w2, f2, -2.0)):
            fd = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]
            api.ttnn_update_cp(run.state, list(w), fd, lam=lam)
        T = W.cp_dense(w1, f1) - 2.0 * W.cp_dense(w2, f2)
        _compare(run, _oracle_sketch(tr, dims, r, p, 3, "f64", T), 1e-12)
    finally:
        run.close()


def test_cp_plus_dense_box_then_recover():
    # the streamed workload in miniature: CP terms and dense boxes into one
    # state, then recovery; F64 plan, exact-rank data plus the box noise
    tr = W.tensor_train(5)
    dims = [5, 4, 6, 4, 5]
    n = len(tr[0])
    run = Run(tr, dims, [4] * n, [2] * n, 8, dtype=api.F64)
    try:
        rng = np.random.default_rng(1)
        T = np.zeros(dims)
        for _ in range(3):
            w, f = W.cp_term(dims, 2, rng)
            fd = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]
            api.ttnn_update_cp(run.state, list(w), fd)
            T += W.cp_dense(w, f)
            off, ext, data = W.box_update(dims, [0, 2, 4], 3, rng, sigma=0.01)
            api.ttnn_update_dense(run.state, torch.from_numpy(np.ascontiguousarray(data)).cuda(),
                                  off, ext)
            T += W.embed_box(dims, off, ext, data)
        t = _otree(tr, dims, 4, 2)
        Om, Ps, Pr = O.sketch_ttnn(T, t, O.Drm(t, 8, "f64"))
        _compare(run, (Om, Ps, Pr), 1e-11)
        got = O.reconstruct(t, run.recover())
        want = O.reconstruct(t, O.recover(t, Om, Ps, Pr)[0])
        assert rel(got, want) <= 1e-9
    finally:
        run.close()


def test_cp_update_rejects_sttnn_and_bad_args():
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    rng = np.random.default_rng(2)
    w, f = W.cp_term(dims, 2, rng)
    fd = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in f]
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.F32, variant=api.VARIANT_STTNN)
    try:
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_cp(run.state, list(w), fd)
        assert ei.value.status == 7
        assert not np.any(run.state_host())
    finally:
        run.close()
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.F32)
    try:
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_cp(run.state, [1.0, float("nan")], fd)
        assert ei.value.status == 1
        assert not np.any(run.state_host())
    finally:
        run.close()


# ---------------------------------------------------------------------------
# TTN-format input (ttnn_update_ttn / ttnn_round)
# ---------------------------------------------------------------------------
from oracle import rounding as OR  # noqa: E402

TTN_TOL = {api.F64: 1e-12, api.F32: 1e-5, api.BF16: 1e-5}


def _ttn_input(tr, dims, R, seed):
    rng = np.random.default_rng(seed)
    n = len(tr[0])
    return W.ttn_cores(tr, dims, [R] * n, rng)


def _dev_cores(cores):
    return [torch.from_numpy(np.ascontiguousarray(cores[v])).cuda() for v in range(len(cores))]


@pytest.mark.parametrize("dtype", [api.F64, api.F32, api.BF16])
@pytest.mark.parametrize("case", sorted(CASES))
def test_ttn_update_matches_oracle(case, dtype):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    cores = _ttn_input(tr, dims, 3, 21)
    run = Run(tr, dims, [r] * n, [p] * n, 42, dtype=dtype)
    try:
        api.ttnn_update_ttn(run.state, _dev_cores(cores), [3] * n, lam=-1.25)
        t = _otree(tr, dims, r, p)
        Om, Ps, Pr = OR.sketch_ttn_input(cores, t, O.Drm(t, 42, FMT[dtype], "round"))
        want = ({v: -1.25 * x for v, x in Om.items()}, {v: -1.25 * x for v, x in Ps.items()},
                -1.25 * Pr)
        _compare(run, want, TTN_TOL[dtype])
    finally:
        run.close()


def test_ttn_update_equals_dense_update_f64():
    # binary64 plans: the structured sketch of a TTN equals the dense pass over
    # its full tensor (same DRMs, no rounding anywhere)
    tr, dims, r, p = CASES["binary5"]
    n = len(tr[0])
    cores = _ttn_input(tr, dims, 4, 3)
    a = Run(tr, dims, [r] * n, [p] * n, 7, dtype=api.F64)
    b = Run(tr, dims, [r] * n, [p] * n, 7, dtype=api.F64)
    try:
        api.ttnn_update_ttn(a.state, _dev_cores(cores), [4] * n)
        dense = torch.from_numpy(np.ascontiguousarray(W.ttn_dense(tr, cores))).cuda()
        api.ttnn_update_dense(b.state, dense)
        assert rel(a.state_host(), b.state_host()) <= 1e-12
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("case", ["toy6", "tt5", "binary5"])
def test_ttn_round_end_to_end(case):
    # rounding an exact-rank TTN whose ranks exceed the targets' true ranks
    # only by zero padding: recovery reproduces the tensor
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    t = _otree(tr, dims, r, p)
    rng = np.random.default_rng(4)
    small = W.ttn_cores(tr, dims, [2] * n, rng)
    T = W.ttn_dense(tr, small)
    # pad every edge rank from 2 to 5 with zeros: same tensor, larger input ranks
    big = {}
    ch, _ = W.children_of(tr[0], tr[1])
    for v in range(n):
        c = small[v]
        pad = [(0, 3)] * c.ndim
        if not ch[v]:
            pad[1:] = [(0, 0)] * (c.ndim - 1)
        big[v] = np.pad(c, pad)
    run = Run(tr, dims, [r] * n, [p] * n, 17, dtype=api.F64, flags=api.FLAG_STRUCTURED_ONLY)
    try:
        out = torch.zeros(run.sizes[2], dtype=torch.float64, device="cuda")
        api.ttnn_round(run.plan, _dev_cores(big), [5] * n, out)
        host = out.cpu().numpy()
        nodes = [api.ttnn_plan_node(run.plan, v) for v in range(n)]
        got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
               .reshape(nd["core_shape"]) for nd in nodes}
        assert rel(O.reconstruct(t, got), T) <= 1e-10
        # and the oracle's rounding of the same input agrees
        sk = OR.sketch_ttn_input(big, t, O.Drm(t, 17, "f64", "round"))
        assert rel(O.reconstruct(t, O.recover(t, *sk)[0]), T) <= 1e-10
    finally:
        run.close()


def test_structured_only_plan_rejects_dense_and_sttnn_rejects_ttn():
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.F32, flags=api.FLAG_STRUCTURED_ONLY)
    try:
        dense = torch.zeros(dims, dtype=torch.float32, device="cuda")
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_dense(run.state, dense)
        assert ei.value.status == 7
    finally:
        run.close()
    cores = _ttn_input(tr, dims, 2, 1)
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.F32, variant=api.VARIANT_STTNN)
    try:
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_ttn(run.state, _dev_cores(cores), [2] * n)
        assert ei.value.status == 7
    finally:
        run.close()
