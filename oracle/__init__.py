"""Plain FP64 CPU oracle for tree tensor network Nystrom (TTNN / STTNN).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (``paper_2412_06111_gb300``) and never
imports it.

Every function follows a passage of Bucci & Verzella, "Randomized algorithms
for streaming low-rank approximation in tree tensor network format"
(arXiv:2412.06111) and is written for a reader to check against the paper by
eye: sketches are formed as products with explicitly materialised Khatri-Rao
/ Kronecker matrices, recovery follows the recovery phase of Sec. 4 step by
step, and library primitives (QR, SVD, matmul) are used only as single steps.

Modules
-------
philox     Philox4x32-10 counter generator and the Gaussian transform (DRMs).
quant      Round-to-nearest-even into fp32 / bf16 / fp8-e4m3 value sets.
tree       Index tree, normalisation, lexicographic order, STTNN reuse sets.
ttnn       DRMs, TTNN sketches, recovery, reconstruction, projector form.
sttnn      STTNN sketches (Sec. 5).
rounding   Sketches of a tensor given in TTN format (Sec. 7).
baselines  HOSVD / TT-SVD / TTN-SVD truncations, GN, MLN, STTA.
bounds     Deterministic (Thm 6.4, 6.7) and expected (Thm 6.6) error bounds.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values fixed by the paper or by mathematics (see each module).
"""
