"""CPU oracle for AlgMortar-PCG (arxiv 2607.22905) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 numpy/scipy restatement of what the GPU path computes, written from
the paper and kept independent of it: it shares no code, tables or helpers with
`paper_2607_22905_b300` and never imports it.  Only the test suite, the smoke check
in `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import or call
anything in this package; the product path must never route through it.

Modules
-------
partition  deterministic recursive graph bisection of the matrix graph (Sec. 3.1)
algmortar  operators of Sec. 3.2, local systems Eq. (A_i), MBFs Eq. (def-phat-local),
           interface problem Eq. (interface-problem-alg), Algorithms 1 and 2, the dense
           reduced preconditioner of Eq. (eq-m-reduced-p), and PCG (Sec. 7)
adjoint    hand-derived gradient of an observation misfit through the TPFA solve
           (not in the paper; the adjoint A lambda = g of the same SPD system)

Every function is pinned by tests/test_oracle_*.py against identities and closed forms
the paper and the mathematics fix (Prop. BWM, Lemmas, Thm. Q-psd, Cor. cor-schur-p,
Prop. bound-eigenvalues, Sec. 5.4 residual structure, Remark tpfa-local-dirichlet,
exact recovery for Lambda = R^E), brute force on tiny inputs and central finite
differences.  Iteration counts of the paper's tables are parity unpinned: they need the
SPE10/SPE11 data, METIS partitions and smoothing, none of which exist here.
"""
