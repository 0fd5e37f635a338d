"""Floating-point bars shared by the parity tests.

VAL_TOL: FP64 hierarchy values computed from identical inputs (one step of
the setup on both sides) agree within 1e-12 of the row's largest magnitude;
the CUDA path sums in other orders (parallel reductions in the power method,
hash-ordered SpGEMM rows are re-sorted but products are the same), which
costs a few units in the last place per operation.

chain_tol(l): the CUDA hierarchy compared with the oracle's own hierarchy at
depth l inherits every earlier level's last-bit differences.  The oracle
itself moves by up to ~2e-12 at level 3 when the fine matrix is perturbed by
one unit in the last place (test_chain_sensitivity), so chained comparisons
get 1e-12 * 4^l."""
VAL_TOL = 1e-12


def chain_tol(l):
    return VAL_TOL * max(1, 4 ** l)
