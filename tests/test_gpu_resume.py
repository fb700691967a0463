"""Checkpoint and resume of parareal (psl1_resume_parareal), through the C ABI:
a solve interrupted after k0 iterations and resumed in a new handle from its
iterate U^{k0} ends where the uninterrupted solve ends, with the same
iteration count, bitwise (every kernel is deterministic and G_old is
recomputed at the checkpoint's states) for every instance still iterating at
k0 -- 1D mixed with the plain and the substep coarse propagator, and 2D FP64
with a one-CTA coarse sweep.  With the 2D sweep split across a cluster the
stored G_old values come from a different summation order than the ones the
resume recomputes (one CTA per unit), so that continuation agrees to rounding
(1e-12).  An instance that had converged before k0 is iterated once more from
its fixed point and stays there to rounding."""
import numpy as np
import pytest

from paper_2510_11023_gb300 import psl1, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["1d-mixed", "1d-mixed-substeps", "2d-fp64", "2d-fp64-split"])
def test_resume_reproduces_uninterrupted_solve(case):
    if case.startswith("1d"):
        wl, prec = workloads.cfg2(B=5, seed=9, P=8, kmin=20, kmax=70, mmin=4, mmax=6), "mixed"
    else:
        wl, prec = workloads.small_batch_2d(P=4), "fp64"
    sub = 2 if case.endswith("substeps") else 1
    split = 4 if case.endswith("split") else 1
    k0 = 2

    def setup(pr):
        pr.set_coarse_substeps(sub)
        if case.startswith("2d"):
            pr.set_sweep_split(split)

    with psl1.Problem(wl, precision=prec) as pr:
        setup(pr)
        pr.keep_iterates(True)
        k_full = pr.solve_parareal(tol=1e-12)
        U_full = pr.get_coeffs("parareal")
        its_full = pr.get_iterations()
        Uk0 = pr.get_iterate(k0)
    assert k_full > k0
    with psl1.Problem(wl, precision=prec) as pr:
        setup(pr)
        k_res = pr.resume_parareal(k0, Uk0, tol=1e-12)
        U_res = pr.get_coeffs("parareal")
        its_res = pr.get_iterations()
    assert k_res == k_full
    for b in range(wl.B):
        if its_full[b] > k0 and split > 1:   # the same continuation, to the rounding of G_old
            assert its_res[b] == its_full[b], b
            assert np.abs(U_res[b] - U_full[b]).max() <= 1e-12 * np.abs(U_full[b]).max(), b
        elif its_full[b] > k0:    # still iterating at the checkpoint: the same continuation, bitwise
            assert its_res[b] == its_full[b] and np.array_equal(U_res[b], U_full[b]), b
        else:                     # converged before it: iterated once more from its fixed point
            assert its_res[b] == k0 + 1, b
            assert np.abs(U_res[b] - U_full[b]).max() <= 1e-13 * np.abs(U_full[b]).max(), b
