"""Inexact early parareal iterations (psl1_set_inexact_fine, MIXED, 1D and 2D).

While an instance's last increment is above the threshold, the F stage of
iteration k runs slices n > k with one FP32 inner solve per fine step; slice
n = k starts from exact states and keeps the refined solve.  The coarse sweep
of those iterations evaluates G with the FP32 step too, and G_old is
recomputed in the refined mode when an instance switches.  Parareal's
properties must survive (Eq. PararealConvergence): after k iterations the
states U^k_{0:k} equal the sequential F sweep S_hyb, the iteration still ends
at S_hyb, graph mode reproduces the host loop bitwise, and the first refined
iteration is exactly one refined iteration from its starting iterate.
Tolerances are those of the mixed path: 1e-13 relative for the exact prefix
(as in the finite-termination test of the refined path), 1e-10 for whole
solves."""
import numpy as np
import pytest

from paper_2510_11023_gb300 import psl1, workloads
from helpers import rel

pytestmark = pytest.mark.gpu
TOL_SOLVE = 1e-10


def _batch():
    return workloads.cfg2(B=6, seed=77, P=16, kmin=32, kmax=96, mmin=4, mmax=12)


def test_exact_prefix_and_fixed_point_with_every_early_slice_inexact():
    # a threshold of 1e-300 keeps every slice n > k inexact in every iteration:
    # only the exactness of slice n = k carries the iteration to S_hyb
    wl = workloads.cfg1(K=48, N=96, P=6)
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        pr.set_inexact_fine(1e-300)
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=0.0)
        assert k == wl.P
        for j in range(k + 1):
            Uj = pr.get_iterate(j)[0]
            assert np.abs(Uj[: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j
        assert rel(pr.get_coeffs("parareal")[0], S) <= 1e-13


def test_inexact_early_iterations_converge_to_serial_with_less_fine_work():
    wl = _batch()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        k0 = pr.solve_parareal(tol=1e-12)
        U0 = pr.get_coeffs("parareal")
        f0 = pr.stats()["flop_fine"]
        pr.set_inexact_fine(1e-4)
        k1 = pr.solve_parareal(tol=1e-12)
        U1 = pr.get_coeffs("parareal")
        f1 = pr.stats()["flop_fine"]
        pr.set_inexact_fine(0.0)          # off again: the refined iteration, bitwise
        k2 = pr.solve_parareal(tol=1e-12)
        U2 = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U0[b], S[b]) < TOL_SOLVE, b
        assert rel(U1[b], S[b]) < TOL_SOLVE, (b, rel(U1[b], S[b]))
        assert np.array_equal(U2[b], U0[b]), b
    assert k2 == k0
    assert k1 <= k0 + 1, (k0, k1)
    if k1 == k0:
        assert f1 < f0, (f0, f1)


def test_inexact_graph_mode_equals_host_loop():
    wl = _batch()
    out = []
    for graph in (False, True):
        with psl1.Problem(wl, precision="mixed") as pr:
            pr.set_inexact_fine(1e-4)
            pr.set_graph(graph)
            pr.solve_parareal(tol=1e-11, allow_not_converged=True)
            out.append((pr.get_coeffs("parareal", flat=True), pr.get_iterations(),
                        [pr.get_errlog(b) for b in range(wl.B)]))
    (Uh, ih, lh), (Ug, ig, lg) = out
    assert np.array_equal(ih, ig)
    assert np.array_equal(Uh, Ug)
    for a, b in zip(lh, lg):
        assert np.array_equal(a, b)


def test_inexact_threshold_rejects_bad_values():
    wl = workloads.cfg1(K=8, N=16, P=4)
    with psl1.Problem(wl, precision="mixed") as pr:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(psl1.PSL1Error) as ei:
                pr.set_inexact_fine(bad)
            assert ei.value.status == -1


def test_inexact_2d_exact_prefix_and_fixed_point():
    # 2D: the inexact slices take the FP32 2D step (one FP32 CG solve, no refinement);
    # the exact prefix and the fixed point S_hyb survive, as in 1D
    wl = workloads.small_batch_2d()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.set_inexact_fine(1e-300)
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=0.0)
        assert k == wl.P
        for j in range(k + 1):
            Uj = pr.get_iterate(j)
            for b in range(wl.B):
                assert np.abs(Uj[b][: j + 1] - S[b][: j + 1]).max() <= 1e-13 * np.abs(S[b]).max(), (j, b)
        pr.set_inexact_fine(1e-4)
        pr.keep_iterates(False)
        pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U[b], S[b]) < TOL_SOLVE, b


@pytest.mark.parametrize("dim", [1, 2])
def test_switch_to_refined_iteration_recomputes_stored_coarse_values(dim):
    # From the first refined iteration k_s of an instance on, the iteration must be
    # Eq. Parareal with the refined G at both call sites.  A resumed solve from
    # U^{k_s} computes G_old = G_n(U^{k_s}_{0:n}) afresh in the refined mode, so one
    # resumed iteration reproduces U^{k_s+1} bitwise only if the switch brought the
    # stored FP32-step values into the refined mode.
    wl = _batch() if dim == 1 else workloads.small_batch_2d()
    tau = 1e-4
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.set_inexact_fine(tau)
        pr.keep_iterates(True)
        pr.solve_parareal(tol=1e-12)
        its = pr.get_iterations()
        logs = [pr.get_errlog(b) for b in range(wl.B)]
        iters = [pr.get_iterate(k) for k in range(int(max(its)) + 1)]
    switch = {}
    for b in range(wl.B):
        ks = next((k for k in range(1, int(its[b])) if logs[b][k - 1] <= tau), None)
        if ks is not None:
            switch.setdefault(ks, []).append(b)
    assert switch, "no instance reached a refined iteration before converging"
    for ks, bs in sorted(switch.items()):
        with psl1.Problem(wl, precision="mixed") as pr:
            pr.resume_parareal(ks, iters[ks], tol=0.0, max_iter=ks + 1, allow_not_converged=True)
            U = pr.get_coeffs("parareal")
        for b in bs:
            assert np.array_equal(U[b], iters[ks + 1][b]), (ks, b)


def test_serial_coarse_solution_ignores_the_inexact_setting():
    wl = _batch()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("coarse")
        C0 = pr.get_coeffs("serial", flat=True)
        pr.set_inexact_fine(1e-4)
        pr.solve_serial("coarse")
        C1 = pr.get_coeffs("serial", flat=True)
    assert np.array_equal(C0, C1)


def test_looser_refinement_keeps_exact_prefix_and_fixed_point():
    # psl1_set_inexact_refinement: refined steps of slices n > k stop at factor * e_{k-1}
    # (e_{-1} = 1).
    # Slice n = k keeps the full target, so U^{k}_{0:k} = S_hyb to 1e-13 after k
    # iterations, and the iteration still ends at S_hyb.
    wl = _batch()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.solve_parareal(tol=1e-12)
        f_full = pr.stats()["flop_fine"]
        k_full = pr.get_iterations().max()
        pr.set_inexact_refinement(1e-2)
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=1e-12)
        f_loose = pr.stats()["flop_fine"]
        for j in range(k + 1):
            Uj = pr.get_iterate(j)
            for b in range(wl.B):
                top = min(j, wl.P)
                assert np.abs(Uj[b][: top + 1] - S[b][: top + 1]).max() <= 1e-13 * np.abs(S[b]).max(), (j, b)
        U = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U[b], S[b]) < TOL_SOLVE, b
    assert k <= k_full + 1
    if k == k_full:
        assert f_loose < f_full, (f_full, f_loose)


def test_looser_refinement_graph_equals_host_and_rejects_bad_values():
    wl = _batch()
    out = []
    for graph in (False, True):
        with psl1.Problem(wl, precision="mixed") as pr:
            pr.set_inexact_fine(1e-4)
            pr.set_inexact_refinement(1e-3)
            pr.set_graph(graph)
            pr.solve_parareal(tol=1e-11, allow_not_converged=True)
            out.append((pr.get_coeffs("parareal", flat=True), pr.get_iterations()))
            for bad in (-1.0, float("nan"), float("inf")):
                with pytest.raises(psl1.PSL1Error) as ei:
                    pr.set_inexact_refinement(bad)
                assert ei.value.status == -1
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


def test_looser_refinement_2d_exact_prefix_and_fixed_point():
    wl = workloads.small_batch_2d()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.set_inexact_fine(1e-4)
        pr.set_inexact_refinement(1e-2)
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=1e-12)
        for j in range(k + 1):
            Uj = pr.get_iterate(j)
            for b in range(wl.B):
                assert np.abs(Uj[b][: j + 1] - S[b][: j + 1]).max() <= 1e-13 * np.abs(S[b]).max(), (j, b)
        U = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U[b], S[b]) < TOL_SOLVE, b
