"""2D coarse sweep shared by a thread-block cluster (psl1_set_sweep_split).

Each CTA of the cluster owns a share of the y node columns. The node-to-mode
results are partial sums that the cluster adds up through distributed shared
memory. Only the summation order changes, so the coarse solution must agree
with the one-CTA sweep to rounding: 1e-12 relative for FP64, 1e-11 for the
mixed path, which refines to a correction of 1e-11 of the iterate. It must also
agree with the oracle's coarse sweep (Eq. CoarsePropagator) at the 2D
tolerance of 1e-10. The split covers cases where some CTAs own no columns
(8 CTAs, 7 node pairs). Parareal with the split sweep must still end at S_hyb
(Eq. PararealConvergence), with inexact early iterations too."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-11)])
def test_split_coarse_solution_matches_one_cta_and_oracle(prec, tol):
    wl = workloads.small_batch_2d()
    out = {}
    with psl1.Problem(wl, precision=prec) as pr:
        for c in (1, 2, 4, 8):
            pr.set_sweep_split(c)
            assert pr.sweep_split() == c
            pr.solve_serial("coarse")
            out[c] = pr.get_coeffs("serial")
    for c in (2, 4, 8):
        for b in range(wl.B):
            assert rel(out[c][b], out[1][b]) < tol, (c, b, rel(out[c][b], out[1][b]))
    for b in range(wl.B):
        ref = O.coarse_sweep(oracle_prob(wl.specs[b], wl.P), wl.u0[b])
        assert rel(out[8][b], ref) < TOL, b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_split_parareal_ends_at_serial_solution(prec):
    wl = workloads.small_batch_2d()
    with psl1.Problem(wl, precision=prec) as pr:
        pr.set_sweep_split(8)
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        if prec == "mixed":
            pr.set_inexact_fine(1e-4)
        pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
    for b in range(wl.B):
        assert rel(U[b], S[b]) < TOL, b


def test_split_graph_mode_equals_host_loop():
    wl = workloads.small_batch_2d()
    res = []
    for graph in (False, True):
        with psl1.Problem(wl, precision="mixed") as pr:
            pr.set_sweep_split(4)
            pr.set_inexact_fine(1e-4)
            pr.set_graph(graph)
            pr.solve_parareal(tol=1e-11, allow_not_converged=True)
            res.append((pr.get_coeffs("parareal", flat=True), pr.get_iterations()))
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][0], res[1][0])


def test_split_setting_is_validated():
    wl = workloads.small_batch_2d()
    with psl1.Problem(wl, precision="mixed") as pr:
        assert pr.sweep_split() in (1, 2, 4, 8)      # the automatic choice
        for bad in (-1, 3, 5, 16):
            with pytest.raises(psl1.PSL1Error) as ei:
                pr.set_sweep_split(bad)
            assert ei.value.status == -1
        pr.set_sweep_split(1)
        assert pr.sweep_split() == 1
    with psl1.Problem(workloads.small_batch(), precision="mixed") as pr:   # 1D: one CTA per instance
        assert pr.sweep_split() == 1
        pr.set_sweep_split(0)
        pr.set_sweep_split(1)
        with pytest.raises(psl1.PSL1Error):
            pr.set_sweep_split(2)
