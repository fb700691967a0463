"""The coarse propagator with c L1 substeps per slice (psl1_set_coarse_substeps)
against the oracle's, through the C ABI: single coarse steps, the parareal
iterates and iteration counts (1D FP64 and mixed, 2D mixed), the limit c = m
(G is F: one iteration), and the rejections.  Tolerance 1e-10 (solves)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _oprob(spec, P, c):
    return O.make_prob(dim=spec.dim, Mx=spec.modes[0], My=spec.modes[1], Qx=spec.qnodes[0] or None,
                       Qy=spec.qnodes[1] or None, N=spec.nsteps, P=P, alpha=spec.alpha, T=spec.T, lo=spec.lo,
                       hi=spec.hi, dpar=spec.dpar, fpar=spec.fpar, coarse_substeps=c)


def _batch(dim):
    # ragged batches whose slices all have m >= 2 fine steps (c = 2 admissible)
    base = workloads.small_batch(P=4) if dim == 1 else workloads.small_batch_2d(P=4)
    keep = [b for b, s in enumerate(base.specs) if s.nsteps // base.P >= 2]
    return workloads.Workload(base.name, base.P, [base.specs[b] for b in keep], [base.u0[b] for b in keep])


@pytest.mark.parametrize("prec,dim", [("fp64", 1), ("mixed", 1), ("mixed", 2)])
def test_substep_coarse_propagator_against_oracle(prec, dim):
    wl = _batch(dim)
    c = 2
    with psl1.Problem(wl, precision=prec) as pr:
        pr.set_coarse_substeps(c)
        pr.solve_serial("coarse")
        Ug = pr.get_coeffs("serial")
        its = pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
        K = pr.get_iterations()
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
    for b, spec in enumerate(wl.specs):
        op = _oprob(spec, wl.P, c)
        assert rel(Ug[b], O.coarse_sweep(op, wl.u0[b])) < TOL, b
        Uo, _, ko = O.parareal(op, wl.u0[b], tol=1e-12)
        assert abs(int(K[b]) - ko) <= (0 if prec == "fp64" else 1), (b, K[b], ko)
        assert rel(U[b], Uo[-1]) < TOL and rel(U[b], S[b]) < TOL, b
    assert its >= 1


def test_substeps_equal_to_m_make_g_the_fine_propagator():
    wl = workloads.cfg1(K=24, N=48, P=6)
    m = 8
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        pr.set_coarse_substeps(m)
        pr.solve_serial("coarse")
        assert rel(pr.get_coeffs("serial")[0], S) < 1e-13
        pr.set_graph(True)
        k = pr.solve_parareal(tol=1e-12)
        assert k == 1 and rel(pr.get_coeffs("parareal")[0], S) < 1e-13


def test_substep_rejections():
    wl = workloads.cfg1(K=16, N=32, P=4)   # m = 8
    with psl1.Problem(wl) as pr, psl1.MLP(nU=8, nH=4, width=16, nout=8) as mlp:
        for bad in (0, 9):
            with pytest.raises(psl1.PSL1Error) as ei:
                pr.set_coarse_substeps(bad)
            assert ei.value.status == -1
        pr.set_coarse_substeps(2)
        with pytest.raises(psl1.PSL1Error):
            pr.set_coarse(mlp)            # the learned correction is defined on the one-step G
        pr.set_coarse_substeps(1)
        pr.set_coarse(mlp)
        with pytest.raises(psl1.PSL1Error):
            pr.set_coarse_substeps(2)
