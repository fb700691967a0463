"""GPU parity of the FP32-pipe paths against the FP64 CPU oracle, through the
C ABI.  Stated tolerances:
  MIXED (double-float transforms, FP32 factor + refinement against the
         FP64-accurate operator): 1e-12 per step, 1e-10 on whole solves;
  FP32  (plain FP32 transforms / assembly / Cholesky, FP64 history and
         correction): 1e-4 per step, 1e-3 on whole solves."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL_STEP = {"mixed": 1e-12, "fp32": 1e-4}
TOL_SOLVE = {"mixed": 1e-10, "fp32": 1e-3}


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("K", [1, 7, 32, 33, 100, 256, 300, 512])
def test_single_step(prec, K):
    spec = workloads.InstanceSpec(modes=(K, 1), nsteps=8, alpha=0.5, dpar=workloads.D_CFG2, fpar=workloads.F_COS)
    rng = np.random.default_rng(K)
    c = rng.standard_normal(K) * np.arange(1, K + 1) ** -1.5
    hist = c + 0.01 * rng.standard_normal(K)
    with psl1.Problem([spec], 2, precision=prec) as pr:
        for te, mu in ((0.0, 0.03), (0.37, 0.2), (0.9, 1e-4)):
            g = pr.step(0, c, te, mu, hist)
            o = O.step(oracle_prob(spec, 2), c, te, mu, hist)
            assert rel(g, o) < TOL_STEP[prec], (K, te, mu, rel(g, o))


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_parareal_and_serial_cfg1(prec):
    wl = workloads.cfg1()
    op = oracle_prob(wl.specs[0], wl.P)
    Uo, _, ko = O.parareal(op, wl.u0[0], tol=1e-10)
    S = O.serial_hyb(op, wl.u0[0])
    W = O.serial_uni(op, wl.u0[0])[:: op.m]
    with psl1.Problem(wl, precision=prec) as pr:
        k = pr.solve_parareal(tol=1e-10, allow_not_converged=True)
        U = pr.get_coeffs("parareal")[0]
        pr.solve_serial("hybrid")
        Sg = pr.get_coeffs("serial")[0]
        pr.solve_serial("uniform")
        Wg = pr.get_coeffs("serial")[0]
    assert rel(Sg, S) < TOL_SOLVE[prec]
    assert rel(Wg, W) < TOL_SOLVE[prec]
    assert rel(U, Uo[-1]) < TOL_SOLVE[prec]
    if prec == "mixed":
        assert k == ko


def test_mixed_ragged_batch_matches_oracle():
    wl = workloads.small_batch()
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
    for b, spec in enumerate(wl.specs):
        op = oracle_prob(spec, wl.P)
        assert rel(S[b], O.serial_hyb(op, wl.u0[b])) < TOL_SOLVE["mixed"]
        assert rel(U[b], O.parareal(op, wl.u0[b], tol=1e-12)[0][-1]) < TOL_SOLVE["mixed"]


def test_mixed_finite_termination_bitwise():
    # the parareal fixed point of the mixed F is the mixed S_hyb, slice by slice
    wl = workloads.cfg1(K=48, N=96, P=6)
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=0.0)
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        for j in range(k + 1):
            Uj = pr.get_iterate(j)[0]
            assert np.abs(Uj[: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j


@pytest.mark.parametrize("fpar", [(1.0,), (0, 1.0), (0.3, -0.2, 0.1, 0.5)])
def test_mixed_step_dominated_by_f(fpar):
    # hist = 0 and a large mu make the step ~ mu F(f(u)): the double-float
    # evaluation of cos u, sin u (with u up to ~10, several multiples of pi/2)
    # and of the other f terms is seen directly at the step tolerance
    K = 40
    spec = workloads.InstanceSpec(modes=(K, 1), nsteps=8, alpha=0.5, dpar=workloads.D_CFG2, fpar=fpar)
    rng = np.random.default_rng(11)
    c = 6.0 * rng.standard_normal(K) / np.arange(1, K + 1)
    with psl1.Problem([spec], 2, precision="mixed") as pr:
        for te, mu in ((0.3, 0.5), (1.7, 2.0)):
            g = pr.step(0, c, te, mu, np.zeros(K))
            o = O.step(oracle_prob(spec, 2), c, te, mu, np.zeros(K))
            assert rel(g, o) < TOL_STEP["mixed"], (fpar, te, mu, rel(g, o))
