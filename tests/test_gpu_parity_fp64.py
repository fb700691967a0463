"""GPU parity of the all-FP64 path against the CPU oracle (tolerance 1e-10
relative, as required of the all-FP64 path), through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _one(K, N=8, P=2, alpha=0.5, dpar=workloads.D_CFG2, fpar=workloads.F_COS, Q=0):
    spec = workloads.InstanceSpec(modes=(K, 1), qnodes=(Q, 0), nsteps=N, alpha=alpha, dpar=dpar, fpar=fpar)
    return spec


@pytest.mark.parametrize("K", [1, 7, 32, 33, 64, 100, 256, 512])
def test_single_step(K):
    spec = _one(K)
    rng = np.random.default_rng(K)
    c = rng.standard_normal(K) * np.arange(1, K + 1) ** -1.5
    hist = c + 0.01 * rng.standard_normal(K)
    with psl1.Problem([spec], 2) as pr:
        for te, mu in ((0.0, 0.03), (0.37, 0.2), (0.9, 1e-4)):
            g = pr.step(0, c, te, mu, hist)
            o = O.step(oracle_prob(spec, 2), c, te, mu, hist)
            assert rel(g, o) < 1e-12, (K, te, mu, rel(g, o))


def test_single_step_manufactured_sources_and_box():
    for fpar, dpar in (((0, 0, 0, 0, 1, 0), workloads.D_CFG1), ((0, 0, 0, 0, 0, 1), (1, 0, 0, 0.5)),
                       ((0.2, 0.1, 0.05, 0.3, 0, 0), (1, 0.5, 0.1, 0.2, 0.1, 0, 0.3, 0))):
        spec = _one(24, dpar=dpar, fpar=fpar, Q=60)
        c = np.linspace(0.3, -0.2, 24) / np.arange(1, 25)
        with psl1.Problem([spec], 2) as pr:
            g = pr.step(0, c, 0.4, 0.05, c)
        assert rel(g, O.step(oracle_prob(spec, 2), c, 0.4, 0.05, c)) < 1e-12
    spec = workloads.InstanceSpec(modes=(20, 1), nsteps=8, alpha=0.5, lo=(-0.5, 0), hi=(1.25, 1),
                                  dpar=workloads.D_CFG2, fpar=(0.1, 0, 0, 0.2))
    c = np.linspace(1, 0, 20) ** 2
    with psl1.Problem([spec], 2) as pr:
        g = pr.step(0, c, 0.2, 0.07, c)
    assert rel(g, O.step(oracle_prob(spec, 2), c, 0.2, 0.07, c)) < 1e-12


@pytest.mark.parametrize("n", [0, 1, 3])
def test_fine_and_coarse_propagators(n):
    wl = workloads.cfg1(K=40, N=64, P=4, alpha=0.35)
    spec, P = wl.specs[0], wl.P
    op = oracle_prob(spec, P)
    U = O.coarse_sweep(op, wl.u0[0])
    with psl1.Problem(wl) as pr:
        V = pr.fine_slice(0, n, U[: n + 1])
        G = pr.coarse_step(0, n, U[: n + 1])
    assert rel(V, O.fine_slice(op, n, U[: n + 1])) < TOL
    assert rel(G, O.coarse_step(op, n, U[: n + 1])) < TOL


@pytest.mark.parametrize("kind", ["hybrid", "uniform", "coarse"])
def test_serial_solvers_cfg1(kind):
    wl = workloads.cfg1()
    op = oracle_prob(wl.specs[0], wl.P)
    ref = {"hybrid": lambda: O.serial_hyb(op, wl.u0[0]),
           "uniform": lambda: O.serial_uni(op, wl.u0[0])[:: op.m],
           "coarse": lambda: O.coarse_sweep(op, wl.u0[0])}[kind]()
    with psl1.Problem(wl) as pr:
        pr.solve_serial(kind)
        g = pr.get_coeffs("serial")[0]
    assert rel(g, ref) < TOL


def test_parareal_iterates_cfg1():
    wl = workloads.cfg1()
    op = oracle_prob(wl.specs[0], wl.P)
    Uo, erro, ko = O.parareal(op, wl.u0[0], tol=1e-10)
    with psl1.Problem(wl) as pr:
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=1e-10)
        assert k == ko
        for j in range(k + 1):
            assert rel(pr.get_iterate(j)[0], Uo[j]) < TOL, j
        e = pr.get_errlog(0)
        assert np.allclose(e, erro, rtol=1e-6, atol=1e-14)
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        U = pr.get_coeffs("parareal")[0]
    assert rel(U, S) < 1e-9


def test_parareal_finite_termination_on_gpu():
    wl = workloads.cfg1(K=24, N=48, P=6)
    with psl1.Problem(wl) as pr:
        pr.keep_iterates(True)
        k = pr.solve_parareal(tol=0.0)
        assert k == wl.P
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")[0]
        for j in range(k + 1):
            Uj = pr.get_iterate(j)[0]
            assert np.abs(Uj[: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j


def test_small_ragged_batch_parareal_and_serial():
    wl = workloads.small_batch()
    with psl1.Problem(wl) as pr:
        pr.solve_parareal(tol=1e-12)
        its = pr.get_iterations()
        U = pr.get_coeffs("parareal")
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.solve_serial("uniform")
        W = pr.get_coeffs("serial")
    for b, spec in enumerate(wl.specs):
        op = oracle_prob(spec, wl.P)
        Uo, _, ko = O.parareal(op, wl.u0[b], tol=1e-12)
        assert its[b] == ko
        assert rel(U[b], Uo[-1]) < TOL
        assert rel(S[b], O.serial_hyb(op, wl.u0[b])) < TOL
        assert rel(W[b], O.serial_uni(op, wl.u0[b])[:: op.m]) < TOL


def test_error_paths():
    wl = workloads.cfg1(K=16, N=16, P=4)
    with psl1.Problem(wl) as pr:
        pr.set_D([-1.0, 0, 0, 0, 0, 0, 0, 0])   # D = -1: the system is not SPD
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.solve_serial("hybrid")
        assert ei.value.status == -2
        pr.set_D(workloads.D_CFG1)
        u0 = wl.u0_concat().copy()
        u0[3] = np.nan
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.set_u0(u0)
        assert ei.value.status == -3
        pr.set_u0(wl.u0_concat())
        pr.solve_serial("hybrid")       # usable again after the failures
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.step(0, np.zeros(16), 0.0, 0.1, np.zeros(16)) if False else pr.fine_slice(0, 9, np.zeros((10, 16)))
        assert ei.value.status == -1
