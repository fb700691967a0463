"""GPU parity of the Chebyshev-Lobatto collocation scheme (the paper's own
spatial discretisation, Sec. 4.1, Eq. NumericalSchemeMainSystem) against the
CPU oracle, through the C ABI: single steps over interval counts 2..64 and
coefficient families, the fine and coarse propagators, the serial solvers
(including the fast history) and parareal on a ragged batch, and the paper's
model problem at its published size.

The library builds its derivative matrix from the paper's explicit diagonal
and trigonometric node differences, the oracle from the negative-sum form:
the two agree to rounding.  Tolerance: 1e-10 relative (FP64), as for the
sine-basis FP64 path.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10
D_MIX = (1.0, 0.5, 0.3, 0.1, 0.2, 0, 0.1, 0)     # (1 + 0.5/(1+u^2) X1 + 0.3 u + 0.1 sin pi x) X0
F_MIX = (0.1, 0.05, 0.02, 0.3, 0, 0, 0, 0)


def _spec(n, N=8, alpha=0.5, dpar=D_MIX, fpar=F_MIX, lo=0.0, hi=1.0):
    return workloads.InstanceSpec(modes=(n, 1), nsteps=N, alpha=alpha, lo=(lo, 0.0), hi=(hi, 1.0), dpar=dpar,
                                  fpar=fpar, basis="cheb")


@pytest.mark.parametrize("n", [2, 3, 16, 33, 64])
def test_collocation_step(n):
    spec = _spec(n, lo=-0.5 if n == 33 else 0.0, hi=1.25 if n == 33 else 1.0)
    rng = np.random.default_rng(n)
    c = 0.3 * rng.standard_normal(n - 1)
    hist = c + 0.01 * rng.standard_normal(n - 1)
    op = oracle_prob(spec, 2)
    with psl1.Problem([spec], 2) as pr:
        for te, mu in ((0.0, 1e-3), (0.4, 0.3)):
            g = pr.step(0, c, te, mu, hist)
            ref = O.step(op, c, te, mu, hist)
            assert rel(g, ref) < 1e-12, (n, mu, rel(g, ref))


def _batch():
    rng = np.random.default_rng(3)
    shapes = [(16, 12, 0.5), (7, 8, 1.0), (40, 16, 0.3), (5, 4, 0.7)]
    P = 4
    specs, u0 = [], []
    for n, N, a in shapes:
        specs.append(_spec(n, N=N, alpha=a))
        x = 0.5 * (1 + np.cos(np.arange(1, n) * np.pi / n))
        u0.append(np.sin(np.pi * x) * (0.5 + 0.2 * rng.standard_normal()))
    return specs, u0, P


def test_collocation_propagators_serial_and_parareal():
    specs, u0, P = _batch()
    with psl1.Problem(specs, P) as pr:
        pr.set_u0(np.concatenate(u0))
        its = pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
        pr.solve_serial("uniform")
        W = pr.get_coeffs("serial")
        pr.solve_serial("uniform-soe")
        Ws = pr.get_coeffs("serial")
        for b, s in enumerate(specs):
            op = oracle_prob(s, P)
            Uc = O.coarse_sweep(op, u0[b])
            assert rel(pr.coarse_step(b, 2, Uc[:3]), O.coarse_sweep(op, u0[b])[3]) < TOL, b
            assert rel(pr.fine_slice(b, 2, Uc[:3]), O.fine_slice(op, 2, Uc[:3])) < TOL, b
            Uo, _, _ = O.parareal(op, u0[b], tol=1e-12)
            assert rel(U[b], Uo[-1]) < TOL, b
            assert rel(S[b], O.serial_hyb(op, u0[b])) < TOL, b
            assert rel(W[b], O.serial_uni(op, u0[b])[:: op.m]) < TOL, b
            assert rel(Ws[b], O.serial_uni_soe(op, u0[b])[:: op.m]) < TOL, b
    assert its >= 1


def test_paper_model_problem_collocation():
    # D = 1 + u, f = sin(pi x) e^{-t}, u0 = x^4 (1-x)^4, alpha = 0.5 on 2^4 intervals,
    # P = 2^8 slices of 2^5 fine steps (Sec. 4.2): parareal reaches the sequential fine
    # solution (the oracle's S_hyb) and stops on the paper's tolerance 1e-10
    wl = workloads.e1_collocation()
    spec, u0 = wl.specs[0], wl.u0[0]
    op = oracle_prob(spec, wl.P)
    S = O.serial_hyb(op, u0)
    with psl1.Problem(wl) as pr:
        pr.set_graph(True)
        k = pr.solve_parareal(tol=1e-10)
        U = pr.get_coeffs("parareal")[0]
        pr.solve_serial("hybrid")
        Sg = pr.get_coeffs("serial")[0]
    assert rel(Sg, S) < TOL
    assert 1 <= k < wl.P and rel(U, S) < 1e-9, (k, rel(U, S))


def test_collocation_rejections():
    spec = _spec(16)
    with pytest.raises(psl1.PSL1Error) as ei:
        psl1.Problem([spec], 2, precision="mixed")
    assert ei.value.status == -1
    with psl1.Problem([spec], 2) as pr, psl1.MLP(nU=8, nH=4, width=16, nout=8) as m:
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.set_coarse(m)
        assert ei.value.status == -1
