"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, library routines (numpy/scipy), brute force, or special
cases that reduce to a textbook scheme.  Citations are to arXiv 2510.11023.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

CFG1_D = (1.0, 0.5, 0, 0, 0, 0, 0, 0)      # D = 1 + 0.5/(1+u^2)
CFG1_F = (0.1, 0, 0, 0, 0, 0, 0, 0)        # f = 0.1 cos u


def cfg1_u0(K):
    # u0 = sin(pi x) + 0.5 sin(3 pi x) with phi_k = sqrt(2) sin(k pi x)
    c = np.zeros(K)
    c[0] = 1.0 / math.sqrt(2.0)
    c[2] = 0.5 / math.sqrt(2.0)
    return c


# ---------------------------------------------------------------- L1 weights
def test_l1_weights_closed_form_alpha_half():
    # Eq. (L1Scheme): b_j = (j+1)^{1-a} - j^{1-a}; at a = 1/2, b_j = sqrt(j+1) - sqrt(j)
    assert O.b(0.5, 0) == 1.0
    assert abs(O.b(0.5, 1) - (math.sqrt(2) - 1)) < 1e-15
    assert abs(O.b(0.5, 2) - (math.sqrt(3) - math.sqrt(2))) < 1e-15
    for j in range(3, 50):
        assert abs(O.b(0.5, j) - (math.sqrt(j + 1) - math.sqrt(j))) < 1e-14


@pytest.mark.parametrize("alpha", [0.2, 0.3, 0.5, 0.7, 0.95])
def test_l1_weights_telescoping_and_monotone(alpha):
    # Sec. 3.1 proof of Prop. 1: b_n + sum_{i=1}^n (b_{n-i} - b_{n-i+1}) = b_0 = 1
    for n in (1, 2, 7, 40, 513):
        s = O.b(alpha, n) + sum(O.b(alpha, n - i) - O.b(alpha, n - i + 1) for i in range(1, n + 1))
        assert abs(s - 1.0) < 1e-13
    bs = [O.b(alpha, j) for j in range(200)]
    assert all(bs[j] > bs[j + 1] > 0 for j in range(199))
    # real index continuity: b(n + r/M) at r = M equals b(n+1)
    for n in range(5):
        assert abs(O.b(alpha, n + 8 / 8) - O.b(alpha, n + 1)) < 1e-15


def test_l1_weights_alpha_one_is_backward_euler():
    # alpha = 1: b_0 = 1, b_x = 0 for x > 0 (abstract: 0 < alpha <= 1)
    assert O.b(1.0, 0) == 1.0
    for x in (0.125, 1, 2.5, 100):
        assert O.b(1.0, x) == 0.0


def test_gamma_closed_forms():
    assert abs(O.gamma2a(0.5) - math.sqrt(math.pi) / 2) < 1e-15
    assert abs(O.gamma2a(1.0) - 1.0) < 1e-15
    assert abs(O.gamma2a(0.0) - 1.0) < 1e-15


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_l1_uniform_operator_order(alpha):
    # Remark (Regularity): for C^2 functions the L1 error is O(dt^{2-alpha});
    # y = t^2 has Caputo derivative 2 t^{2-alpha} / Gamma(3-alpha).
    errs = []
    for n in (32, 64, 128, 256):
        dt = 1.0 / n
        y = (np.arange(n + 1) * dt) ** 2
        errs.append(abs(O.l1_uniform(alpha, dt, y) - 2.0 / math.gamma(3 - alpha)))
    slope = math.log2(errs[-2] / errs[-1])
    assert abs(slope - (2 - alpha)) < 0.05


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.7])
def test_l1_hybrid_operator_consistent(alpha):
    # Eq. (L1Fine): coarse history + fine current interval.  For y = t^2 the
    # error decays with the coarse step at a rate approaching 2 - alpha.
    errs = []
    for P in (16, 32, 64, 128):
        M, dT = 4, 1.0 / P
        n, r = P - 1, M
        Y = (np.arange(n + 1) * dT) ** 2
        yf = (n * dT + np.arange(r + 1) * dT / M) ** 2
        errs.append(abs(O.l1_hybrid(alpha, dT, M, n, r, Y, yf) - 2.0 / math.gamma(3 - alpha)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.2 < s < 2 - alpha + 0.02 for s in slopes)
    assert slopes[-1] > slopes[0]


def test_l1_hybrid_equals_uniform_when_single_interval():
    # n = 0: no coarse history, the hybrid operator is the uniform L1 on the fine grid
    a, M = 0.4, 16
    dT = 0.25
    yf = np.sin(np.arange(M + 1) * dT / M) + 1.0
    for r in range(1, M + 1):
        h = O.l1_hybrid(a, dT, M, 0, r, np.array([yf[0]]), yf[: r + 1])
        u = O.l1_uniform(a, dT / M, yf[: r + 1])
        assert abs(h - u) < 1e-12 * max(1.0, abs(u))


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("Q", [1, 2, 5, 16, 64, 512])
def test_gauss_legendre_vs_numpy(Q):
    x, w = O.gauss_legendre(Q)
    xr, wr = np.polynomial.legendre.leggauss(Q)
    assert np.abs(x - (xr + 1) / 2).max() < 1e-14
    assert np.abs(w - wr / 2).max() < 1e-14
    assert abs(w.sum() - 1.0) < 1e-14


def test_gauss_legendre_exact_on_polynomials():
    Q = 12
    x, w = O.gauss_legendre(Q)
    for deg in range(2 * Q):
        assert abs((w * x**deg).sum() - 1.0 / (deg + 1)) < 1e-14


# ---------------------------------------------------------------- basis / assembly
def test_basis_orthonormal_and_derivative():
    p = O.make_prob(Mx=12, Qx=96, N=4, P=1, alpha=0.5)
    x, _, w = O.nodes(p)
    phi, gx, _ = O.basis(p)
    G = phi.T @ (w[:, None] * phi)
    assert np.abs(G - np.eye(12)).max() < 1e-13
    # derivative table by integration by parts: int_0^1 x phi_k'(x) dx = -int_0^1 phi_k dx
    k = np.arange(1, 13)
    lhs = (w[:, None] * x[:, None] * gx).sum(axis=0)
    ref = -math.sqrt(2) * (1 - np.cos(k * math.pi)) / (k * math.pi)
    assert np.abs(lhs - ref).max() < 1e-13
    assert np.abs((w[:, None] * gx).sum(axis=0)).max() < 1e-12   # phi_k(1) - phi_k(0) = 0


def test_stiffness_constant_D_is_diagonal():
    # a(1; phi_k, phi_l) = (k pi)^2 delta_kl (Eq. AForm with w = 1)
    K = 24
    p = O.make_prob(Mx=K, Qx=4 * K, N=4, P=1, alpha=0.5)
    A = O.stiffness(p, np.ones(p.Q))
    ref = np.diag((np.arange(1, K + 1) * math.pi) ** 2)
    assert np.abs(A - ref).max() < 1e-11 * ref.max()


def test_stiffness_constant_D_2d():
    p = O.make_prob(dim=2, Mx=5, My=4, Qx=32, Qy=32, N=4, P=1, alpha=0.5)
    A = O.stiffness(p, np.ones(p.Q))
    k = np.repeat(np.arange(1, 6), 4)
    l = np.tile(np.arange(1, 5), 5)
    ref = np.diag((k * math.pi) ** 2 + (l * math.pi) ** 2)
    assert np.abs(A - ref).max() < 1e-11 * ref.max()


def test_step_2d_constant_D_is_a_diagonal_solve():
    # D = d0 and f = 0 on a box (Lx, Ly): a(d0; phi_kl, phi_k'l') = d0 pi^2 (k^2/Lx^2 + l^2/Ly^2)
    # delta, so (I + mu A) c = hist decouples mode by mode (Eq. NumericalSchemeFine)
    Mx, My, d0, mu = 6, 5, 1.3, 0.07
    lo, hi = (-0.5, 0.25), (1.0, 2.0)
    p = O.make_prob(dim=2, Mx=Mx, My=My, Qx=48, Qy=48, N=4, P=1, alpha=0.5, lo=lo, hi=hi,
                    dpar=(d0, 0, 0, 0), fpar=(0,))
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    rng = np.random.default_rng(3)
    hist = rng.standard_normal(Mx * My)
    c = rng.standard_normal(Mx * My)
    k = np.repeat(np.arange(1, Mx + 1), My)
    l = np.tile(np.arange(1, My + 1), Mx)
    ref = hist / (1 + mu * d0 * math.pi**2 * (k**2 / Lx**2 + l**2 / Ly**2))
    assert np.abs(O.step(p, c, 0.3, mu, hist) - ref).max() < 1e-12


def test_step_2d_separable_source_closed_form():
    # f = c3 sin(pi x) e^{-t} on the unit square: F_kl = c3 e^{-t} int sin(pi x) phi_k dx int phi_l dy
    #   = c3 e^{-t} delta_k1 (1 - (-1)^l) / (l pi);  with hist = 0 the step is mu F / (1 + mu pi^2 (k^2 + l^2))
    Mx, My, mu, t, c3 = 4, 7, 0.05, 0.4, 0.8
    p = O.make_prob(dim=2, Mx=Mx, My=My, Qx=40, Qy=40, N=4, P=1, alpha=0.5, dpar=(1.0, 0, 0, 0),
                    fpar=(0, 0, 0, c3))
    k = np.repeat(np.arange(1, Mx + 1), My)
    l = np.tile(np.arange(1, My + 1), Mx)
    F = np.where(k == 1, c3 * math.exp(-t) * (1 - np.cos(l * math.pi)) / (l * math.pi), 0.0)
    ref = mu * F / (1 + mu * math.pi**2 * (k**2 + l**2))
    got = O.step(p, np.zeros(Mx * My), t, mu, np.zeros(Mx * My))
    assert np.abs(got - ref).max() < 1e-14


def test_stiffness_toeplitz_hankel_identity():
    # product-to-sum: phi_k' phi_l' = k l pi^2 (cos((k-l) pi x) + cos((k+l) pi x)), so
    # A_kl = k l pi^2 (g_|k-l| + g_{k+l}), g_s = sum_q w_q D_q cos(s pi x_q) -- exact at node level
    K = 20
    p = O.make_prob(Mx=K, N=4, P=1, alpha=0.5)
    x, _, w = O.nodes(p)
    rng = np.random.default_rng(1)
    Dq = 1.0 + rng.random(p.Q)
    A = O.stiffness(p, Dq)
    g = np.array([(w * Dq * np.cos(s * math.pi * x)).sum() for s in range(2 * K + 1)])
    k = np.arange(1, K + 1)
    TH = g[np.abs(k[:, None] - k[None, :])] + g[k[:, None] + k[None, :]]
    ref = np.outer(k, k) * math.pi**2 * TH
    assert np.abs(A - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(A - A.T).max() == 0.0


def test_load_closed_forms():
    K = 10
    p = O.make_prob(Mx=K, Qx=64, N=4, P=1, alpha=0.5)
    F = O.load(p, np.ones(p.Q))          # int_0^1 sqrt2 sin(k pi x) dx
    k = np.arange(1, K + 1)
    ref = math.sqrt(2) * (1 - np.cos(k * math.pi)) / (k * math.pi)
    assert np.abs(F - ref).max() < 1e-13
    x, _, _ = O.nodes(p)
    F2 = O.load(p, np.sin(math.pi * x))  # = delta_k1 / sqrt2
    ref2 = np.zeros(K)
    ref2[0] = 1 / math.sqrt(2)
    assert np.abs(F2 - ref2).max() < 1e-13


def test_eval_nodes_and_families():
    K = 8
    p = O.make_prob(Mx=K, N=4, P=1, alpha=0.5, dpar=CFG1_D, fpar=CFG1_F)
    x, _, _ = O.nodes(p)
    c = cfg1_u0(K)
    u, Dq, fq = O.eval_nodes(p, c, 0.3)
    ue = np.sin(math.pi * x) + 0.5 * np.sin(3 * math.pi * x)
    assert np.abs(u - ue).max() < 1e-14
    assert np.abs(Dq - (1 + 0.5 / (1 + ue**2))).max() < 1e-15
    assert np.abs(fq - 0.1 * np.cos(ue)).max() < 1e-15
    # config-2 D family: (1 + 0.5/(1+u^2)) (1 + 0.2 sin 2 pi x); config-5 in 2D
    p2 = O.make_prob(Mx=K, N=4, P=1, alpha=0.5, dpar=(1, 0.5, 0, 0, 0.2))
    assert abs(O.D(p2, 0.25, 0, 0, 1.0) - 1.25 * 1.2) < 1e-15
    p5 = O.make_prob(dim=2, Mx=4, My=4, N=4, P=1, alpha=0.6, dpar=(1, 0.5, 0, 0, 0, 0, 0, 0.3))
    assert abs(O.D(p5, 0.1, 0.0, 0, 1.0) - (1 + 0.25 * 1.3)) < 1e-15
    pe = O.make_prob(Mx=K, N=4, P=1, alpha=0.5, dpar=(1, 0, 1, 0), fpar=(0, 0, 0, 1))
    assert abs(O.D(pe, 0.3, 0, 0, 0.2) - 1.2) < 1e-15
    assert abs(O.f(pe, 0.5, 0, 1.0, 7.0) - math.exp(-1)) < 1e-15


# ---------------------------------------------------------------- manufactured sources
def test_manufactured_source_1_against_finite_differences():
    from scipy.integrate import quad
    a = 0.5
    p = O.make_prob(Mx=4, N=4, P=1, alpha=a, dpar=CFG1_D, fpar=(0, 0, 0, 0, 1))
    # Caputo derivative of t^a by quadrature of Eq. (Caputo)
    t0 = 0.7
    num = quad(lambda s: a, 0, t0, weight="alg", wvar=(a - 1, -a))[0]
    num /= math.gamma(1 - a)
    assert abs(num - math.gamma(1 + a)) < 1e-8
    uex = lambda x, t: (1 + t**a) * math.sin(math.pi * x)
    Dfun = lambda u: 1 + 0.5 / (1 + u * u)
    h = 1e-4
    for x in (0.13, 0.5, 0.81):
        flux = lambda z: Dfun(uex(z, t0)) * (uex(z + h, t0) - uex(z - h, t0)) / (2 * h)
        div = (flux(x + h) - flux(x - h)) / (2 * h)
        ref = math.gamma(1 + a) * math.sin(math.pi * x) - div
        assert abs(O.src1(p, x, t0) - ref) < 1e-5


def test_manufactured_source_2_against_finite_differences():
    a = 0.4
    p = O.make_prob(Mx=4, N=4, P=1, alpha=a, dpar=(1, 0, 0, 0.5), fpar=(0, 0, 0, 0, 0, 1))
    uex = lambda x, t: (1 + t * t) * math.sin(math.pi * x) / (2 - math.cos(math.pi * x))
    Dfun = lambda x: 1 + 0.5 * math.sin(math.pi * x)
    h = 1e-4
    t0 = 0.6
    for x in (0.1, 0.45, 0.9):
        flux = lambda z: Dfun(z) * (uex(z + h, t0) - uex(z - h, t0)) / (2 * h)
        div = (flux(x + h) - flux(x - h)) / (2 * h)
        cap = 2 * t0 ** (2 - a) / math.gamma(3 - a) * uex(x, 0)
        assert abs(O.src2(p, x, t0) - (cap - div)) < 1e-5


# ---------------------------------------------------------------- Cholesky
def test_cholesky_against_numpy_and_residual():
    rng = np.random.default_rng(7)
    for K in (1, 3, 8, 40):
        B = rng.standard_normal((K, K))
        M = B @ B.T + K * np.eye(K)
        r = rng.standard_normal(K)
        x, st = O.chol_solve(M, r)
        assert st == 0
        assert np.abs(x - np.linalg.solve(M, r)).max() < 1e-12 * np.abs(x).max()
        assert np.linalg.norm(M @ x - r) < 1e-13 * np.linalg.norm(r) * K


def test_cholesky_reports_first_bad_pivot():
    M = np.eye(4)
    M[2, 2] = -1.0
    _, st = O.chol_solve(M, np.ones(4))
    assert st == -3
    M = np.array([[1.0, 2.0], [2.0, 1.0]])
    _, st = O.chol_solve(M, np.ones(2))
    assert st == -2


# ---------------------------------------------------------------- schemes
def test_weak_form_operator_closed_form_and_matrix():
    # the matrix-free weak form (Eq. AForm, node by node) gives
    # (i) pi^2 (k^2 + l^2) v_kl for D = 1 on the unit square (closed form) and
    # (ii) the assembled matrix times v (numpy) for a random positive D, 1D and 2D
    p = O.make_prob(dim=2, Mx=5, My=4, Qx=32, Qy=32, N=4, P=1, alpha=0.5)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(p.K)
    k = np.repeat(np.arange(1, 6), 4)
    l = np.tile(np.arange(1, 5), 5)
    ref = math.pi**2 * (k**2 + l**2) * v
    assert np.abs(O.apply_stiffness(p, np.ones(p.Q), v) - ref).max() < 1e-11 * np.abs(ref).max()
    for q in (O.make_prob(Mx=17, N=4, P=1, alpha=0.5),
              O.make_prob(dim=2, Mx=6, My=7, Qx=14, Qy=12, N=4, P=1, alpha=0.5, lo=(-0.5, 0.25), hi=(1.0, 2.0))):
        Dq = 0.5 + rng.random(q.Q)
        v = rng.standard_normal(q.K)
        ref = O.stiffness(q, Dq) @ v
        assert np.abs(O.apply_stiffness(q, Dq, v) - ref).max() < 1e-12 * np.abs(ref).max()


def test_cg_step_solves_the_same_system_as_cholesky():
    # the two step solves of the oracle reach the same (unique) solution of the SPD
    # system of Eq. NumericalSchemeFine; with D = d0 and f = 0 it is the diagonal solve
    Mx, My, d0, mu = 6, 5, 1.3, 0.07
    lo, hi = (-0.5, 0.25), (1.0, 2.0)
    p = O.make_prob(dim=2, Mx=Mx, My=My, Qx=48, Qy=48, N=4, P=1, alpha=0.5, lo=lo, hi=hi,
                    dpar=(d0, 0, 0, 0), fpar=(0,), solver="cg")
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    rng = np.random.default_rng(3)
    hist = rng.standard_normal(Mx * My)
    k = np.repeat(np.arange(1, Mx + 1), My)
    l = np.tile(np.arange(1, My + 1), Mx)
    ref = hist / (1 + mu * d0 * math.pi**2 * (k**2 / Lx**2 + l**2 / Ly**2))
    assert np.abs(O.step(p, rng.standard_normal(Mx * My), 0.3, mu, hist) - ref).max() < 1e-13
    for dim, Mx, My in ((1, 40, 1), (2, 9, 8)):
        kw = dict(dim=dim, Mx=Mx, My=My, N=12, P=3, alpha=0.6, dpar=(1.0, 0.5, 0, 0, 0.2, 0, 0, 0.3),
                  fpar=(0.05, 0.1, 0.02, 0, 0, 0))
        pc, pg = O.make_prob(**kw), O.make_prob(solver="cg", **kw)
        c = rng.standard_normal(pc.K) / np.arange(1, pc.K + 1)
        hist = c + 0.01 * rng.standard_normal(pc.K)
        for mu in (0.01, 0.8):
            a, b = O.step(pc, c, 0.2, mu, hist), O.step(pg, c, 0.2, mu, hist)
            assert np.abs(a - b).max() < 1e-13 * np.abs(a).max(), (dim, mu)
        U = O.coarse_sweep(pc, c)
        Va, Vb = O.fine_slice(pc, 2, U[:3]), O.fine_slice(pg, 2, U[:3])
        assert np.abs(Va - Vb).max() < 1e-13 * np.abs(Va).max(), dim


def test_cg_step_reproduces_the_stored_dense_solve_at_32x32_modes():
    # at the 32 x 32-mode, 64 x 64-node size the CG solve on the weak form reproduces
    # the dense Cholesky solve stored in tests/golden/step2d_32x32.txt (written from the
    # assembled K x K x Q matrix), so the 64 x 64-mode stored results, which only the
    # CG solve can reach, rest on the same system
    import os
    import sys
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, golden)
    from make_step2d_32x32 import inputs
    spec, P, c, hist, te, mu = inputs()
    p = O.make_prob(dim=2, Mx=32, My=32, N=spec.nsteps, P=P, alpha=spec.alpha, dpar=spec.dpar, fpar=spec.fpar,
                    solver="cg")
    ref = np.loadtxt(os.path.join(golden, "step2d_32x32.txt"))
    assert np.abs(O.step(p, c, te, mu, hist) - ref).max() < 1e-14 * np.abs(ref).max()


def test_openmp_parallel_stage_is_the_same_computation():
    # the OpenMP build runs the parallel stage's slices on all host threads (the
    # paper's threads over coarse intervals, Sec. 4.2); every slice is computed the
    # same way, so parareal and the F stage agree bitwise with the serial build
    p = O.make_prob(Mx=12, N=48, P=6, alpha=0.35, dpar=(1, 0.5, 0, 0, 0.2), fpar=CFG1_F)
    u0 = cfg1_u0(12)
    U1, e1, k1 = O.parareal(p, u0, 1e-12)
    U2, e2, k2 = O.parareal(p, u0, 1e-12, omp=True)
    assert k1 == k2 and np.array_equal(U1, U2) and np.array_equal(e1, e2)
    assert np.array_equal(O.fine_stage(p, U1[0], 2), O.fine_stage(p, U1[0], 2, omp=True))
    F = O.fine_stage(p, U1[0], 2, 5)
    assert np.array_equal(F[3], O.fine_slice(p, 3, U1[0][:4])[-1])
    assert not F[:2].any() and not F[5:].any() and F[2:5].all()


def test_fine_propagator_expanded_equals_difference_form():
    # Eq. (L1Fine): difference form (first line) = expanded form (second line)
    p = O.make_prob(Mx=12, N=48, P=6, alpha=0.35, dpar=(1, 0.5, 0, 0, 0.2), fpar=CFG1_F)
    U = O.coarse_sweep(p, cfg1_u0(12))
    for n in (0, 1, 3, 5):
        Ve = O.fine_slice(p, n, U[: n + 1], diff_form=False)
        Vd = O.fine_slice(p, n, U[: n + 1], diff_form=True)
        assert np.abs(Ve - Vd).max() < 1e-13 * np.abs(Ve).max()


@pytest.mark.parametrize("P", [1, 4])
def test_alpha_one_is_linearly_implicit_backward_euler(P):
    # alpha = 1: all L1 history vanishes and mu = dt, so every solver is the
    # semi-implicit backward Euler scheme, written out here with numpy.
    K, N = 10, 24
    p = O.make_prob(Mx=K, N=N, P=P, alpha=1.0, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(K)
    dt = 1.0 / N
    c = u0.copy()
    BE = [c.copy()]
    for j in range(N):
        _, Dq, fq = O.eval_nodes(p, c, j * dt)
        A = O.stiffness(p, Dq)
        F = O.load(p, fq)
        c = np.linalg.solve(np.eye(K) + dt * A, c + dt * F)
        BE.append(c.copy())
    BE = np.array(BE)
    W = O.serial_uni(p, u0)
    U = O.serial_hyb(p, u0)
    assert np.abs(W - BE).max() < 1e-13
    assert np.abs(U - BE[:: N // P]).max() < 1e-13


def test_single_slice_hybrid_is_uniform():
    # P = 1: no coarse history, the fine sweep is the uniform L1 scheme
    p = O.make_prob(Mx=10, N=40, P=1, alpha=0.6, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(10)
    U, V = O.serial_hyb(p, u0, want_all=True)
    W = O.serial_uni(p, u0)
    assert np.abs(V - W).max() < 1e-13


def test_one_fine_step_per_slice_is_coarse_sweep():
    # M = 1: F_n and G_n are the same step, so S_hyb = coarse sweep
    p = O.make_prob(Mx=10, N=16, P=16, alpha=0.45, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(10)
    assert np.abs(O.serial_hyb(p, u0) - O.coarse_sweep(p, u0)).max() < 1e-13


def test_serial_hyb_differs_from_uniform_at_discretisation_level():
    p = O.make_prob(Mx=16, N=128, P=8, alpha=0.5, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(16)
    U = O.serial_hyb(p, u0)
    W = O.serial_uni(p, u0)
    gap = np.abs(U - W[:: 16]).max()
    assert 1e-6 < gap < 1e-2


def _rand_mlp(K, nU, nH, width, seed):
    nin = nU + nH + 2
    rng = np.random.default_rng(seed)
    n = O.mlp_nparams(nin, width, K)
    return {"params": 0.05 * rng.standard_normal(n), "oscale": 1e-2 * np.ones(K),
            "nU": nU, "nH": nH, "width": width}


@pytest.mark.parametrize("use_mlp", [False, True])
def test_parareal_finite_termination(use_mlp):
    # Eq. (PararealConvergence) and the k >= n saturation: after k iterations
    # U^k_n = S_hyb,n for n <= k, for any coarse propagator.
    K, P = 12, 6
    p = O.make_prob(Mx=K, N=36, P=P, alpha=0.5, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(K)
    S = O.serial_hyb(p, u0)
    mlp = _rand_mlp(K, K, 4, 16, 3) if use_mlp else None
    Ua, err, k = O.parareal(p, u0, tol=0.0, max_iter=P, mlp=mlp)
    assert k == P
    scale = np.abs(S).max()
    for kk in range(P + 1):
        d = np.abs(Ua[kk, : kk + 1] - S[: kk + 1]).max()
        assert d <= 1e-13 * scale, (kk, d)
    assert np.abs(Ua[P] - S).max() <= 1e-13 * scale
    if use_mlp:   # the correction changed the coarse sweep
        assert np.abs(Ua[0] - O.coarse_sweep(p, u0)).max() > 1e-6


def test_parareal_stops_on_increment_and_converges_cfg1():
    # config 1 (alpha = 0.5, K = 32, N = 256, P = 8): converges to S_hyb
    p = O.make_prob(Mx=32, N=256, P=8, alpha=0.5, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(32)
    S = O.serial_hyb(p, u0)
    Ua, err, k = O.parareal(p, u0, tol=1e-10)
    assert k <= 8
    assert err[-1] <= 1e-10 or k == 8
    e = [np.abs(Ua[j] - S).max() / np.abs(S).max() for j in range(k + 1)]
    assert all(e[j + 1] < e[j] for j in range(k - 1))
    assert e[-1] < 1e-9


def test_coarse_step_matches_uniform_scheme_on_coarse_grid():
    # with the coarse grid as the fine grid (N = P), S_uni is the coarse sweep
    p = O.make_prob(Mx=8, N=8, P=8, alpha=0.7, dpar=CFG1_D, fpar=CFG1_F)
    u0 = cfg1_u0(8)
    assert np.abs(O.serial_uni(p, u0) - O.coarse_sweep(p, u0)).max() < 1e-13


# ---------------------------------------------------------------- convergence observables
def _exact2(K, t):
    q = O.make_prob(Mx=K, Qx=256, N=1, P=1, alpha=0.5)
    x, _, _ = O.nodes(q)
    return O.project(q, (1 + t * t) * np.sin(math.pi * x) / (2 - np.cos(math.pi * x)))


def test_time_order_smooth_linear_case_is_one():
    # Reading: the source is lagged to t_n (Eq. NumericalSchemeSequential), an
    # O(dt) consistency error that dominates the L1 order 2 - alpha > 1 for a
    # C^2-in-time solution; the observed order is therefore 1.
    K, a = 16, 0.5
    errs = []
    for N in (32, 64, 128):
        p = O.make_prob(Mx=K, N=N, P=1, alpha=a, dpar=(1, 0, 0, 0.5), fpar=(0, 0, 0, 0, 0, 1))
        W = O.serial_uni(p, _exact2(K, 0.0))
        errs.append(np.linalg.norm(W[-1] - _exact2(K, 1.0)))
    for i in range(2):
        assert abs(math.log2(errs[i] / errs[i + 1]) - 1.0) < 0.05


def test_manufactured_cfg1_converges_first_order():
    # u = (1 + t^a) sin(pi x) (config 1 manufactured case); t^a singularity plus lag
    errs = []
    for N in (32, 64, 128):
        p = O.make_prob(Mx=8, N=N, P=1, alpha=0.5, dpar=CFG1_D, fpar=(0, 0, 0, 0, 1))
        u0 = np.zeros(8)
        u0[0] = 1 / math.sqrt(2)
        W = O.serial_uni(p, u0)
        ex = np.zeros(8)
        ex[0] = 2 / math.sqrt(2)
        errs.append(np.linalg.norm(W[-1] - ex))
    assert errs[0] > errs[1] > errs[2]
    assert 0.8 < math.log2(errs[1] / errs[2]) < 1.2


def test_spectral_decay_in_modes():
    # the sine coefficients of sin(pi x)/(2 - cos(pi x)) are 2 rho^k, rho = 2 - sqrt 3;
    # at fixed dt the Galerkin error against a high-K run decays like rho^K
    N = 16

    def run(K):
        p = O.make_prob(Mx=K, N=N, P=1, alpha=0.5, dpar=(1, 0, 0, 0.5), fpar=(0, 0, 0, 0, 0, 1))
        return O.serial_uni(p, _exact2(K, 0.0))[-1]

    ref = run(40)
    Ks = [4, 6, 8, 10]
    errs = []
    for K in Ks:
        c = run(K)
        errs.append(math.sqrt(np.sum((c - ref[:K]) ** 2) + np.sum(ref[K:] ** 2)))
    slope = np.polyfit(Ks, np.log(errs), 1)[0]
    assert abs(slope - math.log(2 - math.sqrt(3))) < 0.1 * abs(math.log(2 - math.sqrt(3)))


# ---------------------------------------------------------------- Lemma 1
def test_lemma1_closed_form_matches_recursion_exactly():
    # Lemma 1 (two-index Gronwall), equality case in exact rationals
    a, bb, c = Fraction(3, 10), Fraction(11, 10), Fraction(1001, 1000)
    E0 = Fraction(7, 5)
    Kmax, Nmax = 8, 10
    f = [[Fraction(0)] * (Nmax + 1) for _ in range(Kmax + 1)]
    for n in range(1, Nmax + 1):
        f[0][n] = E0
    for k in range(Kmax):
        for n in range(Nmax):
            f[k + 1][n + 1] = a + bb * f[k][n] + c * f[k + 1][n]

    def binom(p_, q_):
        if q_ == -1 and p_ == -1:
            return 1
        if q_ < 0 or p_ < 0 or q_ > p_:
            return 0
        return math.comb(p_, q_)

    for k in range(1, Kmax + 1):
        for n in range(1, Nmax + 1):
            closed = a * sum(binom(i + j, j) * c**i * bb**j
                             for j in range(k) for i in range(n - j))
            closed += E0 * bb**k * sum(binom(j - 1, k - 1) * c ** (j - k) for j in range(k, n))
            assert closed == f[k][n]


# ---------------------------------------------------------------- MLP
def test_mlp_backward_against_finite_differences():
    nin, width, nout, B = 7, 6, 5, 3
    rng = np.random.default_rng(11)
    n = O.mlp_nparams(nin, width, nout)
    assert n == width * nin + width + 2 * (width * width + width) + nout * width + nout
    th = 0.5 * rng.standard_normal(n)
    z = rng.standard_normal((B, nin))
    tg = rng.standard_normal((B, nout))
    g, L = O.mlp_backward(th, nin, width, nout, z, tg)
    y = O.mlp_forward(th, nin, width, nout, z)
    assert abs(L - np.mean((y - tg) ** 2)) < 1e-14
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        Lp = np.mean((O.mlp_forward(tp, nin, width, nout, z) - tg) ** 2)
        Lm = np.mean((O.mlp_forward(tm, nin, width, nout, z) - tg) ** 2)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_mlp_forward_linear_limit():
    # a single sample with all hidden pre-activations equal to zero: silu(0) = 0,
    # so the output is the last bias
    nin, width, nout = 4, 3, 2
    n = O.mlp_nparams(nin, width, nout)
    th = np.zeros(n)
    th[-nout:] = [0.25, -1.5]
    y = O.mlp_forward(th, nin, width, nout, np.ones((1, nin)))
    assert np.all(y == np.array([[0.25, -1.5]]))


def test_adam_first_step_closed_form():
    # first Adam step with zero moments: theta -= lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    th = np.zeros(3)
    m, v = np.zeros(3), np.zeros(3)
    O.adam_step(th, g, m, v, 1, lr=0.01, eps=1e-8)
    assert np.abs(th - (-0.01 * g / (np.abs(g) + 1e-8))).max() < 1e-15


def test_mlp_features_definition():
    # z = [k^2 U_n ; k^2 eta_n(1:nH) ; alpha ; T_n], eta_n the coarse L1 history
    p = O.make_prob(Mx=6, N=12, P=4, alpha=0.5, dpar=CFG1_D, fpar=CFG1_F)
    U = O.coarse_sweep(p, cfg1_u0(6))
    z = O.mlp_features(p, 6, 3, 2, U)
    k2 = np.arange(1, 7) ** 2
    assert np.abs(z[:6] - k2 * U[2]).max() < 1e-15
    eta = O.b(0.5, 2) * (U[1] - U[0]) + O.b(0.5, 1) * (U[2] - U[1])
    assert np.abs(z[6:9] - k2[:3] * eta[:3]).max() < 1e-15
    assert z[9] == 0.5 and abs(z[10] - 0.5) < 1e-15


# ---------------------------------------------------------------- fast history (sum of exponentials)
@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.9])
def test_gauss_jacobi_against_scipy(alpha):
    from scipy.special import roots_jacobi
    t, w = O.gauss_jacobi(10, 0.0, alpha - 1.0)
    t2, w2 = roots_jacobi(10, 0.0, alpha - 1.0)
    assert np.abs(t - t2).max() < 1e-13 and np.abs(w - w2).max() < 1e-12 * w2.max()


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.9, 0.99])
@pytest.mark.parametrize("X", [17, 1024, 8192])
def test_soe_approximates_l1_weights(alpha, X):
    # b(x) = x^{1-a} ((1 + 1/x)^{1-a} - 1) written without cancellation (expm1, log1p)
    s, w = O.soe_nodes(alpha, X)
    x = np.arange(O.SOE_NLOC, X + 1, dtype=np.float64)
    ref = x ** (1 - alpha) * np.expm1((1 - alpha) * np.log1p(1 / x))
    approx = (w[None, :] * np.exp(-np.outer(x, s))).sum(1)
    assert np.abs(approx / ref - 1).max() < 1e-13
    assert len(s) <= 80 and np.all(s > 0) and np.all(w > 0)


def test_soe_uniform_scheme_matches_exact_history():
    # the scheme with the approximated weights stays within rounding of the exact
    # uniform scheme; alpha = 1 has no history (no exponentials) and N < nloc
    # uses only the exact local window
    rng = np.random.default_rng(4)
    for K, N, a in ((12, 200, 0.4), (8, 100, 0.8), (12, 64, 1.0), (9, 15, 0.5)):
        p = O.make_prob(Mx=K, N=N, P=1, alpha=a, dpar=CFG1_D, fpar=CFG1_F)
        u0 = rng.standard_normal(K) / np.arange(1, K + 1) ** 2
        W, Ws = O.serial_uni(p, u0), O.serial_uni_soe(p, u0)
        assert np.abs(Ws - W).max() < 1e-13 * np.abs(W).max(), (K, N, a)
    assert len(O.soe_nodes(1.0, 100)[0]) == 0


# ---------------------------------------------------------------- Chebyshev-Lobatto collocation (Sec. 4.1)
def test_collocation_differentiation_matrix():
    # exact on polynomials of degree <= n (Sec. 4.1: D u = u' for the interpolant), and the
    # negative-sum diagonal equals the explicit form the paper prints, scaled by 2/(b-a)
    n, a, b = 12, 0.2, 1.7
    p = O.make_prob(Mx=n, N=4, P=1, alpha=0.5, basis="cheb", lo=(a, 0), hi=(b, 1))
    x, Dm = O.cheb(p)
    xi = np.cos(np.arange(n + 1) * math.pi / n)
    assert np.abs(x - ((a + b) / 2 + (b - a) / 2 * xi)).max() < 1e-15
    for k in range(n + 1):
        d = k * x ** (k - 1) if k else 0 * x
        assert np.abs(Dm @ x**k - d).max() < 1e-13 * max(1.0, np.abs(d).max()), k
    sc = 2.0 / (b - a)
    diag = np.r_[(2 * n * n + 1) / 6, -xi[1:-1] / (2 * (1 - xi[1:-1] ** 2)), -(2 * n * n + 1) / 6] * sc
    assert np.abs(np.diag(Dm) - diag).max() < 1e-12 * np.abs(diag).max()


def test_collocation_step_is_polynomial_exact():
    # D = d0, f = 0: (I - mu d0 D^2) u = rhs has the polynomial solution p whenever
    # rhs = p - mu d0 p'' at the interior nodes and deg p <= n, p(0) = p(1) = 0
    n, d0, mu = 10, 1.3, 0.05
    p = O.make_prob(Mx=n, N=4, P=1, alpha=0.5, basis="cheb", dpar=(d0, 0, 0, 0), fpar=(0,))
    x, _ = O.cheb(p)
    xi = x[1:-1]
    pv = xi**2 * (1 - xi) ** 2 * (1 + xi)
    # p = x^2 - x^3 - x^4 + x^5 ... expanded: x^2 (1 - 2x + x^2)(1 + x) = x^2 - x^3 - x^4 + x^5
    p2 = 2 - 6 * xi - 12 * xi**2 + 20 * xi**3
    got = O.step(p, np.zeros(n - 1), 0.0, mu, pv - mu * d0 * p2)
    assert np.abs(got - pv).max() < 1e-13


def _cheb_D_numpy(n, a, b):
    # independent construction: derivative of each Lagrange basis polynomial of the
    # nodes, fitted exactly by numpy's Chebyshev series and differentiated there
    from numpy.polynomial import chebyshev as C
    xi = np.cos(np.arange(n + 1) * math.pi / n)
    D = np.zeros((n + 1, n + 1))
    for j in range(n + 1):
        e = np.zeros(n + 1)
        e[j] = 1.0
        c = C.chebfit(xi, e, n)
        D[:, j] = C.chebval(xi, C.chebder(c)) * 2.0 / (b - a)
    return (a + b) / 2 + (b - a) / 2 * xi, D


def test_collocation_alpha_one_is_backward_euler_numpy():
    # alpha = 1: the uniform scheme is linearly-implicit backward Euler of
    # u_t = (D(u) u_x)_x + f, written here with numpy (independent matrices and solve)
    n, N = 10, 20
    dp, fp = (1.0, 0, 1.0, 0, 0.2), (0, 0, 0, 1.0)      # D = (1 + u)(1 + 0.2 sin 2 pi x), f = sin(pi x) e^{-t}
    p = O.make_prob(Mx=n, N=N, P=1, alpha=1.0, basis="cheb", dpar=dp, fpar=fp)
    x, Dn = _cheb_D_numpy(n, 0.0, 1.0)
    u = 0.3 * np.sin(math.pi * x[1:-1])
    W = O.serial_uni(p, u)
    dt = 1.0 / N
    for j in range(N):
        full = np.r_[0.0, u, 0.0]
        Dc = (1 + full) * (1 + 0.2 * np.sin(2 * math.pi * x))
        Nm = (Dn @ np.diag(Dc) @ Dn)[1:-1, 1:-1]
        f = np.sin(math.pi * x[1:-1]) * math.exp(-j * dt)
        u = np.linalg.solve(np.eye(n - 1) - dt * Nm, u + dt * f)
        assert np.abs(W[j + 1] - u).max() < 1e-12, j


def test_collocation_spectral_convergence_manufactured():
    # u = (1 + t^2) sin(pi x)/(2 - cos pi x), D = 1 + 0.5 sin(pi x), source S2: the
    # error at t = T falls geometrically in n until the time-discretisation floor
    errs = []
    for n in (6, 8, 12):
        p = O.make_prob(Mx=n, N=64, P=1, alpha=0.5, T=0.01, basis="cheb", dpar=(1.0, 0, 0, 0.5),
                        fpar=(0, 0, 0, 0, 0, 1.0))
        x, _ = O.cheb(p)
        xi = x[1:-1]
        s = np.sin(math.pi * xi) / (2 - np.cos(math.pi * xi))
        errs.append(np.abs(O.serial_uni(p, s)[-1] - (1 + 0.01**2) * s).max())
    assert errs[0] > 10 * errs[1] > 10 * errs[2] and errs[2] < 1e-5


def test_collocation_parareal_finite_termination_paper_shape():
    # the paper's model problem (D = 1 + u, f = sin(pi x) e^{-t}, u0 = x^4 (1-x)^4, alpha
    # = 0.5) on 2^4 intervals: after k iterations U^k_{0:k} is the sequential F sweep
    n, P, m = 16, 8, 4
    p = O.make_prob(Mx=n, N=P * m, P=P, alpha=0.5, basis="cheb", dpar=(1.0, 0, 1.0, 0), fpar=(0, 0, 0, 1.0))
    x, _ = O.cheb(p)
    u0 = x[1:-1] ** 4 * (1 - x[1:-1]) ** 4
    U, _, k = O.parareal(p, u0, tol=0.0)
    S = O.serial_hyb(p, u0)
    assert k == P
    for j in range(k + 1):
        assert np.abs(U[j][: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j


# ---------------------------------------------------------------- coarse propagator with substeps
def test_coarse_substeps_limits_and_fixed_point():
    # G with c L1 substeps per slice: c = 1 is the paper's G (bitwise), c = m is F itself,
    # so the initial coarse sweep already is S_hyb and one iteration confirms it; any c keeps
    # the exact prefix and the fixed point (Eq. PararealConvergence)
    K, P, m = 12, 6, 4
    kw = dict(Mx=K, N=P * m, P=P, alpha=0.45, dpar=(1, 0.5, 0, 0, 0.2), fpar=CFG1_F)
    u0 = cfg1_u0(K)
    S = O.serial_hyb(O.make_prob(**kw), u0)
    U1, e1, k1 = O.parareal(O.make_prob(**kw), u0, 1e-13)
    Uc1, ec1, kc1 = O.parareal(O.make_prob(coarse_substeps=1, **kw), u0, 1e-13)
    assert k1 == kc1 and np.array_equal(U1, Uc1)
    pm = O.make_prob(coarse_substeps=m, **kw)
    assert np.abs(O.coarse_sweep(pm, u0) - S).max() < 1e-14 * np.abs(S).max()
    Um, em, km = O.parareal(pm, u0, 1e-13)
    assert km == 1 and np.abs(Um[-1] - S).max() < 1e-14 * np.abs(S).max()
    U2, e2, k2 = O.parareal(O.make_prob(coarse_substeps=2, **kw), u0, 0.0)
    for j in range(k2 + 1):
        assert np.abs(U2[j][: j + 1] - S[: j + 1]).max() <= 1e-13 * np.abs(S).max(), j
    # two substeps contract faster than one
    _, ea, _ = O.parareal(O.make_prob(**kw), u0, 0.0, max_iter=3)
    _, eb, _ = O.parareal(O.make_prob(coarse_substeps=2, **kw), u0, 0.0, max_iter=3)
    assert eb[2] < ea[2]
