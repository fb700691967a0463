"""The property that makes inexact early parareal iterations safe, checked on
the CPU with the oracle's own propagators (no GPU).

Parareal (Eq. Parareal with the stored G_old of the flowchart) computes, at
iteration k, U^{k+1}_{n+1} = G_n(U^{k+1}_{0:n}) + F_n(U^k_{0:n}) - G_old(n).
Slices n < k are already exact.  If F is evaluated inexactly only on slices
n > k, then U^{k+1}_{0:k+1} still equals the sequential fine sweep S_hyb
(Eq. PararealConvergence): G_n(U^{k+1}_{0:k}) and G_old(k) have the same
arguments, so U^{k+1}_{k+1} = F_k(U^k_{0:k}), which is exact.  The iteration
therefore still ends at S_hyb after at most P iterations, and converges to
it once the inexactness stops.  Here the inexact F is the oracle's F with a
seeded relative perturbation of 1e-6, a stand-in for the FP32 step."""
import numpy as np

import oracle as O

D = (1.0, 0.5, 0, 0, 0.2, 0, 0, 0)     # (1 + 0.5/(1+u^2)) (1 + 0.2 sin 2 pi x)
F = (0.1, 0, 0, 0, 0, 0, 0, 0)         # 0.1 cos u


def _parareal(op, u0, inexact, tol, rng):
    """Parareal by hand from the oracle's F_n and G_n; inexact(k, e_prev) says
    whether the slices n > k of iteration k take the perturbed F."""
    P, K = op.P, op.K
    U = O.coarse_sweep(op, u0)
    Gold = [O.coarse_step(op, n, U[: n + 1]) for n in range(P)]
    iterates, e_prev = [U.copy()], np.inf
    for k in range(P):
        loose = inexact(k, e_prev)
        Fv = {}
        for n in range(k, P):
            Fv[n] = O.fine_slice(op, n, U[: n + 1])[-1]
            if loose and n > k:
                Fv[n] = Fv[n] * (1.0 + 1e-6 * rng.standard_normal(K))
        Un = U.copy()
        for n in range(k, P):
            g = O.coarse_step(op, n, Un[: n + 1])
            Un[n + 1] = g + Fv[n] - Gold[n]
            Gold[n] = g
        num = max(np.linalg.norm(Un[n] - U[n]) for n in range(P + 1))
        den = max(np.linalg.norm(Un[n]) for n in range(P + 1))
        e_prev = num / den
        U = Un
        iterates.append(U.copy())
        if e_prev <= tol:
            break
    return U, iterates


def _problem(P=8, m=4, K=10, alpha=0.6, seed=3):
    op = O.make_prob(Mx=K, N=P * m, P=P, alpha=alpha, dpar=D, fpar=F)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(K) * np.arange(1, K + 1, dtype=np.float64) ** -2.0
    return op, u0


def test_exact_prefix_with_every_later_slice_inexact():
    op, u0 = _problem()
    S = O.serial_hyb(op, u0)
    U, its = _parareal(op, u0, lambda k, e: True, 0.0, np.random.default_rng(1))
    scale = np.abs(S).max()
    assert len(its) == op.P + 1
    for k, Uk in enumerate(its):
        j = min(k, op.P)
        assert np.abs(Uk[: j + 1] - S[: j + 1]).max() <= 1e-13 * scale, k
    assert np.abs(U - S).max() <= 1e-13 * scale
    # the perturbation is really there: an intermediate iterate is off by ~1e-6 beyond its prefix
    mid = its[2]
    assert np.abs(mid[4:] - S[4:]).max() > 1e-9 * scale


def test_inexact_while_increment_large_converges_to_serial():
    op, u0 = _problem(P=16, m=3, K=12, alpha=0.4, seed=4)
    S = O.serial_hyb(op, u0)
    U, its = _parareal(op, u0, lambda k, e: k == 0 or e > 1e-4, 1e-13, np.random.default_rng(2))
    assert np.abs(U - S).max() <= 1e-11 * np.abs(S).max()
    assert len(its) - 1 < op.P          # converged before the finite-termination bound
