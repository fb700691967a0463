"""Full-size check of the batched 1D workload in the configuration bench.py
times: 256 instances with K in [64, 256], N = 64 m with m in [16, 64],
alpha in {0.3, 0.5, 0.7, 1}, P = 64, mixed precision, parareal run as one
CUDA graph with its device-driven iteration loop, with the refined F in every
iteration and with the inexact early iterations bench.py selects.

The oracle cannot solve 256 full instances in test time, so it recomputes
sampled outputs one at a time.  Parareal's fixed point is the sequential
fine sweep (Eq. PararealConvergence): its states satisfy
U_{n+1} = F_n(U_{0:n}).  For sampled (instance, slice) pairs the oracle's
fine propagator, applied to the GPU's own converged states U_{0:n}, must
give the GPU's U_{n+1}; U_0 must be u0.  Properties that hold at any size
cover the rest of the batch: the iterate equals the GPU's same-precision
serial hybrid solve for every instance, and is finite.
Tolerance: 1e-10 relative (the whole-solve tolerance of the mixed path)."""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _samples(wl):
    """(instance, slice) pairs: the largest K, the longest slice, an alpha = 1
    instance, and one more; first, middle and last slices among them; and two
    instances with K >= 250 and the smallest alpha (the largest mu = dt^a
    Gamma(2-a), the worst-conditioned steps), late slices."""
    K = np.array([s.K for s in wl.specs])
    m = np.array([s.nsteps // wl.P for s in wl.specs])
    a = np.array([s.alpha for s in wl.specs])
    big_k = int(np.argmax(K))
    long_m = int(np.argmax(m * (K < 200)))          # long slice, moderate K (oracle time)
    be = int(np.flatnonzero(a == 1.0)[0])
    other = int(np.argmin(K))
    P = wl.P
    hard = np.flatnonzero((K >= 250) & (a == a.min()))
    hard = hard[np.argsort(m[hard])][:2]             # the two shortest slices among them (oracle time)
    return [(big_k, P - 1), (long_m, 0), (long_m, P // 2), (be, 3 * P // 4), (other, 1), (other, P - 1)] + \
        [(int(hard[0]), P - 2), (int(hard[1]), P // 2 + 7)]


@pytest.mark.parametrize("inexact", [0.0, 1e-5])
def test_full_size_batched_1d_graph_parareal_against_sampled_oracle(inexact):
    # inexact = 1e-5: the early iterations bench.py selects (the FP32 step on
    # slices n > k while the increment exceeds 1e-5)
    wl = workloads.cfg2()               # the benched batch: B = 256, seed 20251011
    assert wl.B == 256 and wl.P == 64
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.set_inexact_fine(inexact)
        pr.set_graph(True)
        k = pr.solve_parareal(tol=1e-12)
        U = pr.get_coeffs("parareal")
        its = pr.get_iterations()
        pr.solve_serial("hybrid")
        S = pr.get_coeffs("serial")
    assert 1 <= k <= wl.P and (its >= 1).all() and (its <= wl.P).all()
    for b in range(wl.B):
        assert np.isfinite(U[b]).all(), b
        assert np.array_equal(U[b][0], wl.u0[b]), b
        assert rel(U[b], S[b]) < TOL, (b, rel(U[b], S[b]))
    for b, n in _samples(wl):
        spec = wl.specs[b]
        V = O.fine_slice(oracle_prob(spec, wl.P), n, U[b][: n + 1])
        assert rel(U[b][n + 1], V[-1]) < TOL, (b, n, spec.K, spec.alpha, rel(U[b][n + 1], V[-1]))
