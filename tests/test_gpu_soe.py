"""GPU parity of the fast (sum-of-exponentials) history of the uniform L1
scheme, through the C ABI.

The library computes each instance's exponentials on the host (Sturm-sequence
bisection and Christoffel weights) and the oracle computes them its own way
(Jacobi-rotation eigenvectors, Newton for Gauss-Legendre): the two sets must
agree.  The GPU solve (the exponential state updated once per step) must match
the oracle's uniform scheme with the approximated weights written out as a
plain sum, and stay within rounding of the exact-history uniform solve.

Tolerances: exponents and weights 1e-12 relative; solves 1e-10 relative (FP64
and mixed), as for the other serial solvers.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _batch():
    # uneven K, N from below the local window (10) to several hundred steps,
    # alpha = 1 (no history), K not a multiple of 32
    rng = np.random.default_rng(12)
    shapes = [(7, 200, 0.3), (33, 64, 0.5), (40, 120, 1.0), (64, 10, 0.7), (19, 300, 0.2)]
    specs, u0 = [], []
    for K, N, a in shapes:
        specs.append(workloads.InstanceSpec(modes=(K, 1), nsteps=N, alpha=a, dpar=workloads.D_CFG2,
                                            fpar=workloads.F_COS))
        u0.append(rng.standard_normal(K) / np.arange(1, K + 1) ** 2)
    return specs, u0


def test_exponentials_agree_with_the_oracle():
    specs, u0 = _batch()
    with psl1.Problem(specs, 2) as pr:
        for b, s in enumerate(specs):
            sg, wg = pr.get_soe(b)
            so, wo = O.soe_nodes(s.alpha, s.nsteps)
            assert len(sg) == len(so), b
            if len(so):
                assert np.abs(sg / so - 1).max() < 1e-12 and np.abs(wg / wo - 1).max() < 1e-12, b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fast_uniform_solve_matches_oracle(prec):
    specs, u0 = _batch()
    P = 2
    with psl1.Problem(specs, P, precision=prec) as pr:
        pr.set_u0(np.concatenate(u0))
        pr.solve_serial("uniform-soe")
        W = pr.get_coeffs("serial")
        pr.solve_serial("uniform-soe")          # replay of the captured graph: same result
        W2 = pr.get_coeffs("serial")
    for b, s in enumerate(specs):
        op = oracle_prob(s, P)
        ref = O.serial_uni_soe(op, u0[b])[:: op.m]
        assert rel(W[b], ref) < TOL, (b, rel(W[b], ref))
        assert np.array_equal(W[b], W2[b])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fast_uniform_solve_matches_exact_history_at_full_size(prec):
    # eight instances of the batched 1D workload (K up to 256, N up to 4096): the
    # fast history stays within rounding of the exact-history uniform solve
    wl = workloads.cfg2(B=8)
    with psl1.Problem(wl, precision=prec) as pr:
        pr.solve_serial("uniform")
        W = pr.get_coeffs("serial")
        pr.solve_serial("uniform-soe")
        Ws = pr.get_coeffs("serial")
        st = pr.stats()
    for b in range(wl.B):
        assert rel(Ws[b], W[b]) < 1e-11, (b, rel(Ws[b], W[b]))
    assert st["kernel_launches"] == 1 + max(s.nsteps for s in wl.specs)
