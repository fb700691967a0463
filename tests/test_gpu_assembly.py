"""Dense stiffness assembly A = Phi'^T diag(w D) Phi' (Eq. AForm) on the tensor
cores (tcgen05, BF16 operands, FP32 accumulation) and by the Toeplitz+Hankel
moments (FP32), through the C ABI, against the oracle's assembled matrix.

Tolerance of the tensor-core result, from its arithmetic: Phi' is rounded to
BF16 (unit roundoff 2^-9) in both operands and w D Phi' is rounded again, so
each term w_q D_q phi_k' phi_l' carries a relative error of at most about
3 * 2^-9; with D > 0, Cauchy-Schwarz bounds the sum of the term magnitudes by
sqrt(A_kk A_ll), hence |A_tc - A|_kl <= 2^-7 sqrt(A_kk A_ll) (FP32
accumulation adds ~Q 2^-24, far below).  The FP32 moments: 1e-4 of the same
scale.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_11023_gb300 import psl1, workloads
from helpers import oracle_prob

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [7, 33, 64, 128, 200, 256])
def test_dense_assembly_against_oracle(K):
    spec = workloads.InstanceSpec(modes=(K, 1), nsteps=4, alpha=0.5, dpar=workloads.D_CFG2, fpar=workloads.F_COS,
                                  lo=(0.25, 0.0), hi=(1.5, 1.0))
    op = oracle_prob(spec, 1)
    x, _, _ = O.nodes(op)
    order = np.argsort(x)
    rng = np.random.default_rng(K)
    units = 3
    Dn = 0.6 + rng.random((units, spec.Q))                   # positive nodal D, oracle node order
    with psl1.Problem([spec], 1) as pr:
        At, ms_t = pr.assemble(0, Dn[:, order], "tensor")
        Am, ms_m = pr.assemble(0, Dn[:, order], "moments")
    assert ms_t > 0 and ms_m > 0
    for u in range(units):
        ref = O.stiffness(op, Dn[u])
        scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.all(np.abs(At[u] - ref) <= 2.0**-7 * scale), (u, np.max(np.abs(At[u] - ref) / scale))
        assert np.all(np.abs(Am[u] - ref) <= 1e-4 * scale), (u, np.max(np.abs(Am[u] - ref) / scale))
        # the tensor-core result is not exact: its error is of BF16 size, not FP32 size
        assert np.max(np.abs(At[u] - ref) / scale) > 1e-6


def test_dense_assembly_rejections():
    spec = workloads.InstanceSpec(modes=(300, 1), nsteps=4, alpha=0.5)
    with psl1.Problem([spec], 1) as pr:
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.assemble(0, np.ones((1, spec.Q)), "tensor")     # K > 256: one MMA covers N <= 256
        assert ei.value.status == -1
        A, _ = pr.assemble(0, np.ones((1, spec.Q)), "moments")
        assert A.shape == (1, 300, 300)
