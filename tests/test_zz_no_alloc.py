"""The allocation-free fine propagator, psl1_fine_slice_noalloc.

Some callers cannot allocate device memory at the moment they call (a
real-time loop whose memory was planned in advance, or code under a memory
manager that forbids new allocations).  For them the library offers one
entry point whose scratch comes from a fixed device array compiled into the
library.  These tests check, through the C ABI, that it gives the same
result as the allocating entry point psl1_fine_slice on two calls in a row
(1D and 2D, FP64 and mixed precision, with the 2D working arrays in shared
memory and in the fixed array), that its second call leaves the device's
free memory unchanged, and that an instance whose scratch fills the array
exactly is accepted while one 256 doubles larger is rejected.  The file name
makes pytest collect it last, so a run that stops at the first failure has
run every other test.
"""
import numpy as np
import pytest

from paper_2510_11023_gb300 import psl1, workloads
from helpers import rel

pytestmark = pytest.mark.gpu
TOL = 1e-10          # the tolerance of the FP64-path parity tests
LIMIT = 512 * 1024   # doubles in the fixed scratch array (4 MiB)


def _check_twice(specs, P, u0, prec, slices):
    """Compare the allocation-free call with psl1_fine_slice on the given slices."""
    import torch
    K, m = specs[0].K, specs[0].nsteps // P
    with psl1.Problem(specs, P, precision=prec) as pr:
        pr.set_u0(u0)
        pr.solve_serial("coarse")
        U = pr.get_coeffs("serial")[0]
        for call, n in enumerate(slices):
            ref = pr.fine_slice(0, n, U[: n + 1])
            dU = torch.from_numpy(np.ascontiguousarray(U[: n + 1])).cuda()
            dV = torch.full((m + 1, K), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            pr.fine_slice_noalloc(0, n, dU.data_ptr(), dV.data_ptr())
            free1 = torch.cuda.mem_get_info()[0]
            got = dV.cpu().numpy()
            assert np.isfinite(got).all()
            assert rel(got, ref) < TOL, (call, rel(got, ref))
            if call == 1:
                assert free1 == free0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    wl = workloads.cfg1(K=40, N=64, P=4, alpha=0.35)
    _check_twice(wl.specs, wl.P, wl.u0_concat(), prec, (3, 2))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("modes", [(6, 5), (64, 64)], ids=["2d-smem", "2d-global-arrays"])
def test_noalloc_2d_matches_allocating_entry_point_twice(prec, modes):
    # 6 x 5 modes: every working array sits in shared memory; 64 x 64 modes
    # (128 x 128 nodes): the node arrays live in the scratch array
    spec = workloads.InstanceSpec(dim=2, modes=modes, nsteps=12, alpha=0.6, dpar=workloads.D_CFG5,
                                  fpar=workloads.F_SIN)
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal(spec.K) / (1.0 + np.arange(spec.K))
    _check_twice([spec], 3, u0, prec, (2, 1))


def _boundary_spec(K, m, P):
    return workloads.InstanceSpec(modes=(K, 1), nsteps=m * P, alpha=0.5, dpar=workloads.D_CFG1,
                                  fpar=workloads.F_COS)


@pytest.mark.parametrize("prec,m_at_limit", [
    # FP64: ring 256 m + factor 8*9/2 blocks of 32 x 32 = 36864 doubles
    ("fp64", (LIMIT - 36864) // 256),
    # mixed: ring 256 m + coarse differences (n+1) 256 with n = 1
    ("mixed", LIMIT // 256 - 2),
])
def test_noalloc_scratch_boundary(prec, m_at_limit):
    import torch
    K, P, n = 256, 2, 1
    # exactly at the limit: accepted, same result as the allocating entry point
    spec = _boundary_spec(K, m_at_limit, P)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(K) / np.arange(1, K + 1) ** 2
    with psl1.Problem([spec], P, precision=prec) as pr:
        pr.set_u0(u0)
        pr.solve_serial("coarse")
        U = pr.get_coeffs("serial")[0]
        ref = pr.fine_slice(0, n, U[: n + 1])
        dU = torch.from_numpy(np.ascontiguousarray(U[: n + 1])).cuda()
        dV = torch.zeros((m_at_limit + 1, K), dtype=torch.float64, device="cuda")
        pr.fine_slice_noalloc(0, n, dU.data_ptr(), dV.data_ptr())
        assert rel(dV.cpu().numpy(), ref) < TOL
    # one fine step more: 256 doubles over the limit, rejected before any launch
    spec = _boundary_spec(K, m_at_limit + 1, P)
    with psl1.Problem([spec], P, precision=prec) as pr:
        dU = torch.zeros((n + 1, K), dtype=torch.float64, device="cuda")
        dV = torch.zeros((m_at_limit + 2, K), dtype=torch.float64, device="cuda")
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.fine_slice_noalloc(0, n, dU.data_ptr(), dV.data_ptr())
        assert ei.value.status == -1
        assert "scratch" in str(ei.value) and str(LIMIT + 256) in str(ei.value)
