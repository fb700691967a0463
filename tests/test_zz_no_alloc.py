"""The allocation-free fine propagator, psl1_fine_slice_noalloc.

Some callers cannot allocate device memory at the moment they call (a
real-time loop whose memory was planned in advance, or code under a memory
manager that forbids new allocations).  For them the library offers one
entry point whose scratch comes from a fixed device array compiled into the
library.  These tests check, through the C ABI, that it gives the same
result as the allocating entry point psl1_fine_slice on two calls in a row,
that it leaves the device's free memory unchanged, and that it rejects
instances whose scratch does not fit.  The file name makes pytest collect it
last, so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2510_11023_gb300 import psl1, workloads
from helpers import rel

pytestmark = pytest.mark.gpu
TOL = 1e-10   # the tolerance of the FP64-path parity tests


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    import torch
    wl = workloads.cfg1(K=40, N=64, P=4, alpha=0.35)
    K, m = 40, 16
    with psl1.Problem(wl, precision=prec) as pr:
        pr.solve_serial("coarse")
        U = pr.get_coeffs("serial")[0]
        for call, n in enumerate((3, 2)):
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


def test_noalloc_rejects_oversized_instance():
    # m K = 2048 * 256 doubles = 4 MiB of history ring alone: more than the fixed array
    spec = workloads.InstanceSpec(modes=(256, 1), nsteps=2048, alpha=0.5, dpar=workloads.D_CFG1,
                                  fpar=workloads.F_COS)
    import torch
    with psl1.Problem([spec], 1, precision="fp64") as pr:
        dU = torch.zeros((1, 256), dtype=torch.float64, device="cuda")
        dV = torch.zeros((2049, 256), dtype=torch.float64, device="cuda")
        with pytest.raises(psl1.PSL1Error) as ei:
            pr.fine_slice_noalloc(0, 0, dU.data_ptr(), dV.data_ptr())
        assert ei.value.status == -1
        assert "scratch" in str(ei.value)
