"""Profiling case of the uniform solver's history stream (k_uni_hist): 96
instances with K = 256 modes and N = 1024 fine steps, mixed precision.  The
fine history is 2 MB per instance, 192 MB in all (larger than the 126 MB L2),
so every history launch streams from HBM.  Runs the uniform serial solve twice
(the first builds its CUDA graph) and prints the second one's wall time.

    python -m paper_2510_11023_gb300.uniform_history_case
"""
import time

import numpy as np

from paper_2510_11023_gb300 import psl1, workloads
def main():
    specs = [workloads.InstanceSpec(modes=(256, 1), nsteps=1024, alpha=0.5, dpar=workloads.D_CFG2,
                                    fpar=workloads.F_COS) for _ in range(96)]
    rng = np.random.default_rng(1)
    u0 = [rng.standard_normal(256) * np.arange(1, 257) ** -2.0 for _ in specs]
    wl = workloads.Workload("uniform history case", 64, specs, u0)
    with psl1.Problem(wl, precision="mixed") as pr:
        pr.solve_serial("uniform")
        t = time.perf_counter()
        pr.solve_serial("uniform")
        dt = time.perf_counter() - t
    hist_bytes = sum(s.K * 8 * s.nsteps * (s.nsteps - 1) / 2 for s in specs)
    print({"uniform_solve_s": dt, "history_bytes": hist_bytes})


if __name__ == "__main__":
    main()
