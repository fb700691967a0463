"""Writes step2d_64x64.txt and fine2d_64x64.txt: the oracle's results at the
64 x 64-mode, 128 x 128-node size of the 2D batched workload, with its
D = 1 + 0.5/(1+u^2) (1 + 0.3 cos 2 pi y) and f = 0.1 sin u, alpha = 0.6:

  step2d_64x64.txt  one L1 step (Eq. NumericalSchemeFine, one linearised SPD
                    solve) from c = u0 of the workload's first instance with
                    hist = c + 0.01 z / (k^2 + l^2) (seed 9), t_e = 0.25 and
                    mu = Gamma(2-a) dt^a for N = 8192;
  fine2d_64x64.txt  the fine propagator F_2 (Eq. FinePropagator, m = 2 fine
                    steps, coarse history of U_0, U_1, U_2) of the same
                    instance with P = 4, N = 8: U_0 = c and
                    U_j = U_{j-1} + 0.05 z_j / (k^2 + l^2) (seeds 21, 22).

The oracle's dense K x K x Q assembly is out of reach at K = 4096, Q = 16384,
so these steps are solved by the oracle's conjugate gradients on the weak
form (solver "cg"; the CPU pins check it against the dense Cholesky solve).
About a few minutes of CPU.  Run from the repository root:
    python tests/golden/make_2d_64x64.py
"""
import dataclasses
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2510_11023_gb300 import workloads  # noqa: E402

STEP = os.path.join(HERE, "step2d_64x64.txt")
FINE = os.path.join(HERE, "fine2d_64x64.txt")


def _smooth(seed, Mx, My):
    k = np.arange(1, Mx + 1)[:, None]
    l = np.arange(1, My + 1)[None, :]
    return (np.random.default_rng(seed).standard_normal((Mx, My)) / (k * k + l * l)).reshape(-1)


def step_inputs():
    """(spec, P, c, hist, te, mu) of the stored step."""
    wl = workloads.cfg5(B=1)
    spec = wl.specs[0]
    c = np.asarray(wl.u0[0], dtype=np.float64)
    hist = c + 0.01 * _smooth(9, *spec.modes)
    mu = O.gamma2a(spec.alpha) * (spec.T / spec.nsteps) ** spec.alpha
    return spec, wl.P, c, hist, 0.25, mu


def fine_inputs():
    """(spec, P, n, U) of the stored fine propagator: P = 4 slices of m = 2 steps."""
    spec, _, c, _, _, _ = step_inputs()
    spec = dataclasses.replace(spec, nsteps=8)
    U = [c]
    for s in (21, 22):
        U.append(U[-1] + 0.05 * _smooth(s, *spec.modes))
    return spec, 4, 2, np.array(U)


def _prob(spec, P):
    return O.make_prob(dim=2, Mx=spec.modes[0], My=spec.modes[1], N=spec.nsteps, P=P, alpha=spec.alpha, T=spec.T,
                       lo=spec.lo, hi=spec.hi, dpar=spec.dpar, fpar=spec.fpar, solver="cg")


def _write(path, what, v):
    with open(path, "w") as f:
        f.write("# oracle %s, 2D 64 x 64 modes, 128 x 128 nodes; written by make_2d_64x64.py\n" % what)
        for x in v:
            f.write("%.17e\n" % x)


def main():
    spec, P, c, hist, te, mu = step_inputs()
    _write(STEP, "step (Eq. NumericalSchemeFine)", O.step(_prob(spec, P), c, te, mu, hist))
    spec, P, n, U = fine_inputs()
    V = O.fine_slice(_prob(spec, P), n, U)
    _write(FINE, "fine propagator F_2 (Eq. FinePropagator), final state", V[-1])


if __name__ == "__main__":
    main()
