"""Writes step2d_32x32.txt: the oracle's one L1 step (Eq. NumericalSchemeFine,
one linearised SPD solve) of the 2D single-instance workload at its full size,
32 x 32 sine modes on 64 x 64 Gauss-Legendre nodes, D = 1 + 0.5/(1+u^2),
f = 0.05 u (1-u).  The CPU oracle needs about two minutes for this step (its
stiffness matrix is a plain K x K x Q sum), so the GPU test compares with this
stored copy.  Run from the repository root:  python tests/golden/make_step2d_32x32.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2510_11023_gb300 import workloads  # noqa: E402

OUT = os.path.join(HERE, "step2d_32x32.txt")


def inputs():
    """(spec, P, c, hist, te, mu) of the stored step: c = u0 of the workload,
    hist = c + 0.01 z / (k^2 + l^2) (seed 9), te = 0.25, mu = Gamma(2-a) dt^a."""
    wl = workloads.cfg3()
    spec = wl.specs[0]
    Mx, My = spec.modes
    k = np.arange(1, Mx + 1)[:, None]
    l = np.arange(1, My + 1)[None, :]
    z = np.random.default_rng(9).standard_normal((Mx, My)) / (k * k + l * l)
    c = np.asarray(wl.u0[0], dtype=np.float64)
    hist = c + 0.01 * z.reshape(-1)
    mu = O.gamma2a(spec.alpha) * (spec.T / spec.nsteps) ** spec.alpha
    return spec, wl.P, c, hist, 0.25, mu


def main():
    spec, P, c, hist, te, mu = inputs()
    p = O.make_prob(dim=2, Mx=spec.modes[0], My=spec.modes[1], N=spec.nsteps, P=P, alpha=spec.alpha, T=spec.T,
                    lo=spec.lo, hi=spec.hi, dpar=spec.dpar, fpar=spec.fpar)
    out = O.step(p, c, te, mu, hist)
    with open(OUT, "w") as f:
        f.write("# oracle step (Eq. NumericalSchemeFine), 2D 32 x 32 modes, 64 x 64 nodes; "
                "written by make_step2d_32x32.py\n")
        for v in out:
            f.write("%.17e\n" % v)


if __name__ == "__main__":
    main()
