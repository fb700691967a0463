"""Helpers shared by the tests: map workload specs onto the oracle's records."""
import numpy as np

import oracle as O


def oracle_prob(spec, P):
    return O.make_prob(dim=spec.dim, Mx=spec.modes[0], My=spec.modes[1], Qx=spec.qnodes[0] or None,
                       Qy=spec.qnodes[1] or None, N=spec.nsteps, P=P, alpha=spec.alpha, T=spec.T,
                       lo=spec.lo, hi=spec.hi, dpar=spec.dpar, fpar=spec.fpar, basis=spec.basis)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
