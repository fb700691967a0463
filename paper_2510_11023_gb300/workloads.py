"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws sizes, parameters and initial coefficients; it holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle
take their inputs from here.

Coefficient families (see include/psl1.h):
  D = (d0 + d1/(1+u^2) X1 + d2 u + d3 sin(pi x)) X0,  X_i = 1 + a_i sin 2pi x + b_i cos 2pi y
      dpar = (d0, d1, d2, d3, a0, b0, a1, b1)
  f = c0 cos u + c1 sin u + c2 u(1-u) + c3 sin(pi x) e^{-t} + c4 S1 + c5 S2
      fpar = (c0, c1, c2, c3, c4, c5, 0, 0)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class InstanceSpec:
    dim: int = 1
    modes: tuple = (32, 1)
    qnodes: tuple = (0, 0)          # 0 selects twice the modes
    nsteps: int = 256
    alpha: float = 0.5
    T: float = 1.0
    lo: tuple = (0.0, 0.0)
    hi: tuple = (1.0, 1.0)
    dpar: tuple = (1.0, 0.5, 0, 0, 0, 0, 0, 0)
    fpar: tuple = (0.1, 0, 0, 0, 0, 0, 0, 0)
    basis: str = "sine"             # "sine" (Galerkin, modes) or "cheb" (collocation, modes[0] intervals)

    @property
    def K(self) -> int:
        if self.basis == "cheb":
            return self.modes[0] - 1
        return self.modes[0] * (self.modes[1] if self.dim == 2 else 1)

    @property
    def Q(self) -> int:
        qx = self.qnodes[0] or 2 * self.modes[0]
        if self.dim == 2:
            return qx * (self.qnodes[1] or 2 * self.modes[1])
        return qx


@dataclass
class Workload:
    name: str
    P: int
    specs: list
    u0: list                          # one float64 array of K coefficients per instance
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return len(self.specs)

    def u0_concat(self) -> np.ndarray:
        return np.concatenate([np.asarray(u, dtype=np.float64) for u in self.u0])


D_CFG1 = (1.0, 0.5, 0, 0, 0, 0, 0, 0)          # 1 + 0.5/(1+u^2)
D_CFG2 = (1.0, 0.5, 0, 0, 0.2, 0, 0, 0)        # (1 + 0.5/(1+u^2)) (1 + 0.2 sin 2 pi x)
F_COS = (0.1, 0, 0, 0, 0, 0, 0, 0)             # 0.1 cos u
D_CFG5 = (1.0, 0.5, 0, 0, 0, 0, 0, 0.3)        # 1 + 0.5/(1+u^2) (1 + 0.3 cos 2 pi y)
F_SIN = (0, 0.1, 0, 0, 0, 0, 0, 0)             # 0.1 sin u


def cfg1(K: int = 32, N: int = 256, P: int = 8, alpha: float = 0.5) -> Workload:
    """1D plain method: K sine modes, 2K Gauss nodes, N L1 steps, P slices,
    u0 = sin(pi x) + 0.5 sin(3 pi x), i.e. c_1 = 1/sqrt2, c_3 = 0.5/sqrt2."""
    u0 = np.zeros(K)
    u0[0] = 1.0 / math.sqrt(2.0)
    if K >= 3:
        u0[2] = 0.5 / math.sqrt(2.0)
    spec = InstanceSpec(modes=(K, 1), nsteps=N, alpha=alpha, dpar=D_CFG1, fpar=F_COS)
    return Workload("1D plain, K=%d N=%d P=%d alpha=%g" % (K, N, P, alpha), P, [spec], [u0])


def cfg1_manufactured(K: int = 32, N: int = 256, P: int = 8, alpha: float = 0.5) -> Workload:
    """Manufactured case u = (1 + t^alpha) sin(pi x) with its source S1."""
    u0 = np.zeros(K)
    u0[0] = 1.0 / math.sqrt(2.0)
    spec = InstanceSpec(modes=(K, 1), nsteps=N, alpha=alpha, dpar=D_CFG1, fpar=(0, 0, 0, 0, 1, 0, 0, 0))
    return Workload("1D manufactured (1+t^a) sin(pi x)", P, [spec], [u0])


def cfg2(B: int = 256, seed: int = 20251011, P: int = 64, kmin: int = 64, kmax: int = 256,
         mmin: int = 16, mmax: int = 64, alphas=(0.3, 0.5, 0.7, 1.0)) -> Workload:
    """1D batched: B instances with K ~ U{kmin..kmax}, N = P m with m ~ U{mmin..mmax}
    (so that P | N; N in [1024, 4096] for the defaults), alpha from `alphas`,
    u0 coefficients z_k k^-2 with z ~ N(0,1), D = (1 + 0.5/(1+u^2))(1 + 0.2 sin 2 pi x),
    f = 0.1 cos u."""
    rng = np.random.default_rng(seed)
    Ks = rng.integers(kmin, kmax + 1, size=B)
    ms = rng.integers(mmin, mmax + 1, size=B)
    al = rng.choice(np.asarray(alphas, dtype=np.float64), size=B)
    specs, u0 = [], []
    for b in range(B):
        K = int(Ks[b])
        specs.append(InstanceSpec(modes=(K, 1), nsteps=int(P * ms[b]), alpha=float(al[b]), dpar=D_CFG2, fpar=F_COS))
        z = rng.standard_normal(K)
        u0.append(z * np.arange(1, K + 1, dtype=np.float64) ** -2.0)
    return Workload("1D batched B=%d K in [%d,%d] N=P*m m in [%d,%d] P=%d" % (B, kmin, kmax, mmin, mmax, P), P,
                    specs, u0, {"seed": seed})


def cfg4_trajectories(n: int, seed: int, K: int = 128, N: int = 4096, P: int = 64,
                      amin: float = 0.2, amax: float = 1.0) -> Workload:
    """Learned-coarse-propagator data: n instances with K = 128, N = 4096, P = 64,
    alpha ~ U[amin, amax], u0 and D, f as in the batched workload."""
    rng = np.random.default_rng(seed)
    specs, u0 = [], []
    for _ in range(n):
        a = float(rng.uniform(amin, amax))
        specs.append(InstanceSpec(modes=(K, 1), nsteps=N, alpha=a, dpar=D_CFG2, fpar=F_COS))
        u0.append(rng.standard_normal(K) * np.arange(1, K + 1, dtype=np.float64) ** -2.0)
    return Workload("1D learned-G data n=%d K=%d N=%d P=%d" % (n, K, N, P), P, specs, u0, {"seed": seed})


def e1(K: int = 16, P: int = 256, m: int = 32, alpha: float = 0.5) -> Workload:
    """The paper's model problem shape (Sec. 4.2): D = 1 + u, f = sin(pi x) e^{-t},
    u0 = x^4 (1-x)^4, alpha = 0.5, 2^4 modes, P = 2^8 slices, m = 2^5 fine steps.
    u0's sine coefficients sqrt2 int_0^1 x^4(1-x)^4 sin(k pi x) dx are taken by
    a 64-point Gauss rule (exact to rounding for this smooth integrand)."""
    xg, wg = np.polynomial.legendre.leggauss(64)
    x, w = (xg + 1) / 2, wg / 2
    k = np.arange(1, K + 1)
    u0 = (w[None, :] * (x**4 * (1 - x) ** 4)[None, :] * math.sqrt(2) * np.sin(np.pi * k[:, None] * x[None, :])).sum(1)
    spec = InstanceSpec(modes=(K, 1), nsteps=P * m, alpha=alpha, dpar=(1.0, 0, 1.0, 0, 0, 0, 0, 0),
                        fpar=(0, 0, 0, 1.0, 0, 0, 0, 0))
    return Workload("paper E1 shape K=%d P=%d m=%d" % (K, P, m), P, [spec], [u0])


def e1_collocation(n: int = 16, P: int = 256, m: int = 32, alpha: float = 0.5) -> Workload:
    """The paper's model problem with its own spatial scheme (Sec. 4.1-4.2):
    Chebyshev-Lobatto collocation on n = 2^4 intervals of [0,1], D = 1 + u,
    f = sin(pi x) e^{-t}, u0 = x^4 (1-x)^4 sampled at the interior nodes
    x_j = (1 + cos(j pi/n))/2, j = 1..n-1, alpha = 0.5, P = 2^8, m = 2^5."""
    x = 0.5 * (1.0 + np.cos(np.arange(1, n) * math.pi / n))
    u0 = x**4 * (1 - x) ** 4
    spec = InstanceSpec(modes=(n, 1), nsteps=P * m, alpha=alpha, dpar=(1.0, 0, 1.0, 0, 0, 0, 0, 0),
                        fpar=(0, 0, 0, 1.0, 0, 0, 0, 0), basis="cheb")
    return Workload("paper model problem, collocation n=%d P=%d m=%d" % (n, P, m), P, [spec], [u0])


def _u0_2d(rng, Mx: int, My: int) -> np.ndarray:
    """c_kl = z_kl / (k^2 + l^2), z ~ N(0, 1), row-major with the y mode fastest."""
    k = np.arange(1, Mx + 1, dtype=np.float64)[:, None]
    l = np.arange(1, My + 1, dtype=np.float64)[None, :]
    return (rng.standard_normal((Mx, My)) / (k * k + l * l)).reshape(-1)


def cfg3(M: int = 32, N: int = 2048, P: int = 128, alpha: float = 0.4, seed: int = 20251012) -> Workload:
    """2D, one instance: Mx = My = M modes, 2M x 2M Gauss nodes, D = 1 + 0.5/(1+u^2),
    f = 0.05 u (1-u), u0 coefficients z / (k^2 + l^2)."""
    rng = np.random.default_rng(seed)
    spec = InstanceSpec(dim=2, modes=(M, M), nsteps=N, alpha=alpha, dpar=D_CFG1, fpar=(0, 0, 0.05, 0, 0, 0, 0, 0))
    return Workload("2D M=%d x %d N=%d P=%d alpha=%g" % (M, M, N, P, alpha), P, [spec], [_u0_2d(rng, M, M)],
                    {"seed": seed})


def cfg5(B: int = 16, M: int = 64, N: int = 8192, P: int = 256, alpha: float = 0.6,
         seed: int = 20251015) -> Workload:
    """2D batched: B instances, Mx = My = M modes, 2M x 2M Gauss nodes,
    D = 1 + 0.5/(1+u^2) (1 + 0.3 cos 2 pi y), f = 0.1 sin u, u0 coefficients z / (k^2 + l^2)."""
    rng = np.random.default_rng(seed)
    specs, u0 = [], []
    for _ in range(B):
        specs.append(InstanceSpec(dim=2, modes=(M, M), nsteps=N, alpha=alpha, dpar=D_CFG5, fpar=F_SIN))
        u0.append(_u0_2d(rng, M, M))
    return Workload("2D batched B=%d M=%d x %d N=%d P=%d alpha=%g" % (B, M, M, N, P, alpha), P, specs, u0,
                    {"seed": seed})


def small_batch_2d(seed: int = 6, P: int = 4) -> Workload:
    """A small ragged 2D batch for parity tests: Mx != My, odd mode counts,
    non-default node counts, a non-unit box, y-dependent D, mixed alpha including 1."""
    rng = np.random.default_rng(seed)
    shapes = [((5, 7), (0, 0)), ((8, 8), (0, 0)), ((12, 9), (26, 20)), ((3, 16), (0, 0))]
    ms = [3, 2, 4, 1]
    al = [0.4, 1.0, 0.6, 0.3]
    dps = [D_CFG1, (1.0, 0.5, 0, 0, 0.1, 0.2, 0, 0.3), (0.8, 0.4, 0, 0.2, 0, 0, 0.2, 0), (1.0, 0.5, 0, 0, 0, 0, 0, 0.3)]
    fps = [(0, 0, 0.05, 0, 0, 0, 0, 0), (0, 0.1, 0, 0, 0, 0, 0, 0), F_COS, (0, 0, 0, 0.5, 0, 0, 0, 0)]
    specs, u0 = [], []
    for b in range(len(shapes)):
        (mx, my), (qx, qy) = shapes[b]
        lo, hi = ((-0.5, 0.25), (1.0, 2.0)) if b == 2 else ((0.0, 0.0), (1.0, 1.0))
        specs.append(InstanceSpec(dim=2, modes=(mx, my), qnodes=(qx, qy), nsteps=P * ms[b], alpha=al[b], lo=lo, hi=hi,
                                  dpar=dps[b], fpar=fps[b]))
        u0.append(_u0_2d(rng, mx, my))
    return Workload("small ragged 2D batch", P, specs, u0, {"seed": seed})


def small_batch(seed: int = 5, B: int = 5, P: int = 4) -> Workload:
    """A small ragged batch for parity tests: uneven K (including K not a multiple
    of 32 and K > 32), uneven m, mixed alpha including alpha = 1."""
    rng = np.random.default_rng(seed)
    Ks = [7, 33, 40, 64, 19][:B]
    ms = [3, 2, 5, 1, 4][:B]
    al = [0.3, 0.5, 1.0, 0.7, 0.45][:B]
    specs, u0 = [], []
    for b in range(B):
        specs.append(InstanceSpec(modes=(Ks[b], 1), nsteps=P * ms[b], alpha=al[b], dpar=D_CFG2, fpar=F_COS))
        u0.append(rng.standard_normal(Ks[b]) * np.arange(1, Ks[b] + 1, dtype=np.float64) ** -2.0)
    return Workload("small ragged batch", P, specs, u0, {"seed": seed})
