"""ctypes wrapper of the plain serial FP64 CPU oracle (``psl1_oracle.c``).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` import it; the product
package never does, and the two share no code.

Every function is a thin marshalling layer over the C oracle; the arithmetic
lives in ``psl1_oracle.c`` (each C function cites the paper's equation it
follows).  The shared library is compiled on first use with gcc
(``-O2 -ffp-contract=off``) if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psl1_oracle.c")
_LIB = os.path.join(_HERE, "_psl1_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_psl1_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

D_, P_ = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)


class Prob(ctypes.Structure):
    """Mirror of ``orc_prob`` (see psl1_oracle.c for the coefficient families)."""

    _fields_ = [
        ("dim", ctypes.c_int), ("Mx", ctypes.c_int), ("My", ctypes.c_int),
        ("Qx", ctypes.c_int), ("Qy", ctypes.c_int), ("N", ctypes.c_int), ("P", ctypes.c_int),
        ("alpha", ctypes.c_double), ("T", ctypes.c_double),
        ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
        ("dpar", ctypes.c_double * 8), ("fpar", ctypes.c_double * 8),
        ("solver", ctypes.c_int), ("basis", ctypes.c_int), ("csub", ctypes.c_int),
    ]

    @property
    def K(self) -> int:
        if self.basis == 1:
            return self.Mx - 1
        return self.Mx * (self.My if self.dim == 2 else 1)

    @property
    def Q(self) -> int:
        return self.Qx * (self.Qy if self.dim == 2 else 1)

    @property
    def m(self) -> int:
        return self.N // self.P


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction).
    omp=True builds the OpenMP variant (_psl1_oracle_omp.so): the same source
    with the parallel stage's loop over slices on all host threads."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                                   *(["-fopenmp"] if omp else []), "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, out)
    return out


def lib(omp: bool = False):
    """The oracle library; omp=True: its OpenMP build (parallel stage on all host threads)."""
    global _lib, _lib_omp
    if (_lib_omp if omp else _lib) is None:
        L = ctypes.CDLL(build(omp=omp))
        pp = ctypes.POINTER(Prob)
        sig = {
            "orc_b": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "orc_gamma2a": (ctypes.c_double, [ctypes.c_double]),
            "orc_gauss_legendre": (None, [ctypes.c_int, D_, D_]),
            "orc_nodes": (ctypes.c_int, [pp, D_, D_, D_]),
            "orc_basis": (ctypes.c_int, [pp, D_, D_, D_]),
            "orc_D": (ctypes.c_double, [pp] + [ctypes.c_double] * 4),
            "orc_f": (ctypes.c_double, [pp] + [ctypes.c_double] * 4),
            "orc_src1": (ctypes.c_double, [pp, ctypes.c_double, ctypes.c_double]),
            "orc_src2": (ctypes.c_double, [pp, ctypes.c_double, ctypes.c_double]),
            "orc_eval_nodes": (ctypes.c_int, [pp, D_, ctypes.c_double, D_, D_, D_]),
            "orc_stiffness": (ctypes.c_int, [pp, D_, D_]),
            "orc_load": (ctypes.c_int, [pp, D_, D_]),
            "orc_apply_stiffness": (ctypes.c_int, [pp, D_, D_, D_]),
            "orc_cheb": (ctypes.c_int, [pp, D_, D_]),
            "orc_project": (ctypes.c_int, [pp, D_, D_]),
            "orc_chol_solve": (ctypes.c_int, [ctypes.c_int, D_, D_, D_]),
            "orc_step": (ctypes.c_int, [pp, D_, ctypes.c_double, ctypes.c_double, D_, D_]),
            "orc_coarse_step": (ctypes.c_int, [pp, ctypes.c_int, D_, D_]),
            "orc_fine_slice": (ctypes.c_int, [pp, ctypes.c_int, D_, D_, ctypes.c_int]),
            "orc_serial_hyb": (ctypes.c_int, [pp, D_, D_, D_]),
            "orc_serial_uni": (ctypes.c_int, [pp, D_, D_]),
            "orc_coarse_sweep": (ctypes.c_int, [pp, D_, D_, D_, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, D_]),
            "orc_fine_stage": (ctypes.c_int, [pp, D_, ctypes.c_int, ctypes.c_int, D_]),
            "orc_gauss_jacobi": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, D_, D_]),
            "orc_soe_nodes": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, D_, D_]),
            "orc_serial_uni_soe": (ctypes.c_int, [pp, D_, ctypes.c_int, ctypes.c_double, D_]),
            "orc_threads": (ctypes.c_int, []),
            "orc_parareal": (ctypes.c_int, [pp, D_, ctypes.c_double, ctypes.c_int, D_, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int, D_, D_, D_, P_]),
            "orc_mlp_nparams": (ctypes.c_long, [ctypes.c_int] * 3),
            "orc_mlp_forward": (ctypes.c_int, [ctypes.c_int] * 3 + [D_, ctypes.c_int, D_, D_, D_]),
            "orc_mlp_backward": (ctypes.c_int, [ctypes.c_int] * 3 + [D_, ctypes.c_int, D_, D_, D_, D_]),
            "orc_adam_step": (None, [ctypes.c_long, D_, D_, D_, D_, ctypes.c_int] + [ctypes.c_double] * 4),
            "orc_mlp_features": (ctypes.c_int, [pp, ctypes.c_int, ctypes.c_int, ctypes.c_int, D_, D_]),
            "orc_l1_uniform": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int, D_]),
            "orc_l1_hybrid": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, D_, D_]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if omp:
            _lib_omp = L
        else:
            _lib = L
    return _lib_omp if omp else _lib


class OracleError(RuntimeError):
    pass


def _chk(st: int, what: str):
    if st != 0:
        raise OracleError(f"oracle {what} failed with status {st}")


def _d(a) -> tuple:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(D_)


def _out(*shape):
    a = np.zeros(shape, dtype=np.float64)
    return a, a.ctypes.data_as(D_)


def make_prob(*, dim=1, Mx, My=1, Qx=None, Qy=None, N, P, alpha, T=1.0, lo=(0.0, 0.0),
              hi=(1.0, 1.0), dpar=(1.0, 0.5, 0, 0, 0, 0, 0, 0), fpar=(0.1, 0, 0, 0, 0, 0, 0, 0),
              solver: str = "cholesky", basis: str = "sine", coarse_substeps: int = 1) -> Prob:
    """Problem record; Qx/Qy default to twice the modes (Gauss-Legendre).
    solver: "cholesky" (dense factor of the assembled matrix) or "cg"
    (conjugate gradients on the weak form, for mode counts whose assembly
    is out of reach); both solve the same SPD system of each step.
    basis: "sine" (Galerkin, Mx modes) or "cheb" (Chebyshev-Lobatto
    collocation, 1D: Mx intervals, the Mx - 1 interior nodal values).
    coarse_substeps: L1 substeps per slice of the coarse propagator (1: the
    paper's one-step G)."""
    p = Prob()
    p.dim, p.Mx = dim, Mx
    p.My = My if dim == 2 else 1
    p.Qx = Qx if Qx else 2 * Mx
    p.Qy = (Qy if Qy else 2 * p.My) if dim == 2 else 1
    p.N, p.P, p.alpha, p.T = N, P, float(alpha), float(T)
    p.lo[0], p.lo[1] = lo
    p.hi[0], p.hi[1] = hi
    dp = list(dpar) + [0.0] * (8 - len(dpar))
    fp = list(fpar) + [0.0] * (8 - len(fpar))
    for i in range(8):
        p.dpar[i], p.fpar[i] = dp[i], fp[i]
    p.solver = {"cholesky": 0, "cg": 1}[solver]
    p.basis = {"sine": 0, "cheb": 1}[basis]
    p.csub = int(coarse_substeps)
    if p.basis == 1 and dim != 1:
        raise ValueError("collocation is 1D")
    if N % P:
        raise ValueError("P must divide N")
    return p


def b(alpha, x) -> float:
    return lib().orc_b(float(alpha), float(x))


def gamma2a(alpha) -> float:
    return lib().orc_gamma2a(float(alpha))


def gauss_legendre(Q: int):
    x, px = _out(Q)
    w, pw = _out(Q)
    lib().orc_gauss_legendre(Q, px, pw)
    return x, w


def nodes(p: Prob):
    (x, px), (y, py), (w, pw) = _out(p.Q), _out(p.Q), _out(p.Q)
    _chk(lib().orc_nodes(ctypes.byref(p), px, py, pw), "nodes")
    return x, y, w


def basis(p: Prob):
    (phi, a), (gx, b_), (gy, c) = _out(p.Q, p.K), _out(p.Q, p.K), _out(p.Q, p.K)
    _chk(lib().orc_basis(ctypes.byref(p), a, b_, c), "basis")
    return phi, gx, gy


def D(p: Prob, x, y, t, u) -> float:
    return lib().orc_D(ctypes.byref(p), float(x), float(y), float(t), float(u))


def f(p: Prob, x, y, t, u) -> float:
    return lib().orc_f(ctypes.byref(p), float(x), float(y), float(t), float(u))


def src1(p: Prob, x, t) -> float:
    return lib().orc_src1(ctypes.byref(p), float(x), float(t))


def src2(p: Prob, x, t) -> float:
    return lib().orc_src2(ctypes.byref(p), float(x), float(t))


def eval_nodes(p: Prob, c, t):
    c, pc = _d(c)
    (u, pu), (Dq, pD), (fq, pf) = _out(p.Q), _out(p.Q), _out(p.Q)
    _chk(lib().orc_eval_nodes(ctypes.byref(p), pc, float(t), pu, pD, pf), "eval_nodes")
    return u, Dq, fq


def stiffness(p: Prob, Dq):
    Dq, pD = _d(Dq)
    A, pA = _out(p.K, p.K)
    _chk(lib().orc_stiffness(ctypes.byref(p), pD, pA), "stiffness")
    return A


def cheb(p: Prob):
    """Chebyshev-Lobatto nodes x_0..x_n (x_0 = hi) and the differentiation matrix."""
    n = p.Mx
    (x, px), (Dm, pD) = _out(n + 1), _out(n + 1, n + 1)
    _chk(lib().orc_cheb(ctypes.byref(p), px, pD), "cheb")
    return x, Dm


def apply_stiffness(p: Prob, Dq, v):
    """(A v)_i by the weak form, node by node, without forming A."""
    Dq, pD = _d(Dq)
    v, pv = _d(v)
    out, po = _out(p.K)
    _chk(lib().orc_apply_stiffness(ctypes.byref(p), pD, pv, po), "apply_stiffness")
    return out


def load(p: Prob, fq):
    fq, pf = _d(fq)
    F, pF = _out(p.K)
    _chk(lib().orc_load(ctypes.byref(p), pf, pF), "load")
    return F


def project(p: Prob, vq):
    vq, pv = _d(vq)
    c, pc = _out(p.K)
    _chk(lib().orc_project(ctypes.byref(p), pv, pc), "project")
    return c


def chol_solve(M, rhs):
    M, pM = _d(M)
    rhs, pr = _d(rhs)
    K = rhs.shape[0]
    x, px = _out(K)
    st = lib().orc_chol_solve(K, pM, pr, px)
    return x, st


def step(p: Prob, cprev, te, mu, hist):
    cprev, pc = _d(cprev)
    hist, ph = _d(hist)
    out, po = _out(p.K)
    _chk(lib().orc_step(ctypes.byref(p), pc, float(te), float(mu), ph, po), "step")
    return out


def coarse_step(p: Prob, n: int, U):
    U, pU = _d(U)
    out, po = _out(p.K)
    _chk(lib().orc_coarse_step(ctypes.byref(p), n, pU, po), "coarse_step")
    return out


def fine_slice(p: Prob, n: int, U, diff_form: bool = False):
    U, pU = _d(U)
    V, pV = _out(p.m + 1, p.K)
    _chk(lib().orc_fine_slice(ctypes.byref(p), n, pU, pV, int(diff_form)), "fine_slice")
    return V


def serial_hyb(p: Prob, u0, want_all: bool = False):
    u0, pu = _d(u0)
    U, pU = _out(p.P + 1, p.K)
    if want_all:
        V, pV = _out(p.N + 1, p.K)
    else:
        V, pV = None, None
    _chk(lib().orc_serial_hyb(ctypes.byref(p), pu, pU, pV), "serial_hyb")
    return (U, V) if want_all else U


def serial_uni(p: Prob, u0):
    u0, pu = _d(u0)
    W, pW = _out(p.N + 1, p.K)
    _chk(lib().orc_serial_uni(ctypes.byref(p), pu, pW), "serial_uni")
    return W


SOE_NLOC = 16      # steps of the exact local window of the fast history
SOE_EPS = 1e-12    # relative accuracy the exponentials are built for


def gauss_jacobi(n: int, ja: float, jb: float):
    """Gauss-Jacobi nodes and weights for (1-t)^ja (1+t)^jb on (-1, 1)."""
    (t, pt), (w, pw) = _out(n), _out(n)
    _chk(lib().orc_gauss_jacobi(int(n), float(ja), float(jb), pt, pw), "gauss_jacobi")
    return t, w


def soe_nodes(alpha: float, X: int, nloc: int = SOE_NLOC, eps: float = SOE_EPS):
    """Exponents s and weights w with b(x) ~ sum_i w_i exp(-s_i x) on [nloc, X]."""
    (s, ps), (w, pw) = _out(512), _out(512)
    L = lib().orc_soe_nodes(float(alpha), int(nloc), int(X), float(eps), 512, ps, pw)
    if L < 0:
        raise OracleError("soe_nodes failed")
    return s[:L], w[:L]


def serial_uni_soe(p: Prob, u0, nloc: int = SOE_NLOC, eps: float = SOE_EPS):
    """The uniform L1 scheme with the sum-of-exponentials weights: (N+1) x K."""
    u0, pu = _d(u0)
    W, pW = _out(p.N + 1, p.K)
    _chk(lib().orc_serial_uni_soe(ctypes.byref(p), pu, int(nloc), float(eps), pW), "serial_uni_soe")
    return W


def _mlp_args(mlp):
    """mlp: dict(params, oscale, nU, nH, width[, nout]) -- nout defaults to len(oscale)."""
    if mlp is None:
        return None, None, 0, 0, 0, 0, None, None
    params, pp = _d(mlp["params"])
    osc, po = _d(mlp["oscale"])
    nout = int(mlp.get("nout", osc.shape[0]))
    return params, pp, int(mlp["nU"]), int(mlp["nH"]), int(mlp["width"]), nout, osc, po


def coarse_sweep(p: Prob, u0, mlp=None):
    u0, pu = _d(u0)
    U, pU = _out(p.P + 1, p.K)
    keep = _mlp_args(mlp)
    _chk(lib().orc_coarse_sweep(ctypes.byref(p), pu, pU, keep[1], keep[2], keep[3], keep[4], keep[5], keep[7]),
         "coarse_sweep")
    return U


def parareal(p: Prob, u0, tol: float, max_iter: int | None = None, mlp=None, omp: bool = False):
    """Returns (U[k, n, :] for k = 0..iters, errlog[:iters], iters).
    omp=True runs the parallel stage of each iteration on all host threads."""
    if max_iter is None:
        max_iter = p.P
    u0, pu = _d(u0)
    Uall, pU = _out(max_iter + 1, p.P + 1, p.K)
    err, pe = _out(max(max_iter, 1))
    it = ctypes.c_int(0)
    keep = _mlp_args(mlp)
    _chk(lib(omp).orc_parareal(ctypes.byref(p), pu, float(tol), int(max_iter), keep[1], keep[2], keep[3],
                               keep[4], keep[5], keep[7], pU, pe, ctypes.byref(it)), "parareal")
    k = it.value
    return Uall[: k + 1], err[:k], k


def fine_stage(p: Prob, U, n0: int = 0, n1: int | None = None, omp: bool = False):
    """F_n(U_{0:n}) for n = n0..n1-1 (rows of a P x K array; the other rows zero).
    U holds at least U_0..U_{n1-1}."""
    n1 = p.P if n1 is None else int(n1)
    U, pU = _d(U)
    F, pF = _out(p.P, p.K)
    _chk(lib(omp).orc_fine_stage(ctypes.byref(p), pU, int(n0), n1, pF), "fine_stage")
    return F


def threads(omp: bool = False) -> int:
    """Host threads of the (OpenMP) parallel stage."""
    return int(lib(omp).orc_threads())


def mlp_nparams(nin, width, nout) -> int:
    return int(lib().orc_mlp_nparams(nin, width, nout))


def mlp_forward(params, nin, width, nout, z, want_pre=False):
    params, pp = _d(params)
    z, pz = _d(np.atleast_2d(z))
    B = z.shape[0]
    y, py = _out(B, nout)
    pre, ppre = (_out(B, 3 * width) if want_pre else (None, None))
    _chk(lib().orc_mlp_forward(nin, width, nout, pp, B, pz, py, ppre), "mlp_forward")
    return (y, pre) if want_pre else y


def mlp_backward(params, nin, width, nout, z, target):
    params, pp = _d(params)
    z, pz = _d(np.atleast_2d(z))
    target, pt = _d(np.atleast_2d(target))
    B = z.shape[0]
    g, pg = _out(params.shape[0])
    loss = ctypes.c_double(0.0)
    _chk(lib().orc_mlp_backward(nin, width, nout, pp, B, pz, pt, pg, ctypes.byref(loss)), "mlp_backward")
    return g, loss.value


def adam_step(param, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam_step(param.shape[0], param.ctypes.data_as(D_), grad.ctypes.data_as(D_),
                        m.ctypes.data_as(D_), v.ctypes.data_as(D_), int(t), lr, b1, b2, eps)


def mlp_features(p: Prob, nU: int, nH: int, n: int, U):
    U, pU = _d(U)
    z, pz = _out(nU + nH + 2)
    _chk(lib().orc_mlp_features(ctypes.byref(p), nU, nH, n, pU, pz), "mlp_features")
    return z


def l1_uniform(alpha, dt, y) -> float:
    """Uniform L1 Caputo operator at t_{n+1} on samples y_0..y_{n+1}."""
    y, py = _d(y)
    return lib().orc_l1_uniform(float(alpha), float(dt), y.shape[0] - 2, py)


def l1_hybrid(alpha, dT, M, n, r, Y, yf) -> float:
    """Hybrid L1 operator at t_{n,r}: coarse samples Y_0..Y_n, fine y_{n,0..r}."""
    Y, pY = _d(Y)
    yf, pf = _d(yf)
    return lib().orc_l1_hybrid(float(alpha), float(dT), int(M), int(n), int(r), pY, pf)
