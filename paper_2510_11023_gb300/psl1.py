"""Thin ctypes binding of the C ABI in ``include/psl1.h``.

Argument marshalling only: every step of the solver runs in the CUDA library
``libpsl1.so``.  There is no fallback; if the library cannot be built or
loaded, or no CUDA device is usable, the calls raise ``PSL1Error``.

Module-level functions carry the C names (``psl1_create``, ...); ``Problem``
is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from .workloads import InstanceSpec, Workload

PREC = {"fp64": 0, "mixed": 1, "fp32": 2}
SERIAL = {"hybrid": 0, "uniform": 1, "coarse": 2, "uniform-soe": 3}
BASIS = {"sine": 0, "cheb": 1}
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_NOT_SPD", -3: "ERR_NONFINITE", -4: "ERR_CUDA", -5: "ERR_TIMEOUT",
          -6: "ERR_NOT_CONVERGED", -7: "ERR_STATE", -8: "ERR_NOMEM"}

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)


class PSL1Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Instance(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("modes", ctypes.c_int * 2), ("qnodes", ctypes.c_int * 2),
                ("nsteps", ctypes.c_int), ("alpha", ctypes.c_double), ("T", ctypes.c_double),
                ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
                ("dpar", ctypes.c_double * 8), ("fpar", ctypes.c_double * 8), ("basis", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations_max", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("ms_total", ctypes.c_double), ("ms_fine", ctypes.c_double), ("ms_coarse", ctypes.c_double),
                ("ms_history", ctypes.c_double), ("fine_steps", ctypes.c_double),
                ("fine_step_modes", ctypes.c_double), ("flop_fine", ctypes.c_double),
                ("flop_coarse", ctypes.c_double), ("flop_serial", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# name -> (restype, argtypes); the exported symbols of include/psl1.h
SIGNATURES = {
    "psl1_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(Instance),
                                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "psl1_set_D": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "psl1_set_f": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "psl1_set_u0": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "psl1_set_u0_dev": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "psl1_solve_serial": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "psl1_solve_parareal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, _I]),
    "psl1_resume_parareal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_double, ctypes.c_int, _I]),
    "psl1_get_coeffs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D]),
    "psl1_get_coeffs_dev": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "psl1_get_iterations": (ctypes.c_int, [ctypes.c_void_p, _I]),
    "psl1_get_errlog": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_int, _I]),
    "psl1_keep_iterates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "psl1_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "psl1_set_inexact_fine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "psl1_set_inexact_refinement": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "psl1_set_coarse_substeps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "psl1_set_sweep_split": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "psl1_get_sweep_split": (ctypes.c_int, [ctypes.c_void_p, _I]),
    "psl1_get_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D]),
    "psl1_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "psl1_get_soe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, _D, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]),
    "psl1_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, _I]),
    "psl1_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _F, _I]),
    "psl1_assemble": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _F, _F]),
    "psl1_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D, _D]),
    "psl1_fine_slice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, _D]),
    "psl1_coarse_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, _D]),
    "psl1_fine_slice_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "psl1_probe_peaks": (ctypes.c_int, [_D, _D]),
    "psl1_probe_dmma": (ctypes.c_int, [_D]),
    "psl1_mlp_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p]),
    "psl1_mlp_nparams": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "psl1_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, _F, _F]),
    "psl1_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, _F, _F]),
    "psl1_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _F, _F]),
    "psl1_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _F, _F, _F, _F]),
    "psl1_mlp_adam_step": (ctypes.c_int, [ctypes.c_void_p, _F, ctypes.c_float]),
    "psl1_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_ulonglong, _F]),
    "psl1_set_coarse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "psl1_mlp_dataset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "psl1_mlp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "psl1_mlp_destroy": (None, [ctypes.c_void_p]),
    "psl1_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "psl1_destroy": (None, [ctypes.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpsl1.so (building it first if needed)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise PSL1Error(-4, f"CUDA library not built: {_build.LIB}")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _err(h) -> str:
    m = load().psl1_last_error(h)
    return m.decode() if m else ""


def _chk(st: int, h):
    if st != 0:
        raise PSL1Error(st, _err(h))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def to_instance(s: InstanceSpec) -> Instance:
    c = Instance()
    c.dim = s.dim
    c.modes[0], c.modes[1] = s.modes
    c.qnodes[0], c.qnodes[1] = s.qnodes
    c.nsteps, c.alpha, c.T = s.nsteps, s.alpha, s.T
    c.lo[0], c.lo[1] = s.lo
    c.hi[0], c.hi[1] = s.hi
    dp = list(s.dpar) + [0.0] * (8 - len(s.dpar))
    fp = list(s.fpar) + [0.0] * (8 - len(s.fpar))
    for i in range(8):
        c.dpar[i], c.fpar[i] = dp[i], fp[i]
    c.basis = BASIS[s.basis]
    return c


# ------------------------------------------------------------------ C names
def psl1_create(specs, P: int, precision: str = "fp64", stream: int | None = None) -> ctypes.c_void_p:
    arr = (Instance * len(specs))(*[to_instance(s) for s in specs])
    h = ctypes.c_void_p()
    _chk(load().psl1_create(ctypes.byref(h), len(specs), arr, int(P), PREC[precision],
                            ctypes.c_void_p(stream) if stream else None), None)
    return h


def psl1_probe_peaks() -> tuple:
    """Measured (FP64, FP32) FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _chk(load().psl1_probe_peaks(ctypes.byref(a), ctypes.byref(b)), None)
    return a.value, b.value


def psl1_probe_dmma() -> float:
    """Measured FP64 tensor-core (DMMA) throughput of the current device, TFLOP/s."""
    a = ctypes.c_double()
    _chk(load().psl1_probe_dmma(ctypes.byref(a)), None)
    return a.value


def psl1_destroy(h) -> None:
    load().psl1_destroy(h)


class Problem:
    """A batch of instances on the device (wraps one psl1 handle)."""

    def __init__(self, workload_or_specs, P: int | None = None, precision: str = "fp64",
                 stream: int | None = None):
        if isinstance(workload_or_specs, Workload):
            wl = workload_or_specs
            self.specs, self.P = list(wl.specs), wl.P
        else:
            self.specs, self.P = list(workload_or_specs), int(P)
        self.K = [s.K for s in self.specs]
        self.offK = np.concatenate([[0], np.cumsum(self.K)]).astype(np.int64)
        self.offU = np.concatenate([[0], np.cumsum([(self.P + 1) * k for k in self.K])]).astype(np.int64)
        self.h = psl1_create(self.specs, self.P, precision, stream)
        self.L = load()
        if isinstance(workload_or_specs, Workload):
            self.set_u0(workload_or_specs.u0_concat())

    def close(self):
        if self.h:
            self.L.psl1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def B(self) -> int:
        return len(self.specs)

    def set_u0(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        assert u0.size == self.offK[-1]
        _chk(self.L.psl1_set_u0(self.h, _dp(u0)), self.h)

    def set_u0_dev(self, ptr: int):
        _chk(self.L.psl1_set_u0_dev(self.h, ctypes.c_void_p(ptr)), self.h)

    def set_D(self, dpar):
        d = np.ascontiguousarray(dpar, dtype=np.float64).reshape(-1)
        _chk(self.L.psl1_set_D(self.h, _dp(d)), self.h)

    def set_f(self, fpar):
        d = np.ascontiguousarray(fpar, dtype=np.float64).reshape(-1)
        _chk(self.L.psl1_set_f(self.h, _dp(d)), self.h)

    def solve_serial(self, kind: str = "hybrid"):
        _chk(self.L.psl1_solve_serial(self.h, SERIAL[kind]), self.h)

    def solve_parareal(self, tol: float = 1e-10, max_iter: int = 0, allow_not_converged: bool = False) -> int:
        it = ctypes.c_int(0)
        st = self.L.psl1_solve_parareal(self.h, float(tol), int(max_iter), ctypes.byref(it))
        if st == -6 and allow_not_converged:
            return it.value
        _chk(st, self.h)
        return it.value

    def resume_parareal(self, k0: int, U, tol: float = 1e-10, max_iter: int = 0,
                        allow_not_converged: bool = False) -> int:
        """Continue parareal from the checkpoint U^{k0} (a list of (P+1) x K arrays or the flat vector)."""
        flat = np.ascontiguousarray(np.concatenate([np.asarray(u).reshape(-1) for u in U])
                                    if isinstance(U, (list, tuple)) else U, dtype=np.float64)
        assert flat.size == self.offU[-1]
        it = ctypes.c_int(0)
        st = self.L.psl1_resume_parareal(self.h, int(k0), _dp(flat), float(tol), int(max_iter), ctypes.byref(it))
        if st == -6 and allow_not_converged:
            return it.value
        _chk(st, self.h)
        return it.value

    def _split(self, flat) -> list:
        return [flat[self.offU[b]:self.offU[b + 1]].reshape(self.P + 1, self.K[b]) for b in range(self.B)]

    def get_coeffs(self, which: str = "parareal", flat: bool = False):
        out = np.zeros(int(self.offU[-1]))
        _chk(self.L.psl1_get_coeffs(self.h, 0 if which == "parareal" else 1, _dp(out)), self.h)
        return out if flat else self._split(out)

    def get_coeffs_dev(self, which: str, ptr: int):
        _chk(self.L.psl1_get_coeffs_dev(self.h, 0 if which == "parareal" else 1, ctypes.c_void_p(ptr)), self.h)

    def get_iterations(self) -> np.ndarray:
        it = np.zeros(self.B, dtype=np.int32)
        _chk(self.L.psl1_get_iterations(self.h, it.ctypes.data_as(_I)), self.h)
        return it

    def get_errlog(self, b: int) -> np.ndarray:
        n = ctypes.c_int(0)
        _chk(self.L.psl1_get_errlog(self.h, b, None, 0, ctypes.byref(n)), self.h)
        out = np.zeros(max(n.value, 1))
        _chk(self.L.psl1_get_errlog(self.h, b, _dp(out), n.value, ctypes.byref(n)), self.h)
        return out[: n.value]

    def keep_iterates(self, on: bool = True):
        _chk(self.L.psl1_keep_iterates(self.h, int(on)), self.h)

    def set_graph(self, on: bool = True):
        """Run parareal as one CUDA graph with a device-driven iteration loop."""
        _chk(self.L.psl1_set_graph(self.h, int(on)), self.h)

    def set_inexact_fine(self, above: float):
        """Inexact early iterations: the FP32 step on slices n > k while the last
        increment exceeds `above` (0: off).  MIXED handles (1D and 2D)."""
        _chk(self.L.psl1_set_inexact_fine(self.h, float(above)), self.h)

    def set_inexact_refinement(self, factor: float):
        """Refined F steps of slices n > k stop refining at factor * e_{k-1} (0: off). MIXED 1D and 2D."""
        _chk(self.L.psl1_set_inexact_refinement(self.h, float(factor)), self.h)

    def get_iterate(self, k: int) -> list:
        out = np.zeros(int(self.offU[-1]))
        _chk(self.L.psl1_get_iterate(self.h, k, _dp(out)), self.h)
        return self._split(out)

    def stats(self) -> dict:
        s = Stats()
        _chk(self.L.psl1_get_stats(self.h, ctypes.byref(s)), self.h)
        return s.as_dict()

    def step(self, b: int, c, te: float, mu: float, hist) -> np.ndarray:
        c = np.ascontiguousarray(c, dtype=np.float64)
        hist = np.ascontiguousarray(hist, dtype=np.float64)
        out = np.zeros(self.K[b])
        _chk(self.L.psl1_step(self.h, b, _dp(c), float(te), float(mu), _dp(hist), _dp(out)), self.h)
        return out

    def fine_slice(self, b: int, n: int, U) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        m = self.specs[b].nsteps // self.P
        V = np.zeros((m + 1, self.K[b]))
        _chk(self.L.psl1_fine_slice(self.h, b, n, _dp(U), _dp(V)), self.h)
        return V

    def assemble(self, b: int, D, method: str = "tensor"):
        """Dense stiffness matrices (units x K x K, FP32) from nodal D (units x Q,
        ascending nodes); returns (A, device ms of the assembly kernel)."""
        D = np.ascontiguousarray(np.atleast_2d(D), dtype=np.float64)
        units, K = D.shape[0], self.K[b]
        A = np.zeros((units, K, K), dtype=np.float32)
        ms = ctypes.c_float(0.0)
        _chk(self.L.psl1_assemble(self.h, b, {"tensor": 0, "moments": 1}[method], units, _dp(D),
                                  A.ctypes.data_as(_F), ctypes.byref(ms)), self.h)
        return A, ms.value

    def set_sweep_split(self, ctas: int = 0):
        """2D: share each coarse-sweep step among a cluster of `ctas` CTAs (1, 2, 4, 8; 0: automatic)."""
        _chk(self.L.psl1_set_sweep_split(self.h, int(ctas)), self.h)

    def sweep_split(self) -> int:
        n = ctypes.c_int(0)
        _chk(self.L.psl1_get_sweep_split(self.h, ctypes.byref(n)), self.h)
        return n.value

    def set_coarse_substeps(self, c: int):
        """L1 substeps per slice of the coarse propagator (1: the paper's one-step G)."""
        _chk(self.L.psl1_set_coarse_substeps(self.h, int(c)), self.h)

    def autotune(self, cache_path: str | None = None) -> bool:
        """Tune the F stage (see psl1_autotune); True if every choice came from the cache."""
        fc = ctypes.c_int(0)
        _chk(self.L.psl1_autotune(self.h, cache_path.encode() if cache_path else None, ctypes.byref(fc)), self.h)
        return bool(fc.value)

    def tuning(self, b: int = 0) -> dict:
        r, g = ctypes.c_float(0), ctypes.c_int(0)
        _chk(self.L.psl1_get_tuning(self.h, b, ctypes.byref(r), ctypes.byref(g)), self.h)
        return {"inner_rtol": r.value, "fstage_ctas": g.value}

    def get_soe(self, b: int):
        """Exponents s and weights w of instance b's fast history."""
        n = ctypes.c_int(0)
        s, w = np.zeros(512), np.zeros(512)
        _chk(self.L.psl1_get_soe(self.h, b, _dp(s), _dp(w), 512, ctypes.byref(n)), self.h)
        return s[: n.value], w[: n.value]

    def fine_slice_noalloc(self, b: int, n: int, d_U: int, d_V: int) -> None:
        """F_n on caller-owned device arrays (pointers), without any allocation."""
        _chk(self.L.psl1_fine_slice_noalloc(self.h, b, n, ctypes.c_void_p(d_U), ctypes.c_void_p(d_V)), self.h)

    def set_coarse(self, mlp: "MLP | None"):
        """Attach a learned coarse correction (None: the plain L1 coarse propagator)."""
        _chk(self.L.psl1_set_coarse(self.h, mlp.h if mlp is not None else None), self.h)
        self._mlp = mlp   # keep it alive while attached

    def coarse_step(self, b: int, n: int, U) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(self.K[b])
        _chk(self.L.psl1_coarse_step(self.h, b, n, _dp(U), _dp(out)), self.h)
        return out


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_F)


class MLP:
    """The learned coarse correction (wraps one psl1_mlp handle)."""

    def __init__(self, nU: int = 128, nH: int = 32, width: int = 512, nout: int = 128, seed: int = 0,
                 stream: int | None = None):
        self.L = load()
        h = ctypes.c_void_p()
        st = self.L.psl1_mlp_create(ctypes.byref(h), nU, nH, width, nout, ctypes.c_ulonglong(seed),
                                    ctypes.c_void_p(stream) if stream else None)
        if st != 0:
            raise PSL1Error(st, (self.L.psl1_mlp_last_error(None) or b"").decode())
        self.h = h
        self.nU, self.nH, self.width, self.nout = nU, nH, width, nout
        self.nin = nU + nH + 2
        n = ctypes.c_longlong(0)
        self._chk(self.L.psl1_mlp_nparams(self.h, ctypes.byref(n)))
        self.nparams = n.value

    def _chk(self, st):
        if st != 0:
            raise PSL1Error(st, (self.L.psl1_mlp_last_error(self.h) or b"").decode())

    def close(self):
        if self.h:
            self.L.psl1_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        s = np.zeros(self.nout, dtype=np.float32)
        self._chk(self.L.psl1_mlp_get_params(self.h, _fp(p), _fp(s)))
        return p, s

    def set_params(self, params=None, oscale=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        s = None if oscale is None else np.ascontiguousarray(oscale, dtype=np.float32)
        self._chk(self.L.psl1_mlp_set_params(self.h, _fp(p) if p is not None else None,
                                             _fp(s) if s is not None else None))

    def forward(self, z) -> np.ndarray:
        z = np.ascontiguousarray(np.atleast_2d(z), dtype=np.float32)
        y = np.zeros((z.shape[0], self.nout), dtype=np.float32)
        self._chk(self.L.psl1_mlp_forward(self.h, z.shape[0], _fp(z), _fp(y)))
        return y

    def loss_grad(self, z, t):
        z = np.ascontiguousarray(np.atleast_2d(z), dtype=np.float32)
        t = np.ascontiguousarray(np.atleast_2d(t), dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float(0)
        self._chk(self.L.psl1_mlp_loss_grad(self.h, z.shape[0], _fp(z), _fp(t), _fp(g), ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, grad, lr: float):
        g = np.ascontiguousarray(grad, dtype=np.float32)
        self._chk(self.L.psl1_mlp_adam_step(self.h, _fp(g), float(lr)))

    def dataset(self, data: Problem, trajectories: bool = False, iterates: int = 0):
        """Build the training set from `data`: S_hyb trajectory samples and/or the
        samples of `iterates` parareal iterations (see psl1_mlp_dataset)."""
        src = (1 if trajectories else 0) | (2 if iterates > 0 else 0)
        self._chk(self.L.psl1_mlp_dataset(self.h, data.h, src, int(iterates)))

    def train(self, data: Problem, epochs: int = 100, batch: int = 512, lr: float = 1e-3, seed: int = 0):
        log = np.zeros(max(epochs, 1), dtype=np.float32)
        self._chk(self.L.psl1_mlp_train(self.h, data.h, int(epochs), int(batch), float(lr),
                                        ctypes.c_ulonglong(seed), _fp(log)))
        return log[:epochs]
