"""Thin ctypes binding of libmmf.so (include/mmf.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; there is no CPU path.  If the
library cannot be loaded or no GPU is usable, the calls raise ``MmfError``.

The ``mmf_*`` functions of the C ABI are exposed under the same names on ``lib()``;
``Context``, ``System`` and ``Batch`` wrap the handles for NumPy callers.
"""

from __future__ import annotations

import atexit
import ctypes
import os
import re
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "libmmf.so")
HEADER = os.path.join(ROOT, "include", "mmf.h")

MMF_OK = 0
MMF_ERR_ARG = -1
MMF_ERR_STATE = -2
MMF_ERR_BUDGET = -3
MMF_ERR_CUDA = -4
MMF_ERR_UNSUPPORTED = -5
MMF_ERR_NOMEM = -6
MMF_ST_NOCONV = 1
MMF_ST_NONFINITE = 2
MMF_ST_CLUSTER = 3
MMF_FP64 = 0
MMF_MIXED = 1
MMF_OPT_JACOBI_N_FP64 = 1
MMF_OPT_JACOBI_N_MIXED = 2
MMF_OPT_LARGE_N = 3
MMF_OPT_REFINE_FULL_N = 4
MMF_OPT_GRAM_KERNEL = 5
MMF_OPT_BT_TC_N = 6
MMF_OPT_JACOBI_SWEEPS = 7
MMF_OPT_BAND_MAX = 8
MMF_OPT_HETRD_TC = 9
MMF_PATH_JACOBI = 0
MMF_PATH_DENSE = 1
MMF_PATH_WHOLE_GPU = 2
MMF_PATH_BAND = 3

_lib = None
_exiting = False


def _at_exit():
    # Handles still alive at interpreter exit are left to the process teardown: releasing them
    # from finalizers that may run after the CUDA runtime has shut down is unsafe.
    global _exiting
    _exiting = True


atexit.register(_at_exit)


class MmfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_PP = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "mmf_ctx_create": (_I, [_I, _SZ, _P, _PP]),
    "mmf_ctx_destroy": (_I, [_P]),
    "mmf_ctx_bytes_in_use": (_SZ, [_P]),
    "mmf_ctx_budget": (_SZ, [_P]),
    "mmf_ctx_set_option": (_I, [_P, _I, _I64]),
    "mmf_ctx_add_rule": (_I, [_P, _I, _I64, _I64, _I, _I, _I, _I, _I]),
    "mmf_ctx_clear_rules": (_I, [_P]),
    "mmf_ctx_load_tuning": (_I, [_P, ctypes.c_char_p]),
    "mmf_sys_create": (_I, [_P, _I, _P, _PP]),
    "mmf_add_mode": (_I, [_P, _D, _I, ctypes.POINTER(_I)]),
    "mmf_add_coupling": (_I, [_P, _I, _I, _P]),
    "mmf_sys_destroy": (_I, [_P]),
    "mmf_dim": (_I64, [_P]),
    "mmf_sys_bandwidth": (_I, [_P]),
    "mmf_build": (_I, [_P, _I, ctypes.POINTER(_I64)]),
    "mmf_hamiltonian": (_I, [_P, _P]),
    "mmf_diagonalise": (_I, [_P]),
    "mmf_quasienergies": (_I, [_P, _P]),
    "mmf_eigenvectors": (_I, [_P, _P]),
    "mmf_time_evolution": (_I, [_P, _D, _I, _P, _P]),
    "mmf_transition_avg": (_I, [_P, _P]),
    "mmf_micromotion": (_I, [_P, _I, _P, _P, _P]),
    "mmf_time_evolution_operator": (_I, [_P, _I, _D, _I, _P, _P]),
    "mmf_batch_create": (_I, [_P, _I, _P, _I, _I, _PP]),
    "mmf_batch_set_times": (_I, [_P, _D, _P]),
    "mmf_batch_upload": (_I, [_P]),
    "mmf_batch_run": (_I, [_P]),
    "mmf_batch_sync": (_I, [_P, _P]),
    "mmf_batch_get": (_I, [_P, _I, _P, _P, _P]),
    "mmf_batch_eigenvectors": (_I, [_P, _I, _P]),
    "mmf_batch_results": (_I, [_P, _P, _P, _P]),
    "mmf_batch_offset": (_I64, [_P, _I, _I]),
    "mmf_batch_size": (_I64, [_P, _I]),
    "mmf_batch_path": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "mmf_batch_bytes": (_SZ, [_P]),
    "mmf_batch_timing": (_I, [_P, _I]),
    "mmf_batch_graph": (_I, [_P, _I]),
    "mmf_batch_stage_ms": (_I, [_P, _P, _P]),
    "mmf_batch_destroy": (_I, [_P]),
    "mmf_quasienergies_dev": (_I, [_P, _P, _P]),
    "mmf_eigenvectors_dev": (_I, [_P, _P, _P]),
    "mmf_time_evolution_dev": (_I, [_P, _D, _I, _P, _P, _P]),
    "mmf_transition_avg_dev": (_I, [_P, _P, _P]),
    "mmf_batch_results_dev": (_I, [_P, _P, _P, _P, _P]),
    "mmf_sys_restrict": (_I, [_P, _I, _P, _PP]),
    "mmf_batch_dressed": (_I, [_P, _P, _P, _P]),
    "mmf_batch_dressed_size": (_I64, [_P, _I]),
    "mmf_batch_dressed_offset": (_I64, [_P, _I, _I]),
    "mmf_dressed_time_evolution": (_I, [_P, _I, _P, _I, _D, _I, _P, _P, _P]),
    "mmf_tridiag_eig_noalloc": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "mmf_serve_create": (_I, [_P, _I, _I, _I, _PP]),
    "mmf_serve_submit": (_I, [_P, _P, _I, _P, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "mmf_serve_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_I)]),
    "mmf_serve_wait": (_I, [_P, ctypes.c_uint64, _I, _P, _P, _P, ctypes.POINTER(_I)]),
    "mmf_serve_stats": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                             ctypes.POINTER(_I64)]),
    "mmf_serve_reset_stats": (_I, [_P]),
    "mmf_serve_plan_stats": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "mmf_serve_destroy": (_I, [_P]),
    "mmf_selftest_tensor_cores": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "mmf_selftest_gram": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "mmf_selftest_split_tf32": (_I, [_I, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "mmf_selftest_hetrd": (_I, [_I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "mmf_strerror": (ctypes.c_char_p, [_I]),
    "mmf_spin_components": (_I, [_I, _P, _P, _I, _P]),
    "mmf_last_error": (ctypes.c_char_p, []),
    "mmf_last_launch_count": (_I, []),
}


def header_symbols() -> List[str]:
    """Names of the functions declared in include/mmf.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^MMF_API\s+[\w\s\*]+?\b(mmf_\w+)\s*\(", txt, flags=re.M)))


def lib():
    """Load libmmf.so (building it first if the CUDA toolkit is present and it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b

            _b.build()
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, allow_numeric: bool = False) -> int:
    if rc == MMF_OK or (allow_numeric and rc > 0):
        return rc
    L = lib()
    msg = L.mmf_last_error().decode() or L.mmf_strerror(rc).decode()
    raise MmfError(rc, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cplx(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def spin_components(S2: int, A, phi=(0.0, 0.0, 0.0), static: bool = False) -> np.ndarray:
    """Coupling matrix of a spin S = S2/2 from Eq. 7's amplitudes and phases (x, y, z):
    sum_i (A_i/2) e^{i phi_i} S_i for a drive sum_i A_i cos(h w t + phi_i) S_i, or the static
    sum_i A_i S_i (static=True).  D x D complex, basis m = S, ..., -S."""
    D = int(S2) + 1
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(3))
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(3))
    V = np.zeros((D, D), dtype=np.complex128)
    _check(lib().mmf_spin_components(int(S2), _ptr(A), _ptr(phi), int(bool(static)), _ptr(V)))
    return V


class Context:
    """A CUDA device + stream binding with an HBM budget (mmf_ctx_*).

    Systems, batches and servers made on a context count as its dependents: the C context is
    destroyed only once the context is closed and every dependent has been closed, whatever the
    order in which Python finalises them."""

    def __init__(self, device: int = 0, budget: int = 0, stream: Optional[int] = None):
        h = ctypes.c_void_p()
        _check(lib().mmf_ctx_create(device, budget, stream, ctypes.byref(h)))
        self.h = h
        self._live = 0
        self._closing = False

    def _acquire(self):
        self._live += 1

    def _release(self):
        self._live -= 1
        if self._closing and self._live <= 0:
            self._destroy()

    def _destroy(self):
        if self.h and not _exiting:
            lib().mmf_ctx_destroy(self.h)
        self.h = None

    def bytes_in_use(self) -> int:
        return int(lib().mmf_ctx_bytes_in_use(self.h))

    def set_option(self, option: int, value: int):
        _check(lib().mmf_ctx_set_option(self.h, option, int(value)))

    def budget(self) -> int:
        return int(lib().mmf_ctx_budget(self.h))

    def add_rule(self, precision: int, n_lo: int, n_hi: int, band_lo: int, band_hi: int,
                 jacobi: int = -1, band: int = -1, bt_tc: int = -1):
        """Per-system solver choices for systems in the given size and band range (-1: no preference)."""
        _check(lib().mmf_ctx_add_rule(self.h, precision, int(n_lo), int(n_hi), int(band_lo), int(band_hi),
                                      int(jacobi), int(band), int(bt_tc)))

    def clear_rules(self):
        _check(lib().mmf_ctx_clear_rules(self.h))

    def load_tuning(self, path: str) -> int:
        """Add the rules of a tuning table file; returns their number."""
        rc = lib().mmf_ctx_load_tuning(self.h, os.fsencode(path))
        if rc < 0:
            _check(rc)
        return rc

    def close(self):
        self._closing = True
        if self._live <= 0:
            self._destroy()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """One driven system (mmf_sys_*) defined from a problem description with attributes
    D, H0, omegas, Ns, couplings (couplings[l][h-1] = V^{l+1,h})."""

    def __init__(self, ctx: Context, problem):
        self.ctx = ctx
        self.h = None
        self.D = int(problem.D)
        h = ctypes.c_void_p()
        H0 = _cplx(problem.H0)
        _check(lib().mmf_sys_create(ctx.h, self.D, _ptr(H0), ctypes.byref(h)))
        self.h = h
        ctx._acquire()
        for l, (w, N) in enumerate(zip(problem.omegas, problem.Ns)):
            mid = ctypes.c_int(-1)
            _check(lib().mmf_add_mode(self.h, float(w), int(N), ctypes.byref(mid)))
            for hh, V in enumerate(problem.couplings[l], start=1):
                _check(lib().mmf_add_coupling(self.h, mid.value, hh, _ptr(_cplx(V))))
        self.n = int(lib().mmf_dim(self.h))

    def bandwidth(self) -> int:
        """Half-bandwidth of this system's H_F."""
        return int(lib().mmf_sys_bandwidth(self.h))

    def build(self, precision: int = MMF_FP64) -> int:
        n = ctypes.c_int64(0)
        _check(lib().mmf_build(self.h, precision, ctypes.byref(n)))
        return int(n.value)

    def hamiltonian(self) -> np.ndarray:
        out = np.zeros((self.n, self.n), dtype=np.complex128)  # column-major data
        _check(lib().mmf_hamiltonian(self.h, _ptr(out)))
        return out.T.copy()

    def diagonalise(self) -> int:
        return _check(lib().mmf_diagonalise(self.h), allow_numeric=True)

    def quasienergies(self) -> np.ndarray:
        E = np.zeros(self.n)
        _check(lib().mmf_quasienergies(self.h, _ptr(E)))
        return E

    def eigenvectors(self) -> np.ndarray:
        Z = np.zeros((self.n, self.n), dtype=np.complex128)
        _check(lib().mmf_eigenvectors(self.h, _ptr(Z)))
        return Z.T.copy()

    def time_evolution(self, t, t0: float = 0.0) -> np.ndarray:
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
        U = np.zeros((t.size, self.D, self.D), dtype=np.complex128)
        _check(lib().mmf_time_evolution(self.h, float(t0), int(t.size), _ptr(t), _ptr(U)))
        return U

    def transition_avg(self) -> np.ndarray:
        P = np.zeros((self.D, self.D))
        _check(lib().mmf_transition_avg(self.h, _ptr(P)))
        return P

    def micromotion(self, t):
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
        UF = np.zeros((t.size, self.D, self.D), dtype=np.complex128)
        reps = np.zeros(self.D, dtype=np.int64)
        _check(lib().mmf_micromotion(self.h, int(t.size), _ptr(t), _ptr(UF), _ptr(reps)))
        return UF, reps

    # device-pointer variants: dst and t are device addresses (e.g. tensor.data_ptr()), stream a
    # cudaStream_t handle (e.g. torch.cuda.current_stream().cuda_stream)
    def quasienergies_dev(self, dst: int, stream: int):
        _check(lib().mmf_quasienergies_dev(self.h, dst, stream))

    def eigenvectors_dev(self, dst: int, stream: int):
        _check(lib().mmf_eigenvectors_dev(self.h, dst, stream))

    def time_evolution_dev(self, t0: float, nt: int, t: int, dst: int, stream: int):
        _check(lib().mmf_time_evolution_dev(self.h, float(t0), int(nt), t, dst, stream))

    def transition_avg_dev(self, dst: int, stream: int):
        _check(lib().mmf_transition_avg_dev(self.h, dst, stream))

    def restrict(self, modes) -> "System":
        """The same system driven by the listed modes only (Sec. 3.3's dressing modes)."""
        m = np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
        h = ctypes.c_void_p()
        _check(lib().mmf_sys_restrict(self.h, int(m.size), _ptr(m), ctypes.byref(h)))
        r = System.__new__(System)
        r.ctx, r.D, r.h = self.ctx, self.D, h
        self.ctx._acquire()
        r.n = int(lib().mmf_dim(h))
        return r

    def dressed_time_evolution(self, dressing, t1: float, t2, precision: int = MMF_FP64):
        """Ud[k] = U_F(t2_k)^dagger U(t2_k, t1) U_F(t1) in the basis dressed by `dressing` (mode
        indices), and the dressed quasienergies Ebar."""
        m = np.ascontiguousarray(np.asarray(dressing, dtype=np.int32))
        t2 = np.ascontiguousarray(np.atleast_1d(np.asarray(t2, dtype=np.float64)))
        Ud = np.zeros((t2.size, self.D, self.D), dtype=np.complex128)
        Eb = np.zeros(self.D)
        _check(lib().mmf_dressed_time_evolution(self.h, int(m.size), _ptr(m), precision, float(t1), int(t2.size),
                                                _ptr(t2), _ptr(Ud), _ptr(Eb)), allow_numeric=True)
        return Ud, Eb

    def time_evolution_operator(self, t, t0: float = 0.0, precision: int = MMF_FP64) -> np.ndarray:
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
        U = np.zeros((t.size, self.D, self.D), dtype=np.complex128)
        _check(lib().mmf_time_evolution_operator(self.h, precision, float(t0), int(t.size), _ptr(t),
                                                 _ptr(U)), allow_numeric=True)
        return U

    def close(self):
        if self.h:
            if not _exiting:
                lib().mmf_sys_destroy(self.h)
            self.h = None
            self.ctx._release()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batch plan over many systems (mmf_batch_*)."""

    def __init__(self, ctx: Context, systems: Sequence[System], precision: int = MMF_FP64, nt: int = 0):
        self.ctx = ctx
        self.systems = list(systems)
        self.count = len(self.systems)
        self.nt = int(nt)
        self.precision = precision
        arr = (ctypes.c_void_p * self.count)(*[s.h.value for s in self.systems])
        h = ctypes.c_void_p()
        self.h = None
        _check(lib().mmf_batch_create(ctx.h, self.count, ctypes.cast(arr, ctypes.c_void_p), precision,
                                      self.nt, ctypes.byref(h)))
        self.h = h
        ctx._acquire()
        self.nE = int(lib().mmf_batch_size(self.h, 0))
        self.nU = int(lib().mmf_batch_size(self.h, 1))
        self.nP = int(lib().mmf_batch_size(self.h, 2))
        self.offE = [int(lib().mmf_batch_offset(self.h, 0, i)) for i in range(self.count)]
        self.offU = [int(lib().mmf_batch_offset(self.h, 1, i)) for i in range(self.count)]
        self.offP = [int(lib().mmf_batch_offset(self.h, 2, i)) for i in range(self.count)]

    def set_times(self, t0: float, t: np.ndarray):
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(self.count, self.nt))
        _check(lib().mmf_batch_set_times(self.h, float(t0), _ptr(t)))

    def upload(self):
        _check(lib().mmf_batch_upload(self.h))

    def run(self):
        _check(lib().mmf_batch_run(self.h))
        return int(lib().mmf_last_launch_count())

    def sync(self) -> np.ndarray:
        st = np.zeros(self.count, dtype=np.int32)
        _check(lib().mmf_batch_sync(self.h, _ptr(st)), allow_numeric=True)
        return st

    def get(self, i: int):
        s = self.systems[i]
        E = np.zeros(s.n)
        U = np.zeros((self.nt, s.D, s.D), dtype=np.complex128)
        P = np.zeros((s.D, s.D))
        _check(lib().mmf_batch_get(self.h, i, _ptr(E), _ptr(U) if self.nt else None, _ptr(P)))
        return E, U, P

    def eigenvectors(self, i: int) -> np.ndarray:
        s = self.systems[i]
        Z = np.zeros((s.n, s.n), dtype=np.complex128)
        _check(lib().mmf_batch_eigenvectors(self.h, i, _ptr(Z)))
        return Z.T.copy()

    def results(self, E=None, U=None, P=None):
        """Packed results into (optionally preallocated, ideally pinned) host arrays."""
        E = np.zeros(self.nE) if E is None else E
        U = np.zeros(max(self.nU, 1), dtype=np.complex128) if U is None else U
        P = np.zeros(self.nP) if P is None else P
        _check(lib().mmf_batch_results(self.h, _ptr(E), _ptr(U), _ptr(P)))
        return E, U, P

    def dressed(self, dress: "Batch"):
        """Sec. 3.3 for every system: this batch is the full systems (times t2, start t1 = t0 of
        set_times), `dress` the same systems restricted to their dressing modes; both run.
        Returns per system (Ud (nt x D x D), Ebar (D))."""
        nu = int(lib().mmf_batch_dressed_size(self.h, 0))
        ne = int(lib().mmf_batch_dressed_size(self.h, 1))
        Ud = np.zeros(max(nu, 1), dtype=np.complex128)
        Eb = np.zeros(max(ne, 1))
        _check(lib().mmf_batch_dressed(self.h, dress.h, _ptr(Ud), _ptr(Eb)))
        out = []
        for i, s in enumerate(self.systems):
            ou = int(lib().mmf_batch_dressed_offset(self.h, 0, i))
            oe = int(lib().mmf_batch_dressed_offset(self.h, 1, i))
            out.append((Ud[ou:ou + self.nt * s.D * s.D].reshape(self.nt, s.D, s.D), Eb[oe:oe + s.D].copy()))
        return out

    def path(self, i: int):
        """(MMF_PATH_* of system i, half-bandwidth used by the band path or 0)."""
        band = ctypes.c_int(0)
        rc = lib().mmf_batch_path(self.h, int(i), ctypes.byref(band))
        if rc < 0:
            _check(rc)
        return rc, band.value

    def results_dev(self, E: int, U: int, P: int, stream: int):
        """Packed results into device buffers (addresses) on the given stream."""
        _check(lib().mmf_batch_results_dev(self.h, E, U, P, stream))

    def unpack(self, E, U, P, i: int):
        s = self.systems[i]
        e = E[self.offE[i]:self.offE[i] + s.n]
        u = U[self.offU[i]:self.offU[i] + self.nt * s.D * s.D].reshape(self.nt, s.D, s.D)
        p = P[self.offP[i]:self.offP[i] + s.D * s.D].reshape(s.D, s.D)
        return e, u, p

    STAGES = ("assemble", "jacobi", "hetrd", "tridiag", "backtransform", "refine_hx", "refine_gram",
              "refine_rest", "outputs")

    def graph(self, enable: bool = True):
        _check(lib().mmf_batch_graph(self.h, 1 if enable else 0))

    def timing(self, max_runs: int):
        _check(lib().mmf_batch_timing(self.h, int(max_runs)))

    def stage_ms(self):
        ms = np.zeros(len(self.STAGES))
        runs = ctypes.c_int(0)
        _check(lib().mmf_batch_stage_ms(self.h, _ptr(ms), ctypes.byref(runs)))
        return dict(zip(self.STAGES, ms.tolist())), int(runs.value)

    def bytes(self) -> int:
        return int(lib().mmf_batch_bytes(self.h))

    def close(self):
        if self.h:
            if not _exiting:
                lib().mmf_batch_destroy(self.h)
            self.h = None
            self.ctx._release()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (mmf_serve_*): submit systems, wait for their results."""

    def __init__(self, ctx: Context, slots: int = 4, max_batch: int = 16, precision: int = MMF_MIXED):
        self.ctx = ctx
        h = ctypes.c_void_p()
        self.h = None
        _check(lib().mmf_serve_create(ctx.h, slots, max_batch, precision, ctypes.byref(h)))
        self.h = h
        ctx._acquire()
        self._shape = {}

    def submit(self, system: System, t, t0: float = 0.0) -> int:
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
        tk = ctypes.c_uint64(0)
        _check(lib().mmf_serve_submit(self.h, system.h, int(t.size), _ptr(t), float(t0), ctypes.byref(tk)))
        self._shape[tk.value] = (system.n, system.D, int(t.size))
        return int(tk.value)

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int(0)
        _check(lib().mmf_serve_poll(self.h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        n, D, nt = self._shape[ticket]
        E = np.zeros(n)
        U = np.zeros((nt, D, D), dtype=np.complex128)
        P = np.zeros((D, D))
        st = ctypes.c_int(0)
        rc = lib().mmf_serve_wait(self.h, ticket, timeout_ms, _ptr(E), _ptr(U) if nt else None, _ptr(P),
                                  ctypes.byref(st))
        if rc != MMF_ERR_STATE:  # anything but a time-out releases the request
            self._shape.pop(ticket, None)
        _check(rc)
        return E, U, P, int(st.value)

    def stats(self):
        p50, p99, mean = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(lib().mmf_serve_stats(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(mean),
                                     ctypes.byref(cnt)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "mean_ms": mean.value, "completed": cnt.value}

    def reset_stats(self):
        _check(lib().mmf_serve_reset_stats(self.h))

    def plan_stats(self):
        c, r, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mmf_serve_plan_stats(self.h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(k)))
        return {"created": c.value, "reused": r.value, "resident": k.value}

    def close(self):
        if self.h:
            if not _exiting:
                lib().mmf_serve_destroy(self.h)
            self.h = None
            self.ctx._release()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
