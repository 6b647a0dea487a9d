"""Python front end of the FP64 CPU oracle (oracle.c) for the multimode Floquet method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the CUDA
path.  A problem is any object with attributes ``D``, ``H0`` (D x D complex),
``omegas``, ``Ns`` and ``couplings`` (``couplings[l][h-1]`` = V^{l+1,h}).

Functions and the passages they follow (arXiv 2005.03426):
  build_hf           Eq. 6 (index read as U^{n-m}) with the layout of Appendix A
  eigh               exact diagonalisation (the paper calls LAPACK, Sec. 3.2): cyclic
                     complex Jacobi, Forsythe & Henrici 1960
  time_evolution     Eq. 3-5 with Eq. 4 read as U_F(t') Ubar U_F(t)^dagger
  transition_avg     time/phase-averaged populations (derived; the paper only names it)
  micromotion        Eq. 5 for one Floquet zone
  rk4                brute-force integration of Eq. 1 in the time domain
  spin_components    Eq. 7 (Sec. 3.4): spin couplings from amplitudes and phases, with the
                     angular-momentum matrices built from their ladder-operator definition
  dressed_time_evolution
                     Sec. 3.3 with Eq. 4: U(t2, t1) in the dressed basis of a subset of modes
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
               "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_dim.restype = i64
        lib.oracle_dim.argtypes = [i32, i32, P]
        lib.oracle_build_hf.restype = i32
        lib.oracle_build_hf.argtypes = [i32, i32, P, P, P, P, P, P]
        lib.oracle_jacobi_eigh.restype = i32
        lib.oracle_jacobi_eigh.argtypes = [i64, P, P, P, i32, f64, P]
        lib.oracle_time_evolution.restype = i32
        lib.oracle_time_evolution.argtypes = [i32, i32, P, P, P, P, f64, i32, P, P]
        lib.oracle_transition_avg.restype = i32
        lib.oracle_transition_avg.argtypes = [i32, i32, P, P, P, f64, P]
        lib.oracle_micromotion.restype = i32
        lib.oracle_micromotion.argtypes = [i32, i32, P, P, P, P, i32, P, P]
        lib.oracle_rk4.restype = i32
        lib.oracle_rk4.argtypes = [i32, i32, P, P, P, P, f64, f64, i64, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _flat(problem):
    D = int(problem.D)
    K = len(problem.omegas)
    N = np.ascontiguousarray(np.array(problem.Ns, dtype=np.int32))
    om = np.ascontiguousarray(np.array(problem.omegas, dtype=np.float64))
    nh = np.ascontiguousarray(np.array([len(c) for c in problem.couplings], dtype=np.int32))
    H0 = np.ascontiguousarray(np.asarray(problem.H0, dtype=np.complex128))
    blocks = [np.asarray(V, dtype=np.complex128) for cl in problem.couplings for V in cl]
    if blocks:
        V = np.ascontiguousarray(np.concatenate([b.reshape(-1) for b in blocks]))
    else:
        V = np.zeros(1, dtype=np.complex128)
    return D, K, N, om, nh, H0, V


def dim(problem) -> int:
    D, K, N, *_ = _flat(problem)
    return int(_load().oracle_dim(D, K, _ptr(N)))


def build_hf(problem) -> np.ndarray:
    """Dense n x n Floquet matrix H_F (complex128)."""
    D, K, N, om, nh, H0, V = _flat(problem)
    n = int(_load().oracle_dim(D, K, _ptr(N)))
    HF = np.zeros((n, n), dtype=np.complex128)
    rc = _load().oracle_build_hf(D, K, _ptr(N), _ptr(om), _ptr(nh), _ptr(H0), _ptr(V), _ptr(HF))
    if rc != 0:
        raise ValueError(f"oracle_build_hf failed: {rc}")
    return HF


def eigh(A: np.ndarray, max_sweeps: int = 60, tol: float = 1e-15):
    """(w ascending, Z with eigenvectors as columns, status, sweeps) by cyclic Jacobi."""
    A = np.array(A, dtype=np.complex128, order="C", copy=True)
    n = A.shape[0]
    w = np.zeros(n, dtype=np.float64)
    Z = np.zeros((n, n), dtype=np.complex128)
    sweeps = ctypes.c_int(0)
    st = _load().oracle_jacobi_eigh(n, _ptr(A), _ptr(w), _ptr(Z), max_sweeps, tol,
                                    ctypes.byref(sweeps))
    return w, Z, int(st), int(sweeps.value)


def time_evolution(problem, E: np.ndarray, Z: np.ndarray, t, t0: float = 0.0) -> np.ndarray:
    """U[k, j, i] = <j| U(t_k, t0) |i>."""
    D, K, N, om, *_ = _flat(problem)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
    E = np.ascontiguousarray(E, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    U = np.zeros((t.size, D, D), dtype=np.complex128)
    _load().oracle_time_evolution(D, K, _ptr(N), _ptr(om), _ptr(E), _ptr(Z), float(t0),
                                  int(t.size), _ptr(t), _ptr(U))
    return U


def transition_avg(problem, E: np.ndarray, Z: np.ndarray, cluster_rel: float = 1e-8) -> np.ndarray:
    """P[i, j] = Pbar_{i -> j}; E ascending."""
    D, K, N, *_ = _flat(problem)
    E = np.ascontiguousarray(E, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    P = np.zeros((D, D), dtype=np.float64)
    _load().oracle_transition_avg(D, K, _ptr(N), _ptr(E), _ptr(Z), float(cluster_rel), _ptr(P))
    return P


def zone_representatives(problem, E: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """The D eigenvectors with the largest weight on the central Fourier block
    sum_i |<i,0|lambda>|^2; ties to the lower eigenvalue index.  Returned in ascending
    eigenvalue order."""
    D, K, N, *_ = _flat(problem)
    b0, s = 0, 1
    for Nk in problem.Ns:
        b0 += Nk * s
        s *= 2 * Nk + 1
    wgt = np.sum(np.abs(Z[b0 * D:(b0 + 1) * D, :]) ** 2, axis=0)
    order = sorted(range(Z.shape[1]), key=lambda l: (-wgt[l], l))
    return np.array(sorted(order[:D]), dtype=np.int64)


def micromotion(problem, Z: np.ndarray, reps, t) -> np.ndarray:
    """UF[k, j, a] = sum_n e^{-i n.w t_k} <j,n|lambda_a>."""
    D, K, N, om, *_ = _flat(problem)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(t, dtype=np.float64)))
    reps = np.ascontiguousarray(np.asarray(reps, dtype=np.int64))
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    UF = np.zeros((t.size, D, D), dtype=np.complex128)
    _load().oracle_micromotion(D, K, _ptr(N), _ptr(om), _ptr(Z), _ptr(reps), int(t.size),
                               _ptr(t), _ptr(UF))
    return UF


def rk4(problem, t0: float, t1: float, steps: int) -> np.ndarray:
    """U(t1, t0) by fixed-step RK4 of i dpsi/dt = H(t) psi (D x D, U[j, i])."""
    D, K, N, om, nh, H0, V = _flat(problem)
    U = np.zeros((D, D), dtype=np.complex128)
    _load().oracle_rk4(D, K, _ptr(om), _ptr(nh), _ptr(H0), _ptr(V), float(t0), float(t1),
                       int(steps), _ptr(U))
    return U


def solve(problem, t=None, t0: float = 0.0, cluster_rel: float = 1e-8):
    """Whole path: H_F -> (E, Z) -> U(t, t0), Pbar.  Returns a dict."""
    HF = build_hf(problem)
    E, Z, st, sw = eigh(HF)
    out = {"HF": HF, "E": E, "Z": Z, "status": st, "sweeps": sw}
    if t is not None:
        out["U"] = time_evolution(problem, E, Z, t, t0)
    out["P"] = transition_avg(problem, E, Z, cluster_rel)
    return out


def spin_operators(S2: int):
    """(S_x, S_y, S_z) for spin S = S2/2 in the basis m = S, S-1, ..., -S: S_z = diag(m) and
    S_+ = S_x + i S_y with <m+1|S_+|m> = sqrt(S(S+1) - m(m+1))."""
    S = S2 / 2.0
    ms = [S - k for k in range(S2 + 1)]
    Sp = np.zeros((S2 + 1, S2 + 1), dtype=np.complex128)
    for a, m_row in enumerate(ms):
        for b, m_col in enumerate(ms):
            if abs(m_row - (m_col + 1.0)) < 1e-12:
                Sp[a, b] = np.sqrt(S * (S + 1.0) - m_col * (m_col + 1.0))
    Sm = Sp.conj().T
    return (Sp + Sm) / 2.0, (Sp - Sm) / 2.0j, np.diag(np.array(ms, dtype=np.complex128))


def spin_components(S2: int, A, phi=(0.0, 0.0, 0.0), static: bool = False) -> np.ndarray:
    """Eq. 7: the coupling sum_i (A_i/2) e^{i phi_i} S_i of the drive sum_i A_i cos(h w t + phi_i) S_i
    (the convention H(t) = H0 + V e^{i h w t} + V^dagger e^{-i h w t}), or sum_i A_i S_i for the
    static part."""
    ops = spin_operators(S2)
    V = np.zeros_like(ops[0])
    for k in range(3):
        c = A[k] if static else 0.5 * A[k] * np.exp(1j * phi[k])
        V = V + c * ops[k]
    return V


class _Restricted:
    """A problem restricted to some of its modes (same levels and static part)."""

    def __init__(self, problem, modes):
        self.D = problem.D
        self.H0 = problem.H0
        self.omegas = [problem.omegas[k] for k in modes]
        self.Ns = [problem.Ns[k] for k in modes]
        self.couplings = [problem.couplings[k] for k in modes]


def dressed_time_evolution(problem, dressing, t1: float, t2: float):
    """Sec. 3.3: the evolution from t1 to t2 expressed in the time-dependent basis of the
    dressing modes (indices into the problem's modes).  The problem restricted to those modes
    gives the micromotion operator U_F(t) of Eq. 5 for one Floquet zone (zone_representatives)
    and its quasienergies Ebar; the full problem gives U(t2, t1) (Eq. 3-4).  Returns
    (U_F(t2)^dagger U(t2, t1) U_F(t1), Ebar)."""
    sub = _Restricted(problem, list(dressing))
    Ed, Zd, _, _ = eigh(build_hf(sub))
    reps = zone_representatives(sub, Ed, Zd)
    UF = micromotion(sub, Zd, reps, np.array([t1, t2], dtype=np.float64))
    E, Z, _, _ = eigh(build_hf(problem))
    U = time_evolution(problem, E, Z, np.array([t2], dtype=np.float64), t1)[0]
    return UF[1].conj().T @ U @ UF[0], Ed[reps]
