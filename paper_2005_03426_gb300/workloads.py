"""Seeded synthetic inputs for the multimode Floquet problem (Eq. 1).

This module only *describes* driven quantum systems: the static Hamiltonian H0 and
the harmonic couplings V^{l,h} of Eq. 1, the drive frequencies and the Fourier
truncations.  It contains none of the method's arithmetic (no Floquet matrix, no
eigensolver, no time evolution), so both the FP64 CPU oracle and the CUDA path
consume exactly the same bytes from it.

Coupling convention (Eq. 1 with "+ h.c." applied to the drive terms only):
    H(t) = H0 + sum_{l,h} ( V^{l,h} e^{+i h w_l t} + V^{l,h}^dagger e^{-i h w_l t} ),
so a real drive  A cos(w t) O  (O Hermitian) enters as V = (A/2) O at harmonic 1.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a
counter-based 64-bit generator, uniform doubles from the top 53 bits, normals by
Box-Muller.  Everything is pure integer/NumPy arithmetic, so the bytes do not
depend on the NumPy version.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream; ``next_u64`` returns mix(seed + k*gamma) for k = 1, 2, ..."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in {lo, ..., hi} (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair; the other is discarded)."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def complex_gaussian(self, sigma: float) -> complex:
        """Circular complex Gaussian: Re, Im i.i.d. N(0, sigma^2/2), so E|g|^2 = sigma^2."""
        s = sigma / math.sqrt(2.0)
        re = self.normal() * s
        im = self.normal() * s
        return complex(re, im)


@dataclass
class Problem:
    """One driven system: D levels, static H0 (D x D Hermitian) and K drive modes.

    ``couplings[l][h-1]`` is V^{l+1,h} (D x D complex), harmonic h >= 1 of mode l+1.
    Mode 1 is the innermost Fourier index of the Floquet matrix (Appendix A).
    """

    D: int
    H0: np.ndarray
    omegas: List[float]
    Ns: List[int]
    couplings: List[List[np.ndarray]] = field(default_factory=list)

    @property
    def K(self) -> int:
        return len(self.omegas)

    @property
    def M(self) -> int:
        m = 1
        for N in self.Ns:
            m *= 2 * N + 1
        return m

    @property
    def n(self) -> int:
        return self.D * self.M

    def nharm(self) -> List[int]:
        return [len(c) for c in self.couplings]

    def period(self) -> float:
        """Time grid period: 2 pi / omega_1 (first mode)."""
        return 2.0 * math.pi / self.omegas[0]


def time_grid(problem: Problem, nt: int) -> np.ndarray:
    """t_k = k T / nt, k = 0..nt-1 with T = 2 pi / omega_1 (includes 0, excludes T)."""
    T = problem.period()
    return np.array([k * T / nt for k in range(nt)], dtype=np.float64)


# ---------------------------------------------------------------- spin operators
def spin_matrices(S2: int):
    """Angular-momentum matrices (Fx, Fy, Fz) for spin S = S2/2 in the |S, m> basis with
    m = S, S-1, ..., -S (standard definition, Sakurai Sec. 3.5)."""
    S = S2 / 2.0
    dim = S2 + 1
    ms = [S - k for k in range(dim)]
    Fz = np.diag(np.array(ms, dtype=np.complex128))
    Fp = np.zeros((dim, dim), dtype=np.complex128)
    for k in range(1, dim):
        m = ms[k]
        Fp[k - 1, k] = math.sqrt(S * (S + 1) - m * (m + 1))
    Fm = Fp.conj().T
    Fx = 0.5 * (Fp + Fm)
    Fy = -0.5j * (Fp - Fm)
    return Fx, Fy, Fz


def hermitian_gaussian(rng: SplitMix64, D: int, sigma: float) -> np.ndarray:
    """V = (G + G^dagger)/2 with G entries circular complex Gaussian of std sigma
    (drawn row-major)."""
    G = np.zeros((D, D), dtype=np.complex128)
    for i in range(D):
        for j in range(D):
            G[i, j] = rng.complex_gaussian(sigma)
    return 0.5 * (G + G.conj().T)


def haar_unitary(rng: SplitMix64, D: int) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of R's
    diagonal moved into Q (Mezzadri, Notices AMS 2007)."""
    Z = np.zeros((D, D), dtype=np.complex128)
    for i in range(D):
        for j in range(D):
            Z[i, j] = rng.complex_gaussian(1.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = d / np.abs(d)
    return Q * ph[None, :]


# ---------------------------------------------------------------- workloads
def two_level(omega: float, N: int = 20, omega0: float = 1.0, Omega: float = 0.5) -> Problem:
    """Linearly driven qubit H = (w0/2) sz + Omega cos(w t) sx  ->  V = (Omega/2) sx."""
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    H0 = 0.5 * omega0 * sz
    V = 0.5 * Omega * sx
    return Problem(D=2, H0=H0, omegas=[float(omega)], Ns=[N], couplings=[[V]])


def qubit_sweep(count: int = 200, N: int = 20, lo: float = 0.2, hi: float = 2.0) -> List[Problem]:
    """Two-level single-mode sweep: omega = linspace(lo, hi, count) inclusive, N Fourier modes
    (n = 2 (2N+1); 82 at N = 20)."""
    ws = np.linspace(lo, hi, count)
    return [two_level(float(w), N=N) for w in ws]


def spin1_bichromatic(Omega1: float, Omega2: float, N1: int = 10, N2: int = 10,
                      omega0: float = 1.0, omega1: float = 1.0,
                      omega2: float = (math.sqrt(5.0) - 1.0) / 2.0) -> Problem:
    """Spin-1: H = w0 Fz + Omega1 cos(w1 t) Fx + Omega2 cos(w2 t) Fz (n = 3 (2N1+1)(2N2+1))."""
    Fx, _, Fz = spin_matrices(2)
    return Problem(D=3, H0=omega0 * Fz, omegas=[omega1, omega2], Ns=[N1, N2],
                   couplings=[[0.5 * Omega1 * Fx], [0.5 * Omega2 * Fz]])


def spin1_amplitude_set(count: int = 64, seed: int = 1, N1: int = 10, N2: int = 10) -> List[Problem]:
    """``count`` seeded amplitude pairs (Omega1, Omega2) ~ U[0.05, 0.5]^2 (n = 1323 at N = 10)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        a1 = rng.uniform_in(0.05, 0.5)
        a2 = rng.uniform_in(0.05, 0.5)
        out.append(spin1_bichromatic(a1, a2, N1=N1, N2=N2))
    return out


def random_multimode(rng: SplitMix64, D: int, Ns: List[int], sigma: float = 0.1,
                     wlo: float = 0.3, whi: float = 1.5) -> Problem:
    """Diagonal H0 with levels U[0,1]; per mode a Hermitian Gaussian coupling (std sigma)
    at harmonic 1 and omega ~ U[wlo, whi]."""
    H0 = np.diag(np.array([rng.uniform() for _ in range(D)], dtype=np.complex128))
    omegas, couplings = [], []
    for _ in Ns:
        couplings.append([hermitian_gaussian(rng, D, sigma)])
        omegas.append(rng.uniform_in(wlo, whi))
    return Problem(D=D, H0=H0, omegas=omegas, Ns=list(Ns), couplings=couplings)


def uneven_batch(count: int = 4096, seed: int = 0, nmax: int = 2000, Dlo: int = 2, Dhi: int = 8,
                 Nlo: int = 4, Nhi: int = 30) -> List[Problem]:
    """Uneven batch: D ~ U{2..8}, K ~ U{1,2}, N_k ~ U{4..30}, (D, K, N) re-drawn until
    n = D prod(2N_k+1) <= nmax; then H0 = diag(U[0,1]), Hermitian couplings sigma = 0.1,
    omega ~ U[0.3, 1.5]."""
    rng = SplitMix64(seed)
    out = []
    while len(out) < count:
        D = rng.integer(Dlo, Dhi)
        K = rng.integer(1, 2)
        Ns = [rng.integer(Nlo, Nhi) for _ in range(K)]
        n = D
        for N in Ns:
            n *= 2 * N + 1
        if n > nmax:
            continue
        out.append(random_multimode(rng, D, Ns))
    return out


def large_instance(seed: int = 3, D: int = 8, N: int = 6, sigma: float = 0.05) -> Problem:
    """D = 8 Haar-rotated H0 (eigenvalues U[0,2]), three modes w = (1, sqrt2, sqrt3)/2,
    Hermitian Gaussian couplings sigma = 0.05, N = (6,6,6) -> n = 17576."""
    rng = SplitMix64(seed)
    lam = np.array([rng.uniform_in(0.0, 2.0) for _ in range(D)])
    Q = haar_unitary(rng, D)
    H0 = (Q * lam[None, :]) @ Q.conj().T
    H0 = 0.5 * (H0 + H0.conj().T)
    omegas = [0.5, math.sqrt(2.0) / 2.0, math.sqrt(3.0) / 2.0]
    couplings = [[hermitian_gaussian(rng, D, sigma)] for _ in range(3)]
    return Problem(D=D, H0=H0, omegas=omegas, Ns=[N, N, N], couplings=couplings)


def driven_lattice(omega: float, D: int = 256, N: int = 3, V0: float = 0.25, t: float = 0.125,
                   V: float = 0.0625, phi: float = 0.0) -> Problem:
    """Harmonically driven 1-D lattice (Sec. 4.2, Eq. 9): D sites, D/2 two-site cells.

    Site m = 1..D (1-based, as in Eq. 9) has the offset (-1)^m V0.  The static hopping from
    site m to m+1 (m = 1..D-1) is t e^{i cos(2 pi m / D)}, with its Hermitian conjugate.  The
    same bonds carry the uniform modulation V cos(w t + phi).  In this module's convention
    that modulation is V^{1,1} = (V/2) e^{i phi} A, with A the real nearest-neighbour adjacency
    (its conjugate term gives the e^{-i w t} part).  One mode, Fourier truncation N, so
    n = D (2N + 1)."""
    H0 = np.zeros((D, D), dtype=np.complex128)
    A = np.zeros((D, D), dtype=np.complex128)
    for m in range(1, D + 1):
        H0[m - 1, m - 1] = V0 if m % 2 == 0 else -V0
    for m in range(1, D):
        h = t * complex(math.cos(math.cos(2.0 * math.pi * m / D)), math.sin(math.cos(2.0 * math.pi * m / D)))
        H0[m - 1, m] = h
        H0[m, m - 1] = h.conjugate()
        A[m - 1, m] = 1.0
        A[m, m - 1] = 1.0
    Vc = 0.5 * V * complex(math.cos(phi), math.sin(phi)) * A
    return Problem(D=D, H0=H0, omegas=[float(omega)], Ns=[N], couplings=[[Vc]])


def lattice_sweep(count: int = 64, lo: float = 0.2, hi: float = 1.0, D: int = 256,
                  N: int = 3) -> List[Problem]:
    """Spectrum-versus-frequency sweep of the driven lattice (Fig. 5's parameters: D = 256,
    V0 = 0.25, t = 0.125, V = 0.0625, phi = 0): omega = linspace(lo, hi, count) inclusive,
    N = 3 (n = 1792 at D = 256)."""
    ws = np.linspace(lo, hi, count)
    return [driven_lattice(float(w), D=D, N=N) for w in ws]


def random_small(seed: int, D: int, Ns: List[int], nharm: List[int] | None = None,
                 sigma: float = 0.3, full_h0: bool = True) -> Problem:
    """Small random test system: Hermitian Gaussian H0 (or diagonal), per mode ``nharm[l]``
    harmonics with Gaussian (generally non-Hermitian) couplings, omega ~ U[0.5, 1.5]."""
    rng = SplitMix64(seed)
    if nharm is None:
        nharm = [1] * len(Ns)
    if full_h0:
        H0 = hermitian_gaussian(rng, D, 1.0)
    else:
        H0 = np.diag(np.array([rng.uniform() for _ in range(D)], dtype=np.complex128))
    omegas, couplings = [], []
    for k, _ in enumerate(Ns):
        omegas.append(rng.uniform_in(0.5, 1.5))
        cl = []
        for _h in range(nharm[k]):
            G = np.zeros((D, D), dtype=np.complex128)
            for i in range(D):
                for j in range(D):
                    G[i, j] = rng.complex_gaussian(sigma)
            cl.append(G)
        couplings.append(cl)
    return Problem(D=D, H0=H0, omegas=omegas, Ns=list(Ns), couplings=couplings)


def serving_stream(count: int, seed: int = 40) -> List[Problem]:
    """Request mix for the serving benchmark: each request is, with equal probability, a driven
    qubit (omega ~ U[0.2, 2], N = 20, n = 82), a spin-1 two-mode system (amplitudes ~ U[0.05, 0.5],
    N = (10, 10), n = 1323) or an uneven-batch draw (n <= 2000)."""
    rng = SplitMix64(seed)
    out = []
    while len(out) < count:
        kind = rng.integer(0, 2)
        if kind == 0:
            out.append(two_level(rng.uniform_in(0.2, 2.0), N=20))
        elif kind == 1:
            a1 = rng.uniform_in(0.05, 0.5)
            a2 = rng.uniform_in(0.05, 0.5)
            out.append(spin1_bichromatic(a1, a2))
        else:
            while True:
                D = rng.integer(2, 8)
                K = rng.integer(1, 2)
                Ns = [rng.integer(4, 30) for _ in range(K)]
                n = D
                for N in Ns:
                    n *= 2 * N + 1
                if n <= 2000:
                    break
            out.append(random_multimode(rng, D, Ns))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (exponential gaps)."""
    rng = SplitMix64(seed)
    t, out = 0.0, []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        out.append(t)
    return np.array(out)
