"""Seeded synthetic inputs for the twisted Wilson flow.

This module is the only code shared by the CUDA path's callers and by the CPU
oracle's callers.  It draws random numbers and builds gauge-link fields; it
holds none of the flow's arithmetic (no staples, forces, integrator, clover or
observables).

Canonical link layout (host and device "canonical" buffers alike): a complex128
array of shape ``(L3, L2, L1, L0, 4, 3, 3)``, i.e. doubles ordered
``[x3][x2][x1][x0][mu][row][col][re,im]`` with ``x0`` fastest.  Extents are
given as ``(L0, L1, L2, L3)``; directions 0 and 1 are the short, twisted plane
of the l x l x 3l x 3l box (Sec. 3.1), directions 2 and 3 the long periodic ones.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), one stream per configuration seeded with the
configuration's seed; uniform u = (x >> 11) * 2**-53; Gaussians by Box-Muller,
omega = sqrt(-2 ln(1-u1)) * (cos, sin)(2 pi u2).  A link is
U = exp(i * amp * sum_a omega_a T_a) with T_a = lambda_a / 2 (Gell-Mann), eight
omegas per link, links drawn in canonical order.  The exponential of the
Hermitian generator is taken with ``torch.linalg.matrix_exp`` (a library
routine, distinct from both exponentials under test).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream started at ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    x = splitmix64(seed, n, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussians(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` (even) standard normals by Box-Muller from uniforms ``offset..offset+n-1``."""
    assert n % 2 == 0
    u = uniforms(seed, n, offset).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    phi = 2.0 * math.pi * u[:, 1]
    out = np.empty((u.shape[0], 2))
    out[:, 0] = r * np.cos(phi)
    out[:, 1] = r * np.sin(phi)
    return out.reshape(-1)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a, shape (8, 3, 3), complex128."""
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0, 0, 1] = g[0, 1, 0] = 1
    g[1, 0, 1], g[1, 1, 0] = -1j, 1j
    g[2, 0, 0], g[2, 1, 1] = 1, -1
    g[3, 0, 2] = g[3, 2, 0] = 1
    g[4, 0, 2], g[4, 2, 0] = -1j, 1j
    g[5, 1, 2] = g[5, 2, 1] = 1
    g[6, 1, 2], g[6, 2, 1] = -1j, 1j
    g[7, 0, 0] = g[7, 1, 1] = 1 / math.sqrt(3)
    g[7, 2, 2] = -2 / math.sqrt(3)
    return g


def _expi(h: np.ndarray, amp: float, device: str = "cpu") -> np.ndarray:
    """exp(i*amp*h) for a stack of Hermitian 3x3 matrices (library exponential)."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(h)).to(device)
    out = torch.linalg.matrix_exp((1j * amp) * t)
    return out.cpu().numpy()


def random_su3(seed: int, n: int, amp: float, offset: int = 0, device: str = "cpu") -> np.ndarray:
    """``n`` matrices exp(i*amp*omega_a*T_a), omegas from uniforms ``offset..``."""
    om = gaussians(seed, 8 * n, offset).reshape(n, 8)
    h = np.einsum("na,aij->nij", om, gell_mann() * 0.5)
    return _expi(h, amp, device)


def sun_generators(N: int) -> np.ndarray:
    """Generalised Gell-Mann matrices lambda_a of SU(N), shape (N^2 - 1, N, N), Tr(l_a l_b) = 2 delta_ab
    (for N = 3 exactly ``gell_mann()``): the symmetric and antisymmetric off-diagonal ones for each
    pair j < k, then the diagonal ones."""
    if N == 3:
        return gell_mann()
    g = []
    for j in range(N):
        for k in range(j + 1, N):
            a = np.zeros((N, N), dtype=np.complex128)
            a[j, k] = a[k, j] = 1
            b = np.zeros((N, N), dtype=np.complex128)
            b[j, k], b[k, j] = -1j, 1j
            g += [a, b]
    for m in range(1, N):
        d = np.zeros((N, N), dtype=np.complex128)
        d[np.arange(m), np.arange(m)] = 1
        d[m, m] = -m
        g.append(d * math.sqrt(2.0 / (m * (m + 1))))
    return np.array(g)


def random_sun(seed: int, n: int, amp: float, N: int, offset: int = 0, device: str = "cpu") -> np.ndarray:
    """``n`` SU(N) matrices exp(i*amp*omega_a*lambda_a/2), N^2 - 1 Gaussian omegas each."""
    if N == 3:
        return random_su3(seed, n, amp, offset, device)
    na = N * N - 1
    om = gaussians(seed, na * n, offset).reshape(n, na)
    h = np.einsum("na,aij->nij", om, sun_generators(N) * 0.5)
    return _expi(h, amp, device)


def n_sites(L) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def random_links(L, seed: int, amp: float, device: str = "cpu", offset: int = 0, N: int = 3) -> np.ndarray:
    """A random SU(N) link field in canonical layout (see module docstring)."""
    L0, L1, L2, L3 = (int(x) for x in L)
    n = n_sites(L) * 4
    return random_sun(seed, n, amp, N, offset, device).reshape(L3, L2, L1, L0, 4, N, N)


def batched_amplitude(seed: int) -> float:
    """Link amplitude of one member of the mixed ensemble: 0.2 + 0.4*u, u the stream's first draw."""
    return 0.2 + 0.4 * float(uniforms(seed, 1)[0])


def batched_member(seed: int, L, device: str = "cpu"):
    """(amplitude, links) of one member of the mixed-size ensemble; omegas follow the first draw."""
    amp = batched_amplitude(seed)
    return amp, random_links(L, seed, amp, device=device, offset=1)


def twist_matrices(k: int = 1, N: int = 3):
    """Clock Gamma_1 = diag(1, w, ..., w^{N-1}) and shift Gamma_2 (e_j -> e_{j+1}), w = exp(2 pi i k/N).

    They satisfy Gamma_1 Gamma_2 = w Gamma_2 Gamma_1, the consistency condition of
    the twist (Sec. 1, Z_12 = exp(2 pi i k / N)).  For even N each is multiplied by an N-th
    root of its inverse determinant so that both lie in SU(N) (a centre phase, which leaves the
    commutation relation unchanged); for N = 3 both determinants are already 1.
    """
    if N == 3:
        w = np.exp(2j * math.pi * k / 3)
        g1 = np.diag([1, w, w * w]).astype(np.complex128)
    else:
        w = np.exp(2j * math.pi * k / N)
        g1 = np.diag([w ** j for j in range(N)]).astype(np.complex128)
    g2 = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        g2[(j + 1) % N, j] = 1
    if N % 2 == 0:
        for g in (g1, g2):
            d = np.linalg.det(g)
            g *= np.exp(-1j * np.angle(d) / N)
    return g1, g2


def twist_eater(L, k: int = 1, N: int = 3) -> np.ndarray:
    """A field whose twisted plaquettes all equal their centre factor (zero twisted action).

    U_0(n) = Gamma_1 where x0 = 0, U_1(n) = Gamma_2 where x1 = 0, every other link
    the unit matrix.  Then P_01(n) = Gamma_1 Gamma_2 Gamma_1^+ Gamma_2^+ = Z_01 at
    x0 = x1 = 0 and P = 1 elsewhere (twist in the (0,1) plane, corner at the origin).
    """
    L0, L1, L2, L3 = (int(x) for x in L)
    g1, g2 = twist_matrices(k, N)
    U = np.zeros((L3, L2, L1, L0, 4, N, N), dtype=np.complex128)
    U[...] = np.eye(N)
    U[:, :, :, 0, 0] = g1
    U[:, :, 0, :, 1] = g2
    return U


def default_twist(k: int = 1) -> np.ndarray:
    """Antisymmetric 4x4 twist tensor n_{mu nu} with n_01 = k, all other planes periodic."""
    n = np.zeros((4, 4), dtype=np.int64)
    n[0, 1], n[1, 0] = k, -k
    return n


def tgf_extent(l: int):
    """The l x l x 3l x 3l box of the twisted gradient-flow scheme (Sec. 3.1)."""
    return (l, l, 3 * l, 3 * l)
