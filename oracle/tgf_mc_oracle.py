"""Plain FP64 CPU oracle of the twisted hybrid Monte Carlo update (heat-bath + over-relaxation).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` do.  It shares no code with the CUDA path and imports nothing from it.

What it computes (Sec. 3.1 of arXiv:2107.03747): ensembles of the twisted Wilson action
S_W = 3b sum_n sum_{mu != nu} Tr[1 - Z*_{mu nu}(n) P_{mu nu}(n)] are generated with a hybrid
algorithm, one heat-bath sweep (Creutz; Fabricius-Haan) followed by L~ over-relaxation sweeps
(Creutz), the paper's references for the update.  With beta = 18 b (= 2N/g0^2, N = 3) the
weight of one link U = U_mu(n) is exp((beta/3) Re Tr[U Sigma]), Sigma the twisted staple sum
of ``tgf_oracle.staple_sum``.  SU(3) is updated in its three SU(2) subgroups (Cabibbo-Marinari):
for the block M of W = U Sigma in rows and columns (i, j), the part proportional to SU(2) is
k v with v in SU(2); the heat-bath draws X in SU(2) with density exp(alpha X_0) dHaar,
alpha = 2 beta k / 3, and sets U <- R U with R = X v^+; over-relaxation sets R = (v^+)^2, which
keeps Re Tr[U Sigma] unchanged.  X_0 is drawn by Kennedy-Pendleton's algorithm (Phys. Lett. B
156 (1985) 393) for alpha > 2 and by Creutz's (Phys. Rev. D 21 (1980) 2308) otherwise.

Order of a sweep: for mu = 0..3, for parity p = 0, 1 (parity of x0+x1+x2+x3): every link
(n, mu) with parity(n) = p, updated from the current field (its staples contain only links
of other directions or of the other parity, so the order inside a pass does not matter);
subgroups (0,1), (0,2), (1,2) in turn.  Every extent must be even.

Random numbers: a counter-based generator, the SplitMix64 output function (Steele, Lea,
Flood, OOPSLA 2014) applied to key + (counter + 1) * 0x9E3779B97F4A7C15, where the key of
configuration c is SplitMix64's output for counter c under the caller's seed, and a draw is
u = ((x >> 11) + 1) 2^-53 in (0, 1].  The draw of slot s of subgroup g of link (site, mu) in
heat-bath sweep number w has counter (((w * 4 + mu) * V + site) * 3 + g) * 260 + s; slots
4a .. 4a+3 serve rejection attempt a < 64, slots 256 and 257 the direction of X.  A subgroup
whose 64 attempts are all rejected is left unchanged.  ``site`` is the canonical site index
x0 + L0 (x1 + L1 (x2 + L2 x3)).

Quaternion convention: X = X0 1 + i (X1 s1 + X2 s2 + X3 s3) with the Pauli matrices s_k,
i.e. [[X0 + i X3, X2 + i X1], [-X2 + i X1, X0 - i X3]].
"""
from __future__ import annotations

import math

import numpy as np

from . import tgf_oracle as O

GOLDEN = 0x9E3779B97F4A7C15
MASK = 0xFFFFFFFFFFFFFFFF
SLOTS = 260
ATTEMPTS = 64
SUBGROUPS = ((0, 1), (0, 2), (1, 2))


# --------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------

def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 values."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def hash64(key: int, counter) -> np.ndarray:
    """Output number ``counter`` of the SplitMix64 stream started at state ``key``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key & MASK) + (c + np.uint64(1)) * np.uint64(GOLDEN))


def config_key(seed: int, cfg: int) -> int:
    return int(hash64(seed, cfg))


def uniform(key: int, counter) -> np.ndarray:
    """Draws in (0, 1] with 53 random bits."""
    x = hash64(key, counter)
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def draw_counter(sweep: int, mu: int, V: int, site, sub: int, slot) -> np.ndarray:
    site = np.asarray(site, dtype=np.uint64)
    return ((((np.uint64(sweep) * np.uint64(4) + np.uint64(mu)) * np.uint64(V) + site) * np.uint64(3)
             + np.uint64(sub)) * np.uint64(SLOTS) + np.asarray(slot, dtype=np.uint64))


# --------------------------------------------------------------------------
# SU(2) pieces
# --------------------------------------------------------------------------

def su2_part(M: np.ndarray) -> np.ndarray:
    """Quaternion (x0, x1, x2, x3) of the part of the 2x2 complex matrices M proportional to SU(2)."""
    x0 = 0.5 * (M[..., 0, 0].real + M[..., 1, 1].real)
    x1 = 0.5 * (M[..., 0, 1].imag + M[..., 1, 0].imag)
    x2 = 0.5 * (M[..., 0, 1].real - M[..., 1, 0].real)
    x3 = 0.5 * (M[..., 0, 0].imag - M[..., 1, 1].imag)
    return np.stack([x0, x1, x2, x3], axis=-1)


def qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of quaternions in the convention of the module docstring."""
    a0, av = a[..., 0], a[..., 1:]
    b0, bv = b[..., 0], b[..., 1:]
    c0 = a0 * b0 - np.sum(av * bv, axis=-1)
    cv = a0[..., None] * bv + b0[..., None] * av - np.cross(av, bv)
    return np.concatenate([c0[..., None], cv], axis=-1)


def qconj(a: np.ndarray) -> np.ndarray:
    return np.concatenate([a[..., :1], -a[..., 1:]], axis=-1)


def q_to_mat(a: np.ndarray) -> np.ndarray:
    m = np.empty(a.shape[:-1] + (2, 2), dtype=np.complex128)
    m[..., 0, 0] = a[..., 0] + 1j * a[..., 3]
    m[..., 0, 1] = a[..., 2] + 1j * a[..., 1]
    m[..., 1, 0] = -a[..., 2] + 1j * a[..., 1]
    m[..., 1, 1] = a[..., 0] - 1j * a[..., 3]
    return m


def sample_x0(alpha: np.ndarray, key: int, counter0: np.ndarray):
    """X0 with density sqrt(1 - X0^2) exp(alpha X0) on [-1, 1] for each entry of alpha.

    counter0: counter of slot 0 of each entry.  Returns (X0, accepted)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    x0 = np.zeros_like(alpha)
    done = np.zeros(alpha.shape, dtype=bool)
    kp = alpha > 2.0
    for a in range(ATTEMPTS):
        todo = ~done
        if not todo.any():
            break
        r = [uniform(key, counter0 + np.uint64(4 * a + j)) for j in range(4)]
        # Kennedy-Pendleton: lambda^2 = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 alpha), accept if r4^2 <= 1 - lambda^2
        with np.errstate(divide="ignore", invalid="ignore"):
            lam2 = -(np.log(r[0]) + np.cos(2.0 * math.pi * r[1]) ** 2 * np.log(r[2])) / (2.0 * alpha)
            ok_kp = r[3] * r[3] <= 1.0 - lam2
            x_kp = 1.0 - 2.0 * lam2
            # Creutz: X0 = 1 + ln(e^{-2 alpha} + (1 - e^{-2 alpha}) r1) / alpha, accept if r2^2 <= 1 - X0^2
            small = alpha < 1e-8
            e2a = np.exp(-2.0 * alpha)
            x_cr = np.where(small, 2.0 * r[0] - 1.0, 1.0 + np.log(e2a + (1.0 - e2a) * r[0]) / np.where(small, 1.0, alpha))
            ok_cr = r[1] * r[1] <= 1.0 - x_cr * x_cr
        ok = np.where(kp, ok_kp, ok_cr) & todo
        x0 = np.where(ok, np.where(kp, x_kp, x_cr), x0)
        done |= ok
    return x0, done


def random_su2(x0: np.ndarray, key: int, counter0: np.ndarray) -> np.ndarray:
    """Quaternion (X0, |X| n) with n uniform on the sphere from slots 256, 257."""
    cth = 2.0 * uniform(key, counter0 + np.uint64(256)) - 1.0
    phi = 2.0 * math.pi * uniform(key, counter0 + np.uint64(257))
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    r = np.sqrt(np.maximum(0.0, 1.0 - x0 * x0))
    return np.stack([x0, r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth], axis=-1)


# --------------------------------------------------------------------------
# sweeps
# --------------------------------------------------------------------------

def parity_mask(L) -> np.ndarray:
    x = O.coords(L)
    return (x[0] + x[1] + x[2] + x[3]) % 2


def site_index(L) -> np.ndarray:
    x = O.coords(L)
    return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))


def _update_links(U_mu, S_mu, beta, kind, key, sweep, mu, V, sites):
    """Cabibbo-Marinari update of the links U_mu (n, 3, 3) with staple sums S_mu (n, 3, 3)."""
    U = U_mu.copy()
    W = np.matmul(U, S_mu)
    for g, (i, j) in enumerate(SUBGROUPS):
        M = W[:, [i, j], :][:, :, [i, j]]
        x = su2_part(M)
        k = np.sqrt(np.sum(x * x, axis=-1))
        live = k > 1e-300
        v = np.where(live[:, None], x / np.where(live, k, 1.0)[:, None], np.array([1.0, 0, 0, 0]))
        if kind == "hb":
            c0 = draw_counter(sweep, mu, V, sites, g, 0)
            x0, acc = sample_x0(2.0 * beta * k / 3.0, key, c0)
            X = random_su2(x0, key, c0)
            R = qmul(X, qconj(v))
            R = np.where(acc[:, None], R, np.array([1.0, 0, 0, 0]))
        else:
            vd = qconj(v)
            R = qmul(vd, vd)
            R = np.where(live[:, None], R, np.array([1.0, 0, 0, 0]))
        R2 = q_to_mat(R)
        E = np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape).copy()
        E[:, i, i] = R2[:, 0, 0]
        E[:, i, j] = R2[:, 0, 1]
        E[:, j, i] = R2[:, 1, 0]
        E[:, j, j] = R2[:, 1, 1]
        U = np.matmul(E, U)
        W = np.matmul(E, W)
    return U


def sweep(U: np.ndarray, twist, beta: float, kind: str, seed: int = 0, cfg: int = 0,
          sweep_index: int = 0) -> np.ndarray:
    """One heat-bath (kind='hb') or over-relaxation (kind='or') sweep of every link; returns the
    new field (canonical layout, see ``tgf_oracle``)."""
    L = O.extents_of(U)
    if any(l % 2 for l in L):
        raise ValueError("checkerboard sweeps need even extents")
    V = L[0] * L[1] * L[2] * L[3]
    key = config_key(seed, cfg)
    U = U.copy()
    par = parity_mask(L)
    sid = site_index(L)
    for mu in range(4):
        for p in (0, 1):
            Ud = O.links_by_dir(U)
            S = O.staple_sum(Ud, L, twist, mu)
            sel = par == p
            new = _update_links(U[..., mu, :, :][sel], S[sel], beta, kind, key, sweep_index, mu, V, sid[sel])
            Umu = U[..., mu, :, :]
            Umu[sel] = new
            U[..., mu, :, :] = Umu
    return U


def hybrid(U: np.ndarray, twist, beta: float, n_or: int, seed: int, cfg: int, hb_index: int) -> np.ndarray:
    """One hybrid sweep: a heat-bath sweep (numbered hb_index) and n_or over-relaxation sweeps."""
    U = sweep(U, twist, beta, "hb", seed, cfg, hb_index)
    for _ in range(n_or):
        U = sweep(U, twist, beta, "or", seed, cfg, 0)
    return U


# --------------------------------------------------------------------------
# closed forms used by the pins
# --------------------------------------------------------------------------

def su3_one_link_re_tr(x: float, qmax: int = 40) -> float:
    """<Re Tr U> for U in SU(3) with weight exp(x Re Tr U) (Haar measure): d/dx ln Z(x) with
    Z(x) = sum_q det[I_{q+i-j}(x)]_{i,j=0..2}, the one-link SU(N) integral written as a sum of
    Toeplitz determinants of modified Bessel functions (the U(N) integral is the q = 0 term)."""
    from scipy.special import iv

    def Z(y):
        tot = 0.0
        for q in range(-qmax, qmax + 1):
            m = np.array([[iv(q + i - j, y) for j in range(3)] for i in range(3)])
            tot += np.linalg.det(m)
        return tot

    h = 1e-5 * max(1.0, x)
    return (math.log(Z(x + h)) - math.log(Z(x - h))) / (2 * h)


def x0_mean(alpha: float) -> float:
    """<X0> for the density sqrt(1 - X0^2) exp(alpha X0) on [-1, 1]: I_2(alpha) / I_1(alpha)."""
    from scipy.special import iv

    return float(iv(2, alpha) / iv(1, alpha))
