"""Plain FP64 CPU oracle of the twisted Wilson flow and its observables.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares no
code with the CUDA path and imports nothing from it.

It is written to be checked against the paper by eye: numpy arrays over all
sites, ``np.roll`` for neighbours, ``np.matmul`` for 3x3 products, and every
formula written as printed (or, where the paper relies on an outside
definition, as that definition states it).  No blocking, fusion or reordering.

Conventions (Sec. 3.1 of arXiv:2107.03747):
  * extents ``L = (L0, L1, L2, L3)``; directions 0, 1 form the short twisted
    plane (the paper's 1, 2), 2, 3 the long periodic directions;
  * a link field is a complex128 array of shape ``(L3, L2, L1, L0, 4, 3, 3)``
    (x0 fastest, then mu, row, col); ``U[..., mu, :, :]`` is U_mu(n);
  * the twist tensor ``n`` is an antisymmetric integer 4x4 array; the plaquette
    factor Z_{mu nu}(n) = exp(2 pi i n_{mu nu} / N) (N = 3 for the paper's SU(3); every
    function takes N from the field's last axis) at the plaquettes whose
    corner has x_mu = c_mu and x_nu = c_nu (``corner``, default the origin,
    the 0-based reading of "x_1 = x_2 = 1"), and 1 everywhere else.
"""
from __future__ import annotations

import math

import numpy as np

NC = 3


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------

def _axis(mu: int) -> int:
    """Array axis of direction mu in a per-direction field of shape (L3, L2, L1, L0, ...)."""
    return 3 - mu


def shift(A: np.ndarray, mu: int, s: int) -> np.ndarray:
    """The field n -> A(n + s*mu_hat) with periodic indexing."""
    return np.roll(A, -s, axis=_axis(mu))


def dag(A: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(A, -1, -2))


def mm(*ms: np.ndarray) -> np.ndarray:
    out = ms[0]
    for m in ms[1:]:
        out = np.matmul(out, m)
    return out


def tr(A: np.ndarray) -> np.ndarray:
    return np.trace(A, axis1=-2, axis2=-1)


def links_by_dir(U: np.ndarray):
    """[U_0, U_1, U_2, U_3], each of shape (L3, L2, L1, L0, 3, 3)."""
    return [U[..., mu, :, :] for mu in range(4)]


def extents_of(U: np.ndarray):
    L3, L2, L1, L0 = U.shape[:4]
    return (L0, L1, L2, L3)


def coords(L):
    """Coordinate arrays x_mu(n), each of shape (L3, L2, L1, L0)."""
    L0, L1, L2, L3 = L
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0), indexing="ij")
    return [x0, x1, x2, x3]


def twist_factor(L, twist, mu: int, nu: int, corner=(0, 0, 0, 0), N: int = NC) -> np.ndarray:
    """Z_{mu nu}(n) over all sites (Sec. 3.1, the centre factor of the twisted plaquettes).

    Z_{mu nu} = exp(2 pi i n_{mu nu} / N) where x_mu = corner_mu and x_nu = corner_nu,
    and 1 elsewhere; Z_{nu mu} = Z_{mu nu}^* follows from n antisymmetric.
    """
    x = coords(L)
    z = np.ones(x[0].shape, dtype=np.complex128)
    k = int(twist[mu][nu]) % N
    if k != 0 and mu != nu:
        where = (x[mu] == corner[mu]) & (x[nu] == corner[nu])
        z[where] = np.exp(2j * math.pi * int(twist[mu][nu]) / N)
    return z[..., None, None]


# --------------------------------------------------------------------------
# action (Sec. 3.1: S_W = 3b sum_n sum_{mu != nu} Tr[1 - Z*_{mu nu}(n) P_{mu nu}(n)])
# --------------------------------------------------------------------------

def plaquette(Ud, mu: int, nu: int) -> np.ndarray:
    """P_{mu nu}(n) = U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+  (Sec. 3.1)."""
    return mm(Ud[mu], shift(Ud[nu], mu, 1), dag(shift(Ud[mu], nu, 1)), dag(Ud[nu]))


def reduced_action(U: np.ndarray, twist, corner=(0, 0, 0, 0)) -> float:
    """s = sum_n sum_{mu<nu} Re Tr[1 - Z*_{mu nu} P_{mu nu}].

    With b = 1/lambda_0 = 1/(3 g0^2) (Sec. 3.1) this is g0^2 S_W / 2: the sum over
    ordered pairs mu != nu counts each plaquette twice with complex-conjugate traces.
    """
    L = extents_of(U)
    Ud = links_by_dir(U)
    N = U.shape[-1]
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            z = twist_factor(L, twist, mu, nu, corner, N)
            zp = np.conj(z) * plaquette(Ud, mu, nu)
            s += float(np.sum(np.real(tr(np.eye(N) - zp))))
    return s


def wilson_action_ordered(U: np.ndarray, twist, corner=(0, 0, 0, 0)) -> float:
    """sum_n sum_{mu != nu} Tr[1 - Z*_{mu nu} P_{mu nu}] over ordered pairs, as printed (Sec. 3.1)."""
    L = extents_of(U)
    Ud = links_by_dir(U)
    s = 0.0 + 0.0j
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            z = twist_factor(L, twist, mu, nu, corner, U.shape[-1])
            s += np.sum(tr(np.eye(U.shape[-1]) - np.conj(z) * plaquette(Ud, mu, nu)))
    return complex(s)


# --------------------------------------------------------------------------
# flow force Z_mu(n) = -g0^2 d S_W / d U_mu(n)  (Wilson flow, Sec. 3.1)
# --------------------------------------------------------------------------

def proj_ta(M: np.ndarray) -> np.ndarray:
    """Traceless anti-Hermitian part: (M - M^+)/2 - tr(M - M^+)/(2N) * 1."""
    N = M.shape[-1]
    A = 0.5 * (M - dag(M))
    return A - (tr(A) / N)[..., None, None] * np.eye(N)


def staple_sum(Ud, L, twist, mu: int, corner=(0, 0, 0, 0)) -> np.ndarray:
    """Sigma_mu(n) such that Re Tr[U_mu(n) Sigma_mu(n)] is the sum of Re Tr[Z* P] over the
    six plaquettes that contain U_mu(n).

    Forward  (plaquette P_{mu nu}(n)):       Z*_{mu nu}(n)     U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
    Backward (plaquette P_{nu mu}(n-nu)):    Z_{mu nu}(n-nu)   U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu)
    (the backward factor is Z*_{nu mu}(n-nu) = Z_{mu nu}(n-nu)).
    """
    S = np.zeros_like(Ud[mu])
    for nu in range(4):
        if nu == mu:
            continue
        z = twist_factor(L, twist, mu, nu, corner, Ud[mu].shape[-1])
        fwd = np.conj(z) * mm(shift(Ud[nu], mu, 1), dag(shift(Ud[mu], nu, 1)), dag(Ud[nu]))
        z_m = shift(z, nu, -1)
        Unu_m = shift(Ud[nu], nu, -1)
        bwd = z_m * mm(dag(shift(Unu_m, mu, 1)), dag(shift(Ud[mu], nu, -1)), Unu_m)
        S = S + fwd + bwd
    return S


def force(U: np.ndarray, twist, corner=(0, 0, 0, 0)) -> np.ndarray:
    """Z_mu(n) = -g0^2 d_{n,mu} S_W for every link, shape like U.

    Lie derivative d^a f = d/ds f(exp(s T^a) U)|_0 with anti-Hermitian T^a,
    tr(T^a T^b) = -delta^{ab}/2.  From g0^2 S_W = 2 s and d^a s = -Re Tr(T^a Omega)
    with Omega = U_mu Sigma_mu, Z = 2 T^a Re Tr(T^a Omega) = -P_ta(Omega).
    """
    L = extents_of(U)
    Ud = links_by_dir(U)
    Z = np.empty_like(U)
    for mu in range(4):
        Om = mm(Ud[mu], staple_sum(Ud, L, twist, mu, corner))
        Z[..., mu, :, :] = -proj_ta(Om)
    return Z


# --------------------------------------------------------------------------
# exponential: Taylor series with scaling and squaring (Moler & Van Loan, 1978/2003)
# --------------------------------------------------------------------------

def expm(X: np.ndarray) -> np.ndarray:
    """exp(X) for a stack of 3x3 matrices.

    Scale by 2^-s so that ||X 2^-s||_F <= 1/2, sum the Taylor series until the
    added term is below 1e-18 in Frobenius norm (at most 30 terms), then square s times.
    """
    nrm = np.sqrt(np.sum(np.abs(X) ** 2, axis=(-2, -1)))
    s = np.maximum(0, np.ceil(np.log2(np.maximum(nrm, 1e-300) / 0.5))).astype(np.int64)
    out = np.empty_like(X)
    for sv in np.unique(s):
        sel = s == sv
        Y = X[sel] / (2.0 ** sv)
        T = np.broadcast_to(np.eye(X.shape[-1], dtype=X.dtype), Y.shape).copy()
        term = T.copy()
        for k in range(1, 31):
            term = np.matmul(term, Y) / k
            T = T + term
            if np.max(np.abs(term)) < 1e-18:
                break
        for _ in range(int(sv)):
            T = np.matmul(T, T)
        out[sel] = T
    return out


# --------------------------------------------------------------------------
# Runge-Kutta integrator of the Wilson flow (Luscher, JHEP 08 (2010) 071, Sec. 3.2; cited in Sec. 1)
# --------------------------------------------------------------------------

def rk3_step(U: np.ndarray, eps: float, twist, corner=(0, 0, 0, 0)) -> np.ndarray:
    """One step V_t -> V_{t+eps}:

      W0 = V_t
      W1 = exp(1/4 Z0) W0
      W2 = exp(8/9 Z1 - 17/36 Z0) W1
      V_{t+eps} = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,     Z_i = eps Z(W_i).

    Every force of a stage is taken from the field of that stage before any link changes.
    """
    W0 = U
    Z0 = eps * force(W0, twist, corner)
    W1 = np.matmul(expm(0.25 * Z0), W0)
    Z1 = eps * force(W1, twist, corner)
    W2 = np.matmul(expm(8.0 / 9.0 * Z1 - 17.0 / 36.0 * Z0), W1)
    Z2 = eps * force(W2, twist, corner)
    return np.matmul(expm(0.75 * Z2 - 8.0 / 9.0 * Z1 + 17.0 / 36.0 * Z0), W2)


def euler_step(U: np.ndarray, eps: float, twist, corner=(0, 0, 0, 0)) -> np.ndarray:
    """First-order step V_{t+eps} = exp(eps Z(V_t)) V_t (used only to test the integrator's order)."""
    return np.matmul(expm(eps * force(U, twist, corner)), U)


# --------------------------------------------------------------------------
# clover field strength and observables (Sec. 3.1, eqs. gmunu, qlatt)
# --------------------------------------------------------------------------

def clover(Ud, L, twist, mu: int, nu: int, corner=(0, 0, 0, 0)) -> np.ndarray:
    """C_{mu nu}(n) = sum of the four twisted leaves of eq. (gmunu):

      Z*(n)         P_{mu nu}(n)    = U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
      Z*(n-nu)      P_{-nu mu}(n)   = U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu) U_mu(n)^+
      Z*(n-mu)      P_{nu -mu}(n)   = U_nu(n) U_mu(n-mu+nu)^+ U_nu(n-mu)^+ U_mu(n-mu)
      Z*(n-mu-nu)   P_{-mu -nu}(n)  = U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu) U_nu(n-nu)

    with U_{-mu}(n) = U_mu(n-mu)^+ and Z = Z_{mu nu}.
    """
    z = twist_factor(L, twist, mu, nu, corner, Ud[mu].shape[-1])
    Um, Un = Ud[mu], Ud[nu]
    l1 = np.conj(z) * mm(Um, shift(Un, mu, 1), dag(shift(Um, nu, 1)), dag(Un))
    Un_mn = shift(Un, nu, -1)  # U_nu(n-nu)
    l2 = np.conj(shift(z, nu, -1)) * mm(dag(Un_mn), shift(Um, nu, -1), shift(Un_mn, mu, 1), dag(Um))
    Um_mm = shift(Um, mu, -1)  # U_mu(n-mu)
    l3 = np.conj(shift(z, mu, -1)) * mm(Un, dag(shift(Um_mm, nu, 1)), dag(shift(Un, mu, -1)), Um_mm)
    Um_mmn = shift(Um_mm, nu, -1)  # U_mu(n-mu-nu)
    Un_mmn = shift(Un_mn, mu, -1)  # U_nu(n-mu-nu)
    l4 = np.conj(shift(shift(z, mu, -1), nu, -1)) * mm(dag(Um_mm), dag(Un_mmn), Um_mmn, Un_mn)
    return l1 + l2 + l3 + l4


def field_strength(U: np.ndarray, twist, traceless: bool = False, corner=(0, 0, 0, 0)):
    """G^cl_{mu nu}(n) = -(i/8) (C_{mu nu} - C_{mu nu}^+) for all ordered pairs; G[mu][nu].

    ``traceless`` subtracts tr(G)/3 (eq. gmunu prints no projection; off by default).
    """
    L = extents_of(U)
    Ud = links_by_dir(U)
    G = [[None] * 4 for _ in range(4)]
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            C = clover(Ud, L, twist, mu, nu, corner)
            g = (-1j / 8.0) * (C - dag(C))
            if traceless:
                g = g - (tr(g) / g.shape[-1])[..., None, None] * np.eye(g.shape[-1])
            G[mu][nu] = g
    return G


def levi_civita(m: int, n: int, r: int, s: int) -> int:
    """epsilon_{mnrs} with epsilon_{0123} = +1."""
    p = [m, n, r, s]
    if len(set(p)) < 4:
        return 0
    sign = 1
    for i in range(4):
        for j in range(i + 1, 4):
            if p[i] > p[j]:
                sign = -sign
    return sign


def measure(U: np.ndarray, twist, traceless: bool = False, corner=(0, 0, 0, 0)) -> dict:
    """Observables at the current flow time.

    E  = (1/V) sum_n 1/2 Tr[G_{mu nu} G_{mu nu}]            (clover energy density, Sec. 3.1)
    Q  = 1/(16 pi^2) sum_n Tr[G_{mu nu} Gt_{mu nu}],  Gt_{mu nu} = 1/2 eps_{mu nu rho sigma} G_{rho sigma}  (eq. qlatt)
    P  = (1/(6V)) sum_n sum_{mu<nu} 1/3 Re Tr[Z* P_{mu nu}] (average twisted plaquette)
    S  = sum_n sum_{mu<nu} Re Tr[1 - Z* P_{mu nu}]           (= g0^2 S_W / 2)
    Sums over mu, nu run over all ordered pairs where the formula says so.
    """
    L = extents_of(U)
    V = L[0] * L[1] * L[2] * L[3]
    G = field_strength(U, twist, traceless, corner)
    e = 0.0
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                e += 0.5 * float(np.sum(np.real(tr(mm(G[mu][nu], G[mu][nu])))))
    q = 0.0 + 0.0j
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            for rho in range(4):
                for sig in range(4):
                    eps = levi_civita(mu, nu, rho, sig)
                    if eps:
                        q += 0.5 * eps * np.sum(tr(mm(G[mu][nu], G[rho][sig])))
    Ud = links_by_dir(U)
    p = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            z = twist_factor(L, twist, mu, nu, corner, U.shape[-1])
            p += float(np.sum(np.real(tr(np.conj(z) * plaquette(Ud, mu, nu))))) / U.shape[-1]
    return {
        "E": e / V,
        "Q": float(np.real(q)) / (16.0 * math.pi ** 2),
        "P": p / (6.0 * V),
        "S": reduced_action(U, twist, corner),
    }


def charge_density(U: np.ndarray, twist, traceless: bool = False, corner=(0, 0, 0, 0)) -> np.ndarray:
    """q(n) = 1/(16 pi^2) Tr[G_{mu nu}(n) Gt_{mu nu}(n)] per site (the summand of eq. qlatt), shape (L3, L2, L1, L0)."""
    G = field_strength(U, twist, traceless, corner)
    q = 0.0
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            for rho in range(4):
                for sig in range(4):
                    eps = levi_civita(mu, nu, rho, sig)
                    if eps:
                        q = q + 0.5 * eps * tr(mm(G[mu][nu], G[rho][sig]))
    return np.real(q) / (16.0 * math.pi ** 2)


def slice_charge(U: np.ndarray, twist, direction: int = 3, traceless: bool = False, corner=(0, 0, 0, 0)) -> np.ndarray:
    """q(x0, t) of Sec. 4: the charge density summed over the three directions other than
    `direction` (a long one, so the sum includes both short directions); entry x is the slice
    x_direction = x (lattice units)."""
    q = charge_density(U, twist, traceless, corner)
    axes = tuple(a for a in range(4) if a != _axis(direction))
    return np.sum(q, axis=axes)


def slice_correlator(q_slices, Q, keep_cut: float = 0.5):
    """C(d) = <q(x0 + d) q(x0) delta_Q> / <delta_Q> (eq. qcorr) for an ensemble, averaged over the
    source x0 (translation invariance); q_slices[c][x], Q[c] per configuration.
    Returns (C as an array over d = 0..T-1, number of configurations kept) or (None, 0)."""
    q = np.asarray(q_slices, dtype=np.float64)
    keep = np.abs(np.asarray(Q, dtype=np.float64)) < keep_cut
    if not np.any(keep):
        return None, 0
    T = q.shape[1]
    C = np.zeros(T)
    for c in np.nonzero(keep)[0]:
        for d in range(T):
            C[d] += np.mean(np.roll(q[c], -d) * q[c])
    return C / np.sum(keep), int(np.sum(keep))


def flow(U: np.ndarray, eps: float, t_end: float, twist, measure_every: int = 1,
         traceless: bool = False, corner=(0, 0, 0, 0)):
    """Integrate the flow from t = 0 to t_end with RK3 steps of size eps.

    n = floor(t_end/eps + 1e-9) full steps, then one step of eps' = t_end - n eps if
    eps' > 1e-12 * eps.  Observables are recorded before every measure_every-th step
    and once at t_end.  Returns (final links, list of (t, E, Q, P, S)).
    """
    n = int(math.floor(t_end / eps + 1e-9))
    rest = t_end - n * eps
    steps = [eps] * n + ([rest] if rest > 1e-12 * eps else [])
    records = []
    for i, h in enumerate(steps):
        if i % measure_every == 0:
            m = measure(U, twist, traceless, corner)
            records.append((i * eps, m["E"], m["Q"], m["P"], m["S"]))
        U = rk3_step(U, h, twist, corner)
    m = measure(U, twist, traceless, corner)
    records.append((n * eps + (rest if len(steps) > n else 0.0), m["E"], m["Q"], m["P"], m["S"]))
    return U, records


def flow_steps(t_end: float, eps: float):
    """(number of full steps, size of the final partial step or 0)."""
    n = int(math.floor(t_end / eps + 1e-9))
    rest = t_end - n * eps
    return n, (rest if rest > 1e-12 * eps else 0.0)


# --------------------------------------------------------------------------
# coupling lambda_TGF (eqs. lambdat, calA, theta3, lambdat_latt, latt_norm)
# --------------------------------------------------------------------------

def _theta_terms(a: float) -> int:
    """Largest |m| with exp(-pi a m^2) above 1e-40, so the dropped tail is below double rounding."""
    return int(math.ceil(math.sqrt(92.0 / (math.pi * a)))) + 2


def theta3_direct(x: float) -> float:
    """theta_3(0, i x) = sum_m exp(-pi x m^2)  (first form of eq. theta3)."""
    mmax = _theta_terms(x)
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    return float(np.sum(np.exp(-math.pi * x * m * m)))


def theta3_dual(x: float) -> float:
    """theta_3(0, i x) = x^-1/2 sum_m exp(-pi m^2 / x)  (second form of eq. theta3, z = 0)."""
    mmax = _theta_terms(1.0 / x)
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    return float(np.sum(np.exp(-math.pi * m * m / x))) / math.sqrt(x)


def calA(x: float, N: int = 3) -> float:
    """A(x) = x^2 theta3^2(0,ix) (theta3^2(0,ix) - theta3^2(0, i x N^2))  (eq. calA)."""
    t1 = theta3_direct(x)
    tN = theta3_direct(x * N * N)
    return x * x * t1 * t1 * (t1 * t1 - tN * tN)


def lattice_norm_inverse(c: float, Lt: int, N: int = 3) -> float:
    """N^-1(c, Lt) of eq. (latt_norm).

    (c^4/128) sum_{mu != nu} sum'_q exp(-c^2 Lt^2 qhat^2 / 4) sin^2(q_nu) cos^2(q_mu/2) / qhat^2,
    q_mu = 2 pi n_mu / Lt with n_mu = 0..Lt-1 for all four directions, qhat_mu = 2 sin(q_mu/2);
    the primed sum drops the momenta whose two twisted-plane components both satisfy
    Lt q_i = 0 mod 2 N pi, i.e. n_0 = n_1 = 0 (mod N).
    """
    q = 2.0 * math.pi * np.arange(Lt) / Lt
    Q = np.meshgrid(q, q, q, q, indexing="ij")  # Q[mu] over (n0, n1, n2, n3)
    n = np.arange(Lt)
    N0, N1 = np.meshgrid(n, n, indexing="ij")
    excl2 = ((N0 % N) == 0) & ((N1 % N) == 0)
    keep = ~np.broadcast_to(excl2[:, :, None, None], (Lt, Lt, Lt, Lt))
    qhat2 = sum(4.0 * np.sin(Q[m] / 2.0) ** 2 for m in range(4))
    qh = np.where(keep, qhat2, 1.0)
    w = np.where(keep, np.exp(-0.25 * c * c * Lt * Lt * qh) / qh, 0.0)
    tot = 0.0
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            tot += float(np.sum(w * np.sin(Q[nu]) ** 2 * np.cos(Q[mu] / 2.0) ** 2))
    return c ** 4 / 128.0 * tot


def lattice_norm(c: float, Lt: int, N: int = 3) -> float:
    return 1.0 / lattice_norm_inverse(c, Lt, N)


def continuum_norm(c: float, N: int = 3) -> float:
    """Continuum value of N(c): lambda = 128 pi^2 t^2 <E>/(3 N A(pi c^2)) (eq. lambdat) equals
    N <t^2 E>/3 (eq. lambdat_latt) when N(c) = 128 pi^2 / (N A(pi c^2))."""
    return 128.0 * math.pi ** 2 / (N * calA(math.pi * c * c, N))


def lambda_tgf(c: float, Lt: int, t: float, E, Q, N: int = 3):
    """lambda_TGF = N(c, Lt) <t^2 E delta_Q> / (3 <delta_Q>), delta_Q = 1 if |Q| < 0.5 (eq. lambdat_latt).

    Returns (lambda, number of configurations kept); lambda is None when none is kept.
    """
    E = np.asarray(E, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    d = (np.abs(Q) < 0.5).astype(np.float64)
    kept = int(np.sum(d))
    if kept == 0:
        return None, 0
    return lattice_norm(c, Lt, N) * t * t * float(np.sum(E * d)) / (3.0 * float(np.sum(d))), kept
