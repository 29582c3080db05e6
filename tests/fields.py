"""Hand-built link fields and field transformations used by the tests.

These are test constructions with known answers (closed forms, symmetries); they
contain no part of the flow or of the observables.
"""
import math

import numpy as np

from paper_2107_03747_gb300 import inputs as I


def unit_field(L):
    L0, L1, L2, L3 = L
    U = np.zeros((L3, L2, L1, L0, 4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def gauge_transform(U, Lam):
    """U_mu(n) -> Lam(n) U_mu(n) Lam(n+mu)^+ with periodic Lam of shape (L3, L2, L1, L0, 3, 3)."""
    out = np.empty_like(U)
    for mu in range(4):
        Lp = np.roll(Lam, -1, axis=3 - mu)
        out[..., mu, :, :] = Lam @ U[..., mu, :, :] @ np.conj(np.swapaxes(Lp, -1, -2))
    return out


def random_gauge(L, seed, amp=2.0):
    L0, L1, L2, L3 = L
    return I.random_su3(seed, L0 * L1 * L2 * L3, amp).reshape(L3, L2, L1, L0, 3, 3)


def reflect_x3(U):
    """Parity in direction 3: x3 -> -x3, U'_mu(n) = U_mu(Rn) (mu != 3), U'_3(n) = U_3(Rn - 3)^+."""
    L3 = U.shape[0]
    r = (-np.arange(L3)) % L3
    r1 = (-np.arange(L3) - 1) % L3
    out = U[r].copy()
    out[..., 3, :, :] = np.conj(np.swapaxes(U[r1][..., 3, :, :], -1, -2))
    return out


def single_link(L, theta, site=(0, 0, 0, 0), mu=0):
    """All links 1 except U_mu(site) = exp(i theta lambda_3 / 2) = diag(e^{i th/2}, e^{-i th/2}, 1)."""
    U = unit_field(L)
    x0, x1, x2, x3 = site
    U[x3, x2, x1, x0, mu] = np.diag([np.exp(0.5j * theta), np.exp(-0.5j * theta), 1.0])
    return U


H3 = np.diag([1.0, -1.0, 0.0])


def abelian_flux(U, a, b, m):
    """Multiply in a constant abelian field of flux f = 2 pi m/(L_a L_b) per plaquette of plane (a, b).

    U_b(n) *= exp(i f x_a H), and at x_a = L_a - 1 also U_a(n) *= exp(-i f L_a x_b H), H = diag(1,-1,0).
    Every plaquette P_ab then equals exp(i f H); all other planes are unchanged.
    """
    L3, L2, L1, L0 = U.shape[:4]
    Lx = (L0, L1, L2, L3)
    f = 2.0 * math.pi * m / (Lx[a] * Lx[b])
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0), indexing="ij")
    x = [x0, x1, x2, x3]
    ph_b = np.exp(1j * f * x[a][..., None] * np.diag(H3)[None, :])
    out = U.copy()
    out[..., b, :, :] = out[..., b, :, :] * ph_b[..., None, :]  # right-multiply by a diagonal
    wrap = x[a] == Lx[a] - 1
    ph_a = np.exp(-1j * f * Lx[a] * x[b][..., None] * np.diag(H3)[None, :])
    ua = out[..., a, :, :]
    ua[wrap] = ua[wrap] * ph_a[wrap][:, None, :]
    out[..., a, :, :] = ua
    return out, f
