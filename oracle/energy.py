"""Discrete energies and norms of Sec. 3 and App. A, in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (App. A): for cell-centred f, g the plain inner product is
(f||g) = sum_ij f_ij g_ij and the norms carry the cell area, ||f||_p^p = h^2 sum |f|^p.
||grad_h f||_2^2 = h^2 (sum over east-west edges of (D_x f)^2 + sum over north-south
edges of (D_y f)^2); with periodic boundaries there are m x n edges of each kind.

Every function takes ny_neumann: False for periodic boundaries (A.8)-(A.9); True for
periodic in x and homogeneous Neumann in y (A.7), Sec. 4.5, where a ghost row holds
the boundary row's value, so the n-1 interior north-south edges carry differences and
the two boundary edges carry none.

Pins (tests/test_oracle.py, tests/test_oracle_neumann.py): Green's identity
||grad_h f||^2 = -h^2 (f||Delta_h f), the spectral inverse Laplacian against a dense
linear solve, and the exact discrete energy identities of both schemes, for both
boundary rules.
"""
from __future__ import annotations

import numpy as np


def lap(f, h, ny_neumann=False):
    """Five-point Delta_h (App. A); arrays are (n, m)."""
    south, north = np.roll(f, 1, 0), np.roll(f, -1, 0)
    if ny_neumann:                       # ghost rows = boundary rows (A.7)
        south[0], north[-1] = f[0], f[-1]
    return (south + north + np.roll(f, 1, 1) + np.roll(f, -1, 1) - 4.0 * f) / (h * h)


def grad_sq(f, h, ny_neumann=False):
    """||grad_h f||_2^2: h^2 * sum of squared edge differences / h^2 (App. A)."""
    dx = np.roll(f, -1, 1) - f
    dy = np.diff(f, axis=0) if ny_neumann else np.roll(f, -1, 0) - f
    return float(np.sum(dx * dx) + np.sum(dy * dy))


def _dct_matrix(n):
    """Orthonormal cosine basis of the cell-centred Neumann grid: row q is
    cos(pi q (j + 1/2) / n), j = 0..n-1, scaled to unit length."""
    j = np.arange(n)
    C = np.cos(np.pi * np.arange(n)[:, None] * (j[None, :] + 0.5) / n) * np.sqrt(2.0 / n)
    C[0] /= np.sqrt(2.0)
    return C


def inv_neg_lap(f, h, ny_neumann=False):
    """xi with -Delta_h xi = f and xi of mean zero (App. A, (A.16)), for mean-zero f.
    Solved exactly in the eigenbasis of the five-point operator: Fourier modes in
    periodic directions, lambda = (4/h^2) sin^2(pi p/m); with ny_neumann the cosine
    modes cos(pi q (j + 1/2)/n) in y, lambda = (4/h^2) sin^2(pi q/(2n)) (each is an
    exact eigenvector of Delta_h under the ghost rule (A.7)); periodic y otherwise,
    lambda = (4/h^2) sin^2(pi q/n)."""
    n, m = f.shape
    p = np.arange(m)
    q = np.arange(n)
    sy = np.sin(np.pi * q / (2 * n)) if ny_neumann else np.sin(np.pi * q / n)
    lam = (4.0 / h**2) * (np.sin(np.pi * p / m)[None, :] ** 2 + sy[:, None] ** 2)
    lam[0, 0] = 1.0
    fx = np.fft.fft(f, axis=1)
    if ny_neumann:
        C = _dct_matrix(n)
        xh = (C @ fx) / lam
        xh[0, 0] = 0.0
        return np.real(np.fft.ifft(C.T @ xh, axis=1))
    xh = np.fft.fft(fx, axis=0) / lam
    xh[0, 0] = 0.0
    return np.real(np.fft.ifft2(xh))


def norm_m1_sq(f, h, ny_neumann=False):
    """||f||_{-1}^2 = h^2 (f || -Delta_h^{-1} f) for mean-zero f (App. A, (A.17)-(A.18))."""
    return float(h * h * np.sum(f * inv_neg_lap(f - f.mean(), h, ny_neumann)))


def F(phi, h, eps, ny_neumann=False):
    """Discrete energy F(phi), Sec. 3, (3.1):
    1/4 ||phi||_4^4 + alpha/2 ||phi||_2^2 - ||grad_h phi||_2^2 + 1/2 ||Delta_h phi||_2^2."""
    alpha = 1.0 - eps
    h2 = h * h
    L = lap(phi, h, ny_neumann)
    return float(0.25 * h2 * np.sum(phi**4) + 0.5 * alpha * h2 * np.sum(phi**2) - grad_sq(phi, h, ny_neumann)
                 + 0.5 * h2 * np.sum(L * L))


def pseudo_F(phi, psi, h, eps, M, ny_neumann=False):
    """Pseudo energy script-F(phi, psi) = F(phi) + 1/(2M) ||psi||_{-1}^2, Sec. 3, (3.2)."""
    return F(phi, h, eps, ny_neumann) + norm_m1_sq(psi, h, ny_neumann) / (2.0 * M)


def tilde_F(phi, phi_prev, psi, h, eps, M, ny_neumann=False):
    """Second-order energy tilde-F = script-F(phi, psi) + 1/2 ||grad_h(phi - phi_prev)||^2, Sec. 3.4, (3.26)."""
    return pseudo_F(phi, psi, h, eps, M, ny_neumann) + 0.5 * grad_sq(phi - phi_prev, h, ny_neumann)


def mass(phi, h):
    """h^2 (phi || 1), the conserved quantity of Sec. 3.3."""
    return float(h * h * np.sum(phi))


def pin_energy(phi, W, phihat, h):
    """Pinning energy h^2 sum W (phi - phihat)^2, the discrete form of the term added
    to E in Sec. 4.6."""
    return float(h * h * np.sum(W * (phi - phihat) ** 2))


def scheme2_identity_terms(phi_new, phi_k, phi_km1, psi_new, psi_k, h, eps, M, beta, s, ny_neumann=False,
                           W=None, phihat=None):
    """Both sides of the exact energy identity of Sec. 3.4, (3.28):
    tildeF^{k+1} + s beta/M ||psi^{k+1/2}||_{-1}^2 + s^4/2 ||grad_h D_s^2 phi^k||^2 = tildeF^k.
    Returns (lhs, rhs)."""
    nn = ny_neumann
    tf_new = tilde_F(phi_new, phi_k, psi_new, h, eps, M, nn)
    tf_old = tilde_F(phi_k, phi_km1, psi_k, h, eps, M, nn)
    psi_half = 0.5 * (psi_new + psi_k)
    diss = s * beta / M * norm_m1_sq(psi_half, h, nn) + 0.5 * grad_sq(phi_new - 2.0 * phi_k + phi_km1, h, nn)
    if W is not None:   # the pinned energy: the midpoint form makes its change exact (difference of squares)
        tf_new += pin_energy(phi_new, W, phihat, h)
        tf_old += pin_energy(phi_k, W, phihat, h)
    return tf_new + diss, tf_old


def scheme1_identity_terms(phi_new, phi_k, psi_new, psi_k, h, eps, M, beta, s, ny_neumann=False):
    """Both sides of the exact form of the first-order stability estimate (Sec. 3.4,
    first theorem), obtained by keeping every term of the convex-splitting argument:
    F^{k+1} + G4 + alpha/2 ||d||^2 + 1/2 ||Delta_h d||^2 + ||grad_h d||^2
      + s beta/M ||psi^{k+1}||_{-1}^2 + 1/(2M) ||psi^{k+1} - psi^k||_{-1}^2 = F^k (pseudo energies),
    with d = phi^{k+1} - phi^k and G4 = h^2 sum[(a-b) a^3 - (a^4-b^4)/4] >= 0.
    Returns (lhs, rhs)."""
    alpha = 1.0 - eps
    h2 = h * h
    a, b = phi_new, phi_k
    d = a - b
    G4 = h2 * float(np.sum(d * a**3 - 0.25 * (a**4 - b**4)))
    nn = ny_neumann
    Ld = lap(d, h, nn)
    diss = (G4 + 0.5 * alpha * h2 * float(np.sum(d * d)) + 0.5 * h2 * float(np.sum(Ld * Ld)) + grad_sq(d, h, nn)
            + s * beta / M * norm_m1_sq(psi_new, h, nn) + norm_m1_sq(psi_new - psi_k, h, nn) / (2.0 * M))
    return pseudo_F(a, psi_new, h, eps, M, nn) + diss, pseudo_F(b, psi_k, h, eps, M, nn)


def pfc_scheme1_identity_terms(phi_new, phi_k, h, eps, M, s, ny_neumann=False):
    """Exact energy balance of the first-order convex-splitting scheme of the PFC
    equation (1): with d = phi^{k+1} - phi^k = s M Delta_h mu,
      F^{k+1} + G4 + alpha/2 ||d||^2 + 1/2 ||Delta_h d||^2 + ||grad_h d||^2
        + ||d||_{-1}^2 / (s M) = F^k,
    the MPFC balance of scheme 1 without the inertial terms (G4 as there).
    Returns (lhs, rhs)."""
    alpha = 1.0 - eps
    h2 = h * h
    a, b = phi_new, phi_k
    d = a - b
    G4 = h2 * float(np.sum(d * a**3 - 0.25 * (a**4 - b**4)))
    Ld = lap(d, h, ny_neumann)
    diss = (G4 + 0.5 * alpha * h2 * float(np.sum(d * d)) + 0.5 * h2 * float(np.sum(Ld * Ld))
            + grad_sq(d, h, ny_neumann) + norm_m1_sq(d, h, ny_neumann) / (s * M))
    return F(a, h, eps, ny_neumann) + diss, F(b, h, eps, ny_neumann)


def pfc_scheme2_identity_terms(phi_new, phi_k, phi_km1, h, eps, M, s, ny_neumann=False):
    """Exact energy balance of the second-order scheme for the PFC equation (1), the
    analogue of (3.28) without the inertial terms: with
    tildeF(phi, phi_prev) = F(phi) + 1/2 ||grad_h(phi - phi_prev)||^2 and
    d = phi^{k+1} - phi^k = s M Delta_h mu^{k+1/2},
      tildeF^{k+1} + ||d||_{-1}^2 / (s M) + 1/2 ||grad_h(phi^{k+1} - 2 phi^k + phi^{k-1})||^2 = tildeF^k.
    Returns (lhs, rhs)."""
    nn = ny_neumann
    d = phi_new - phi_k
    t_new = F(phi_new, h, eps, nn) + 0.5 * grad_sq(phi_new - phi_k, h, nn)
    t_old = F(phi_k, h, eps, nn) + 0.5 * grad_sq(phi_k - phi_km1, h, nn)
    diss = norm_m1_sq(d, h, nn) / (s * M) + 0.5 * grad_sq(phi_new - 2.0 * phi_k + phi_km1, h, nn)
    return t_new + diss, t_old
