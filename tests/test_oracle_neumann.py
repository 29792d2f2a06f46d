"""Pins of the oracle's mixed boundary conditions (Sec. 4.5: periodic in x,
homogeneous Neumann in y, ghost rule (A.7) of App. A).

References: closed-form eigenvectors of the Neumann Laplacian, an independently
assembled matrix, a dense Newton solve, Green's identities (whose boundary sums
vanish for Neumann conditions, App. A), the exact energy identity of Sec. 3.4, and
the mirror extension: a problem with the ghost rule (A.7) in y is the periodic
problem on the doubled domain whose data are mirrored about the upper boundary,
restricted to the lower half.  That last pin checks the whole Neumann time step
against the periodic one, which tests/test_oracle.py pins separately.
"""
import math

import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs


def _consistent_u(oracle, scheme, p, S, phi0, phik=None):
    """u0 = (phi0, mu0, kappa0) with N2 = S2, N3 = S3 exactly (current boundary rule)."""
    c, gam, theta = oracle.scheme_consts(p, scheme)
    kap = S[2] + theta * oracle.laplacian(phi0, p.h)
    g = phi0 ** 3 if scheme == 1 else 0.25 * (phi0 ** 2 + phik ** 2) * (phi0 + phik)
    mu = S[1] + g + gam * phi0 + oracle.laplacian(kap, p.h)
    return phi0.copy(), mu, kap


def _mirror(f):
    """(n, m) -> (2n, m): rows 0..n-1 as given, then the same rows reversed."""
    return np.concatenate([f, f[::-1]], axis=0)


@pytest.mark.parametrize("m,n,p_,q_", [(16, 16, 1, 0), (16, 8, 3, 2), (8, 12, 0, 5), (8, 8, 4, 7)])
def test_cosine_modes_are_eigenvectors(oracle_mod, m, n, p_, q_):
    """cos(2 pi p x / L_x) cos(pi q y / L_y) is an eigenvector of Delta_h under (A.7)
    with eigenvalue -(4/h^2)(sin^2(pi p/m) + sin^2(pi q/(2n)))."""
    h = 0.37
    X, Y = inputs.cell_centres(m, n, h)
    f = np.cos(2 * np.pi * p_ * X / (m * h) + 0.3) * np.cos(np.pi * q_ * Y / (n * h))
    lam = 4.0 / h ** 2 * (math.sin(math.pi * p_ / m) ** 2 + math.sin(math.pi * q_ / (2 * n)) ** 2)
    with oracle_mod.boundary(True):
        lf = oracle_mod.laplacian(f, h)
    np.testing.assert_allclose(lf, -lam * f, atol=1e-12 * max(lam, 1.0))


def test_laplacian_three_ways_symmetric_and_constant_kernel(oracle_mod):
    """The C oracle's stencil, the assembled matrix of bruteforce.py and energy.lap
    agree; the matrix is symmetric and annihilates constants."""
    from oracle import bruteforce, energy
    m, n, h = 12, 10, 0.6
    f = inputs.noise_field(m, n, 0.1, 0.3, 17)
    L = bruteforce.lap_matrix(m, n, h, ny_neumann=True)
    with oracle_mod.boundary(True):
        a = oracle_mod.laplacian(f, h)
    np.testing.assert_allclose(a.ravel(), L @ f.ravel(), atol=1e-12)
    np.testing.assert_allclose(energy.lap(f, h, ny_neumann=True), a, atol=1e-12)
    np.testing.assert_allclose(L, L.T, atol=0)
    np.testing.assert_allclose(L @ np.ones(m * n), 0.0, atol=1e-12)
    # and it is not the periodic operator
    assert np.abs(L - bruteforce.lap_matrix(m, n, h)).max() > 1.0


def test_green_identities_neumann(oracle_mod):
    """Green's first and second identities with vanishing boundary sums (App. A)."""
    from oracle import energy
    h = 0.5
    f = inputs.noise_field(24, 16, 0.1, 0.3, 7)
    g = inputs.noise_field(24, 16, -0.2, 0.5, 8)
    with oracle_mod.boundary(True):
        lf, lg = oracle_mod.laplacian(f, h), oracle_mod.laplacian(g, h)
    lhs = energy.grad_sq(f, h, ny_neumann=True)
    rhs = -h * h * float(np.sum(f * lf))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert abs(float(np.sum(f * lg)) - float(np.sum(lf * g))) <= 1e-12 * float(np.sum(np.abs(f * lg)))


def test_inverse_laplacian_neumann_vs_dense(oracle_mod):
    """The '-1' norm's Poisson solve with the cosine basis against a dense solve."""
    from oracle import bruteforce, energy
    m, n, h = 8, 12, 0.7
    f = inputs.noise_field(m, n, 0.0, 1.0, 3)
    f -= f.mean()
    xi = energy.inv_neg_lap(f, h, ny_neumann=True)
    L = bruteforce.lap_matrix(m, n, h, ny_neumann=True)
    xd, *_ = np.linalg.lstsq(-L, f.ravel(), rcond=None)
    xd -= xd.mean()
    np.testing.assert_allclose(xi.ravel(), xd, atol=1e-12)
    with oracle_mod.boundary(True):
        np.testing.assert_allclose(-oracle_mod.laplacian(xi, h), f, atol=1e-12)


@pytest.mark.parametrize("scheme", [1, 2])
def test_smoother_local_equations_neumann(oracle_mod, scheme):
    """After a red-black sweep with omega = 1, every black cell, boundary rows
    included, satisfies rows 1 and 3 of its cell system exactly under (A.7): the
    ghost of a boundary cell is its own new value."""
    m = 16
    p = oracle_mod.Params(m=m, n=m, h=0.5, s=0.3, omega=1.0)
    consts = oracle_mod.scheme_consts(p, scheme)
    phik = inputs.noise_field(m, m, 0.07, 0.05, 5)
    psik = inputs.noise_field(m, m, 0.0, 0.01, 6)
    psik -= psik.mean()
    pk = phik if scheme == 2 else None
    with oracle_mod.boundary(True):
        S = oracle_mod.source(scheme, p, phik, phik, psik)
        u0 = _consistent_u(oracle_mod, scheme, p, S, phik + 0.01 * inputs.noise_field(m, m, 0, 1, 9), phik)
        u1 = oracle_mod.smooth(scheme, consts, p.h, u0, S, phik=pk, sweeps=1, omega=1.0)
        r = oracle_mod.residual(scheme, consts, p.h, u1, S, phik=pk)
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    black = (ii + jj) % 2 == 1
    assert np.abs(r[0][black]).max() < 1e-13 * max(np.abs(S[0]).max(), 1.0)
    assert np.abs(r[2][black]).max() < 1e-12 * (np.abs(S[2]).max() + np.abs(u1[2]).max())
    # the boundary rows hold black cells too
    assert black[0].any() and black[-1].any()


@pytest.mark.parametrize("scheme,s", [(1, 0.01), (1, 1.0), (2, 0.05), (2, 5.0)])
def test_vcycle_equals_dense_newton_neumann(oracle_mod, scheme, s):
    """Unique solvability (Sec. 3.3): the FAS V-cycle and plain Newton on the
    assembled Neumann system reach the same u at 8 x 8."""
    from oracle import bruteforce
    m = 8
    p = oracle_mod.Params(m=m, n=m, h=0.5, s=s, ny_neumann=1)
    consts = oracle_mod.scheme_consts(p, scheme)
    phik = inputs.noise_field(m, m, 0.07, 0.05, 21)
    psik = inputs.noise_field(m, m, 0.0, 0.01, 22)
    psik -= psik.mean()
    pk = phik if scheme == 2 else None
    with oracle_mod.boundary(True):
        S = oracle_mod.source(scheme, p, phik, phik, psik)
    sol = oracle_mod.Solver(p)
    (phi, mu, ka), cyc, res, _ = sol.solve(scheme, (phik, np.zeros_like(phik), np.zeros_like(phik)), S, phik=pk,
                                          tol=1e-13)
    assert res <= 1e-13
    (bphi, bmu, bka), bres = bruteforce.newton_solve(scheme, consts, p.h, S, phik=pk, ny_neumann=True)
    assert bres < 1e-12
    for a, b in ((phi, bphi), (mu, bmu), (ka, bka)):
        np.testing.assert_allclose(a, b, atol=1e-10 * max(np.abs(b).max(), 1.0))


@pytest.mark.parametrize("scheme", [1, 2])
def test_mirror_extension_equals_neumann(oracle_mod, scheme):
    """A Neumann-in-y run on n rows equals the periodic run on 2n rows from the
    mirrored data (rows 0..n-1), step by step, to the solve tolerance; and it
    differs from the periodic run on n rows."""
    m, n, h, s = 16, 16, 0.5, 0.05
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 31)
    neu = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, ny_neumann=1))
    ext = oracle_mod.Solver(oracle_mod.Params(m=m, n=2 * n, h=h, s=s))
    per = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s))
    neu.set_state(phi0)
    ext.set_state(_mirror(phi0))
    per.set_state(phi0)
    for k in range(4):
        for sol in (neu, ext, per):
            r = sol.step(scheme, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
            assert r["status"] == 0
        a = neu.get_state()[0]
        b = ext.get_state()[0]
        np.testing.assert_allclose(a, b[:n], atol=1e-11)
        np.testing.assert_allclose(b[n:], b[:n][::-1], atol=1e-11)   # the extension stays mirrored
    assert np.abs(neu.get_state()[0] - per.get_state()[0]).max() > 1e-5


def test_mass_and_energy_identity_neumann(oracle_mod):
    """No-flux boundaries keep the mass (Sec. 3.3) and the exact energy identity
    (3.28) of scheme 2 holds with the Neumann energies (boundary sums vanish)."""
    from oracle import energy
    m, n, h, s = 32, 24, 1.0, 0.1
    p = oracle_mod.Params(m=m, n=n, h=h, s=s, beta=0.9, ny_neumann=1)
    sol = oracle_mod.Solver(p)
    phi0 = inputs.paper_smooth_field(m, n, h) + 0.02 * inputs.noise_field(m, n, 0, 1, 2)
    sol.set_state(phi0)
    m0 = energy.mass(phi0, h)
    for k in range(4):
        phi_k, phi_km1, psi_k = sol.get_state()
        r = sol.step(2, tol=1e-12, guess=oracle_mod.GUESS_EXTRAP)
        assert r["status"] == 0
        phi_n, _, psi_n = sol.get_state()
        lhs, rhs = energy.scheme2_identity_terms(phi_n, phi_k, phi_km1, psi_n, psi_k, h, p.eps, p.M, p.beta, s,
                                                 ny_neumann=True)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs), (k, lhs, rhs)
        assert abs(energy.mass(phi_n, h) - m0) <= 1e-9 * (k + 1)
