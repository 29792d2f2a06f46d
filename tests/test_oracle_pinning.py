"""Pins of the oracle's pinning term (Sec. 4.6): the second-order scheme with the
pinned potential mu~ = mu + 2 (phi^{k+1/2} - phihat) W.

References: the special case of a constant weight and target, which must reproduce
the unpinned scheme with alpha -> alpha + 2 W (tests/test_oracle.py pins that one);
the exact energy identity (3.28) with the pinning energy added (its change is exact,
a difference of squares, because the term is taken at the midpoint); an
independently written dense Newton solve; and the smoother's local equations.
"""
import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs


def _strips(m, n, w0, width):
    """Weight w0 in horizontal strips of `width` rows at the top and bottom, 0 between
    (the shape of the pinning weight of Sec. 4.6)."""
    W = np.zeros((n, m))
    W[:width] = w0
    W[-width:] = w0
    return W


def _crystal(m, n, h, phis, eps, shift=0.0):
    return inputs.one_mode_crystal(m, n, h, phis, eps, shift)


def test_constant_pinning_is_a_shift_of_alpha(oracle_mod):
    """W = w0 and phihat = c0 everywhere: phi follows the unpinned scheme with
    eps' = eps - 2 w0, and mu~ = mu' - 2 w0 c0 (Sec. 4.6 with Sec. 3.2)."""
    m, h, s, eps, w0, c0 = 32, 0.5, 0.05, 0.3, 0.07, 0.2
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 3)
    a = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, eps=eps))
    a.set_pinning(np.full((m, m), w0), np.full((m, m), c0))
    b = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, eps=eps - 2 * w0))
    a.set_state(phi0)
    b.set_state(phi0)
    for k in range(4):
        ra = a.step(2, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
        rb = b.step(2, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
        assert ra["status"] == 0 and rb["status"] == 0
        np.testing.assert_allclose(a.get_state()[0], b.get_state()[0], atol=1e-11)
        ua, ub = a.get_u(), b.get_u()
        np.testing.assert_allclose(ua[1], ub[1] - 2 * w0 * c0, atol=1e-10)
    # and the weight does change the dynamics compared with no pinning
    c = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, eps=eps))
    c.set_state(phi0)
    for k in range(4):
        c.step(2, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
    assert np.abs(c.get_state()[0] - a.get_state()[0]).max() > 1e-6


@pytest.mark.parametrize("s", [0.01, 0.1, 1.0])
def test_pinned_energy_identity(oracle_mod, s):
    """(3.28) with the pinning energy h^2 sum W (phi - phihat)^2 added to tildeF holds
    exactly for the discrete solution, with a weight that varies in space."""
    from oracle import energy
    m, n, h, eps = 32, 32, 1.0, 0.6
    p = oracle_mod.Params(m=m, n=n, h=h, s=s, beta=0.2, eps=eps, M=2.0)
    W = _strips(m, n, 2.0, 4)
    phihat = _crystal(m, n, h, 0.395, eps, shift=0.3)
    sol = oracle_mod.Solver(p)
    sol.set_pinning(W, phihat)
    sol.set_state(_crystal(m, n, h, 0.395, eps) + 0.01 * inputs.noise_field(m, n, 0, 1, 4))
    for k in range(4):
        phi_k, phi_km1, psi_k = sol.get_state()
        r = sol.step(2, tol=1e-12, guess=oracle_mod.GUESS_EXTRAP)
        assert r["status"] == 0
        phi_n, _, psi_n = sol.get_state()
        lhs, rhs = energy.scheme2_identity_terms(phi_n, phi_k, phi_km1, psi_n, psi_k, h, p.eps, p.M, p.beta, s,
                                                 W=W, phihat=phihat)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs), (k, lhs, rhs)
        # without the pinning energy the balance is off
        l0, r0 = energy.scheme2_identity_terms(phi_n, phi_k, phi_km1, psi_n, psi_k, h, p.eps, p.M, p.beta, s)
        assert abs(l0 - r0) > 1e-7 * abs(r0)


@pytest.mark.parametrize("s", [0.05, 2.0])
def test_vcycle_equals_dense_newton_pinned(oracle_mod, s):
    from oracle import bruteforce
    m = 8
    p = oracle_mod.Params(m=m, n=m, h=0.5, s=s)
    consts = oracle_mod.scheme_consts(p, 2)
    phik = inputs.noise_field(m, m, 0.07, 0.05, 21)
    psik = inputs.noise_field(m, m, 0.0, 0.01, 22)
    psik -= psik.mean()
    W = _strips(m, m, 2.0, 2)
    phihat = inputs.noise_field(m, m, 0.1, 0.1, 23)
    S = oracle_mod.source(2, p, phik, phik, psik, W=W, phihat=phihat)
    sol = oracle_mod.Solver(p)
    sol.set_pinning(W, phihat)
    (phi, mu, ka), cyc, res, _ = sol.solve(2, (phik, np.zeros_like(phik), np.zeros_like(phik)), S, phik=phik,
                                          tol=1e-13)
    assert res <= 1e-13
    (bphi, bmu, bka), bres = bruteforce.newton_solve(2, consts, p.h, S, phik=phik, W=W)
    assert bres < 1e-12
    for a, b in ((phi, bphi), (mu, bmu), (ka, bka)):
        np.testing.assert_allclose(a, b, atol=1e-10 * max(np.abs(b).max(), 1.0))


def test_smoother_local_equations_pinned(oracle_mod):
    """After a red-black sweep with omega = 1, every black cell satisfies rows 1 and 3
    exactly and row 2 up to the linearisation error of the cubic, with the pinning
    weight in row 2."""
    m = 16
    p = oracle_mod.Params(m=m, n=m, h=0.5, s=0.3, omega=1.0)
    consts = oracle_mod.scheme_consts(p, 2)
    phik = inputs.noise_field(m, m, 0.07, 0.05, 5)
    psik = inputs.noise_field(m, m, 0.0, 0.01, 6)
    psik -= psik.mean()
    W = _strips(m, m, 2.0, 3) + 0.5
    phihat = inputs.noise_field(m, m, 0.1, 0.1, 7)
    S = oracle_mod.source(2, p, phik, phik, psik, W=W, phihat=phihat)
    rng = np.random.default_rng(9)
    u0 = [phik + 0.01 * rng.uniform(-1, 1, (m, m)), rng.normal(size=(m, m)), rng.normal(size=(m, m))]
    u1 = oracle_mod.smooth(2, consts, p.h, u0, S, phik=phik, sweeps=1, omega=1.0, W=W)
    r = oracle_mod.residual(2, consts, p.h, u1, S, phik=phik, W=W)
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    black = (ii + jj) % 2 == 1
    assert np.abs(r[0][black]).max() < 1e-13 * max(np.abs(S[0]).max(), 1.0)
    assert np.abs(r[2][black]).max() < 1e-12 * (np.abs(S[2]).max() + np.abs(u1[2]).max())
    # row 2: r2 = g(phi_new) - [g(p) + g'(p)(phi_new - p)] with p the value before the visit
    p0, pn = u0[0], u1[0]
    g = lambda x: 0.25 * (x ** 2 + phik ** 2) * (x + phik)
    dg = lambda x: 0.25 * (3 * x ** 2 + 2 * x * phik + phik ** 2)
    lin_err = g(pn) - (g(p0) + dg(p0) * (pn - p0))
    np.testing.assert_allclose(r[1][black], lin_err[black], atol=1e-12)


def test_scheme1_with_pinning_is_refused(oracle_mod):
    m = 16
    sol = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=0.5, s=0.1))
    sol.set_pinning(np.ones((m, m)), np.zeros((m, m)))
    sol.set_state(inputs.noise_field(m, m, 0.07, 0.05, 1))
    assert sol.step(1)["rc"] != 0
    assert sol.step(2)["rc"] == 0
