"""Pins of the oracle's PFC variant: d_t phi = M Delta mu, the purely parabolic
special case of the MPFC equation (Sec. 1, (1)), solved by the same convex-splitting
schemes and FAS machinery (row 1 of N becomes phi - s M Delta_h mu, S1 = phi^k).

References: exact discrete energy balances of both schemes (the MPFC ones of Sec. 3.4
with the inertial terms removed), the overdamped limit of the MPFC schemes (beta ->
infinity with M / beta fixed), a dense Newton solve, mass conservation, and the time
order under step halving.
"""
import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs


def _solver(oracle_mod, m, h, s, **kw):
    return oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, model=1, **kw))


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("s", [0.01, 0.1, 1.0, 10.0])
def test_pfc_exact_energy_balance(oracle_mod, scheme, s):
    from oracle import energy
    m, h, eps, M = 32, 1.0, 0.3, 1.5
    sol = _solver(oracle_mod, m, h, s, eps=eps, M=M)
    sol.set_state(inputs.paper_smooth_field(m, m, h) + 0.02 * inputs.noise_field(m, m, 0, 1, 2))
    for k in range(4):
        phk, phkm1, _ = sol.get_state()
        r = sol.step(scheme, tol=1e-12, guess=oracle_mod.GUESS_EXTRAP)
        assert r["status"] == 0
        phn = sol.get_state()[0]
        if scheme == 1:
            lhs, rhs = energy.pfc_scheme1_identity_terms(phn, phk, h, eps, M, s)
        else:
            lhs, rhs = energy.pfc_scheme2_identity_terms(phn, phk, phkm1, h, eps, M, s)
        assert abs(lhs - rhs) <= 1e-9 * abs(rhs), (k, lhs, rhs)


@pytest.mark.parametrize("scheme", [1, 2])
def test_overdamped_limit_of_mpfc(oracle_mod, scheme):
    """MPFC with damping beta and mobility beta M tends to PFC with mobility M as beta
    grows (the inertial term becomes negligible): the gap shrinks like 1/beta."""
    m, h, s, M = 32, 0.5, 0.05, 1.0
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 5)
    pfc = _solver(oracle_mod, m, h, s, M=M)
    pfc.set_state(phi0)
    for _ in range(3):
        pfc.step(scheme, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
    ref = pfc.get_state()[0]
    gaps = []
    for beta in (1e4, 1e6):
        mp_ = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, beta=beta, M=beta * M))
        mp_.set_state(phi0)
        for _ in range(3):
            mp_.step(scheme, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)
        gaps.append(np.abs(mp_.get_state()[0] - ref).max())
    assert gaps[1] < 1e-6 and gaps[1] < 0.05 * gaps[0], gaps


@pytest.mark.parametrize("scheme,s", [(1, 0.05), (2, 0.05), (2, 5.0)])
def test_pfc_vcycle_equals_dense_newton(oracle_mod, scheme, s):
    from oracle import bruteforce
    m = 8
    p = oracle_mod.Params(m=m, n=m, h=0.5, s=s, model=1)
    consts = oracle_mod.scheme_consts(p, scheme)
    assert abs(consts[0] - s * p.M) < 1e-15          # c = s M for PFC
    phik = inputs.noise_field(m, m, 0.07, 0.05, 21)
    S = oracle_mod.source(scheme, p, phik, phik, inputs.noise_field(m, m, 0, 1, 22))
    np.testing.assert_array_equal(S[0], phik)          # S1 = phi^k: no velocity term
    sol = oracle_mod.Solver(p)
    pk = phik if scheme == 2 else None
    (phi, mu, ka), cyc, res, _ = sol.solve(scheme, (phik, np.zeros_like(phik), np.zeros_like(phik)), S, phik=pk,
                                          tol=1e-13)
    assert res <= 1e-13
    (bphi, bmu, bka), bres = bruteforce.newton_solve(scheme, consts, p.h, S, phik=pk)
    for a, b in ((phi, bphi), (mu, bmu), (ka, bka)):
        np.testing.assert_allclose(a, b, atol=1e-10 * max(np.abs(b).max(), 1.0))


@pytest.mark.parametrize("scheme", [1, 2])
def test_pfc_mass(oracle_mod, scheme):
    from oracle import energy
    m, h = 48, 0.5
    sol = _solver(oracle_mod, m, h, 0.2)
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    sol.set_state(phi0)
    m0 = energy.mass(phi0, h)
    for k in range(6):
        assert sol.step(scheme, tol=1e-12, guess=oracle_mod.GUESS_EXTRAP)["status"] == 0
        assert abs(energy.mass(sol.get_state()[0], h) - m0) <= 1e-9 * (k + 1)


@pytest.mark.parametrize("scheme,order", [(1, 1.0), (2, 2.0)])
def test_pfc_time_order(oracle_mod, scheme, order):
    """Errors against a fine-step reference fall like s^order under step halving."""
    m, h, T = 32, 1.0, 0.8
    phi0 = inputs.paper_smooth_field(m, m, h)

    def run(s):
        sol = _solver(oracle_mod, m, h, s)
        sol.set_state(phi0)
        for _ in range(int(round(T / s))):
            assert sol.step(scheme, tol=1e-13, guess=oracle_mod.GUESS_EXTRAP)["status"] == 0
        return sol.get_state()[0]

    ref = run(T / 256)
    errs = [np.abs(run(T / k) - ref).max() for k in (8, 16, 32)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.25 for r in rates), (errs, rates)
