"""Pin of whole time steps of the oracle by the single-Fourier-mode closed form.

About a constant state phibar, a grid function phibar + a e, with e an eigenvector of
Delta_h (eigenvalue lam < 0), stays of that form under both schemes up to terms of order
a^3: the cubic's quadratic part feeds only the mean and the doubled mode, and those come
back into e at third order.  The mode's amplitude then follows a scalar linear recurrence
written here directly from the schemes' equations (Sec. 3.1: the first-order scheme with psi
eliminated; Sec. 3.2: the second-order scheme, chi(phi, phi^k) phi^{k+1/2} linearised about
phibar; the PFC special case of Sec. 1 with the same chemical potentials).  The oracle reaches
the same amplitudes by sources, the three-field operator, FAS V-cycles and the psi update,
so a dropped term, a wrong sign or a wrong coefficient in any of them moves the amplitude by
far more than the tolerance used here.
"""
import math

import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs

AMP = 1e-5          # mode amplitude: the neglected cubic terms are ~AMP^2 relative
RTOL = 1e-9          # bound on |a_oracle - a_closed| / max|a| over the steps (seen: 2e-10)


def _mode(m, n, h, p_, q_, neumann):
    """A real eigenvector of Delta_h and its eigenvalue: cos in x (periodic); in y cos of
    the periodic kind, or cos(pi q y / L_y) under the Neumann ghost rule (A.7)."""
    X, Y = inputs.cell_centres(m, n, h)
    if neumann:
        e = np.cos(2 * np.pi * p_ * X / (m * h) + 0.4) * np.cos(np.pi * q_ * Y / (n * h))
        lam = -4.0 / h ** 2 * (math.sin(math.pi * p_ / m) ** 2 + math.sin(math.pi * q_ / (2 * n)) ** 2)
    else:
        e = np.cos(2 * np.pi * (p_ * X / (m * h) + q_ * Y / (n * h)) + 0.4)
        lam = -4.0 / h ** 2 * (math.sin(math.pi * p_ / m) ** 2 + math.sin(math.pi * q_ / n) ** 2)
    return e, lam


def _closed_form(scheme, model, P, phibar, lam, a_prev, a0, b0, steps):
    """Mode amplitudes (a^k, psi amplitude b^k) for k = 1..steps, from the schemes:

    first order (Sec. 3.1): a1 - a0 = c1 lam mu1 + b0 / (beta + 1/s),
        mu1 = (3 phibar^2 + alpha + lam^2) a1 + 2 lam a0,  b1 = (a1 - a0) / s;
    second order (Sec. 3.2): a1 - a0 = c2 lam mu + 2 b0 / (beta + 2/s),
        mu = (3/2 phibar^2 + alpha/2 + lam^2/2)(a1 + a0) + lam (3 a0 - a_prev),
        b1 = (2/s)(a1 - a0) - b0;
    PFC (Sec. 1, d_t phi = M Delta mu): the same mu, a1 - a0 = s M lam mu, no psi.
    c1 = sM/(beta + 1/s), c2 = sM/(beta + 2/s), alpha = 1 - eps.
    """
    alpha = 1.0 - P.eps
    s, M, beta = P.s, P.M, P.beta
    out = []
    for _ in range(steps):
        if scheme == 1:
            c = s * M if model == 1 else s * M / (beta + 1.0 / s)
            forcing = 0.0 if model == 1 else b0 / (beta + 1.0 / s)
            # a1 (1 - c lam (3 phibar^2 + alpha + lam^2)) = a0 + c lam 2 lam a0 + forcing
            a1 = (a0 * (1.0 + 2.0 * c * lam * lam) + forcing) / (1.0 - c * lam * (3 * phibar ** 2 + alpha + lam * lam))
            b1 = (a1 - a0) / s
        else:
            c = s * M if model == 1 else s * M / (beta + 2.0 / s)
            forcing = 0.0 if model == 1 else 2.0 * b0 / (beta + 2.0 / s)
            k = 1.5 * phibar ** 2 + 0.5 * alpha + 0.5 * lam * lam
            # a1 - a0 = c lam (k (a1 + a0) + lam (3 a0 - a_prev)) + forcing
            a1 = (a0 + c * lam * (k * a0 + lam * (3 * a0 - a_prev)) + forcing) / (1.0 - c * lam * k)
            b1 = 2.0 / s * (a1 - a0) - b0
        if model == 1:
            b1 = None
        out.append((a1, b1))
        a_prev, a0, b0 = a0, a1, (b1 if b1 is not None else 0.0)
    return out


def _amp(f, phibar, e):
    return float(np.sum((f - phibar) * e) / np.sum(e * e))


CASES = [
    # scheme, model, neumann, m, n, h, p, q, phibar, s
    (1, 0, False, 16, 16, 0.5, 1, 2, 0.07, 0.01),
    (2, 0, False, 16, 16, 0.5, 1, 2, 0.07, 0.01),
    (1, 0, False, 32, 16, 0.9, 3, 1, -0.285, 0.5),
    (2, 0, False, 32, 16, 0.9, 3, 1, -0.285, 0.5),
    (2, 0, False, 16, 32, 0.7, 2, 5, 0.2, 5.0),
    (1, 1, False, 16, 16, 0.5, 2, 1, 0.07, 0.01),
    (2, 1, False, 16, 16, 0.5, 2, 1, 0.07, 0.1),
    (1, 0, True, 16, 16, 0.6, 1, 3, 0.1, 0.05),
    (2, 0, True, 16, 16, 0.6, 1, 3, 0.1, 0.05),
]


@pytest.mark.parametrize("scheme,model,neumann,m,n,h,p_,q_,phibar,s", CASES)
def test_single_mode_steps_follow_the_linear_recurrence(oracle_mod, scheme, model, neumann, m, n, h, p_, q_,
                                                        phibar, s):
    P = oracle_mod.Params(m=m, n=n, h=h, s=s, ny_neumann=int(neumann), model=model)
    e, lam = _mode(m, n, h, p_, q_, neumann)
    # distinct history amplitudes, so the extrapolated phi~ and the psi^k forcing both act
    a_prev, a0 = 0.7 * AMP, AMP
    b0 = 0.0 if model == 1 else 0.3 * AMP / s
    sol = oracle_mod.Solver(P)
    sol.set_state(phibar + a0 * e, phibar + a_prev * e, None if model == 1 else b0 * e)
    steps = 3
    want = _closed_form(scheme, model, P, phibar, lam, a_prev, a0, b0, steps)
    scale = max(abs(a) for a, _ in want + [(a0, None)])
    for k in range(steps):
        r = sol.step(scheme, tol=1e-15, max_cycles=60)
        assert r["status"] == 0, r
        phi, _, psi = sol.get_state()
        a_got = _amp(phi, phibar, e)
        a_want, b_want = want[k]
        assert abs(a_got - a_want) <= RTOL * scale, (k, a_got, a_want)
        # the rest of phi is the constant phibar up to second order in the amplitude
        assert np.max(np.abs(phi - phibar - a_got * e)) <= 10 * AMP * AMP + 1e-13
        if b_want is not None:
            b_got = _amp(psi, 0.0, e)
            # psi^{k+1} is a difference quotient of phi: its error is that of a over s, times 2
            assert abs(b_got - b_want) <= 2.0 * RTOL * scale / s, (k, b_got, b_want)


def test_the_recurrence_separates_the_schemes(oracle_mod):
    """The closed forms differ by much more than the tolerance between schemes, models and
    with a wrong neighbour coefficient, so the pin above can tell them apart."""
    P = oracle_mod.Params(m=16, n=16, h=0.5, s=0.01)
    _, lam = _mode(16, 16, 0.5, 1, 2, False)
    base = _closed_form(1, 0, P, 0.07, lam, 0.7 * AMP, AMP, 0.3 * AMP / P.s, 3)
    other = [_closed_form(2, 0, P, 0.07, lam, 0.7 * AMP, AMP, 0.3 * AMP / P.s, 3),
             _closed_form(1, 1, P, 0.07, lam, 0.7 * AMP, AMP, 0.3 * AMP / P.s, 3),
             _closed_form(1, 0, P, 0.07, lam, 0.7 * AMP, AMP, 0.0, 3)]
    P4 = oracle_mod.Params(m=16, n=16, h=0.5, s=0.01, M=4.0)   # the 4 sM/(h^2 (beta + 2/s)) misprint's size
    other.append(_closed_form(1, 0, P4, 0.07, lam, 0.7 * AMP, AMP, 0.3 * AMP / P.s, 3))
    for o in other:
        assert max(abs(x[0] - y[0]) for x, y in zip(base, o)) > 1e3 * RTOL * AMP
