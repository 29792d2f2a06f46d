"""The CUDA path against the single-Fourier-mode closed form of the schemes (Sec. 3.1,
3.2 and the PFC case of Sec. 1), with no oracle in between: a small eigenmode of Delta_h
about a constant state, stepped by the FP64 and the FP32-inner solvers, keeps the amplitude
that the scalar linear recurrence of tests/test_oracle_modes.py gives, for both schemes,
periodic and Neumann-in-y grids.  Solved to a scaled residual of 3e-15, the amplitude's
error is the neglected cubic order (~1e-10 relative at amplitude 1e-5) plus ~3e-10 from the
tolerance."""
import numpy as np
import pytest

from test_oracle_modes import AMP, _amp, _closed_form, _mode

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL_GPU = 2e-9


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import mpfc
    mpfc.load()
    return mpfc


class _P:
    """The parameters the closed form reads."""

    def __init__(self, s, M=1.0, beta=0.9, eps=0.025):
        self.s, self.M, self.beta, self.eps = s, M, beta, eps


CASES = [
    # scheme, model, neumann, m, n, h, p, q, phibar, s
    (1, 0, False, 64, 64, 0.5, 1, 2, 0.07, 0.01),
    (2, 0, False, 96, 160, 0.7, 3, 2, -0.285, 0.5),
    (2, 1, False, 64, 64, 0.5, 2, 1, 0.07, 0.1),
    (1, 0, True, 64, 96, 0.6, 1, 3, 0.1, 0.05),
    (2, 0, True, 64, 96, 0.6, 1, 3, 0.1, 0.05),
    (1, 0, False, 128, 64, 0.5, 5, 3, 0.07, 2.0),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32_inner"])
@pytest.mark.parametrize("scheme,model,neumann,m,n,h,p_,q_,phibar,s", CASES)
def test_single_mode_steps_on_the_gpu(mp, precision, scheme, model, neumann, m, n, h, p_, q_, phibar, s):
    prm = mp.default_params(m=m, n=n, h=h, dt=s, M=1.0, beta=0.9, epsilon=0.025, tol=3e-15, max_cycles=100,
                            model=mp.MPFC_MODEL_PFC if model else mp.MPFC_MODEL_MPFC,
                            bc=mp.MPFC_BC_NEUMANN_Y if neumann else mp.MPFC_BC_PERIODIC,
                            precision=mp.MPFC_FP32_INNER if precision == "fp32_inner" else mp.MPFC_FP64)
    e, lam = _mode(m, n, h, p_, q_, neumann)
    a_prev, a0 = 0.7 * AMP, AMP
    b0 = 0.0 if model == 1 else 0.3 * AMP / s
    g = mp.Solver(prm)
    g.set_state(phibar + a0 * e, phibar + a_prev * e, None if model == 1 else b0 * e)
    steps = 3
    want = _closed_form(scheme, model, _P(s), phibar, lam, a_prev, a0, b0, steps)
    scale = max(abs(a) for a, _ in want + [(a0, None)])
    for k in range(steps):
        info = g.step(scheme, 1)[0]
        assert info["status"] == 0 and info["res"] <= 3e-15, (k, info)
        phi, _, psi = g.get_state()
        a_got = _amp(phi, phibar, e)
        a_want, b_want = want[k]
        assert abs(a_got - a_want) <= RTOL_GPU * scale, (k, a_got, a_want)
        assert np.max(np.abs(phi - phibar - a_got * e)) <= 10 * AMP * AMP + 1e-13
        if b_want is not None:
            assert abs(_amp(psi, 0.0, e) - b_want) <= 2.0 * RTOL_GPU * scale / s, k
