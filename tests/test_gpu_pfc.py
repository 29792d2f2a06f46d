"""Parity of the CUDA path with the oracle for the PFC variant (Sec. 1, (1):
d_t phi = M Delta mu with the same convex-splitting schemes): FP64 steps in lockstep
at <= 1e-10 relative per step, the FP32-inner form within its bound of 1e-8 of the
oracle solved to 1e-13, a batch that follows its single instances, and the energies."""
import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import mpfc
    mpfc.load()
    return mpfc


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("scheme,m,n,s,steps", [(1, 64, 64, 0.05, 8), (2, 64, 64, 0.05, 8), (2, 96, 160, 1.0, 4),
                                                (1, 128, 64, 2.0, 4)])
def test_pfc_lockstep(mp, oracle_mod, scheme, m, n, s, steps):
    h = 0.5
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 3)
    g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, model=mp.MPFC_MODEL_PFC))
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, model=1))
    o.set_state(phi0)
    for k in range(steps):
        ro = o.step(scheme, tol=1e-10, guess=1)
        assert ro["status"] == 0
        rg = g.step_cycles(scheme, ro["cycles"])
        assert rg["status"] == 0
        pg, _, psig = g.get_state()
        po, _, psio = o.get_state()
        assert relerr(pg, po) <= 1e-10, (k, relerr(pg, po))
        assert np.abs(psig - psio).max() <= 1e-10 * np.abs(po).max() / s


@pytest.mark.parametrize("scheme", [1, 2])
def test_pfc_fp32_inner(mp, oracle_mod, scheme):
    m, h, s = 96, 0.5, 0.2
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 4)
    g = mp.Solver(mp.default_params(m=m, n=m, h=h, dt=s, model=mp.MPFC_MODEL_PFC, precision=mp.MPFC_FP32_INNER))
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s, model=1))
    o.set_state(phi0)
    for k in range(5):
        info = g.step(scheme, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10
        assert o.step(scheme, tol=1e-13, guess=1)["status"] == 0
        assert relerr(g.get_state()[0], o.get_state()[0]) <= 1e-8, k


@pytest.mark.parametrize("scheme", [1, 2])
def test_pfc_batch_follows_singles(mp, scheme):
    mix = [dict(m=64, n=64, epsilon=0.03), dict(m=96, n=160, epsilon=0.08), dict(m=32, n=32, epsilon=0.2)]
    ps = [mp.default_params(h=0.5, dt=0.1, model=mp.MPFC_MODEL_PFC, **kw) for kw in mix]
    b = mp.BatchSolver(ps)
    singles = []
    for i, p in enumerate(ps):
        phi0 = inputs.noise_field(p.m, p.n, 0.05 + 0.01 * i, 0.05, 20 + i)
        b.set_state(i, phi0)
        g = mp.Solver(p)
        g.set_state(phi0)
        singles.append(g)
    for step in range(3):
        rc, st, cy = b.step(scheme, 1)
        assert rc == 0 and all(x == 0 for x in st)
        for i, g in enumerate(singles):
            info = g.step(scheme, 1)[0]
            assert cy[i] == info["cycles"]
            ref = g.get_state()[0]
            assert np.abs(b.get_state(i)[0] - ref).max() <= 1e-12 * np.abs(ref).max()
    # a batch mixing the two models is refused
    ps2 = [ps[0], mp.default_params(h=0.5, dt=0.1, m=64, n=64)]
    assert mp.load().mpfc_batch_workspace_bytes(2, (mp.mpfc_params * 2)(*ps2)) == 0


def test_pfc_energy(mp, oracle_mod):
    from oracle import energy
    m, h, s = 64, 0.5, 0.1
    g = mp.Solver(mp.default_params(m=m, n=m, h=h, dt=s, model=mp.MPFC_MODEL_PFC))
    g.set_state(inputs.noise_field(m, m, 0.07, 0.05, 5))
    g.step(2, 3)
    phi, phip, _ = g.get_state()
    e = g.energy()
    ref_f = energy.F(phi, h, 0.025)
    assert abs(e["F"] - ref_f) < 1e-11 * abs(ref_f)
    assert e["pseudoF"] == e["F"]                       # no kinetic energy in the PFC model
    ref_t = ref_f + 0.5 * energy.grad_sq(phi - phip, h)
    assert abs(e["tildeF"] - ref_t) < 1e-10 * abs(ref_t)
