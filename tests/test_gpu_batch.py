"""Batched ensemble: every instance of a mixed batch follows the single-instance
solver (itself in lockstep parity with the oracle) step by step, and a fixed-cycle
batched step matches the oracle directly."""
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


MIX = [dict(m=64, n=64, epsilon=0.03, beta=0.7), dict(m=96, n=160, epsilon=0.08, beta=1.2),
       dict(m=128, n=128, epsilon=0.05, beta=0.9), dict(m=32, n=32, epsilon=0.02, beta=1.5),
       dict(m=128, n=64, epsilon=0.1, beta=0.5)]


def _params(mp, kw, s=0.01):
    return mp.default_params(h=0.5, dt=s, **kw)


@pytest.mark.parametrize("scheme", [1, 2])
def test_batch_follows_single_instances(mp, scheme):
    ps = [_params(mp, kw) for kw in MIX]
    b = mp.BatchSolver(ps)
    singles = []
    for i, p in enumerate(ps):
        phi0 = inputs.noise_field(p.m, p.n, 0.05 + 0.01 * i, 0.05, 10 + i)
        b.set_state(i, phi0)
        g = mp.Solver(p)
        g.set_state(phi0)
        singles.append(g)
    for step in range(4):
        rc, st, cy = b.step(scheme, 1)
        assert rc == 0 and all(x == 0 for x in st)
        for i, g in enumerate(singles):
            info = g.step(scheme, 1)[0]
            assert cy[i] == info["cycles"], (step, i)
            a, ref = b.get_state(i)[0], g.get_state()[0]
            assert np.abs(a - ref).max() <= 1e-12 * np.abs(ref).max(), (step, i)


def test_batch_fixed_cycles_match_oracle(mp, oracle_mod):
    ps = [_params(mp, kw) for kw in MIX[:3]]
    b = mp.BatchSolver(ps)
    orcs = []
    for i, p in enumerate(ps):
        phi0 = inputs.noise_field(p.m, p.n, 0.07, 0.05, 20 + i)
        b.set_state(i, phi0)
        o = oracle_mod.Solver(oracle_mod.Params(m=p.m, n=p.n, h=p.h, s=p.dt, eps=p.epsilon, beta=p.beta))
        o.set_state(phi0)
        orcs.append(o)
    for step in range(3):
        rc, st = b.step_cycles(1, 3)
        assert rc == 0
        for i, o in enumerate(orcs):
            o.step(1, fixed_cycles=3, guess=1)
            a, ref = b.get_state(i)[0], o.get_state()[0]
            assert np.abs(a - ref).max() <= 1e-10 * np.abs(ref).max(), (step, i)


def test_batch_failure_is_per_instance(mp):
    ps = [_params(mp, kw) for kw in MIX[:3]]
    b = mp.BatchSolver(ps)
    good = []
    for i, p in enumerate(ps):
        phi0 = inputs.noise_field(p.m, p.n, 0.07, 0.05, 30 + i)
        if i == 1:
            phi0[2, 3] = np.nan
        b.set_state(i, phi0)
        good.append(phi0)
    rc, st, cy = b.step(1, 2, raise_on_error=False)
    assert rc == mp.MPFC_ERR_DIVERGED
    assert st[1] == mp.MPFC_ERR_DIVERGED and st[0] == 0 and st[2] == 0
    assert np.isnan(b.get_state(1)[0]).any()          # state kept as set, not advanced
    assert not np.array_equal(b.get_state(0)[0], good[0])


def test_autotuner_keeps_results(mp, tmp_path):
    from paper_1208_2643_gb300 import tuning
    ps = [_params(mp, kw) for kw in MIX]
    b = mp.BatchSolver(ps)
    for i, p in enumerate(ps):
        b.set_state(i, inputs.noise_field(p.m, p.n, 0.07, 0.05, 40 + i))
    ref = None
    chosen = tuning.autotune(b, scheme=1, cache_path=str(tmp_path / "tiles.json"), reps=2)
    assert chosen and all(tx * ty >= 64 for tx, ty, _ in chosen.values())
    rc, st, cy = b.step(1, 2)
    assert rc == 0
    # a second batch reads the cache and gets the same tiles
    b2 = mp.BatchSolver(ps)
    chosen2 = tuning.autotune(b2, scheme=1, cache_path=str(tmp_path / "tiles.json"), reps=2)
    assert {k: v[:2] for k, v in chosen.items()} == {k: tuple(v[:2]) for k, v in chosen2.items()}


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_batch_nonfinite_instance_diverges_alone(mp, bad):
    """One instance with a NaN or infinity in phi reports DIVERGED and keeps its state;
    the other instances step as the single-instance solver does."""
    ps = [_params(mp, kw) for kw in MIX[:3]]
    b = mp.BatchSolver(ps)
    phis = []
    for i, p in enumerate(ps):
        phi0 = inputs.noise_field(p.m, p.n, 0.05 + 0.01 * i, 0.05, 10 + i)
        if i == 1:
            phi0[3, 4] = bad
        b.set_state(i, phi0)
        phis.append(phi0)
    rc, st, cy = b.step(1, 2, raise_on_error=False)
    assert rc == mp.MPFC_ERR_DIVERGED
    assert st[1] == mp.MPFC_ERR_DIVERGED and st[0] == 0 and st[2] == 0
    kept = b.get_state(1)[0]
    ok = ~np.isnan(phis[1])
    assert np.array_equal(np.isnan(kept), np.isnan(phis[1])) and np.array_equal(kept[ok], phis[1][ok])
    for i in (0, 2):
        g = mp.Solver(ps[i])
        g.set_state(phis[i])
        g.step(1, 2)
        ref = g.get_state()[0]
        assert np.abs(b.get_state(i)[0] - ref).max() <= 1e-12 * np.abs(ref).max()
