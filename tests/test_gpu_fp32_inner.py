"""The mixed-precision form (FP64 outer defect correction around FP32 inner V-cycles).

It is a different iteration from the FP64 V-cycle, so it is not compared in lockstep:
each step must reach the same FP64 scaled-residual tolerance, and its phi must stay
within a stated bound of the FP64 oracle's solution of the same step (solved to
1e-13): relative max-norm error <= 1e-8 per step.
"""
import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUND = 1e-8


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import mpfc
    mpfc.load()
    return mpfc


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("scheme,m,n,h,s,steps", [(1, 64, 64, 0.5, 0.01, 10), (2, 96, 160, 0.5, 0.05, 6),
                                                  (1, 128, 128, 0.5, 0.02, 6), (2, 64, 64, 1.0, 1.0, 4)])
def test_fp32_inner_matches_fp64_oracle(mp, oracle_mod, scheme, m, n, h, s, steps):
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 1)
    g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, precision=mp.MPFC_FP32_INNER))
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s))
    o.set_state(phi0)
    worst = 0.0
    for k in range(steps):
        info = g.step(scheme, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10
        r = o.step(scheme, tol=1e-13, guess=1)
        assert r["status"] == 0
        # the oracle continues from its own (tighter) state; compare this step's phi
        e = relerr(g.get_state()[0], o.get_state()[0])
        worst = max(worst, e)
        assert e <= BOUND, (k, e)


@pytest.mark.parametrize("inner", [1, 3, 4, 6])
@pytest.mark.parametrize("scheme,m,s", [(1, 128, 0.02), (2, 96, 1.0)])
def test_fp32_inner_cycle_counts_match_fp64_oracle(mp, oracle_mod, inner, scheme, m, s):
    """Other numbers of FP32 inner V-cycles per FP64 outer iteration (the benchmark runs
    3 and 4 on some workloads) reach the same tolerance and stay within the mixed form's
    1e-8 of the oracle solved to 1e-13, step by step; the outer iterations per step do
    not grow with more inner cycles."""
    n = m
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 1)
    outers = {}
    for ic in (2, inner):
        g = mp.Solver(mp.default_params(m=m, n=n, h=0.5, dt=s, precision=mp.MPFC_FP32_INNER, inner_cycles=ic))
        g.set_state(phi0)
        o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=0.5, s=s))
        o.set_state(phi0)
        cyc = []
        for k in range(4):
            info = g.step(scheme, 1)[0]
            assert info["status"] == 0 and info["res"] <= 1e-10
            cyc.append(info["cycles"])
            assert o.step(scheme, tol=1e-13, guess=1)["status"] == 0
            assert relerr(g.get_state()[0], o.get_state()[0]) <= BOUND, (ic, k)
        outers[ic] = sum(cyc)
        g.close()
    if inner > 2:
        assert outers[inner] <= outers[2], outers


def test_fp32_inner_stream_mode_matches_graph(mp):
    m = 64
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    out = []
    for mode in (mp.MPFC_LAUNCH_GRAPH, mp.MPFC_LAUNCH_STREAM):
        g = mp.Solver(mp.default_params(m=m, n=m, precision=mp.MPFC_FP32_INNER))
        g.set_launch_mode(mode)
        g.set_state(phi0)
        infos = g.step(1, 3)
        out.append((g.get_state()[0], [i["cycles"] for i in infos]))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_fp32_inner_mass_conservation(mp):
    m = 128
    g = mp.Solver(mp.default_params(m=m, n=m, precision=mp.MPFC_FP32_INNER))
    g.set_state(inputs.noise_field(m, m, 0.07, 0.05, 2))
    m0 = g.mass()
    g.step(1, 20)
    assert abs(g.mass() - m0) < 1e-8 * abs(m0)


@pytest.mark.parametrize("m,n", [(64, 64), (128, 128), (96, 160), (64, 96)])
@pytest.mark.parametrize("scheme", [1, 2])
def test_fp32_tail_is_bitwise_the_per_level_cycle(mp, m, n, scheme):
    """The inner V-cycles' small levels run in one CTA with the levels in shared memory
    give exactly the bits of the per-level launches (whole steps, same outer counts)."""
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 5)
    runs = []
    for tail_cells in (0, 16 * 16, 64 * 64):
        g = mp.Solver(mp.default_params(m=m, n=n, h=0.5, dt=0.05, precision=mp.MPFC_FP32_INNER))
        g.set_launch_shape(4, 0, 4 * torch.cuda.get_device_properties(0).multi_processor_count, tail_cells, 1)
        g.set_state(phi0)
        infos = g.step(scheme, 3)
        runs.append(([i["cycles"] for i in infos], g.get_state()))
        g.close()
    for cyc, st in runs[1:]:
        assert cyc == runs[0][0]
        for a, b in zip(st, runs[0][1]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 1e39])
def test_fp32_inner_nonfinite_state_diverges_and_keeps_state(mp, bad):
    """A NaN, an infinity or a value beyond the binary32 range in phi makes the FP64
    defect non-finite; the step reports DIVERGED and leaves the state as it was (the
    FP32 conversions carry non-finite values through instead of mapping them to
    finite ones), and a good state steps normally afterwards."""
    m = 64
    g = mp.Solver(mp.default_params(m=m, n=m, precision=mp.MPFC_FP32_INNER))
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    phi0[5, 7] = bad
    g.set_state(phi0)
    rc, infos = g.step(1, 2, raise_on_error=False)
    assert rc == mp.MPFC_ERR_DIVERGED
    assert infos[0]["status"] == mp.MPFC_ERR_DIVERGED
    phi = g.get_state()[0]
    assert np.array_equal(np.isnan(phi), np.isnan(phi0))
    ok = ~np.isnan(phi0)
    assert np.array_equal(phi[ok], phi0[ok])
    g.set_state(inputs.noise_field(m, m, 0.07, 0.05, 1))
    info = g.step(1, 1)[0]
    assert info["status"] == 0 and info["res"] <= 1e-10


@pytest.mark.parametrize("case", ["periodic1", "periodic2", "ragged2", "neumann2", "pinned2", "odd_sweeps1",
                                  "large1", "largeneumann2"])
def test_fp32_tiled_sweeps_are_bitwise_the_two_launch_sweeps(mp, case):
    """One-launch red-black sweeps over shared-memory tiles (out of place, in pairs)
    give exactly the bits of two in-place half-sweep launches, for every tile height,
    over whole steps (same outer counts, same state).  The large cases have interior
    tiles, which are staged by tensor copies (the others by cp.async)."""
    scheme = int(case[-1])
    m, n = {"ragged2": (96, 160), "neumann2": (128, 64), "large1": (384, 256),
            "largeneumann2": (256, 192)}.get(case, (128, 128))
    kw = dict(m=m, n=n, h=0.5, dt=0.05, precision=mp.MPFC_FP32_INNER)
    if "neumann" in case:
        kw["bc"] = mp.MPFC_BC_NEUMANN_Y
    if case.startswith("pinned"):
        kw["pinning"] = 1
    if case.startswith("odd"):
        kw.update(nu1=3, nu2=1)
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 7)
    runs = []
    for rows in (0, 4, 8, 16, 32):
        g = mp.Solver(mp.default_params(**kw))
        g.set_launch_shape(4, 0, 4 * torch.cuda.get_device_properties(0).multi_processor_count, 0, 1)
        g.set_fp32_sweep(rows, 0)
        if case.startswith("pinned"):
            W = np.zeros((n, m))
            W[n // 4: n // 2, :] = 2.0
            g.set_pinning(W, 0.5 * phi0)
        g.set_state(phi0)
        infos = g.step(scheme, 3)
        assert all(i["status"] == 0 for i in infos)
        runs.append(([i["cycles"] for i in infos], g.get_state()))
        g.close()
    for cyc, st in runs[1:]:
        assert cyc == runs[0][0]
        for a, b in zip(st, runs[0][1]):
            assert np.array_equal(a, b)


def test_fp32_tiled_sweep_wait_timeout_diverges_and_recovers(mp):
    """The tiled sweep's waits for its tensor copies are bounded.  Through the test hook
    the copies of tile (1, 1) are not issued (no out-of-bounds access): the owning CTA's
    wait runs out after 2e6 clock cycles, the CTA writes NaN into its output tiles and
    returns, and the step reports DIVERGED with its state unchanged.  With the hook off,
    the same step converges to the bits of the two-launch sweeps."""
    m, n = 384, 256
    kw = dict(m=m, n=n, h=0.5, dt=0.05, precision=mp.MPFC_FP32_INNER)
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 11)
    lib = mp.load()
    runs = []
    for rows in (0, 16):
        g = mp.Solver(mp.default_params(**kw))
        g.set_fp32_sweep(rows, 0)
        g.set_state(phi0)
        if rows:
            try:
                assert lib.mpfc_fp32_test_withhold_copy(1, 2000000) == 0
                rc, infos = g.step(1, 1, raise_on_error=False)
            finally:
                assert lib.mpfc_fp32_test_withhold_copy(0, 0) == 0
            assert rc == mp.MPFC_ERR_DIVERGED and infos[0]["status"] == mp.MPFC_ERR_DIVERGED
            assert np.array_equal(g.get_state()[0], phi0)
        info = g.step(1, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10
        runs.append((info["cycles"], g.get_state()))
        g.close()
    assert runs[1][0] == runs[0][0]
    for a, b in zip(runs[1][1], runs[0][1]):
        assert np.array_equal(a, b)
    assert lib.mpfc_fp32_test_withhold_copy(2, 0) == mp.MPFC_ERR_INVALID


def test_fp32_sweep_setting_checked(mp):
    g = mp.Solver(mp.default_params(m=64, n=64, precision=mp.MPFC_FP32_INNER))
    for bad in (3, 12, 64, -1):
        with pytest.raises(mp.MPFCError):
            g.set_fp32_sweep(bad, 0)
    f = mp.Solver(mp.default_params(m=64, n=64))
    with pytest.raises(mp.MPFCError):
        f.set_fp32_sweep(16, 0)
