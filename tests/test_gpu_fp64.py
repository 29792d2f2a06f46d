"""Parity of the FP64 CUDA path (through the C ABI) with the CPU oracle.

Kernel-level checks run every building block on the same seeded inputs as the
oracle routine of the same name, at sizes that are not multiples of the 32 x 8
thread tiles.  Step-level checks run whole time steps in lockstep (the GPU takes
the oracle's V-cycle count) and require max-norm relative error <= 1e-10 per
step, the bar the solver is built to.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def make(mp, m, n, h, s, **kw):
    return mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, **kw))


def rand_fields(m, n, seed):
    phik = inputs.noise_field(m, n, 0.07, 0.05, seed)
    phikm1 = inputs.noise_field(m, n, 0.07, 0.05, seed + 1)
    psik = inputs.noise_field(m, n, 0.0, 0.02, seed + 2)
    psik -= psik.mean()
    return phik, phikm1, psik


SIZES = [(96, 160), (64, 64)]


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("m,n", SIZES)
def test_source(mp, oracle_mod, scheme, m, n):
    h, s = 0.7, 0.05
    g = make(mp, m, n, h, s)
    p = oracle_mod.Params(m=m, n=n, h=h, s=s)
    phik, phikm1, psik = rand_fields(m, n, 3)
    Sg = g.op_source(scheme, dev(phik), dev(phikm1), dev(psik))
    So = oracle_mod.source(scheme, p, phik, phikm1, psik)
    for a, b in zip(Sg, So):
        if np.abs(b).max() == 0:
            assert np.abs(host(a)).max() == 0
        else:
            assert relerr(host(a), b) < 1e-13


def _level_inputs(oracle_mod, mp, scheme, m, n, h, s, level, seed):
    g = make(mp, m, n, h, s)
    ml, nl, hl = g.level_size(level)
    p = oracle_mod.Params(m=m, n=n, h=h, s=s)
    consts = oracle_mod.scheme_consts(p, scheme)
    rng = np.random.default_rng(seed)
    u = [0.07 + 0.05 * rng.uniform(-1, 1, (nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    S = [rng.normal(scale=0.05, size=(nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    phik = 0.07 + 0.05 * rng.uniform(-1, 1, (nl, ml)) if scheme == 2 else None
    return g, consts, hl, u, S, phik


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("level", [0, 1, 3])
def test_residual(mp, oracle_mod, scheme, level):
    g, consts, hl, u, S, phik = _level_inputs(oracle_mod, mp, scheme, 96, 160, 0.5, 0.3, level, 5)
    rg = g.op_residual(scheme, level, [dev(x) for x in u], [dev(x) for x in S], dev(phik) if phik is not None else None)
    ro = oracle_mod.residual(scheme, consts, hl, u, S, phik)
    for a, b in zip(rg, ro):
        assert relerr(host(a), b) < 1e-13


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("omega", [1.0, 0.8])
@pytest.mark.parametrize("level,sweeps", [(0, 1), (0, 3), (2, 2)])
def test_smooth(mp, oracle_mod, scheme, omega, level, sweeps):
    m, n, h, s = 96, 160, 0.5, 0.3
    g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, omega=omega))
    ml, nl, hl = g.level_size(level)
    p = oracle_mod.Params(m=m, n=n, h=h, s=s)
    consts = oracle_mod.scheme_consts(p, scheme)
    phik = inputs.noise_field(ml, nl, 0.07, 0.05, 8)
    S = oracle_mod.source(scheme, oracle_mod.Params(m=ml, n=nl, h=hl, s=s), phik, phik,
                          inputs.noise_field(ml, nl, 0, 0.01, 9))
    rng = np.random.default_rng(10)
    u = [phik + 0.01 * rng.uniform(-1, 1, (nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    pk = phik if scheme == 2 else None
    ug = g.op_smooth(scheme, level, [dev(x) for x in u], [dev(x) for x in S], dev(pk) if pk is not None else None,
                     sweeps)
    uo = oracle_mod.smooth(scheme, consts, hl, u, S, pk, sweeps=sweeps, omega=omega)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("level", [0, 2])
def test_restrict_tau(mp, oracle_mod, scheme, level):
    m, n, h, s = 96, 160, 0.5, 0.3
    g, consts, hl, u, S, phik = _level_inputs(oracle_mod, mp, scheme, m, n, h, s, level, 12)
    p = oracle_mod.Params(m=m, n=n, h=h, s=s)
    phik_c = oracle_mod.restrict(phik) if scheme == 2 else None
    uc, Sc = g.op_restrict(scheme, level, [dev(x) for x in u], [dev(x) for x in S],
                           dev(phik) if phik is not None else None, dev(phik_c) if phik_c is not None else None)
    r = oracle_mod.residual(scheme, consts, hl, u, S, phik)
    uco = [oracle_mod.restrict(x) for x in u]
    No = oracle_mod.apply_N(scheme, consts, 2 * hl, *uco, phik_c)
    Sco = [a + oracle_mod.restrict(b) for a, b in zip(No, r)]
    for a, b in zip(uc, uco):
        assert relerr(host(a), b) < 1e-14
    for a, b in zip(Sc, Sco):
        assert relerr(host(a), b) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_prolong(mp, oracle_mod, level):
    g = make(mp, 96, 160, 0.5, 0.3)
    mc, nc, _ = g.level_size(level + 1)
    mf, nf, _ = g.level_size(level)
    rng = np.random.default_rng(13)
    new = [rng.normal(size=(nc, mc)) for _ in range(3)]
    old = [rng.normal(size=(nc, mc)) for _ in range(3)]
    fine = [rng.normal(size=(nf, mf)) for _ in range(3)]
    out = g.op_prolong(level, [dev(x) for x in new], [dev(x) for x in old], [dev(x) for x in fine])
    for a, c_new, c_old, f in zip(out, new, old, fine):
        assert relerr(host(a), oracle_mod.prolong_add(c_new - c_old, f)) < 1e-14


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("m,n,s", [(64, 64, 0.3), (96, 160, 10.0), (128, 32, 0.01), (64, 96, 1.0), (64, 64, 200.0)])
def test_coarse_solve(mp, oracle_mod, scheme, m, n, s):
    g = make(mp, m, n, 0.5, s)
    L = g.levels - 1
    mc, nc, hc = g.level_size(L)
    p = oracle_mod.Params(m=m, n=n, h=0.5, s=s)
    consts = oracle_mod.scheme_consts(p, scheme)
    rng = np.random.default_rng(14)
    S = [rng.normal(scale=0.05, size=(nc, mc)) + 0.07 * (i == 0) for i in range(3)]
    phik = 0.07 + 0.05 * rng.uniform(-1, 1, (nc, mc)) if scheme == 2 else None
    u0 = [np.full((nc, mc), 0.07), np.zeros((nc, mc)), np.zeros((nc, mc))]
    ug = g.op_coarse_solve(scheme, [dev(x) for x in u0], [dev(x) for x in S], dev(phik) if phik is not None else None)
    uo, _ = oracle_mod.coarse_newton(scheme, consts, hc, u0, S, phik)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11
    # and it really solves N(u) = S
    r = oracle_mod.residual(scheme, consts, hc, [host(x) for x in ug], S, phik)
    assert max(np.abs(x).max() for x in r) < 1e-11 * max(1.0, max(np.abs(x).max() for x in S))


def _lockstep(mp, oracle_mod, scheme, m, n, h, s, steps, phi0, omega=0.8, guess=1, tol=1e-10):
    g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, omega=omega, guess=guess, tol=tol))
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, omega=omega))
    o.set_state(phi0)
    worst = 0.0
    for k in range(steps):
        ro = o.step(scheme, tol=tol, guess=guess)
        assert ro["status"] == 0
        rg = g.step_cycles(scheme, ro["cycles"])
        assert rg["status"] == 0
        pg, _, psig = g.get_state()
        po, _, psio = o.get_state()
        e = relerr(pg, po)
        worst = max(worst, e)
        assert e <= 1e-10, (k, e)
        assert np.abs(psig - psio).max() <= 1e-10 * max(np.abs(psio).max(), np.abs(po).max() / s)
    return g, o, worst


@pytest.mark.parametrize("scheme", [1, 2])
def test_steps_lockstep_64(mp, oracle_mod, scheme):
    """The 64^2 first-order workload (h = 0.5, eps = 0.025, beta = 0.9, s = 0.01, 20 steps,
    phi0 = 0.07 + 0.05 U) for both schemes, lockstep with the oracle."""
    phi0 = inputs.noise_field(64, 64, 0.07, 0.05, 1)
    _lockstep(mp, oracle_mod, scheme, 64, 64, 0.5, 0.01, 20, phi0)


def test_steps_lockstep_ragged_scheme2(mp, oracle_mod):
    phi0 = inputs.crystallite_field(96, 160, np.pi / 4, -0.285, 0.25, count=2, radius_cells=12, seed=2)
    _lockstep(mp, oracle_mod, 2, 96, 160, np.pi / 4, 0.05, 6, phi0)


def test_steps_lockstep_coarsest_4x6(mp, oracle_mod):
    """64 x 96: the hierarchy ends on a 4 x 6 grid (24 cells), the coarsest solve's
    32-row register path; 128 x 32 ends on 16 x 4 (64 cells, shared-memory path)."""
    for m, n in ((64, 96), (128, 32)):
        phi0 = inputs.noise_field(m, n, 0.07, 0.05, 7)
        _lockstep(mp, oracle_mod, 1, m, n, 0.5, 0.05, 4, phi0)


def test_steps_lockstep_undamped(mp, oracle_mod):
    phi0 = inputs.noise_field(64, 64, 0.07, 0.05, 1)
    _lockstep(mp, oracle_mod, 1, 64, 64, 0.5, 0.01, 5, phi0, omega=1.0, guess=0)


def test_own_cycle_count_matches_oracle(mp, oracle_mod):
    """Without lockstep the GPU's device-side tolerance test picks the oracle's cycle counts."""
    m, h, s = 64, 0.5, 0.01
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    g = make(mp, m, m, h, s)
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=m, h=h, s=s))
    o.set_state(phi0)
    infos = g.step(1, 10)
    oc = [o.step(1, tol=1e-10, guess=1)["cycles"] for _ in range(10)]
    assert [i["cycles"] for i in infos] == oc
    assert relerr(g.get_state()[0], o.get_state()[0]) < 1e-10


def test_headline_size_one_step(mp, oracle_mod):
    """One lockstep step at the 1024^2 headline size (all cells compared)."""
    m, h, s = 1024, 0.5, 0.01
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    _lockstep(mp, oracle_mod, 1, m, m, h, s, 1, phi0)


def test_mass_and_energy(mp, oracle_mod):
    from oracle import energy
    m, h, s = 96, 0.5, 0.05
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    g = make(mp, m, m, h, s)
    g.set_state(phi0)
    g.step(2, 3)
    phi, phip, psi = g.get_state()
    assert abs(g.mass() - energy.mass(phi, h)) < 1e-12 * abs(energy.mass(phi, h))
    e = g.energy()
    assert abs(e["F"] - energy.F(phi, h, 0.025)) < 1e-11 * abs(energy.F(phi, h, 0.025))
    ref_p = energy.pseudo_F(phi, psi, h, 0.025, 1.0)
    ref_t = energy.tilde_F(phi, phip, psi, h, 0.025, 1.0)
    assert abs(e["pseudoF"] - ref_p) < 1e-10 * abs(ref_p)
    assert abs(e["tildeF"] - ref_t) < 1e-10 * abs(ref_t)


def test_mass_conserved_over_many_steps(mp):
    m, h, s = 128, 0.5, 0.01
    g = make(mp, m, m, h, s)
    g.set_state(inputs.noise_field(m, m, 0.07, 0.05, 1))
    m0 = g.mass()
    g.step(1, 50)
    assert abs(g.mass() - m0) < 1e-8 * abs(m0)


def test_not_converged_keeps_state(mp):
    m = 64
    g = mp.Solver(mp.default_params(m=m, n=m, max_cycles=1, tol=1e-14))
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    g.set_state(phi0)
    rc, infos = g.step(1, 3, raise_on_error=False)
    assert rc == mp.MPFC_ERR_NOT_CONVERGED
    assert infos[0]["status"] == mp.MPFC_ERR_NOT_CONVERGED and infos[0]["cycles"] == 1
    assert np.array_equal(g.get_state()[0], phi0)


def test_diverged_on_nan(mp):
    m = 32
    g = make(mp, m, m, 0.5, 0.01)
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    phi0[3, 4] = np.nan
    g.set_state(phi0)
    rc, infos = g.step(1, 2, raise_on_error=False)
    assert rc == mp.MPFC_ERR_DIVERGED
    # a good state afterwards steps normally again
    g.set_state(inputs.noise_field(m, m, 0.07, 0.05, 1))
    assert g.step(1, 1)[0]["status"] == 0


def test_invalid_arguments(mp):
    import ctypes
    lib = mp.load()
    p = mp.default_params(m=62, n=64)   # 62 -> 31 is odd: hierarchy stops at a coarse grid too big for the dense solve
    assert mp.workspace_bytes(p) == 0
    p = mp.default_params(m=64, n=64)
    nbytes = mp.workspace_bytes(p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    assert lib.mpfc_create(ctypes.byref(p), ws.data_ptr(), nbytes - 1024, None, ctypes.byref(h)) == mp.MPFC_ERR_WORKSPACE
    assert lib.mpfc_create(ctypes.byref(p), ws.data_ptr() + 8, nbytes, None, ctypes.byref(h)) == mp.MPFC_ERR_WORKSPACE
    g = make(mp, 64, 64, 0.5, 0.01)
    assert lib.mpfc_step(g.h, 3, 1, None) == mp.MPFC_ERR_INVALID


def test_checkpoint_resume_bitwise(mp):
    m, h, s = 64, 0.5, 0.05
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    a = make(mp, m, m, h, s)
    a.set_state(phi0)
    a.step(2, 10)
    b = make(mp, m, m, h, s)
    b.set_state(phi0)
    b.step(2, 5)
    st = b.get_state()
    c = make(mp, m, m, h, s)
    c.set_state(*st)
    c.step(2, 5)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)


def test_multi_step_call_equals_single_steps(mp):
    m = 64
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    a = make(mp, m, m, 0.5, 0.01)
    a.set_state(phi0)
    a.step(1, 6)
    b = make(mp, m, m, 0.5, 0.01)
    b.set_state(phi0)
    for _ in range(6):
        b.step(1, 1)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_stream_launch_mode_matches_graph(mp):
    """The same kernels launched one by one (host-side loop test) give bitwise the same steps."""
    m = 96
    phi0 = inputs.noise_field(m, m, 0.07, 0.05, 1)
    res = []
    for mode in (mp.MPFC_LAUNCH_GRAPH, mp.MPFC_LAUNCH_STREAM):
        g = make(mp, m, m, 0.5, 0.05)
        g.set_launch_mode(mode)
        g.set_state(phi0)
        infos = g.step(2, 4)
        res.append((g.get_state()[0], [i["cycles"] for i in infos]))
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][0], res[1][0])


def test_smoother_reciprocal_error_bound(mp):
    """The cell solve's reciprocal (Newton-Raphson step from the single-precision
    reciprocal) stays within 2^-44 relative of the IEEE double quotient."""
    lib = mp.load()
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(1.0, 2.0, 4096), 10.0 ** rng.uniform(-3, 12, 4096), [1.0, 3.0, 7.0, 1e10]])
    xd = dev(x)
    y = torch.empty_like(xd)
    assert lib.mpfc_probe_rcp(xd.data_ptr(), y.data_ptr(), x.size, None) == 0
    rel = np.abs(host(y) * x - 1.0)
    assert rel.max() < 2.0 ** -44, rel.max()


def test_integer_pipe_conversions_match_ieee(mp):
    """binary64 -> binary32 round-to-nearest-even, truncation and exact widening, done on
    the integer pipes, against the IEEE conversions (numpy) over the normal range."""
    import ctypes
    lib = mp.load()
    lib.mpfc_probe_convert.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p]
    rng = np.random.default_rng(5)
    mags = 2.0 ** rng.uniform(-120, 120, 20000)
    x = np.concatenate([mags * rng.choice([-1, 1], mags.size), [0.0, -0.0, 1.0, -1.5, 3.4e38, 1.2e-38],
                        np.nextafter(np.float32(1.0), np.float32(2.0)).astype(np.float64) + np.array([1e-12, -1e-12, 0])])
    # exact ties: binary32 midpoints
    f = rng.uniform(1, 2, 1000).astype(np.float32).astype(np.float64)
    x = np.concatenate([x, f + 2.0 ** -24, f - 2.0 ** -24])
    xd = dev(x)
    rn = torch.empty(x.size, dtype=torch.float32, device="cuda")
    tr = torch.empty_like(rn)
    back = torch.empty_like(xd)
    assert lib.mpfc_probe_convert(xd.data_ptr(), rn.data_ptr(), tr.data_ptr(), back.data_ptr(), x.size, None) == 0
    torch.cuda.synchronize()
    ref = x.astype(np.float32)
    got = rn.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(back.cpu().numpy(), ref.astype(np.float64))
    t = tr.cpu().numpy().astype(np.float64)
    nz = x != 0
    assert np.all(np.abs(t[nz] - x[nz]) <= np.abs(x[nz]) * 2.0 ** -23)
    assert np.all(np.abs(t[nz]) <= np.abs(x[nz]))


def _rz32(x):
    """binary64 -> binary32 rounded toward zero (numpy rounds to nearest): the nearest
    conversion, stepped one binary32 toward zero where it went past |x|."""
    with np.errstate(over="ignore", invalid="ignore"):
        f = x.astype(np.float32)
        past = np.isfinite(x) & (np.abs(f.astype(np.float64)) > np.abs(x))
    f[past] = np.nextafter(f[past], np.float32(0.0))
    return f


def test_integer_pipe_conversions_special_values(mp):
    """Outside the normal binary32 range the conversions equal the IEEE ones too:
    NaN stays NaN, infinities and overflow give infinities (FLT_MAX toward zero),
    binary32 underflow gives the correctly rounded subnormal or zero, and the widening
    of binary32 subnormals, infinities and NaN is exact."""
    import ctypes
    lib = mp.load()
    lib.mpfc_probe_convert.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p]
    fmax = float(np.finfo(np.float32).max)
    x = np.array([np.nan, -np.nan, np.inf, -np.inf, 1e39, -1e39, 1e300, -1e300, fmax, -fmax,
                  fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), 2.0 ** 128, 1e-39, -1e-39, 1e-45, 7e-46,
                  1.4e-45, 1e-300, -1e-300, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150,
                  2.0 ** -150 * 1.0000001, 3 * 2.0 ** -151, 0.0, -0.0, 5e-324])
    rng = np.random.default_rng(11)
    x = np.concatenate([x, rng.uniform(-1, 1, 2000) * 2.0 ** rng.uniform(-160, -120, 2000),
                        rng.uniform(-1, 1, 200) * 2.0 ** rng.uniform(126, 140, 200)])
    xd = dev(x)
    rn = torch.empty(x.size, dtype=torch.float32, device="cuda")
    tr = torch.empty_like(rn)
    back = torch.empty_like(xd)
    assert lib.mpfc_probe_convert(xd.data_ptr(), rn.data_ptr(), tr.data_ptr(), back.data_ptr(), x.size, None) == 0
    torch.cuda.synchronize()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float32)
    got = rn.cpu().numpy()
    nan = np.isnan(x)
    assert np.all(np.isnan(got[nan]))
    assert np.array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    tz = tr.cpu().numpy()
    assert np.all(np.isnan(tz[nan]))
    assert np.array_equal(tz[~nan].view(np.uint32), _rz32(x)[~nan].view(np.uint32))
    b = back.cpu().numpy()
    assert np.all(np.isnan(b[nan]))
    assert np.array_equal(b[~nan], ref[~nan].astype(np.float64))


@pytest.mark.parametrize("ctas", [1, 8, 16])
@pytest.mark.parametrize("case", ["periodic1", "periodic2", "ragged2", "neumann2", "pinned2"])
def test_tail_cluster_is_bitwise_the_per_level_cycle(mp, case, ctas):
    """The coarse levels run as one launch, of one CTA or of a thread-block cluster
    (barriers between the phases), give exactly the bits of the per-level launches,
    over several steps."""
    probe = mp.Solver(mp.default_params(m=64, n=64))
    try:
        probe.set_launch_shape(1, 0, 4 * torch.cuda.get_device_properties(0).multi_processor_count, 64 * 64, ctas)
    except mp.MPFCError:
        pytest.skip(f"this GPU holds no {ctas}-CTA cluster")
    finally:
        probe.close()
    scheme = int(case[-1])
    m, n = (96, 160) if case.startswith("ragged") else (128, 128)
    kw = {}
    if case.startswith("neumann"):
        kw["bc"] = mp.MPFC_BC_NEUMANN_Y
    if case.startswith("pinned"):
        kw["pinning"] = 1
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 3)
    runs = []
    for tail_cells in (0, 16 * 16, 32 * 32, 64 * 64):
        g = mp.Solver(mp.default_params(m=m, n=n, h=0.5, dt=0.05, **kw))
        if case.startswith("pinned"):
            W = np.zeros((n, m))
            W[:10] = 2.0
            W[-10:] = 2.0
            g.set_pinning(W, inputs.noise_field(m, n, 0.1, 0.05, 4))
        g.set_launch_shape(1, 0, 4 * torch.cuda.get_device_properties(0).multi_processor_count, tail_cells, ctas)
        g.set_state(phi0)
        infos = g.step(scheme, 3)
        runs.append(([i["cycles"] for i in infos], g.get_state()))
        g.close()
    for cyc, st in runs[1:]:
        assert cyc == runs[0][0]
        for a, b in zip(st, runs[0][1]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("case", ["periodic1", "periodic2", "ragged1", "ragged2", "neumann2", "pinned2"])
def test_transfer_split_is_bitwise_the_per_coarse_cell_transfers(mp, case):
    """The restriction with four threads per coarse cell and the prolongation with one
    thread per fine cell give exactly the bits of the one-thread-per-coarse-cell kernels,
    over several steps: on every per-level launch (no tail, down to a 6 x 10 coarsest
    grid on the ragged case, where a warp's last quads lie past the grid), on the levels
    of at most 64^2 cells only, and beside the default coarse tail."""
    scheme = int(case[-1])
    m, n = (96, 160) if case.startswith("ragged") else (128, 128)
    kw = {}
    if case.startswith("neumann"):
        kw["bc"] = mp.MPFC_BC_NEUMANN_Y
    if case.startswith("pinned"):
        kw["pinning"] = 1
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 13)
    runs = []
    for tail_cells, split in ((0, 0), (0, 1 << 30), (0, 64 * 64), (256, 1 << 30)):
        g = mp.Solver(mp.default_params(m=m, n=n, h=0.5, dt=0.05, **kw))
        if case.startswith("pinned"):
            W = np.zeros((n, m))
            W[:10] = 2.0
            W[-10:] = 2.0
            g.set_pinning(W, inputs.noise_field(m, n, 0.1, 0.05, 4))
        g.set_launch_shape(1, 0, 16, tail_cells, 1)
        g.set_transfer_split(split)
        g.set_state(phi0)
        infos = g.step(scheme, 3)
        assert all(i["status"] == 0 for i in infos)
        runs.append(([i["cycles"] for i in infos], g.get_state()))
        g.close()
    for cyc, st in runs[1:]:
        assert cyc == runs[0][0]
        for a, b in zip(st, runs[0][1]):
            assert np.array_equal(a, b)


def test_transfer_split_rules(mp):
    g = mp.Solver(mp.default_params(m=64, n=64))
    with pytest.raises(mp.MPFCError):
        g.set_transfer_split(-1)
    g.set_transfer_split(1 << 20)
    g.set_launch_shape(1, 0, 16, 0, 1)
    assert g.launch_counts(1) == (6, 4 * 11 + 2)   # the same launches, other thread layouts
    g.close()


def test_launch_counts(mp):
    """Kernels per step and per V-cycle under the default launch shape: 64^2 has levels
    64, 32, 16, 8, 4; the levels of at most 16 x 16 cells run as one launch, so two
    levels keep their 11 launches (4 + 4 sweeps, restriction, tau, prolongation)."""
    g = mp.Solver(mp.default_params(m=64, n=64))
    assert g.launch_counts(1) == (6, 2 * 11 + 2)
    assert g.launch_counts(2) == (6 + 4, 2 * 11 + 2)
    g.set_launch_shape(1, 0, 608, 0, 1)   # no tail: every level above the coarsest, and the coarse solve
    assert g.launch_counts(1) == (6, 4 * 11 + 2)
    h = mp.Solver(mp.default_params(m=64, n=64, precision=mp.MPFC_FP32_INNER))
    with pytest.raises(mp.MPFCError):
        h.launch_counts(1)


@pytest.mark.parametrize("scheme", [1, 2])
def test_launch_shape_does_not_change_results(mp, scheme):
    """Block shapes, programmatic dependent launch and the coarse tails are a tuning
    choice: every shape gives the bits of the default one (128 x 96, 4 steps)."""
    m, n = 128, 96
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 9)
    # the last shape puts every level in the tail, so the convergence test is k_resnorm over all
    # cells instead of the residual of the finest level's last half sweep plus k_resnorm_red
    shapes = [None, (8, 0, 0, 0, 1), (2, 38912, 0, 1024, 1), (4, 1 << 20, 1 << 20, 256, 8), (1, 0, 608, 64 * 64, 1),
              (1, 0, 608, 1 << 20, 1)]
    runs = []
    for sh in shapes:
        g = mp.Solver(mp.default_params(m=m, n=n, h=0.5, dt=0.05))
        if sh is not None:
            g.set_launch_shape(*sh)
        g.set_state(phi0)
        infos = g.step(scheme, 4)
        runs.append(([i["cycles"] for i in infos], g.get_state(), [i["res"] for i in infos]))
        g.close()
    for cyc, st, res in runs[1:]:
        assert cyc == runs[0][0]
        for a, b in zip(st, runs[0][1]):
            assert np.array_equal(a, b)
        # the same residual norm, summed in another order and partly from registers
        np.testing.assert_allclose(res, runs[0][2], rtol=1e-5)


def test_launch_shape_rules(mp):
    g = mp.Solver(mp.default_params(m=64, n=64))
    for bad in ((3, 0, 0, 0, 1), (1, -1, 0, 0, 1), (1, 0, -1, 0, 1), (1, 0, 0, -5, 1), (1, 0, 0, 0, 4)):
        with pytest.raises(mp.MPFCError):
            g.set_launch_shape(*bad)
    with pytest.raises(mp.MPFCError):   # the FP32 sweep timer wants a mixed-precision handle
        g.fp32_time_smooth(0, 1)
    h = mp.Solver(mp.default_params(m=64, n=64, precision=mp.MPFC_FP32_INNER))
    assert h.fp32_time_smooth(0, 2) > 0.0
    with pytest.raises(mp.MPFCError):
        h.fp32_time_smooth(h.levels, 1)


@pytest.mark.parametrize("scheme", [1, 2])
def test_initial_residual_equals_oracle(mp, oracle_mod, scheme):
    """After the initial guess only row 1 of the residual is evaluated (rows 2 and 3 hold
    by construction); the reported initial norm equals the oracle's full residual norm
    after its own guess, step after step, also under the Neumann rule."""
    for kw, okw in (({}, {}), ({"bc": mp.MPFC_BC_NEUMANN_Y}, {"ny_neumann": 1})):
        m, n, h, s = 64, 96, 0.5, 0.05
        phi0 = inputs.noise_field(m, n, 0.07, 0.05, 12)
        g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, **kw))
        g.set_state(phi0)
        o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, **okw))
        o.set_state(phi0)
        for k in range(3):
            ro = o.step(scheme, tol=1e-10, guess=1)
            rg = g.step_cycles(scheme, ro["cycles"])
            assert abs(rg["res0"] - ro["res0"]) <= 1e-9 * ro["res0"], (k, rg["res0"], ro["res0"])
        g.close()
