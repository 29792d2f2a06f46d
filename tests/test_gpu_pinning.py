"""Parity of the FP64 CUDA path with the oracle for the pinning term of Sec. 4.6
(second-order scheme, pinned potential mu~ = mu + 2 (phi^{k+1/2} - phihat) W).

Every kernel that the term touches (source, smoother, residual, restriction with
the coarse operator, coarsest solve) is compared with the oracle routine on the same
inputs and the same level weights (2x2 averages of W); whole steps run in lockstep
at <= 1e-10 relative per step, on the strained-crystal setting of Sec. 4.6 at a test
size.  The pinning energy is checked against the oracle's formula.
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


def strips(m, n, w0, width):
    W = np.zeros((n, m))
    W[:width] = w0
    W[-width:] = w0
    return W


def level_weight(oracle_mod, W, level):
    for _ in range(level):
        W = oracle_mod.restrict(W)
    return W


def pinned(mp, m, n, h, s, W, phihat, **kw):
    g = mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, pinning=1, **kw))
    g.set_pinning(W, phihat)
    return g


M, N, H, S = 96, 160, 0.5, 0.3


@pytest.fixture(scope="module")
def setup(mp, oracle_mod):
    W = strips(M, N, 2.0, 8) + 0.25 * (inputs.noise_field(M, N, 0.0, 1.0, 40) > 0.5)
    phihat = inputs.one_mode_crystal(M, N, H, 0.395, 0.6, shift=0.4)
    return W, phihat


def test_source_pinned(mp, oracle_mod, setup):
    W, phihat = setup
    g = pinned(mp, M, N, H, S, W, phihat)
    phik = inputs.noise_field(M, N, 0.07, 0.05, 8)
    phikm1 = inputs.noise_field(M, N, 0.07, 0.05, 9)
    psik = inputs.noise_field(M, N, 0, 0.01, 10)
    Sg = g.op_source(2, dev(phik), dev(phikm1), dev(psik))
    So = oracle_mod.source(2, oracle_mod.Params(m=M, n=N, h=H, s=S), phik, phikm1, psik, W=W, phihat=phihat)
    for a, b in zip(Sg, So):
        assert relerr(host(a), b) < 1e-13


@pytest.mark.parametrize("level,sweeps", [(0, 1), (0, 3), (2, 2)])
def test_smooth_residual_pinned(mp, oracle_mod, setup, level, sweeps):
    W, phihat = setup
    g = pinned(mp, M, N, H, S, W, phihat)
    ml, nl, hl = g.level_size(level)
    Wl = level_weight(oracle_mod, W, level)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=M, n=N, h=H, s=S), 2)
    phik = inputs.noise_field(ml, nl, 0.07, 0.05, 11)
    Sx = oracle_mod.source(2, oracle_mod.Params(m=ml, n=nl, h=hl, s=S), phik, phik,
                           inputs.noise_field(ml, nl, 0, 0.01, 12))
    rng = np.random.default_rng(13)
    u = [phik + 0.01 * rng.uniform(-1, 1, (nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    ug = g.op_smooth(2, level, [dev(x) for x in u], [dev(x) for x in Sx], dev(phik), sweeps)
    uo = oracle_mod.smooth(2, consts, hl, u, Sx, phik, sweeps=sweeps, W=Wl)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11
    rg = g.op_residual(2, level, [dev(x) for x in u], [dev(x) for x in Sx], dev(phik))
    ro = oracle_mod.residual(2, consts, hl, u, Sx, phik, W=Wl)
    for a, b in zip(rg, ro):
        assert relerr(host(a), b) < 1e-12


@pytest.mark.parametrize("level", [0, 2])
def test_restrict_tau_pinned(mp, oracle_mod, setup, level):
    W, phihat = setup
    g = pinned(mp, M, N, H, S, W, phihat)
    ml, nl, hl = g.level_size(level)
    Wl, Wc = level_weight(oracle_mod, W, level), level_weight(oracle_mod, W, level + 1)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=M, n=N, h=H, s=S), 2)
    phik = inputs.noise_field(ml, nl, 0.07, 0.05, 14)
    Sx = oracle_mod.source(2, oracle_mod.Params(m=ml, n=nl, h=hl, s=S), phik, phik,
                           inputs.noise_field(ml, nl, 0, 0.01, 15))
    rng = np.random.default_rng(16)
    u = [phik + 0.01 * rng.uniform(-1, 1, (nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    pkc = oracle_mod.restrict(phik)
    uc, Sc = g.op_restrict(2, level, [dev(x) for x in u], [dev(x) for x in Sx], dev(phik), dev(pkc))
    r = oracle_mod.residual(2, consts, hl, u, Sx, phik, W=Wl)
    uco = [oracle_mod.restrict(x) for x in u]
    No = oracle_mod.apply_N(2, consts, 2 * hl, *uco, pkc, W=Wc)
    for a, b in zip(Sc, [x + oracle_mod.restrict(y) for x, y in zip(No, r)]):
        assert relerr(host(a), b) < 1e-12


def test_coarse_solve_pinned(mp, oracle_mod, setup):
    W, phihat = setup
    g = pinned(mp, M, N, H, 10.0, W, phihat)
    L = g.levels - 1
    mc, nc, hc = g.level_size(L)
    Wc = level_weight(oracle_mod, W, L)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=M, n=N, h=H, s=10.0), 2)
    rng = np.random.default_rng(17)
    Sx = [rng.normal(scale=0.05, size=(nc, mc)) + 0.07 * (i == 0) for i in range(3)]
    phik = 0.07 + 0.05 * rng.uniform(-1, 1, (nc, mc))
    u0 = [np.full((nc, mc), 0.07), np.zeros((nc, mc)), np.zeros((nc, mc))]
    ug = g.op_coarse_solve(2, [dev(x) for x in u0], [dev(x) for x in Sx], dev(phik))
    uo, _ = oracle_mod.coarse_newton(2, consts, hc, u0, Sx, phik, W=Wc)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11


def test_steps_lockstep_strained_crystal(mp, oracle_mod):
    """The strained-crystal setting of Sec. 4.6 at a test size: eps = 0.6, M = 15^2,
    h = 4 pi / (16 sqrt 3), s = 0.025 h^2, scheme 2, weight 2 in strips at the top and
    bottom of a crystal slab, target = the slab shifted by 4 % of 2 pi."""
    from oracle import energy
    m, n = 64, 48
    h = 4 * np.pi / (16 * np.sqrt(3.0))
    s = 0.025 * h * h
    eps, Mob, beta = 0.6, 15.0 ** 2, 0.2
    slab = inputs.one_mode_crystal(m, n, h, 0.395, eps)
    liquid = np.full((n, m), 0.57)
    rows = np.arange(n)[:, None] * np.ones((1, m))
    inside = (rows >= 8) & (rows < n - 8)
    phi0 = np.where(inside, slab, liquid)
    W = np.zeros((n, m))
    band = int(round(np.pi / h))
    W[8:8 + band] = 2.0
    W[n - 8 - band:n - 8] = 2.0
    phihat = np.where(inside, inputs.one_mode_crystal(m, n, h, 0.395, eps, shift=0.04 * 2 * np.pi), liquid)
    g = pinned(mp, m, n, h, s, W, phihat, epsilon=eps, M=Mob, beta=beta, tol=1e-10)
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, eps=eps, M=Mob, beta=beta))
    o.set_pinning(W, phihat)
    o.set_state(phi0)
    for k in range(6):
        ro = o.step(2, tol=1e-10, guess=1)
        assert ro["status"] == 0
        rg = g.step_cycles(2, ro["cycles"])
        assert rg["status"] == 0
        pg, _, psig = g.get_state()
        po, _, psio = o.get_state()
        assert relerr(pg, po) <= 1e-10, (k, relerr(pg, po))
    e = g.energy()
    ref = energy.pin_energy(pg, W, phihat, h)
    assert abs(e["pinning"] - ref) <= 1e-12 * abs(ref)


def test_pinning_rules(mp, setup):
    W, phihat = setup
    m = 64
    g = mp.Solver(mp.default_params(m=m, n=m))
    with pytest.raises(mp.MPFCError):
        g.set_pinning(np.ones((m, m)), np.zeros((m, m)))          # handle created without pinning
    p = pinned(mp, m, m, 0.5, 0.1, np.ones((m, m)), np.zeros((m, m)))
    p.set_state(inputs.noise_field(m, m, 0.07, 0.05, 1))
    rc, _ = p.step(1, 1, raise_on_error=False)
    assert rc == mp.MPFC_ERR_INVALID                                 # scheme 1 refused while pinned
    assert p.step(2, 1)[0]["status"] == 0
    # switched off, it follows the unpinned solver
    q = mp.Solver(mp.default_params(m=m, n=m, dt=0.1))
    p.set_pinning(None)
    st = p.get_state()
    q.set_state(st[0], st[1], st[2])
    p.step(2, 2)
    q.step(2, 2)
    assert np.abs(p.get_state()[0] - q.get_state()[0]).max() == 0.0
    for kw in (dict(guess=mp.MPFC_GUESS_LEARNED),):
        assert mp.workspace_bytes(mp.default_params(m=m, n=m, pinning=1, **kw)) == 0


def test_fp32_inner_pinned_strained_crystal(mp, oracle_mod):
    """The mixed-precision form with the pinning term (its FP32 linearisation takes
    gam + W + g'): each step within 1e-8 of the oracle's pinned step solved to 1e-13."""
    m, n = 64, 48
    h = 4 * np.pi / (16 * np.sqrt(3.0))
    s = 0.025 * h * h
    eps, Mob, beta = 0.6, 15.0 ** 2, 0.2
    slab = inputs.one_mode_crystal(m, n, h, 0.395, eps)
    rows = np.arange(n)[:, None] * np.ones((1, m))
    inside = (rows >= 8) & (rows < n - 8)
    phi0 = np.where(inside, slab, 0.57)
    W = np.zeros((n, m))
    band = int(round(np.pi / h))
    W[8:8 + band] = 2.0
    W[n - 8 - band:n - 8] = 2.0
    phihat = np.where(inside, inputs.one_mode_crystal(m, n, h, 0.395, eps, shift=0.04 * 2 * np.pi), 0.57)
    g = pinned(mp, m, n, h, s, W, phihat, epsilon=eps, M=Mob, beta=beta, precision=mp.MPFC_FP32_INNER)
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, eps=eps, M=Mob, beta=beta))
    o.set_pinning(W, phihat)
    o.set_state(phi0)
    for k in range(4):
        info = g.step(2, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10
        assert o.step(2, tol=1e-13, guess=1)["status"] == 0
        assert relerr(g.get_state()[0], o.get_state()[0]) <= 1e-8, k
