"""Parity of the FP64 CUDA path with the oracle under the mixed boundary conditions
of Sec. 4.5 (periodic in x, homogeneous Neumann in y, ghost rule (A.7) of App. A).

Kernel-level checks compare every building block with the oracle routine of the
same name on the same seeded inputs (ragged sizes, several levels); step-level
checks run whole time steps in lockstep at <= 1e-10 relative per step, the same bar
as the periodic path.  The mirror-extension check compares the GPU's Neumann run
with its own periodic run on the doubled, mirrored domain.
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


def neu(mp, m, n, h, s, **kw):
    return mp.Solver(mp.default_params(m=m, n=n, h=h, dt=s, bc=mp.MPFC_BC_NEUMANN_Y, **kw))


def _level_fields(oracle_mod, scheme, ml, nl, hl, s, seed):
    phik = inputs.noise_field(ml, nl, 0.07, 0.05, seed)
    with oracle_mod.boundary(True):
        S = oracle_mod.source(scheme, oracle_mod.Params(m=ml, n=nl, h=hl, s=s), phik, phik,
                              inputs.noise_field(ml, nl, 0, 0.01, seed + 1))
    rng = np.random.default_rng(seed + 2)
    u = [phik + 0.01 * rng.uniform(-1, 1, (nl, ml)), rng.normal(size=(nl, ml)), rng.normal(size=(nl, ml))]
    return phik, S, u


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("omega", [1.0, 0.8])
@pytest.mark.parametrize("level,sweeps", [(0, 1), (0, 3), (2, 2)])
def test_smooth_neumann(mp, oracle_mod, scheme, omega, level, sweeps):
    m, n, h, s = 96, 160, 0.5, 0.3
    g = neu(mp, m, n, h, s, omega=omega)
    ml, nl, hl = g.level_size(level)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=m, n=n, h=h, s=s), scheme)
    phik, S, u = _level_fields(oracle_mod, scheme, ml, nl, hl, s, 8)
    pk = phik if scheme == 2 else None
    ug = g.op_smooth(scheme, level, [dev(x) for x in u], [dev(x) for x in S], dev(pk) if pk is not None else None,
                     sweeps)
    with oracle_mod.boundary(True):
        uo = oracle_mod.smooth(scheme, consts, hl, u, S, pk, sweeps=sweeps, omega=omega)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("level", [0, 2])
def test_residual_restrict_tau_neumann(mp, oracle_mod, scheme, level):
    m, n, h, s = 96, 160, 0.5, 0.3
    g = neu(mp, m, n, h, s)
    ml, nl, hl = g.level_size(level)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=m, n=n, h=h, s=s), scheme)
    phik, S, u = _level_fields(oracle_mod, scheme, ml, nl, hl, s, 12)
    pk = phik if scheme == 2 else None
    with oracle_mod.boundary(True):
        r = oracle_mod.residual(scheme, consts, hl, u, S, pk)
        uco = [oracle_mod.restrict(x) for x in u]
        pkc = oracle_mod.restrict(phik) if scheme == 2 else None
        No = oracle_mod.apply_N(scheme, consts, 2 * hl, *uco, pkc)
    rg = g.op_residual(scheme, level, [dev(x) for x in u], [dev(x) for x in S], dev(pk) if pk is not None else None)
    for a, b in zip(rg, r):
        assert relerr(host(a), b) < 1e-12
    uc, Sc = g.op_restrict(scheme, level, [dev(x) for x in u], [dev(x) for x in S],
                           dev(pk) if pk is not None else None, dev(pkc) if pkc is not None else None)
    for a, b in zip(uc, uco):
        assert relerr(host(a), b) < 1e-14
    for a, b in zip(Sc, [x + oracle_mod.restrict(y) for x, y in zip(No, r)]):
        assert relerr(host(a), b) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_prolong_neumann(mp, oracle_mod, level):
    g = neu(mp, 96, 160, 0.5, 0.3)
    mc, nc, _ = g.level_size(level + 1)
    mf, nf, _ = g.level_size(level)
    rng = np.random.default_rng(13)
    new = [rng.normal(size=(nc, mc)) for _ in range(3)]
    old = [rng.normal(size=(nc, mc)) for _ in range(3)]
    fine = [rng.normal(size=(nf, mf)) for _ in range(3)]
    out = g.op_prolong(level, [dev(x) for x in new], [dev(x) for x in old], [dev(x) for x in fine])
    with oracle_mod.boundary(True):
        ref = [oracle_mod.prolong_add(a - b, f) for a, b, f in zip(new, old, fine)]
        per_ref = None
    with oracle_mod.boundary(False):
        per_ref = oracle_mod.prolong_add(new[0] - old[0], fine[0])
    for a, b in zip(out, ref):
        assert relerr(host(a), b) < 1e-14
    assert np.abs(ref[0] - per_ref).max() > 1e-3   # the boundary rows differ from the periodic rule


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("m,n,s", [(64, 64, 0.3), (96, 160, 10.0), (128, 32, 0.01)])
def test_coarse_solve_neumann(mp, oracle_mod, scheme, m, n, s):
    g = neu(mp, m, n, 0.5, s)
    mc, nc, hc = g.level_size(g.levels - 1)
    consts = oracle_mod.scheme_consts(oracle_mod.Params(m=m, n=n, h=0.5, s=s), scheme)
    rng = np.random.default_rng(14)
    S = [rng.normal(scale=0.05, size=(nc, mc)) + 0.07 * (i == 0) for i in range(3)]
    phik = 0.07 + 0.05 * rng.uniform(-1, 1, (nc, mc)) if scheme == 2 else None
    u0 = [np.full((nc, mc), 0.07), np.zeros((nc, mc)), np.zeros((nc, mc))]
    ug = g.op_coarse_solve(scheme, [dev(x) for x in u0], [dev(x) for x in S], dev(phik) if phik is not None else None)
    with oracle_mod.boundary(True):
        uo, _ = oracle_mod.coarse_newton(scheme, consts, hc, u0, S, phik)
        r = oracle_mod.residual(scheme, consts, hc, [host(x) for x in ug], S, phik)
    for a, b in zip(ug, uo):
        assert relerr(host(a), b) < 1e-11
    assert max(np.abs(x).max() for x in r) < 1e-11 * max(1.0, max(np.abs(x).max() for x in S))


def _lockstep(mp, oracle_mod, scheme, m, n, h, s, steps, phi0, tol=1e-10, **kw):
    g = neu(mp, m, n, h, s, tol=tol, **kw)
    g.set_state(phi0)
    okw = {"eps": kw["epsilon"]} if "epsilon" in kw else {}
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, ny_neumann=1, **okw))
    o.set_state(phi0)
    for k in range(steps):
        ro = o.step(scheme, tol=tol, guess=1)
        assert ro["status"] == 0
        rg = g.step_cycles(scheme, ro["cycles"])
        assert rg["status"] == 0
        pg, _, psig = g.get_state()
        po, _, psio = o.get_state()
        assert relerr(pg, po) <= 1e-10, (k, relerr(pg, po))
        assert np.abs(psig - psio).max() <= 1e-10 * max(np.abs(psio).max(), np.abs(po).max() / s)
    return g, o


@pytest.mark.parametrize("scheme", [1, 2])
def test_steps_lockstep_neumann_64(mp, oracle_mod, scheme):
    phi0 = inputs.noise_field(64, 64, 0.07, 0.05, 1)
    _lockstep(mp, oracle_mod, scheme, 64, 64, 0.5, 0.01, 10, phi0)


def test_steps_lockstep_neumann_polycrystal_like(mp, oracle_mod):
    """The polycrystal setting of Sec. 4.5 at a test size: scheme 2, eps = 0.25,
    mean density 0.285, seeds near the bottom boundary, ragged 96 x 160 grid."""
    m, n, h = 96, 160, 804.0 / 2048
    phi0 = np.full((n, m), 0.285)
    rng = np.random.default_rng(5)
    for cx in (16, 48, 80):   # three small random perturbations along y = 0
        phi0[0:6, cx - 3:cx + 3] += 0.3 * rng.uniform(-1, 1, (6, 6))
    _lockstep(mp, oracle_mod, 2, m, n, h, 1.0, 5, phi0, epsilon=0.25)


def test_mirror_extension_gpu(mp):
    """The GPU's Neumann run equals its periodic run on the doubled, mirrored domain."""
    m, n, h, s = 64, 64, 0.5, 0.05
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 31)
    a = neu(mp, m, n, h, s, tol=1e-12)
    b = mp.Solver(mp.default_params(m=m, n=2 * n, h=h, dt=s, tol=1e-12))
    a.set_state(phi0)
    b.set_state(np.concatenate([phi0, phi0[::-1]], axis=0))
    for scheme in (1, 2):
        a.step(scheme, 3)
        b.step(scheme, 3)
        pa, pb = a.get_state()[0], b.get_state()[0]
        assert np.abs(pa - pb[:n]).max() < 1e-9
        assert np.abs(pb[n:] - pb[:n][::-1]).max() < 1e-9


def test_mass_and_energy_neumann(mp, oracle_mod):
    from oracle import energy
    m, n, h, s = 96, 64, 0.5, 0.05
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 1)
    g = neu(mp, m, n, h, s)
    g.set_state(phi0)
    m0 = g.mass()
    g.step(2, 3)
    phi, phip, psi = g.get_state()
    assert abs(g.mass() - m0) < 1e-9 * abs(m0)
    e = g.energy()
    ref_f = energy.F(phi, h, 0.025, ny_neumann=True)
    ref_p = energy.pseudo_F(phi, psi, h, 0.025, 1.0, ny_neumann=True)
    ref_t = energy.tilde_F(phi, phip, psi, h, 0.025, 1.0, ny_neumann=True)
    assert abs(e["F"] - ref_f) < 1e-11 * abs(ref_f)
    assert abs(e["pseudoF"] - ref_p) < 1e-10 * abs(ref_p)
    assert abs(e["tildeF"] - ref_t) < 1e-10 * abs(ref_t)
    # and the periodic formulas give something else on this state
    assert abs(energy.pseudo_F(phi, psi, h, 0.025, 1.0) - ref_p) > 1e-8 * abs(ref_p)


def test_neumann_rejected_where_not_built(mp):
    """The mixed conditions are built for single instances with the analytic guesses (FP64
    and FP32-inner): the learned guess and the batch refuse them."""
    bad = [dict(guess=mp.MPFC_GUESS_LEARNED)]
    for kw in bad:
        assert mp.workspace_bytes(mp.default_params(m=64, n=64, bc=mp.MPFC_BC_NEUMANN_Y, **kw)) == 0
    assert mp.workspace_bytes(mp.default_params(m=64, n=64, bc=2)) == 0
    lib = mp.load()
    import ctypes
    arr = (mp.mpfc_params * 2)(mp.default_params(m=64, n=64, bc=mp.MPFC_BC_NEUMANN_Y),
                               mp.default_params(m=64, n=64, bc=mp.MPFC_BC_NEUMANN_Y))
    assert lib.mpfc_batch_workspace_bytes(2, arr) == 0


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("m,n,h,s,eps", [(64, 64, 0.5, 0.2, 0.025), (96, 160, 804.0 / 2048, 1.0, 0.25)])
def test_fp32_inner_neumann(mp, oracle_mod, scheme, m, n, h, s, eps):
    """The mixed-precision form under the Sec. 4.5 conditions: every step within 1e-8 of
    the oracle's Neumann step solved to 1e-13 (the form's bound on periodic grids), and
    the FP32 tail of the inner cycles bit for bit the per-level launches."""
    if m == 96:
        phi0 = np.full((n, m), 0.285)
        rng = np.random.default_rng(5)
        for cx in (16, 48, 80):
            phi0[0:6, cx - 3:cx + 3] += 0.3 * rng.uniform(-1, 1, (6, 6))
    else:
        phi0 = inputs.noise_field(m, n, 0.07, 0.05, 8)
    g = neu(mp, m, n, h, s, epsilon=eps, precision=mp.MPFC_FP32_INNER)
    g.set_state(phi0)
    o = oracle_mod.Solver(oracle_mod.Params(m=m, n=n, h=h, s=s, eps=eps, ny_neumann=1))
    o.set_state(phi0)
    for k in range(4):
        info = g.step(scheme, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10
        assert o.step(scheme, tol=1e-13, guess=1)["status"] == 0
        assert relerr(g.get_state()[0], o.get_state()[0]) <= 1e-8, k
    runs = []
    for tail_cells in (0, 32 * 32):
        a = neu(mp, m, n, h, s, epsilon=eps, precision=mp.MPFC_FP32_INNER)
        a.set_launch_shape(4, 0, 4 * torch.cuda.get_device_properties(0).multi_processor_count, tail_cells, 1)
        a.set_state(phi0)
        infos = a.step(scheme, 3)
        runs.append(([i["cycles"] for i in infos], a.get_state()))
        a.close()
    assert runs[0][0] == runs[1][0]
    for x, y in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(x, y)
