"""The CUDA path at the largest grid it accepts: 32768 x 32768 = 2^30 cells (planes of
8 GiB, a 120 GiB FP64 workspace), where 32-bit cell indices reach their limit and
plane offsets pass 2^33 bytes.

The oracle cannot run grids this size, so it computes sampled outputs one at a time:
each sampled cell's neighbourhood is cut out as a 16 x 16 periodic patch (same
colouring; the periodic wrap of the patch lies outside the cell's domain of
dependence) from the seeded generator's values at those cells, and the oracle's
source (App. B.1/B.2), residual and red-black sweep on the patch give the cell's
value (tests/test_oracle_patches.py shows on the CPU that this reproduces the
whole-grid oracle bit for bit).  Inputs are built on the device by the same
counter-based generator, bit for bit.  Whole time steps (FP64, and FP32 inner cycles
with FP64 defect correction) are checked by properties: convergence to the tolerance,
conservation of mass, and the two forms' agreement at the sampled cells.
"""
import numpy as np
import pytest

import patches
from paper_1208_2643_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

M = N = 32768
H, S_DT = 0.5, 0.3
PATCH = patches.PATCH


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < (230 << 30):
        pytest.skip("needs a GPU with at least 230 GiB")
    from paper_1208_2643_gb300 import mpfc
    mpfc.load()
    return mpfc


def _samples():
    return patches.sample_cells(M, N, 24)


def _patch(ci, cj):
    return patches.patch(M, N, ci, cj)


# generator fields: (mean, amplitude, seed)
F_PHIK, F_PHIKM1, F_PSIK = (0.07, 0.05, 31), (0.07, 0.05, 38), (0.0, 0.01, 32)
F_MU, F_KA = (0.0, 1.0, 33), (0.0, 1.0, 34)
F_S = [(0.0, 1.0, 35), (0.0, 1.0, 36), (0.0, 1.0, 37)]


def _dev(f):
    return inputs.noise_field_torch(M, N, *f, device="cuda")


def _at(f, rows, cols):
    return patches.at(M, f, rows, cols)


def _gather(t, cells):
    i = torch.tensor([c[0] for c in cells], device=t.device)
    j = torch.tensor([c[1] for c in cells], device=t.device)
    return t[j, i].cpu().numpy()


def _close(got, want, tol):
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= tol * scale, (np.abs(got - want).max(), scale)


@pytest.mark.parametrize("scheme", [1, 2])
def test_max_size_kernels_at_sampled_cells(mp, oracle_mod, scheme):
    """Source, residual and one red-black sweep (level 0, omega = 0.8) of the 2^30-cell
    grid at 32 sampled cells (corners, edges, random) against the oracle on patches:
    source and residual to 1e-13, the sweep to 1e-11 (relative to the largest sampled
    value), as the kernel-level tests require at small sizes."""
    cells = _samples()
    g = mp.Solver(mp.default_params(m=M, n=N, h=H, dt=S_DT))
    lib, s = g.lib, g.stream
    p = oracle_mod.Params(m=PATCH, n=PATCH, h=H, s=S_DT)
    consts = oracle_mod.scheme_consts(p, scheme)

    phik = _dev(F_PHIK)
    phikm1 = _dev(F_PHIKM1) if scheme == 2 else phik
    psik = _dev(F_PSIK)
    Sg = g.op_source(scheme, phik, phikm1, psik)
    s.synchronize()
    got = [_gather(x, cells) for x in Sg]
    del Sg, psik
    if scheme == 2:
        del phikm1
    want = [[], [], []]
    for ci, cj in cells:
        rows, cols, (r, c) = _patch(ci, cj)
        f_prev = F_PHIKM1 if scheme == 2 else F_PHIK
        So = oracle_mod.source(scheme, p, _at(F_PHIK, rows, cols), _at(f_prev, rows, cols), _at(F_PSIK, rows, cols))
        for k in range(3):
            want[k].append(So[k][r, c])
    for a, b in zip(got, want):
        _close(a, np.array(b), 1e-13)

    phi = phik.clone() if scheme == 2 else phik
    u = [phi, _dev(F_MU), _dev(F_KA)]
    S = [_dev(f) for f in F_S]
    pk = phik if scheme == 2 else None
    r = g.op_residual(scheme, 0, u, S, pk)
    s.synchronize()
    got_r = [_gather(x, cells) for x in r]
    del r
    rc = lib.mpfc_op_smooth(g.h, scheme, 0, *[x.data_ptr() for x in u], *[x.data_ptr() for x in S],
                            pk.data_ptr() if pk is not None else None, 1)
    assert rc == 0
    s.synchronize()
    got_u = [_gather(x, cells) for x in u]
    want_r, want_u = [[], [], []], [[], [], []]
    for ci, cj in cells:
        rows, cols, (rr, cc) = _patch(ci, cj)
        up = [_at(F_PHIK, rows, cols), _at(F_MU, rows, cols), _at(F_KA, rows, cols)]
        Sp = [_at(f, rows, cols) for f in F_S]
        pkp = up[0] if scheme == 2 else None
        ro = oracle_mod.residual(scheme, consts, H, up, Sp, pkp)
        uo = oracle_mod.smooth(scheme, consts, H, up, Sp, pkp, sweeps=1, omega=0.8)
        for k in range(3):
            want_r[k].append(ro[k][rr, cc])
            want_u[k].append(uo[k][rr, cc])
    for a, b in zip(got_r, want_r):
        _close(a, np.array(b), 1e-13)
    for a, b in zip(got_u, want_u):
        _close(a, np.array(b), 1e-11)
    del u, S, phik, pk, phi
    g.close()
    torch.cuda.empty_cache()


def test_max_size_steps_converge_and_conserve_mass(mp):
    """One time step of scheme 1 at 2^30 cells in FP64 and in the mixed form (FP32 inner
    V-cycles, FP64 outer defect correction, tiled FP32 sweeps on the finest levels):
    both converge to the scaled residual 1e-10, the mass moves by no more than the
    inexact solve allows (50 tol per unit area, as for the 512^2 run), and the two
    results agree at the sampled cells to 1e-8 relative, the mixed form's bound."""
    cells = _samples()
    area = (M * H) ** 2
    phi0 = _dev(F_PHIK)
    mass0 = float(phi0.sum()) * H * H   # torch's own reduction of the input
    out = {}
    for prec in (mp.MPFC_FP64, mp.MPFC_FP32_INNER):
        g = mp.Solver(mp.default_params(m=M, n=N, h=H, dt=0.01, precision=prec))
        g.set_state(phi0)
        assert abs(g.mass() - mass0) <= 1e-12 * abs(mass0)
        info = g.step(1, 1)[0]
        assert info["status"] == 0 and info["res"] <= 1e-10, info
        assert abs(g.mass() - mass0) <= 50 * 1e-10 * area
        out[prec] = _gather(g.get_state(device=True)[0], cells)
        g.close()
        torch.cuda.empty_cache()
    a, b = out[mp.MPFC_FP32_INNER], out[mp.MPFC_FP64]
    assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
