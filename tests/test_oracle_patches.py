"""The patch method of the largest-grid tests (tests/test_gpu_max_size.py), checked on
the CPU: the oracle's source, residual and red-black sweep computed on 16 x 16 patches
give, at each sampled cell, exactly the values the oracle computes on the whole grid
(same operations on the same operands, so bit for bit)."""
import numpy as np
import pytest

import patches

F_PHIK, F_PHIKM1, F_PSIK = (0.07, 0.05, 31), (0.07, 0.05, 38), (0.0, 0.01, 32)
F_MU, F_KA = (0.0, 1.0, 33), (0.0, 1.0, 34)
F_S = [(0.0, 1.0, 35), (0.0, 1.0, 36), (0.0, 1.0, 37)]


@pytest.mark.parametrize("scheme", [1, 2])
def test_patches_reproduce_the_whole_grid(oracle_mod, scheme):
    m, n, h, s = 64, 48, 0.5, 0.3
    allr, allc = list(range(n)), list(range(m))
    full = {f: patches.at(m, f, allr, allc) for f in (F_PHIK, F_PHIKM1, F_PSIK, F_MU, F_KA, *F_S)}
    p = oracle_mod.Params(m=m, n=n, h=h, s=s)
    consts = oracle_mod.scheme_consts(p, scheme)
    f_prev = F_PHIKM1 if scheme == 2 else F_PHIK
    S_full = oracle_mod.source(scheme, p, full[F_PHIK], full[f_prev], full[F_PSIK])
    u = [full[F_PHIK], full[F_MU], full[F_KA]]
    S = [full[f] for f in F_S]
    pk = full[F_PHIK] if scheme == 2 else None
    r_full = oracle_mod.residual(scheme, consts, h, u, S, pk)
    u_full = oracle_mod.smooth(scheme, consts, h, u, S, pk, sweeps=1, omega=0.8)
    pp = oracle_mod.Params(m=patches.PATCH, n=patches.PATCH, h=h, s=s)
    for ci, cj in patches.sample_cells(m, n, 12):
        rows, cols, (r, c) = patches.patch(m, n, ci, cj)
        Sp = oracle_mod.source(scheme, pp, patches.at(m, F_PHIK, rows, cols), patches.at(m, f_prev, rows, cols),
                               patches.at(m, F_PSIK, rows, cols))
        up = [patches.at(m, f, rows, cols) for f in (F_PHIK, F_MU, F_KA)]
        Spp = [patches.at(m, f, rows, cols) for f in F_S]
        pkp = up[0] if scheme == 2 else None
        rp = oracle_mod.residual(scheme, consts, h, up, Spp, pkp)
        uo = oracle_mod.smooth(scheme, consts, h, up, Spp, pkp, sweeps=1, omega=0.8)
        for k in range(3):
            assert Sp[k][r, c] == S_full[k][cj, ci]
            assert rp[k][r, c] == r_full[k][cj, ci]
            assert uo[k][r, c] == u_full[k][cj, ci]
