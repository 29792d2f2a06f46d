"""The oracle's all-cores build (OpenMP over independent cells, reductions serial)
gives exactly the bits of the serial build: same V-cycle counts, same residual
histories, same fields, for both schemes, periodic and Neumann-in-y grids, with the
smoother's colours, the operator, the source and the transfers all above the size
where the parallel loops engage."""
import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs


@pytest.mark.parametrize("scheme,ny", [(1, 0), (2, 0), (2, 1)])
def test_threaded_oracle_is_bitwise_serial(oracle_mod, scheme, ny):
    orc = oracle_mod
    used = orc.threads(4)
    assert used == 4
    m, n = 128, 96
    phi0 = inputs.noise_field(m, n, 0.07, 0.05, 3)
    p = orc.Params(m=m, n=n, h=0.5, s=0.05, ny_neumann=ny)
    a, b = orc.Solver(p), orc.Solver(p, threaded=True)
    a.set_state(phi0)
    b.set_state(phi0)
    for _ in range(3):
        ra = a.step(scheme, tol=1e-10, guess=orc.GUESS_EXTRAP)
        rb = b.step(scheme, tol=1e-10, guess=orc.GUESS_EXTRAP)
        assert ra["status"] == 0 and rb["status"] == 0
        assert ra["cycles"] == rb["cycles"]
        assert np.array_equal(ra["hist"], rb["hist"])
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(x, y)
        for x, y in zip(a.get_u(), b.get_u()):
            assert np.array_equal(x, y)
