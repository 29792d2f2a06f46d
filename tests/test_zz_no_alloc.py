"""mpfc_mass_noalloc: the allocation-free variant of the mass reduction.

Some callers cannot let a library allocate device memory: an application whose own
memory pool has reserved all of the GPU's memory, or a plug-in whose host forbids
allocations outside the host's allocator.  They get the mass of a device field
through this entry point, whose scratch is a static device array.  This file is
collected last on purpose: it checks the entry point against mpfc_mass, the
workspace-based one, on two calls in a row (and against the oracle's mass), up to
the largest grid it accepts, and must pass alone in a fresh process as well as after
the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1208_2643_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MPFC_ERR_TOO_LARGE = -6   # include/mpfc.h


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2643_gb300 import mpfc
    L = mpfc.load()
    L.mpfc_mass_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_double)]
    L.mpfc_mass_noalloc.restype = ctypes.c_int
    return L


def noalloc_mass(lib, phi_dev, m, n, h, stream):
    out = ctypes.c_double()
    rc = lib.mpfc_mass_noalloc(phi_dev.data_ptr(), m, n, h, stream.cuda_stream, ctypes.byref(out))
    return rc, out.value


# 2048 x 2048 is the largest grid accepted: every block slot of the scratch is used and
# each thread sums its full share of cells
@pytest.mark.parametrize("m,n,h", [(96, 160, 0.5), (1024, 1024, 0.5), (2048, 2048, 0.5)])
def test_noalloc_mass_matches_workspace_mass_twice(lib, m, n, h):
    from oracle import energy
    from paper_1208_2643_gb300 import mpfc
    solver = mpfc.Solver(mpfc.default_params(m=m, n=n, h=h, dt=0.01))
    stream = solver.stream
    solver.set_state(inputs.noise_field(m, n, 0.07, 0.05, 1))
    for call in range(2):
        ref = solver.mass()                       # existing entry point (workspace partials)
        phi = solver.get_state(device=True)[0]
        rc, got = noalloc_mass(lib, phi, m, n, h, stream)
        assert rc == mpfc.MPFC_OK
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
        exact = energy.mass(phi.cpu().numpy(), h)     # the oracle's h^2 sum phi
        assert abs(got - exact) <= 1e-12 * abs(exact), (call, got, exact)
        solver.step(1, 1)                         # a different field for the second call


@pytest.mark.parametrize("m,n", [(4096, 2048), (2048, 2049), (2049, 2048)])
def test_noalloc_rejects_too_large(lib, m, n):
    """Grids past 2048 x 2048 cells are refused before any launch (the 16-element
    array here is never read)."""
    from paper_1208_2643_gb300 import mpfc
    phi = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    rc = lib.mpfc_mass_noalloc(phi.data_ptr(), m, n, 0.5, None, ctypes.byref(out))
    assert rc == MPFC_ERR_TOO_LARGE
    assert "2048" in mpfc.strerror(rc)
