"""mpfc_mass_noalloc: the allocation-free variant of the mass reduction.

Callers that cannot allocate device memory (inside a stream capture, under a host
that owns the GPU's memory, or in loops that cannot take cudaMalloc's implicit
synchronisation) get the mass of a device field through this entry point, whose
scratch is a static device array.  This file is collected last on purpose: it
checks the new entry point against mpfc_mass, the workspace-based one, on two calls
in a row, and must pass alone in a fresh process as well as after the other tests.
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


@pytest.mark.parametrize("m,n,h", [(96, 160, 0.5), (1024, 1024, 0.5)])
def test_noalloc_mass_matches_workspace_mass_twice(lib, m, n, h):
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
        solver.step(1, 1)                         # a different field for the second call


def test_noalloc_rejects_too_large(lib):
    from paper_1208_2643_gb300 import mpfc
    phi = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    rc = lib.mpfc_mass_noalloc(phi.data_ptr(), 4096, 2048, 0.5, None, ctypes.byref(out))
    assert rc == MPFC_ERR_TOO_LARGE
    assert "2048" in mpfc.strerror(rc)
