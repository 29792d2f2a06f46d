"""Plain FP64 CPU oracle of the MPFC convex-splitting schemes and their FAS solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never links, loads or calls it, and it shares no
code with the CUDA path (the only shared module is the seeded input generator,
which holds none of the method's arithmetic).

Parts:
  * ``mpfc_oracle.c`` (plain serial C, FP64): Delta_h, the FAS operator N and
    source S of App. B.1/B.2, the red-black nonlinear block Gauss-Seidel
    smoother, 2x2 restriction, bilinear prolongation, dense-Newton coarsest
    solve, the V-cycle, and the time steps of Sec. 3.1/3.2.
  * ``energy.py`` (numpy): the discrete energies F, script-F, tilde-F of
    Sec. 3 and the "-1" norm of App. A (periodic Poisson solve by FFT).
  * ``bruteforce.py`` (numpy): dense-Jacobian Newton on all 3mn unknowns.

Every function cites the passage of the paper it follows.  Parity status of
each part is in the module docstrings; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpfc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmpfc_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libmpfc_oracle_omp.so")


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc (plain -O2, no fast-math, no FMA contraction
    so the arithmetic follows the source order), once serial and once with OpenMP
    (the all-cores build: parallel loops over independent cells only, identical
    bits).  Returns the serial library's path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared"]
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            subprocess.run(base + extra + ["-o", lib, _SRC, "-lm"], check=True)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("h", ctypes.c_double), ("M", ctypes.c_double),
                ("eps", ctypes.c_double), ("beta", ctypes.c_double), ("s", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("newton", ctypes.c_int),
                ("coarse_cells", ctypes.c_int), ("omega", ctypes.c_double), ("model", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("res0", ctypes.c_double),
                ("res", ctypes.c_double)]


_lib = None
_lib_omp = None
_D = ctypes.POINTER(ctypes.c_double)


def _load(threaded: bool = False):
    """The serial library, or with `threaded` the OpenMP build of the same source."""
    global _lib, _lib_omp
    if threaded:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(ctypes.CDLL(_LIB_OMP))
            _lib_omp.orc_set_boundary(_load().orc_get_boundary())
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def threads(n: int = 0) -> int:
    """Sets the OpenMP build's thread count (n > 0) and returns the count it uses."""
    return int(_load(True).orc_set_threads(n))


def _declare(lib):
    """Argument types of the oracle library's entry points."""
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.POINTER(_Params)]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_levels.argtypes = [ctypes.c_void_p]
    lib.orc_set_state.argtypes = [ctypes.c_void_p, _D, _D, _D]
    lib.orc_get_state.argtypes = [ctypes.c_void_p, _D, _D, _D]
    lib.orc_get_u.argtypes = [ctypes.c_void_p, _D, _D, _D]
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, ctypes.POINTER(_Info), _D]
    lib.orc_solve.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double,
                              ctypes.c_int, _D, _D]
    lib.orc_laplacian.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
    lib.orc_apply_N.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_residual.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_double] + [_D] * 10
    lib.orc_source.argtypes = [ctypes.c_int, ctypes.POINTER(_Params), _D, _D, _D, _D, _D, _D]
    lib.orc_smooth.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double] + [_D] * 7
    lib.orc_restrict.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
    lib.orc_prolong_add.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
    lib.orc_cramer3.argtypes = [_D, _D, _D]
    lib.orc_gauss_solve.argtypes = [ctypes.c_int, _D, _D, _D]
    lib.orc_coarse_newton.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double] + [_D] * 7
    lib.orc_scheme_consts.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _D, _D, _D]
    lib.orc_num_levels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_set_boundary.argtypes = [ctypes.c_int]
    lib.orc_set_pinning.argtypes = [ctypes.c_void_p, _D, _D]
    lib.orc_apply_N_pinned.argtypes = lib.orc_apply_N.argtypes[:11] + [_D, _D, _D, _D]
    lib.orc_smooth_pinned.argtypes = lib.orc_smooth.argtypes + [_D]
    lib.orc_coarse_newton_pinned.argtypes = lib.orc_coarse_newton.argtypes + [_D]
    lib.orc_source_pinned.argtypes = [ctypes.c_int, ctypes.POINTER(_Params), _D, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    return lib


def _p(a):
    """Pointer to a C-contiguous float64 numpy array (None -> NULL)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_boundary(ny_neumann: bool) -> None:
    """Boundary rule of every following call: periodic (App. A, (A.8)-(A.9)), or with
    ny_neumann periodic in x and homogeneous Neumann in y ((A.7), Sec. 4.5)."""
    _load().orc_set_boundary(1 if ny_neumann else 0)
    if _lib_omp is not None:
        _lib_omp.orc_set_boundary(1 if ny_neumann else 0)


class boundary:
    """Context manager: the given boundary rule inside, periodic again on exit."""

    def __init__(self, ny_neumann: bool):
        self.ny = ny_neumann

    def __enter__(self):
        set_boundary(self.ny)
        return self

    def __exit__(self, *exc):
        set_boundary(False)
        return False


@dataclass
class Params:
    """Problem parameters (Sec. 3, App. B).  Arrays are shaped (n, m): row j, column i."""
    m: int
    n: int
    h: float
    M: float = 1.0
    eps: float = 0.025
    beta: float = 0.9
    s: float = 0.01
    nu1: int = 2
    nu2: int = 2
    newton: int = 1
    coarse_cells: int = 4
    omega: float = 0.8
    ny_neumann: int = 0   # 1: homogeneous Neumann in y (Sec. 4.5); applied by Solver around each call
    model: int = 0        # 0: MPFC (2); 1: PFC (1), d_t phi = M Delta mu

    def c_struct(self) -> _Params:
        return _Params(self.m, self.n, self.h, self.M, self.eps, self.beta, self.s, self.nu1, self.nu2,
                       self.newton, self.coarse_cells, self.omega, self.model)


def scheme_consts(p: Params, scheme: int):
    """(c, gam, theta) of the FAS operator N for scheme 1 (App. B.1) or 2 (App. B.2)."""
    lib = _load()
    c, g, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_scheme_consts(ctypes.byref(p.c_struct()), scheme, ctypes.byref(c), ctypes.byref(g), ctypes.byref(t))
    return c.value, g.value, t.value


def num_levels(m: int, n: int, coarse_cells: int = 4) -> int:
    return _load().orc_num_levels(m, n, coarse_cells)


def laplacian(f, h):
    """Five-point Delta_h with the current ghost rule (App. A; see set_boundary)."""
    f = _f64(f)
    out = np.empty_like(f)
    _load().orc_laplacian(f.shape[1], f.shape[0], h, _p(f), _p(out))
    return out


def apply_N(scheme, consts, h, phi, mu, kappa, phik=None, W=None):
    """N(u) of App. B.1/B.2 on one grid; W: pinning weight on the grid (Sec. 4.6)."""
    phi, mu, kappa = _f64(phi), _f64(mu), _f64(kappa)
    phik = _f64(phik) if phik is not None else np.zeros_like(phi)
    out = [np.empty_like(phi) for _ in range(3)]
    c, g, t = consts
    args = (scheme, c, g, t, phi.shape[1], phi.shape[0], h, _p(phi), _p(mu), _p(kappa), _p(phik))
    if W is None:
        _load().orc_apply_N(*args, *[_p(o) for o in out])
    else:
        _load().orc_apply_N_pinned(*args, _p(_f64(W)), *[_p(o) for o in out])
    return out


def residual(scheme, consts, h, u, S, phik=None, W=None):
    """r = S - N(u)."""
    if W is not None:
        N = apply_N(scheme, consts, h, *u, phik, W)
        return [_f64(a) - b for a, b in zip(S, N)]
    phi, mu, kappa = [_f64(x) for x in u]
    S1, S2, S3 = [_f64(x) for x in S]
    phik = _f64(phik) if phik is not None else np.zeros_like(phi)
    out = [np.empty_like(phi) for _ in range(3)]
    c, g, t = consts
    _load().orc_residual(scheme, c, g, t, phi.shape[1], phi.shape[0], h, _p(phi), _p(mu), _p(kappa), _p(S1),
                         _p(S2), _p(S3), _p(phik), *[_p(o) for o in out])
    return out


def source(scheme, p: Params, phik, phikm1, psik, W=None, phihat=None):
    """S of App. B.1 (scheme 1) or App. B.2 (scheme 2); with a pinning weight W and
    target phihat, the pinned scheme-2 source of Sec. 4.6."""
    phik, phikm1, psik = _f64(phik), _f64(phikm1), _f64(psik)
    out = [np.empty_like(phik) for _ in range(3)]
    if W is None:
        _load().orc_source(scheme, ctypes.byref(p.c_struct()), _p(phik), _p(phikm1), _p(psik), *[_p(o) for o in out])
    else:
        _load().orc_source_pinned(scheme, ctypes.byref(p.c_struct()), _p(phik), _p(phikm1), _p(psik), _p(_f64(W)),
                                  _p(_f64(phihat)), *[_p(o) for o in out])
    return out


def smooth(scheme, consts, h, u, S, phik=None, sweeps=1, newton=1, omega=0.8, W=None):
    """Red-black nonlinear block Gauss-Seidel sweeps (App. B), relaxed by omega; returns new u."""
    phi, mu, kappa = [_f64(x).copy() for x in u]
    S1, S2, S3 = [_f64(x) for x in S]
    phik = _f64(phik) if phik is not None else np.zeros_like(phi)
    c, g, t = consts
    args = (scheme, c, g, t, newton, omega, sweeps, phi.shape[1], phi.shape[0], h, _p(phi), _p(mu), _p(kappa), _p(S1),
            _p(S2), _p(S3), _p(phik))
    if W is None:
        _load().orc_smooth(*args)
    else:
        _load().orc_smooth_pinned(*args, _p(_f64(W)))
    return phi, mu, kappa


def restrict(fine):
    fine = _f64(fine)
    nc, mc = fine.shape[0] // 2, fine.shape[1] // 2
    out = np.empty((nc, mc))
    _load().orc_restrict(mc, nc, _p(fine), _p(out))
    return out


def prolong_add(coarse, fine):
    """Returns fine + P coarse (cell-centred bilinear)."""
    coarse = _f64(coarse)
    out = _f64(fine).copy()
    _load().orc_prolong_add(coarse.shape[1], coarse.shape[0], _p(coarse), _p(out))
    return out


def cramer3(A, r):
    A, r = _f64(A).reshape(9).copy(), _f64(r).copy()
    x = np.empty(3)
    _load().orc_cramer3(_p(A), _p(r), _p(x))
    return x


def coarse_newton(scheme, consts, h, u, S, phik=None, W=None):
    phi, mu, kappa = [_f64(x).copy() for x in u]
    S1, S2, S3 = [_f64(x) for x in S]
    phik = _f64(phik) if phik is not None else np.zeros_like(phi)
    c, g, t = consts
    args = (scheme, c, g, t, phi.shape[1], phi.shape[0], h, _p(phi), _p(mu), _p(kappa), _p(S1), _p(S2), _p(S3),
            _p(phik))
    if W is None:
        it = _load().orc_coarse_newton(*args)
    else:
        it = _load().orc_coarse_newton_pinned(*args, _p(_f64(W)))
    return (phi, mu, kappa), it


GUESS_PREV, GUESS_EXTRAP, GUESS_GIVEN = 0, 1, 2


class Solver:
    """Time stepper of Sec. 3.1 (scheme 1) / Sec. 3.2 (scheme 2) with the FAS solver."""

    def __init__(self, p: Params, threaded: bool = False):
        """threaded: run on the OpenMP build (all host cores unless threads() says
        otherwise); its results are bitwise those of the serial build."""
        self.p = p
        self._lib = _load(threaded)
        self._ctx = self._lib.orc_create(ctypes.byref(p.c_struct()))
        if not self._ctx:
            raise ValueError("invalid grid size")
        self.levels = self._lib.orc_levels(self._ctx)

    def __del__(self):
        if getattr(self, "_ctx", None):
            self._lib.orc_destroy(self._ctx)
            self._ctx = None

    def set_pinning(self, weight=None, target=None):
        """Pinning of Sec. 4.6 (scheme 2): weight W >= 0 and target phihat on the grid;
        weight None switches it off."""
        if weight is None:
            self._lib.orc_set_pinning(self._ctx, None, None)
        else:
            self._pin = (_f64(weight), _f64(target))
            self._lib.orc_set_pinning(self._ctx, _p(self._pin[0]), _p(self._pin[1]))

    def set_state(self, phi, phi_prev=None, psi=None):
        phi = _f64(phi)
        self._lib.orc_set_state(self._ctx, _p(phi), _p(_f64(phi_prev)) if phi_prev is not None else None,
                                _p(_f64(psi)) if psi is not None else None)

    def get_state(self):
        shp = (self.p.n, self.p.m)
        a, b, c = np.empty(shp), np.empty(shp), np.empty(shp)
        self._lib.orc_get_state(self._ctx, _p(a), _p(b), _p(c))
        return a, b, c

    def get_u(self):
        shp = (self.p.n, self.p.m)
        a, b, c = np.empty(shp), np.empty(shp), np.empty(shp)
        self._lib.orc_get_u(self._ctx, _p(a), _p(b), _p(c))
        return a, b, c

    def step(self, scheme, tol=1e-10, max_cycles=100, guess=GUESS_PREV, fixed_cycles=0, phi0=None):
        """One time step; returns dict(cycles, status, res0, res, hist)."""
        info = _Info()
        hist = np.zeros(max(max_cycles, fixed_cycles, 1))
        ph0 = _f64(phi0) if phi0 is not None else None
        with boundary(self.p.ny_neumann):
            st = self._lib.orc_step(self._ctx, scheme, guess, _p(ph0), tol, max_cycles, fixed_cycles,
                                    ctypes.byref(info), _p(hist))
        return dict(cycles=info.cycles, status=info.status, res0=info.res0, res=info.res,
                    hist=hist[:info.cycles].copy(), rc=st)

    def solve(self, scheme, u, S, phik=None, tol=1e-10, max_cycles=100):
        """V-cycles on N(u) = S from the given u; returns (u, cycles, res, hist)."""
        phi, mu, kappa = [_f64(x).copy() for x in u]
        S1, S2, S3 = [_f64(x) for x in S]
        hist = np.zeros(max(max_cycles, 1))
        res = ctypes.c_double()
        pk = _f64(phik) if phik is not None else None
        with boundary(self.p.ny_neumann):
            cyc = self._lib.orc_solve(self._ctx, scheme, _p(phi), _p(mu), _p(kappa), _p(S1), _p(S2), _p(S3),
                                      _p(pk), tol, max_cycles, _p(hist), ctypes.byref(res))
        return (phi, mu, kappa), cyc, res.value, hist[:cyc].copy()
