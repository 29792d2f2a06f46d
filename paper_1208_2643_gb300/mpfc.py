"""Python binding of libmpfc (argument marshalling only; every step runs in the CUDA library).

The names follow include/mpfc.h.  PyTorch supplies device memory (the workspace and
any field tensors) and the CUDA stream; the library never falls back to a CPU path:
if libmpfc.so cannot be loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

MPFC_OK = 0
MPFC_ERR_INVALID = -1
MPFC_ERR_WORKSPACE = -2
MPFC_ERR_CUDA = -3
MPFC_ERR_NOT_CONVERGED = -4
MPFC_ERR_DIVERGED = -5

MPFC_FP64 = 0
MPFC_FP32_INNER = 1

MPFC_LAUNCH_GRAPH = 0
MPFC_LAUNCH_STREAM = 1

MPFC_GUESS_PREV = 0
MPFC_GUESS_EXTRAP = 1
MPFC_GUESS_LEARNED = 2

MPFC_BC_PERIODIC = 0
MPFC_BC_NEUMANN_Y = 1

MPFC_MODEL_MPFC = 0
MPFC_MODEL_PFC = 1


class mpfc_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("h", ctypes.c_double), ("M", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("beta", ctypes.c_double), ("dt", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("coarsest", ctypes.c_int),
                ("omega", ctypes.c_double), ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("precision", ctypes.c_int), ("guess", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("bc", ctypes.c_int), ("pinning", ctypes.c_int), ("model", ctypes.c_int)]


class mpfc_step_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("res0", ctypes.c_double),
                ("res_final", ctypes.c_double)]


class mpfc_energy_t(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("pseudoF", ctypes.c_double), ("tildeF", ctypes.c_double),
                ("pinning", ctypes.c_double)]


_lib = None
_VP = ctypes.c_void_p


class MPFCError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libmpfc.so (building it first if needed); raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmpfc.so not found at {path}; run paper_1208_2643_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.mpfc_default_params.argtypes = [P(mpfc_params)]
    lib.mpfc_default_params.restype = None
    lib.mpfc_workspace_bytes.argtypes = [P(mpfc_params)]
    lib.mpfc_workspace_bytes.restype = ctypes.c_size_t
    lib.mpfc_create.argtypes = [P(mpfc_params), _VP, ctypes.c_size_t, _VP, P(_VP)]
    lib.mpfc_destroy.argtypes = [_VP]
    lib.mpfc_destroy.restype = None
    lib.mpfc_set_state.argtypes = [_VP, _VP, _VP, _VP]
    lib.mpfc_get_state.argtypes = [_VP, _VP, _VP, _VP]
    lib.mpfc_step.argtypes = [_VP, ctypes.c_int, ctypes.c_int, P(mpfc_step_info)]
    lib.mpfc_step_cycles.argtypes = [_VP, ctypes.c_int, ctypes.c_int, P(mpfc_step_info)]
    lib.mpfc_step_async.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
    lib.mpfc_records.argtypes = [_VP, P(mpfc_step_info), ctypes.c_int, P(ctypes.c_int)]
    lib.mpfc_probe_fp64_fma.argtypes = [_VP, _VP, P(ctypes.c_double)]
    lib.mpfc_probe_rcp.argtypes = [_VP, _VP, ctypes.c_int, _VP]
    lib.mpfc_set_launch_mode.argtypes = [_VP, ctypes.c_int]
    lib.mpfc_fp32_time_smooth.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    lib.mpfc_launch_counts.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.mpfc_set_launch_shape.argtypes = [_VP] + [ctypes.c_int] * 5
    lib.mpfc_set_transfer_split.argtypes = [_VP, ctypes.c_int]
    lib.mpfc_set_guess_gate.argtypes = [_VP, ctypes.c_double]
    lib.mpfc_set_fp32_sweep.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
    lib.mpfc_fp32_test_withhold_copy.argtypes = [ctypes.c_int, ctypes.c_longlong]
    lib.mpfc_op_learned_guess.argtypes = [_VP]
    lib.mpfc_guess_correction.argtypes = [_VP, _VP]
    lib.mpfc_batch_workspace_bytes.argtypes = [ctypes.c_int, P(mpfc_params)]
    lib.mpfc_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.mpfc_batch_create.argtypes = [ctypes.c_int, P(mpfc_params), _VP, ctypes.c_size_t, _VP, P(_VP)]
    lib.mpfc_batch_destroy.argtypes = [_VP]
    lib.mpfc_batch_destroy.restype = None
    lib.mpfc_batch_set_state.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP]
    lib.mpfc_batch_get_state.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP]
    lib.mpfc_batch_step.argtypes = [_VP, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)]
    lib.mpfc_batch_step_cycles.argtypes = [_VP, ctypes.c_int, ctypes.c_int, P(ctypes.c_int)]
    lib.mpfc_batch_levels.argtypes = [_VP]
    lib.mpfc_batch_set_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mpfc_batch_time_smooth.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_float)]
    lib.mpfc_mass.argtypes = [_VP, P(ctypes.c_double)]
    lib.mpfc_energy.argtypes = [_VP, P(mpfc_energy_t)]
    lib.mpfc_set_pinning.argtypes = [_VP, _VP, _VP]
    lib.mpfc_strerror.argtypes = [ctypes.c_int]
    lib.mpfc_strerror.restype = ctypes.c_char_p
    lib.mpfc_levels.argtypes = [_VP]
    lib.mpfc_level_size.argtypes = [_VP, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double)]
    lib.mpfc_op_source.argtypes = [_VP, ctypes.c_int] + [_VP] * 6
    lib.mpfc_op_smooth.argtypes = [_VP, ctypes.c_int, ctypes.c_int] + [_VP] * 7 + [ctypes.c_int]
    lib.mpfc_op_residual.argtypes = [_VP, ctypes.c_int, ctypes.c_int] + [_VP] * 10
    lib.mpfc_op_restrict.argtypes = [_VP, ctypes.c_int, ctypes.c_int] + [_VP] * 14
    lib.mpfc_op_prolong.argtypes = [_VP, ctypes.c_int] + [_VP] * 9
    lib.mpfc_op_coarse_solve.argtypes = [_VP, ctypes.c_int] + [_VP] * 7
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load(build_if_missing=False).mpfc_strerror(status).decode()
    except Exception:
        return f"status {status}"


def _check(rc, where):
    if rc != MPFC_OK:
        raise MPFCError(rc, where)


def default_params(**kw) -> mpfc_params:
    p = mpfc_params()
    load().mpfc_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def workspace_bytes(p: mpfc_params) -> int:
    return int(load().mpfc_workspace_bytes(ctypes.byref(p)))


def _ptr(t):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.dtype == np.float64 and t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


class Solver:
    """One MPFC instance on the current CUDA device: workspace, state and stepping."""

    def __init__(self, params: mpfc_params | None = None, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmpfc needs a CUDA device")
        self._torch = torch
        self.lib = load()
        self.p = params if params is not None else default_params(**kw)
        nbytes = workspace_bytes(self.p)
        if nbytes == 0:
            raise MPFCError(MPFC_ERR_INVALID, "mpfc_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = _VP()
        _check(self.lib.mpfc_create(ctypes.byref(self.p), aligned, nbytes, self.stream.cuda_stream, ctypes.byref(h)),
               "mpfc_create")
        self.h = h
        self.shape = (self.p.n, self.p.m)
        self.levels = self.lib.mpfc_levels(self.h)

    def close(self):
        """Destroys the handle and releases its workspace once the work queued on the
        handle's stream has finished."""
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.mpfc_destroy(self.h)
            self.h = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_size(self, level):
        m, n, hl = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(self.lib.mpfc_level_size(self.h, level, ctypes.byref(m), ctypes.byref(n), ctypes.byref(hl)),
               "mpfc_level_size")
        return m.value, n.value, hl.value

    def _dev(self, a):
        torch = self._torch
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")
        return a.to(device="cuda", dtype=torch.float64).contiguous()

    def set_state(self, phi, phi_prev=None, psi=None):
        """Copies (phi^k, phi^{k-1}, psi^k) in; numpy arrays (host) or tensors (device)."""
        args = [phi, phi_prev, psi]
        keep = []
        ptrs = []
        for a in args:
            if a is None:
                ptrs.append(None)
            elif isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                ptrs.append(a.ctypes.data)
            else:
                a = a.contiguous()
                keep.append(a)
                ptrs.append(a.data_ptr())
        _check(self.lib.mpfc_set_state(self.h, *ptrs), "mpfc_set_state")
        self.stream.synchronize()

    def get_state(self, device=False):
        """Returns (phi^k, phi^{k-1}, psi^k) as numpy arrays (or device tensors)."""
        torch = self._torch
        if device:
            outs = [torch.empty(self.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
            _check(self.lib.mpfc_get_state(self.h, *[o.data_ptr() for o in outs]), "mpfc_get_state")
            return outs
        outs = [np.empty(self.shape) for _ in range(3)]
        _check(self.lib.mpfc_get_state(self.h, *[o.ctypes.data for o in outs]), "mpfc_get_state")
        return outs

    def step(self, scheme: int, nsteps: int = 1, raise_on_error=True):
        """Advances nsteps steps; returns a list of dicts (cycles, status, res0, res)."""
        infos = (mpfc_step_info * max(nsteps, 1))()
        rc = self.lib.mpfc_step(self.h, scheme, nsteps, infos)
        out = [dict(cycles=i.cycles, status=i.status, res0=i.res0, res=i.res_final) for i in infos[:nsteps]]
        if rc != MPFC_OK and raise_on_error:
            raise MPFCError(rc, "mpfc_step")
        return out if raise_on_error else (rc, out)

    def launch_counts(self, scheme: int):
        """(launches per FP64 step besides the V-cycles, launches per V-cycle)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.mpfc_launch_counts(self.h, scheme, ctypes.byref(a), ctypes.byref(b)), "mpfc_launch_counts")
        return a.value, b.value

    def fp32_time_smooth(self, level: int = 0, sweeps: int = 1) -> float:
        """Milliseconds of `sweeps` FP32 red-black sweeps of one level (mixed-precision handles)."""
        ms = ctypes.c_float()
        _check(self.lib.mpfc_fp32_time_smooth(self.h, level, sweeps, ctypes.byref(ms)), "mpfc_fp32_time_smooth")
        return ms.value

    def set_launch_mode(self, mode: int):
        _check(self.lib.mpfc_set_launch_mode(self.h, mode), "mpfc_set_launch_mode")

    def set_launch_shape(self, rows: int, small_cells: int, pdl_blocks: int, tail_cells: int = 0, tail_ctas: int = 1):
        """Block rows of large launches, the cell count below which launches use one-warp
        blocks, the largest grid launched with programmatic dependent launch, and the
        levels (at most tail_cells cells) run as one launch of tail_ctas CTAs."""
        _check(self.lib.mpfc_set_launch_shape(self.h, rows, small_cells, pdl_blocks, tail_cells, tail_ctas),
               "mpfc_set_launch_shape")

    def set_transfer_split(self, fine_cells: int):
        """FP64 grid transfers onto or from fine levels of at most fine_cells cells with four
        threads per coarse cell (restriction) and one per fine cell (prolongation)."""
        _check(self.lib.mpfc_set_transfer_split(self.h, fine_cells), "mpfc_set_transfer_split")

    def set_fp32_sweep(self, tile_rows: int, min_cells: int = 0):
        """Mixed-precision handles: inner sweeps as one launch over 64 x tile_rows tiles
        on levels of at least min_cells cells (tile_rows 0: two launches per sweep)."""
        _check(self.lib.mpfc_set_fp32_sweep(self.h, tile_rows, min_cells), "mpfc_set_fp32_sweep")

    def set_guess_gate(self, res0_threshold: float):
        """Learned guess: run the network only when the extrapolated guess's scaled
        residual is at least res0_threshold (0: on every step)."""
        _check(self.lib.mpfc_set_guess_gate(self.h, res0_threshold), "mpfc_set_guess_gate")

    def step_async(self, scheme: int, nsteps: int = 1):
        """Enqueues steps without synchronising (records via records())."""
        _check(self.lib.mpfc_step_async(self.h, scheme, nsteps), "mpfc_step_async")

    def records(self, max_records: int = 1024):
        """Synchronises and returns (status, records, count) of the steps since the last call."""
        infos = (mpfc_step_info * max(max_records, 1))()
        cnt = ctypes.c_int()
        rc = self.lib.mpfc_records(self.h, infos, max_records, ctypes.byref(cnt))
        n = min(cnt.value, max_records)
        return rc, [dict(cycles=i.cycles, status=i.status, res0=i.res0, res=i.res_final) for i in infos[:n]], cnt.value

    def step_cycles(self, scheme: int, ncycles: int):
        info = mpfc_step_info()
        _check(self.lib.mpfc_step_cycles(self.h, scheme, ncycles, ctypes.byref(info)), "mpfc_step_cycles")
        return dict(cycles=info.cycles, status=info.status, res0=info.res0, res=info.res_final)

    def mass(self) -> float:
        v = ctypes.c_double()
        _check(self.lib.mpfc_mass(self.h, ctypes.byref(v)), "mpfc_mass")
        return v.value

    def set_pinning(self, weight=None, target=None):
        """Pinning of Sec. 4.6 (scheme 2): weight W >= 0 and target phihat, (n, m) numpy
        arrays or device tensors; weight None switches it off."""
        if weight is None:
            _check(self.lib.mpfc_set_pinning(self.h, None, None), "mpfc_set_pinning")
            return
        import numpy as np
        keep = []
        ptrs = []
        for a in (weight, target):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                ptrs.append(a.ctypes.data)
            else:
                ptrs.append(_ptr(a))
        _check(self.lib.mpfc_set_pinning(self.h, ptrs[0], ptrs[1]), "mpfc_set_pinning")

    def energy(self):
        e = mpfc_energy_t()
        _check(self.lib.mpfc_energy(self.h, ctypes.byref(e)), "mpfc_energy")
        return dict(F=e.F, pseudoF=e.pseudoF, tildeF=e.tildeF, pinning=e.pinning)

    # component entry points (device tensors in and out)
    def op_source(self, scheme, phik, phikm1, psik):
        torch = self._torch
        S = [torch.empty(self.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        _check(self.lib.mpfc_op_source(self.h, scheme, _ptr(phik), _ptr(phikm1), _ptr(psik), *[_ptr(s) for s in S]),
               "mpfc_op_source")
        return S

    def op_smooth(self, scheme, level, u, S, phik=None, sweeps=1):
        u = [x.clone() for x in u]
        _check(self.lib.mpfc_op_smooth(self.h, scheme, level, *[_ptr(x) for x in u], *[_ptr(s) for s in S],
                                       _ptr(phik), sweeps), "mpfc_op_smooth")
        return u

    def op_residual(self, scheme, level, u, S, phik=None):
        torch = self._torch
        r = [torch.empty_like(u[0]) for _ in range(3)]
        _check(self.lib.mpfc_op_residual(self.h, scheme, level, *[_ptr(x) for x in u], *[_ptr(s) for s in S],
                                         _ptr(phik), *[_ptr(x) for x in r]), "mpfc_op_residual")
        return r

    def op_restrict(self, scheme, level, u, S, phik=None, phik_c=None):
        torch = self._torch
        m, n, _ = self.level_size(level + 1)
        uc = [torch.empty((n, m), dtype=torch.float64, device="cuda") for _ in range(3)]
        Sc = [torch.empty((n, m), dtype=torch.float64, device="cuda") for _ in range(3)]
        _check(self.lib.mpfc_op_restrict(self.h, scheme, level, *[_ptr(x) for x in u], *[_ptr(s) for s in S],
                                         _ptr(phik), _ptr(phik_c), *[_ptr(x) for x in uc], *[_ptr(x) for x in Sc]),
               "mpfc_op_restrict")
        return uc, Sc

    def op_prolong(self, level, uc_new, uc_old, u):
        u = [x.clone() for x in u]
        _check(self.lib.mpfc_op_prolong(self.h, level, *[_ptr(x) for x in uc_new], *[_ptr(x) for x in uc_old],
                                        *[_ptr(x) for x in u]), "mpfc_op_prolong")
        return u

    def op_coarse_solve(self, scheme, u, S, phik=None):
        u = [x.clone() for x in u]
        _check(self.lib.mpfc_op_coarse_solve(self.h, scheme, *[_ptr(x) for x in u], *[_ptr(s) for s in S],
                                             _ptr(phik)), "mpfc_op_coarse_solve")
        return u


def probe_fp64_tflops(stream=None) -> float:
    """Measured FP64 FMA rate of the current GPU (2 flops per FMA), in TFLOP/s."""
    import torch
    lib = load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    scratch = torch.empty(sms * 8 * 256, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(lib.mpfc_probe_fp64_fma(scratch.data_ptr(), st.cuda_stream, ctypes.byref(v)), "mpfc_probe_fp64_fma")
    return v.value


class BatchSolver:
    """Many independent instances advanced together (mpfc_batch_*)."""

    def __init__(self, params_list, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmpfc needs a CUDA device")
        self._torch = torch
        self.lib = load()
        self.count = len(params_list)
        self.params = (mpfc_params * self.count)(*params_list)
        nbytes = int(self.lib.mpfc_batch_workspace_bytes(self.count, self.params))
        if nbytes == 0:
            raise MPFCError(MPFC_ERR_INVALID, "mpfc_batch_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.workspace.data_ptr() + 255) & ~255
        h = _VP()
        _check(self.lib.mpfc_batch_create(self.count, self.params, aligned, nbytes, self.stream.cuda_stream,
                                          ctypes.byref(h)), "mpfc_batch_create")
        self.h = h
        self.levels = self.lib.mpfc_batch_levels(self.h)

    def close(self):
        """Destroys the handle and releases its workspace (as Solver.close)."""
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.mpfc_batch_destroy(self.h)
            self.h = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, inst, phi, phi_prev=None, psi=None):
        keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in (phi, phi_prev, psi)]
        _check(self.lib.mpfc_batch_set_state(self.h, inst, *[a.ctypes.data if a is not None else None for a in keep]),
               "mpfc_batch_set_state")
        self.stream.synchronize()

    def get_state(self, inst):
        p = self.params[inst]
        outs = [np.empty((p.n, p.m)) for _ in range(3)]
        _check(self.lib.mpfc_batch_get_state(self.h, inst, *[o.ctypes.data for o in outs]), "mpfc_batch_get_state")
        return outs

    def step(self, scheme, nsteps=1, raise_on_error=True):
        st = (ctypes.c_int * self.count)()
        cy = (ctypes.c_int * self.count)()
        rc = self.lib.mpfc_batch_step(self.h, scheme, nsteps, st, cy)
        if rc != MPFC_OK and raise_on_error:
            raise MPFCError(rc, "mpfc_batch_step")
        return rc, list(st), list(cy)

    def step_cycles(self, scheme, ncycles):
        st = (ctypes.c_int * self.count)()
        rc = self.lib.mpfc_batch_step_cycles(self.h, scheme, ncycles, st)
        return rc, list(st)

    def set_tile(self, level, tx, ty):
        _check(self.lib.mpfc_batch_set_tile(self.h, level, tx, ty), "mpfc_batch_set_tile")

    def time_smooth(self, scheme, level, reps=5):
        ms = ctypes.c_float()
        _check(self.lib.mpfc_batch_time_smooth(self.h, scheme, level, reps, ctypes.byref(ms)), "mpfc_batch_time_smooth")
        return ms.value
