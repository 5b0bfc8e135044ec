"""GB300 solver for pressurized phase-field fracture (Heister & Wick, arXiv 1806.09924).

A thin ctypes binding over the C ABI of ``include/pff.h`` (libpff.so, built
in-tree by ``paper_1806_09924_gb300.build``).  The binding only marshals
arguments: every step of the hot path runs in the library's CUDA kernels.
Device buffers may be PyTorch CUDA tensors (their ``data_ptr()`` is passed),
host buffers are numpy arrays.  Importing the package fails loudly if the
library has not been built.

Module-level functions carry the C names (``pff_create_mesh`` ...); the
``Problem`` class wraps one handle with the same operations as methods.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpff.so")

PFF_OK = 0
PFF_ERR_INVALID_ARG = -1
PFF_ERR_OOM = -2
PFF_ERR_NOT_CONVERGED = -3
PFF_ERR_NAN = -6
PFF_ERR_CUDA = -8
PFF_ERR_CAPACITY = -9
PFF_PREC_FP64 = 0
PFF_PREC_MIXED = 1
PFF_APPLY_AUTO = 0
PFF_APPLY_ASSEMBLED = 1
PFF_APPLY_MATFREE = 2
PFF_PC_AMG = 0
PFF_PC_JACOBI = 1
PFF_PC_AMG_TRI = 2


class PffOptions(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("c", ctypes.c_double), ("tol_newton", ctypes.c_double),
        ("tol_step", ctypes.c_double), ("tol_linear", ctypes.c_double), ("max_newton", ctypes.c_int),
        ("max_halvings", ctypes.c_int), ("cycle_lock", ctypes.c_int), ("krylov_restart", ctypes.c_int),
        ("max_krylov", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("amg_theta", ctypes.c_double),
        ("amg_coarse_max", ctypes.c_int), ("apply_variant", ctypes.c_int), ("precond", ctypes.c_int),
        ("cheb_ratio", ctypes.c_double), ("tol_active", ctypes.c_double),
        ("atol_newton", ctypes.c_double), ("tol_change", ctypes.c_double),
        ("spmv_group", ctypes.c_int), ("amg_reuse", ctypes.c_int), ("amg_reuse_tol", ctypes.c_double),
        ("precond_overlap", ctypes.c_int), ("cheb_degree_coarse", ctypes.c_int),
        ("forcing_max", ctypes.c_double), ("iter_graph", ctypes.c_int),
        ("amg_rebuild_phi", ctypes.c_double), ("amg_age_phi", ctypes.c_int),
        ("amg_levels_phi", ctypes.c_int), ("cheb_degree_phi", ctypes.c_int),
        ("amg_rotations", ctypes.c_int),
    ]


class PffStepReport(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("converged", ctypes.c_int), ("newton_its", ctypes.c_int),
        ("krylov_its", ctypes.c_int), ("krylov_its_max", ctypes.c_int), ("active", ctypes.c_int),
        ("changed", ctypes.c_int), ("locked", ctypes.c_int), ("ties", ctypes.c_int),
        ("linesearch_fails", ctypes.c_int), ("rho0", ctypes.c_double), ("rho", ctypes.c_double),
        ("time_ms", ctypes.c_double), ("amg_builds_u", ctypes.c_int), ("amg_builds_phi", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PffRequest(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n_cells", ctypes.c_int32 * 3),
        ("axis_coords", ctypes.POINTER(ctypes.c_double) * 3),
        ("E", ctypes.c_double), ("nu", ctypes.c_double), ("Gc", ctypes.c_double),
        ("kappa", ctypes.c_double), ("eps", ctypes.c_double), ("l0", ctypes.c_double),
        ("n_steps", ctypes.c_int), ("schedule", ctypes.POINTER(ctypes.c_double)),
        ("n_cod", ctypes.c_int), ("cod_x", ctypes.POINTER(ctypes.c_double)),
        ("keep_solution", ctypes.c_int), ("reserved", ctypes.c_int),
    ]


class PffRequestResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("done", ctypes.c_int), ("newton_its", ctypes.c_int),
        ("krylov_its", ctypes.c_int), ("converged_steps", ctypes.c_int), ("reserved", ctypes.c_int),
        ("n_dofs", ctypes.c_int64), ("bytes", ctypes.c_int64), ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double), ("tcv", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class PffServerStats(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64),
        ("peak_reserved_bytes", ctypes.c_int64), ("queued", ctypes.c_int), ("running", ctypes.c_int),
        ("finished", ctypes.c_int), ("max_running", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PffError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pff error {code}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "pff_default_options": (None, [ctypes.POINTER(PffOptions)]),
    "pff_check_options": (ctypes.c_int, [ctypes.POINTER(PffOptions)]),
    "pff_create_mesh": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(_D), ctypes.POINTER(_P)]),
    "pff_set_material": (ctypes.c_int, [_P] + [ctypes.c_double] * 5),
    "pff_set_pressure": (ctypes.c_int, [_P, ctypes.c_double]),
    "pff_set_crack": (ctypes.c_int, [_P, ctypes.c_double]),
    "pff_set_state": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "pff_newton_step": (ctypes.c_int, [_P, ctypes.POINTER(PffOptions), ctypes.POINTER(PffStepReport)]),
    "pff_end_loading_step": (ctypes.c_int, [_P]),
    "pff_solve_loading_steps": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(PffOptions),
                                               ctypes.POINTER(PffStepReport)]),
    "pff_eval_tcv_cod": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "pff_get_solution": (ctypes.c_int, [_P, _P, _P, _P]),
    "pff_set_stream": (ctypes.c_int, [_P, _P]),
    "pff_get_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "pff_destroy": (None, [_P]),
    "pff_last_error": (ctypes.c_char_p, []),
    "pff_residual_dev": (ctypes.c_int, [_P, _P]),
    "pff_active_set_dev": (ctypes.c_int, [_P, ctypes.c_double, _P, _P]),
    "pff_assemble": (ctypes.c_int, [_P]),
    "pff_apply_jacobian_dev": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "pff_precond_setup": (ctypes.c_int, [_P, ctypes.POINTER(PffOptions)]),
    "pff_precond_apply_dev": (ctypes.c_int, [_P, _P, _P]),
    "pff_linear_solve_dev": (ctypes.c_int, [_P, ctypes.POINTER(PffOptions), _P, _P,
                                            ctypes.POINTER(ctypes.c_int)]),
    "pff_set_state_dev": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "pff_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "pff_profile_select": (ctypes.c_int, [ctypes.c_char_p]),
    "pff_profile_report": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
    "pff_launch_count": (ctypes.c_longlong, []),
    "pff_eval_tcv_cod_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "pff_cell_indicators_dev": (ctypes.c_int, [_P, _P]),
    "pff_refine_axes": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_D)]),
    "pff_transfer_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "pff_mark_axes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_D),
                                     ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(_D)]),
    "pff_batch_solve": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(_D), ctypes.POINTER(PffOptions),
                                       ctypes.POINTER(ctypes.POINTER(PffStepReport)), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "pff_request_bytes": (ctypes.c_int64, [ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]),
    "pff_server_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(PffOptions),
                                         ctypes.POINTER(_P)]),
    "pff_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(PffRequest), ctypes.POINTER(ctypes.c_int64)]),
    "pff_server_result": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(PffRequestResult)]),
    "pff_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double,
                                       ctypes.POINTER(PffRequestResult)]),
    "pff_server_cod": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    "pff_server_solution": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
    "pff_server_release": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pff_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(PffServerStats)]),
    "pff_server_destroy": (None, [_P]),
    "pff_memory_usage": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.c_int]),
}

PFF_NOALLOC_MAX_POINTS = 1024
PFF_FIELD_U, PFF_FIELD_PHI, PFF_FIELD_PHI_OLD, PFF_FIELD_PHI_PREV = 1, 2, 4, 8
PFF_FIELD_ALL = 15

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpff.so (raises if it has not been built) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_1806_09924_gb300/build.py`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PFF_OK:
        raise PffError(rc, load_library().pff_last_error().decode(errors="replace"))


def options(**kw) -> PffOptions:
    """Solver options: library defaults overridden by keyword arguments."""
    o = PffOptions()
    load_library().pff_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def check_options(o: PffOptions) -> None:
    """pff_check_options: raises PffError naming the first out-of-range field."""
    _check(load_library().pff_check_options(ctypes.byref(o)))


def _host(a, dtype=np.float64):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def _dev(t, dtype_name: str, numel: int):
    """Device pointer of a CUDA tensor (checked) or a raw integer address."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device buffers must be contiguous CUDA tensors")
    if str(t.dtype) != dtype_name:
        raise ValueError(f"expected {dtype_name}, got {t.dtype}")
    if t.numel() < numel:
        raise ValueError(f"buffer too small: {t.numel()} < {numel}")
    return ctypes.c_void_p(t.data_ptr())


class Problem:
    """One phase-field fracture problem on a tensor-product mesh (owns a pff_problem)."""

    def __init__(self, coords: Sequence[np.ndarray]):
        lib = load_library()
        self._lib = lib
        self.dim = len(coords)
        self._coords = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
        nc = (ctypes.c_int32 * self.dim)(*[len(c) - 1 for c in self._coords])
        ptrs = (_D * self.dim)(*[c.ctypes.data_as(_D) for c in self._coords])
        h = _P()
        _check(lib.pff_create_mesh(self.dim, nc, ptrs, ctypes.byref(h)))
        self._h = h
        d, nn, nd = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.pff_get_sizes(h, ctypes.byref(d), ctypes.byref(nn), ctypes.byref(nd)))
        self.n_nodes, self.n_dofs = nn.value, nd.value

    # ---- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.pff_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---- set-up
    def set_material(self, E, nu, Gc, kappa, eps):
        _check(self._lib.pff_set_material(self._h, E, nu, Gc, kappa, eps))

    def set_pressure(self, p):
        _check(self._lib.pff_set_pressure(self._h, p))

    def set_crack(self, l0):
        _check(self._lib.pff_set_crack(self._h, l0))

    def set_state(self, u=None, phi=None, phi_old=None, phi_prev=None, steps_done=0):
        bufs = [_host(a) for a in (u, phi, phi_old, phi_prev)]
        _check(self._lib.pff_set_state(self._h, *[b[1] for b in bufs], int(steps_done)))

    def set_state_dev(self, u=None, phi=None, phi_old=None, phi_prev=None, steps_done=0):
        n = self.n_nodes
        _check(self._lib.pff_set_state_dev(self._h, _dev(u, "torch.float64", n * self.dim),
                                           _dev(phi, "torch.float64", n), _dev(phi_old, "torch.float64", n),
                                           _dev(phi_prev, "torch.float64", n), int(steps_done)))

    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", None)
        _check(self._lib.pff_set_stream(self._h, ctypes.c_void_p(ptr)))

    # ---- solver
    def newton_step(self, opts: Optional[PffOptions] = None) -> dict:
        r = PffStepReport()
        o = opts if opts is not None else options()
        rc = self._lib.pff_newton_step(self._h, ctypes.byref(o), ctypes.byref(r))
        _check(rc)
        return r.as_dict()

    def end_loading_step(self):
        _check(self._lib.pff_end_loading_step(self._h))

    def solve_loading_steps(self, pressures, opts: Optional[PffOptions] = None,
                            raise_on_error: bool = True) -> List[dict]:
        p, pp = _host(pressures)
        n = len(p)
        reps = (PffStepReport * max(n, 1))()
        o = opts if opts is not None else options()
        rc = self._lib.pff_solve_loading_steps(self._h, n, pp, ctypes.byref(o), reps)
        if raise_on_error:
            _check(rc)
        return [reps[i].as_dict() for i in range(n)]

    def eval_tcv_cod(self, pts=()):
        pts_arr, pptr = _host(np.asarray(pts, dtype=np.float64).reshape(-1))
        npts = pts_arr.size // (self.dim - 1)
        tcv = ctypes.c_double()
        cod = np.zeros(max(npts, 1))
        _check(self._lib.pff_eval_tcv_cod(self._h, npts, pptr, ctypes.byref(tcv),
                                          cod.ctypes.data_as(ctypes.c_void_p)))
        return tcv.value, cod[:npts]

    def eval_tcv_cod_noalloc(self, pts=()):
        """pff_eval_tcv_cod without device allocation (fixed scratch, at most
        PFF_NOALLOC_MAX_POINTS points)."""
        pts_arr, pptr = _host(np.asarray(pts, dtype=np.float64).reshape(-1))
        npts = pts_arr.size // (self.dim - 1)
        tcv = ctypes.c_double()
        cod = np.zeros(max(npts, 1))
        _check(self._lib.pff_eval_tcv_cod_noalloc(self._h, npts, pptr, ctypes.byref(tcv),
                                                  cod.ctypes.data_as(ctypes.c_void_p)))
        return tcv.value, cod[:npts]

    def get_solution(self):
        u = np.empty((self.n_nodes, self.dim))
        phi = np.empty(self.n_nodes)
        act = np.empty(self.n_nodes, dtype=np.uint8)
        _check(self._lib.pff_get_solution(self._h, u.ctypes.data_as(ctypes.c_void_p),
                                          phi.ctypes.data_as(ctypes.c_void_p),
                                          act.ctypes.data_as(ctypes.c_void_p)))
        return u, phi, act

    # ---- adaptive refinement
    @property
    def coords(self):
        return [c.copy() for c in self._coords]

    @property
    def n_cells(self) -> int:
        return int(np.prod([len(c) - 1 for c in self._coords]))

    def cell_indicators_dev(self, eta2):
        _check(self._lib.pff_cell_indicators_dev(self._h, _dev(eta2, "torch.float64", self.n_cells)))

    def refine_axes(self, theta, h_band, phi_band):
        """pff_refine_axes: the refined axis coordinates (the problem is unchanged)."""
        outs = [np.empty(2 * (len(c) - 1) + 1) for c in self._coords]
        ptrs = (_D * self.dim)(*[o.ctypes.data_as(_D) for o in outs])
        nc = (ctypes.c_int32 * self.dim)()
        _check(self._lib.pff_refine_axes(self._h, float(theta), float(h_band), float(phi_band), nc, ptrs))
        return [outs[a][:nc[a] + 1].copy() for a in range(self.dim)]

    def transfer_state(self, dst: "Problem", fields: int = PFF_FIELD_ALL):
        """pff_transfer_state: interpolate this problem's fields onto dst's nodes."""
        _check(self._lib.pff_transfer_state(self._h, dst._h, int(fields)))

    # ---- component entry points (device buffers)
    def residual_dev(self, F):
        _check(self._lib.pff_residual_dev(self._h, _dev(F, "torch.float64", self.n_dofs)))

    def active_set_dev(self, c=1.0, active=None, indicator=None):
        _check(self._lib.pff_active_set_dev(self._h, c, _dev(active, "torch.uint8", self.n_nodes),
                                            _dev(indicator, "torch.float64", self.n_nodes)))

    def assemble(self):
        _check(self._lib.pff_assemble(self._h))

    def apply_jacobian_dev(self, variant, x, y):
        _check(self._lib.pff_apply_jacobian_dev(self._h, variant, _dev(x, "torch.float64", self.n_dofs),
                                                _dev(y, "torch.float64", self.n_dofs)))

    def precond_setup(self, opts: Optional[PffOptions] = None):
        o = opts if opts is not None else options()
        _check(self._lib.pff_precond_setup(self._h, ctypes.byref(o)))

    def precond_apply_dev(self, r, z):
        _check(self._lib.pff_precond_apply_dev(self._h, _dev(r, "torch.float64", self.n_dofs),
                                               _dev(z, "torch.float64", self.n_dofs)))

    def linear_solve_dev(self, b, x, opts: Optional[PffOptions] = None) -> int:
        o = opts if opts is not None else options()
        it = ctypes.c_int()
        _check(self._lib.pff_linear_solve_dev(self._h, ctypes.byref(o), _dev(b, "torch.float64", self.n_dofs),
                                              _dev(x, "torch.float64", self.n_dofs), ctypes.byref(it)))
        return it.value


def profile_enable(on: bool = True):
    """Enable / disable per-kernel event timing (resets the totals)."""
    _check(load_library().pff_profile_enable(1 if on else 0))


def profile_select(name=None):
    """Time only launches of kernel `name` (None: all instrumented launches)."""
    _check(load_library().pff_profile_select(name.encode() if name else None))


def profile_report() -> dict:
    """Per-kernel {"count", "ms", "bytes"} totals since profile_enable."""
    import json
    lib = load_library()
    need = lib.pff_profile_report(None, 0)
    buf = ctypes.create_string_buffer(need + 16)
    lib.pff_profile_report(buf, need + 16)
    return json.loads(buf.value.decode())


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(load_library().pff_launch_count())


def batch_solve(problems, schedules, opts: Optional[PffOptions] = None, workers: int = 0):
    """Solve independent problems concurrently (pff_batch_solve).

    Returns (reports, status): reports[i] is the list of step-report dicts of
    problems[i], status[i] its return code."""
    lib = load_library()
    n = len(problems)
    o = opts if opts is not None else options()
    scheds = [np.ascontiguousarray(s, dtype=np.float64).reshape(-1) for s in schedules]
    reps = [(PffStepReport * max(len(s), 1))() for s in scheds]
    handles = (_P * max(n, 1))(*[p.handle for p in problems])
    steps = (ctypes.c_int * max(n, 1))(*[len(s) for s in scheds])
    sp = (_D * max(n, 1))(*[s.ctypes.data_as(_D) for s in scheds])
    rp = (ctypes.POINTER(PffStepReport) * max(n, 1))(
        *[ctypes.cast(r, ctypes.POINTER(PffStepReport)) for r in reps])
    st = (ctypes.c_int * max(n, 1))()
    lib.pff_batch_solve(n, handles, steps, sp, ctypes.byref(o), rp, int(workers), st)
    return ([[reps[i][k].as_dict() for k in range(len(scheds[i]))] for i in range(n)],
            [st[i] for i in range(n)])


def mark_axes(coords, slab_eta2, slab_minphi, theta, h_band, phi_band):
    """pff_mark_axes: refined axis coordinates from host slab sums and minima (no device)."""
    lib = load_library()
    dim = len(coords)
    xs = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
    ss = [np.ascontiguousarray(v, dtype=np.float64) for v in slab_eta2]
    ms = [np.ascontiguousarray(v, dtype=np.float64) for v in slab_minphi]
    for x, sv, mv in zip(xs, ss, ms):
        if sv.size != x.size - 1 or mv.size != x.size - 1:
            raise ValueError("slab arrays need one value per interval")
    outs = [np.empty(2 * (x.size - 1) + 1) for x in xs]
    nc = (ctypes.c_int32 * dim)(*[x.size - 1 for x in xs])
    arr = lambda lst: (_D * dim)(*[v.ctypes.data_as(_D) for v in lst])  # noqa: E731
    nout = (ctypes.c_int32 * dim)()
    _check(lib.pff_mark_axes(dim, nc, arr(xs), arr(ss), arr(ms), float(theta), float(h_band),
                             float(phi_band), nout, arr(outs)))
    return [outs[a][:nout[a] + 1].copy() for a in range(dim)]


def memory_usage(reset_peak: bool = False):
    """(current, peak) device bytes held by the library (all problems)."""
    cur, peak = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().pff_memory_usage(ctypes.byref(cur), ctypes.byref(peak), 1 if reset_peak else 0))
    return cur.value, peak.value


def request_bytes(dim: int, n_cells) -> int:
    """Device bytes the server's admission test reserves for a problem of this size."""
    nc = (ctypes.c_int32 * 3)(*(list(n_cells) + [1] * (3 - len(n_cells))))
    return int(load_library().pff_request_bytes(int(dim), nc))


class Server:
    """Continuous-batching request server (pff_server_*): a device-memory budget,
    worker threads with their own streams, FIFO admission."""

    def __init__(self, budget_bytes: int, workers: int, opts: Optional[PffOptions] = None):
        lib = load_library()
        self._lib = lib
        o = opts if opts is not None else options()
        h = _P()
        _check(lib.pff_server_create(int(budget_bytes), int(workers), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._meta = {}

    def submit(self, w, pressures=None, cod_x=(), keep_solution: bool = False) -> int:
        """Queue a request for ``workloads.Workload`` w (its mesh, material, crack and,
        unless given, its pressure schedule)."""
        coords = [np.ascontiguousarray(c, dtype=np.float64) for c in w.coords]
        sched = np.ascontiguousarray(w.pressures if pressures is None else pressures, dtype=np.float64)
        cx = np.ascontiguousarray(cod_x, dtype=np.float64).reshape(-1)
        r = PffRequest()
        r.dim = w.dim
        for a in range(w.dim):
            r.n_cells[a] = len(coords[a]) - 1
            r.axis_coords[a] = coords[a].ctypes.data_as(_D)
        r.E, r.nu, r.Gc, r.kappa, r.eps, r.l0 = w.E, w.nu, w.Gc, w.kappa, w.eps, w.l0
        r.n_steps = len(sched)
        r.schedule = sched.ctypes.data_as(_D)
        r.n_cod = len(cx)
        r.cod_x = cx.ctypes.data_as(_D)
        r.keep_solution = 1 if keep_solution else 0
        rid = ctypes.c_int64()
        _check(self._lib.pff_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        nn = int(np.prod([len(c) for c in coords]))
        self._meta[rid.value] = (w.dim, nn, len(cx))
        return rid.value

    def result(self, rid: int) -> dict:
        res = PffRequestResult()
        _check(self._lib.pff_server_result(self._h, rid, ctypes.byref(res)))
        return res.as_dict()

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        res = PffRequestResult()
        _check(self._lib.pff_server_wait(self._h, rid, float(timeout), ctypes.byref(res)))
        return res.as_dict()

    def cod(self, rid: int) -> np.ndarray:
        out = np.zeros(self._meta[rid][2])
        _check(self._lib.pff_server_cod(self._h, rid, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def solution(self, rid: int):
        d, nn, _ = self._meta[rid]
        u = np.zeros((nn, d))
        phi = np.zeros(nn)
        act = np.zeros(nn, dtype=np.uint8)
        _check(self._lib.pff_server_solution(self._h, rid, u.ctypes.data_as(ctypes.c_void_p),
                                             phi.ctypes.data_as(ctypes.c_void_p),
                                             act.ctypes.data_as(ctypes.c_void_p)))
        return u, phi, act

    def release(self, rid: int):
        _check(self._lib.pff_server_release(self._h, rid))
        self._meta.pop(rid, None)

    def stats(self) -> dict:
        st = PffServerStats()
        _check(self._lib.pff_server_stats_get(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pff_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def problem_from_workload(w, crack: bool = True) -> Problem:
    """Create a Problem for a ``workloads.Workload`` (mesh, material, crack)."""
    P = Problem(w.coords)
    P.set_material(w.E, w.nu, w.Gc, w.kappa, w.eps)
    if crack:
        P.set_crack(w.l0)
    return P


# C-named module-level aliases (argument marshalling only)
def pff_create_mesh(coords):
    return Problem(coords)


def pff_set_material(P, E, nu, Gc, kappa, eps):
    P.set_material(E, nu, Gc, kappa, eps)


def pff_set_pressure(P, p):
    P.set_pressure(p)


def pff_set_crack(P, l0):
    P.set_crack(l0)


def pff_newton_step(P, opts=None):
    return P.newton_step(opts)


def pff_solve_loading_steps(P, pressures, opts=None):
    return P.solve_loading_steps(pressures, opts)


def pff_eval_tcv_cod(P, pts):
    return P.eval_tcv_cod(pts)


def pff_get_solution(P):
    return P.get_solution()


def pff_destroy(P):
    P.close()


load_library()
