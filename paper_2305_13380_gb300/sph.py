"""Thin Python binding of the C ABI in ``include/sph.h`` (ctypes).

Argument marshalling only: every step of the SPH path runs in the CUDA
library ``_lib/libsph.so``.  Tensors are torch CUDA tensors (torch provides
the device memory and the stream); they must be contiguous with the dtypes the
header states.  If the library is missing the import of a function raises: no
part of the path has a CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from .build import LIB

SPH_OK = 0
SPH_E_INVAL = -1
SPH_E_NOMEM = -2
SPH_E_H_NOCONV = -3
SPH_E_REBUILD = -4
SPH_E_BOX = -5
SPH_E_TIMEOUT = -6
SPH_E_CUDA = -7
SPH_E_CAPACITY = -8

SPH_ST_H_NOCONV = 1
SPH_ST_REBUILD = 2
SPH_ST_BOX = 4
SPH_ST_CAPACITY = 8
SPH_ST_NEG_U = 16

SPH_FLAG_SYNC = 1
SPH_FLAG_COUNT_PAIRS = 2
SPH_FLAG_TIMING = 4
SPH_FLAG_TREE = 8
SPH_FLAG_AXIS_SORT = 16
SPH_FLAG_SYMMETRIC = 32
SPH_HIER_ADAPT = 1
SPH_HIER_WAKEUP = 2
SPH_HIER_PREDICT = 4
SPH_HIER_KEEP_CELLS = 8
SPH_KERNEL_CUBIC, SPH_KERNEL_QUARTIC, SPH_KERNEL_WENDLAND_C2 = 0, 1, 2

TIMING_GROUPS = ("build", "gather", "density", "force", "integrate")

_P = C.c_void_p


class sph_params(C.Structure):
    _fields_ = [("box_size", C.c_double), ("gamma", C.c_double), ("eta", C.c_double),
                ("alpha_v", C.c_double), ("beta_v", C.c_double), ("eps_balsara", C.c_double),
                ("h_tol", C.c_double), ("cfl", C.c_double), ("cell_margin", C.c_double),
                ("max_h_iter", C.c_int32), ("flags", C.c_int32), ("n_leaf", C.c_int32),
                ("kernel", C.c_int32), ("lanes_per_target", C.c_int32)]


class sph_cells(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_c", C.c_int32), ("n_c_dev", _P), ("cell_start", _P),
                ("perm", _P)]


class sph_particles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, _P) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")]


DENSITY_FIELDS = ("h", "rho", "f", "div_v", "curl_v", "P", "c", "balsara")


class sph_density_out(C.Structure):
    _fields_ = [(k, _P) for k in DENSITY_FIELDS + ("n_iter",)]


FORCE_FIELDS = ("ax", "ay", "az", "du_dt", "v_sig")


class sph_force_out(C.Structure):
    _fields_ = [(k, _P) for k in FORCE_FIELDS]


POOL_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h", "ax", "ay", "az", "du_dt", "v_sig",
               "rho", "f", "div_v", "curl_v", "P", "c", "balsara", "dt")


class sph_pool(C.Structure):
    _fields_ = [("n_sims", C.c_int32), ("n_total", C.c_int64), ("sim_offset", _P),
                ("box_size", _P)] + [(k, _P) for k in POOL_FIELDS] + [("n_iter", _P)]


class sph_sphenix_params(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("alpha_v_max", "ell", "beta_c", "alpha_c_min", "alpha_c_max")]


class sph_sphenix_state(C.Structure):
    _fields_ = [(k, _P) for k in ("alpha_v", "alpha_c", "div_v_prev", "v_sig", "lap_u")]


class SPHError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {error_string(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library {LIB} is missing: run __graft_entry__.build()")
        L = C.CDLL(LIB)
        L.sph_default_params.argtypes = [C.POINTER(sph_params)]
        L.sph_default_params.restype = None
        L.sph_create.argtypes = [C.POINTER(_P), C.POINTER(sph_params), _P]
        L.sph_destroy.argtypes = [_P]
        L.sph_destroy.restype = None
        L.sph_error_string.argtypes = [C.c_int]
        L.sph_error_string.restype = C.c_char_p
        L.sph_status.argtypes = [_P, C.POINTER(C.c_int32)]
        L.sph_build_cells.argtypes = [_P, C.c_int64, _P, _P, _P, _P, C.POINTER(sph_cells)]
        L.sph_cells_sync.argtypes = [_P, C.POINTER(sph_cells)]
        L.sph_cells_copy.argtypes = [_P, C.POINTER(sph_cells), _P, _P]
        L.sph_density.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles), _P,
                                  C.POINTER(sph_density_out)]
        L.sph_force.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles),
                                C.POINTER(sph_density_out), C.POINTER(sph_force_out)]
        L.sph_step.argtypes = [_P, C.POINTER(sph_pool)]
        L.sph_hier_substep.argtypes = [_P, C.POINTER(sph_pool), _P, _P, C.c_double, C.c_int32, C.c_int64,
                                       C.c_int32, _P, C.POINTER(C.c_int64)]
        L.sph_hier_substep_dev.argtypes = [_P, C.POINTER(sph_pool), _P, _P, C.c_double, C.c_int32, _P,
                                           C.c_int32, _P]
        L.sph_time_bins.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles),
                                    C.POINTER(sph_density_out), _P, C.c_double, C.c_double, C.c_int32, _P]
        L.sph_density_active.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles), _P, _P,
                                         C.POINTER(sph_density_out)]
        L.sph_force_active.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles),
                                       C.POINTER(sph_density_out), _P, C.POINTER(sph_force_out)]
        L.sph_sphenix_default_params.restype = None
        L.sph_sphenix_default_params.argtypes = [C.POINTER(sph_sphenix_params)]
        L.sph_sphenix_gradient.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles),
                                           C.POINTER(sph_density_out), C.POINTER(sph_sphenix_params),
                                           C.c_double, C.POINTER(sph_sphenix_state)]
        L.sph_force_sphenix.argtypes = [_P, C.POINTER(sph_cells), C.POINTER(sph_particles),
                                        C.POINTER(sph_density_out), _P, _P, C.POINTER(sph_force_out)]
        L.sph_step_sphenix.argtypes = [_P, C.POINTER(sph_pool), C.POINTER(sph_sphenix_params), _P, _P]
        L.sph_conservation.argtypes = [_P, C.POINTER(sph_pool), _P]
        L.sph_pair_counts.argtypes = [_P, C.POINTER(C.c_int64)]
        L.sph_kernel_times.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.sph_build_cells_static.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_double, C.c_double,
                                             _P, C.c_int64, _P, _P, _P, _P]
        L.sph_reserve.argtypes = [_P, C.c_int64, C.c_int32]
        L.sph_tree_counts.argtypes = [_P, C.POINTER(C.c_int64)]
        L.sph_fof.argtypes = [_P, C.c_int64, _P, _P, _P, C.c_double, _P]
        L.sph_pool_move.argtypes = [C.POINTER(sph_pool), C.POINTER(sph_pool), C.c_int32, _P, _P, C.c_int32,
                                    _P]
        for f in ("sph_create", "sph_status", "sph_build_cells", "sph_cells_sync", "sph_cells_copy",
                  "sph_density",
                  "sph_force", "sph_step", "sph_conservation", "sph_pair_counts",
                  "sph_kernel_times", "sph_build_cells_static", "sph_reserve", "sph_tree_counts",
                  "sph_pool_move", "sph_fof"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().sph_error_string(int(code)).decode()


def _check(rc: int, what: str):
    if rc != SPH_OK:
        raise SPHError(rc, what)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return _P(t.data_ptr())


def sph_default_params(**overrides) -> sph_params:
    p = sph_params()
    lib().sph_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Context:
    """Owns an ``sph_ctx`` bound to a CUDA stream (torch's current one by default)."""

    def __init__(self, params: sph_params | None = None, stream: torch.cuda.Stream | None = None):
        self.params = params if params is not None else sph_default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _P()
        _check(lib().sph_create(C.byref(h), C.byref(self.params), _P(self.stream.cuda_stream)),
               "sph_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().sph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sph_create(params: sph_params | None = None, stream=None) -> Context:
    return Context(params, stream)


def sph_destroy(ctx: Context):
    ctx.close()


def sph_status(ctx: Context) -> int:
    s = C.c_int32(0)
    _check(lib().sph_status(ctx.handle, C.byref(s)), "sph_status")
    return s.value


def sph_build_cells(ctx: Context, x, y, z, h) -> sph_cells:
    cells = sph_cells()
    n = int(x.shape[0])
    _check(lib().sph_build_cells(ctx.handle, n, _ptr(x, torch.float64), _ptr(y, torch.float64),
                                 _ptr(z, torch.float64), _ptr(h, torch.float32), C.byref(cells)),
           "sph_build_cells")
    cells._keep = (x, y, z, h)
    return cells


def sph_fof(ctx: Context, x, y, z, link_len: float, group=None):
    """Friends-of-friends groups (int32 CUDA tensor): group[i] = the smallest
    index of i's group, friends closer than link_len (minimum image in the
    context's periodic box)."""
    n = int(x.shape[0])
    if group is None:
        group = torch.empty(n, dtype=torch.int32, device=x.device)
    _check(lib().sph_fof(ctx.handle, n, _ptr(x, torch.float64), _ptr(y, torch.float64),
                         _ptr(z, torch.float64), float(link_len), _ptr(group, torch.int32)), "sph_fof")
    return group


def sph_cells_sync(ctx: Context, cells: sph_cells) -> int:
    _check(lib().sph_cells_sync(ctx.handle, C.byref(cells)), "sph_cells_sync")
    return cells.n_c


def sph_cells_copy(ctx: Context, cells: sph_cells):
    """Host copies (numpy int32) of cell_start (n_c^3 + 1) and perm (n)."""
    import numpy as np
    sph_cells_sync(ctx, cells)
    nc = cells.n_c
    cs = np.zeros(nc ** 3 + 1, dtype=np.int32)
    perm = np.zeros(max(int(cells.n), 1), dtype=np.int32)
    _check(lib().sph_cells_copy(ctx.handle, C.byref(cells), cs.ctypes.data_as(_P),
                                perm.ctypes.data_as(_P)), "sph_cells_copy")
    return cs, perm[:int(cells.n)]


def particles(p: dict) -> sph_particles:
    """Marshals a dict of CUDA tensors x, y, z (float64) and vx, vy, vz, m, u (float32)."""
    s = sph_particles(int(p["x"].shape[0]), *(
        [_ptr(p[k], torch.float64) for k in ("x", "y", "z")] +
        [_ptr(p[k], torch.float32) for k in ("vx", "vy", "vz", "m", "u")]))
    s._keep = p
    return s


def density_out(d: dict) -> sph_density_out:
    s = sph_density_out(*([_ptr(d[k], torch.float32) for k in DENSITY_FIELDS] +
                          [_ptr(d.get("n_iter"), torch.int32)]))
    s._keep = d
    return s


def force_out(f: dict) -> sph_force_out:
    s = sph_force_out(*[_ptr(f[k], torch.float32) for k in FORCE_FIELDS])
    s._keep = f
    return s


def sph_density(ctx: Context, cells: sph_cells, part: sph_particles, h_in, out: sph_density_out):
    _check(lib().sph_density(ctx.handle, C.byref(cells), C.byref(part), _ptr(h_in, torch.float32),
                             C.byref(out)), "sph_density")


def sph_force(ctx: Context, cells: sph_cells, part: sph_particles, dens: sph_density_out,
              out: sph_force_out):
    _check(lib().sph_force(ctx.handle, C.byref(cells), C.byref(part), C.byref(dens),
                           C.byref(out)), "sph_force")


def sph_hier_substep_dev(ctx: Context, pl: sph_pool, bins, t_begin, dt_max: float, max_bin: int, tick,
                         adapt: bool = True, wakeup: bool = False, sync=None, predict: bool = False) -> None:
    """One sub-step with the tick in a device int64 tensor (read, then
    replaced by the next tick); waits for nothing, so it can be captured in a
    CUDA graph."""
    opts = (SPH_HIER_ADAPT if adapt else 0) | (SPH_HIER_WAKEUP if wakeup else 0) | \
        (SPH_HIER_PREDICT if predict else 0)
    _check(lib().sph_hier_substep_dev(ctx.handle, C.byref(pl), _ptr(bins, torch.int32), _ptr(t_begin, torch.int64),
                                      C.c_double(dt_max), C.c_int32(max_bin), _ptr(tick, torch.int64),
                                      C.c_int32(opts), None if sync is None else _ptr(sync, torch.uint8)),
           "sph_hier_substep_dev")


def sph_hier_substep(ctx: Context, pl: sph_pool, bins, t_begin, dt_max: float, max_bin: int, t_now: int,
                     adapt: bool = True, wakeup: bool = False, sync=None, predict: bool = False,
                     keep_cells: bool = False) -> int:
    """One sub-step of the time-step hierarchy; returns the new tick.  sync is
    an optional uint8 device tensor of flags (cleared by the call)."""
    t_next = C.c_int64(0)
    opts = (SPH_HIER_ADAPT if adapt else 0) | (SPH_HIER_WAKEUP if wakeup else 0) | \
        (SPH_HIER_PREDICT if predict else 0) | (SPH_HIER_KEEP_CELLS if keep_cells else 0)
    _check(lib().sph_hier_substep(ctx.handle, C.byref(pl), _ptr(bins, torch.int32), _ptr(t_begin, torch.int64),
                                  C.c_double(dt_max), C.c_int32(max_bin), C.c_int64(t_now), C.c_int32(opts),
                                  None if sync is None else _ptr(sync, torch.uint8), C.byref(t_next)),
           "sph_hier_substep")
    return int(t_next.value)


def sph_time_bins(ctx: Context, cells: sph_cells, part: sph_particles, dens: sph_density_out, v_sig,
                  cfl: float, dt_max: float, max_bin: int, bins):
    """Time bins with the first limiter into ``bins`` (int32 CUDA tensor)."""
    _check(lib().sph_time_bins(ctx.handle, C.byref(cells), C.byref(part), C.byref(dens),
                               _ptr(v_sig, torch.float32), C.c_double(cfl), C.c_double(dt_max),
                               C.c_int32(max_bin), _ptr(bins, torch.int32)), "sph_time_bins")


def sph_density_active(ctx: Context, cells: sph_cells, part: sph_particles, h_in, active,
                       out: sph_density_out):
    """sph_density on the particles whose uint8 ``active`` entry is nonzero."""
    _check(lib().sph_density_active(ctx.handle, C.byref(cells), C.byref(part), _ptr(h_in, torch.float32),
                                    _ptr(active, torch.uint8), C.byref(out)), "sph_density_active")


def sph_force_active(ctx: Context, cells: sph_cells, part: sph_particles, dens: sph_density_out, active,
                     out: sph_force_out):
    """sph_force on the particles whose uint8 ``active`` entry is nonzero."""
    _check(lib().sph_force_active(ctx.handle, C.byref(cells), C.byref(part), C.byref(dens),
                                  _ptr(active, torch.uint8), C.byref(out)), "sph_force_active")


def pool(sim_offset, box_size, arrays: dict) -> sph_pool:
    """Marshals a pool of simulations: sim_offset (int64, n_sims+1), box_size
    (float64, n_sims) and the per-particle arrays of ``POOL_FIELDS`` (dt is a
    float64 array of n_sims)."""
    n_sims = int(box_size.shape[0])
    vals = []
    for k in POOL_FIELDS:
        dt = torch.float64 if k in ("x", "y", "z", "dt") else torch.float32
        vals.append(_ptr(arrays[k], dt))
    s = sph_pool(n_sims, int(arrays["x"].shape[0]), _ptr(sim_offset, torch.int64),
                 _ptr(box_size, torch.float64), *vals, _ptr(arrays.get("n_iter"), torch.int32))
    s._keep = (sim_offset, box_size, arrays)
    return s


def sph_pool_move(spread: sph_pool, packed: sph_pool, n_ranges: int, starts, offsets, to_packed: bool,
                  stream=None):
    """Moves whole simulations between a spread pool and a packed one
    (starts / offsets: int64 device tensors of n_ranges and n_ranges + 1)."""
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().sph_pool_move(C.byref(spread), C.byref(packed), int(n_ranges), _ptr(starts, torch.int64),
                               _ptr(offsets, torch.int64), 1 if to_packed else 0, C.c_void_p(st.cuda_stream)),
           "sph_pool_move")


def sph_tree_counts(ctx: Context) -> dict:
    """Nested-grid diagnostics of the last build and density."""
    v = (C.c_int64 * 4)()
    _check(lib().sph_tree_counts(ctx.handle, v), "sph_tree_counts")
    return {"groups": int(v[0]), "list_free_targets": int(v[1]), "reverse_pairs": int(v[2]),
            "fallback_targets": int(v[3])}


def sph_reserve(ctx: Context, n_total: int, n_sims: int = 1):
    """Allocates the context's scratch for n_total particles in n_sims
    simulations up front."""
    _check(lib().sph_reserve(ctx.handle, C.c_int64(n_total), C.c_int32(n_sims)), "sph_reserve")


def sph_step(ctx: Context, pl: sph_pool):
    _check(lib().sph_step(ctx.handle, C.byref(pl)), "sph_step")


def sph_sphenix_default_params(**overrides) -> sph_sphenix_params:
    x = sph_sphenix_params()
    lib().sph_sphenix_default_params(C.byref(x))
    for k, v in overrides.items():
        setattr(x, k, v)
    return x


def sphenix_state(alpha_v, alpha_c, div_v_prev, v_sig, lap_u=None) -> sph_sphenix_state:
    """Marshals the SPHENIX per-particle arrays (float32 CUDA tensors)."""
    f = torch.float32
    s = sph_sphenix_state(_ptr(alpha_v, f), _ptr(alpha_c, f), _ptr(div_v_prev, f), _ptr(v_sig, f),
                          _ptr(lap_u, f))
    s._keep = (alpha_v, alpha_c, div_v_prev, v_sig, lap_u)
    return s


def sph_sphenix_gradient(ctx: Context, cells: sph_cells, part: sph_particles, dens: sph_density_out,
                         x: sph_sphenix_params, dt: float, st: sph_sphenix_state):
    _check(lib().sph_sphenix_gradient(ctx.handle, C.byref(cells), C.byref(part), C.byref(dens),
                                      C.byref(x), C.c_double(dt), C.byref(st)), "sph_sphenix_gradient")


def sph_force_sphenix(ctx: Context, cells: sph_cells, part: sph_particles, dens: sph_density_out,
                      alpha_v, alpha_c, out: sph_force_out):
    f = torch.float32
    _check(lib().sph_force_sphenix(ctx.handle, C.byref(cells), C.byref(part), C.byref(dens),
                                   _ptr(alpha_v, f), _ptr(alpha_c, f), C.byref(out)), "sph_force_sphenix")


def sph_step_sphenix(ctx: Context, pl: sph_pool, x: sph_sphenix_params, alpha_v, alpha_c):
    f = torch.float32
    _check(lib().sph_step_sphenix(ctx.handle, C.byref(pl), C.byref(x), _ptr(alpha_v, f), _ptr(alpha_c, f)),
           "sph_step_sphenix")


def sph_conservation(ctx: Context, pl: sph_pool, out):
    _check(lib().sph_conservation(ctx.handle, C.byref(pl), _ptr(out, torch.float64)),
           "sph_conservation")


def sph_pair_counts(ctx: Context):
    v = (C.c_int64 * 2)()
    _check(lib().sph_pair_counts(ctx.handle, v), "sph_pair_counts")
    return int(v[0]), int(v[1])


def sph_kernel_times(ctx: Context):
    """{group: (milliseconds, launches)} since the last query (SPH_FLAG_TIMING)."""
    ms = (C.c_double * len(TIMING_GROUPS))()
    calls = (C.c_int64 * len(TIMING_GROUPS))()
    _check(lib().sph_kernel_times(ctx.handle, ms, calls), "sph_kernel_times")
    return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(TIMING_GROUPS)}


STATIC_MAX_N = 65536


def sph_build_cells_static(x, y, z, h, box_size: float, cell_margin: float, cell_start, perm,
                           n_c_out=None, status_out=None, stream=None):
    """The allocation-free cell build: every buffer is the caller's (CUDA
    tensors), the library's scratch is a fixed array inside the library."""
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().sph_build_cells_static(
        int(x.shape[0]), _ptr(x, torch.float64), _ptr(y, torch.float64), _ptr(z, torch.float64),
        _ptr(h, torch.float32), float(box_size), float(cell_margin), _ptr(cell_start, torch.int32),
        int(cell_start.shape[0]), _ptr(perm, torch.int32), _ptr(n_c_out, torch.int32),
        _ptr(status_out, torch.int32), _P(st.cuda_stream)), "sph_build_cells_static")


# ---- allocation helpers (marshalling of outputs) ----------------------------

def to_device(p: dict, device="cuda") -> dict:
    """Input dict of numpy arrays -> CUDA tensors with the ABI dtypes."""
    out = {}
    for k in ("x", "y", "z"):
        out[k] = torch.as_tensor(p[k], dtype=torch.float64, device=device).contiguous()
    for k in ("vx", "vy", "vz", "m", "u"):
        out[k] = torch.as_tensor(p[k], dtype=torch.float32, device=device).contiguous()
    out["h0"] = torch.as_tensor(p["h0"], dtype=torch.float32, device=device).contiguous()
    return out


def alloc_density(n: int, device="cuda", n_iter: bool = True) -> dict:
    d = {k: torch.empty(n, dtype=torch.float32, device=device) for k in DENSITY_FIELDS}
    if n_iter:
        d["n_iter"] = torch.empty(n, dtype=torch.int32, device=device)
    return d


def alloc_force(n: int, device="cuda") -> dict:
    return {k: torch.empty(n, dtype=torch.float32, device=device) for k in FORCE_FIELDS}
