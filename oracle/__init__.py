"""Python handle on the FP64 CPU oracle (``oracle/sph_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The library under
``paper_2305_13380_gb300/`` never imports it and shares no code with it.

The oracle computes the SPH sums of SWIFT (Schaller et al. 2024) Sec. 3.1-3.2
straight from their definitions in double precision; see the header of
``sph_oracle.c`` for the readings of the paper it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

GAMMA_K = 1.825742  # H/h of the 3-D cubic spline (Dehnen & Aly 2012 convention)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("L", C.c_double)] + [
        (k, C.c_void_p) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u")]


class _Config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("eta", C.c_double), ("alpha_v", C.c_double),
                ("beta_v", C.c_double), ("eps_balsara", C.c_double), ("h_tol", C.c_double),
                ("max_iter", C.c_int32), ("brute", C.c_int32)]


_DENS_F = ("h", "rho", "drho_dh", "n_hat", "dn_dh", "div_v", "curl_x", "curl_y", "curl_z",
           "curl_norm", "f", "P", "c", "B")
_DENS_I = ("n_ngb", "n_iter")


class _DensOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _DENS_F + _DENS_I]


class _DensState(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("h", "rho", "f", "P", "c", "B")]


_FORCE_F = ("ax", "ay", "az", "du_dt", "v_sig")


class _ForceOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _FORCE_F + ("n_pairs",)]


class _SphenixCfg(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("alpha_v_max", "ell", "beta_c", "alpha_c_min",
                                          "alpha_c_max")]


_GRAD_F = ("lap_u", "v_c", "alpha_v_ngb", "alpha_c")


class _GradOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _GRAD_F]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.oracle_w.restype = C.c_double
        L.oracle_w.argtypes = [C.c_double]
        L.oracle_dw_dq.restype = C.c_double
        L.oracle_dw_dq.argtypes = [C.c_double]
        L.oracle_gamma_k.restype = C.c_double
        L.oracle_set_kernel.argtypes = [C.c_int]
        L.oracle_wrap.restype = C.c_double
        L.oracle_wrap.argtypes = [C.c_double, C.c_double]
        L.oracle_cell_coord.restype = C.c_int32
        L.oracle_cell_coord.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.oracle_tree_order.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_int32, C.c_void_p, C.c_void_p]
        L.oracle_build_cells.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_double, C.c_int32, C.c_void_p, C.c_void_p]
        L.oracle_fof.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                 C.c_double, C.c_void_p]
        L.oracle_density.argtypes = [C.POINTER(_Particles), C.POINTER(_Config), C.c_void_p,
                                     C.c_int64, C.c_void_p, C.POINTER(_DensOut)]
        L.oracle_density_at.argtypes = [C.POINTER(_Particles), C.POINTER(_Config), C.c_void_p,
                                        C.c_int64, C.c_void_p, C.POINTER(_DensOut)]
        L.oracle_force.argtypes = [C.POINTER(_Particles), C.POINTER(_Config),
                                   C.POINTER(_DensState), C.c_int64, C.c_void_p,
                                   C.POINTER(_ForceOut)]
        L.oracle_neighbours.argtypes = [C.POINTER(_Particles), C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
        L.oracle_sphenix_alpha_v.restype = None
        L.oracle_sphenix_alpha_v.argtypes = [C.c_int64, C.POINTER(_SphenixCfg), C.c_double] + \
            [C.c_void_p] * 7
        L.oracle_sphenix_gradient.argtypes = [C.POINTER(_Particles), C.POINTER(_Config),
                                              C.POINTER(_SphenixCfg), C.POINTER(_DensState),
                                              C.c_void_p, C.c_void_p, C.c_double, C.c_int64,
                                              C.c_void_p, C.POINTER(_GradOut)]
        L.oracle_sphenix_force.argtypes = [C.POINTER(_Particles), C.POINTER(_Config),
                                           C.POINTER(_DensState), C.c_void_p, C.c_void_p,
                                           C.c_int64, C.c_void_p, C.POINTER(_ForceOut),
                                           C.c_void_p]
        L.oracle_step.argtypes = [C.c_int64, C.c_double, C.POINTER(_Config), C.c_double] + \
            [C.c_void_p] * 14 + [C.c_void_p, C.POINTER(C.c_double)]
        _lib = L
    return _lib


@dataclass
class Physics:
    """Physical constants of the "Minimal" SPH flavour (Sec. 3.2)."""
    gamma: float = 5.0 / 3.0
    eta: float = 1.2348
    alpha_v: float = 0.8
    beta_v: float = 3.0
    eps_balsara: float = 1e-4
    h_tol: float = 1e-13
    max_iter: int = 200
    kernel: int = 0  # 0 cubic spline, 1 quartic spline, 2 Wendland C2 (Sec. 3.1)


@dataclass
class Sphenix:
    """Constants of the SPHENIX flavour (Sec. 3.3)."""
    alpha_v_max: float = 2.0
    ell: float = 0.05
    beta_c: float = 1.0
    alpha_c_min: float = 0.0
    alpha_c_max: float = 1.0


def _sphenix_cfg(X: Sphenix):
    return _SphenixCfg(X.alpha_v_max, X.ell, X.beta_c, X.alpha_c_min, X.alpha_c_max)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Keep:
    """Keeps the float64 copies alive for the duration of a call."""

    def __init__(self):
        self.items = []

    def __call__(self, a):
        a = _d(a)
        self.items.append(a)
        return _ptr(a)


def _particles(keep, p):
    n = int(np.asarray(p["x"]).shape[0])
    return _Particles(n, float(p["L"]), *[keep(p[k]) for k in
                                          ("x", "y", "z", "vx", "vy", "vz", "m", "u")])


KERNELS = {"cubic": 0, "quartic": 1, "wendland_c2": 2}


def set_kernel(kernel: int):
    """Selects the kernel of the following oracle calls."""
    _check(lib().oracle_set_kernel(int(kernel)), "set_kernel")


def _config(phys: Physics, brute: bool):
    set_kernel(phys.kernel)
    return _Config(phys.gamma, phys.eta, phys.alpha_v, phys.beta_v, phys.eps_balsara,
                   phys.h_tol, phys.max_iter, 1 if brute else 0)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def w(q: float, kernel: int = 0) -> float:
    set_kernel(kernel)
    return lib().oracle_w(float(q))


def dw_dq(q: float, kernel: int = 0) -> float:
    set_kernel(kernel)
    return lib().oracle_dw_dq(float(q))


def gamma_k(kernel: int = 0) -> float:
    """H/h of the kernel."""
    set_kernel(kernel)
    return lib().oracle_gamma_k()


def cell_coord(x: float, L: float, n_c: int) -> int:
    return lib().oracle_cell_coord(float(x), float(L), int(n_c))


def wrap(x: float, L: float) -> float:
    return lib().oracle_wrap(float(x), float(L))


def build_cells(x, y, z, L: float, n_c: int):
    """Stable counting sort of particles into the n_c^3 cell grid (Sec. 2.1)."""
    keep = _Keep()
    n = int(np.asarray(x).shape[0])
    cell_start = np.zeros(n_c ** 3 + 1, dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().oracle_build_cells(n, keep(x), keep(y), keep(z), float(L), int(n_c),
                                    _ptr(cell_start), _ptr(perm)), "build_cells")
    return cell_start, perm[:n]


def fof(x, y, z, L: float, b: float):
    """Friends-of-friends groups with linking length b in the periodic box of
    side L (Sec. 7.1): group[i] = the smallest index of i's group."""
    keep = _Keep()
    n = int(np.asarray(x).shape[0])
    group = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().oracle_fof(n, keep(x), keep(y), keep(z), float(L), float(b), _ptr(group)), "fof")
    return group[:n]


def tree_order(x, y, z, L: float, n_c: int):
    """Depth-first order of the nested grids below the n_c^3 top cells
    (Sec. 2.1, Sec. 9.1): top cells ascending, then the child indices of
    depths 1..10, ties by input index.  Returns (cell_start, perm)."""
    keep = _Keep()
    n = int(np.asarray(x).shape[0])
    cell_start = np.zeros(n_c ** 3 + 1, dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().oracle_tree_order(n, keep(x), keep(y), keep(z), float(L), int(n_c),
                                   _ptr(cell_start), _ptr(perm)), "tree_order")
    return cell_start, perm[:n]


def density(p: dict, h0, targets=None, phys: Physics = Physics(), brute: bool = False) -> dict:
    """Density loop + smoothing-length solve for the given targets (all by default).

    ``p`` holds x, y, z, vx, vy, vz, m, u (length n) and the box side L;
    ``h0`` the starting guess of h for all n particles."""
    keep = _Keep()
    P = _particles(keep, p)
    n = P.n
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else int(tg.shape[0])
    out = {k: np.zeros(nt) for k in _DENS_F}
    out.update({k: np.zeros(nt, dtype=np.int32) for k in _DENS_I})
    D = _DensOut(*[_ptr(out[k]) for k in _DENS_F + _DENS_I])
    cfg = _config(phys, brute)
    _check(lib().oracle_density(C.byref(P), C.byref(cfg), keep(h0), nt, _ptr(tg), C.byref(D)),
           "density")
    return out


def density_at(p: dict, h_t, targets=None, phys: Physics = Physics(),
               brute: bool = False) -> dict:
    """Density-loop sums at the given smoothing length h_t[t] of each target (no solve)."""
    keep = _Keep()
    P = _particles(keep, p)
    n = P.n
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else int(tg.shape[0])
    out = {k: np.zeros(nt) for k in _DENS_F}
    out.update({k: np.zeros(nt, dtype=np.int32) for k in _DENS_I})
    D = _DensOut(*[_ptr(out[k]) for k in _DENS_F + _DENS_I])
    cfg = _config(phys, brute)
    _check(lib().oracle_density_at(C.byref(P), C.byref(cfg), keep(h_t), nt, _ptr(tg),
                                   C.byref(D)), "density_at")
    return out


def force(p: dict, state: dict, targets=None, phys: Physics = Physics(),
          brute: bool = False) -> dict:
    """Force loop for the given targets; ``state`` holds h, rho, f, P, c, B for all n."""
    keep = _Keep()
    P = _particles(keep, p)
    n = P.n
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else int(tg.shape[0])
    S = _DensState(*[keep(state[k]) for k in ("h", "rho", "f", "P", "c", "B")])
    out = {k: np.zeros(nt) for k in _FORCE_F}
    out["n_pairs"] = np.zeros(nt, dtype=np.int32)
    F = _ForceOut(*[_ptr(out[k]) for k in _FORCE_F + ("n_pairs",)])
    cfg = _config(phys, brute)
    _check(lib().oracle_force(C.byref(P), C.byref(cfg), C.byref(S), nt, _ptr(tg), C.byref(F)),
           "force")
    return out


def neighbours(p: dict, targets, R, brute: bool = False, cap: int = 4096):
    """Indices j != t with minimum-image distance < R[t], per target (list of arrays)."""
    keep = _Keep()
    P = _particles(keep, p)
    tg = np.ascontiguousarray(targets, dtype=np.int64)
    Rr = np.ascontiguousarray(R, dtype=np.float64)
    nt = int(tg.shape[0])
    nbr = np.zeros(nt * cap, dtype=np.int32)
    cnt = np.zeros(nt, dtype=np.int64)
    _check(lib().oracle_neighbours(C.byref(P), nt, _ptr(tg), _ptr(Rr), 1 if brute else 0, cap,
                                   _ptr(nbr), _ptr(cnt)), "neighbours")
    if np.any(cnt > cap):
        raise RuntimeError("neighbour capacity exceeded")
    return [np.sort(nbr[t * cap:t * cap + cnt[t]]) for t in range(nt)]


def density_force(p: dict, h0, phys: Physics = Physics(), brute: bool = False):
    """Density then force on every particle; returns (density dict, force dict)."""
    d = density(p, h0, None, phys, brute)
    f = force(p, d, None, phys, brute)
    return d, f


def step(s: dict, cfl: float, phys: Physics = Physics(), brute: bool = False) -> float:
    """One KDK step in place on the state dict s (x, y, z, vx, vy, vz, m, u, h,
    ax, ay, az, du_dt, v_sig, L); returns dt.  s must hold float64 arrays."""
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "ax", "ay", "az", "du_dt", "v_sig"):
        if not (isinstance(s[k], np.ndarray) and s[k].dtype == np.float64 and s[k].flags.c_contiguous):
            s[k] = _d(s[k])
    n = int(s["x"].shape[0])
    cfg = _config(phys, brute)
    rho = np.zeros(n)
    dt = C.c_double(0.0)
    args = [_ptr(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "ax", "ay", "az",
                                 "du_dt", "v_sig")]
    _check(lib().oracle_step(n, float(s["L"]), C.byref(cfg), float(cfl), *args, _ptr(rho),
                             C.byref(dt)), "step")
    s["rho"] = rho
    return dt.value


def sphenix_alpha_v(dt: float, h, c, div_v, div_v_prev, v_sig, alpha, X: Sphenix = Sphenix(),
                    phys: Physics = Physics()):
    """SPHENIX viscosity parameters after a step dt (eqs. "sphenix_visc1"-"sphenix_visc4")."""
    set_kernel(phys.kernel)
    keep = _Keep()
    n = int(np.asarray(h).shape[0])
    out = np.zeros(n)
    cfg = _sphenix_cfg(X)
    lib().oracle_sphenix_alpha_v(n, C.byref(cfg), float(dt), keep(h), keep(c), keep(div_v),
                                 keep(div_v_prev), keep(v_sig), keep(alpha), _ptr(out))
    return out


def sphenix_gradient(p: dict, state: dict, alpha_v, alpha_c, dt: float, targets=None,
                     X: Sphenix = Sphenix(), phys: Physics = Physics(),
                     brute: bool = False) -> dict:
    """SPHENIX gradient pass (lap u, v_c, largest neighbour alpha_V) and the updated
    conduction parameter alpha_c of the targets; ``alpha_v`` are the updated
    viscosity parameters of all n particles, ``alpha_c`` the old conduction ones."""
    keep = _Keep()
    P = _particles(keep, p)
    n = P.n
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else int(tg.shape[0])
    S = _DensState(*[keep(state[k]) for k in ("h", "rho", "f", "P", "c", "B")])
    out = {k: np.zeros(nt) for k in _GRAD_F}
    O = _GradOut(*[_ptr(out[k]) for k in _GRAD_F])
    cfg = _config(phys, brute)
    xc = _sphenix_cfg(X)
    _check(lib().oracle_sphenix_gradient(C.byref(P), C.byref(cfg), C.byref(xc), C.byref(S),
                                         keep(alpha_v), keep(alpha_c), float(dt), nt, _ptr(tg),
                                         C.byref(O)), "sphenix_gradient")
    return out


def sphenix_force(p: dict, state: dict, alpha_v, alpha_c, targets=None,
                  phys: Physics = Physics(), brute: bool = False) -> dict:
    """SPHENIX force loop for the given targets (``du_cond``: the conduction part of du/dt)."""
    keep = _Keep()
    P = _particles(keep, p)
    n = P.n
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else int(tg.shape[0])
    S = _DensState(*[keep(state[k]) for k in ("h", "rho", "f", "P", "c", "B")])
    out = {k: np.zeros(nt) for k in _FORCE_F + ("du_cond",)}
    out["n_pairs"] = np.zeros(nt, dtype=np.int32)
    F = _ForceOut(*[_ptr(out[k]) for k in _FORCE_F + ("n_pairs",)])
    cfg = _config(phys, brute)
    _check(lib().oracle_sphenix_force(C.byref(P), C.byref(cfg), C.byref(S), keep(alpha_v),
                                      keep(alpha_c), nt, _ptr(tg), C.byref(F),
                                      _ptr(out["du_cond"])), "sphenix_force")
    return out


def sphenix_evaluate(p: dict, h0, alpha_v, alpha_c, div_v_prev, v_sig_prev, dt: float,
                     X: Sphenix = Sphenix(), phys: Physics = Physics(), brute: bool = False):
    """One SPHENIX force evaluation in the library's order: density, viscosity
    update, gradient pass with the conduction update, force.  Returns
    (density dict, alpha_v, gradient dict, force dict)."""
    d = density(p, h0, None, phys, brute)
    av = sphenix_alpha_v(dt, d["h"], d["c"], d["div_v"], div_v_prev, v_sig_prev, alpha_v, X, phys)
    g = sphenix_gradient(p, d, av, alpha_c, dt, None, X, phys, brute)
    f = sphenix_force(p, d, av, g["alpha_c"], None, phys, brute)
    return d, av, g, f


def sphenix_step(s: dict, cfl: float, X: Sphenix = Sphenix(), phys: Physics = Physics(),
                 brute: bool = False) -> float:
    """One KDK step of SPHENIX in place on the state dict s (the keys of
    ``step`` plus alpha_v, alpha_c and div_v, the divergence of the previous
    evaluation), in the order of ``step`` with sphenix_evaluate as the force
    evaluation on the predicted v and u; returns dt."""
    for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "ax", "ay", "az", "du_dt", "v_sig",
              "alpha_v", "alpha_c", "div_v"):
        s[k] = _d(s[k]).copy()
    L = float(s["L"])
    dt = float(np.min(cfl * gamma_k(phys.kernel) * s["h"] / s["v_sig"]))
    if not (dt > 0.0) or not np.isfinite(dt):
        raise RuntimeError("oracle sphenix_step: no finite positive time-step")
    wrap = lib().oracle_wrap
    for k in ("x", "y", "z"):
        v = "v" + k
        s[v] = s[v] + 0.5 * dt * s["a" + k]
        s[k] = np.array([wrap(float(q), L) for q in s[k] + s[v] * dt])
    s["u"] = s["u"] + 0.5 * dt * s["du_dt"]
    pred = dict(L=L, x=s["x"], y=s["y"], z=s["z"], m=s["m"],
                vx=s["vx"] + 0.5 * dt * s["ax"], vy=s["vy"] + 0.5 * dt * s["ay"],
                vz=s["vz"] + 0.5 * dt * s["az"], u=s["u"] + 0.5 * dt * s["du_dt"])
    d, av, g, f = sphenix_evaluate(pred, s["h"], s["alpha_v"], s["alpha_c"], s["div_v"],
                                   s["v_sig"], dt, X, phys, brute)
    s["h"], s["rho"], s["div_v"] = d["h"], d["rho"], d["div_v"]
    s["alpha_v"], s["alpha_c"] = av, g["alpha_c"]
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        s[k] = f[k]
    for k in ("x", "y", "z"):
        s["v" + k] = s["v" + k] + 0.5 * dt * s["a" + k]
    s["u"] = s["u"] + 0.5 * dt * s["du_dt"]
    return dt


def time_bins(h, v_sig, cfl: float, dt_max: float, max_bin: int, kernel: int = 0):
    """Per-particle time bins of the power-of-two time-step hierarchy (Sec. 2.4,
    "Local time-step optimisations"): the CFL step dt_i = C_CFL gamma_K h_i / v_sig,i,
    and bin_i = the smallest b in [0, max_bin] with dt_max 2^-b <= dt_i (max_bin if
    none; bin 0 where v_sig <= 0).  The definition in FP64: dt_i is one FP64
    expression and dt_max 2^-b is exact.  A kernel that decides in a lower precision
    agrees except where dt_i lies within its rounding of a power-of-two boundary
    (``bin_edge_band``)."""
    h = np.asarray(h, dtype=np.float64)
    v = np.asarray(v_sig, dtype=np.float64)
    c = float(cfl) * gamma_k(kernel)
    with np.errstate(divide="ignore"):
        dt = np.where(v > 0, c * h / np.where(v > 0, v, 1.0), np.inf)
    bins = np.full(h.shape, max_bin, dtype=np.int32)
    for b in range(max_bin, -1, -1):
        bins = np.where(np.ldexp(float(dt_max), -b) <= dt, b, bins)
    return bins


def bin_edge_band(h, v_sig, cfl: float, dt_max: float, max_bin: int, kernel: int = 0,
                  rel: float = 1e-6):
    """True where the CFL step dt_i lies within a relative distance rel of one of
    the bin boundaries dt_max 2^-b (b = 0..max_bin): there a bin decided in FP32
    may differ by one from the FP64 definition."""
    h = np.asarray(h, dtype=np.float64)
    v = np.asarray(v_sig, dtype=np.float64)
    c = float(cfl) * gamma_k(kernel)
    with np.errstate(divide="ignore"):
        dt = np.where(v > 0, c * h / np.where(v > 0, v, 1.0), np.inf)
    near = np.zeros(h.shape, dtype=bool)
    for b in range(0, max_bin + 1):
        e = np.ldexp(float(dt_max), -b)
        near |= np.abs(dt - e) <= rel * e
    return near


def limit_time_bins(p: dict, h, bins, kernel: int = 0, scale: float = 1.0):
    """The first time-step limiter (Sec. 3.4, "Time-step limiter", Delta = 4):
    a particle's step is at most 4 times the smallest step of the particles it
    interacts with in the force loop (j != i, r_ij < max(H_i, H_j)), i.e.
    bin_i <- max(bin_i, max_j bin_j - 2), applied once.  Brute force over all
    pairs with minimum-image distances (small inputs).  scale multiplies the
    interaction radius (tests use 1 +- 1e-5 to bound pairs at the edge)."""
    x = np.stack([np.asarray(p[k], dtype=np.float64) for k in ("x", "y", "z")], 1)
    L = float(p["L"])
    H = gamma_k(kernel) * np.asarray(h, dtype=np.float64)
    bins = np.asarray(bins, dtype=np.int32)
    out = bins.copy()
    for i in range(len(bins)):
        d = x - x[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        nb = (r < scale * np.maximum(H, H[i])) & (np.arange(len(bins)) != i)
        if nb.any():
            out[i] = max(bins[i], int(bins[nb].max()) - 2)
    return out


def hier_substep(s: dict, bins, t_begin, dt_max: float, max_bin: int, t_now: int, adapt: bool,
                 cfl: float = 0.1, phys: Physics = Physics(), wakeup: bool = False, sync=None,
                 predict: bool = False) -> int:
    """One sub-step of the power-of-two time-step hierarchy (Sec. 2.4), in place
    on the state dict s (float64 arrays: x, y, z, vx, vy, vz and u half-kicked
    for each particle's current step, m, h, ax, ay, az, du_dt, v_sig, the
    density results rho, f, P, c, B, div_v; and L) and on bins / t_begin
    (integer arrays).  Time runs on ticks of dt_max 2^-max_bin; a particle in
    bin b steps 2^(max_bin - b) ticks.  Every particle drifts to the next end
    of a step; the particles whose step ends there (the active ones) get the
    density and the force at the predicted v and u of every particle, their
    second half kick, a new bin (adapt: the CFL bin limited against the
    neighbours' bins -- proposed ones for active neighbours, held ones for
    inactive neighbours; else the old one;
    shortened until the new step divides the tick) and the first half kick of
    the new step.

    The second and third limiters of Sec. 3.4 ("Time-step limiter") end the
    current step of an inactive particle j at the new tick: its velocity and
    energy are kicked to the tick with its last a and du/dt, it takes a new bin
    (shortened until its step divides the tick), the first half kick of that
    step, and t_begin = tick.
      wakeup: after the active particles have their new bins, every inactive j
        with an active force-loop neighbour i (r_ij < max(H_i, H_j)) whose new
        step is more than 4 times shorter (bin_i - 2 > bin_j) is woken with
        bin max_i (bin_i - 2) (Saitoh & Makino 2009);
      sync: a boolean array of flagged particles (say, touched by a source
        term between sub-steps); a flagged inactive one is synchronised with
        its CFL bin (adapt; the limiter of the active ones then sees that bin)
        or its held bin, raised to its wake-up bin if it has one.  The flags
        are cleared in place.
    predict: the drift also carries every particle's smoothing length and
    density over the interval with its last velocity divergence held fixed,
    dh/dt = h div_v / 3 and the continuity equation drho/dt = -rho div_v
    (h e^(div_v dt / 3), rho e^(-div_v dt)), and its pressure and sound speed
    from the equation of state (Sec. 3.2) at the predicted density and u.  The
    active particles' values are then replaced by their density loop (h is
    its starting guess).
    Returns the new tick."""
    n = len(bins)
    step = np.left_shift(np.int64(1), (max_bin - bins).astype(np.int64))
    tau = float(np.ldexp(dt_max, -max_bin))
    t_next = int(np.min(t_begin + step))
    dt = (t_next - t_now) * tau
    wrap = lib().oracle_wrap
    L = float(s["L"])
    for k in ("x", "y", "z"):
        s[k] = np.array([wrap(float(q), L) for q in s[k] + s["v" + k] * dt])
    w = ((t_next - t_begin) - 0.5 * step) * tau
    pred = dict(L=L, x=s["x"], y=s["y"], z=s["z"], m=s["m"], vx=s["vx"] + s["ax"] * w,
                vy=s["vy"] + s["ay"] * w, vz=s["vz"] + s["az"] * w, u=s["u"] + s["du_dt"] * w)
    if predict:
        dv = np.asarray(s["div_v"], dtype=np.float64) * dt
        s["h"] = s["h"] * np.exp(dv / 3.0)
        s["rho"] = s["rho"] * np.exp(-dv)
        s["P"] = (phys.gamma - 1.0) * pred["u"] * s["rho"]
        s["c"] = np.sqrt(phys.gamma * s["P"] / s["rho"])
    act = np.where(t_begin + step == t_next)[0]
    d = density(pred, s["h"], act, phys)
    for k in ("h", "rho", "f", "P", "c", "B", "div_v"):
        s[k][act] = d[k]
    f = force(pred, s, act, phys)
    for k in ("ax", "ay", "az", "du_dt", "v_sig"):
        s[k][act] = f[k]
    inactive = np.ones(n, dtype=bool)
    inactive[act] = False
    flagged = np.zeros(n, dtype=bool) if sync is None else np.asarray(sync, dtype=bool).copy()
    synced = flagged & inactive
    if adapt:
        # the limiter compares an active particle's proposed bin with the bins
        # its force-loop neighbours step in: the proposals of the active ones
        # (and of the synchronised ones), the bins that the other inactive
        # ones hold for their current step
        b0 = time_bins(s["h"], s["v_sig"], cfl, dt_max, max_bin, phys.kernel)
        held = inactive & ~synced
        b0[held] = bins[held]
        new = limit_time_bins(pred, s["h"], b0, phys.kernel)[act]
    else:
        new = bins[act].copy()

    def aligned(b):
        b = min(max(int(b), 0), max_bin)
        while b < max_bin and t_next % (1 << (max_bin - b)) != 0:
            b += 1
        return b

    for q, i in enumerate(act):
        b = aligned(new[q])
        h_old, h_new = 0.5 * step[i] * tau, 0.5 * (1 << (max_bin - b)) * tau
        for k in ("x", "y", "z"):
            s["v" + k][i] += s["a" + k][i] * (h_old + h_new)
        s["u"][i] += s["du_dt"][i] * (h_old + h_new)
        bins[i] = b
        t_begin[i] = t_next
    # the steps that end early: requested bin of each interrupted particle
    want = {int(j): int(b0[j]) if adapt else int(bins[j]) for j in np.where(synced)[0]}
    if wakeup and len(act):
        X = np.stack([s["x"], s["y"], s["z"]], 1)
        H = gamma_k(phys.kernel) * np.asarray(s["h"], dtype=np.float64)
        for j in np.where(inactive)[0]:
            d = X[act] - X[j]
            d -= L * np.round(d / L)
            r = np.sqrt((d * d).sum(1))
            nb = r < np.maximum(H[act], H[j])
            if nb.any():
                w = int(bins[act][nb].max()) - 2
                if w > bins[j]:
                    want[int(j)] = max(want.get(int(j), w), w)
    for j, b in sorted(want.items()):
        b = aligned(b)
        # end of the current step at the tick, then the first half of the new
        w = ((t_next - t_begin[j]) - 0.5 * step[j]) * tau + 0.5 * (1 << (max_bin - b)) * tau
        for k in ("x", "y", "z"):
            s["v" + k][j] += s["a" + k][j] * w
        s["u"][j] += s["du_dt"][j] * w
        bins[j] = b
        t_begin[j] = t_next
    if sync is not None:
        sync[...] = False
    return t_next
