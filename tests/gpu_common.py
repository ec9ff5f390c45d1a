"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same inputs (the GPU's float32 inputs, upcast)."""
import math

import numpy as np

GAMMA_K = 1.825742

# Tolerances of the CUDA path (FP32 pair arithmetic) against the FP64 oracle.
# rho and h: 1e-5 relative.  Accelerations and du/dt: 1e-4 of their rms.
# The other density outputs are derived from the same FP32 sums; their bounds
# follow from the arithmetic: f, P, c and v_sig inherit the rho/h error
# (1e-5 relative); div_v and |curl v| are sums with cancellation, bounded by
# 1e-4 of their rms plus the h error times their size; B is bounded in
# absolute terms by the div/curl errors relative to their sum.
TOL = dict(h=1e-5, rho=1e-5, f=1e-5, P=1e-5, c=1e-5, v_sig=1e-5, acc=1e-4, du=1e-4,
           divcurl=1e-4, balsara=2e-4)


def as_f32(p):
    """The float32 rounding the GPU sees, as float64 arrays for the oracle."""
    q = dict(p)
    for k in ("vx", "vy", "vz", "m", "u", "h0"):
        q[k] = np.asarray(p[k], dtype=np.float32).astype(np.float64)
    return q


def expected_nc(h0_f32, L, margin=0.05, n=None):
    """Cells per side from the definition in include/sph.h."""
    hmax = float(np.max(np.asarray(h0_f32, dtype=np.float32)))
    nc = int(math.floor(L / (GAMMA_K * hmax * (1.0 + margin))))
    if n is not None:
        lim = 8.0 * n + 216.0
        cap = int(round(lim ** (1.0 / 3.0)))
        while (cap + 1) ** 3 <= lim:
            cap += 1
        while cap > 3 and cap ** 3 > lim:
            cap -= 1
        nc = min(nc, cap)
    return max(nc, 1)


def run_gpu(p, margin=0.05, count_pairs=False, h_tol=1e-4, tree=False, n_leaf=16, h_start=None,
            axis=False, kernel=0, extra_flags=0, lanes=0):
    """build -> density -> (rebuild while the status asks) -> force on cuda:0.
    tree: nested grids below the top cells; axis: sorted interactions on the
    uniform grid; h_start: starting guess of h (default p["h0"]); kernel:
    SPH_KERNEL_* of the context; extra_flags: further SPH_FLAG_* bits; lanes:
    lanes per target of the uniform loops (0: automatic)."""
    import torch
    from paper_2305_13380_gb300 import sph
    flags = sph.SPH_FLAG_COUNT_PAIRS if count_pairs else 0
    if tree:
        flags |= sph.SPH_FLAG_TREE
    if axis:
        flags |= sph.SPH_FLAG_AXIS_SORT
    flags |= extra_flags
    params = sph.sph_default_params(box_size=float(p["L"]), cell_margin=margin, flags=flags,
                                    h_tol=h_tol, n_leaf=n_leaf, kernel=kernel, lanes_per_target=lanes)
    ctx = sph.Context(params)
    t = sph.to_device(p)
    n = int(t["x"].shape[0])
    part = sph.particles(t)
    d = sph.alloc_density(n)
    f = sph.alloc_force(n)
    h_in = t["h0"] if h_start is None else torch.as_tensor(
        np.asarray(h_start, dtype=np.float32), device="cuda")
    rebuilds = 0
    for _ in range(8):
        cells = sph.sph_build_cells(ctx, t["x"], t["y"], t["z"], h_in)
        sph.sph_density(ctx, cells, part, h_in, sph.density_out(d))
        st = sph.sph_status(ctx)
        if not st & sph.SPH_ST_REBUILD:
            break
        rebuilds += 1
        h_in = d["h"].clone()
    assert st == 0, f"device status {st}"
    pairs_d = sph.sph_pair_counts(ctx)[0] if count_pairs else None
    sph.sph_force(ctx, cells, part, sph.density_out(d), sph.force_out(f))
    assert sph.sph_status(ctx) == 0
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in d.items()}
    out.update({k: v.cpu().numpy() for k, v in f.items()})
    if count_pairs:
        out["pairs"] = (pairs_d, sph.sph_pair_counts(ctx)[1])
    out["rebuilds"] = rebuilds
    out["_ctx"], out["_cells"] = ctx, cells
    return out


def support_bound(q, k=20):
    """Upper bound on each particle's support H_j = gamma_K h_j of the cubic
    spline from the positions alone.  With d_k the distance to the k-th nearest
    particle (itself the first), H = 2 d_k puts k particles at q <= 1/2, where
    w(q) >= w(1/2) = 2/pi, so sum_j w(r_ij / H) >= 2k/pi, which reaches
    (gamma_K eta)^3 = 11.458 (eta = 1.2348) once k >= 18.  The partition
    condition's left side grows with h, so H_j <= 2 d_k for k = 20.
    Returns (bound, cKDTree of the positions, positions)."""
    from scipy.spatial import cKDTree
    L = float(q["L"])
    X = np.stack([np.mod(np.asarray(q[c], dtype=np.float64), L) for c in ("x", "y", "z")], 1)
    tree = cKDTree(X, boxsize=L)
    d, _ = tree.query(X, k=k)
    return 2.0 * d[:, -1], tree, X


def rel_err(a, b):
    return np.abs(a - b) / np.abs(b)


def coord_floor(cell, h):
    """Relative error floor of quantities set by neighbour distances when
    positions are FP32 offsets of magnitude up to two cells of side `cell`.
    Each coordinate is rounded once from FP64 (error <= ulp(cell)/2) and once
    when the periodic-image offset is added (<= ulp(2 cell)/2 = ulp(cell)),
    so a pair difference is off by at most 2 ulp(cell) <= 2^-22 cell per
    component and a distance by sqrt(3) 2^-22 cell.  For a neighbour at
    r ~ H/2 that is 2 sqrt(3) 2^-22 cell / H relative; sums over the ~50
    neighbours stay within that worst single-distance figure."""
    return 2.0 * np.sqrt(3.0) * 2.0 ** -22 * cell / (GAMMA_K * np.asarray(h))


def compare(g, od, of, idx=None, cell=None, vmax=None):
    """Asserts the GPU outputs g (indexed by idx) against oracle density od and
    force of (already restricted to the same particles).

    With `cell` (the grid's cell size) every bound gets the coordinate-rounding
    floor d_i = coord_floor(cell, h_i) of each particle.  Quantities that are
    sums of gradient terms carry d_i times the sum of their absolute terms;
    with int_0^1 |w'(q)| 4 pi q^2 dq = 5.6 for the cubic spline, that sum is
    5.6 / H_i times the term's velocity or pressure factor: 2 vmax for the
    divergence and curl, 2 P/rho for the acceleration, 4 vmax P/rho for du/dt."""
    sel = (lambda a: a) if idx is None else (lambda a: a[idx])
    report = {}
    if cell is None:
        floor = np.zeros_like(od["h"])
    else:
        floor = coord_floor(cell, od["h"])
    H = GAMMA_K * od["h"]
    vm = 0.0 if vmax is None else vmax
    Prho = od["P"] / od["rho"]
    for k_g, k_o, tol in (("h", "h", TOL["h"]), ("rho", "rho", TOL["rho"]), ("f", "f", TOL["f"]),
                          ("P", "P", TOL["P"]), ("c", "c", TOL["c"])):
        err = rel_err(sel(g[k_g]), od[k_o])
        lim = tol + floor if k_g != "c" else tol
        e = (err / lim).max()
        report[k_g] = err.max()
        assert e <= 1.0, f"{k_g}: max relative error {err.max():.3e} (worst ratio to bound {e:.2f})"
    dvc = {}
    for k_g, k_o in (("div_v", "div_v"), ("curl_v", "curl_norm")):
        ref = od[k_o]
        scale = np.sqrt(np.mean(ref ** 2)) + 1e-300
        err = np.abs(sel(g[k_g]) - ref)
        # the h-error term: the gradient sums scale as H^-5 through the
        # kernel gradient, so a relative h error d moves them by ~5 d
        lim = TOL["divcurl"] * scale + 5 * TOL["h"] * np.abs(ref) + floor * 5.6 * 2 * vm / H
        dvc[k_g] = lim
        e = (err / lim).max()
        report[k_g] = err.max() / scale
        assert e <= 1.0, f"{k_g}: max error / rms {err.max() / scale:.3e} (worst ratio {e:.2f})"
    err = np.abs(sel(g["balsara"]) - od["B"])
    denom = np.abs(od["div_v"]) + od["curl_norm"] + 1e-4 * od["c"] / od["h"]
    lim = TOL["balsara"] + 2 * (dvc["div_v"] + dvc["curl_v"]) / denom * (cell is not None)
    e = (err / lim).max()
    report["balsara"] = err.max()
    assert e <= 1.0, f"balsara: max abs error {err.max():.3e} (worst ratio {e:.2f})"
    a_ref = np.stack([of["ax"], of["ay"], of["az"]], 1)
    a_gpu = np.stack([sel(g["ax"]), sel(g["ay"]), sel(g["az"])], 1)
    rms = np.sqrt(np.mean(np.sum(a_ref ** 2, 1)))
    err = np.abs(a_gpu - a_ref).max(1)
    lim = TOL["acc"] * rms + floor * 5.6 * 2 * Prho / H
    e = (err / lim).max()
    report["a"] = err.max() / rms
    assert e <= 1.0, f"a: max error / rms|a| {err.max() / rms:.3e} (worst ratio {e:.2f})"
    rms_u = np.sqrt(np.mean(of["du_dt"] ** 2))
    err = np.abs(sel(g["du_dt"]) - of["du_dt"])
    lim = TOL["du"] * rms_u + floor * 5.6 * 4 * vm * Prho / H
    e = (err / lim).max()
    report["du_dt"] = err.max() / rms_u
    assert e <= 1.0, f"du_dt: max error / rms {err.max() / rms_u:.3e} (worst ratio {e:.2f})"
    err = rel_err(sel(g["v_sig"]), of["v_sig"])
    lim = TOL["v_sig"] + floor
    e = (err / lim).max()
    report["v_sig"] = err.max()
    assert e <= 1.0, f"v_sig: max relative error {err.max():.3e} (worst ratio {e:.2f})"
    return report
