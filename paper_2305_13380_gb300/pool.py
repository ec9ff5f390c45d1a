"""Pools of independent simulations advanced together by ``sph_step``.

A pool keeps every simulation's particles in one set of device arrays
(structure of arrays, simulation s owns ``[sim_offset[s], sim_offset[s+1])``),
so one ``sph_step`` call runs each kernel once for all simulations.  The step
of a pool can be captured in a CUDA graph and replayed: every size that
depends on the data (cells per side, cell and block counts) is computed on the
device, so the captured launches stay valid while the particles move.

This module only marshals arrays and calls the C ABI; all arithmetic runs in
the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sph

_F64 = ("x", "y", "z")
_F32_IN = ("vx", "vy", "vz", "u", "m")
_F32_OUT = ("h", "ax", "ay", "az", "du_dt", "v_sig", "rho", "f", "div_v", "curl_v", "P", "c",
            "balsara")


class Pool:
    """Device state of several simulations.

    ``sims`` is a list of dicts with x, y, z, vx, vy, vz, m, u, h0 and L (as
    produced by ``inputs``).  The first ``step()`` (or ``start()``) has zero
    signal velocities, hence dt = 0: it only evaluates density and force."""

    def __init__(self, sims, params: sph.sph_params | None = None, stream=None,
                 device="cuda"):
        self.n_sims = len(sims)
        counts = [len(s["x"]) for s in sims]
        self.offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        cat = lambda k, dt: torch.as_tensor(  # noqa: E731
            np.concatenate([np.asarray(s[k], dtype=dt) for s in sims]), device=device)
        self.a = {}
        for k in _F64:
            self.a[k] = cat(k, np.float64).contiguous()
        for k in _F32_IN:
            self.a[k] = cat(k, np.float32).contiguous()
        self.a["h"] = cat("h0", np.float32).contiguous()
        for k in _F32_OUT[1:]:
            self.a[k] = torch.zeros(self.n, dtype=torch.float32, device=device)
        self.a["dt"] = torch.zeros(self.n_sims, dtype=torch.float64, device=device)
        self.sim_offset = torch.as_tensor(self.offsets, device=device)
        self.box = torch.as_tensor(np.array([s["L"] for s in sims], dtype=np.float64),
                                   device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        p = params if params is not None else sph.sph_default_params()
        self.params = p
        self.ctx = sph.Context(p, self.stream)
        self.pool = sph.pool(self.sim_offset, self.box, self.a)
        self.graph = None

    def step(self):
        with torch.cuda.stream(self.stream):
            sph.sph_step(self.ctx, self.pool)

    def start(self):
        """Density + force of the initial state (a step with dt = 0).  It runs
        on a synchronous context, which rebuilds the cells with larger ones when
        a starting guess of h was too small for its cell."""
        q = sph.sph_params.from_buffer_copy(self.params)
        q.flags = q.flags | sph.SPH_FLAG_SYNC
        first = sph.Context(q, self.stream)
        with torch.cuda.stream(self.stream):
            sph.sph_step(first, self.pool)
        self.stream.synchronize()
        first.close()

    def capture(self):
        """Captures one step in a CUDA graph (after a warm-up step, so that
        the context's scratch is allocated and the launch shapes are set)."""
        self.step()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            sph.sph_step(self.ctx, self.pool)
        self.graph = g
        return g

    def replay(self):
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def status(self) -> int:
        return sph.sph_status(self.ctx)

    def sim_slice(self, s: int) -> slice:
        return slice(int(self.offsets[s]), int(self.offsets[s + 1]))

    def host(self, keys=("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax", "ay", "az",
                         "du_dt", "v_sig")) -> dict:
        self.stream.synchronize()
        return {k: self.a[k].cpu().numpy() for k in keys}


class Group:
    """Pools stepped together, each with its own parameters (say, lattice
    boxes on the uniform grid and clustered boxes on nested grids): every
    step forks the pools onto their own streams from the first pool's stream
    and joins them back, so their kernels overlap on the device, and one CUDA
    graph captures the whole step."""

    def __init__(self, pools: list[Pool]):
        if not pools:
            raise ValueError("a group needs at least one pool")
        self.pools = pools
        self.stream = pools[0].stream
        self.graph = None

    def start(self):
        for P in self.pools:
            P.start()

    def step(self):
        main = self.stream
        for P in self.pools[1:]:
            P.stream.wait_stream(main)
        for P in self.pools:
            with torch.cuda.stream(P.stream):
                sph.sph_step(P.ctx, P.pool)
        for P in self.pools[1:]:
            main.wait_stream(P.stream)

    def capture(self):
        """One graph for the step of every pool (after a warm-up step)."""
        self.step()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.step()
        self.graph = g
        return g

    def replay(self):
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def synchronize(self):
        """Waits for the step (a replayed graph runs on the first pool's stream)."""
        self.stream.synchronize()
        for P in self.pools[1:]:
            P.stream.synchronize()

    def status(self) -> int:
        self.synchronize()
        st = 0
        for P in self.pools:
            st |= P.status()
        return st

