"""Serving many live simulations on one GPU: resident state, admission by an
HBM budget, and continuous batching of step requests.

State.  Every admitted simulation keeps its particles resident in one device
store (structure of arrays, one contiguous range per simulation, handed out
by a first-fit allocator).  A simulation is admitted only while its range fits
in the store, so the resident set never exceeds the budget it was sized for.
Registered simulations may outnumber what the store holds: each keeps a
pinned host copy, and a request for one that is not resident admits it,
evicting the least recently used idle simulations (their state copied back to
the host after their last batch) until its range fits.

Requests.  A request asks for one KDK step of one simulation.  Requests of the
same simulation run in arrival order, one at a time.

Continuous batching.  Up to `slots` batches are in flight, each on its own
CUDA stream with its own context and arena.  Whenever a slot is free, the
pending requests (oldest first, at most one per simulation, up to the arena's
particle capacity) form a batch: their simulations' ranges are gathered into
the arena (one index kernel per field), one sph_step advances all of them in
one launch per kernel, and the results are scattered back.  Requests that
arrive while other batches run are admitted as soon as a slot and arena room
free up, and their batch overlaps the running ones on the device.

Every step of the SPH computation runs in the CUDA library (sph_step); this
module only moves state between the store and the arenas and keeps the books.
A simulation's step does not depend on which others share its batch (every
kernel works per simulation and sums in a fixed order), so results in the mix
equal results alone.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import sph

F64 = ("x", "y", "z")
F32 = ("vx", "vy", "vz", "u", "m", "h", "ax", "ay", "az", "du_dt", "v_sig", "rho", "f", "div_v",
       "curl_v", "P", "c", "balsara")
STATE_BYTES = 8 * len(F64) + 4 * len(F32)
# context scratch per particle of an arena: cell keys and counts, sorted
# copies and lists (~570 B) plus the nested grids' keys, orders, groups and
# their ranges, copies, lists (8 lanes x 32 entries) and reverse pairs
# (~2350 B), for 1.25 n + 64 particles of capacity; rounded up
SCRATCH_BYTES = 3700


class Store:
    """Device SoA of `capacity` particles with a first-fit range allocator."""

    def __init__(self, capacity: int, device="cuda"):
        self.capacity = int(capacity)
        self.a = {k: torch.zeros(self.capacity, dtype=torch.float64, device=device) for k in F64}
        self.a.update({k: torch.zeros(self.capacity, dtype=torch.float32, device=device) for k in F32})
        self.free = [(0, self.capacity)]  # sorted (start, length)

    def alloc(self, n: int):
        for i, (s, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, ln - n)
                return s
        return None

    def release(self, start: int, n: int):
        self.free.append((start, n))
        self.free.sort()
        merged = []
        for s, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == s:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((s, ln))
        self.free = merged

    def view(self, start: int, n: int) -> dict:
        return {k: v[start:start + n] for k, v in self.a.items()}


@dataclasses.dataclass
class Sim:
    sid: int
    n: int
    L: float
    start: int
    busy: bool = False
    steps: int = 0
    resident: bool = True
    host: dict | None = None       # pinned copy of the state (registered simulations)
    last_event: object = None      # completion of the last batch that touched the state
    ready: object = None           # completion of its upload, for the next batch to wait on
    last_use: int = 0


@dataclasses.dataclass
class Request:
    rid: int
    sid: int
    t_arrival: float   # seconds on the server's clock
    t_done: float = float("nan")
    batch: int = -1


class _Slot:
    def __init__(self, params: sph.sph_params, capacity: int, max_sims: int, device="cuda"):
        self.stream = torch.cuda.Stream()
        self.ctx = sph.Context(params, self.stream)
        self.capacity = capacity
        self.a = {k: torch.zeros(capacity, dtype=torch.float64, device=device) for k in F64}
        self.a.update({k: torch.zeros(capacity, dtype=torch.float32, device=device) for k in F32})
        self.a["dt"] = torch.zeros(max_sims, dtype=torch.float64, device=device)
        self.off_h = torch.zeros(max_sims + 1, dtype=torch.int64).pin_memory()
        self.box_h = torch.zeros(max_sims, dtype=torch.float64).pin_memory()
        self.meta_h = torch.zeros(3 * max_sims, dtype=torch.int64).pin_memory()
        self.off = torch.zeros(max_sims + 1, dtype=torch.int64, device=device)
        self.box = torch.zeros(max_sims, dtype=torch.float64, device=device)
        self.meta = torch.zeros(3 * max_sims, dtype=torch.int64, device=device)
        self.begin = torch.cuda.Event(enable_timing=True)
        self.done = torch.cuda.Event(enable_timing=True)
        self.requests: list[Request] = []
        self.particles = 0
        self.sims: list[Sim] = []


class Server:
    """Continuous-batching server of SPH step requests.

    budget_bytes bounds the device memory of the store, the arenas and the
    contexts' scratch; `slots` batches may be in flight; each arena holds up to
    `batch_particles` particles (default: what the budget leaves)."""

    def __init__(self, budget_bytes: int, store_particles: int, slots: int = 3,
                 batch_particles: int | None = None, max_batch_sims: int = 256,
                 params: sph.sph_params | None = None):
        self.params = params if params is not None else sph.sph_default_params(
            flags=sph.SPH_FLAG_TREE)
        store_bytes = store_particles * STATE_BYTES
        left = budget_bytes - store_bytes
        per_slot_particle = STATE_BYTES + SCRATCH_BYTES
        fit = left // (slots * per_slot_particle)
        if batch_particles is None:
            batch_particles = fit
        if batch_particles < 1 or batch_particles > fit:
            raise ValueError(f"budget {budget_bytes / 1e9:.1f} GB holds the store and "
                             f"{fit} particles per slot; asked {batch_particles}")
        self.store = Store(store_particles)
        self.store_pool = sph.pool(torch.tensor([0, store_particles], dtype=torch.int64, device="cuda"),
                                   torch.ones(1, dtype=torch.float64, device="cuda"),
                                   dict(self.store.a, dt=torch.zeros(1, dtype=torch.float64, device="cuda")))
        self.slots = [_Slot(self.params, int(batch_particles), max_batch_sims) for _ in range(slots)]
        for sl in self.slots:
            # no step of a slot allocates: its latency carries no cudaMalloc
            sph.sph_reserve(sl.ctx, int(batch_particles), max_batch_sims)
        self.batch_particles = int(batch_particles)
        self.max_batch_sims = max_batch_sims
        self.sims: dict[int, Sim] = {}
        self.pending: collections.deque[Request] = collections.deque()
        self.waiting_sims: collections.deque[tuple[int, dict]] = collections.deque()
        self.finished: list[Request] = []
        self.n_batches = 0
        self.updates = 0
        self.ref = torch.cuda.Event(enable_timing=True)
        self.t0 = None
        self.status = 0
        self.admit_ctx = None
        self.batch_log: list[tuple[int, int, float]] = []  # (simulations, particles, device ms)
        # registered simulations live in pinned host memory when not resident;
        # evictions and uploads run on their own stream
        self.transfer = torch.cuda.Stream()
        self.uploads = 0
        self.evictions = 0
        self.use_clock = 0

    # -------------------------------------------------------------- clock --
    def start_clock(self):
        torch.cuda.synchronize()
        self.ref.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # ---------------------------------------------------------- admission --
    def admit(self, sid: int, sim: dict) -> bool:
        """Makes a simulation resident (upload and first density + force)
        if the store has room; otherwise it waits for room."""
        n = len(sim["x"])
        if n > self.batch_particles:
            raise ValueError(f"simulation {sid} ({n} particles) exceeds the batch capacity")
        start = self.store.alloc(n)
        if start is None:
            self.waiting_sims.append((sid, sim))
            return False
        v = self.store.view(start, n)
        for k in F64:
            v[k].copy_(torch.as_tensor(np.asarray(sim[k], dtype=np.float64)))
        for k, src in (("vx", "vx"), ("vy", "vy"), ("vz", "vz"), ("u", "u"), ("m", "m"), ("h", "h0")):
            v[k].copy_(torch.as_tensor(np.asarray(sim[src], dtype=np.float32)))
        for k in ("ax", "ay", "az", "du_dt", "v_sig"):
            v[k].zero_()
        # first density + force (a step with dt = 0) on a synchronous context,
        # which rebuilds the cells when a starting h was too small
        if self.admit_ctx is None:
            q = sph.sph_params.from_buffer_copy(self.params)
            q.flags |= sph.SPH_FLAG_SYNC
            self.admit_ctx = sph.Context(q)
        off = torch.tensor([0, n], dtype=torch.int64, device="cuda")
        box = torch.tensor([float(sim["L"])], dtype=torch.float64, device="cuda")
        arr = dict(v)
        arr["dt"] = torch.zeros(1, dtype=torch.float64, device="cuda")
        sph.sph_step(self.admit_ctx, sph.pool(off, box, arr))
        torch.cuda.current_stream().synchronize()
        self.sims[sid] = Sim(sid, n, float(sim["L"]), start)
        return True

    # ------------------------------------------ registered simulations --
    def register(self, sid: int, sim: dict):
        """A live simulation whose state may leave the device: its state is
        kept in pinned host memory, it is made resident (evicting idle
        simulations if the store is full) and gets its first density + force.
        Later requests admit it again whenever it was evicted."""
        n = len(sim["x"])
        if n > self.batch_particles or n > self.store.capacity:
            raise ValueError(f"simulation {sid} ({n} particles) exceeds the batch or store capacity")
        host = {k: torch.empty(n, dtype=torch.float64, pin_memory=True) for k in F64}
        host.update({k: torch.zeros(n, dtype=torch.float32, pin_memory=True) for k in F32})
        for k in F64:
            host[k].copy_(torch.as_tensor(np.asarray(sim[k], dtype=np.float64)))
        for k, src in (("vx", "vx"), ("vy", "vy"), ("vz", "vz"), ("u", "u"), ("m", "m"), ("h", "h0")):
            host[k].copy_(torch.as_tensor(np.asarray(sim[src], dtype=np.float32)))
        sm = Sim(sid, n, float(sim["L"]), -1, resident=False, host=host)
        self.sims[sid] = sm
        if not self._make_resident(sm, set()):
            raise RuntimeError("no room in the store even after evicting every idle simulation")
        # first density + force on the transfer stream (synchronous context)
        if self.admit_ctx is None:
            q = sph.sph_params.from_buffer_copy(self.params)
            q.flags |= sph.SPH_FLAG_SYNC
            self.admit_ctx = sph.Context(q, self.transfer)
        with torch.cuda.stream(self.transfer):
            off = torch.tensor([0, n], dtype=torch.int64, device="cuda")
            box = torch.tensor([sm.L], dtype=torch.float64, device="cuda")
            arr = self.store.view(sm.start, n)
            arr["dt"] = torch.zeros(1, dtype=torch.float64, device="cuda")
            sph.sph_step(self.admit_ctx, sph.pool(off, box, arr))
        self.transfer.synchronize()
        sm.ready = None

    def _make_resident(self, sm: Sim, exclude: set) -> bool:
        """Gives a registered simulation a range of the store and uploads its
        state (on the transfer stream), evicting the least recently used idle
        simulations (not busy, not in `exclude`) while no range fits."""
        if sm.resident:
            return True
        while True:
            start = self.store.alloc(sm.n)
            if start is not None:
                break
            idle = [o for o in self.sims.values()
                    if o.resident and not o.busy and o.host is not None and o.sid not in exclude]
            if not idle:
                return False
            self._evict(min(idle, key=lambda o: o.last_use))
        sm.start, sm.resident = start, True
        v = self.store.view(start, sm.n)
        with torch.cuda.stream(self.transfer):
            for k in F64 + F32:
                v[k].copy_(sm.host[k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.transfer)
        sm.ready = ev
        self.uploads += 1
        return True

    def _evict(self, sm: Sim):
        """Copies a resident simulation's state to its pinned host copy after
        its last batch, and frees its range (the next upload into that range
        runs after the copy, on the same stream)."""
        v = self.store.view(sm.start, sm.n)
        with torch.cuda.stream(self.transfer):
            if sm.last_event is not None:
                self.transfer.wait_event(sm.last_event)
            for k in F64 + F32:
                sm.host[k].copy_(v[k], non_blocking=True)
        self.store.release(sm.start, sm.n)
        sm.resident, sm.start, sm.ready = False, -1, None
        self.evictions += 1

    def retire(self, sid: int):
        """Frees a simulation's range and admits waiting ones that now fit."""
        s = self.sims.pop(sid)
        self.store.release(s.start, s.n)
        while self.waiting_sims:
            wsid, wsim = self.waiting_sims[0]
            if not any(ln >= len(wsim["x"]) for _, ln in self.store.free):
                break
            self.waiting_sims.popleft()
            self.admit(wsid, wsim)

    def host_state(self, sid: int, keys=("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax",
                                         "ay", "az", "du_dt", "v_sig")) -> dict:
        torch.cuda.synchronize()
        s = self.sims[sid]
        if not s.resident:
            return {k: s.host[k].numpy().copy() for k in keys}
        v = self.store.view(s.start, s.n)
        return {k: v[k].cpu().numpy() for k in keys}

    # ------------------------------------------------------------ requests --
    def submit(self, sid: int, t_arrival: float, rid: int):
        self.pending.append(Request(rid, sid, t_arrival))

    def _form_batch(self, slot: _Slot) -> bool:
        reqs, sims, total = [], [], 0
        taken = set()
        kept = collections.deque()
        while self.pending and len(reqs) < self.max_batch_sims:
            r = self.pending.popleft()
            s = self.sims[r.sid]
            if s.busy or r.sid in taken or total + s.n > slot.capacity:
                kept.append(r)
                continue
            if not s.resident and not self._make_resident(s, taken):
                kept.append(r)  # no room until running batches finish
                continue
            reqs.append(r)
            sims.append(s)
            taken.add(r.sid)
            total += s.n
        # requests left behind keep their order ahead of later arrivals
        kept.extend(self.pending)
        self.pending = kept
        if not reqs:
            return False
        ns = len(sims)
        counts = np.array([s.n for s in sims], dtype=np.int64)
        slot.off_h[0] = 0
        slot.off_h[1:ns + 1] = torch.from_numpy(np.cumsum(counts))
        slot.box_h[:ns] = torch.tensor([s.L for s in sims], dtype=torch.float64)
        slot.meta_h[:ns] = torch.from_numpy(np.array([s.start for s in sims], dtype=np.int64))
        st = slot.stream
        slot.done = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            for sm in sims:
                if sm.ready is not None:  # freshly uploaded
                    st.wait_event(sm.ready)
                    sm.ready = None
            slot.begin.record(st)
            slot.off[:ns + 1].copy_(slot.off_h[:ns + 1], non_blocking=True)
            slot.box[:ns].copy_(slot.box_h[:ns], non_blocking=True)
            slot.meta[:ns].copy_(slot.meta_h[:ns], non_blocking=True)
            view = {k: v[:total] for k, v in slot.a.items() if k != "dt"}
            view["dt"] = slot.a["dt"][:ns]
            packed = sph.pool(slot.off[:ns + 1], slot.box[:ns], view)
            # gather the simulations out of the store, step them, put them back
            sph.sph_pool_move(self.store_pool, packed, ns, slot.meta[:ns], slot.off[:ns + 1], True, st)
            sph.sph_step(slot.ctx, packed)
            sph.sph_pool_move(self.store_pool, packed, ns, slot.meta[:ns], slot.off[:ns + 1], False, st)
            slot.done.record(st)
        self.use_clock += 1
        for s in sims:
            s.busy = True
            s.last_event = slot.done
            s.last_use = self.use_clock
        for r in reqs:
            r.batch = self.n_batches
        slot.requests, slot.sims = reqs, sims
        slot.particles = total
        self.n_batches += 1
        self.updates += total
        return True

    def poll(self) -> int:
        """Completes finished batches; returns how many slots are free."""
        free = 0
        for slot in self.slots:
            if slot.requests and slot.done.query():
                t = self.ref.elapsed_time(slot.done) / 1e3
                self.batch_log.append((len(slot.sims), slot.particles, slot.begin.elapsed_time(slot.done)))
                self.status |= sph.sph_status(slot.ctx)
                for r in slot.requests:
                    r.t_done = t
                    self.finished.append(r)
                for s in slot.sims:
                    s.busy = False
                    s.steps += 1
                slot.requests, slot.sims = [], []
            if not slot.requests:
                free += 1
        return free

    def schedule(self):
        for slot in self.slots:
            if not slot.requests and self.pending:
                if not self._form_batch(slot):
                    break

    def run(self, trace, idle_sleep: float = 2e-5) -> dict:
        """Replays `trace` (a list of (t_arrival seconds, sim id)) in real time
        and returns latency and throughput figures."""
        trace = sorted(trace)
        self.start_clock()
        i = 0
        n = len(trace)
        while len(self.finished) < n:
            t = self.now()
            while i < n and trace[i][0] <= t:
                self.submit(trace[i][1], trace[i][0], i)
                i += 1
            self.poll()
            self.schedule()
            if i < n and not any(s.requests for s in self.slots) and not self.pending:
                time.sleep(max(0.0, min(trace[i][0] - self.now(), 1e-3)))
            else:
                time.sleep(idle_sleep)
        torch.cuda.synchronize()
        wall = self.now()
        lat = np.array([r.t_done - r.t_arrival for r in self.finished])
        log = np.array(self.batch_log[-self.n_batches:] or [(0, 0, 0.0)], dtype=np.float64)
        return {"requests": n, "batches": self.n_batches, "wall_s": wall,
                "batch_sims_mean": float(log[:, 0].mean()), "batch_particles_mean": float(log[:, 1].mean()),
                "batch_ms_mean": float(log[:, 2].mean()), "batch_ms_max": float(log[:, 2].max()),
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3),
                "particle_updates": int(self.updates),
                "particle_updates_per_s": self.updates / wall,
                "mean_sims_per_batch": n / max(self.n_batches, 1),
                "device_status": int(self.status)}


def poisson_trace(n_requests: int, rate: float, sims: list[int], seed: int = 0):
    """Poisson arrivals at `rate` per second, each for a uniformly chosen
    simulation."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    who = rng.choice(np.asarray(sims), n_requests)
    return [(float(a), int(b)) for a, b in zip(t, who)]
