"""Continuous-batching server: results in the mix equal results alone,
requests of one simulation complete in order, admission by the store's
budget."""
import numpy as np
import pytest

from paper_2305_13380_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2305_13380_gb300 import build
    build.build()


def _sims(k, n_min=1000, n_max=3000):
    return {s: inputs.two_spheres(seed=s, n_min=n_min, n_max=n_max) for s in range(k)}


def test_served_mix_equals_alone():
    import torch
    from paper_2305_13380_gb300 import pool, serve, sph
    sims = _sims(12)
    total = sum(len(p["x"]) for p in sims.values())
    prm = sph.sph_default_params(flags=sph.SPH_FLAG_TREE)
    # small arenas force several batches of mixed simulations
    srv = serve.Server(budget_bytes=4 << 30, store_particles=total, slots=3, batch_particles=9000,
                       params=prm)
    for sid, p in sims.items():
        assert srv.admit(sid, p)
    trace = serve.poisson_trace(36, rate=2000.0, sims=list(sims), seed=3)
    out = srv.run(trace)
    assert out["device_status"] == 0
    assert out["batches"] < len(trace)  # requests were batched
    steps = {sid: sum(1 for _, s in trace if s == sid) for sid in sims}
    # requests of one simulation complete in arrival order
    by_sim = {}
    for r in sorted(srv.finished, key=lambda r: r.rid):
        by_sim.setdefault(r.sid, []).append(r)
    for rs in by_sim.values():
        done = [r.t_done for r in rs]
        assert all(a < b for a, b in zip(done, done[1:]))
        assert all(r.t_done >= r.t_arrival for r in rs)
    for sid, p in sims.items():
        got = srv.host_state(sid)
        alone = pool.Pool([p], prm)
        alone.start()
        for _ in range(steps[sid]):
            alone.step()
        ref = alone.host()
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "ax", "du_dt", "v_sig"):
            assert np.array_equal(got[k], ref[k]), (sid, k)
    torch.cuda.synchronize()


def test_admission_waits_for_room():
    import torch
    from paper_2305_13380_gb300 import serve, sph
    sims = _sims(4, 2000, 2000)
    n = len(sims[0]["x"])
    srv = serve.Server(budget_bytes=2 << 30, store_particles=2 * n + 10, slots=1, batch_particles=4 * n,
                       params=sph.sph_default_params(flags=sph.SPH_FLAG_TREE))
    admitted = [srv.admit(s, p) for s, p in sims.items()]
    assert admitted == [True, True, False, False]
    srv.retire(0)
    assert set(srv.sims) == {1, 2}
    srv.retire(1)
    assert set(srv.sims) == {2, 3}
    torch.cuda.synchronize()


def test_pool_move_round_trip():
    # whole simulations gathered out of a spread store into a packed arena and
    # moved back: every field lands where it belongs, nothing else changes
    import torch
    from paper_2305_13380_gb300 import sph
    g = torch.Generator(device="cuda").manual_seed(0)
    n_store, ranges = 1000, [(700, 50), (10, 120), (400, 1), (900, 99)]
    keys = sph.POOL_FIELDS[:-1]

    def arrays(n):
        a = {k: torch.rand(n, generator=g, device="cuda",
                           dtype=torch.float64 if k in ("x", "y", "z") else torch.float32) for k in keys}
        a["dt"] = torch.zeros(1, dtype=torch.float64, device="cuda")
        return a
    store = arrays(n_store)
    before = {k: v.clone() for k, v in store.items()}
    total = sum(n for _, n in ranges)
    arena = arrays(total + 7)
    off = torch.tensor([0] + list(np.cumsum([n for _, n in ranges])), dtype=torch.int64, device="cuda")
    starts = torch.tensor([s for s, _ in ranges], dtype=torch.int64, device="cuda")
    box = torch.ones(1, dtype=torch.float64, device="cuda")
    sp = sph.pool(torch.tensor([0, n_store], dtype=torch.int64, device="cuda"), box, store)
    pk = sph.pool(torch.tensor([0, total + 7], dtype=torch.int64, device="cuda"), box, arena)
    sph.sph_pool_move(sp, pk, len(ranges), starts, off, True)
    torch.cuda.synchronize()
    for k in keys:
        for r, (s, n) in enumerate(ranges):
            o = int(off[r])
            assert torch.equal(arena[k][o:o + n], store[k][s:s + n]), k
    for k in keys:
        arena[k][:total] *= 2
    sph.sph_pool_move(sp, pk, len(ranges), starts, off, False)
    torch.cuda.synchronize()
    for k in keys:
        exp = before[k].clone()
        for s, n in ranges:
            exp[s:s + n] *= 2
        assert torch.equal(store[k], exp), k


def test_budgeted_store_pages_simulations_and_keeps_results():
    # the store holds about a third of the registered simulations: requests
    # admit simulations by evicting idle ones to host memory, and every
    # simulation's state still equals its run alone
    import torch
    from paper_2305_13380_gb300 import pool, serve, sph
    sims = _sims(9, 1500, 1500)
    n = len(sims[0]["x"])
    prm = sph.sph_default_params(flags=sph.SPH_FLAG_TREE)
    srv = serve.Server(budget_bytes=2 << 30, store_particles=3 * n + 100, slots=2, batch_particles=2 * n,
                       params=prm)
    for sid, p in sims.items():
        srv.register(sid, p)
    trace = serve.poisson_trace(30, rate=500.0, sims=list(sims), seed=4)
    out = srv.run(trace)
    assert out["device_status"] == 0
    assert srv.evictions > 0 and srv.uploads > len(sims)
    steps = {sid: sum(1 for _, s in trace if s == sid) for sid in sims}
    for sid, p in sims.items():
        got = srv.host_state(sid)
        alone = pool.Pool([p], prm)
        alone.start()
        for _ in range(steps[sid]):
            alone.step()
        ref = alone.host()
        for k in ("x", "vx", "u", "h", "rho", "ax", "du_dt", "v_sig"):
            assert np.array_equal(got[k], ref[k]), (sid, k)
    torch.cuda.synchronize()
