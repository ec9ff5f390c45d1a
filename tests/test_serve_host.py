"""Host-side books of the server (CPU): the store's range allocator and the
request trace."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_store_ranges_first_fit_and_merge(monkeypatch):
    from paper_2305_13380_gb300 import serve
    st = serve.Store(100, device="cpu")
    a = st.alloc(30)
    b = st.alloc(30)
    c = st.alloc(30)
    assert (a, b, c) == (0, 30, 60)
    assert st.alloc(20) is None
    st.release(b, 30)
    assert st.alloc(40) is None
    assert st.alloc(25) == 30
    st.release(a, 30)
    st.release(30, 25)
    assert st.free == [(0, 60), (90, 10)]
    assert st.alloc(60) == 0


def test_poisson_trace_rate_and_choice():
    from paper_2305_13380_gb300 import serve
    tr = serve.poisson_trace(20000, rate=1000.0, sims=[3, 5, 7], seed=1)
    t = np.array([a for a, _ in tr])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 1000.0) < 30.0
    who = np.array([s for _, s in tr])
    assert set(who) == {3, 5, 7}
