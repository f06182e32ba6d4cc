"""Serving loop (rb_submit / rb_poll) on the GPU: continuous batching over
several resident events of different durations, detector sets and bin counts.

* every result in the mix equals the same request evaluated alone (bitwise:
  each walker is computed by one warp, independent of the others), also when
  several requests share one launch and the launch is padded;
* requests overlap on the device (more than one in flight) when slots and the
  memory budget allow it, and are serialised when the budget admits one;
* admission refusal (RB_EBUSY), poll timeouts and unknown tickets.
"""
import time

import numpy as np
import pytest
import torch

import synth
from tests._events import inject

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2404_11397_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def events(rb):
    specs = [(64.0, ("H1", "L1"), 100), (128.0, ("H1", "L1", "V1"), 500), (64.0, ("H1",), 300),
             (128.0, ("L1", "V1"), 800)]
    out = []
    for T, sites, B in specs:
        ev = inject(synth.make_event("C2", T=T, sites=sites))
        out.append(rb.Event.from_synth(ev, n_bins=B))
    return out


def _alone(rb, event, th, mode="mixed"):
    L, G = rb.loglike_grad(event, torch.tensor(th, device="cuda"), mode=mode)
    return L.cpu().numpy(), G.cpu().numpy()


@pytest.mark.parametrize("use_graphs", [True, False])
def test_mix_equals_alone(rb, events, use_graphs):
    pool = synth.walkers("C2", 3000)
    rng = np.random.default_rng(7)
    srv = rb.Server(max_slots=4, max_walkers=4096, use_graphs=use_graphs)
    reqs = []
    for i in range(24):
        e = int(rng.integers(0, len(events)))
        W = int(rng.integers(1, 3000))
        off = int(rng.integers(0, 3000 - W + 1))
        th = pool[off:off + W]
        reqs.append((srv.submit(events[e], th, want_grad=True), e, th))
    for i, (t, e, th) in enumerate(reqs):
        if i == 12:
            srv._req.clear()  # the rest are sized from the library's record of each ticket
        st, L, G = srv.poll(t, timeout_us=-1)
        assert st == rb.RB_OK
        La, Ga = _alone(rb, events[e], th)
        np.testing.assert_array_equal(L, La)
        np.testing.assert_array_equal(G, Ga)
    stats = srv.stats()
    assert stats["completed"] == stats["submitted"] == 24
    launches = stats["graph_launches"] if use_graphs else stats["plain_launches"]
    assert 1 <= launches <= 24
    if use_graphs:
        assert stats["graphs_captured"] >= 1 and stats["graphs_captured"] + stats["graph_updates"] == launches
    assert stats["walkers_requested"] == sum(th.shape[0] for _, _, th in reqs)
    assert 0 <= stats["walkers_run"] - stats["walkers_requested"] < 256 * launches
    srv.close()


def test_pending_requests_share_launches(rb, events):
    """With one slot, requests for the same event that queue behind a running
    launch are packed into the next one; each still gets its own results."""
    pool = synth.walkers("C2", 4096)
    srv = rb.Server(max_slots=1, max_walkers=8192)
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(40):
        W = int(rng.integers(1, 700))
        th = pool[(37 * i) % 3000:(37 * i) % 3000 + W]
        e = 1 if i % 4 else 3
        reqs.append((srv.submit(events[e], th, want_grad=i % 5 != 0), e, th, i % 5 != 0))
    for t, e, th, g in reqs:
        st, L, G = srv.poll(t, timeout_us=-1)
        assert st == rb.RB_OK and (G is not None) == g
        La, Ga = _alone(rb, events[e], th)
        np.testing.assert_array_equal(L, La)
        if g:
            np.testing.assert_array_equal(G, Ga)
    stats = srv.stats()
    assert stats["completed"] == 40
    assert stats["graph_launches"] < 40  # some launches carried several requests
    srv.close()


def test_requests_overlap_and_budget_serialises(rb, events):
    pool = synth.walkers("C2", 4096)
    srv = rb.Server(max_slots=8, max_walkers=4096)
    ts = [srv.submit(events[1], pool, want_grad=True) for _ in range(16)]
    for t in ts:
        assert srv.poll(t, 4096)[0] == rb.RB_OK
    assert srv.stats()["max_in_flight"] > 1
    srv.close()
    # a budget that admits one 4096-walker request at a time
    one = 4096 * (8 * 27 + 1024)
    srv = rb.Server(max_slots=8, max_walkers=4096, hbm_budget_bytes=one)
    ts = [srv.submit(events[1], pool, want_grad=True) for _ in range(8)]
    for t in ts:
        assert srv.poll(t, 4096)[0] == rb.RB_OK
    assert srv.stats()["max_in_flight"] == 1
    srv.close()


def test_admission_refusal_and_polls(rb, events):
    pool = synth.walkers("C2", 4096)
    srv = rb.Server(max_slots=1, max_queue=1, max_walkers=4096)
    accepted, busy = [], 0
    for _ in range(64):
        try:
            accepted.append(srv.submit(events[1], pool, want_grad=True))
        except rb.RBError as e:
            assert e.status == rb.RB_EBUSY
            busy += 1
    assert busy > 0 and accepted
    st, _, _ = srv.poll(accepted[-1], 4096, timeout_us=0)
    assert st in (rb.RB_OK, rb.RB_PENDING)
    for t in accepted:
        st = rb.RB_PENDING
        deadline = time.time() + 60
        while st != rb.RB_OK and time.time() < deadline:
            st, L, G = srv.poll(t, 4096, timeout_us=1000)
            assert st in (rb.RB_OK, rb.RB_ETIMEDOUT)
        assert st == rb.RB_OK
    with pytest.raises(rb.RBError) as e:
        srv.poll(accepted[0], 4096)  # already collected
    assert e.value.status == rb.RB_ENOTFOUND
    srv._req.clear()
    with pytest.raises(rb.RBError) as e:
        srv.poll(accepted[0])  # nor known to the library
    assert e.value.status == rb.RB_ENOTFOUND
    assert srv.stats()["rejected"] == busy
    srv.close()
