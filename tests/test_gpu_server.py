"""The continuous-batching server: every replan served in a mix of sessions
(two dynamics kinds, uneven K and T, requests arriving while batches run) is
bitwise the replan of that session alone; the device-memory budget rejects
sessions it cannot hold."""
import time

import numpy as np
import pytest

import paper_2607_06499_b300 as pkg
from paper_2607_06499_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _wait(srv, tk, sid, timeout=30.0):
    t0 = time.time()
    while True:
        r = srv.poll(tk, sid)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "server did not answer"
        time.sleep(1e-4)


def test_server_results_equal_alone_over_two_rounds():
    scenes = [W.make("batch_instance", seed=s, n_replans=3) for s in range(10)]
    scenes += [W.make("arm_blocked", seed=s, K=700 + 50 * s, n_replans=3) for s in range(3)]
    srv = pkg.Server(mem_budget_bytes=8 << 30, max_batch=6, n_streams=3)
    sids = [srv.open(sc["cfg"], sc["radius"].shape[0]) for sc in scenes]
    alone = [pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0]) for sc in scenes]
    for rnd in range(2):
        tickets = []
        for sid, sc in zip(sids, scenes):   # arrive one by one while batches run
            tickets.append(srv.submit(sid, sc["x0"], W.history(sc, rnd), sc["radius"]))
        for i, (sid, sc) in enumerate(zip(sids, scenes)):
            u, diag, lat = _wait(srv, tickets[i], sid)
            u_ref, d_ref = alone[i].replan(sc["x0"], W.history(sc, rnd), sc["radius"])
            assert diag["status"] == 0 and lat > 0
            assert np.array_equal(u, u_ref), (rnd, i)
            assert diag["mode"] == d_ref["mode"] and diag["counter"] == rnd
    st = srv.stats()
    assert st["replans"] == 2 * len(scenes) and st["sessions_open"] == len(scenes)
    for sid in sids:
        srv.close_session(sid)
    srv.close()
    for pl in alone:
        pl.close()


def test_server_budget_rejects_and_releases():
    sc = W.make("unicycle", seed=0, K=4096)
    srv = pkg.Server(mem_budget_bytes=3 << 20, max_sessions=8)
    sid = srv.open(sc["cfg"], sc["radius"].shape[0])   # ~2.2 MB session
    assert sid is not None
    assert srv.open(sc["cfg"], sc["radius"].shape[0]) is None
    assert srv.stats()["sessions_rejected"] == 1
    srv.close_session(sid)
    assert srv.open(sc["cfg"], sc["radius"].shape[0]) is not None
    srv.close()


def test_server_replaces_a_queued_request():
    sc = W.make("unicycle", seed=1, K=16384, n_replans=4)
    srv = pkg.Server(mem_budget_bytes=8 << 30, n_streams=1)
    sids = [srv.open(sc["cfg"], sc["radius"].shape[0]) for _ in range(6)]
    # keep the single slot busy, then submit twice to one session
    for s in sids[:5]:
        srv.submit(s, sc["x0"], W.history(sc, 0), sc["radius"], want_result=False)
    t1 = srv.submit(sids[5], sc["x0"], W.history(sc, 0), sc["radius"])
    t2 = srv.submit(sids[5], sc["x0"], W.history(sc, 1), sc["radius"])
    r1 = _wait(srv, t1, sids[5])
    r2 = _wait(srv, t2, sids[5])
    if srv.stats()["superseded"] == 1:   # t2 arrived while t1 was still queued
        assert np.array_equal(r1[0], r2[0])
    else:                               # t1 had already been launched
        assert r2[1]["counter"] == r1[1]["counter"] + 1
    srv.close()


def test_server_sessions_closed_while_queued():
    """Sessions closed while their requests wait in the queue, under one
    instance per launch and one stream (the queue stays long): the stale queue
    entries are dropped, slots and pooled planners are reused, and the
    surviving sessions' replans still equal their replans alone."""
    sc = W.make("unicycle", seed=2, K=16384, n_replans=8)
    srv = pkg.Server(mem_budget_bytes=8 << 30, max_sessions=16, max_batch=1, n_streams=1)
    keep = srv.open(sc["cfg"], sc["radius"].shape[0])
    alone = pkg.Planner(sc["cfg"], n_obs_max=sc["radius"].shape[0])
    for rnd in range(6):
        churn = [srv.open(sc["cfg"], sc["radius"].shape[0]) for _ in range(6)]
        for s in churn:
            srv.submit(s, sc["x0"], W.history(sc, rnd), sc["radius"], want_result=False)
        tk = srv.submit(keep, sc["x0"], W.history(sc, rnd), sc["radius"])
        for s in churn[::-1]:   # most of these are still queued
            srv.close_session(s)
        u, diag, _ = _wait(srv, tk, keep)
        u_ref, _ = alone.replan(sc["x0"], W.history(sc, rnd), sc["radius"])
        assert diag["status"] == 0 and diag["counter"] == rnd
        assert np.array_equal(u, u_ref), rnd
    assert srv.stats()["sessions_open"] == 1
    srv.close()
    alone.close()
