"""Serving: region requests submitted to the native server, batched on the
GPU, against the region fit run directly and against themselves run alone."""
import numpy as np
import pytest
import torch

import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _requests():
    return [fields.region_request(700 + k, n_sources=n, side=side)
            for k, (n, side) in enumerate([(3, 48), (6, 80), (1, 33), (9, 120)])]


def _collect(srv, tickets):
    out = {}
    for t in tickets:
        r = None
        for _ in range(600):
            r = srv.poll(t, wait_ms=100)
            if r is not None:
                break
        assert r is not None, "request did not finish"
        assert r["code"] == 0, (r["code"], hex(r["device_error"]))
        out[t] = r
    return out


def test_request_result_equals_the_region_fit(cel):
    req = _requests()[1]
    srv = cel.Server(req.model, workers=1)
    res = _collect(srv, [srv.submit(req)])
    srv.close()
    (r,) = res.values()
    ctx = cel.Context(req.model)
    dp = cel.DeviceProblem(req)
    fit = cel.Fit(ctx, dp, range(req.n_sources))
    passes, _ = fit.run(max_passes=5, max_iter=50, pass_tol=1e-3)
    st = fit.results()[0].cpu().numpy()
    assert r["passes"] == passes
    assert np.array_equal(r["theta"], dp.theta.cpu().numpy())
    assert np.array_equal(r["status"], st)


def test_a_request_arriving_mid_run_joins_at_a_pass_boundary(cel):
    """Continuous batching: a request submitted while another runs is
    admitted before that one finishes, and its result is bitwise the one it
    gets alone."""
    import time
    big = fields.region_request(777, n_sources=64, side=400)
    small = fields.region_request(702, n_sources=2, side=40)
    srv = cel.Server(big.model, workers=1)
    # the small request alone first: it also leaves the worker set up and
    # idle, so the big request is admitted as soon as it is submitted
    alone = _collect(srv, [srv.submit(small)]).popitem()[1]
    t_big = srv.submit(big)
    time.sleep(0.02)                       # the big request is on the GPU
    t_small = srv.submit(small)
    res = _collect(srv, [t_small, t_big])
    srv.close()
    b, s = res[t_big], res[t_small]
    assert b["passes"] >= 2
    # admitted after the big request started and before it finished ...
    assert b["t_start_s"] < s["t_start_s"] < b["t_done_s"]
    assert s["batch_requests"] == 2
    # ... with the result it has alone
    assert s["passes"] == alone["passes"]
    assert np.array_equal(s["theta"], alone["theta"])
    assert np.array_equal(s["status"], alone["status"])


def test_alone_equals_batched_with_others(cel):
    reqs = _requests()
    alone = {}
    srv = cel.Server(reqs[0].model, workers=1)
    for k, q in enumerate(reqs):
        alone[k] = _collect(srv, [srv.submit(q)]).popitem()[1]
        assert alone[k]["batch_requests"] == 1
    srv.close()
    # the same requests queued together start as one running set (one
    # segmented fit; requests leave it as their segments stop)
    srv = cel.Server(reqs[0].model, workers=1, start_paused=True)
    order = [2, 0, 3, 1]
    tickets = {k: srv.submit(reqs[k]) for k in order}
    srv.pause(False)
    mixed = _collect(srv, [tickets[k] for k in order])
    st = srv.stats()
    srv.close()
    assert st["batches"] == 1 and st["worker_error"] == 0 and st["launches"] > 0
    for k in order:
        m = mixed[tickets[k]]
        assert m["batch_requests"] == len(reqs)
        assert m["passes"] == alone[k]["passes"]
        assert np.array_equal(m["theta"], alone[k]["theta"]), k
        assert np.array_equal(m["status"], alone[k]["status"]), k


def test_admission_and_errors(cel):
    reqs = _requests()
    srv = cel.Server(reqs[0].model, workers=1, device_bytes=1 << 16)
    with pytest.raises(cel.CelesteError) as e:
        srv.submit(reqs[3])
    assert e.value.code == cel.ETOOLARGE
    srv.close()
    srv = cel.Server(reqs[0].model, workers=1, start_paused=True, queue_bytes=1)
    with pytest.raises(cel.CelesteError) as e:
        srv.submit(reqs[2])
    assert e.value.code == cel.EAGAIN
    srv.close()
    srv = cel.Server(reqs[0].model, workers=1, start_paused=True)
    bad = fields.region_request(701, n_sources=2, side=40)
    bad.patch_x0 = bad.patch_x0.copy()
    bad.patch_x0[0] = 39          # patch sticks out of its image
    with pytest.raises(cel.CelesteError) as e:
        srv.submit(bad)
    assert e.value.code == -1
    t = srv.submit(reqs[2])
    assert srv.poll(t) is None    # queued while paused
    srv.pause(False)
    _collect(srv, [t])
    with pytest.raises(cel.CelesteError):
        srv.poll(t)               # collected tickets are forgotten
    srv.close()
