"""The allocation-free entry point (celeste_elbo_grad_hess_noalloc).

It serves callers that must not allocate device memory (a locked or
defragmenting memory pool, a host program that owns every allocation), so
it keeps its intermediates in one fixed device array shared by all calls.
This file is collected last: the entry point must give the same results as
celeste_elbo_grad_hess whether it runs alone in a fresh process or after
every other test, and on consecutive calls that reuse the shared array.
"""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu

TOL_ELBO = 1e-5      # the parity tests' tolerances
TOL_DERIV = 1e-4


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _outputs(n, dev):
    return (torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n, 27), float("nan"), dtype=torch.float64, device=dev),
            torch.full((n, 27, 27), float("nan"), dtype=torch.float64, device=dev))


def _close(a, b):
    e, er, g, H = (t.cpu().numpy() for t in a)
    re, rer, rg, rH = (t.cpu().numpy() for t in b)
    assert np.all(np.abs(e - re) <= TOL_ELBO * np.abs(re))
    assert np.all(np.abs(er - rer) <= TOL_ELBO * np.maximum(np.abs(rer), 1.0))
    gs = np.abs(rg).max(axis=1, keepdims=True)
    assert np.all(np.abs(g - rg) <= TOL_DERIV * (np.abs(rg) + 1e-3 * gs))
    hs = np.abs(rH).reshape(len(rH), -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(H - rH) <= TOL_DERIV * (np.abs(rH) + 1e-3 * hs))


def _blend():
    return fields.batched(seed=61, n_sources=9, min_side=15, max_side=45, max_images_per_band=2,
                          max_neighbours=4)


def test_noalloc_matches_existing_entry_point_on_consecutive_calls(cel):
    p = _blend()
    dev = torch.device("cuda")
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    model = p.model
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    for sources in (list(range(p.n_sources)), [7, 2, 5]):
        plan = cel.Plan(ctx, dp, sources)
        ref = cel.elbo_grad_hess(plan)
        ctx.synchronize()
        out = _outputs(len(sources), dev)
        cel.elbo_grad_hess_noalloc(model, dp, sources, out, device_error=err)
        torch.cuda.synchronize()
        assert int(err[0]) == 0
        _close(out, ref)


def test_noalloc_matches_the_oracle(cel):
    """The FP64 oracle at the parity tests' tolerances, for the source with
    the most neighbours of the blend."""
    p = _blend()
    dev = torch.device("cuda")
    dp = cel.DeviceProblem(p)
    s = int(np.argmax(np.diff(p.nbr_ptr)))
    assert p.nbr_ptr[s + 1] > p.nbr_ptr[s]
    out = _outputs(1, dev)
    cel.elbo_grad_hess_noalloc(p.model, dp, [s], out)
    torch.cuda.synchronize()
    e, er, g, H = (t.cpu().numpy()[0] for t in out)
    ref = oracle.elbo_grad_hess(p, s)
    sc = oracle.abs_sum_scales(p, s)
    assert abs(e - ref["elbo"]) <= TOL_ELBO * abs(ref["elbo"])
    assert abs(er - ref["elbo_rel"]) <= TOL_ELBO * max(abs(ref["elbo_rel"]), sc["elbo"])
    assert np.all(np.abs(g - ref["grad"]) <= TOL_DERIV * np.maximum(np.abs(ref["grad"]), sc["grad"]))
    assert np.all(np.abs(H - ref["hess"]) <= TOL_DERIV * np.maximum(np.abs(ref["hess"]), sc["hess"]))


def test_noalloc_allocates_no_device_memory(cel):
    p = _blend()
    dev = torch.device("cuda")
    dp = cel.DeviceProblem(p)
    srcs = list(range(p.n_sources))
    out = _outputs(len(srcs), dev)
    cel.elbo_grad_hess_noalloc(p.model, dp, srcs, out)      # first call: set-up, module loads
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        cel.elbo_grad_hess_noalloc(p.model, dp, srcs, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 >= free0


def test_noalloc_on_a_side_stream_equals_the_default_stream(cel):
    p = _blend()
    dev = torch.device("cuda")
    dp = cel.DeviceProblem(p)
    srcs = [0, 3, 8]
    ref = _outputs(len(srcs), dev)
    cel.elbo_grad_hess_noalloc(p.model, dp, srcs, ref)
    side = torch.cuda.Stream()
    out = _outputs(len(srcs), dev)
    side.wait_stream(torch.cuda.current_stream())
    cel.elbo_grad_hess_noalloc(p.model, dp, srcs, out, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)


def test_noalloc_reports_non_finite_values_in_its_error_word(cel):
    p = _blend()
    p.theta[4, 1] = float("nan")      # galaxy mean log flux of one source
    dev = torch.device("cuda")
    dp = cel.DeviceProblem(p)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    cel.elbo_grad_hess_noalloc(p.model, dp, [4], _outputs(1, dev), device_error=err)
    torch.cuda.synchronize()
    assert int(err[0]) & cel.DERR_NONFINITE


def test_noalloc_rejects_requests_beyond_its_limits(cel):
    p = fields.plain_source(side=15)
    dp = cel.DeviceProblem(p)
    dev = torch.device("cuda")
    too_many = list(range(1025))      # more sources than CELESTE_NOALLOC_MAX_SOURCES
    with pytest.raises(cel.CelesteError, match="-8"):
        cel.elbo_grad_hess_noalloc(p.model, dp, too_many, _outputs(1025, dev))
    # a few large patches: within the pair and tile limits, beyond the bytes
    big = fields.batched(seed=62, n_sources=24, min_side=101, max_side=101,
                         max_images_per_band=6, max_neighbours=3)
    dbig = cel.DeviceProblem(big)
    srcs = list(range(big.n_sources))
    assert 5_000 < big.visits(srcs) // 256 < 32_768
    with pytest.raises(cel.CelesteError, match="-8"):
        cel.elbo_grad_hess_noalloc(big.model, dbig, srcs, _outputs(len(srcs), dev))


def test_noalloc_refuses_a_stream_under_capture(cel):
    p = _blend()
    dev = torch.device("cuda")
    dp = cel.DeviceProblem(p)
    out = _outputs(2, dev)
    cel.elbo_grad_hess_noalloc(p.model, dp, [0, 1], out)   # set-up outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    raised = None
    with torch.cuda.graph(graph, stream=side):
        try:
            cel.elbo_grad_hess_noalloc(p.model, dp, [0, 1], out, stream=side)
        except cel.CelesteError as e:
            raised = e
    assert raised is not None and "-1" in str(raised)
