"""The full-field ELBO (Eq. elbo over every pixel of every image) on the GPU
against the FP64 oracle, and against the per-source objective it contains."""
import numpy as np
import pytest
import torch

import fields
import oracle
from oracle import elbo as OE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1803_00113_gb300 import celeste
    return celeste


def _kl_sum(p):
    return sum(float(OE.kl_source(OE.Theta.from_vector(torch.as_tensor(p.theta[s])), p.model))
               for s in range(p.n_sources))


@pytest.mark.parametrize("kind", ["field", "blend"])
def test_field_elbo_matches_oracle(cel, kind):
    if kind == "field":
        p = fields.single_field(seed=5, n_sources=40, height=300, width=250)
    else:
        p = fields.batched(seed=71, n_sources=12, min_side=15, max_side=41, max_images_per_band=2,
                           max_neighbours=4)
    assert p.nbr_ptr[-1] > 0
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    fe = cel.FieldElbo(ctx, dp)
    out = fe().cpu().numpy().copy()
    again = fe().cpu().numpy()
    ctx.synchronize()
    assert np.array_equal(out, again)                  # deterministic
    ref = oracle.full_field_elbo(p)
    kl = _kl_sum(p)
    assert abs(out[0] - ref) <= 1e-6 * abs(ref), (out[0], ref)
    assert abs(out[2] - kl) <= 1e-5 * abs(kl) + 1e-3, (out[2], kl)
    assert abs(out[1] - (ref + kl)) <= 1e-6 * abs(ref), (out[1], ref + kl)


def test_field_change_equals_the_source_change(cel):
    """Moving one source changes the whole ELBO by exactly its own L_s change:
    L_s holds every term that depends on theta_s."""
    p = fields.batched(seed=72, n_sources=10, min_side=15, max_side=41, max_images_per_band=2,
                       max_neighbours=4)
    s = int(np.argmax(np.diff(p.nbr_ptr)))              # a source with neighbours
    ctx = cel.Context(p.model)
    dp = cel.DeviceProblem(p)
    fe = cel.FieldElbo(ctx, dp)
    plan = cel.Plan(ctx, dp, [s])
    F0 = float(fe()[0])
    L0 = float(cel.elbo(plan)[0][0])
    th = p.theta.copy()
    th[s, 21:23] += 0.3                                  # shift the position
    th[s, 1] += 0.05                                     # and the flux
    dp.set_theta(th)
    F1 = float(fe()[0])
    L1 = float(cel.elbo(plan)[0][0])
    ctx.synchronize()
    assert abs(L1 - L0) > 1.0
    assert abs((F1 - F0) - (L1 - L0)) <= 1e-4 * abs(L1 - L0) + 1e-6 * abs(F0), (F1 - F0, L1 - L0)
