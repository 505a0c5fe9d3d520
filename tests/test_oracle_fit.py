"""Pins of the oracle's region fit (block coordinate ascent, Sec. 4.3, 4.4).

The fit is a schedule around the per-source subsolver, so it is pinned by
what block coordinate ascent must satisfy: the schedule and stopping rule
(checked with a stand-in subsolver), independence of sources that share a
colour (their order inside a class cannot matter, and a region of isolated
sources is the union of their independent fits), and the bookkeeping
identity: the summed gains of the accepted block steps equal the change of
the full-field ELBO (Eq. elbo over every pixel), which holds only if each
L_s contains every term that depends on theta_s.
"""
import numpy as np
import pytest

import fields
import oracle
from oracle import newton as ON


def _blend(seed=51, n=2, side=15):
    return fields.batched(seed=seed, n_sources=n, min_side=side, max_side=side,
                          max_images_per_band=1, max_neighbours=n - 1)


def test_overlap_classes_are_proper_greedy_and_restricted_to_the_region():
    p = fields.batched(seed=9, n_sources=60, min_side=15, max_side=41, max_images_per_band=2,
                       max_neighbours=6)
    nbrs = {s: set(int(t) for t in p.nbr_idx[p.nbr_ptr[s]:p.nbr_ptr[s + 1]])
            for s in range(p.n_sources)}
    assert any(nbrs.values())
    rng = np.random.default_rng(0)
    for region in (range(p.n_sources), sorted(rng.choice(p.n_sources, 35, replace=False))):
        region = [int(s) for s in region]
        classes = ON.overlap_classes(p, region)
        color = {s: c for c, cls in enumerate(classes) for s in cls}
        assert sorted(color) == sorted(region)
        for c, cls in enumerate(classes):
            assert cls == sorted(cls) and cls
            for s in cls:
                # proper: no two members of a class overlap
                assert not (nbrs[s] & set(cls))
                # greedy by ascending id: every smaller colour is taken by a
                # smaller-id neighbour inside the region
                lower = {color[t] for t in nbrs[s] if t in color and t < s}
                assert set(range(c)) <= lower


class _FakeSubsolver:
    """Stands in for newton_fit: records calls, returns scripted gains."""

    def __init__(self, gains_per_pass, n_region):
        self.calls = []
        self.gains = gains_per_pass
        self.n = n_region

    def __call__(self, work, s, theta, delta, max_iter, trace):
        k = len(self.calls) // self.n          # pass index
        self.calls.append((k, s, float(delta), max_iter))
        g = self.gains[min(k, len(self.gains) - 1)] / self.n
        trace.append(dict(status=ON.ST_ACCEPTED, elbo=0.0, theta=theta, delta=delta))
        trace.append(dict(status=ON.ST_CONVERGED, elbo=g, theta=theta, delta=delta))
        return theta + 1.0, delta, ON.ST_CONVERGED, 2


def test_region_fit_schedule_and_stopping_rule(monkeypatch):
    p = fields.batched(seed=9, n_sources=12, min_side=15, max_side=21, max_images_per_band=1,
                       max_neighbours=3)
    classes = ON.overlap_classes(p)
    assert len(classes) >= 2
    n = p.n_sources
    order = [s for c in classes for s in c]
    for gains, max_passes, expect in (([10.0, 0.5, 1e-4, 5.0], 5, 3),    # stops on a small pass
                                      ([10.0, 1.0], 2, 2),               # capped
                                      ([0.0], 5, 1),                     # nothing to gain
                                      ([10.0, 12e-3, 11e-3], 5, 3)):     # boundary: <= tol * n
        fake = _FakeSubsolver(gains, n)
        monkeypatch.setattr(ON, "newton_fit", fake)
        r = ON.region_fit(p, max_passes=max_passes, max_iter=7, pass_tol=1e-3)
        assert r["passes"] == expect, (gains, r["passes"])
        assert len(fake.calls) == expect * n
        for k in range(expect):
            chunk = fake.calls[k * n:(k + 1) * n]
            assert [s for _, s, _, _ in chunk] == order          # classes in colour order
            assert all(d == ON.DELTA0 and m == 7 for _, _, d, m in chunk)  # fresh calls
        np.testing.assert_allclose(r["pass_gains"], [gains[min(k, len(gains) - 1)]
                                                     for k in range(expect)])
        np.testing.assert_allclose(r["theta"], p.theta + expect, rtol=0, atol=1e-12)
        assert all(v == 2 * expect for v in r["iters"].values())


def test_isolated_sources_fit_independently_and_in_any_order():
    p = fields.batched(seed=12, n_sources=2, min_side=15, max_side=15, max_images_per_band=1,
                       max_neighbours=0)
    assert p.nbr_ptr[-1] == 0
    assert ON.overlap_classes(p) == [[0, 1]]
    r = ON.region_fit(p, max_passes=1, max_iter=3)
    rr = ON.region_fit(p, max_passes=1, max_iter=3, order=lambda c: c[::-1])
    assert np.array_equal(r["theta"], rr["theta"])
    for s in range(2):
        th, _, st, it = ON.newton_fit(p, s, max_iter=3)
        assert np.array_equal(r["theta"][s], th)
        assert r["status"][s] == st and r["iters"][s] == it


def test_fit_gains_equal_the_change_of_the_full_field_elbo():
    p = _blend()
    assert p.nbr_ptr[-1] > 0, "the sources must overlap"
    L0 = oracle.full_field_elbo(p)
    r = ON.region_fit(p, max_passes=2, max_iter=3, pass_tol=0.0)
    assert r["passes"] == 2 and len(r["gains"]) >= 2
    assert all(g > 0 for g in r["gains"])     # every accepted block step climbs
    L1 = oracle.full_field_elbo(p, r["theta"])
    total = float(np.sum(r["gains"]))
    assert abs((L1 - L0) - total) <= 1e-9 * abs(L0) + 1e-7 * abs(total), (L1 - L0, total)
