"""The seeded generators behind every workload (CPU): the recipe each workload states (sizes,
ranges, duration laws, bursty and Zipf times, degree skew) holds, and the draws are
deterministic and independent of the thread count."""
import numpy as np
import pytest

import synth
from synth import WORKLOADS, scaled


def test_tiny_workload_recipe():
    el = synth.rmat(WORKLOADS[1].graph)
    assert el.n == 1 << 13 and el.src.shape[0] == 100_000
    for a in (el.src, el.dst):
        assert a.min() >= 0 and a.max() < el.n
    assert el.t.max() < 1 << 20 and el.lam.min() >= 1 and el.lam.max() <= 100
    assert abs(el.lam.mean() - 50.5) < 0.5          # U[1, 100]
    assert abs(el.t.mean() / (1 << 19) - 1) < 0.01   # U[0, 2^20)


def test_medium_laws_at_smaller_size():
    """Geometric durations with mean 50 (p = 1/50 on {1, 2, ...}); 80% of departures in 10
    Gaussian bursts of sigma 2^12 over [0, 2^24), the rest uniform; R-MAT degree skew."""
    spec = scaled(WORKLOADS[2].graph, 16, 1 << 21)
    el = synth.rmat(spec)
    lam = el.lam.astype(np.float64)
    assert lam.min() >= 1 and abs(lam.mean() - 50.0) < 0.5
    assert abs((lam == 1).mean() - 1 / 50) < 0.002   # P(1) = p
    assert el.t.max() < 1 << 24
    hist = np.bincount(el.t >> 12, minlength=1 << 12)  # bins one sigma wide
    top = np.sort(hist)[::-1]
    assert top[:80].sum() / el.t.size > 0.75  # the bursts: about 60 of 4096 bins hold 80%
    assert top[1000:].sum() / el.t.size > 0.12  # the uniform fifth spreads everywhere
    deg = np.bincount(el.src, minlength=el.n)
    assert deg.max() > 20 * deg.mean()
    # ids pass through a multiplicative bijection: R-MAT's largest hub (all-'a' path, id 0) stays
    # at 0, the next hubs are scattered over the id range
    hubs = np.argsort(deg)[::-1][:10]
    assert hubs[0] == 0 and np.median(hubs[1:]) > el.n / 64


def test_zipf_times_of_the_large_workload():
    """Departure rank r - 1 with P(r) proportional to r^-1.2 over 2^31 ranks (Hoermann-
    Derflinger rejection-inversion): P(t = 0) = 1 / H(2^31, 1.2) and P(t = 1) = 2^-1.2 / H."""
    spec = scaled(WORKLOADS[5].graph, 14, 1 << 20)
    el = synth.rmat(spec)
    H = sum(r ** -1.2 for r in range(1, 200001)) + ((200000.5) ** -0.2 - (2 ** 31 + 0.5) ** -0.2) / 0.2
    p0, p1 = 1 / H, 2 ** -1.2 / H
    assert abs((el.t == 0).mean() - p0) < 0.003
    assert abs((el.t == 1).mean() - p1) < 0.002
    assert el.lam.dtype == np.uint16 and el.lam.min() >= 1 and el.lam.max() <= 4096


def test_deterministic_and_thread_independent():
    spec = scaled(WORKLOADS[2].graph, 12, 1 << 16)
    a = synth.rmat(spec, nthreads=1)
    b = synth.rmat(spec, nthreads=4)
    for x, y in ((a.src, b.src), (a.dst, b.dst), (a.t, b.t), (a.lam, b.lam)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("key", [1, 2, 3, 4])
def test_query_sets_match_their_recipe(key):
    spec = WORKLOADS[key].graph
    el = synth.rmat(scaled(spec, 12, 1 << 15) if key != 1 else spec)
    qs = synth.workload_queries(key, el, count=16 if key != 1 else None)
    out_deg = np.bincount(el.src, minlength=el.n)
    in_deg = np.bincount(el.dst, minlength=el.n)
    for q in qs:
        assert 0 <= q.vertex < el.n and q.ta <= q.tw <= synth.C_MIRROR
        assert (out_deg if q.kind == synth.EA else in_deg)[q.vertex] > 0
    if key == 2:
        assert [q.kind for q in qs] == [synth.EA] * 16 + [synth.LD] * 16
        assert all((q.ta, q.tw) == (0, synth.C_MIRROR) for q in qs)
