"""Full-size parity for the large workloads (2^28 and 2^31 edges).  Labels are checked by
the any-size certificate (closed under every usable edge, every finite label witnessed,
exact when durations are >= 1), one query against the oracle's full scan at 2^28 edges,
and latest departure against the oracle on a smaller graph of the same laws."""
import numpy as np
import pytest

import oracle
import synth
from oracle import UNREACHED, Oracle
from synth import EA, LD, Query

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def labels(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def batched_graph():
    w = synth.WORKLOADS[3]
    el = synth.rmat(w.graph)
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    g.index(256)
    yield el, g
    g.close()


def test_batched_workload_full_size(batched_graph):
    el, g = batched_graph
    qs = synth.workload_queries(3, el)[:32]
    g.set_tuning(lanes=16)
    out = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    stats = g.batch(qs, out)
    torch.cuda.synchronize()
    got = labels(out)
    for i in range(0, len(qs), 4):
        q = qs[i]
        assert oracle.certify_ea(el, q.vertex, q.ta, q.tw, q.strict, got[i]) == (0, 0), q
        assert got[i][q.vertex] == q.ta
        assert stats[i].reached == int((got[i] != UNREACHED).sum())
    orc = Oracle(el)
    want = orc.query(qs[1])
    assert np.array_equal(got[1], want)
    assert stats[1].relaxed_edges == orc.admissible(qs[1], want)


def test_served_workload_full_size_alone_and_in_the_mix(batched_graph):
    """Workload 4: the resident workload-3 graph, a 70/30 mix with log-uniform windows
    submitted while others run; each answer equals the same query alone."""
    el, g = batched_graph
    qs = synth.workload_queries(4, el, count=48)
    alone = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    g.set_tuning(lanes=1)
    g.batch(qs, alone, want_stats=False)
    server = kx.kairos_serve_create(g.handle, max_slots=16, rounds_per_slice=3)
    outs = [torch.empty(el.n, dtype=torch.int32, device="cuda") for _ in qs]
    try:
        tickets = [kx.kairos_serve_submit(server, q, o) for q, o in zip(qs, outs)]
        infos = [kx.kairos_serve_poll(server, t, -1) for t in tickets]
    finally:
        kx.kairos_serve_destroy(server)
    torch.cuda.synchronize()
    ref = labels(alone)
    for i, q in enumerate(qs):
        assert infos[i].status == kx.KAIROS_OK
        got = labels(outs[i])
        assert np.array_equal(got, ref[i]), q
        if q.kind == EA and i % 6 == 0:
            assert oracle.certify_ea(el, q.vertex, q.ta, q.tw, q.strict, got) == (0, 0), q


def test_large_skewed_full_size():
    """Workload 5: 2^26 vertices, 2^31 edges, Zipf(1.2) times, 16-bit durations."""
    w = synth.WORKLOADS[5]
    el = synth.rmat(w.graph)
    assert el.lam.dtype == np.uint16 and el.m == 1 << 31
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream(), skip_reverse=True)
    g.index(256)
    qs = [q for q in synth.workload_queries(5, el, count=2) if q.kind == EA]
    g.set_tuning(lanes=2)
    out = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    stats = g.batch(qs, out)
    torch.cuda.synchronize()
    got = labels(out)
    g.close()
    for i, q in enumerate(qs):
        assert got[i][q.vertex] == q.ta
        assert stats[i].relaxed_edges > 0
        assert oracle.certify_ea(el, q.vertex, q.ta, q.tw, q.strict, got[i]) == (0, 0), q


@pytest.mark.parametrize("theta", [16, 4096])
def test_large_skewed_laws_smaller_graph_against_oracle(theta):
    """Workload 5's laws (skew a = .65, Zipf times with heavy ties near 0, 16-bit durations)
    at 2^20 vertices; both query kinds label by label, index threshold swept."""
    spec = synth.scaled(synth.WORKLOADS[5].graph, 20, 1 << 24)
    el = synth.rmat(spec)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index(theta)
    g.set_tuning(lanes=4)
    vs = synth.pick_vertices(el, 4, 0xC500, True, True)
    qs = [Query(k, v, 0, synth.C_MIRROR) for v in vs for k in (EA, LD)] + [Query(EA, vs[0], 5, 1 << 20, 1)]
    out = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    stats = g.batch(qs, out)
    got = labels(out)
    g.close()
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), q
        assert stats[i].relaxed_edges == orc.admissible(q, want)
