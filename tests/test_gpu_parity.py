"""GPU parity: the CUDA path, called through the C ABI, against the oracle on the same
seeded inputs.  All arithmetic is exact uint32, so every comparison is bit-exact."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import C_MIRROR, UNREACHED, Oracle
from synth import EA, LD, Query

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
NO_INDEX = kx.KAIROS_NO_INDEX


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kx.lib()
    yield


def labels(x):
    if hasattr(x, "cpu"):
        return x.cpu().numpy().view(np.uint32).reshape(x.shape)
    return np.asarray(x).view(np.uint32)


def dev_out(n, rows=None):
    shape = (n,) if rows is None else (rows, n)
    return torch.full(shape, 0x5A5A5A5A, dtype=torch.int32, device="cuda")


def gpu_batch(g, n, queries, on_device=True):
    out = dev_out(n, len(queries)) if on_device else np.full((len(queries), n), 0x5A5A5A5A, np.uint32)
    stats = kx.kairos_batch_query(g.handle, n, queries, out)
    return labels(out), stats


class Edges:
    def __init__(self, n, rows):
        r = np.array(rows, dtype=np.int64).reshape(-1, 4)
        self.n = n
        self.src = r[:, 0].astype(np.int32)
        self.dst = r[:, 1].astype(np.int32)
        self.t = r[:, 2].astype(np.uint32)
        self.lam = r[:, 3].astype(np.uint32)


# ---- the hand-worked example ----------------------------------------------------------

def test_hand_worked_example():
    gj = json.load(open(os.path.join(HERE, "golden", "hand_example.json")))
    el = Edges(gj["n"], gj["edges_u_v_t_lam"])
    g = kx.Graph.from_edges(el)
    for th in (1, NO_INDEX):
        g.index(th)
        qs = [Query(EA if c["kind"] == "EA" else LD, c["vertex"], c["ta"], c["tw"], c["strict"]) for c in gj["cases"]]
        got, stats = gpu_batch(g, el.n, qs)
        for i, c in enumerate(gj["cases"]):
            assert got[i].tolist() == c["expect"], c
            if "admissible" in c:
                assert stats[i].relaxed_edges == c["admissible"]
    g.close()


# ---- tiny workload: every query kind, predicate, index threshold and lane width ----------

@pytest.fixture(scope="module")
def tiny():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    yield el, orc, g
    g.close()


def tiny_queries(el, count=12):
    srcs = synth.pick_vertices(el, count, 0x9100, True, True)
    wins = [(0, (1 << 20) - 1), (0, C_MIRROR), (200_000, 700_000), (500_000, 500_900)]
    qs = []
    for i, v in enumerate(srcs):
        ta, tw = wins[i % len(wins)]
        qs.append(Query(EA if i % 2 == 0 else LD, v, ta, tw, (i // 2) % 2))
    return qs


def test_single_query_calls_match_oracle(tiny):
    el, orc, g = tiny
    g.index(NO_INDEX)
    q = synth.workload_queries(1, el)[0]
    want = orc.query(q)
    out = dev_out(el.n)
    g.earliest_arrival(q.vertex, q.ta, q.tw, out)
    assert np.array_equal(labels(out), want)
    host = np.zeros(el.n, np.uint32)
    g.earliest_arrival(q.vertex, q.ta, q.tw, host)
    assert np.array_equal(host, want)
    want_ld = orc.latest_departure(q.vertex, 0, (1 << 20) - 1)
    g.latest_departure(q.vertex, 0, (1 << 20) - 1, out)
    assert np.array_equal(labels(out), want_ld)
    g.latest_departure(q.vertex, 0, (1 << 20) - 1, host)
    assert np.array_equal(host, want_ld)


@pytest.mark.parametrize("theta", [1, 16, 256, 4096, NO_INDEX])
def test_index_threshold_invariance(tiny, theta):
    el, orc, g = tiny
    g.index(theta)
    g.set_tuning(lanes=1)
    qs = tiny_queries(el)
    got, stats = gpu_batch(g, el.n, qs)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), (theta, q)
        assert stats[i].relaxed_edges == orc.admissible(q, want), (theta, q)
        assert stats[i].reached == int((want != UNREACHED).sum())


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("on_device", [True, False])
def test_lane_widths(tiny, lanes, on_device):
    el, orc, g = tiny
    g.index(64)
    g.set_tuning(lanes=lanes)
    qs = tiny_queries(el, 37)  # ragged: not a multiple of any lane width
    got, stats = gpu_batch(g, el.n, qs, on_device)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), (lanes, q)
        assert stats[i].relaxed_edges == orc.admissible(q, want)
    g.set_tuning(lanes=1)


@pytest.mark.parametrize("warp_max,chunk,dense", [(32, 32, 0), (32, 64, 1), (100, 32, 1_000_000), (4096, 2048, 1)])
def test_work_shapes(tiny, warp_max, chunk, dense):
    """Grid-wide chunking of long ranges and the dense bitmap sweep give identical labels."""
    el, orc, g = tiny
    g.index(16)
    g.set_tuning(lanes=4, warp_max_edges=warp_max, chunk_edges=chunk, dense_div=dense)
    qs = tiny_queries(el, 9)
    got, stats = gpu_batch(g, el.n, qs)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), q
        assert stats[i].relaxed_edges == orc.admissible(q, want)
    g.set_tuning(lanes=1, warp_max_edges=128, chunk_edges=512, dense_div=16)


# ---- random multigraphs: zero durations, self-loops, parallel edges, ties -----------------

@pytest.mark.parametrize("seed", range(6))
def test_random_multigraphs(seed):
    n, m = 60 + 17 * seed, 400 + 131 * seed
    el = synth.random_small(n, m, 0x9200 + seed, t_max=40, lam_max=4, lam_min=0)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index([1, 4, NO_INDEX][seed % 3])
    g.set_tuning(lanes=[1, 8, 32][seed % 3], warp_max_edges=32, chunk_edges=32)
    qs = []
    for i in range(40):
        d = lambda k: synth.draw(0x9300 + seed, i, k)
        ta = synth.below(d(1), 20)
        qs.append(Query(i % 2, synth.below(d(0), n), ta, ta + synth.below(d(2), 40), (i // 2) % 2))
    got, stats = gpu_batch(g, n, qs)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), q
        assert stats[i].relaxed_edges == orc.admissible(q, want)
    g.close()


def test_device_resident_input_and_torch_allocator():
    el = synth.random_small(300, 3000, 0x9400, t_max=1000, lam_max=20, lam_min=1)
    orc = Oracle(el)
    cols = [torch.from_numpy(a.astype(np.int32) if a.dtype != np.int32 else a).cuda()
            for a in (el.src, el.dst, el.t.view(np.int32), el.lam.view(np.int32))]
    alloc = kx.TorchAllocator()
    g = kx.Graph(el.n, *cols, stream=torch.cuda.current_stream(), allocator=alloc)
    g.index(8)
    qs = [Query(k, v, 0, 2000) for k in (EA, LD) for v in (1, 7, 299)]
    got, _ = gpu_batch(g, el.n, qs)
    for i, q in enumerate(qs):
        assert np.array_equal(got[i], orc.query(q))
    g.close()


def test_uint16_durations():
    spec = synth.scaled(synth.WORKLOADS[5].graph, 12, 40_000)
    el = synth.rmat(spec)
    assert el.lam.dtype == np.uint16
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index(64)
    vs = synth.pick_vertices(el, 4, 0x9500, True, True)
    qs = [Query(k, v, 0, C_MIRROR) for v in vs for k in (EA, LD)]
    got, stats = gpu_batch(g, el.n, qs)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want)
        assert stats[i].relaxed_edges == orc.admissible(q, want)
    g.close()


# ---- edge cases and errors ----------------------------------------------------------------

def test_edge_cases():
    # a single vertex, no edges
    g = kx.Graph(1, *(np.zeros(0, t) for t in (np.int32, np.int32, np.uint32, np.uint32)))
    out = dev_out(1)
    g.earliest_arrival(0, 5, 9, out)
    assert labels(out).tolist() == [5]
    g.latest_departure(0, 5, 9, out)
    assert labels(out).tolist() == [9]
    g.close()
    # isolated source; ta == tw; window end at KAIROS_TIME_MAX
    el = Edges(4, [(1, 2, 3, 1), (2, 3, 4, 0), (2, 3, 4, 0), (3, 3, 7, 2), (1, 1, 0, 0)])
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    for q in [Query(EA, 0, 0, 10), Query(EA, 1, 3, 3), Query(EA, 1, 3, 4), Query(LD, 3, 0, C_MIRROR),
              Query(EA, 1, 0, C_MIRROR, 1), Query(LD, 2, 4, 4)]:
        got, _ = gpu_batch(g, 4, [q])
        assert np.array_equal(got[0], orc.query(q)), q
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival(4, 0, 1, dev_out(4))
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival(0, 5, 4, dev_out(4))
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    with pytest.raises(kx.KairosError) as e:
        g.latest_departure(0, 0, 0xFFFFFFFF, dev_out(4))
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()
    # t + lambda beyond KAIROS_TIME_MAX, and a vertex id out of range, are rejected at build
    bad = Edges(3, [(0, 1, 0xFFFFFFF0, 0x20)])
    with pytest.raises(kx.KairosError) as e:
        kx.Graph.from_edges(bad)
    assert e.value.status == kx.KAIROS_ERR_OVERFLOW
    bad = Edges(3, [(0, 3, 1, 1)])
    with pytest.raises(kx.KairosError) as e:
        kx.Graph.from_edges(bad)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    # latest departure on a graph built without the reverse direction
    g = kx.Graph.from_edges(Edges(3, [(0, 1, 1, 1)]), skip_reverse=True)
    with pytest.raises(kx.KairosError) as e:
        g.latest_departure(1, 0, 5, dev_out(3))
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()


# ---- the medium workload at full size ----------------------------------------------------------

@pytest.fixture(scope="module")
def medium():
    el = synth.rmat(synth.WORKLOADS[2].graph)
    g = kx.Graph.from_edges(el)
    g.index(synth.WORKLOADS[2].theta)
    yield el, g
    g.close()


def test_medium_full_size_sampled_against_oracle(medium):
    """Full 2^25-edge workload in the launch shape the benchmark times: every answer of both
    kinds is certified at full size (earliest arrival directly, latest departure through the
    mirrored graph), and a sample of each kind is compared label by label with the oracle's
    scans, with exact relaxed-edge counts."""
    el, g = medium
    qs = synth.workload_queries(2, el)
    g.autotune(qs)  # the launch shape the benchmark times
    got, stats = gpu_batch(g, el.n, qs)
    orc = Oracle(el)
    for i in (0, 1, 63, 64, 65, 127):
        want = orc.query(qs[i])
        assert np.array_equal(got[i], want), qs[i]
        assert stats[i].relaxed_edges == orc.admissible(qs[i], want)
    assert {q.kind for q in qs} == {EA, LD}
    res = oracle.Certifier(el).check_all(qs, lambda i: got[i])
    assert res == [(0, 0)] * len(qs), [(qs[i], r) for i, r in enumerate(res) if r != (0, 0)][:4]
    for i, q in enumerate(qs):
        assert got[i][q.vertex] == (q.ta if q.kind == EA else q.tw)
        assert stats[i].reached == int((got[i] != UNREACHED).sum())
    g.set_tuning(lanes=1)


# ---- failure paths: device waits and the round cap give up with a status ----------------------

def test_device_wait_and_round_cap_return_timeout(tiny, monkeypatch):
    """A wait limit of zero polls makes every grid-barrier wait run out (nothing can satisfy
    it in time): the call must return KAIROS_ERR_TIMEOUT, not hang or fault, and the
    context must stay usable.  Likewise a round cap below the rounds a query needs."""
    el, orc, g = tiny
    g.index(64)
    g.set_tuning(lanes=1)
    q = synth.workload_queries(1, el)[0]
    out = dev_out(el.n)
    monkeypatch.setenv("KAIROS_SPIN_LIMIT", "0")
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival(q.vertex, q.ta, q.tw, out)
    assert e.value.status == kx.KAIROS_ERR_TIMEOUT
    monkeypatch.delenv("KAIROS_SPIN_LIMIT")
    monkeypatch.setenv("KAIROS_ROUND_CAP", "1")
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival(q.vertex, q.ta, q.tw, out)
    assert e.value.status == kx.KAIROS_ERR_TIMEOUT
    monkeypatch.delenv("KAIROS_ROUND_CAP")
    g.earliest_arrival(q.vertex, q.ta, q.tw, out)
    assert np.array_equal(labels(out), orc.query(q))


def test_captured_batch_replays_and_recaptures(tiny):
    """On a graph with its own stream and device outputs, a repeated batch is captured into
    a CUDA graph and replayed; each replay recomputes the labels, and a different batch is
    captured afresh."""
    el, orc, _ = tiny
    stream = torch.cuda.Stream()
    g = kx.Graph.from_edges(el, stream=stream)
    g.index(64)
    g.set_tuning(lanes=8)
    n = el.n
    with torch.cuda.stream(stream):
        for qs in (tiny_queries(el, 20), tiny_queries(el, 13)[::-1]):
            out = torch.empty((len(qs), n), dtype=torch.int32, device="cuda")
            want = [orc.query(q) for q in qs]
            for rep in range(3):
                out.fill_(0x5A5A5A5A)
                stats = g.batch(qs, out, want_stats=(rep == 1))
                got = labels(out)
                for i in range(len(qs)):
                    assert np.array_equal(got[i], want[i]), (rep, qs[i])
                if rep == 1:
                    assert [s.relaxed_edges for s in stats] == [orc.admissible(q, w) for q, w in zip(qs, want)]
    torch.cuda.synchronize()
    assert g.info().graph_launches == 6  # both batches, three calls each, ran as graphs
    g.close()


@pytest.mark.parametrize("lanes,mode", [(1, 1), (2, 1), (8, 1), (32, 1), (2, 2), (4, 2), (16, 2), (32, 2)])
def test_relax_modes(tiny, lanes, mode):
    """relax_mode 1 (unconditional fire-and-forget minima, bitmap frontier) and 2 (checked
    minima over candidate segments only) give the same labels and counts, including zero
    durations and both predicates."""
    el, orc, g = tiny
    g.index(16)
    g.set_tuning(lanes=lanes, relax_mode=mode, warp_max_edges=64, chunk_edges=64)
    qs = tiny_queries(el, 21)
    got, stats = gpu_batch(g, el.n, qs)
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), q
        assert stats[i].relaxed_edges == orc.admissible(q, want)
    el2 = synth.random_small(90, 900, 0x9600 + lanes, t_max=30, lam_max=3, lam_min=0)
    orc2 = Oracle(el2)
    g2 = kx.Graph.from_edges(el2)
    g2.index(4)
    g2.set_tuning(lanes=lanes, relax_mode=mode)
    qs2 = [Query(i % 2, (7 * i) % 90, i % 5, 20 + i % 13, (i // 2) % 2) for i in range(24)]
    got2, _ = gpu_batch(g2, el2.n, qs2)
    for i, q in enumerate(qs2):
        assert np.array_equal(got2[i], orc2.query(q)), q
    g2.close()
    g.set_tuning(lanes=1, relax_mode=0, warp_max_edges=128, chunk_edges=512)


@pytest.mark.parametrize("lanes", [1, 4, 16])
def test_concurrent_launches(tiny, lanes):
    """Two launches in flight on two streams and workspaces (tuning.concurrent = 2): the same
    labels and counts as the oracle, on the graph's own stream (captured and replayed) and
    on the default stream, with device outputs; host outputs fall back to one stream."""
    el, orc, _ = tiny
    n = el.n
    qs = tiny_queries(el, 2 * lanes + 3)  # ragged, both kinds, at least three launches
    want = [orc.query(q) for q in qs]
    counts = [orc.admissible(q, w) for q, w in zip(qs, want)]
    stream = torch.cuda.Stream()
    for own_stream in (True, False):
        g = kx.Graph.from_edges(el, stream=stream if own_stream else None)
        g.index(16)
        g.set_tuning(lanes=lanes, concurrent=2, warp_max_edges=32, chunk_edges=64)
        with torch.cuda.stream(stream if own_stream else torch.cuda.default_stream()):
            for rep in range(3):
                out = torch.full((len(qs), n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
                stats = g.batch(qs, out, want_stats=(rep != 1))
                got = labels(out)
                for i in range(len(qs)):
                    assert np.array_equal(got[i], want[i]), (own_stream, rep, qs[i])
                if stats:
                    assert [s.relaxed_edges for s in stats] == counts
        host = np.full((len(qs), n), 0x5A5A5A5A, np.uint32)
        stats = g.batch(qs, host)
        assert all(np.array_equal(host[i], want[i]) for i in range(len(qs)))
        assert [s.relaxed_edges for s in stats] == counts
        torch.cuda.synchronize()
        g.close()


class BudgetAllocator(kx.TorchAllocator):
    """Device allocations through PyTorch, refused (NULL) once `budget` bytes would be live:
    device out-of-memory injected on the host."""

    def __init__(self, budget):
        super().__init__()
        self.budget = budget
        self.live = {}

    def _alloc(self, nbytes, ctx):
        if sum(self.live.values()) + int(nbytes) > self.budget:
            return None
        p = super()._alloc(nbytes, ctx)
        if p:
            self.live[int(p)] = int(nbytes)
        return p

    def _free(self, ptr, ctx):
        if ptr:
            self.live.pop(int(ptr), None)
        super()._free(ptr, ctx)


def test_allocator_refusals_return_oom(tiny):
    """A refused allocation at graph build or at query time returns KAIROS_ERR_OOM, gives
    back what was taken, and leaves the graph usable once memory is available again."""
    el, orc, _ = tiny
    A = BudgetAllocator(0)
    with pytest.raises(kx.KairosError) as e:
        kx.Graph.from_edges(el, allocator=A)
    assert e.value.status == kx.KAIROS_ERR_OOM
    assert not A.live
    A.budget = 1 << 62
    g = kx.Graph.from_edges(el, allocator=A)
    A.budget = sum(A.live.values()) + 4096  # the graph fits, a 32-lane workspace does not
    g.set_tuning(lanes=32)
    qs = tiny_queries(el, 32)
    out = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    with pytest.raises(kx.KairosError) as e:
        g.batch(qs, out, want_stats=False)
    assert e.value.status == kx.KAIROS_ERR_OOM
    A.budget = 1 << 62
    g.batch(qs, out, want_stats=False)
    got = labels(out)
    for i, q in enumerate(qs):
        assert np.array_equal(got[i], orc.query(q)), q
    g.close()
    torch.cuda.synchronize()
    assert not A.live  # closing the graph gave back every allocation
