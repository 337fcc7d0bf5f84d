"""GPU parity of the time-ordered edge-map (relax_mode 3: one sweep of the edges in departure
order, block by block, with frontier fix-ups inside a block) through the C ABI against the
oracle, bit-exact (integer times): both query kinds and predicates, windows, 32 and 64 lanes
with ragged lane counts, host and device outputs, two launches in flight, block sizes from a
few edges to one block, zero durations and equal departure times (chains inside one instant),
16-bit durations, the medium workload at full size (every answer certified), the fix-up
round cap, and the same labels as the frontier kernel."""
import numpy as np
import pytest

import oracle
import synth
from oracle import C_MIRROR, UNREACHED, Oracle
from synth import EA, LD, Query

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kx.lib()
    yield


def labels(x):
    return x.cpu().numpy().view(np.uint32).reshape(x.shape)


def run(g, n, qs, on_device=True):
    if on_device:
        out = torch.full((len(qs), n), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        st = kx.kairos_batch_query(g.handle, n, qs, out)
        return labels(out), st
    out = np.full((len(qs), n), 0x5A5A5A5A, np.uint32)
    st = kx.kairos_batch_query(g.handle, n, qs, out)
    return out, st


def mixed_queries(el, count, seed):
    vs = synth.pick_vertices(el, count, seed, True, True)
    wins = [(0, (1 << 20) - 1), (0, C_MIRROR), (200_000, 700_000), (500_000, 500_900), (1000, 1000)]
    return [Query(EA if i % 2 == 0 else LD, v, *wins[i % len(wins)], (i // 3) % 2) for i, v in enumerate(vs)]


@pytest.fixture(scope="module")
def tiny():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    g.index(64)
    yield el, orc, g
    g.close()


def check(orc, qs, got, stats):
    for i, q in enumerate(qs):
        want = orc.query(q)
        assert np.array_equal(got[i], want), q
        assert stats[i].relaxed_edges == orc.admissible(q, want), q
        assert stats[i].reached == int((want != UNREACHED).sum()), q


@pytest.mark.parametrize("lanes", [32, 64])
@pytest.mark.parametrize("on_device", [True, False])
@pytest.mark.parametrize("block_edges", [0, 37, 100_000])
def test_stream_mode_matches_oracle(tiny, lanes, on_device, block_edges):
    el, orc, g = tiny
    g.set_tuning(lanes=lanes, relax_mode=3, block_edges=block_edges, concurrent=1)
    qs = mixed_queries(el, 71, 0xB100 + lanes)  # ragged: not a multiple of the lane width
    got, stats = run(g, el.n, qs, on_device)
    check(orc, qs, got, stats)
    g.set_tuning(lanes=1, relax_mode=0, block_edges=0)


@pytest.mark.parametrize("lanes", [32, 64])
@pytest.mark.parametrize("concurrent", [2, 4])
def test_stream_mode_launches_in_flight_and_replay(tiny, lanes, concurrent):
    """Launches are dealt to two or four streams and workspaces; the call repeats as a
    captured CUDA graph with identical labels."""
    el, orc, g = tiny
    g.set_tuning(lanes=lanes, relax_mode=3, concurrent=concurrent, block_edges=2000)
    qs = mixed_queries(el, 3 * lanes + 5, 0xB200)
    before = g.info().graph_launches
    first, stats = run(g, el.n, qs)
    again, _ = run(g, el.n, qs)
    assert g.info().graph_launches > before
    assert np.array_equal(first, again)
    check(orc, qs, first, stats)
    g.set_tuning(lanes=1, relax_mode=0, concurrent=1, block_edges=0)


@pytest.mark.parametrize("seed", range(8))
def test_stream_mode_random_multigraphs(seed):
    """Zero durations, self-loops, parallel edges and many equal departure times: chains
    within one instant and within one block are finished by the fix-up rounds."""
    n, m = 50 + 23 * seed, 500 + 211 * seed
    el = synth.random_small(n, m, 0xB300 + seed, t_max=30 + 10 * seed, lam_max=3 + seed, lam_min=0)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=[32, 64][seed % 2], relax_mode=3, block_edges=[1, 7, 64, 100_000][seed % 4])
    qs = []
    for i in range(90):
        d = lambda k: synth.draw(0xB400 + seed, i, k)
        ta = synth.below(d(1), 20)
        qs.append(Query(i % 2, synth.below(d(0), n), ta, ta + synth.below(d(2), 60), (i // 2) % 2))
    got, stats = run(g, n, qs)
    check(orc, qs, got, stats)
    g.close()


def test_stream_mode_uint16_durations_and_frontier_kernel_agree():
    spec = synth.scaled(synth.WORKLOADS[5].graph, 14, 1 << 18)
    el = synth.rmat(spec)
    assert el.lam.dtype == np.uint16
    orc = Oracle(el)
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    g.index(16)
    vs = synth.pick_vertices(el, 40, 0xB500, True, True)
    qs = [Query(k, v, 0, C_MIRROR) for v in vs for k in (EA, LD)]
    g.set_tuning(lanes=64, relax_mode=3)
    got, stats = run(g, el.n, qs)
    check(orc, qs, got, stats)
    g.set_tuning(lanes=16, relax_mode=0)
    got2, stats2 = run(g, el.n, qs)
    assert np.array_equal(got, got2)
    assert [s.relaxed_edges for s in stats] == [s.relaxed_edges for s in stats2]
    g.close()


def test_stream_mode_edge_cases():
    # one vertex, no edges
    class E:
        pass

    el = E()
    el.n, el.src, el.dst = 1, np.zeros(0, np.int32), np.zeros(0, np.int32)
    el.t, el.lam = np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=32, relax_mode=3)
    got, _ = run(g, 1, [Query(EA, 0, 5, 9), Query(LD, 0, 5, 9)])
    assert got[0].tolist() == [5] and got[1].tolist() == [9]
    g.close()
    # window end at the largest finite time, ta == tw, an isolated source
    el = synth.random_small(40, 300, 0xB600, t_max=50, lam_max=5, lam_min=0)
    el.t[0], el.lam[0] = C_MIRROR - 3, 3
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=64, relax_mode=3, block_edges=16)
    qs = [Query(EA, 1, 0, C_MIRROR), Query(LD, 2, 0, C_MIRROR), Query(EA, 3, 7, 7), Query(LD, 4, 9, 9, 1),
          Query(EA, int(el.src[0]), C_MIRROR - 3, C_MIRROR)]
    got, stats = run(g, el.n, qs)
    check(orc, qs, got, stats)
    # invalid shapes are refused
    with pytest.raises(kx.KairosError):
        g.set_tuning(lanes=16, relax_mode=3)
    with pytest.raises(kx.KairosError):
        g.set_tuning(lanes=64, relax_mode=0)
    with pytest.raises(kx.KairosError):
        g.set_tuning(lanes=16, relax_mode=0, concurrent=4)
    g.close()


def test_stream_mode_fix_up_round_cap_returns_timeout(monkeypatch):
    """A cap of one fix-up round per block on a graph whose blocks need more returns
    KAIROS_ERR_TIMEOUT (no fault, no hang); the next call without the cap succeeds."""
    class E:
        pass

    # a zero-duration chain 29 -> 28 -> ... -> 0 at one instant: the time order lists the edge
    # out of 1 first, so the sweep relaxes only the first hop and each later hop is one fix-up
    el = E()
    el.n = 30
    el.src = np.arange(29, 0, -1, dtype=np.int32)
    el.dst = el.src - 1
    el.t = np.full(29, 4, np.uint32)
    el.lam = np.zeros(29, np.uint32)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=32, relax_mode=3)
    qs = [Query(EA, 29, 0, 10), Query(LD, 0, 0, 10)]
    monkeypatch.setenv("KAIROS_ROUND_CAP", "1")
    with pytest.raises(kx.KairosError) as e:
        run(g, el.n, qs)
    assert e.value.status == kx.KAIROS_ERR_TIMEOUT
    monkeypatch.delenv("KAIROS_ROUND_CAP")
    got, stats = run(g, el.n, qs)
    check(orc, qs, got, stats)
    g.close()


def test_stream_mode_medium_full_size_certified():
    """The 2^25-edge medium workload, 64 lanes: every answer of both kinds certified, two
    compared label by label with the oracle, and the labels equal the frontier kernel's."""
    el = synth.rmat(synth.WORKLOADS[2].graph)
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    g.index(synth.WORKLOADS[2].theta)
    qs = synth.workload_queries(2, el)
    g.set_tuning(lanes=64, relax_mode=3, concurrent=2)
    out = torch.empty((len(qs), el.n), dtype=torch.int32, device="cuda")
    stats = g.batch(qs, out)
    res = oracle.Certifier(el).check_all(qs, lambda i: labels(out[i]))
    assert res == [(0, 0)] * len(qs), [(qs[i], r) for i, r in enumerate(res) if r != (0, 0)][:4]
    orc = Oracle(el)
    for i in (0, 64):
        want = orc.query(qs[i])
        assert np.array_equal(labels(out[i]), want)
        assert stats[i].relaxed_edges == orc.admissible(qs[i], want)
    g.set_tuning(lanes=16, relax_mode=0, concurrent=1)
    ref = torch.empty_like(out)
    stats2 = g.batch(qs, ref)
    assert torch.equal(out, ref)
    assert [s.relaxed_edges for s in stats] == [s.relaxed_edges for s in stats2]
    g.close()


@pytest.mark.parametrize("shape", [dict(lanes=1, relax_mode=0), dict(lanes=16, relax_mode=0, concurrent=2),
                                   dict(lanes=64, relax_mode=3, concurrent=2)])
def test_page_locked_host_outputs(tiny, shape):
    """Outputs in page-locked host memory: written by the kernels through their device mapping
    with one launch in flight, staged and moved by the copy engine (inside the captured graph)
    with two; the same labels as the oracle, in one call or repeated (graph replay)."""
    el, orc, g = tiny
    g.set_tuning(**shape)
    qs = mixed_queries(el, 70, 0xB800)
    host_t = torch.full((len(qs), el.n), 0x5A5A5A5A, dtype=torch.int32, pin_memory=True)
    host = host_t.numpy().view(np.uint32)
    for _ in range(2):
        stats = kx.kairos_batch_query(g.handle, el.n, qs, host)
        check(orc, qs, host, stats)
        host[:] = 0x5A5A5A5A
    row_t = torch.full((el.n,), 0x5A5A5A5A, dtype=torch.int32, pin_memory=True)
    q = qs[0]
    g.earliest_arrival(q.vertex, q.ta, q.tw, row_t.numpy().view(np.uint32))
    assert np.array_equal(row_t.numpy().view(np.uint32), orc.query(q))
    g.set_tuning(lanes=1, relax_mode=0, concurrent=1)
