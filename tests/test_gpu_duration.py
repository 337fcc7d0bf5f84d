"""GPU parity of shortest durations (kairos_shortest_duration, through the C ABI) against the
oracle's one-pass (total, arrival) pair scan on the same seeded inputs; bit-exact."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import UNREACHED, Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kx.lib()
    yield


def labels(x):
    if hasattr(x, "cpu"):
        return x.cpu().numpy().view(np.uint32)
    return np.asarray(x).view(np.uint32)


def gpu_sd(g, n, s, ta, tw, strict=0, on_device=True):
    out = (torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") if on_device
           else np.full(n, 0x5A5A5A5A, np.uint32))
    st = g.shortest_duration(s, ta, tw, out, strict)
    return labels(out), st


class Edges:
    def __init__(self, n, rows):
        r = np.array(rows, dtype=np.int64).reshape(-1, 4)
        self.n = n
        self.src = r[:, 0].astype(np.int32)
        self.dst = r[:, 1].astype(np.int32)
        self.t = r[:, 2].astype(np.uint32)
        self.lam = r[:, 3].astype(np.uint32)


def test_hand_worked_example():
    gj = json.load(open(os.path.join(HERE, "golden", "hand_example.json")))
    el = Edges(gj["n"], gj["edges_u_v_t_lam"])
    g = kx.Graph.from_edges(el)
    for c in gj["shortest_duration_cases"]:
        for on_device in (True, False):
            got, _ = gpu_sd(g, el.n, c["vertex"], c["ta"], c["tw"], c["strict"], on_device)
            assert got.tolist() == c["expect"], c
    g.close()


@pytest.mark.parametrize("strict", [0, 1])
def test_random_multigraphs(strict):
    """Parallel edges, self-loops, zero durations, few distinct times (many ties)."""
    for seed in range(6):
        n, m = 300 + 97 * seed, 6000 + 1500 * seed
        el = synth.random_small(n, m, 0x7B00 + seed, t_max=40 + 10 * seed, lam_max=6, lam_min=0)
        orc = Oracle(el)
        g = kx.Graph.from_edges(el)
        out_deg = np.bincount(el.src, minlength=n)
        for k, s in enumerate(np.flatnonzero(out_deg)[[0, 5, 11]]):
            ta = [0, 3, 10][k]
            tw = [10**6, 30, 25 + seed][k]
            want = orc.shortest_duration(int(s), ta, tw, strict)
            got, st = gpu_sd(g, n, int(s), ta, tw, strict, on_device=bool(k % 2))
            assert np.array_equal(got, want), (seed, s, ta, tw)
            assert 1 <= st.rounds <= n + 1
        g.close()


def test_tiny_workload_and_uint16():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    el16 = synth.EdgeList(el.n, el.src, el.dst, el.t, el.lam.astype(np.uint16))
    srcs = synth.pick_vertices(el, 4, 0x5D5D, True, False)
    for edges in (el, el16):
        g = kx.Graph.from_edges(edges)
        for i, s in enumerate(srcs):
            ta, tw = (0, 2**20 - 1) if i % 2 == 0 else (1 << 18, 3 << 18)
            want = orc.shortest_duration(s, ta, tw, i % 2)
            assert np.array_equal(gpu_sd(g, el.n, s, ta, tw, i % 2)[0], want), (s, ta, tw)
        g.close()


def test_dijkstra_graph():
    """The always-available static graph of the oracle's Dijkstra pin, on the GPU."""
    n = 60
    st = synth.random_small(n, 200, 0x7C00, t_max=0, lam_max=5, lam_min=1)
    H = 5 * n + 5
    rows = [(int(u), int(v), tt, int(l)) for u, v, l in zip(st.src, st.dst, st.lam) for tt in range(0, H + 1, 1)]
    el = Edges(n, rows)
    g = kx.Graph.from_edges(el)
    orc = Oracle(el)
    for s in (0, 7):
        want = orc.shortest_duration(s, 0, 2 * H)
        assert np.array_equal(gpu_sd(g, n, s, 0, 2 * H)[0], want)
    g.close()


def test_edge_cases():
    el = Edges(5, [(0, 1, 5, 1), (1, 2, 7, 0), (2, 3, 7, 2), (3, 0, 20, 1)])
    g = kx.Graph.from_edges(el)
    assert gpu_sd(g, 5, 4, 0, 100)[0].tolist() == [UNREACHED] * 4 + [0]
    assert gpu_sd(g, 5, 0, 6, 100)[0].tolist() == [0] + [UNREACHED] * 4
    assert gpu_sd(g, 5, 0, 0, 100)[0].tolist() == [0, 1, 1, 3, UNREACHED]
    assert gpu_sd(g, 5, 0, 0, 100, strict=1)[0].tolist() == [0, 1, 1, UNREACHED, UNREACHED]
    for s, ta, tw, strict in ((5, 0, 1, 0), (0, 3, 2, 0), (0, 0, 0xFFFFFFFF, 0), (0, 0, 10, 2)):
        with pytest.raises(kx.KairosError) as e:
            gpu_sd(g, 5, s, ta, tw, strict)
        assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()
    g = kx.Graph.from_edges(el, skip_reverse=True)
    with pytest.raises(kx.KairosError) as e:
        gpu_sd(g, 5, 0, 0, 100)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()


def test_medium_workload_full_size():
    w = synth.WORKLOADS[2]
    el = synth.rmat(w.graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index(w.theta)
    for i, s in enumerate(synth.pick_vertices(el, 2, 0x5D5E, True, False)):
        ta, tw = (0, (1 << 24) - 1) if i == 0 else (1 << 22, 3 << 22)
        assert np.array_equal(gpu_sd(g, el.n, s, ta, tw)[0], orc.shortest_duration(s, ta, tw, 0)), (s, ta, tw)
    g.close()


# ---- temporal BFS: the same computation with unit costs --------------------------------

def gpu_bfs(g, n, s, ta, tw, strict=0, on_device=True):
    out = (torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") if on_device
           else np.full(n, 0x5A5A5A5A, np.uint32))
    st = g.temporal_bfs(s, ta, tw, out, strict)
    return labels(out), st


def test_temporal_bfs_hand_example_and_random_graphs():
    gj = json.load(open(os.path.join(HERE, "golden", "hand_example.json")))
    el = Edges(gj["n"], gj["edges_u_v_t_lam"])
    g = kx.Graph.from_edges(el)
    for c in gj["temporal_bfs_cases"]:
        for on_device in (True, False):
            assert gpu_bfs(g, el.n, c["vertex"], c["ta"], c["tw"], c["strict"], on_device)[0].tolist() == c["expect"], c
    g.close()
    for seed in range(4):
        n, m = 400 + 131 * seed, 8000 + 1000 * seed
        el = synth.random_small(n, m, 0x7D00 + seed, t_max=50, lam_max=5, lam_min=0)
        orc = Oracle(el)
        g = kx.Graph.from_edges(el)
        out_deg = np.bincount(el.src, minlength=n)
        for k, s in enumerate(np.flatnonzero(out_deg)[[1, 7]]):
            for strict in (0, 1):
                ta, tw = (0, 10**6) if k == 0 else (5, 40)
                want = orc.temporal_bfs(int(s), ta, tw, strict)
                assert np.array_equal(gpu_bfs(g, n, int(s), ta, tw, strict, bool(strict))[0], want), (seed, s, strict)
        g.close()


def test_temporal_bfs_tiny_workload():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    for i, s in enumerate(synth.pick_vertices(el, 4, 0x5D5F, True, False)):
        ta, tw = (0, 2**20 - 1) if i % 2 == 0 else (1 << 18, 3 << 18)
        want = orc.temporal_bfs(s, ta, tw, i % 2)
        got, st = gpu_bfs(g, el.n, s, ta, tw, i % 2)
        assert np.array_equal(got, want), (s, ta, tw)
        # alternating with shortest durations on the same graph reuses the per-graph state
        assert np.array_equal(gpu_sd(g, el.n, s, ta, tw, i % 2)[0], orc.shortest_duration(s, ta, tw, i % 2))
    g.close()
