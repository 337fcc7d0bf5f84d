"""GPU parity of fastest paths (kairos_fastest_path, through the C ABI) against the oracle's
one-pass (start, arrival) pair scan on the same seeded inputs; bit-exact."""
import json
import os

import numpy as np
import pytest

import oracle
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


def gpu_fastest(g, n, s, ta, tw, strict=0, on_device=True, want_stats=False):
    out = (torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") if on_device
           else np.full(n, 0x5A5A5A5A, np.uint32))
    st = g.fastest_path(s, ta, tw, out, strict, want_stats)
    return labels(out), st


def start_times(el, s, ta, tw):
    m = (el.src == s) & (el.t >= ta) & (el.t.astype(np.uint64) + el.lam.astype(np.uint64) <= tw)
    return sorted(set(int(x) for x in el.t[m]))


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
    for lanes in (1, 4, 32):
        g.set_tuning(lanes=lanes)
        for c in gj["fastest_cases"]:
            for on_device in (True, False):
                got, _ = gpu_fastest(g, el.n, c["vertex"], c["ta"], c["tw"], c["strict"], on_device)
                assert got.tolist() == c["expect"], (lanes, c)
    g.close()


@pytest.mark.parametrize("strict", [0, 1])
def test_random_multigraphs(strict):
    """Multigraphs with parallel edges, self-loops, zero durations and few distinct times, so
    that sources have many departure times and labels tie often; several lane widths and
    both index settings."""
    for seed in range(6):
        n, m = 300 + 97 * seed, 6000 + 1500 * seed
        el = synth.random_small(n, m, 0x7A00 + seed, t_max=40 + 10 * seed, lam_max=6, lam_min=0)
        orc = Oracle(el)
        g = kx.Graph.from_edges(el)
        g.index(1 if seed % 2 else kx.KAIROS_NO_INDEX)
        g.set_tuning(lanes=(1, 2, 4, 8, 16, 32)[seed])
        out_deg = np.bincount(el.src, minlength=n)
        for k, s in enumerate(np.flatnonzero(out_deg)[[0, 5, 11]]):
            ta = [0, 3, 10][k]
            tw = [10**6, 30, 25 + seed][k]
            want = orc.fastest(int(s), ta, tw, strict)
            got, st = gpu_fastest(g, n, int(s), ta, tw, strict, on_device=bool(k % 2), want_stats=True)
            assert np.array_equal(got, want), (seed, s, ta, tw)
            assert st.start_times == len(start_times(el, int(s), ta, tw))
        g.close()


def test_tiny_workload_counts():
    """The 10^5-edge workload graph: labels, and the relaxed-edge total equals the sum over
    the source's start times of the oracle's admissible-edge counts."""
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index(64)
    g.set_tuning(lanes=16)
    srcs = synth.pick_vertices(el, 4, 0xFA57, True, False)
    for i, s in enumerate(srcs):
        ta, tw = (0, 2**20 - 1) if i % 2 == 0 else (1 << 18, 3 << 18)
        want = orc.fastest(s, ta, tw, i % 2)
        got, st = gpu_fastest(g, el.n, s, ta, tw, i % 2, want_stats=True)
        assert np.array_equal(got, want), (s, ta, tw)
        D = start_times(el, s, ta, tw)
        te = sum(orc.admissible(synth.Query(synth.EA, s, d, tw, i % 2), orc.earliest_arrival(s, d, tw, i % 2))
                 for d in D)
        assert st.start_times == len(D) and st.relaxed_edges == te
        assert st.launches == (len(D) + 15) // 16
    g.close()


def test_many_start_times_several_passes():
    """A source with 3000 distinct departure times (more than one pass of start-time lanes)."""
    n = 800
    rng_rows = []
    for i in range(3000):
        rng_rows.append((0, 1 + synth.below(synth.draw(0x5A1, i, 0), n - 1), 3 * i, 1 + synth.below(synth.draw(0x5A1, i, 1), 50)))
    bg = synth.random_small(n, 20000, 0x5A2, t_max=9000, lam_max=40, lam_min=1)
    rows = rng_rows + list(zip(bg.src.tolist(), bg.dst.tolist(), bg.t.tolist(), bg.lam.tolist()))
    el = Edges(n, rows)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=32)
    want = orc.fastest(0, 0, 10**6, 0)
    got, st = gpu_fastest(g, n, 0, 0, 10**6, 0, want_stats=True)
    assert np.array_equal(got, want)
    assert st.start_times >= 3000 and st.launches == (st.start_times + 31) // 32
    g.close()


def test_edge_cases():
    el = Edges(5, [(0, 1, 5, 1), (1, 2, 7, 0), (2, 3, 7, 2), (3, 0, 20, 1)])
    g = kx.Graph.from_edges(el)
    g.set_tuning(lanes=4)
    # a source without out-edges, and a window that excludes every out-edge of the source
    got, st = gpu_fastest(g, 5, 4, 0, 100, want_stats=True)
    assert got.tolist() == [UNREACHED, UNREACHED, UNREACHED, UNREACHED, 0] and st.start_times == 0
    got, _ = gpu_fastest(g, 5, 0, 6, 100)
    assert got.tolist() == [0, UNREACHED, UNREACHED, UNREACHED, UNREACHED]
    # the zero-duration edge chains within one instant (Succeeds) but not under StrictlySucceeds
    assert gpu_fastest(g, 5, 0, 0, 100)[0].tolist() == [0, 1, 2, 4, UNREACHED]
    assert gpu_fastest(g, 5, 0, 0, 100, strict=1)[0].tolist() == [0, 1, 2, UNREACHED, UNREACHED]
    for bad in (dict(s=5, ta=0, tw=1), dict(s=0, ta=3, tw=2), dict(s=0, ta=0, tw=0xFFFFFFFF)):
        with pytest.raises(kx.KairosError) as e:
            gpu_fastest(g, 5, bad["s"], bad["ta"], bad["tw"])
        assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    with pytest.raises(kx.KairosError) as e:
        gpu_fastest(g, 5, 0, 0, 10, strict=2)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()


def test_uint16_durations_and_medium_workload():
    """Full-size medium workload graph (2^25 edges) for three sources, and the same queries on
    a copy whose durations are stored as uint16."""
    w = synth.WORKLOADS[2]
    el = synth.rmat(w.graph)
    orc = Oracle(el)
    g = kx.Graph.from_edges(el)
    g.index(w.theta)
    g.set_tuning(lanes=16)
    srcs = synth.pick_vertices(el, 3, 0xFA58, True, False)
    wants = []
    for i, s in enumerate(srcs):
        ta, tw = (0, (1 << 24) - 1) if i != 1 else (1 << 22, 3 << 22)
        want = orc.fastest(s, ta, tw, 0)
        got, _ = gpu_fastest(g, el.n, s, ta, tw)
        assert np.array_equal(got, want), (s, ta, tw)
        wants.append((s, ta, tw, want))
    g.close()
    el16 = synth.EdgeList(el.n, el.src, el.dst, el.t, el.lam.astype(np.uint16))
    assert np.array_equal(el16.lam.astype(np.uint32), el.lam)
    g = kx.Graph.from_edges(el16)
    g.index(w.theta)
    g.set_tuning(lanes=32)
    for s, ta, tw, want in wants:
        assert np.array_equal(gpu_fastest(g, el.n, s, ta, tw)[0], want)
    g.close()
