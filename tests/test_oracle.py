"""Pins for the oracle, checked against things other than itself: a hand-worked example,
brute force over simple paths, textbook reductions, the mirror identity between the two
query kinds, the identity between fastest paths and earliest arrival over start times, and
invariants that the definitions fix.  CPU only."""
import json
import os
from collections import deque

import numpy as np
import pytest

import oracle
import synth
from oracle import (C_MIRROR, UNREACHED, Oracle, brute_earliest_arrival, brute_fastest,
                    brute_latest_departure, brute_shortest_duration, brute_temporal_bfs, certify_ea,
                    mirror_edges)
from synth import EA, LD, Query

HERE = os.path.dirname(os.path.abspath(__file__))


class Edges:
    def __init__(self, n, src, dst, t, lam):
        self.n = n
        self.src = np.asarray(src, np.int32)
        self.dst = np.asarray(dst, np.int32)
        self.t = np.asarray(t, np.uint32)
        self.lam = np.asarray(lam, np.uint32)


def from_rows(n, rows):
    r = np.array(rows, dtype=np.int64).reshape(-1, 4)
    return Edges(n, r[:, 0], r[:, 1], r[:, 2], r[:, 3])


def test_hand_worked_example():
    g = json.load(open(os.path.join(HERE, "golden", "hand_example.json")))
    el = from_rows(g["n"], g["edges_u_v_t_lam"])
    orc = Oracle(el)
    for c in g["cases"]:
        q = Query(EA if c["kind"] == "EA" else LD, c["vertex"], c["ta"], c["tw"], c["strict"])
        got = orc.query(q)
        assert got.tolist() == c["expect"], c
        brute = (brute_earliest_arrival if q.kind == EA else brute_latest_departure)(
            el.n, el.src, el.dst, el.t, el.lam, q.vertex, q.ta, q.tw, q.strict)
        assert brute.tolist() == c["expect"], c
        if "admissible" in c:
            assert orc.admissible(q, got) == c["admissible"]
    for c in g["fastest_cases"]:
        got = orc.fastest(c["vertex"], c["ta"], c["tw"], c["strict"])
        assert got.tolist() == c["expect"], c
        brute = brute_fastest(el.n, el.src, el.dst, el.t, el.lam, c["vertex"], c["ta"], c["tw"], c["strict"])
        assert brute.tolist() == c["expect"], c
    for c in g["temporal_bfs_cases"]:
        got = orc.temporal_bfs(c["vertex"], c["ta"], c["tw"], c["strict"])
        assert got.tolist() == c["expect"], c
        brute = brute_temporal_bfs(el.n, el.src, el.dst, el.t, el.lam, c["vertex"], c["ta"], c["tw"], c["strict"])
        assert brute.tolist() == c["expect"], c
    for c in g["shortest_duration_cases"]:
        got = orc.shortest_duration(c["vertex"], c["ta"], c["tw"], c["strict"])
        assert got.tolist() == c["expect"], c
        brute = brute_shortest_duration(el.n, el.src, el.dst, el.t, el.lam, c["vertex"], c["ta"], c["tw"],
                                        c["strict"])
        assert brute.tolist() == c["expect"], c


def _tiny_cases(count):
    for seed in range(count):
        n = 2 + seed % 7
        m = 1 + (seed * 7) % 18
        el = synth.random_small(n, m, 0x7100 + seed, t_max=6, lam_max=3, lam_min=0)
        d = lambda k: synth.draw(0x7200 + seed, 0, k)
        v = synth.below(d(0), n)
        ta = synth.below(d(1), 4)
        tw = ta + synth.below(d(2), 8)
        yield el, v, ta, tw


@pytest.mark.parametrize("strict", [0, 1])
def test_brute_force_tiny_graphs(strict):
    """Thousands of tiny multigraphs with self-loops, parallel edges and zero durations."""
    checked = 0
    for el, v, ta, tw in _tiny_cases(1500):
        orc = Oracle(el)
        used = set()
        want = brute_earliest_arrival(el.n, el.src, el.dst, el.t, el.lam, v, ta, tw, strict, used)
        got = orc.earliest_arrival(v, ta, tw, strict)
        assert np.array_equal(got, want), (el.src, el.dst, el.t, el.lam, v, ta, tw)
        assert orc.admissible(Query(EA, v, ta, tw, strict), got) == len(used)
        used = set()
        want = brute_latest_departure(el.n, el.src, el.dst, el.t, el.lam, v, ta, tw, strict, used)
        got = orc.latest_departure(v, ta, tw, strict)
        assert np.array_equal(got, want), (el.src, el.dst, el.t, el.lam, v, ta, tw)
        assert orc.admissible(Query(LD, v, ta, tw, strict), got) == len(used)
        checked += 1
    assert checked == 1500


def _bfs(n, src, dst, s):
    adj = [[] for _ in range(n)]
    for u, v in zip(src, dst):
        adj[int(u)].append(int(v))
    dist = [-1] * n
    dist[s] = 0
    dq = deque([s])
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                dq.append(v)
    return dist


def test_reduction_static_reachability():
    """Every edge at t = 0 with zero duration: earliest arrival reaches exactly the
    vertices BFS reaches, all at time 0."""
    for seed in range(20):
        el = synth.random_small(40, 90, 0x7300 + seed, t_max=0, lam_max=0)
        s = seed % 40
        got = Oracle(el).earliest_arrival(s, 0, 5)
        dist = _bfs(el.n, el.src, el.dst, s)
        assert [g == 0 for g in got] == [d >= 0 for d in dist]
        assert all(g in (0, UNREACHED) for g in got)


@pytest.mark.parametrize("strict", [0, 1])
def test_reduction_hop_distance(strict):
    """A static graph whose every edge is present at each integer time 0..H with duration 1:
    earliest arrival from s at time 0 is the BFS hop distance d (Succeeds), or 2d - 1
    (StrictlySucceeds: every later hop must wait one more instant)."""
    H = 12
    for seed in range(10):
        st = synth.random_small(30, 45, 0x7400 + seed, t_max=0, lam_max=0)
        rows = [(int(u), int(v), tt, 1) for u, v in zip(st.src, st.dst) for tt in range(H + 1)]
        el = from_rows(30, rows)
        s = seed
        got = Oracle(el).earliest_arrival(s, 0, H + 1, strict)
        dist = _bfs(30, st.src, st.dst, s)
        for v in range(30):
            d = dist[v]
            want = 0 if v == s else (UNREACHED if d < 0 else (d if not strict else 2 * d - 1))
            if want != UNREACHED and want > H + 1:
                want = UNREACHED
            assert got[v] == want, (v, d)


@pytest.fixture(scope="module")
def tiny_workload():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    return el, Oracle(el)


@pytest.mark.parametrize("strict", [0, 1])
def test_latest_departure_equals_mirrored_earliest_arrival(tiny_workload, strict):
    """Two independent routes to latest departure: the direct descending scan, and C minus
    earliest arrival on the reversed, time-mirrored graph over [C - tw, C - ta]."""
    el, orc = tiny_workload
    ms, md, mt, ml = mirror_edges(el.src, el.dst, el.t, el.lam)
    morc = Oracle(Edges(el.n, ms, md, mt, ml))
    xs = synth.pick_vertices(el, 6, 0x7500 + strict, False, True)
    for k, x in enumerate(xs):
        ta, tw = [(0, C_MIRROR), (1000, 900_000), (300_000, 700_000)][k % 3]
        ld = orc.latest_departure(x, ta, tw, strict)
        ea = morc.earliest_arrival(x, C_MIRROR - tw, C_MIRROR - ta, strict)
        back = np.where(ea == UNREACHED, UNREACHED, np.uint32(C_MIRROR) - ea).astype(np.uint32)
        assert np.array_equal(ld, back)
        assert orc.admissible(Query(LD, x, ta, tw, strict), ld) == \
            morc.admissible(Query(EA, x, C_MIRROR - tw, C_MIRROR - ta, strict), ea)


@pytest.mark.parametrize("strict", [0, 1])
def test_invariants_tiny_workload(tiny_workload, strict):
    el, orc = tiny_workload
    srcs = synth.pick_vertices(el, 5, 0x7600 + strict, True, False)
    for s in srcs:
        ea = orc.earliest_arrival(s, 0, (1 << 20) - 1, strict)
        assert ea[s] == 0
        assert certify_ea(el, s, 0, (1 << 20) - 1, strict, ea) == (0, 0)
        # window extension: labels finite under a narrower end stay equal; new ones exceed it
        for tw1 in (200_000, 600_000):
            e1 = orc.earliest_arrival(s, 0, tw1, strict)
            fin = e1 != UNREACHED
            assert np.array_equal(e1[fin], ea[fin])
            assert np.all(ea[~fin & (ea != UNREACHED)] > tw1)
        # later window start never helps (for v != s)
        e_late = orc.earliest_arrival(s, 100_000, (1 << 20) - 1, strict)
        mask = np.arange(el.n) != s
        assert np.all(ea[mask].astype(np.uint64) <= e_late[mask].astype(np.uint64))
        # mirrored statements for latest departure: a later window end never hurts
        ld = orc.latest_departure(s, 0, 600_000, strict)
        ld2 = orc.latest_departure(s, 0, 900_000, strict)
        both = (ld != UNREACHED) & mask
        assert np.all(ld2[both] >= ld[both])
        assert np.all(ld2[mask & (ld != UNREACHED)] != UNREACHED)


def test_certificate_rejects_planted_mistakes(tiny_workload):
    """The any-size certificate accepts the oracle's labels and rejects each kind of
    single-label mistake."""
    el, orc = tiny_workload
    s = synth.pick_vertices(el, 1, 0x7700, True, False)[0]
    tw = (1 << 20) - 1
    ea = orc.earliest_arrival(s, 0, tw, 0)
    assert certify_ea(el, s, 0, tw, 0, ea)[0] == 0
    reached = np.flatnonzero((ea != UNREACHED) & (np.arange(el.n) != s))
    unreached = np.flatnonzero(ea == UNREACHED)
    assert reached.size > 10 and unreached.size > 0
    v = int(reached[reached.size // 2])
    for bad in (ea[v] + 1, ea[v] - 1, UNREACHED):
        x = ea.copy()
        x[v] = bad
        assert certify_ea(el, s, 0, tw, 0, x)[0] == 1, bad
    x = ea.copy()
    x[int(unreached[0])] = tw
    assert certify_ea(el, s, 0, tw, 0, x)[0] == 1
    x = ea.copy()
    x[s] = 1
    assert certify_ea(el, s, 0, tw, 0, x)[0] == 1


def test_time_order_is_the_stable_sort():
    """The oracle's radix time order equals a library stable sort by departure time (ties by
    edge index), on times with many ties and on the extremes of the 32-bit range."""
    lib = oracle._load()
    rng = np.random.default_rng(0x50127)
    cases = [np.zeros(0, np.uint32), np.array([7], np.uint32),
             np.array([0xFFFFFFFF, 0, 0xFFFFFFFF, 1, 0, 0x80000000, 2047, 2048, 1 << 22], np.uint32),
             rng.integers(0, 5, 10_000).astype(np.uint32),
             rng.integers(0, 1 << 32, 100_000, dtype=np.uint64).astype(np.uint32),
             (rng.zipf(1.2, 100_000) % (1 << 31)).astype(np.uint32)]
    for t in cases:
        perm = np.empty(t.size, np.uint32)
        assert lib.oracle_time_order(t.size, t.ctypes.data, perm.ctypes.data) == 0
        assert np.array_equal(perm, np.argsort(t, kind="stable").astype(np.uint32))


@pytest.mark.parametrize("strict", [0, 1])
def test_certifier_both_kinds(tiny_workload, strict):
    """The batch certifier accepts the oracle's earliest-arrival and latest-departure labels
    (latest departure through the mirrored graph) and rejects single-label mistakes in
    either kind."""
    el, orc = tiny_workload
    cert = oracle.Certifier(el)
    vs = synth.pick_vertices(el, 3, 0x7800 + strict, True, True)
    qs = [Query(k, v, ta, tw, strict) for v in vs for k in (EA, LD)
          for ta, tw in ((0, C_MIRROR), (1000, 900_000))]
    labs = [orc.query(q) for q in qs]
    assert cert.check_all(qs, lambda i: labs[i], threads=4) == [(0, 0)] * len(qs)
    assert cert.check_all(qs, lambda i: labs[i], threads=2, group=3) == [(0, 0)] * len(qs)
    for i, q in enumerate(qs[:4]):
        lab = labs[i]
        reached = np.flatnonzero((lab != UNREACHED) & (np.arange(el.n) != q.vertex))
        unreached = np.flatnonzero(lab == UNREACHED)
        assert reached.size > 10 and unreached.size > 0
        v = int(reached[reached.size // 3])
        for bad in (lab[v] + 1, lab[v] - 1, UNREACHED):
            x = lab.copy()
            x[v] = bad
            assert cert.check(q, x)[0] == 1, (q, bad)
            # the rows form refutes the same mistake and only in that query of its group
            same = [j for j in range(len(qs)) if qs[j].kind == q.kind]
            res = cert.check_group([qs[j] for j in same], [x if j == i else labs[j] for j in same])
            assert [r[0] for r in res] == [1 if j == i else 0 for j in same], (q, bad)
        x = lab.copy()
        x[int(unreached[0])] = q.tw if q.kind == EA else q.ta
        assert cert.check(q, x)[0] == 1, q
        assert cert.check_group([q], [x])[0][0] == 1, q


def test_invalid_arguments_rejected():
    el = from_rows(3, [(0, 1, 1, 1)])
    orc = Oracle(el)
    with pytest.raises(ValueError):
        orc.earliest_arrival(3, 0, 5)
    with pytest.raises(ValueError):
        orc.earliest_arrival(0, 6, 5)
    with pytest.raises(ValueError):
        orc.latest_departure(0, 0, 0xFFFFFFFF)


def test_empty_graph_and_isolated_source():
    el = Edges(4, [], [], [], [])
    orc = Oracle(el)
    assert orc.earliest_arrival(2, 3, 9).tolist() == [UNREACHED, UNREACHED, 3, UNREACHED]
    assert orc.latest_departure(1, 3, 9).tolist() == [UNREACHED, 9, UNREACHED, UNREACHED]


# ---- fastest paths --------------------------------------------------------------------

def start_times(el, s, ta, tw):
    """Distinct departure times of s's usable out-edges (t >= ta, t + lam <= tw)."""
    m = (el.src == s) & (el.t >= ta) & (el.t.astype(np.uint64) + el.lam <= tw)
    return sorted(set(int(x) for x in el.t[m]))


def fastest_by_start_times(orc, el, s, ta, tw, strict):
    """min over start times d of EA_[d, tw](v) - d: every path starting at d is a candidate
    of EA from d, and EA from d is the end of a path starting at or after d."""
    best = np.full(el.n, UNREACHED, np.uint64)
    for d in start_times(el, s, ta, tw):
        ea = orc.earliest_arrival(s, d, tw, strict).astype(np.uint64)
        ok = ea != UNREACHED
        best[ok] = np.minimum(best[ok], ea[ok] - d)
    best[s] = 0
    return best.astype(np.uint32)


@pytest.mark.parametrize("strict", [0, 1])
def test_fastest_brute_force_tiny_graphs(strict):
    """The one-pass pair scan against enumeration of simple paths, on the tiny multigraphs
    (self-loops, parallel edges, zero durations)."""
    for el, v, ta, tw in _tiny_cases(1500):
        got = Oracle(el).fastest(v, ta, tw, strict)
        want = brute_fastest(el.n, el.src, el.dst, el.t, el.lam, v, ta, tw, strict)
        assert np.array_equal(got, want), (el.src, el.dst, el.t, el.lam, v, ta, tw)


@pytest.mark.parametrize("strict", [0, 1])
def test_fastest_equals_min_over_start_times(tiny_workload, strict):
    """On the 10^5-edge workload graph: the pair scan equals the minimum, over the source's
    departure times d, of earliest arrival from d minus d (the pinned earliest-arrival scan)."""
    el, orc = tiny_workload
    for k in range(4):
        s = int(np.flatnonzero(np.bincount(el.src, minlength=el.n))[7 * k + 3])
        ta, tw = (0, 2**20 - 1) if k % 2 == 0 else (1 << 18, 3 << 18)
        got = orc.fastest(s, ta, tw, strict)
        assert np.array_equal(got, fastest_by_start_times(orc, el, s, ta, tw, strict)), (s, ta, tw)


def test_fastest_reductions():
    """(1) Every edge at t = 0 with zero duration: duration 0 on exactly the BFS-reachable set.
    (2) A chain s -> 1 -> ... -> k with edge i at time i and duration 1 (plus slower early
    copies): the fastest duration to vertex j is j (one path, no waiting).  (3) Waiting
    counts: a later direct edge beats an earlier two-hop path with a long layover."""
    for seed in range(10):
        el = synth.random_small(40, 90, 0x7500 + seed, t_max=0, lam_max=0)
        s = seed % 40
        got = Oracle(el).fastest(s, 0, 5)
        dist = _bfs(el.n, el.src, el.dst, s)
        assert [g == 0 for g in got] == [d >= 0 for d in dist]
        assert all(g in (0, UNREACHED) for g in got)
    k = 8
    rows = [(i, i + 1, i, 1) for i in range(k)] + [(i, i + 1, 0, 3) for i in range(1, k)]
    got = Oracle(from_rows(k + 1, rows)).fastest(0, 0, 100)
    assert got.tolist() == list(range(k + 1))
    rows = [(0, 1, 0, 1), (1, 2, 50, 1), (0, 2, 60, 5)]
    got = Oracle(from_rows(3, rows)).fastest(0, 0, 100)
    assert got.tolist() == [0, 1, 5]  # 0->1->2 takes 0..51; the direct edge takes 5


@pytest.mark.parametrize("strict", [0, 1])
def test_fastest_invariants(tiny_workload, strict):
    """fp[v] <= ea[v] - ta (the earliest-arrival path starts at or after ta); fp is finite
    exactly where ea is; every finite fp is at most tw - ta."""
    el, orc = tiny_workload
    for s in (3, 99, 1234):
        ta, tw = 1 << 17, (1 << 20) - 1
        fp = orc.fastest(s, ta, tw, strict).astype(np.int64)
        ea = orc.earliest_arrival(s, ta, tw, strict).astype(np.int64)
        reached = ea != UNREACHED
        assert np.array_equal(fp != UNREACHED, reached)
        assert np.all(fp[reached] <= ea[reached] - ta)
        assert np.all(fp[reached] <= tw - ta)


# ---- shortest duration ----------------------------------------------------------------

@pytest.mark.parametrize("strict", [0, 1])
def test_shortest_duration_brute_force_tiny_graphs(strict):
    """The one-pass (total, arrival) pair scan against enumeration of simple paths."""
    for el, v, ta, tw in _tiny_cases(1500):
        got = Oracle(el).shortest_duration(v, ta, tw, strict)
        want = brute_shortest_duration(el.n, el.src, el.dst, el.t, el.lam, v, ta, tw, strict)
        assert np.array_equal(got, want), (el.src, el.dst, el.t, el.lam, v, ta, tw)


@pytest.mark.parametrize("strict", [0, 1])
def test_shortest_duration_reduces_to_dijkstra(strict):
    """A static weighted graph whose every edge is present at each integer time 0..H (waiting
    is free and H exceeds every path's length): the least total duration is the static
    shortest-path distance (scipy's Dijkstra), under either predicate (durations >= 1)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    for seed in range(6):
        n = 40
        st = synth.random_small(n, 100, 0x7600 + seed, t_max=0, lam_max=5, lam_min=1)
        H = 5 * n + 5
        rows = [(int(u), int(v), tt, int(l)) for u, v, l in zip(st.src, st.dst, st.lam) for tt in range(H + 1)]
        el = from_rows(n, rows)
        s = seed
        got = Oracle(el).shortest_duration(s, 0, 2 * H, strict)
        w = {}
        for u, v, l in zip(st.src, st.dst, st.lam):  # parallel edges: the lightest counts
            if u != v:
                w[(int(u), int(v))] = min(w.get((int(u), int(v)), 99), int(l))
        M = csr_matrix(([x for x in w.values()], ([k[0] for k in w], [k[1] for k in w])), shape=(n, n))
        dist = dijkstra(M, indices=s)
        want = [0 if v == s else (UNREACHED if np.isinf(dist[v]) else int(dist[v])) for v in range(n)]
        assert got.tolist() == want, seed


def test_shortest_duration_reductions_and_invariants(tiny_workload):
    """(1) All edges at t = 0 with zero duration: 0 exactly on the BFS-reachable set.
    (2) On the 10^5-edge graph: sd <= fp (waiting only adds to a path's duration), sd is
    finite exactly where earliest arrival is, and sd[v] >= the smallest duration of v's
    usable in-edges."""
    for seed in range(10):
        el = synth.random_small(40, 90, 0x7700 + seed, t_max=0, lam_max=0)
        s = seed % 40
        got = Oracle(el).shortest_duration(s, 0, 5)
        dist = _bfs(el.n, el.src, el.dst, s)
        assert [g == 0 for g in got] == [d >= 0 for d in dist]
    el, orc = tiny_workload
    for s in (3, 99, 1234):
        for strict in (0, 1):
            ta, tw = 1 << 17, (1 << 20) - 1
            sd = orc.shortest_duration(s, ta, tw, strict).astype(np.int64)
            fp = orc.fastest(s, ta, tw, strict).astype(np.int64)
            ea = orc.earliest_arrival(s, ta, tw, strict)
            reached = ea != UNREACHED
            assert np.array_equal(sd != UNREACHED, reached)
            assert np.all(sd[reached] <= fp[reached])
            usable = (el.t >= ta) & (el.t.astype(np.int64) + el.lam <= tw)
            minin = np.full(el.n, np.iinfo(np.int64).max)
            np.minimum.at(minin, el.dst[usable], el.lam[usable].astype(np.int64))
            others = reached.copy()
            others[s] = False
            assert np.all(sd[others] >= minin[others])


# ---- temporal BFS (least number of edges) ----------------------------------------------

@pytest.mark.parametrize("strict", [0, 1])
def test_temporal_bfs_brute_force_tiny_graphs(strict):
    for el, v, ta, tw in _tiny_cases(1500):
        got = Oracle(el).temporal_bfs(v, ta, tw, strict)
        want = brute_temporal_bfs(el.n, el.src, el.dst, el.t, el.lam, v, ta, tw, strict)
        assert np.array_equal(got, want), (el.src, el.dst, el.t, el.lam, v, ta, tw)


@pytest.mark.parametrize("strict", [0, 1])
def test_temporal_bfs_reductions_and_invariants(tiny_workload, strict):
    """(1) Every edge of a static graph present at each integer time 0..H with duration 1: the
    level of v is its static BFS distance (H exceeds every path).  (2) On the 10^5-edge graph
    (durations >= 1): finite exactly where earliest arrival is, and at most the shortest
    duration (a least-duration path has at least that many edges, each lasting >= 1)."""
    H = 70
    for seed in range(6):
        st = synth.random_small(30, 45, 0x7800 + seed, t_max=0, lam_max=0)
        rows = [(int(u), int(v), tt, 1) for u, v in zip(st.src, st.dst) for tt in range(H + 1)]
        got = Oracle(from_rows(30, rows)).temporal_bfs(seed, 0, H + 1, strict)
        dist = _bfs(30, st.src, st.dst, seed)
        assert got.tolist() == [UNREACHED if d < 0 else d for d in dist], seed
    el, orc = tiny_workload
    for s in (3, 99, 1234):
        ta, tw = 1 << 17, (1 << 20) - 1
        hops = orc.temporal_bfs(s, ta, tw, strict).astype(np.int64)
        sd = orc.shortest_duration(s, ta, tw, strict).astype(np.int64)
        reached = orc.earliest_arrival(s, ta, tw, strict) != UNREACHED
        assert np.array_equal(hops != UNREACHED, reached)
        assert np.all(hops[reached] <= sd[reached])


# ---- temporal connected components --------------------------------------------------------

def _canonical(labels):
    """Relabel a component labelling by the smallest vertex of each component."""
    labels = np.asarray(labels)
    first = {}
    for v, c in enumerate(labels.tolist()):
        first.setdefault(c, v)
    return np.array([first[c] for c in labels.tolist()], np.uint32)


@pytest.mark.parametrize("seed", range(40))
def test_temporal_cc_brute_force(seed):
    """Union-find over the window's usable edges equals breadth-first search on tiny graphs
    (self-loops, parallel edges, zero durations, windows cutting edges at both ends)."""
    n = 5 + seed % 13
    el = synth.random_small(n, 3 + 2 * seed, 0x7C00 + seed, t_max=30, lam_max=6, lam_min=0)
    for ta, tw in ((0, 40), (5, 20), (12, 12), (0, C_MIRROR)):
        got = oracle.temporal_cc(el, ta, tw)
        want = oracle.brute_temporal_cc(n, el.src, el.dst, el.t, el.lam, ta, tw)
        assert got.tolist() == want.tolist(), (seed, ta, tw)


def test_temporal_cc_equals_scipy_components():
    """A library routine on the same snapshot: scipy's connected components of the window's
    usable edges, relabelled by each component's smallest vertex."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp

    el = synth.rmat(synth.WORKLOADS[1].graph)
    for ta, tw in ((0, (1 << 20) - 1), (100_000, 300_000), (500_000, 500_300)):
        use = (el.t >= ta) & (el.t.astype(np.uint64) + el.lam <= tw)
        a = sp.coo_matrix((np.ones(int(use.sum())), (el.src[use], el.dst[use])), shape=(el.n, el.n))
        _, lab = csgraph.connected_components(a, directed=True, connection="weak")
        got = oracle.temporal_cc(el, ta, tw)
        assert got.tolist() == _canonical(lab).tolist()
        assert all(got[v] <= v for v in range(el.n))
