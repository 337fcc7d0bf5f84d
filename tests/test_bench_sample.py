"""The benchmark's bounded oracle sample (bench.CpuSample): the queries over a graph's most
recent departures give, on the sub-graph of the edges departing in their window, exactly the
labels of the same queries on the whole graph, as its description claims; and the sample keeps
every such edge and no other.  CPU only."""
import numpy as np

import bench
import synth
from oracle import Oracle


def test_sample_labels_equal_whole_graph_labels():
    el = synth.rmat(synth.scaled(synth.WORKLOADS[5].graph, 14, 1 << 19))  # Zipf departures, 16-bit durations
    s = bench.CpuSample(el, 50_000, count=16)  # a tenth of the edges (the benchmark takes 2^24 of 2^31)
    assert 0 < s.sub.m < el.m
    assert s.sub.m == int((el.t >= s.T).sum()) and bool((s.sub.t >= s.T).all())
    assert len(s.queries) == 16 and {q.kind for q in s.queries} == {synth.EA, synth.LD}
    whole, sub = Oracle(el), Oracle(s.sub)
    reached = 0
    for q in s.queries:
        want = whole.query(q)
        assert np.array_equal(sub.query(q), want), q
        reached += int((want != 0xFFFFFFFF).sum())
    assert reached > 16  # the sample queries reach beyond their own sources
