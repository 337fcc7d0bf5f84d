"""The autotune cache of the binding (host logic, CPU only): a hit installs the stored launch
shape without measuring; another graph, threshold, sample, GPU or library build misses."""
import json

import numpy as np
import pytest

import synth
import paper_2401_02563_gb300 as kx


class FakeGraph(kx.Graph):
    def __init__(self, el, theta=256):
        self.n, self.m = el.n, len(el.src)
        self.theta = theta
        self.fingerprint = kx.graph_fingerprint(el.n, el.src, el.dst, el.t, el.lam)
        self.handle = object()

    def close(self):  # nothing was built
        self.handle = None


@pytest.fixture
def fake_library(monkeypatch):
    calls = {"autotune": 0, "set": []}

    def autotune(handle, sample, min_lanes=1):
        calls["autotune"] += 1
        t = kx.kairos_tuning()
        t.lanes, t.warp_max_edges, t.chunk_edges, t.concurrent = 16, 512, 1024, 2
        return t

    def set_tuning(handle, **fields):
        calls["set"].append(fields)
        return fields

    monkeypatch.setattr(kx, "kairos_autotune", autotune)
    monkeypatch.setattr(kx, "kairos_set_tuning", set_tuning)
    monkeypatch.setattr(kx, "_device_name", lambda: "GPU-A")
    monkeypatch.setattr(kx, "_library_digest", lambda: "lib-1")
    return calls


def test_hit_installs_stored_shape_without_measuring(tmp_path, fake_library):
    el = synth.random_small(50, 300, 0x1111, t_max=100, lam_max=5)
    qs = [synth.Query(synth.EA, 3, 0, 100), synth.Query(synth.LD, 7, 0, 100)]
    path = str(tmp_path / "tune.json")
    g = FakeGraph(el)
    g.autotune(qs, cache=path)
    assert fake_library["autotune"] == 1 and not fake_library["set"]
    stored = json.load(open(path))
    assert len(stored) == 1 and list(stored.values())[0]["lanes"] == 16
    FakeGraph(el).autotune(qs, cache=path)  # same graph, threshold, sample: a hit
    assert fake_library["autotune"] == 1
    assert fake_library["set"][-1]["concurrent"] == 2 and fake_library["set"][-1]["chunk_edges"] == 1024


def test_misses(tmp_path, fake_library, monkeypatch):
    el = synth.random_small(50, 300, 0x1111, t_max=100, lam_max=5)
    other = synth.random_small(50, 300, 0x2222, t_max=100, lam_max=5)
    qs = [synth.Query(synth.EA, 3, 0, 100)]
    path = str(tmp_path / "tune.json")
    FakeGraph(el).autotune(qs, cache=path)
    FakeGraph(other).autotune(qs, cache=path)                       # another graph
    FakeGraph(el, theta=16).autotune(qs, cache=path)                # another index threshold
    FakeGraph(el).autotune([synth.Query(synth.EA, 4, 0, 100)], cache=path)  # another sample
    monkeypatch.setattr(kx, "_device_name", lambda: "GPU-B")
    FakeGraph(el).autotune(qs, cache=path)                          # another GPU model
    monkeypatch.setattr(kx, "_library_digest", lambda: "lib-2")
    FakeGraph(el).autotune(qs, cache=path)                          # another library build
    assert fake_library["autotune"] == 6 and not fake_library["set"]
    assert len(json.load(open(path))) == 6


def test_fingerprint_host_and_sizes():
    el = synth.random_small(50, 300, 0x1111, t_max=100, lam_max=5)
    a = kx.graph_fingerprint(el.n, el.src, el.dst, el.t, el.lam)
    assert a == kx.graph_fingerprint(el.n, el.src.copy(), el.dst.copy(), el.t.copy(), el.lam.copy())
    t2 = el.t.copy()
    t2[0] += 1
    assert a != kx.graph_fingerprint(el.n, el.src, el.dst, t2, el.lam)
    assert a != kx.graph_fingerprint(el.n + 1, el.src, el.dst, el.t, el.lam)
    e = np.zeros(0, np.int32)
    assert kx.graph_fingerprint(4, e, e, e.astype(np.uint32), e.astype(np.uint32))
