"""The earliest-arrival entry point that allocates no device memory, for callers that
cannot allocate while they query (a process that gave all device memory to its own pool,
or code running while another library captures a CUDA graph).  Its labels must equal the
oracle's and those of the ordinary entry point, exactly (integer times: tolerance 0), on
calls in a row that reuse the library's fixed scratch array; the call must allocate
nothing; and graphs beyond the array's limits must be refused.  This file is collected
last."""
import numpy as np
import pytest

import synth
from oracle import UNREACHED, Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _labels(t):
    return t.cpu().numpy().view(np.uint32)


class CountingAllocator(kx.TorchAllocator):
    """Device allocations through PyTorch, recorded; refused (NULL) once `budget` bytes
    would be live."""

    def __init__(self):
        super().__init__()
        self.budget = 1 << 62
        self.live = {}
        self.calls = 0

    def _alloc(self, nbytes, ctx):
        self.calls += 1
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


def test_no_alloc_matches_the_oracle_and_the_allocating_entry_point_on_two_calls():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    n = el.n
    orc = Oracle(el)
    A = CountingAllocator()
    g = kx.Graph.from_edges(el, allocator=A)
    g.index(64)
    g.set_tuning(warp_max_edges=32, chunk_edges=64)  # exercise the split-range lists too
    srcs = synth.pick_vertices(el, 2, 0xA110C, True, False)
    windows = [(0, (1 << 20) - 1), (100_000, 800_000)]
    wants = []
    for s, (ta, tw) in zip(srcs, windows):
        want = torch.empty(n, dtype=torch.int32, device="cuda")
        g.earliest_arrival(s, ta, tw, want)
        wants.append(_labels(want))
    # from here on any device allocation by the library is refused and would show up
    torch.cuda.synchronize()
    A.budget = sum(A.live.values())
    live, calls = dict(A.live), A.calls
    bufs = [torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") for _ in range(3)]
    # the first call on the device looks up the fixed array (the driver may load the
    # library's device code then); device memory is compared from after it
    g.earliest_arrival_noalloc(srcs[1], *windows[1], bufs[2])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for s, (ta, tw), want, got in zip(srcs, windows, wants, bufs):
        g.earliest_arrival_noalloc(s, ta, tw, got)
        lab = _labels(got)
        assert np.array_equal(lab, want), (s, ta, tw)
        assert np.array_equal(lab, orc.earliest_arrival(s, ta, tw)), (s, ta, tw)
        assert int((lab != UNREACHED).sum()) > 1
    torch.cuda.synchronize()
    assert A.calls == calls and A.live == live
    # a device allocation is at least one 2 MiB page: none may have happened
    assert torch.cuda.mem_get_info()[0] > free0 - (1 << 20)
    assert np.array_equal(_labels(bufs[2]), wants[1])
    A.budget = 1 << 62
    g.close()


def test_no_alloc_at_the_vertex_limit_medium_graph():
    """The 2^20-vertex, 2^25-edge workload graph is exactly at the vertex limit; with the
    default split shape its long ranges fit the fixed lists, and the labels equal the
    oracle's.  With 32-edge splits they do not fit, and the call refuses."""
    el = synth.rmat(synth.WORKLOADS[2].graph)
    assert el.n == 1 << 20
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    g.index(synth.WORKLOADS[2].theta)
    (s,) = synth.pick_vertices(el, 1, 0xA1100, True, False)
    out = torch.empty(el.n, dtype=torch.int32, device="cuda")
    want = Oracle(el).earliest_arrival(s, 0, synth.C_MIRROR)
    for _ in range(2):
        out.fill_(0x5A5A5A5A)
        g.earliest_arrival_noalloc(s, 0, synth.C_MIRROR, out)
        assert np.array_equal(_labels(out), want)
    g.set_tuning(warp_max_edges=32, chunk_edges=512)
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival_noalloc(s, 0, synth.C_MIRROR, out)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    assert "split-range" in str(e.value)
    g.close()


def test_no_alloc_round_cap_returns_timeout(monkeypatch):
    """A round cap below what the query needs makes the call return KAIROS_ERR_TIMEOUT (a
    bounded wait, no fault); the next call without the cap succeeds."""
    el = synth.rmat(synth.WORKLOADS[1].graph)
    g = kx.Graph.from_edges(el)
    (s,) = synth.pick_vertices(el, 1, 0xA1101, True, False)
    out = torch.empty(el.n, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("KAIROS_ROUND_CAP", "1")
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival_noalloc(s, 0, (1 << 20) - 1, out)
    assert e.value.status == kx.KAIROS_ERR_TIMEOUT
    monkeypatch.delenv("KAIROS_ROUND_CAP")
    g.earliest_arrival_noalloc(s, 0, (1 << 20) - 1, out)
    assert np.array_equal(_labels(out), Oracle(el).earliest_arrival(s, 0, (1 << 20) - 1))
    g.close()


def test_no_alloc_rejects_what_it_cannot_hold():
    n = (1 << 20) + 1
    src = np.array([0], np.int32)
    g = kx.Graph(n, src, np.array([1], np.int32), np.array([5], np.uint32), np.array([1], np.uint32))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival_noalloc(0, 0, 10, out)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    host = np.zeros(4, np.uint32)
    g.close()
    g = kx.Graph(4, src, np.array([1], np.int32), np.array([5], np.uint32), np.array([1], np.uint32))
    with pytest.raises(kx.KairosError) as e:
        g.earliest_arrival_noalloc(0, 0, 10, host)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()
