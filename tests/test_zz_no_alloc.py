"""The earliest-arrival entry point that allocates no device memory, for callers that
cannot allocate while they query (a process that gave all device memory to its own pool,
or code running while another library captures a CUDA graph).  Its labels must equal
those of the ordinary entry point, exactly (integer times: tolerance 0), on two calls in a
row that reuse the library's fixed scratch array.  This file is collected last."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


def _labels(t):
    return t.cpu().numpy().view(np.uint32)


def test_no_alloc_matches_the_allocating_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    el = synth.rmat(synth.WORKLOADS[1].graph)
    n = el.n
    g = kx.Graph.from_edges(el)
    g.index(64)
    g.set_tuning(warp_max_edges=32, chunk_edges=64)  # exercise the split-range lists too
    srcs = synth.pick_vertices(el, 2, 0xA110C, True, False)
    windows = [(0, (1 << 20) - 1), (100_000, 800_000)]
    for s, (ta, tw) in zip(srcs, windows):
        want = torch.empty(n, dtype=torch.int32, device="cuda")
        g.earliest_arrival(s, ta, tw, want)
        got = torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        kx.kairos_earliest_arrival_noalloc(g.handle, n, s, ta, tw, got)
        assert np.array_equal(_labels(got), _labels(want)), (s, ta, tw)
        assert int((_labels(got) != 0xFFFFFFFF).sum()) > 1
    g.close()


def test_no_alloc_rejects_what_it_cannot_hold():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = (1 << 20) + 1
    src = np.array([0], np.int32)
    g = kx.Graph(n, src, np.array([1], np.int32), np.array([5], np.uint32), np.array([1], np.uint32))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(kx.KairosError) as e:
        kx.kairos_earliest_arrival_noalloc(g.handle, n, 0, 0, 10, out)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    host = np.zeros(4, np.uint32)
    g.close()
    g = kx.Graph(4, src, np.array([1], np.int32), np.array([5], np.uint32), np.array([1], np.uint32))
    with pytest.raises(kx.KairosError) as e:
        kx.kairos_earliest_arrival_noalloc(g.handle, 4, 0, 0, 10, host)
    assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    g.close()
