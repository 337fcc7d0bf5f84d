"""GPU parity of temporal connected components (kairos_temporal_cc) against the oracle's
union-find, label by label (integer labels: bit-exact): windows cutting edges at both ends,
random multigraphs with self-loops and zero durations, 16-bit durations, the 2^25-edge medium
graph at full size, and host, page-locked host and device outputs."""
import numpy as np
import pytest

import oracle
import synth
from oracle import C_MIRROR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev_labels(g, n, ta, tw):
    out = torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    g.temporal_cc(ta, tw, out)
    return out.cpu().numpy().view(np.uint32)


def test_tiny_workload_windows():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    g = kx.Graph.from_edges(el)
    for ta, tw in ((0, (1 << 20) - 1), (0, C_MIRROR), (100_000, 300_000), (500_000, 500_300), (7, 7)):
        want = oracle.temporal_cc(el, ta, tw)
        assert np.array_equal(dev_labels(g, el.n, ta, tw), want), (ta, tw)
        host = np.zeros(el.n, np.uint32)
        g.temporal_cc(ta, tw, host)
        assert np.array_equal(host, want)
        pinned = torch.zeros(el.n, dtype=torch.int32, pin_memory=True)
        g.temporal_cc(ta, tw, pinned.numpy().view(np.uint32))
        assert np.array_equal(pinned.numpy().view(np.uint32), want)
    with pytest.raises(kx.KairosError):
        g.temporal_cc(5, 4, np.zeros(el.n, np.uint32))
    g.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_multigraphs(seed):
    n, m = 40 + 31 * seed, 60 + 150 * seed
    el = synth.random_small(n, m, 0xCC00 + seed, t_max=50, lam_max=5, lam_min=0)
    g = kx.Graph.from_edges(el)
    for ta, tw in ((0, 60), (10, 30), (25, 25)):
        assert np.array_equal(dev_labels(g, n, ta, tw), oracle.temporal_cc(el, ta, tw)), (seed, ta, tw)
    g.close()


def test_uint16_and_medium_full_size():
    spec = synth.scaled(synth.WORKLOADS[5].graph, 14, 1 << 18)
    el = synth.rmat(spec)
    g = kx.Graph.from_edges(el)
    for ta, tw in ((0, C_MIRROR), (1000, 1 << 20)):
        assert np.array_equal(dev_labels(g, el.n, ta, tw), oracle.temporal_cc(el, ta, tw))
    g.close()
    el = synth.rmat(synth.WORKLOADS[2].graph)
    g = kx.Graph.from_edges(el, stream=torch.cuda.Stream())
    from oracle import selectivity as sel
    T = sel.recent_start(el.t, 5)  # the paper's window: the most recent departures to the end
    for ta, tw in ((0, C_MIRROR), (T, C_MIRROR)):
        assert np.array_equal(dev_labels(g, el.n, ta, tw), oracle.temporal_cc(el, ta, tw)), (ta, tw)
    g.close()
