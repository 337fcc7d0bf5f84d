"""The continuous-batching server: queries of both kinds, predicates and windows submitted
while others run; every result equals the oracle and the same query answered alone."""
import time

import numpy as np
import pytest

import synth
from oracle import Oracle, UNREACHED
from synth import EA, LD, Query

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module")
def served():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    el = synth.rmat(synth.WORKLOADS[1].graph)
    g = kx.Graph.from_edges(el)
    g.index(64)
    yield el, Oracle(el), g
    g.close()


def mixed_queries(el, count, seed):
    vs = synth.pick_vertices(el, count, seed, True, True)
    qs = []
    for i, v in enumerate(vs):
        d = lambda k: synth.draw(seed, i, k)
        L = 1 + synth.below(d(1), 1 << 20)
        ta = synth.below(d(2), (1 << 20) - L + 1)
        kind = EA if synth.below(d(3), 10) < 7 else LD
        qs.append(Query(kind, v, ta, ta + L - 1, synth.below(d(4), 2)))
    return qs


def checksum(lab):
    v = np.arange(1, lab.size + 1, dtype=np.uint64)
    return int(np.sum(v * lab.astype(np.uint64), dtype=np.uint64))


def wait(server, ticket):
    info = kx.kairos_serve_poll(server, ticket, -1)
    assert info.status == kx.KAIROS_OK, info.status
    return info


@pytest.mark.parametrize("slots,slice_rounds,concurrent", [(2, 1, 1), (4, 2, 1), (32, 4, 1), (4, 2, 2), (16, 1, 2)])
def test_served_results_equal_oracle_and_alone(served, slots, slice_rounds, concurrent):
    """concurrent = 2: the two sessions' slices run at once on their own streams."""
    el, orc, g = served
    qs = mixed_queries(el, 45, 0xB000 + slots + 7 * concurrent)
    alone = np.zeros((len(qs), el.n), np.uint32)
    g.set_tuning(lanes=1, concurrent=1)
    g.batch(qs, alone, want_stats=False)
    g.set_tuning(concurrent=concurrent)
    server = kx.kairos_serve_create(g.handle, max_slots=slots, rounds_per_slice=slice_rounds)
    try:
        outs, tickets = [], []
        # three waves: later waves arrive while earlier queries are still on the device
        for wave in range(3):
            for q in qs[wave * 15:(wave + 1) * 15]:
                o = torch.full((el.n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") if len(outs) % 2 \
                    else np.full(el.n, 0x5A5A5A5A, np.uint32)
                outs.append(o)
                tickets.append(kx.kairos_serve_submit(server, q, o))
            time.sleep(0.002)
        infos = [wait(server, t) for t in tickets]
    finally:
        kx.kairos_serve_destroy(server)
        g.set_tuning(concurrent=1)
    for i, q in enumerate(qs):
        got = outs[i].cpu().numpy().view(np.uint32) if hasattr(outs[i], "cpu") else outs[i]
        want = orc.query(q)
        assert np.array_equal(got, want), q
        assert np.array_equal(got, alone[i])
        assert infos[i].reached == int((want != UNREACHED).sum())
        assert infos[i].checksum == checksum(want)
        assert infos[i].relaxed_edges == orc.admissible(q, want)
        assert infos[i].latency_ms > 0


def test_busy_and_not_ready(served):
    el, orc, g = served
    qs = mixed_queries(el, 200, 0xB100)
    server = kx.kairos_serve_create(g.handle, max_slots=2, queue_capacity=8, rounds_per_slice=1)
    accepted, busy = [], 0
    try:
        for q in qs:
            o = np.empty(el.n, np.uint32)
            try:
                accepted.append((q, o, kx.kairos_serve_submit(server, q, o)))
            except kx.KairosError as e:
                assert e.status == kx.KAIROS_ERR_BUSY
                busy += 1
        assert busy > 0
        for q, o, t in accepted:
            wait(server, t)
            assert np.array_equal(o, orc.query(q))
        with pytest.raises(kx.KairosError):
            kx.kairos_serve_poll(server, 10 ** 9, 0)
    finally:
        kx.kairos_serve_destroy(server)
