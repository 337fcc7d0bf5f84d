"""One query stream over several server replicas (kairos_router_*), with two replicas of the
same graph on one GPU standing in for one replica per GPU: every answer equals the oracle's
and the same query alone, host buffers are spread over both replicas by load, device buffers
go to a replica on their device, and tickets poll back through the router."""
import threading

import numpy as np
import pytest

import synth
from oracle import UNREACHED, Oracle
from synth import EA, LD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2401_02563_gb300 as kx  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def checksum(lab):
    """sum over v of (v + 1) * label[v], mod 2^64 (uint64 arithmetic wraps)."""
    v = np.arange(1, lab.size + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int((v * lab.astype(np.uint64)).sum(dtype=np.uint64))


def test_router_two_replicas_one_device():
    el = synth.rmat(synth.WORKLOADS[1].graph)
    orc = Oracle(el)
    graphs = [kx.Graph.from_edges(el, stream=torch.cuda.Stream()) for _ in range(2)]
    for g in graphs:
        g.index(64)
    servers = [kx.kairos_serve_create(g.handle, max_slots=8, rounds_per_slice=2) for g in graphs]
    router = kx.kairos_router_create(servers)
    try:
        # a served-style mix on this graph: 70/30 kinds, log-uniform windows over its time span
        vs = synth.pick_vertices(el, 60, 0xD100, True, True)
        wins = synth.log_uniform_windows(60, 0xD101, 1 << 20, 10.0, 20.0)
        qs = [synth.Query(EA if i % 10 < 7 else LD, v, ta, tw) for i, (v, (ta, tw)) in enumerate(zip(vs, wins))]
        host = [np.full(el.n, 0x5A5A5A5A, np.uint32) for _ in qs]
        dev = [torch.full((el.n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda") for _ in qs]
        # host buffers from two submitting threads, then device buffers
        tickets = [None] * len(qs)

        def submit(part):
            for i in range(part, len(qs), 2):
                tickets[i] = kx.kairos_router_submit(router, qs[i], host[i])

        th = [threading.Thread(target=submit, args=(p,)) for p in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        infos = [kx.kairos_router_poll(router, t, -1) for t in tickets]
        dt = [kx.kairos_router_submit(router, q, d) for q, d in zip(qs, dev)]
        dinfos = [kx.kairos_router_poll(router, t, -1) for t in dt]
        sub, done = kx.kairos_router_replica_counts(router, 2)
        assert sum(sub) == 2 * len(qs) and sub == done
        assert min(sub) > 0  # both replicas took work
        for i, q in enumerate(qs):
            want = orc.query(q)
            assert infos[i].status == kx.KAIROS_OK and dinfos[i].status == kx.KAIROS_OK
            assert np.array_equal(host[i], want), q
            assert np.array_equal(dev[i].cpu().numpy().view(np.uint32), want), q
            assert infos[i].reached == int((want != UNREACHED).sum())
            assert infos[i].checksum == checksum(want) == dinfos[i].checksum
        with pytest.raises(kx.KairosError) as e:  # a ticket is polled once
            kx.kairos_router_poll(router, tickets[0], 0)
        assert e.value.status == kx.KAIROS_ERR_INVALID_ARG
    finally:
        kx.kairos_router_destroy(router)
        for s in servers:
            kx.kairos_serve_destroy(s)
        for g in graphs:
            g.close()
