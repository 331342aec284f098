"""Served request loop: each request's result is the same in the mix (waves of
continuous batching, overlapping on two streams) as alone (one synchronous
launch per request in arrival order), and both match the oracle replaying the
requests in admission order.

Tolerance: lookups compare byte for byte. For find-or-put, a key that occurs
once in its request compares byte for byte; for a key repeated inside one
request, exactly one copy reports PUT if the key was new and the others FOUND
(which copy wins is not unique). The stored sets of every table are equal."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_tables(nt, seeds):
    import paper_2406_09255_gb300 as m
    return [m.Table(m.ICEBERG, 36, 1 << (10 + i % 3), 1 << (7 + i % 3), seed=seeds[i])
            for i in range(nt)]


def per_request_equal(a, b, keys):
    """a, b: status arrays of one request; keys: its keys (numpy)."""
    if np.array_equal(a, b):
        return True
    uniq, inv, cnt = np.unique(keys, return_inverse=True, return_counts=True)
    single = cnt[inv] == 1
    if not np.array_equal(a[single], b[single]):
        return False
    rep = ~single
    if not (np.isin(a[rep], (1, 2)).all() and np.isin(b[rep], (1, 2)).all()):
        return False
    pa = np.bincount(inv, weights=(a == 2), minlength=len(uniq))
    pb = np.bincount(inv, weights=(b == 2), minlength=len(uniq))
    return np.array_equal(pa, pb)


@pytest.mark.parametrize("realtime", [False, True])
def test_mix_equals_alone_equals_oracle(realtime):
    from paper_2406_09255_gb300.serve import Server, make_requests, run_sequential
    nt = 5
    seeds = [7000 + i for i in range(nt)]
    rate = 0 if not realtime else 20000.0
    reqs_a = make_requests(240, nt, rate, min_size=16, max_size=6000, rng_seed=11)
    reqs_b = make_requests(240, nt, rate, min_size=16, max_size=6000, rng_seed=11)
    ta, tb = make_tables(nt, seeds), make_tables(nt, seeds)
    srv = Server(ta, seeds)
    srv.plan(reqs_a, seed=3)
    out_a = srv.run(reqs_a, realtime=realtime)
    assert srv.waves < len(reqs_a)  # requests were batched together
    base = Server(tb, seeds)
    base.plan(reqs_b, seed=3)
    out_b = run_sequential(base, reqs_b, realtime=False)
    # the oracle, in admission order
    orc = [oracle.Table(oracle.ICEBERG, 36, t.cfg.num_buckets, t.cfg.num_buckets_backyard,
                        fpw0=t.cfg.fields_per_word, fpw1=t.cfg.fields_per_word_backyard,
                        seed=t.cfg.seed) for t in ta]
    for ra, rb in zip(out_a, out_b):
        assert ra.rid == rb.rid and ra.done >= ra.arrival
        ka = ra.keys.cpu().numpy().view(np.uint64)
        assert np.array_equal(ka, rb.keys.cpu().numpy().view(np.uint64))
        sa, sb = ra.status.cpu().numpy(), rb.status.cpu().numpy()
        o = orc[ra.table]
        so = o.find(ka) if ra.op == "find" else o.insert(ka)
        assert (so != oracle.FULL).all()
        assert per_request_equal(sa, sb, ka), (ra.rid, ra.op)
        assert per_request_equal(sa, so, ka), (ra.rid, ra.op)
    for x, y, o in zip(ta, tb, orc):
        sx = np.sort(x.enumerate()[0].cpu().numpy().view(np.uint64))
        sy = np.sort(y.enumerate()[0].cpu().numpy().view(np.uint64))
        assert np.array_equal(sx, sy)
        assert np.array_equal(sx, np.sort(o.enumerate()))
