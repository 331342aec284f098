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


def _oracle_tables(tables):
    return [oracle.Table(oracle.ICEBERG, t.cfg.key_bits, t.cfg.num_buckets,
                         t.cfg.num_buckets_backyard, fpw0=t.cfg.fields_per_word,
                         fpw1=t.cfg.fields_per_word_backyard, seed=t.cfg.seed) for t in tables]


@pytest.mark.parametrize("realtime", [False, True])
def test_mix_equals_alone_equals_oracle(realtime):
    from paper_2406_09255_gb300.serve import Server, make_requests, run_sequential
    nt = 5
    seeds = [7000 + i for i in range(nt)]
    rate = 0 if not realtime else 20000.0
    reqs_a = make_requests(240, nt, rate, min_size=16, max_size=6000, rng_seed=11)
    reqs_b = make_requests(240, nt, rate, min_size=16, max_size=6000, rng_seed=11)
    ta, tb = make_tables(nt, seeds), make_tables(nt, seeds)
    srv = Server(ta, seeds, keep_results=True)
    srv.plan(reqs_a, seed=3)
    out_a = srv.run(reqs_a, realtime=realtime)
    assert srv.waves < len(reqs_a)  # requests were batched together
    base = Server(tb, seeds, keep_results=True)
    base.plan(reqs_b, seed=3)
    out_b = run_sequential(base, reqs_b, realtime=False)
    # the oracle, in admission order, on keys computed on the host from each
    # request's recipe (the device generator must have produced the same)
    orc = _oracle_tables(ta)
    for ra, rb in zip(out_a, out_b):
        assert ra.rid == rb.rid and ra.done >= ra.arrival and not ra.rejected
        kc = srv.request_keys(ra).numpy().view(np.uint64)
        assert np.array_equal(ra.keys.cpu().numpy().view(np.uint64), kc)
        assert np.array_equal(rb.keys.cpu().numpy().view(np.uint64), kc)
        sa, sb = ra.status.cpu().numpy(), rb.status.cpu().numpy()
        o = orc[ra.table]
        so = o.find(kc) if ra.op == "find" else o.insert(kc)
        assert (so != oracle.FULL).all()
        assert per_request_equal(sa, sb, kc), (ra.rid, ra.op)
        assert per_request_equal(sa, so, kc), (ra.rid, ra.op)
    for x, y, o in zip(ta, tb, orc):
        sx = np.sort(x.enumerate()[0].cpu().numpy().view(np.uint64))
        sy = np.sort(y.enumerate()[0].cpu().numpy().view(np.uint64))
        assert np.array_equal(sx, sy)
        assert np.array_equal(sx, np.sort(o.enumerate()))


def test_admission_by_memory_and_headroom():
    """A 6,000-key arena: a request that does not fit next to the one in
    flight waits (and so does the request behind it) and is admitted once the
    first completes; a write request whose fresh keys exceed its table's
    headroom (max_fill = 0.3 of its slots) is rejected; a request whose
    deadline has passed when it is considered is cancelled. Every admitted
    request's result equals the one-at-a-time run's and the oracle's."""
    from paper_2406_09255_gb300.serve import FIND, FOP, Request, Server, run_sequential
    nt = 3
    seeds = [7100 + i for i in range(nt)]

    def requests():
        return [Request(0, 0, FOP, 4000, 0.0), Request(1, 1, FOP, 3000, 0.0),
                Request(2, 2, FIND, 500, 0.0), Request(3, 0, FOP, 20000, 0.0),
                Request(4, 2, FOP, 800, 0.0), Request(5, 1, FIND, 100, 0.0, deadline=0.0)]

    ta, tb = make_tables(nt, seeds), make_tables(nt, seeds)
    srv = Server(ta, seeds, keep_results=True, fill_cap=0.9, max_fill=0.3, arena_keys=6000)
    reqs = srv.plan(requests(), seed=5)
    srv.run(reqs, realtime=False)
    r = {q.rid: q for q in reqs}
    assert 1 in srv.held_for_memory
    assert r[1].admitted >= r[0].done and r[2].admitted >= r[0].done
    assert r[3].rejected == "table headroom" and r[3].status is None
    # a request whose deadline passed before it could be admitted is cancelled
    assert r[5].rejected == "cancelled" and r[5].status is None
    assert srv.rejected == 2 and srv.arena.used() == 0
    base = Server(tb, seeds, keep_results=True, fill_cap=0.9, max_fill=0.3)
    rb = {q.rid: q for q in run_sequential(base, base.plan(requests(), seed=5), realtime=False)}
    assert rb[3].rejected == "table headroom"
    orc = _oracle_tables(ta)
    for rid in (0, 1, 2, 4):
        kc = srv.request_keys(r[rid]).numpy().view(np.uint64)
        assert np.array_equal(r[rid].keys.cpu().numpy().view(np.uint64), kc)
        sa, sb = r[rid].status.cpu().numpy(), rb[rid].status.cpu().numpy()
        o = orc[r[rid].table]
        so = o.find(kc) if r[rid].op == FIND else o.insert(kc)
        assert per_request_equal(sa, sb, kc) and per_request_equal(sa, so, kc), rid


def test_device_generator_matches_the_definition():
    """The request-key generator kernel (input generation for the served
    benchmark) writes exactly the keys workloads.request_keys defines, for
    odd and even key widths, at arbitrary arena offsets."""
    from paper_2406_09255_gb300 import workloads as W
    out = torch.full((50000,), -1, dtype=torch.int64, device=DEV)
    reqs, off = [], 7
    for i, (n, nf, hi, w) in enumerate([(1000, 300, 5000, 48), (77, 0, 0, 33), (4096, 4096, 0, 40),
                                        (5000, 2000, 123456, 31), (1, 0, 9, 20)]):
        reqs.append(dict(out_off=off, n=n, n_fresh=nf, fresh_base=10 * i, re_hi=hi,
                         re_seed=W.splitmix(9, i), miss_base=1 << 18, key_bits=w, seed=100 + i))
        off += n + 13
    W.request_keys_device(reqs, out)
    torch.cuda.synchronize()
    got = out.cpu()
    for d in reqs:
        want = W.request_keys(d["n"], d["n_fresh"], d["fresh_base"], d["re_hi"], d["re_seed"],
                              d["miss_base"], d["key_bits"], d["seed"])
        assert torch.equal(got[d["out_off"]: d["out_off"] + d["n"]], want)
    # positions between requests are left alone
    assert (got[:7] == -1).all()
