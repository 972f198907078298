"""The serving loop: requests admitted by HBM footprint and sorted in
continuous batches on several streams give, for every request, exactly the
result of sorting it alone (and the oracle's)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def _requests(num, seed, rate, smax):
    from paper_1808_00963_gb300.serve import make_request
    out = []
    for i, (t, kind, size, sd) in enumerate(gen.trace(num, seed, rate, smin=1000, smax=smax)):
        s = gen.make_set(kind, size, sd)
        r = make_request(i, t, s.chars, s.offsets, s.max_len)
        r.meta["set"] = s
        out.append(r)
    return out


@pytest.mark.parametrize("mode", ["served", "plain"])
def test_each_result_same_alone_and_in_the_mix(mode):
    import torch

    import paper_1808_00963_gb300 as ss
    from paper_1808_00963_gb300.serve import Server
    reqs = _requests(36, 5, rate=3000.0, smax=60000)
    srv = Server(budget_bytes=2 << 30, streams=3, batch_max=16, big=30000, mode=mode)
    stats = srv.run(reqs)
    assert not stats["errors"]
    for r in reqs:
        s = r.meta["set"]
        gp = r.perm.numpy().view(np.uint32)
        gl = r.lcp.numpy().view(np.uint32)
        wp, wl = oracle.sort(s.chars, s.offsets, s.max_len)
        assert np.array_equal(gp, wp) and np.array_equal(gl, wl), r.rid
        # alone, on its own
        ch = torch.from_numpy(s.chars).cuda()
        of = torch.from_numpy(s.offsets.view(np.int64)).cuda()
        p, l = ss.sort(ch, of, max_len=s.max_len)
        assert np.array_equal(p.cpu().numpy().view(np.uint32), gp)
        assert np.array_equal(l.cpu().numpy().view(np.uint32), gl)
    if mode == "served":
        assert stats["mean_batch"] > 1.0


def test_admission_respects_budget():
    from paper_1808_00963_gb300.serve import Server
    reqs = _requests(12, 6, rate=1e6, smax=20000)
    budget = max(r.footprint for r in reqs) + 1  # room for about one request at a time
    srv = Server(budget_bytes=budget, streams=4, batch_max=8, big=10**9, mode="served")
    stats = srv.run(reqs)
    assert not stats["errors"]
    assert srv.free == budget
    assert all(r.done >= r.start >= 0 for r in reqs)


@pytest.mark.slow
def test_served_requests_up_to_millions_of_strings():
    """Requests of configuration 5's size range (log-uniform 1k..5M strings,
    mixed generators), many at once so that batches and requests sorted alone
    on the multi-block path overlap on four streams: every result passes the
    oracle's O(n + D) checker and equals the request sorted alone."""
    import torch

    import paper_1808_00963_gb300 as ss
    from paper_1808_00963_gb300.serve import Server
    reqs = _requests(24, 17, rate=400.0, smax=5_000_000)
    assert max(r.n for r in reqs) > 1_000_000
    srv = Server(budget_bytes=16 << 30, streams=4, mode="served")
    stats = srv.run(reqs)
    assert not stats["errors"]
    for r in reqs:
        s = r.meta["set"]
        gp = r.perm.numpy().view(np.uint32)
        gl = r.lcp.numpy().view(np.uint32)
        assert oracle.check(s.chars, s.offsets, gp, gl, s.max_len) == -1, r.rid
        ch = torch.from_numpy(s.chars).cuda()
        of = torch.from_numpy(s.offsets.view(np.int64)).cuda()
        p, l = ss.sort(ch, of, max_len=s.max_len)
        assert np.array_equal(p.cpu().numpy().view(np.uint32), gp)
        assert np.array_equal(l.cpu().numpy().view(np.uint32), gl)


@pytest.mark.slow
def test_served_trickle_of_requests_keeps_every_result():
    """Requests arriving one by one (mostly single-request groups, sorted
    asynchronously, two groups in flight per worker stream, some small
    batches between them): every result of 400 requests, replaying a pool of
    40 sets of 1k..3M strings, equals its set sorted alone, and the pool sets
    pass the oracle's O(n + D) checker.  (This pattern once exposed batch
    descriptors read before their upload had landed.)"""
    import dataclasses

    import torch

    import paper_1808_00963_gb300 as ss
    from paper_1808_00963_gb300.serve import Server, make_request
    spec = gen.trace(400, 23, 900.0, smin=1000, smax=3_000_000)
    pool = [gen.make_set(k, n, sd) for (_, k, n, sd) in spec[:40]]
    expected = []
    for st in pool:
        ch = torch.from_numpy(st.chars).cuda()
        of = torch.from_numpy(st.offsets.view(np.int64)).cuda()
        p, l = ss.sort(ch, of, max_len=st.max_len)
        hp, hl = p.cpu().numpy().view(np.uint32), l.cpu().numpy().view(np.uint32)
        assert oracle.check(st.chars, st.offsets, hp, hl, st.max_len) == -1, st.name
        expected.append((hp.copy(), hl.copy()))
    base = [make_request(i, 0.0, st.chars, st.offsets, st.max_len) for i, st in enumerate(pool)]
    reqs = [dataclasses.replace(base[j % len(pool)], rid=j, arrival=t, meta={"pool": j % len(pool)})
            for j, (t, _, _, _) in enumerate(spec)]
    bad = []

    def verify(r):
        hp, hl = expected[r.meta["pool"]]
        if not (np.array_equal(r.perm.numpy().view(np.uint32), hp)
                and np.array_equal(r.lcp.numpy().view(np.uint32), hl)):
            bad.append(r.rid)

    stats = Server(budget_bytes=16 << 30, streams=4, mode="served", on_done=verify).run(reqs)
    assert not stats["errors"]
    assert not bad, bad[:10]
    assert stats["mean_batch"] < 4.0  # mostly small groups
