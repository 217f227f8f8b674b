"""GPU tests of the serving loop: concurrent (continuous-batching) execution
gives every request the same bits as running it alone and as the direct API,
with 1024-, 2048- and 3072-bit keys in one mix (the 3072-bit kernels overlap
the 2048-bit ones);
admission respects the HBM budget; queued requests can be cancelled; a bad
request fails on its own without disturbing the others."""

import numpy as np
import pytest
import torch

import oracle
from paper_2504_03909_b300 import native, paillier as P, synth

pytestmark = pytest.mark.gpu

MFULL, FFULL = 3000, 6
GH_BITS = 38


def _dataset(n_bits, seed):
    p, q = synth.gen_primes(n_bits, seed)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(MFULL, seed + 10)
    r = synth.gen_r(p * q, n_bits, 2 * MFULL, seed + 10, p, q)
    m = P.encode(torch.from_numpy(gh.reshape(-1)).cuda())
    ct = P.encrypt(key, m, P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct.view(2, MFULL, -1))
    # the same g/h values packed one plaintext per sample (B = 38 covers 3000 samples)
    g_d, h_d = torch.from_numpy(gh[0].copy()).cuda(), torch.from_numpy(gh[1].copy()).cuda()
    ctm_gh = P.ct_prepare(key, P.encrypt_gh(key, P.encode_gh(g_d, h_d, GH_BITS), P.to_limb_tensor(r[:MFULL])))
    bins = {K: torch.from_numpy(synth.gen_bins_uniform(FFULL, MFULL, K, seed + K)).cuda() for K in (8, 16, 256)}
    node = torch.from_numpy(synth.gen_tree_levels(MFULL, 3, seed)[2]).cuda()
    P.sync()
    return dict(key=key, ctm=ctm, ctm_gh=ctm_gh, bins=bins, node=node, m=m.cpu().numpy().view(np.uint64))


@pytest.fixture(scope="module")
def data():
    return {1024: _dataset(1024, 1), 2048: _dataset(2048, 2), 3072: _dataset(3072, 3)}


REQUESTS = [  # (n_bits, M, F, K, use_node); 3072-bit requests run beside 2048-bit ones (mixed key lengths)
    (1024, 3000, 6, 16, False), (3072, 2000, 5, 16, True), (2048, 1200, 4, 8, False), (1024, 17, 2, 8, True),
    (2048, 3000, 6, 16, True), (3072, 3000, 6, 8, False), (1024, 2500, 5, 16, True), (2048, 1, 1, 8, False),
    (1024, 999, 3, 8, False), (2048, 2047, 6, 16, False), (3072, 1, 1, 8, False),
]


def _submit(srv, data, req):
    nb, M, F, K, use_node = req
    d = data[nb]
    node = d["node"] if use_node else None
    return srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], node=node, num_nodes=4 if use_node else 1,
                      gh_stride=MFULL, bins_stride=MFULL)


def _direct(data, req):
    nb, M, F, K, use_node = req
    d = data[nb]
    ctm = d["ctm"][:, :M].contiguous()
    bins = d["bins"][K][:F, :M].contiguous()
    nn = 4 if use_node else 1
    node = d["node"][:M].contiguous() if use_node else torch.zeros(M, dtype=torch.int32, device="cuda")
    h, c = P.hist_aggregate(d["key"], ctm, bins, node, nn, K)
    s = P.decrypt_u64(d["key"], h.reshape(-1, 2 * d["key"].L))
    P.sync()
    return s.view(nn, F, K, 2).cpu(), c.cpu()


def test_mix_equals_alone_equals_direct(data):
    mix = P.Server(slots=4, hbm_budget=8 << 30)
    tickets = [_submit(mix, data, rq) for rq in REQUESTS]
    got_mix = []
    for t, s, c in tickets:
        st, lat = mix.wait(t)
        assert st == native.REQ_DONE and lat > 0
        got_mix.append((s.clone(), c.clone()))
    stats = mix.stats()
    mix.close()
    assert stats["completed"] == len(REQUESTS) and stats["peak_running"] >= 2
    alone = P.Server(slots=1, hbm_budget=8 << 30)
    for rq, (sm, cm) in zip(REQUESTS, got_mix):
        t, s, c = _submit(alone, data, rq)
        assert alone.wait(t)[0] == native.REQ_DONE
        assert torch.equal(s, sm) and torch.equal(c, cm)
        sd, cd = _direct(data, rq)
        assert torch.equal(s, sd) and torch.equal(c, cd)
    alone.close()


# cells per packed ciphertext: the server's rule (these requests have few cells,
# so it decrypts them directly), short chains, one cell (no packing), as many as fit
PACK_SLOTS = (0, 3, 1, 10_000)


def test_packed_requests_equal_unpacked(data):
    srv = P.Server(slots=3, hbm_budget=8 << 30)
    for rq in REQUESTS[:4]:
        nb, M, F, K, use_node = rq
        d = data[nb]
        node = d["node"] if use_node else None
        nn = 4 if use_node else 1
        kw = dict(node=node, num_nodes=nn, gh_stride=MFULL, bins_stride=MFULL)
        t1, s1, c1 = srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], **kw)
        runs = [srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], pack_bits=40, pack_slots=ps, **kw)
                for ps in PACK_SLOTS]
        most = (nb - 2) // 40
        chosen = [P.Server.request_plan(d["key"], M, F, K, num_nodes=nn, pack_bits=40, pack_slots=ps)[0]
                  for ps in PACK_SLOTS]
        assert chosen == [0, 3, 0, most]
        assert srv.wait(t1)[0] == native.REQ_DONE
        for t2, s2, c2 in runs:
            assert srv.wait(t2)[0] == native.REQ_DONE
            assert torch.equal(s1, s2) and torch.equal(c1, c2)
    srv.close()


def test_automatic_packing_of_larger_requests(data):
    """Requests with enough cells that the server's rule packs them (3,072
    cells: 3 per packed ciphertext at least 1,024 packed ciphertexts), at each
    key size, give the unpacked request's sums."""
    srv = P.Server(slots=4, hbm_budget=8 << 30)
    for nb in (1024, 2048, 3072):
        d = data[nb]
        M, F, K = MFULL, FFULL, 256
        assert P.Server.request_plan(d["key"], M, F, K, pack_bits=40)[0] == 3
        kw = dict(gh_stride=MFULL, bins_stride=MFULL)
        t1, s1, c1 = srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], **kw)
        t2, s2, c2 = srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], pack_bits=40, **kw)
        assert srv.wait(t1)[0] == native.REQ_DONE and srv.wait(t2)[0] == native.REQ_DONE
        assert torch.equal(s1, s2) and torch.equal(c1, c2)
    srv.close()


def test_gh_packed_requests_equal_unpacked(data):
    """Requests over one g/h-packed ciphertext array (half the histogram
    products and decryptions) give the sums of the two-array requests, with
    and without ciphertext packing, mixed with unpacked requests."""
    srv = P.Server(slots=4, hbm_budget=8 << 30)
    for rq in REQUESTS[:4]:
        nb, M, F, K, use_node = rq
        d = data[nb]
        node = d["node"] if use_node else None
        kw = dict(node=node, num_nodes=4 if use_node else 1, bins_stride=MFULL)
        t1, s1, c1 = srv.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], gh_stride=MFULL, **kw)
        t2, s2, c2 = srv.submit(d["key"], d["ctm_gh"], M, F, K, d["bins"][K], gh_bits=GH_BITS, **kw)
        packed = [srv.submit(d["key"], d["ctm_gh"], M, F, K, d["bins"][K], gh_bits=GH_BITS, pack_bits=1,
                             pack_slots=ps, **kw) for ps in PACK_SLOTS]
        for t in (t1, t2):
            assert srv.wait(t)[0] == native.REQ_DONE
        assert torch.equal(s1, s2) and torch.equal(c1, c2)
        for t3, s3, c3 in packed:
            assert srv.wait(t3)[0] == native.REQ_DONE
            assert torch.equal(s1, s3) and torch.equal(c1, c3)
    with pytest.raises(native.PaillierError):
        srv.submit(data[1024]["key"], data[1024]["ctm_gh"], 10, 1, 8, data[1024]["bins"][8], gh_bits=20)
    srv.close()


def test_served_sums_equal_plaintext_histogram(data):
    srv = P.Server(slots=2, hbm_budget=4 << 30)
    rq = (1024, 2500, 5, 16, True)
    t, s, c = _submit(srv, data, rq)
    assert srv.wait(t)[0] == native.REQ_DONE
    d = data[1024]
    m = d["m"]
    node = d["node"].cpu().numpy()[:2500]
    bins = d["bins"][16].cpu().numpy()[:5, :2500]
    sums, counts = oracle.plain_histogram(m[:MFULL][:2500], m[MFULL:][:2500], bins, node, 4, 16)
    assert s.numpy().view(np.uint64).reshape(-1).tolist() == [
        sums[v][f][b][k] for v in range(4) for f in range(5) for b in range(16) for k in range(2)]
    assert c.numpy().reshape(-1).tolist() == [counts[v][f][b] for v in range(4) for f in range(5) for b in range(16)]
    srv.close()


def test_budget_admission_limits_concurrency(data):
    # a budget that fits one request of this size but not two
    big = (1024, 3000, 6, 16, False)
    d = data[1024]
    need = P.Server.request_bytes(d["key"], d["ctm"], 3000, 6, 16, d["bins"][16])
    assert need > 0
    srv = P.Server(slots=4, hbm_budget=need + need // 2)
    ts = [_submit(srv, data, big) for _ in range(3)]
    for t, _, _ in ts:
        assert srv.wait(t)[0] == native.REQ_DONE
    assert srv.stats()["peak_running"] == 1
    srv.close()
    tiny = P.Server(slots=2, hbm_budget=need // 2)
    with pytest.raises(native.PaillierError) as e:
        _submit(tiny, data, big)
    assert e.value.code == native.PL_EBUSY
    tiny.close()


def test_cancel_and_isolated_failure(data):
    srv = P.Server(slots=1, hbm_budget=8 << 30)
    t1, s1, c1 = _submit(srv, data, (2048, 3000, 6, 16, False))
    t2, _, _ = _submit(srv, data, (2048, 3000, 6, 16, False))
    srv.cancel(t2)
    assert srv.poll(t2)[0] == native.REQ_CANCELLED
    # a request whose bins exceed its K fails alone; the next request is unaffected
    d = data[1024]
    t3, _, _ = srv.submit(d["key"], d["ctm"], 500, 3, 8, d["bins"][16], gh_stride=MFULL, bins_stride=MFULL)
    t4, s4, c4 = _submit(srv, data, (1024, 999, 3, 8, False))
    assert srv.wait(t1)[0] == native.REQ_DONE
    st3 = srv.wait(t3)[0]
    assert st3 == native.REQ_FAILED and srv.poll(t3)[2] == native.PL_EDEVICE
    assert srv.wait(t4)[0] == native.REQ_DONE
    sd, cd = _direct(data, (1024, 999, 3, 8, False))
    assert torch.equal(s4, sd) and torch.equal(c4, cd)
    st = srv.stats()
    assert st["failed"] == 1 and st["cancelled"] == 1 and st["completed"] == 2
    srv.close()
    P.sync()  # the library's own status word is untouched by served requests


def test_split_launches_and_priorities_give_the_same_bits(data):
    """The device scheduling policy (launches of bounded work, one stream
    priority per size class) changes when the GPU changes hands, not what is
    computed: with a budget small enough to split every request into one
    launch per feature, packing range and decryption range (2,048 ciphertexts
    at least), requests in all three classes, and every large request moved to
    the medium-priority stream mid-request by aging, every request gives the
    bits of the default policy alone and of the direct API."""
    reqs = REQUESTS + [(1024, 3000, 6, 256, False), (2048, 2500, 5, 256, False), (3072, 2000, 4, 256, False)]
    # promote_ms ~0: every large request moves to the medium stream before its second launch group
    split = P.Server(slots=4, hbm_budget=8 << 30, chunk_imad=1e7, small_imad=2e11, large_imad=2.5e11,
                     promote_ms=1e-6)
    tickets = [_submit(split, data, rq) for rq in reqs]
    nb, M, F, K, use_node = reqs[-2]
    d = data[nb]
    packed = split.submit(d["key"], d["ctm"], M, F, K, d["bins"][K], gh_stride=MFULL, bins_stride=MFULL,
                          pack_bits=40)
    gh = split.submit(d["key"], d["ctm_gh"], M, F, K, d["bins"][K], bins_stride=MFULL, gh_bits=GH_BITS,
                      pack_bits=1)
    got = []
    for t, s_, c_ in tickets + [packed, gh]:
        assert split.wait(t)[0] == native.REQ_DONE
        got.append((s_.clone(), c_.clone()))
    pol = split.policy_stats()
    split.close()
    # every root-only request split into one launch per feature, plus its decryption ranges (two or
    # more where it has over 2,048 cells); some requests ran at high priority, not all
    want_groups = sum((1 if use_node else F_) + -(-2 * F_ * K_ * (4 if use_node else 1) // 2048)
                      for _, _, F_, K_, use_node in reqs)
    cls = pol["per_class"]
    assert pol["launch_groups"] >= want_groups and sum(cls) == len(reqs) + 2 and cls[0] > 0 and cls[2] > 0
    assert pol["promoted"] == cls[2]  # aging moved every large request to the medium stream
    alone = P.Server(slots=1, hbm_budget=8 << 30)
    for rq, (sm, cm) in zip(reqs, got):
        t, s_, c_ = _submit(alone, data, rq)
        assert alone.wait(t)[0] == native.REQ_DONE
        assert torch.equal(s_, sm) and torch.equal(c_, cm)
        sd, cd = _direct(data, rq)
        assert torch.equal(s_, sd) and torch.equal(c_, cd)
    # the packed and g/h-packed requests against their two-array twin
    assert torch.equal(got[-2][0], got[len(reqs) - 2][0]) and torch.equal(got[-1][0], got[len(reqs) - 2][0])
    alone.close()


def test_reserved_slots_hold_back_large_requests_only(data):
    """Admission by size class: with 3 slots and 1 reserved for small
    requests, at most 2 large requests run at once; small requests submitted
    behind queued large ones still complete, with the right bits."""
    srv = P.Server(slots=3, hbm_budget=8 << 30, small_imad=1e9, large_imad=1e9, reserved_slots=1)
    big = (2048, 3000, 6, 16, False)   # modelled work well above 1e9: large
    small = (1024, 17, 2, 8, True)     # below 1e9: small
    ts = [_submit(srv, data, big) for _ in range(5)] + [_submit(srv, data, small) for _ in range(3)]
    for t, _, _ in ts:
        assert srv.wait(t)[0] == native.REQ_DONE
    pol = srv.policy_stats()
    srv.close()
    assert pol["peak_nonsmall"] <= 2 and pol["per_class"] == [3, 0, 5]
    sd, cd = _direct(data, small)
    for t, s_, c_ in ts[5:]:
        assert torch.equal(s_, sd) and torch.equal(c_, cd)
    with pytest.raises(native.PaillierError):
        P.Server(slots=2, hbm_budget=1 << 30, reserved_slots=2)
