"""The bounds-checked library (build.py --checked: device-side checks on every
gathered sample id, chunk partial, sorted position, window-table entry, CKKS
cluster exchange and slot permutation) runs the main paths (encryption as one
launch at 1024-bit and as two at 2048-bit) without a single failed check, and
gives the same integers as the normal library.  It stands
in for compute-sanitizer, which this pool does not offer."""

import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2504_03909_b300 import native

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _workload() -> dict:
    """Paillier level with ragged nodes (batched and per-node), packing, g/h
    packing; CKKS through clusters and through one CTA per polynomial."""
    from paper_2504_03909_b300 import ckks as G, paillier as P, synth

    out = {}
    n_bits, M, F, K, nodes = 1024, 2000, 6, 16, 4
    p, q = synth.gen_primes(n_bits, 21)
    key = P.Key.from_primes(n_bits, p, q)
    gh = synth.gen_gh(M, 21)
    r = synth.gen_r(p * q, n_bits, 2 * M, 21, p, q)
    bins = torch.from_numpy(synth.gen_bins_uniform(F, M, K, 21)).cuda()
    node = torch.from_numpy(synth.rng_misc(21).integers(-1, nodes, size=M).astype(np.int32)).cuda()
    ct = P.encrypt(key, P.encode(torch.from_numpy(gh.reshape(-1)).cuda()), P.to_limb_tensor(r))
    ctm = P.ct_prepare(key, ct.view(2, M, -1))
    hist, cnt = P.hist_aggregate(key, ctm, bins, node, nodes, K)
    hist_pn, _ = P.hist_aggregate(key, ctm, bins, node, nodes, K, per_node=True)
    cells = hist.reshape(-1, 2 * key.L)
    out.update(ct=ct, hist=hist, hist_pn=hist_pn, cnt=cnt, sums=P.decrypt_u64(key, cells),
               packed_sums=P.decrypt_packed_u64(key, P.pack(key, cells, 40), cells.shape[0], 40))
    B = 38
    g_d, h_d = torch.from_numpy(gh[0].copy()).cuda(), torch.from_numpy(gh[1].copy()).cuda()
    ct1 = P.encrypt_gh(key, P.encode_gh(g_d, h_d, B), P.to_limb_tensor(r[:M]))
    h1, _ = P.hist_aggregate_gh(key, P.ct_prepare(key, ct1), bins, node, nodes, K)
    out.update(ct_gh=ct1, sums_gh=P.decrypt_gh(key, h1.reshape(-1, 2 * key.L), B))

    # 2048-bit encryption large enough to take the two-launch path (first stage
    # at 2 lanes, second at 4)
    p2, q2 = synth.gen_primes(2048, 22)
    key2 = P.Key.from_primes(2048, p2, q2)
    M2 = 4000
    m2 = P.encode(torch.from_numpy(synth.gen_gh(M2 // 2, 22).reshape(-1)).cuda())
    out.update(ct2048=P.encrypt(key2, m2, P.to_limb_tensor(synth.gen_r(p2 * q2, 2048, M2, 22, p2, q2))))

    log_n = 10
    N, qc = 1 << log_n, synth.ckks_prime(log_n)
    ctx = G.Context(log_n, qc, 2.0 ** 40)
    s_, a_, e_ = synth.ckks_secret(N, 4), synth.ckks_uniform(N, qc, 4), synth.ckks_gaussian(N, 4, 1)
    s_d, a_d = torch.from_numpy(s_).cuda(), torch.from_numpy(a_.view(np.int64)).cuda()
    b_d = ctx.keygen(s_d, a_d, torch.from_numpy(e_).cuda())
    z = synth.rng_misc(6).normal(size=(2, 3, N // 2)) * 100
    rnd = [torch.from_numpy(x).cuda() for x in (synth.ckks_ternary((3, N), 4, 2), synth.ckks_gaussian((3, N), 4, 3),
                                                synth.ckks_gaussian((3, N), 4, 4))]
    for tag, limit in (("cl", 64), ("one", 0)):
        ctx.set_cluster_limit(limit)
        msg = ctx.encode(torch.from_numpy(z[0].copy()).cuda(), torch.from_numpy(z[1].copy()).cuda())
        c = ctx.encrypt(b_d, a_d, msg, *rnd)
        d = ctx.decrypt(ctx.sum([c, c]), s_d)
        zr, zi = ctx.decode(d)
        out.update({f"ckks_msg_{tag}": msg, f"ckks_ct_{tag}": c, f"ckks_dec_{tag}": d, f"ckks_zr_{tag}": zr,
                    f"ckks_zi_{tag}": zi})
    P.sync()  # raises PL_EDEVICE in the checked build if any check failed
    return {k: v.cpu().numpy() for k, v in out.items()}


def _run_to(path: str) -> None:
    np.savez(path, **_workload())


def _report_chain() -> None:
    """In the checked build: a report at site 3 surfaces once at paillier_sync."""
    from paper_2504_03909_b300 import paillier as P
    native.call("paillier_test_bounds_report", 3, torch.cuda.current_stream().cuda_stream)
    try:
        P.sync()
    except native.PaillierError as e:
        assert e.code == native.PL_EDEVICE and "0x8" in str(e), str(e)
    else:
        raise AssertionError("the report did not reach paillier_sync")
    P.sync()  # cleared


def test_checked_build_runs_clean_and_matches(tmp_path):
    lib = os.path.join(ROOT, "paper_2504_03909_b300", "libpaillier_b300_checked.so")
    if not os.path.exists(lib):
        pytest.skip("checked library not built (python -m paper_2504_03909_b300.build --checked)")
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, PAILLIER_B300_LIB="checked", PYTHONPATH=os.pathsep.join([ROOT, HERE]))
    code = ("import sys, test_gpu_checked as t; from paper_2504_03909_b300 import native; "
            "assert native.LIB_PATH.endswith('_checked.so'); t._run_to(sys.argv[1]); t._report_chain()")
    res = subprocess.run([sys.executable, "-c", code, path], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    checked = dict(np.load(path))
    assert not native.LIB_PATH.endswith("_checked.so")
    normal = _workload()
    for k, v in normal.items():
        if v.dtype.kind == "f":
            assert np.allclose(checked[k], v, rtol=0, atol=1e-6 * max(1.0, np.abs(v).max())), k
        else:
            assert np.array_equal(checked[k], v), k
    assert np.array_equal(normal["hist"], normal["hist_pn"])
    assert np.array_equal(normal["ckks_ct_cl"], normal["ckks_ct_one"])
    # the normal build has no report path
    with pytest.raises(native.PaillierError):
        native.call("paillier_test_bounds_report", 3, torch.cuda.current_stream().cuda_stream)
