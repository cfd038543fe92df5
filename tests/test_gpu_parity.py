"""GPU parity of every hot-path step against the FP64 oracle, through the C ABI.

Sizes span several SFT chunks, ragged binary tiles, ragged f0 blocks and
ragged last chunks.  Bar: peakgram bits, rho and quantised weights bit-exact; bins and
unweighted counts bit-exact outside the oracle's tie band; weighted counts
and power sums within 1e-5 relative of FP64 on the same quantised weights;
toplists identical except for entries within the score error of the k-th.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_04873_gb300 import bsh, synth
from _common import small_mid
from gpu_common import REL_TOL, check_dense, check_toplists, device_problem, oracle_scores

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_peakgram_median_bit_exact():
    pr = synth.mid(n_sky=4, n_per_det=150, n_ap=2, n_P=2, n_T=2)
    power = torch.as_tensor(pr.power, device="cuda")
    rho, bits = bsh.make_peakgram(power, 101, 1.6, pr.W)
    assert bsh.sync_status() == bsh.OK
    orho, obits = oracle.peakgram(pr.power, 101, 1.6, W=pr.W)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), obits)
    assert np.array_equal(rho.cpu().numpy(), orho)


@pytest.mark.parametrize("K", [90, 101, 333])
def test_peakgram_direct_and_ragged(K):
    rng = np.random.default_rng(K)
    r = (-np.log1p(-rng.random((77, K)))).astype(np.float32)
    W = -(-(-(-K // 32)) // 4) * 4
    rho, bits = bsh.make_peakgram(torch.as_tensor(r, device="cuda"), 0, 1.6, W)
    orho, obits = oracle.peakgram(r, 0, 1.6, W=W)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), obits)
    if K >= 101:
        rho, bits = bsh.make_peakgram(torch.as_tensor(r, device="cuda"), 101, 1.6, W)
        orho, obits = oracle.peakgram(r, 101, 1.6, W=W)
        assert np.array_equal(bits.cpu().numpy().view(np.uint32), obits)
        assert np.array_equal(rho.cpu().numpy(), orho)


@pytest.mark.parametrize("window,K", [(3, 3), (7, 70), (31, 64), (101, 101), (101, 164), (101, 230),
                                      (201, 2000), (63, 127)])
@pytest.mark.parametrize("ties", [False, True])
def test_peakgram_sliding_median(window, K, ties):
    # the sliding running median (one segment of 63 bins per thread, the median moving to its
    # successor or predecessor as the window slides) against the oracle's sort per bin: window
    # sizes from 3 up, rows that end inside the first and second segments, and rows of small
    # integers whose windows hold many equal values
    rng = np.random.default_rng(1000 * window + K)
    if ties:
        r = rng.integers(0, 6, size=(41, K)).astype(np.float32) + 0.5
    else:
        r = (-np.log1p(-rng.random((41, K)))).astype(np.float32)
    W = -(-(-(-K // 32)) // 4) * 4
    rho, bits = bsh.make_peakgram(torch.as_tensor(r, device="cuda"), window, 1.6, W)
    assert bsh.sync_status() == bsh.OK
    orho, obits = oracle.peakgram(r, window, 1.6, W=W)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), obits)
    assert np.array_equal(rho.cpu().numpy(), orho)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("n_per_det", [300, 2500])
def test_weights(dtype, n_per_det):
    # both sides evaluate Eq. (22) in the same order (explicit wave-frame basis, every
    # operation rounded on its own, the normalisation sum over SFTs in ascending order), so
    # the stored weights are identical, not merely close; 2 x 2500 SFTs span two tiles of
    # the kernel's sequential sum.  Includes a sky point on the pole (the basis' special case)
    pr = synth.mid(n_sky=37, n_per_det=n_per_det, n_ap=2, n_P=2, n_T=2)
    skyv = pr.sky.copy()
    skyv[0] = [0.0, 0.0, 1.0]
    skyv[1] = [0.0, 0.0, -1.0]
    sky = torch.as_tensor(skyv, device="cuda")
    arms = torch.as_tensor(pr.arms, device="cuda")
    Sn = torch.as_tensor(pr.Sn, device="cuda")
    w, sw, sw2 = bsh.weights(sky, arms, Sn, True, dtype)
    assert bsh.sync_status() == bsh.OK
    oq = oracle.quantize(oracle.weights(skyv, pr.arms, pr.Sn, norm=True), dtype)
    gw = w.double().cpu().numpy()
    assert np.array_equal(gw, oq), f"{int((gw != oq).sum())} weights differ"
    assert np.allclose(sw.cpu().numpy(), gw.sum(axis=1), rtol=1e-12)
    assert np.allclose(sw2.cpu().numpy(), (gw * gw).sum(axis=1), rtol=1e-12)
    assert np.allclose(sw.cpu().numpy(), pr.N, rtol=1e-2)
    # unnormalised weights as well
    w, _, _ = bsh.weights(sky, arms, Sn, False, dtype)
    oq = oracle.quantize(oracle.weights(skyv, pr.arms, pr.Sn, norm=False), dtype)
    assert np.array_equal(w.double().cpu().numpy(), oq)


@pytest.fixture(scope="module")
def mid_small():
    # 6 sky points in 2 patches, 300 SFTs (3 chunks, ragged), 36 binaries (ragged tile),
    # 90 f0 templates (3 blocks of 30)
    pr = small_mid(n_sky=6, n_per_det=150, n_ap=4, n_P=3, n_T=3, patch_size=3, top_k=40)
    return pr


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32", "f64"])
def test_count_dense_batched(mid_small, dtype):
    pr = mid_small
    dp, op, wq = device_problem(pr, dtype)
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d = op.count_dense()
    check_dense(gu[0], gw[0], d)
    plan.close()


@pytest.mark.parametrize("threads,chunk,acc,direct", [(128, 64, 0, 1), (256, 256, 0, 1), (256, 64, 0, 0),
                                                      (128, 256, 1, 0), (256, 64, 1, 0), (256, 128, 1, 0),
                                                      (256, 128, 2, 0), (256, 64, 2, 1), (256, 256, 2, 0)])
def test_count_dense_tile_shapes(mid_small, threads, chunk, acc, direct):
    # every accumulation variant and both ways of forming the binary term (the byte-table
    # accumulation exists only with the per-warp term; the tensor-core one with 256 threads)
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k, threads=threads, sft_chunk=chunk)
    plan.set_direct(direct)
    plan.set_accumulate(acc)
    t = plan.tile()
    assert t["threads"] == threads and t["accumulate"] == acc and t["direct"] == direct
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.close()


def test_per_term_plans_keep_predicated_adds(mid_small):
    pr = mid_small
    dp, _, _ = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    assert plan.set_direct(1) == 1
    plan.set_accumulate(1)
    assert plan.tile()["accumulate"] == 0
    plan.set_direct(0)
    plan.set_accumulate(1)
    assert plan.tile()["accumulate"] == 1 and plan.tile()["direct"] == 0
    plan.close()


def test_autotune_keeps_parity(mid_small):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    tile = plan.autotune()
    assert tile["threads"] in (128, 256) and tile["sft_chunk"] in (32, 64, 128, 256)
    assert tile["accumulate"] in (0, 1)
    assert bsh.sync_status() == bsh.OK
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense())
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


def test_count_dense_plain_is_fp64_exact(mid_small):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f64")
    plan = bsh.Plan([dp], bsh.MODE_PLAIN, top_k=pr.top_k)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    check_dense(gu[0], gw[0], op.count_dense(), exact_w=True)
    plan.close()


@pytest.mark.parametrize("mode", [bsh.MODE_BATCHED, bsh.MODE_PLAIN])
def test_toplist_matches_full_sort(mid_small, mode):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16" if mode == bsh.MODE_BATCHED else "f64")
    plan = bsh.Plan([dp], mode, top_k=pr.top_k)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, pr.top_k, tol=2e-4)
    plan.close()


def test_toplist_large_k_multiple_selects():
    # k small relative to the items so the per-CTA selection runs many times
    pr = small_mid(n_sky=12, n_per_det=64, n_ap=8, n_P=4, n_T=4, patch_size=4, top_k=7)
    dp, op, wq = device_problem(pr, "f32")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=7)
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    _, sc = oracle_scores(op, wq)
    by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
    check_toplists(plan, dp, 0, by_patch, 7, tol=2e-4)


def test_power_sum_and_rerank(mid_small):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(10)
    assert bsh.sync_status() == bsh.OK
    lists = bsh.cands_to_numpy(cands, n)
    per_s = pr.B * pr.n_f0
    for r, g in enumerate(lists):
        for c in g:
            s, rem = divmod(int(c["template_id"]), per_s)
            b, j = divmod(rem, pr.n_f0)
            P = op.power_sum(s, b, j)
            assert abs(c["power"] - P) <= REL_TOL * P
            sP = oracle.power_significance(P, wq[s].sum(), (wq[s] ** 2).sum())
            assert abs(c["s_p"] - sP) < 1e-4
    finals = bsh.cands_to_numpy(final, nf)
    for r, f in enumerate(finals):
        assert f.size == min(10, lists[r].size)
        ref = np.sort(lists[r]["s_p"])[::-1][:10]
        assert np.array_equal(np.sort(f["s_p"])[::-1], ref)
        assert np.all(np.diff(f["s_p"]) <= 0)


def test_injection_ranks_first():
    from _common import inject_on_track, oracle_inputs
    pr = synth.tiny()
    inj = synth.TINY_INJECTION
    b_inj = (inj["Om_index"] * pr.T_asc.shape[1] + inj["T_index"]) * pr.a_p.size + inj["ap_index"]
    pr.power = inject_on_track(pr, pr.power, inj["sky"], b_inj, inj["f0_index"], inj["excess"])
    dp = bsh.DeviceProblem(pr, w_dtype="f64")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    cands, n = plan.toplist()
    assert bsh.sync_status() == bsh.OK
    top = bsh.cands_to_numpy(cands, n)[0]
    assert top[0]["template_id"] == (inj["sky"] * pr.B + b_inj) * pr.n_f0 + inj["f0_index"]
    assert top[0]["n_unw"] == pr.N


def test_multi_problem_batch():
    probs = synth.batching(n_patch=3, size_lo=2, size_hi=4, n_per_det=70, n_bin=3)
    for p in probs:
        p.n_f0 = 40
    dps = [device_problem(p, "f16") for p in probs]
    plan = bsh.Plan([d[0] for d in dps], bsh.MODE_BATCHED, top_k=15)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        check_dense(gu[q], gw[q], op.count_dense())
    plan.number_count()
    assert bsh.sync_status() == bsh.OK
    for q, (dp, op, wq) in enumerate(dps):
        _, sc = oracle_scores(op, wq)
        pr = dp.pr
        by_patch = [sc[pr.patch_start[p]:pr.patch_start[p + 1]] for p in range(len(pr.patch_start) - 1)]
        check_toplists(plan, dp, q, by_patch, 15, tol=2e-4)


def test_forced_exact_ties():
    pr = synth.precision_stress(n_sky=4, n_per_det=100, n_ap=4, n_P=3, n_T=3)
    dp, op, wq = device_problem(pr, "f32")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=10)
    gu, gw = plan.count_dense()
    assert bsh.sync_status() == bsh.OK
    d = op.count_dense()
    # exact ties are decided identically (x + 1/2 is an exact integer): compare everything
    assert np.array_equal(gu[0].cpu().numpy()[0, ::4], d["n_unw"][0, ::4])
    check_dense(gu[0], gw[0], d)


def test_device_detects_understated_velocity_bound(mid_small):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16")
    dp.v_max *= 0.5
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    assert bsh.sync_status() == bsh.ERR_RANGE
    assert bsh.sync_status() == bsh.OK


def test_graph_replay_matches_eager(mid_small):
    pr = mid_small
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    c1, n1 = plan.toplist()
    f1, nf1 = plan.power_sum(8)
    ref = (c1.clone(), n1.clone(), f1.clone(), nf1.clone())
    for _ in range(3):
        f2, nf2 = plan.graph_launch(8)
    assert bsh.sync_status() == bsh.OK
    assert torch.equal(plan.cands, ref[0]) and torch.equal(plan.n_cands, ref[1])
    assert torch.equal(f2, ref[2]) and torch.equal(nf2, ref[3])
