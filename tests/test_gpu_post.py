"""GPU parity of the post-processing (Sec. V.E) against the oracle, through the C ABI.

Cluster labels, the option-B keep flags and the best cluster are integer outcomes of
FP64 threshold decisions taken on identically ordered expressions: bit-exact.
Centroids and summed significances are FP64 sums in another order: 1e-12 relative.
Candidate parameters decode template ids exactly as the oracle does.
"""
import math

import numpy as np
import pytest

from oracle import postprocess as opp
from paper_1904_04873_gb300 import bsh, synth
from _common import orbit_of
from gpu_common import device_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PPD = dict(T_c=900.0, T_obs=3.15e7, v_over_c=1e-4, P_F=2.0, m_a=1.6, m_Om=1.6, m_t=1.6,
           obliquity=synth.OBLIQUITY, d_cluster=math.sqrt(14.0), d_cut=0.0, d_coinc=3.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1904_04873_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def cloud(n, seed, n_blobs=12, spread=0.6, noise_frac=0.3):
    """Seeded candidate parameters: blobs of a few resolutions' size plus a scattered background."""
    rng = np.random.default_rng(seed)
    p0 = np.array([200.05, 0.3, -0.2, 8.0, 2 * math.pi / (15 * 86400.0), 1.0e5])
    r0 = opp.resolutions(p0[None], PPD)[0]
    centres = p0 + rng.normal(size=(n_blobs, 6)) * r0 * 40.0
    k = rng.integers(n_blobs, size=n)
    p = centres[k] + rng.normal(size=(n, 6)) * r0 * spread
    bg = rng.random(n) < noise_frac
    p[bg] = p0 + rng.normal(size=(bg.sum(), 6)) * r0 * 60.0
    sig = rng.normal(5.0, 2.0, size=n)
    sig[rng.random(n) < 0.05] = -1.0
    valid = (rng.random(n) > 0.05).astype(np.int32)
    return p, sig, valid


def _cluster_gpu(p, sig, valid, **kw):
    pp = bsh.post_params(**{**PPD, **kw})
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    out = bsh.cluster(t(p, torch.float64), t(sig, torch.float64), t(valid, torch.int32), pp)
    assert bsh.sync_status() == bsh.OK
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("n,seed,cut", [(300, 1, 0.0), (2500, 2, 0.0), (2500, 3, 3.0), (4000, 4, 2.0)])
def test_cluster_matches_oracle(n, seed, cut):
    p, sig, valid = cloud(n, seed)
    label, keep, cen, csig, best = _cluster_gpu(p, sig, valid, d_cut=cut)
    ol, ok, oc, ocs, ob = opp.cluster(p, sig, valid.astype(bool), PPD, PPD["d_cluster"], cut)
    assert np.array_equal(label, ol)
    assert np.array_equal(keep, ok)
    roots = np.nonzero(ol == np.arange(n))[0]
    assert roots.size > 5 and roots.size < n
    assert np.allclose(cen[roots], oc[roots], rtol=1e-12, atol=0)
    assert np.allclose(csig[roots], ocs[roots], rtol=1e-12, atol=1e-12)
    others = np.setdiff1d(np.arange(n), roots)
    assert np.isnan(cen[others]).all() and np.all(csig[others] == 0.0)
    assert best[0] == ob


def test_cluster_edge_cases():
    # nothing valid; a single candidate; identical candidates
    p, sig, valid = cloud(50, 5)
    label, keep, cen, csig, best = _cluster_gpu(p, sig, np.zeros(50, np.int32))
    assert np.all(label == -1) and best[0] == -1
    label, keep, cen, csig, best = _cluster_gpu(p[:1], sig[:1], np.ones(1, np.int32))
    assert label[0] == 0 and keep[0] == 1 and best[0] == 0
    assert np.allclose(cen[0], p[0], rtol=1e-15, atol=0)        # (w x) / w, rounded twice
    same = np.repeat(p[:1], 7, axis=0)
    label, keep, cen, csig, best = _cluster_gpu(same, np.full(7, 2.0), np.ones(7, np.int32))
    assert np.all(label == 0) and csig[0] == 14.0


def test_coincidences_match_oracle():
    pa, sa, va = cloud(400, 6)     # same seed: the two lists share their blobs
    pb, sb, vb = cloud(300, 6)
    pp = bsh.post_params(**PPD)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    pairs, cen, sig, n = bsh.coincidences(t(pa, torch.float64), t(sa, torch.float64), t(va, torch.int32),
                                          t(pb, torch.float64), t(sb, torch.float64), t(vb, torch.int32), pp,
                                          cap=20000)
    assert bsh.sync_status() == bsh.OK
    n = int(n.item())
    ref = opp.coincidences(pa[va.astype(bool)], sa[va.astype(bool)], pb[vb.astype(bool)], sb[vb.astype(bool)], PPD,
                           PPD["d_coinc"])
    ia, ib = np.nonzero(va)[0], np.nonzero(vb)[0]
    ref = {(int(ia[i]), int(ib[j])): (c, s) for i, j, c, s in ref}
    assert n == len(ref) and n > 50
    got = pairs[:n].cpu().numpy()
    cen = cen[:n].cpu().numpy()
    sig = sig[:n].cpu().numpy()
    for e, (i, j) in enumerate(got):
        c, s = ref[(int(i), int(j))]
        assert np.allclose(cen[e], c, rtol=1e-14, atol=0) and sig[e] == s


def _cands_array(ids, regions, per_region, n_valid):
    """bsh_cand records with the given template ids (other fields arbitrary)."""
    raw = np.zeros((regions, per_region), dtype=bsh.CAND_DTYPE)
    raw["template_id"] = ids.reshape(regions, per_region)
    raw["s_h"] = np.linspace(9.0, 1.0, regions * per_region).reshape(regions, per_region)
    raw["s_p"] = -raw["s_h"]
    return (torch.as_tensor(raw.view(np.uint8).reshape(regions, per_region, 32), device="cuda"),
            torch.as_tensor(np.asarray(n_valid, np.int32), device="cuda"))


@pytest.mark.parametrize("bank", [False, True])
def test_candidate_parameters(bank):
    pr = synth.eccentric(n_sky=6, n_per_det=60, n_ap=3, n_P=2, n_T=2, n_kap=2, n_eta=1, e_max=0.05, patch_size=3,
                         top_k=20)
    if bank:
        pr = synth.grid_as_bank(pr)
    dp, op, wq = device_problem(pr, "f16")
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=20)
    rng = np.random.default_rng(8)
    regions, per = plan.regions, 20
    ids = np.empty((regions, per), np.int64)
    per_s = pr.B * pr.n_f0
    for r in range(regions):
        s0, s1 = pr.patch_start[r], pr.patch_start[r + 1]
        ids[r] = rng.integers(s0 * per_s, s1 * per_s, size=per)
    n_valid = [per, 13]
    cands, n_c = _cands_array(ids, regions, per, n_valid)
    pp = bsh.post_params(**PPD)
    for stat in (0, 1):
        params, sig, valid = bsh.cand_params(plan, 0, cands, n_c, stat, pp)
        assert bsh.sync_status() == bsh.OK
        params, sig, valid = params.cpu().numpy(), sig.cpu().numpy(), valid.cpu().numpy()
        exp_valid = np.concatenate([np.arange(per) < n_valid[r] for r in range(regions)])
        assert np.array_equal(valid.astype(bool), exp_valid)
        ref = opp.candidate_params(ids.reshape(-1), pr.F0, pr.n_f0, pr.B, 900.0, pr.sky, synth.OBLIQUITY,
                                   lambda b: orbit_of(pr, b)[:3])
        assert np.array_equal(params[exp_valid], ref[exp_valid])
        raw = cands.cpu().numpy().view(bsh.CAND_DTYPE).reshape(-1)
        want = raw["s_p" if stat else "s_h"].astype(np.float64)
        assert np.array_equal(sig[exp_valid], want[exp_valid])
    plan.close()


def test_search_to_best_cluster_recovers_an_injection():
    # tiny search with an injected track: toplist -> parameters -> clusters -> the best
    # cluster's centroid lies within 2 parameter-space bins (Eq. (44)) of the injection
    from _common import inject_on_track
    pr = synth.tiny()
    inj = synth.TINY_INJECTION
    b_inj = (inj["Om_index"] * pr.T_asc.shape[1] + inj["T_index"]) * pr.a_p.size + inj["ap_index"]
    pr.power = inject_on_track(pr, pr.power, inj["sky"], b_inj, inj["f0_index"], inj["excess"])
    dp = bsh.DeviceProblem(pr, w_dtype="f32")
    dp.prepare()
    plan = bsh.Plan([dp], bsh.MODE_BATCHED, top_k=pr.top_k)
    plan.number_count()
    cands, n = plan.toplist()
    final, nf = plan.power_sum(50)
    ppd = dict(PPD, T_obs=30 * synth.DAY, m_a=1.0, m_Om=1.0, m_t=1.0)
    pp = bsh.post_params(**ppd)
    params, sig, valid = bsh.cand_params(plan, 0, final, nf, 1, pp)
    label, keep, cen, csig, best = bsh.cluster(params, sig, valid, pp)
    assert bsh.sync_status() == bsh.OK
    best = int(best.item())
    assert best >= 0
    c = cen[best].cpu().numpy()
    ap, Om, Ta = pr.a_p[inj["ap_index"]], pr.Omega[inj["Om_index"]], pr.T_asc[inj["Om_index"], inj["T_index"]]
    n = pr.sky[inj["sky"]]
    truth = np.array([(pr.F0 + inj["f0_index"]) / 900.0, n[0],
                      math.cos(synth.OBLIQUITY) * n[1] + math.sin(synth.OBLIQUITY) * n[2], ap, Om, Ta])
    rt = opp.resolutions(truth[None], ppd)[0]
    rc = opp.resolutions(c[None], ppd)[0]
    assert math.sqrt(opp.distance2(truth, rt, c, rc)) < 2.0
    plan.close()
