"""FP16/BF16 tensor cores past the formats' exact integer range
(CCW_PRECISION_INEXACT), against the oracle's int64 Eq. CCW.

The workload: literal score (Eq. CCW on the facies codes) of a 3-facies TI at
level J = 4, where the operands (code sums of 16 x 16 blocks) reach 512: past
BF16's exact integers (256), within FP16's (2048). Checked per step (one
batch of data events):
  * without the flag BF16 is refused, FP16 is exact;
  * with it, every BF16 score is within the bound the format fixes: both
    operands rounded to nearest (unit roundoff u = 2^-8) give a product within
    2u of the exact one, all products are non-negative, so
    |S~ - S| <= 2^-7 S + 1 (the 1 covers FP32 accumulation and the rounding
    of the score to an integer); the step's maximum relative error is printed;
  * the search's rankings equal the oracle's up to near-ties: mismatch counts
    (exact) agree at every rank, scores within the bound, and where no two of
    the oracle's first K + 1 scores lie within twice the bound the ranked
    candidates and the pick are identical.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INEXACT = 4
F, J, T, OV = 3, 4, 64, 16


@pytest.fixture(scope="module")
def setup():
    import paper_2404_00441_gb300 as ccw
    ccw.load()
    ti = configs.channel_lens_ti_1000()
    g = ccw.TI(torch.from_numpy(ti).cuda(), F, J, T, OV)
    return ccw, ti, g, O.OracleTI(ti, F, J)


def events(ti, n, seed):
    rng = np.random.default_rng(seed)
    return configs.structured_events(ti, T, OV, n, rng, n_hd=3, F=F)


def bound(s):
    return np.ldexp(np.abs(s).astype(np.float64), -7) + 1.0


def test_refused_without_the_flag_and_fp16_exact(setup):
    ccw, ti, g, o = setup
    de, hd = events(ti, 12, 1)
    with pytest.raises(ccw.CCWError):
        ccw.ccf_map(g, torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda(), score_mode=1,
                    precision=2)
    sc, mm = ccw.ccf_map(g, torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda(),
                         score_mode=1, precision=1)
    sc, mm = sc.cpu().numpy(), mm.cpu().numpy()
    for i in range(len(de)):
        ref = o.search(T, de[i], hd[i], K=1, score_mode=1, maps=True)
        assert np.array_equal(sc[i], ref["scores"]) and np.array_equal(mm[i], ref["mis"])


@pytest.mark.parametrize("step", range(3))
def test_bf16_past_the_exact_range_maps_within_the_bound(setup, step):
    ccw, ti, g, o = setup
    de, hd = events(ti, 16, 10 + step)
    sc, mm = ccw.ccf_map(g, torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda(),
                         score_mode=1, precision=2 | INEXACT)
    sc, mm = sc.cpu().numpy().astype(np.int64), mm.cpu().numpy()
    worst = 0.0
    for i in range(len(de)):
        ref = o.search(T, de[i], hd[i], K=1, score_mode=1, maps=True)
        s = ref["scores"]
        assert np.array_equal(mm[i], ref["mis"])               # mismatches stay exact
        assert np.all(np.abs(sc[i] - s) <= bound(s)), i
        if s.max() > 0:
            worst = max(worst, float(np.abs(sc[i] - s).max() / s.max()))
    assert worst <= 2.0 ** -7
    print(f"\nstep {step}: max relative CCF error (BF16 past 256, vs int64 oracle) = {worst:.3e}")


@pytest.mark.parametrize("K", [1, 5])
def test_bf16_past_the_exact_range_rankings_up_to_near_ties(setup, K):
    ccw, ti, g, o = setup
    de, hd = events(ti, 24, 30 + K)
    ctr = torch.from_numpy(np.stack([np.arange(24), np.arange(24) * 7], 1).astype(np.int32)).cuda()
    res = ccw.ccf_search(g, torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda(), k=K,
                         score_mode=1, seed=77, ctr=ctr, precision=2 | INEXACT)
    idx = res["topk_idx"].cpu().numpy()
    mis = res["topk_mis"].cpu().numpy()
    pick = res["pick"].cpu().numpy()
    identical = 0
    for i in range(len(de)):
        ref = o.search(T, de[i], hd[i], K=K + 1, score_mode=1, seed=77, r=i, p=7 * i,
                       maps=True)
        s, m = ref["scores"], ref["mis"]
        ro = ref["topk_idx"]
        n = min(K, len(ro))
        assert np.array_equal(mis[i, :n], m[ro[:n]]), i
        assert np.all(np.abs(s[idx[i, :n]] - s[ro[:n]]) <= 2 * bound(s[ro[:n]])), i
        top = s[ro[:n + 1]]
        close = np.any(np.abs(np.diff(top)) <= 2 * bound(top[1:])) if n + 1 <= len(ro) else False
        if not close:
            assert np.array_equal(idx[i, :n], ro[:n]), i
            assert pick[i] in ro[:n]
            identical += 1
    # with K = 5 most events hold a near-tie among their first six scores
    assert identical >= (len(de) // 4 if K == 1 else 1)
