"""GPU pattern-reproduction statistics (ccw_eval_*) against the numpy
definitions of workloads/stats.py: exact counts, exact variogram ratios."""
import numpy as np
import pytest

from workloads import configs, stats, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ev():
    import paper_2404_00441_gb300 as m
    m.load()
    from paper_2404_00441_gb300 import evaluate
    return evaluate


def test_proportions_and_variograms_match_numpy(ev):
    rng = np.random.default_rng(0)
    reals = np.stack([synth.channel_lens_ti(130, 97, seed=s, tol=0.3) for s in (1, 2, 3)])
    reals[1, :5, :7] = 2
    t = torch.from_numpy(reals).cuda()
    p = ev.proportions(t, 3).cpu().numpy()
    for i in range(3):
        assert np.array_equal(p[i], stats.proportions(reals[i], 3))
    lags = (1, 2, 5, 17, 96, 200)
    for axis, np_axis in ((0, 1), (1, 0)):
        for f in (0, 1, 2):
            g = ev.variogram(t, f, axis, lags).cpu().numpy()
            for i in range(3):
                ok = [h for h in lags if h < reals.shape[2 - axis]]
                ref = stats.indicator_variogram(reals[i], f, np_axis, ok)
                assert np.allclose(g[i][:len(ok)], ref, rtol=1e-13, atol=0)
    # 3D along z
    cube = (rng.random((2, 9, 11, 13)) < 0.4).astype(np.uint8)
    g = ev.variogram(torch.from_numpy(cube).cuda(), 1, 2, (1, 3)).cpu().numpy()
    for i in range(2):
        for j, h in enumerate((1, 3)):
            d = (cube[i, h:] == 1).astype(int) - (cube[i, :-h] == 1).astype(int)
            assert abs(g[i, j] - 0.5 * np.mean(d * d)) < 1e-13


@pytest.mark.parametrize("down", [1, 2, 4])
def test_pattern_histograms_match_numpy(ev, down):
    ti = configs.ribbon_ti_250()
    reals = np.stack([ti[:200, :180], ti[50:250, 70:250]])
    h = ev.pattern_histogram(torch.from_numpy(np.ascontiguousarray(reals)).cuda(), 2, w=4,
                             down=down).cpu().numpy()
    ref = stats.ensemble_histogram(list(reals), 2, k=down, w=4)
    dense = np.zeros_like(h)
    for code, c in ref.items():
        dense[code] = c
    assert np.array_equal(h, dense)
    # the divergence of a histogram with itself is 0, and matches numpy otherwise
    h2 = ev.pattern_histogram(torch.from_numpy(np.ascontiguousarray(reals[:1])).cuda(), 2, w=4,
                              down=down)
    assert ev.js_divergence(torch.from_numpy(h), torch.from_numpy(h)) == 0.0
    ref2 = stats.ensemble_histogram(list(reals[:1]), 2, k=down, w=4)
    assert abs(ev.js_divergence(torch.from_numpy(h), h2) - stats.js_divergence(ref, ref2)) < 1e-12


def _pairs_by_flood_fill(real, f, lags, axis):
    """Host counts from a 4-connected labelling (scipy.ndimage.label):
    (pairs of facies f at lag h along the axis, pairs in one component)."""
    from scipy import ndimage
    lab, _ = ndimage.label(real == f)
    out = []
    for h in lags:
        a, b = (lab[:, :-h], lab[:, h:]) if axis == 0 else (lab[:-h, :], lab[h:, :])
        both = (a > 0) & (b > 0)
        out.append((int(both.sum()), int((both & (a == b)).sum())))
    return np.array(out, np.int64)


@pytest.mark.parametrize("kind", ["ribbons", "random", "spiral"])
def test_connection_probability_matches_flood_fill(ev, kind):
    """The GPU probability of connection (union-find labelling, Sec. 5.3)
    gives exactly the pair counts of a breadth-first labelling, on channel
    layouts, percolation-like random fields and a long spiral (one component
    whose union-find chains are long)."""
    rng = np.random.default_rng(3)
    if kind == "ribbons":
        reals = np.stack([synth.ribbon_ti(180, 150, n_ribbons=8, seed=s, target=0.3, tol=0.2)
                          for s in (1, 2, 3)])
    elif kind == "random":
        reals = (rng.random((4, 97, 131)) < 0.55).astype(np.uint8)
    else:
        n = 121
        sp = np.zeros((n, n), np.uint8)
        lo, hi = 0, n - 1
        while lo <= hi:   # square spiral of width-1 corridors
            sp[lo, lo:hi + 1] = 1
            sp[lo:hi + 1, hi] = 1
            if lo + 2 <= hi:
                sp[hi, lo + 2:hi + 1] = 1
                sp[lo + 2:hi + 1, lo + 2] = 1
                sp[lo + 2, lo + 2:lo + 4] = 1
            lo += 4
            hi -= 4
        reals = np.stack([sp, 1 - sp])
    lags = (1, 2, 3, 8, 25, 64)
    t = torch.from_numpy(np.ascontiguousarray(reals)).cuda()
    for f in (0, 1):
        for axis in (0, 1):
            got = ev.connectivity_counts(t, f, lags, axis).cpu().numpy()
            for i in range(len(reals)):
                assert np.array_equal(got[i], _pairs_by_flood_fill(reals[i], f, lags, axis)), (
                    f, axis, i)
    # the probability equals the numpy definition (stats, axis 1 = x there)
    p = ev.connection_probability(t, 1, lags, 0)
    for i in range(len(reals)):
        ref = stats.connection_probability(reals[i], 1, lags, axis=1)
        assert np.allclose(p[i], ref, equal_nan=True, rtol=0, atol=0)
