"""Host-side logic on the CPU: gap calibration of the learned proposal, the
autotuner's candidate tilings, the lattice helper of the binding, and the
pattern statistics used to compare ensembles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_calibrate_gap_meets_the_target_miss_rate():
    from paper_2404_00441_gb300.proposal import calibrate_gap
    rng = np.random.default_rng(0)
    n = 5000
    gap = rng.random(n)
    # misses concentrate at small gaps
    hit = rng.random(n) < np.clip(gap * 4, 0, 1)
    gap[:50] = -1.0   # no proposals
    g, h = torch.from_numpy(gap), torch.from_numpy(hit)
    for target in (0.01, 0.05, 0.2):
        th = calibrate_gap(h, g, target)
        sel = gap >= th
        assert np.mean(~hit[sel]) <= target + 1e-12
        # the next smaller gap would break the target (theta is the smallest)
        smaller = np.sort(gap[(gap >= 0) & (gap < th)])
        if smaller.size:
            sel2 = gap >= smaller[-1]
            assert np.mean(~hit[sel2]) > target
    assert calibrate_gap(torch.zeros(3, dtype=torch.bool), torch.full((3,), -1.0), 0.1) == float("inf")
    assert calibrate_gap(torch.zeros(3, dtype=torch.bool), torch.ones(3), 0.0) == float("inf")


def test_autotune_candidates_respect_the_documented_tilings():
    from paper_2404_00441_gb300 import autotune

    class T2:
        ndim = 2

    class T3:
        ndim = 3

    c2 = autotune.candidates(T2(), (0, 1, 2))
    c3 = autotune.candidates(T3(), (0, 1, 2))
    assert {t for p, t in c2 if p == 0} == {1, 2, 4, 8}
    assert {t for p, t in c3 if p == 0} == {1, 2, 4}
    for cands, ndim in ((c2, 2), (c3, 3)):
        for p, t in cands:
            if p == 0:
                continue
            nt, mt, fl = t & 0xFFFF, (t >> 16) & 0xFF, t >> 24
            assert nt in (16, 32, 64, 128) and 1 <= mt <= 4 and mt * nt <= 512
            assert fl <= 63 and ((fl >> 3) & 3) != 3 and not (fl & 32 and fl & 4)
            if ndim == 3:
                assert fl & 2   # streamed operands only in 3D
    assert len(set(c2)) == len(c2) and len(set(c3)) == len(c3)


def test_lattice_helper_matches_the_oracle():
    from oracle import oracle as O
    from paper_2404_00441_gb300 import ccw
    for grid, T, Ov in (((250, 250), 40, 10), ((2000, 2000), 64, 16), ((30, 22), 40, 10),
                        ((200, 200, 100), 24, 6), ((512, 512), 48, 12)):
        n, gp = ccw.lattice(grid, T, Ov)
        rn, rgp = O.lattice(len(grid), grid, T, Ov)
        assert tuple(n) == tuple(rn[:len(grid)]) and tuple(gp) == tuple(rgp[:len(grid)])


def test_pattern_statistics_basic_properties():
    from workloads import stats
    rng = np.random.default_rng(1)
    a = (rng.random((40, 50)) < 0.3).astype(np.uint8)
    b = (rng.random((40, 50)) < 0.6).astype(np.uint8)
    ha, hb = stats.pattern_histogram(a, 2), stats.pattern_histogram(b, 2)
    assert stats.js_divergence(ha, ha) == 0.0
    assert abs(stats.js_divergence(ha, hb) - stats.js_divergence(hb, ha)) < 1e-15
    assert 0.0 < stats.js_divergence(ha, hb) <= 1.0
    assert sum(ha.values()) == (40 - 3) * (50 - 3)
    # mode downsampling: ties go to the lower code
    blk = np.array([[0, 1], [1, 0]], np.uint8)
    assert stats.mode_downsample(blk, 2, 2)[0, 0] == 0
    # variogram of a constant field is zero, of a checkerboard 1 at odd lags
    assert np.all(stats.indicator_variogram(np.ones((8, 8), np.uint8), 1, 1, (1, 2)) == 0)
    cb = (np.indices((8, 8)).sum(0) % 2).astype(np.uint8)
    assert np.allclose(stats.indicator_variogram(cb, 1, 1, (1, 2, 3)), [0.5, 0.0, 0.5])
