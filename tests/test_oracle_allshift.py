"""Pins of the oracle's all-shift (polyphase) candidate option: every fine
origin of the training image is a candidate, instead of the multiples of
s = 2^J that the decimated level-J grid keeps (Sec. 3.2, 4.3). CPU only."""
import numpy as np
import pytest
from scipy import signal

from oracle import oracle as O
from workloads import synth


def _event(rng, T, d, F, p_known=0.5):
    de = rng.integers(0, F, size=(T,) * d).astype(np.uint8)
    de[rng.random((T,) * d) >= p_known] = O.UNKNOWN
    return de


def _block_sums(x, s):
    """Closed form of the scaled-Haar approximation: sums over s^d blocks."""
    if x.ndim == 2:
        ny, nx = x.shape
        return x.reshape(ny // s, s, nx // s, s).sum(axis=(1, 3))
    nz, ny, nx = x.shape
    return x.reshape(nz // s, s, ny // s, s, nx // s, s).sum(axis=(1, 3, 5))


@pytest.mark.parametrize("shape,J,T", [((30, 34), 1, 8), ((36, 40), 2, 8), ((14, 16, 18), 1, 4)])
@pytest.mark.parametrize("score_mode", [0, 1])
def test_allshift_score_map_equals_library_correlation(shape, J, T, score_mode):
    """The score of the window at every fine origin c is
    sum_f sum_q I_f(c + q) b_f(floor(q / s)): a 'valid' correlation of each
    indicator (or of the codes) with the data event's block sums expanded
    to fine cells (np.kron with a block of ones)."""
    F, s, d = 3, 2 ** J, len(shape)
    rng = np.random.default_rng(J + 3 * d + score_mode)
    ti = synth.random_field_ti(shape, F, seed=11 + J)
    t = O.OracleTI(ti, F, J)
    de = _event(rng, T, d, F)
    res = t.search(T, de, K=3, maps=True, all_shift=True, score_mode=score_mode)
    ones = np.ones((s,) * d, np.int64)
    chans = range(F) if score_mode == 0 else [None]
    ref = 0
    for f in chans:
        if f is None:
            img, ev = ti.astype(np.int64), np.where(de == O.UNKNOWN, 0, de).astype(np.int64)
        else:
            img, ev = (ti == f).astype(np.int64), (de == f).astype(np.int64)
        w = np.kron(_block_sums(ev, s), ones)
        ref = ref + signal.correlate(img, w, mode="valid", method="direct")
    assert res["scores"].shape[0] == ref.size
    np.testing.assert_array_equal(res["scores"], ref.ravel())


@pytest.mark.parametrize("d", [2, 3])
def test_level0_allshift_is_the_decimated_search(d):
    """At J = 0 every fine origin is already a level-0 candidate."""
    shape = (24, 26) if d == 2 else (12, 14, 10)
    rng = np.random.default_rng(d)
    ti = synth.random_field_ti(shape, 3, seed=4)
    t = O.OracleTI(ti, 3, 0)
    T = 6 if d == 2 else 4
    de = _event(rng, T, d, 3)
    hd = np.where(rng.random((T,) * d) < 0.2, rng.integers(0, 3, (T,) * d),
                  O.UNKNOWN).astype(np.uint8)
    a = t.search(T, de, hd=hd, K=5, maps=True, seed=3, r=1, p=2)
    b = t.search(T, de, hd=hd, K=5, maps=True, seed=3, r=1, p=2, all_shift=True)
    for k in ("scores", "mis", "topk_idx", "topk_score", "topk_mis"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["pick"] == b["pick"]


def test_phase_zero_candidates_are_the_decimated_ones():
    """The all-shift candidates at multiples of s are the decimated
    candidates, with the same scores and mismatches."""
    J, T, s = 2, 16, 4
    rng = np.random.default_rng(9)
    ti = synth.random_field_ti((64, 56), 3, seed=5)
    t = O.OracleTI(ti, 3, J)
    de = _event(rng, T, 2, 3)
    hd = np.where(rng.random((T, T)) < 0.1, rng.integers(0, 3, (T, T)), O.UNKNOWN).astype(np.uint8)
    dec = t.search(T, de, hd=hd, K=2, maps=True)
    alls = t.search(T, de, hd=hd, K=2, maps=True, all_shift=True)
    cy, cx = t.cand_shape(T)
    fy, fx = ti.shape[0] - T + 1, ti.shape[1] - T + 1
    sc = alls["scores"].reshape(fy, fx)[::s, ::s][:cy, :cx]
    mm = alls["mis"].reshape(fy, fx)[::s, ::s][:cy, :cx]
    np.testing.assert_array_equal(sc.ravel(), dec["scores"])
    np.testing.assert_array_equal(mm.ravel(), dec["mis"])


def test_allshift_mismatch_topk_and_pick():
    """Mismatches are the brute-force hard-data disagreements at every fine
    origin; the top-K and the pick follow a full sort of the maps by the key
    (mismatches, -score, index) and the Philox draw of the header."""
    rng = np.random.default_rng(12)
    ti = synth.random_field_ti((40, 36), 3, seed=6)
    t = O.OracleTI(ti, 3, 1)
    T, K = 8, 6
    de = _event(rng, T, 2, 3)
    hd = np.where(rng.random((T, T)) < 0.15, rng.integers(0, 3, (T, T)), O.UNKNOWN).astype(np.uint8)
    res = t.search(T, de, hd=hd, K=K, maps=True, all_shift=True, seed=5, r=2, p=7)
    fy, fx = ti.shape[0] - T + 1, ti.shape[1] - T + 1
    mis = np.zeros((fy, fx), np.int64)
    for y in range(fy):
        for x in range(fx):
            win = ti[y:y + T, x:x + T]
            mis[y, x] = np.sum((hd != O.UNKNOWN) & (win != hd))
    np.testing.assert_array_equal(res["mis"], mis.ravel())
    order = np.lexsort((np.arange(fx * fy), -res["scores"], res["mis"]))
    np.testing.assert_array_equal(res["topk_idx"], order[:K])
    u = int(O.philox4x32_10([2, 7, 0, 0], [5, 0])[0])
    assert res["pick"] == order[(u * K) >> 32]


@pytest.mark.parametrize("path_random", [0, 1])
def test_allshift_simulation_pastes_ti_crops(path_random):
    """With all-shift candidates the first patch is the TI crop at its fine
    pick origin (its unshared core survives), and hard data are honoured."""
    ti = synth.ribbon_ti(90, 84, n_ribbons=5, seed=4, target=0.3, tol=0.2)
    T, Ov, J = 16, 4, 1
    t = O.OracleTI(ti, 2, J)
    grid = (40, 28)                      # T + k (T - OR): no padding
    fx = 90 - T + 1
    for r in range(4):
        out, log = t.simulate(grid, T, Ov, K=3, path_random=path_random, seed=8, r=r,
                              all_shift=1)
        c = int(log[0, 0])
        crop = ti[c // fx:c // fx + T, c % fx:c % fx + T]
        flips = O.path_flips(2, 8, r, path_random)
        ys = range(Ov, T) if flips & 2 else range(0, T - Ov)
        xs = range(Ov, T) if flips & 1 else range(0, T - Ov)
        oy = grid[1] - T if flips & 2 else 0
        ox = grid[0] - T if flips & 1 else 0
        for y in ys:
            for x in xs:
                assert out[oy + y, ox + x] == crop[y, x]
    field = synth.ribbon_ti(40, 28, n_ribbons=3, seed=9, target=0.3, tol=0.3)
    cells, vals = synth.sample_hard_data(field, 25, seed=3)
    out, _ = t.simulate(grid, T, Ov, K=3, hd_cells=cells, hd_vals=vals, seed=2, all_shift=1)
    assert np.array_equal(out[cells[:, 1], cells[:, 0]], vals)
