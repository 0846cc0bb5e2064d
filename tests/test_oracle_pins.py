"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names the passage of the paper, or the piece of mathematics, that
fixes the expected value. They run on the CPU only.
"""
import os

import numpy as np
import pytest
from scipy import signal

from oracle import oracle as O
from workloads import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def block_sum(x, s):
    """Closed form of the scaled-Haar approximation: sums over s^d blocks."""
    if x.ndim == 2:
        ny, nx = x.shape
        return x.reshape(ny // s, s, nx // s, s).sum(axis=(1, 3))
    nz, ny, nx = x.shape
    return x.reshape(nz // s, s, ny // s, s, nx // s, s).sum(axis=(1, 3, 5))


# --------------------------------------------------------------- DWT pins --
@pytest.mark.parametrize("shape", [(16, 16), (32, 48), (16, 16, 16), (8, 32, 16)])
@pytest.mark.parametrize("J", [0, 1, 2, 3, 4])
def test_dwt_idwt_round_trip(shape, J):
    """Sec. 3.1 / abstract: the Inverse-DWT restores the image exactly."""
    s = 2 ** J
    if any(n % s for n in shape):
        pytest.skip("shape not divisible")
    rng = np.random.default_rng(J * 7 + len(shape))
    x = rng.integers(-300, 300, size=shape)
    pyr = O.dwt(x, J)
    assert pyr.size == x.size
    assert np.array_equal(O.idwt(pyr, shape, J), x)


def test_paper_subband_size_example():
    """Sec. 4.3 size example and Sec. 3.1 sub-band size 1/4^j (golden file)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_subband_sizes.txt"))
            if l.strip() and not l.startswith("#") and not l.startswith("columns")]
    for nx, ny, J, ax, ay, cnt in [tuple(int(v) for v in r) for r in rows]:
        x = np.zeros((ny, nx), dtype=np.int64)
        bands, cA = O.pyramid_views(O.dwt(x, J), (ny, nx), J)
        assert cA.shape == (ay, ax) and cA.size == cnt
        for j in range(1, J + 1):
            for b in range(1, 4):
                assert bands[(j, b)].size * 4 ** j == nx * ny


@pytest.mark.parametrize("shape,J", [((16, 16), 1), ((32, 32), 2), ((16, 32), 3),
                                     ((8, 8, 8), 1), ((16, 8, 16), 2)])
def test_scaled_approximation_is_block_sum(shape, J):
    """Closed form: scaled-Haar cA_J = sum of each 2^J-block."""
    rng = np.random.default_rng(3)
    x = rng.integers(0, 8, size=shape)
    _, cA = O.pyramid_views(O.dwt(x, J), shape, J)
    assert np.array_equal(cA, block_sum(x, 2 ** J))


def _haar_1d(kind, j, k, n):
    """Sampled Haar function of Sec. 4.2 on pixels [0, n): phi = 1 on [0, 1),
    psi = +1 on [0, 1/2), -1 on [1/2, 1); dilated by 2^j, shifted by k and
    normalised by 2^(-j/2)."""
    v = np.zeros(n)
    w = 2 ** j
    if kind == "phi":
        v[k * w:(k + 1) * w] = 1.0
    else:
        v[k * w:k * w + w // 2] = 1.0
        v[k * w + w // 2:(k + 1) * w] = -1.0
    return v * 2.0 ** (-j / 2.0)


@pytest.mark.parametrize("shape,J", [((8, 8), 1), ((8, 16), 2), ((16, 16), 3),
                                     ((8, 8, 8), 2)])
def test_coefficients_are_inner_products_with_haar_basis(shape, J):
    """Sec. 3.1: a = <TI, phi_{J,k}> and Z^B = <TI, psi^B_{j,k}> for the
    separable Haar basis built from phi and psi of Sec. 4.2. Band b has the
    wavelet psi along axis a when bit a of b is set (x is axis 0). The
    orthonormal transform must equal these inner products, and the scaled one
    must equal them times 2^(d j / 2)."""
    rng = np.random.default_rng(11)
    x = rng.integers(0, 5, size=shape).astype(np.float64)
    d = len(shape)
    dims_xyz = shape[::-1]
    orth = O.dwt_orth(x, J)
    scal = O.dwt(x.astype(np.int64), J)
    bo, ao = O.pyramid_views(orth, shape, J)
    bs, as_ = O.pyramid_views(scal, shape, J)

    def basis(j, b, kxyz):
        vecs = []
        for a in range(d):
            kind = "psi" if (b >> a) & 1 else "phi"
            vecs.append(_haar_1d(kind, j, kxyz[a], dims_xyz[a]))
        # numpy axis order is reversed (z, y, x)
        out = vecs[0][None, :] if d == 2 else vecs[0][None, None, :]
        if d == 2:
            out = vecs[1][:, None] * vecs[0][None, :]
        else:
            out = vecs[2][:, None, None] * vecs[1][None, :, None] * vecs[0][None, None, :]
        return out

    for j in range(1, J + 1):
        for b in range(1, 2 ** d):
            band_o = bo[(j, b)]
            for idx in np.ndindex(band_o.shape):
                kxyz = idx[::-1]
                ip = float((x * basis(j, b, kxyz)).sum())
                assert band_o[idx] == pytest.approx(ip, abs=1e-9)
                assert bs[(j, b)][idx] == pytest.approx(ip * 2.0 ** (d * j / 2.0), abs=1e-6)
    for idx in np.ndindex(ao.shape):
        ip = float((x * basis(J, 0, idx[::-1])).sum())
        assert ao[idx] == pytest.approx(ip, abs=1e-9)
        assert as_[idx] == pytest.approx(ip * 2.0 ** (d * J / 2.0), abs=1e-6)


# --------------------------------------------------------------- CCW pins --
def _random_event(rng, T, d, F, p_known=0.5):
    shape = (T,) * d
    de = rng.integers(0, F, size=shape).astype(np.uint8)
    de[rng.random(shape) >= p_known] = O.UNKNOWN
    return de


@pytest.mark.parametrize("J", [0, 1])
@pytest.mark.parametrize("score_mode", [0, 1])
def test_ccw_map_equals_library_correlation_2d(J, score_mode):
    """Eq. CCW is a 'valid' cross-correlation of cA_J(TI) with cA_J(OR); with
    the one-hot reading it is summed over the facies indicators. Checked
    against scipy.signal.correlate on block sums computed here."""
    rng = np.random.default_rng(5 + J)
    F, T = 3, 4
    ti = synth.random_field_ti((12, 12), F, seed=J)
    t = O.OracleTI(ti, F, J)
    de = _random_event(rng, T, 2, F)
    res = t.search(T, de, K=3, score_mode=score_mode, maps=True)
    s = 2 ** J
    known = de != O.UNKNOWN
    if score_mode == 0:
        ref = 0
        for f in range(F):
            a = block_sum((ti == f).astype(np.int64), s)
            b = block_sum((known & (de == f)).astype(np.int64), s)
            ref = ref + signal.correlate(a, b, mode="valid", method="direct")
    else:
        a = block_sum(ti.astype(np.int64), s)
        b = block_sum(np.where(known, de, 0).astype(np.int64), s)
        ref = signal.correlate(a, b, mode="valid", method="direct")
    assert np.array_equal(res["scores"].reshape(ref.shape), ref)


def test_ccw_map_equals_library_correlation_3d():
    rng = np.random.default_rng(9)
    F, T, J = 4, 4, 1
    ti = synth.random_field_ti((8, 10, 12), F, seed=4)
    t = O.OracleTI(ti, F, J)
    de = _random_event(rng, T, 3, F)
    res = t.search(T, de, K=2, maps=True)
    ref = 0
    for f in range(F):
        a = block_sum((ti == f).astype(np.int64), 2)
        b = block_sum(((de != O.UNKNOWN) & (de == f)).astype(np.int64), 2)
        ref = ref + signal.correlate(a, b, mode="valid", method="direct")
    assert np.array_equal(res["scores"].reshape(ref.shape), ref)


def test_level0_one_hot_score_is_agreement_count():
    """At J = 0 (CCSIM, Sec. 2.1) the one-hot score of a candidate is the
    number of known cells whose facies agrees: n_known - Hamming distance."""
    rng = np.random.default_rng(1)
    ti = synth.random_field_ti((20, 24), 2, seed=8)
    T = 6
    t = O.OracleTI(ti, 2, 0)
    de = _random_event(rng, T, 2, 2, p_known=0.4)
    res = t.search(T, de, K=1, maps=True)
    known = de != O.UNKNOWN
    cy, cx = t.cand_shape(T)
    for c in range(cy * cx):
        y, x = divmod(c, cx)
        win = ti[y:y + T, x:x + T]
        ham = int(((win != de) & known).sum())
        assert res["scores"][c] == known.sum() - ham


def test_planted_pattern_is_found_at_level0():
    """A full data event cut from the TI at c* scores T^d there, the maximum
    at J = 0; the rank-1 candidate carries the same pattern (c* itself unless
    an identical pattern has a lower index)."""
    ti = synth.ribbon_ti(60, 60, n_ribbons=4, seed=3, target=0.3, tol=0.2)
    T = 8
    t = O.OracleTI(ti, 2, 0)
    cy, cx = t.cand_shape(T)
    rng = np.random.default_rng(2)
    for _ in range(5):
        c = int(rng.integers(0, cy * cx))
        y, x = divmod(c, cx)
        de = ti[y:y + T, x:x + T].copy()
        res = t.search(T, de, K=1)
        best = int(res["topk_idx"][0])
        by, bx = divmod(best, cx)
        assert res["topk_score"][0] == T * T
        assert best <= c
        assert np.array_equal(ti[by:by + T, bx:bx + T], de)


def test_topk_and_pick_follow_full_sort_and_philox():
    """Ranking = full sort by (mismatch asc, score desc, index asc), checked
    with numpy.lexsort on the oracle's own maps; pick = topk[u K >> 32]."""
    rng = np.random.default_rng(4)
    F, T, J = 3, 8, 1
    ti = synth.random_field_ti((40, 36), F, seed=2)
    t = O.OracleTI(ti, F, J)
    for trial in range(6):
        de = _random_event(rng, T, 2, F, p_known=0.3)
        hd = np.full((T, T), O.UNKNOWN, np.uint8)
        for _ in range(3):
            qy, qx = rng.integers(0, T, size=2)
            hd[qy, qx] = rng.integers(0, F)
            de[qy, qx] = hd[qy, qx]
        K = int(rng.integers(1, 7))
        seed = int(rng.integers(0, 2 ** 63))
        res = t.search(T, de, hd, K=K, seed=seed, r=trial, p=3 * trial + 1, maps=True)
        idx = np.arange(res["scores"].size)
        order = np.lexsort((idx, -res["scores"], res["mis"]))
        assert np.array_equal(res["topk_idx"], order[:K])
        u = int(O.philox4x32_10([trial, 3 * trial + 1, 0, 0],
                                [seed & 0xFFFFFFFF, seed >> 32])[0])
        assert res["pick"] == order[(u * K) >> 32]


def test_mismatch_is_brute_force_hard_data_disagreement():
    """Sec. 4.4 conditional check: count of hard data in the window that the
    candidate's fine TI pattern contradicts."""
    rng = np.random.default_rng(6)
    F, T, J = 3, 8, 2
    ti = synth.random_field_ti((33, 41), F, seed=5)
    t = O.OracleTI(ti, F, J)
    de = _random_event(rng, T, 2, F, p_known=0.2)
    hd = np.full((T, T), O.UNKNOWN, np.uint8)
    pts = rng.integers(0, T, size=(5, 2))
    for qy, qx in pts:
        hd[qy, qx] = rng.integers(0, F)
    res = t.search(T, de, hd, K=1, maps=True)
    cy, cx = t.cand_shape(T)
    s = 2 ** J
    for c in range(cy * cx):
        y, x = divmod(c, cx)
        win = ti[s * y:s * y + T, s * x:s * x + T]
        assert res["mis"][c] == int(((win != hd) & (hd != O.UNKNOWN)).sum())


def test_feasible_hard_data_give_zero_mismatch():
    """Hard data sampled from a TI patch are honoured exactly by the chosen
    candidate (mismatch 0), as Sec. 5.2 expects of conditional simulation."""
    ti = synth.channel_lens_ti(200, 200, seed=2, tol=0.15)
    T, J = 16, 2
    t = O.OracleTI(ti, 3, J)
    cy, cx = t.cand_shape(T)
    rng = np.random.default_rng(8)
    for _ in range(4):
        c = int(rng.integers(0, cy * cx))
        y, x = divmod(c, cx)
        patch = ti[4 * y:4 * y + T, 4 * x:4 * x + T]
        hd = np.full((T, T), O.UNKNOWN, np.uint8)
        sel = rng.random((T, T)) < 0.05
        hd[sel] = patch[sel]
        res = t.search(T, hd.copy(), hd, K=5, maps=False)
        assert res["topk_mis"][0] == 0


# ------------------------------------------------------- reconstruct pins --
@pytest.mark.parametrize("shape,J,T", [((40, 44), 0, 8), ((40, 44), 1, 8), ((64, 72), 2, 16),
                                       ((64, 48), 3, 16), ((24, 20, 28), 1, 8),
                                       ((24, 32, 16), 2, 8)])
def test_reconstruct_equals_ti_crop(shape, J, T):
    """Algorithm 1, line 13 and Sec. 3.2 ('information is not lost'): the
    Inverse-DWT of the selected approximation block plus the TI's detail
    coefficients is exactly the TI crop at s * candidate origin."""
    ti = synth.random_field_ti(shape, 5, seed=J)
    t = O.OracleTI(ti, 5, J)
    s = 2 ** J
    cs = t.cand_shape(T)
    rng = np.random.default_rng(J)
    for c in rng.integers(0, int(np.prod(cs)), size=5):
        pos = np.unravel_index(int(c), cs)          # numpy order (z,) y, x
        sl = tuple(slice(s * p, s * p + T) for p in pos)
        assert np.array_equal(t.reconstruct(T, int(c)), ti[sl])


# ----------------------------------------------------------- lattice pins --
def test_lattice_and_candidate_counts_of_workloads():
    """Sec. 4.1 lattice (patches of edge T stepping by T - OR) on the
    workload shapes; candidate counts follow the level-J TI size of Sec. 4.3."""
    cases = [  # ndim, grid, T, O, expected patches per axis
        (2, (250, 250), 40, 10, (8, 8, 1)),
        (2, (2000, 2000), 64, 16, (42, 42, 1)),
        (2, (1000, 1000), 64, 16, (21, 21, 1)),
        (3, (200, 200, 100), 24, 6, (11, 11, 6)),
        (3, (100, 100, 100), 24, 6, (6, 6, 6)),
        (2, (512, 512), 48, 12, (14, 14, 1)),
    ]
    for ndim, grid, T, Ov, exp in cases:
        n, gp = O.lattice(ndim, grid, T, Ov)
        assert n == exp
        for a in range(ndim):
            assert gp[a] >= grid[a] and gp[a] - (T - Ov) < grid[a] or n[a] == 1
    ti1 = np.zeros((250, 250), np.uint8)
    assert O.OracleTI(ti1, 2, 1).num_candidates(40) == 106 * 106
    assert O.OracleTI(ti1, 2, 2).num_candidates(64) == 47 * 47
    assert O.OracleTI(ti1, 2, 2).num_candidates(48) == 51 * 51
    assert O.OracleTI(np.zeros((1000, 1000), np.uint8), 3, 2).num_candidates(64) == 235 * 235
    assert O.OracleTI(np.zeros((120, 150, 180), np.uint8), 4, 1).num_candidates(24) == 79 * 64 * 49


# ----------------------------------------------------------- Philox pins ---
def read_philox_kat():
    """The published Philox4x32-10 known-answer vectors
    (tests/golden/philox4x32_10_kat.txt): [(ctr, key, out)]."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_matches_published_known_answers():
    """Philox4x32-10 (SC'11) of the oracle reproduces the published
    known-answer vectors, one block at a time and in a batch."""
    rows = read_philox_kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert [int(x) for x in O.philox4x32_10(ctr, key)] == out
        got = O.philox_many(np.array([ctr, ctr], np.uint32), key)
        assert got.tolist() == [out, out]


def test_philox_output_is_uniform_and_sensitive():
    """Beyond the known answers: 32-bit words are uniform (chi-square on the
    top byte) and every input word changes every output word."""
    words = O.philox_many(np.array([[i, 7, 0, 0] for i in range(4000)], np.uint32), [123, 456])
    top = (words.reshape(-1) >> 24).astype(np.int64)
    hist = np.bincount(top, minlength=256)
    exp = top.size / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 340          # 255 dof, p ~ 1e-3
    base = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    for pos in range(6):
        ctr, key = [1, 2, 3, 4], [5, 6]
        if pos < 4:
            ctr[pos] ^= 1
        else:
            key[pos - 4] ^= 1
        alt = O.philox4x32_10(ctr, key)
        assert np.all(alt != base)
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(alt, base))
        assert 40 < flips < 88


# ---------------------------------------------------------- simulate pins --
@pytest.mark.parametrize("path_random", [0, 1])
def test_first_patch_core_is_a_ti_crop(path_random):
    """Algorithm 1, lines 5-6 and 14: the first patch is a random TI patch
    pasted, unmirrored, at the path's origin corner; the part of it that no
    later patch overlaps survives unchanged in the realization."""
    ti = synth.ribbon_ti(120, 120, n_ribbons=6, seed=4, target=0.3, tol=0.2)
    T, Ov, J = 16, 4, 1
    t = O.OracleTI(ti, 2, J)
    grid = (70, 58)                      # (nx, ny)
    seed = 99
    seen = set()
    for r in range(8):
        out, log = t.simulate(grid, T, Ov, K=3, path_random=path_random, seed=seed, r=r)
        assert log[0, 3] & 1                           # uniform first pick
        pat = t.reconstruct(T, int(log[0, 0]))         # [qy, qx]
        flips = O.path_flips(2, seed, r, path_random)
        seen.add(flips)
        # along a forward axis the first window is [0, T) and later patches
        # share [T - O, T); along a reversed axis it is the far corner and
        # later patches share [0, O) of it
        rng_q, to_out = [], []
        for a in range(2):
            if (flips >> a) & 1:
                rng_q.append(range(Ov, T))
                to_out.append(grid[a] - T)
            else:
                rng_q.append(range(0, T - Ov))
                to_out.append(0)
        checked = 0
        for qy in rng_q[1]:
            for qx in rng_q[0]:
                x, y = qx + to_out[0], qy + to_out[1]
                if 0 <= x < grid[0] and 0 <= y < grid[1]:
                    assert out[y, x] == pat[qy, qx]
                    checked += 1
        assert checked > 0
    assert (len(seen) > 1) == bool(path_random)


def test_hard_data_are_honoured_in_realizations():
    """Sec. 5.2: conditional realizations reproduce every hard datum."""
    ti = synth.channel_lens_ti(200, 200, seed=2, tol=0.15)
    field = synth.channel_lens_ti(200, 200, seed=3, tol=0.15)
    cells, vals = synth.sample_hard_data(field, 60, seed=4)
    t = O.OracleTI(ti, 3, 2)
    out, log = t.simulate((200, 200), 32, 8, K=5, hd_cells=cells, hd_vals=vals, seed=3)
    assert np.array_equal(out[cells[:, 1], cells[:, 0]], vals)
    assert np.all(out < 3)
    assert np.all(log[:, 3] & 2)


@pytest.mark.parametrize("path_random", [0, 1])
def test_first_patch_core_is_a_ti_crop_3d(path_random):
    """The 3D form of the first-patch pin: a uniform TI patch pasted,
    unmirrored, at the path's origin corner; the part no later patch
    overlaps ([0, T - OR) along each forward axis, [OR, T) along a mirrored
    one) survives in the realization."""
    ti = synth.tube_lobe_ti_3d(48, 40, 36, seed=5)
    T, Ov, J = 8, 2, 1
    t = O.OracleTI(ti, 4, J)
    grid = (20, 14, 14)                  # T + k (T - OR) on every axis: no padding
    seed = 77
    seen = set()
    for r in range(8):
        out, log = t.simulate(grid, T, Ov, K=3, path_random=path_random, seed=seed, r=r)
        assert log[0, 3] & 1
        pat = t.reconstruct(T, int(log[0, 0]))          # [qz, qy, qx]
        flips = O.path_flips(3, seed, r, path_random)
        seen.add(flips)
        rq, org = [], []
        for a in range(3):
            if (flips >> a) & 1:
                rq.append(np.arange(Ov, T))
                org.append(grid[a] - T)
            else:
                rq.append(np.arange(0, T - Ov))
                org.append(0)
        qz, qy, qx = np.meshgrid(rq[2], rq[1], rq[0], indexing="ij")
        got = out[qz + org[2], qy + org[1], qx + org[0]]
        assert np.array_equal(got, pat[qz, qy, qx])
    assert (len(seen) > 1) == bool(path_random)


def test_hard_data_are_honoured_in_3d_realizations():
    """Sec. 5.2 in 3D: every hard datum is reproduced."""
    ti = synth.tube_lobe_ti_3d(48, 40, 36, seed=5)
    field = synth.tube_lobe_ti_3d(26, 22, 18, seed=6)
    cells, vals = synth.sample_hard_data(field, 80, seed=7)
    t = O.OracleTI(ti, 4, 1)
    out, log = t.simulate((26, 22, 18), 8, 2, K=4, hd_cells=cells, hd_vals=vals, seed=3,
                          path_random=1)
    assert np.array_equal(out[cells[:, 2], cells[:, 1], cells[:, 0]], vals)
    assert np.all(out < 4) and np.all(log[:, 3] & 2)
