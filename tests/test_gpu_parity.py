"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer path, so every comparison is exact (scores, mismatches, ranks,
picks, pasted cells, realizations, patch logs).
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import configs, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccw():
    import paper_2404_00441_gb300 as m
    m.load()
    return m


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.cpu().numpy()


# ------------------------------------------------------------ TI prepare --
def block_layout_from_pyramid(pyr, shape, J):
    """Map the oracle's Mallat pyramid to the per-block in-place layout of
    ccw_ti_export(what=2): a level-j band-b coefficient with band index k
    lives in block k >> (J - j), at in-block position
    ((k mod 2^(J-j)) * 2^j + (2^(j-1) if bit a of b else 0)) per axis."""
    d = len(shape)
    s = 2 ** J
    bands, cA = O.pyramid_views(pyr, shape, J)
    cshape = tuple(n // s for n in shape)
    out = np.zeros(cshape + (s,) * d, np.int64)          # [.., by, bx, cy, cx]
    for idx in np.ndindex(cA.shape):
        out[idx + (0,) * d] = cA[idx]
    for (j, b), arr in bands.items():
        for idx in np.ndindex(arr.shape):
            blk, pos = [], []
            for ax in range(d):                    # numpy axis ax <-> spatial axis d-1-ax
                k = idx[ax]
                sa = d - 1 - ax
                blk.append(k >> (J - j))
                pos.append((k % (1 << (J - j))) * (1 << j) + ((1 << (j - 1)) if (b >> sa) & 1 else 0))
            out[tuple(blk) + tuple(pos)] = arr[idx]
    return out.reshape(cshape + (s ** d,))


@pytest.mark.parametrize("case", [("2d", 3, 2, (60, 52)), ("2d", 2, 1, (41, 37)), ("2d", 5, 3, (64, 40)),
                                  ("3d", 4, 1, (18, 22, 14)), ("3d", 3, 2, (16, 24, 20))])
def test_ti_prepare_matches_oracle(ccw, case):
    _, F, J, shape = case
    ti = synth.random_field_ti(shape, F, seed=F + J)
    T = 2 ** J * 2
    g = ccw.TI(dev(ti), F, J, T, 0)
    o = O.OracleTI(ti, F, J)
    cA_ind, cA_code, pyr, ti_c = o.arrays()
    assert np.array_equal(host(g.export(3)), ti_c)
    assert np.array_equal(host(g.export(0)).astype(np.int64), cA_ind[:F - 1])
    assert np.array_equal(host(g.export(1)).astype(np.int64), cA_code)
    assert np.array_equal(host(g.export(2)).astype(np.int64),
                          block_layout_from_pyramid(pyr, o.shape, J))
    assert g.n_cand == o.num_candidates(T)


# ---------------------------------------------------------------- CCF map --
MAP_CASES = [
    # name, TI factory, F, J, T, O
    ("c1geom", lambda: configs.ribbon_ti_250(), 2, 1, 40, 10),
    ("c2geom", lambda: synth.channel_lens_ti(300, 260, seed=2, tol=0.2), 3, 2, 64, 16),
    ("j0", lambda: synth.random_field_ti((50, 70), 3, seed=1), 3, 0, 8, 2),
    ("f8j3", lambda: synth.random_field_ti((96, 120), 8, seed=3), 8, 3, 32, 8),
    ("3d", lambda: synth.tube_lobe_ti_3d(40, 36, 30, seed=5), 4, 1, 12, 2),
]


@pytest.mark.parametrize("case", MAP_CASES, ids=[c[0] for c in MAP_CASES])
@pytest.mark.parametrize("score_mode", [0, 1])
def test_ccf_map_matches_oracle(ccw, case, score_mode):
    name, mk, F, J, T, Ov = case
    ti = mk()
    if score_mode == 1 and (F - 1) ** 2 * T ** ti.ndim * 2 ** (J * ti.ndim) >= 2 ** 24:
        pytest.skip("literal score beyond the exact bound")
    rng = np.random.default_rng(len(name) + score_mode)
    de, hd = configs.structured_events(ti, T, Ov, 6, rng, n_hd=3, F=F)
    de[0] = 255                   # an empty data event
    hd[0] = 255
    g = ccw.TI(dev(ti), F, J, T, Ov)
    o = O.OracleTI(ti, F, J)
    sc, mm = ccw.ccf_map(g, dev(de), dev(hd), score_mode=score_mode)
    sc, mm = host(sc), host(mm)
    for b in range(de.shape[0]):
        ref = o.search(T, de[b], hd[b], K=1, score_mode=score_mode, maps=True)
        assert np.array_equal(sc[b], ref["scores"]), f"score map {b}"
        assert np.array_equal(mm[b], ref["mis"]), f"mismatch map {b}"


# -------------------------------------------------------------- CCF search --
@pytest.mark.parametrize("case", MAP_CASES, ids=[c[0] for c in MAP_CASES])
@pytest.mark.parametrize("K", [1, 5, 64])
def test_ccf_search_matches_oracle(ccw, case, K):
    name, mk, F, J, T, Ov = case
    ti = mk()
    rng = np.random.default_rng(K + len(name))
    B = 9
    de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=2, F=F)
    de[3] = 255
    hd[3] = 255
    seed = int(rng.integers(0, 2 ** 63))
    ctr = np.stack([rng.integers(0, 1000, B), rng.integers(0, 5000, B)], axis=1).astype(np.uint32)
    g = ccw.TI(dev(ti), F, J, T, Ov)
    o = O.OracleTI(ti, F, J)
    res = ccw.ccf_search(g, dev(de), dev(hd), k=K, seed=seed, ctr=dev(ctr.view(np.int32)))
    res = {k: host(v) for k, v in res.items()}
    for b in range(B):
        ref = o.search(T, de[b], hd[b], K=K, seed=seed, r=int(ctr[b, 0]), p=int(ctr[b, 1]))
        n = ref["n"]
        assert res["pick"][b] == ref["pick"], f"pick {b}"
        assert np.array_equal(res["topk_idx"][b, :n], ref["topk_idx"])
        assert np.array_equal(res["topk_score"][b, :n], ref["topk_score"])
        assert np.array_equal(res["topk_mis"][b, :n], ref["topk_mis"])
        assert np.all(res["topk_idx"][b, n:] == -1)
    assert g.status() == 0


def test_ccf_search_more_k_than_candidates(ccw):
    """P_c < K: only P_c ranked entries, the rest -1."""
    ti = synth.random_field_ti((12, 14), 3, seed=9)
    T, J = 8, 1
    g = ccw.TI(dev(ti), 3, J, T, 2)
    o = O.OracleTI(ti, 3, J)
    assert g.n_cand == 4 * 3
    rng = np.random.default_rng(0)
    de, hd = configs.structured_events(ti, T, 2, 4, rng, n_hd=1, F=3)
    ctr = np.arange(8, dtype=np.uint32).reshape(4, 2)
    res = ccw.ccf_search(g, dev(de), dev(hd), k=20, seed=5, ctr=dev(ctr.view(np.int32)))
    for b in range(4):
        ref = o.search(T, de[b], hd[b], K=20, seed=5, r=int(ctr[b, 0]), p=int(ctr[b, 1]))
        assert ref["n"] == 12
        assert np.array_equal(host(res["topk_idx"])[b, :12], ref["topk_idx"])
        assert np.all(host(res["topk_idx"])[b, 12:] == -1)
        assert host(res["pick"])[b] == ref["pick"]


# ------------------------------------------------------------ IDWT paste --
@pytest.mark.parametrize("shape,F,J,T", [((80, 90), 3, 2, 16), ((64, 64), 2, 4, 32),
                                         ((30, 26, 22), 4, 1, 8), ((24, 32, 28), 3, 2, 8)])
def test_idwt_paste_matches_oracle(ccw, shape, F, J, T):
    ti = synth.random_field_ti(shape, F, seed=J)
    g = ccw.TI(dev(ti), F, J, T, 0)
    o = O.OracleTI(ti, F, J)
    d = ti.ndim
    rng = np.random.default_rng(1)
    B = 6
    picks = rng.integers(0, g.n_cand, B).astype(np.int32)
    gshape = tuple(n + 10 for n in shape)      # numpy order
    gdims = gshape[::-1]
    origins = np.zeros((B, 3), np.int32)
    for b in range(B):
        for a in range(d):
            origins[b, a] = rng.integers(-T // 2, gdims[a] - T // 2)
    sg = np.full(gshape, 255, np.uint8)
    out = host(ccw.idwt_paste(g, dev(picks), dev(origins), dev(sg)))
    ref = np.full(gshape, 255, np.uint8)
    for b in range(B):
        pat = o.reconstruct(T, int(picks[b]))
        sl_dst, sl_src = [], []
        for a in range(d):                    # numpy axis a <-> spatial d-1-a
            sa = d - 1 - a
            lo = origins[b, sa]
            s0, s1 = max(lo, 0), min(lo + T, gdims[sa])
            sl_dst.append(slice(s0, s1))
            sl_src.append(slice(s0 - lo, s1 - lo))
        ref[tuple(sl_dst)] = pat[tuple(sl_src)]
    covered = np.zeros(gshape, int)
    for b in range(B):
        sl = []
        for a in range(d):
            sa = d - 1 - a
            lo = origins[b, sa]
            sl.append(slice(max(lo, 0), min(lo + T, gdims[sa])))
        covered[tuple(sl)] += 1
    # cells covered by one destination are defined; overlaps are unspecified
    once = covered == 1
    assert np.array_equal(out[once], ref[once])
    assert np.all(out[covered == 0] == 255)
