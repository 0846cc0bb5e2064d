"""GPU parity of the tensor-core CCF (FP16 / BF16 operands, FP32 accumulation
in tensor memory) against the CPU oracle. Within the exact integer range of
the 16-bit formats the results are bit-identical to the oracle's."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # name, TI factory, F, J, T, O
    ("c1geom", lambda: configs.ribbon_ti_250(), 2, 1, 40, 10),
    ("c3geom", lambda: configs.ribbon_ti_250(), 2, 2, 64, 16),
    ("c2geom", lambda: synth.channel_lens_ti(300, 260, seed=2, tol=0.2), 3, 2, 64, 16),
    ("j0", lambda: synth.random_field_ti((50, 70), 3, seed=1), 3, 0, 8, 2),
    ("f5j3", lambda: synth.random_field_ti((96, 120), 5, seed=3), 5, 3, 32, 8),
]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tensor_ccf_map_matches_oracle(ccw, case, precision):
    name, mk, F, J, T, Ov = case
    ti = mk()
    rng = np.random.default_rng(len(name) + 10 * precision)
    B = 21                    # spans two N-tiles of 16
    de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=2, F=F)
    de[4] = 255
    hd[4] = 255
    g = ccw.TI(dev(ti), F, J, T, Ov)
    o = O.OracleTI(ti, F, J)
    sc, mm = ccw.ccf_map(g, dev(de), dev(hd), precision=precision)
    sc, mm = sc.cpu().numpy(), mm.cpu().numpy()
    for b in range(B):
        ref = o.search(T, de[b], hd[b], K=1, maps=True)
        assert np.array_equal(sc[b], ref["scores"]), f"score map {b}"
        assert np.array_equal(mm[b], ref["mis"]), f"mismatch map {b}"


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("K", [1, 5, 64])
def test_tensor_ccf_search_matches_oracle(ccw, precision, K):
    ti = synth.channel_lens_ti(300, 260, seed=2, tol=0.2)
    F, J, T, Ov = 3, 2, 64, 16
    rng = np.random.default_rng(K + precision)
    B = 40
    de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=3, F=F)
    de[7] = 255
    hd[7] = 255
    seed = int(rng.integers(0, 2 ** 63))
    ctr = np.stack([rng.integers(0, 99, B), rng.integers(0, 999, B)], 1).astype(np.uint32)
    g = ccw.TI(dev(ti), F, J, T, Ov)
    o = O.OracleTI(ti, F, J)
    res = ccw.ccf_search(g, dev(de), dev(hd), k=K, seed=seed, ctr=dev(ctr.view(np.int32)),
                         precision=precision)
    res = {k2: v.cpu().numpy() for k2, v in res.items()}
    for b in range(B):
        ref = o.search(T, de[b], hd[b], K=K, seed=seed, r=int(ctr[b, 0]), p=int(ctr[b, 1]))
        n = ref["n"]
        assert res["pick"][b] == ref["pick"], f"pick {b}"
        assert np.array_equal(res["topk_idx"][b, :n], ref["topk_idx"])
        assert np.array_equal(res["topk_score"][b, :n], ref["topk_score"])
        assert np.array_equal(res["topk_mis"][b, :n], ref["topk_mis"])


@pytest.mark.parametrize("precision", [1, 2])
def test_tensor_simulation_matches_oracle(ccw, precision):
    """Many realizations through the tensor-core wave step (c3 geometry on a
    smaller grid) and a hard-data 3-facies case, bit-exact."""
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 2, 64, 16)
    out, log = ccw.simulate(g, (200, 170), n_real=12, topk=1, seed=33, real_base=5,
                            precision=precision, want_log=True)
    out, log = out.cpu().numpy(), log.cpu().numpy()
    o = O.OracleTI(ti, 2, 2)
    for i in range(12):
        ref, rlog = o.simulate((200, 170), 64, 16, K=1, seed=33, r=5 + i)
        assert np.array_equal(log[i], rlog)
        assert np.array_equal(out[i], ref)
    ti3 = configs.channel_lens_ti_1000()
    field = synth.channel_lens_ti(300, 260, seed=3, tol=0.2)
    cells, vals = synth.sample_hard_data(field, 40, seed=4)
    g3 = ccw.TI(dev(ti3), 3, 2, 64, 16)
    out, log = ccw.simulate(g3, (300, 260), n_real=2, topk=5, seed=9, hd_cells=dev(cells),
                            hd_vals=dev(vals), precision=precision, path_random=1,
                            want_log=True)
    o3 = O.OracleTI(ti3, 3, 2)
    for i in range(2):
        ref, rlog = o3.simulate((300, 260), 64, 16, K=5, hd_cells=cells, hd_vals=vals, seed=9,
                                r=i, path_random=1)
        assert np.array_equal(log.cpu().numpy()[i], rlog)
        assert np.array_equal(out.cpu().numpy()[i], ref)


def test_tensor_precision_bounds(ccw):
    """BF16 is exact up to 256: the one-hot score at J = 4 (2D) fits, the
    literal score of 3 facies (operands up to 512) does not and is refused;
    the 3D tensor-core path keeps per-thread K-lists, so K > 8 is refused."""
    ti = synth.random_field_ti((128, 128), 3, seed=1)
    g = ccw.TI(dev(ti), 3, 4, 32, 16)
    de = torch.full((1, 32, 32), 255, dtype=torch.uint8, device="cuda")
    ccw.ccf_map(g, de, precision=2)
    with pytest.raises(ccw.CCWError, match="exact integer range"):
        ccw.ccf_map(g, de, score_mode=1, precision=2)
    ti3 = synth.random_field_ti((20, 20, 20), 2, seed=1)
    g3 = ccw.TI(dev(ti3), 2, 1, 8, 2)
    de3 = torch.full((1, 8, 8, 8), 255, dtype=torch.uint8, device="cuda")
    ccw.ccf_search(g3, de3, k=8, precision=1)
    with pytest.raises(ccw.CCWError, match="K <= 8"):
        ccw.ccf_search(g3, de3, k=9, precision=1)


CASES_3D = [
    # name, TI factory, F, J, T, O
    ("tube_j1", lambda: synth.tube_lobe_ti_3d(60, 50, 40, seed=5), 4, 1, 12, 2),
    ("rand_j0", lambda: synth.random_field_ti((22, 26, 18), 3, seed=4), 3, 0, 6, 2),
    ("rand_j2", lambda: synth.random_field_ti((48, 40, 44), 2, seed=6), 2, 2, 16, 4),
]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", CASES_3D, ids=[c[0] for c in CASES_3D])
def test_streamed_tensor_ccf_3d_matches_oracle(ccw, case, precision):
    """3D on the tensor cores (operands streamed through shared-memory
    stages): maps and K = 1 / 5 searches equal the oracle's."""
    name, mk, F, J, T, Ov = case
    ti = mk()
    rng = np.random.default_rng(len(name) + 7 * precision)
    B = 19
    de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=2, F=F)
    de[3] = 255
    hd[3] = 255
    g = ccw.TI(dev(ti), F, J, T, Ov)
    o = O.OracleTI(ti, F, J)
    sc, mm = ccw.ccf_map(g, dev(de), dev(hd), precision=precision)
    sc, mm = sc.cpu().numpy(), mm.cpu().numpy()
    for b in range(B):
        ref = o.search(T, de[b], hd[b], K=1, maps=True)
        assert np.array_equal(sc[b], ref["scores"]), f"score map {b}"
        assert np.array_equal(mm[b], ref["mis"]), f"mismatch map {b}"
    ctr = torch.from_numpy(np.stack([np.arange(B), np.arange(B) * 3], 1).astype(np.int32)).cuda()
    for K in (1, 5):
        res = ccw.ccf_search(g, dev(de), dev(hd), k=K, seed=17, ctr=ctr, precision=precision)
        for b in range(B):
            ref = o.search(T, de[b], hd[b], K=K, seed=17, r=b, p=3 * b)
            n = ref["n"]
            assert int(res["pick"][b]) == ref["pick"], f"pick {b} K {K}"
            assert np.array_equal(res["topk_idx"][b][:n].cpu().numpy(), ref["topk_idx"])
            assert np.array_equal(res["topk_score"][b][:n].cpu().numpy(), ref["topk_score"])


@pytest.mark.parametrize("precision", [1, 2])
def test_streamed_tensor_3d_simulation_bit_exact(ccw, precision):
    """Whole 3D simulations with hard data on the streamed tensor-core CCF
    equal the oracle's realizations and patch logs."""
    ti = synth.tube_lobe_ti_3d(60, 50, 40, seed=5)
    field = synth.tube_lobe_ti_3d(50, 44, 30, seed=6)
    cells, vals = synth.sample_hard_data(field, 40, seed=7)
    g = ccw.TI(dev(ti), 4, 1, 12, 2)
    out, log = ccw.simulate(g, (50, 44, 30), n_real=2, topk=5, seed=9, hd_cells=dev(cells),
                            hd_vals=dev(vals), path_random=1, precision=precision, want_log=True)
    o = O.OracleTI(ti, 4, 1)
    for i in range(2):
        ref, rlog = o.simulate((50, 44, 30), 12, 2, K=5, path_random=1, hd_cells=cells,
                               hd_vals=vals, seed=9, r=i)
        assert np.array_equal(log.cpu().numpy()[i], rlog)
        assert np.array_equal(out.cpu().numpy()[i], ref)
