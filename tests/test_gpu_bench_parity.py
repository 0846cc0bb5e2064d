"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (precision and CCF tiling from workloads.configs.BENCH_TILE).

* 2000x2000 3-facies workload: every hard datum honoured, every cell equal to
  the Inverse-DWT pattern of the last patch covering it, and sampled patches
  re-searched by the oracle on the data event rebuilt from the logged pastes
  (identical ranking, scores, mismatches and pick) -- in the benchmarked
  BF16 tiling, the library's FP16 tiling and on the FP32 lanes.
* 64 x 1000^2 and 256 x 512^2 binary batches: whole realizations at the
  start, middle and end of the batch equal the oracle's simulation.
* 3D mixed-size batch: sampled patches of the first realization of each grid
  size re-searched by the oracle as above.
* Table 2 geometry (20 x 512^2 with hard data, top-5) at each level J:
  sampled patches of the first and last realization, as above.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccw():
    import paper_2404_00441_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def replay_check(o, ti_shape_nd, grid, T, Ov, K, seed, r, out, log, cells, vals, n_sample,
                 rng_seed=0):
    """Replays the logged pastes of one realization in raster order (Algorithm
    1) on the host; at sampled patches the oracle searches the rebuilt data
    event and must give the logged ranking and pick; at the end the replayed
    grid must equal the realization."""
    d = len(grid)
    npch, gp = O.lattice(d, grid, T, Ov)
    S = T - Ov
    shape = tuple(gp[:d])[::-1]
    hd_img = np.full(shape, 255, np.uint8)
    state = np.full(shape, 255, np.uint8)
    if cells is not None:
        hd_img[tuple(cells[:, a] for a in range(d - 1, -1, -1))] = vals
        assert np.array_equal(out[tuple(cells[:, a] for a in range(d - 1, -1, -1))], vals)
    n_patches = int(np.prod(npch[:d]))
    rng = np.random.default_rng(rng_seed)
    sample = set(rng.choice(n_patches, min(n_sample, n_patches), replace=False).tolist())
    sample |= {0, 1, npch[0], n_patches - 1}
    for p in range(n_patches):
        ip = [p % npch[0], (p // npch[0]) % npch[1], p // (npch[0] * npch[1])]
        win = tuple(slice(S * ip[a], S * ip[a] + T) for a in range(d - 1, -1, -1))
        hw = hd_img[win]
        if p in sample:
            de = np.where(hw != 255, hw, state[win])
            ref = o.search(T, de, hw, K=K, seed=seed, r=r, p=p)
            e = log[p]
            assert e[0] == ref["pick"], f"pick of patch {p}"
            n = ref["n"]
            if n:
                assert np.array_equal(e[4:4 + n], ref["topk_idx"]), f"ranking of patch {p}"
                sel = list(ref["topk_idx"]).index(ref["pick"])
                assert e[1] == ref["topk_score"][sel] and e[2] == ref["topk_mis"][sel]
        assert log[p, 3] & 2
        pat = o.reconstruct(T, int(log[p, 0]))
        state[win] = np.where(hw != 255, hw, pat)
    crop = tuple(slice(0, grid[a]) for a in range(d - 1, -1, -1))
    assert np.array_equal(state[crop], out)


@pytest.mark.parametrize("form", ["bench", "fp16_library_tile", "fp32_lanes"])
def test_c2_full_size_sampled(ccw, form):
    w = configs.workload("c2")
    prec, tile = {"bench": configs.bench_tile("c2"), "fp16_library_tile": (1, 0),
                  "fp32_lanes": (0, 0)}[form]
    ti, F, J, T, Ov, K, grid = w["ti"], w["F"], w["J"], w["T"], w["O"], w["K"], w["grid"]
    cells, vals = w["hd"]
    g = ccw.TI(dev(ti), F, J, T, Ov)
    out, log = ccw.simulate(g, grid, n_real=1, topk=K, seed=w["seed"], hd_cells=dev(cells),
                            hd_vals=dev(vals), want_log=True, precision=prec, ccf_tile=tile)
    out, log = out.cpu().numpy()[0], log.cpu().numpy()[0]
    replay_check(O.OracleTI(ti, F, J), ti.shape, grid, T, Ov, K, w["seed"], 0, out, log, cells,
                 vals, n_sample=24)


@pytest.mark.parametrize("name", ["c3", "c5"])
def test_batched_full_size_realizations(ccw, name):
    """All realizations of the batch in one call, in the benchmarked tiling;
    realizations at the start, middle and end equal the oracle's."""
    w = configs.workload(name)
    prec, tile = configs.bench_tile(name)
    g = ccw.TI(dev(w["ti"]), w["F"], w["J"], w["T"], w["O"])
    out, log = ccw.simulate(g, w["grid"], n_real=w["n_real"], topk=w["K"], seed=w["seed"],
                            want_log=True, precision=prec, ccf_tile=tile)
    o = O.OracleTI(w["ti"], w["F"], w["J"])
    for r in (0, w["n_real"] // 2 - 1, w["n_real"] - 1):
        ref, rlog = o.simulate(w["grid"], w["T"], w["O"], K=w["K"], seed=w["seed"], r=r)
        assert np.array_equal(log[r].cpu().numpy(), rlog), f"patch log of realization {r}"
        assert np.array_equal(out[r].cpu().numpy(), ref), f"realization {r}"


@pytest.mark.parametrize("name", ["t2_j1_h1000", "t2_j2_h2000", "t2_j3_h1000"])
def test_table2_batch_sampled(ccw, name):
    """The Table 2 geometry (20 x 512^2, T 32, OR 8, top-5, 1000 or 2000 hard
    data) in the benchmarked tiling of its level; sampled patches of the
    first and last realization re-searched by the oracle, both replayed."""
    w = configs.workload(name)
    prec, tile = configs.bench_tile(name)
    cells, vals = w["hd"]
    g = ccw.TI(dev(w["ti"]), w["F"], w["J"], w["T"], w["O"])
    out, log = ccw.simulate(g, w["grid"], n_real=w["n_real"], topk=w["K"], seed=w["seed"],
                            hd_cells=dev(cells), hd_vals=dev(vals), want_log=True,
                            precision=prec, ccf_tile=tile)
    o = O.OracleTI(w["ti"], w["F"], w["J"])
    for r in (0, w["n_real"] - 1):
        replay_check(o, w["ti"].shape, w["grid"], w["T"], w["O"], w["K"], w["seed"], r,
                     out[r].cpu().numpy(), log[r].cpu().numpy(), cells, vals, n_sample=8,
                     rng_seed=r)


def test_3d_mixed_batch_sampled(ccw):
    """The 3D batch (8 x 200x200x100 + 8 x 100^3, 1000 hard data per size) in
    the benchmarked tiling; sampled patches of realization 0 of each size."""
    w = configs.workload("c4")
    prec, tile = configs.bench_tile("c4")
    g = ccw.TI(dev(w["ti"]), w["F"], w["J"], w["T"], w["O"])
    groups = [dict(grid=s["grid"], n_real=s["n_real"], real_base=s["real_base"],
                   hd_cells=dev(s["hd"][0]), hd_vals=dev(s["hd"][1])) for s in w["groups"]]
    res = ccw.simulate_groups(g, groups, topk=w["K"], seed=w["seed"], precision=prec,
                              ccf_tile=tile, want_log=True)
    o = O.OracleTI(w["ti"], w["F"], w["J"])
    for s, (out, log) in zip(w["groups"], res):
        replay_check(o, w["ti"].shape, s["grid"], w["T"], w["O"], w["K"], w["seed"],
                     s["real_base"], out[0].cpu().numpy(), log[0].cpu().numpy(), s["hd"][0],
                     s["hd"][1], n_sample=4, rng_seed=1)
