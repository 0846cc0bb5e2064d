"""GPU parity of whole simulations (Algorithm 1) against the CPU oracle.

The CUDA path runs patches in wavefronts; the oracle runs the raster path one
patch at a time. Realizations and patch logs must be identical.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_pair(ccw, ti, F, J, T, Ov, grid, K, n_real=1, real_base=0, hd=None, seed=11,
             path_random=0, score_mode=0):
    g = ccw.TI(dev(ti), F, J, T, Ov)
    hc = hv = None
    if hd is not None:
        hc, hv = dev(hd[0]), dev(hd[1])
    out, log = ccw.simulate(g, grid, n_real=n_real, topk=K, seed=seed, hd_cells=hc, hd_vals=hv,
                            real_base=real_base, path_random=path_random,
                            score_mode=score_mode, want_log=True)
    out, log = out.cpu().numpy(), log.cpu().numpy()
    o = O.OracleTI(ti, F, J)
    for i in range(n_real):
        ref, rlog = o.simulate(grid, T, Ov, K=K, score_mode=score_mode,
                               path_random=path_random,
                               hd_cells=None if hd is None else hd[0],
                               hd_vals=None if hd is None else hd[1], seed=seed,
                               r=real_base + i)
        assert np.array_equal(log[i], rlog), f"patch log of realization {i}"
        assert np.array_equal(out[i], ref), f"realization {i}"
    return out, log


def test_c1_full_workload(ccw):
    """Binary ribbon TI 250x250, one 250x250 realization, T40/OR10/J1, K=1."""
    w = configs.workload("c1")
    run_pair(ccw, w["ti"], w["F"], w["J"], w["T"], w["O"], w["grid"], w["K"], seed=w["seed"])


def test_three_facies_hard_data_top5(ccw):
    """c2 geometry (T64/OR16/J2, K=5, 3 facies, hard data) on a 520x456 grid,
    two realizations with a realization offset and randomised paths."""
    ti = configs.channel_lens_ti_1000()
    field = synth.channel_lens_ti(520, 456, seed=3, tol=0.2)
    hd = synth.sample_hard_data(field, 80, seed=4)
    run_pair(ccw, ti, 3, 2, 64, 16, (520, 456), 5, n_real=2, real_base=7, hd=hd, seed=5,
             path_random=1)


def test_literal_score_mode(ccw):
    ti = synth.channel_lens_ti(200, 180, seed=2, tol=0.2)
    run_pair(ccw, ti, 3, 1, 16, 4, (90, 70), 3, score_mode=1, seed=3)


def test_grid_smaller_than_template(ccw):
    ti = configs.ribbon_ti_250()
    run_pair(ccw, ti, 2, 1, 40, 10, (30, 22), 2, n_real=3, seed=8)


def test_no_overlap(ccw):
    """OR = 0: every data event is empty (uniform picks, Algorithm 1 line 6)."""
    ti = configs.ribbon_ti_250()
    run_pair(ccw, ti, 2, 1, 20, 0, (70, 50), 1, seed=2)


def test_3d_four_facies_hard_data(ccw):
    ti = synth.tube_lobe_ti_3d(60, 50, 40, seed=5)
    field = synth.tube_lobe_ti_3d(50, 44, 30, seed=6)
    hd = synth.sample_hard_data(field, 40, seed=7)
    run_pair(ccw, ti, 4, 1, 12, 2, (50, 44, 30), 5, n_real=2, hd=hd, seed=9, path_random=1)


def test_many_realizations_one_call(ccw):
    ti = configs.ribbon_ti_250()
    run_pair(ccw, ti, 2, 2, 32, 8, (100, 84), 4, n_real=6, real_base=100, seed=21)


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_grid_sizes_in_one_batch(ccw, precision):
    """Several grid sizes advance in one batch (ccw_simulate_groups); every
    realization equals the oracle's simulation of its own grid."""
    if precision == 0:
        ti = synth.tube_lobe_ti_3d(60, 50, 40, seed=5)
        F, J, T, Ov, K = 4, 1, 12, 2, 5
        grids = [(50, 44, 30), (30, 26, 22)]
        fields = [synth.tube_lobe_ti_3d(*g, seed=6 + i) for i, g in enumerate(grids)]
    else:
        ti = configs.channel_lens_ti_1000()
        F, J, T, Ov, K = 3, 2, 64, 16, 5
        grids = [(300, 260), (150, 120)]
        fields = [synth.channel_lens_ti(*g, seed=6 + i, tol=0.3) for i, g in enumerate(grids)]
    hds = [synth.sample_hard_data(f, 30, seed=9 + i) for i, f in enumerate(fields)]
    g = ccw.TI(dev(ti), F, J, T, Ov)
    groups = [dict(grid=grids[0], n_real=2, real_base=0, hd_cells=dev(hds[0][0]),
                   hd_vals=dev(hds[0][1])),
              dict(grid=grids[1], n_real=3, real_base=10, hd_cells=dev(hds[1][0]),
                   hd_vals=dev(hds[1][1]))]
    res = ccw.simulate_groups(g, groups, topk=K, seed=4, path_random=1, precision=precision,
                              want_log=True)
    o = O.OracleTI(ti, F, J)
    for gi, (out, log) in enumerate(res):
        out, log = out.cpu().numpy(), log.cpu().numpy()
        for i in range(groups[gi]["n_real"]):
            ref, rlog = o.simulate(grids[gi], T, Ov, K=K, path_random=1, hd_cells=hds[gi][0],
                                   hd_vals=hds[gi][1], seed=4, r=groups[gi]["real_base"] + i)
            assert np.array_equal(log[i], rlog), f"group {gi} realization {i} log"
            assert np.array_equal(out[i], ref), f"group {gi} realization {i}"


@pytest.mark.parametrize("precision,tile", [(0, 0), (2, 0x10020), (1, 0xa020020)])
def test_realization_lanes_give_the_same_simulations(ccw, precision, tile):
    """Realizations split into lanes whose wavefront chains run on separate
    streams (ccf_tile bits 20-22) give exactly the one-lane simulations, in
    one grid size and across two; sampled realizations equal the oracle's."""
    ti = configs.ribbon_ti_250()
    F, J, T, Ov, K = 2, 2, 48, 12, 3
    g = ccw.TI(dev(ti), F, J, T, Ov)
    grids = [(200, 160), (120, 100)]
    groups = [dict(grid=grids[0], n_real=11, real_base=0), dict(grid=grids[1], n_real=5,
                                                                 real_base=20)]
    ref = None
    for lanes in (1, 2, 3, 4, 8):
        res = ccw.simulate_groups(g, groups, topk=K, seed=13, path_random=1, precision=precision,
                                  ccf_tile=tile | ((lanes - 1) << 20), want_log=True)
        got = [(o.cpu().numpy(), lg.cpu().numpy()) for o, lg in res]
        if ref is None:
            ref = got
            continue
        for (o0, l0), (o1, l1) in zip(ref, got):
            assert np.array_equal(l0, l1), lanes
            assert np.array_equal(o0, o1), lanes
    o = O.OracleTI(ti, F, J)
    for gi, i in ((0, 0), (0, 10), (1, 4)):
        out, rlog = o.simulate(grids[gi], T, Ov, K=K, path_random=1, seed=13,
                               r=groups[gi]["real_base"] + i)
        assert np.array_equal(ref[gi][1][i], rlog) and np.array_equal(ref[gi][0][i], out)
