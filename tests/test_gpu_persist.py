"""The one-kernel simulation (ccw_params.ccf_tile bit 30): every wavefront of
a call in one cooperative kernel, bit-exact against the oracle's raster path
(Algorithm 1), plus its refusals and its bounded grid-barrier wait."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from workloads import configs, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PERSIST = 1 << 30


def tile(nt, mt=0):
    return PERSIST | nt | (mt << 16)


@pytest.fixture(scope="module")
def ccw():
    import paper_2404_00441_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check(ccw, ti, F, J, T, Ov, grid, K, n_real=1, real_base=0, hd=None, seed=11,
          path_random=0, score_mode=0, precision=2, ccf_tile=tile(32)):
    g = ccw.TI(dev(ti), F, J, T, Ov)
    hc = hv = None
    if hd is not None:
        hc, hv = dev(hd[0]), dev(hd[1])
    out, log = ccw.simulate(g, grid, n_real=n_real, topk=K, seed=seed, hd_cells=hc, hd_vals=hv,
                            real_base=real_base, path_random=path_random, score_mode=score_mode,
                            want_log=True, precision=precision, ccf_tile=ccf_tile)
    out, log = out.cpu().numpy(), log.cpu().numpy()
    o = O.OracleTI(ti, F, J)
    for i in range(n_real):
        ref, rlog = o.simulate(grid, T, Ov, K=K, score_mode=score_mode, path_random=path_random,
                               hd_cells=None if hd is None else hd[0],
                               hd_vals=None if hd is None else hd[1], seed=seed,
                               r=real_base + i)
        assert np.array_equal(log[i], rlog), f"patch log of realization {i}"
        assert np.array_equal(out[i], ref), f"realization {i}"


@pytest.mark.parametrize("nt", [16, 64])
def test_ribbon_250_full(ccw, nt):
    w = configs.workload("c1")
    check(ccw, w["ti"], w["F"], w["J"], w["T"], w["O"], w["grid"], w["K"], seed=w["seed"],
          ccf_tile=tile(nt))


@pytest.mark.parametrize("precision", [1, 2])
def test_three_facies_hard_data_top5_mirrored(ccw, precision):
    ti = configs.channel_lens_ti_1000()
    field = synth.channel_lens_ti(520, 456, seed=3, tol=0.2)
    hd = synth.sample_hard_data(field, 80, seed=4)
    check(ccw, ti, 3, 2, 64, 16, (520, 456), 5, n_real=2, real_base=7, hd=hd, seed=5,
          path_random=1, precision=precision)


def test_many_realizations_narrow_groups(ccw):
    """More items per wavefront than CTAs: one warp per item in the gather
    and paste phases, several N-tiles per CTA."""
    ti = configs.ribbon_ti_250()
    check(ccw, ti, 2, 2, 32, 8, (100, 84), 4, n_real=96, real_base=100, seed=21,
          ccf_tile=tile(64))


@pytest.mark.parametrize("J,T,Ov", [(0, 15, 5), (1, 16, 4), (3, 32, 8)])
def test_levels_and_odd_template(ccw, J, T, Ov):
    ti = synth.channel_lens_ti(160, 150, seed=2, tol=0.2)
    field = synth.channel_lens_ti(90, 77, seed=5, tol=0.3)
    hd = synth.sample_hard_data(field, 25, seed=6)
    check(ccw, ti, 3, J, T, Ov, (90, 77), 3, n_real=2, hd=hd, seed=3, path_random=1)


def test_literal_score(ccw):
    ti = synth.channel_lens_ti(200, 180, seed=2, tol=0.2)
    check(ccw, ti, 3, 1, 16, 4, (90, 70), 3, score_mode=1, seed=3, precision=1)


def test_empty_events_only(ccw):
    """Grids smaller than the template and no overlap: every data event is
    empty (uniform draws, Algorithm 1 line 6)."""
    ti = configs.ribbon_ti_250()
    check(ccw, ti, 2, 1, 40, 10, (30, 22), 2, n_real=3, seed=8)
    check(ccw, ti, 2, 1, 20, 0, (70, 50), 1, seed=2)


def test_mixed_grid_sizes(ccw):
    ti = configs.channel_lens_ti_1000()
    F, J, T, Ov, K = 3, 2, 64, 16, 5
    grids = [(300, 260), (150, 120)]
    fields = [synth.channel_lens_ti(*gr, seed=6 + i, tol=0.3) for i, gr in enumerate(grids)]
    hds = [synth.sample_hard_data(f, 30, seed=9 + i) for i, f in enumerate(fields)]
    g = ccw.TI(dev(ti), F, J, T, Ov)
    groups = [dict(grid=grids[0], n_real=2, real_base=0, hd_cells=dev(hds[0][0]),
                   hd_vals=dev(hds[0][1])),
              dict(grid=grids[1], n_real=3, real_base=10, hd_cells=dev(hds[1][0]),
                   hd_vals=dev(hds[1][1]))]
    res = ccw.simulate_groups(g, groups, topk=K, seed=4, path_random=1, precision=2,
                              ccf_tile=tile(32), want_log=True)
    o = O.OracleTI(ti, F, J)
    for gi, (out, log) in enumerate(res):
        out, log = out.cpu().numpy(), log.cpu().numpy()
        for i in range(groups[gi]["n_real"]):
            ref, rlog = o.simulate(grids[gi], T, Ov, K=K, path_random=1, hd_cells=hds[gi][0],
                                   hd_vals=hds[gi][1], seed=4, r=groups[gi]["real_base"] + i)
            assert np.array_equal(log[i], rlog), f"group {gi} realization {i} log"
            assert np.array_equal(out[i], ref), f"group {gi} realization {i}"


def test_refusals(ccw):
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 1, 40, 10)
    for kw in (dict(vt_ext=4), dict(boundary_cut=1), dict(topk=9)):
        args = dict(n_real=1, topk=2, seed=1, precision=2, ccf_tile=tile(32))
        args.update(kw)
        with pytest.raises(ccw.CCWError):
            ccw.simulate(g, (120, 100), **args)
    with pytest.raises(ccw.CCWError):   # FP32 lanes have no persistent form
        ccw.simulate(g, (120, 100), n_real=1, topk=1, precision=0, ccf_tile=tile(32))


def test_barrier_timeout_is_reported_and_the_next_call_is_clean(ccw):
    """A grid-barrier wait limited to one poll gives up: the call returns
    CCW_ETIMEOUT (the kernel records it, stops every CTA at its next barrier,
    waits for its own copies and frees its tensor memory); with the default
    limit restored the next call is exact."""
    lib = ccw.load()
    lib.ccw_set_barrier_polls.argtypes = [C.c_int64]
    w = configs.workload("c1")
    g = ccw.TI(dev(w["ti"]), w["F"], w["J"], w["T"], w["O"])
    assert lib.ccw_set_barrier_polls(1) == 0
    try:
        with pytest.raises(ccw.CCWError) as ei:
            ccw.simulate(g, w["grid"], n_real=4, topk=1, seed=w["seed"], precision=2,
                         ccf_tile=tile(16))
        assert "error -4" in str(ei.value)
    finally:
        assert lib.ccw_set_barrier_polls(0) == 0
    torch.cuda.synchronize()
    check(ccw, w["ti"], w["F"], w["J"], w["T"], w["O"], w["grid"], w["K"], seed=w["seed"],
          ccf_tile=tile(16))
