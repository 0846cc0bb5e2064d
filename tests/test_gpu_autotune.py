"""Every CCF tiling the autotuner may pick gives identical simulations (the
arithmetic is exact in all of them), and the tuner returns one of them."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("ndim", [2, 3])
def test_all_tilings_agree_and_tuner_picks_one(ccw, ndim, tmp_path, monkeypatch):
    from paper_2404_00441_gb300 import autotune
    monkeypatch.setenv("CCW_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    if ndim == 2:
        ti = configs.channel_lens_ti_1000()[:400, :400].copy()
        F, J, T, O, K = 3, 2, 32, 8, 5
        grids = [(200, 180), (96, 80)]
        field = synth.channel_lens_ti(200, 180, seed=3, tol=0.3)
    else:
        ti = synth.tube_lobe_ti_3d(60, 50, 40, seed=5)
        F, J, T, O, K = 4, 1, 12, 2, 3
        grids = [(40, 36, 24), (30, 26, 22)]
        field = synth.tube_lobe_ti_3d(40, 36, 24, seed=6)
    cells, vals = synth.sample_hard_data(field, 25, seed=4)
    g = ccw.TI(dev(ti), F, J, T, O)
    groups = [dict(grid=grids[0], n_real=3, real_base=0, hd_cells=dev(cells), hd_vals=dev(vals)),
              dict(grid=grids[1], n_real=2, real_base=5)]
    ref = None
    cands = autotune.candidates(g, (0, 1, 2) if ndim == 2 else (0,))
    ran = 0
    for prec, tile in cands:
        try:
            res = ccw.simulate_groups(g, groups, topk=K, seed=7, path_random=1, precision=prec,
                                      ccf_tile=tile, want_log=True)
        except ccw.CCWError:
            continue   # refused (shared memory or exactness bound)
        ran += 1
        got = [(o.cpu().numpy(), l.cpu().numpy()) for o, l in res]
        if ref is None:
            ref = got
            continue
        for (o0, l0), (o1, l1) in zip(ref, got):
            assert np.array_equal(l0, l1), (prec, hex(tile))
            assert np.array_equal(o0, o1), (prec, hex(tile))
    assert ran >= 3
    prec, tile, times = autotune.tune(g, groups, topk=K, seed=7,
                                      precisions=(0, 1, 2) if ndim == 2 else (0,))
    assert (prec, tile & ~(7 << 20)) in cands and len(times) >= ran
    # cached
    assert autotune.tune(g, groups, topk=K, seed=7,
                         precisions=(0, 1, 2) if ndim == 2 else (0,))[:2] == (prec, tile)
    with pytest.raises(ccw.CCWError):
        ccw.simulate_groups(g, groups, topk=K, seed=7, precision=0, ccf_tile=3)
