"""GPU parity, against the CPU oracle, of the two variants of the search-and-
paste step:

- non-causal conditioning (Sec. 4.4): the hard data of a virtual template,
  the window grown by ``vt_ext`` cells along the forward directions of the
  path, join every candidate's mismatch count;
- the minimum-error boundary cut of image quilting (Sec. 2) at paste.

Realizations and patch logs must be identical, on the FP32 lanes and on the
tensor cores (resident and streamed operands).
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


def run_pair(ccw, ti, F, J, T, Ov, grid, K, hd=None, n_real=2, real_base=0, seed=11,
             path_random=1, vt=0, cut=0, precision=0, ccf_tile=0):
    g = ccw.TI(dev(ti), F, J, T, Ov)
    hc = hv = None
    if hd is not None:
        hc, hv = dev(hd[0]), dev(hd[1])
    out, log = ccw.simulate(g, grid, n_real=n_real, topk=K, seed=seed, hd_cells=hc,
                            hd_vals=hv, real_base=real_base, path_random=path_random,
                            precision=precision, want_log=True, ccf_tile=ccf_tile, vt_ext=vt,
                            boundary_cut=cut)
    out, log = out.cpu().numpy(), log.cpu().numpy()
    o = O.OracleTI(ti, F, J)
    for i in range(n_real):
        ref, rlog = o.simulate(grid, T, Ov, K=K, path_random=path_random,
                               hd_cells=None if hd is None else hd[0],
                               hd_vals=None if hd is None else hd[1], seed=seed,
                               r=real_base + i, vt_ext=vt, cut=cut)
        assert np.array_equal(log[i], rlog), f"patch log of realization {i}"
        assert np.array_equal(out[i], ref), f"realization {i}"
    return out, log


def _hd_2d(nx, ny, n, seed):
    field = synth.channel_lens_ti(nx, ny, seed=seed, tol=0.2)
    return synth.sample_hard_data(field, n, seed=seed + 1)


# streamed tensor-core operands: 16 events per N-tile, one M-tile, bit 25
STREAMED_2D = 16 | (1 << 16) | (2 << 24)


@pytest.mark.parametrize("precision,tile", [(0, 0), (2, 0), (2, STREAMED_2D), (1, 1 << 24 | 32 | 1 << 16)])
@pytest.mark.parametrize("vt", [4, 16])
def test_virtual_template_2d(ccw, precision, tile, vt):
    """Dense hard data, mirrored paths, K = 3: the virtual data change the
    picks and both sides count them alike, including data whose TI position
    falls outside the TI."""
    ti = synth.channel_lens_ti(200, 180, seed=2, tol=0.2)
    hd = _hd_2d(120, 100, 150, 3)
    _, log = run_pair(ccw, ti, 3, 1, 16, 4, (120, 100), 3, hd=hd, real_base=3, seed=5, vt=vt,
                      precision=precision, ccf_tile=tile)
    # the variant is not a no-op on this input
    o = O.OracleTI(ti, 3, 1)
    _, plain = o.simulate((120, 100), 16, 4, K=3, path_random=1, hd_cells=hd[0],
                          hd_vals=hd[1], seed=5, r=3)
    assert not np.array_equal(log[0], plain)


@pytest.mark.parametrize("precision", [0, 1])
def test_virtual_template_3d(ccw, precision):
    ti = synth.tube_lobe_ti_3d(48, 40, 36, seed=5)
    field = synth.tube_lobe_ti_3d(24, 20, 16, seed=6)
    hd = synth.sample_hard_data(field, 60, seed=7)
    run_pair(ccw, ti, 4, 1, 8, 2, (24, 20, 16), 3, hd=hd, seed=9, vt=4, precision=precision)


@pytest.mark.parametrize("J,T,Ov", [(0, 12, 4), (1, 16, 4), (2, 32, 8)])
@pytest.mark.parametrize("precision", [0, 2])
def test_boundary_cut_2d(ccw, J, T, Ov, precision):
    """Boundary-cut paste on mirrored paths, without and with hard data."""
    ti = synth.ribbon_ti(160, 150, n_ribbons=7, seed=4, target=0.3, tol=0.2)
    out, _ = run_pair(ccw, ti, 2, J, T, Ov, (100, 90), 2, n_real=3, seed=6, cut=1,
                      precision=precision)
    hd = _hd_2d(100, 90, 40, 8)
    hd = (hd[0], np.minimum(hd[1], 1).astype(np.uint8))
    run_pair(ccw, ti, 2, J, T, Ov, (100, 90), 2, hd=hd, n_real=2, seed=7, cut=1,
             precision=precision)


def test_cut_and_virtual_template_c2_geometry(ccw):
    """Both variants at the three-facies geometry (T64 / OR16 / J2, K = 5,
    hard data) on the BF16 tensor cores."""
    ti = configs.channel_lens_ti_1000()
    hd = _hd_2d(232, 200, 60, 11)
    run_pair(ccw, ti, 3, 2, 64, 16, (232, 200), 5, hd=hd, real_base=1, seed=4, vt=16, cut=1,
             precision=2)


def test_variants_are_refused_outside_their_range(ccw):
    ti2 = dev(synth.ribbon_ti(300, 300, n_ribbons=7, seed=4, target=0.3, tol=0.2))
    g = ccw.TI(ti2, 2, 1, 16, 4)
    with pytest.raises(ccw.CCWError):
        ccw.simulate(g, (40, 40), vt_ext=17)
    with pytest.raises(ccw.CCWError):
        ccw.simulate(g, (40, 40), vt_ext=-1)
    with pytest.raises(ccw.CCWError):
        ccw.simulate(g, (40, 40), boundary_cut=2)
    big = ccw.TI(ti2, 2, 3, 136, 32)    # templates above 128 cells have no cut
    with pytest.raises(ccw.CCWError):
        ccw.simulate(big, (300, 300), boundary_cut=1)
    ti3 = dev(synth.tube_lobe_ti_3d(32, 32, 32, seed=5))
    g3 = ccw.TI(ti3, 4, 1, 8, 2)
    with pytest.raises(ccw.CCWError):
        ccw.simulate(g3, (16, 16, 16), boundary_cut=1)
