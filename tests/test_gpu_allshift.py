"""All-shift (polyphase) candidates on the GPU (ccw_params.all_shift): every
fine origin of the cropped TI is a candidate (the undecimated reading of
Sec. 3.2); the library searches the s^2 phases of the TI's level-J planes
with the tensor-core CCF and pastes TI crops. Realizations and patch logs
(fine candidate indices) must equal the oracle's all-shift simulation."""
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
    # name, F, J, T, O, grid, K, n_hd, vt_ext, precision, tile
    ("ribbon_j1", 2, 1, 16, 4, (70, 58), 3, 0, 0, 2, 0),
    ("facies3_j2_hd", 3, 2, 16, 4, (90, 77), 5, 25, 0, 2, 0),
    ("facies3_j2_fp16_lanes", 3, 2, 16, 4, (90, 77), 5, 25, 0, 1, 1 << 20),
    ("facies3_j1_lane_epilogue", 3, 1, 12, 2, (60, 50), 12, 10, 0, 2, 0x1010010),
    ("facies3_j2_virtual", 3, 2, 16, 4, (90, 77), 3, 40, 8, 2, 0),
    ("facies3_j3", 3, 3, 32, 8, (100, 90), 2, 15, 0, 2, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_allshift_simulation_matches_oracle(ccw, case):
    name, F, J, T, Ov, grid, K, n_hd, vt_ext, precision, tile = case
    if F == 2:
        ti = synth.ribbon_ti(120, 110, n_ribbons=6, seed=4, target=0.3, tol=0.2)
    else:
        ti = synth.channel_lens_ti(150, 140, seed=2, tol=0.2)
    hd = None
    if n_hd:
        field = synth.channel_lens_ti(grid[0], grid[1], seed=5, tol=0.3) if F == 3 else \
            synth.ribbon_ti(grid[0], grid[1], n_ribbons=4, seed=5, target=0.3, tol=0.3)
        hd = synth.sample_hard_data(field, n_hd, seed=6)
    g = ccw.TI(dev(ti), F, J, T, Ov)
    out, log = ccw.simulate(g, grid, n_real=2, topk=K, seed=17, real_base=3, path_random=1,
                            hd_cells=None if hd is None else dev(hd[0]),
                            hd_vals=None if hd is None else dev(hd[1]), want_log=True,
                            precision=precision, ccf_tile=tile, vt_ext=vt_ext, all_shift=1)
    out, log = out.cpu().numpy(), log.cpu().numpy()
    o = O.OracleTI(ti, F, J)
    for i in range(2):
        ref, rlog = o.simulate(grid, T, Ov, K=K, path_random=1, seed=17, r=3 + i,
                               hd_cells=None if hd is None else hd[0],
                               hd_vals=None if hd is None else hd[1], vt_ext=vt_ext,
                               all_shift=1)
        assert np.array_equal(log[i], rlog), f"{name}: patch log of realization {i}"
        assert np.array_equal(out[i], ref), f"{name}: realization {i}"


def test_allshift_refusals(ccw):
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 1, 16, 4)
    for kw in (dict(precision=0), dict(precision=2, ccf_tile=0x2010010),
               dict(precision=2, boundary_cut=1), dict(precision=2, ccf_tile=(1 << 30) | 32)):
        with pytest.raises(ccw.CCWError):
            ccw.simulate(g, (60, 50), n_real=1, topk=2, seed=1, all_shift=1, **kw)
