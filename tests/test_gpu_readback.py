"""Host read-back of ccw_simulate_groups (out_host).

With page-locked host buffers and unmirrored paths the library copies each
band of output rows to the host inside the captured graph, as soon as the
last patch row over it is pasted; otherwise it copies after the crop. Either
way the host buffer must hold exactly the device output, which must be the
same as a call without a host buffer (and, for one realization, the
oracle's).
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


def host(shape, pinned=True):
    t = torch.full(shape, 77, dtype=torch.uint8)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("lanes_tile", [0, 0x100000])
@pytest.mark.parametrize("pinned", [True, False])
def test_2d_read_back_equals_device_output(ccw, lanes_tile, pinned):
    """Ribbon TI, 5 realizations of 200 x 150 (T40/OR10/J1, K 3), one or two
    realization lanes; the second call reuses the buffers, the third brings
    new ones (the streamed graph is built again)."""
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 1, 40, 10)
    grid, n_real, seed = (200, 150), 5, 31
    shape = (n_real, 150, 200)
    ref, _ = ccw.simulate(g, grid, n_real=n_real, topk=3, seed=seed, precision=2,
                          ccf_tile=lanes_tile)
    ref = ref.cpu().numpy()
    want0, _ = O.OracleTI(ti, 2, 1).simulate(grid, 40, 10, K=3, seed=seed, r=0)
    assert np.array_equal(ref[0], want0)
    out = torch.empty(shape, dtype=torch.uint8, device="cuda")
    for call in range(3):
        h = host(shape, pinned)
        if call == 2:
            out = torch.empty(shape, dtype=torch.uint8, device="cuda")
        ccw.simulate(g, grid, n_real=n_real, topk=3, seed=seed, precision=2,
                     ccf_tile=lanes_tile, out=out, out_host=h)
        assert np.array_equal(h.numpy(), ref), f"call {call}: host copy"
        assert np.array_equal(out.cpu().numpy(), ref), f"call {call}: device output"


def test_2d_mirrored_paths_copy_after_the_crop(ccw):
    """path_random = 1: every realization mirrors its own axes, so the copy
    runs after the crop; the host buffer still equals the device output."""
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 1, 40, 10)
    grid, n_real = (180, 130), 4
    ref, _ = ccw.simulate(g, grid, n_real=n_real, topk=1, seed=5, path_random=1, precision=2)
    h = host((n_real, 130, 180))
    ccw.simulate(g, grid, n_real=n_real, topk=1, seed=5, path_random=1, precision=2, out_host=h)
    assert np.array_equal(h.numpy(), ref.cpu().numpy())


def test_3d_groups_with_hard_data_read_back(ccw):
    """3D 4-facies TI, two grid sizes in one call with hard data (T24/OR6/J1,
    K 5), bands along z; the first group is copied to the host, the second
    is not."""
    ti = configs.tube_ti_3d()
    g = ccw.TI(dev(ti), 4, 1, 24, 6)
    field = synth.tube_lobe_ti_3d(56, 44, 40, seed=6)
    cells, vals = synth.sample_hard_data(field, 60, seed=3)
    specs = [dict(grid=(56, 44, 40), n_real=3, real_base=0,
                  hd_cells=dev(cells), hd_vals=dev(vals)),
             dict(grid=(30, 30, 24), n_real=2, real_base=3)]
    ref = ccw.simulate_groups(g, specs, topk=5, seed=9, precision=1)
    ref = [r[0].cpu().numpy() for r in ref]
    h = host((3, 40, 44, 56))
    specs2 = [dict(specs[0], out_host=h), specs[1]]
    for _ in range(2):
        h.fill_(77)
        res = ccw.simulate_groups(g, specs2, topk=5, seed=9, precision=1)
        assert np.array_equal(h.numpy(), ref[0])
        assert np.array_equal(res[0][0].cpu().numpy(), ref[0])
        assert np.array_equal(res[1][0].cpu().numpy(), ref[1])


def test_bad_host_buffer_is_rejected(ccw):
    ti = configs.ribbon_ti_250()
    g = ccw.TI(dev(ti), 2, 1, 40, 10)
    with pytest.raises(ValueError):
        ccw.simulate(g, (100, 100), n_real=2,
                     out_host=torch.empty((2, 100, 99), dtype=torch.uint8))
