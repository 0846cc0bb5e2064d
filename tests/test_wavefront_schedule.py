"""The CUDA path runs the patches of one wavefront w = i_x + 2 i_y (+ 4 i_z)
together. With T >= 2 OR this gives exactly the raster-order result of
Algorithm 1: patches of one wavefront never share a cell, and every patch
that shares a cell with patch p comes before p in both orders. Checked here
on the CPU with the oracle's own search and reconstruction steps driven in
wavefront order (2D and 3D, forward and mirrored paths), which also pins the
oracle's loop of Algorithm 1 (window placement, data event, paste, crop)
against a restatement of it."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from workloads import synth


def wave_of(ip):
    return ip[0] + 2 * ip[1] + (4 * ip[2] if len(ip) > 2 else 0)


@pytest.mark.parametrize("T,Ov", [(16, 4), (16, 8), (24, 6), (12, 2)])
@pytest.mark.parametrize("d", [2, 3])
def test_wavefront_dependencies(T, Ov, d):
    S = T - Ov
    n = (5, 4, 3)[:d]
    pats = list(itertools.product(*[range(k) for k in n]))
    def overlap(a, b):
        return all(abs(x - y) * S < T for x, y in zip(a, b))
    def raster(ip):
        idx = 0
        for ax in reversed(range(d)):
            idx = idx * n[ax] + ip[ax]
        return idx
    for a in pats:
        for b in pats:
            if a == b or not overlap(a, b):
                continue
            assert wave_of(a) != wave_of(b)
            assert (raster(a) < raster(b)) == (wave_of(a) < wave_of(b))


def test_wavefront_driver_equals_raster_simulation():
    ti = synth.channel_lens_ti(160, 150, seed=2, tol=0.2)
    F, J, T, Ov, K = 3, 1, 16, 4, 3
    grid = (75, 61)
    cells, vals = synth.sample_hard_data(synth.channel_lens_ti(75, 61, seed=3, tol=0.3), 20, 4)
    o = O.OracleTI(ti, F, J)
    seed, r = 17, 2
    ref, rlog = o.simulate(grid, T, Ov, K=K, hd_cells=cells, hd_vals=vals, seed=seed, r=r)
    npch, gp = O.lattice(2, grid, T, Ov)
    S = T - Ov
    hd = np.full((gp[1], gp[0]), 255, np.uint8)
    hd[cells[:, 1], cells[:, 0]] = vals
    sg = np.full((gp[1], gp[0]), 255, np.uint8)
    order = sorted(range(npch[0] * npch[1]),
                   key=lambda p: (wave_of((p % npch[0], p // npch[0])), p))
    order = order[::-1]                          # reversed inside each wave too
    order = sorted(order, key=lambda p: wave_of((p % npch[0], p // npch[0])))
    for p in order:
        iy, ix = divmod(p, npch[0])
        win = (slice(S * iy, S * iy + T), slice(S * ix, S * ix + T))
        hw = hd[win]
        de = np.where(hw != 255, hw, sg[win])
        res = o.search(T, de, hw, K=K, seed=seed, r=r, p=p)
        assert res["pick"] == rlog[p, 0]
        sg[win] = np.where(hw != 255, hw, o.reconstruct(T, res["pick"]))
    assert np.array_equal(sg[:grid[1], :grid[0]], ref)


@pytest.mark.parametrize("cut", [0, 1])
def test_rows_before_the_next_patch_row_are_final_2d(cut):
    """The host read-back copies output rows y < (i + 1)(T - OR) as soon as
    patch row i is pasted: no later patch, boundary cut included, writes
    them. Checked in raster order on the oracle (the wavefront order reaches
    the same states, test above): the realization after the first i + 1
    patch rows agrees there with the finished one."""
    ti = synth.ribbon_ti(120, 110, n_ribbons=6, seed=4)
    T, Ov = 16, 4
    S = T - Ov
    grid = (95, 83)
    o = O.OracleTI(ti, 2, 1)
    npch, _ = O.lattice(2, grid, T, Ov)
    full, _ = o.simulate(grid, T, Ov, K=2, seed=5, r=1, cut=cut)
    for i in range(npch[1] - 1):
        part, _ = o.simulate(grid, T, Ov, K=2, seed=5, r=1, cut=cut,
                             max_patches=(i + 1) * npch[0])
        y1 = min(grid[1], (i + 1) * S)
        assert np.array_equal(part[:y1], full[:y1]), i
        # and the next rows are not final yet: the next patch row writes them
        assert not np.array_equal(part[y1:], full[y1:]), i


def test_slabs_before_the_next_patch_slab_are_final_3d():
    """The same in 3D along z: after patch slab i the cells z < (i + 1)(T - OR)
    are final."""
    ti = synth.tube_lobe_ti_3d(40, 36, 32, seed=5)
    T, Ov = 8, 2
    S = T - Ov
    grid = (26, 24, 22)
    o = O.OracleTI(ti, 4, 1)
    npch, _ = O.lattice(3, grid, T, Ov)
    full, _ = o.simulate(grid, T, Ov, K=3, seed=9, r=0)
    per_slab = npch[0] * npch[1]
    for i in range(npch[2] - 1):
        part, _ = o.simulate(grid, T, Ov, K=3, seed=9, r=0, max_patches=(i + 1) * per_slab)
        z1 = min(grid[2], (i + 1) * S)
        assert np.array_equal(part[:z1], full[:z1]), i


def drive_in_wavefronts(o, grid, T, Ov, K, cells, vals, seed, r, flips):
    """Algorithm 1 restated with the oracle's search and reconstruction
    steps, patches in wavefront order (reversed inside each wave), on a path
    mirrored along the axes set in `flips`: the grid sits at the high end of
    the padded lattice along a mirrored axis, whose patch origins run from
    the high end down; the patterns themselves are not mirrored. Returns the
    cropped realization."""
    d = len(grid)
    npch, gp = O.lattice(d, grid, T, Ov)
    S = T - Ov
    off = [gp[a] - grid[a] if flips >> a & 1 else 0 for a in range(d)]
    shape = tuple(gp[a] for a in reversed(range(d)))
    hd = np.full(shape, 255, np.uint8)
    for c, v in zip(cells, vals):
        idx = tuple(c[a] + off[a] for a in reversed(range(d)))
        hd[idx] = min(hd[idx], v)
    sg = np.full(shape, 255, np.uint8)
    pats = list(itertools.product(*[range(npch[a]) for a in reversed(range(d))]))
    ips = [tuple(reversed(q)) for q in pats]              # (ix, iy[, iz])
    def raster(ip):
        idx = 0
        for a in reversed(range(d)):
            idx = idx * npch[a] + ip[a]
        return idx
    order = sorted(ips, key=lambda ip: (wave_of(ip), -raster(ip)))
    for ip in order:
        p = raster(ip)
        org = [gp[a] - T - S * ip[a] if flips >> a & 1 else S * ip[a] for a in range(d)]
        win = tuple(slice(org[a], org[a] + T) for a in reversed(range(d)))
        hw = hd[win]
        de = np.where(hw != 255, hw, sg[win])
        res = o.search(T, de, hw, K=K, seed=seed, r=r, p=p)
        sg[win] = np.where(hw != 255, hw, o.reconstruct(T, res["pick"]))
    crop = tuple(slice(off[a], off[a] + grid[a]) for a in reversed(range(d)))
    return sg[crop]


def test_wavefront_driver_equals_raster_simulation_mirrored():
    """Mirrored paths (path_random = 1): each of the three non-trivial flips
    of a 2D path, hard data included."""
    ti = synth.channel_lens_ti(160, 150, seed=2, tol=0.2)
    F, J, T, Ov, K = 3, 1, 16, 4, 3
    grid = (75, 61)
    cells, vals = synth.sample_hard_data(synth.channel_lens_ti(75, 61, seed=3, tol=0.3), 20, 4)
    o = O.OracleTI(ti, F, J)
    seed = 23
    seen = set()
    for r in range(64):
        flips = O.path_flips(2, seed, r)
        if flips == 0 or flips in seen:
            continue
        seen.add(flips)
        ref, _ = o.simulate(grid, T, Ov, K=K, path_random=1, hd_cells=cells, hd_vals=vals,
                            seed=seed, r=r)
        got = drive_in_wavefronts(o, grid, T, Ov, K, cells, vals, seed, r, flips)
        assert np.array_equal(got, ref), (r, flips)
    assert seen == {1, 2, 3}


def test_wavefront_driver_equals_raster_simulation_3d():
    """3D (w = i_x + 2 i_y + 4 i_z), forward and one mirrored path, hard
    data included."""
    ti = synth.tube_lobe_ti_3d(36, 32, 30, seed=5)
    F, J, T, Ov, K = 4, 1, 8, 2, 3
    grid = (22, 20, 18)
    cells, vals = synth.sample_hard_data(synth.tube_lobe_ti_3d(22, 20, 18, seed=6), 25, 7)
    o = O.OracleTI(ti, F, J)
    seed = 31
    ref, _ = o.simulate(grid, T, Ov, K=K, hd_cells=cells, hd_vals=vals, seed=seed, r=0)
    got = drive_in_wavefronts(o, grid, T, Ov, K, cells, vals, seed, 0, 0)
    assert np.array_equal(got, ref)
    r = next(r for r in range(64) if O.path_flips(3, seed, r) == 7)
    ref, _ = o.simulate(grid, T, Ov, K=K, path_random=1, hd_cells=cells, hd_vals=vals,
                        seed=seed, r=r)
    got = drive_in_wavefronts(o, grid, T, Ov, K, cells, vals, seed, r, 7)
    assert np.array_equal(got, ref)
