"""Pins of the oracle's two extensions of the paste-and-search loop:

- the minimum-error boundary cut of image quilting (Efros and Freeman; the
  IQ method the paper reviews in Sec. 2), used as an alternative paste;
- the non-causal conditioning of Sec. 4.4: hard data in a virtual template
  (the template grown along the forward directions of the path) join the
  mismatch count.

Expected values come from brute force over all cut paths, from a search
with a larger template on a padded training image, and from hand-placed
hard data. CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from workloads import synth


# ------------------------------------------------------- boundary cut pins --
def _all_paths(rows, cols):
    """Every column sequence with steps of at most one column."""
    paths = [[c] for c in range(cols)]
    for _ in range(rows - 1):
        paths = [p + [c] for p in paths for c in (p[-1] - 1, p[-1], p[-1] + 1)
                 if 0 <= c < cols]
    return paths


def _brute_cut(err):
    """The cheapest path; among equal costs the one whose columns, read from
    the last row up, are lexicographically smallest."""
    rows, cols = err.shape
    paths = _all_paths(rows, cols)
    cost = [sum(int(err[y, p[y]]) for y in range(rows)) for p in paths]
    best = min(cost)
    return min((p for p, c in zip(paths, cost) if c == best), key=lambda p: p[::-1])


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 4), (5, 1), (4, 2), (6, 3), (7, 4), (8, 4)])
def test_min_cut_equals_brute_force(rows, cols):
    """The dynamic program returns the cheapest 8-connected top-to-bottom
    path, ties resolved towards lower columns from the bottom row up."""
    rng = np.random.default_rng(100 * rows + cols)
    for p_one in (0.2, 0.5, 0.8):
        for _ in range(12):
            err = (rng.random((rows, cols)) < p_one).astype(np.uint8)
            assert list(O.min_cut(err)) == _brute_cut(err)


def test_min_cut_closed_forms():
    """No disagreement: the cut hugs column 0 (the whole strip takes the new
    pattern). One clean column among disagreeing ones: the cut follows it."""
    assert list(O.min_cut(np.zeros((9, 5), np.uint8))) == [0] * 9
    err = np.ones((9, 5), np.uint8)
    err[:, 3] = 0
    assert list(O.min_cut(err)) == [3] * 9


def _quilt(old, new, Ov, flips):
    """Reference paste of one 2D window through the boundary cuts, written
    from the definition: path frame = window mirrored along flipped axes;
    costs 1 where the grid already holds a value that differs from the
    pattern; a simulated cell takes the pattern only on the far side of both
    the column cut of the left strip and the row cut of the top strip."""
    fo, fn = old.copy(), new.copy()
    if flips & 1:
        fo, fn = fo[:, ::-1], fn[:, ::-1]
    if flips & 2:
        fo, fn = fo[::-1, :], fn[::-1, :]
    T = fo.shape[0]
    err = ((fo != O.UNKNOWN) & (fo != fn)).astype(np.uint8)   # [y', x']
    cv = _brute_cut(err[:, :Ov])          # column of the cut in each row y'
    ch = _brute_cut(err[:Ov, :].T)        # row of the cut in each column x'
    yp, xp = np.mgrid[0:T, 0:T]
    take = (fo == O.UNKNOWN) | ((xp >= np.asarray(cv)[yp]) & (yp >= np.asarray(ch)[xp]))
    out = np.where(take, fn, fo)
    if flips & 2:
        out = out[::-1, :]
    if flips & 1:
        out = out[:, ::-1]
    return out


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("flip", [0, 1])
def test_two_patch_quilt_matches_definition(axis, flip):
    """Two patches side by side (or one above the other): the second is
    pasted through the boundary cuts against the first, in the path frame of
    the realization (mirrored when the path runs backwards)."""
    ti = synth.ribbon_ti(64, 64, n_ribbons=5, seed=7, target=0.3, tol=0.2)
    t = O.OracleTI(ti, 2, 1)
    T, Ov, S = 8, 4, 4
    grid = (T + S, T) if axis == 0 else (T, T + S)
    seed = 5
    rs = [r for r in range(64) if O.path_flips(2, seed, r, 1) >> axis & 1 == flip]
    nontrivial = 0
    for r in rs[:10]:
        out, log = t.simulate(grid, T, Ov, K=4, path_random=1, seed=seed, r=r, cut=1)
        flips = O.path_flips(2, seed, r, 1)
        sg = np.full(out.shape, O.UNKNOWN, np.uint8)   # [y, x]
        for p in range(2):
            pat = t.reconstruct(T, int(log[p, 0]))
            i = [0, 0]
            i[axis] = p
            org = []
            for a in range(2):
                n = grid[a]
                org.append(n - T - S * i[a] if flips >> a & 1 else S * i[a])
            win = (slice(org[1], org[1] + T), slice(org[0], org[0] + T))
            before = sg[win].copy()
            sg[win] = _quilt(before, pat, Ov, flips)
            if p == 1:
                nontrivial += int(np.any((sg[win] != pat) & (before != O.UNKNOWN)))
        assert np.array_equal(out, sg)
    assert nontrivial > 0   # some cut kept cells of the first patch


def test_cut_without_overlap_or_conflict_is_plain_paste():
    """With no overlap there is nothing to cut, so cut = 1 equals the full
    paste; the same holds for a single-facies training image, whose patterns
    never disagree."""
    ti = synth.ribbon_ti(80, 80, n_ribbons=5, seed=8, target=0.3, tol=0.2)
    t = O.OracleTI(ti, 2, 1)
    a, la = t.simulate((40, 36), 8, 0, K=3, seed=2, cut=0)
    b, lb = t.simulate((40, 36), 8, 0, K=3, seed=2, cut=1)
    assert np.array_equal(a, b) and np.array_equal(la, lb)
    t0 = O.OracleTI(np.zeros((40, 40), np.uint8), 2, 1)
    a, la = t0.simulate((30, 30), 8, 2, K=3, seed=2, cut=0)
    b, lb = t0.simulate((30, 30), 8, 2, K=3, seed=2, cut=1)
    assert np.array_equal(a, b) and np.array_equal(la, lb)


def test_cut_is_two_dimensional():
    t = O.OracleTI(np.zeros((16, 16, 16), np.uint8), 2, 0)
    with pytest.raises(ValueError):
        t.simulate((8, 8, 8), 4, 2, cut=1)


# ----------------------------------------------------- virtual template pins --
@pytest.mark.parametrize("d,J,T,E", [(2, 0, 6, 3), (2, 1, 8, 4), (3, 0, 4, 2), (3, 1, 4, 2)])
@pytest.mark.parametrize("side", ["high", "low"])
def test_virtual_mismatch_equals_padded_larger_template(d, J, T, E, side):
    """A hard datum of the virtual template at offset q counts like an
    in-template datum of a template grown to T + E: on the training image
    padded by E cells with a code no datum has, the grown template's
    mismatch map over the same candidates equals the virtual one, the
    padding standing for positions outside the training image."""
    s, F = 2 ** J, 3
    rng = np.random.default_rng(17 * d + 5 * J + (side == "low"))
    n = 24 if d == 2 else 12
    ti = rng.integers(0, F, size=(n,) * d).astype(np.uint8)
    t = O.OracleTI(ti, F, J)
    # virtual data: offsets of the grown window outside the template
    lo, hi = (0, T + E) if side == "high" else (-E, T)
    vhd = []
    while len(vhd) < 6:
        q = [int(v) for v in rng.integers(lo, hi, size=d)]
        if all(0 <= v < T for v in q) or any(w[:d] == q for w in vhd):
            continue
        vhd.append(q + [0] * (3 - d) + [int(rng.integers(0, F))])
    de = np.full((T,) * d, O.UNKNOWN, np.uint8)
    de.flat[int(rng.integers(0, de.size))] = 1          # one known cell
    res = t.search(T, de, K=2, maps=True, vhd=vhd)
    # the padded image, code F outside the original
    tip = np.full((n + E,) * d, F, np.uint8)
    core = tuple(slice(0, n) if side == "high" else slice(E, E + n) for _ in range(d))
    tip[core] = ti
    tp = O.OracleTI(tip, F + 1, J)
    Tp, sh = T + E, (0 if side == "high" else E)
    de2 = np.full((Tp,) * d, O.UNKNOWN, np.uint8)
    de2[tuple(slice(sh, sh + T) for _ in range(d))] = de
    hd2 = np.full((Tp,) * d, O.UNKNOWN, np.uint8)
    for v in vhd:
        idx = tuple(v[a] + sh for a in range(d))[::-1]   # numpy order z, y, x
        hd2[idx] = v[3]
    res2 = tp.search(Tp, de2, hd=hd2, K=2, maps=True)
    assert tp.cand_shape(Tp) == t.cand_shape(T)
    assert np.array_equal(res["mis"], res2["mis"])
    assert res["mis"].max() > 0


@pytest.mark.parametrize("path_random,r", [(0, 0), (1, 0), (1, 1), (1, 2), (1, 3)])
def test_first_patch_gathers_virtual_hard_data(path_random, r):
    """The first patch of a realization: its data event is the hard data in
    its window, and the hard data within E cells beyond its forward edges
    (mirrored with the path) form the virtual template; the log record
    equals a direct search with that list."""
    ti = synth.channel_lens_ti(96, 96, seed=2, tol=0.2)
    t = O.OracleTI(ti, 3, 1)
    T, Ov, E, seed = 16, 4, 8, 11
    grid = (40, 28)                      # T + k S: the lattice needs no padding
    flips = O.path_flips(2, seed, r, path_random)
    org = [grid[a] - T if flips >> a & 1 else 0 for a in range(2)]
    _, gp = O.lattice(2, grid, T, Ov)
    assert tuple(gp[:2]) == grid
    rng = np.random.default_rng(r + 10 * path_random)
    cells, vals = [], []
    # two data inside the first window, six in its virtual extension
    def fwd(a, v):   # window offset of path-frame offset v along axis a
        return T - 1 - v if flips >> a & 1 else v
    while len(cells) < 2:
        c = [org[a] + fwd(a, int(rng.integers(0, T))) for a in range(2)]
        if c not in cells:
            cells.append(c)
    while len(cells) < 8:
        v = [int(rng.integers(0, T + E)) for _ in range(2)]
        if v[0] < T and v[1] < T:
            continue
        c = [org[a] + fwd(a, v[a]) for a in range(2)]
        if c not in cells:
            cells.append(c)
    vals = [int(v) for v in rng.integers(0, 3, size=len(cells))]
    hd_cells = np.asarray(cells, np.int32)
    hd_vals = np.asarray(vals, np.uint8)
    _, log = t.simulate(grid, T, Ov, K=4, path_random=path_random, hd_cells=hd_cells,
                        hd_vals=hd_vals, seed=seed, r=r, max_patches=1, vt_ext=E)
    win = np.full((T, T), O.UNKNOWN, np.uint8)
    vhd = []
    for (x, y), v in zip(cells, vals):
        qx, qy = x - org[0], y - org[1]
        if 0 <= qx < T and 0 <= qy < T:
            win[qy, qx] = v
        else:
            vhd.append([qx, qy, 0, v])
    assert len(vhd) == 6
    res = t.search(T, win, hd=win, K=4, seed=seed, r=r, p=0, vhd=vhd)
    sel = list(res["topk_idx"]).index(res["pick"])
    assert log[0, 0] == res["pick"]
    assert log[0, 1] == res["topk_score"][sel] and log[0, 2] == res["topk_mis"][sel]
    assert list(log[0, 4:4 + res["n"]]) == list(res["topk_idx"])


def test_virtual_template_without_hard_data_changes_nothing():
    """With no hard data beyond the template the grown template adds no
    mismatch, so vt_ext > 0 equals vt_ext = 0."""
    ti = synth.ribbon_ti(80, 80, n_ribbons=5, seed=9, target=0.3, tol=0.2)
    t = O.OracleTI(ti, 2, 1)
    a, la = t.simulate((40, 36), 8, 2, K=3, seed=4)
    b, lb = t.simulate((40, 36), 8, 2, K=3, seed=4, vt_ext=8)
    assert np.array_equal(a, b) and np.array_equal(la, lb)


def test_virtual_template_improves_conditioning():
    """The purpose of the non-causal check: with dense hard data the picks
    that honour the data ahead of the template are preferred, so fewer
    pasted cells disagree with hard data that later patches re-impose."""
    ti = synth.channel_lens_ti(160, 160, seed=2, tol=0.2)
    field = synth.channel_lens_ti(160, 160, seed=3, tol=0.2)
    cells, vals = synth.sample_hard_data(field, 300, seed=4)
    t = O.OracleTI(ti, 3, 1)

    def conflicts(vt):
        total = 0
        for r in range(3):
            out, log = t.simulate((96, 96), 16, 4, K=3, hd_cells=cells[cells.max(1) < 96],
                                  hd_vals=vals[cells.max(1) < 96], seed=6, r=r, vt_ext=vt)
            # disagreement of the realization with hard data one cell away:
            # a patch that ignored data ahead leaves isolated re-imposed cells
            hd = np.full(out.shape, O.UNKNOWN, np.uint8)
            sel = cells.max(1) < 96
            hd[cells[sel, 1], cells[sel, 0]] = vals[sel]
            ys, xs = np.nonzero(hd != O.UNKNOWN)
            for y, x in zip(ys, xs):
                nb = out[max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]
                total += int(np.sum(nb != hd[y, x]))
        return total
    assert conflicts(4) < conflicts(0)


def test_boundary_cut_keeps_channels_connected():
    """The purpose of the quilting cut: seams between patches break fewer
    channels, so the E-W probability of connection (Sec. 5.3) of the
    ribbon workload's channels at long lags is higher than with the full
    paste (4 realizations of the 250 x 250 workload, T 40, OR 10, J 1, K 3)."""
    from workloads import configs, stats
    w = configs.workload("c1")
    t = O.OracleTI(w["ti"], w["F"], w["J"])

    def conn(cut):
        reals = [t.simulate(w["grid"], w["T"], w["O"], K=3, seed=21, r=r, cut=cut,
                            want_log=False)[0] for r in range(4)]
        return np.nanmean([stats.connection_probability(x, 1, (64, 128), axis=1)
                           for x in reals], 0)
    plain, cut = conn(0), conn(1)
    assert np.all(cut > plain)
