"""Pins of the validation statistics (host): the probability of connection
of Sec. 5.3 against a breadth-first flood fill written here and against
hand-made channel layouts, and the ANODI ratio of Sec. 5.5 against its
closed forms. CPU only."""
from collections import deque

import numpy as np

from workloads import stats


def _brute_connection(real, f, lags, axis):
    """Flood-fill labels (4-neighbours), then the pair count by loops."""
    ny, nx = real.shape
    lab = np.zeros((ny, nx), np.int64)
    nxt = 0
    for y in range(ny):
        for x in range(nx):
            if real[y, x] != f or lab[y, x]:
                continue
            nxt += 1
            lab[y, x] = nxt
            q = deque([(y, x)])
            while q:
                cy, cx = q.popleft()
                for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    yy, xx = cy + dy, cx + dx
                    if 0 <= yy < ny and 0 <= xx < nx and real[yy, xx] == f and not lab[yy, xx]:
                        lab[yy, xx] = nxt
                        q.append((yy, xx))
    out = []
    for h in lags:
        n = c = 0
        for y in range(ny):
            for x in range(nx):
                y2, x2 = (y, x + h) if axis == 1 else (y + h, x)
                if y2 >= ny or x2 >= nx:
                    continue
                if lab[y, x] and lab[y2, x2]:
                    n += 1
                    c += lab[y, x] == lab[y2, x2]
        out.append(np.nan if n == 0 else c / n)
    return np.asarray(out)


def test_connection_probability_equals_flood_fill():
    rng = np.random.default_rng(3)
    for p in (0.45, 0.55, 0.65):
        for axis in (0, 1):
            real = (rng.random((23, 31)) < p).astype(np.uint8)
            lags = (1, 2, 5, 9)
            np.testing.assert_array_equal(stats.connection_probability(real, 1, lags, axis),
                                          _brute_connection(real, 1, lags, axis))


def test_connection_probability_closed_forms():
    """One E-W channel: every pair is connected. Two N-S bars 5 apart: no
    pair at lag 5 is; a bridge between them connects every pair."""
    real = np.zeros((9, 20), np.uint8)
    real[4, :] = 1
    assert np.all(stats.connection_probability(real, 1, (1, 3, 19), axis=1) == 1.0)
    bars = np.zeros((9, 20), np.uint8)
    bars[:, 3] = bars[:, 8] = 1
    assert stats.connection_probability(bars, 1, (5,), axis=1)[0] == 0.0
    assert np.isnan(stats.connection_probability(bars, 1, (4,), axis=1)[0])
    bars[0, 3:9] = 1
    assert stats.connection_probability(bars, 1, (5,), axis=1)[0] == 1.0
    # diagonal neighbours are not connected (4-connectivity): (0, 0) and
    # (0, 2) touch (1, 1) only at corners
    v = np.zeros((3, 3), np.uint8)
    v[0, 0] = v[1, 1] = v[0, 2] = 1
    assert stats.connection_probability(v, 1, (2,), axis=1)[0] == 0.0
    v[0, 1] = 1
    assert stats.connection_probability(v, 1, (2,), axis=1)[0] == 1.0


def test_anodi_ratio_closed_forms():
    """Identical ensembles give r = 1; doubling A's between-realization
    variability at equal within-realization error doubles r, doubling its
    within error halves it (Sec. 5.5 equation)."""
    rng = np.random.default_rng(5)
    ti = (rng.random((40, 40)) < 0.3).astype(np.uint8)
    reals = [(rng.random((40, 40)) < 0.3).astype(np.uint8) for _ in range(4)]
    va = stats.anodi_variability(reals, ti, 2, ks=(1, 2))
    assert va[0].shape == (2,) and np.all(va[0] > 0) and np.all(va[1] > 0)
    assert abs(stats.anodi_ratio(va, va) - 1.0) < 1e-12
    assert abs(stats.anodi_ratio((2 * va[0], va[1]), va) - 2.0) < 1e-12
    assert abs(stats.anodi_ratio((va[0], 2 * va[1]), va) - 0.5) < 1e-12


def test_copies_of_the_ti_have_no_within_error():
    rng = np.random.default_rng(6)
    ti = (rng.random((32, 32)) < 0.4).astype(np.uint8)
    between, within = stats.anodi_variability([ti, ti, ti], ti, 2, ks=(1, 2))
    assert np.all(between == 0.0) and np.all(within == 0.0)
