"""Pattern-reproduction statistics of categorical realizations (host, numpy).

Used to compare ensembles (learned proposal vs full search, a variant vs the
plain method) at equal accuracy: facies proportions, indicator variograms
along the two axes and the probability of connection along an axis (the two
validation metrics of Sec. 5.3), and the Jensen-Shannon divergence of w x w
pattern histograms at mode-downsampled resolutions, from which the between-
and within-realization variabilities and the ratio of the ANODI comparison
(Sec. 5.5) are formed. ANODI's own pattern clustering and multidimensional
scaling are not reproduced: exact histograms of small windows stand in.
"""
from __future__ import annotations

import numpy as np


def proportions(real: np.ndarray, F: int) -> np.ndarray:
    """Facies fractions [F] of a realization (any shape)."""
    return np.bincount(real.ravel(), minlength=F)[:F] / real.size


def indicator_variogram(real: np.ndarray, f: int, axis: int, lags) -> np.ndarray:
    """gamma(h) = 0.5 E[(I(x) - I(x + h e_axis))^2] of the indicator of f,
    for 2D realizations [ny, nx]; axis 1 = x (E-W), 0 = y (N-S)."""
    ind = (real == f).astype(np.float64)
    out = []
    for h in lags:
        if axis == 1:
            d = ind[:, h:] - ind[:, :-h]
        else:
            d = ind[h:, :] - ind[:-h, :]
        out.append(0.5 * np.mean(d * d))
    return np.asarray(out)


def connection_probability(real: np.ndarray, f: int, lags, axis: int = 1) -> np.ndarray:
    """Probability of connection (Sec. 5.3) of facies f at each lag h: among
    the cell pairs (x, x + h e_axis) of a 2D realization [ny, nx] that are
    both of facies f, the fraction lying in one 4-connected component of
    facies f. axis 1 = x (E-W), 0 = y (N-S). NaN where no such pair exists."""
    from scipy import ndimage
    lab, _ = ndimage.label(real == f)   # the default structure is 4-connected
    out = []
    for h in lags:
        if axis == 1:
            a, b = lab[:, :-h], lab[:, h:]
        else:
            a, b = lab[:-h, :], lab[h:, :]
        both = (a > 0) & (b > 0)
        n = int(both.sum())
        out.append(np.nan if n == 0 else float(np.sum(both & (a == b))) / n)
    return np.asarray(out)


def mode_downsample(real: np.ndarray, k: int, F: int) -> np.ndarray:
    """Most frequent facies of every k x k block (ties to the lower code)."""
    ny, nx = (real.shape[0] // k) * k, (real.shape[1] // k) * k
    b = real[:ny, :nx].reshape(ny // k, k, nx // k, k).transpose(0, 2, 1, 3).reshape(
        ny // k, nx // k, k * k)
    counts = np.stack([(b == f).sum(-1) for f in range(F)], -1)
    return counts.argmax(-1).astype(np.uint8)


def pattern_histogram(real: np.ndarray, F: int, w: int = 4) -> dict:
    """Counts of every w x w pattern (encoded base F) in a 2D realization."""
    ny, nx = real.shape
    code = np.zeros((ny - w + 1, nx - w + 1), dtype=np.int64)
    for dy in range(w):
        for dx in range(w):
            code = code * F + real[dy:dy + ny - w + 1, dx:dx + nx - w + 1].astype(np.int64)
    vals, cnt = np.unique(code, return_counts=True)
    return dict(zip(vals.tolist(), cnt.tolist()))


def js_divergence(h1: dict, h2: dict) -> float:
    """Jensen-Shannon divergence (base 2) of two pattern histograms."""
    keys = sorted(set(h1) | set(h2))
    p = np.array([h1.get(k, 0) for k in keys], np.float64)
    q = np.array([h2.get(k, 0) for k in keys], np.float64)
    p /= p.sum()
    q /= q.sum()
    m = 0.5 * (p + q)

    def kl(a, b):
        nz = a > 0
        return float(np.sum(a[nz] * np.log2(a[nz] / b[nz])))

    return 0.5 * kl(p, m) + 0.5 * kl(q, m)


def ensemble_histogram(reals, F: int, k: int = 1, w: int = 4) -> dict:
    h: dict = {}
    for r in reals:
        rr = r if k == 1 else mode_downsample(r, k, F)
        for key, c in pattern_histogram(rr, F, w).items():
            h[key] = h.get(key, 0) + c
    return h


def summary(reals, ti: np.ndarray, F: int, lags=(1, 2, 4, 8, 16, 32), ks=(1, 2, 4)) -> dict:
    """Per-realization proportions and variograms, and the JS divergence of
    the ensemble's pattern histograms to the TI's at each resolution."""
    props = np.stack([proportions(r, F) for r in reals])
    vx = np.stack([indicator_variogram(r, 1, 1, lags) for r in reals])
    vy = np.stack([indicator_variogram(r, 1, 0, lags) for r in reals])
    js = [js_divergence(ensemble_histogram(reals, F, k), ensemble_histogram([ti], F, k))
          for k in ks]
    return dict(props=props, vario_x=vx, vario_y=vy, js=np.asarray(js))


def anodi_variability(reals, ti: np.ndarray, F: int, ks=(1, 2, 4), w: int = 4):
    """The two components of the ANODI comparison (Sec. 5.5) at each
    resolution k (mode downsampling by k): between = the mean JS divergence
    of the w x w pattern histograms over all pairs of realizations (spatial
    uncertainty), within = their mean JS divergence to the TI's (pattern
    reproduction error). Returns (between[len(ks)], within[len(ks)])."""
    between, within = [], []
    for k in ks:
        def down(x):
            return x if k == 1 else mode_downsample(x, k, F)
        hs = [pattern_histogram(down(r), F, w) for r in reals]
        ht = pattern_histogram(down(ti), F, w)
        pairs = [js_divergence(hs[i], hs[j]) for i in range(len(hs))
                 for j in range(i + 1, len(hs))]
        between.append(float(np.mean(pairs)))
        within.append(float(np.mean([js_divergence(h, ht) for h in hs])))
    return np.asarray(between), np.asarray(within)


def anodi_ratio(var_a, var_b, weights=None) -> float:
    """r(A, B) = sum_p w_p d_between(A, B) / d_within(A, B) (Sec. 5.5) with
    d_between = between_A / between_B and d_within = within_A / within_B per
    resolution p, from two anodi_variability results; equal weights by
    default. Above 1: A does better than B."""
    (ba, wa), (bb, wb) = var_a, var_b
    w = np.full(len(ba), 1.0 / len(ba)) if weights is None else np.asarray(weights, float)
    return float(np.sum(w * (ba / bb) / (wa / wb)))


def ci95(x: np.ndarray) -> tuple:
    """Mean and half-width of the 95 % confidence interval of the mean
    (normal approximation) along axis 0."""
    m = x.mean(0)
    h = 1.96 * x.std(0, ddof=1) / np.sqrt(x.shape[0])
    return m, h
