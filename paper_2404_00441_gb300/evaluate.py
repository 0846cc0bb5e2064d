"""Pattern-reproduction statistics of realizations on the GPU (libccw's
``ccw_eval_*`` kernels): facies proportions, indicator variograms, the
probability of connection and w x w pattern histograms at mode-downsampled
resolutions, with the Jensen-Shannon
divergence between two histograms (computed on the host from the counts).
Used to compare ensembles (e.g. the learned proposal vs the full search) and
an ensemble with its training image, as in the validation of Sec. 5.2-5.3.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import ccw


def _lib():
    lib = ccw.load()
    if not getattr(lib, "_eval_ready", False):
        P, i32 = C.c_void_p, C.c_int32
        lib.ccw_eval_proportions.argtypes = [P, i32, P, i32, P, P]
        lib.ccw_eval_variogram.argtypes = [P, i32, P, i32, i32, P, i32, P, P]
        lib.ccw_eval_patterns.argtypes = [P, i32, P, i32, i32, i32, P, P, P]
        lib.ccw_eval_connectivity.argtypes = [P, i32, P, i32, i32, P, i32, P, P, P]
        lib.ccw_eval_last_error.restype = C.c_char_p
        lib._eval_ready = True
    return lib


def _check(rc):
    if rc != 0:
        raise ccw.CCWError(_lib().ccw_eval_last_error().decode())


def _dims(reals: torch.Tensor):
    shp = list(reals.shape[1:])[::-1]
    return (C.c_int32 * 3)(*(shp + [1] * (3 - len(shp))))


def proportions(reals: torch.Tensor, n_facies: int, stream=None) -> torch.Tensor:
    """Facies fractions float64 [n_real, n_facies] (host tensor) of uint8
    realizations."""
    lib = _lib()
    n = reals.shape[0]
    out = torch.empty((n, n_facies), dtype=torch.int64, device=reals.device)
    _check(lib.ccw_eval_proportions(ccw._ptr(reals), n, _dims(reals), n_facies, ccw._ptr(out),
                                    ccw._stream(stream)))
    vol = reals[0].numel()
    # divided on the host: torch may divide by a scalar through its
    # reciprocal, which is not the correctly rounded quotient
    return torch.from_numpy(out.cpu().numpy() / vol)


def variogram(reals: torch.Tensor, facies: int, axis: int, lags, stream=None) -> torch.Tensor:
    """Indicator variogram float64 [n_real, len(lags)] (host tensor) of
    `facies` along axis (0 = x, 1 = y, 2 = z): 0.5 * (differing pairs) / pairs."""
    lib = _lib()
    n = reals.shape[0]
    lg = torch.tensor(list(lags), dtype=torch.int32, device=reals.device)
    out = torch.empty((n, len(lags)), dtype=torch.int64, device=reals.device)
    _check(lib.ccw_eval_variogram(ccw._ptr(reals), n, _dims(reals), facies, axis, ccw._ptr(lg),
                                  len(lags), ccw._ptr(out), ccw._stream(stream)))
    shape = list(reals.shape[1:])[::-1]
    n_axis = shape[axis]
    per_line = reals[0].numel() // n_axis
    pairs = torch.tensor([(n_axis - h) * per_line if 0 <= h < n_axis else float("nan")
                          for h in lags], dtype=torch.float64, device=reals.device)
    return torch.from_numpy(0.5 * out.cpu().numpy() / pairs.cpu().numpy())   # NaN: no pair


def pattern_histogram(reals: torch.Tensor, n_facies: int, w: int = 4, down: int = 1,
                      stream=None) -> torch.Tensor:
    """Counts int64 [n_facies^(w*w)] of the w x w patterns of all 2D
    realizations after mode downsampling by `down`."""
    lib = _lib()
    n, ny, nx = reals.shape
    bins = n_facies ** (w * w)
    hist = torch.empty((bins,), dtype=torch.int32, device=reals.device)
    scratch = (torch.empty((n, ny // down, nx // down), dtype=torch.uint8, device=reals.device)
               if down > 1 else None)
    _check(lib.ccw_eval_patterns(ccw._ptr(reals), n, _dims(reals), n_facies, down, w,
                                 ccw._ptr(scratch) if scratch is not None else None,
                                 ccw._ptr(hist), ccw._stream(stream)))
    return hist.to(torch.int64)


def connectivity_counts(reals: torch.Tensor, facies: int, lags, axis: int = 0,
                        stream=None) -> torch.Tensor:
    """``ccw_eval_connectivity``: int64 [n_real, len(lags), 2] = (cell pairs
    (c, c + h e_axis) both of `facies`, those in one 4-connected component
    of it) of 2D realizations; axis 0 = x (E-W), 1 = y (N-S)."""
    lib = _lib()
    n, ny, nx = reals.shape
    lg = torch.tensor(list(lags), dtype=torch.int32, device=reals.device)
    labels = torch.empty((n * (nx * ny + 1),), dtype=torch.int32, device=reals.device)
    out = torch.empty((n, len(lags), 2), dtype=torch.int64, device=reals.device)
    _check(lib.ccw_eval_connectivity(ccw._ptr(reals), n, _dims(reals), facies, axis,
                                     ccw._ptr(lg), len(lags), ccw._ptr(labels), ccw._ptr(out),
                                     ccw._stream(stream)))
    return out


def connection_probability(reals: torch.Tensor, facies: int, lags, axis: int = 0,
                           stream=None) -> np.ndarray:
    """Probability of connection (Sec. 5.3) float64 [n_real, len(lags)] of
    `facies` along axis 0 = x (E-W) or 1 = y (N-S): connected pairs over
    pairs, NaN where no pair exists."""
    c = connectivity_counts(reals, facies, lags, axis, stream).cpu().numpy()
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(c[..., 0] > 0, c[..., 1] / np.maximum(c[..., 0], 1), np.nan)


def js_divergence(h1: torch.Tensor, h2: torch.Tensor) -> float:
    """Jensen-Shannon divergence (base 2) of two pattern histograms."""
    p = h1.double().cpu().numpy()
    q = h2.double().cpu().numpy()
    p = p / p.sum()
    q = q / q.sum()
    m = 0.5 * (p + q)

    def kl(a, b):
        nz = a > 0
        return float(np.sum(a[nz] * np.log2(a[nz] / b[nz])))

    return 0.5 * kl(p, m) + 0.5 * kl(q, m)
