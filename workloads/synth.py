"""Seeded synthetic inputs shaped like the paper's categorical training images.

This module only draws inputs. It holds none of the simulation method's
arithmetic (no wavelet, no correlation, no selection), so both the CPU oracle
and the CUDA path can take their inputs from it.

The paper's own training images (Channel, Stonewall, Ganges delta, the
multi-facies TI; Sec. 5.1-5.8) are not available, so these generators stand
in for them:

* ``ribbon_ti``   -- binary E-W sinuous channels (stand-in for the Channel TI,
  Sec. 5.1; channel continuity is E-W as in Sec. 5.3).
* ``channel_lens_ti`` -- 3 facies: sinuous channels (1) and elliptical lenses
  (2) over a background (0); stand-in for the multi-facies TI of Sec. 5.8.
* ``tube_lobe_ti_3d`` -- 4 facies 3D: sinuous channel tubes with a core (1) and
  a margin (2), lobes (3), background (0); the paper only proposes 3D as future
  work (Sec. 6).
* ``sample_hard_data`` -- conditioning points drawn uniformly without
  replacement from a second field, as Sec. 5.2 draws hard data from an initial
  realization.

Every array is C-ordered with x fastest: 2D arrays are ``[ny, nx]``, 3D
arrays ``[nz, ny, nx]``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "ribbon_ti",
    "channel_lens_ti",
    "tube_lobe_ti_3d",
    "sample_hard_data",
    "random_field_ti",
]


def _rng(seed: int, tag: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(tag)]))


def _ribbons(nx: int, ny: int, count: int, rng: np.random.Generator,
             amp=(5.0, 25.0), lam=(60.0, 250.0), width=(6, 12),
             ytop=None) -> np.ndarray:
    """Boolean mask of ``count`` E-W ribbons y = c + A sin(2 pi x / lam + phi)."""
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)[:, None]
    out = np.zeros((ny, nx), dtype=bool)
    lo = 0.0 if ytop is None else ytop[0]
    hi = float(ny) if ytop is None else ytop[1]
    for _ in range(count):
        c = rng.uniform(lo, hi)
        a = rng.uniform(*amp)
        lm = rng.uniform(*lam)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        w = int(rng.integers(width[0], width[1] + 1))
        yc = c + a * np.sin(2.0 * np.pi * x / lm + ph)
        out |= np.abs(y - yc[None, :]) < (w / 2.0)
    return out


def ribbon_ti(nx: int = 250, ny: int = 250, n_ribbons: int = 12, seed: int = 1,
              target: float = 0.28, tol: float = 0.03,
              max_tries: int = 10000) -> np.ndarray:
    """Binary ribbon TI (u8, values 0/1), channel fraction within target +- tol.

    The draw is repeated with tags 0, 1, 2, ... of the same seed until the
    channel fraction lands in range, so the result is a pure function of the
    arguments.
    """
    for tag in range(max_tries):
        rng = _rng(seed, tag)
        m = _ribbons(nx, ny, n_ribbons, rng)
        frac = float(m.mean())
        if abs(frac - target) <= tol:
            return m.astype(np.uint8)
    raise RuntimeError("ribbon_ti: no draw reached the target fraction")


def channel_lens_ti(nx: int = 1000, ny: int = 1000, seed: int = 2,
                    target=(0.55, 0.30, 0.15), tol: float = 0.03) -> np.ndarray:
    """3-facies TI: background 0, channels 1, elliptical lenses 2 (u8).

    Channels are added one at a time until facies 1 reaches its target, then
    lenses (drawn over the background only, so channels cut through them)
    until facies 2 reaches its target.
    """
    rng = _rng(seed, 0)
    ti = np.zeros((ny, nx), dtype=np.uint8)
    scale = nx / 250.0
    x = np.arange(nx, dtype=np.float64)
    yy = np.arange(ny, dtype=np.float64)[:, None]
    xx = np.arange(nx, dtype=np.float64)[None, :]
    for _ in range(10000):
        if (ti == 1).mean() >= target[1]:
            break
        c = rng.uniform(0, ny)
        a = rng.uniform(5, 25) * scale
        lm = rng.uniform(60, 250) * scale
        ph = rng.uniform(0, 2 * np.pi)
        w = rng.uniform(6, 12) * scale
        yc = c + a * np.sin(2 * np.pi * x / lm + ph)
        ti[np.abs(yy - yc[None, :]) < w / 2] = 1
    for _ in range(100000):
        if (ti == 2).mean() >= target[2]:
            break
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ax = rng.uniform(8, 30) * scale
        ay = rng.uniform(3, 10) * scale
        th = rng.uniform(-0.4, 0.4)
        dx, dy = xx - cx, yy - cy
        u = (dx * np.cos(th) + dy * np.sin(th)) / ax
        v = (-dx * np.sin(th) + dy * np.cos(th)) / ay
        ti[(u * u + v * v <= 1.0) & (ti == 0)] = 2
    p = np.array([(ti == f).mean() for f in range(3)])
    if np.any(np.abs(p - np.asarray(target)) > tol):
        raise RuntimeError(f"channel_lens_ti: proportions {p} off target")
    return ti


def tube_lobe_ti_3d(nx: int = 180, ny: int = 150, nz: int = 120, seed: int = 5,
                    target=(0.60, 0.18, 0.10, 0.12)) -> np.ndarray:
    """4-facies 3D TI [nz, ny, nx]: background 0, tube core 1, tube margin 2,
    lobes 3. Tubes run along x with a sinuous centreline in y and a gentle
    undulation in z; the margin is a shell around the core."""
    rng = _rng(seed, 0)
    ti = np.zeros((nz, ny, nx), dtype=np.uint8)
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    core = np.zeros(ti.shape, dtype=bool)
    shell = np.zeros(ti.shape, dtype=bool)
    for _ in range(2000):
        if core.mean() >= target[1]:
            break
        cy, cz = rng.uniform(0, ny), rng.uniform(0, nz)
        a = rng.uniform(5, 20)
        lm = rng.uniform(50, 180)
        ph = rng.uniform(0, 2 * np.pi)
        az = rng.uniform(1, 5)
        lz = rng.uniform(80, 250)
        rc = rng.uniform(2.5, 5.0)
        rm = rc + rng.uniform(0.6, 1.3)
        yc = cy + a * np.sin(2 * np.pi * x / lm + ph)
        zc = cz + az * np.sin(2 * np.pi * x / lz)
        d2 = (y - yc) ** 2 + ((z - zc) * 1.5) ** 2
        core |= d2 < rc * rc
        shell |= d2 < rm * rm
    ti[shell] = 2
    ti[core] = 1
    lobes = np.zeros(ti.shape, dtype=bool)
    for _ in range(5000):
        if ((ti == 0) & lobes).mean() + 0.0 >= target[3]:
            break
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        ax, ay, az = rng.uniform(8, 25), rng.uniform(6, 18), rng.uniform(2, 5)
        lobes |= (((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2
                  + ((z - cz) / az) ** 2) <= 1.0
    ti[lobes & (ti == 0)] = 3
    return ti


def random_field_ti(shape, n_facies: int, seed: int) -> np.ndarray:
    """Unstructured i.i.d. categorical field (u8) for small edge-case tests."""
    return _rng(seed, 7).integers(0, n_facies, size=shape, dtype=np.uint8)


def sample_hard_data(field: np.ndarray, n: int, seed: int):
    """Draw ``n`` distinct cells uniformly from ``field``.

    Returns ``(cells, vals)``: ``cells`` is int32 ``[n, ndim]`` in (x, y[, z])
    order and ``vals`` is u8 ``[n]`` with the field's value at each cell.
    """
    rng = _rng(seed, 0)
    flat = rng.choice(field.size, size=n, replace=False)
    idx = np.unravel_index(flat, field.shape)        # (z,) y, x
    cells = np.stack(idx[::-1], axis=1).astype(np.int32)
    vals = field.reshape(-1)[flat].astype(np.uint8)
    return np.ascontiguousarray(cells), np.ascontiguousarray(vals)
