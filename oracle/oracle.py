"""ctypes front-end of the plain C oracle (``ccw_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The CUDA library and its
Python binding never import this module.

Arrays follow the C convention of the oracle: x fastest, so a 2D grid is a
numpy array ``[ny, nx]`` and a 3D grid ``[nz, ny, nx]``; dims tuples are
``(nx, ny[, nz])``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libccw_oracle.so")
UNKNOWN = 255

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2) into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    i32, i64, u32, u64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    lib.orc_philox4x32_10.argtypes = [P, P, P]
    lib.orc_philox_many.argtypes = [C.c_int64, P, P, P]
    lib.orc_dwt.argtypes = [P, C.c_int, P, C.c_int, P]
    lib.orc_idwt.argtypes = [P, C.c_int, P, C.c_int, P]
    lib.orc_dwt_orth.argtypes = [P, C.c_int, P, C.c_int, P]
    lib.orc_ti_prepare.argtypes = [P, C.c_int, P, C.c_int, C.c_int]
    lib.orc_ti_prepare.restype = P
    lib.orc_ti_free.argtypes = [P]
    lib.orc_ti_info.argtypes = [P, P]
    lib.orc_ti_get.argtypes = [P, P, P, P, P]
    lib.orc_num_candidates.argtypes = [P, C.c_int]
    lib.orc_num_candidates.restype = i64
    lib.orc_search.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int, u64, u32, u32,
                               P, P, P, P, P, P]
    lib.orc_reconstruct.argtypes = [P, C.c_int, i32, P]
    lib.orc_lattice.argtypes = [C.c_int, P, C.c_int, C.c_int, P, P]
    lib.orc_path_flips.argtypes = [C.c_int, u64, u32, C.c_int]
    lib.orc_path_flips.restype = u32
    lib.orc_simulate.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_int, P, P, u64, u32, i64, P, P]
    lib.orc_simulate_ext.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, C.c_int, C.c_int, P, P, u64, u32, i64, P,
                                     P]
    lib.orc_search_allshift.argtypes = [P, C.c_int, P, P, P, C.c_int, C.c_int, C.c_int, u64,
                                        u32, u32, P, P, P, P, P, P]
    lib.orc_num_candidates_allshift.argtypes = [P, C.c_int]
    lib.orc_num_candidates_allshift.restype = i64
    lib.orc_search_virtual.argtypes = [P, C.c_int, P, P, P, C.c_int, C.c_int, C.c_int, u64,
                                       u32, u32, P, P, P, P, P, P]
    lib.orc_min_cut.argtypes = [P, C.c_int, C.c_int, P]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims3(dims):
    d = list(dims) + [1] * (3 - len(dims))
    return np.asarray(d, dtype=np.int32)


# ---------------------------------------------------------------- Philox ---
def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_many(ctr, key) -> np.ndarray:
    """Philox4x32-10 blocks of the counters ctr [n, 4] under one key: [n, 4]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _load().orc_philox_many(c.shape[0], _p(c), _p(k), _p(out))
    return out


# ------------------------------------------------------------------ DWT ---
def dwt(x: np.ndarray, levels: int) -> np.ndarray:
    """J-level scaled Haar DWT; x is [ny, nx] or [nz, ny, nx] of integers.
    Returns the flat pyramid (level-1 detail bands, ..., level-J detail
    bands, then cA_J)."""
    x = np.ascontiguousarray(x, dtype=np.int64)
    out = np.zeros(x.size, dtype=np.int64)
    rc = _load().orc_dwt(_p(x), x.ndim, _p(_dims3(x.shape[::-1])), levels, _p(out))
    if rc != 0:
        raise ValueError(f"orc_dwt failed ({rc})")
    return out


def idwt(pyr: np.ndarray, shape, levels: int) -> np.ndarray:
    pyr = np.ascontiguousarray(pyr, dtype=np.int64)
    out = np.zeros(int(np.prod(shape)), dtype=np.int64)
    rc = _load().orc_idwt(_p(pyr), len(shape), _p(_dims3(tuple(shape)[::-1])), levels, _p(out))
    if rc != 0:
        raise ValueError(f"orc_idwt failed ({rc})")
    return out.reshape(shape)


def dwt_orth(x: np.ndarray, levels: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size, dtype=np.float64)
    rc = _load().orc_dwt_orth(_p(x), x.ndim, _p(_dims3(x.shape[::-1])), levels, _p(out))
    if rc != 0:
        raise ValueError(f"orc_dwt_orth failed ({rc})")
    return out


def pyramid_views(pyr: np.ndarray, shape, levels: int):
    """Split a flat pyramid into {(j, b): band array} and cA (numpy shapes)."""
    d = len(shape)
    nb = (1 << d) - 1
    off = 0
    bands = {}
    for j in range(1, levels + 1):
        bshape = tuple(n >> j for n in shape)
        v = int(np.prod(bshape))
        for b in range(1, nb + 1):
            bands[(j, b)] = pyr[off:off + v].reshape(bshape)
            off += v
    ashape = tuple(n >> levels for n in shape)
    cA = pyr[off:off + int(np.prod(ashape))].reshape(ashape)
    return bands, cA


# ------------------------------------------------------------- TI state ---
class OracleTI:
    """The oracle's training-image state: cropped TI, per-facies indicator
    cA_J, code cA_J and the full code pyramid (Algorithm 1, line 2)."""

    def __init__(self, ti: np.ndarray, n_facies: int, level: int):
        ti = np.ascontiguousarray(ti, dtype=np.uint8)
        self._lib = _load()
        self.ndim = ti.ndim
        self.F = n_facies
        self.J = level
        self.h = self._lib.orc_ti_prepare(_p(ti), ti.ndim, _p(_dims3(ti.shape[::-1])),
                                          n_facies, level)
        if not self.h:
            raise ValueError("orc_ti_prepare rejected the training image")
        info = np.zeros(10, dtype=np.int32)
        self._lib.orc_ti_info(self.h, _p(info))
        self.s = int(info[3])
        self.n = tuple(int(v) for v in info[4:4 + self.ndim])        # (nx, ny[, nz])
        self.nc = tuple(int(v) for v in info[7:7 + self.ndim])
        self.shape = self.n[::-1]
        self.cshape = self.nc[::-1]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.orc_ti_free(h)
            self.h = None

    def arrays(self):
        ncv = int(np.prod(self.nc))
        nv = int(np.prod(self.n))
        cA_ind = np.zeros(ncv * self.F, dtype=np.int64)
        cA_code = np.zeros(ncv, dtype=np.int64)
        pyr = np.zeros(nv, dtype=np.int64)
        ti = np.zeros(nv, dtype=np.uint8)
        self._lib.orc_ti_get(self.h, _p(cA_ind), _p(cA_code), _p(pyr), _p(ti))
        return (cA_ind.reshape((self.F,) + self.cshape), cA_code.reshape(self.cshape),
                pyr, ti.reshape(self.shape))

    def num_candidates(self, T: int) -> int:
        return int(self._lib.orc_num_candidates(self.h, T))

    def cand_shape(self, T: int):
        tj = T // self.s
        return tuple(n - tj + 1 for n in self.cshape)

    def search(self, T, de, hd=None, K=1, score_mode=0, seed=0, r=0, p=0, maps=False,
               vhd=None, all_shift=False):
        """Best-match search for one data event (numpy [T]*d u8, 255 = unknown).
        vhd: hard data of a virtual template, int [n][4] rows (qx, qy, qz, code)
        of fine offsets from the window origin (any sign). all_shift: every
        fine origin is a candidate (indices over the fine candidate grid).
        Returns dict(topk_idx, topk_score, topk_mis, pick[, scores, mis])."""
        de = np.ascontiguousarray(de, dtype=np.uint8)
        hdp = None
        if hd is not None:
            hd = np.ascontiguousarray(hd, dtype=np.uint8)
            hdp = _p(hd)
        P = (int(self._lib.orc_num_candidates_allshift(self.h, T)) if all_shift
             else self.num_candidates(T))
        sc = np.zeros(P, dtype=np.int64) if maps else None
        mm = np.zeros(P, dtype=np.int32) if maps else None
        ti_idx = np.full(K, -1, dtype=np.int32)
        ti_sc = np.zeros(K, dtype=np.int64)
        ti_mm = np.zeros(K, dtype=np.int32)
        pick = np.zeros(1, dtype=np.int32)
        if all_shift:
            v = np.ascontiguousarray(np.asarray([] if vhd is None else vhd,
                                                dtype=np.int32).reshape(-1, 4))
            nk = self._lib.orc_search_allshift(self.h, T, _p(de), hdp, _p(v) if len(v) else None,
                                               len(v), K, score_mode, seed, r, p,
                                               _p(sc) if maps else None,
                                               _p(mm) if maps else None, _p(ti_idx), _p(ti_sc),
                                               _p(ti_mm), _p(pick))
        elif vhd is None:
            nk = self._lib.orc_search(self.h, T, _p(de), hdp, K, score_mode, seed, r, p,
                                      _p(sc) if maps else None, _p(mm) if maps else None,
                                      _p(ti_idx), _p(ti_sc), _p(ti_mm), _p(pick))
        else:
            v = np.ascontiguousarray(np.asarray(vhd, dtype=np.int32).reshape(-1, 4))
            nk = self._lib.orc_search_virtual(self.h, T, _p(de), hdp, _p(v), len(v), K,
                                              score_mode, seed, r, p,
                                              _p(sc) if maps else None,
                                              _p(mm) if maps else None, _p(ti_idx), _p(ti_sc),
                                              _p(ti_mm), _p(pick))
        if nk < 0:
            raise ValueError(f"orc_search failed ({nk})")
        out = dict(n=nk, topk_idx=ti_idx[:nk], topk_score=ti_sc[:nk], topk_mis=ti_mm[:nk],
                   pick=int(pick[0]))
        if maps:
            out["scores"] = sc
            out["mis"] = mm
        return out

    def reconstruct(self, T: int, pick: int) -> np.ndarray:
        pat = np.zeros(T ** self.ndim, dtype=np.uint8)
        rc = self._lib.orc_reconstruct(self.h, T, int(pick), _p(pat))
        if rc != 0:
            raise ValueError(f"orc_reconstruct failed ({rc})")
        return pat.reshape((T,) * self.ndim)

    def simulate(self, grid, T, O, K=1, score_mode=0, path_random=0, hd_cells=None,
                 hd_vals=None, seed=0, r=0, max_patches=-1, want_log=True, vt_ext=0, cut=0,
                 all_shift=0):
        """One realization along the raster path (Algorithm 1). grid = (nx, ny[, nz]).
        vt_ext grows the virtual template of the non-causal conditioning; cut = 1
        pastes through the minimum-error boundary cuts (2D); all_shift = 1
        searches every fine origin of the TI (log indices over the fine grid).
        Returns (realization numpy array, patch log [n_patches, 4+K] or None)."""
        g = _dims3(grid)
        npch, gp = lattice(self.ndim, grid, T, O)
        n_patches = int(np.prod(npch))
        out = np.zeros(tuple(grid)[::-1], dtype=np.uint8)
        log = np.zeros((n_patches, 4 + K), dtype=np.int32) if want_log else None
        if hd_cells is None or len(hd_cells) == 0:
            n_hd, hc, hv = 0, None, None
        else:
            hc = np.ascontiguousarray(hd_cells, dtype=np.int32)
            hv = np.ascontiguousarray(hd_vals, dtype=np.uint8)
            n_hd = len(hv)
        rc = self._lib.orc_simulate_ext(self.h, _p(g), T, O, K, score_mode, path_random,
                                        vt_ext, cut, all_shift, n_hd,
                                        _p(hc) if n_hd else None,
                                        _p(hv) if n_hd else None, seed, r, max_patches,
                                        _p(out), _p(log) if want_log else None)
        if rc != 0:
            raise ValueError(f"orc_simulate failed ({rc})")
        return out, log


def lattice(ndim, grid, T, O):
    """(patches per axis, padded extent per axis), both (nx, ny, nz)."""
    n = np.zeros(3, dtype=np.int32)
    gp = np.zeros(3, dtype=np.int32)
    rc = _load().orc_lattice(ndim, _p(_dims3(grid)), T, O, _p(n), _p(gp))
    if rc != 0:
        raise ValueError("bad lattice")
    return tuple(int(v) for v in n), tuple(int(v) for v in gp)


def path_flips(ndim, seed, r, path_random=1) -> int:
    return int(_load().orc_path_flips(ndim, seed, r, path_random))


def min_cut(err) -> np.ndarray:
    """Minimum-error boundary cut of image quilting through a [rows, cols]
    0/1 cost array: the column of the cut in every row."""
    e = np.ascontiguousarray(err, dtype=np.uint8)
    rows, cols = e.shape
    cut = np.zeros(rows, dtype=np.int32)
    rc = _load().orc_min_cut(_p(e), rows, cols, _p(cut))
    if rc != 0:
        raise ValueError(f"orc_min_cut failed ({rc})")
    return cut
