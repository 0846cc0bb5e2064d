"""ctypes binding of the C ABI in include/ccw.h (argument marshalling only).

Tensors passed in must be contiguous CUDA tensors of the stated dtype on the
current device; calls run on ``torch.cuda.current_stream()`` unless a stream is
given. There is no CPU fallback: if ``libccw.so`` is missing the import of the
library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libccw.so")
_lib = None

CCW_UNKNOWN = 255
CCW_MAX_TOPK = 64
LOG_FLAG_UNIFORM = 1
LOG_FLAG_DONE = 2
LOG_FLAG_PROPOSAL = 4


class CCWError(RuntimeError):
    pass


class _Params(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("grid", C.c_int32 * 3), ("topk", C.c_int32),
                ("n_real", C.c_int32), ("real_base", C.c_int32), ("path_random", C.c_int32),
                ("score_mode", C.c_int32), ("precision", C.c_int32), ("learned", C.c_int32),
                ("ccf_tile", C.c_int32), ("vt_ext", C.c_int32),
                ("boundary_cut", C.c_int32), ("all_shift", C.c_int32)]


class _Group(C.Structure):
    _fields_ = [("grid", C.c_int32 * 3), ("n_real", C.c_int32), ("real_base", C.c_int32),
                ("hd_cells_dev", C.c_void_p), ("hd_vals_dev", C.c_void_p), ("n_hd", C.c_int32),
                ("out_dev", C.c_void_p), ("patch_log_dev", C.c_void_p),
                ("event_counts_dev", C.c_void_p), ("out_host", C.c_void_p)]


class _Desc(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("n_facies", C.c_int32), ("level", C.c_int32),
                ("scale", C.c_int32), ("templ", C.c_int32), ("overlap", C.c_int32),
                ("dims", C.c_int32 * 3), ("coarse", C.c_int32 * 3), ("cand", C.c_int32 * 3),
                ("n_cand", C.c_int64)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libccw.so (built in-tree by ``paper_2404_00441_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: run paper_2404_00441_gb300.build.build() "
                          "(nvcc, sm_103a) first; there is no CPU fallback")
    lib = C.CDLL(_LIB_PATH)
    P, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    lib.ccw_ti_prepare.argtypes = [P, i32, P, i32, i32, i32, i32, P, C.POINTER(P)]
    lib.ccw_ti_describe.argtypes = [P, C.POINTER(_Desc)]
    lib.ccw_ti_free.argtypes = [P]
    lib.ccw_ti_free.restype = None
    lib.ccw_ti_export.argtypes = [P, i32, P, P]
    lib.ccw_simulate.argtypes = [P, C.POINTER(_Params), P, P, i32, u64, P, P, P]
    lib.ccw_simulate_groups.argtypes = [P, C.POINTER(_Params), C.POINTER(_Group), i32, u64, P]
    lib.ccw_ccf_search.argtypes = [P, i32, P, P, i32, i32, u64, P, P, P, P, P, P]
    lib.ccw_ccf_map.argtypes = [P, i32, P, P, i32, P, P, P]
    lib.ccw_idwt_paste.argtypes = [P, i32, P, P, P, P, P]
    lib.ccw_ti_status.argtypes = [P, P, C.POINTER(i32)]
    lib.ccw_last_error.restype = C.c_char_p
    lib.ccw_profile_enable.argtypes = [i32]
    lib.ccw_profile_read.argtypes = [C.POINTER(i64), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.ccw_launch_count.restype = i64
    lib.ccw_profile_read_phases.argtypes = [C.POINTER(C.c_double)]
    lib.ccw_profile_read_proposal.argtypes = [C.POINTER(C.c_double)]
    lib.ccw_set_nn_path.argtypes = [C.c_int32]
    f32 = C.c_float
    lib.ccw_net_create.argtypes = [i32, i32, u64, C.POINTER(P)]
    lib.ccw_net_free.argtypes = [P]
    lib.ccw_net_free.restype = None
    lib.ccw_net_param_count.argtypes = [P]
    lib.ccw_net_param_count.restype = i64
    lib.ccw_net_get.argtypes = [P, i32, P]
    lib.ccw_net_set.argtypes = [P, P]
    lib.ccw_net_embed.argtypes = [P, P, i32, i32, P, P]
    lib.ccw_net_train_step.argtypes = [P, P, i32, P, i32, f32, f32, f32, i32, i32, P, P]
    lib.ccw_net_last_error.restype = C.c_char_p
    lib.ccw_ti_attach_proposal.argtypes = [P, P, i32, f32, P]
    lib.ccw_proposal_query.argtypes = [P, P, i32, P, P, P, P]
    lib.ccw_proposal_inputs.argtypes = [P, i32, P, P, P, i32, P, P]
    lib.ccw_proposal_stats.argtypes = [P, C.POINTER(i64), P]
    lib.ccw_philox_host.argtypes = [i64, P, P, P]
    lib.ccw_philox_dev.argtypes = [i64, P, P, P, P]
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise CCWError(f"ccw error {rc}: {load().ccw_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _host_ptr(t, shape):
    """A host output buffer: a contiguous CPU uint8 tensor of `shape` (pinned
    for the streamed read-back)."""
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous() or t.dtype != torch.uint8 or tuple(t.shape) != shape:
        raise ValueError(f"out_host must be a contiguous CPU uint8 tensor of shape {shape}")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _i3(v):
    v = list(v) + [1] * (3 - len(v))
    return (C.c_int32 * 3)(*v)


def lattice(grid, T, O):
    """Patches per axis and padded extent (Sec. 4.1 lattice), host-side."""
    S = T - O
    n, gp = [], []
    for g in grid:
        extra = max(g - T, 0)
        n.append(1 + (extra + S - 1) // S)
        gp.append(T + (n[-1] - 1) * S)
    return tuple(n), tuple(gp)


class TI:
    """A training image prepared on the GPU (``ccw_ti_prepare``).

    ``ti`` is a uint8 CUDA tensor [ny, nx] or [nz, ny, nx]."""

    def __init__(self, ti: torch.Tensor, n_facies: int, level: int, templ: int, overlap: int,
                 stream=None):
        lib = load()
        if ti.dtype != torch.uint8:
            raise ValueError("TI must be uint8")
        self.ndim = ti.dim()
        dims = _i3(list(ti.shape)[::-1])
        h = C.c_void_p()
        _check(lib.ccw_ti_prepare(_ptr(ti), self.ndim, dims, n_facies, level, templ, overlap,
                                  _stream(stream), C.byref(h)))
        self._h = h
        self._lib = lib
        d = _Desc()
        _check(lib.ccw_ti_describe(h, C.byref(d)))
        self.n_facies = d.n_facies
        self.level = d.level
        self.scale = d.scale
        self.templ = d.templ
        self.overlap = d.overlap
        self.dims = tuple(d.dims[:self.ndim])
        self.coarse = tuple(d.coarse[:self.ndim])
        self.cand = tuple(d.cand[:self.ndim])
        self.n_cand = int(d.n_cand)

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ccw_ti_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def export(self, what: int, stream=None) -> torch.Tensor:
        cshape = self.coarse[::-1]
        sd = self.scale ** self.ndim
        if what == 0:
            out = torch.empty((self.n_facies - 1,) + cshape, dtype=torch.float32, device="cuda")
        elif what == 1:
            out = torch.empty(cshape, dtype=torch.float32, device="cuda")
        elif what == 2:
            out = torch.empty(cshape + (sd,), dtype=torch.int16, device="cuda")
        elif what == 3:
            out = torch.empty(self.dims[::-1], dtype=torch.uint8, device="cuda")
        elif what == 4:
            out = torch.empty((16, self.n_cand, 64), dtype=torch.bfloat16, device="cuda")
        else:
            raise ValueError(what)
        _check(self._lib.ccw_ti_export(self._h, what, _ptr(out), _stream(stream)))
        return out

    def attach_proposal(self, net, n_prop=64, gap_theta=0.0, stream=None):
        """``ccw_ti_attach_proposal``: tables of the TI windows under every mask
        type; ``net`` None detaches."""
        _check(self._lib.ccw_ti_attach_proposal(self._h, None if net is None else net.handle,
                                                n_prop, float(gap_theta), _stream(stream)))
        self.n_prop = n_prop if net is not None else 0

    def proposal_query(self, counts: torch.Tensor, stream=None):
        """``ccw_proposal_query`` on block counts uint8 [n, F, tj*tj]:
        (proposals int32 [n, n_prop], gaps float [n], mask types int32 [n])."""
        n = counts.shape[0]
        prop = torch.full((n, self.n_prop), -1, dtype=torch.int32, device=counts.device)
        gap = torch.empty((n,), dtype=torch.float32, device=counts.device)
        typ = torch.empty((n,), dtype=torch.int32, device=counts.device)
        _check(self._lib.ccw_proposal_query(self._h, _ptr(counts), n, _ptr(prop), _ptr(gap),
                                            _ptr(typ), _stream(stream)))
        return prop, gap, typ

    def proposal_inputs(self, what, counts=None, cand=None, types=None, stream=None):
        """``ccw_proposal_inputs``: encoder inputs float [n, F, tj, tj] from
        block counts (what 0; returns (x, mask types)) or from TI windows of
        candidates under mask types (what 1; returns x)."""
        tj = self.templ // self.scale
        if what == 0:
            n = counts.shape[0]
            types = torch.empty((n,), dtype=torch.int32, device=counts.device)
        else:
            n = cand.shape[0]
        dev = (counts if what == 0 else cand).device
        out = torch.empty((n, self.n_facies, tj, tj), dtype=torch.float32, device=dev)
        _check(self._lib.ccw_proposal_inputs(self._h, what, _ptr(counts), _ptr(cand),
                                             _ptr(types), n, _ptr(out), _stream(stream)))
        return (out, types) if what == 0 else out

    def proposal_stats(self, stream=None):
        """``ccw_proposal_stats``: (non-empty patches, patches with proposals,
        patches settled by the proposal) since the last read."""
        v = (C.c_int64 * 3)()
        _check(self._lib.ccw_proposal_stats(self._h, v, _stream(stream)))
        return tuple(int(x) for x in v)

    def status(self, stream=None) -> int:
        v = C.c_int32()
        _check(self._lib.ccw_ti_status(self._h, _stream(stream), C.byref(v)))
        return v.value


def simulate(ti: TI, grid, n_real=1, topk=1, seed=0, hd_cells=None, hd_vals=None, real_base=0,
             path_random=0, score_mode=0, precision=0, want_log=False, out=None, log=None,
             learned=0, ccf_tile=0, vt_ext=0, boundary_cut=0, all_shift=0, out_host=None,
             stream=None):
    """``ccw_simulate``: returns (realizations uint8 [n_real, *grid[::-1]], log or None).
    With ``out_host`` (a CPU uint8 tensor of that shape, pinned for the
    streamed copy) the realizations are also copied into it, through
    ``ccw_simulate_groups``' host read-back."""
    lib = load()
    p = _Params()
    p.ndim = ti.ndim
    p.grid = _i3(grid)
    p.topk = topk
    p.n_real = n_real
    p.real_base = real_base
    p.path_random = path_random
    p.score_mode = score_mode
    p.precision = precision
    p.learned = learned
    p.ccf_tile = ccf_tile
    p.vt_ext = vt_ext
    p.boundary_cut = boundary_cut
    p.all_shift = all_shift
    shape = (n_real,) + tuple(grid)[::-1]
    if out is None:
        out = torch.empty(shape, dtype=torch.uint8, device="cuda")
    npch, _ = lattice(grid, ti.templ, ti.overlap)
    n_patches = 1
    for v in npch:
        n_patches *= v
    if want_log and log is None:
        log = torch.empty((n_real, n_patches, 4 + topk), dtype=torch.int32, device="cuda")
    n_hd = 0 if hd_vals is None else int(hd_vals.numel())
    if out_host is not None:
        g = (_Group * 1)()
        g[0].grid = _i3(grid)
        g[0].n_real = n_real
        g[0].real_base = real_base
        g[0].hd_cells_dev = _ptr(hd_cells) if n_hd else None
        g[0].hd_vals_dev = _ptr(hd_vals) if n_hd else None
        g[0].n_hd = n_hd
        g[0].out_dev = _ptr(out)
        g[0].patch_log_dev = _ptr(log) if want_log else None
        g[0].event_counts_dev = None
        g[0].out_host = _host_ptr(out_host, shape)
        _check(lib.ccw_simulate_groups(ti.handle, C.byref(p), g, 1, seed & (2 ** 64 - 1),
                                       _stream(stream)))
        return out, (log if want_log else None)
    _check(lib.ccw_simulate(ti.handle, C.byref(p), _ptr(hd_cells) if n_hd else None,
                            _ptr(hd_vals) if n_hd else None, n_hd, seed & (2 ** 64 - 1),
                            _ptr(out), _ptr(log) if want_log else None, _stream(stream)))
    return out, (log if want_log else None)


def simulate_groups(ti: TI, groups, topk=1, seed=0, path_random=0, score_mode=0, precision=0,
                    want_log=False, want_counts=False, learned=0, ccf_tile=0, vt_ext=0,
                    boundary_cut=0, all_shift=0, stream=None):
    """``ccw_simulate_groups``: several grid sizes in one batch. ``groups`` is
    a list of dicts with keys grid, n_real, real_base and optionally hd_cells,
    hd_vals (CUDA tensors), out (the CUDA output) and out_host (a CPU copy of
    it, pinned for the streamed read-back). Returns a list of (realizations,
    log or None)."""
    lib = load()
    p = _Params()
    p.ndim = ti.ndim
    p.grid = _i3([1] * ti.ndim)
    p.topk = topk
    p.n_real = 1
    p.path_random = path_random
    p.score_mode = score_mode
    p.precision = precision
    p.learned = learned
    p.ccf_tile = ccf_tile
    p.vt_ext = vt_ext
    p.boundary_cut = boundary_cut
    p.all_shift = all_shift
    arr = (_Group * len(groups))()
    results = []
    keep = []
    for i, g in enumerate(groups):
        grid = tuple(g["grid"])
        n_real = int(g["n_real"])
        shape = (n_real,) + grid[::-1]
        out = g.get("out")
        if out is None:
            out = torch.empty(shape, dtype=torch.uint8, device="cuda")
        elif tuple(out.shape) != shape or out.dtype != torch.uint8:
            raise ValueError(f"out must be a CUDA uint8 tensor of shape {shape}")
        npch, _ = lattice(grid, ti.templ, ti.overlap)
        n_patches = 1
        for v in npch:
            n_patches *= v
        log = (torch.empty((n_real, n_patches, 4 + topk), dtype=torch.int32, device="cuda")
               if want_log else None)
        tjd = (ti.templ // ti.scale) ** ti.ndim
        counts = (torch.empty((n_real, n_patches, ti.n_facies, tjd), dtype=torch.uint8,
                              device="cuda") if want_counts else None)
        hc, hv = g.get("hd_cells"), g.get("hd_vals")
        n_hd = 0 if hv is None else int(hv.numel())
        arr[i].grid = _i3(grid)
        arr[i].n_real = n_real
        arr[i].real_base = int(g.get("real_base", 0))
        arr[i].hd_cells_dev = _ptr(hc) if n_hd else None
        arr[i].hd_vals_dev = _ptr(hv) if n_hd else None
        arr[i].n_hd = n_hd
        arr[i].out_dev = _ptr(out)
        arr[i].patch_log_dev = _ptr(log) if want_log else None
        arr[i].event_counts_dev = _ptr(counts) if want_counts else None
        arr[i].out_host = _host_ptr(g.get("out_host"), shape)
        keep.append((hc, hv))
        results.append((out, log, counts) if want_counts else (out, log))
    _check(lib.ccw_simulate_groups(ti.handle, C.byref(p), arr, len(groups), seed & (2 ** 64 - 1),
                                   _stream(stream)))
    return results


def ccf_search(ti: TI, de: torch.Tensor, hd=None, k=1, score_mode=0, seed=0, ctr=None,
               precision=0, stream=None):
    """``ccw_ccf_search`` on B data events de uint8 [B, T(, T), T]."""
    lib = load()
    B = de.shape[0]
    if ctr is None:
        ctr = torch.zeros((B, 2), dtype=torch.int32, device="cuda")
    dev = de.device
    ti_idx = torch.empty((B, k), dtype=torch.int32, device=dev)
    ti_sc = torch.empty((B, k), dtype=torch.int32, device=dev)
    ti_mm = torch.empty((B, k), dtype=torch.int32, device=dev)
    pick = torch.empty((B,), dtype=torch.int32, device=dev)
    _check(lib.ccw_ccf_search(ti.handle, B, _ptr(de), _ptr(hd), k, score_mode | (precision << 4),
                              seed & (2 ** 64 - 1), _ptr(ctr), _ptr(ti_idx), _ptr(ti_sc),
                              _ptr(ti_mm), _ptr(pick), _stream(stream)))
    return dict(topk_idx=ti_idx, topk_score=ti_sc, topk_mis=ti_mm, pick=pick)


def ccf_map(ti: TI, de: torch.Tensor, hd=None, score_mode=0, precision=0, stream=None):
    """``ccw_ccf_map``: (scores int32 [B, P_c], mismatches int32 [B, P_c])."""
    lib = load()
    B = de.shape[0]
    sc = torch.empty((B, ti.n_cand), dtype=torch.int32, device=de.device)
    mm = torch.empty((B, ti.n_cand), dtype=torch.int32, device=de.device)
    _check(lib.ccw_ccf_map(ti.handle, B, _ptr(de), _ptr(hd), score_mode | (precision << 4),
                           _ptr(sc), _ptr(mm),
                           _stream(stream)))
    return sc, mm


def idwt_paste(ti: TI, picks: torch.Tensor, origins: torch.Tensor, sg: torch.Tensor,
               stream=None):
    """``ccw_idwt_paste`` into sg (uint8, [ny, nx] or [nz, ny, nx]) in place."""
    lib = load()
    _check(lib.ccw_idwt_paste(ti.handle, int(picks.numel()), _ptr(picks), _ptr(origins),
                              _ptr(sg), _i3(list(sg.shape)[::-1]), _stream(stream)))
    return sg


def profile_enable(on: bool = True):
    _check(load().ccw_profile_enable(1 if on else 0))


def profile_read():
    """(timed launches, total ms, candidate evaluations, multiply-adds)."""
    n = C.c_int64()
    ms, ce, mac = C.c_double(), C.c_double(), C.c_double()
    _check(load().ccw_profile_read(C.byref(n), C.byref(ms), C.byref(ce), C.byref(mac)))
    return n.value, ms.value, ce.value, mac.value


def profile_read_phases():
    """(events ms, CCF ms, finish ms) of the profiled simulations since the
    last read."""
    v = (C.c_double * 3)()
    _check(load().ccw_profile_read_phases(v))
    return tuple(float(x) for x in v)


def profile_read_proposal():
    """(encoder ms, nearest-window selection + re-rank ms) of the profiled
    learned simulations since the last read."""
    v = (C.c_double * 2)()
    _check(load().ccw_profile_read_proposal(v))
    return tuple(float(x) for x in v)


def set_nn_path(path: int):
    """``ccw_set_nn_path``: 0 auto (tensor cores for small tables), 1 never the
    tensor cores, 2 one CTA per data event, 3 as 0 with twelve data events per
    tensor-core CTA whenever they fit."""
    _check(load().ccw_set_nn_path(int(path)))


def philox_host(ctr, key):
    """``ccw_philox_host``: Philox4x32-10 blocks of the counters ``ctr``
    (uint32 array [n, 4]) under ``key`` (2 words), computed on the host by the
    library's own generator; returns a uint32 array [n, 4]."""
    import numpy as np
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty_like(c)
    _check(load().ccw_philox_host(c.shape[0], c.ctypes.data_as(C.c_void_p),
                                  k.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p)))
    return out


def philox_dev(ctr: torch.Tensor, key, stream=None) -> torch.Tensor:
    """``ccw_philox_dev``: the same blocks computed on the GPU; ``ctr`` is a
    CUDA int32/uint32-valued tensor [n, 4] (int32 storage), returns [n, 4]."""
    import numpy as np
    if ctr.dim() != 2 or ctr.shape[1] != 4 or ctr.dtype != torch.int32:
        raise ValueError("ctr must be an int32 CUDA tensor [n, 4]")
    out = torch.empty_like(ctr)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    _check(load().ccw_philox_dev(ctr.shape[0], _ptr(ctr), k.ctypes.data_as(C.c_void_p),
                                 _ptr(out), _stream(stream)))
    return out


def launch_count() -> int:
    return int(load().ccw_launch_count())


class Net:
    """The learned proposal's encoder (``ccw_net_*``)."""

    def __init__(self, in_ch: int, tj: int, seed: int = 0):
        lib = load()
        h = C.c_void_p()
        rc = lib.ccw_net_create(in_ch, tj, seed & (2 ** 64 - 1), C.byref(h))
        if rc != 0:
            raise CCWError(lib.ccw_net_last_error().decode())
        self._h, self._lib = h, lib
        self.in_ch, self.tj = in_ch, tj
        self.n_params = int(lib.ccw_net_param_count(h))

    def __del__(self):
        try:
            if self._h and self._h.value:
                self._lib.ccw_net_free(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _chk(self, rc):
        if rc != 0:
            raise CCWError(self._lib.ccw_net_last_error().decode())

    def get(self, what=0):
        import numpy as np
        out = np.zeros(self.n_params, dtype=np.float32)
        self._chk(self._lib.ccw_net_get(self._h, what, out.ctypes.data_as(C.c_void_p)))
        return out

    def set(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._chk(self._lib.ccw_net_set(self._h, p.ctypes.data_as(C.c_void_p)))

    def embed(self, x: torch.Tensor, bf16=0, stream=None) -> torch.Tensor:
        n = x.shape[0]
        out = torch.empty((n, 64), dtype=torch.float32, device=x.device)
        self._chk(self._lib.ccw_net_embed(self._h, _ptr(x), n, bf16, _ptr(out), _stream(stream)))
        return out

    def train_step(self, anchors, cands, tau=0.1, lr=1e-3, wd=1e-4, bf16=1, apply=1,
                   stream=None) -> torch.Tensor:
        loss = torch.zeros(1, dtype=torch.float32, device=anchors.device)
        self._chk(self._lib.ccw_net_train_step(self._h, _ptr(anchors), anchors.shape[0],
                                               _ptr(cands), cands.shape[0], tau, lr, wd, bf16,
                                               apply, _ptr(loss), _stream(stream)))
        return loss
