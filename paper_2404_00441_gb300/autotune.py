"""Autotuner of the CCF tiling: picks the precision (FP32 lanes, FP16 or BF16
tensor cores) and the ``ccf_tile`` value of ``ccw_params`` by timing whole
simulation calls of the caller's batch shape. Every choice gives the same
results (the arithmetic is exact in all of them), so the tuner only looks at
time.

Results are cached in a JSON file (``CCW_AUTOTUNE_CACHE``, default
``~/.cache/paper_2404_00441_gb300/autotune.json``) keyed by the device and
the batch shape.
"""
from __future__ import annotations

import json
import os

import torch

from . import ccw


def _cache_path() -> str:
    p = os.environ.get("CCW_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2404_00441_gb300",
                        "autotune.json")


LANES = (2, 3, 4, 6, 8)   # realization lanes tried on the best tiling


def candidates(ti: "ccw.TI", precisions=(0, 1, 2)):
    """(precision, ccf_tile) pairs the library accepts for this TI."""
    out = []
    for p in precisions:
        if p == 0:
            for nb in ((1, 2, 4, 8) if ti.ndim == 2 else (1, 2, 4)):
                out.append((0, nb))
        else:
            # tensor cores: bit 24 = lanes-on-candidates epilogue, bit 25 =
            # streamed operands (the only form in 3D)
            # bit 26 = three stages in the streamed kernel, bit 29 = four
            # (else two); bits 27-28 = template rows per stage Tj / 2^v
            streamed = (2, 6, 2 | 8, 2 | 16, 6 | 8, 6 | 16, 2 | 16 | 32, 2 | 8 | 32)
            flags = (0, 1) + streamed if ti.ndim == 2 else streamed
            for fl in flags:
                for nt in (16, 32, 64, 128):
                    for mt in (1, 2, 4):
                        if mt * nt <= 512:
                            out.append((p, nt | (mt << 16) | (fl << 24)))
    return out


def _key(ti, groups, topk, score_mode, learned, precisions, vt_ext=0, boundary_cut=0):
    dev = torch.cuda.get_device_name()
    shape = [(tuple(g["grid"]), int(g["n_real"]), 0 if g.get("hd_vals") is None
              else int(g["hd_vals"].numel())) for g in groups]
    return json.dumps([dev, ti.dims, ti.n_facies, ti.level, ti.templ, ti.overlap, shape, topk,
                       score_mode, learned, list(precisions), vt_ext, boundary_cut])


def _time_call(fn, reps):
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(ti: "ccw.TI", groups, topk=1, seed=0, score_mode=0, learned=0, precisions=(0, 1, 2),
         reps=2, use_cache=True, vt_ext=0, boundary_cut=0):
    """Times every candidate tiling on simulate_groups(ti, groups, ...), then
    the fastest one with the realizations split into 2-8 concurrent lanes,
    and returns (precision, ccf_tile, {"p<precision>/<tile>": ms}).
    Candidates the library refuses (shared memory, exactness bounds) are
    skipped."""
    key = _key(ti, groups, topk, score_mode, learned, precisions, vt_ext, boundary_cut)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        c = cache[key]
        return c["precision"], c["ccf_tile"], c["times"]
    times = {}
    best = None
    for prec, tile in candidates(ti, precisions):
        def call():
            ccw.simulate_groups(ti, groups, topk=topk, seed=seed, score_mode=score_mode,
                                precision=prec, learned=learned, ccf_tile=tile,
                                vt_ext=vt_ext, boundary_cut=boundary_cut)
        try:
            call()   # builds the plan and captures its graph
        except ccw.CCWError:
            continue
        ms = _time_call(call, reps)
        times[f"p{prec}/{tile:#x}"] = ms
        if best is None or ms < best[2]:
            best = (prec, tile, ms)
    if best is None:
        raise ccw.CCWError("no tiling accepted for this batch")
    # second stage: the best tiling with the realizations split into lanes
    # whose wavefront chains run concurrently (ccf_tile bits 20-22)
    total_real = sum(int(g["n_real"]) for g in groups)
    if not learned and not (best[1] >> 30) & 1:
        for lanes in LANES:
            if lanes > total_real:
                break
            prec, tile = best[0], best[1] | ((lanes - 1) << 20)

            def call():
                ccw.simulate_groups(ti, groups, topk=topk, seed=seed, score_mode=score_mode,
                                    precision=prec, learned=learned, ccf_tile=tile,
                                    vt_ext=vt_ext, boundary_cut=boundary_cut)
            try:
                call()
            except ccw.CCWError:
                continue
            ms = _time_call(call, reps)
            times[f"p{prec}/{tile:#x}"] = ms
            if ms < best[2]:
                best = (prec, tile, ms)
    if use_cache:
        cache[key] = {"precision": best[0], "ccf_tile": best[1], "times": times}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best[0], best[1], times
