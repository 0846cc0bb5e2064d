"""ccw_ccf_search_noalloc: the search for callers that cannot allocate device
memory while they run (a serving process that reserved all of HBM for its own
pool, a latency-critical loop that must not pay for a driver allocation). It
must give exactly what ccw_ccf_search gives, call after call, although every
call reuses the same scratch array compiled into the library.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCRATCH_BYTES = 4 * 1024 * 1024          # CCW_NOALLOC_SCRATCH_BYTES in include/ccw.h


@pytest.fixture(scope="module")
def env():
    import paper_2404_00441_gb300 as ccw
    lib = ccw.load()
    P, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
    lib.ccw_ccf_search_noalloc.argtypes = [P, i32, P, P, i32, i32, u64, P, P, P, P, P, P]
    lib.ccw_ccf_search.argtypes = [P, i32, P, P, i32, i32, u64, P, P, P, P, P, P]
    lib.ccw_last_error.restype = C.c_char_p
    return ccw, lib


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _call(lib, fn, g, de, hd, k, seed, ctr):
    B = de.shape[0]
    outs = [torch.full((B, k), -7, dtype=torch.int32, device="cuda") for _ in range(3)]
    pick = torch.full((B,), -7, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(g.handle, B, _p(de), _p(hd), k, 0, seed, _p(ctr), _p(outs[0]),
                          _p(outs[1]), _p(outs[2]), _p(pick), stream)
    assert rc == 0, lib.ccw_last_error()
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs] + [pick.cpu().numpy()]


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_noalloc_search_equals_search_on_two_calls_in_a_row(env, case):
    ccw, lib = env
    rng = np.random.default_rng(3)
    if case == "2d":
        ti = configs.ribbon_ti_250()
        F, J, T, Ov, K = 2, 1, 40, 10, 5
    else:
        from workloads import synth
        ti = synth.tube_lobe_ti_3d(44, 40, 36, seed=5)
        F, J, T, Ov, K = 4, 1, 12, 2, 7
    g = ccw.TI(torch.from_numpy(ti).cuda(), F, J, T, Ov)
    for call in range(2):
        B = 12 + call * 5
        de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=2, F=F)
        de[call] = 255                       # one empty data event per call
        hd[call] = 255
        ctr = torch.from_numpy(
            np.stack([rng.integers(0, 99, B), rng.integers(0, 999, B)], 1).astype(np.int32)
        ).cuda()
        de_t, hd_t = torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda()
        seed = int(rng.integers(0, 2 ** 62))
        ref = _call(lib, "ccw_ccf_search", g, de_t, hd_t, K, seed, ctr)
        got = _call(lib, "ccw_ccf_search_noalloc", g, de_t, hd_t, K, seed, ctr)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), f"call {call}"


def test_noalloc_rejects_batches_beyond_the_scratch_array(env):
    ccw, lib = env
    ti = configs.ribbon_ti_250()
    g = ccw.TI(torch.from_numpy(ti).cuda(), 2, 1, 40, 10)
    tiles = 2 * 7                      # 106 x 106 candidates in 64 x 16 tiles
    k = 64
    B = SCRATCH_BYTES // (8 * tiles * k) + 1
    de = torch.full((B, 40, 40), 255, dtype=torch.uint8, device="cuda")
    ctr = torch.zeros((B, 2), dtype=torch.int32, device="cuda")
    outs = [torch.empty((B, k), dtype=torch.int32, device="cuda") for _ in range(3)]
    pick = torch.empty((B,), dtype=torch.int32, device="cuda")
    rc = lib.ccw_ccf_search_noalloc(g.handle, B, _p(de), None, k, 0, 1, _p(ctr), _p(outs[0]),
                                    _p(outs[1]), _p(outs[2]), _p(pick), None)
    assert rc == -1
    assert b"scratch" in lib.ccw_last_error()


def test_noalloc_search_stays_out_of_the_profiler(env):
    """With profiling on, the search that allocates nothing still gives the
    search's results and adds no timed launch: the profiler's events and
    counters would need allocations."""
    ccw, lib = env
    rng = np.random.default_rng(5)
    ti = configs.ribbon_ti_250()
    F, J, T, Ov, K = 2, 1, 40, 10, 3
    g = ccw.TI(torch.from_numpy(ti).cuda(), F, J, T, Ov)
    B = 9
    de, hd = configs.structured_events(ti, T, Ov, B, rng, n_hd=2, F=F)
    ctr = torch.from_numpy(np.stack([np.arange(B), np.arange(B) + 3], 1).astype(np.int32)).cuda()
    de_t, hd_t = torch.from_numpy(de).cuda(), torch.from_numpy(hd).cuda()
    ref = _call(lib, "ccw_ccf_search", g, de_t, hd_t, K, 17, ctr)
    ccw.profile_enable(True)
    try:
        ccw.profile_read()
        for _ in range(2):
            got = _call(lib, "ccw_ccf_search_noalloc", g, de_t, hd_t, K, 17, ctr)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
        launches = ccw.profile_read()[0]
    finally:
        ccw.profile_enable(False)
    assert launches == 0
