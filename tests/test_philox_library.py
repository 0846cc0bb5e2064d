"""The library's Philox4x32-10 (the generator of every draw of Algorithm 1)
against the published known-answer vectors and against the oracle's own
Philox, written separately in plain C, on 10^6 counters: on the host
(ccw_philox_host, the kernels' source compiled for the CPU) and on the GPU
(ccw_philox_dev)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def counters(n, seed=0):
    """10^6-scale counters: the (realization, patch, purpose, 0) words the
    library draws with, plus random full-range words."""
    rng = np.random.default_rng(seed)
    c = np.zeros((n, 4), np.uint32)
    h = n // 2
    c[:h, 0] = np.arange(h) % 4096             # realization
    c[:h, 1] = np.arange(h) // 4096            # patch
    c[:h, 2] = np.arange(h) % 2                # purpose (0 pick, 1 path)
    c[h:] = rng.integers(0, 2 ** 32, size=(n - h, 4), dtype=np.uint64).astype(np.uint32)
    return c


@pytest.fixture(scope="module")
def ccw():
    import paper_2404_00441_gb300 as m
    from paper_2404_00441_gb300 import build
    build.build()
    m.load()
    return m


def test_library_philox_known_answers_host(ccw):
    for ctr, key, out in kat_rows():
        assert ccw.philox_host(np.array([ctr], np.uint32), key).tolist() == [out]


@pytest.mark.parametrize("key", [(0, 0), (2, 0), (0xDEADBEEF, 0x12345678)])
def test_library_philox_equals_oracle_on_a_million_counters_host(ccw, key):
    c = counters(1_000_000, seed=key[0] & 0xFF)
    assert np.array_equal(ccw.philox_host(c, key), O.philox_many(c, key))


@pytest.mark.gpu
def test_library_philox_equals_oracle_on_a_million_counters_gpu(ccw):
    torch = pytest.importorskip("torch")
    rows = kat_rows()
    kat = np.array([r[0] for r in rows], np.uint32)
    for ctr, key, out in rows:
        got = ccw.philox_dev(torch.from_numpy(np.array([ctr], np.uint32).view(np.int32)).cuda(),
                             key).cpu().numpy().view(np.uint32)
        assert got.tolist() == [out]
    assert kat.shape == (3, 4)
    for key in [(0, 0), (2, 0), (0xDEADBEEF, 0x12345678)]:
        c = counters(1_000_000, seed=key[0] & 0xFF)
        got = ccw.philox_dev(torch.from_numpy(c.view(np.int32)).cuda(), key)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy().view(np.uint32), O.philox_many(c, key))
