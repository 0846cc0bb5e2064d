"""The benchmark's JSON contract, checked on the CPU: the line assembled from
measurements carries every required key, and the reference arm (the oracle
on the host cores) prints a complete line."""
import json
import os
import subprocess
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(**kw):
    a = dict(steps=5, warmup=3, workload="c2", gpus=1)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_line_has_every_required_key():
    m = dict(total_ms=30.0, kern_ms=20.0, instr_ms=40.0, macs=1e10, cand_evals=5e8, n_launch=620,
             launches=1870, clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
             precision=2, tile=0xA040010, ndim=2, total_real=1, cells_per_step=4e6,
             e2e_ms=31.0, h2d=3600, d2h=4000000, learned=None, autotune={"chosen": "x"})
    line = bench.ours_line(_args(), 1, m)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "gpu_launches", "clocks", "e2e"):
        assert k in line, k
    assert line["config"]["workload"].startswith("c2")
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert line["roofline"]["bound"] == "tensor" and "k_ccf_tcs" in line["roofline"]["kernel"]
    assert abs(line["value"] - 5 * 4e6 / 0.030) < 1e-6 * line["value"]
    assert abs(line["roofline"]["frac"] - line["roofline"]["achieved"] / line["roofline"]["peak"]) < 1e-12
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    assert line["dtype"] == "bf16" and line["scaling"] == "weak"
    json.dumps(line)
    m32 = dict(m, precision=0, tile=1)
    line32 = bench.ours_line(_args(), 1, m32)
    assert line32["roofline"]["bound"] == "alu" and line32["dtype"] == "f32"


def test_reference_arm_prints_a_complete_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "c1", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "1"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_realization_parallel_oracle_baseline():
    """The all-cores oracle figure: one spawned process per realization, the
    clock started together after every worker has prepared its TI."""
    from workloads import synth
    ti = synth.ribbon_ti(120, 120, n_ribbons=6, seed=4, target=0.3, tol=0.2)
    w = dict(ti=ti, F=2, J=1, grid=(100, 90), T=16, O=4, K=3, hd=None, seed=3)
    wall = bench.oracle_parallel(w, 12, 2)
    assert 0.0 < wall < 60.0
    assert bench.host_cores() >= 1


def test_gpus_flag_starts_that_many_ranks():
    """`bench.py --gpus N` outside a launcher runs N ranks under
    torch.distributed.run on 127.0.0.1 with the same arguments."""
    cmd = bench.rank_command(["--gpus", "4", "--steps", "2"], 4)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=4" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-4:] == ["--gpus", "4", "--steps", "2"]
