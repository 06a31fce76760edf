"""Host logic of bench.py's multi-GPU path on CPU: two gloo ranks.

With N > 1 every rank runs its own replica and its own shard of the alpha
sweep; the timed region is bracketed by barriers and the slowest rank's time
is the job's time.  These checks run the sharding and the cross-rank
reductions as two gloo processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w = bench.dist_init("gloo")
    items = list(range(64))
    mine = bench.shard(items, r, w)
    bench.barrier()
    t_max = bench.max_over_ranks(1.0 + r)
    n_sum = bench.sum_over_ranks(len(mine))
    out[rank] = (tuple(mine), t_max, n_sum)
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    a, b = out[0], out[1]
    assert set(a[0]).isdisjoint(b[0]) and set(a[0]) | set(b[0]) == set(range(64))
    assert a[1] == b[1] == 2.0  # the slowest rank's time
    assert a[2] == b[2] == 64.0  # every instance counted once


@pytest.mark.parametrize("n,world", [(64, 1), (64, 3), (5, 8), (0, 2)])
def test_shard_partitions(n, world):
    items = list(range(n))
    parts = [bench.shard(items, r, world) for r in range(world)]
    assert sum(parts, []) == items
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_single_rank_reductions_are_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.sum_over_ranks(7) == 7.0


def test_reference_arm_prints_one_contract_line():
    # The reference arm (the oracle on the host cores) runs without a GPU and
    # prints one JSON line with the keys the benchmark contract asks for.
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--workload", "dambreak_small_dp0.02"], cwd=root, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "dambreak_small_dp0.02" and d["steps"] == 2


def test_accuracy_errors_per_window_and_from_files(tmp_path):
    # Probe series of the two forms that differ by a known amount after
    # 0.15 s: the windows before it report zero, the ones after it the
    # difference over Hc (wave) and rho0 g Hc (pressure); the comparison read
    # back from the files that --accuracy-dir writes is the same.
    from paper_2306_01959_gb300 import workloads as wl

    case = wl.by_name("dambreak_obstacle_dp0.01")
    hc = case.column[2]
    a = [(0.01 * (k + 1), [0.5, 0.4], [100.0, 200.0]) for k in range(30)]
    b = [(t, [w + (0.011 if t > 0.15 else 0.0) for w in wv], [p + (981.0 if t > 0.15 else 0.0) for p in pv])
         for t, wv, pv in a]
    out = bench.accuracy_errors({"mixed": a, "fp64": b}, case.name, 0.3)
    assert out["mixed_vs_fp64"]["0.1"] == {"wave_over_Hc": 0.0, "pressure_over_rho0_g_Hc": 0.0}
    assert abs(out["mixed_vs_fp64"]["0.2"]["wave_over_Hc"] - round(0.011 / hc, 5)) < 1e-12
    assert abs(out["mixed_vs_fp64"]["0.3"]["pressure_over_rho0_g_Hc"] - round(981.0 / (1000.0 * 9.81 * hc), 5)) < 1e-12
    assert "mixed_vs_mixed_nudged_1nm" not in out
    for name, rows in (("mixed", a), ("fp64", b)):
        (tmp_path / f"accuracy_{case.name}_{name}.json").write_text(
            json.dumps({"workload": case.name, "physical_time_s": 0.3, "rows": rows,
                        "fp64_reference": "each ordered pair" if name == "fp64" else None}))
    r = subprocess.run([sys.executable, "bench.py", "--accuracy-from", str(tmp_path)], capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.abspath(bench.__file__)), check=True)
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert got["mixed_vs_fp64"] == out["mixed_vs_fp64"] and got["fp64_reference"] == "each ordered pair"
