"""The device arm's JSON line (the bench contract) from a synthetic run
result: every required key, the whole-job arithmetic and JSON-serialisable
values, checked on the CPU."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _res(nc=314_389):
    stage_ms = {name: 0.1 for name in bench.STAGES}
    stage_ms["network"] = 1.6
    return dict(elapsed_ms=50.0, net_ms=[1.6, 1.6], stage_ms=stage_ms, launches=240,
                clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 16},
                e2e_s=0.0625, nc=nc, nf=2_596_650, nv=330_000, fp64=None, fp32=None, paper=None,
                affine_frac=0.9)


def test_line_has_the_contract_keys_and_arithmetic():
    args = argparse.Namespace(steps=20, warmup=3, nz=37, no_fp64=True, no_cpu_baseline=True)
    line = bench.result_line(_res(), args, 1, 50.0)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] == 400.0 and line["ms_per_step"] == 2.5 and line["steps"] == 20
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["dtype"] == "bf16"
    assert "workload" in line["config"] and "model" not in line["config"]
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "tensor" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(r["achieved"] - bench.network_flops_per_patch() * 314_389 / 1.6e-3 / 1e12) < 1e-9
    e = line["e2e"]
    assert e["value"] == 20 / 0.0625 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] == 240 and set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    assert line["stages"]["parallelepiped_cells"] == 0.9
    json.dumps(line)


def test_whole_job_value_scales_with_ranks():
    args = argparse.Namespace(steps=10, warmup=3, nz=37, no_fp64=True, no_cpu_baseline=True)
    one = bench.result_line(_res(), args, 1, 20.0)
    four = bench.result_line(_res(), args, 4, 20.0)      # 4 replicas in the same (slowest-rank) time
    assert four["value"] == 4 * one["value"] and four["n_gpus"] == 4
    assert four["config"]["parallelism"] == "replicas x4"
