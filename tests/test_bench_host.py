"""Host logic of bench.py (no GPU): the algorithmic byte model behind the roofline figures,
checked against counts worked out by hand, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_pass_bytes_at_256_hand_counted():
    # 2/3 rule at 256: K = 85, Mx = My = 171, Mz = 86
    M, L1, L2 = 171 * 171 * 86, 256 * 171 * 86, 256 * 256 * 86
    assert (M, L1, L2) == (2514726, 3764736, 5636096)
    b = bench.pass_bytes(256)
    assert b["p1_x_inverse_curl"] == 3 * M * 16 + 6 * L1 * 16
    assert b["p3_z_c2r_cross_r2c"] == 9 * L2 * 16
    assert b["p5_x_forward_project"] == 3 * L1 * 16 + 6 * M * 16
    # per right-hand side: 3.07 GB in FP64, 1.72 GB with FP32 intermediates
    assert round(sum(b.values()) / 1e9, 2) == 3.07
    assert round(sum(bench.pass_bytes(256, esz=8).values()) / 1e9, 2) == 1.72
    # fp32 form in a step: k written as 8-byte values, stage inputs 6/7 of the time 8 bytes
    b32 = bench.pass_bytes(256, esz=8, ksz=8, ysz=(6 * 8 + 16) / 7)
    assert b32["p5_x_forward_project"] == 3 * L1 * 8 + 3 * M * (64 / 7) + 3 * M * 8


def test_step_kernel_bytes_hand_counted():
    cells = 3 * 171 * 171 * 86
    b = bench.step_kernel_bytes(256)
    # stage sums: BS5 inputs 2..8 read u and 1,2,3,4,5,6,6 k's and write one field: 41 fields
    assert b["stage_sum"] == 41 * cells * 16
    # error norm: u_n, u_{n+1} and the 7 k's with b_j != bhat_j
    assert b["err_norm_partials"] == 9 * cells * 16
    b8 = bench.step_kernel_bytes(256, ksz=8)
    # fp32: k's and intermediate outputs 8 bytes, u and u_{n+1} 16
    assert b8["stage_sum"] == cells * (7 * 16 + 27 * 8 + 6 * 8 + 16)
    assert b8["err_norm_partials"] == cells * (2 * 16 + 7 * 8)


def test_at_error_interpolates_log_log():
    curve = [{"l2_error": 1e-6, "rhs_evals": 100}, {"l2_error": 1e-8, "rhs_evals": 400}]
    assert bench.at_error(curve, 1e-7, "rhs_evals") == pytest.approx(200.0, rel=1e-12)
    assert bench.at_error(curve, 1e-9, "rhs_evals") is None


def test_reference_arm_prints_one_contract_line():
    # a small grid keeps the test short; the arm is the same code at 256^3
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "4",
                        "--warmup", "0", "--grid", "32"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    for key in ("metric", "unit", "n_gpus", "steps", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in d
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    # the oracle runs on every host core the memory allows (here 4 jobs: up to 4 workers)
    assert d["cpu_baseline"]["cores"] == min(4, bench.cpu_workers(4, 32))
    assert d["cpu_baseline"]["nproc"] >= d["cpu_baseline"]["cores"]
    assert d["config"]["grid"] == [32, 32, 32]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]
