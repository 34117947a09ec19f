"""Host logic of bench.py (CPU): the algorithmic byte model of one sweep launch
(the numerator of the roofline fraction), the rule that an ncu traffic record
counts only for the kernel source and the sweep kernel it was captured from,
and the reference arm's JSON line (the oracle on the host cores).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# the 2048 x 2048 power grid in 32 x 32 tiles (plan statistics)
GRID2048 = {"nports": 516096, "sum_p2": 65282048, "sum_tri": 32899072}


@pytest.mark.parametrize("prec,kernel,alg,ovh", [
    # packed symmetric kernels read the blocks on and above the diagonal:
    # algorithmic 2 B x 32,899,072 + 516,096 ports x 5 wave words of 4 B (the
    # twin's outgoing wave, c, the new outgoing wave, the twin's pair for the
    # residual); overhead per port: the port's own pair (8 B), twin index and
    # run byte (5 B), residual coefficients (8 B)
    (3, 11, 2 * 32899072 + 516096 * 20, 516096 * 21),
    (2, 11, 2 * 32899072 + 516096 * 20, 516096 * 21),
    (3, 9, 2 * 32899072 + 516096 * 20, 516096 * 21),
    (1, 9, 4 * 32899072 + 516096 * 20, 516096 * 21),
    # full-matrix kernels read every entry; FP64 waves and coefficients
    (1, 1, 4 * 65282048 + 516096 * 20, 516096 * 21),
    (0, 1, 8 * 65282048 + 516096 * 40, 516096 * (16 + 5 + 16)),
    # the double-float FP64 sweep reads the packed blocks as 8-byte hi/lo pairs
    (0, 12, 8 * 32899072 + 516096 * 40, 516096 * (16 + 5 + 16)),
])
def test_sweep_bytes_follow_the_byte_model(prec, kernel, alg, ovh):
    assert bench.sweep_bytes(dict(GRID2048, sweep_kernel=kernel), prec) == (alg, ovh)


def test_fp16_sweep_bytes_of_the_bench_line():
    # 65.8 MB of stored entries + 10.3 MB of wave words: 76.12 MB per sweep
    # (algorithmic_bytes_per_launch); 10.8 MB of port metadata apart
    assert bench.sweep_bytes(dict(GRID2048, sweep_kernel=11), 3) == (76120064, 10838016)


def test_batched_sweep_bytes_count_every_column():
    # the batched sweep reads every entry once for all R columns
    alg, ovh = bench.sweep_bytes(dict(GRID2048, sweep_kernel=11), 2, nrhs=64)
    assert alg == 2 * 65282048 + 516096 * 5 * 4 * 64
    assert ovh == 516096 * (2 * 4 * 64 + 5 + 16)


def test_traffic_record_needs_its_own_source_and_kernel(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as fh:
        rec = json.load(fh)
    monkeypatch.setattr(bench, "sweep_kernel_source_hash", lambda: rec["kernel_source_sha256"])
    for name, prec in (("fp32", 1), ("bf16", 2), ("fp16", 3)):
        entry = rec["per_launch"][name]
        for k in entry["sweep_kernels"]:
            assert bench.traffic_record(prec, {"sweep_kernel": k}, "power_grid") == entry["bytes"]
        others = [k for k in range(1, 12) if k not in entry["sweep_kernels"]]
        assert all(bench.traffic_record(prec, {"sweep_kernel": k}, "power_grid") is None for k in others)
        k0 = entry["sweep_kernels"][0]
        assert bench.traffic_record(prec, {"sweep_kernel": k0}, "thermal") is None
    # a changed kernel source voids the record
    monkeypatch.setattr(bench, "sweep_kernel_source_hash", lambda: "0" * 64)
    assert bench.traffic_record(3, {"sweep_kernel": rec["per_launch"]["fp16"]["sweep_kernels"][0]},
                                "power_grid") is None


def test_recorded_traffic_is_near_the_algorithmic_bytes():
    # the ncu DRAM bytes of a cold sweep launch read every stored byte once:
    # within 10% of the byte model (padding of the 16x16 blocks adds, cached
    # port data subtracts)
    with open(os.path.join(ROOT, "profiles", "sweep_traffic.json")) as fh:
        rec = json.load(fh)
    for name, prec in (("fp32", 1), ("bf16", 2), ("fp16", 3)):
        entry = rec["per_launch"][name]
        alg, ovh = bench.sweep_bytes(dict(GRID2048, sweep_kernel=entry["sweep_kernels"][0]), prec)
        model = alg + ovh
        assert abs(entry["bytes"] / model - 1) < 0.1, (name, entry["bytes"], model)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["higher_is_better"] is True and line["value"] > 0
    assert abs(line["value"] - bench.SAMPLE_N ** 2 / (line["ms_per_step"] * 1e-3)) <= 1e-6 * line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench.host_cores() and cb["value"] == line["value"]
    assert cb["sample"] and cb["cpu_model"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # the workload named is the sample the arm times, and which workload it samples
    assert line["config"]["workload"].startswith("power grid 512x512")
    assert line["config"]["sample_of"].startswith("power grid 2048x2048")
    assert line["config"]["n"] == bench.SAMPLE_N ** 2


def test_profiling_options_name_their_workload(monkeypatch):
    # the smaller thermal grid and the band-solve choice that the profile
    # commands use reach the line's config; the defaults keep the benchmark's
    # 128 x 128 x 32 grid with 400 boxes
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "thermal", "--thermal-grid", "96",
                                      "--thermal-boxes", "225", "--band-solve", "1"])
    args = bench.parse()
    cfg = bench.workload_config(args)
    assert args.band_solve == 1
    assert cfg["n"] == 96 * 96 * 32 and "96x96x32" in cfg["workload"] and "225 random boxes" in cfg["workload"]
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "thermal"])
    args = bench.parse()
    cfg = bench.workload_config(args)
    assert args.band_solve == 0
    assert cfg["n"] == 524288 and "128x128x32" in cfg["workload"] and "400 random boxes" in cfg["workload"]
