"""The JSON contract of bench.py's reference arm (the FP64 oracle timed on the
host cores), which runs without a GPU: one line with the metric, unit and
config of the GPU arm, a ``cpu_baseline`` that describes the run and an
``e2e`` object with no host-device traffic; ranks other than 0 exit at once."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    # a 2048^3 workload keeps the test short; the contract does not depend on the size
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "3", "--size", "2048"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0 and d["unit"] == "TFLOP/s"
    assert d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["config"]["workload"] and d["config"]["m"] == d["config"]["n"] == d["config"]["k"] == 2048
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def _synthetic_run():
    """An ``out`` dict and legs shaped like a full default run of bench.py."""
    mode_entry = {"tflops": 512.3456789, "ms": 68.123456, "rel_fro_vs_fp64": 4.1234567e-7,
                  "selected": "fp16x"}
    points = [{"size": n, "s": s, "modes": {m: dict(mode_entry) for m in
                                            ("fp32", "tf32x", "fp16x", "fp16x_scaled", "auto",
                                             "auto_tuned")},
               "cublas_cgemm_tflops": 76.2, "auto_pick_by_tol": {"0": "tf32x", "0.001": "fp16x"},
               "auto_speedup_vs_fp32": 12.1 + s, "auto_err_ratio_vs_fp32": 0.13 + s / 100}
              for n in (1024, 2048, 4096, 8192, 16384) for s in (0, 8, 20, 40)]
    variant = {"s_per_slice": 1.95e-3, "s_per_slice_eager": 2.1e-3, "slices_timed": 16,
               "tflops": 250.0, "amplitude_rel_err_vs_fp64": 9.6e-7,
               "routing": {"gemms": {"fp16x": 1, "fp32": 700},
                           "fraction": {"fp16x": 0.001, "fp32": 0.999},
                           "flops_fraction": {"fp16x": 0.0, "fp16x_scaled": 0.93, "tf32x": 0.07,
                                              "fp32": 0.0, "bf16x3": 0.0}}}
    contraction = {"workload": "x" * 400, "auto": dict(variant), "auto_t0.5": dict(variant),
                   "auto_paper_rule": dict(variant), "fp32": dict(variant, s_per_slice=11.6e-3),
                   "speedup_vs_fp32": 5.9, "speedup_vs_fp32_t0.5": 7.4}
    legs = {
        "candidates": {m: dict(mode_entry) for m in ("tf32x", "bf16x3", "auto_3m", "fp16x_3m")},
        "hbm_kernels": {"peak_gbs": 6784.5, "exp_stats": {"GB/s": 6300.0, "frac": 0.93, "ms": 1.0,
                                                          "bytes": 1}},
        "sweep": {"workload": "y" * 300, "points": points},
        "sgemm": {"points": points[:4]},
        "contraction": contraction,
        "contraction_seed2_order": dict(contraction),
        "plain_small": {"s_per_batch_grouped_cuda_graph": 5.0e-4, "fidelity_vs_fp64": 1 - 1.4e-13},
        "differentiation": {"auto_s": 0.15, "fp32_s": 0.41, "speedup_vs_fp32": 2.7,
                            "auto_grad_rel_l2_vs_fp64": 1.2e-5, "fp32_grad_rel_l2_vs_fp64": 2.5e-5,
                            "cheapest_order": {"auto_s": 0.129, "fp32_s": 0.139}},
        "precision_at_scale": dict(contraction, sampled_slices_fidelity_vs_fp64=1 - 4.4e-13),
    }
    out = {"metric": "m", "value": 512.0, "unit": "TFLOP/s", "n_gpus": 1, "steps": 20,
           "warmup": 5, "ms_per_step": 68.7, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64", "data": "synthetic",
           "config": {"workload": "CGEMM m=n=k=16384 " + "z" * 120, "m": 16384},
           "gpu_launches": 160, "clocks": {"sm_mhz": 1462.0, "sm_max_mhz": 2070.0, "reasons": []},
           "stages": {k: {"ms_per_step": 1.0, "launches": 20} for k in
                      ("stats", "select", "split", "gemm_tc", "gemm_simt")},
           "roofline": {"bound": "tensor", "achieved": 1595.0, "peak": 1714.8, "unit": "TFLOP/s",
                        "frac": 0.93, "traffic": 1.5e11, "kernel": "cgemm_tc_kernel (fp16x)",
                        "peak_source": "measured bf16 sustained"},
           "error": {"rel_fro_vs_fp64": 4.1e-7, "sample": "16 output rows"},
           "cpu_baseline": {"value": 0.12, "unit": "TFLOP/s", "cores": 16, "kind": "oracle",
                            "sample": "16 of 16384 output rows"},
           "fp32": {"simt_tflops": 40.6, "cublas_cgemm_tflops": 76.2},
           "e2e": {"value": 420.0, "unit": "TFLOP/s", "h2d_bytes_per_step": 2 * 16384 ** 2 * 8,
                   "d2h_bytes_per_step": 16384 ** 2 * 8}}
    return out, legs


def test_contract_line_is_short_and_keeps_the_contract_keys():
    sys.path.insert(0, ROOT)
    import bench

    out, legs = _synthetic_run()
    line = bench.contract_line(out, legs)
    text = json.dumps(line)
    assert len(text) <= bench.LINE_LIMIT, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "gpu_launches", "clocks", "roofline", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["d2h_bytes_per_step"] > 0
    summ = line["legs"]
    assert summ["contraction_5x6_d14"]["fp32_ms_per_slice"] > summ["contraction_5x6_d14"][
        "auto_ms_per_slice"]
    assert "precision_5x8_d12" in summ and "differentiation_4x5_d12" in summ
    # a failed leg keeps a short error, and an oversized summary is trimmed, not the contract
    legs["sweep"] = {"error": "RuntimeError: " + "e" * 2000}
    legs.update({f"extra{i}": {"error": "x" * 500} for i in range(20)})
    line = bench.contract_line(out, legs)
    assert len(json.dumps(line)) <= bench.LINE_LIMIT
    assert line["roofline"]["frac"] == 0.93 and line["e2e"]["value"] == 420.0


def test_legs_go_to_stderr_and_file(tmp_path, capsys):
    sys.path.insert(0, ROOT)
    import bench

    _, legs = _synthetic_run()
    path = tmp_path / "sub" / "legs.json"
    bench.emit_legs(legs, str(path))
    err = capsys.readouterr().err.splitlines()
    assert [json.loads(ln)["leg"] for ln in err] == list(legs)
    assert json.load(open(path))["sweep"]["points"][0]["size"] == 1024
