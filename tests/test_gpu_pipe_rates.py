"""The per-SM issue rates behind bench.py's SFU and FP32 rooflines, measured on the GPU.

bench.py divides the kernels' algorithmic transcendental and FP32 work by peaks built
from per-SM issue rates (ex2.approx 32 per clock, lg2.approx 16, FFMA 122 lane operations).
This test measures those rates with a microbenchmark (tests/pipe_rates.cu: independent
chains of one PTX instruction, two 1024-thread blocks per SM) while nvidia-smi samples the
SM clock of the same GPU, and checks them against bench.py's constants.  Run with -s to
see the measured rates.
"""
import json
import os
import shutil
import statistics
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_sfu_and_fp32_issue_rates_match_bench_constants(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "pipe_rates")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    os.path.join(HERE, "pipe_rates.cu"), "-o", exe], check=True)
    import bench
    smi = subprocess.Popen(["nvidia-smi", f"--id={bench.smi_device_id(0)}", "--query-gpu=clocks.sm",
                            "--format=csv,noheader,nounits", "-lms", "50"],
                           stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    try:
        run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    finally:
        smi.terminate()
        clocks_out, _ = smi.communicate(timeout=10)
    assert run.returncode == 0, run.stdout + run.stderr
    res = json.loads(run.stdout)
    mhz = [float(x) for x in clocks_out.split() if x.replace(".", "").isdigit()]
    busy = [m for m in mhz if m > 0.8 * max(mhz)] if mhz else []
    if not busy:
        pytest.skip("nvidia-smi gave no SM clock samples")
    sm_mhz = statistics.median(busy)
    per_clk = {k: v * 1e9 / (res["sms"] * sm_mhz * 1e6) for k, v in res["total_gops"].items()}
    print(json.dumps({"sms": res["sms"], "sm_mhz_median": sm_mhz, "total_gops": res["total_gops"],
                      "per_sm_per_clk": {k: round(v, 2) for k, v in per_clk.items()}}))
    expect = {"ex2.approx.ftz.f32": bench.MUFU_EX2_PER_CLK_SM, "lg2.approx.ftz.f32": bench.MUFU_LG2_PER_CLK_SM,
              "fma.rn.f32": bench.FP32_PER_CLK_SM}
    for name, want in expect.items():
        assert abs(per_clk[name] - want) <= 0.1 * want, (name, per_clk[name], want)
