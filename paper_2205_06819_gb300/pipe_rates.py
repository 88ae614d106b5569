"""Measure the per-SM issue rates of the SFU approximations and of FFMA on the local GPU
(the denominators of the forward kernel's SFU roofline).

    python -m paper_2205_06819_gb300.pipe_rates

compiles csrc/pipe_rates.cu for sm_103a into the package's build folder, runs it while
nvidia-smi samples the SM clock, and prints one JSON line: total rates (G instructions/s)
and rates per SM per clock at the median sampled clock.
"""
from __future__ import annotations

import json
import os
import statistics
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    src = os.path.join(HERE, "csrc", "pipe_rates.cu")
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "pipe_rates")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", src, "-o", exe],
                   check=True)
    smi = subprocess.Popen(["nvidia-smi", "--id=0", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits",
                            "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    try:
        run = subprocess.run([exe], capture_output=True, text=True)
    finally:
        smi.terminate()
        clocks_out, _ = smi.communicate(timeout=10)
    if run.returncode != 0:
        sys.stdout.write(run.stdout + run.stderr)
        return run.returncode
    res = json.loads(run.stdout)
    mhz = [float(x) for x in clocks_out.split() if x.replace(".", "").isdigit()]
    busy = [m for m in mhz if m > 0.8 * max(mhz)] if mhz else []
    sm_mhz = statistics.median(busy) if busy else None
    res["sm_mhz_median"] = sm_mhz
    if sm_mhz:
        res["per_sm_per_clk"] = {k: round(v * 1e9 / (res["sms"] * sm_mhz * 1e6), 2)
                                 for k, v in res["total_gops"].items()}
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
