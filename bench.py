#!/usr/bin/env python
"""Benchmark of the batched galaxy-model log-likelihood on GB300.

Default workload: 1024 parameter vectors against one 80x80-spaxel galaxy with 5x5
oversampling and a Gaussian PSF of FWHM 2.5" (Dehnen bulge with gamma in [0, 2], one
exponential disc, NFW halo, 64 radial quadrature nodes), float32 compute with float64
chi-square accumulation.  One step = logL of the whole batch (one persistent launch, in the
shape bang_model_tune chose for it).

Prints one JSON line: device-timed evals/s (`value`), end-to-end evals/s through the C
ABI with host buffers (`e2e`), the roofline of the dominant kernel (the SFU and FP32 work
of the step's own algorithm against the measured per-SM issue rates), the launch shape,
SM clocks sampled during the timed region, the GPU, its SM count and the host's cores
(`device`), and the FP64 CPU oracle timed on a bounded sample (`cpu_baseline`, whose
`parity` compares the oracle's chi^2 of the rows it evaluated with the timed batch's logL).
Side lines, each in one tuned launch with its own roofline and launch shape: the paper's
one-kernel-per-task form on the same batch (`plain_gpu`), logL + gradient for 256 rows
(`fwd_adjoint`), the 64-galaxy uneven batch (`uneven`, with the plain form), the 128x128
Moffat two-disc workload (`largest`, with the plain form on 32 rows; `largest_grad`, 1024
rows), the single row's latency in three forms (`single`) and the radial-table option
(`radial_table`).  ``--impl reference`` times the oracle alone in the same format.

Multi-GPU: launched by torchrun, every rank evaluates its own batch (weak scaling, no
collective on the data path); the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2205_06819_gb300 import synth  # noqa: E402

L2_FLUSH_BYTES = 256 << 20          # > 129 MB of L2
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT_NOMINAL = 152
SM_MAX_MHZ_NOMINAL = 2070.0
# Per-SM issue rates measured on GB300 (sm_103a) by a microbenchmark of independent
# chains of each PTX instruction (ex2.approx issues at twice the rate of lg2.approx).
MUFU_EX2_PER_CLK_SM = 32.0
MUFU_LG2_PER_CLK_SM = 16.0
# measured FFMA rate, lane operations per clock per SM (128 nominal); a packed two-lane
# FMA does two lane operations in two FMA-pipe cycles, so the lane rate is the same
FP32_PER_CLK_SM = 122.0
# DRAM traffic of one forward launch from an ncu capture, valid only for the kernel source
# it was taken on (sha256 prefix of bang_forward.cu + bang_device.cuh); otherwise null.
NCU_TRAFFIC = {"stamp": "a8a345c8424ec33f", "bytes_per_launch": 404480}
# Pipe activity of the forward kernel from the same kind of capture (ncu --set full on one
# timed launch of the tuned benchmark batch): SFU (xu) and FMA pipes, issue active, thread
# instructions per fine point; stamp-checked like the traffic.
NCU_PIPES = {"stamp": "a8a345c8424ec33f", "pipe_xu_pct": 35.3, "pipe_fma_pct": 32.0, "pipe_fma_cycles_pct": 45.8,
             "issue_active_pct": 66.5, "thread_instr_per_point": 436}


def kernel_stamp() -> str:
    h = hashlib.sha256()
    for f in ("bang_forward.cu", "bang_device.cuh"):
        with open(os.path.join(ROOT, "paper_2205_06819_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batched", choices=synth.WORKLOADS)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain-form and adjoint side measurements")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (bang_model_tune) before timing")
    ap.add_argument("--rows", type=int, default=0,
                    help="time only the first R rows of the workload's batch (small cases for ncu captures; "
                         "not a headline number)")
    ap.add_argument("--grad", action="store_true",
                    help="time logL + gradient (bang_loglike_grad_batch) instead of logL")
    ap.add_argument("--bulge-table", type=int, default=0,
                    help="radial-table option with T radii (0: per-point quadrature, the method as defined)")
    ap.add_argument("--bulge-kind", type=int, default=0,
                    help="1 Hernquist / 2 Jaffe closed-form bulge instead of the Dehnen quadrature")
    ap.add_argument("--psf-mode", type=int, default=0,
                    help="PSF mode bits: 1 circular window, 2 centre sampling, 4 flux-weighted moments")
    ap.add_argument("--list-workloads", action="store_true",
                    help="print the five workloads as JSON lines (no GPU) and exit")
    return ap.parse_args()


def workload_json(name: str) -> dict:
    """One workload as plain data: its galaxies (grid, oversampling, PSF), rows, model and
    the padded fine points per evaluation."""
    import dataclasses
    wl = synth.workload(name)
    gals = [dataclasses.asdict(g) for g in wl.galaxies]
    if len(gals) > 1:   # the uneven batch: distinct galaxy specs with their counts
        uniq = {}
        for g in gals:
            key = json.dumps(g, sort_keys=True)
            uniq.setdefault(key, [g, 0])[1] += 1
        gals = [dict(g, count=n) for g, n in uniq.values()]
    return {"workload": wl.name, "description": wl.description, "galaxies": gals,
            "rows_per_galaxy": wl.rows_per_galaxy, "rows": wl.batch, "n_discs": wl.n_discs, "n_quad": wl.n_quad,
            "nparams": wl.nparams, "gamma_fixed": wl.gamma_fixed, "gradient": wl.grad,
            "padded_fine_points_per_row": points_per_eval(wl.galaxies[0]) if len(wl.galaxies) == 1 else "per galaxy"}


# ----------------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def smi_device_id(cuda_ordinal: int) -> str:
    """The identifier nvidia-smi needs for CUDA device `cuda_ordinal`: its PCI address
    (nvidia-smi numbers GPUs in PCI order, which is not the CUDA ordinal once
    CUDA_VISIBLE_DEVICES remaps them), else its UUID, else the ordinal itself."""
    try:
        import torch
        p = torch.cuda.get_device_properties(cuda_ordinal)
    except Exception:   # no torch or no device: the ordinal is all there is
        return str(cuda_ordinal)
    dom, bus, dev = (getattr(p, k, None) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
    if isinstance(dom, int) and isinstance(bus, int) and isinstance(dev, int):
        return f"{dom:08X}:{bus:02X}:{dev:02X}.0"
    uuid = getattr(p, "uuid", None)
    if uuid:
        u = str(uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    return str(cuda_ordinal)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region, on the
    GPU that CUDA device `cuda_ordinal` is."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, cuda_ordinal: int):
        self.smi_id = smi_device_id(cuda_ordinal)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.smi_id}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "gpu": self.smi_id}


def measured_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f)
    except OSError:
        return {}


def points_per_eval(spec: synth.GalaxySpec) -> int:
    sig = spec.psf_fwhm_arcsec / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    h = int(math.floor(3.0 * sig / (spec.spaxel_arcsec / spec.oversample))) if spec.psf_fwhm_arcsec > 0 else 0
    return (spec.oversample * spec.nx + 2 * h) * (spec.oversample * spec.ny + 2 * h)


# SFU (MUFU) operations per padded fine point, by issue class: "half" are the functions the
# SFU issues at 16 per clock per SM (lg2, rcp, rsqrt, sqrt), "full" is ex2 (32 per clock).
#  forward (eval_point): per radial node below the far series split KF (TAIL_SPLIT) one lg2
#    and one ex2 (q^(g-4); q^(2g-7) = (q^(g-4))^2 q by multiplications); the nodes from KF on
#    as a series in 1 / w (one reciprocal and the two powers w^(g-4), w^(2g-7)); per point 13 +
#    (n_discs - 1) / 2 half-rate (the bulge's 1/(x+1) and log2 w, sqrt R, rsqrt r2, the bulge
#    velocity's 1/(x+1) and log2 u, the NFW m(x) (two reciprocals, or a log and a
#    reciprocal), a disc fit's log for y <= 1 (half the points), sqrt v, 1/B, sqrt sigma^2,
#    1/Sigma) and 3 + n_discs ex2 (the bulge's two per-point powers, the bulge velocity power,
#    each disc's exponential).  The points within ~2-3 bulge scales of the centre (a few
#    per cent of a grid), which take the mid split's nodes or every node, are counted as the
#    others: the count is a lower bound of the work;
#  adjoint (point_vjp): per radial node below the mid split K (MID_SPLIT: the adjoint uses
#    the mid level only) one lg2 and two ex2 (q^(g-4) and u/w), the upper nodes as three
#    series (one reciprocal, two ex2); per point the forward
#    recomputation's operations plus 1/(3-g), 1/R (twice), 1/(1+x) of the halo derivative,
#    the two divisions of the reverse sweep: 18 + (n_discs - 1) / 2 half-rate and 3 + n_discs
#    ex2.
TAIL_SPLIT = {64: 18, 128: 36}   # first radial node of the far-level series (TailRule::KF)
FAR_TERMS = 14                    # its terms (kFarTerms): two-lane Horner steps per point
MID_SPLIT = {64: 24, 128: 48}    # the mid level's split (TailRule::K), the adjoint's series
MID_TERMS = 8                     # its terms (kTailTerms)


def sfu_ops_per_point(n_quad: int, n_discs: int, adjoint: bool = False) -> dict:
    if adjoint:
        k = MID_SPLIT[n_quad]
        return {"half": k + 19.0 + 0.5 * (n_discs - 1), "full": 2.0 * k + 5.0 + n_discs}
    k = TAIL_SPLIT[n_quad]
    return {"half": k + 14.0 + 0.5 * (n_discs - 1), "full": k + 5.0 + n_discs}


def sfu_ops_per_point_node_by_node(n_quad: int, n_discs: int, adjoint: bool = False) -> dict:
    """The SFU operations of a pass with every radial node evaluated one by one (the plain
    form of the same sum)."""
    if adjoint:
        return {"half": n_quad + 18.0 + 0.5 * (n_discs - 1), "full": 2.0 * n_quad + 3.0 + n_discs}
    return {"half": n_quad + 13.0 + 0.5 * (n_discs - 1), "full": n_quad + 3.0 + n_discs}


def _batch_points(wl: synth.Workload, gal_idx=None, rows: int | None = None) -> float:
    if rows is None:
        return float(sum(points_per_eval(g) for g in wl.galaxies) * wl.rows_per_galaxy)
    per = [points_per_eval(g) for g in wl.galaxies]
    return float(sum(per[0 if gal_idx is None else int(gal_idx[b])] for b in range(rows)))


def sfu_work(wl: synth.Workload, gal_idx=None, rows: int | None = None, grad: bool = False):
    """Algorithmic SFU work of one batch: (operations, SM-cycles at the measured per-SM issue
    rates).  A logL step is the forward pass over every padded fine point; a logL + gradient
    step is the forward seed pass plus the adjoint pass over the same points."""
    pts = _batch_points(wl, gal_idx, rows)
    ops = cyc = 0.0
    for adj in ((False, True) if grad else (False,)):
        c = sfu_ops_per_point(wl.n_quad, wl.n_discs, adj)
        ops += pts * (c["half"] + c["full"])
        cyc += pts * (c["half"] / MUFU_LG2_PER_CLK_SM + c["full"] / MUFU_EX2_PER_CLK_SM)
    return ops, cyc


def algorithmic_sfu_ops(wl: synth.Workload, gal_idx=None, rows: int | None = None, grad: bool = False) -> float:
    """Transcendental (SFU) operations of one batch (see sfu_ops_per_point)."""
    return sfu_work(wl, gal_idx, rows, grad)[0]


def algorithmic_fp32_ops(wl: synth.Workload, gal_idx=None, rows: int | None = None, grad: bool = False) -> float:
    """FP32 instructions of one batch: per padded fine point 6 per radial node below the
    far series split (the argument of the logarithm, the exponent, and the two weighted sums
    with the (q^(g-4))^2 q product), 2 FAR_TERMS lane operations for the series (two-lane
    Horner steps) and ~200 for geometry, velocities, discs and light weighting; per galaxy
    the PSF stencil (separable: 4 channels x (fine rows x nx + nx x ny) x (os + 2h); two-
    dimensional: 4 x nx x ny x (os + 2h)^2) and ~40 per spaxel for the chi-square.  A
    gradient step adds the adjoint pass: per point 13 per radial node below the mid split (the
    six sums), 6 MID_TERMS lane operations for the three series and ~400 for the forward
    recomputation and the reverse sweep, and the transposed stencil (the forward's count).
    Forward points counted at the far level, as in sfu_ops_per_point."""
    def per_row(spec):
        sig = spec.psf_fwhm_arcsec / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        h = int(math.floor(3.0 * sig / (spec.spaxel_arcsec / spec.oversample))) if spec.psf_fwhm_arcsec > 0 else 0
        L = spec.oversample + 2 * h
        if spec.psf_kind == 1:
            psf = 4.0 * spec.nx * spec.ny * L * L
        else:
            psf = 4.0 * ((spec.oversample * spec.ny + 2 * h) * spec.nx + spec.nx * spec.ny) * L
        fwd = points_per_eval(spec) * (6.0 * TAIL_SPLIT[wl.n_quad] + 2.0 * FAR_TERMS + 200.0) + psf \
            + 40.0 * spec.nx * spec.ny
        if grad:
            fwd += points_per_eval(spec) * (13.0 * MID_SPLIT[wl.n_quad] + 6.0 * MID_TERMS + 400.0) + psf
        return fwd
    per = [per_row(g) for g in wl.galaxies]
    if rows is None:
        return float(sum(per) * wl.rows_per_galaxy)
    return float(sum(per[0 if gal_idx is None else int(gal_idx[b])] for b in range(rows)))


def combine_max(local: float, dist, device) -> float:
    """The maximum of a per-rank number over all ranks (the job takes as long as its slowest
    rank); the identity without torch.distributed."""
    if dist is None:
        return local
    import torch
    t = torch.tensor([local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_batch_seed(workload_id: int, rank: int) -> int:
    """Each rank evaluates its own batch of the same size (weak scaling)."""
    return synth.batch_seed(workload_id) + 1000 * rank


def roofline_block(wl: synth.Workload, step_s: float, gal_idx=None, rows: int | None = None, grad: bool = False,
                   mhz: float = SM_MAX_MHZ_NOMINAL, sms: int = SM_COUNT_NOMINAL) -> dict:
    """The roofline of one timed step over its two arithmetic pipes: achieved = algorithmic SFU
    operations / step time; peak = the same operations over the time the SFU needs for them
    at the measured per-SM issue rates of their classes (sms x clock); sfu_frac = that time /
    the measured time, fp32.frac the same for the FP32 count against the measured FFMA rate,
    frac = the larger of the two (the pipe that bounds the step).  node_by_node_sfu_frac is
    the SFU time the same step would need with every radial node evaluated one by one, over
    the measured time (above 1 when the series beats that SFU bound)."""
    ops, cyc = sfu_work(wl, gal_idx, rows, grad)
    t_sfu = cyc / (sms * mhz * 1e6)
    fp32 = algorithmic_fp32_ops(wl, gal_idx, rows, grad)
    fp32_peak = sms * mhz * 1e6 * FP32_PER_CLK_SM
    t_fp32 = fp32 / fp32_peak
    pts = _batch_points(wl, gal_idx, rows)
    nbn = sfu_ops_per_point_node_by_node(wl.n_quad, wl.n_discs)
    t_nbn = pts * (nbn["half"] / MUFU_LG2_PER_CLK_SM + nbn["full"] / MUFU_EX2_PER_CLK_SM) / (sms * mhz * 1e6)
    if grad:
        c = sfu_ops_per_point_node_by_node(wl.n_quad, wl.n_discs, True)
        t_nbn += pts * (c["half"] / MUFU_LG2_PER_CLK_SM + c["full"] / MUFU_EX2_PER_CLK_SM) / (sms * mhz * 1e6)
    return {"bound": "alu", "achieved": ops / step_s / 1e9, "peak": ops / t_sfu / 1e9, "unit": "G SFU op/s",
            "frac": max(t_sfu, t_fp32) / step_s,
            "sfu_frac": t_sfu / step_s,
            "node_by_node_sfu_frac": t_nbn / step_s,
            "fp32": {"achieved": fp32 / step_s / 1e9, "peak": fp32_peak / 1e9, "unit": "G FP32 lane-op/s",
                     "frac": t_fp32 / step_s},
            "t_roof_over_t_meas": max(t_sfu, t_fp32) / step_s,
            "sfu_sm_cycles_per_point": cyc / _batch_points(wl, gal_idx, rows),
            "peak_basis": f"{sms} SMs x {mhz:.0f} MHz (MEASURED_PEAKS sm_max_mhz) x measured per-SM issue rates: "
                          f"lg2/rcp/rsqrt/sqrt {MUFU_LG2_PER_CLK_SM:.0f}/clk, ex2 {MUFU_EX2_PER_CLK_SM:.0f}/clk, "
                          f"FFMA {FP32_PER_CLK_SM:.0f} lanes/clk, for the step's own operation mix"}


# ----------------------------------------------------------------------------- data
def make_model(wl: synth.Workload, rank: int, torch, bulge_table: int = 0, bulge_kind: int = 0, psf_mode: int = 0):
    """Seeded synthetic galaxies: noise-free maps from the library at each galaxy's
    theta_true plus noise; the batch is rows_per_galaxy rows per galaxy."""
    from paper_2205_06819_gb300.model import Galaxy, Model
    wid = synth.workload_id(wl.name)
    box = synth.prior_box(wl.n_discs, wl.gamma_fixed)
    tts = [synth.draw_theta_true(box, synth.dataset_seed(wid, g)) for g in range(len(wl.galaxies))]
    probes = [Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec,
                     np.ones((4, s.ny, s.nx), np.float32), np.ones((4, s.ny, s.nx), np.float32),
                     psf_kind=s.psf_kind, moffat_beta=s.moffat_beta) for s in wl.galaxies]
    probe = Model(probes, n_discs=wl.n_discs, n_quad=wl.n_quad, bulge_kind=bulge_kind, psf_mode=psf_mode)
    gi = np.arange(len(wl.galaxies), dtype=np.int32)
    true = probe.maps(torch.from_numpy(np.stack(tts).astype(np.float32)).cuda(), gi if len(gi) > 1 else None)
    probe.close()
    gals = []
    for g, s in enumerate(wl.galaxies):
        data, err, mask = synth.noisy_data(true[g].cpu().numpy().astype(np.float64), seed=synth.dataset_seed(wid, g))
        gals.append(Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec, data, err, mask,
                           psf_kind=s.psf_kind, moffat_beta=s.moffat_beta))
    model = Model(gals, n_discs=wl.n_discs, n_quad=wl.n_quad, bulge_table=bulge_table, bulge_kind=bulge_kind,
                  psf_mode=psf_mode)
    seed = rank_batch_seed(wid, rank)
    theta = np.concatenate([synth.draw_theta_batch(box, tts[g], wl.rows_per_galaxy, seed + 7 * g)
                            for g in range(len(gals))]).astype(np.float32)
    gal_idx = np.repeat(gi, wl.rows_per_galaxy) if len(gals) > 1 else None
    return model, gals, theta, gal_idx


def cpu_oracle_sample(wl, gal, theta, seconds: float, gpu_logL=None):
    """The FP64 oracle, as it stands, on consecutive rows until the time budget is spent.
    With ``gpu_logL`` (the timed batch's logL from the CUDA path) the oracle's chi^2 of the
    rows it evaluated is also compared with the GPU's, as a parity sample of the bench run."""
    import oracle
    oracle.build()
    og = oracle.Galaxy(gal.nx, gal.ny, gal.oversample, gal.psf_fwhm_arcsec, gal.kpc_per_arcsec,
                       psf_kind=gal.psf_kind, moffat_beta=gal.moffat_beta,
                       data=np.asarray(gal.data, np.float64), err=np.asarray(gal.err, np.float64), mask=gal.mask)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    n = 0
    B = theta.shape[0]
    ref_chi2 = []
    while n < max(B, 1 << 30):
        _, c2 = oracle.loglike(og, theta[n % B:n % B + 1].astype(np.float64), n_discs=wl.n_discs, n_quad=wl.n_quad)
        if n < B:
            ref_chi2.append(float(c2[0]))
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    # the same oracle on one thread, a few rows (about a third of the budget)
    t1 = time.perf_counter()
    n1 = 0
    while True:
        oracle.loglike(og, theta[n1 % B:n1 % B + 1].astype(np.float64), n_discs=wl.n_discs, n_quad=wl.n_quad,
                       nthreads=1)
        n1 += 1
        if time.perf_counter() - t1 > seconds / 3:
            break
    dt1 = time.perf_counter() - t1
    oracle.loglike(og, theta[:1].astype(np.float64), n_discs=wl.n_discs, n_quad=wl.n_quad,
                   nthreads=cores)   # restore the thread count
    out = {"value": n / dt, "unit": "logL evals/s", "cores": cores, "kind": "oracle",
           "single_thread_value": n1 / dt1, "single_thread_sample": f"{n1} rows, {dt1:.1f} s",
           "sample": f"{n} oracle calls on consecutive rows of the {B}-row batch (OpenMP over fine-grid rows), "
                     f"{dt:.1f} s"}
    if gpu_logL is not None and ref_chi2:
        k = len(ref_chi2)
        ref = np.asarray(ref_chi2)
        gpu_chi2 = -2.0 * (np.asarray(gpu_logL[:k], np.float64) + oracle.norm_const(og))
        rel = np.abs(gpu_chi2 - ref) / ref
        out["parity"] = {"rows": k, "max_rel_chi2_err": float(rel.max()), "median_rel_chi2_err": float(np.median(rel)),
                         "tolerance": 1e-5, "pass": bool(rel.max() < 1e-5)}
    return out


def time_plain(model, theta, logL, B):
    """The same batch through the paper's one-kernel-per-task form (bang_loglike_plain)."""
    import torch
    from paper_2205_06819_gb300 import _lib
    per_row = 9
    model.loglike_plain(theta[:8])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = model.loglike_plain(theta)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ref = model.loglike(theta)
    fin = torch.isfinite(ref)
    rel = ((out[fin] - ref[fin]).abs() / ref[fin].abs()).max().item()
    return {"value": B / ms * 1e3, "unit": "logL evals/s", "ms_per_batch": ms, "launches": per_row * B,
            "max_rel_logL_vs_fused": rel,
            "form": "one kernel per task per parameter vector, 64 threads/block, intermediates in HBM"}


def time_table(wl, torch, T=1024, steps=20):
    """The same workload with the radial-table option (bulge_table = T): logL and
    logL + gradient, device-timed, with the largest chi^2 difference to the default mode."""
    model, _, theta_np, gal_idx = make_model(wl, 0, torch, bulge_table=T)
    exact, _, _, _ = make_model(wl, 0, torch)
    theta = torch.from_numpy(theta_np).cuda()
    B = theta.shape[0]
    model.tune(B, gal_idx)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    for _ in range(3):
        model.loglike(theta, gal_idx, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        model.loglike(theta, gal_idx, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    model.loglike_grad(theta, gal_idx)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(3):
        model.loglike_grad(theta, gal_idx)
    e1.record()
    torch.cuda.synchronize()
    gms = e0.elapsed_time(e1) / 3
    ref = exact.loglike(theta, gal_idx)
    fin = torch.isfinite(ref)
    rel = ((out[fin] - ref[fin]).abs() / ref[fin].abs()).max().item()
    model.close()
    exact.close()
    return {"value": B / ms * 1e3, "unit": "logL evals/s", "ms_per_batch": ms, "table_radii": T,
            "fwd_adjoint_evals_s": B / gms * 1e3, "max_rel_logL_vs_per_point_quadrature": rel,
            "form": "bulge Sigma and sigma^2 from a per-row table of the same radial quadrature, "
                    "4-point Lagrange interpolation in log R"}


def _event_time(torch, fn, steps, flush=None):
    """Mean device time (ms) of fn() over `steps` calls, each bracketed by CUDA events on the
    current stream, the L2 flushed between calls outside the events."""
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xff)
        starts[k].record(stream)
        fn()
        ends[k].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps


def time_workload(name, torch, grad=False, rows=None, steps=5, warmup=2, mhz=SM_MAX_MHZ_NOMINAL,
                  sms=SM_COUNT_NOMINAL, flush=None, forward_too=False, plain_rows=0):
    """One workload (or its first `rows` rows) in one launch after the autotuner has chosen
    its shape: device-timed logL (or logL + gradient) evaluations per second and the SFU
    roofline of the timed step.  With plain_rows, also the paper's one-kernel-per-task form
    (bang_loglike_plain) on the first plain_rows rows, and its largest relative logL
    difference from the fused launch."""
    wl = synth.workload(name)
    model, _, theta_np, gal_idx = make_model(wl, 0, torch)
    if rows:
        theta_np = np.ascontiguousarray(theta_np[:rows])
        gal_idx = None if gal_idx is None else np.ascontiguousarray(gal_idx[:rows])
    B = theta_np.shape[0]
    model.tune(B, gal_idx, grad=grad)
    theta = torch.from_numpy(theta_np).cuda()
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    if grad:
        def call():
            model.loglike_grad(theta, gal_idx)
    else:
        def call():
            model.loglike(theta, gal_idx, out=out)
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ms = _event_time(torch, call, steps, flush)
    metric = "logL+gradient evals/s" if grad else "logL evals/s"
    res = {"value": B / ms * 1e3, "unit": metric, "ms_per_step": ms, "rows": B, "steps": steps,
           "workload": f"{wl.name}: {wl.description}", "launch": model.launch_info(B, gal_idx, grad),
           "roofline": roofline_block(wl, ms / 1e3, gal_idx, B, grad, mhz, sms)}
    if forward_too:
        fms = _event_time(torch, lambda: model.loglike(theta, gal_idx, out=out), steps, flush)
        res["forward_only_ms"] = fms
        res["grad_over_forward"] = ms / fms
    if plain_rows:
        n = min(plain_rows, B)
        tp = theta[:n]
        gp = None if gal_idx is None else np.ascontiguousarray(gal_idx[:n])
        model.loglike_plain(tp[:1], None if gp is None else gp[:1])
        torch.cuda.synchronize()
        pms = _event_time(torch, lambda: model.loglike_plain(tp, gp), 1)
        ref = model.loglike(tp, gp)
        got = model.loglike_plain(tp, gp)
        fin = torch.isfinite(ref)
        res["plain_gpu"] = {"value": n / pms * 1e3, "unit": "logL evals/s", "rows": n, "ms": pms,
                            "max_rel_logL_vs_fused": ((got[fin] - ref[fin]).abs() / ref[fin].abs()).max().item(),
                            "form": "one kernel per task per parameter vector (bang_loglike_plain)"}
    model.close()
    return res


def time_single(torch, steps=50):
    """The single-row workload (30x30, os 3, gamma = 1, one row): latency of one evaluation
    by the fused launch, by the paper's one-kernel-per-task chain (float32), and by the
    float64 check path (every step in float64), with the relative logL differences."""
    import time as _t
    wl = synth.workload("single")
    model, _, theta_np, _ = make_model(wl, 0, torch)
    theta = torch.from_numpy(theta_np).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        model.loglike(theta, out=out)
        model.loglike_plain(theta)
    torch.cuda.synchronize()
    fused = _event_time(torch, lambda: model.loglike(theta, out=out), steps)
    plain = _event_time(torch, lambda: model.loglike_plain(theta), steps)
    th64 = torch.from_numpy(theta_np.astype(np.float64))
    l64 = model.loglike_fp64(th64)          # synchronous: timed by the host clock
    t0 = _t.perf_counter()
    n = 5
    for _ in range(n):
        l64 = model.loglike_fp64(th64)
    fp64_ms = (_t.perf_counter() - t0) / n * 1e3
    l32 = float(model.loglike(theta).cpu()[0])
    lp = float(model.loglike_plain(theta).cpu()[0])
    model.close()
    return {"workload": f"single: {wl.description}", "unit": "ms per evaluation",
            "fused_f32_ms": fused, "plain_f32_ms": plain, "fp64_check_path_ms": fp64_ms,
            "fused_evals_s": 1e3 / fused, "plain_evals_s": 1e3 / plain, "fp64_evals_s": 1e3 / fp64_ms,
            "rel_logL_fused_vs_fp64": abs(l32 - float(l64[0])) / abs(float(l64[0])),
            "rel_logL_plain_vs_fused": abs(lp - l32) / abs(l32),
            "note": "one row cannot fill the GPU: latency, not throughput; the float64 path is "
                    "synchronous and timed by the host clock"}


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = synth.workload(args.workload)
    wid = synth.workload_id(wl.name)
    box = synth.prior_box(wl.n_discs, wl.gamma_fixed)
    s = wl.galaxies[0]
    tt = synth.draw_theta_true(box, synth.dataset_seed(wid))
    g0 = oracle.Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec, psf_kind=s.psf_kind,
                       moffat_beta=s.moffat_beta)
    data, err, mask = synth.noisy_data(oracle.maps(g0, tt, n_discs=wl.n_discs, n_quad=wl.n_quad),
                                       seed=synth.dataset_seed(wid))
    og = oracle.Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec, psf_kind=s.psf_kind,
                       moffat_beta=s.moffat_beta, data=data.astype(np.float64), err=err.astype(np.float64), mask=mask)
    theta = synth.draw_theta_batch(box, tt, wl.batch, synth.batch_seed(wid)).astype(np.float32).astype(np.float64)
    rows_per_step = 1
    k = 0
    for _ in range(args.warmup):
        oracle.loglike(og, theta[k % wl.batch:k % wl.batch + rows_per_step], n_discs=wl.n_discs, n_quad=wl.n_quad)
        k += rows_per_step
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.loglike(og, theta[k % wl.batch:k % wl.batch + rows_per_step], n_discs=wl.n_discs, n_quad=wl.n_quad)
        k += rows_per_step
    dt = time.perf_counter() - t0
    value = args.steps * rows_per_step / dt
    line = {
        "impl": "reference", "metric": "logL evals/s", "value": value, "unit": "logL evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.description}", "rows_per_step": rows_per_step},
        "cpu_baseline": {"value": value, "unit": "logL evals/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{rows_per_step} row per step of the {wl.batch}-row batch"},
        "e2e": {"value": value, "unit": "logL evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_2205_06819_gb300 import build as bmod
    bmod.build()
    wl = synth.workload(args.workload)
    model, gals, theta_np, gal_idx = make_model(wl, rank, torch, bulge_table=args.bulge_table,
                                                bulge_kind=args.bulge_kind, psf_mode=args.psf_mode)
    gal = gals[0]
    B_full = theta_np.shape[0]
    if args.rows:
        theta_np = np.ascontiguousarray(theta_np[:args.rows])
        gal_idx = None if gal_idx is None else np.ascontiguousarray(gal_idx[:args.rows])
    if not args.no_tune:
        model.tune(theta_np.shape[0], gal_idx, grad=args.grad)
    B, P = theta_np.shape
    if args.grad:
        def call(th, out):
            return model.loglike_grad(th, gal_idx)
    else:
        def call(th, out):
            return model.loglike(th, gal_idx, out=out)
    # kernels per step: decode, forward, finalize (+ the table kernel; + adjoint and gradient map)
    launches_per_step = 3 + (1 if args.bulge_table else 0) + (2 if args.grad else 0)
    headline = not (args.rows or args.grad or args.bulge_table or args.bulge_kind or args.psf_mode)
    theta = torch.from_numpy(theta_np).cuda()
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        call(theta, logL)
    torch.cuda.synchronize()

    # device-timed steps (L2 flushed between steps, outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        res = call(theta, logL)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = combine_max(sum(step_ms) / 1e3, dist, "cuda")
    value = ws * B * args.steps / dev_s
    assert np.isfinite((res[0] if args.grad else logL).cpu().numpy()).any()

    # end to end through the C ABI with pinned host buffers
    th_host = torch.from_numpy(theta_np).pin_memory()
    out_host = torch.empty(B, dtype=torch.float64).pin_memory()
    for _ in range(2):
        call(th_host, out_host)
    e2e_t = []
    barrier()
    for k in range(max(3, args.steps // 4)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call(th_host, out_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = combine_max(sum(e2e_t), dist, "cuda")
    e2e_value = ws * B * len(e2e_t) / e2e_s

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL))
    step_s = dev_s / args.steps
    pipes = NCU_PIPES if NCU_PIPES["stamp"] == kernel_stamp() else None
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["stamp"] == kernel_stamp() else None
    roof = roofline_block(wl, step_s, gal_idx, B, args.grad, mhz, sms)
    roof["traffic"] = None if args.grad else traffic
    roof["ncu_pipes"] = None if args.grad else pipes

    metric = "logL+gradient evals/s" if args.grad else "logL evals/s"
    line = {
        "metric": metric, "value": value, "unit": metric, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.description}", "rows": B, "rows_of_workload": B_full,
                   "path": ("logL + gradient" if args.grad else "logL")
                   + (f", radial table T={args.bulge_table}" if args.bulge_table else "")
                   + (f", closed-form bulge kind {args.bulge_kind}" if args.bulge_kind else "")
                   + (f", psf_mode {args.psf_mode}" if args.psf_mode else ""),
                   "padded_fine_points_per_row": points_per_eval(wl.galaxies[0]) if len(wl.galaxies) == 1 else
                   "per galaxy", "n_quad": wl.n_quad, "galaxies": len(wl.galaxies),
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "launch": model.launch_info(B, gal_idx, args.grad)},
        "e2e": {"value": e2e_value, "unit": metric, "h2d_bytes_per_step": int(B * P * 4),
                "d2h_bytes_per_step": int(B * 8 + (B * P * 4 if args.grad else 0))},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "clocks": clk,
        "wall_s_timed": wall,
        "device": {"name": props.name, "sms": sms, "host_cores": os.cpu_count(), "torch": torch.__version__,
                   "cuda": torch.version.cuda},
    }
    if not headline:
        line["note"] = ("profiling or variant case (--rows / --grad / --bulge-table / --bulge-kind / --psf-mode), "
                        "not the headline configuration")
        if args.bulge_table or args.bulge_kind or args.psf_mode:
            line["roofline"] = None        # the SFU counts are the per-point quadrature's
    if ws == 1 and headline and not args.no_extras and len(wl.galaxies) == 1:
        line["plain_gpu"] = time_plain(model, theta, logL, B)
        model.close()
        side = dict(torch=torch, mhz=mhz, sms=sms, flush=flush)
        # the other workloads, each in one tuned launch: logL + gradient (256 rows), the
        # uneven batch (64 galaxies x 64 rows), the largest (4096 rows; its gradient on the
        # first 1024), and the single row's latency in three forms
        line["fwd_adjoint"] = time_workload("adjoint", grad=True, steps=10, forward_too=True, **side)
        line["uneven"] = time_workload("uneven", steps=5, plain_rows=4096, **side)
        line["largest"] = time_workload("largest", steps=3, plain_rows=32, **side)
        line["largest_grad"] = time_workload("largest", grad=True, rows=1024, steps=3, **side)
        line["single"] = time_single(torch)
        line["radial_table"] = time_table(wl, torch)
        line["cpu_baseline"] = cpu_oracle_sample(wl, gal, theta_np, args.cpu_seconds, logL.cpu().numpy())
    elif ws == 1:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.list_workloads:
        for name in synth.WORKLOADS:
            print(json.dumps(workload_json(name)))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
