"""Parity report: the CUDA library against the FP64 oracle on every workload at full size.

For each of the five workloads (single, batched, adjoint, uneven, largest) this builds the
seeded synthetic galaxy(ies) from the oracle's noise-free maps, runs the whole batch on the
GPU in the launch shape the benchmark uses, and compares a sample of rows with the oracle:
relative error of chi^2 (the theta-dependent part of logL) and of logL, per-map element
errors (B, sigma, M/L relative; v relative to the map's largest |v|), and for the
gradient workloads the gradient error relative to the oracle gradient's norm.

    python tests/parity_report.py [--rows N] [--grad-rows N] [--bulge-table T] [--out file.json]

Prints one JSON object per workload.  Needs a GPU; the oracle uses all host cores.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset  # noqa: E402


def map_errors(got, ref):
    out = {}
    for c, name in enumerate(["B", "v", "sigma", "ML"]):
        if name == "v":
            out[name] = float(np.abs(got[c] - ref[c]).max() / max(np.abs(ref[c]).max(), 1e-30))
        else:
            out[name] = float((np.abs(got[c] - ref[c]) / np.abs(ref[c])).max())
    return out


def report(name, rows, grad_rows, torch, Model, bulge_table=0):
    wl = synth.workload(name)
    wid = synth.workload_id(name)
    box = synth.prior_box(wl.n_discs, wl.gamma_fixed)
    t0 = time.time()
    dss = []
    for g, spec in enumerate(wl.galaxies):
        tt = synth.draw_theta_true(box, synth.dataset_seed(wid, g))
        dss.append(Dataset(spec, tt, n_discs=wl.n_discs, n_quad=wl.n_quad, seed=synth.dataset_seed(wid, g)))
    gal_idx = np.repeat(np.arange(len(dss), dtype=np.int32), wl.rows_per_galaxy)
    theta = np.concatenate([synth.draw_theta_batch(box, d.theta_true, wl.rows_per_galaxy, synth.batch_seed(wid) + 7 * g)
                            for g, d in enumerate(dss)]).astype(np.float32)
    m = Model([d.model_galaxy() for d in dss], n_discs=wl.n_discs, n_quad=wl.n_quad, bulge_table=bulge_table)
    tt_ = torch.from_numpy(theta).cuda()
    gi = gal_idx if len(dss) > 1 else None
    logL = m.loglike(tt_, gi).cpu().numpy()
    rng = np.random.default_rng(wid)
    nb = theta.shape[0]
    pick = np.unique(np.concatenate([[0, nb - 1], rng.choice(nb, min(rows, nb), replace=False)]))[:max(1, min(rows, nb))]
    res = {"workload": name, "bulge_table": bulge_table, "rows_total": int(theta.shape[0]),
           "rows_checked": [int(b) for b in pick]}
    chi_rel, logl_rel, maps_err = [], [], {"B": 0.0, "v": 0.0, "sigma": 0.0, "ML": 0.0}
    maps = m.maps(torch.from_numpy(theta[pick]).cuda(), gal_idx[pick] if gi is not None else None)
    for k, b in enumerate(pick):
        d = dss[gal_idx[b]]
        ref_l, ref_c = d.oracle_loglike(theta[b:b + 1])
        c = -2 * (logL[b] + oracle.norm_const(d.og))
        chi_rel.append(abs(c - ref_c[0]) / ref_c[0])
        logl_rel.append(abs(logL[b] - ref_l[0]) / abs(ref_l[0]))
        me = map_errors(maps[k].cpu().numpy(), d.oracle_maps(theta[b]))
        for key in maps_err:
            maps_err[key] = max(maps_err[key], me[key])
    res["max_rel_chi2"] = float(max(chi_rel))
    res["max_rel_logL"] = float(max(logl_rel))
    res["max_map_err"] = maps_err
    if wl.grad and grad_rows > 0:
        gpick = pick[:grad_rows]
        _, grad = m.loglike_grad(tt_, gi)
        grad = grad.cpu().numpy()
        gerr, gcomp = [], []
        for b in gpick:
            d = dss[gal_idx[b]]
            _, ref = oracle.loglike_grad(d.og, theta[b:b + 1].astype(np.float64), n_discs=wl.n_discs,
                                         n_quad=wl.n_quad)
            nrm = np.linalg.norm(ref[0])
            gerr.append(float(np.linalg.norm(grad[b] - ref[0]) / nrm))
            gcomp.append(float(np.abs(grad[b] - ref[0]).max() / nrm))
        res["grad_rows_checked"] = [int(b) for b in gpick]
        res["max_rel_grad_norm"] = max(gerr)
        res["max_grad_component_over_norm"] = max(gcomp)
    res["seconds"] = time.time() - t0
    m.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=6)
    ap.add_argument("--grad-rows", type=int, default=2)
    ap.add_argument("--workloads", default=",".join(synth.WORKLOADS))
    ap.add_argument("--out", default=None)
    ap.add_argument("--bulge-table", type=int, default=0, help="radial-table option of the library (0: off)")
    args = ap.parse_args()
    import torch
    oracle.build()
    from paper_2205_06819_gb300 import build as b
    b.build()
    from paper_2205_06819_gb300.model import Model
    out = []
    for name in args.workloads.split(","):
        r = report(name, args.rows, args.grad_rows, torch, Model, args.bulge_table)
        print(json.dumps(r), flush=True)
        out.append(r)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
