"""Training and evaluation of the learned warm start (not in the paper).

    python -m paper_1703_08015_gb300.warmstart --n-train 2000 --n-heldout 200 \\
        --out paper_1703_08015_gb300/weights/unet_spheres64.npz --report report.json

1. Seeded sphere packs of side 64 (radius 4-12, fluid fraction uniform in
   0.1-0.6, only geometries whose pore space winds around the periodic x
   axis); the training and held-out sets come from different seeds.
2. Steady states of the training set from the solver itself (FP32 storage of
   the shifted PDFs, batched, run to residual < 1e-6).
3. Adam training of the U-Net in ``nn.py`` with the library's own forward and
   backward kernels.
4. On the held-out set: time and steps to residual < 1e-6 from rest and from
   the network's prediction, FP32-storage and FP64 solvers, with and without
   the period-2 filter (lbm_filter_period2), with the velocity and
   permeability of every converged run against the filtered FP64 zero start.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import lbm
from . import nn


STORAGES = {"f64": lbm.LBM_STORE_F64, "f32s": lbm.LBM_STORE_F32S, "f32": lbm.LBM_STORE_F32,
            "f16s": lbm.LBM_STORE_F16S}
# (label, storage, start, period-2 filter); the first is the baseline
CASES_FULL = [("f64_zero_plain", "f64", "zero", False), ("f64_zero", "f64", "zero", True),
              ("f64_warm", "f64", "warm", True), ("f32s_zero", "f32s", "zero", True),
              ("f32s_warm", "f32s", "warm", True), ("f32s_warm_plain", "f32s", "warm", False)]
CASES_F32S = [("f32s_zero", "f32s", "zero", True), ("f32s_warm", "f32s", "warm", True)]


def evaluate(net, masks, cases, tau=0.6, force=1e-6, target=1e-6, max_steps=150000, device="cuda", log=None):
    """Per held-out geometry and case: steps and wall time to residual < target
    (tiling, initialisation and network inference included), permeability,
    and the velocity error of the converged field and of the prediction
    against the first filtered zero start (the most accurate field)."""
    nu = (tau - 0.5) / 3.0
    rows = []
    for k, m in enumerate(masks):
        row = {"fluid_fraction": float(m.mean())}
        fl = m.astype(bool)
        fields = {}
        for label, form, start, filt, *fin in cases:
            r = nn.solve_to_steady(m, net if start == "warm" else None, tau=tau, force=force,
                                   storage=STORAGES[form], target=target, max_steps=max_steps,
                                   filter_period2=filt, finish=STORAGES[fin[0]] if fin else None,
                                   device=device)
            fields[label] = r.pop("u")
            row[label] = r
        ref_label = next(c[0] for c in cases if c[2] == "zero" and c[3])
        u_ref, k_ref = fields[ref_label], row[ref_label]["permeability"]
        nrm = float(np.sqrt(np.sum(u_ref * u_ref)))
        for label in fields:
            d = fields[label] - u_ref
            row[label]["u_rel_err"] = float(np.sqrt(np.sum(d * d))) / nrm
            row[label]["permeability_rel_err"] = abs(row[label]["permeability"] / k_ref - 1.0)
        _, u_pred = nn.predict_fields(net, m, force, nu)
        d = u_pred[:, fl] - u_ref
        row["prediction_u_rel_l2"] = float(np.sqrt(np.sum(d * d))) / nrm
        k_pred = nu * float(np.sum(u_pred[0][fl])) / m.size / force
        row["prediction_permeability_rel_err"] = abs(k_pred / k_ref - 1.0)
        rows.append(row)
        if log:
            s = ", ".join(f"{c[0]} {row[c[0]]['steps']}" for c in cases)
            log(f"held-out {k + 1}/{len(masks)} fluid {row['fluid_fraction']:.2f}: {s}; "
                f"prediction error u {row['prediction_u_rel_l2']:.3f}")
    return rows


def summarize(rows, cases):
    """Per case: geometries converged, median steps, total time over the
    geometries where every case converged, speedups against the first case
    and against the filtered zero start of the same storage."""
    labels = [lb for lb, *_ in cases]
    ok = [r for r in rows if all(r[lb]["converged"] for lb in labels)]
    out = {"geometries": len(rows), "all_converged": len(ok)}
    if not ok:
        return out
    tot = {lb: sum(r[lb]["seconds"] for r in ok) for lb in labels}
    for lb, form, start, filt, *_ in cases:
        steps = np.array([r[lb]["steps"] for r in ok])
        e = {"converged": sum(r[lb]["converged"] for r in rows), "steps_median": float(np.median(steps)),
             "steps_mean": float(steps.mean()), "seconds_total": tot[lb],
             "speedup_vs_" + labels[0]: tot[labels[0]] / tot[lb],
             "u_rel_err_median": float(np.median([r[lb]["u_rel_err"] for r in ok])),
             "permeability_rel_err_max": max(r[lb]["permeability_rel_err"] for r in ok),
             "fallbacks": sum(bool(r[lb].get("fallback")) for r in rows),
             "switched": sum(r[lb].get("switched_at") is not None for r in rows)}
        zero = f"{form}_zero"
        if start == "warm" and zero in labels:
            ratio = np.array([r[lb]["steps"] / r[zero]["steps"] for r in ok])
            e["steps_ratio_vs_" + zero + "_median"] = float(np.median(ratio))
            e["speedup_vs_" + zero] = tot[zero] / tot[lb]
            e["faster_than_" + zero + "_fraction"] = float(np.mean([r[lb]["seconds"] < r[zero]["seconds"]
                                                                     for r in ok]))
        out[lb] = e
    out["prediction_u_rel_l2_median"] = float(np.median([r["prediction_u_rel_l2"] for r in rows]))
    out["prediction_permeability_rel_err_median"] = float(np.median([r["prediction_permeability_rel_err"]
                                                                     for r in rows]))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-heldout", type=int, default=200)
    ap.add_argument("--n-heldout-f64", type=int, default=50, help="held-out geometries also solved in FP64")
    ap.add_argument("--side", type=int, default=64)
    ap.add_argument("--seed-train", type=int, default=1)
    ap.add_argument("--seed-heldout", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tau", type=float, default=0.6)
    ap.add_argument("--force", type=float, default=1e-6)
    ap.add_argument("--max-steps", type=int, default=150000)
    ap.add_argument("--out", default=nn.WEIGHTS)
    ap.add_argument("--report", default=None)
    ap.add_argument("--eval-only", action="store_true", help="load --out instead of training")
    args = ap.parse_args(argv)

    import torch

    dev = torch.device("cuda")
    t_start = time.perf_counter()

    def log(msg):
        print(f"[{time.perf_counter() - t_start:7.1f} s] {msg}", flush=True)

    nu = (args.tau - 0.5) / 3.0
    report = {"args": vars(args)}
    if args.eval_only:
        net = nn.UNet.load(args.out, device=dev)
    else:
        masks, infos = nn.sample_geometries(args.n_train, args.seed_train, args.side)
        log(f"{len(masks)} training geometries")
        fields, steps = nn.steady_states(masks, args.tau, args.force, max_steps=args.max_steps, device=dev, log=log)
        keep = [i for i, s in enumerate(steps) if s is not None]
        log(f"{len(keep)} converged; steps median {np.median([steps[i] for i in keep]):.0f}")
        idx = torch.as_tensor(keep, device=dev)
        fields = fields.index_select(0, idx)
        masks_dev = torch.from_numpy(np.stack([masks[i] for i in keep])).to(dev)
        net = nn.UNet(seed=0, device=dev)
        log(f"U-Net: {net.n_params} parameters")
        hist = nn.train(net, masks_dev, fields, args.force, nu, epochs=args.epochs, batch=args.batch, lr=args.lr,
                        log=log)
        del fields
        torch.cuda.empty_cache()
        net.save(args.out, n_train=len(keep), epochs=args.epochs, batch=args.batch, lr=args.lr, tau=args.tau,
                 side=args.side, seed_train=args.seed_train, loss_final=hist[-1][1])
        report["train"] = {"geometries": len(keep), "not_converged": len(steps) - len(keep),
                           "steps_median": float(np.median([steps[i] for i in keep])),
                           "steps_max": int(max(steps[i] for i in keep)), "loss": hist}
        log(f"saved {args.out}")
    held, _ = nn.sample_geometries(args.n_heldout, args.seed_heldout, args.side)
    n64 = min(args.n_heldout_f64, len(held))
    rows = evaluate(net, held[:n64], CASES_FULL, args.tau, args.force, max_steps=args.max_steps, device=dev, log=log)
    rows += evaluate(net, held[n64:], CASES_F32S, args.tau, args.force, max_steps=args.max_steps, device=dev,
                     log=log)
    report["heldout_all_cases"] = summarize(rows[:n64], CASES_FULL)
    report["heldout_f32s"] = summarize(rows, CASES_F32S)
    report["rows"] = rows
    log(json.dumps({k: v for k, v in report.items() if k.startswith("heldout")}))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    return report


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
