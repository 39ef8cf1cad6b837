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
   the network's prediction, FP32-storage and FP64 solvers, with the
   permeability of every converged run against the FP64 zero start.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import lbm
from . import nn


def evaluate(net, masks, tau=0.6, force=1e-6, forms=("f32s",), target=1e-6, max_steps=150000, device="cuda",
             log=None):
    """Per held-out geometry: zero and warm start for every storage form; the
    warm start's prediction error against the converged zero-start field."""
    storages = {"f64": lbm.LBM_STORE_F64, "f32s": lbm.LBM_STORE_F32S, "f32": lbm.LBM_STORE_F32,
                "f16s": lbm.LBM_STORE_F16S}
    nu = (tau - 0.5) / 3.0
    rows = []
    for k, m in enumerate(masks):
        row = {"fluid_fraction": float(m.mean())}
        fl = m.astype(bool)
        u_ref = None
        for form in forms:
            for start, model in (("zero", None), ("warm", net)):
                r = nn.solve_to_steady(m, model, tau=tau, force=force, storage=storages[form], target=target,
                                       max_steps=max_steps, device=device)
                u = r.pop("u")
                if form == forms[0] and start == "zero":
                    u_ref = u
                row[f"{form}_{start}"] = r
        _, u_pred = nn.predict_fields(net, m, force, nu)
        d = u_pred[:, fl] - u_ref
        row["prediction_u_rel_l2"] = float(np.sqrt(np.sum(d * d) / np.sum(u_ref * u_ref)))
        k_pred = nu * float(np.sum(u_pred[0][fl])) / m.size / force
        k_ref = row[f"{forms[0]}_zero"]["permeability"]
        row["prediction_permeability_rel_err"] = abs(k_pred / k_ref - 1.0)
        for form in forms:
            for start in ("zero", "warm"):
                r = row[f"{form}_{start}"]
                for base in {f"{form}_zero", f"{forms[0]}_zero"}:
                    r["permeability_rel_err_vs_" + base] = abs(r["permeability"] / row[base]["permeability"] - 1.0)
        rows.append(row)
        if log:
            s = ", ".join(f"{f}: {row[f + '_zero']['steps']} -> {row[f + '_warm']['steps']} steps" for f in forms)
            log(f"held-out {k + 1}/{len(masks)} fluid {row['fluid_fraction']:.2f}: {s}; "
                f"prediction error u {row['prediction_u_rel_l2']:.3f}")
    return rows


def summarize(rows, forms):
    out = {}
    base = "f64_zero" if "f64" in forms else f"{forms[0]}_zero"
    for form in forms:
        ok = [r for r in rows if r[f"{form}_zero"]["converged"] and r[f"{form}_warm"]["converged"]]
        if not ok:
            continue
        sr = np.array([r[f"{form}_warm"]["steps"] / r[f"{form}_zero"]["steps"] for r in ok])
        tr = np.array([r[f"{form}_warm"]["seconds"] / r[f"{form}_zero"]["seconds"] for r in ok])
        tz = sum(r[f"{form}_zero"]["seconds"] for r in ok)
        tw = sum(r[f"{form}_warm"]["seconds"] for r in ok)
        out[form] = {
            "geometries": len(ok),
            "zero_start_not_converged": sum(not r[f"{form}_zero"]["converged"] for r in rows),
            "warm_start_fallbacks": sum(bool(r[f"{form}_warm"].get("fallback")) for r in rows),
            "steps_ratio_median": float(np.median(sr)), "steps_ratio_mean": float(sr.mean()),
            "time_ratio_median": float(np.median(tr)),
            "total_seconds_zero": tz, "total_seconds_warm": tw, "speedup_total": tz / tw,
            "warm_faster_fraction": float(np.mean(tr < 1.0)),
            "max_permeability_rel_err_warm_vs_" + base: max(r[f"{form}_warm"]["permeability_rel_err_vs_" + base]
                                                            for r in ok),
        }
    if "f64" in forms:
        ok = [r for r in rows if r["f64_zero"]["converged"]]
        for form in forms:
            for start in ("zero", "warm"):
                key = f"{form}_{start}"
                t = sum(r[key]["seconds"] for r in ok)
                out.setdefault("vs_f64_zero", {})[key] = sum(r["f64_zero"]["seconds"] for r in ok) / t
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
    rows = evaluate(net, held[:n64], args.tau, args.force, forms=("f64", "f32s"), max_steps=args.max_steps,
                    device=dev, log=log)
    rows += evaluate(net, held[n64:], args.tau, args.force, forms=("f32s",), max_steps=args.max_steps, device=dev,
                     log=log)
    report["heldout_f64_and_f32s"] = summarize(rows[:n64], ("f64", "f32s"))
    report["heldout_f32s"] = summarize(rows, ("f32s",))
    report["rows"] = rows
    log(json.dumps({k: v for k, v in report.items() if k.startswith("heldout")}))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    return report


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
