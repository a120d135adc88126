"""Train the learned closure on cells labelled by the exact GPU closure.

    python -m paper_2606_15622_gb300.train_surrogate --cells 2000000 \
        --epochs 20 --out paper_2606_15622_gb300/weights/surrogate_full.fpw

Training cells are drawn half from the Couette-like and half from the
cavity-like distributions (populations.training_cells), in chunks, labelled
with fp_closure_exact in FP64; cells the exact closure flags or whose
dimensionless coefficients exceed 1e6 are dropped.  Every training step runs
in libfpclosure's kernels (forward, loss + gradient, backward, Adam).  A
held-out set (fresh seeds) measures the error of the network alone and of
the surrogate closure with its exact fallback; the report is written beside
the weights as JSON.

    python -m paper_2606_15622_gb300.train_surrogate --features lite \
        --out paper_2606_15622_gb300/weights/surrogate_lite.fpw

trains the network on the 16 LITE inputs instead (same cells, same targets,
same loss); its held-out report measures what the low-order inputs lose
against the exact closure, beside the full-input network's.
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import api
from . import populations as P
from . import surrogate as S


def build_training_set(n_cells, seed, eps2_hat, chunk=250_000, log=print, features="full", cylinder_fraction=0.0):
    parts = []
    done = 0
    k = 0
    while done < n_cells:
        n = min(chunk, n_cells - done)
        t0 = time.time()
        pop = P.training_cells(n, seed=seed * 1000 + k, cylinder_fraction=cylinder_fraction)
        ts = S.TrainingSet(pop, eps2_hat=eps2_hat, features=features)
        parts.append(ts)
        done += n
        k += 1
        log(f"  labelled {done}/{n_cells} cells ({len(ts)} kept) in {time.time() - t0:.1f} s")
    out = parts[0]
    out.f = torch.cat([p.f for p in parts])
    out.t = torch.cat([p.t for p in parts])
    out.aux = torch.cat([p.aux for p in parts])
    out.src = torch.cat([p.src for p in parts])
    out.tau = torch.cat([p.tau for p in parts])
    return out


def evaluate(s: S.Surrogate, n_cells, seed, eps2_hat):
    """Error of the network and of the surrogate closure against the exact
    FP64 closure on fresh cells; fallback rate."""
    pop = P.training_cells(n_cells, seed=seed)
    dev = torch.device("cuda")
    v = torch.from_numpy(pop.v64).to(dev)
    off = torch.from_numpy(pop.offsets).to(dev)
    tau = torch.from_numpy(pop.tau).to(dev)
    prm = api.default_params(eps2_hat=eps2_hat)
    mom, y_ex, fl_ex = api.fp_closure_exact(v, off, tau, params=prm, prec="fp64")
    if s.features_set == "lite":
        y_s, fl_s = s.closure_lite(api.fp_moments_lite(v, off), tau, params=prm)
        fb = (fl_s & api.FALLBACK_FLAGS) != 0     # cells given the linear drift
    else:
        y_s, fl_s = s.closure(mom, tau, params=prm)
        fb = (fl_s & api.FLAG_FALLBACK) != 0
    torch.cuda.synchronize()
    t_ex = S.dimensionless(y_ex, mom, tau)
    t_s = S.dimensionless(y_s, mom, tau)
    ok = fl_ex == 0
    rel = ((t_s - t_ex).norm(dim=1) / t_ex.norm(dim=1))[ok]
    net = ~fb & ok
    rel_net = ((t_s - t_ex).norm(dim=1) / t_ex.norm(dim=1))[net]
    sd = s.y_sigma[:9].double()
    std_err = (((t_s - t_ex) / sd) ** 2).sum(1).sqrt()[ok]
    lin = torch.zeros_like(t_ex)
    lin[:, [0, 3, 5]] = -1.0
    rel_lin = ((lin - t_ex).norm(dim=1) / t_ex.norm(dim=1))[ok]

    def q(x, p):
        return float(torch.quantile(x.float().cpu(), p)) if x.numel() else float("nan")

    full = S.error_report(s, mom, tau, y_ex, fl_ex, eps2_hat, params=prm,
                          lite=api.fp_moments_lite(v, off) if s.features_set == "lite" else None)
    return {
        "report": full,
        "cells": n_cells, "seed": seed, "inputs": s.features_set,
        "fallback_rate": float(fb.double().mean()),
        "range_flag_rate": float(((fl_s & api.FLAG_RANGE) != 0).double().mean()),
        "energy_flag_rate": float(((fl_s & api.FLAG_ENERGY) != 0).double().mean()),
        "rel_err_surrogate": {"median": q(rel, 0.5), "p95": q(rel, 0.95), "max": float(rel.max())},
        "rel_err_network_cells": {"median": q(rel_net, 0.5), "p95": q(rel_net, 0.95),
                                  "max": float(rel_net.max()) if rel_net.numel() else None},
        "standardised_l2_mean": float(std_err.mean()),
        "rel_err_linear_closure": {"median": q(rel_lin, 0.5), "p95": q(rel_lin, 0.95)},
    }


def evaluate_cylinder(s: S.Surrogate, eps2_hat):
    """The learned closure's error on the Mach-10 cylinder population
    (131072 cells, FP64 moments) against the exact FP64 closure."""
    pop = P.cylinder()
    dev = torch.device("cuda")
    v = torch.from_numpy(pop.v64).to(dev)
    off = torch.from_numpy(pop.offsets).to(dev)
    tau = torch.from_numpy(pop.tau).to(dev)
    prm = api.default_params(eps2_hat=eps2_hat)
    mom, y_ex, fl_ex = api.fp_closure_exact(v, off, tau, params=prm, prec="fp64")
    lite = api.fp_moments_lite(v, off) if s.features_set == "lite" else None
    rep = S.error_report(s, mom, tau, y_ex, fl_ex, eps2_hat, params=prm, lite=lite)
    torch.cuda.synchronize()
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-decay", type=float, default=0.85, help="per-epoch learning-rate factor")
    ap.add_argument("--eps2-hat", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--eval-cells", type=int, default=131072)
    ap.add_argument("--lam-drift", type=float, default=0.1, help="weight of the induced-drift term of the loss")
    ap.add_argument("--lam-energy", type=float, default=1.0, help="weight of the energy-residual term of the loss")
    ap.add_argument("--cylinder-fraction", type=float, default=0.0,
                    help="fraction of the training cells drawn from cylinder-like populations (fresh seeds)")
    ap.add_argument("--eval-cylinder", action="store_true",
                    help="also report the error on the Mach-10 cylinder population (FP64 moments)")
    ap.add_argument("--features", choices=sorted(S.FEATURE_SETS), default="full",
                    help="network inputs: the 25 high-order moments or the 16 LITE inputs")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights",
                                                  "surrogate_full.fpw"))
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    print(f"labelling {args.cells} training cells")
    ts = build_training_set(args.cells, args.seed, args.eps2_hat, features=args.features,
                            cylinder_fraction=args.cylinder_fraction)
    t_label = time.time() - t0
    s = S.Surrogate(eps2_hat=args.eps2_hat, seed=args.seed, features=args.features)
    s.init_params()
    S.fit_scalers(s, ts)
    tr = S.Trainer(s, batch=args.batch, lr=args.lr, lam_drift=args.lam_drift, lam_energy=args.lam_energy)
    t1 = time.time()
    hist = tr.fit(ts, epochs=args.epochs, seed=args.seed, log=print, lr_decay=args.lr_decay)
    t_train = time.time() - t1
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    s.save(args.out)
    rep = {"inputs": args.features, "training_cells": len(ts), "cylinder_fraction": args.cylinder_fraction,
           "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
           "lr_decay": args.lr_decay, "lam_drift": args.lam_drift, "lam_energy": args.lam_energy,
           "loss_history": hist, "label_seconds": t_label, "train_seconds": t_train,
           "held_out": evaluate(s, args.eval_cells, seed=987654, eps2_hat=args.eps2_hat)}
    if args.eval_cylinder:
        rep["cylinder"] = evaluate_cylinder(s, args.eps2_hat)
        print(json.dumps(rep["cylinder"], indent=1))
    with open(args.out + ".json", "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep["held_out"], indent=1))


if __name__ == "__main__":
    main()
