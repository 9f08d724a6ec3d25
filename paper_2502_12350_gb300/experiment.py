"""Learned vs plain preconditioned FWI on the 160x160x80 workload.

Trains the GN-diagonal network on exact labels of seeded models of the
layered family (same acquisition as the inversion: 12 shots, 64 receivers,
1500 steps; 400 training and 20 held-out models by default), reports the
held-out accuracy of the network against the pseudo-Hessian, then inverts a
further model from the same blurred start once per preconditioner arm:
none, the pseudo-Hessian (the plain method), the learned diagonal (falling
back to the pseudo-Hessian step when the learned step fails Armijo) and the
exact GN diagonal recomputed at every iterate.  Writes a JSON report with
misfit against wall time for every arm.

With --test-models and --waters the comparison is made on several inverted
models: each arm's water level (the floor of its preconditioning diagonal,
as a fraction of its maximum) is first chosen on a validation model by the
lowest final misfit, then every test model is inverted by every arm at its
chosen level, and the report gives, per model, each arm's final misfit, wall
time and the wall time at which it reached the plain (pseudo-Hessian) run's
final misfit.

    python -m paper_2502_12350_gb300.experiment --out report.json
    python -m paper_2502_12350_gb300.experiment --out report.json --train-models 80 \
        --heldout-models 20 --arms pseudo,learned --waters 0.002,0.01,0.05 \
        --val-model 5100 --test-models 5420,5421,5422
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train-models", type=int, default=400)
    ap.add_argument("--heldout-models", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--nt", type=int, default=1500)
    ap.add_argument("--nx", type=int, default=160)
    ap.add_argument("--ny", type=int, default=160)
    ap.add_argument("--nz", type=int, default=80)
    ap.add_argument("--test-model", type=int, default=5420)
    ap.add_argument("--water", type=float, default=0.05,
                    help="water level of the preconditioning diagonals (fraction of the max)")
    ap.add_argument("--save-net", default=None, help="write the trained network (.npz)")
    ap.add_argument("--load-net", default=None,
                    help="use a trained network (.npz) instead of labelling and training")
    ap.add_argument("--arms", default="none,pseudo,learned,exact")
    ap.add_argument("--waters", default=None,
                    help="comma list: choose each arm's water level on --val-model")
    ap.add_argument("--val-model", type=int, default=5100)
    ap.add_argument("--test-models", default=None, help="comma list of inverted models")
    args = ap.parse_args(argv)

    from . import build, cnn, fwi, learned, mamute, synth
    build.build()
    dev = torch.device("cuda", 0)
    ctx = mamute.Context(0)
    report = {"config": vars(args)}

    def wl(mid):
        return synth.fwi_small(model_id=mid, nt=args.nt, nx=args.nx, ny=args.ny, nz=args.nz)

    net = cnn.Net(ctx, seed=1)
    # training models 5000 .. 5000+n-1, held-out models right after them,
    # the inverted model after those
    train_ids = list(range(5000, 5000 + args.train_models))
    test_ids = list(range(5000 + args.train_models, 5000 + args.train_models + args.heldout_models))
    assert args.test_model not in train_ids + test_ids
    if args.load_net:
        z = np.load(args.load_net)
        ws = [z[f"w{l}"] for l in range(cnn.LAYERS)]
        bs = [z[f"b{l}"] for l in range(cnn.LAYERS)]
        net = cnn.Net(ctx, weights=(ws, bs))
        net.offset = float(z["offset"])
        report["loaded_net"] = args.load_net
    else:
        t0 = time.perf_counter()
        data = learned.dataset(ctx, net, wl, train_ids, seed=1)
        held = learned.dataset(ctx, net, wl, test_ids, seed=2, set_offset=False)
        report["offset"] = net.offset
        torch.cuda.synchronize()
        report["label_seconds"] = time.perf_counter() - t0
        report["label_seconds_per_model"] = report["label_seconds"] / (len(train_ids) + len(test_ids))
        t0 = time.perf_counter()
        hist = learned.train(net, data, args.epochs, lr=args.lr,
                             log=lambda m: print(m) if m.split(":")[0].endswith("0") else None)
        torch.cuda.synchronize()
        report["train_seconds"] = time.perf_counter() - t0
        report["train_loss"] = hist
        errs = learned.log_errors(net, held)
        report["heldout_log_rms"] = {"network": [e[0] for e in errs],
                                     "pseudo_hessian_rescaled": [e[1] for e in errs]}
        print("held-out RMS log error (network, rescaled P): %.3f %.3f" %
              (np.mean([e[0] for e in errs]), np.mean([e[1] for e in errs])))
        del data, held
        if args.save_net:
            ws, bs = net.weights()
            np.savez(args.save_net, offset=net.offset, **{f"w{l}": ws[l] for l in range(cnn.LAYERS)},
                     **{f"b{l}": bs[l] for l in range(cnn.LAYERS)})

    def invert(mid, kind, water):
        w = wl(mid)
        g = mamute.grid_of(w)
        vt = torch.from_numpy(w.vel).to(dev)
        dobs = torch.empty((int(w.rec_offset[-1]), w.nt), device=dev)
        ctx.model(g, vt, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs)
        vmin, vmax = float(w.vel.min()) * 0.9, float(w.vel.max()) * 1.1
        prob = fwi.Problem(ctx, w, dobs, vmin, vmax)
        res = fwi.run(prob, w.vel_init.astype(np.float64), args.iters, precond=kind, net=net,
                      water=water)
        err = float(np.sqrt(np.mean((res.vel - w.vel) ** 2)))
        print(mid, kind, water, "final misfit", res.history[-1][1], "model error", err,
              "time", res.history[-1][0], flush=True)
        return {"history": [(t, J, k) for t, J, k in res.history], "model_rms_error": err,
                "gradients": res.n_gradients, "forward_models": res.n_forward, "water": water,
                "initial_model_rms_error": float(np.sqrt(np.mean((w.vel_init - w.vel) ** 2)))}

    def time_to(runs, target):
        for kind in runs:
            runs[kind]["seconds_to_plain_final_misfit"] = None if target is None else next(
                (t for t, J, _ in runs[kind]["history"] if J <= target), None)

    arms = args.arms.split(",")
    if args.test_models:
        assert args.val_model not in train_ids + test_ids
        water = {k: args.water for k in arms}
        if args.waters:
            levels = [float(v) for v in args.waters.split(",")]
            val = {k: {str(lv): invert(args.val_model, k, lv) for lv in levels} for k in arms}
            report["validation"] = {k: {lv: r["history"][-1][1] for lv, r in v.items()}
                                    for k, v in val.items()}
            water = {k: float(min(v, key=lambda lv: v[lv]["history"][-1][1]))
                     for k, v in val.items()}
        report["chosen_water"] = water
        models = {}
        for mid in [int(v) for v in args.test_models.split(",")]:
            assert mid not in train_ids + test_ids + [args.val_model]
            runs = {k: invert(mid, k, water[k]) for k in arms}
            time_to(runs, runs["pseudo"]["history"][-1][1] if "pseudo" in runs else None)
            models[str(mid)] = runs
        report["fwi_models"] = models
        summary = {}
        for mid, runs in models.items():
            summary[mid] = {k: {"final_misfit": r["history"][-1][1], "seconds": r["history"][-1][0],
                                "seconds_to_plain_final_misfit": r["seconds_to_plain_final_misfit"],
                                "model_rms_error": r["model_rms_error"]} for k, r in runs.items()}
        report["summary"] = summary
        with open(args.out, "w") as f:
            json.dump(report, f, indent=1)
        ctx.close()
        return

    w = wl(args.test_model)
    report["initial_model_rms_error"] = float(np.sqrt(np.mean((w.vel_init - w.vel) ** 2)))
    runs = {kind: invert(args.test_model, kind, args.water) for kind in arms}
    # wall time for each run to reach the plain run's final misfit
    time_to(runs, runs["pseudo"]["history"][-1][1] if "pseudo" in runs else None)
    report["fwi"] = runs
    with open(args.out, "w") as f:
        json.dump(report, f, indent=1)
    ctx.close()


if __name__ == "__main__":
    main()
