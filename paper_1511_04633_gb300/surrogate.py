"""Learned warm start: training data, training loop and time-to-steady-state.

The surrogate network (CUDA kernels behind ``dmrt_surrogate_*``) maps a
cavity's (Ra, wall type) to an approximate steady state.  This module

* builds training data: steady states of seeded cavities, solved by the
  lattice Boltzmann ensemble (``dmrt_ensemble_*``) and packed on the device;
* trains the network with the library's own forward / backward / Adam
  kernels (contiguous batches, visited in a seeded random order);
* measures what the warm start gains: steps and wall time until the hot-wall
  Nu_3D stays within a relative tolerance of its converged value, and until
  the residual falls below the convergence threshold, from rest and from the
  network's prediction.

Orchestration only: every arithmetic step runs in the library's kernels;
torch provides device memory.

The trained parameters ship with the package (``weights/``); this module
writes them (``--save-params``) and reads them back (``load_surrogate``).

    python -m paper_1511_04633_gb300.surrogate --grid 32 --train 48 --epochs 30
    python -m paper_1511_04633_gb300.surrogate --time-steps 3     # time the training step
    python -m paper_1511_04633_gb300.surrogate --time-steps 3 --layer 16,16   # one conv layer
    python -m paper_1511_04633_gb300.surrogate --test 0 --epochs 60 \
        --save-params paper_1511_04633_gb300/weights/warm_start_64cube.npz
"""

from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import dmrt, inputs

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
# the network trained on 512 steady states of 64^3 cavities (log10 Ra in [3, 6],
# wall types 1-3, draws of seed 2024), written by main() with --save-params
DEFAULT_PARAMS = os.path.join(WEIGHTS_DIR, "warm_start_64cube.npz")
# the seeded draws of that training run: the first 512 trained it, the rest
# are held out
TRAIN_SEED, TRAIN_COUNT = 2024, 512


def held_out_draws(count, grid=64):
    """The cavities (Ra, wall) of the training run's seeded draws that it
    did not train on."""
    draws = inputs.ensemble_draws(TRAIN_COUNT + count, seed=TRAIN_SEED, edges=(grid,), log10_ra=(3.0, 6.0))
    return draws[TRAIN_COUNT:]


def _to_bf16_bits(p):
    """float32 -> bfloat16 bit patterns, rounded to nearest even (the
    conversion the BF16 network applies to its master weights)."""
    b = np.ascontiguousarray(p, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def bias_mask(depth, channels, features=8, out=5):
    """Which entries of the flat parameter vector are biases, from the
    layout include/dmrt.h states: layer by layer (a_0, s_0, then a_l, s_l
    for l = 1..D, then d_l, h_l for l = D-1..0, then the 1x1 head), each
    layer's weights [tap][cout][cin] followed by its cout biases."""
    c = list(channels)[:depth + 1]
    layers = [(features, c[0], 27), (c[0], c[0], 27)]
    for l in range(1, depth + 1):
        layers += [(c[l - 1], c[l], 27), (c[l], c[l], 27)]
    for l in range(depth - 1, -1, -1):
        layers += [(c[l + 1], c[l], 27), (c[l], c[l], 27)]
    layers.append((c[0], out, 1))
    mask = []
    for cin, cout, taps in layers:
        mask += [False] * (taps * cout * cin) + [True] * cout
    return np.array(mask)


def save_params(sur, path, info=None):
    """Write a BF16 network's configuration and parameters.  The BF16
    network multiplies with its weights rounded to bfloat16 and adds its
    biases in FP32, so the file holds the weights rounded the same way and
    the biases as they are (about half the bytes of FP32): a network loaded
    from it predicts exactly what the saved one did."""
    if sur.storage != dmrt.STORE_BF16:
        raise ValueError("save_params stores the weights of a BF16 network")
    p = sur.params()
    mask = bias_mask(sur.depth, sur.channels)
    if mask.size != p.size:
        raise ValueError(f"layout of {mask.size} parameters for a network of {p.size}")
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez_compressed(path, weights_bf16=_to_bf16_bits(p[~mask]), biases=p[mask].astype(np.float32),
                        grid=sur.grid, depth=sur.depth, channels=np.array(sur.channels),
                        info=json.dumps(info or {}))


def load_surrogate(path=DEFAULT_PARAMS, max_batch=1):
    """A BF16 surrogate with the parameters of a file written by save_params.
    Returns (surrogate, info dict)."""
    with np.load(path) as z:
        depth, channels = int(z["depth"]), tuple(int(c) for c in z["channels"])
        sur = dmrt.Surrogate(int(z["grid"]), depth, channels, dmrt.STORE_BF16, max_batch=max_batch)
        mask = bias_mask(depth, channels)
        if mask.size != sur.param_count:
            raise ValueError(f"{path}: layout of {mask.size} parameters for a network of {sur.param_count}")
        p = np.empty(mask.size, np.float32)
        p[~mask] = (z["weights_bf16"].astype(np.uint32) << 16).view(np.float32)
        p[mask] = z["biases"]
        sur.set_params(p)
        info = json.loads(str(z["info"]))
    return sur, info


def steady_dataset(n, draws, tol=1e-6, max_steps=200_000, group=64, storage=dmrt.STORE_F32):
    """Steady states of cubic n^3 cavities, one per draw {"Ra", "wall"}, solved
    to residual < tol (1e-6 leaves errors far below what the network learns).

    Returns (Ra [N], wall [N], targets: CUDA tensor [N][n^3][5], info)."""
    import torch

    count = len(draws)
    tgt = torch.empty((count, n ** 3, 5), dtype=torch.float32, device="cuda")
    u = torch.empty((3, n, n, n), dtype=torch.float32, device="cuda")
    th = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    rho = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    residual = np.zeros(count)
    steps = []
    t0 = time.perf_counter()
    for g0 in range(0, count, group):
        part = draws[g0:g0 + group]
        ens = dmrt.Ensemble([{"grid": (n, n, n), "Ra": d["Ra"], "wall": d["wall"]} for d in part],
                            storage=storage)
        ens.autotune(trials=2)
        ok, st, conv = ens.run_to_steady(tol, max_steps)
        steps.append(st)
        residual[g0:g0 + len(part)] = ens.residual()
        for k in range(len(part)):
            dmrt.dmrt_ensemble_fields(ens.e, k, rho=rho, u=u, theta=th)
            uc = math.sqrt(ens.params(k)["gbeta"] * n)
            dmrt.dmrt_surrogate_target_from_fields(u, th, rho, n, uc, tgt[g0 + k])
            torch.cuda.synchronize()
        ens.close()
    ra = np.array([d["Ra"] for d in draws], dtype=np.float64)
    wall = np.array([d["wall"] for d in draws], dtype=np.int32)
    info = {"seconds": time.perf_counter() - t0, "steps_per_group": steps,
            "max_residual": float(np.max(residual)), "converged": int(np.sum(residual < tol))}
    return ra, wall, tgt, info


def learning_rate(lr, it, total, warmup):
    """Linear warm-up over `warmup` iterations, then cosine decay to zero."""
    if it < warmup:
        return lr * (it + 1) / warmup
    frac = (it - warmup) / max(total - warmup, 1)
    return max(lr * 0.5 * (1.0 + math.cos(math.pi * frac)), 1e-7)


def train(sur, ra, wall, targets, epochs, batch, lr=5e-4, seed=0, log=None, warmup=None):
    """Adam over contiguous batches visited in a seeded random order, with a
    linear warm-up and cosine decay of the learning rate.  Returns the mean
    loss of every epoch; stops early if the loss becomes non-finite or grows
    a thousandfold (the caller sees the short history)."""
    rng = np.random.default_rng(seed)
    count = len(ra)
    nb = count // batch
    total = epochs * nb
    if warmup is None:
        warmup = max(1, total // 20)
    history = []
    it = 0
    first = None
    for ep in range(epochs):
        acc = 0.0
        for b in rng.permutation(nb):
            lo = b * batch
            loss = sur.train_step(ra[lo:lo + batch], wall[lo:lo + batch], targets[lo:lo + batch],
                                  learning_rate(lr, it, total, warmup))
            first = loss if first is None else first
            if not math.isfinite(loss) or loss > 1e3 * first:
                history.append(loss)
                if log:
                    log(f"training diverged at iteration {it}: loss {loss}")
                return history
            acc += loss
            it += 1
        history.append(acc / max(nb, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {history[-1]:.5g}")
    return history


def solve(cav, tol=1e-7, max_steps=2_000_000, chunk=None):
    """Step a cavity to residual < tol, recording (steps, Nu_3D) after every
    residual interval.  Returns (steps, seconds, records)."""
    import torch

    K = chunk or cav.params["residual_interval"]
    records = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        cav.step(K)
        steps += K
        records.append((steps, cav.nusselt(0)[0], time.perf_counter() - t0))
        if cav.residual() < tol:
            break
    return steps, time.perf_counter() - t0, records


def time_to_nu(records, nu_ref, rtol):
    """First (steps, seconds) after which Nu_3D stays within rtol of nu_ref."""
    for i, (s, nu, t) in enumerate(records):
        if all(abs(v - nu_ref) <= rtol * abs(nu_ref) for _, v, _ in records[i:]):
            return s, t
    return None, None


def compare_warm_start(sur, grid, Ra, wall, tol=1e-7, nu_rtol=1e-3, max_steps=2_000_000,
                       storage=dmrt.STORE_F32, ref_tol=1e-9):
    """From-rest against warm-started solve of one cubic cavity.  The Nu
    reference is the from-rest solve continued to residual < ref_tol (a
    residual of 1e-7 per step still leaves drifts of a few 1e-4 in Nu)."""
    import torch

    cold = dmrt.Cavity((grid,) * 3, Ra, wall_type=wall, storage=storage)
    s_cold, t_cold, rec_cold = solve(cold, tol, max_steps)
    nu_at_tol = cold.nusselt(0)[0]
    s_ref, _, rec_ref = solve(cold, ref_tol, max(s_cold, 10_000))
    nu_ref = cold.nusselt(0)[0]
    rec_cold = rec_cold + [(s + s_cold, nu, t) for s, nu, t in rec_ref]
    cold.close()
    warm = dmrt.Cavity((grid,) * 3, Ra, wall_type=wall, storage=storage)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.warm_start(warm, Ra, wall)
    t_pred = time.perf_counter() - t0
    s_warm, t_warm, rec_warm = solve(warm, tol, max_steps)
    nu_warm = warm.nusselt(0)[0]
    warm.close()
    n_cold = time_to_nu(rec_cold, nu_ref, nu_rtol)
    n_warm = time_to_nu(rec_warm, nu_ref, nu_rtol)
    return {
        "grid": grid, "Ra": Ra, "wall": wall, "tol": tol, "nu_rtol": nu_rtol,
        "nu_reference": nu_ref, "reference_extra_steps": s_ref,
        "nu_from_rest_at_tol": nu_at_tol, "nu_warm_at_tol": nu_warm,
        "nu_rel_diff": abs(nu_warm - nu_ref) / nu_ref,
        "from_rest": {"steps_to_residual": s_cold, "seconds_to_residual": t_cold,
                      "steps_to_nu": n_cold[0], "seconds_to_nu": n_cold[1]},
        "warm": {"predict_seconds": t_pred, "steps_to_residual": s_warm,
                 "seconds_to_residual": t_warm + t_pred,
                 "steps_to_nu": n_warm[0],
                 "seconds_to_nu": None if n_warm[1] is None else n_warm[1] + t_pred},
    }


def time_steps(args):
    """Wall time of training steps and predictions of the configured network
    on zero targets (one warm-up step first)."""
    import torch

    ch = tuple(int(c) for c in args.channels.split(","))
    sur = dmrt.Surrogate(args.grid, args.depth, ch,
                         dmrt.STORE_BF16 if args.storage == "bf16" else dmrt.STORE_F32,
                         max_batch=args.batch, seed=args.seed)
    t = torch.zeros((args.batch, args.grid ** 3, 5), device="cuda")
    ra = [10.0 ** (3 + 3 * k / max(args.batch - 1, 1)) for k in range(args.batch)]
    wall = [1 + k % 3 for k in range(args.batch)]
    sur.train_step(ra, wall, t, 1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.time_steps):
        sur.train_step(ra, wall, t, 1e-4)
    torch.cuda.synchronize()
    step = (time.perf_counter() - t0) / args.time_steps
    t0 = time.perf_counter()
    for _ in range(args.time_steps):
        sur.predict(ra[:1], wall[:1])
    torch.cuda.synchronize()
    pred = (time.perf_counter() - t0) / args.time_steps
    res = {"train_step_ms": step * 1e3, "predict_ms": pred * 1e3, "params": sur.param_count,
           "grid": args.grid, "batch": args.batch}
    print(json.dumps(res), flush=True)
    return res


def time_layer(args):
    """Calls of one 3^3 convolution layer of the network (dmrt_nn_conv3d,
    bf16, leaky ReLU) on seeded random activations and weights at the
    configured grid and batch: one warm-up call, then --time-steps timed
    calls (each synchronises)."""
    import torch

    cin, cout = (int(c) for c in args.layer.split(","))
    n, batch = args.grid, args.batch
    x = torch.from_numpy(inputs.random_targets((batch, n, n, n, cin), seed=1)).to(torch.bfloat16).cuda()
    w = torch.from_numpy(inputs.random_weights(27 * cout * cin, seed=2, scale=0.2)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(inputs.random_weights(cout, seed=3, scale=0.5)).cuda()
    y = torch.empty((batch, n, n, n, cout), dtype=torch.bfloat16, device="cuda")
    dmrt.dmrt_nn_conv3d(x, w, b, y, batch, n, cin, cout, 3, act=1)
    t0 = time.perf_counter()
    for _ in range(args.time_steps):
        dmrt.dmrt_nn_conv3d(x, w, b, y, batch, n, cin, cout, 3, act=1)
    per_call = (time.perf_counter() - t0) / args.time_steps
    res = {"layer": [cin, cout], "grid": n, "batch": batch, "call_ms": per_call * 1e3,
           "tensor_core_errors": dmrt.dmrt_nn_tensor_core_errors(reset=True)}
    print(json.dumps(res), flush=True)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the warm-start surrogate and measure its gain")
    ap.add_argument("--grid", type=int, default=64, help="network (and training cavity) grid")
    ap.add_argument("--depth", type=int, default=3)
    ap.add_argument("--channels", type=str, default="16,32,64,128")
    ap.add_argument("--storage", choices=["f32", "bf16"], default="bf16")
    ap.add_argument("--train", type=int, default=512, help="training cavities")
    ap.add_argument("--test", type=int, default=4, help="held-out cavities")
    ap.add_argument("--target-grid", type=int, default=128, help="grid of the warm-started solves")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--data-tol", type=float, default=1e-6, help="residual of the training states")
    ap.add_argument("--ra", type=str, default="3,6", help="log10 Ra range")
    ap.add_argument("--max-steps", type=int, default=200_000)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--out", type=str, default="")
    ap.add_argument("--save-params", type=str, default="",
                    help="write the trained parameters (BF16 network) to this .npz file")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="only time this many training steps (zero targets) and predictions")
    ap.add_argument("--layer", type=str, default="",
                    help="with --time-steps: time one 3^3 convolution layer CIN,COUT instead")
    args = ap.parse_args(argv)
    import torch

    if args.time_steps > 0:
        return time_layer(args) if args.layer else time_steps(args)

    lo, hi = (float(v) for v in args.ra.split(","))
    draws = inputs.ensemble_draws(args.train + args.test, seed=args.seed, edges=(args.grid,),
                                  log10_ra=(lo, hi))
    train_draws, test_draws = draws[:args.train], draws[args.train:]
    ra, wall, tgt, info = steady_dataset(args.grid, train_draws, tol=args.data_tol,
                                         max_steps=args.max_steps)
    print(json.dumps({"dataset": info}), flush=True)
    ch = tuple(int(c) for c in args.channels.split(","))
    sur = dmrt.Surrogate(args.grid, args.depth, ch,
                         dmrt.STORE_BF16 if args.storage == "bf16" else dmrt.STORE_F32,
                         max_batch=args.batch, seed=args.seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = train(sur, ra, wall, tgt, args.epochs, args.batch, args.lr, seed=args.seed,
                 log=lambda m: print(m, flush=True))
    t_train = time.perf_counter() - t0
    results = {"params": sur.param_count, "train_seconds": t_train, "loss_first": hist[0],
               "loss_last": hist[-1], "epochs_run": len(hist), "dataset": info, "cases": []}
    if not math.isfinite(hist[-1]) or len(hist) < args.epochs:
        print(json.dumps({"error": "training diverged", "history": hist}), flush=True)
        return results
    if args.save_params:
        info = {"grid": args.grid, "depth": args.depth, "channels": ch, "train": args.train,
                "seed": args.seed, "log10_ra": [lo, hi], "epochs": args.epochs, "batch": args.batch,
                "lr": args.lr, "data_tol": args.data_tol, "loss_first": hist[0], "loss_last": hist[-1],
                "dataset_seconds": info["seconds"], "train_seconds": t_train}
        save_params(sur, args.save_params, info)
        loaded, _ = load_surrogate(args.save_params)
        probe_ra, probe_wall = [float(train_draws[0]["Ra"])], [int(train_draws[0]["wall"])]
        same = np.array_equal(loaded.predict(probe_ra, probe_wall), sur.predict(probe_ra, probe_wall))
        print(json.dumps({"saved": args.save_params, "reloaded_predicts_the_same": bool(same)}), flush=True)
        loaded.close()
    for d in test_draws:
        r = compare_warm_start(sur, args.target_grid, d["Ra"], d["wall"], max_steps=args.max_steps * 8)
        results["cases"].append(r)
        print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(results, fh, indent=1)
    return results


if __name__ == "__main__":
    main()
