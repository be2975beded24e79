"""Train the learned pressure guess on the GPU and measure what it saves.

Training pairs come from the solver itself, generated on the fly so that no
pair is seen twice: for a Gaussian direction v (walls zero) on an
N^3 cosine-mapped grid at Re drawn from [re_lo, re_hi], w = L_U v (the
momentum predictor of Eq. 10), r = D w and phi = (D G)^+ r by the exact
tensor-product solve, all through the C-ABI in float64.  U is the smooth
sample vortex flow of the synthetic inputs.  Every step is one
fv_unet_train_step (forward, backward, Adam on the device).

Evaluation at larger grids on held-out directions: the relative error of
the guess, and SIMPLE passes and device time of one Krylov-vector
evaluation (eps = 1e-8) with the plain loop (exact first pass) against the
loop whose first pass is the guess; and conjugate-gradient iterations and
device time of the multigrid pressure solve (relative residual --mg-rtol)
from zero against the same solve started from the guess.

    python -m paper_1704_08521_gb300.unet_train --train 64,80,96,112,128 \
        --steps 600 --eval 200,256 --rhs 4 [--save params.npy]

Prints one JSON object.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def gaussian_direction(shape, gen, torch):
    """Standard-normal velocity vector with zero wall entries (device)."""
    nz, ny, nx = shape
    v = torch.randn(3, nz, ny, nx, dtype=torch.float64, device="cuda", generator=gen)
    v[0, :, :, 0] = 0.0
    v[1, :, 0, :] = 0.0
    v[2, 0, :, :] = 0.0
    return v.reshape(-1)


def make_pair(fv, g, U, v, torch):
    w = torch.empty_like(v)
    fv.ns_jacvec(g, U, v, w, prec="fp64")
    r = torch.empty(g.n_cell, dtype=torch.float64, device="cuda")
    fv.ns_divergence(g, w, r)
    phi = torch.empty_like(r)
    fv.fv_pressure_solve(g, r, phi, prec="fp64")
    return r, phi


def timed(torch, fn, reps=3):
    """Median device time (ms) of fn() over reps calls after one warm-up."""
    fn()
    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        res = fn()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out)), res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", default="64,80,96,112,128")
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--re", default="1850,1950")
    ap.add_argument("--eval", default="200,256")
    ap.add_argument("--rhs", type=int, default=4)
    ap.add_argument("--eps", type=float, default=1e-8)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--save", default=None)
    ap.add_argument("--mg-rtol", type=float, default=1e-8)
    a = ap.parse_args(argv)

    import torch
    import paper_1704_08521_gb300 as fv
    import synth

    train = sorted((int(s) for s in a.train.split(",")), reverse=True)
    re_lo, re_hi = (float(s) for s in a.re.split(","))
    gen = torch.Generator(device="cuda").manual_seed(a.seed)
    rng = np.random.default_rng(a.seed)
    net = fv.UNet(seed=a.seed)

    grids, flows = {}, {}
    for n in train:
        grids[n] = fv.Grid(n, n, n, map="cosine", alpha=0.0, re=1900.0)
        flows[n] = torch.tensor(synth.vortex_base_flow((n, n, n), "cosine", 0.0), device="cuda")

    losses = []
    t0 = time.time()
    train_ms = 0.0
    for step in range(a.steps):
        n = train[step % len(train)]
        g = grids[n]
        g.set_re(float(rng.uniform(re_lo, re_hi)))
        v = gaussian_direction(g.shape, gen, torch)
        r, phi = make_pair(fv, g, flows[n], v, torch)
        lr = a.lr if step < 0.7 * a.steps else 0.25 * a.lr
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        losses.append(net.train_step(g, r, phi, lr))
        e1.record()
        torch.cuda.synchronize()
        train_ms += e0.elapsed_time(e1)
    wall = time.time() - t0
    k = max(1, len(train))
    summary = {
        "train_sizes": train, "steps": a.steps, "lr": a.lr, "re": [re_lo, re_hi],
        "loss_first": float(np.mean(losses[:k])), "loss_last": float(np.mean(losses[-k:])),
        "train_step_ms_mean": train_ms / max(1, a.steps), "train_wall_s": wall,
        "n_param": net.n_param, "eval": [],
    }
    if a.save:
        p = torch.empty(net.n_param, dtype=torch.float32, device="cuda")
        net.get_params(params=p)
        np.save(a.save, p.cpu().numpy())
    del grids, flows

    for n in (int(s) for s in a.eval.split(",")):
        for re in (1900.0, 1950.0):
            g = fv.Grid(n, n, n, map="cosine", alpha=0.0, re=re)
            U = torch.tensor(synth.vortex_base_flow((n, n, n), "cosine", 0.0), device="cuda")
            rows = []
            for s in range(a.rhs):
                v = torch.tensor(synth.gaussian_velocity((n, n, n), 50000 + s), device="cuda")
                r, phi = make_pair(fv, g, U, v, torch)
                guess = torch.empty_like(phi)
                ms_guess_only, _ = timed(torch, lambda: net.guess(g, r, guess))
                gs = guess - guess.mean()
                ph = phi - phi.mean()
                err = float(torch.linalg.vector_norm(gs - ph) / torch.linalg.vector_norm(ph))
                err_max = float((gs - ph).abs().max() / ph.abs().max())
                out = torch.empty_like(v)
                ms_plain, st_plain = timed(torch, lambda: fv.simple_krylov_solve(
                    g, U, v, out, eps=a.eps, prec="mixed"))
                ms_guess, st_guess = timed(torch, lambda: fv.simple_krylov_solve_guess(
                    g, net, U, v, out, eps=a.eps, prec="mixed"))
                phi_tpf = torch.empty_like(phi)
                ms_tpf, _ = timed(torch, lambda: fv.fv_pressure_solve(g, r, phi_tpf, prec="mixed"))
                # the multigrid pressure solve to rtol from zero and from the guess
                phi_mg = torch.empty_like(phi)
                ms_mg0, st_mg0 = timed(torch, lambda: fv.fv_pressure_solve_mg(g, r, phi_mg, rtol=a.mg_rtol))

                def mg_from_guess():
                    net.guess(g, r, guess)
                    return fv.fv_pressure_solve_mg(g, r, phi_mg, guess=guess, rtol=a.mg_rtol)
                ms_mg1, st_mg1 = timed(torch, mg_from_guess)
                rows.append({"guess_rel_err": err, "guess_rel_err_max": err_max, "passes_plain": st_plain["passes"],
                             "passes_guess": st_guess["passes"], "ms_plain": ms_plain,
                             "ms_guess": ms_guess, "ms_net": ms_guess_only, "ms_exact_solve": ms_tpf,
                             "mg_iters_zero": st_mg0["iterations"], "mg_iters_guess": st_mg1["iterations"],
                             "ms_mg_zero": ms_mg0, "ms_mg_guess": ms_mg1})
            agg = {key: float(np.mean([row[key] for row in rows])) for key in rows[0]}
            # exact solves the loop needed: plain = passes; guess = passes - 1
            agg["exact_solves_saved"] = agg["passes_plain"] - (agg["passes_guess"] - 1)
            summary["eval"].append({"n": n, "re": re, **agg})
            del g
            torch.cuda.empty_cache()
    print(json.dumps(summary))
    return summary


if __name__ == "__main__":
    main()
