"""Learned warm start: generate training data with the solver, train the
neural operator with libqn's own BF16 forward/backward/AdamW kernels, and
compare warm-started solves with zero-start solves.

  python -m paper_2502_03611_gb300.warmstart --n 255 --G 64 --train 4096 --test 256

Workload: -Lap u + u^3 = f on the n^3 interior grid (Dirichlet 0), f a
Dirichlet-consistent Gaussian random field with power spectrum
(1 + |k|^2)^-2 rescaled to RMS `scale` (1 = unit variance). Training data:
solutions of the quasi-Newton method itself (BF16x3 mode products, FP64
residual, tolerance 1e-10), restricted with the library's trilinear transfer
to the coarse G^3 grid. Every solver and network step runs in libqn; torch
holds device memory and synthesises the GRF inputs.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

import numpy as np

from . import qn
from .inputs import grf_source_torch, random_field


def init_params(C: int, M: int, L: int, seed: int = 1234) -> np.ndarray:
    """Seeded initial parameters (uniform, fan-in scaled; biases zero)."""
    n = int(qn.load_library().qn_net_param_count(C, M, L))
    p = np.zeros(n, dtype=np.float64)
    u = random_field((n,), seed)                  # U(-1, 1)
    o = 0
    p[o:o + C] = u[o:o + C]                       # wl (fan-in 1)
    o += 2 * C                                    # bl = 0
    K = M ** 3
    for _ in range(L):
        k = K * C * C
        p[o:o + k] = u[o:o + k] * math.sqrt(3.0 / C) * 0.5   # R: per-mode C x C mixing
        o += k
        p[o:o + C * C] = u[o:o + C * C] * math.sqrt(3.0 / C)  # W
        o += C * C + C                                          # b = 0
    p[o:o + C] = u[o:o + C] * math.sqrt(3.0 / C)               # wp
    o += C + 1
    assert o == n
    return p.astype(np.float32)


def generate(ctx, G: int, n: int, seeds, scale: float, tol: float = 1e-10):
    """Solve each GRF problem with the library and restrict f and U to G^3."""
    import torch
    N = len(seeds)
    f_c = torch.empty(N * G ** 3, dtype=torch.float32, device="cuda")
    u_c = torch.empty(N * G ** 3, dtype=torch.float32, device="cuda")
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    its = []
    for k, s in enumerate(seeds):
        f = grf_source_torch(n, s, scale=scale).reshape(-1).contiguous()
        U.zero_()
        res, _ = qn.qn_solve(ctx, U, f, tol=tol, max_it=200)
        if res["status"] != 0:
            raise RuntimeError(f"training solve {s} failed: {res}")
        its.append(res["iterations"])
        qn.qn_interp3d(f, n, f_c[k * G ** 3:(k + 1) * G ** 3], G)
        qn.qn_interp3d(U, n, u_c[k * G ** 3:(k + 1) * G ** 3], G)
    return f_c, u_c, its


def train(net, f_c, u_c, in_scale: float, out_scale: float, epochs: int, batch: int, lr: float,
          wd: float = 1e-4, seed: int = 0, log_every: int = 0):
    """AdamW training of qn_net on (in_scale f_c, u_c / out_scale); cosine
    learning-rate decay. in_scale, out_scale make inputs and targets unit RMS."""
    import torch
    G3 = net.G ** 3
    N = f_c.numel() // G3
    target = (u_c / out_scale).contiguous()
    f_c = (f_c * in_scale).contiguous()
    rng = np.random.default_rng(seed)
    steps_per_epoch = N // batch
    total = epochs * steps_per_epoch
    fb = torch.empty(batch * G3, dtype=torch.float32, device="cuda")
    tb = torch.empty(batch * G3, dtype=torch.float32, device="cuda")
    losses = []
    step = 0
    for ep in range(epochs):
        perm = rng.permutation(N)
        ep_loss = []
        for s in range(steps_per_epoch):
            idx = torch.from_numpy(perm[s * batch:(s + 1) * batch]).cuda()
            fb.copy_(f_c.view(N, G3).index_select(0, idx).reshape(-1))
            tb.copy_(target.view(N, G3).index_select(0, idx).reshape(-1))
            cur_lr = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            want = (s == steps_per_epoch - 1) or (log_every and s % log_every == 0)
            loss = net.train_step(fb, tb, batch, cur_lr, wd, want_loss=want)
            if want:
                ep_loss.append(loss)
            step += 1
        losses.append(statistics.mean(ep_loss))
    return losses


def evaluate(ctx, net, n: int, seeds, scale: float, in_scale: float, out_scale: float, tol: float = 1e-10):
    """Zero-start vs warm-start solves (time to tol with CUDA events, warm time
    includes the restriction, the network and the prolongation)."""
    import torch
    stream = torch.cuda.current_stream()
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    out = []
    for s in seeds:
        f = grf_source_torch(n, s, scale=scale).reshape(-1).contiguous()
        row = {"seed": s}
        for mode in ("zero", "warm"):
            U.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "zero":
                res, _ = qn.qn_solve(ctx, U, f, tol=tol, max_it=200)
                used = False
            else:
                res = qn.qn_solve_warm(ctx, net, U, f, in_scale=in_scale, out_scale=out_scale, tol=tol, max_it=200)
                used = res["used_warm"]
            e1.record(stream)
            torch.cuda.synchronize()
            row[mode] = {"iterations": res["iterations"], "ms": e0.elapsed_time(e1), "status": res["status"],
                         "rel": res["rel"]}
            if mode == "warm":
                row[mode]["used_warm"] = used
        # quality of U0 alone: ||F(U0)|| / ||f|| and its error against the solution
        Ustar = U.clone()
        U.zero_()
        qn.qn_solve(ctx, U, f, tol=tol, max_it=200)
        Ustar.copy_(U)
        net.predict(f, n, U, in_scale, out_scale)
        st = qn.qn_residual(ctx, U, f)
        row["u0_rel_residual"] = st["rel"]
        row["u0_rel_error"] = float(torch.linalg.vector_norm(U - Ustar) / torch.linalg.vector_norm(Ustar))
        out.append(row)
    return out


def summarise(rows):
    z_it = [r["zero"]["iterations"] for r in rows]
    w_it = [r["warm"]["iterations"] for r in rows]
    z_ms = [r["zero"]["ms"] for r in rows]
    w_ms = [r["warm"]["ms"] for r in rows]
    return {"cases": len(rows),
            "zero_iterations_mean": statistics.mean(z_it), "warm_iterations_mean": statistics.mean(w_it),
            "zero_ms_median": statistics.median(z_ms), "warm_ms_median": statistics.median(w_ms),
            "iterations_saved_mean": statistics.mean(z - w for z, w in zip(z_it, w_it)),
            "warm_used_fraction": sum(r["warm"]["used_warm"] for r in rows) / len(rows),
            "u0_rel_residual_median": statistics.median(r["u0_rel_residual"] for r in rows),
            "u0_rel_error_median": statistics.median(r["u0_rel_error"] for r in rows),
            "all_converged": all(r["zero"]["status"] == 0 and r["warm"]["status"] == 0 for r in rows)}


def run(n=255, G=64, modes=6, blocks=4, ntrain=4096, ntest=256, scale=1.0, epochs=12, batch=8, lr=2e-3,
        train_seed0=0, test_seed0=100000, log=print, precision="bf16x3", also=()):
    """Generate the training solves and evaluate with a `precision` context; `also`: more
    precisions whose zero / warm solves are evaluated on the same held-out seeds (their
    summaries under summ["by_precision"])."""
    import torch
    ctx = qn.QnContext(3, n, precision)
    t0 = time.time()
    f_c, u_c, its = generate(ctx, G, n, range(train_seed0, train_seed0 + ntrain), scale)
    t_gen = time.time() - t0
    out_scale = float(torch.sqrt(torch.mean(u_c.double() ** 2)))
    in_scale = 1.0 / float(torch.sqrt(torch.mean(f_c.double() ** 2)))
    net = qn.QnNet(G, modes, blocks, max_batch=batch)
    net.set_params(init_params(32, modes, blocks))
    t0 = time.time()
    losses = train(net, f_c, u_c, in_scale, out_scale, epochs, batch, lr)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    rows = evaluate(ctx, net, n, range(test_seed0, test_seed0 + ntest), scale, in_scale, out_scale)
    summ = summarise(rows)
    summ["precision"] = precision
    by = {precision: summarise(rows)}
    for p in also:
        c2 = qn.QnContext(3, n, p)
        by[p] = summarise(evaluate(c2, net, n, range(test_seed0, test_seed0 + ntest), scale, in_scale, out_scale))
        c2.close()
    if also:
        summ["by_precision"] = by
    summ.update({"n": n, "G": G, "modes": modes, "blocks": blocks, "params": int(net.nparams),
                 "train_samples": ntrain, "epochs": epochs, "batch": batch, "scale": scale,
                 "train_solve_iterations_mean": statistics.mean(its), "data_gen_s": round(t_gen, 1),
                 "train_s": round(t_train, 1), "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
                 "in_scale": in_scale, "out_scale": out_scale})
    log(json.dumps(summ))
    return summ, net, rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--G", type=int, default=64)
    ap.add_argument("--modes", type=int, default=6)
    ap.add_argument("--blocks", type=int, default=4)
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--precision", default="bf16x3", choices=("bf16x3", "bf16x6"))
    ap.add_argument("--also", nargs="*", default=[], choices=("bf16x3", "bf16x6"))
    a = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    summ, _, rows = run(a.n, a.G, a.modes, a.blocks, a.train, a.test, a.scale, a.epochs, a.batch, a.lr,
                        precision=a.precision, also=tuple(a.also))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump({"summary": summ, "rows": rows}, fh)


if __name__ == "__main__":
    main()
