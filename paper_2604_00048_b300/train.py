"""Training and evaluation of the lambda network (the learned-lambda smoother).

Training step (all arithmetic in the library's kernels; this module only sequences calls):
    lambda, log lambda = g_theta(x, w)                          ws_tcn_forward (training)
    z = (W + D^T Lambda D)^{-1} W x                             ws_smooth_batch
    L = mean_t,s (z - clean)^2, dL/dz, dL/dlog lambda          ws_solve_adjoint_mse (the loss
                                                                fused into the adjoint, Eqs. 4-5)
    dL/dtheta                                                   ws_tcn_backward
    theta <- Adam(theta, dL/dtheta)                             ws_adam_step, ws_tcn_pack
The clean signal is known because the series are synthetic (the paper trains on masked
hold-out observations of real data; with a generator the clean curve is the better target).

Checkpoints: a flat little-endian file, header "WSTCN001", then int64 step count, int64
batches drawn, float64 log lambda range, and the FP32 master weights, Adam m and v.

    python -m paper_2604_00048_b300.train --series 2097152 --batch 4096 --epochs 1 --out tcn.ckpt
"""
from __future__ import annotations

import argparse
import math
import struct
import sys
import time

import numpy as np
import torch

from . import synth, ws

MAGIC = b"WSTCN001"


def save_checkpoint(path: str, net: "ws.Tcn", batches: int) -> None:
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<qqdd", net.step_count, batches, net.log_lam[0], net.log_lam[1]))
        for t in (net.theta, net.m, net.v):
            f.write(t.detach().cpu().numpy().astype("<f4").tobytes())


def load_checkpoint(path: str, device="cuda"):
    """Returns (net, batches drawn)."""
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a lambda-network checkpoint")
        step, batches, lmin, lmax = struct.unpack("<qqdd", f.read(32))
        n = ws.TCN_PARAMS
        arrs = [np.frombuffer(f.read(4 * n), dtype="<f4") for _ in range(3)]
    net = ws.Tcn(torch.from_numpy(arrs[0].copy()).to(device), (lmin, lmax))
    net.m.copy_(torch.from_numpy(arrs[1].copy()))
    net.v.copy_(torch.from_numpy(arrs[2].copy()))
    net.step_count = step
    return net, batches


def batch(rc: synth.Recipe, first: int, n: int, device="cuda"):
    out = synth.generate_tile(rc, n, series0=first, device=device, want_clean=True)
    return out["x"], out["w"], out["clean"][:, 0, :].contiguous()


def train_step(net: "ws.Tcn", x, w, clean, lr: float, d: int = 2):
    """One Adam step on one batch; returns the batch loss (mean squared error to clean, as
    a one-element tensor). The loss and its gradient are formed inside the adjoint's sweeps
    (ws_solve_adjoint_mse): dL/dz is never written to memory."""
    lam, _ = net.forward(x[:, 0, :], w, training=True, want_loglam=False)
    z, _ = ws.smooth(x, w, lam, d)
    _, glam, loss, _ = ws.smooth_adjoint_mse(w, lam, z, clean[:, None, :], d, scale=2.0 / clean.numel(),
                                             want_gx=False, log_lambda=True)
    net.backward(glam)
    net.step(lr)
    return loss.sum().reshape(1)


def learned_smooth(net: "ws.Tcn", x, w, d: int = 2, refine: bool = False):
    lam, _ = net.forward(x[:, 0, :], w, want_loglam=False)
    z, st = ws.smooth(x, w, lam, d, refine=refine)
    return z, lam, st


def rmse(z, clean) -> float:
    return float(torch.sqrt(torch.mean((z[:, 0, :].double() - clean.double()) ** 2)).item())


def train(series: int, batch_size: int, epochs: float, lr: float, seed: int = 0, net=None, batches_done: int = 0,
          time_limit: float = math.inf, log_every: int = 50, ckpt: str | None = None, device="cuda"):
    rc = synth.RECIPES["learned"]
    net = net or ws.Tcn(ws.tcn_init(seed, device=device))
    n_batches = int(math.ceil(epochs * series / batch_size))
    per_epoch = max(1, series // batch_size)
    t0 = time.time()
    hist = []
    b = batches_done
    while b < n_batches and time.time() - t0 < time_limit:
        first = (b % per_epoch) * batch_size
        x, w, clean = batch(rc, first, batch_size, device)
        # cosine decay to 10% of lr over the run
        lr_b = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * b / max(1, n_batches))))
        loss = train_step(net, x, w, clean, lr_b)
        b += 1
        if b % log_every == 0 or b == n_batches:
            hist.append((b, float(loss.item())))
            print(f"batch {b}/{n_batches} loss {hist[-1][1]:.3e} ({time.time() - t0:.0f} s)", file=sys.stderr,
                  flush=True)
            if ckpt:
                save_checkpoint(ckpt, net, b)
    return net, b, hist


def evaluate(net: "ws.Tcn", n: int = 262144, T: int = 730, seed_shift: int = 1000, device="cuda", chunk: int = 65536):
    """RMSE to the clean signal of the learned-lambda smoother and of the GCV-grid smoother
    on n new series (same generator, another seed)."""
    base = synth.RECIPES["learned"]
    rc = synth.Recipe(**{**base.__dict__, "seed": base.seed + seed_shift, "T": T})
    se_l = se_g = 0.0
    cnt = 0
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        out = synth.generate_tile(rc, m, series0=s0, device=device, want_clean=True)
        x, w, clean = out["x"], out["w"], out["clean"][:, 0, :]
        zl, _, _ = learned_smooth(net, x, w, refine=True)
        zg, _, _, _ = ws.gcv_smooth(x, w, None, 2, refine=True, want_scores=False)
        se_l += float(torch.sum((zl[:, 0, :].double() - clean.double()) ** 2).item())
        se_g += float(torch.sum((zg[:, 0, :].double() - clean.double()) ** 2).item())
        cnt += clean.numel()
    return math.sqrt(se_l / cnt), math.sqrt(se_g / cnt)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--series", type=int, default=2097152)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--epochs", type=float, default=1.0)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--time-limit", type=float, default=math.inf)
    ap.add_argument("--out", default="tcn.ckpt")
    ap.add_argument("--resume", default=None)
    ap.add_argument("--eval", type=int, default=65536)
    args = ap.parse_args()
    net, done = (load_checkpoint(args.resume) if args.resume else (None, 0))
    net, b, hist = train(args.series, args.batch, args.epochs, args.lr, args.seed, net, done, args.time_limit,
                         ckpt=args.out)
    save_checkpoint(args.out, net, b)
    if args.eval:
        rl, rg = evaluate(net, n=args.eval)
        print(f"eval on {args.eval} new series: RMSE learned {rl:.5f}  GCV {rg:.5f}", flush=True)


if __name__ == "__main__":
    main()
