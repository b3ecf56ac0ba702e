"""Training and Monte-Carlo evaluation of the learned false-alarm surrogate.

Orchestration only: the noise, the periodograms, their maxima, the pattern
features, the network and its whole training loop (minibatch draws, learning
rate schedule, Adam, validation loss, choice of the kept weights) all run in
liblsp.so (lsp_batch, lsp_fap_features, lsp_fap_train, lsp_fap_predict); this
module draws sampling patterns (synth.noise_batch) and hands arrays to the C
ABI.  The evaluation compares the library's quantiles with the empirical
quantiles of brute-force Monte Carlo, the yardstick the surrogate is measured against.

  python -m paper_1007_1658_gb300.surrogate [--quick] [--out model.lspfap] [--evaluate-only]

trains on noise periodograms the batched engine generates and evaluates the
trained network against brute-force Monte Carlo on held-out patterns,
printing one JSON report (--evaluate-only: evaluate the model in --out).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import lsp, synth

LEVELS = np.array([0.05, 0.10, 0.25, 0.50, 0.75, 0.90, 0.95, 0.98, 0.99])
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fap_surrogate.lspfap")


class DevicePatterns:
    """A batch of sampling patterns resident on the GPU."""

    def __init__(self, b: synth.Batch, device):
        import torch
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.batch = b
        self.n = b.n
        self.t_off, self.t, self.f0, self.df, self.nf = d(b.t_off), d(b.t), d(b.f0), d(b.df), d(b.nf)
        nt = np.diff(b.t_off).astype(np.float32)
        self.counts = d(np.column_stack([nt, b.nf.astype(np.float32)]))
        self.total = int(b.t_off[-1])


def mc_maxima(ctx: lsp.Context, pats: DevicePatterns, n_real: int, seed: int, max_floats: float = 6e8):
    """Largest noise peak of n_real noise realizations of every pattern:
    a [n_real, n] float32 device tensor, realizations drawn in chunks whose
    noise buffer stays under max_floats values."""
    import torch
    chunk = max(1, min(n_real, int(max_floats // max(1, pats.total))))
    out = torch.empty((n_real, pats.n), dtype=torch.float32, device=pats.t.device)
    arg = torch.empty((chunk, pats.n), dtype=torch.int32, device=pats.t.device)
    r = 0
    while r < n_real:
        k = min(chunk, n_real - r)
        ctx.batch(pats.t_off, pats.t, pats.f0, pats.df, pats.nf, seed=seed + r, n_real=k,
                  maxP=out[r:r + k], argmax=arg[:k])
        r += k
    return out


def train(ctx: lsp.Context, n_patterns=65535, n_real=4, steps=4000, batch=4096, lr=3e-4, lr_final=0.05,
          warmup_steps=100, weight_decay=3.0, hidden=256, seed=2024, n_val=2048, val_real=8, eval_every=100,
          verbose=True):
    """Train the surrogate on n_patterns x n_real noise periodograms through
    lsp_fap_train (the loop, the validation loss and the choice of the kept
    weights all run in the library), validating on n_val patterns x val_real
    realizations.  Each pattern has only n_real noisy targets, so without
    weight decay the network starts to fit the patterns' own noise after about
    one epoch; the default decoupled weight decay keeps the training and
    validation losses together to the end of the run."""
    import torch
    dev = torch.device("cuda", ctx.device)
    t0 = time.perf_counter()
    b = synth.noise_batch(n_curves=n_patterns, seed=seed)
    vb = synth.noise_batch(n_curves=n_val, seed=seed + 1)
    pats = DevicePatterns(b, dev)
    vpats = DevicePatterns(vb, dev)
    t_gen = time.perf_counter() - t0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    targets = mc_maxima(ctx, pats, n_real, seed=seed * 7919 + 1).reshape(-1).contiguous()
    ev[1].record()
    vtargets = mc_maxima(ctx, vpats, val_real, seed=seed * 7919 + 2).contiguous()
    feats = ctx.fap_features(pats.t_off, pats.t, pats.f0, pats.df, pats.nf)
    vfeats = ctx.fap_features(vpats.t_off, vpats.t, vpats.f0, vpats.df, vpats.nf)
    ctx.fap_init(feats, hidden=hidden, seed=seed)
    rep = ctx.fap_train(feats, pats.counts, targets, vfeats, vpats.counts, vtargets, steps=steps, batch=batch, lr=lr,
                        lr_final=lr_final, warmup_steps=warmup_steps, weight_decay=weight_decay,
                        eval_every=eval_every, seed=seed)
    torch.cuda.synchronize(dev)
    if verbose:
        hist = zip(rep["val_history"], rep["train_history"])
        for e, (v, tl) in enumerate(hist):
            print("pass %3d  train %.4f  val %.4f" % (e, tl, v), flush=True)
    steps_at = [0] + [min(steps, (e + 1) * eval_every) for e in range(rep["evaluations"] - 1)] if eval_every else [0, steps]
    return {"patterns": n_patterns, "realizations": n_real, "periodograms": n_patterns * n_real,
            "terms": int(b.terms) * n_real, "steps": steps, "batch": batch, "lr": lr, "lr_final": lr_final,
            "warmup_steps": warmup_steps, "weight_decay": weight_decay, "val_patterns": n_val,
            "val_realizations": val_real, "gpu_s_data": ev[0].elapsed_time(ev[1]) / 1e3,
            "gpu_s_train": rep["gpu_ms"] / 1e3, "cpu_s_patterns": t_gen, "val_loss_eq3": rep["val_loss_initial"],
            "val_loss_best": rep["val_loss_best"], "best_step": rep["best_step"],
            "train_loss_last": rep["train_loss_last"],
            "val_history": [(s_, round(v, 5)) for s_, v in zip(steps_at, rep["val_history"])],
            "train_history": [(s_, round(v, 5)) for s_, v in zip(steps_at, rep["train_history"])]}


def hidden_of(ctx: lsp.Context) -> int:
    """Hidden width of the context's network, from its parameter count."""
    n = ctx.fap_get_params().size - 64
    # 32H + H + 2(H^2 + H) + 9H + 9 = 2H^2 + 44H + 9
    return int(round((-44 + np.sqrt(44 * 44 - 8 * (9 - n))) / 4))


def evaluate(ctx: lsp.Context, n_patterns=256, n_real=10000, seed=777001):
    """Held-out patterns: surrogate quantiles and Eq. 3's against brute-force
    Monte Carlo with n_real noise realizations each; GPU seconds of both."""
    import torch
    dev = torch.device("cuda", ctx.device)
    b = synth.noise_batch(n_curves=n_patterns, seed=seed)
    pats = DevicePatterns(b, dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ctx.fap_predict(pats.t_off, pats.t, pats.f0, pats.df, pats.nf)  # warm-up
    torch.cuda.synchronize(dev)
    ev[0].record()
    q_sur = ctx.fap_predict(pats.t_off, pats.t, pats.f0, pats.df, pats.nf)
    ev[1].record()
    maxP = mc_maxima(ctx, pats, n_real, seed=seed * 31 + 5)
    ev[2].record()
    torch.cuda.synchronize(dev)
    q_sur = q_sur.cpu().numpy().astype(np.float64)
    # the same weights evaluated with FP32 activations
    ctx32 = lsp.Context(ctx.device, mlp_fp32=1)
    ctx32.fap_set_params(ctx.fap_get_params(), hidden=hidden_of(ctx))
    q32 = ctx32.fap_predict(pats.t_off, pats.t, pats.f0, pats.df, pats.nf).cpu().numpy().astype(np.float64)
    # Eq. 3's quantiles from the library's own head: a freshly initialized
    # network has a zero output layer, and z = 0 is Eq. 3 exactly
    feats = ctx32.fap_features(pats.t_off, pats.t, pats.f0, pats.df, pats.nf)
    ctx32.fap_init(feats, hidden=4, seed=1)
    q_eq3 = ctx32.fap_predict(pats.t_off, pats.t, pats.f0, pats.df, pats.nf).cpu().numpy().astype(np.float64)
    ctx32.close()
    m = np.sort(maxP.cpu().numpy().astype(np.float64), axis=0)
    idx = np.minimum(n_real - 1, np.ceil(LEVELS * n_real).astype(int) - 1)   # empirical quantiles
    q_mc = m[idx, :].T
    rel_sur = np.abs(q_sur - q_mc) / q_mc
    rel_32 = np.abs(q32 - q_mc) / q_mc
    rel_eq3 = np.abs(q_eq3 - q_mc) / q_mc
    t_sur = ev[0].elapsed_time(ev[1]) / 1e3
    t_mc = ev[1].elapsed_time(ev[2]) / 1e3
    return {"patterns": n_patterns, "realizations": n_real, "levels": LEVELS.tolist(),
            "mean_rel_err_surrogate": rel_sur.mean(axis=0).tolist(),
            "p95_rel_err_surrogate": np.percentile(rel_sur, 95, axis=0).tolist(),
            "mean_rel_err_surrogate_fp32_activations": rel_32.mean(axis=0).tolist(),
            "mean_rel_err_eq3": rel_eq3.mean(axis=0).tolist(),
            "max_level_mean_rel_err_surrogate": float(rel_sur.mean(axis=0).max()),
            "max_level_mean_rel_err_eq3": float(rel_eq3.mean(axis=0).max()),
            "gpu_s_surrogate": t_sur, "gpu_s_mc": t_mc, "gpu_s_ratio": t_mc / max(t_sur, 1e-9),
            "mc_terms": int(b.terms) * n_real}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="small run (minutes -> seconds)")
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--evaluate-only", action="store_true",
                    help="evaluate the model in --out against Monte Carlo, no training")
    args = ap.parse_args()
    ctx = lsp.Context(0)
    if args.evaluate_only:
        ctx.fap_load(args.out)
        print(json.dumps({"evaluation": evaluate(ctx), "model": os.path.basename(args.out)}), flush=True)
        return
    if args.quick:
        tr = train(ctx, n_patterns=4096, n_real=4, steps=args.steps or 400, batch=2048, lr=1e-3, n_val=512,
                   eval_every=100)
        jd = evaluate(ctx, n_patterns=64, n_real=2000)
    else:
        tr = train(ctx, steps=args.steps or 4000)
        jd = evaluate(ctx)
    ctx.fap_save(args.out)
    print(json.dumps({"train": tr, "evaluation": jd, "model": os.path.basename(args.out)}), flush=True)


if __name__ == "__main__":
    main()
