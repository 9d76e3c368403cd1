"""Learned troubled-cell indicator: data from the criterion, training, evaluation.

Orchestration only: every step runs in libdolinc's kernels (stage, criterion,
features, network forward/backward/Adam).  The criterion labels the cells of
seeded four-quadrant Riemann runs in which it also drives the limiter of flagged
faces; the network is trained on (features, labels) sampled along those runs and
then replaces the criterion as the limiter's switch, the criterion measuring its
misclassification rate.

The limiter of flagged faces is either ENO3-DOLINC (Sec 2.4) or the first-order
fallback (each side's own cell average).  On these Riemann problems ENO3-DOLINC
alone does not keep the runs bounded: its far values are inverted from the cell's
Gauss differentials, which carry the jump at the cell's other faces, so a flagged
cell's face values can all exceed its average and drain it; the fallback is the
default here.
"""
import numpy as np

from . import (MLP, Mesh, Scheme, dolinc_criterion, dolinc_indicator_features, dolinc_indicator_infer, dolinc_rk_step,
               dolinc_set_flags, dolinc_sync_status, workspace)


def riemann_runs(make_workload, seeds, steps, sample_every, precision="fp32", kappa=4.0, eps=1e-3,
                 limiter="first_order_flagged"):
    """Yields (x24 [n,24] float32 cuda, labels [n] uint8 cuda) samples along criterion-
    limited runs of the given seeds.  make_workload(seed) -> synth workload dict."""
    import torch
    for seed in seeds:
        w = make_workload(seed)
        M = Mesh(w["mesh"])
        sch = Scheme(precision=precision, limiter=limiter, **w["scheme"])
        flags = torch.zeros(M.n_cells, dtype=torch.uint8, device="cuda")
        dolinc_set_flags(M, flags)
        ws = workspace(M, sch)
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        x = torch.zeros((M.n_cells, 24), dtype=torch.float32, device="cuda")
        for step in range(steps):
            dolinc_criterion(M, sch, u, flags, ws, kappa, eps)
            if step % sample_every == 0:
                dolinc_indicator_features(M, sch, u, x, ws)
                yield x.clone(), flags.clone()
            dolinc_rk_step(M, sch, w["dt"], u, ws)
        dolinc_sync_status(M, ws)
        dolinc_set_flags(M, None)


def train(net, X, Y, epochs=20, batch=8192, lr=2e-3, pos_weight=None, seed=0):
    """Adam on shuffled minibatches; returns the per-epoch mean losses."""
    import torch
    n = X.shape[0]
    if pos_weight is None:
        pos = float(Y.float().mean().item())
        pos_weight = min(20.0, (1.0 - pos) / max(pos, 1e-6))
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        Xs, Ys = X[perm].contiguous(), Y[perm].contiguous()
        tot, nb = 0.0, 0
        for b in range(0, n - batch + 1, batch):
            net.train_step(Xs[b:b + batch], Ys[b:b + batch], lr, pos_weight, loss)
            tot += loss.item()
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist, pos_weight


def confusion(pred, label):
    pred, label = np.asarray(pred).astype(bool), np.asarray(label).astype(bool)
    tp = int((pred & label).sum())
    fp = int((pred & ~label).sum())
    fn = int((~pred & label).sum())
    tn = int((~pred & ~label).sum())
    n = max(tp + fp + fn + tn, 1)
    return dict(accuracy=(tp + tn) / n, misclassified=(fp + fn) / n, recall=tp / max(tp + fn, 1),
                precision=tp / max(tp + fp, 1), flagged=(tp + fp) / n, troubled=(tp + fn) / n)


def run_with(w, switch, steps, precision="fp32", net=None, kappa=4.0, eps=1e-3, flagged_limiter="first_order_flagged"):
    """Advance one workload with the limiter driven by `switch`: 'none' (fixed stencil),
    'criterion', 'network' or 'all' (ENO3 everywhere); flagged faces take
    `flagged_limiter`.  Returns (state in caller order, finite flag, seconds per step of
    indicator + stage, flagged fraction)."""
    import torch
    M = Mesh(w["mesh"])
    limiter = {"none": "none", "all": "eno3_all"}.get(switch, flagged_limiter)
    flagged = limiter in ("eno3_flagged", "first_order_flagged")
    sch = Scheme(precision=precision, limiter=limiter, **w["scheme"])
    flags = torch.zeros(M.n_cells, dtype=torch.uint8, device="cuda")
    if flagged:
        dolinc_set_flags(M, flags)
    ws = workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    frac = 0.0
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        if switch == "criterion":
            dolinc_criterion(M, sch, u, flags, ws, kappa, eps)
        elif switch == "network":
            dolinc_indicator_infer(M, sch, net, u, None, flags, ws)     # inputs gathered inside the network kernel
        dolinc_rk_step(M, sch, w["dt"], u, ws)
    e1.record()
    torch.cuda.synchronize()
    if flagged:
        frac = float(flags.float().mean().item())
    finite = True
    try:
        dolinc_sync_status(M, ws)
    except Exception:
        finite = False
    st = M.from_lib(u.cpu().numpy())
    finite = finite and bool(np.all(np.isfinite(st)))
    if flagged:
        dolinc_set_flags(M, None)
    return st, finite, e0.elapsed_time(e1) / 1e3 / steps, frac


__all__ = ["riemann_runs", "train", "confusion", "run_with", "MLP"]
