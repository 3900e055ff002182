"""Learned adaptation indicator: data generation, training and deployment helpers.

The indicator is a per-element MLP (features of `Mesh.features`, 3 hidden layers of 64, GELU,
logits for coarsen / keep / refine) that predicts the density-gradient indicator `horizon` steps
ahead, so that adaptation can run less often.  Every numeric step runs in the library's kernels
(features, forward, backward, Adam); this module only sequences them.

Labels: from a snapshot of a plain run, a copy of the mesh is advanced `horizon` steps without
adaptation and the density-gradient indicator of that future state, on the same leaves, is the
label of each leaf.
"""
from __future__ import annotations

import numpy as np

from . import fr
from . import workloads as W


def init_params(in_dim: int, seed: int) -> np.ndarray:
    """Uniform fan-in scaled initial weights (sqrt(6/fan_in)) and zero biases, from splitmix64."""
    n = fr.mlp_param_count(in_dim)
    r = W.random_uniform(n, seed) * 2.0 - 1.0
    out = np.zeros(n, dtype=np.float32)
    off = 0
    for fan_in, rows in ((in_dim, 64), (64, 64), (64, 64), (64, 3)):
        nw = fan_in * rows
        out[off:off + nw] = r[off:off + nw] * np.sqrt(6.0 / fan_in)
        off += nw + rows  # biases stay zero
    return out


def collect_pairs(cfg: dict, snapshots: int, horizon: int = 20, every: int = 10, warmup: int = 0):
    """Feature/label pairs from a plain run of `cfg` (density-gradient indicator).

    Returns (X, y): CUDA tensors, BF16 [n][in] and int8 [n] in {-1, 0, 1}.
    """
    import torch
    base = dict(cfg, indicator=0)
    run = fr.Mesh(base)
    probe = fr.Mesh(dict(base, init_passes=0))
    for _ in range(warmup):
        run.step(every)
        run.adapt()
    Xs, ys = [], []
    for _ in range(snapshots):
        run.step(every)
        run.adapt()
        Xs.append(run.features())
        probe.set_state(run.leaves(), run.state())
        probe.set_time(run.info()["t"])
        probe.step(horizon)
        f, _ = probe.flags()
        ys.append(torch.from_numpy(f).cuda())
    run.close()
    probe.close()
    return torch.cat(Xs), torch.cat(ys)


def class_weights(y) -> np.ndarray:
    """Inverse-frequency class weights (coarsen, keep, refine), normalised to mean 1."""
    yy = y.cpu().numpy().astype(np.int64) + 1
    cnt = np.bincount(yy, minlength=3).astype(np.float64)
    w = np.where(cnt > 0, cnt.sum() / (3.0 * np.maximum(cnt, 1.0)), 0.0)
    return w


def train(X, y, epochs: int = 5, batch: int = 4096, lr: float = 2e-3, seed: int = 7,
          class_w=None, log=None):
    """Adam on the weighted cross-entropy; returns FP32 parameters (numpy) and the loss history."""
    import torch
    n, in_dim = X.shape
    params = torch.from_numpy(init_params(in_dim, seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    cw = class_weights(y) if class_w is None else np.asarray(class_w, dtype=np.float64)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        perm = np.random.default_rng(seed + 1000 * (ep + 1)).permutation(n)  # seeded shuffle
        permt = torch.from_numpy(perm).cuda()
        Xp, yp = X[permt].contiguous(), y[permt].contiguous()
        tot, nb = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            fr.mlp_train_step(params, m, v, step, Xp[b0:b0 + batch], yp[b0:b0 + batch], cw, lr, loss)
            step += 1
            tot += float(loss.item()) if (nb % 50 == 0) else 0.0
            nb += 1
        hist.append(tot / max(1, (nb + 49) // 50))
        if log:
            log("epoch %d: loss %.4f" % (ep, hist[-1]))
    return params.cpu().numpy(), hist


def accuracy(params, X, y):
    """Fraction of samples whose argmax class equals the label, and the confusion matrix."""
    import torch
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    _, flags = fr.mlp_forward(p, X)
    f = flags.cpu().numpy().astype(np.int64) + 1
    t = y.cpu().numpy().astype(np.int64) + 1
    conf = np.zeros((3, 3), dtype=np.int64)
    np.add.at(conf, (t, f), 1)
    return float((f == t).mean()), conf


def deploy_run(cfg: dict, steps: int, every: int, params=None) -> dict:
    """Runs `steps` steps adapting every `every` steps (0: never, the initial mesh throughout);
    wall time of steps and adaptations, the final and the mean leaf count."""
    import time

    import torch
    m = fr.Mesh(cfg)
    if params is not None:
        m.set_learned_indicator(params)
    ts = ta = 0.0
    n_adapt = 0
    chunk = every if every > 0 else 30
    Ms = []
    for _ in range(steps // chunk):
        Ms.append(m.M)
        torch.cuda.synchronize()
        a = time.perf_counter()
        m.step(chunk)
        torch.cuda.synchronize()
        b = time.perf_counter()
        if every > 0:
            m.adapt()
            n_adapt += 1
        torch.cuda.synchronize()
        c = time.perf_counter()
        ts += b - a
        ta += c - b
    nm = m.norms()
    out = dict(l2_rho=nm["l2_rho"], t=nm["t"], M_final=m.M, M_mean=float(np.mean(Ms)), steps_s=ts,
               adapt_s=ta, total_s=ts + ta, adaptations=n_adapt, adaptation_pct=100.0 * ta / (ts + ta))
    m.close()
    torch.cuda.empty_cache()
    return out


def experiment(steps: int = 120, snapshots: int = 30, log=print) -> dict:
    """Train on the 3D p=2 tube (labels: the deployment's plain indicator 20 steps ahead), deploy
    on the four-tube 3D p=3 setup adapting every 30 steps, against the plain indicator every 10."""
    import time

    import torch
    cfg4 = W.config("vortex3d_p3_multi")
    cfg3 = dict(W.config("vortex3d_p2_tube"), precision=4,
                th_refine=cfg4["th_refine"], th_coarsen=cfg4["th_coarsen"])
    t0 = time.perf_counter()
    X, y = collect_pairs(cfg3, snapshots=snapshots, horizon=20, every=10)
    t_collect = time.perf_counter() - t0
    n = X.shape[0]
    ntr = int(0.9 * n)
    t0 = time.perf_counter()
    params, hist = train(X[:ntr], y[:ntr], epochs=6, batch=4096, lr=2e-3, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    acc, conf = accuracy(params, X[ntr:], y[ntr:])
    res = dict(pairs=int(n), collect_s=t_collect, train_s=t_train, loss_history=hist,
               heldout_accuracy=acc, confusion=conf.tolist())
    del X, y
    torch.cuda.empty_cache()
    res["plain_f64_every10"] = deploy_run(dict(cfg4, precision=0, indicator=0), steps, 10)
    res["learned_f64_every30"] = deploy_run(dict(cfg4, precision=0, indicator=3), steps, 30, params)
    res["learned_double_word_every30"] = deploy_run(dict(cfg4, precision=4, indicator=3), steps, 30,
                                                    params)
    return res


def experiment_long(steps: int = 990, snapshots: int = 30, log=print) -> dict:
    """The same training as `experiment`; deployment on the four 3D p=3 tubes for `steps` steps
    (a multiple of 10 and 30, so every arm ends at the same time; each vortex moves about 20
    finest cells) in four arms -- plain indicator every 10 and every
    30 steps, learned indicator every 30, no adaptation -- in FP64 and in the double-word form."""
    import time

    import torch
    cfg4 = W.config("vortex3d_p3_multi")
    cfg3 = dict(W.config("vortex3d_p2_tube"), precision=4,
                th_refine=cfg4["th_refine"], th_coarsen=cfg4["th_coarsen"])
    t0 = time.perf_counter()
    X, y = collect_pairs(cfg3, snapshots=snapshots, horizon=20, every=10)
    t_collect = time.perf_counter() - t0
    n = X.shape[0]
    ntr = int(0.9 * n)
    t0 = time.perf_counter()
    params, hist = train(X[:ntr], y[:ntr], epochs=6, batch=4096, lr=2e-3, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    acc, conf = accuracy(params, X[ntr:], y[ntr:])
    res = dict(steps=steps, pairs=int(n), collect_s=t_collect, train_s=t_train, loss_history=hist,
               heldout_accuracy=acc, confusion=conf.tolist())
    del X, y
    torch.cuda.empty_cache()
    for prec, pname in ((0, "f64"), (4, "double_word")):
        arms = (("plain_every10", 0, 10), ("plain_every30", 0, 30), ("learned_every30", 3, 30),
                ("no_adaptation", 0, 0))
        for arm, ind, every in arms:
            key = "%s_%s" % (arm, pname)
            res[key] = deploy_run(dict(cfg4, precision=prec, indicator=ind), steps, every,
                                  params if ind == 3 else None)
            log("%s: %s" % (key, res[key]))
    return res


def bench_forward(n: int = 2_000_000, n_in: int = 55, reps: int = 10, seed: int = 1) -> dict:
    """Times the tensor-core inference (fr_mlp_forward) on n seeded synthetic feature rows: CUDA
    events around each call (which includes its status check and synchronisation)."""
    import torch
    npar = fr.mlp_param_count(n_in)
    P = torch.from_numpy(((W.random_uniform(npar, seed) - 0.5) * 0.5).astype(np.float32)).cuda()
    X = torch.from_numpy(((W.random_uniform(n * n_in, seed + 1) - 0.5) * 6).astype(np.float32))
    X = X.reshape(n, n_in).cuda().to(torch.bfloat16)
    fr.mlp_forward(P, X)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fr.mlp_forward(P, X)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms)) * 1e-3
    macs = n_in * 64 + 2 * 64 * 64 + 64 * 3
    return dict(rows=n, in_dim=n_in, ms=t * 1e3, tflops=2.0 * macs * n / t / 1e12,
                gbs=n * (2 * n_in + 12 + 1) / t / 1e9)


def bench_train(batch: int = 65536, n_in: int = 55, reps: int = 20, seed: int = 1) -> dict:
    """Times one tensor-core training step (fr_mlp_train_step: gradient of a batch and the Adam
    update, including the call's status check) on seeded synthetic features and labels."""
    import torch
    npar = fr.mlp_param_count(n_in)
    P = torch.from_numpy(((W.random_uniform(npar, seed) - 0.5) * 0.5).astype(np.float32)).cuda()
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    X = torch.from_numpy(((W.random_uniform(batch * n_in, seed + 1) - 0.5) * 6).astype(np.float32))
    X = X.reshape(batch, n_in).cuda().to(torch.bfloat16)
    y = torch.from_numpy((np.floor(W.random_uniform(batch, seed + 2) * 3) - 1).astype(np.int8)).cuda()
    cw = [1.5, 0.5, 2.0]
    fr.mlp_train_step(P, m, v, 0, X, y, cw, 1e-3)
    ms = []
    for k in range(1, reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fr.mlp_train_step(P, m, v, k, X, y, cw, 1e-3)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = float(np.median(ms)) * 1e-3
    macs = n_in * 64 + 2 * 64 * 64 + 64 * 3
    # forward, backward-data, weight gradients and the recomputed pre-activations: ~4 passes
    return dict(batch=batch, in_dim=n_in, ms=t * 1e3, samples_per_s=batch / t,
                tflops_4pass=4 * 2.0 * macs * batch / t / 1e12)


if __name__ == "__main__":
    import json
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "--bench-train":
        b = int(sys.argv[2]) if len(sys.argv) > 2 else 65536
        n_in = int(sys.argv[3]) if len(sys.argv) > 3 else 55
        print(json.dumps(bench_train(b, n_in)))
        sys.exit(0)
    if len(sys.argv) > 1 and sys.argv[1] == "--bench-forward":
        n = int(sys.argv[2]) if len(sys.argv) > 2 else 2_000_000
        n_in = int(sys.argv[3]) if len(sys.argv) > 3 else 55
        print(json.dumps(bench_forward(n, n_in)))
        sys.exit(0)
    if len(sys.argv) > 1 and sys.argv[1] == "--long":
        out = experiment_long(int(sys.argv[3]) if len(sys.argv) > 3 else 990)
        print(json.dumps(out))
        if len(sys.argv) > 2:
            with open(sys.argv[2], "w") as fh:
                json.dump(out, fh, indent=1)
        sys.exit(0)
    out = experiment()
    print(json.dumps(out))
    if len(sys.argv) > 1:
        with open(sys.argv[1], "w") as fh:
            json.dump(out, fh, indent=1)
