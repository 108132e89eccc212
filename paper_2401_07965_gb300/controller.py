"""Learned schedule controller: training data from the method's own traces, GPU
training with the library's network kernels, and helpers to run a learned or a
plain schedule on the same grid.

What the network learns.  A plain run on a fine uniform beta grid records, at
every step, the energy fluctuation sigma = sqrt(var E) and the 8 statistics the
controller sees.  The reweighting of Eq. (Q) loses about dbeta^2 var(E) of the
population's effective size per step, so steps of size proportional to
sigma^-p (p = 1: constant energy-histogram overlap, the adaptive-step practice
Sec. 5 cites) balance that loss along the anneal.  In hindsight, on the trace,

    s_i = mean_{j >= i}(sigma_j^p) / sigma_i^p

is the step at beta_i relative to the average remaining step (the quantity the
controller re-plans with), and the sweep weight of a step is w_i, one of

    const: 1    isig: (mean sigma / sigma_i)^(1/2)    isig1: mean sigma / sigma_i
    acc:   (mean a / a_i)^(1/2)   (a: Metropolis acceptance rate)

normalised to mean 1 over the steps the spacing above would take, t_i = w_i /
(sum_j sigma_j^p w_j / sum_j sigma_j^p).  Labels are clipped to s in [0.2, 5],
t in [0.5, 2].  The network maps (beta, <E>/N, var(E)/N, ln Q, rho_t, family
entropy, acceptance, L) to (s, t); traces come from the 2D Ising L=16 and L=64
ferromagnets and 3D +-J spin glasses with L=4, 6, 8, each on several grids
(step sizes) and sweep numbers so that the step-size dependent features (ln Q,
rho_t) are seen over their range.

Run as a module to train: python -m paper_2401_07965_gb300.controller --out FILE
"""
from __future__ import annotations

import os

import numpy as np

from . import pa

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "controller_weights.npz")
NPARAM = pa.PA_MLP_NPARAM
SHAPES = [(64, 8), (64,), (64, 64), (64,), (2, 64), (2,)]

# trace workloads: (dim, L, couplings, R, beta_f); each on grids of 200 and 400
# steps with 5 and 10 sweeps per step
TRACE_SHAPES = [
    (2, 16, ("ferro",), 1000, 1.0),
    (2, 64, ("ferro",), 100000, 1.0),
    (3, 4, ("ea", 3, 0), 50000, 3.0),
    (3, 6, ("ea", 3, 64), 50000, 3.0),
    (3, 8, ("ea", 3, 128), 50000, 3.0),
]
TRACE_GRIDS = ((200, 5), (200, 10), (400, 5), (400, 10))


def bf16_bits(x32):
    b = np.ascontiguousarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for shp in SHAPES:
        if len(shp) == 2:
            parts.append(rng.normal(0, np.sqrt(2.0 / shp[1]), shp).ravel())
        else:
            parts.append(np.zeros(shp))
    flat = np.concatenate(parts).astype(np.float32)
    flat[-2:] = 1.0  # outputs start at the plain schedule (s = t = 1)
    return flat


def controlled_run(dim, L, couplings, R, betas, plain_units, plain_theta, params_bits=None,
                   seed=1, budget=0, theta_min=2, theta_max=40, u_max=8, resampler="systematic",
                   stream=None, sweep_threads=None):
    """A single run on the schedule grid `betas`, driven by the network (params_bits) or,
    with params_bits None, by plain steps of plain_units grid points and plain_theta sweeps."""
    n = len(betas) - 1
    pop = pa.Population(dim, L, R, betas, np.full(n, plain_theta, np.uint32), resampler, seed,
                        couplings=couplings, stream=stream, sweep_threads=sweep_threads)
    pa.pa_set_controller(pop.ctx, params_bits, 0 if params_bits is None else 1, plain_units,
                         plain_theta, theta_min, theta_max, budget, u_max)
    return pop


def run_to_end(pop, chunk=16):
    """Launch steps until the controller reports that beta_f is reached (at most one
    step per grid point, so the loop is bounded)."""
    for _ in range(pop.n_steps // chunk + 2):
        try:
            pop.step(chunk)
        except pa.PAError as e:
            if e.status == pa.PA_ERR_DONE:
                return pop
            raise
        pa.pa_sync(pop.ctx)
    raise RuntimeError("controlled run did not reach the final beta")


def smooth(y, w=7):
    """Moving average with edge padding (window w, odd)."""
    k = np.ones(w) / w
    return np.convolve(np.pad(np.asarray(y, np.float64), (w // 2, w // 2), mode="edge"), k,
                       mode="valid")


def hindsight_labels(sigma, acc, p=1.0, rule="isig"):
    """Targets (s, t) of the rows of one uniform-grid trace (see the module text)."""
    sig = np.maximum(smooth(sigma), 1e-9)
    dens = sig ** p
    n = len(dens)
    rem = np.cumsum(dens[::-1])[::-1] / np.arange(n, 0, -1)
    s = rem / dens
    a = np.maximum(smooth(acc), 1e-6)
    if rule == "const":
        w = np.ones(n)
    elif rule == "isig":
        w = np.sqrt(sig.mean() / sig)
    elif rule == "isig1":
        w = sig.mean() / sig
    elif rule == "acc":
        w = np.sqrt(a.mean() / a)
    else:
        raise ValueError(rule)
    t = w / (np.sum(dens * w) / np.sum(dens))
    return np.clip(s, 0.2, 5.0), np.clip(t, 0.5, 2.0)


def trace_arrays(rows, N):
    sig = np.sqrt(np.maximum([(r["e2"] - r["e"] ** 2) * N * N for r in rows], 0.0))
    acc = np.array([r["accept_rate"] for r in rows])
    if len(acc) > 1:
        acc[0] = acc[1]  # no sweeps before step 0
    X = np.array([r["features"] for r in rows], np.float32)
    return X, sig, acc


def collect(seeds=(1, 2), shapes=TRACE_SHAPES, grids=TRACE_GRIDS, stream=None):
    """Plain fine-grid runs with the controller in plain mode (it records the features).
    Returns a list of (name, X, sigma, acceptance)."""
    out = []
    for dim, L, cpl, R, bf in shapes:
        for n, theta in grids:
            for seed in seeds:
                c = cpl if cpl[0] == "ferro" else (cpl[0], cpl[1], cpl[2] + seed)
                pop = controlled_run(dim, L, c, R, np.linspace(0.0, bf, n + 1), 1, theta, None,
                                     seed=seed, stream=stream)
                run_to_end(pop)
                X, sig, acc = trace_arrays(pop.trace(), L ** dim)
                pop.close()
                out.append((f"d{dim}L{L}n{n}t{theta}s{seed}", X, sig, acc))
    return out


def dataset(traces, p=1.0, rule="isig"):
    Xs, Ys = [], []
    for _, X, sig, acc in traces:
        s, t = hindsight_labels(sig, acc, p, rule)
        Xs.append(X)
        Ys.append(np.stack([s, t], 1).astype(np.float32))
    return np.concatenate(Xs), np.concatenate(Ys)


def train(X, Y, iters=3000, lr=3e-3, seed=0, log_every=0, decay=False):
    """Full-batch Adam on the device with pa_mlp_gradients / pa_mlp_adam (learning
    rate lr, or lr on a cosine decay to lr/20 with decay=True)."""
    import torch
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    B = X.shape[0]
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(Y, np.float32)).to(dev)
    Md = torch.ones_like(Yd)
    w = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    g = torch.zeros_like(w)
    wbf = torch.zeros(NPARAM, dtype=torch.int16, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    scratch = torch.empty(pa.pa_mlp_scratch_bytes(B), dtype=torch.uint8, device=dev)
    history = []
    for it in range(1, iters + 1):
        pa.pa_mlp_gradients(w.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Md.data_ptr(), B,
                            g.data_ptr(), loss.data_ptr(), scratch.data_ptr(), scratch.numel(),
                            stream)
        lr_it = lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * (it - 1) / iters))) if decay else lr
        pa.pa_mlp_adam(w.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), wbf.data_ptr(), it,
                       lr_it, stream)
        if log_every and it % log_every == 0:
            history.append((it, float(loss.item())))
    torch.cuda.synchronize()
    return w.cpu().numpy(), wbf.cpu().numpy().view(np.uint16), history


def predict(bits, X):
    import torch
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    Yd = torch.zeros((X.shape[0], 2), dtype=torch.float32, device=dev)
    Bd = torch.from_numpy(np.ascontiguousarray(bits, np.uint16).view(np.int16)).to(dev)
    pa.pa_mlp_forward(Bd.data_ptr(), Xd.data_ptr(), X.shape[0], Yd.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


def save(bits, path=WEIGHTS, **meta):
    np.savez(path, params_bf16=np.asarray(bits, np.uint16), **meta)


def load(path=WEIGHTS):
    with np.load(path) as z:
        return z["params_bf16"].astype(np.uint16)


def main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="train the schedule controller on the GPU")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--p", type=float, default=1.0)
    ap.add_argument("--rule", default="isig", choices=["const", "isig", "isig1", "acc"])
    ap.add_argument("--iters", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    t0 = time.time()
    traces = collect()
    t1 = time.time()
    X, Y = dataset(traces, a.p, a.rule)
    w, bits, hist = train(X, Y, a.iters, a.lr, a.seed, log_every=max(a.iters // 10, 1),
                          decay=True)
    t2 = time.time()
    pred = predict(bits, X)
    rms = np.sqrt(np.mean((pred - Y) ** 2, 0))
    save(bits, a.out, p=a.p, rule=a.rule, rows=X.shape[0], rms_s=rms[0], rms_t=rms[1])
    print(json.dumps({"rows": int(X.shape[0]), "traces": len(traces), "collect_s": t1 - t0,
                      "train_s": t2 - t1, "loss": hist, "rms_s": float(rms[0]),
                      "rms_t": float(rms[1]), "p": a.p, "rule": a.rule, "out": a.out}))


if __name__ == "__main__":
    main()
