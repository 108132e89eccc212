"""The learned schedule controller's network and decision rule, written plainly
(test infrastructure only).

Network: x (8) -> relu(W1 x + b1) (64) -> relu(W2 h1 + b2) (64) -> W3 h2 + b3 (2),
parameters in the order W1[64][8], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]
(4866 values), rounded to BF16 (round to nearest even) for inference.

* forward64 / grads64: FP64 forward and backward of the masked mean squared
  error sum mask (y - yt)^2 / (2B), the reference for the GPU gradients.
* forward32: the FP32 evaluation in the device's order (products summed in
  index order starting from 0, bias added last, no fused multiply-add).
* decide: the controller's choice of the next step from the outputs.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 8, 64, 2
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n]).reshape(shp)
        o += n
    return out


def bf16_bits(x32):
    """float32 -> BF16 bit patterns, round to nearest even."""
    b = np.ascontiguousarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def bf16_to_f32(bits):
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def bf16_round(x32):
    return bf16_to_f32(bf16_bits(x32))


def forward64(flat, X):
    p = unpack(np.asarray(flat, np.float64))
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    return h2 @ p["W3"].T + p["b3"], (z1, h1, z2, h2)


def grads64(flat, X, Yt, mask):
    """d/dparams of sum mask (y - yt)^2 / (B * OUT), in the flat layout."""
    X = np.asarray(X, np.float64)
    B = X.shape[0]
    p = unpack(np.asarray(flat, np.float64))
    Y, (z1, h1, z2, h2) = forward64(flat, X)
    d = 2.0 * mask * (Y - Yt) / (B * OUT)
    loss = float((mask * (Y - Yt) ** 2).sum() / (B * OUT))
    gW3 = d.T @ h2
    gb3 = d.sum(0)
    dh2 = (d @ p["W3"]) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)]), loss


def forward32(bits, x):
    """One feature vector through the BF16 network in the device's FP32 order."""
    p = unpack(bf16_to_f32(bits))
    x = np.asarray(x, np.float32)
    f = np.float32
    h1 = np.zeros(HID, np.float32)
    for t in range(HID):
        acc = f(0.0)
        for k in range(IN):
            acc = f(acc + f(p["W1"][t, k] * x[k]))
        acc = f(acc + p["b1"][t])
        h1[t] = acc if acc > 0 else f(0.0)
    h2 = np.zeros(HID, np.float32)
    for t in range(HID):
        acc = f(0.0)
        for k in range(HID):
            acc = f(acc + f(p["W2"][t, k] * h1[k]))
        acc = f(acc + p["b2"][t])
        h2[t] = acc if acc > 0 else f(0.0)
    out = np.zeros(OUT, np.float32)
    for t in range(OUT):
        acc = f(0.0)
        for k in range(HID):
            acc = f(acc + f(p["W3"][t, k] * h2[k]))
        out[t] = f(acc + p["b3"][t])
    return out


def decide(out, k, used, cfg):
    """Next step (grid points u, sweeps theta) from the network outputs, the grid
    index k and the sweeps used so far.  cfg: K, use_mlp, plain_units, plain_theta,
    theta_min, theta_max, budget, u_max, theta_c (float32)."""
    f = np.float32
    D = cfg["K"] - k
    if D <= 0:
        return None
    Brem = max(cfg["budget"] - used, 0)
    s, t = f(out[0]), f(out[1])
    ok = (cfg["use_mlp"] and np.isfinite(s) and np.isfinite(t) and f(0.05) <= s <= f(20.0)
          and f(0.05) <= t <= f(20.0))
    if ok:
        nrem = f(f(Brem) / f(cfg["theta_c"]))
        ubar = f(f(D) / max(nrem, f(1.0)))
        uf = np.rint(f(s * ubar))
        u = int(min(max(uf, f(1.0)), f(cfg["u_max"])))
        tf = np.rint(f(t * f(cfg["theta_c"])))
        th = int(min(max(tf, f(cfg["theta_min"])), f(cfg["theta_max"])))
    else:
        u, th = cfg["plain_units"], cfg["plain_theta"]
    u = min(u, D)
    if ok:
        need = (D - u + cfg["u_max"] - 1) // cfg["u_max"]
        cap = Brem - cfg["theta_min"] * need
        if th > cap:
            th = cap if cap > cfg["theta_min"] else cfg["theta_min"]
    return u, th
