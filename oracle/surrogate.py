"""CPU oracle of the learned surrogate kernel (FP64, BF16 storage emulated) -- TEST INFRASTRUCTURE ONLY.

The paper has no learned part: the surrogate is a network that predicts a source's spreading kernel (the
column of p, Sec. 3.1) from its local diffusivity patch, with the explicit FD march as the fallback when
the prediction fails a mass/positivity gate.  Definition followed here (and by the CUDA path):

* features of source s: a 17^3 patch centred on s (offsets o = -8..8 per axis), 16 channels, of which
  seven are used:
  ch0 = clamp(log10(D)/8 + 1, -0.5, 1.5) in the domain (D = 0 -> -0.5), 0 outside;
  ch1 = 1 in the domain, 0 outside;  ch2 = 1 at the source cell, 0 elsewhere;
  ch3, ch4, ch5 = o_x / 8, o_y / 8, o_z / 8 and ch6 = |o|^2 / 256 on every voxel of the patch (the
  network is translation-equivariant with a 9^3 receptive field, so without these a voxel more than 4
  cells from the source could not tell where the source is; all four are exact in BF16).
* 4 layers z_l = conv3d_same(a_{l-1}, W_l) + b_l, 3^3 taps, 16 -> 16 channels, zero padding;
  a_l = relu(z_l) for l = 1..3, stored in BF16 (the GPU keeps activations in BF16); the features and
  the weights are BF16 too; sums are exact here (FP64) and FP32 on the GPU.
* head: y = exp(z_4[channel 0]) on in-domain cells, 0 outside; mass m = sum y (FP64).
* gate: accept when |m - 1| <= 1e-3 (y >= 0 holds by construction); the stored kernel is then y / m.
* training loss per sample: the generalised Kullback-Leibler divergence of the prediction from the FD
  kernel k over in-domain cells, sum_v (y_v - k_v z_v + k_v ln k_v - k_v) with y = exp(z), z = z_4
  channel 0 (0 ln 0 = 0).  It is >= 0 with equality at y = k, and its gradient with respect to z is y - k:
  mass predicted where the kernel has none is penalised directly, which is what the mass gate checks.
  The gradient flows back through the relu layers (hand-derived below).

Pins (tests/test_surrogate_oracle.py): conv3d against scipy.ndimage.correlate; every weight and bias
gradient of the hand-derived backward against float64 autograd through torch's conv3d (1e-12 relative on
every entry, interior and edge patches); the BF16-emulating forward against the same chain in torch with
torch's BF16 cast at the same points; central finite differences off the relu kinks; BF16 rounding
against torch's bfloat16 cast.
"""
from __future__ import annotations

import numpy as np

P = 17            # patch side
HALF = 8          # patch radius
C = 16            # channels of every layer
LAYERS = 4
GATE_TOL = 1e-3


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64.  Goes through float32, as
    the GPU rounds FP32 values."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(D, shape, s) -> np.ndarray:
    """[16, 17, 17, 17] feature patch (channel, z, y, x) of source s, BF16-rounded."""
    nx, ny, nz = shape
    Dv = np.asarray(D, dtype=np.float64).reshape(nz, ny, nx)
    sx, sy, sz = s % nx, (s // nx) % ny, s // (nx * ny)
    f = np.zeros((C, P, P, P))
    for k in range(P):
        z = sz - HALF + k
        if not 0 <= z < nz:
            continue
        for j in range(P):
            y = sy - HALF + j
            if not 0 <= y < ny:
                continue
            for i in range(P):
                x = sx - HALF + i
                if not 0 <= x < nx:
                    continue
                d = Dv[z, y, x]
                f[0, k, j, i] = min(max(np.log10(d) / 8.0 + 1.0, -0.5), 1.5) if d > 0 else -0.5
                f[1, k, j, i] = 1.0
    f[2, HALF, HALF, HALF] = 1.0
    o = np.arange(P) - HALF
    f[3] = (o / 8.0)[None, None, :]
    f[4] = (o / 8.0)[None, :, None]
    f[5] = (o / 8.0)[:, None, None]
    f[6] = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2) / 256.0
    return bf16_round(f)


def conv3d_same(a, W, b):
    """z[co, v] = b[co] + sum_{tap, ci} a[ci, v + tap] W[tap, co, ci], taps (dz, dy, dx) in [-1,1]^3 with
    tap index (dx+1) + 3(dy+1) + 9(dz+1); zero padding.  a: [C, P, P, P], W: [27, C, C], b: [C]."""
    ap = np.zeros((a.shape[0], P + 2, P + 2, P + 2))
    ap[:, 1:-1, 1:-1, 1:-1] = a
    z = np.zeros((W.shape[1], P, P, P)) + np.asarray(b)[:, None, None, None]
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                sl = ap[:, 1 + dz:1 + dz + P, 1 + dy:1 + dy + P, 1 + dx:1 + dx + P]
                z += np.einsum("oc,czyx->ozyx", W[t], sl)
    return z


def conv3d_same_grad_input(g, W):
    """d(sum g*z)/da for z = conv3d_same(a, W, b): a correlation of g with the flipped, transposed taps."""
    gp = np.zeros((g.shape[0], P + 2, P + 2, P + 2))
    gp[:, 1:-1, 1:-1, 1:-1] = g
    out = np.zeros((W.shape[2], P, P, P))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                sl = gp[:, 1 - dz:1 - dz + P, 1 - dy:1 - dy + P, 1 - dx:1 - dx + P]
                out += np.einsum("oc,ozyx->czyx", W[t], sl)
    return out


def conv3d_same_grad_weight(a, g):
    """dW[tap, co, ci] = sum_v a[ci, v + tap] g[co, v]."""
    ap = np.zeros((a.shape[0], P + 2, P + 2, P + 2))
    ap[:, 1:-1, 1:-1, 1:-1] = a
    dW = np.zeros((27, g.shape[0], a.shape[0]))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                sl = ap[:, 1 + dz:1 + dz + P, 1 + dy:1 + dy + P, 1 + dx:1 + dx + P]
                dW[t] = np.einsum("czyx,ozyx->oc", sl, g)
    return dW


def forward(feat, Ws, bs, emulate_bf16=True):
    """Returns (y, m, cache): y [P,P,P] head output, m its FP64 mass, cache for backward."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = rnd(feat)
    acts, zs = [a], []
    for l in range(LAYERS):
        z = conv3d_same(a, rnd(Ws[l]), bs[l])
        zs.append(z)
        if l + 1 < LAYERS:
            a = rnd(np.maximum(z, 0.0))
            acts.append(a)
    mask = feat[1] > 0.5
    y = np.where(mask, np.exp(zs[-1][0]), 0.0)
    return y, float(y.sum()), (acts, zs, mask)


def backward(Ws, cache, dz, emulate_bf16=True):
    """Gradients (dWs, dbs) of sum(dz * z_4[0]) through the convolutions and the relus."""
    rnd = bf16_round if emulate_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts, zs, mask = cache
    g = np.zeros((C, P, P, P))
    g[0] = np.where(mask, dz, 0.0)
    dWs, dbs = [None] * LAYERS, [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        dWs[l] = conv3d_same_grad_weight(acts[l], g)
        dbs[l] = g.sum(axis=(1, 2, 3))
        if l > 0:
            ga = conv3d_same_grad_input(g, rnd(Ws[l]))
            g = ga * (zs[l - 1] > 0.0)
    return dWs, dbs


EPS = 1e-9


def loss_grad(cache, k):
    """Loss sum_v (y - k z + k ln k - k) over in-domain cells, y = exp(z), and its gradient y - k with
    respect to z (0 outside the domain)."""
    _, zs, mask = cache
    kk = np.asarray(k, dtype=np.float64)
    z = zs[-1][0]
    y = np.exp(z)
    klnk = np.where(kk > 0.0, kk * np.log(np.where(kk > 0.0, kk, 1.0)), 0.0)
    return float(np.where(mask, y - kk * z + klnk - kk, 0.0).sum()), np.where(mask, y - kk, 0.0)


def gate(m: float) -> bool:
    return abs(m - 1.0) <= GATE_TOL


def init_params(seed: int, noise: float = 0.02):
    """Delta-kernel prior plus small noise: channel 0 carries the source marker through the relu layers
    (centre taps 1) and layer 4 maps it to z = ln(eps) + |ln eps| * a0, i.e. z = 0 at the source and ln(eps)
    elsewhere; all other weights start N(0, noise); layer 4 keeps only output channel 0."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    L = -np.log(EPS)
    for l in range(LAYERS):
        W = rng.normal(0.0, noise, size=(27, C, C))
        b = np.zeros(C)
        if l == 0:
            W[13, 0, :] = 0.0
            W[13, 0, 2] = 1.0
        elif l < LAYERS - 1:
            W[13, 0, :] = 0.0
            W[13, 0, 0] = 1.0
        else:
            W[:, 1:, :] = 0.0
            W[13, 0, 0] = L
            b[0] = -L
        Ws.append(bf16_round(W))
        bs.append(b.astype(np.float32).astype(np.float64))
    return Ws, bs
