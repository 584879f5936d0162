"""FP64 oracle of the learned curvature (27 -> 128 -> 128 -> 1 ReLU MLP).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

The learned curvature is not in the paper; it stands in for the height-function
curvature the paper computes from volume fractions (Sec. 2.6).  This module
restates, in plain numpy FP64:

* the canonical orientation of a 3x3x3 volume-fraction stencil: reflect every
  axis whose Youngs normal component (same sums and order as the HF oracle) is
  negative, then order the axes by increasing |n| (stable, lower axis first);
  curvature is invariant under these 48 cube symmetries;
* the input encoding: each C value is rounded to float32 and split into a
  bfloat16 head and a bfloat16 tail (head + tail carries ~16 mantissa bits),
  giving 27 heads and 27 tails padded to 32 + 32 = 64 inputs;
* the forward pass as the tensor-core kernels compute it: layer 1 and 2 from
  bfloat16 operands (weights, inputs, and the layer-1 activation rounded to
  bfloat16), ReLU, the output layer from the layer-2 activation unrounded;
* the backward pass (mean-squared relative error loss) and Adam;
* the fallback rules of the learned curvature: height functions where the
  learned value leaves |kappa h| <= 1 or where the 3x3x3 stencil holds a cell
  with C > 0 that is not face-connected to the centre through such cells.

Parameters are one flat float vector in this order: W1[128][64], b1[128],
W2[128][128], b2[128], w3[128], b3[1].
"""
from __future__ import annotations

import numpy as np

D_IN = 64  # 27 heads + 5 pad, 27 tails + 5 pad
H = 128
N_PARAMS = H * D_IN + H + H * H + H + H + 1


def bf16_round(x):
    """Round to bfloat16 (round to nearest even) via float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split_bf16(x):
    """x (FP64) -> (head, tail), both bfloat16 values: head = bf16(f32(x)),
    tail = bf16(f32(x) - head)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    hi = bf16_round(f)
    lo = bf16_round((f - hi).astype(np.float32))
    return hi, lo


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * D_IN].reshape(H, D_IN); o += H * D_IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3]).astype(np.float64)


def init_params(seed=0):
    """He-uniform initial weights (layer 1 fan-in counts the 27 real inputs)."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((H, D_IN))
    lim1 = np.sqrt(6.0 / 27.0)
    W1[:, :27] = rng.uniform(-lim1, lim1, (H, 27))
    W1[:, 32:59] = W1[:, :27]  # a tail feeds the same unit as its head
    b1 = np.zeros(H)
    lim2 = np.sqrt(6.0 / H)
    W2 = rng.uniform(-lim2, lim2, (H, H))
    b2 = np.zeros(H)
    w3 = rng.uniform(-np.sqrt(3.0 / H), np.sqrt(3.0 / H), H)
    b3 = np.array([0.2])
    return pack(W1, b1, W2, b2, w3, b3)


# ------------------------------------------------------------ stencils
def youngs_normal(blk):
    """blk[..., dz, dy, dx] (3x3x3): n = -grad C with 1-2-1 weights, summed in
    the height-function order (b2 outer, b1 inner) for each axis."""
    w = (1.0, 2.0, 1.0)
    n = np.zeros(blk.shape[:-3] + (3,))
    for d in range(3):
        t1, t2 = [(1, 2), (0, 2), (0, 1)][d]
        g = np.zeros(blk.shape[:-3])
        for b2 in (-1, 0, 1):
            for b1 in (-1, 0, 1):
                op = [0, 0, 0]
                om = [0, 0, 0]
                op[d], om[d] = 1, -1
                op[t1] += b1
                om[t1] += b1
                op[t2] += b2
                om[t2] += b2
                cp = blk[..., op[2] + 1, op[1] + 1, op[0] + 1]
                cm = blk[..., om[2] + 1, om[1] + 1, om[0] + 1]
                g = g + (w[b1 + 1] * w[b2 + 1]) * (cp - cm)
        n[..., d] = -g
    return n


def canonical_stencil(blk):
    """Canonically oriented stencil: (..., 27) in z-major order of the canonical
    axes (u2, u1, u0) with u_k the offset along the axis of k-th smallest |n|."""
    blk = np.asarray(blk, dtype=np.float64)
    flat = blk.reshape(-1, 3, 3, 3)
    n = youngs_normal(flat)
    out = np.zeros((flat.shape[0], 27))
    for i in range(flat.shape[0]):
        sgn = [(-1 if n[i, a] < 0.0 else 1) for a in range(3)]
        m = [abs(n[i, a]) for a in range(3)]
        # ascending |n|, stable (lower axis first on ties)
        o = [0, 1, 2]
        for a2 in (1, 2):
            b2 = a2
            while b2 > 0 and m[o[b2]] < m[o[b2 - 1]]:
                o[b2], o[b2 - 1] = o[b2 - 1], o[b2]
                b2 -= 1
        k = 0
        for u2 in (-1, 0, 1):
            for u1 in (-1, 0, 1):
                for u0 in (-1, 0, 1):
                    d = [0, 0, 0]
                    d[o[0]] = sgn[o[0]] * u0
                    d[o[1]] = sgn[o[1]] * u1
                    d[o[2]] = sgn[o[2]] * u2
                    out[i, k] = flat[i, d[2] + 1, d[1] + 1, d[0] + 1]
                    k += 1
    return out.reshape(blk.shape[:-3] + (27,))


def encode(stencils27):
    """(..., 27) FP64 -> (..., 64) bfloat16 values: heads, 5 zeros, tails, 5 zeros."""
    hi, lo = split_bf16(stencils27)
    z = np.zeros(hi.shape[:-1] + (5,))
    return np.concatenate([hi, z, lo, z], axis=-1)


def gather_stencils(C, cells):
    """3x3x3 blocks (periodic) around linear cell ids of C[nz, ny, nx]."""
    nz, ny, nx = C.shape
    cells = np.asarray(cells, dtype=np.int64)
    x = cells % nx
    y = (cells // nx) % ny
    z = cells // (nx * ny)
    blk = np.zeros((len(cells), 3, 3, 3))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                blk[:, dz + 1, dy + 1, dx + 1] = C[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
    return blk


def fragmented(blk):
    """True if a cell of the 3x3x3 block (blk[dz, dy, dx]) with C > 0 cannot be
    reached from the centre by face steps through cells with C > 0 (breadth-
    first search from the centre)."""
    blk = np.asarray(blk)
    pos = {(z, y, x) for z in range(3) for y in range(3) for x in range(3) if blk[z, y, x] > 0.0}
    seen = set()
    if (1, 1, 1) in pos:
        seen.add((1, 1, 1))
        todo = [(1, 1, 1)]
        while todo:
            z, y, x = todo.pop()
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                q = (z + dz, y + dy, x + dx)
                if q in pos and q not in seen:
                    seen.add(q)
                    todo.append(q)
    return seen != pos


def learned_curvature(C, p, mode, hf_kh, hf_st, cells=None):
    """kappa*h and status on the interface cells (0 < C < 1) of C[nz, ny, nx]:
    mode 1 the network's value (status 5) everywhere; mode 2 the height-function
    value and status (hf_kh, hf_st, flat arrays) where the network's value has
    |y| > 1 or the stencil is fragmented.  Returns (cells, kh, st, y, frag)."""
    flat = np.asarray(C).reshape(-1)
    if cells is None:
        cells = np.nonzero((flat > 0.0) & (flat < 1.0))[0]
    blk = gather_stencils(np.asarray(C), cells)
    X = encode(canonical_stencil(blk))
    y, _ = forward(p, X, emulate=True)
    frag = np.array([fragmented(b) for b in blk], dtype=bool)
    kh = y.copy()
    st = np.full(len(cells), 5, dtype=np.uint8)
    if mode == 2:
        fb = (np.abs(y) > 1.0) | frag
        kh[fb] = np.asarray(hf_kh).reshape(-1)[cells[fb]]
        st[fb] = np.asarray(hf_st).reshape(-1)[cells[fb]]
    return cells, kh, st, y, frag


# ------------------------------------------------------------- network
def forward(p, X, emulate=True):
    """y (FP64) for inputs X (B, 64).  With emulate, weights are rounded to
    bfloat16 and the layer-1 activation too, as in the tensor-core kernels."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    if emulate:
        W1, W2 = bf16_round(W1), bf16_round(W2)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    h1r = bf16_round(h1) if emulate else h1
    z2 = h1r @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    return y, (X, z1, h1r, z2, h2)


def loss_weights(t, floor=0.05):
    return 1.0 / np.maximum(np.abs(t), floor) ** 2


def loss_and_grad(p, X, t, emulate=True):
    """Mean squared relative error (denominator max(|t|, 0.05)) and its gradient
    (backprop of the forward above, roundings passed straight through)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    W1e, W2e = (bf16_round(W1), bf16_round(W2)) if emulate else (W1, W2)
    y, (X, z1, h1r, z2, h2) = forward(p, X, emulate)
    B = X.shape[0]
    wgt = loss_weights(t)
    r = y - t
    loss = float(np.mean(wgt * r * r))
    dy = 2.0 * wgt * r / B
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dh2 = np.outer(dy, w3) * (z2 > 0.0)
    dW2 = dh2.T @ h1r
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2e) * (z1 > 0.0)
    dW1 = dh1.T @ X
    db1 = dh1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------- analytic labels
def ellipsoid_mean_curvature(x, axes):
    """Sum of principal curvatures of the ellipsoid sum x_i^2/a_i^2 = 1 at the
    surface point x (body frame): (|gF|^2 tr H - gF^T H gF) / |gF|^3 for
    F = sum x_i^2/a_i^2 - 1 (positive: convex, reference phase inside)."""
    a2 = np.asarray(axes, dtype=np.float64) ** 2
    g = 2.0 * x / a2
    Hd = 2.0 / a2
    gn2 = np.sum(g * g, axis=-1)
    return (gn2 * np.sum(Hd) - np.sum(g * g * Hd, axis=-1)) / gn2 ** 1.5


def ellipsoid_closest_point(p, axes, iters=60):
    """Closest surface point of the ellipsoid to points p (body frame, outside or
    inside): x_i = a_i^2 p_i / (a_i^2 + t) with t the root of
    sum (a_i p_i / (a_i^2 + t))^2 = 1, found by bisection on its monotone branch."""
    a2 = np.asarray(axes, dtype=np.float64) ** 2
    p = np.asarray(p, dtype=np.float64)

    def f(t):
        return np.sum((np.sqrt(a2) * p / (a2 + t[..., None])) ** 2, axis=-1) - 1.0

    lo = np.full(p.shape[:-1], -np.min(a2) + 1e-12)
    hi = np.full(p.shape[:-1], np.max(a2) * 4 + np.sum(p * p, axis=-1) * 4)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        lo = np.where(fm > 0, mid, lo)
        hi = np.where(fm > 0, hi, mid)
    t = 0.5 * (lo + hi)
    return a2 * p / (a2 + t[..., None])
