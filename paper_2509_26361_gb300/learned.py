"""Learned curvature: data, training and evaluation driven through the C ABI.

The network (27 -> 128 -> 128 -> 1, ReLU, bf16 operands with FP32
accumulation) maps the canonically oriented 3x3x3 volume-fraction stencil of an
interface cell to kappa*h; height functions (Sec. 2.6) stay the fallback and
the reference it is measured against.  Every arithmetic step runs in the library's kernels: Front2VOF
makes the fractions, the gather kernel encodes the stencils, the training
kernel computes the loss gradient and the Adam kernel updates the weights.
This module only orchestrates them and computes the analytic labels on the
host (``curvature_data``).

Command line (GPU):
    python -m paper_2509_26361_gb300.learned train --out DIR [--stencils 2000000]
    python -m paper_2509_26361_gb300.learned eval --params FILE [--out DIR]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import curvature_data as D
from . import ebit

PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "mlp_curvature_params.npy")
RADIUS_BINS = (2.0, 4.0, 8.0, 16.0, 32.0, math.inf)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def finite_level(phi):
    """Level sets evaluated only near each shape carry -inf (or +inf) far away;
    the library needs finite values (only their signs matter there)."""
    return np.where(np.isfinite(phi), phi, np.sign(phi))


def stencil_set(n, ells, mlp, inside=1, with_hf=False):
    """Interface stencils of one grid: fractions from the library's Front2VOF
    on exact-crossing markers, encoded stencils and fragment flags from the
    gather kernel, analytic labels from the markers' centroids.  Returns a
    dict of device tensors X (bf16 [m, 64]), t (f32 [m]) and host arrays."""
    n3 = (n, n, n)
    f = D.ellipsoid_fields(n3, ells, inside)
    g = ebit.Grid(n, n, n)
    try:
        g.init(_dev(finite_level(f.phi)), _dev(finite_level(f.phi_faces)), _dev(f.s_exact))
        C = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        g.front2vof(C, flags=ebit.EBIT_FULL)
        cb, s = g.get_state()
        Ch = C.cpu().numpy().reshape(-1)
        cells = np.nonzero((Ch > 0.0) & (Ch < 1.0))[0].astype(np.int32)
        cent = D.interface_centroids(n3, cb.cpu().numpy(), s.cpu().numpy(), cells)
        lab = D.curvature_labels(n3, ells, f, cent, cells, inside)
        X, fr = mlp.gather(C, n3, _dev(cells), with_frag=True)
        out = {"cells": cells, "label": lab, "frag": fr.cpu().numpy().astype(bool), "X": X, "C": C, "n3": n3}
        if with_hf:
            kh = torch.zeros_like(C)
            st = torch.zeros(C.shape, dtype=torch.uint8, device="cuda")
            g.curvature(C, kh, st, mode=ebit.EBIT_CURV_HF, flags=ebit.EBIT_FULL)
            out["hf_kh"] = kh.reshape(-1)[_dev(cells).long()].cpu().numpy()
            out["hf_st"] = st.reshape(-1)[_dev(cells).long()].cpu().numpy()
        g.sync()
        return out
    finally:
        g.close()


def training_set(mlp, stencils=2_000_000, seed=3, n=256, bubble_every=4, log=print):
    """About ``stencils`` labelled stencils from seeded grids of spheres and
    ellipsoids with semi-axes between 2 and 32 cells (log-uniform, 30 %
    spheres).  Grids alternate between 150 shapes over the whole range and
    2000 small shapes (2 to 8 cells), so that small radii, whose shapes carry
    few interface cells each, are not rare.  Every ``bubble_every``-th grid
    swaps the phases (negative curvature).  Fragmented stencils (height-function
    fallback) and stencils without a finite label are left out."""
    rng = np.random.default_rng(seed)
    Xs, ts = [], []
    total = 0
    grid = 0
    while total < stencils:
        if grid % 2 == 0:
            ells = D.random_ellipsoids(rng, 150, 2.0, 32.0, n, log_uniform=True, sphere_fraction=0.3)
        else:
            ells = D.random_ellipsoids(rng, 2000, 2.0, 8.0, n, log_uniform=True, sphere_fraction=0.3)
        inside = 0 if (bubble_every and grid % bubble_every == bubble_every - 1) else 1
        st = stencil_set(n, ells, mlp, inside)
        keep = np.isfinite(st["label"]) & ~st["frag"] & (np.abs(st["label"]) <= 1.0)
        kidx = _dev(np.nonzero(keep)[0].astype(np.int64))
        Xs.append(st["X"][kidx])
        ts.append(_dev(st["label"][keep].astype(np.float32)))
        total += int(keep.sum())
        log(f"grid {grid}: {len(ells)} shapes, {int(keep.sum())} stencils (inside={inside}), total {total}")
        grid += 1
    X = torch.cat(Xs)
    t = torch.cat(ts)
    # a seeded subset of the requested size, mixed over the grids
    pick = _dev(rng.permutation(t.numel())[:stencils].astype(np.int64))
    return X[pick].contiguous(), t[pick].contiguous()


def train(mlp, X, t, epochs=400, batch=16384, lr0=2e-3, lr1=2e-5, seed=0, log=print):
    """Adam with a cosine learning-rate decay from lr0 to lr1; a fresh
    permutation of the rows every epoch (the training kernel reads the rows
    through the index array).  Returns the mean loss per epoch."""
    m = t.numel()
    rng = np.random.default_rng(seed)
    steps_per_epoch = m // batch
    total = epochs * steps_per_epoch
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        perm = _dev(rng.permutation(m).astype(np.int32))
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        for b in range(steps_per_epoch):
            lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * step / max(total - 1, 1)))
            mlp.train_step(X, t, lr, loss, idx=perm[b * batch:(b + 1) * batch], batch=batch)
            acc += loss
            step += 1
        mlp.sync()
        hist.append(float(acc.item()) / (steps_per_epoch * batch))
        log(f"epoch {ep}: loss {hist[-1]:.3e}")
    return hist


def _rms(e):
    return float(np.sqrt(np.mean(e * e))) if len(e) else float("nan")


def fp64_network(params, X):
    """The network evaluated in FP64 from the FP32 master parameters, with no
    bfloat16 rounding of weights or activations: the function the tensor-core
    pass approximates.  Used only to state that pass's precision error.
    X: encoded stencils (bf16 [m, 64], device); returns kappa*h (FP64, host)."""
    p = np.asarray(params, dtype=np.float64)
    W1 = p[:8192].reshape(128, 64)
    b1 = p[8192:8320]
    W2 = p[8320:24704].reshape(128, 128)
    b2, w3, b3 = p[24704:24832], p[24832:24960], p[24960]
    x = X.float().cpu().numpy().astype(np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def precision_error(mlp, X):
    """kappa*h of the tensor-core pass (bf16 operands, FP32 accumulation)
    against the unrounded FP64 network on the same encoded stencils."""
    y = mlp.forward(X).double().cpu().numpy()
    ref = fp64_network(mlp.get_params().cpu().numpy(), X)
    d = y - ref
    return {"stencils": int(len(y)), "rms": _rms(d), "max_abs": float(np.max(np.abs(d))) if len(d) else 0.0,
            "rms_ref": _rms(ref)}


def time_training(X, t, steps=200, batch=16384, warmup=10, seed=0):
    """Training throughput of the library's kernels (forward, backward and
    Adam per step, rows read through a random index array as in train()):
    stencil passes per second over ``steps`` steps of a fresh network, timed
    with CUDA events on the network's stream."""
    mlp = ebit.Mlp(init_params(seed))
    rng = np.random.default_rng(seed)
    m = t.numel()
    idx = [_dev(rng.integers(0, m, batch).astype(np.int32)) for _ in range(8)]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    for k in range(warmup):
        mlp.train_step(X, t, 1e-3, loss, idx=idx[k % 8], batch=batch)
    mlp.sync()
    # the network was created on the default stream, which is torch's current one here
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        mlp.train_step(X, t, 1e-3, loss, idx=idx[k % 8], batch=batch)
    e1.record()
    mlp.sync()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mlp.close()
    return {"steps": steps, "batch": batch, "ms_per_step": ms / steps,
            "stencil_passes_per_s": steps * batch / (ms * 1e-3),
            "flops_per_stencil_pass": 1.2e5, "tflops": steps * batch * 1.2e5 / (ms * 1e-3) / 1e12}


def evaluate(mlp, seed=33, n=256, count=64, amin=4.0, amax=32.0, repeats=5, path=None, train_steps=0):
    """The learned-curvature benchmark grid: ``count`` seeded ellipsoids with
    semi-axes U[amin, amax] cells and random rotations.  RMS kappa*h error
    against the analytic labels for height functions (where they give a value),
    the network alone, and the network with height-function fallback; binned
    by the local radius 2/|kappa| in cells; stencils per second of the
    height-function pass and the learned pass on the same interface list; the
    tensor-core pass against the unrounded FP64 network; and, with
    ``train_steps``, the training throughput on this grid's labelled stencils."""
    if path is not None:
        mlp.set_path(path)
    rng = np.random.default_rng(seed)
    ells = D.random_ellipsoids(rng, count, amin, amax, n)
    st = stencil_set(n, ells, mlp, 1, with_hf=True)
    cells, lab = st["cells"], st["label"]
    ok = np.isfinite(lab)
    n3 = st["n3"]
    g = ebit.Grid(*n3)
    g.set_mlp(mlp)
    C = st["C"]
    kh = torch.zeros_like(C)
    stt = torch.zeros(C.shape, dtype=torch.uint8, device="cuda")
    res = {"grid": n, "ellipsoids": count, "semi_axes_cells": [amin, amax], "interface_cells": int(len(cells))}
    idx = _dev(cells.astype(np.int64))
    vals = {}
    times = {}
    for name, mode in (("hf", ebit.EBIT_CURV_HF), ("mlp", ebit.EBIT_CURV_MLP), ("mlp_hf", ebit.EBIT_CURV_MLP_HF)):
        g.curvature(C, kh, stt, mode=mode, flags=ebit.EBIT_FULL)  # warm-up
        g.profile(True)
        for _ in range(repeats):
            g.curvature(C, kh, stt, mode=mode, flags=ebit.EBIT_FULL)
        prof = g.profile_read()
        g.profile(False)
        times[name] = {k: v[0] / repeats for k, v in prof.items()}
        vals[name] = (kh.reshape(-1)[idx].cpu().numpy(), stt.reshape(-1)[idx].cpu().numpy())
    # the other inference path on the same list (same network, same values)
    prev = getattr(mlp, "path", ebit.EBIT_MLP_PATH_TCGEN05)
    other = ebit.EBIT_MLP_PATH_MMA if prev == ebit.EBIT_MLP_PATH_TCGEN05 else ebit.EBIT_MLP_PATH_TCGEN05
    mlp.set_path(other)
    g.curvature(C, kh, stt, mode=ebit.EBIT_CURV_MLP, flags=ebit.EBIT_FULL)
    g.profile(True)
    for _ in range(repeats):
        g.curvature(C, kh, stt, mode=ebit.EBIT_CURV_MLP, flags=ebit.EBIT_FULL)
    prof = g.profile_read()
    g.profile(False)
    times["mlp_other_path"] = {k: v[0] / repeats for k, v in prof.items()}
    other_kh = kh.reshape(-1)[idx].cpu().numpy()
    mlp.set_path(prev)
    g.close()
    res["path"] = "tcgen05" if prev == ebit.EBIT_MLP_PATH_TCGEN05 else "mma.sync"
    res["other_path"] = "mma.sync" if prev == ebit.EBIT_MLP_PATH_TCGEN05 else "tcgen05"
    res["paths_max_abs_diff"] = float(np.max(np.abs(other_kh - vals["mlp"][0]))) if len(cells) else 0.0
    hf_k, hf_s = vals["hf"]
    hf_ok = ok & (hf_s >= 1) & (hf_s <= 3)
    res["hf_no_value"] = int(np.sum(ok & ~((hf_s >= 1) & (hf_s <= 3))))
    res["fragmented"] = int(np.sum(st["frag"]))
    mh_k, mh_s = vals["mlp_hf"]
    res["mlp_hf_fallback"] = int(np.sum(mh_s != 5))
    rad = 2.0 / np.maximum(np.abs(lab), 1e-30) / 1.0  # kappa*h -> 2/(kappa h) cells
    rows = []
    for lo, hi in zip(RADIUS_BINS[:-1], RADIUS_BINS[1:]):
        b = ok & (rad >= lo) & (rad < hi)
        bh = b & hf_ok
        rows.append({"radius_cells": [lo, hi], "cells": int(b.sum()), "hf_cells": int(bh.sum()),
                     "rms_hf": _rms(hf_k[bh] - lab[bh]), "rms_mlp": _rms(vals["mlp"][0][b] - lab[b]),
                     "rms_mlp_hf": _rms(mh_k[b] - lab[b]),
                     "rms_mlp_on_hf_cells": _rms(vals["mlp"][0][bh] - lab[bh])})
    res["bins"] = rows
    res["rms_hf"] = _rms(hf_k[hf_ok] - lab[hf_ok])
    res["rms_mlp"] = _rms(vals["mlp"][0][ok] - lab[ok])
    res["rms_mlp_hf"] = _rms(mh_k[ok] - lab[ok])
    res["rms_mlp_on_hf_cells"] = _rms(vals["mlp"][0][hf_ok] - lab[hf_ok])
    m = len(cells)
    t_hf = times["hf"].get("hf", float("nan"))
    t_list = times["mlp"].get("hf", 0.0)
    t_mlp = times["mlp"].get("mlp", float("nan"))
    t_mlp_hf = times["mlp_hf"].get("hf", 0.0) + times["mlp_hf"].get("mlp", float("nan"))
    res["ms"] = times
    res["hf_stencils_per_s"] = m / (t_hf * 1e-3)
    res["mlp_stencils_per_s"] = m / ((t_list + t_mlp) * 1e-3)
    res["mlp_hf_stencils_per_s"] = m / (t_mlp_hf * 1e-3)
    t_o = times["mlp_other_path"].get("hf", 0.0) + times["mlp_other_path"].get("mlp", float("nan"))
    res["mlp_other_path_stencils_per_s"] = m / (t_o * 1e-3)
    res["bf16_vs_fp64"] = precision_error(mlp, st["X"])
    if train_steps:
        keep = np.nonzero(ok & ~st["frag"] & (np.abs(lab) <= 1.0))[0]
        kidx = _dev(keep.astype(np.int64))
        res["training"] = time_training(st["X"][kidx].contiguous(), _dev(lab[keep].astype(np.float32)),
                                        steps=train_steps)
    return res


def init_params(seed=0):
    """He-uniform initial weights in the library's layout (W1[128][64], b1,
    W2[128][128], b2, w3, b3); a tail input starts with its head's weights."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((128, 64))
    W1[:, :27] = rng.uniform(-1.0, 1.0, (128, 27)) * math.sqrt(6.0 / 27.0)
    W1[:, 32:59] = W1[:, :27]
    W2 = rng.uniform(-1.0, 1.0, (128, 128)) * math.sqrt(6.0 / 128.0)
    w3 = rng.uniform(-1.0, 1.0, 128) * math.sqrt(3.0 / 128.0)
    return np.concatenate([W1.ravel(), np.zeros(128), W2.ravel(), np.zeros(128), w3, [0.1]])


def save_params(mlp, path):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.save(path, mlp.get_params().cpu().numpy().astype(np.float32))


def load_network(path=PARAMS_FILE):
    """A network with the stored parameters (float32 vector, see include/ebit.h)."""
    p = np.load(path)
    return ebit.Mlp(p.astype(np.float64))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=("train", "eval"))
    ap.add_argument("--out", default=".")
    ap.add_argument("--params", default=PARAMS_FILE)
    ap.add_argument("--stencils", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--seed", type=int, default=3)
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)

    def log(msg):
        print(msg, flush=True)

    if a.cmd == "train":
        t0 = time.time()
        mlp = ebit.Mlp(init_params(a.seed))
        X, t = training_set(mlp, a.stencils, seed=a.seed, log=log)
        t1 = time.time()
        torch.cuda.synchronize()
        t2 = time.time()
        hist = train(mlp, X, t, epochs=a.epochs, batch=a.batch, seed=a.seed, log=log)
        torch.cuda.synchronize()
        t3 = time.time()
        path = os.path.join(a.out, "mlp_curvature_params.npy")
        save_params(mlp, path)
        rep = {"stencils": int(t.numel()), "epochs": a.epochs, "batch": a.batch, "seed": a.seed,
               "data_seconds": t1 - t0, "train_seconds": t3 - t2, "loss_per_epoch": hist}
        rep["eval"] = evaluate(mlp)
        with open(os.path.join(a.out, "train_report.json"), "w") as fh:
            json.dump(rep, fh, indent=1)
        log(json.dumps(rep["eval"], indent=1))
    else:
        mlp = load_network(a.params)
        res = evaluate(mlp)
        with open(os.path.join(a.out, "eval_report.json"), "w") as fh:
            json.dump(res, fh, indent=1)
        log(json.dumps(res, indent=1))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
