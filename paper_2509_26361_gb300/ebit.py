"""Thin Python binding of libebit.so (the C ABI in include/ebit.h).

Functions carry the C names and only marshal arguments: torch tensors supply
device memory (``data_ptr()``) and the CUDA stream; every step of the EBIT path
runs in the library's CUDA kernels.  There is no CPU fallback: importing works
without a GPU, but any call needs the compiled library and a CUDA device and
raises ``EbitError`` otherwise.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

EBIT_OK = 0
EBIT_EINVAL = -1
EBIT_ENONFINITE = -2
EBIT_ECUDA = -3
EBIT_ETIMEOUT = -4
EBIT_ENOMEM = -5
EBIT_ECFL = -6
EBIT_WINCONSISTENT = 1

EBIT_INCREMENTAL = 0
EBIT_FULL = 1
EBIT_ASYNC = 2
EBIT_CURV_HF = 0
EBIT_CURV_MLP = 1
EBIT_CURV_MLP_HF = 2
EBIT_DESC_DENSE = 1

ST_NONE, ST_HF_X, ST_HF_Y, ST_HF_Z, ST_NO_HF, ST_MLP = 0, 1, 2, 3, 4, 5
EBIT_MLP_PATH_MMA, EBIT_MLP_PATH_TCGEN05 = 0, 1
# tile shapes of a batch (cells per tile edge along x, y, z), in ABI order
TILE_SHAPES = ((8, 8, 8), (16, 8, 4), (32, 4, 4))
EBIT_BATCH_MAX_CTAS = 8

COUNTER_NAMES = ("markers", "annihilate", "multi", "inconsistent", "cfl")


class EbitError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ebit error {code}: {msg}")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("flags", ctypes.c_int)]


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in COUNTER_NAMES + ("tiles", "nonfinite")]


_lib = None
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
# every callback pair ever installed: an object keeps the pair it was created
# with until it is destroyed, so none may be collected
_allocators = []


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libebit.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise EbitError(EBIT_ECUDA, f"CUDA library missing: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ebit_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.ebit_destroy.argtypes = [P]
    lib.ebit_destroy.restype = None
    lib.ebit_init.argtypes = [P, P, P, P]
    lib.ebit_set_state.argtypes = [P, P, P]
    lib.ebit_get_state.argtypes = [P, P, P]
    lib.ebit_advect_sweep.argtypes = [P, I, P, D]
    lib.ebit_front2vof.argtypes = [P, P, I]
    lib.ebit_curvature.argtypes = [P, P, P, P, I, I]
    lib.ebit_counters.argtypes = [P, ctypes.POINTER(_Counters)]
    lib.ebit_reset_counters.argtypes = [P]
    lib.ebit_sync.argtypes = [P]
    lib.ebit_band_tiles.argtypes = [P]
    lib.ebit_profile.argtypes = [P, I]
    lib.ebit_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    lib.ebit_advect_sweep_noalloc.argtypes = [I, I, I, D, I, P, P, P, D, P, P, P]
    lib.ebit_join.argtypes = [P]
    lib.ebit_event_record.argtypes = [P, P]
    lib.ebit_mlp_nparams.argtypes = []
    lib.ebit_mlp_create.argtypes = [P, ctypes.POINTER(ctypes.c_void_p)]
    lib.ebit_mlp_destroy.argtypes = [P]
    lib.ebit_mlp_destroy.restype = None
    lib.ebit_mlp_set_params.argtypes = [P, P]
    lib.ebit_mlp_get_params.argtypes = [P, P]
    lib.ebit_mlp_gather.argtypes = [P, P, I, I, I, P, I, P, P]
    lib.ebit_mlp_forward.argtypes = [P, P, I, P]
    lib.ebit_mlp_gradient.argtypes = [P, P, P, I, P]
    lib.ebit_mlp_train_step.argtypes = [P, P, P, P, I, ctypes.c_float, P]
    lib.ebit_mlp_sync.argtypes = [P]
    lib.ebit_mlp_set_path.argtypes = [P, I]
    lib.ebit_mlp_last_error.argtypes = [P]
    lib.ebit_mlp_last_error.restype = ctypes.c_char_p
    lib.ebit_set_mlp.argtypes = [P, P]
    lib.ebit_last_error.argtypes = [P]
    lib.ebit_last_error.restype = ctypes.c_char_p
    lib.ebit_batch_create.argtypes = [I, ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_void_p)]
    lib.ebit_batch_destroy.argtypes = [P]
    lib.ebit_selftest_bounded_waits.argtypes = [P, P]
    lib.ebit_selftest_f64_to_f32.argtypes = [P, P, I, P]
    lib.ebit_refine_mask.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
    lib.ebit_one_fluid.argtypes = [P, P, P, P, D, D, D, D, D, P, P, P]
    lib.ebit_pack_bricks.argtypes = [P, I, P, P, P, P, ctypes.POINTER(ctypes.c_int)]
    lib.ebit_unpack_bricks.argtypes = [P, I, P, P, P, P]
    lib.ebit_batch_destroy.restype = None
    lib.ebit_batch_size.argtypes = [P]
    lib.ebit_batch_instance.argtypes = [P, I]
    lib.ebit_batch_instance.restype = P
    lib.ebit_batch_set_velocity.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double)]
    lib.ebit_batch_advect_sweep.argtypes = [P, I, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double)]
    lib.ebit_mlp_load.argtypes = [P, P, ctypes.c_size_t]
    lib.ebit_batch_run.argtypes = [P, I, I, I]
    lib.ebit_batch_graph_active.argtypes = [P]
    lib.ebit_batch_graph_note.argtypes = [P]
    lib.ebit_batch_graph_note.restype = ctypes.c_char_p
    lib.ebit_batch_sync.argtypes = [P]
    lib.ebit_batch_launch_shape.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.ebit_batch_set_launch_shape.argtypes = [P, I]
    lib.ebit_batch_autotune.argtypes = [P, I, ctypes.POINTER(ctypes.c_double)]
    lib.ebit_batch_tile_shape.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.ebit_batch_set_tile_shape.argtypes = [P, I]
    lib.ebit_batch_last_error.argtypes = [P]
    lib.ebit_batch_last_error.restype = ctypes.c_char_p
    lib.ebit_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, P]
    _lib = lib
    return lib


def _check(ctx, code):
    if code < 0:
        msg = load().ebit_last_error(ctx).decode() if ctx else ""
        raise EbitError(code, msg)
    return code


def _dev(t: torch.Tensor, dtype, numel=None, name="tensor"):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise TypeError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _any(t: torch.Tensor, dtype, numel, name):
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name}: need a contiguous {dtype} tensor of {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------- C names
def ebit_set_allocator(alloc=None, free=None):
    """Route the library's device allocations through ``alloc(nbytes) -> int``
    (a device pointer aligned to 256 bytes, or 0 when it cannot allocate) and
    ``free(ptr)``; both None restores cudaMalloc / cudaFree.  Objects created
    afterwards keep this pair for their whole life."""
    lib = load()
    if alloc is None and free is None:
        return _check(None, lib.ebit_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
    if alloc is None or free is None:
        fa = _ALLOC_FN(lambda n, u: alloc(n) or None) if alloc is not None else _ALLOC_FN()
        ff = _FREE_FN(lambda ptr, u: free(ptr)) if free is not None else _FREE_FN()
        return _check(None, lib.ebit_set_allocator(fa, ff, None))
    fa = _ALLOC_FN(lambda n, u: alloc(n) or None)
    ff = _FREE_FN(lambda ptr, u: free(ptr))
    _allocators.append((fa, ff))
    return _check(None, lib.ebit_set_allocator(fa, ff, None))


def ebit_selftest_f64_to_f32(x):
    """The gather's bit-pattern double -> float rounding over a float64 CUDA tensor."""
    xp = _dev(x, torch.float64, name="x")
    out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    _check(None, load().ebit_selftest_f64_to_f32(xp, _dev(out, torch.float32, name="out"), int(x.numel()),
                                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def ebit_create(nx, ny, nz, h, stream=None, flags=0):
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    d = _Desc(int(nx), int(ny), int(nz), float(h), ctypes.c_void_p(sp), int(flags))
    out = ctypes.c_void_p()
    code = lib.ebit_create(ctypes.byref(d), ctypes.byref(out))
    if code != EBIT_OK:
        raise EbitError(code, "ebit_create failed")
    return out


def ebit_destroy(ctx):
    load().ebit_destroy(ctx)


def ebit_init(ctx, n, phi_nodes, phi_faces=None, s_exact=None):
    pf = None if phi_faces is None else _dev(phi_faces, torch.float64, 3 * n, "phi_faces")
    se = None if s_exact is None else _dev(s_exact, torch.float64, 3 * n, "s_exact")
    return _check(ctx, load().ebit_init(ctx, _dev(phi_nodes, torch.float64, n, "phi_nodes"), pf, se))


def ebit_set_state(ctx, n, cb, s):
    return _check(ctx, load().ebit_set_state(ctx, _any(cb, torch.uint8, n, "cb"), _any(s, torch.float64, 3 * n, "s")))


def ebit_get_state(ctx, n, cb, s):
    return _check(ctx, load().ebit_get_state(ctx, _any(cb, torch.uint8, n, "cb"), _any(s, torch.float64, 3 * n, "s")))


def ebit_advect_sweep(ctx, n, d, u_face, dt):
    return _check(ctx, load().ebit_advect_sweep(ctx, int(d), _dev(u_face, torch.float64, n, "u_face"), float(dt)))


def ebit_front2vof(ctx, n, C, flags=EBIT_INCREMENTAL):
    return _check(ctx, load().ebit_front2vof(ctx, _dev(C, torch.float64, n, "C"), int(flags)))


def ebit_curvature(ctx, n, C, kappa_h, status, mode=EBIT_CURV_HF, flags=EBIT_INCREMENTAL):
    return _check(ctx, load().ebit_curvature(ctx, _dev(C, torch.float64, n, "C"),
                                             _dev(kappa_h, torch.float64, n, "kappa_h"),
                                             _dev(status, torch.uint8, n, "status"), int(mode), int(flags)))


def ebit_counters(ctx):
    c = _Counters()
    code = load().ebit_counters(ctx, ctypes.byref(c))
    _check(ctx, code)
    return {k: int(getattr(c, k)) for k in COUNTER_NAMES + ("tiles", "nonfinite")}, code


def ebit_reset_counters(ctx):
    return _check(ctx, load().ebit_reset_counters(ctx))


def ebit_sync(ctx):
    return _check(ctx, load().ebit_sync(ctx))


def ebit_join(ctx):
    return _check(ctx, load().ebit_join(ctx))


def ebit_event_record(ctx, event):
    """Record a torch.cuda.Event where the context's last Front2VOF/curvature
    output is complete (see include/ebit.h).  torch creates the CUDA event on
    its first record, so an unused event is recorded once first."""
    if not event.cuda_event:
        event.record()
    return _check(ctx, load().ebit_event_record(ctx, ctypes.c_void_p(event.cuda_event)))


def ebit_band_tiles(ctx):
    return int(load().ebit_band_tiles(ctx))


PROF_KINDS = ("sweep", "band", "f2v", "hf", "mlp", "advect", "fp64", "scan", "coupling")


def ebit_profile(ctx, enable):
    return _check(ctx, load().ebit_profile(ctx, int(bool(enable))))


def ebit_profile_read(ctx):
    ms = (ctypes.c_double * len(PROF_KINDS))()
    n = (ctypes.c_int64 * len(PROF_KINDS))()
    _check(ctx, load().ebit_profile_read(ctx, ms, n))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROF_KINDS) if n[i]}


def ebit_advect_sweep_noalloc(n3, h, d, cb_in, s_in, u_face, dt, cb_out, s_out, stream=None):
    """One sweep with no device allocation (see include/ebit.h); all tensors on
    the device, at most 64^3 cells."""
    nx, ny, nz = (int(v) for v in n3)
    n = nx * ny * nz
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    code = load().ebit_advect_sweep_noalloc(
        nx, ny, nz, float(h), int(d), _dev(cb_in, torch.uint8, n, "cb_in"), _dev(s_in, torch.float64, 3 * n, "s_in"),
        _dev(u_face, torch.float64, n, "u_face"), float(dt), _dev(cb_out, torch.uint8, n, "cb_out"),
        _dev(s_out, torch.float64, 3 * n, "s_out"), ctypes.c_void_p(sp))
    if code < 0:
        raise EbitError(code, "ebit_advect_sweep_noalloc failed")
    return code


def ebit_last_error(ctx):
    return load().ebit_last_error(ctx).decode()


def ebit_selftest_bounded_waits(stream=None):
    """Runs the self-test of the bounded device waits (see include/ebit.h);
    returns (code, report) with report the six ints it fills."""
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rep = (ctypes.c_int * 6)()
    code = load().ebit_selftest_bounded_waits(ctypes.c_void_p(sp), rep)
    return code, list(rep)


# ------------------------------------------------------- learned curvature
def _mcheck(mlp, code):
    if code < 0:
        raise EbitError(code, load().ebit_mlp_last_error(mlp).decode())
    return code


def ebit_mlp_nparams():
    return int(load().ebit_mlp_nparams())


def ebit_mlp_create(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    out = ctypes.c_void_p()
    code = load().ebit_mlp_create(ctypes.c_void_p(sp), ctypes.byref(out))
    if code != EBIT_OK:
        raise EbitError(code, "ebit_mlp_create failed")
    return out


def ebit_mlp_destroy(mlp):
    load().ebit_mlp_destroy(mlp)


def ebit_mlp_set_params(mlp, params):
    return _mcheck(mlp, load().ebit_mlp_set_params(mlp, _any(params, torch.float32, ebit_mlp_nparams(), "params")))


def ebit_mlp_get_params(mlp, params):
    return _mcheck(mlp, load().ebit_mlp_get_params(mlp, _any(params, torch.float32, ebit_mlp_nparams(), "params")))


def ebit_mlp_gather(mlp, C, n3, cells, X, frag=None):
    nx, ny, nz = (int(v) for v in n3)
    m = cells.numel()
    fp = None if frag is None else _dev(frag, torch.uint8, m, "frag")
    return _mcheck(mlp, load().ebit_mlp_gather(mlp, _dev(C, torch.float64, nx * ny * nz, "C"), nx, ny, nz,
                                               _dev(cells, torch.int32, m, "cells"), m,
                                               _dev(X, torch.bfloat16, 64 * m, "X"), fp))


def ebit_mlp_forward(mlp, X, y):
    m = y.numel()
    return _mcheck(mlp, load().ebit_mlp_forward(mlp, _dev(X, torch.bfloat16, 64 * m, "X"), m,
                                                _dev(y, torch.float32, m, "y")))


def ebit_mlp_gradient(mlp, X, t, grad):
    b = t.numel()
    return _mcheck(mlp, load().ebit_mlp_gradient(mlp, _dev(X, torch.bfloat16, 64 * b, "X"),
                                                 _dev(t, torch.float32, b, "t"), b,
                                                 _any(grad, torch.float32, ebit_mlp_nparams(), "grad")))


def ebit_mlp_train_step(mlp, X, t, lr, loss=None, idx=None, batch=None):
    """One Adam step on rows idx[:batch] of (X, t), or on all of them without idx."""
    if idx is None:
        b = t.numel()
        if X.numel() != 64 * b:
            raise ValueError("X must have 64 values per label")
        ip = None
    else:
        b = int(batch if batch is not None else idx.numel())
        if b > idx.numel():
            raise ValueError("batch larger than the index array")
        ip = _dev(idx, torch.int32, idx.numel(), "idx")
    lp = None if loss is None else _dev(loss, torch.float32, 1, "loss")
    return _mcheck(mlp, load().ebit_mlp_train_step(mlp, _dev(X, torch.bfloat16, X.numel(), "X"),
                                                   _dev(t, torch.float32, t.numel(), "t"), ip, b, float(lr), lp))


def ebit_mlp_sync(mlp):
    return _mcheck(mlp, load().ebit_mlp_sync(mlp))


def ebit_mlp_load(ctx, params):
    p = torch.as_tensor(params, dtype=torch.float32).contiguous()
    n = ebit_mlp_nparams()
    if p.numel() != n:
        raise ValueError(f"params: need {n} floats")
    return _check(ctx, load().ebit_mlp_load(ctx, ctypes.c_void_p(p.data_ptr()), 4 * n))


def ebit_set_mlp(ctx, mlp):
    return _check(ctx, load().ebit_set_mlp(ctx, mlp))


class Mlp:
    """The learned-curvature network on the device (parameters, Adam state)."""

    def __init__(self, params=None, stream=None):
        self.h = ebit_mlp_create(stream)
        self.path = EBIT_MLP_PATH_TCGEN05
        self.nparams = ebit_mlp_nparams()
        if params is not None:
            self.set_params(params)

    def close(self):
        if self.h is not None:
            ebit_mlp_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = torch.as_tensor(params, dtype=torch.float32).contiguous().cuda()
        ebit_mlp_set_params(self.h, p)

    def get_params(self):
        p = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        ebit_mlp_get_params(self.h, p)
        return p

    def gather(self, C, n3, cells, with_frag=False):
        X = torch.empty((cells.numel(), 64), dtype=torch.bfloat16, device="cuda")
        fr = torch.empty(cells.numel(), dtype=torch.uint8, device="cuda") if with_frag else None
        ebit_mlp_gather(self.h, C, n3, cells, X, fr)
        return (X, fr) if with_frag else X

    def forward(self, X):
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        ebit_mlp_forward(self.h, X, y)
        return y

    def gradient(self, X, t):
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        ebit_mlp_gradient(self.h, X, t, g)
        return g

    def train_step(self, X, t, lr, loss=None, idx=None, batch=None):
        return ebit_mlp_train_step(self.h, X, t, lr, loss, idx, batch)

    def sync(self):
        return ebit_mlp_sync(self.h)

    def set_path(self, path):
        """EBIT_MLP_PATH_MMA (warp-level MMA) or EBIT_MLP_PATH_TCGEN05."""
        r = _mcheck(self.h, load().ebit_mlp_set_path(self.h, int(path)))
        self.path = int(path)
        return r


# ----------------------------------------------------------------- batches
def _bcheck(b, code):
    if code < 0:
        raise EbitError(code, load().ebit_batch_last_error(b).decode())
    return code


def ebit_batch_create(n3s, hs=None, stream=None):
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    n = len(n3s)
    descs = (_Desc * n)()
    for i, n3 in enumerate(n3s):
        h = float(hs[i]) if hs is not None else 1.0 / n3[0]
        descs[i] = _Desc(int(n3[0]), int(n3[1]), int(n3[2]), h, ctypes.c_void_p(sp), 0)
    out = ctypes.c_void_p()
    code = lib.ebit_batch_create(n, descs, ctypes.byref(out))
    if code != EBIT_OK:
        raise EbitError(code, "ebit_batch_create failed")
    return out


def ebit_batch_set_velocity(b, n3s, u_fields, dts):
    """u_fields[i] = (u_x, u_y, u_z) device float64 tensors of instance i."""
    n = len(n3s)
    ptrs = (ctypes.c_void_p * (3 * n))()
    for i in range(n):
        N = n3s[i][0] * n3s[i][1] * n3s[i][2]
        for d in range(3):
            ptrs[3 * i + d] = _dev(u_fields[i][d], torch.float64, N, "u_face").value
    dt = (ctypes.c_double * n)(*[float(v) for v in dts])
    return _bcheck(b, load().ebit_batch_set_velocity(b, ptrs, dt))


class Batch:
    """Independent instances advanced by one persistent launch per split sweep.
    ``instance(i)`` is a :class:`Grid` view of instance i (state access,
    Front2VOF, curvature, counters)."""

    def __init__(self, n3s, hs=None, device="cuda", stream=None):
        self.n3s = [tuple(int(v) for v in n3) for n3 in n3s]
        self.hs = [float(hs[i]) if hs is not None else 1.0 / n3[0] for i, n3 in enumerate(self.n3s)]
        self.device = torch.device(device)
        self.b = ebit_batch_create(self.n3s, self.hs, stream)
        self._views = [Grid._view(load().ebit_batch_instance(self.b, i), self.n3s[i], self.hs[i], self.device)
                       for i in range(len(self.n3s))]
        self._u = None

    def __len__(self):
        return len(self.n3s)

    def instance(self, i):
        return self._views[i]

    def set_velocity(self, u_fields, dts):
        self._u = [tuple(u) for u in u_fields]  # keep the device fields alive
        return ebit_batch_set_velocity(self.b, self.n3s, self._u, dts)

    def sweep(self, d, u=None, dts=None):
        """One split sweep along d; ``u`` (instance i's u_d device tensor at u[i])
        and ``dts`` replace the stored velocity of d and the time steps."""
        up = dp = None
        if u is not None:
            up = (ctypes.c_void_p * len(self.n3s))()
            for i, n3 in enumerate(self.n3s):
                up[i] = _dev(u[i], torch.float64, n3[0] * n3[1] * n3[2], "u_face").value
                self._keep = getattr(self, "_keep", {})
                self._keep[(d, i)] = u[i]
        if dts is not None:
            dp = (ctypes.c_double * len(self.n3s))(*[float(v) for v in dts])
        return _bcheck(self.b, load().ebit_batch_advect_sweep(self.b, int(d), up, dp))

    def run(self, first_step, steps, graph=True):
        return _bcheck(self.b, load().ebit_batch_run(self.b, int(first_step), int(steps), int(bool(graph))))

    def graph_active(self):
        """0 none, 1 stream capture, 2 graph built node by node."""
        return int(load().ebit_batch_graph_active(self.b))

    def graph_note(self):
        return load().ebit_batch_graph_note(self.b).decode()

    def sync(self):
        return _bcheck(self.b, load().ebit_batch_sync(self.b))

    def launch_shape(self):
        c, m = ctypes.c_int(), ctypes.c_int()
        _bcheck(self.b, load().ebit_batch_launch_shape(self.b, ctypes.byref(c), ctypes.byref(m)))
        return c.value, m.value

    def set_launch_shape(self, ctas_per_sm):
        return _bcheck(self.b, load().ebit_batch_set_launch_shape(self.b, int(ctas_per_sm)))

    def tile_shape(self):
        """(shape id, (tx, ty, tz)) of the band tiles in use."""
        dims = (ctypes.c_int * 3)()
        sh = _bcheck(self.b, load().ebit_batch_tile_shape(self.b, dims))
        return sh, tuple(int(v) for v in dims)

    def set_tile_shape(self, shape):
        """Re-tile every instance with tile shape ``shape`` (an index of TILE_SHAPES)."""
        return _bcheck(self.b, load().ebit_batch_set_tile_shape(self.b, int(shape)))

    def autotune(self, sweeps=6):
        """Time every tile shape and launch shape on a copy of the state, keep
        the fastest pair; returns {(tx, ty, tz): [ms for 1, 2, ... blocks/SM]}."""
        ms = (ctypes.c_double * (len(TILE_SHAPES) * EBIT_BATCH_MAX_CTAS))()
        _bcheck(self.b, load().ebit_batch_autotune(self.b, int(sweeps), ms))
        out = {}
        for sh, dims in enumerate(TILE_SHAPES):
            row = [float(v) for v in ms[sh * EBIT_BATCH_MAX_CTAS:(sh + 1) * EBIT_BATCH_MAX_CTAS]]
            out[dims] = [v for v in row if v > 0.0]
        return out

    def close(self):
        if self.b is not None:
            for v in self._views:
                v.ctx = None
            load().ebit_batch_destroy(self.b)
            self.b = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ convenience
class Grid:
    """One EBIT context with its device buffers (torch tensors on ``device``).

    ``shape`` is (nz, ny, nx); every array is idx-ordered like the C ABI.
    """

    def __init__(self, nx, ny, nz, h=None, device="cuda", stream=None, dense=False):
        self.n3 = (int(nx), int(ny), int(nz))
        self.N = self.n3[0] * self.n3[1] * self.n3[2]
        self.h = float(h if h is not None else 1.0 / nx)
        self.device = torch.device(device)
        self.shape = (self.n3[2], self.n3[1], self.n3[0])
        self.ctx = ebit_create(nx, ny, nz, self.h, stream, EBIT_DESC_DENSE if dense else 0)

    @classmethod
    def _view(cls, ctx, n3, h, device):
        """A Grid over a context owned elsewhere (a batch instance)."""
        g = cls.__new__(cls)
        g.n3 = tuple(int(v) for v in n3)
        g.N = g.n3[0] * g.n3[1] * g.n3[2]
        g.h = float(h)
        g.device = torch.device(device)
        g.shape = (g.n3[2], g.n3[1], g.n3[0])
        g.ctx = ctypes.c_void_p(ctx)
        g._owned = False
        return g

    def close(self):
        if self.ctx is not None and getattr(self, "_owned", True):
            ebit_destroy(self.ctx)
        self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi_nodes, phi_faces=None, s_exact=None):
        return ebit_init(self.ctx, self.N, phi_nodes, phi_faces, s_exact)

    def set_state(self, cb, s):
        return ebit_set_state(self.ctx, self.N, cb, s)

    def get_state(self):
        cb = torch.empty(self.shape, dtype=torch.uint8, device=self.device)
        s = torch.empty((3,) + self.shape, dtype=torch.float64, device=self.device)
        ebit_get_state(self.ctx, self.N, cb, s)
        return cb, s

    def sweep(self, d, u_face, dt):
        return ebit_advect_sweep(self.ctx, self.N, d, u_face, dt)

    def step(self, n, u_fields, dt):
        """Three split sweeps: x-y-z on even steps, z-y-x on odd steps."""
        for d in ((0, 1, 2) if n % 2 == 0 else (2, 1, 0)):
            self.sweep(d, u_fields[d], dt)

    def front2vof(self, C, flags=EBIT_INCREMENTAL):
        return ebit_front2vof(self.ctx, self.N, C, flags)

    def curvature(self, C, kappa_h, status, mode=EBIT_CURV_HF, flags=EBIT_INCREMENTAL):
        return ebit_curvature(self.ctx, self.N, C, kappa_h, status, mode, flags)

    def counters(self):
        return ebit_counters(self.ctx)[0]

    def reset_counters(self):
        return ebit_reset_counters(self.ctx)

    def sync(self):
        return ebit_sync(self.ctx)

    def join(self):
        return ebit_join(self.ctx)

    def record_done(self, event):
        return ebit_event_record(self.ctx, event)

    def band_tiles(self):
        return ebit_band_tiles(self.ctx)

    def set_mlp(self, mlp):
        return ebit_set_mlp(self.ctx, None if mlp is None else mlp.h)

    def load_mlp(self, params):
        """Parameters (float32, host or device) into a network the context owns."""
        return ebit_mlp_load(self.ctx, params)

    @property
    def tiles(self):
        """Number of 8^3 tiles (bricks) of the grid."""
        t = 1
        for v in self.n3:
            t *= (v + 7) // 8
        return t

    def one_fluid(self, C, kh=None, st=None, sigma=0.0, rho1=1.0, rho2=1.0, mu1=1.0, mu2=1.0, force=True, out=None):
        """Eq. 6 properties (rho, mu per cell) and, with force, the face-centred
        well-balanced surface-tension force [3, nz, ny, nx] from C and the
        curvature output (kh, st); out = (rho, mu, f) reuses buffers."""
        if out is not None:
            rho, mu, f = out
        else:
            rho = torch.empty(self.shape, dtype=torch.float64, device=self.device)
            mu = torch.empty_like(rho)
            f = torch.empty((3,) + self.shape, dtype=torch.float64, device=self.device) if force else None
        _check(self.ctx, load().ebit_one_fluid(
            self.ctx, _dev(C, torch.float64, self.N, "C"),
            _dev(kh, torch.float64, self.N, "kh") if force else None,
            _dev(st, torch.uint8, self.N, "st") if force else None,
            float(sigma), float(rho1), float(rho2), float(mu1), float(mu2),
            _dev(rho, torch.float64), _dev(mu, torch.float64), _dev(f, torch.float64) if force else None))
        return rho, mu, f

    def refine_mask(self):
        """(mask uint8 tensor of the grid's shape, count): the cells that the
        AMR rule of Sec. 2.5 refines (3x3x3 around every interfacial cell)."""
        mask = torch.empty(self.shape, dtype=torch.uint8, device=self.device)
        n = ctypes.c_int64()
        _check(self.ctx, load().ebit_refine_mask(self.ctx, _dev(mask, torch.uint8, self.N, "mask"), ctypes.byref(n)))
        return mask, int(n.value)

    def pack_bricks(self):
        """The narrow-band brick store of the state: dict of device tensors
        tiles [n] int32, cb [n, 512] uint8, s [n, 3, 512] float64, bg [tiles] uint8."""
        lib = load()
        n = ctypes.c_int()
        _check(self.ctx, lib.ebit_pack_bricks(self.ctx, 0, None, None, None, None, ctypes.byref(n)))
        cap = max(int(n.value), 1)
        t = torch.empty(cap, dtype=torch.int32, device=self.device)
        cb = torch.empty((cap, 512), dtype=torch.uint8, device=self.device)
        s = torch.empty((cap, 3, 512), dtype=torch.float64, device=self.device)
        bg = torch.empty(self.tiles, dtype=torch.uint8, device=self.device)
        _check(self.ctx, lib.ebit_pack_bricks(self.ctx, cap, _dev(t, torch.int32), _dev(cb, torch.uint8),
                                              _dev(s, torch.float64), _dev(bg, torch.uint8), ctypes.byref(n)))
        k = int(n.value)
        return {"tiles": t[:k], "cb": cb[:k], "s": s[:k], "bg": bg}

    def unpack_bricks(self, store):
        """Replace the state with the one a brick store describes."""
        t, cb, s, bg = store["tiles"], store["cb"], store["s"], store["bg"]
        k = int(t.numel())
        if bg.numel() != self.tiles:
            raise ValueError(f"bg must have {self.tiles} entries")
        return _check(self.ctx, load().ebit_unpack_bricks(
            self.ctx, k, _dev(t.contiguous(), torch.int32) if k else None,
            _dev(cb.contiguous(), torch.uint8) if k else None, _dev(s.contiguous(), torch.float64) if k else None,
            _dev(bg.contiguous(), torch.uint8)))

    def profile(self, enable=True):
        return ebit_profile(self.ctx, enable)

    def profile_read(self):
        return ebit_profile_read(self.ctx)
