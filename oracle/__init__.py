"""CPU FP64 oracle for the 3D EBIT kinematics path (arxiv 2509.26361).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2509_26361_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``ebit_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so every operation rounds separately, in the written order).
This module compiles it with gcc on first use and exposes numpy-level functions.

State layout (a documented format, not shared code): arrays are indexed
``[k, j, i]`` (x fastest).  ``cb`` is the packed colour byte per node -- bit 0 the
node colour, bit 1+a the colour of the face normal to axis ``a`` whose lowest
corner is that node.  ``s`` has shape ``(3, nz, ny, nx)``: ``s[a]`` the marker
offset on the a-edge leaving each node (0 when the edge carries no marker).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebit_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libebit_oracle.so")
_lock = threading.Lock()
_lib = None

CNT_NAMES = ("markers", "annihilate", "multi", "inconsistent", "cfl")


def build(force: bool = False) -> str:
    """Compile the oracle C source into a shared library (gcc, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.oracle_init.argtypes = [I, I, I, P, P, P, P, P]
            lib.oracle_init.restype = None
            lib.oracle_sweep.argtypes = [I, I, I, I, P, D, P, P, P, P, P]
            lib.oracle_sweep.restype = None
            lib.oracle_front2vof.argtypes = [I, I, I, P, P, P]
            lib.oracle_front2vof.restype = ctypes.c_long
            lib.oracle_hf.argtypes = [I, I, I, P, P, P]
            lib.oracle_hf.restype = None
            lib.oracle_surface_volume.argtypes = [I, I, I, P, P, P]
            lib.oracle_surface_volume.restype = D
            lib.oracle_cube_volume.argtypes = [P, P, P, P, P]
            lib.oracle_cube_volume.restype = D
            lib.oracle_circle_root.argtypes = [P, D, P]
            lib.oracle_circle_root.restype = D
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(cb: np.ndarray):
    nz, ny, nx = cb.shape
    return nx, ny, nz


class State:
    """EBIT state on the host: packed colour bytes + FP64 edge offsets."""

    def __init__(self, cb: np.ndarray, s: np.ndarray):
        assert cb.dtype == np.uint8 and cb.ndim == 3
        assert s.dtype == np.float64 and s.shape == (3,) + cb.shape
        self.cb = np.ascontiguousarray(cb)
        self.s = np.ascontiguousarray(s)

    def copy(self) -> "State":
        return State(self.cb.copy(), self.s.copy())

    @property
    def shape(self):
        return self.cb.shape

    def node_colour(self) -> np.ndarray:
        return self.cb & 1

    def face_colour(self, a: int) -> np.ndarray:
        return (self.cb >> (1 + a)) & 1


def init(phi_nodes: np.ndarray, phi_faces: np.ndarray | None = None,
         s_exact: np.ndarray | None = None) -> State:
    """Markers from a level set sampled at the nodes (colour = phi >= 0; linear root).

    ``phi_faces`` (shape (3, nz, ny, nx)) gives phi at the face centres, used for the
    colour of saddle faces; if None the mean of the 4 corner values is used.
    ``s_exact`` (same shape, NaN where absent) overrides the linear root on
    sign-change edges with a given offset (exact shape intersections).
    """
    phi = np.ascontiguousarray(phi_nodes, dtype=np.float64)
    nx, ny, nz = phi.shape[2], phi.shape[1], phi.shape[0]
    cb = np.zeros(phi.shape, np.uint8)
    s = np.zeros((3,) + phi.shape, np.float64)
    pf = None if phi_faces is None else np.ascontiguousarray(phi_faces, dtype=np.float64)
    se = None if s_exact is None else np.ascontiguousarray(s_exact, dtype=np.float64)
    _load().oracle_init(nx, ny, nz, _ptr(phi), None if pf is None else _ptr(pf),
                        None if se is None else _ptr(se), _ptr(cb), _ptr(s))
    return State(cb, s)


def sweep(st: State, d: int, u: np.ndarray, lam: float) -> tuple[State, np.ndarray]:
    """One split advection along axis d.  ``u``: u_d on the d-normal faces (same
    indexing as nodes); ``lam`` = dt/h.  Returns the new state and the counters."""
    nx, ny, nz = _dims(st.cb)
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == st.cb.shape
    cb2 = np.zeros_like(st.cb)
    s2 = np.zeros_like(st.s)
    cnt = np.zeros(len(CNT_NAMES), np.int64)
    _load().oracle_sweep(nx, ny, nz, int(d), _ptr(u), float(lam), _ptr(st.cb), _ptr(st.s),
                         _ptr(cb2), _ptr(s2), _ptr(cnt))
    return State(cb2, s2), cnt


def front2vof(st: State) -> tuple[np.ndarray, int]:
    """Volume fraction of every cell; returns (C, number of inconsistent cells)."""
    nx, ny, nz = _dims(st.cb)
    C = np.zeros(st.cb.shape, np.float64)
    nbad = _load().oracle_front2vof(nx, ny, nz, _ptr(st.cb), _ptr(st.s), _ptr(C))
    return C, int(nbad)


def hf_curvature(C: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Height-function kappa*h and status (0 none, 1+d axis d, 4 no stencil)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    nz, ny, nx = C.shape
    kh = np.zeros_like(C)
    stt = np.zeros(C.shape, np.uint8)
    _load().oracle_hf(nx, ny, nz, _ptr(C), _ptr(kh), _ptr(stt))
    return kh, stt


def surface_volume(st: State) -> tuple[float, int]:
    """Volume enclosed by all fan triangles, with one global origin (cell units)."""
    nx, ny, nz = _dims(st.cb)
    nt = ctypes.c_long(0)
    v = _load().oracle_surface_volume(nx, ny, nz, _ptr(st.cb), _ptr(st.s), ctypes.byref(nt))
    return float(v), int(nt.value)


def cube_volume(K, F, E) -> tuple[float, int, int]:
    """Volume fraction of one unit cube from 8 corner colours (id = dx|dy<<1|dz<<2),
    6 face colours (x0,x1,y0,y1,z0,z1) and 12 edge offsets (x: dy+2dz, y: 4+dx+2dz,
    z: 8+dx+2dy).  Returns (C, loops, bad)."""
    K = np.ascontiguousarray(K, dtype=np.int32)
    F = np.ascontiguousarray(F, dtype=np.int32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    nl = ctypes.c_int(0)
    bad = ctypes.c_int(0)
    v = _load().oracle_cube_volume(_ptr(K), _ptr(F), _ptr(E), ctypes.byref(nl), ctypes.byref(bad))
    return float(v), int(nl.value), int(bad.value)


def circle_root(P1, P2, P3, P4, ylin: float) -> tuple[float, int]:
    """Circle-fit crossing of the grid line x = 0 (returns y and a validity mask:
    bit 0 circle P1P2P3, bit 1 circle P2P3P4)."""
    P = np.ascontiguousarray(np.array([P1, P2, P3, P4], dtype=np.float64).ravel())
    w = ctypes.c_int(0)
    y = _load().oracle_circle_root(_ptr(P), float(ylin), ctypes.byref(w))
    return float(y), int(w.value)


def step(st: State, n: int, u_fields, lam: float, counters: np.ndarray | None = None) -> State:
    """One full time step: three split sweeps, x-y-z on even steps and z-y-x on odd
    steps.  ``u_fields[d]`` is u_d on the d-normal faces; ``lam`` = dt/h (may carry a
    time factor)."""
    order = (0, 1, 2) if n % 2 == 0 else (2, 1, 0)
    for d in order:
        st, c = sweep(st, d, u_fields[d], lam)
        if counters is not None:
            counters += c
    return st


def e_mass(C_series_sums, C0_sum: float) -> float:
    """Mass error (Eq. 9): time-averaged |V(t) - V(0)| / V(0)."""
    sums = np.asarray(C_series_sums, dtype=np.float64)
    return float(np.mean(np.abs(sums - C0_sum)) / C0_sum)


def e_shape(C_T: np.ndarray, C_0: np.ndarray) -> float:
    """Shape error (Eq. 10): L1 difference of volume fractions over the initial volume."""
    return float(np.sum(np.abs(C_T - C_0)) / np.sum(C_0))
