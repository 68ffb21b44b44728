"""FP64 CPU oracle for the short-range non-bonded path (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library and its Python binding never touch it, and it shares no code with
them: the arithmetic lives in ``nb_oracle.c`` (plain C, FP64), compiled with
gcc into ``oracle/_build/liboracle.so``.

Functions here only marshal NumPy arrays into the C routines; each C routine
cites the passage it follows.
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ewald_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CLUSTER = 8


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, FP contraction off so FP32 predicates round
    exactly as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *_SRCS, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            F = ctypes.c_float
            I = ctypes.c_int
            D = ctypes.c_double
            common = [I64, P, P, P, I, P, P, P, F, F, F, F, F, F, I64, P, I64, P]
            L.orc_forces_allpairs.argtypes = common + [P, P, P]
            L.orc_forces_allpairs.restype = I64
            L.orc_forces_cells.argtypes = common + [P, P, P]
            L.orc_forces_cells.restype = I64
            L.orc_forces_subset.argtypes = common + [I64, P, P, P, P]
            L.orc_forces_subset.restype = None
            L.orc_backward_allpairs.argtypes = common + [P, D, P, P, P, P, P, P]
            L.orc_backward_allpairs.restype = I64
            L.orc_pair_terms.argtypes = [I64, P, P, P, P, P, P, I, P, P, F, F, F, F, P]
            L.orc_pair_terms.restype = None
            L.orc_pairs.argtypes = [I64, P, P, F, I64, P, I64, P, I64, P]
            L.orc_pairs.restype = I64
            L.orc_combine_lb.argtypes = [I, P, P, P, P, P, P]
            L.orc_combine_lb.restype = None
            L.orc_lb_chain.argtypes = [I, P, P, P, P, P, P, P, P, P]
            L.orc_lb_chain.restype = None
            L.orc_wrap_f32.argtypes = [I64, P, P]
            L.orc_wrap_f32.restype = None
            L.orc_binning.argtypes = [I64, P, P, P, P]
            L.orc_binning.restype = I64
            L.orc_grid_dims.argtypes = [I64, P, P, P]
            L.orc_grid_dims.restype = None
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = I
            L.orc_set_threads.argtypes = [I]
            L.orc_set_threads.restype = None
            L.orc_set_table.argtypes = [I]
            L.orc_set_table.restype = None
            L.orc_ewald_recip.argtypes = [I64, P, P, P, D, D, I, I, I, P, P, P]
            L.orc_ewald_recip.restype = I
            L.orc_ewald_corrections.argtypes = [I64, P, P, P, D, D, I64, P, I64, P, D, P, P, P]
            L.orc_ewald_corrections.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (timing only)."""
    lib().orc_set_threads(int(n))


@contextlib.contextmanager
def tabulated(n: int):
    """Within the block, the forward functions (forces, forces_subset)
    evaluate the radial functions by linear interpolation of n-interval
    tables on [0, rc] instead of directly (see nb_oracle.c, tab_t)."""
    lib().orc_set_table(int(n))
    try:
        yield
    finally:
        lib().orc_set_table(0)


def combine_lb(sigma, epsilon):
    """Lorentz-Berthelot type-pair tables (sig_tab, eps_tab, A, B), FP64 [T, T]."""
    s = _c(sigma, np.float32)
    e = _c(epsilon, np.float32)
    T = s.shape[0]
    out = [np.zeros((T, T)) for _ in range(4)]
    lib().orc_combine_lb(T, _p(s), _p(e), *[_p(o) for o in out])
    return tuple(out)


def _args(sys, pos=None, q=None):
    pos = _c(sys.pos if pos is None else pos, np.float32)
    q = _c(sys.q if q is None else q, np.float32)
    typ = _c(sys.type, np.int32)
    _, _, A, B = combine_lb(sys.sigma, sys.epsilon)
    box = _c(sys.box, np.float32)
    ex = _c(sys.excl, np.int32).reshape(-1, 2)
    p14 = _c(sys.pairs14, np.int32).reshape(-1, 2)
    keep = (pos, q, typ, A, B, box, ex, p14)
    args = [pos.shape[0], _p(pos), _p(q), _p(typ), sys.n_types, _p(A), _p(B), _p(box),
            sys.cutoff, sys.switch_dist, sys.ewald_alpha, sys.coulomb_k,
            sys.scale14_lj, sys.scale14_coul, ex.shape[0], _p(ex), p14.shape[0], _p(p14)]
    return args, keep


def forces(sys, method: str = "allpairs", pos=None, q=None, with_scale: bool = False, with_sq: bool = False):
    """FP64 forces [N,3], energies (E_LJ, E_Coul), virial [6] and pair count.

    method: "allpairs" (plain O(N^2) sum) or "cells" (cell-list traversal).
    with_scale: also return (sum |e_LJ|, sum |e_Coul|) over pairs, the scale
    of the rounding error of each summed energy.
    with_sq (with with_scale): then also (sum e_LJ^2, sum e_Coul^2), the
    scale of the random part of that error.
    """
    args, keep = _args(sys, pos, q)
    n = args[0]
    F = np.zeros((n, 3))
    E = np.zeros(6)
    W = np.zeros(6)
    fn = lib().orc_forces_allpairs if method == "allpairs" else lib().orc_forces_cells
    npairs = fn(*args, _p(F), _p(E), _p(W))
    del keep
    if with_scale and with_sq:
        return F, E[:2].copy(), W, int(npairs), E[2:4].copy(), E[4:6].copy()
    if with_scale:
        return F, E[:2].copy(), W, int(npairs), E[2:4].copy()
    return F, E[:2].copy(), W, int(npairs)


def pair_terms(sys, xi, xj, qi, qj, ti, tj):
    """FP64 terms of given pairs with unit weights: [m, 4] = (E_LJ, E_Coul,
    dU/dr, A r^-12 + B r^-6), d = x_j - x_i as given (see nb_oracle.c,
    orc_pair_terms)."""
    xi, xj = _c(xi, np.float32), _c(xj, np.float32)
    qi, qj = _c(qi, np.float32), _c(qj, np.float32)
    ti, tj = _c(ti, np.int32), _c(tj, np.int32)
    _, _, A, B = combine_lb(sys.sigma, sys.epsilon)
    m = xi.shape[0]
    out = np.zeros((m, 4))
    lib().orc_pair_terms(m, _p(xi), _p(xj), _p(qi), _p(qj), _p(ti), _p(tj), sys.n_types, _p(A), _p(B),
                         sys.cutoff, sys.switch_dist, sys.ewald_alpha, sys.coulomb_k, _p(out))
    return out


def forces_subset(sys, atoms, pos=None, q=None):
    """FP64 forces and half pair energies on selected atoms only."""
    args, keep = _args(sys, pos, q)
    at = _c(atoms, np.int64)
    m = at.shape[0]
    F = np.zeros((m, 3))
    E4 = np.zeros((m, 6))
    npair = np.zeros(m, np.int64)
    lib().orc_forces_subset(*args, m, _p(at), _p(F), _p(E4), _p(npair))
    del keep
    return F, E4[:, :2].copy(), npair


def backward(sys, G, gE: float = 0.0, pos=None, q=None, with_scale: bool = False):
    """Adjoint of L = sum G.F + gE*E: dL/dx [N,3], dL/dq [N], dL/dA, dL/dB [T,T]
    (and, with with_scale, the sums of |pair contribution| of dL/dA, dL/dB)."""
    args, keep = _args(sys, pos, q)
    n = args[0]
    T = sys.n_types
    Gd = _c(G, np.float64)
    dx = np.zeros((n, 3))
    dq = np.zeros(n)
    dA = np.zeros((T, T))
    dB = np.zeros((T, T))
    aA = np.zeros((T, T))
    aB = np.zeros((T, T))
    lib().orc_backward_allpairs(*args, _p(Gd), float(gE), _p(dx), _p(dq), _p(dA), _p(dB), _p(aA), _p(aB))
    del keep
    if with_scale:
        return dx, dq, dA, dB, aA, aB
    return dx, dq, dA, dB


def lb_chain(sys, dA, dB):
    """(dL/dsig_tab, dL/deps_tab, dL/dsigma_t, dL/deps_t) from table gradients."""
    sig_tab, eps_tab, _, _ = combine_lb(sys.sigma, sys.epsilon)
    T = sys.n_types
    e = _c(sys.epsilon, np.float32)
    dA = _c(dA, np.float64)
    dB = _c(dB, np.float64)
    dst = np.zeros((T, T))
    det = np.zeros((T, T))
    ds = np.zeros(T)
    de = np.zeros(T)
    lib().orc_lb_chain(T, _p(sig_tab), _p(eps_tab), _p(dA), _p(dB), _p(e), _p(dst), _p(det), _p(ds), _p(de))
    return dst, det, ds, de


def pairs(sys, pos=None, cap: int | None = None):
    """Unique in-range, non-excluded pairs (i < j) as int32 [M, 2], sorted."""
    pos = _c(sys.pos if pos is None else pos, np.float32)
    box = _c(sys.box, np.float32)
    ex = _c(sys.excl, np.int32).reshape(-1, 2)
    p14 = _c(sys.pairs14, np.int32).reshape(-1, 2)
    L = lib()
    if cap is None:
        cap = 0
        cap = int(L.orc_pairs(pos.shape[0], _p(pos), _p(box), sys.cutoff, ex.shape[0], _p(ex),
                              p14.shape[0], _p(p14), 0, None))
    ij = np.zeros((max(cap, 1), 2), np.int32)
    n = int(L.orc_pairs(pos.shape[0], _p(pos), _p(box), sys.cutoff, ex.shape[0], _p(ex),
                        p14.shape[0], _p(p14), cap, _p(ij)))
    ij = ij[:min(n, cap)]
    order = np.lexsort((ij[:, 1], ij[:, 0]))
    return ij[order]


def wrap_f32(pos, box):
    p = _c(pos, np.float32).copy()
    b = _c(box, np.float32)
    lib().orc_wrap_f32(p.shape[0], _p(p), _p(b))
    return p


def grid_dims(n: int, box):
    b = _c(box, np.float32)
    nx = ctypes.c_int()
    ny = ctypes.c_int()
    lib().orc_grid_dims(n, _p(b), ctypes.byref(nx), ctypes.byref(ny))
    return nx.value, ny.value


def binning(pos, box):
    """Sorted slot order (padding = -1) and padded column starts of one system."""
    p = _c(pos, np.float32)
    b = _c(box, np.float32)
    n = p.shape[0]
    nx, ny = grid_dims(n, b)
    perm = np.full(n + (CLUSTER - 1) * nx * ny + CLUSTER, -1, np.int64)
    cs = np.zeros(nx * ny + 1, np.int64)
    npad = int(lib().orc_binning(n, _p(p), _p(b), _p(perm), _p(cs)))
    return perm[:npad], cs, (nx, ny)
