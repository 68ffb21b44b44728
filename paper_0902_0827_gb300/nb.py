"""Python binding of the C ABI in ``include/acenb.h`` (argument marshalling only).

Every step of the computation runs in the CUDA library ``_build/libacenb.so``.
PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback: if the library cannot be loaded, :func:`lib` raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import build as _build

NB_OK = 0
STATUS_NAMES = {
    0: "NB_OK", 1: "NB_ERR_INVALID_ARG", 2: "NB_ERR_BOX_TOO_SMALL", 3: "NB_ERR_CUDA", 4: "NB_ERR_OOM",
    5: "NB_ERR_NOT_BUILT", 6: "NB_ERR_OVERFLOW", 7: "NB_ERR_LIST_STALE", 8: "NB_ERR_TIMEOUT",
    9: "NB_ERR_NONFINITE", 10: "NB_ERR_CAPACITY", 11: "NB_ERR_UNSUPPORTED", 12: "NB_ERR_TOO_LARGE",
}
# every symbol include/acenb.h declares
EXPORTS = ("nb_create", "nb_create_batch", "nb_build_cells", "nb_forces", "nb_forces_batch", "nb_step", "nb_backward",
           "nb_get_status", "nb_set_stream", "nb_destroy", "nb_set_tuning", "nb_get_tuning", "nb_get_sizes",
           "nb_debug_cells", "nb_debug_pairs", "nb_debug_fill", "nb_debug_pair_terms", "nb_debug_philox", "nb_status_string",
           "nb_set_lj_params", "nb_set_profiling", "nb_get_profile", "nb_forces_noalloc", "nb_type_gradients",
           "nb_set_pme", "nb_pme_forces", "nb_set_tables", "nb_md_init", "nb_md_step", "nb_md_minimize",
           "nb_bonded_forces",
           "nb_md_set_step", "nb_fp32_peak_launch")


class NbError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        name = STATUS_NAMES.get(code, str(code))
        super().__init__(f"{where}: {name}" if where else name)


class nb_params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("box", ctypes.c_float * 3), ("cutoff", ctypes.c_float),
        ("switch_dist", ctypes.c_float), ("ewald_alpha", ctypes.c_float), ("coulomb_k", ctypes.c_float),
        ("n_types", ctypes.c_int32), ("sigma", ctypes.c_void_p), ("epsilon", ctypes.c_void_p),
        ("comb_rule", ctypes.c_int32), ("sigma_tab", ctypes.c_void_p), ("eps_tab", ctypes.c_void_p),
        ("n_excl", ctypes.c_int32), ("excl", ctypes.c_void_p), ("n_14", ctypes.c_int32),
        ("pairs14", ctypes.c_void_p), ("scale14_lj", ctypes.c_float), ("scale14_coul", ctypes.c_float),
        ("flags", ctypes.c_uint32),
    ]


class nb_tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("stage_capacity", ctypes.c_int32),
                ("list_capacity", ctypes.c_int32), ("list_split", ctypes.c_int32),
                ("group_clusters", ctypes.c_int32)]


class nb_pme_params(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32 * 3), ("order", ctypes.c_int32), ("flags", ctypes.c_int32)]


class nb_md_params(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_void_p),
        ("n_bonds", ctypes.c_int32), ("bonds", ctypes.c_void_p), ("bond_k", ctypes.c_void_p),
        ("bond_r0", ctypes.c_void_p),
        ("n_angles", ctypes.c_int32), ("angles", ctypes.c_void_p), ("angle_k", ctypes.c_void_p),
        ("angle_theta0", ctypes.c_void_p),
        ("n_dihedrals", ctypes.c_int32), ("dihedrals", ctypes.c_void_p), ("dihedral_k", ctypes.c_void_p),
        ("dihedral_n", ctypes.c_void_p), ("dihedral_phase", ctypes.c_void_p),
        ("n_waters", ctypes.c_int32), ("waters", ctypes.c_void_p), ("water_roh", ctypes.c_float),
        ("water_rhh", ctypes.c_float),
        ("dt", ctypes.c_float), ("gamma", ctypes.c_float), ("temperature", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("shake_max_iter", ctypes.c_int32), ("shake_tolerance", ctypes.c_float),
        ("flags", ctypes.c_uint32),
    ]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"CUDA library not built: {path}")
            _build.build()
        L = ctypes.CDLL(path)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "nb_create": ([ctypes.POINTER(nb_params), P, ctypes.POINTER(P)], ctypes.c_int),
            "nb_create_batch": ([I32, ctypes.POINTER(nb_params), P, ctypes.POINTER(P)], ctypes.c_int),
            "nb_build_cells": ([P, P], ctypes.c_int),
            "nb_forces": ([P, P, P, P, P, P, P], ctypes.c_int),
            "nb_forces_batch": ([P, P, P, P, P, P, P], ctypes.c_int),
            "nb_step": ([P, P, P, P, P, P, P], ctypes.c_int),
            "nb_backward": ([P, P, P, P, P, P, P, P, P, P], ctypes.c_int),
            "nb_get_status": ([P], ctypes.c_int),
            "nb_set_stream": ([P, P], ctypes.c_int),
            "nb_destroy": ([P], None),
            "nb_set_tuning": ([P, ctypes.POINTER(nb_tuning)], ctypes.c_int),
            "nb_get_tuning": ([P, ctypes.POINTER(nb_tuning)], ctypes.c_int),
            "nb_get_sizes": ([P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I64)], ctypes.c_int),
            "nb_debug_cells": ([P, P, ctypes.POINTER(I64), P, ctypes.POINTER(I64)], ctypes.c_int),
            "nb_debug_pairs": ([P, P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64)], ctypes.c_int),
            "nb_debug_fill": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64)], ctypes.c_int),
            "nb_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "nb_set_lj_params": ([P, P, P, P, P], ctypes.c_int),
            "nb_set_profiling": ([P, I32], ctypes.c_int),
            "nb_get_profile": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)], ctypes.c_int),
            "nb_forces_noalloc": ([ctypes.POINTER(nb_params), P, P, P, P, P, P, P], ctypes.c_int),
            "nb_type_gradients": ([P, P, P, P, P], ctypes.c_int),
            "nb_set_pme": ([P, ctypes.POINTER(nb_pme_params)], ctypes.c_int),
            "nb_pme_forces": ([P, P, P, P, P, P], ctypes.c_int),
            "nb_set_tables": ([P, I32], ctypes.c_int),
            "nb_md_init": ([P, ctypes.POINTER(nb_md_params)], ctypes.c_int),
            "nb_md_step": ([P, P, P, P, P, I32, P], ctypes.c_int),
            "nb_md_minimize": ([P, P, P, P, I32, ctypes.c_float, P], ctypes.c_int),
            "nb_bonded_forces": ([P, P, P, P], ctypes.c_int),
            "nb_md_set_step": ([P, ctypes.c_uint64], ctypes.c_int),
            "nb_debug_pair_terms": ([P, I64, P, P, P, P, P], ctypes.c_int),
            "nb_debug_philox": ([I64, P, P, P, P], ctypes.c_int),
            "nb_fp32_peak_launch": ([I64, P, P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != NB_OK:
        raise NbError(code, where)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _tptr(t, host_ok=False):
    """Device pointer of a contiguous CUDA tensor (None passes NULL).  With
    host_ok, a contiguous page-locked CPU tensor is accepted too: under
    unified addressing its address is also its device address, and the
    kernels read and write it across the host link."""
    if t is None:
        return None
    ok = t.is_cuda or (host_ok and t.device.type == "cpu" and t.is_pinned())
    if not ok or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor" + (" or page-locked CPU tensor" if host_ok else ""))
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_params(systems):
    """nb_params array for a list of systems plus the host arrays it points to
    (keep them alive until the library has copied them)."""
    keep = []
    arr = (nb_params * len(systems))()
    for k, s in enumerate(systems):
        sig, eps = _f32(s.sigma), _f32(s.epsilon)
        ex, p14 = _i32(s.excl).reshape(-1, 2), _i32(s.pairs14).reshape(-1, 2)
        keep += [sig, eps, ex, p14]
        p = arr[k]
        p.n_atoms = int(s.n_atoms)
        for a in range(3):
            p.box[a] = float(s.box[a])
        p.cutoff, p.switch_dist = float(s.cutoff), float(s.switch_dist)
        p.ewald_alpha, p.coulomb_k = float(s.ewald_alpha), float(s.coulomb_k)
        p.n_types = int(sig.shape[0])
        p.sigma, p.epsilon = _ptr(sig), _ptr(eps)
        p.comb_rule = 0
        p.n_excl, p.excl = int(ex.shape[0]), _ptr(ex)
        p.n_14, p.pairs14 = int(p14.shape[0]), _ptr(p14)
        p.scale14_lj, p.scale14_coul = float(s.scale14_lj), float(s.scale14_coul)
        p.flags = 0
    return arr, keep


def forces_noalloc(system, pos, q, typ, F, energy=None, virial=None):
    """nb_forces_noalloc: one small system, no device allocation by the library
    (scratch in its static device array).  Outputs are caller-owned tensors."""
    arr, keep = make_params([system])
    code = lib().nb_forces_noalloc(arr, _tptr(pos), _tptr(q), _tptr(typ), _tptr(F), _tptr(energy),
                                   _tptr(virial), _stream_handle())
    del keep
    _check(code, "nb_forces_noalloc")


class Nonbonded:
    """One context of the library: a single system or a batch of systems.

    ``systems`` are objects with the attributes of
    :class:`paper_0902_0827_gb300.systems.System` (box, cutoff, switch_dist,
    ewald_alpha, coulomb_k, sigma, epsilon, excl, pairs14, scale factors and
    n_atoms).  For a batch, per-atom tensors are the systems' arrays
    concatenated in order.
    """

    def __init__(self, systems, stream=None):
        L = lib()
        single = not isinstance(systems, (list, tuple))
        self.systems = [systems] if single else list(systems)
        arr, self._keep = make_params(self.systems)
        h = ctypes.c_void_p()
        st = stream if stream is not None else _stream_handle()
        _check(L.nb_create_batch(len(self.systems), arr, st, ctypes.byref(h)), "nb_create_batch")
        self._keep = []
        self.h = h
        self.n_sys = len(self.systems)
        self.n_atoms = int(sum(s.n_atoms for s in self.systems))
        self.n_types = int(self.systems[0].sigma.shape[0])

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            lib().nb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        lib().nb_set_stream(self.h, _stream_handle())

    # -- compute ---------------------------------------------------------
    def build(self, pos):
        self._sync_stream()
        _check(lib().nb_build_cells(self.h, _tptr(pos)), "nb_build_cells")

    def forces(self, pos, q, typ, F=None, energy=True, virial=True):
        """Forces [N,3] (FP32), energies [n_sys,2] and virials [n_sys,6] (FP64)."""
        import torch
        self._sync_stream()
        dev = pos.device
        if F is None:
            F = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=dev)
        E = torch.empty((self.n_sys, 2), dtype=torch.float64, device=dev) if energy is True else energy
        W = torch.empty((self.n_sys, 6), dtype=torch.float64, device=dev) if virial is True else virial
        E = E if E is not False else None
        W = W if W is not False else None
        _check(lib().nb_forces(self.h, _tptr(pos), _tptr(q), _tptr(typ), _tptr(F), _tptr(E), _tptr(W)),
               "nb_forces")
        return F, E, W

    def step(self, pos, q, typ, F=None, energy=True, virial=True):
        """Rebuild from pos and evaluate (nb_step): the results of
        build(pos) followed by forces(pos, q, typ), in fewer kernels.  The
        arrays may be CUDA tensors or page-locked CPU tensors (read and
        written by the kernels in place; results are there once the stream
        has completed); new outputs go where pos is."""
        import torch
        self._sync_stream()
        dev = pos.device
        pin = dev.type == "cpu"

        def new(shape, dtype):
            return torch.empty(shape, dtype=dtype, device=dev, pin_memory=pin)

        if F is None:
            F = new((self.n_atoms, 3), torch.float32)
        E = new((self.n_sys, 2), torch.float64) if energy is True else energy
        W = new((self.n_sys, 6), torch.float64) if virial is True else virial
        E = E if E is not False else None
        W = W if W is not False else None
        _check(lib().nb_step(self.h, _tptr(pos, True), _tptr(q, True), _tptr(typ, True), _tptr(F, True),
                             _tptr(E, True), _tptr(W, True)), "nb_step")
        return F, E, W

    def set_tables(self, n_intervals: int = 4096):
        """Radial functions by linear interpolation of n-interval tables on
        [0, rc] (0 restores direct evaluation)."""
        _check(lib().nb_set_tables(self.h, int(n_intervals)), "nb_set_tables")

    def md_init(self, top, dt=0.002, gamma=1.0, temperature=300.0, seed=2009, shake_max_iter=10,
                shake_tolerance=1e-6):
        """Attach the MD state: ``top`` has the attributes of
        :class:`paper_0902_0827_gb300.systems.MDTopology`."""
        keep = []

        def arr(a, dt_):
            a = np.ascontiguousarray(a, dtype=dt_)
            keep.append(a)
            return _ptr(a)

        p = nb_md_params()
        p.mass = arr(top.mass, np.float32)
        p.n_bonds = len(top.bonds)
        p.bonds, p.bond_k, p.bond_r0 = arr(top.bonds, np.int32), arr(top.bond_k, np.float32), arr(top.bond_r0, np.float32)
        p.n_angles = len(top.angles)
        p.angles, p.angle_k = arr(top.angles, np.int32), arr(top.angle_k, np.float32)
        p.angle_theta0 = arr(top.angle_theta0, np.float32)
        p.n_dihedrals = len(top.dihedrals)
        p.dihedrals, p.dihedral_k = arr(top.dihedrals, np.int32), arr(top.dihedral_k, np.float32)
        p.dihedral_n, p.dihedral_phase = arr(top.dihedral_n, np.int32), arr(top.dihedral_phase, np.float32)
        p.n_waters = len(top.waters)
        p.waters = arr(top.waters, np.int32)
        p.water_roh, p.water_rhh = float(top.water_roh), float(top.water_rhh)
        p.dt, p.gamma, p.temperature = float(dt), float(gamma), float(temperature)
        p.seed, p.shake_max_iter, p.shake_tolerance, p.flags = int(seed), int(shake_max_iter), float(shake_tolerance), 0
        _check(lib().nb_md_init(self.h, ctypes.byref(p)), "nb_md_init")
        del keep

    def md_step(self, pos, vel, q, typ, n_steps=1, energy=None):
        """Advance pos and vel (CUDA FP32 [N,3], in place) by n_steps; energy
        (FP64 [6] tensor or None) receives E_LJ, E_Coul, E_bond, E_angle,
        E_dihedral, E_kin after the last step."""
        self._sync_stream()
        _check(lib().nb_md_step(self.h, _tptr(pos), _tptr(vel), _tptr(q), _tptr(typ), int(n_steps), _tptr(energy)),
               "nb_md_step")

    def md_minimize(self, pos, q, typ, n_steps, max_disp=0.01, energy=None):
        """Capped steepest descent of pos (CUDA FP32 [N,3], in place) over
        n_steps moves of at most max_disp A; energy (FP64 [6] tensor or None)
        receives the energies at the final positions."""
        self._sync_stream()
        _check(lib().nb_md_minimize(self.h, _tptr(pos), _tptr(q), _tptr(typ), int(n_steps), float(max_disp),
                                    _tptr(energy)), "nb_md_minimize")

    def bonded_forces(self, pos):
        import torch
        self._sync_stream()
        F = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=pos.device)
        E = torch.empty((3,), dtype=torch.float64, device=pos.device)
        _check(lib().nb_bonded_forces(self.h, _tptr(pos), _tptr(F), _tptr(E)), "nb_bonded_forces")
        return F, E

    def md_set_step(self, step: int):
        _check(lib().nb_md_set_step(self.h, int(step)), "nb_md_set_step")

    def set_pme(self, grid=None, order: int = 4):
        """Enable smooth PME on the grid (K1, K2, K3) with B-splines of the
        given order (nb_forces then returns the full Ewald electrostatics), or
        disable it with grid=None."""
        if grid is None:
            _check(lib().nb_set_pme(self.h, None), "nb_set_pme")
            return
        p = nb_pme_params()
        for a in range(3):
            p.grid[a] = int(grid[a])
        p.order, p.flags = int(order), 0
        _check(lib().nb_set_pme(self.h, ctypes.byref(p)), "nb_set_pme")

    def pme_forces(self, pos, q, F=None):
        """Long-range part alone: forces [N,3] (FP32), energies (E_recip,
        E_self, E_excl) and virial [6] (FP64)."""
        import torch
        self._sync_stream()
        dev = pos.device
        if F is None:
            F = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=dev)
        E = torch.empty((3,), dtype=torch.float64, device=dev)
        W = torch.empty((6,), dtype=torch.float64, device=dev)
        _check(lib().nb_pme_forces(self.h, _tptr(pos), _tptr(q), _tptr(F), _tptr(E), _tptr(W)), "nb_pme_forces")
        return F, E, W

    def backward(self, pos, q, typ, dLdF, dLdE=None, want=("pos", "q", "sig", "eps")):
        import torch
        self._sync_stream()
        dev = pos.device
        T = self.n_types
        gpos = torch.empty((self.n_atoms, 3), dtype=torch.float32, device=dev) if "pos" in want else None
        gq = torch.empty((self.n_atoms,), dtype=torch.float32, device=dev) if "q" in want else None
        gs = torch.empty((T, T), dtype=torch.float64, device=dev) if "sig" in want else None
        ge = torch.empty((T, T), dtype=torch.float64, device=dev) if "eps" in want else None
        _check(lib().nb_backward(self.h, _tptr(pos), _tptr(q), _tptr(typ), _tptr(dLdF), _tptr(dLdE),
                                 _tptr(gpos), _tptr(gq), _tptr(gs), _tptr(ge)), "nb_backward")
        return gpos, gq, gs, ge

    def type_gradients(self, gsig_tab, geps_tab):
        """Per-type (sigma, epsilon) gradients from type-pair gradients (Lorentz-Berthelot)."""
        import torch
        gs = torch.empty((self.n_types,), dtype=torch.float64, device=gsig_tab.device)
        ge = torch.empty((self.n_types,), dtype=torch.float64, device=gsig_tab.device)
        self._sync_stream()
        _check(lib().nb_type_gradients(self.h, _tptr(gsig_tab.contiguous()), _tptr(geps_tab.contiguous()),
                                       _tptr(gs), _tptr(ge)), "nb_type_gradients")
        return gs, ge

    def set_lj_params(self, sigma, epsilon):
        """Replace the per-type LJ parameters (Lorentz-Berthelot) of the context."""
        sig, eps = _f32(sigma), _f32(epsilon)
        _check(lib().nb_set_lj_params(self.h, _ptr(sig), _ptr(eps), None, None), "nb_set_lj_params")

    def status(self, raise_on_error: bool = True) -> int:
        code = int(lib().nb_get_status(self.h))
        if raise_on_error and code != NB_OK:
            raise NbError(code, "device status")
        return code

    def set_profiling(self, on: bool):
        _check(lib().nb_set_profiling(self.h, int(bool(on))), "nb_set_profiling")

    def profile(self):
        """(summed force-kernel milliseconds, launches) since profiling was enabled."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().nb_get_profile(self.h, ctypes.byref(ms), ctypes.byref(n)), "nb_get_profile")
        return ms.value, n.value

    # -- tuning / debug --------------------------------------------------
    def tuning(self) -> dict:
        t = nb_tuning()
        _check(lib().nb_get_tuning(self.h, ctypes.byref(t)), "nb_get_tuning")
        return {k: getattr(t, k) for k, _ in nb_tuning._fields_}

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        t = nb_tuning(**cur)
        _check(lib().nb_set_tuning(self.h, ctypes.byref(t)), "nb_set_tuning")

    def sizes(self):
        n, s, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().nb_get_sizes(self.h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(c)), "nb_get_sizes")
        return n.value, s.value, c.value

    def debug_cells(self):
        _, _, cap = self.sizes()
        perm = np.empty(cap, np.int32)
        ns, nc = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nb_debug_cells(self.h, None, ctypes.byref(ns), None, ctypes.byref(nc)), "nb_debug_cells")
        cs = np.empty(nc.value + 1, np.int64)
        _check(lib().nb_debug_cells(self.h, _ptr(perm), ctypes.byref(ns), _ptr(cs), ctypes.byref(nc)),
               "nb_debug_cells")
        return perm[:ns.value].copy(), cs

    def debug_pair_terms(self, xqi, xqj, ti, tj):
        """The forward kernel's pair arithmetic for given pairs
        (nb_debug_pair_terms): xqi, xqj [n,4] float32, ti, tj [n] int32 on the
        GPU; returns [n,8] float32 (E_LJ, E_Coul, r2, 0, F_j, 0)."""
        import torch
        xqi, xqj, ti, tj = (t.contiguous() for t in (xqi, xqj, ti, tj))
        out = torch.empty((xqi.shape[0], 8), dtype=torch.float32, device=xqi.device)
        self._sync_stream()
        _check(lib().nb_debug_pair_terms(self.h, xqi.shape[0], _tptr(xqi), _tptr(xqj), _tptr(ti), _tptr(tj),
                                         _tptr(out)), "nb_debug_pair_terms")
        return out

    def debug_pairs(self, cap: int | None = None):
        n, no = ctypes.c_int64(), ctypes.c_int64()
        if cap is None:
            _check(lib().nb_debug_pairs(self.h, None, 0, ctypes.byref(n), ctypes.byref(no)), "nb_debug_pairs")
            cap = n.value
        ij = np.empty((max(cap, 1), 2), np.int32)
        _check(lib().nb_debug_pairs(self.h, _ptr(ij), cap, ctypes.byref(n), ctypes.byref(no)), "nb_debug_pairs")
        m = min(n.value, cap)
        ij = ij[:m]
        order = np.lexsort((ij[:, 1], ij[:, 0]))
        return ij[order], n.value, no.value

    def debug_fill(self):
        """(tiles visited, tile halves evaluated) of the last debug_pairs run."""
        t, h = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().nb_debug_fill(self.h, ctypes.byref(t), ctypes.byref(h)), "nb_debug_fill")
        return t.value, h.value


def debug_philox(ctr, key):
    """Philox4x32-10 on the device (nb_debug_philox): ctr [n,4], key [n,2]
    uint32 tensors on the GPU; returns [n,4] uint32 outputs (int32 storage)."""
    import torch
    assert ctr.dtype == torch.int32 and key.dtype == torch.int32
    ctr, key = ctr.contiguous(), key.contiguous()
    out = torch.empty_like(ctr)
    _check(lib().nb_debug_philox(ctr.shape[0], _tptr(ctr), _tptr(key), _tptr(out), _stream_handle()),
           "nb_debug_philox")
    return out


def fp32_peak_launch(iters: int, sink):
    """Launch the FP32 FMA throughput kernel (nb_fp32_peak_launch) on the
    current stream; returns the FLOP it performs.  Time it with CUDA events."""
    flop = ctypes.c_double()
    _check(lib().nb_fp32_peak_launch(int(iters), _stream_handle(), _tptr(sink), ctypes.byref(flop)),
           "nb_fp32_peak_launch")
    return flop.value


def concat_inputs(systems: Sequence, device="cuda"):
    """Concatenated (pos, q, type) tensors of a list of systems on the device."""
    import torch
    pos = np.concatenate([s.pos for s in systems]).astype(np.float32)
    q = np.concatenate([s.q for s in systems]).astype(np.float32)
    t = np.concatenate([s.type for s in systems]).astype(np.int32)
    return (torch.from_numpy(pos).to(device), torch.from_numpy(q).to(device), torch.from_numpy(t).to(device))


def _autograd():
    import torch

    class NonbondedFn(torch.autograd.Function):
        """(F, E) = NonbondedFn.apply(pos, q, sigma, epsilon, ctx, types).

        forward: cell-list rebuild + forces and energies (E is [n_sys, 2]:
        LJ, Coulomb).  backward: the library's adjoint kernel with the pair
        list recomputed from a fresh build, giving dL/dpos (Hessian-vector
        product plus the energy term), dL/dq and per-type dL/dsigma, dL/deps.
        sigma/epsilon are per-type tensors; the context's LJ table is updated
        from them when their values change.
        """

        @staticmethod
        def forward(fctx, pos, q, sigma, epsilon, nbctx, typ):
            sig = sigma.detach().double().cpu().numpy().astype(np.float32)
            eps = epsilon.detach().double().cpu().numpy().astype(np.float32)
            key = (sig.tobytes(), eps.tobytes())
            if getattr(nbctx, "_lj_key", None) != key:
                nbctx.set_lj_params(sig, eps)
                nbctx._lj_key = key
            nbctx.build(pos)
            F, E, _ = nbctx.forces(pos, q, typ, virial=False)
            fctx.save_for_backward(pos, q)
            fctx.nb = nbctx
            fctx.typ = typ
            fctx.sig_meta = (sigma.dtype, sigma.device, epsilon.dtype, epsilon.device)
            return F, E

        @staticmethod
        def backward(fctx, gF, gE):
            pos, q = fctx.saved_tensors
            nbctx = fctx.nb
            gF = torch.zeros_like(pos) if gF is None else gF.contiguous().float()
            gE = None if gE is None else gE.contiguous().double()
            nbctx.build(pos)  # the pair list is recomputed, not stored
            gpos, gq, gs_tab, ge_tab = nbctx.backward(pos, q, fctx.typ, gF, gE)
            gs, ge = nbctx.type_gradients(gs_tab, ge_tab)
            sd, sdev, ed, edev = fctx.sig_meta
            return gpos, gq, gs.to(sdev, sd), ge.to(edev, ed), None, None

    return NonbondedFn


_fn_cache = None


def nonbonded(pos, q, sigma, epsilon, nbctx, typ):
    """Differentiable (F, E) through the library's forward and adjoint kernels."""
    global _fn_cache
    if _fn_cache is None:
        _fn_cache = _autograd()
    return _fn_cache.apply(pos, q, sigma, epsilon, nbctx, typ)
