"""The C-ABI library builds, loads and exports every symbol include/acenb.h
declares; host-side validation rejects bad parameters before touching a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_0902_0827_gb300 import build as B
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "acenb.h")


def declared_symbols():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    B.build()
    L = nb.lib()
    decl = declared_symbols()
    assert len(decl) >= 14
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(nb.EXPORTS)


def test_status_strings():
    L = nb.lib()
    for code in range(13):
        s = L.nb_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0


def _params(sys):
    p = nb.nb_params()
    sig, eps = np.ascontiguousarray(sys.sigma, np.float32), np.ascontiguousarray(sys.epsilon, np.float32)
    ex = np.ascontiguousarray(sys.excl, np.int32)
    p.n_atoms = sys.n_atoms
    for a in range(3):
        p.box[a] = 30.0  # a valid box for the 9 A cutoff
    p.cutoff, p.switch_dist, p.ewald_alpha, p.coulomb_k = sys.cutoff, sys.switch_dist, sys.ewald_alpha, sys.coulomb_k
    p.n_types = sig.shape[0]
    p.sigma, p.epsilon = sig.ctypes.data_as(ctypes.c_void_p), eps.ctypes.data_as(ctypes.c_void_p)
    p.n_excl, p.excl = ex.shape[0], ex.ctypes.data_as(ctypes.c_void_p) if ex.size else None
    p.scale14_lj, p.scale14_coul = 0.5, 1 / 1.2
    return p, (sig, eps, ex)


def _create(p):
    h = ctypes.c_void_p()
    return nb.lib().nb_create(ctypes.byref(p), None, ctypes.byref(h)), h


def test_host_validation_without_gpu():
    s = S._water_system(S.rng_for(30), 8, "w")
    p, keep = _params(s)
    # box barely above 2 rc is fine on the host side; exactly 2 rc is too small
    p.box[0] = 18.0
    assert _create(p)[0] == 2  # NB_ERR_BOX_TOO_SMALL
    p, keep = _params(s)
    p.cutoff = -1.0
    assert _create(p)[0] == 1
    p, keep = _params(s)
    bad = np.array([[0, 99]], np.int32)
    p.n_excl, p.excl = 1, bad.ctypes.data_as(ctypes.c_void_p)
    assert _create(p)[0] == 1
    p, keep = _params(s)
    p.n_types = 65
    big = np.ones(65, np.float32)
    p.sigma = p.epsilon = big.ctypes.data_as(ctypes.c_void_p)
    assert _create(p)[0] == 11  # NB_ERR_UNSUPPORTED
    p, keep = _params(s)
    p.flags = 1
    assert _create(p)[0] == 1
    # an empty system (N >= 1 is required)
    p, keep = _params(s)
    p.n_atoms = 0
    assert _create(p)[0] == 1
    # more than 16 topology partners (excluded + scaled 1-4) of one atom
    s20 = S._water_system(S.rng_for(31), 7, "w21")
    p, keep = _params(s20)
    ex17 = np.array([[0, j] for j in range(1, 18)], np.int32)
    p.n_excl, p.excl = 17, ex17.ctypes.data_as(ctypes.c_void_p)
    assert _create(p)[0] == 11  # NB_ERR_UNSUPPORTED
    h = ctypes.c_void_p()
    assert nb.lib().nb_create(None, None, ctypes.byref(h)) == 1
    assert nb.lib().nb_build_cells(None, None) == 1
    assert nb.lib().nb_get_status(None) == 1


def test_oracle_and_product_share_no_code():
    root = os.path.dirname(HDR)
    pkg = os.path.join(os.path.dirname(root), "paper_0902_0827_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")) and "_build" not in dirpath:
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "nb_oracle" not in txt, f
    osrc = open(os.path.join(os.path.dirname(root), "oracle", "nb_oracle.c")).read()
    assert "acenb" not in osrc and "nb_internal" not in osrc
