"""Pins of the oracle's tabulated radial functions (the paper's lookup-table
variant: radial parts of the van der Waals and electrostatic terms linearly
interpolated from n-point tables; n = 4096 in its error figure), against
what the mathematics and the paper fix:

* at a table point the interpolated pair energy equals the direct one (to
  FP32 rounding of the table);
* at the midpoint of an interval the error is the linear-interpolation
  error of each radial function, (f(a) + f(b))/2 - f((a+b)/2), in closed form;
* the error against direct evaluation falls as h^2 (4x per halving of h);
* with n = 4096 the relative force error is below the paper's 1e-4.
"""

import dataclasses

import numpy as np
import pytest

import oracle
from paper_0902_0827_gb300 import systems as S

SIG, EPS = 3.4, 0.238


def lj_dimer(r):
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]], np.float32)
    assert float(pos[1, 0]) - float(pos[0, 0]) == r  # exact in FP32
    return S.System("dimer", pos, np.zeros(2, np.float32), np.zeros(2, np.int32),
                    np.array([SIG], np.float32), np.array([EPS], np.float32), np.full(3, 30.0, np.float32),
                    np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), 9.0, 7.5, 0.0)


def lj_direct(r):
    """LJ energy of the FP32 parameters at r (no switch below rs)."""
    s, e = float(np.float32(SIG)), float(np.float32(EPS))
    A, B = 4.0 * e * s ** 12, 4.0 * e * s ** 6
    return A / r ** 12 - B / r ** 6, A, B


def test_interpolation_is_exact_at_table_points():
    n, rc = 4096, 9.0
    k = 1365
    r = k * rc / n  # 12285 / 4096, exact in FP32
    with oracle.tabulated(n):
        _, Et, _, _ = oracle.forces(lj_dimer(r))
    Ed, _, _ = lj_direct(r)
    assert abs(Et[0] - Ed) <= 1e-6 * abs(Ed)


@pytest.mark.parametrize("k", [1000, 1200, 1365])
def test_midpoint_error_is_the_linear_interpolation_error(k):
    n, rc = 4096, 9.0
    a, b = k * rc / n, (k + 1) * rc / n
    m = 0.5 * (a + b)
    with oracle.tabulated(n):
        _, Et, _, _ = oracle.forces(lj_dimer(m))
    Em, A, B = lj_direct(m)
    # (f(a) + f(b))/2 - f(m) for f = r^-12 and r^-6, combined with A and -B
    lerp_err = A * (0.5 * (a ** -12 + b ** -12) - m ** -12) - B * (0.5 * (a ** -6 + b ** -6) - m ** -6)
    assert abs(lerp_err) > 100 * 6e-8 * abs(Em)  # the effect is far above FP32 table rounding
    assert abs((Et[0] - Em) - lerp_err) <= 0.01 * abs(lerp_err) + 2e-7 * abs(Em)


def water_box_small():
    return S._water_system(S.rng_for(31), 512, "w512")


def test_error_falls_as_h_squared():
    s = water_box_small()
    Fd, Ed, _, _ = oracle.forces(s, method="cells")
    errs = []
    for n in (1024, 2048, 4096):
        with oracle.tabulated(n):
            F, _, _, _ = oracle.forces(s, method="cells")
        errs.append(np.linalg.norm(F - Fd) / np.linalg.norm(Fd))
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.0 <= e1 / e2 <= 5.0, errs


def test_paper_bound_at_4096_points():
    s = S.solvated_chain()
    Fd, Ed, Wd, nd, Es = oracle.forces(s, method="cells", with_scale=True)
    with oracle.tabulated(4096):
        F, E, W, n = oracle.forces(s, method="cells")
    assert n == nd  # membership does not depend on the radial functions
    assert np.linalg.norm(F - Fd) / np.linalg.norm(Fd) <= 1e-4
    for c in range(2):
        assert abs(E[c] - Ed[c]) <= 1e-4 * Es[c]
