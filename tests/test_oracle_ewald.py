"""Pins of the reciprocal-space oracle (direct Ewald sum, Ewald corrections,
smooth PME) against results the mathematics fixes, independently of the
oracle's own formulas:

* the Madelung constant of rock salt (1.747564594633, a textbook value) from
  the real-space + reciprocal + self energies of a periodic NaCl crystal;
* independence of the total electrostatic energy, forces and virial from the
  splitting parameter alpha (a wrong sign or factor in any one of the four
  parts breaks it);
* forces = -grad E by central differences, for the direct sum and for PME;
* virial = -dE/d(strain) by finite differences of a homogeneous deformation,
  the shear components through a brute-force triclinic Ewald sum;
* the smooth PME energy, forces and virial converging to the direct sum as
  the grid and the B-spline order grow;
* cardinal B-spline closed forms (values at the integers, unit partition);
* a molecule whose pairs are all excluded but one scaled 1-4 pair, alone in a
  large box: its total electrostatic energy is that one pair's s14 ke qq/r.
"""

import dataclasses
import math

import numpy as np
import pytest

import oracle
import oracle.ewald as ew
from paper_0902_0827_gb300 import systems as S

MADELUNG_NACL = 1.747564594633


def rock_salt(d=2.8, n_cells=4, alpha=0.35, rc=11.0):
    """Periodic NaCl: n_cells^3 conventional cubic cells of edge 2d, +1 on
    the FCC sites, -1 on the sites shifted by (d, 0, 0); no LJ."""
    a = 2.0 * d
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts, qs = [], []
    for o in np.ndindex(n_cells, n_cells, n_cells):
        for b in fcc:
            pts.append((np.array(o) + b) * a)
            qs.append(1.0)
            pts.append(((np.array(o) + b + [0.5, 0, 0]) % n_cells) * a)
            qs.append(-1.0)
    n = len(qs)
    return S.System("nacl", np.array(pts, np.float32), np.array(qs, np.float32), np.zeros(n, np.int32),
                    np.array([1.0], np.float32), np.array([0.0], np.float32), np.full(3, n_cells * a, np.float32),
                    np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), rc, rc - 1.0, alpha)


def coulomb_only(s, kmax):
    """Total Ewald electrostatics of s: real space (the short-range oracle
    minus its charge-free LJ part) + reciprocal + self + corrections."""
    F, E, W, _ = oracle.forces(s, method="allpairs")
    F0, E0, W0, _ = oracle.forces(s, method="allpairs", q=np.zeros_like(s.q))
    Fr, Er, Wr = ew.ewald_recip(s, kmax)
    Fc, Es, Ep, Wc = ew.ewald_corrections(s)
    return F - F0 + Fr + Fc, E[1] + Er + Es + Ep, W - W0 + Wr + Wc


def test_rock_salt_madelung_constant():
    d = 2.8
    s = rock_salt(d)
    F, E, W = coulomb_only(s, 14)
    # E = -(N/2) M ke q^2 / d for N ions of charge +-1
    M = -E / (0.5 * s.n_atoms * s.coulomb_k / d)
    assert abs(M - MADELUNG_NACL) <= 5e-6 * MADELUNG_NACL
    # every ion sits at a centre of symmetry: no force
    assert np.abs(F).max() <= 1e-3
    # Coulomb energy is homogeneous of degree -1: trace of the virial = E
    assert abs(W[:3].sum() - E) <= 1e-4 * abs(E)
    # cubic symmetry: isotropic diagonal, no shear
    assert np.ptp(W[:3]) <= 1e-6 * abs(E)
    assert np.abs(W[3:]).max() <= 1e-6 * abs(E)


def water216(alpha):
    return dataclasses.replace(S._water_system(S.rng_for(30), 216, "w216"), ewald_alpha=alpha)


def test_total_electrostatics_independent_of_alpha():
    F1, E1, W1 = coulomb_only(water216(0.45), 20)
    F2, E2, W2 = coulomb_only(water216(0.55), 22)
    assert abs(E1 - E2) <= 2e-5 * abs(E1)
    assert np.linalg.norm(F1 - F2) / np.linalg.norm(F1) <= 2e-5
    assert np.abs(W1 - W2).max() <= 1e-4 * np.abs(W1).max()


def test_direct_sum_forces_are_minus_gradient():
    s = water216(0.32)
    F, _, _ = ew.ewald_recip(s, 12)
    h = np.float32(2.0 ** -8)  # exact in FP32 at these coordinates
    for i in (0, 5, 300, 647):
        for a in range(3):
            p = s.pos.copy()
            p[i, a] += h
            Ep = ew.ewald_recip(s, 12, pos=p)[1]
            p[i, a] -= 2 * h
            Em = ew.ewald_recip(s, 12, pos=p)[1]
            fd = -(Ep - Em) / (2.0 * float(h))
            assert abs(fd - F[i, a]) <= 1e-4 * max(1.0, abs(F[i, a]))


def test_pme_forces_are_minus_gradient():
    s = water216(0.32)
    grid, order = (24, 20, 28), 6
    F, _, _ = ew.spme(s, grid, order)
    x = s.pos.astype(np.float64)
    h = 1e-5
    for i in (1, 100, 646):
        for a in range(3):
            p = x.copy()
            p[i, a] += h
            Ep = ew.spme(s, grid, order, pos=p)[1]
            p[i, a] -= 2 * h
            Em = ew.spme(s, grid, order, pos=p)[1]
            assert abs(-(Ep - Em) / (2 * h) - F[i, a]) <= 1e-5 * max(1.0, abs(F[i, a]))


def strained(s, a, eps):
    """s under x_a -> (1 + eps) x_a (box and coordinates)."""
    p = s.pos.astype(np.float64).copy()
    L = s.box.astype(np.float64).copy()
    p[:, a] *= 1.0 + eps
    L[a] *= 1.0 + eps
    return p, L


def test_diagonal_virial_is_minus_strain_derivative():
    s = water216(0.32)
    _, _, W = ew.spme(s, (32, 32, 32), 6)
    _, _, Wd = ew.ewald_recip(s, 12)
    h = 1e-6
    for a in range(3):
        Es = []
        for e in (h, -h):
            p, L = strained(s, a, e)
            Es.append(ew.spme(dataclasses.replace(s, box=L), (32, 32, 32), 6, pos=p)[1])
        fd = -(Es[0] - Es[1]) / (2 * h)
        assert abs(fd - W[a]) <= 1e-6 * np.abs(W).max()
        # the direct sum's virial agrees with PME's at this accuracy
        assert abs(Wd[a] - W[a]) <= 1e-4 * np.abs(W).max()


def triclinic_recip_energy(r, q, hmat, alpha, ke, kmax):
    """Brute-force Ewald reciprocal energy for a general cell (columns of
    hmat are the cell vectors): m = k . h^-1 over integer k, |k_a| <= kmax."""
    hinv = np.linalg.inv(hmat)
    V = abs(np.linalg.det(hmat))
    e = 0.0
    rng = range(-kmax, kmax + 1)
    for k in np.array([(i, j, l) for i in rng for j in rng for l in rng if (i, j, l) != (0, 0, 0)]):
        m = k @ hinv
        m2 = m @ m
        Sm = np.sum(q * np.exp(2j * np.pi * (r @ m)))
        e += math.exp(-np.pi ** 2 * m2 / alpha ** 2) / m2 * abs(Sm) ** 2
    return ke / (2 * np.pi * V) * e


def test_shear_virial_by_triclinic_finite_difference():
    rng = np.random.default_rng(11)
    L = np.array([9.0, 10.0, 11.0])
    r = rng.uniform(0, 1, size=(8, 3)) * L
    q = rng.normal(size=8)
    q -= q.mean()
    s = S.System("tri", r.astype(np.float32), q.astype(np.float32), np.zeros(8, np.int32),
                 np.array([1.0], np.float32), np.array([0.0], np.float32), L.astype(np.float32),
                 np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32), 4.0, 3.0, 0.3)
    kmax = 6
    _, E, W = ew.ewald_recip(s, kmax)
    r32 = s.pos.astype(np.float64)
    q32 = s.q.astype(np.float64)
    h0 = np.diag(s.box.astype(np.float64))
    a32, ke32 = float(np.float32(0.3)), float(np.float32(s.coulomb_k))  # parameters are FP32 values
    assert abs(triclinic_recip_energy(r32, q32, h0, a32, ke32, kmax) - E) <= 1e-9 * abs(E)
    h = 1e-6
    for k, (a, b) in zip((3, 4, 5), ((0, 1), (0, 2), (1, 2))):
        Es = []
        for e in (h, -h):
            D = np.eye(3)
            D[a, b] += e  # x_a -> x_a + e x_b
            Es.append(triclinic_recip_energy(r32 @ D.T, q32, D @ h0, a32, ke32, kmax))
        fd = -(Es[0] - Es[1]) / (2 * h)
        assert abs(fd - W[k]) <= 1e-6 * max(1.0, np.abs(W).max())


@pytest.mark.parametrize("grid,order,tol", [((32, 32, 32), 6, 1e-5), ((64, 64, 64), 8, 1e-8)])
def test_pme_converges_to_the_direct_sum(grid, order, tol):
    s = water216(0.32)
    Fd, Ed, Wd = ew.ewald_recip(s, 14)
    F, E, W = ew.spme(s, grid, order)
    assert abs(E - Ed) <= tol * abs(Ed)
    assert np.linalg.norm(F - Fd) / np.linalg.norm(Fd) <= tol
    assert np.abs(W - Wd).max() <= 10 * tol * np.abs(Wd).max()


def test_bspline_closed_forms():
    # cubic (order 4) cardinal B-spline: 1/6, 2/3, 1/6 at x = 1, 2, 3
    assert np.allclose(ew.bspline(np.array([0.0, 1.0, 2.0, 3.0, 4.0]), 4), [0, 1 / 6, 2 / 3, 1 / 6, 0], atol=1e-15)
    x = np.linspace(0.0, 1.0, 17)
    for n in (3, 4, 5, 6, 8):
        w = ew.bspline(x[:, None] + np.arange(n)[None, :], n)
        assert np.allclose(w.sum(1), 1.0, atol=1e-13)  # partition of unity
        assert np.allclose(ew.bspline(x, n), ew.bspline(n - x, n), atol=1e-14)  # symmetry
        dw = ew.dbspline(x[:, None] + np.arange(n)[None, :], n)
        assert np.allclose(dw.sum(1), 0.0, atol=1e-12)


def test_fully_excluded_molecule_keeps_only_its_scaled_1_4_pair():
    # four charged atoms on a bent chain, 1-2 and 1-3 pairs excluded, one
    # 1-4 pair scaled: alone in a 100 A box the electrostatic energy is that
    # pair's s14 ke q0 q3 / r (the periodic images of the molecule's dipole
    # contribute ~ ke p^2 / L^3 to the energy and ~ ke q p / L^3 to forces,
    # below 1e-3 here)
    pos = np.array([[50.0, 50.0, 50.0], [51.5, 50.0, 50.0], [52.0, 51.4, 50.0], [53.5, 51.6, 50.6]])
    q = np.array([0.3, -0.5, 0.4, -0.2])
    ex = np.array([[0, 1], [1, 2], [2, 3], [0, 2], [1, 3]], np.int32)
    s = S.System("mol", pos.astype(np.float32), q.astype(np.float32), np.zeros(4, np.int32),
                 np.array([1.0], np.float32), np.array([0.0], np.float32), np.full(3, 100.0, np.float32),
                 ex, np.array([[0, 3]], np.int32), 9.0, 7.5, 0.3)
    F, E, W = coulomb_only(s, 44)
    p = s.pos.astype(np.float64)
    d = p[0] - p[3]
    r = np.linalg.norm(d)
    c = s.scale14_coul * s.coulomb_k * float(s.q[0]) * float(s.q[3])
    assert abs(E - c / r) <= 1e-3
    f0 = c * d / r ** 3
    Fx = np.zeros((4, 3))
    Fx[0], Fx[3] = f0, -f0
    assert np.abs(F - Fx).max() <= 1e-3
