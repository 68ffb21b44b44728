"""FP64 oracle of the molecular-dynamics step (TEST INFRASTRUCTURE).

Section "Molecular dynamics on the GPU" lists bonded force terms,
velocity-Verlet integration with a Langevin thermostat, PME and holonomic
hydrogen-bond constraints by M-SHAKE (positions) and RATTLE (velocities);
section "Performance" runs DHFR with them.  The paper prints no formula for
any of these; the forms below are the readings recorded in the design notes:

* bonds U = k (r - r0)^2, angles U = k (theta - theta0)^2, dihedrals
  U = k (1 + cos(n phi - delta)) with the IUPAC sign of phi
  (phi = atan2(|b2| b1 . (b2 x b3), (b1 x b2) . (b2 x b3)), b1 = x_j - x_i,
  b2 = x_k - x_j, b3 = x_l - x_k), every displacement the minimum image;
* one step of length dt (ps) from (x, v, F(x)):
    O  v <- c v + sqrt((1 - c^2) kT / m) xi,  c = exp(-gamma dt / 2)
    B  v <- v + (dt/2) F / m
    A  x' <- x + dt v, then M-SHAKE: x'' = x' + sum_k lambda_k s_ik r_k / m_i
       with the constraint vectors r_k of x, lambda from Newton iterations on
       |r_k''|^2 = d_k^2 (the 3 x 3 linearised system solved exactly each
       iteration), and v <- v + (x'' - x') / dt
    F(x'')
    B  v <- v + (dt/2) F / m
    O  v <- c v + sqrt((1 - c^2) kT / m) xi'
    RATTLE  v <- v + sum_k mu_k s_ik r_k'' / m_i with r_k'' . (v_a - v_b) = 0
  (a Langevin velocity Verlet in the O-B-A-B-O arrangement; gamma = 0 is
  plain velocity Verlet with SHAKE/RATTLE);
* the Gaussian numbers xi come from the counter-based generator
  Philox4x32-10 (Salmon et al., SC 2011), counter (atom, step, stream, 0),
  key (seed low, seed high), each 32-bit output turned into a 24-bit uniform
  u = ((x >> 8) + 1/2) 2^-24 and pairs of uniforms into normals by the
  Box-Muller transform;
* units: kcal/mol, A, amu, ps; F / m in kcal/mol/A/amu times 418.4 is A/ps^2.

Only the tests, the smoke check and the CPU legs of the benchmark use this.
"""

from __future__ import annotations

import dataclasses

import numpy as np

KCAL_PER_AMU = 418.4   # (A/ps)^2 per kcal/mol/amu
KB = 0.0019872041      # kcal/mol/K


def min_image(d, L):
    return d - L * np.rint(d / L)


# ----------------------------------------------------------------- bonded


def bonded(top, pos, box):
    """(F [N,3], (E_bond, E_angle, E_dihedral), W [6]) in FP64."""
    x = np.asarray(pos, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    n = x.shape[0]
    F = np.zeros((n, 3))
    W = np.zeros((3, 3))
    E = [0.0, 0.0, 0.0]

    def add(idx, f, y):
        np.add.at(F, idx, f)
        W[...] += np.einsum("ia,ib->ab", y, f)

    if len(top.bonds):
        i, j = top.bonds[:, 0], top.bonds[:, 1]
        d = min_image(x[j] - x[i], L)
        r = np.linalg.norm(d, axis=1)
        k, r0 = top.bond_k.astype(np.float64), top.bond_r0.astype(np.float64)
        E[0] = float((k * (r - r0) ** 2).sum())
        fi = (2.0 * k * (r - r0) / r)[:, None] * d  # -dU/dx_i
        add(i, fi, np.zeros_like(d))
        add(j, -fi, d)
    if len(top.angles):
        i, j, kk = top.angles[:, 0], top.angles[:, 1], top.angles[:, 2]
        a = min_image(x[i] - x[j], L)
        b = min_image(x[kk] - x[j], L)
        la, lb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
        cr = np.cross(a, b)
        s = np.linalg.norm(cr, axis=1)
        c = np.einsum("ij,ij->i", a, b)
        th = np.arctan2(s, c)
        k, t0 = top.angle_k.astype(np.float64), top.angle_theta0.astype(np.float64)
        E[1] = float((k * (th - t0) ** 2).sum())
        dU = 2.0 * k * (th - t0)
        cos, sin = c / (la * lb), s / (la * lb)
        ah, bh = a / la[:, None], b / lb[:, None]
        dth_da = (cos[:, None] * ah - bh) / (la * sin)[:, None]
        dth_db = (cos[:, None] * bh - ah) / (lb * sin)[:, None]
        fi, fk = -dU[:, None] * dth_da, -dU[:, None] * dth_db
        add(i, fi, a)
        add(kk, fk, b)
        add(j, -fi - fk, np.zeros_like(a))
    if len(top.dihedrals):
        i, j, kk, l = (top.dihedrals[:, c] for c in range(4))
        b1 = min_image(x[j] - x[i], L)
        b2 = min_image(x[kk] - x[j], L)
        b3 = min_image(x[l] - x[kk], L)
        n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
        lb2 = np.linalg.norm(b2, axis=1)
        phi = np.arctan2(lb2 * np.einsum("ij,ij->i", b1, n2), np.einsum("ij,ij->i", n1, n2))
        k = top.dihedral_k.astype(np.float64)
        m = top.dihedral_n.astype(np.float64)
        dl = top.dihedral_phase.astype(np.float64)
        E[2] = float((k * (1.0 + np.cos(m * phi - dl))).sum())
        dU = -k * m * np.sin(m * phi - dl)
        n1s, n2s = np.einsum("ij,ij->i", n1, n1), np.einsum("ij,ij->i", n2, n2)
        gi = -(lb2 / n1s)[:, None] * n1
        gl = (lb2 / n2s)[:, None] * n2
        p1 = (np.einsum("ij,ij->i", b1, b2) / lb2 ** 2)[:, None]
        p3 = (np.einsum("ij,ij->i", b3, b2) / lb2 ** 2)[:, None]
        gj = -(1.0 + p1) * gi + p3 * gl
        gk = -(1.0 + p3) * gl + p1 * gi
        z = np.zeros_like(b1)
        add(i, -dU[:, None] * gi, z)
        add(j, -dU[:, None] * gj, b1)
        add(kk, -dU[:, None] * gk, b1 + b2)
        add(l, -dU[:, None] * gl, b1 + b2 + b3)
    Wv = np.array([W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]])
    return F, tuple(E), Wv


# ------------------------------------------------------------ Philox / noise

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon et al. 2011) on uint64 arrays
    holding 32-bit values; returns four uint64 arrays of 32-bit outputs."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.uint64(k0 & _MASK)
    k1 = np.uint64(k1 & _MASK)
    for rnd in range(10):
        p0 = np.uint64(_M0) * c0
        p1 = np.uint64(_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
    return c0, c1, c2, c3


def uniforms24(x):
    """((x >> 8) + 1/2) 2^-24: a uniform on (0, 1) exact in FP32."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def normals(atoms, step: int, stream: int, seed: int):
    """Three standard normals per atom from one Philox block:
    counter (atom, step, stream, 0), key (seed & 0xffffffff, seed >> 32)."""
    a = np.asarray(atoms, dtype=np.uint64)
    o = philox4x32_10(a, np.full_like(a, step), np.full_like(a, stream), np.zeros_like(a),
                      seed & _MASK, (seed >> 32) & _MASK)
    u = [uniforms24(t) for t in o]
    r0 = np.sqrt(-2.0 * np.log(u[0]))
    r1 = np.sqrt(-2.0 * np.log(u[2]))
    return np.stack([r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
                     r1 * np.cos(2 * np.pi * u[3])], 1)


# ---------------------------------------------------------- constraints

# rigid water: constraint k joins atoms (A[k], B[k]) of (O, H1, H2)
_CA = np.array([0, 0, 1])
_CB = np.array([1, 2, 2])


def _coupling(mw):
    """C_kl = s(a_k, l)/m_{a_k} - s(b_k, l)/m_{b_k}, s(i, l) = +1 if i is the
    first atom of constraint l, -1 if the second: r_k changes by
    sum_l lambda_l C_kl r_l when atom i moves by sum_l lambda_l s(i,l) r_l / m_i.
    mw [nw, 3] masses of (O, H1, H2) -> [nw, 3, 3]."""
    s = np.zeros((3, 3))
    for l in range(3):
        s[_CA[l], l] = 1.0
        s[_CB[l], l] = -1.0
    return s[_CA][None] / mw[:, _CA, None] - s[_CB][None] / mw[:, _CB, None], s


def shake(top, x_ref, x_new, box, mass, tol=1e-12, max_iter=100):
    """M-SHAKE of every water: returns (constrained positions, displacement
    x'' - x', iterations used).  x_ref satisfies the constraints."""
    L = np.asarray(box, dtype=np.float64)
    w = top.waters
    if len(w) == 0:
        return x_new.copy(), np.zeros_like(x_new), 0
    mw = mass[w]
    d2 = np.array([top.water_roh, top.water_roh, top.water_rhh], dtype=np.float64) ** 2
    C, s = _coupling(mw)
    r = min_image(x_ref[w[:, _CA]] - x_ref[w[:, _CB]], L)      # [nw, 3 constraints, 3]
    u = min_image(x_new[w[:, _CA]] - x_new[w[:, _CB]], L)
    lam = np.zeros((len(w), 3))
    it = 0
    for it in range(1, max_iter + 1):
        rr = u + np.einsum("wkl,wl,wlc->wkc", C, lam, r)
        g = np.einsum("wkc,wkc->wk", rr, rr) - d2
        if np.max(np.abs(g) / d2) < tol:
            break
        J = 2.0 * np.einsum("wkc,wkl,wlc->wkl", rr, C, r)
        lam = lam - np.linalg.solve(J, g[..., None])[..., 0]
    disp = np.einsum("il,wl,wlc->wic", s, lam, r) / mw[..., None]  # [nw, atom, 3]
    out = x_new.copy()
    out[w] = x_new[w] + disp
    dfull = np.zeros_like(x_new)
    dfull[w] = disp
    return out, dfull, it


def rattle(top, x, v, box, mass):
    """Project water velocities so that r_k . (v_a - v_b) = 0 (r_k of x)."""
    L = np.asarray(box, dtype=np.float64)
    w = top.waters
    if len(w) == 0:
        return v.copy()
    mw = mass[w]
    C, s = _coupling(mw)
    r = min_image(x[w[:, _CA]] - x[w[:, _CB]], L)
    dv = v[w[:, _CA]] - v[w[:, _CB]]
    A = np.einsum("wkl,wkc,wlc->wkl", C, r, r)
    b = -np.einsum("wkc,wkc->wk", r, dv)
    mu = np.linalg.solve(A, b[..., None])[..., 0]
    out = v.copy()
    out[w] = v[w] + np.einsum("il,wl,wlc->wic", s, mu, r) / mw[..., None]
    return out


# ----------------------------------------------------------------- the step


@dataclasses.dataclass
class MDParams:
    dt: float = 0.002           # ps
    gamma: float = 1.0          # 1/ps (0: NVE)
    temperature: float = 300.0  # K
    seed: int = 2009
    pme: tuple | None = None    # (grid, order) or None (real space only)


def forces_at(sys, top, x, prm: MDParams):
    """Total forces and potential energies at positions x (FP64 array; the
    non-bonded terms take its FP32 rounding, as the library does)."""
    from . import forces as nb_forces
    from . import ewald
    x32 = x.astype(np.float32)
    L = sys.box.astype(np.float64)
    x32 = np.mod(x32.astype(np.float64), L).astype(np.float32)
    x32 = np.where(x32 >= sys.box, x32 - sys.box, x32).astype(np.float32)
    F, E, _, _ = nb_forces(sys, method="cells", pos=x32)
    e_c = E[1]
    if prm.pme is not None:
        Fr, Er, _ = ewald.spme(sys, prm.pme[0], prm.pme[1], pos=x32.astype(np.float64))
        Fc, Es, Ep, _ = ewald.ewald_corrections(sys, pos=x32)
        F = F + Fr + Fc
        e_c = e_c + Er + Es + Ep
    Fb, Eb, _ = bonded(top, x, sys.box)
    return F + Fb, np.array([E[0], e_c, Eb[0], Eb[1], Eb[2]])


def minimize_step(sys, top, x, F, max_disp: float):
    """One move of the library's energy minimiser (the paper prints none; a
    plain capped steepest descent in mass-weighted coordinates): x' = x +
    h F / m with h = max_disp / max_i |F_i| / m_i, then M-SHAKE of every
    water from x.  F: total forces at x (forces_at)."""
    m = top.mass.astype(np.float64)
    g = np.linalg.norm(F, axis=1) / m
    gmax = float(g.max())
    h = max_disp / gmax if gmax > 0.0 else 0.0
    xn = x + h * F / m[:, None]
    xc, _, _ = shake(top, x, xn, sys.box, m)
    return xc


def kinetic(v, mass):
    return 0.5 * float((mass[:, None] * v * v).sum()) / KCAL_PER_AMU


def step(sys, top, x, v, F, step_index: int, prm: MDParams):
    """One step; returns (x, v, F, energies [E_lj, E_coul, E_bond, E_angle,
    E_dihedral, E_kin])."""
    m = top.mass.astype(np.float64)
    dt = prm.dt
    c = np.exp(-prm.gamma * dt / 2.0)
    sig = np.sqrt((1.0 - c * c) * KB * prm.temperature * KCAL_PER_AMU / m)[:, None]
    idx = np.arange(len(m))
    if prm.gamma > 0:
        v = c * v + sig * normals(idx, step_index, 0, prm.seed)
    v = v + 0.5 * dt * KCAL_PER_AMU * F / m[:, None]
    xn = x + dt * v
    xc, disp, _ = shake(top, x, xn, sys.box, m)
    v = v + disp / dt
    F, Ep = forces_at(sys, top, xc, prm)
    v = v + 0.5 * dt * KCAL_PER_AMU * F / m[:, None]
    if prm.gamma > 0:
        v = c * v + sig * normals(idx, step_index, 1, prm.seed)
    v = rattle(top, xc, v, sys.box, m)
    return xc, v, F, np.concatenate([Ep, [kinetic(v, m)]])
