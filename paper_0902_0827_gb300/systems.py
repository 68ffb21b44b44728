"""Seeded synthetic molecular systems shaped like the paper's workloads.

This module only builds inputs (coordinates, charges, types, parameters,
exclusion and 1-4 lists).  It contains none of the non-bonded arithmetic, so
both the FP64 oracle and the CUDA path can consume its output.

Every system is returned as a :class:`System` holding canonical FP32 arrays with
coordinates already wrapped into ``[0, L)`` per axis.

Workloads (stand-ins for the paper's benchmark systems, none of which ships
with this code; section "Performance" and section "Molecular dynamics on the
GPU"):

* ``lj_fcc``      - 256-atom Lennard-Jones FCC crystal, rc 8.5, switch 7.5.
* ``water_box``   - TIP3P-shaped rigid waters on a jittered grid at 1 g/cm^3.
* ``solvated_chain`` - 2,500-atom self-avoiding chain + 7,000 waters in a
  62.2 A box (shaped like the DHFR benchmark: 23,500 atoms, R = 9 A,
  switch 7.5 A).
* ``water_ensemble`` - many water boxes with log-uniform atom counts.
* ``big_water``   - 333,333 waters (about 1.0 M atoms).
* ``dhfr_chain_md`` - the solvated chain with parameters fit for dynamics.

Seeds follow ``PCG64(902827 + k)`` for workload ``k``.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# TIP3P geometry and parameters (kcal/mol, Angstrom, e).
TIP3P_QO = -0.834
TIP3P_QH = 0.417
TIP3P_ROH = 0.9572
TIP3P_THETA = math.radians(104.52)
TIP3P_SIGMA_O = 3.1507
TIP3P_EPS_O = 0.1521
# Water number density at 1.0 g/cm^3: N_A / M_w  (M_w = 18.015 g/mol).
WATER_NUMBER_DENSITY = 6.02214076e23 / 18.015 * 1e-24  # per A^3
COULOMB_K = 332.0636  # kcal A / (mol e^2), the NAMD/CHARMM value
SEED_BASE = 902827


@dataclasses.dataclass
class System:
    """One periodic system in canonical FP32 form.

    pos:   float32 [N, 3], wrapped into [0, L) per axis.
    q:     float32 [N] charges (e).
    type:  int32 [N] LJ type index into sigma/epsilon.
    sigma, epsilon: float32 [T] per-type LJ parameters (A, kcal/mol).
    box:   float32 [3] orthorhombic edge lengths.
    excl:  int32 [n_excl, 2] excluded pairs (1-2, 1-3), i != j.
    pairs14: int32 [n_14, 2] scaled 1-4 pairs, disjoint from excl.
    """

    name: str
    pos: np.ndarray
    q: np.ndarray
    type: np.ndarray
    sigma: np.ndarray
    epsilon: np.ndarray
    box: np.ndarray
    excl: np.ndarray
    pairs14: np.ndarray
    cutoff: float
    switch_dist: float
    ewald_alpha: float
    coulomb_k: float = COULOMB_K
    scale14_lj: float = 0.5
    scale14_coul: float = 1.0 / 1.2

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.sigma.shape[0])

    def params(self) -> dict:
        return dict(cutoff=self.cutoff, switch_dist=self.switch_dist,
                    ewald_alpha=self.ewald_alpha, coulomb_k=self.coulomb_k,
                    scale14_lj=self.scale14_lj, scale14_coul=self.scale14_coul)


def rng_for(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + k))


def wrap_canonical(pos64: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L) and round to FP32, keeping x < L."""
    box32 = np.asarray(box, dtype=np.float32)
    p = np.mod(pos64, box32.astype(np.float64))
    p32 = p.astype(np.float32)
    for a in range(3):
        col = p32[:, a]
        col[(col >= box32[a]) | (col < 0)] = np.float32(0.0)
    return np.ascontiguousarray(p32)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_body_frame() -> np.ndarray:
    """O at origin, H1/H2 in the xy plane, bisector along +x."""
    h = TIP3P_THETA / 2
    return np.array([[0.0, 0.0, 0.0],
                     [TIP3P_ROH * math.cos(h), TIP3P_ROH * math.sin(h), 0.0],
                     [TIP3P_ROH * math.cos(h), -TIP3P_ROH * math.sin(h), 0.0]])


def _min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    return d - box * np.round(d / box)


def _place_waters(rng, oxygens: np.ndarray, box: np.ndarray,
                  avoid: np.ndarray | None = None, min_dist: float = 1.3,
                  max_rounds: int = 200) -> np.ndarray:
    """Random orientations for waters at the given O sites.

    An orientation is redrawn while any atom of the water lies closer than
    ``min_dist`` to an atom of another water (or of ``avoid``).
    Returns FP64 positions [3*n, 3] in O, H1, H2 order.
    """
    from scipy.spatial import cKDTree

    n = oxygens.shape[0]
    body = _water_body_frame()
    R = _random_rotations(rng, n)
    bad = np.arange(n)
    for _ in range(max_rounds):
        xyz = oxygens[:, None, :] + np.einsum("nij,kj->nki", R, body)
        flat = np.mod(xyz.reshape(-1, 3), box)
        mol = np.repeat(np.arange(n), 3)
        pts = flat
        owner = mol
        if avoid is not None and avoid.shape[0]:
            pts = np.concatenate([flat, np.mod(avoid, box)])
            owner = np.concatenate([mol, np.full(avoid.shape[0], -1)])
        tree = cKDTree(pts, boxsize=box)
        pairs = tree.query_pairs(min_dist, output_type="ndarray")
        if pairs.size:
            oi, oj = owner[pairs[:, 0]], owner[pairs[:, 1]]
            clash = oi != oj
            cand = np.concatenate([oi[clash], oj[clash]])
            bad = np.unique(cand[cand >= 0])
        else:
            bad = np.empty(0, dtype=np.int64)
        if bad.size == 0:
            return xyz.reshape(-1, 3)
        R[bad] = _random_rotations(rng, bad.size)
    raise RuntimeError("could not place waters without clashes")


def _grid_sites(n_side: int, box: np.ndarray) -> np.ndarray:
    g = np.arange(n_side)
    sp = box / n_side
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    return (np.stack([gx, gy, gz], -1).reshape(-1, 3) + 0.5) * sp


def water_topology(n_waters: int, first_atom: int = 0):
    """1-2 (O-H) and 1-3 (H-H) exclusions of rigid 3-site waters."""
    base = first_atom + 3 * np.arange(n_waters)
    ex = np.concatenate([np.stack([base, base + 1], 1),
                         np.stack([base, base + 2], 1),
                         np.stack([base + 1, base + 2], 1)])
    return ex.astype(np.int32)


def lj_fcc(k: int = 0) -> System:
    """256 single-type LJ atoms on an FCC lattice, 0.0213 atoms/A^3."""
    rng = rng_for(k)
    ncell = 4
    n = 4 * ncell ** 3
    L = (n / 0.0213) ** (1.0 / 3.0)
    a = L / ncell
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(ncell)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None]) * a).reshape(-1, 3)
    pos = pos + rng.uniform(-0.05, 0.05, size=pos.shape)
    box = np.full(3, L)
    return System("lj_fcc", wrap_canonical(pos, box), np.zeros(n, np.float32),
                  np.zeros(n, np.int32), np.array([3.4], np.float32),
                  np.array([0.238], np.float32), box.astype(np.float32),
                  np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32),
                  cutoff=8.5, switch_dist=7.5, ewald_alpha=0.0)


def fcc_lattice_constant(n_cells: int = 4, density: float = 0.0213) -> float:
    return ((4 * n_cells ** 3 / density) ** (1.0 / 3.0)) / n_cells


def _water_system(rng, n_waters: int, name: str, jitter: float = 0.15,
                  cutoff: float = 9.0, switch_dist: float = 7.5,
                  alpha: float = 0.32) -> System:
    L = (n_waters / WATER_NUMBER_DENSITY) ** (1.0 / 3.0)
    box = np.full(3, L)
    n_side = int(math.ceil(n_waters ** (1.0 / 3.0)))
    sites = _grid_sites(n_side, box)
    pick = rng.permutation(sites.shape[0])[:n_waters]
    ox = sites[pick] + rng.uniform(-jitter, jitter, size=(n_waters, 3))
    xyz = _place_waters(rng, ox, box)
    n = 3 * n_waters
    q = np.tile(np.array([TIP3P_QO, TIP3P_QH, TIP3P_QH], np.float32), n_waters)
    typ = np.tile(np.array([0, 1, 1], np.int32), n_waters)
    return System(name, wrap_canonical(xyz, box), q, typ,
                  np.array([TIP3P_SIGMA_O, 0.0], np.float32),
                  np.array([TIP3P_EPS_O, 0.0], np.float32), box.astype(np.float32),
                  water_topology(n_waters), np.zeros((0, 2), np.int32),
                  cutoff=cutoff, switch_dist=switch_dist, ewald_alpha=alpha)


def water_box(k: int = 1, n_waters: int = 2048) -> System:
    """TIP3P-shaped water box (2,048 waters, L ~ 39.4 A by default)."""
    return _water_system(rng_for(k), n_waters, "water_box")


def _self_avoiding_chain(rng, n: int, box: np.ndarray, bond: float = 1.5,
                         clearance: float = 2.4, max_tries: int = 2000) -> np.ndarray:
    """Random-walk chain with fixed bond length; a step is rejected while any
    earlier atom other than its bonded predecessor lies within ``clearance``
    under periodic boundaries."""
    pos = np.empty((n, 3))
    pos[0] = box / 2
    i = 1
    backtracks = 0
    while i < n:
        placed = False
        prev = pos[:i - 1]
        for _ in range(max_tries):
            v = rng.normal(size=3)
            v *= bond / np.linalg.norm(v)
            cand = pos[i - 1] + v
            if i >= 2:
                d = _min_image(prev - cand, box)
                if np.min(np.einsum("ij,ij->i", d, d)) < clearance * clearance:
                    continue
            pos[i] = cand
            placed = True
            break
        if placed:
            i += 1
        else:
            backtracks += 1
            i = max(1, i - 5)
            if backtracks > 10000:
                raise RuntimeError("chain growth stuck")
    return pos


def chain_topology(n: int):
    """Linear chain: 1-2 and 1-3 exclusions, (i, i+3) scaled 1-4 pairs."""
    i = np.arange(n)
    ex12 = np.stack([i[:-1], i[:-1] + 1], 1)
    ex13 = np.stack([i[:-2], i[:-2] + 2], 1)
    p14 = np.stack([i[:-3], i[:-3] + 3], 1)
    return np.concatenate([ex12, ex13]).astype(np.int32), p14.astype(np.int32)


def solvated_chain(k: int = 2, n_chain: int = 2500, n_waters: int = 7000,
                   L: float = 62.2) -> System:
    """Solvated-protein-shaped system: chain + TIP3P waters (23,500 atoms)."""
    rng = rng_for(k)
    box = np.full(3, L)
    chain = _self_avoiding_chain(rng, n_chain, box)
    n_types_chain = 20
    ctype = rng.integers(0, n_types_chain, size=n_chain).astype(np.int32)
    sig = rng.uniform(1.0, 4.0, size=n_types_chain)
    eps = rng.uniform(0.01, 0.2, size=n_types_chain)
    cq = rng.normal(0.0, 0.3, size=n_chain)
    cq -= cq.mean()
    # Water O sites: a jittered grid, refined until enough sites clear the chain.
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(chain, box), boxsize=box)
    n_side = int(math.ceil(n_waters ** (1.0 / 3.0)))
    while True:
        sites = _grid_sites(n_side, box)
        sites = np.mod(sites + rng.uniform(-0.15, 0.15, size=sites.shape), box)
        dmin, _ = tree.query(sites, k=1)
        ok = np.nonzero(dmin > 2.6)[0]
        if ok.size >= n_waters:
            break
        n_side += 1
    pick = ok[rng.permutation(ok.size)[:n_waters]]
    wat = _place_waters(rng, sites[pick], box, avoid=chain)
    pos = np.concatenate([chain, wat])
    q = np.concatenate([cq.astype(np.float32),
                        np.tile(np.array([TIP3P_QO, TIP3P_QH, TIP3P_QH], np.float32), n_waters)])
    typ = np.concatenate([ctype, np.tile(np.array([20, 21, 21], np.int32), n_waters)])
    sigma = np.concatenate([sig, [TIP3P_SIGMA_O, 0.0]]).astype(np.float32)
    epsilon = np.concatenate([eps, [TIP3P_EPS_O, 0.0]]).astype(np.float32)
    cex, c14 = chain_topology(n_chain)
    excl = np.concatenate([cex, water_topology(n_waters, first_atom=n_chain)])
    return System("solvated_chain", wrap_canonical(pos, box), q.astype(np.float32),
                  typ.astype(np.int32), sigma, epsilon, box.astype(np.float32),
                  excl, c14, cutoff=9.0, switch_dist=7.5, ewald_alpha=0.32)


# CHARMM's TIP3P gives the water hydrogens a small LJ sphere (epsilon
# 0.046 kcal/mol, Rmin/2 0.2245 A, so sigma = 2 Rmin/2 / 2^(1/6) = 0.4000 A).
TIP3P_SIGMA_H_CHARMM = 0.4000
TIP3P_EPS_H_CHARMM = 0.046


def dhfr_chain_md(k: int = 2, n_chain: int = 2500, n_waters: int = 7000, L: float = 62.2) -> System:
    """The solvated chain prepared for dynamics (section "Performance": the
    DHFR run): the chain and waters of solvated_chain(k) with heavy-atom LJ
    sizes on the chain (sigma 3.0..4.0 A per type, seeded) and CHARMM's
    TIP3P hydrogen LJ.  With sigma_H = 0 the Lorentz-Berthelot epsilon of
    every pair with a water H is zero, so a negatively charged chain atom and
    an H attract without any repulsion and the dynamics collapses them; the
    parity workload solvated_chain keeps its own parameters."""
    s = solvated_chain(k, n_chain, n_waters, L)
    rng = rng_for(100 + k)
    sigma = s.sigma.astype(np.float64).copy()
    eps = s.epsilon.astype(np.float64).copy()
    n_types_chain = sigma.size - 2
    sigma[:n_types_chain] = rng.uniform(3.0, 4.0, size=n_types_chain)
    sigma[-1], eps[-1] = TIP3P_SIGMA_H_CHARMM, TIP3P_EPS_H_CHARMM
    return dataclasses.replace(s, name="dhfr_chain_md", sigma=sigma.astype(np.float32),
                               epsilon=eps.astype(np.float32))


MIN_ENSEMBLE_WATERS = 199  # keeps L >= 2 rc + 0.1 A at rc = 9 A


def ensemble_sizes(k: int = 3, n_sys: int = 64, lo: int = 500, hi: int = 20000) -> np.ndarray:
    """Water counts of the ensemble: atoms log-uniform in [lo, hi], whole waters,
    clamped so every box satisfies L >= 2 rc + 0.1 A."""
    rng = rng_for(k)
    atoms = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_sys))
    w = np.maximum(np.rint(atoms / 3.0).astype(np.int64), MIN_ENSEMBLE_WATERS)
    return w


def water_ensemble(k: int = 3, n_sys: int = 64, lo: int = 500, hi: int = 20000) -> list[System]:
    """Independent TIP3P-shaped boxes with log-uniform atom counts."""
    sizes = ensemble_sizes(k, n_sys, lo, hi)
    out = []
    for s, nw in enumerate(sizes):
        rng = np.random.Generator(np.random.PCG64([SEED_BASE + k, s]))
        out.append(_water_system(rng, int(nw), f"ensemble_{s}"))
    return out


def big_water(k: int = 4, n_waters: int = 333_333) -> System:
    """Large water box (333,333 waters, about 1.0 M atoms, L ~ 215 A)."""
    return _water_system(rng_for(k), n_waters, "big_water")


# ---------------------------------------------------------------------------
# Molecular-dynamics inputs: masses, bonded terms and rigid-water constraints
# (section "Molecular dynamics on the GPU": bonded terms, velocity-Verlet
# integration, Langevin thermostat, M-SHAKE/RATTLE constraints).  The chain
# gets CHARMM-like parameters of an sp3 carbon backbone (the random-walk
# geometry does not sit at their minimum, so it relaxes at the start of a
# run).

MASS_CHAIN = 12.011   # amu (carbon-like beads)
MASS_O = 15.9994
MASS_H = 1.008
TIP3P_RHH = 2.0 * TIP3P_ROH * math.sin(0.5 * TIP3P_THETA)
BOND_K, BOND_R0 = 300.0, 1.5               # U = k (r - r0)^2, kcal/mol/A^2, A
ANGLE_K, ANGLE_THETA0 = 50.0, math.radians(111.0)  # U = k (theta - theta0)^2
DIHEDRAL_K, DIHEDRAL_N, DIHEDRAL_PHASE = 0.2, 3, 0.0  # U = k (1 + cos(n phi - delta))


@dataclasses.dataclass
class MDTopology:
    """Bonded terms (int32 indices, FP32 parameters), rigid 3-site waters
    (O, H1, H2) and per-atom masses of one system."""

    mass: np.ndarray          # float32 [N] (amu)
    bonds: np.ndarray         # int32 [nb, 2]
    bond_k: np.ndarray        # float32 [nb]
    bond_r0: np.ndarray       # float32 [nb]
    angles: np.ndarray        # int32 [na, 3], the middle atom is the vertex
    angle_k: np.ndarray
    angle_theta0: np.ndarray  # radians
    dihedrals: np.ndarray     # int32 [nd, 4]
    dihedral_k: np.ndarray
    dihedral_n: np.ndarray    # int32
    dihedral_phase: np.ndarray  # radians
    waters: np.ndarray        # int32 [nw, 3]
    water_roh: float = TIP3P_ROH
    water_rhh: float = TIP3P_RHH


def md_topology(sys: System, n_chain: int = 0) -> MDTopology:
    """MD inputs of a water box (n_chain = 0) or of the solvated chain (its
    first n_chain atoms form the chain, the rest are waters)."""
    n = sys.n_atoms
    nw = (n - n_chain) // 3
    mass = np.concatenate([np.full(n_chain, MASS_CHAIN), np.tile([MASS_O, MASS_H, MASS_H], nw)])
    waters = (n_chain + 3 * np.arange(nw))[:, None] + np.arange(3)[None, :]
    i = np.arange(max(n_chain, 0))
    bonds = np.stack([i[:-1], i[:-1] + 1], 1) if n_chain > 1 else np.zeros((0, 2), np.int64)
    angles = np.stack([i[:-2], i[:-2] + 1, i[:-2] + 2], 1) if n_chain > 2 else np.zeros((0, 3), np.int64)
    dih = np.stack([i[:-3], i[:-3] + 1, i[:-3] + 2, i[:-3] + 3], 1) if n_chain > 3 else np.zeros((0, 4), np.int64)
    return MDTopology(
        mass=mass.astype(np.float32),
        bonds=bonds.astype(np.int32), bond_k=np.full(len(bonds), BOND_K, np.float32),
        bond_r0=np.full(len(bonds), BOND_R0, np.float32),
        angles=angles.astype(np.int32), angle_k=np.full(len(angles), ANGLE_K, np.float32),
        angle_theta0=np.full(len(angles), ANGLE_THETA0, np.float32),
        dihedrals=dih.astype(np.int32), dihedral_k=np.full(len(dih), DIHEDRAL_K, np.float32),
        dihedral_n=np.full(len(dih), DIHEDRAL_N, np.int32),
        dihedral_phase=np.full(len(dih), DIHEDRAL_PHASE, np.float32),
        waters=waters.astype(np.int32))


def hmr_masses(top: MDTopology, h_mass: float = 4.032) -> MDTopology:
    """Hydrogen mass repartitioning (section "Molecular dynamics on the GPU",
    after Feenstra et al.): each water H gets h_mass and its O gives up the
    difference, so every molecule keeps its mass (allows 4 fs steps)."""
    m = top.mass.astype(np.float64).copy()
    w = top.waters
    for h in (1, 2):
        m[w[:, 0]] -= h_mass - m[w[:, h]]
        m[w[:, h]] = h_mass
    return dataclasses.replace(top, mass=m.astype(np.float32))


def initial_velocities(top: MDTopology, temperature: float = 300.0, seed: int = 11) -> np.ndarray:
    """Seeded Maxwell-Boltzmann velocities (A/ps) at the temperature (K):
    each component N(0, kT/m) with kT in kcal/mol and 1 kcal/mol/amu =
    418.4 A^2/ps^2; the centre-of-mass velocity removed."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 200 + seed))
    kT = 0.0019872041 * temperature
    m = top.mass.astype(np.float64)
    v = rng.normal(size=(m.size, 3)) * np.sqrt(kT * 418.4 / m)[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v.astype(np.float32)


def make(name: str, **kw):
    table = {"lj_fcc": lj_fcc, "water_box": water_box, "solvated_chain": solvated_chain,
             "water_ensemble": water_ensemble, "big_water": big_water, "dhfr_chain_md": dhfr_chain_md}
    return table[name](**kw)


def target_forces(sys: System, seed: int = 7) -> np.ndarray:
    """Seeded random force targets F_target for the fitting loss."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 100 + seed))
    return rng.normal(0.0, 10.0, size=(sys.n_atoms, 3)).astype(np.float32)
