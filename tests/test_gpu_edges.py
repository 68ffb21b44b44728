"""GPU edge cases against the FP64 oracle: the maximum number of LJ types
(forward and adjoint), a droplet that leaves most columns of a large box
empty, a lone atom, pairs placed at the cutoff boundary in FP32, and a pair
list capacity that is too small (reported, not trapped)."""

import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

F_RMS, F_MAX, E_REL, W_REL = 5e-6, 1e-3, 1e-6, 1e-5

import parity  # noqa: E402


def run_forward(s):
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    _, n, _ = ctx.debug_pairs(cap=0)
    torch.cuda.synchronize()
    ctx.status()
    return F.cpu().numpy().astype(np.float64), E[0].cpu().numpy(), W[0].cpu().numpy(), n


def check_forward(s, bars=(E_REL,) * 3, notes=("",) * 3):
    F, E, W, n = run_forward(s)
    Fo, Eo, Wo, no, Es, Eq = oracle.forces(s, method="allpairs", with_scale=True, with_sq=True)
    assert n == no
    if np.linalg.norm(Fo) > 0:
        assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= F_RMS
    assert np.abs(F - Fo).max() <= F_MAX
    if np.abs(Eo).max() > 0:
        parity.check_energy(s.name, E, Eo, Es, bars=bars, notes=notes, Eq=Eq)
    else:
        assert np.abs(E).max() <= 1e-12
    if np.abs(Wo).max() > 0:
        assert np.abs(W - Wo).max() <= W_REL * np.abs(Wo).max()
    return F, E, W


def many_types(T=64, seed=3):
    """The 256-atom FCC crystal (nearest neighbours 4.05 A apart) with T
    random LJ types (sigma 2.5..3.5 A, eps 0.01..0.2) and neutral random
    charges, Ewald on: nearly every type pair occurs within the cutoff."""
    s = S.lj_fcc()
    rng = np.random.default_rng(seed)
    n = s.n_atoms
    typ = rng.integers(0, T, size=n).astype(np.int32)
    sig = rng.uniform(2.5, 3.5, size=T).astype(np.float32)
    eps = rng.uniform(0.01, 0.2, size=T).astype(np.float32)
    q = rng.normal(0.0, 0.3, size=n)
    q = (q - q.mean()).astype(np.float32)
    return dataclasses.replace(s, name="types64", type=typ, sigma=sig, epsilon=eps, q=q, ewald_alpha=0.32)


def test_sixty_four_types_forward():
    check_forward(many_types())


def test_sixty_four_types_adjoint():
    s = many_types()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    G = np.random.default_rng(4).normal(size=(s.n_atoms, 3)).astype(np.float32)
    Gd = torch.from_numpy(G).cuda()
    gpos, gq, gs_tab, ge_tab = ctx.backward(pos, q, t, Gd, None)
    torch.cuda.synchronize()
    ctx.status()
    dx, dq, dA, dB, aA, aB = oracle.backward(s, G.astype(np.float64), 0.0, with_scale=True)
    gpos = gpos.cpu().numpy()
    gq = gq.cpu().numpy()
    assert np.linalg.norm(gpos - dx) / np.linalg.norm(dx) <= 1e-4
    assert np.linalg.norm(gq - dq) / np.linalg.norm(dq) <= 1e-4


def test_droplet_leaves_most_columns_empty():
    # 300 waters packed into one corner of a box eight times their volume
    w = S._water_system(S.rng_for(22), 300, "w300")
    L = w.box * 2.0
    s = dataclasses.replace(w, name="droplet", box=L.astype(np.float32))
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    perm, cs = ctx.debug_cells()
    counts = np.diff(cs)
    assert (counts == 0).mean() > 0.5  # most columns are empty
    # 300 randomly oriented waters: the Coulomb sum cancels (FP32 floor)
    check_forward(s, bars=(E_REL, "floor", "floor"), notes=("", "water Coulomb sum cancels", "water Coulomb sum cancels"))


def test_lone_atom():
    s = S.System("one", np.array([[1.0, 2.0, 3.0]], np.float32), np.array([0.5], np.float32),
                 np.zeros(1, np.int32), np.array([3.0], np.float32), np.array([0.2], np.float32),
                 np.full(3, 25.0, np.float32), np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32),
                 9.0, 7.5, 0.32)
    F, E, W, n = run_forward(s)
    assert n == 0
    assert np.all(F == 0.0) and np.all(E == 0.0) and np.all(W == 0.0)


def test_pairs_straddling_the_cutoff():
    # pairs at FP32 distances just below, at and just above rc, also across
    # the periodic boundary: the membership predicate decides exactly as the
    # oracle's
    rc = np.float32(9.0)
    L = np.float32(30.0)
    pts = []
    for k, d in enumerate([np.nextafter(rc, np.float32(0)), rc, np.nextafter(rc, np.float32(20))]):
        y = np.float32(3.0 + 7.0 * k)
        pts += [[np.float32(1.0), y, np.float32(5.0)], [np.float32(1.0) + d, y, np.float32(5.0)]]
        # the same separation across the x boundary
        pts += [[np.float32(0.5), y, np.float32(20.0)], [np.float32(0.5) - d + L, y, np.float32(20.0)]]
    pos = np.array(pts, np.float32)
    n = pos.shape[0]
    s = S.System("edge", pos, np.where(np.arange(n) % 2 == 0, 0.4, -0.4).astype(np.float32),
                 np.zeros(n, np.int32), np.array([3.0], np.float32), np.array([0.2], np.float32),
                 np.full(3, L, np.float32), np.zeros((0, 2), np.int32), np.zeros((0, 2), np.int32),
                 float(rc), 7.5, 0.32)
    F, E, W, ng = run_forward(s)
    no = len(oracle.pairs(s))
    assert ng == no
    Fo, Eo, Wo, npo = oracle.forces(s, method="allpairs")
    assert np.abs(F - Fo).max() <= F_MAX


def test_list_capacity_overflow_is_reported():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    ctx.set_tuning(list_capacity=64)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    ctx.forces(pos, q, t)
    assert ctx.status(raise_on_error=False) == 10  # NB_ERR_CAPACITY


def test_tuning_is_validated_and_default_split_is_one():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    for bad in (dict(list_split=-1), dict(list_split=9), dict(blocks_per_sm=0), dict(blocks_per_sm=9),
                dict(group_clusters=2), dict(group_clusters=3), dict(group_clusters=16)):
        with pytest.raises(nb.NbError):
            ctx.set_tuning(**bad)
    pos, q, t = nb.concat_inputs([s])
    outs = {}
    for split in (0, 1, 1, 2):  # 0 selects the default split (1); every split repeats bit for bit
        ctx.set_tuning(list_split=split)
        ctx.build(pos)
        F, E, W = ctx.forces(pos, q, t)
        torch.cuda.synchronize()
        outs.setdefault(split, []).append((F.clone(), E.clone(), W.clone()))
    ctx.status()
    a, b, c = outs[0][0], outs[1][0], outs[1][1]
    for x, y in ((a, b), (b, c)):
        assert all(torch.equal(u, v) for u, v in zip(x, y))
    # another split only moves where the FP32 sums are cut
    F2, F1 = outs[2][0][0].double(), a[0].double()
    assert (torch.linalg.norm(F2 - F1) / torch.linalg.norm(F1)).item() < 1e-6


def test_group_size_change_needs_a_new_build_and_keeps_parity():
    # the i-group size (4 or 8 clusters) is a build parameter: after a change
    # the forces are refused until the next build, which then agrees with the
    # oracle at the same bars
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    ctx.forces(pos, q, t)
    ctx.set_tuning(group_clusters=4)
    with pytest.raises(nb.NbError) as e:
        ctx.forces(pos, q, t)
    assert e.value.code == 5  # NB_ERR_NOT_BUILT
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    _, n, _ = ctx.debug_pairs(cap=0)
    torch.cuda.synchronize()
    ctx.status()
    Fo, Eo, Wo, no, Es, Eq = oracle.forces(s, method="allpairs", with_scale=True, with_sq=True)
    assert n == no
    parity.check_forces("water_box group4", F.double().cpu().numpy(), Fo)
    parity.check_energy("water_box group4", E[0].cpu().numpy(), Eo, Es, bars=(E_REL, "floor", "floor"), Eq=Eq)
    assert ctx.tuning()["group_clusters"] == 4


@pytest.mark.parametrize("which", ["water_x", "chain_y"])
def test_orthorhombic_boxes(which):
    # non-cubic boxes (different column counts per axis, a vacuum gap along
    # the stretched axis): cells and pairs bit-exact, forces, energies and
    # virial within the bars
    if which == "water_x":
        w = S._water_system(S.rng_for(23), 900, "w900")
        s = dataclasses.replace(w, name="water_x", box=(w.box * np.array([1.35, 1.0, 1.0])).astype(np.float32))
    else:
        c = S.solvated_chain(k=24, n_chain=300, n_waters=900, L=31.0)
        s = dataclasses.replace(c, name="chain_y", box=(c.box * np.array([1.0, 1.2, 1.0])).astype(np.float32))
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    perm, cs = ctx.debug_cells()
    operm, ocs, _ = oracle.binning(s.pos, s.box)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(perm.astype(np.int64), operm)
    ctx.forces(pos, q, t)
    ij, n, _ = ctx.debug_pairs()
    ctx.status()
    assert np.array_equal(ij, oracle.pairs(s))
    check_forward(s, bars=(E_REL, "floor", "floor"), notes=("", "water Coulomb sum cancels", "water Coulomb sum cancels"))


def sixteen_partners():
    """A 200-atom chain in 600 waters where every interior chain atom has the
    maximum of 16 topology partners: excluded (i, i +- 1..4) and scaled 1-4
    (i, i +- 5..8), partners spread over several clusters."""
    c = S.solvated_chain(k=25, n_chain=200, n_waters=600, L=26.0)
    n = 200
    ex = [(i, i + d) for d in range(1, 5) for i in range(n - d)]
    p14 = [(i, i + d) for d in range(5, 9) for i in range(n - d)]
    wex = c.excl[c.excl.min(axis=1) >= n]  # the waters' own exclusions
    excl = np.concatenate([np.array(ex, np.int32), wex.astype(np.int32)])
    return dataclasses.replace(c, name="chain_k16", excl=excl, pairs14=np.array(p14, np.int32))


@pytest.mark.parametrize("group", [1, 8])
def test_sixteen_topology_partners_per_atom(group):
    s = sixteen_partners()
    counts = np.bincount(np.concatenate([s.excl.ravel(), s.pairs14.ravel()]), minlength=s.n_atoms)
    assert counts.max() == 16
    ctx = nb.Nonbonded(s)
    if group != 1:
        ctx.set_tuning(group_clusters=group, list_split=2)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    ij, n, _ = ctx.debug_pairs()
    torch.cuda.synchronize()
    ctx.status()
    assert np.array_equal(ij, oracle.pairs(s))
    Fo, Eo, Wo, no, Es, Eq = oracle.forces(s, method="allpairs", with_scale=True, with_sq=True)
    F = F.double().cpu().numpy()
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= F_RMS
    assert np.abs(F - Fo).max() <= F_MAX
    parity.check_energy(f"chain_k16 g{group}", E[0].cpu().numpy(), Eo, Es, bars=(E_REL, "floor", "floor"),
                        notes=("", "water Coulomb sum cancels", "water Coulomb sum cancels"), Eq=Eq)
    W = W[0].cpu().numpy()
    assert np.abs(W - Wo).max() <= W_REL * np.abs(Wo).max()
