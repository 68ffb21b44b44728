"""Full-size parity of the largest workload: the 999,999-atom water box
(333,333 TIP3P-shaped waters, L ~ 215 A, rc 9 A, Ewald alpha 0.32), built and
evaluated with the default launch configuration, against the FP64 oracle's
cell-list evaluation of every atom (a few seconds on the host cores)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

import parity  # noqa: E402


def test_million_atom_water_box_full_parity():
    s = S.big_water()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    _, n_gpu, n_eval = ctx.debug_pairs(cap=0)
    torch.cuda.synchronize()
    ctx.status()
    F = F.cpu().numpy().astype(np.float64)
    E = E[0].cpu().numpy()
    W = W[0].cpu().numpy()
    Fo, Eo, Wo, n_oracle, Es, Eq = oracle.forces(s, method="cells", with_scale=True, with_sq=True)
    # the same unique pair set size (every pair evaluated once)
    assert n_gpu == n_oracle
    assert n_eval == n_gpu
    case = "water_1M"
    parity.check_forces(case, F, Fo)
    # E_LJ to 1e-6; the water Coulomb sum cancels to 1/6000 of sum |e_ij|: FP32 floor
    parity.check_energy(case, E, Eo, Es, bars=(parity.E_REL, "floor", "floor"),
                        notes=("", "water Coulomb sum cancels", "water Coulomb sum cancels"), Eq=Eq)
    parity.check_virial(case, W, Wo)


@pytest.mark.parametrize("n_waters", [100_000, 333_333])
def test_long_columns_sort_bit_exact(n_waters):
    # columns of about 8 nx atoms: 264 (100,000 waters: columns on both
    # sides of the 256-atom switch from rank sort to the bitonic network in
    # one build) and 400 (the 1 M-atom box: all bitonic)
    s = S.big_water() if n_waters == 333_333 else S._water_system(S.rng_for(44), n_waters, "w100k")
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    perm, cs = ctx.debug_cells()
    ctx.status()
    operm, ocs, _ = oracle.binning(s.pos, s.box)
    sizes = np.diff(ocs)
    print("column sizes", sizes.min(), sizes.max())
    assert np.array_equal(cs, ocs)
    assert np.array_equal(perm.astype(np.int64), operm)
