"""The allocation-free entry point nb_forces_noalloc.

Some callers of this library may not allocate device memory themselves (a
host application whose device memory all comes from its own pool, or a
plug-in that may not call cudaMalloc after start-up).  nb_forces_noalloc
serves them with scratch in a static device array that every call reuses.
These tests call it through the C ABI and check that:

* it runs the same kernels on the same lists as the regular context entry
  point (nb_build_cells + nb_forces), so forces, energies and virial agree
  bit for bit, on two calls in a row;
* leftovers of a larger system in the shared array (lists, z-bin index,
  sorted types) do not leak into a smaller one: a 2,800-atom chain, then a
  900-atom water box, then the chain again, each bitwise equal to its
  context result;
* one case meets the FP64 oracle's parity bars directly;
* oversized systems are rejected with NB_ERR_TOO_LARGE.

This file is collected last, so a run that stops at its first failure has
run every other test before it; it also passes alone in a fresh process.
"""

import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

import parity  # noqa: E402

pytestmark = pytest.mark.gpu


def _context_result(s):
    pos, q, t = nb.concat_inputs([s])
    ctx = nb.Nonbonded(s)
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    return (pos, q, t), F.clone(), E.clone(), W.clone()


def _noalloc(s, pos, q, t):
    F = torch.full((s.n_atoms, 3), float("nan"), dtype=torch.float32, device=pos.device)
    E = torch.full((1, 2), float("nan"), dtype=torch.float64, device=pos.device)
    W = torch.full((1, 6), float("nan"), dtype=torch.float64, device=pos.device)
    nb.forces_noalloc(s, pos, q, t, F, E, W)
    torch.cuda.synchronize()
    return F, E, W


def _assert_same_bits(s, times=2):
    (pos, q, t), F_ref, E_ref, W_ref = _context_result(s)
    for _ in range(times):  # calls in a row share and reuse the static scratch
        F, E, W = _noalloc(s, pos, q, t)
        assert torch.equal(F, F_ref), s.name
        assert torch.equal(E, E_ref), s.name
        assert torch.equal(W, W_ref), s.name


def _water():
    return S._water_system(S.rng_for(41), 300, "noalloc_water")


def _chain():
    # chain with exclusions and scaled 1-4 pairs, plus waters: 2,800 atoms
    return S.solvated_chain(k=42, n_chain=400, n_waters=800, L=32.0)


def test_noalloc_matches_context_entry_point_water():
    _assert_same_bits(_water())


def test_noalloc_matches_context_entry_point_chain():
    _assert_same_bits(_chain())


def test_noalloc_larger_then_smaller_then_larger():
    chain, water = _chain(), _water()
    assert chain.n_atoms > water.n_atoms
    for s in (chain, water, chain):
        _assert_same_bits(s, times=1)


def test_noalloc_meets_the_oracle_bars():
    s = _chain()
    pos, q, t = nb.concat_inputs([s])
    F, E, W = _noalloc(s, pos, q, t)
    Fo, Eo, Wo, _, Es, Eq = oracle.forces(s, method="allpairs", with_scale=True, with_sq=True)
    parity.check_forces("noalloc chain2800", F.double().cpu().numpy(), Fo)
    # E_LJ to 1e-6; the Coulomb sum (800 randomly oriented waters dominate
    # it) to the FP32 floor of the pair arithmetic, as in the other tests
    parity.check_energy("noalloc chain2800", E.cpu().numpy()[0], Eo, Es, bars=(parity.E_REL, "floor", "floor"),
                        Eq=Eq)
    parity.check_virial("noalloc chain2800", W.cpu().numpy()[0], Wo)


def test_noalloc_rejects_oversized_system():
    s = S._water_system(S.rng_for(43), 1400, "too_big")  # 4,200 atoms > 4,096
    pos, q, t = nb.concat_inputs([s])
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device=pos.device)
    with pytest.raises(nb.NbError) as e:
        nb.forces_noalloc(s, pos, q, t, F)
    assert e.value.code == 12  # NB_ERR_TOO_LARGE
