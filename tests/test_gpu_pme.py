"""Smooth PME on the GPU against the FP64 oracle: the long-range part alone
(reciprocal sum, self term, excluded and 1-4 corrections) against the
oracle's smooth PME on the same grid and order, the full electrostatics of
nb_forces with PME against real space + PME + corrections, PME against the
direct Ewald sum, bit-identical reruns, CUDA-graph replay and the
unsupported combinations.

Tolerances.  The oracle is FP64 throughout; the GPU spreads FP32 B-spline
weights into a fixed-point grid and runs FP32 FFTs, whose rounding error is
about u log2(K1 K2 K3) ~ 1e-6 relative (u = 2^-24), so the reciprocal-space
energy, forces and virial are held to 5e-6 relative (measured: 1.3e-6).  The self term sums
q^2 in fixed point (the FMA-exact hi + lo parts of q^2, each rounded to
2^-36: at most 2^-37 per atom, the same for every atom of a kind) and scales
it in FP64 (1e-10).  The pair
corrections are FP32 pair arithmetic (erff, expf, a division: a few ulp
per pair, the same for every rigid water), held to 1e-6.  The total forces of
nb_forces keep the short-range bound (relative RMS 5e-6), since the
reciprocal forces are a small part of the total.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle.ewald as ew
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

REC_REL = 5e-6
SELF_REL = 1e-10
CORR_REL = 1e-6
F_RMS, F_MAX, E_REL, W_REL = 5e-6, 1e-3, 1e-6, 1e-5

import parity  # noqa: E402


def pme_gpu(s, grid, order):
    ctx = nb.Nonbonded(s)
    ctx.set_pme(grid, order)
    pos, q, _ = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, W = ctx.pme_forces(pos, q)
    torch.cuda.synchronize()
    ctx.status()
    return ctx, F.double().cpu().numpy(), E.cpu().numpy(), W.cpu().numpy()


def pme_oracle(s, grid, order):
    Fr, Er, Wr = ew.spme(s, grid, order)
    Fc, Es, Ep, Wc = ew.ewald_corrections(s)
    return Fr, Er, Wr, Fc, Es, Ep, Wc


def report(name, **kw):
    print(name, " ".join(f"{k}={v:.3e}" for k, v in kw.items()))


@pytest.mark.parametrize("which,grid,order", [("water", (40, 40, 40), 4), ("chain", (64, 64, 64), 4),
                                              ("water", (48, 40, 36), 6), ("water", (32, 32, 32), 8)])
def test_long_range_part_matches_oracle_pme(which, grid, order):
    s = S.water_box() if which == "water" else S.solvated_chain()
    _, F, E, W = pme_gpu(s, grid, order)
    Fr, Er, Wr, Fc, Es, Ep, Wc = pme_oracle(s, grid, order)
    # forces: reciprocal and corrections together, as the library returns them
    Fo = Fr + Fc
    rel = np.linalg.norm(F - Fo) / np.linalg.norm(Fo)
    erec = abs(E[0] - Er) / abs(Er)
    eself = abs(E[1] - Es) / abs(Es)
    epair = abs(E[2] - Ep) / abs(Ep)
    Wo = Wr + Wc
    wrel = np.abs(W - Wo).max() / np.abs(Wo).max()
    report(f"pme {which} {grid} n={order}", f_rms=rel, e_rec=erec, e_self=eself, e_pair=epair, w=wrel)
    tag = f"pme {which} {grid} n={order}"
    parity.record(tag, "force rel RMS", rel, REC_REL)
    parity.record(tag, "E_recip |dE|/|E|", erec, REC_REL)
    parity.record(tag, "E_self |dE|/|E|", eself, SELF_REL)
    parity.record(tag, "E_pair corr |dE|/|E|", epair, CORR_REL)
    parity.record(tag, "virial max|dW|/max|W|", wrel, REC_REL)
    assert rel <= REC_REL
    assert erec <= REC_REL
    assert eself <= SELF_REL
    assert epair <= CORR_REL
    assert wrel <= REC_REL


def test_nb_forces_with_pme_is_the_full_electrostatics():
    s = S.solvated_chain()
    grid, order = (64, 64, 64), 4
    ctx = nb.Nonbonded(s)
    ctx.set_pme(grid, order)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    F = F.double().cpu().numpy()
    E = E[0].cpu().numpy()
    W = W[0].cpu().numpy()
    Fs, Eo, Wo, _, Esc = oracle.forces(s, method="cells", with_scale=True)
    Fr, Er, Wr, Fc, Es, Ep, Wc = pme_oracle(s, grid, order)
    Ft = Fs + Fr + Fc
    rel = np.linalg.norm(F - Ft) / np.linalg.norm(Ft)
    report("full", f_rms=rel, f_max=np.abs(F - Ft).max())
    assert rel <= F_RMS
    assert np.abs(F - Ft).max() <= F_MAX
    ec = Eo[1] + Er + Es + Ep
    scale = Esc[1] + abs(Er) + abs(Es) + abs(Ep)
    # the literal relative errors of E_LJ and of the full Ewald E_Coul (real
    # space + reciprocal + self + exclusion/1-4 corrections: terms up to 80
    # times larger than the total, whose errors must stay below 1e-6 of it)
    parity.check_energy(f"pme {s.name}", E, np.array([Eo[0], ec]), np.array([Esc[0], scale]))
    Wt = Wo + Wr + Wc
    assert np.abs(W - Wt).max() <= W_REL * np.abs(Wt).max()


def test_pme_converges_to_the_direct_ewald_sum():
    s = S.water_box()
    _, F, E, W = pme_gpu(s, (64, 64, 64), 8)
    Fd, Ed, Wd = ew.ewald_recip(s, 20)
    Fc, Es, Ep, Wc = ew.ewald_corrections(s)
    rel = np.linalg.norm(F - (Fd + Fc)) / np.linalg.norm(Fd + Fc)
    report("pme vs direct", f_rms=rel, e=abs(E[0] - Ed) / abs(Ed))
    assert rel <= 2e-5
    assert abs(E[0] - Ed) <= 2e-5 * abs(Ed)


def test_pme_reruns_are_bit_identical_and_graph_replay_agrees():
    s = S.solvated_chain()
    ctx = nb.Nonbonded(s)
    ctx.set_pme((64, 64, 64), 4)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    outs = []
    for _ in range(2):
        F, E, W = ctx.forces(pos, q, t)
        outs.append((F.clone(), E.clone(), W.clone()))
    N = pos.shape[0]
    F = torch.empty((N, 3), device="cuda")
    E = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    W = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.build(pos)
        ctx.forces(pos, q, t, F=F, energy=E, virial=W)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            ctx.build(pos)
            ctx.forces(pos, q, t, F=F, energy=E, virial=W)
    torch.cuda.current_stream().wait_stream(side)
    F.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ctx.status()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    assert torch.equal(F, outs[0][0])
    assert torch.equal(E, outs[0][1])
    assert torch.equal(W, outs[0][2])


def test_disable_and_unsupported_combinations():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F0, E0, _ = ctx.forces(pos, q, t)
    ctx.set_pme((40, 40, 40), 4)
    F1, E1, _ = ctx.forces(pos, q, t)
    assert not torch.equal(F0, F1)
    G = torch.zeros_like(F1)
    with pytest.raises(nb.NbError) as ei:
        ctx.backward(pos, q, t, G)
    assert ei.value.code == 11  # NB_ERR_UNSUPPORTED: no PME adjoint
    ctx.set_pme(None)
    F2, E2, _ = ctx.forces(pos, q, t)
    assert torch.equal(F0, F2) and torch.equal(E0, E2)
    with pytest.raises(nb.NbError) as ei:
        ctx.set_pme((40, 40, 40), 5)
    assert ei.value.code == 11
    batch = nb.Nonbonded([s, s])
    with pytest.raises(nb.NbError) as ei:
        batch.set_pme((40, 40, 40), 4)
    assert ei.value.code == 11
    torch.cuda.synchronize()


def test_neutral_pair_of_excluded_charges_alone():
    # an excluded +q/-q pair in a large box: the corrections cancel the
    # reciprocal sum's intramolecular part, so what is left is the periodic
    # images' dipole interaction, about ke 2 pi p^2 / (3 V) = 3.6e-3 here --
    # a sign error would leave ~ke q^2/r = 73
    pos = np.array([[20.0, 20.0, 20.0], [21.0, 20.5, 20.2]], np.float32)
    s = S.System("dimer", pos, np.array([0.5, -0.5], np.float32), np.zeros(2, np.int32),
                 np.array([1.0], np.float32), np.array([0.0], np.float32), np.full(3, 40.0, np.float32),
                 np.array([[0, 1]], np.int32), np.zeros((0, 2), np.int32), 9.0, 7.5, 0.35)
    _, F, E, W = pme_gpu(s, (48, 48, 48), 6)
    assert abs(E.sum()) <= 1e-2
    assert np.abs(F).max() <= 1e-2
    Fr, Er, Wr, Fc, Es, Ep, Wc = pme_oracle(s, (48, 48, 48), 6)
    assert abs(E.sum() - (Er + Es + Ep)) <= REC_REL * (abs(Er) + abs(Es) + abs(Ep))
    assert np.abs(F - (Fr + Fc)).max() <= REC_REL * np.abs(Fr).max()


@pytest.mark.parametrize("group", [4, 8])
def test_pme_with_group_tiles(group):
    # nb_forces with PME when the short-range kernel runs 4- or 8-cluster
    # i-groups (and nb_step, which forks PME before the lists): the same
    # full electrostatics as with single-cluster groups, to FP32 rounding
    s = S.solvated_chain()
    pos, q, t = nb.concat_inputs([s])
    out = []
    for g in (1, group):
        ctx = nb.Nonbonded(s)
        ctx.set_pme((64, 64, 64), 4)
        if g != 1:
            ctx.set_tuning(group_clusters=g, list_split=2)
        ctx.build(pos)
        F, E, W = ctx.forces(pos, q, t)
        F2, E2, W2 = ctx.step(pos, q, t)
        torch.cuda.synchronize()
        ctx.status()
        assert torch.equal(F, F2) and torch.equal(E, E2) and torch.equal(W, W2)
        out.append((F.double().cpu().numpy(), E[0].cpu().numpy(), W[0].cpu().numpy()))
    (F1, E1, W1), (Fg, Eg, Wg) = out
    assert np.linalg.norm(Fg - F1) / np.linalg.norm(F1) <= 1e-6
    # FP32 partial sums cut at different places: within the literal bar
    assert np.all(np.abs(Eg - E1) <= 1e-6 * np.abs(E1))
    assert np.abs(Wg - W1).max() <= 1e-6 * np.abs(W1).max()
