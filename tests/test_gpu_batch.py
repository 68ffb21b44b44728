"""Batched form: many independent water boxes of uneven size in one
persistent launch, captured in a CUDA graph, against the FP64 oracle per
system and against separate per-system contexts; the autotuner keeps parity."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import autotune
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

import parity  # noqa: E402

# Literal energy bars of the water boxes: E_LJ 1e-6; the Coulomb sum of
# randomly oriented TIP3P-shaped waters cancels to 1/6000 of sum |e_ij| and is
# held to the FP32 floor of the pair arithmetic (parity.fp32_floor).
BARS = (parity.E_REL, "floor", "floor")
NOTES = ("", "water Coulomb sum cancels", "water Coulomb sum cancels")


def check_system(F, E, W, s, case):
    Fo, Eo, Wo, _, Es, Eq = oracle.forces(s, method="cells", with_scale=True, with_sq=True)
    parity.check_forces(case, F, Fo)
    parity.check_energy(case, E, Eo, Es, bars=BARS, notes=NOTES, Eq=Eq)
    parity.check_virial(case, W, Wo)


def test_ensemble_graph_matches_oracle_per_system():
    systems = S.water_ensemble()
    assert len(systems) == 64
    ctx = nb.Nonbonded(systems)
    pos, q, t = nb.concat_inputs(systems)
    N = pos.shape[0]
    F = torch.empty((N, 3), device="cuda")
    E = torch.empty((64, 2), dtype=torch.float64, device="cuda")
    W = torch.empty((64, 6), dtype=torch.float64, device="cuda")
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
    torch.cuda.synchronize()
    ctx.status()
    Fh, Eh, Wh = F.double().cpu().numpy(), E.cpu().numpy(), W.cpu().numpy()
    off = 0
    rng = np.random.default_rng(0)
    pick = set(rng.choice(64, 12, replace=False).tolist()) | {int(np.argmin([s.n_atoms for s in systems])),
                                                              int(np.argmax([s.n_atoms for s in systems]))}
    for k, s in enumerate(systems):
        if k in pick:
            check_system(Fh[off:off + s.n_atoms], Eh[k], Wh[k], s, f"ensemble64[{k}] n={s.n_atoms}")
        off += s.n_atoms


def test_batch_equals_separate_contexts():
    systems = S.water_ensemble(n_sys=8, k=31)
    ctx = nb.Nonbonded(systems)
    pos, q, t = nb.concat_inputs(systems)
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    off = 0
    for k, s in enumerate(systems):
        c1 = nb.Nonbonded(s)
        p1, q1, t1 = nb.concat_inputs([s])
        c1.build(p1)
        F1, E1, W1 = c1.forces(p1, q1, t1)
        torch.cuda.synchronize()
        # same kernels, same per-atom summation order: identical bits
        assert torch.equal(F[off:off + s.n_atoms], F1)
        assert torch.equal(E[k], E1[0]) and torch.equal(W[k], W1[0])
        off += s.n_atoms
    ctx.status()


def test_autotuner_picks_a_valid_configuration_and_keeps_parity():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    rec = autotune.autotune(ctx, pos, q, t, candidates=[dict(blocks_per_sm=b, list_split=c)
                                                        for b in (1, 3) for c in (1, 4)], reps=2)
    assert rec["best"] in [c for _, c in rec["table"]]
    assert ctx.tuning()["blocks_per_sm"] == rec["best"]["blocks_per_sm"]
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    check_system(F.double().cpu().numpy(), E.cpu().numpy()[0], W.cpu().numpy()[0], s, "water_box autotuned")
