"""nb_step (rebuild + forces in one call, the charges and types packed by the
column sort) against nb_build_cells + nb_forces on the same inputs: forces,
energies and virial bit for bit, alone, in a batch, with smooth PME and with
tables; the context is built afterwards; a bad type index is reported; the
arrays may be page-locked host memory (same bits)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu


def _two_calls(systems, setup=None):
    ctx = nb.Nonbonded(systems if len(systems) > 1 else systems[0])
    if setup:
        setup(ctx)
    pos, q, t = nb.concat_inputs(systems)
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    return (pos, q, t), F.clone(), E.clone(), W.clone()


def _one_call(systems, inp, setup=None):
    ctx = nb.Nonbonded(systems if len(systems) > 1 else systems[0])
    if setup:
        setup(ctx)
    pos, q, t = inp
    F, E, W = ctx.step(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    return ctx, F, E, W


CASES = {
    "solvated_chain": (lambda: [S.solvated_chain()], None),
    "water_box": (lambda: [S.water_box()], None),
    "batch3": (lambda: S.water_ensemble()[:3], None),
    "chain_pme": (lambda: [S.solvated_chain()], lambda c: c.set_pme((64, 64, 64), 4)),
    "water_tables": (lambda: [S.water_box()], lambda c: c.set_tables(4096)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_step_equals_build_then_forces(name):
    make, setup = CASES[name]
    systems = make()
    inp, F0, E0, W0 = _two_calls(systems, setup)
    ctx, F1, E1, W1 = _one_call(systems, inp, setup)
    assert torch.equal(F1, F0), name
    assert torch.equal(E1, E0), name
    assert torch.equal(W1, W0), name
    # the step leaves the context built on these positions
    F2, E2, W2 = ctx.forces(*inp)
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(F2, F0) and torch.equal(E2, E0) and torch.equal(W2, W0)


def test_step_reports_a_bad_type():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    t[5] = s.n_types  # out of range
    ctx.step(pos, q, t)
    torch.cuda.synchronize()
    with pytest.raises(nb.NbError) as e:
        ctx.status()
    assert e.value.code == 1  # NB_ERR_INVALID_ARG (a type index outside [0, T))


@pytest.mark.parametrize("group", [1, 4])
def test_fill_counters_are_consistent(group):
    # every pair sits in an evaluated half, every evaluated half in a visited
    # tile, for single-cluster and four-cluster i-groups
    s = S.solvated_chain()
    ctx = nb.Nonbonded(s)
    ctx.set_tuning(group_clusters=group)
    pos, q, t = nb.concat_inputs([s])
    ctx.step(pos, q, t)
    _, n, _ = ctx.debug_pairs(cap=0)
    tiles, halves = ctx.debug_fill()
    ctx.status()
    print("group", group, "pairs", n, "tiles", tiles, "halves", halves, "lane fill", n / (32 * halves))
    assert 0 < n <= 32 * halves <= 64 * tiles
    assert halves <= 2 * tiles
    assert 0.2 < n / (32 * halves) < 0.9


@pytest.mark.parametrize("pme", [False, True])
def test_step_replays_from_a_cuda_graph(pme):
    # the bench's timed step: nb_step captured once on a side stream and
    # replayed; the results equal those of plain calls bit for bit
    s = S.solvated_chain()
    ctx = nb.Nonbonded(s)
    if pme:
        ctx.set_pme((64, 64, 64), 4)
    pos, q, t = nb.concat_inputs([s])
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    E = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    W = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.step(pos, q, t, F=F, energy=E, virial=W)
    torch.cuda.synchronize()
    F0, E0, W0 = F.clone(), E.clone(), W.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        ctx.step(pos, q, t, F=F, energy=E, virial=W)  # the context moves to this stream outside the capture
        with torch.cuda.graph(g, stream=side):
            ctx.step(pos, q, t, F=F, energy=E, virial=W)
    torch.cuda.current_stream().wait_stream(side)
    F.zero_()
    E.zero_()
    W.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(F, F0) and torch.equal(E, E0) and torch.equal(W, W0)


@pytest.mark.parametrize("pme", [False, True])
def test_step_on_page_locked_host_arrays(pme):
    # inputs and outputs in page-locked host memory, read and written by the
    # kernels in place: the same bits as with device arrays, plain and from
    # a CUDA graph
    s = S.solvated_chain()
    ctx = nb.Nonbonded(s)
    if pme:
        ctx.set_pme((64, 64, 64), 4)
    pos, q, t = nb.concat_inputs([s])
    F0, E0, W0 = ctx.step(pos, q, t)
    torch.cuda.synchronize()
    hpos, hq, ht = (x.cpu().pin_memory() for x in (pos, q, t))
    F, E, W = ctx.step(hpos, hq, ht)
    torch.cuda.synchronize()
    ctx.status()
    assert F.device.type == "cpu" and F.is_pinned()
    assert torch.equal(F, F0.cpu()) and torch.equal(E, E0.cpu()) and torch.equal(W, W0.cpu())
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        ctx.step(hpos, hq, ht, F=F, energy=E, virial=W)
        with torch.cuda.graph(g, stream=side):
            ctx.step(hpos, hq, ht, F=F, energy=E, virial=W)
    torch.cuda.current_stream().wait_stream(side)
    F.zero_()
    E.zero_()
    W.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(F, F0.cpu()) and torch.equal(E, E0.cpu()) and torch.equal(W, W0.cpu())


def test_step_rejects_pageable_host_arrays():
    s = S.water_box()
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    with pytest.raises(ValueError):
        ctx.step(pos.cpu(), q, t)
