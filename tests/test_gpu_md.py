"""The MD step on the GPU (nb_md_init / nb_md_step / nb_bonded_forces)
against the FP64 oracle of oracle/md.py.

Tolerances.  Bonded terms are FP32 (atan2f, cross products of A-sized
vectors): forces to 1e-5 relative RMS.  One step moves positions by dt v
(~0.01 A) in FP32 coordinates of up to 62 A, whose rounding is ~4e-6 A, so
positions are compared to 2e-5 A (minimum image) and velocities to 1e-5
relative RMS; after a few steps both grow with the FP32 differences of the
forces.  Constraints hold to the FP32 resolution of the coordinates.
"""

import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle.md as omd
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu


def setup(s, top, gamma=0.0, dt=0.001, pme=None, seed=2009):
    ctx = nb.Nonbonded(s)
    if pme:
        ctx.set_pme(*pme)
    ctx.md_init(top, dt=dt, gamma=gamma, temperature=300.0, seed=seed)
    pos, q, t = nb.concat_inputs([s])
    return ctx, pos, q, t


def min_image(d, L):
    return d - L * np.rint(d / L)


def test_bonded_forces_match_oracle():
    s = S.solvated_chain()
    top = S.md_topology(s, n_chain=2500)
    ctx, pos, q, t = setup(s, top)
    F, E = ctx.bonded_forces(pos)
    torch.cuda.synchronize()
    ctx.status()
    Fo, Eo, _ = omd.bonded(top, s.pos.astype(np.float64), s.box)
    F = F.double().cpu().numpy()
    rel = np.linalg.norm(F - Fo) / np.linalg.norm(Fo)
    print("bonded f_rms", rel)
    assert rel <= 1e-5
    for k in range(3):
        assert abs(E[k].item() - Eo[k]) <= 1e-6 * max(abs(Eo[k]), 1.0)


def water(nw=512, seed=41):
    s = S._water_system(S.rng_for(seed), nw, f"w{nw}")
    return s, S.md_topology(s)


@pytest.mark.parametrize("gamma", [0.0, 5.0])
def test_one_step_matches_oracle(gamma):
    s, top = water()
    ctx, pos, q, t = setup(s, top, gamma=gamma)
    v0 = S.initial_velocities(top, 300.0)
    vel = torch.from_numpy(v0).cuda()
    E = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_step(pos, vel, q, t, 1, E)
    torch.cuda.synchronize()
    ctx.status()
    prm = omd.MDParams(dt=0.001, gamma=gamma, temperature=300.0, seed=2009)
    x = s.pos.astype(np.float64)
    F, _ = omd.forces_at(s, top, x, prm)
    xo, vo, _, Eo = omd.step(s, top, x, v0.astype(np.float64), F, 0, prm)
    L = s.box.astype(np.float64)
    dx = np.abs(min_image(pos.double().cpu().numpy() - xo, L)).max()
    vg = vel.double().cpu().numpy()
    rv = np.linalg.norm(vg - vo) / np.linalg.norm(vo)
    print("step gamma", gamma, "max dx", dx, "v rel", rv)
    assert dx <= 2e-5
    assert rv <= 1e-5
    Eg = E.cpu().numpy()
    assert abs(Eg[5] - Eo[5]) <= 1e-5 * Eo[5]  # kinetic energy


def test_solvated_chain_with_pme_three_steps():
    s = S.solvated_chain()
    top = S.md_topology(s, n_chain=2500)
    pme = ((64, 64, 64), 4)
    ctx, pos, q, t = setup(s, top, gamma=1.0, dt=0.002, pme=pme)
    v0 = S.initial_velocities(top, 300.0)
    vel = torch.from_numpy(v0).cuda()
    E = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_step(pos, vel, q, t, 3, E)
    torch.cuda.synchronize()
    ctx.status()
    prm = omd.MDParams(dt=0.002, gamma=1.0, temperature=300.0, seed=2009, pme=pme)
    x = s.pos.astype(np.float64)
    v = v0.astype(np.float64)
    F, _ = omd.forces_at(s, top, x, prm)
    for k in range(3):
        x, v, F, Eo = omd.step(s, top, x, v, F, k, prm)
    L = s.box.astype(np.float64)
    dx = np.abs(min_image(pos.double().cpu().numpy() - x, L)).max()
    rv = np.linalg.norm(vel.double().cpu().numpy() - v) / np.linalg.norm(v)
    Eg = E.cpu().numpy()
    print("chain 3 steps max dx", dx, "v rel", rv, "E", Eg, Eo)
    assert dx <= 1e-4
    assert rv <= 1e-4
    assert abs(Eg[5] - Eo[5]) <= 1e-4 * Eo[5]
    for k in range(2, 5):
        assert abs(Eg[k] - Eo[k]) <= 1e-4 * max(abs(Eo[k]), 1.0)


def test_constraints_hold_and_nve_energy_is_conserved():
    s, top = water(nw=512)
    ctx, pos, q, t = setup(s, top, gamma=0.0, dt=0.001)
    vel = torch.from_numpy(S.initial_velocities(top, 300.0)).cuda()
    E = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_step(pos, vel, q, t, 50, E)  # relax the synthetic start
    torch.cuda.synchronize()
    E0 = E.sum().item()
    ke = []
    tot = []
    for _ in range(20):
        ctx.md_step(pos, vel, q, t, 10, E)
        e = E.cpu().numpy()
        tot.append(e.sum())
        ke.append(e[5])
    ctx.status()
    x = pos.double().cpu().numpy()
    L = s.box.astype(np.float64)
    w = top.waters
    for (a, b), d in (((0, 1), top.water_roh), ((0, 2), top.water_roh), ((1, 2), top.water_rhh)):
        r = np.linalg.norm(min_image(x[w[:, a]] - x[w[:, b]], L), axis=1)
        assert np.abs(r - d).max() < 5e-5
    print("NVE drift", tot[-1] - E0, "KE", np.mean(ke))
    assert abs(tot[-1] - E0) < 0.01 * np.mean(ke)


def test_md_is_deterministic_and_graph_capturable():
    s, top = water(nw=216, seed=43)
    v0 = torch.from_numpy(S.initial_velocities(top, 300.0)).cuda()
    outs = []
    for _ in range(2):
        ctx, pos, q, t = setup(s, top, gamma=2.0, dt=0.002)
        vel = v0.clone()
        ctx.md_step(pos, vel, q, t, 20)
        torch.cuda.synchronize()
        outs.append((pos.clone(), vel.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    # graph: 10 steps captured once, replayed twice = 20 steps from the
    # same state (the device step counter numbers the noise)
    ctx, pos, q, t = setup(s, top, gamma=2.0, dt=0.002)
    vel = v0.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.md_step(pos, vel, q, t, 0)  # forces at the start (not captured)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            ctx.md_step(pos, vel, q, t, 10)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    # capture executed nothing: state, forces and step counter are those of
    # the start
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ctx.status()
    assert torch.equal(pos, outs[0][0]) and torch.equal(vel, outs[0][1])


def test_shake_iteration_cap_reports_timeout_and_context_stays_usable():
    # The M-SHAKE Newton loop is the library's one bounded device-side
    # iteration.  A water stretched by 0.2 A cannot meet the 1e-6 relative
    # tolerance in one iteration: the step records NB_ERR_TIMEOUT in the
    # status word (no trap, no fault) and the context keeps working.
    s, top = water(nw=216, seed=44)
    x = s.pos.copy()
    w0 = top.waters[0]
    x[w0[1]] += np.float32(0.2) * (x[w0[1]] - x[w0[0]]) / np.linalg.norm(x[w0[1]] - x[w0[0]])
    s1 = dataclasses.replace(s, pos=oracle.wrap_f32(x, s.box))
    vel0 = torch.from_numpy(S.initial_velocities(top, 300.0)).cuda()
    for max_iter, want in ((1, 8), (10, 0)):
        ctx = nb.Nonbonded(s1)
        ctx.md_init(top, dt=0.001, gamma=0.0, temperature=300.0, seed=1, shake_max_iter=max_iter)
        pos, q, t = nb.concat_inputs([s1])
        vel = vel0.clone()
        ctx.md_step(pos, vel, q, t, 1)
        assert ctx.status(raise_on_error=False) == want  # 8 = NB_ERR_TIMEOUT
        ctx.md_step(pos, vel, q, t, 1)  # the next step runs (converged from the now nearer start)
        torch.cuda.synchronize()
        assert torch.isfinite(pos).all() and torch.isfinite(vel).all()
        ctx.status(raise_on_error=False)


def test_device_philox_matches_the_known_answer_vectors():
    # the device generator of the Langevin noise against the published
    # Philox4x32-10 outputs (the same vectors pin the oracle's generator)
    import test_oracle_md as tom
    rows = tom.philox_kat()
    ctr = torch.tensor(np.array([r[0] for r in rows], np.uint32).view(np.int32), device="cuda")
    key = torch.tensor(np.array([r[1] for r in rows], np.uint32).view(np.int32), device="cuda")
    out = nb.debug_philox(ctr, key).cpu().numpy().view(np.uint32)
    want = np.array([r[2] for r in rows], np.uint32)
    assert np.array_equal(out, want)
    # and agrees with the oracle word for word on 4096 counters of the MD
    # noise layout (atom, step, stream, 0) with a 64-bit seed
    n = 4096
    a = np.arange(n, dtype=np.uint32)
    c = np.stack([a, np.full(n, 77, np.uint32), np.full(n, 1, np.uint32), np.zeros(n, np.uint32)], 1)
    seed = 0x123456789ABCDEF0
    k = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32), (n, 1))
    got = nb.debug_philox(torch.tensor(c.view(np.int32), device="cuda"),
                          torch.tensor(k.view(np.int32), device="cuda")).cpu().numpy().view(np.uint32)
    o = omd.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], seed & 0xFFFFFFFF, seed >> 32)
    assert np.array_equal(got, np.stack([np.asarray(v, np.uint32) for v in o], 1))


def test_minimize_matches_oracle_and_lowers_the_energy():
    # the MD-ready solvated chain with PME 64^3: one capped steepest-descent
    # move against the oracle's, then 40 more moves lower the energy
    s = S.dhfr_chain_md()
    top = S.md_topology(s, n_chain=2500)
    pme = ((64, 64, 64), 4)
    ctx, pos, q, t = setup(s, top, pme=pme)
    E0 = torch.empty(6, dtype=torch.float64, device="cuda")
    E1 = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_minimize(pos, q, t, 0, 0.01, E0)   # energies at the start
    ctx.md_minimize(pos, q, t, 1, 0.01, E1)
    torch.cuda.synchronize()
    ctx.status()
    prm = omd.MDParams(pme=pme)
    x = s.pos.astype(np.float64)
    F, Eo0 = omd.forces_at(s, top, x, prm)
    x1 = omd.minimize_step(s, top, x, F, 0.01)
    _, Eo1 = omd.forces_at(s, top, x1, prm)
    L = s.box.astype(np.float64)
    dx = np.abs(min_image(pos.double().cpu().numpy() - x1, L)).max()
    e0, e1 = E0.cpu().numpy(), E1.cpu().numpy()
    print("minimize max dx", dx, "E0", e0, Eo0, "E1", e1, Eo1)
    assert dx <= 2e-5
    for k in range(5):
        assert abs(e0[k] - Eo0[k]) <= 1e-5 * max(abs(Eo0[k]), 1.0), k
        assert abs(e1[k] - Eo1[k]) <= 1e-4 * max(abs(Eo1[k]), 1.0), k
    assert e1[:5].sum() < e0[:5].sum()
    E2 = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_minimize(pos, q, t, 40, 0.01, E2)
    torch.cuda.synchronize()
    ctx.status()
    assert E2[:5].sum().item() < e1[:5].sum()
    assert E2[5].item() == 0.0


def test_step_with_tabulated_radial_functions_matches_oracle():
    # the MD step on the 4096-interval tables (the paper's production
    # setting) against the oracle's step on its own tables
    s, top = water()
    ctx, pos, q, t = setup(s, top, gamma=5.0)
    ctx.set_tables(4096)
    v0 = S.initial_velocities(top, 300.0)
    vel = torch.from_numpy(v0).cuda()
    E = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.md_step(pos, vel, q, t, 2, E)
    torch.cuda.synchronize()
    ctx.status()
    prm = omd.MDParams(dt=0.001, gamma=5.0, temperature=300.0, seed=2009)
    x, v = s.pos.astype(np.float64), v0.astype(np.float64)
    with oracle.tabulated(4096):
        F, _ = omd.forces_at(s, top, x, prm)
        for k in range(2):
            x, v, F, Eo = omd.step(s, top, x, v, F, k, prm)
    L = s.box.astype(np.float64)
    dx = np.abs(min_image(pos.double().cpu().numpy() - x, L)).max()
    rv = np.linalg.norm(vel.double().cpu().numpy() - v) / np.linalg.norm(v)
    Eg = E.cpu().numpy()
    print("tables: max dx", dx, "v rel", rv, "E", Eg[:2], Eo[:2])
    assert dx <= 4e-5
    assert rv <= 2e-5
    assert abs(Eg[0] - Eo[0]) <= 1e-5 * abs(Eo[0])
