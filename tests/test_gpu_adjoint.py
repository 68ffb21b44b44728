"""GPU parity of the adjoint (nb_backward, nb_type_gradients, NonbondedFn)
against the FP64 oracle.  Bar: relative RMS <= 1e-4 per result (dL/dx,
dL/dq); the type-pair and per-type parameter gradients are sums over many
pairs of both signs, so, like the energies, their error is measured against
their summation scale (the sum of |pair contribution|, reported by the
oracle): |delta| <= 1e-4 x scale; reruns bit-identical."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

ADJ_RMS = 1e-4


def rel_rms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ok = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), ok), "non-finite pattern differs"
    return np.linalg.norm(a[ok] - b[ok]) / max(np.linalg.norm(b[ok]), 1e-300)


def gpu_backward(s, G, gE, group=1):
    ctx = nb.Nonbonded(s)
    if group != 1:
        ctx.set_tuning(group_clusters=group, list_split=2)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    Gd = torch.from_numpy(np.ascontiguousarray(G, np.float32)).cuda()
    gEd = torch.tensor([[gE, gE]], dtype=torch.float64, device="cuda")
    gpos, gq, gs_tab, ge_tab = ctx.backward(pos, q, t, Gd, gEd)
    gs, ge = ctx.type_gradients(gs_tab, ge_tab)
    torch.cuda.synchronize()
    ctx.status()
    return [x.cpu().numpy() for x in (gpos, gq, gs_tab, ge_tab, gs, ge)]


def param_scales(s, aA, aB):
    """Summation scales of dL/dsig_ab, dL/deps_ab and of the per-type values."""
    sig_tab, eps_tab, _, _ = oracle.combine_lb(s.sigma, s.epsilon)
    s6 = sig_tab ** 6
    c1, c2 = 48 * eps_tab * s6 * sig_tab ** 5, 24 * eps_tab * sig_tab ** 5
    c3, c4 = 4 * s6 * s6, 4 * s6
    sc_sig = aA * c1 + aB * c2
    sc_eps = aA * c3 + aB * c4
    # per type: the Lorentz-Berthelot chain factors are at most 1 (sigma) and
    # eps_b / (2 sqrt(eps_t eps_b)) (epsilon)
    e = s.epsilon.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        fe = np.where(e[None, :] > 0, e[None, :] / (2 * np.sqrt(e[:, None] * e[None, :])), 0.0)
    np.fill_diagonal(fe, 1.0)
    return sc_sig, sc_eps, sc_sig.sum(1), (sc_eps * fe).sum(1)


def check_params(s, gs_tab, ge_tab, gs, ge, dst, det, ds, de, aA, aB):
    sc_sig, sc_eps, sc_s, sc_e = param_scales(s, aA, aB)
    used = np.unique(s.type)
    sub = np.ix_(used, used)
    assert np.all(np.abs(gs_tab[sub] - dst[sub]) <= ADJ_RMS * sc_sig[sub] + 1e-12)
    assert np.all(np.abs(ge_tab[sub] - det[sub]) <= ADJ_RMS * sc_eps[sub] + 1e-12)
    fin = np.isfinite(de)
    assert np.array_equal(np.isfinite(ge), fin)
    assert np.all(np.abs(gs[used] - ds[used]) <= ADJ_RMS * sc_s[used] + 1e-12)
    u = used[fin[used]]
    assert np.all(np.abs(ge[u] - de[u]) <= ADJ_RMS * sc_e[u] + 1e-12)


CASES = {
    "water_tiny": lambda: S._water_system(S.rng_for(11), 216, "w216"),
    "chain_small": lambda: S.solvated_chain(k=42, n_chain=400, n_waters=800, L=32.0),
    "lj_fcc": lambda: S.lj_fcc(),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("gE", [0.0, 0.7])
def test_adjoint_matches_oracle(name, gE):
    s = CASES[name]()
    rng = np.random.default_rng(5)
    G = rng.normal(0.0, 1.0, size=(s.n_atoms, 3)).astype(np.float32)
    gpos, gq, gs_tab, ge_tab, gs, ge = gpu_backward(s, G, gE)
    dx, dq, dA, dB, aA, aB = oracle.backward(s, G.astype(np.float64), gE, with_scale=True)
    dst, det, ds, de = oracle.lb_chain(s, dA, dB)
    assert rel_rms(gpos, dx) <= ADJ_RMS
    if np.any(s.q != 0):
        assert rel_rms(gq, dq) <= ADJ_RMS
    check_params(s, gs_tab, ge_tab, gs, ge, dst, det, ds, de, aA, aB)


@pytest.mark.parametrize("group", [4, 8])
def test_adjoint_of_group_tiles_matches_oracle(group):
    # the adjoint kernel of 4- and 8-cluster i-groups (the autotuner's other
    # tile shapes), on the chain with exclusions and 1-4 pairs
    s = CASES["chain_small"]()
    rng = np.random.default_rng(6)
    G = rng.normal(0.0, 1.0, size=(s.n_atoms, 3)).astype(np.float32)
    gpos, gq, gs_tab, ge_tab, gs, ge = gpu_backward(s, G, 0.7, group=group)
    dx, dq, dA, dB, aA, aB = oracle.backward(s, G.astype(np.float64), 0.7, with_scale=True)
    dst, det, ds, de = oracle.lb_chain(s, dA, dB)
    assert rel_rms(gpos, dx) <= ADJ_RMS
    assert rel_rms(gq, dq) <= ADJ_RMS
    check_params(s, gs_tab, ge_tab, gs, ge, dst, det, ds, de, aA, aB)


def test_fitting_loss_on_solvated_chain():
    # L = sum |F - F_target|^2 with seeded random targets: G = 2 (F - F_target)
    s = S.solvated_chain()
    Ft = S.target_forces(s)
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    ctx.build(pos)
    F, E, _ = ctx.forces(pos, q, t, virial=False)
    G = 2.0 * (F - torch.from_numpy(Ft).cuda())
    gpos, gq, gs_tab, ge_tab = ctx.backward(pos, q, t, G.contiguous(), None)
    gs, ge = ctx.type_gradients(gs_tab, ge_tab)
    torch.cuda.synchronize()
    ctx.status()
    Gh = G.double().cpu().numpy()
    dx, dq, dA, dB, aA, aB = oracle.backward(s, Gh, 0.0, with_scale=True)
    dst, det, ds, de = oracle.lb_chain(s, dA, dB)
    assert rel_rms(gpos.cpu().numpy(), dx) <= ADJ_RMS
    assert rel_rms(gq.cpu().numpy(), dq) <= ADJ_RMS
    check_params(s, gs_tab.cpu().numpy(), ge_tab.cpu().numpy(), gs.cpu().numpy(), ge.cpu().numpy(),
                 dst, det, ds, de, aA, aB)
    # FP64 finite differences of L in a few charges: L is quadratic in each
    # q_k, so the central difference with the FP64 oracle is exact
    Fo = oracle.forces(s, method="cells")[0]

    def L_of(qv):
        Fq = oracle.forces(s, method="cells", q=qv)[0]
        return ((Fq - Ft) ** 2).sum()

    rng = np.random.default_rng(9)
    for k in rng.choice(s.n_atoms, 3, replace=False):
        qp = s.q.copy(); qp[k] = np.float32(qp[k] + 0.125)
        qm = s.q.copy(); qm[k] = np.float32(qm[k] - 0.125)
        fd = (L_of(qp) - L_of(qm)) / (float(qp[k]) - float(qm[k]))
        # the GPU adjoint uses G from the FP32 forward; compare loosely in
        # absolute terms against the scale of dL/dq
        assert abs(gq[k].item() - fd) <= 1e-3 * np.abs(dq).max() + 1e-4 * abs(fd)


def test_autograd_function():
    s = S.solvated_chain(k=42, n_chain=400, n_waters=800, L=32.0)
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    pos = pos.clone().requires_grad_(True)
    q = q.clone().requires_grad_(True)
    sig = torch.tensor(s.sigma, dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(s.epsilon, dtype=torch.float64, requires_grad=True)
    Ft = torch.from_numpy(S.target_forces(s)).cuda()
    F, E = nb.nonbonded(pos, q, sig, eps, ctx, t)
    loss = ((F - Ft) ** 2).sum() + 0.3 * E.sum()
    loss.backward()
    torch.cuda.synchronize()
    ctx.status()
    Fh = F.detach().double().cpu().numpy()
    G = 2.0 * (Fh - Ft.double().cpu().numpy())
    dx, dq, dA, dB, aA, aB = oracle.backward(s, G, 0.3, with_scale=True)
    _, _, ds, de = oracle.lb_chain(s, dA, dB)
    assert rel_rms(pos.grad.cpu().numpy(), dx) <= ADJ_RMS
    assert rel_rms(q.grad.cpu().numpy(), dq) <= ADJ_RMS
    used = np.unique(s.type)
    _, _, sc_s, sc_e = param_scales(s, aA, aB)
    assert np.all(np.abs(sig.grad.numpy()[used] - ds[used]) <= ADJ_RMS * sc_s[used] + 1e-12)
    # types with eps = 0 have an undefined eps gradient (NaN on both sides)
    ge, fin = eps.grad.numpy(), np.isfinite(de)
    assert np.array_equal(np.isfinite(ge), fin)
    u = used[fin[used]]
    assert np.all(np.abs(ge[u] - de[u]) <= ADJ_RMS * sc_e[u] + 1e-12)


def test_adjoint_reruns_bitwise_identical():
    s = S._water_system(S.rng_for(12), 400, "w400")
    ctx = nb.Nonbonded(s)
    pos, q, t = nb.concat_inputs([s])
    G = torch.randn((s.n_atoms, 3), generator=torch.Generator().manual_seed(3)).cuda()
    outs = []
    for _ in range(3):
        ctx.build(pos)
        outs.append([x.clone() for x in ctx.backward(pos, q, t, G, None)])
    torch.cuda.synchronize()
    ctx.status()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert torch.equal(a, b)
