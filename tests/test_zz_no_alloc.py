"""The allocation-free entry point nb_forces_noalloc.

Some callers of this library may not allocate device memory themselves (a
host application whose device memory all comes from its own pool, or a
plug-in that may not call cudaMalloc after start-up).  nb_forces_noalloc
serves them with scratch in a static device array.  These tests call it
through the C ABI and check that two calls in a row reproduce the regular
context entry point (nb_build_cells + nb_forces) within the parity
tolerances used elsewhere, and that oversized systems are rejected.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

pytestmark = pytest.mark.gpu

F_RMS, F_MAX, E_REL = 5e-6, 1e-3, 1e-6


def _reference(s):
    pos, q, t = nb.concat_inputs([s])
    ctx = nb.Nonbonded(s)
    ctx.build(pos)
    F, E, W = ctx.forces(pos, q, t)
    torch.cuda.synchronize()
    ctx.status()
    return (pos, q, t), F.clone(), E.clone(), W.clone()


def _check_against(s):
    (pos, q, t), F_ref, E_ref, W_ref = _reference(s)
    for _ in range(2):  # two calls in a row share and reuse the static scratch
        F = torch.full_like(F_ref, float("nan"))
        E = torch.full((1, 2), float("nan"), dtype=torch.float64, device=F.device)
        W = torch.full((1, 6), float("nan"), dtype=torch.float64, device=F.device)
        nb.forces_noalloc(s, pos, q, t, F, E, W)
        torch.cuda.synchronize()
        Fd, Fr = F.double(), F_ref.double()
        assert torch.isfinite(Fd).all()
        rel = (torch.linalg.norm(Fd - Fr) / torch.linalg.norm(Fr)).item()
        assert rel <= F_RMS and (Fd - Fr).abs().max().item() <= F_MAX
        assert torch.allclose(E, E_ref, rtol=E_REL, atol=E_REL)
        assert torch.allclose(W, W_ref, rtol=1e-5, atol=1e-5 * W_ref.abs().max().item())


def test_noalloc_matches_context_entry_point_water():
    _check_against(S._water_system(S.rng_for(41), 300, "noalloc_water"))


def test_noalloc_matches_context_entry_point_chain():
    # chain with exclusions and scaled 1-4 pairs, plus waters
    _check_against(S.solvated_chain(k=42, n_chain=400, n_waters=800, L=32.0))


def test_noalloc_rejects_oversized_system():
    s = S._water_system(S.rng_for(43), 1400, "too_big")  # 4,200 atoms > 4,096
    pos, q, t = nb.concat_inputs([s])
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device=pos.device)
    with pytest.raises(nb.NbError) as e:
        nb.forces_noalloc(s, pos, q, t, F)
    assert e.value.code == 12  # NB_ERR_TOO_LARGE
