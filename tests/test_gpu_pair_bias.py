"""The forward kernel's FP32 pair arithmetic against the FP64 oracle, pair by
pair (nb_debug_pair_terms against oracle.pair_terms on every unique in-range
pair of the water box and of the solvated chain).

Why pair by pair: a summed energy of many terms of both signs (the Coulomb
energy of neutral molecules cancels to 1/6000 of sum |e_ij| in the water box)
inherits any bias of the pair arithmetic that differs between its terms, so
the relative error of each pair term must be centred on zero at every
distance, not only small.  Bars, per 1 A bin of r:
* mean relative error of E_Coul and of E_LJ (the latter relative to
  A r^-12 + B r^-6, which vanishes neither where E_LJ changes sign nor where
  the switch reaches zero) within 1e-8 (or 5 standard errors of the bin mean
  when the bin is small);
* rms relative error below 5e-7, and of the pair force below 1e-6.
The MUFU approximations of rsqrt, rcp and ex2 carry mean errors of -5e-9,
up to +6e-9 and -5e-8 on this GPU (amplified twelvefold in r^-12 for
rsqrt), and the FP32 type-pair coefficients A, B differ from their FP64
values by up to 6e-8 (constant per type pair); the pair arithmetic refines
or replaces the approximations and adds the coefficients' FP32 remainders
in the energy, which this test guards.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_0902_0827_gb300 import nb
from paper_0902_0827_gb300 import systems as S

import parity  # noqa: E402
from pairs_util import imaged_pairs  # noqa: E402

pytestmark = pytest.mark.gpu

BIAS, RMS, F_RMS_PAIR = 1e-8, 5e-7, 1e-6


def gpu_pair_terms(s, ij, xi, xj):
    ctx = nb.Nonbonded(s)
    i, j = ij[:, 0], ij[:, 1]
    xqi = torch.tensor(np.concatenate([xi, s.q[i][:, None]], 1), device="cuda")
    xqj = torch.tensor(np.concatenate([xj, s.q[j][:, None]], 1), device="cuda")
    out = ctx.debug_pair_terms(xqi, xqj, torch.tensor(s.type[i], device="cuda"),
                               torch.tensor(s.type[j], device="cuda"))
    torch.cuda.synchronize()
    ctx.status()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("which", ["water_box", "solvated_chain"])
def test_pair_terms_are_unbiased_at_every_distance(which):
    s = getattr(S, which)()
    ij, xi, xj = imaged_pairs(s)
    g = gpu_pair_terms(s, ij, xi, xj)
    o = oracle.pair_terms(s, xi, xj, s.q[ij[:, 0]], s.q[ij[:, 1]], s.type[ij[:, 0]], s.type[ij[:, 1]])
    d = xj.astype(np.float64) - xi.astype(np.float64)
    r = np.sqrt((d * d).sum(1))
    fj_ref = -(o[:, 2] / r)[:, None] * d  # force on j: -dU/dr d / r
    fj = g[:, 4:7]
    frel = np.linalg.norm(fj - fj_ref) / np.linalg.norm(fj_ref)
    parity.record(f"pairs {which}", "pair force rel RMS", frel, F_RMS_PAIR)
    assert frel <= F_RMS_PAIR
    for b in range(1, 9):
        m = (r >= b) & (r < b + 1)
        for lab, col, scale in (("E_Coul", 1, np.abs(o[:, 1])), ("E_LJ", 0, o[:, 3])):
            mm = m & (scale > 0)
            if mm.sum() < 100:
                continue
            rel = (g[mm, col] - o[mm, col]) / scale[mm]
            mean, rms = rel.mean(), np.sqrt((rel ** 2).mean())
            bar = max(BIAS, 5 * rms / np.sqrt(mm.sum()))
            parity.record(f"pairs {which} r {b}-{b + 1} A", f"{lab} mean rel err", mean, bar)
            parity.record(f"pairs {which} r {b}-{b + 1} A", f"{lab} rms rel err", rms, RMS)
            assert abs(mean) <= bar, (which, b, lab, mean, bar)
            assert rms <= RMS, (which, b, lab, rms)
