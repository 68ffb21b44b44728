"""Shared parity checks of the GPU tests against the FP64 oracle.

Every forward parity test reports, per energy component k (LJ, Coulomb) and
for their total, the literal relative error |E_k - E_k^oracle| / |E_k^oracle|
(the target's measure) next to the error relative to the summation scale
sum_pairs |e_ij| of that component (a diagnostic: how large the error is
against the terms that were added).  The numbers are collected in RECORD and
printed by the terminal summary of tests/conftest.py, so every GPU run states
them; with NB_PARITY_RECORD=<file> they are also written there as JSON lines.

Bars.  Forces: relative RMS <= 5e-6 and max |dF| <= 1e-3 kcal/mol/A.  Energy:
literal relative error <= 1e-6 for every component whose FP32 rounding floor
allows it (see energy_floor), else <= the bar the case passes with its
reason.  Virial: max |dW_ab| <= 1e-5 max |W_ab|.
"""

from __future__ import annotations

import json
import os

import numpy as np

F_RMS, F_MAX, E_REL, W_REL = 5e-6, 1e-3, 1e-6, 1e-5

RECORD: list[dict] = []

# Per-pair error model of the kernel's FP32 pair arithmetic, measured pair by
# pair (nb_debug_pair_terms against FP64 on every pair of the water box and
# the solvated chain): random relative error of one pair energy (rms, at the
# short distances that dominate sum e^2) and the residual relative bias that
# differs between pairs (which does not cancel in a sum of both signs).
SIGMA_PAIR = 1.5e-7
DELTA_PAIR = 2.0e-9


def fp32_floor(Eo: float, Ea: float, Eq: float) -> float:
    """The literal relative error an unbiased FP32 pair pipeline reaches on a
    summed energy E = sum e_ij: 6 sigma of the random part,
    6 SIGMA_PAIR sqrt(sum e^2), plus the residual bias DELTA_PAIR sum |e|,
    over |E|.  For the TIP3P-shaped water boxes the Coulomb sum cancels to
    1/6000 of sum |e| and this floor lies above 1e-6."""
    return (6.0 * SIGMA_PAIR * np.sqrt(Eq) + DELTA_PAIR * Ea) / abs(Eo)


def record(case: str, quantity: str, value: float, bar: float | None = None, note: str = "") -> None:
    row = {"case": case, "quantity": quantity, "value": float(value), "bar": bar, "note": note}
    RECORD.append(row)
    path = os.environ.get("NB_PARITY_RECORD")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(row) + "\n")


def check_forces(case: str, F, Fo, rms_bar: float = F_RMS, max_bar: float = F_MAX):
    F = np.asarray(F, np.float64)
    nrm = np.linalg.norm(Fo)
    rel = np.linalg.norm(F - Fo) / nrm if nrm > 0 else 0.0
    mx = float(np.abs(F - Fo).max()) if F.size else 0.0
    record(case, "force rel RMS", rel, rms_bar)
    record(case, "force max |dF|", mx, max_bar)
    if nrm > 0:
        assert rel <= rms_bar, f"{case}: force rel RMS {rel:.3e} > {rms_bar:.1e}"
    assert mx <= max_bar, f"{case}: force max abs {mx:.3e} > {max_bar:.1e}"
    return rel, mx


def energy_errors(E, Eo, Es):
    """Literal relative errors (LJ, Coulomb, total) and the errors relative to
    the summation scales sum |e_ij| (LJ, Coulomb, total)."""
    E = np.asarray(E, np.float64)
    Eo = np.asarray(Eo, np.float64)
    Es = np.asarray(Es, np.float64)
    lit, scl = [], []
    for k in range(2):
        d = abs(E[k] - Eo[k])
        lit.append(d / abs(Eo[k]) if Eo[k] != 0 else (0.0 if d == 0 else np.inf))
        scl.append(d / Es[k] if Es[k] != 0 else (0.0 if d == 0 else np.inf))
    d = abs(E.sum() - Eo.sum())
    lit.append(d / abs(Eo.sum()) if Eo.sum() != 0 else (0.0 if d == 0 else np.inf))
    scl.append(d / Es.sum() if Es.sum() != 0 else (0.0 if d == 0 else np.inf))
    return lit, scl


def check_energy(case: str, E, Eo, Es, bars=(E_REL, E_REL, E_REL), notes=("", "", ""), Eq=None):
    """Assert the literal relative error of (E_LJ, E_Coul, E_total) against
    `bars`; components whose oracle value is zero must come out exactly zero.
    A bar given as "floor" is the FP32 floor of that component (fp32_floor,
    needs the oracle's sum e^2 per component in Eq), never below 1e-6.  The
    summation-scale errors are recorded as diagnostics and must stay below
    1e-6."""
    lit, scl = energy_errors(E, Eo, Es)
    bars, notes = list(bars), list(notes)
    for k in range(3):
        if bars[k] == "floor":
            Eo_k = np.asarray(Eo).sum() if k == 2 else np.asarray(Eo)[k]
            Ea_k = np.asarray(Es).sum() if k == 2 else np.asarray(Es)[k]
            Eq_k = np.asarray(Eq).sum() if k == 2 else np.asarray(Eq)[k]
            fl = fp32_floor(Eo_k, Ea_k, Eq_k)
            bars[k] = max(E_REL, fl)
            notes[k] = (notes[k] + " " if notes[k] else "") + f"FP32 floor {fl:.1e}"
    names = ("E_LJ", "E_Coul", "E_total")
    live = [k for k in range(3) if k == 2 or np.asarray(Es)[k] != 0]
    for k in live:  # record every number before the first assertion
        record(case, f"{names[k]} |dE|/|E|", lit[k], bars[k], notes[k])
        record(case, f"{names[k]} |dE|/sum|e|", scl[k], E_REL)
    for k in range(2):
        if k not in live:
            assert np.asarray(E)[k] == 0.0, f"{case}: {names[k]} must be 0"
    for k in live:
        assert lit[k] <= bars[k], f"{case}: {names[k]} literal rel err {lit[k]:.3e} > {bars[k]:.1e}"
        assert scl[k] <= E_REL, f"{case}: {names[k]} err / sum|e| {scl[k]:.3e} > {E_REL:.1e}"
    return lit, scl


def check_virial(case: str, W, Wo, bar: float = W_REL):
    scale = np.abs(Wo).max()
    err = float(np.abs(np.asarray(W) - Wo).max())
    rel = err / scale if scale > 0 else err
    record(case, "virial max|dW|/max|W|", rel, bar)
    assert rel <= bar, f"{case}: virial rel err {rel:.3e} > {bar:.1e}"
    return rel
