"""FP64 oracle of the reciprocal-space electrostatics (TEST INFRASTRUCTURE).

Section "Molecular dynamics on the GPU" evaluates the long-range part of the
electrostatics by smooth particle-mesh Ewald with the FFT library; section
"Validation" uses a 64^3 grid.  Three pieces, each following its definition:

* ``ewald_recip``: the Ewald reciprocal sum over reciprocal lattice vectors
  (plain definition, C), with forces and virial;
* ``ewald_corrections``: the self term and the excluded / scaled 1-4 pair
  terms a reciprocal sum over all pairs needs (C);
* ``spme``: smooth PME taken in the order of its algorithm (Essmann et al.):
  cardinal B-spline charge spreading on a K1 x K2 x K3 grid, FFT (NumPy's, a
  library primitive), multiplication by B(m) C(m), gradient through the
  B-spline derivatives, virial from the per-vector energies.

Only the tests, the smoke check and the CPU legs of the benchmark use this.
"""

from __future__ import annotations

import numpy as np

from . import _c, _p, lib


def _f32(x) -> float:
    """A parameter as the FP32 value the library's parameter block carries."""
    return float(np.float32(x))


def ewald_recip(sys, kmax, pos=None, q=None):
    """Direct reciprocal-space Ewald sum: (F [N,3], E, W [6]) in FP64."""
    pos = _c(sys.pos if pos is None else pos, np.float32)
    q = _c(sys.q if q is None else q, np.float32)
    box = _c(sys.box, np.float32)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(1)
    W = np.zeros(6)
    kx, ky, kz = (kmax, kmax, kmax) if np.isscalar(kmax) else kmax
    rc = lib().orc_ewald_recip(n, _p(pos), _p(q), _p(box), _f32(sys.ewald_alpha), _f32(sys.coulomb_k),
                               int(kx), int(ky), int(kz), _p(F), _p(E), _p(W))
    if rc != 0:
        raise MemoryError("orc_ewald_recip")
    return F, float(E[0]), W


def ewald_corrections(sys, pos=None, q=None):
    """(F [N,3], E_self, E_pairs, W [6]) of the Ewald-consistent corrections."""
    pos = _c(sys.pos if pos is None else pos, np.float32)
    q = _c(sys.q if q is None else q, np.float32)
    box = _c(sys.box, np.float32)
    ex = _c(sys.excl, np.int32).reshape(-1, 2)
    p14 = _c(sys.pairs14, np.int32).reshape(-1, 2)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(2)
    W = np.zeros(6)
    lib().orc_ewald_corrections(n, _p(pos), _p(q), _p(box), _f32(sys.ewald_alpha), _f32(sys.coulomb_k),
                                ex.shape[0], _p(ex), p14.shape[0], _p(p14), _f32(sys.scale14_coul),
                                _p(F), _p(E), _p(W))
    return F, float(E[0]), float(E[1]), W


def bspline(x, n: int):
    """Cardinal B-spline M_n(x) (support [0, n]) by the two-term recursion."""
    x = np.asarray(x, dtype=np.float64)
    if n == 2:
        return np.where((x >= 0.0) & (x <= 2.0), 1.0 - np.abs(x - 1.0), 0.0)
    return (x * bspline(x, n - 1) + (n - x) * bspline(x - 1.0, n - 1)) / (n - 1)


def dbspline(x, n: int):
    """dM_n/dx = M_{n-1}(x) - M_{n-1}(x - 1)."""
    return bspline(x, n - 1) - bspline(x - 1.0, n - 1)


def spme_moduli(K: int, n: int) -> np.ndarray:
    """|b(m)|^2 for m = 0..K-1: 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2."""
    m = np.arange(K)
    k = np.arange(n - 1)
    s = (bspline(k + 1.0, n)[None, :] * np.exp(2j * np.pi * np.outer(m, k) / K)).sum(1)
    return 1.0 / np.abs(s) ** 2


def spme(sys, grid, order: int = 4, pos=None, q=None):
    """Smooth PME reciprocal energy, forces and virial in FP64 (no
    corrections): (F [N,3], E, W [6]).  Even orders only: for odd n the
    B-spline modulus sum vanishes at the Nyquist index of an even grid."""
    if order % 2 or order < 4:
        raise ValueError("smooth PME is defined here for even orders >= 4")
    x = np.asarray(sys.pos if pos is None else pos, dtype=np.float64)
    qv = np.asarray(sys.q if q is None else q, dtype=np.float64)
    L = np.asarray(sys.box, dtype=np.float64)
    K = np.asarray(grid, dtype=np.int64)
    n = order
    alpha, ke = _f32(sys.ewald_alpha), _f32(sys.coulomb_k)
    V = float(np.prod(L))
    x = x - L * np.floor(x / L)
    u = x * K / L
    fl = np.floor(u)
    f = u - fl
    j = np.arange(n)
    # per atom and axis: grid indices (floor(u) - j) mod K, weights M_n(f + j)
    idx = [((fl[:, a:a + 1].astype(np.int64) - j[None, :]) % K[a]) for a in range(3)]
    w = [bspline(f[:, a:a + 1] + j[None, :], n) for a in range(3)]
    dw = [dbspline(f[:, a:a + 1] + j[None, :], n) * (K[a] / L[a]) for a in range(3)]
    Q = np.zeros(tuple(K))
    ww = (qv[:, None, None, None] * w[0][:, :, None, None] * w[1][:, None, :, None] * w[2][:, None, None, :])
    ii = np.broadcast_to(idx[0][:, :, None, None], ww.shape)
    jj = np.broadcast_to(idx[1][:, None, :, None], ww.shape)
    kk = np.broadcast_to(idx[2][:, None, None, :], ww.shape)
    np.add.at(Q, (ii.ravel(), jj.ravel(), kk.ravel()), ww.ravel())
    FQ = np.fft.fftn(Q)
    mi = [np.fft.fftfreq(int(K[a])) * K[a] for a in range(3)]
    mx, my, mz = np.meshgrid(mi[0] / L[0], mi[1] / L[1], mi[2] / L[2], indexing="ij")
    msq = mx * mx + my * my + mz * mz
    msq[0, 0, 0] = 1.0
    C = np.exp(-np.pi ** 2 * msq / alpha ** 2) / (np.pi * V * msq)
    C[0, 0, 0] = 0.0
    bm = [spme_moduli(int(K[a]), n) for a in range(3)]
    B = bm[0][:, None, None] * bm[1][None, :, None] * bm[2][None, None, :]
    Em = 0.5 * ke * B * C * np.abs(FQ) ** 2
    E = float(Em.sum())
    conv = ke * np.real(np.fft.ifftn(B * C * FQ)) * Q.size
    cv = conv[ii, jj, kk]  # [N, n, n, n]
    Fx = -qv * (dw[0][:, :, None, None] * w[1][:, None, :, None] * w[2][:, None, None, :] * cv).sum((1, 2, 3))
    Fy = -qv * (w[0][:, :, None, None] * dw[1][:, None, :, None] * w[2][:, None, None, :] * cv).sum((1, 2, 3))
    Fz = -qv * (w[0][:, :, None, None] * w[1][:, None, :, None] * dw[2][:, None, None, :] * cv).sum((1, 2, 3))
    c = 2.0 * (1.0 + np.pi ** 2 * msq / alpha ** 2) / msq
    W = np.array([(Em * (1.0 - c * mx * mx)).sum(), (Em * (1.0 - c * my * my)).sum(),
                  (Em * (1.0 - c * mz * mz)).sum(), (Em * (-c * mx * my)).sum(),
                  (Em * (-c * mx * mz)).sum(), (Em * (-c * my * mz)).sum()])
    return np.stack([Fx, Fy, Fz], 1), E, W
