"""Host-side helper shared by tests: the unique pairs of a system with the
exact-shift minimum image applied in FP32 (the membership convention of the
library and the oracle: s = x_j - x_i; s > L/2 -> x_j - L; s < -L/2 ->
x_i - L), so that d = x_j' - x_i' as given reproduces the kernel's
displacement.  No pair arithmetic here."""

import numpy as np

import oracle


def imaged_pairs(s):
    ij = oracle.pairs(s).astype(np.int64)
    i, j = ij[:, 0], ij[:, 1]
    xi = s.pos[i].astype(np.float32).copy()
    xj = s.pos[j].astype(np.float32).copy()
    L = s.box.astype(np.float32)
    h = (L * np.float32(0.5)).astype(np.float32)
    d = (xj - xi).astype(np.float32)
    for a in range(3):
        up = d[:, a] > h[a]
        dn = d[:, a] < -h[a]
        xj[up, a] = (xj[up, a] - L[a]).astype(np.float32)
        xi[dn, a] = (xi[dn, a] - L[a]).astype(np.float32)
    return ij, xi, xj
