"""Which condition estimate the FP64 leaf fallback of FP32 factors uses,
checked on the oracle's assembly of the 1023^2 recipe (log10 a ~ U[-4, 4] per
pixel, leaf 16).

The cheap lower bound kappa_hat = (max L_ii / min L_ii)^2 of a leaf block's
condition number grows with the coefficient contrast, so at contrast 1e8 a
large share of the leaves would exceed the 1e6 threshold and be eliminated
again in FP64; the Jacobi-scaled condition number kappa(D A_II D)
(D = diag(A_II)^{-1/2}), which bounds the accuracy of a Cholesky
factorization, exceeds it on almost none.  The fallback therefore tests the
scaled condition number (its 1-norm form, computed on the GPU from the FP32
band factor).
"""
import numpy as np

import workloads as W
from oracle import fd


def _leaf_blocks(count):
    p = W.config_problem(1)
    A = fd.assemble(p.ns, p.a, p.b).tocsr()
    n, m = p.ns[0], p.leaf
    idx = np.arange(1, m)
    out = []
    for c in range(count):
        cy, cx = divmod(c, (n + 1) // m)
        X, Y = np.meshgrid(cx * m + idx, cy * m + idx)
        g = ((X - 1) + n * (Y - 1)).ravel()
        out.append(A[g][:, g].toarray())
    return out


def test_cheap_estimate_flags_many_leaves_the_scaled_condition_few():
    blocks = _leaf_blocks(192)
    hat, full, scaled = [], [], []
    for B in blocks:
        d = np.diag(np.linalg.cholesky(B))
        hat.append((d.max() / d.min()) ** 2)
        ev = np.linalg.eigvalsh(B)
        full.append(ev[-1] / ev[0])
        s = 1.0 / np.sqrt(np.diag(B))
        ev = np.linalg.eigvalsh(B * s[:, None] * s[None, :])
        scaled.append(ev[-1] / ev[0])
    hat, full, scaled = np.array(hat), np.array(full), np.array(scaled)
    # the diagonal of a triangular factor holds its eigenvalues: kappa_hat <= kappa(A_II)
    assert np.all(hat <= full * (1 + 1e-8))
    assert np.mean(hat > 1e6) >= 0.25
    assert np.mean(scaled > 1e6) <= 0.02
