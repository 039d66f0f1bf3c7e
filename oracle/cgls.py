"""FP64 CGLS on the oracle operators (TEST INFRASTRUCTURE ONLY).

Conjugate gradients on the normal equations A^T A x = A^T y of the
least-squares problem of Eq. 5 (Sec. 3: non-regularised least squares solved
by conjugate gradients), x0 = 0, textbook recurrences (Hestenes-Stiefel
CGLS), every quantity in double precision.
"""
import numpy as np


def cgls(forward, adjoint, y, iters):
    """forward(x) -> A x, adjoint(r) -> A^T r (numpy FP64).  Returns the
    iterates x_1..x_iters and the residual norms ||y - A x_k||."""
    r = np.array(y, dtype=np.float64)
    s = adjoint(r)
    x = np.zeros_like(s)
    p = s.copy()
    gamma = float(np.sum(s * s))
    xs, res = [], []
    for _ in range(iters):
        q = forward(p)
        alpha = gamma / float(np.sum(q * q))
        x = x + alpha * p
        r = r - alpha * q
        s = adjoint(r)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        xs.append(x.copy())
        res.append(float(np.linalg.norm(r)))
    return xs, res
