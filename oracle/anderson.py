"""Anderson acceleration on the polarisation divergence p (Sec. 2.3, Algorithm 1).

The paper accelerates every 2 or 3 iterations from the 4 previous couples of
fields and residuals, applied to p instead of u^f.  It does not print the
formulation; the reading used here (stated in the design notes) is:

* q_m is the field actually sent to the transforms at iteration m, and
  g_m = p_{m+1} the raw polarisation divergence it produces at the next
  iteration; the residual of the couple is f_m = g_m - q_m.
* The last `depth` couples are kept (cleared at each load step).
* At iteration m with m % period == period - 1 and a full history, the new
  field is q = sum_j c_j g_j with c = argmin || sum_j c_j f_j ||_2 subject to
  sum_j c_j = 1 (least squares on the differences f_j - f_last).
* The step is skipped (q = p_m) when the 3x3 normal matrix of those
  differences has a Cholesky pivot below 1e-8 of its diagonal entry: the
  residual differences are then too close to collinear for a well-determined mix.

Parity unpinned beyond self-consistency: there is no closed form for the
accelerated iterates; the fixed point they converge to is pinned elsewhere.
"""

import numpy as np

PIVOT_TOL = 1e-8


def normal_matrix_ok(A, tol=PIVOT_TOL):
    """True when every Cholesky pivot of A exceeds tol times its diagonal entry."""
    m = A.shape[0]
    L = np.zeros_like(A)
    for k in range(m):
        d = A[k, k] - np.dot(L[k, :k], L[k, :k])
        if not (A[k, k] > 0.0) or not (d > tol * A[k, k]):
            return False
        L[k, k] = np.sqrt(d)
        for i in range(k + 1, m):
            L[i, k] = (A[i, k] - np.dot(L[i, :k], L[k, :k])) / L[k, k]
    return True


def coefficients(fs):
    """Mixing coefficients c (sum 1) minimising ||sum_j c_j f_j||_2, or None when skipped."""
    F = np.stack([np.asarray(f, dtype=np.float64).ravel() for f in fs], axis=1)
    fl = F[:, -1]
    Dm = F[:, :-1] - fl[:, None]
    if not normal_matrix_ok(Dm.T @ Dm):
        return None
    gamma = np.linalg.lstsq(Dm, -fl, rcond=None)[0]
    return np.append(gamma, 1.0 - gamma.sum())


def accelerate_now(m, period, history_len, depth):
    return (m % period == period - 1) and history_len == depth
