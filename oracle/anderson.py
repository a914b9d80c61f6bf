"""Anderson acceleration on the polarisation divergence p (Sec. 2.3, Algorithm 1).

The paper accelerates every 2 or 3 iterations from the 4 previous couples of
fields and residuals, applied to p instead of u^f.  It does not print the
formulation; the reading used here is:

* q_m is the field actually sent to the transforms at iteration m, and
  g_m = p_{m+1} the raw polarisation divergence it produces at the next
  iteration; the residual of the couple is f_m = g_m - q_m.
* The last `depth` couples are kept (cleared at each load step).
* At iteration m with m % period == period - 1 and a full history, the new
  field is q = sum_j c_j g_j with c = argmin || sum_j c_j f_j ||_2 subject to
  sum_j c_j = 1 (least squares on the differences f_j - f_last).
* The step is skipped (q = p_m) when the residual differences are numerically
  dependent: some difference makes an angle with the span of the previous ones
  whose squared sine is below 1e-8 (the Cholesky pivots of their normal matrix
  relative to its diagonal entries; a measure that, like the mixing
  coefficients, does not depend on the scale of each difference).  The mix is
  undetermined for exactly dependent differences, and the paper's FP64 p-form
  iteration gives an exactly collinear history (a laminate's) an angle of its
  own through rounding alone, a squared sine that stays below 1e-8 down to
  tolerances of 1e-10, while genuinely three-dimensional histories sit above
  1e-3 (both measured in the tests); the threshold separates the two.

Pinned: for an affine fixed-point map the mix of dimension + 1 couples is the
fixed point, and the residual of the mix is M times the minimal residual (which
tells a mix of the g_j from a mix of the q_j); the solver on a problem with 3
free node components lands on its solution right after its first mix.  Beyond
these identities the accelerated iterates of a general problem have no closed
form: their parity is self-consistency (the fixed point they reach is pinned
elsewhere).
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


class Mixer:
    """The solver loop's bookkeeping of the couples (Algorithm 1, "Anderson ... on p").

    At iteration m the loop has the field p_m it just computed.  The couple of the previous
    iteration is completed with it (q_{m-1}, g_{m-1} = p_m), the oldest couple is dropped
    beyond `depth`, and the field sent to the transforms is q_m = p_m, or, on an
    acceleration iteration with a full history and a well-determined mix, the combination
    sum_j c_j g_j of the stored couples.
    """

    def __init__(self, depth, period, enabled=True):
        self.depth, self.period, self.enabled = depth, period, enabled
        self.hist = []  # (q_j, g_j)
        self.q_prev = None

    def propose(self, m, p):
        """The field q_m to transform at iteration m, and whether it is an Anderson mix."""
        if self.q_prev is not None:
            self.hist.append((self.q_prev, p))
            if len(self.hist) > self.depth:
                self.hist.pop(0)
        q, mixed = p, False
        if self.enabled and accelerate_now(m, self.period, len(self.hist), self.depth):
            c = coefficients([g_ - q_ for q_, g_ in self.hist])
            if c is not None:
                q = sum(cj * g_ for cj, (_, g_) in zip(c, self.hist))
                mixed = True
        self.q_prev = q
        return q, mixed
