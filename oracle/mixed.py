"""Normal-mixed loading (the porous-medium example of Sec. 3.2, Eq. NMBC1).

Test infrastructure: only tests/, the smoke check and bench.py's CPU legs may use this
package.  Plain, slow FP64 NumPy.

The paper imposes the volume average of grad u* with one component controlled and
adjusts the other components at each iteration so that the volume-averaged stress
vanishes in them (<P_rs> = 0); it does not say how.  Reading (small strain, symmetric
stress): the free components form a subset F of the
six symmetric strain components (Voigt order 11, 22, 33, 23, 13, 12, bit k of `mask`);
after the residual of iteration m, with <sigma> the mean stress over the voxel points,
the strain of u* takes the increment

    d eps_F = - (C0_FF)^-1 <sigma>_F ,   d eps_k = 0 for k not in F,

C0 the isotropic reference stiffness (lambda0, mu0): sigma_ii = lambda0 tr eps + 2 mu0
eps_ii, sigma_ij = 2 mu0 eps_ij.  The increment is added symmetrically to A (u*_q =
A_qi x_i, so eps* = sym A) and leaves its skew part alone.  A step has converged when the
equilibrium error is below tol and the mixed error ||<sigma>_F|| / ||<sigma>|| (tensor
Frobenius norms, both off-diagonal entries counted) is below tol too.  A later load step
with the same mask starts its free components from the values the previous one ended with.
"""

import numpy as np

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def free_components(mask):
    return [k for k in range(6) if (mask >> k) & 1]


def mixed_increment(mean_sig, mask, lam0, mu0):
    """d eps (3x3 symmetric) cancelling the free components of mean_sig to first order in
    the reference stiffness."""
    F = free_components(mask)
    d = np.zeros((3, 3))
    normal = [k for k in F if k < 3]
    if normal:
        # C0 restricted to the free normal components: lam0 + 2 mu0 on the diagonal, lam0 off it
        M = np.full((len(normal), len(normal)), lam0) + 2.0 * mu0 * np.eye(len(normal))
        rhs = np.array([-mean_sig[k, k] for k in normal])
        x = np.linalg.solve(M, rhs)
        for k, v in zip(normal, x):
            d[k, k] = v
    for k in F:
        if k >= 3:
            i, j = VOIGT[k]
            d[i, j] = d[j, i] = -mean_sig[i, j] / (2.0 * mu0)
    return d


def mixed_error(mean_sig, mask):
    """||<sigma>_F|| / ||<sigma>||, both off-diagonal entries counted; 0 for zero stress."""
    tot = float(np.sum(mean_sig * mean_sig))
    if tot == 0.0:
        return 0.0
    s = 0.0
    for k in free_components(mask):
        i, j = VOIGT[k]
        s += mean_sig[i, j] ** 2 * (1.0 if i == j else 2.0)
    return float(np.sqrt(s / tot))


def nmbc1_bc():
    """Eq. NMBC1 on every axis: on the faces normal to axis a, component a Dirichlet
    (u^f_a = 0) and the two tangential components traction-free."""
    bc = []
    for a in range(3):
        row = ["N", "N", "N"]
        row[a] = "D"
        bc.append([list(row), list(row)])
    return bc
