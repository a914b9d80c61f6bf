"""Algorithm 1 (Sec. 2.4): one load step of the accelerated displacement fixed point.

Per iteration m, in the order of Algorithm 1:

  a1  G = grad_d u^f + grad_d u*                      (voxel points)
  a2  P = F(G, committed state)                        (the behaviour law)
  a3  D = div_d P  (+ D*, zero for traction-free faces)
  a4  err = h1 sqrt(S_D / S_P) vs eps  (Eq. equilibrium_condition; S_D = sum of D^2
      over the transformed node components, S_P = sum over voxel points of
      ||P||_F^2 / n_ppv: squared L2 norms, which makes err dimensionless)
      p  = div_d (R0 : grad_d u^f) - D                (Eq. div_pol)
  a5  Anderson on p                                    (anderson.py)
  a6  forward DT of each component of p                (Table 1, x then y then z)
  a7  B0 / 2mu0 Green operator                         (Eqs. NSGO1_*, NSGO2_*)
  a8  inverse DT -> u^f                                (dismissed nodes = 0)

On convergence the committed state is updated from the converged strain (a9).
"""

from dataclasses import dataclass, field

import numpy as np

from . import anderson as anderson_mod
from . import mixed as mixed_mod
from .bc import Grid
from .green import c0_green_apply, c0_unsupported, green_factor
from .laws import b0_apply, c0_apply, phase_groups, stress
from .stencils import div, full_nodes, grad, grad_full, n_points
from .transforms import dt3d_forward, dt3d_inverse


@dataclass
class Report:
    iterations: int
    converged: bool
    err: list = field(default_factory=list)
    accelerated: list = field(default_factory=list)
    mean_P: np.ndarray = None
    mean_G: np.ndarray = None
    mixed_err: list = field(default_factory=list)
    A: np.ndarray = None


class Problem:
    """Plain-data problem built from a synthetic.Workload."""

    def __init__(self, wl, fast=None):
        self.wl = wl
        self.grid = Grid(wl.n, wl.bc, wl.h)
        self.scheme = wl.scheme
        self.npp = n_points(wl.scheme)
        self.lambda0 = 0.0 if wl.green == "MU0" else float(wl.lambda0)
        self.mu0 = float(wl.mu0)
        self.groups = phase_groups(wl.phase, len(wl.materials))
        self.fast = fast
        self.masks = [self.grid.dof_mask(q) for q in range(3)]
        self.c0 = wl.green == "C0"
        if self.c0:
            why = c0_unsupported(self.grid, wl.scheme)
            if why:
                raise ValueError(why)
        self.factors = [green_factor(self.grid, q, wl.scheme, self.lambda0, self.mu0) for q in range(3)]
        self.state = None
        shp = (self.npp,) + self.grid.n
        if any(m.law == 2 for m in wl.materials):  # J2: (eps^p, p)
            self.state = {"ep": np.zeros((self.npp, 3, 3) + self.grid.n), "p": np.zeros(shp)}
        if any(m.law == 7 for m in wl.materials):  # logarithmic J2: (H^p, p)
            self.state = self.state or {}
            self.state["Hp"] = np.zeros((self.npp, 3, 3) + self.grid.n)
            self.state["pl"] = np.zeros(shp)
        if any(m.law == 6 for m in wl.materials):  # crystal plasticity: (F^p, Gamma)
            self.state = self.state or {}
            self.state["Fp"] = np.broadcast_to(np.eye(3)[None, :, :, None, None, None],
                                               (self.npp, 3, 3) + self.grid.n).copy()
            self.state["gam"] = np.zeros(shp)
        self.uf = np.zeros(self.grid.node_shape)
        self.mixed_A = None  # the affine part of u* the last mixed load step ended with
        self.mixed_mask = 0  # that step's mask

    # --- a0: prescribed displacement and its discrete gradient ------------------------
    def ustar_full(self, A=None, b=None, Q=None):
        """u* on the full (n+1)^3 node grid: u*_q = A[q] . x + b[q] + sum_k Q[q][k] m_k(x),
        m = (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2) (affine plus the quadratic terms of
        bending and torsion loads)."""
        A = self.wl.A if A is None else A
        b = self.wl.b if b is None else b
        Q = getattr(self.wl, "Q", np.zeros((3, 6))) if Q is None else Q
        n, h = self.grid.n, self.grid.h
        x = [np.arange(n[a] + 1) * h[a] for a in range(3)]
        X = np.meshgrid(*x, indexing="ij")
        mono = [X[0] * X[0], X[1] * X[1], X[2] * X[2], X[1] * X[2], X[0] * X[2], X[0] * X[1]]
        return np.stack([A[q, 0] * X[0] + A[q, 1] * X[1] + A[q, 2] * X[2] + b[q]
                         + sum(Q[q][k] * mono[k] for k in range(6)) for q in range(3)])

    def grad_ustar(self, A=None, b=None, Q=None, Us=None):
        """Discrete gradient of u* at the voxel points (the scheme's stencil on the node values);
        Us: a node field (3, N1, N2, N3) on the stored node grid added to the closed-form u*
        (Sec. 2.2: u* is any field carrying the Dirichlet values)."""
        u = self.ustar_full(A, b, Q)
        if Us is not None:
            u = u + full_nodes(np.asarray(Us, dtype=np.float64), self.grid)
        return grad_full(u, self.grid, self.scheme)

    # --- pieces of one iteration ------------------------------------------------------
    def residual(self, uf, Gs, T=None, Tf=None):
        """a1-a4 and p: returns (p, D, P, G, S_D, S_P); T: uniform Neumann tractions
        T[axis][face][component] (D = div P + D*, the ghosts of P* = 2 t)."""
        Gf = grad(uf, self.grid, self.scheme)
        G = Gf + Gs
        P, _ = stress(G, self.wl.materials, self.groups, self.state)
        D = div(P, self.grid, self.scheme, T, Tf)
        for q in range(3):
            D[q][~self.masks[q]] = 0.0
        S_D = float(np.sum(D * D))
        S_P = float(np.sum(P * P)) / self.npp
        r0 = c0_apply if self.c0 else b0_apply
        p = div(r0(Gf, self.lambda0, self.mu0), self.grid, self.scheme) - D
        for q in range(3):
            p[q][~self.masks[q]] = 0.0
        return p, D, P, G, S_D, S_P

    def error(self, S_D, S_P):
        if S_P > 0.0:
            return self.grid.h[0] * np.sqrt(S_D / S_P)
        return 0.0 if S_D == 0.0 else np.inf

    def green_update(self, q_field):
        """a6-a8: u^f = iDT(DGO(DT(q)))."""
        g = self.grid
        out = np.zeros(g.node_shape)
        if self.c0:  # the three components couple at each node position (green.c0_green_apply)
            ph = []
            for q in range(3):
                full = np.zeros(g.N)
                full[g.dof_slices(q)] = dt3d_forward(q_field[q], g.kind[q], g.n, fast=self.fast)
                ph.append(full)
            uh = c0_green_apply(g, self.lambda0, self.mu0, ph, self.scheme)
            for q in range(3):
                out[q] = dt3d_inverse(uh[q][g.dof_slices(q)], g.kind[q], g.n, g.N, fast=self.fast)
            return out
        for q in range(3):
            spec = dt3d_forward(q_field[q], g.kind[q], g.n, fast=self.fast)
            spec = spec * self.factors[q]
            out[q] = dt3d_inverse(spec, g.kind[q], g.n, g.N, fast=self.fast)
        return out

    # --- Algorithm 1, one load step -----------------------------------------------------
    def solve_step(self, A=None, b=None, uf0=None, max_iter=None, tol=None, anderson=True, Q=None, mixed=0,
                   T=None, Tf=None, Us=None):
        """One load step.  mixed: bit mask of the symmetric strain components (Voigt order
        11, 22, 33, 23, 13, 12) of u* that are adjusted so that the mean stress vanishes in
        them (normal-mixed loading, mixed.py); the other components of A are imposed.
        T: uniform tractions T[axis][face][component] on the faces where that component is
        Neumann (stencils.add_traction_ghosts), or None for traction-free faces; Tf: per-face
        traction fields {(axis, face): t (3, n_b, n_c)} added to T; Us: u* as a node field on
        the stored node grid, added to the closed-form u*."""
        wl = self.wl
        tol = wl.tol if tol is None else tol
        max_iter = wl.max_iter if max_iter is None else max_iter
        A = np.array(wl.A if A is None else A, dtype=np.float64)
        if mixed and mixed == self.mixed_mask:  # free components start where the last mixed step ended
            for k in mixed_mod.free_components(mixed):
                i, j = mixed_mod.VOIGT[k]
                A[i, j] = self.mixed_A[i, j]
                A[j, i] = self.mixed_A[j, i]
        Gs = self.grad_ustar(A, b, Q, Us)
        uf = self.uf.copy() if uf0 is None else np.array(uf0, dtype=np.float64)
        mixer = anderson_mod.Mixer(wl.anderson_depth, wl.anderson_period, enabled=anderson)
        rep = Report(iterations=0, converged=False)
        for m in range(max_iter + 1):
            p, D, P, G, S_D, S_P = self.residual(uf, Gs, T, Tf)
            err = self.error(S_D, S_P)
            rep.err.append(err)
            rep.iterations = m
            mean_sig = None
            if mixed:
                Pm = P.mean(axis=(0, 3, 4, 5))
                mean_sig = 0.5 * (Pm + Pm.T)
                rep.mixed_err.append(mixed_mod.mixed_error(mean_sig, mixed))
            if err < tol and (not mixed or rep.mixed_err[-1] < tol):
                rep.converged = True
                break
            if m == max_iter:
                break
            if np.isnan(err) or not (np.isfinite(S_D) and np.isfinite(S_P)):
                break  # diverged (err is +inf, and the iteration goes on, while P is still zero)
            q, mixed_step = mixer.propose(m, p)
            if mixed_step:
                rep.accelerated.append(m)
            uf = self.green_update(q)
            if mixed:  # the free strain components of u* for the next iteration
                A = A + mixed_mod.mixed_increment(mean_sig, mixed, float(wl.lambda0), float(wl.mu0))
                Gs = self.grad_ustar(A, b, Q, Us)
        self.uf = uf
        if mixed:
            self.mixed_A = A.copy()
            self.mixed_mask = mixed
            rep.A = A.copy()
        rep.mean_P = P.mean(axis=(0, 3, 4, 5))
        rep.mean_G = G.mean(axis=(0, 3, 4, 5))
        if self.state is not None and rep.converged:
            _, self.state = stress(G, wl.materials, self.groups, self.state)
        self.last = {"P": P, "G": G, "D": D}
        return uf, rep


def node_field_full(problem, uf):
    """Total displacement u = u^f + u* on the full node grid (for reporting)."""
    return full_nodes(uf, problem.grid) + problem.ustar_full()
