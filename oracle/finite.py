"""Finite-strain laws at the voxel points (test infrastructure: only tests/, the smoke
check and the benchmark's CPU baseline use the oracle).

Kinematics (Sec. 3.1.2, Sec. 3.4): F = 1 + grad u with (grad u)_qi = d u_q / d x_i.  With
the library's index convention G[i, q] = D_i u_q the deformation gradient is F = 1 + G^T,
and the tensor the divergence acts on is S[i, q] = P[q, i], P the first Piola-Kirchhoff
stress (div P)_q = d P_qi / d x_i.

* SVK_CUBIC: St-Venant-Kirchhoff, second Piola-Kirchhoff Pi = C : E, E = (F^T F - 1)/2,
  C the cubic stiffness (C11, C12, C44) rotated by the grain orientation; P = F Pi
  (Sec. 3.1.2, written there for isotropic C).
* NEO_HOOKE: psi = mu/2 (J^(-2/3) tr(F^T F) - 3) + K/2 (J - 1)^2, Pi = d psi / d E,
  P = F Pi (Appendix B).
* CP_FCC: multiplicative crystal plasticity F = F^e F^p (Sec. 3.4) with the 12
  {111}<110> systems, Pi = C : E^e, E^e = (F^eT F^e - 1)/2, L^p = sum_s gdot_s m_s (x) n_s,
  and the power-law flow gdot_s = gdot0 |tau_s / tau_c|^n sign(tau_s) with Voce hardening
  tau_c = tau0 + (tau_inf - tau0)(1 - exp(-h0 Gamma / (tau_inf - tau0))), Gamma the
  cumulated slip.  Integration over a load increment dt (implicit in Pi, after
  Kalidindi, Bronkhorst and Anand 1992): F^p_{n+1} = (1 + sum_s dgamma_s P_s) F^p_n,
  Pi = C : (A - 1)/2 - sum_s dgamma_s C : sym(A P_s), A = F^p_n^{-T} F^T F F^p_n^{-1},
  tau_s = Pi : P_s (the Mandel stress with C^e ~ 1 in the resolved shear), tau_c at the
  committed Gamma_n.  params = (C11, C12, C44, gdot0, n, tau0, tau_inf, h0, dt).
  Pinned by the single-slip recursion under simple shear; the full-field solve through
  this law by a two-crystal laminate past yield (traction continuity solved independently,
  tests/test_oracle_laminate_nonlinear.py); the full-field polycrystal response is parity
  unpinned beyond that.
* LOG_J2: perfect von Mises plasticity in the logarithmic framework the paper uses for the
  porous medium (Sec. 3.2, after Miehe, Apel and Lambrecht): Hencky strain H = log(F^T F)/2
  split additively, H = H^e + H^p; the stress conjugate to H is T = 2 mu dev H^e + K tr H^e 1
  (K = lambda + 2 mu / 3); f = sqrt(3/2 dev T : dev T) - sigma0 <= 0 with normality in H^p.
  Reading (the paper calls T the Cauchy stress and gives no integration): backward-Euler
  radial return from the committed (H^p_n, p_n) on the trial H^e = H - H^p_n; the second
  Piola-Kirchhoff stress is T : dH/dE = T : d log C / d C (E = (C - 1)/2), evaluated in the
  eigenbasis of C = sum_a lam_a N_a (x) N_a with the divided differences of the logarithm
  (theta_aa = 1 / lam_a, theta_ab = (log lam_a - log lam_b) / (lam_a - lam_b)); P = F S.
  params = (lambda, mu, sigma0).
"""

import numpy as np

from .laws import quat_to_rotation, rotated_cubic

I3 = np.eye(3)


def deformation_gradient(G):
    """G (npp, 3, 3, m) with G[r, i, q] = D_i u_q  ->  F (npp, m, 3, 3)."""
    return I3 + np.moveaxis(G, 3, 1).swapaxes(2, 3)


def to_S(P):
    """First Piola P (npp, m, 3, 3) [q, i] -> S (npp, 3, 3, m) with S[i, q] = P[q, i]."""
    return np.moveaxis(P.swapaxes(2, 3), 1, 3)


def svk_cubic(G, params, quat):
    C = rotated_cubic(params[:3], quat)
    F = deformation_gradient(G)
    E = 0.5 * (np.einsum("rmki,rmkj->rmij", F, F) - I3)
    Pi = np.einsum("ijkl,rmkl->rmij", C, E)
    return to_S(F @ Pi)


def neo_hooke(G, params):
    mu, K = params[:2]
    F = deformation_gradient(G)
    Cr = np.einsum("rmki,rmkj->rmij", F, F)
    J = np.linalg.det(F)
    Ci = np.linalg.inv(Cr)
    I1 = np.trace(Cr, axis1=2, axis2=3)
    Jm23 = J ** (-2.0 / 3.0)
    Pi = (mu * Jm23)[..., None, None] * (I3 - (I1 / 3.0)[..., None, None] * Ci) \
        + (K * (J - 1.0) * J)[..., None, None] * Ci
    return to_S(F @ Pi)


def fcc_slip_systems():
    """The 12 {111}<110> systems (unit slip directions m, unit plane normals n), crystal frame."""
    normals = [np.array(v, float) for v in [(1, 1, 1), (-1, 1, 1), (1, -1, 1), (1, 1, -1)]]
    dirs = [np.array(v, float) for v in [(1, -1, 0), (1, 0, -1), (0, 1, -1), (1, 1, 0), (1, 0, 1), (0, 1, 1)]]
    ms, ns = [], []
    for nv in normals:
        for d in dirs:
            if abs(d @ nv) < 1e-12:
                ms.append(d / np.linalg.norm(d))
                ns.append(nv / np.linalg.norm(nv))
    assert len(ms) == 12
    return np.array(ms), np.array(ns)


def voce(gam, tau0, tau_inf, h0):
    return tau0 + (tau_inf - tau0) * (1.0 - np.exp(-h0 * gam / (tau_inf - tau0)))


def cp_update(F, Fp_n, gam_n, C, Ps, gdot0, nexp, tau0, tau_inf, h0, dt, tol=1e-12, max_newton=200):
    """One implicit increment at every point.  F, Fp_n: (m, 3, 3); gam_n: (m,); C: 3x3x3x3;
    Ps: (S, 3, 3) Schmid tensors m_s (x) n_s in the sample frame.
    Returns (P first Piola (m, 3, 3), Fp_{n+1}, gam_{n+1}, newton iterations used)."""
    mpts = F.shape[0]
    Fpi = np.linalg.inv(Fp_n)
    Fe_tr = F @ Fpi
    A = np.einsum("mki,mkj->mij", Fe_tr, Fe_tr)
    Pi_tr = np.einsum("ijkl,mkl->mij", C, 0.5 * (A - I3))
    B = np.einsum("mik,skj->msij", A, Ps)
    Cs = np.einsum("ijkl,mskl->msij", C, 0.5 * (B + B.swapaxes(2, 3)))
    tauc = voce(gam_n, tau0, tau_inf, h0)

    def slip(Pi):
        tau = np.einsum("mij,sij->ms", Pi, Ps)
        x = tau / tauc[:, None]
        ax = np.abs(x)
        dg = dt * gdot0 * ax ** nexp * np.sign(x)
        ddg = dt * gdot0 * nexp * ax ** (nexp - 1.0) / tauc[:, None]
        return dg, ddg

    def resid(Pi):
        dg, ddg = slip(Pi)
        return Pi - Pi_tr + np.einsum("ms,msij->mij", dg, Cs), dg, ddg

    # start on the yield surface of the most stressed system (or at the trial stress if below)
    tau_tr = np.abs(np.einsum("mij,sij->ms", Pi_tr, Ps)).max(axis=1)
    s0 = np.minimum(1.0, tauc / np.maximum(tau_tr, 1e-300))
    Pi = Pi_tr * s0[:, None, None]
    R, dg, ddg = resid(Pi)
    scale = np.maximum(np.abs(Pi_tr).reshape(mpts, 9).max(axis=1), tauc)
    it_used = 0
    for it in range(max_newton):
        rn = np.abs(R).reshape(mpts, 9).max(axis=1)
        active = rn > tol * scale
        if not active.any():
            break
        it_used = it + 1
        Jm = np.tile(np.eye(9), (mpts, 1, 1)) + np.einsum("msa,ms,sb->mab", Cs.reshape(mpts, -1, 9), ddg,
                                                           Ps.reshape(-1, 9))
        d = np.linalg.solve(Jm[active], -R[active].reshape(-1, 9, 1)).reshape(-1, 3, 3)
        d = 0.5 * (d + d.swapaxes(1, 2))
        # backtracking on the max-norm of the residual
        step = np.ones(d.shape[0])
        Pa, Ra = Pi[active], R[active]
        r0 = np.abs(Ra).reshape(-1, 9).max(axis=1)
        newP = Pa + d
        for _ in range(60):
            Rt, _, _ = resid_sub(newP, Pi_tr[active], Cs[active], Ps, tauc[active], gdot0, nexp, dt)
            rt = np.abs(Rt).reshape(-1, 9).max(axis=1)
            bad = ~(rt < r0) & (step > 1e-12)
            if not bad.any():
                break
            step = np.where(bad, 0.5 * step, step)
            newP = Pa + step[:, None, None] * d
        Pi[active] = newP
        R, dg, ddg = resid(Pi)
    L = np.einsum("ms,sij->mij", dg, Ps)
    Fp = (I3 + L) @ Fp_n
    gam = gam_n + np.abs(dg).sum(axis=1)
    Fpi_new = np.linalg.inv(Fp)
    Fe = F @ Fpi_new
    P = Fe @ Pi @ Fpi_new.swapaxes(1, 2)
    return P, Fp, gam, it_used


def resid_sub(Pi, Pi_tr, Cs, Ps, tauc, gdot0, nexp, dt):
    tau = np.einsum("mij,sij->ms", Pi, Ps)
    x = tau / tauc[:, None]
    dg = dt * gdot0 * np.abs(x) ** nexp * np.sign(x)
    return Pi - Pi_tr + np.einsum("ms,msij->mij", dg, Cs), dg, None


def cp_fcc(G, params, quat, Fp_n, gam_n):
    """CP_FCC at the points of one phase.  G (npp, 3, 3, m); Fp_n (npp, 3, 3, m); gam_n (npp, m).
    Returns (S (npp, 3, 3, m), Fp_{n+1}, gam_{n+1})."""
    C11, C12, C44, gdot0, nexp, tau0, tau_inf, h0, dt = params[:9]
    R = quat_to_rotation(quat)
    C = rotated_cubic((C11, C12, C44), quat)
    mc, nc = fcc_slip_systems()
    Ps = np.einsum("si,sj->sij", mc @ R.T, nc @ R.T)
    npp, m = G.shape[0], G.shape[3]
    F = deformation_gradient(G).reshape(npp * m, 3, 3)
    Fpn = np.moveaxis(Fp_n, 3, 1).reshape(npp * m, 3, 3)
    P, Fp, gam, _ = cp_update(F, Fpn, gam_n.reshape(npp * m), C, Ps, gdot0, nexp, tau0, tau_inf, h0, dt)
    S = to_S(P.reshape(npp, m, 3, 3))
    return S, np.moveaxis(Fp.reshape(npp, m, 3, 3), 1, 3), gam.reshape(npp, m)


def _log_divided_differences(w):
    """theta[..., a, b] = (log w_a - log w_b) / (w_a - w_b), 1 / w_a on the diagonal and in
    the limit of equal eigenvalues (log1p keeps nearby pairs accurate)."""
    wa = w[..., :, None]
    wb = w[..., None, :]
    r = (wa - wb) / wb
    with np.errstate(divide="ignore", invalid="ignore"):
        th = np.log1p(r) / (wb * r)
    near = np.abs(r) < 1e-10
    return np.where(near, 1.0 / (0.5 * (wa + wb)), th)


def log_j2(G, params, Hp_n, p_n):
    """G (npp, 3, 3, m); Hp_n (npp, 3, 3, m) committed plastic Hencky strain, p_n (npp, m)
    cumulated plastic strain.  Returns (S[i, q] = P[q, i], Hp, p)."""
    lam, mu, sigma0 = params[:3]
    K = lam + 2.0 * mu / 3.0
    F = deformation_gradient(G)  # (npp, m, 3, 3)
    C = np.einsum("rmki,rmkj->rmij", F, F)
    w, V = np.linalg.eigh(C)  # C = V diag(w) V^T
    H = np.einsum("rmia,rma,rmja->rmij", V, 0.5 * np.log(w), V)
    Hp = np.moveaxis(Hp_n, 3, 1)  # (npp, m, 3, 3)
    He = H - Hp
    tr = np.trace(He, axis1=2, axis2=3)
    dev = He - (tr / 3.0)[..., None, None] * I3
    s_tr = 2.0 * mu * dev
    seq = np.sqrt(1.5 * np.einsum("rmij,rmij->rm", s_tr, s_tr))
    f = seq - sigma0
    yld = f > 0.0
    dp = np.where(yld, f / (3.0 * mu), 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(yld, sigma0 / seq, 1.0)
        nflow = np.where(yld[..., None, None], 1.5 * s_tr / seq[..., None, None], 0.0)
    s = scale[..., None, None] * s_tr
    T = s + (K * tr)[..., None, None] * I3
    Hp_new = Hp + dp[..., None, None] * nflow
    # S = T : d log C / d C in the eigenbasis of C
    Tt = np.einsum("rmia,rmij,rmjb->rmab", V, T, V)
    St = _log_divided_differences(w) * Tt
    S = np.einsum("rmia,rmab,rmjb->rmij", V, St, V)
    return to_S(F @ S), np.moveaxis(Hp_new, 1, 3), p_n + dp
