"""Small-strain constitutive laws evaluated at the voxel points.

G[r, i, q] = D_i u_q; the small strain is eps = (G + G^T)/2 and P = sigma
(symmetric) in small strain (Sec. 2.2).

* ISO_ELASTIC: sigma = lambda tr(eps) 1 + 2 mu eps (Sec. 3.1.1; the standard
  2 mu factor is used).
* CUBIC_ELASTIC: sigma = C^g : eps with the cubic stiffness (C11, C12, C44) of
  Sec. 3.3 rotated into the sample frame: C^g_ijkl = R_ia R_jb R_kc R_ld C_abcd,
  R the rotation of the grain's unit quaternion (w, x, y, z).
* J2_LINHARD: von Mises plasticity with linear isotropic hardening, radial
  return from the committed (eps^p, p): the small-strain form of the J2 law
  of Sec. 3.2 with yield stress sigma_y + H p.
* B0_LINEAR: P = 2 mu G + lambda G (.) I -- the B0 preconditioner itself
  (Sec. 2.6.3), a test law for which one fixed-point iteration is exact.
* SVK_CUBIC, NEO_HOOKE, CP_FCC: finite-strain laws, in oracle/finite.py.
"""

import numpy as np

ISO_ELASTIC = 0
CUBIC_ELASTIC = 1
J2_LINHARD = 2
B0_LINEAR = 3
SVK_CUBIC = 4
NEO_HOOKE = 5
CP_FCC = 6
LOG_J2 = 7  # finite strain (finite.log_j2)

I3 = np.eye(3)


def quat_to_rotation(qt):
    """Rotation matrix of a unit quaternion (w, x, y, z) (crystal frame -> sample frame)."""
    w, x, y, z = (float(v) for v in qt)
    nrm = np.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def cubic_tensor(C11, C12, C44):
    """Fourth-order cubic stiffness in the crystal frame."""
    C = np.zeros((3, 3, 3, 3))
    for a in range(3):
        for b in range(3):
            if a == b:
                C[a, a, a, a] = C11
            else:
                C[a, a, b, b] = C12
                C[a, b, a, b] = C44
                C[a, b, b, a] = C44
    return C


def rotated_cubic(params, quat):
    R = quat_to_rotation(quat)
    C = cubic_tensor(*params)
    return np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C)


def iso_tensor(lam, mu):
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = lam * I3[i, j] * I3[k, l] + mu * (I3[i, k] * I3[j, l] + I3[i, l] * I3[j, k])
    return C


def phase_groups(phase, n_phases):
    """Flat voxel indices of each phase."""
    flat = np.asarray(phase).ravel()
    order = np.argsort(flat, kind="stable")
    counts = np.bincount(flat, minlength=n_phases)
    bounds = np.concatenate([[0], np.cumsum(counts)])
    return [order[bounds[p]:bounds[p + 1]] for p in range(n_phases)]


def _sym(Gv):
    return 0.5 * (Gv + np.swapaxes(Gv, 1, 2))


def j2_return(eps, ep_n, p_n, lam, mu, sy, H):
    """Radial return, small strain, linear isotropic hardening.  eps, ep_n: (npp, 3, 3, m)."""
    ee = eps - ep_n
    tr = ee[:, 0, 0] + ee[:, 1, 1] + ee[:, 2, 2]
    sig = 2.0 * mu * ee + lam * tr[:, None, None] * I3[None, :, :, None]
    trs = sig[:, 0, 0] + sig[:, 1, 1] + sig[:, 2, 2]
    s = sig - (trs / 3.0)[:, None, None] * I3[None, :, :, None]
    q = np.sqrt(1.5 * np.einsum("rijm,rijm->rm", s, s))
    f = q - (sy + H * p_n)
    plastic = f > 0.0
    dp = np.where(plastic, f / (3.0 * mu + H), 0.0)
    qs = np.where(plastic, q, 1.0)
    nflow = 1.5 * s / qs[:, None, None]
    sig = sig - 2.0 * mu * dp[:, None, None] * nflow
    ep = ep_n + dp[:, None, None] * nflow
    return sig, ep, p_n + dp


def stress(G, materials, groups, state=None):
    """First Piola stress (= Cauchy in small strain) at every voxel point.

    G: (npp, 3, 3, n1, n2, n3).  state: dict with 'ep' (npp,3,3,n1,n2,n3) and
    'p' (npp,n1,n2,n3) for J2 phases, or None.  Returns (P, new_state or None).
    """
    npp = G.shape[0]
    shp = G.shape
    Gf = G.reshape(npp, 3, 3, -1)
    P = np.zeros_like(Gf)
    from . import finite
    new_state = None
    if state is not None:
        new_state = {}
        if "ep" in state:
            new_state["ep"] = state["ep"].reshape(npp, 3, 3, -1).copy()
            new_state["p"] = state["p"].reshape(npp, -1).copy()
        if "Fp" in state:
            new_state["Fp"] = state["Fp"].reshape(npp, 3, 3, -1).copy()
            new_state["gam"] = state["gam"].reshape(npp, -1).copy()
        if "Hp" in state:
            new_state["Hp"] = state["Hp"].reshape(npp, 3, 3, -1).copy()
            new_state["pl"] = state["pl"].reshape(npp, -1).copy()
    for ph, mat in enumerate(materials):
        idx = groups[ph]
        if idx.size == 0:
            continue
        Gv = Gf[..., idx]
        if mat.law == ISO_ELASTIC:
            lam, mu = mat.params[:2]
            eps = _sym(Gv)
            tr = eps[:, 0, 0] + eps[:, 1, 1] + eps[:, 2, 2]
            P[..., idx] = 2.0 * mu * eps + lam * tr[:, None, None] * I3[None, :, :, None]
        elif mat.law == CUBIC_ELASTIC:
            C = rotated_cubic(mat.params[:3], mat.quat)
            P[..., idx] = np.einsum("ijkl,rklm->rijm", C, _sym(Gv))
        elif mat.law == B0_LINEAR:
            lam, mu = mat.params[:2]
            diag = np.einsum("riim->rim", Gv)
            out = 2.0 * mu * Gv
            for i in range(3):
                out[:, i, i] += lam * diag[:, i]
            P[..., idx] = out
        elif mat.law == J2_LINHARD:
            lam, mu, sy, H = mat.params[:4]
            if state is None:
                ep_n = np.zeros_like(Gv)
                p_n = np.zeros((npp, idx.size))
            else:
                ep_n = new_state["ep"][..., idx]
                p_n = new_state["p"][..., idx]
            sig, ep, p = j2_return(_sym(Gv), ep_n, p_n, lam, mu, sy, H)
            P[..., idx] = sig
            if new_state is not None:
                new_state["ep"][..., idx] = ep
                new_state["p"][..., idx] = p
        elif mat.law == SVK_CUBIC:
            P[..., idx] = finite.svk_cubic(Gv, mat.params, mat.quat)
        elif mat.law == NEO_HOOKE:
            P[..., idx] = finite.neo_hooke(Gv, mat.params)
        elif mat.law == CP_FCC:
            if state is None:
                Fp_n = np.broadcast_to(I3[None, :, :, None], (npp, 3, 3, idx.size)).copy()
                gam_n = np.zeros((npp, idx.size))
            else:
                Fp_n = new_state["Fp"][..., idx]
                gam_n = new_state["gam"][..., idx]
            S, Fp, gam = finite.cp_fcc(Gv, mat.params, mat.quat, Fp_n, gam_n)
            P[..., idx] = S
            if new_state is not None:
                new_state["Fp"][..., idx] = Fp
                new_state["gam"][..., idx] = gam
        elif mat.law == LOG_J2:
            if state is None:
                Hp_n = np.zeros((npp, 3, 3, idx.size))
                pl_n = np.zeros((npp, idx.size))
            else:
                Hp_n = new_state["Hp"][..., idx]
                pl_n = new_state["pl"][..., idx]
            S, Hp, pl = finite.log_j2(Gv, mat.params, Hp_n, pl_n)
            P[..., idx] = S
            if new_state is not None:
                new_state["Hp"][..., idx] = Hp
                new_state["pl"][..., idx] = pl
        else:
            raise ValueError(f"unknown law {mat.law}")
    P = P.reshape(shp)
    if new_state is not None:
        out = {}
        if "ep" in new_state:
            out["ep"] = new_state["ep"].reshape(shp)
            out["p"] = new_state["p"].reshape((npp,) + shp[3:])
        if "Fp" in new_state:
            out["Fp"] = new_state["Fp"].reshape(shp)
            out["gam"] = new_state["gam"].reshape((npp,) + shp[3:])
        if "Hp" in new_state:
            out["Hp"] = new_state["Hp"].reshape(shp)
            out["pl"] = new_state["pl"].reshape((npp,) + shp[3:])
        new_state = out
    return P, new_state


def c0_apply(G, lambda0, mu0):
    """R0 : G for the C0 preconditioner, 2 mu0 G + lambda0 tr(G) 1 (Eq. TF_C0_behavior)."""
    out = 2.0 * mu0 * G
    tr = G[:, 0, 0] + G[:, 1, 1] + G[:, 2, 2]
    for i in range(3):
        out[:, i, i] += lambda0 * tr
    return out


def b0_apply(G, lambda0, mu0):
    """R0 : G for the B0 preconditioner, 2 mu0 G + lambda0 G (.) I (Sec. 2.6.3)."""
    out = 2.0 * mu0 * G
    for i in range(3):
        out[:, i, i] += lambda0 * G[:, i, i]
    return out
