"""Oracle constitutive laws pinned by textbook results (T8), and the synthetic inputs."""

import os

import numpy as np
import pytest
from scipy.optimize import brentq

import synthetic as syn
from oracle.laws import (CUBIC_ELASTIC, ISO_ELASTIC, J2_LINHARD, cubic_tensor, iso_tensor,
                         quat_to_rotation, rotated_cubic, stress)
from synthetic.workloads import Material

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "materials.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _point(G, mats, state=None):
    """Evaluate the law on a single voxel point."""
    G = np.asarray(G, dtype=np.float64).reshape(1, 3, 3, 1, 1, 1)
    groups = [np.array([0])] + [np.array([], dtype=np.int64)] * (len(mats) - 1)
    P, st = stress(G, mats, groups, state)
    return P[0, :, :, 0, 0, 0], st


def test_cubic_identity_rotation_reproduces_constants():
    g = _golden()
    C = rotated_cubic((g["C11"], g["C12"], g["C44"]), (1.0, 0.0, 0.0, 0.0))
    assert C[0, 0, 0, 0] == g["C11"] and C[0, 0, 1, 1] == g["C12"] and C[0, 1, 0, 1] == g["C44"]
    # uniaxial strain along a cube axis: sigma_11 = C11 eps, sigma_22 = C12 eps
    P, _ = _point(np.diag([1e-3, 0, 0]), [Material(CUBIC_ELASTIC, (168.0, 121.0, 75.0))])
    assert np.allclose(np.diag(P), [0.168, 0.121, 0.121], rtol=1e-14)


def test_cubic_rotation_invariants():
    q = syn.shoemake_quaternions(5, 1)
    for qt in q:
        R = quat_to_rotation(qt)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1) < 1e-14
        C = rotated_cubic((168.0, 121.0, 75.0), qt)
        # bulk modulus: 1 : C : 1 / 9 = (C11 + 2 C12) / 3
        K = np.einsum("iijj->", C) / 9.0
        assert abs(K - (168.0 + 2 * 121.0) / 3.0) < 1e-11
        # full symmetric invariants: C_ijij and the Frobenius norm
        C0 = cubic_tensor(168.0, 121.0, 75.0)
        assert abs(np.einsum("ijij->", C) - np.einsum("ijij->", C0)) < 1e-10
        assert abs(np.sum(C * C) - np.sum(C0 * C0)) < 1e-8
        # major and minor symmetries
        assert np.allclose(C, C.transpose(1, 0, 2, 3)) and np.allclose(C, C.transpose(2, 3, 0, 1))


def test_cubic_with_zener_ratio_one_is_isotropic():
    lam, mu = 2.0, 1.5
    C = rotated_cubic((lam + 2 * mu, lam, mu), syn.shoemake_quaternions(1, 4)[0])
    assert np.allclose(C, iso_tensor(lam, mu), atol=1e-13)


def test_isotropic_hooke():
    lam, mu = 1.2, 0.8
    rng = np.random.default_rng(1)
    G = rng.standard_normal((3, 3)) * 1e-3
    P, _ = _point(G, [Material(ISO_ELASTIC, (lam, mu))])
    eps = 0.5 * (G + G.T)
    assert np.allclose(P, lam * np.trace(eps) * np.eye(3) + 2 * mu * eps, atol=1e-16)


def test_j2_simple_shear_closed_form():
    E, nu, sy, H = 200000.0, 0.3, 300.0, 2000.0
    lam, mu = syn.iso_lame(E, nu)
    mat = [Material(J2_LINHARD, (lam, mu, sy, H))]
    for gam in [1e-4, 2e-3, 1e-2]:
        e12 = 0.5 * gam
        G = np.zeros((3, 3))
        G[0, 1] = G[1, 0] = e12
        P, _ = _point(G, mat, {"ep": np.zeros((1, 3, 3, 1, 1, 1)), "p": np.zeros((1, 1, 1, 1))})
        if np.sqrt(3.0) * 2 * mu * e12 <= sy:
            ref = 2 * mu * e12
        else:
            s3 = np.sqrt(3.0)
            ep12 = (2 * s3 * mu * e12 - sy) / (2 * s3 * mu + 2 * H / s3)
            ref = 2 * mu * (e12 - ep12)
        assert abs(P[0, 1] - ref) < 1e-9 * abs(ref)


def test_j2_uniaxial_stress_tangent():
    """Uniaxial stress: sigma = sigma_y + E H / (E + H) (eps - sigma_y / E) beyond yield."""
    E, nu, sy, H = 200000.0, 0.3, 300.0, 2000.0
    lam, mu = syn.iso_lame(E, nu)
    mat = [Material(J2_LINHARD, (lam, mu, sy, H))]
    st0 = {"ep": np.zeros((1, 3, 3, 1, 1, 1)), "p": np.zeros((1, 1, 1, 1))}
    for eps in [1e-3, 4e-3, 1e-2]:
        def lateral(e):
            P, _ = _point(np.diag([eps, e, e]), mat, st0)
            return P[1, 1]
        e_t = brentq(lateral, -eps, eps, xtol=1e-16)
        P, _ = _point(np.diag([eps, e_t, e_t]), mat, st0)
        ref = sy + E * H / (E + H) * (eps - sy / E) if E * eps > sy else E * eps
        assert abs(P[0, 0] - ref) < 1e-7 * ref


def test_phase_maps_are_exact():
    ph = syn.centred_sphere((32, 32, 32), 8)
    j = np.arange(32)
    d2 = ((2 * j[:, None, None] + 1 - 32) ** 2 + (2 * j[None, :, None] + 1 - 32) ** 2
          + (2 * j[None, None, :] + 1 - 32) ** 2)
    assert np.array_equal(ph == 1, d2 <= 256)
    n = (9, 7, 5)
    v, seeds = syn.voronoi(n, 6, 3)
    c = [(2 * np.arange(k) + 1) * 128 for k in n]
    for x in range(n[0]):
        for y in range(n[1]):
            for z in range(n[2]):
                d = [(c[0][x] - s[0]) ** 2 + (c[1][y] - s[1]) ** 2 + (c[2][z] - s[2]) ** 2 for s in seeds]
                assert v[x, y, z] == int(np.argmin(d))
    a = syn.random_spheres((24, 24, 24), 0.3, 2, 4, 4)
    assert abs((a == 1).mean() - 0.3) < 0.1 and (a == 1).mean() >= 0.3
