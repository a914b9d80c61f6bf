"""Pins of the Anderson step and of how the solver loop feeds it (Sec. 2.3, Algorithm 1).

The paper states only that the acceleration acts on p, every 2 or 3 iterations, from the
last 4 couples.  The reading (type-II Anderson on the couples (q_j, g_j = p_{j+1})) is pinned
here by what it implies for an affine fixed-point map g(q) = M q + b, whose residual
f(q) = g(q) - q is affine too:

* with as many couples as the dimension + 1, the constrained least squares cancels the
  residual exactly (sum c_j f_j = 0 with sum c_j = 1), so the mixed field sum c_j g_j IS the
  fixed point: one accepted step lands on it to rounding;
* with fewer couples, the residual of the mixed field is M r, r = sum c_j f_j the minimal
  residual, whereas mixing the q_j instead would leave exactly r (so the test tells the
  two apart);
* in the oracle's solver, a linear-elastic problem with 3 free node components (a 2x2x2
  grid with Dirichlet faces everywhere: one interior node) makes the map q -> p of one
  iteration affine in dimension 3: the iteration after the first accepted Anderson step
  has a zero residual to rounding.  A couple paired with the wrong g, or a combination of
  the wrong fields, fails this.

The skip rule (the angle test on the residual differences) is pinned by its own
definition: a history whose differences are collinear is refused and one at a right angle
is accepted, independently of the scale of each difference; and its threshold by where
the rounding of the paper's FP64 iteration puts exactly collinear histories (laminates)
and where genuinely three-dimensional ones sit.
"""

import numpy as np

from oracle import anderson
from oracle.solver import Problem
from synthetic.workloads import ISO_ELASTIC, Material, Workload, axis_bc, iso_lame


def _affine(dim, seed, contraction=0.8):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
    M = Q @ np.diag(contraction * rng.uniform(-1.0, 1.0, dim)) @ Q.T + 0.05 * rng.standard_normal((dim, dim))
    b = rng.standard_normal(dim)
    return M, b


def _run_mixer(M, b, depth, period, iters):
    """Drive anderson.Mixer exactly as the solver loop does, with p_{m+1} = g(q_m)."""
    mixer = anderson.Mixer(depth, period)
    p = b.copy()  # p_0 = g(0)
    trace = []
    for m in range(iters):
        q, mixed = mixer.propose(m, p)
        trace.append((m, q.copy(), mixed, [(qq.copy(), gg.copy()) for qq, gg in mixer.hist]))
        p = M @ q + b
    return trace


def test_full_history_lands_on_the_fixed_point_of_an_affine_map():
    M, b = _affine(3, 5)
    x_star = np.linalg.solve(np.eye(3) - M, b)
    trace = _run_mixer(M, b, depth=4, period=3, iters=6)
    m, q, mixed, hist = trace[5]  # first iteration with m % 3 == 2 and 4 couples
    assert mixed and len(hist) == 4
    assert not any(t[2] for t in trace[:5])
    assert np.linalg.norm(q - x_star) < 1e-12 * np.linalg.norm(x_star)
    # and the couples are (q_j, g(q_j)): each stored g is the map applied to its own q
    for qq, gg in hist:
        assert np.allclose(gg, M @ qq + b, rtol=0, atol=1e-14)


def test_the_mix_combines_the_g_fields_type_two():
    dim = 6
    M, b = _affine(dim, 9)
    trace = _run_mixer(M, b, depth=4, period=3, iters=6)
    m, q, mixed, hist = trace[5]
    assert mixed
    fs = [g_ - q_ for q_, g_ in hist]
    c = anderson.coefficients(fs)
    r = sum(cj * f for cj, f in zip(c, fs))          # the minimal residual of the history
    q_bar = sum(cj * q_ for cj, (q_, _) in zip(c, hist))
    assert np.allclose(q, q_bar + r, rtol=0, atol=1e-13)   # sum c_j g_j = sum c_j q_j + r
    f_new = M @ q + b - q
    assert np.allclose(f_new, M @ r, rtol=0, atol=1e-13)   # type II: f(sum c g) = M r
    assert np.linalg.norm(f_new - r) > 1e-3 * np.linalg.norm(r)  # a mix of the q_j would give r


def test_skip_rule_is_the_angle_between_differences_and_ignores_their_scale():
    e = np.eye(4)
    last = np.array([1.0, 2.0, 3.0, 4.0])
    # differences e0 and 1e6 e1 (scaled): orthogonal -> accepted
    ok = anderson.coefficients([last + e[0], last + 1e6 * e[1], last])
    assert ok is not None
    # differences e0 and e0 + 1e-5 e1: sin^2 of the angle 1e-10 < 1e-8 -> skipped
    assert anderson.coefficients([last + e[0], last + e[0] + 1e-5 * e[1], last]) is None
    # the same pair scaled by 1e-9 and 1e9: still skipped (scale-free)
    assert anderson.coefficients([last + 1e-9 * e[0], last + 1e9 * (e[0] + 1e-5 * e[1]), last]) is None
    # at sin^2 = 1e-6 (angle 1e-3 rad) the mix is kept
    assert anderson.coefficients([last + e[0], last + e[0] + 1e-3 * e[1], last]) is not None


def _three_dof_problem():
    n = (2, 2, 2)
    phase = np.zeros(n, dtype=np.uint16)
    phase[0, 0, 0] = phase[1, 1, 0] = phase[1, 0, 1] = 1
    m0 = Material(ISO_ELASTIC, iso_lame(1.0, 0.3))
    m1 = Material(ISO_ELASTIC, iso_lame(20.0, 0.2))
    lam0 = 0.5 * (m0.params[0] + m1.params[0])
    mu0 = 0.5 * (m0.params[1] + m1.params[1])
    A = np.array([[1e-3, 2e-4, 0.0], [0.0, -3e-4, 1e-4], [5e-4, 0.0, 2e-4]])
    return Workload("three_dof", n, phase, [m0, m1], axis_bc("D", "D", "D"), scheme="HEX1",
                    lambda0=lam0, mu0=mu0, tol=1e-300, max_iter=6, A=A, h=(1.0, 1.3, 0.8))


def test_solver_lands_on_the_solution_after_the_first_anderson_step_with_three_free_dofs():
    wl = _three_dof_problem()
    pr = Problem(wl)
    assert sum(int(mk.sum()) for mk in pr.masks) == 3
    _, rep = pr.solve_step()
    assert rep.accelerated == [5]
    err = rep.err
    # the plain fixed point is still far from the solution before the mix ...
    assert err[5] > 1e-4 * err[0]
    # ... and the mix of 4 couples in dimension 3 lands on it to rounding
    assert err[6] < 1e-12 * err[0], err


def test_without_anderson_the_same_problem_converges_only_geometrically():
    wl = _three_dof_problem()
    pr = Problem(wl)
    _, rep = pr.solve_step(anderson=False)
    assert rep.accelerated == []
    assert rep.err[6] > 1e-6 * rep.err[0]


def _pivot_ratios_of_a_solve(wl, tol):
    """Every normal matrix the oracle's Anderson step tests during a solve, as the smallest
    Cholesky pivot relative to its diagonal entry (sin^2 of the angle between a residual
    difference and the span of the previous ones)."""
    seen = []
    orig = anderson.normal_matrix_ok

    def spy(A, tol_=anderson.PIVOT_TOL):
        m = A.shape[0]
        L = np.zeros_like(A)
        worst = 1.0
        for k in range(m):
            d = A[k, k] - np.dot(L[k, :k], L[k, :k])
            worst = min(worst, d / A[k, k] if A[k, k] > 0 else 0.0)
            if d <= 0:
                break
            L[k, k] = np.sqrt(d)
            for i in range(k + 1, m):
                L[i, k] = (A[i, k] - np.dot(L[i, :k], L[k, :k])) / L[k, k]
        seen.append(worst)
        return orig(A, tol_)

    anderson.normal_matrix_ok = spy
    try:
        Problem(wl).solve_step(tol=tol)
    finally:
        anderson.normal_matrix_ok = orig
    return seen


def test_skip_threshold_sits_between_rounding_and_genuine_mixes():
    """Why 1e-8: a laminate's residual sequence is one-dimensional, so its residual differences
    are collinear in exact arithmetic and only the FP64 rounding of the paper's p-form
    iteration (f = g - q, a cancellation of two O(|p|) fields) gives them an angle.  That
    rounding angle grows as the residual shrinks; down to tolerance 1e-10 its pivot ratio
    stays below 1e-8, so every such mix is skipped.  Genuinely three-dimensional histories
    (a sphere composite, a polycrystal) sit above 1e-3.  A threshold of 1e-12 would admit the
    rounding-determined mixes of the laminates at tolerance 1e-9 and below."""
    import synthetic as syn

    noise = []
    for wl in (syn.x_laminate(n=(36, 4, 4), period=6, scheme="TETRA2"),
               syn.y_laminate(n=(6, 36, 4), period=6, scheme="HEX1")):
        for tol in (1e-6, 1e-8, 1e-10):
            noise += _pivot_ratios_of_a_solve(wl, tol)
    assert max(noise) < anderson.PIVOT_TOL
    assert max(noise) > 1e-12  # a threshold of 1e-12 would not have rejected all of them
    genuine = []
    for wl in (syn.sphere_inclusion_32(n=16, radius=4),
               syn.voronoi_polycrystal(n=(24, 18, 16), grains=12, tol=1e-8)):
        genuine += _pivot_ratios_of_a_solve(wl, wl.tol)
    assert min(genuine) > 1e-3
