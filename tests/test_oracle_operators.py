"""Pins of the oracle's sum-factorised operators BP1.0, BP3.5 and BP3.0
(Algorithms 1-5) against brute-force element matrices built from the
quadrature sums of Section 4, exact-integration invariants, closed forms
and symmetry -- chosen so that a dropped term, a wrong sign, a wrong index
or a transposed operand fails at least one of them."""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import fem_synth
import oracle


def _mesh(nx=2, jitter=0.15, seed=11):
    return fem_synth.box_mesh(nx, jitter=jitter, seed=seed)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- dense ---

@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_bp1_equals_dense_mass(N):
    v = _mesh()
    q = fem_synth.field(2, v.shape[0], (N + 1) ** 3)
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    got = oracle.bp1(N, wJ, q)
    for e in range(v.shape[0]):
        M = oracle.dense_element(N, v[e], "gauss", stiff=False)
        assert _rel(got[e], M @ q[e]) < 1e-13


@pytest.mark.parametrize("N,lam", [(1, 1.0), (2, 0.0), (3, 1.0), (4, 2.5)])
def test_bp35_equals_dense_gll_operator(N, lam):
    v = _mesh()
    q = fem_synth.field(2, v.shape[0], (N + 1) ** 3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    got = oracle.bp35(N, G, lam, q)
    for e in range(v.shape[0]):
        A = oracle.dense_element(N, v[e], "gll", stiff=True, lam=lam)
        assert _rel(got[e], A @ q[e]) < 1e-12


@pytest.mark.parametrize("N,lam", [(1, 1.0), (2, 0.0), (3, 1.0), (4, 2.5)])
def test_bp30_equals_dense_gauss_operator(N, lam):
    v = _mesh()
    q = fem_synth.field(2, v.shape[0], (N + 1) ** 3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    got = oracle.bp30(N, G, lam, q)
    for e in range(v.shape[0]):
        A = oracle.dense_element(N, v[e], "gauss", stiff=True, lam=lam)
        assert _rel(got[e], A @ q[e]) < 1e-12


def test_dense_element_matrices_are_symmetric():
    v = _mesh()[3]
    for rule, stiff in (("gauss", False), ("gll", True), ("gauss", True)):
        A = oracle.dense_element(3, v, rule, stiff=stiff, lam=0.7)
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())


# ------------------------------------------------------- mass invariants ---

def _fd_detJ(v8, r, s, t, h=0.25):
    X = np.zeros((3, 3))
    for col, d in enumerate(np.eye(3)):
        xp, _ = oracle.trilinear(v8, r + h * d[0], s + h * d[1], t + h * d[2])
        xm, _ = oracle.trilinear(v8, r - h * d[0], s - h * d[1], t - h * d[2])
        X[:, col] = (xp - xm) / (2 * h)
    return np.linalg.det(X)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 10, 15])
def test_bp1_volume(N):
    """1^T M 1 = volume (1 interpolates to 1, sum of w detJ = volume)."""
    v = _mesh(nx=3)
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    one = np.ones((v.shape[0], (N + 1) ** 3))
    assert abs(oracle.bp1(N, wJ, one).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 6])
def test_bp1_energy_is_exact_integral(N):
    """q^T M q = integral of u^2 |J| over the reference cube for u in Q^N:
    the N+2 point Gauss rule integrates degree 2N+2 per direction exactly.
    Reference by a 14-point numpy Gauss rule and a finite-difference |J|."""
    v = _mesh(nx=2, jitter=0.2)[:3]
    b = oracle.Basis(N)
    rng = np.random.default_rng(N)
    xg, wg = npleg.leggauss(14)
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    for e in range(v.shape[0]):
        # u(r,s,t) = pr(r) ps(s) pt(t) + po(r) (a second separable term)
        polys = [np.polynomial.Polynomial(rng.standard_normal(N + 1)) for _ in range(4)]
        u = lambda r, s, t: polys[0](r) * polys[1](s) * polys[2](t) + polys[3](r)  # noqa: E731
        q = np.array([u(b.r[i], b.r[j], b.r[k])
                      for k in range(N + 1) for j in range(N + 1) for i in range(N + 1)])
        Mq = oracle.bp1(N, wJ[e:e + 1], q[None])[0]
        ref = 0.0
        for (a, ra), (bb, sb), (c, tc) in itertools.product(enumerate(xg), repeat=3):
            ref += wg[a] * wg[bb] * wg[c] * u(ra, sb, tc) ** 2 * _fd_detJ(v[e], ra, sb, tc)
        assert abs(q @ Mq - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("N", [1, 2, 4])
def test_bp1_affine_kronecker_closed_form(N):
    """On an undistorted cube M^e = detJ (M1 x M1 x M1) with M1 the exact 1D
    Lagrange mass matrix (numpy polynomial products and integrals)."""
    h = 0.5
    v = fem_synth.box_mesh(2, jitter=0.0)[:1]
    b = oracle.Basis(N)
    n = N + 1
    L = []
    for i in range(n):
        others = np.delete(b.r, i)
        L.append(np.polynomial.Polynomial.fromroots(others) / np.prod(b.r[i] - others))
    M1 = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            P = (L[i] * L[j]).integ()
            M1[i, j] = P(1.0) - P(-1.0)
    Me = (h / 2) ** 3 * np.kron(np.kron(M1, M1), M1)
    wJ, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    q = fem_synth.field(5, 1, n ** 3)
    assert _rel(oracle.bp1(N, wJ, q)[0], Me @ q[0]) < 1e-11


# -------------------------------------------------- stiffness invariants ---

@pytest.mark.parametrize("N", [1, 2, 3, 7, 12, 15])
def test_stiffness_annihilates_constants(N):
    v = _mesh(nx=2)
    one = np.ones((v.shape[0], (N + 1) ** 3))
    G35, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    G30, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    scale35 = np.abs(oracle.bp35(N, G35, 0.0, fem_synth.field(3, v.shape[0], (N + 1) ** 3))).max()
    scale30 = np.abs(oracle.bp30(N, G30, 0.0, fem_synth.field(3, v.shape[0], (N + 1) ** 3))).max()
    assert np.abs(oracle.bp35(N, G35, 0.0, one)).max() < 1e-13 * scale35
    assert np.abs(oracle.bp30(N, G30, 0.0, one)).max() < 1e-13 * scale30
    # with lambda: A 1 = lambda M 1, and the sum over everything is lambda * vol
    assert abs(oracle.bp30(N, G30, 2.0, one).sum() - 2.0) < 1e-12
    if N >= 2:
        assert abs(oracle.bp35(N, G35, 2.0, one).sum() - 2.0) < 1e-12


def _linear_field(v, N, a, nodes):
    """u = a . x at each element's GLL nodes (physical coordinates from the map)."""
    E = v.shape[0]
    n = N + 1
    q = np.zeros((E, n ** 3))
    for e in range(E):
        p = 0
        for k, j, i in itertools.product(range(n), repeat=3):
            x, _ = oracle.trilinear(v[e], nodes[i], nodes[j], nodes[k])
            q[e, p] = a @ x
            p += 1
    return q


@pytest.mark.parametrize("N", [1, 2, 3, 5, 9])
def test_linear_field_energy(N):
    """q^T S q = |a|^2 vol for u = a.x (physical gradient a everywhere; the
    integrand |a|^2 w detJ is integrated exactly by Gauss rules, and by GLL
    rules for N >= 2)."""
    v = _mesh(nx=2, jitter=0.2)
    b = oracle.Basis(N)
    a = np.array([0.3, -1.2, 0.7])
    q = _linear_field(v, N, a, b.r)
    G30, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    e30 = np.sum(q * oracle.bp30(N, G30, 0.0, q))
    assert abs(e30 - a @ a) < 1e-12
    if N >= 2:
        G35, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
        e35 = np.sum(q * oracle.bp35(N, G35, 0.0, q))
        assert abs(e35 - a @ a) < 1e-12


def _grad_energy_ref(A, polys_sum, N, npts=14):
    """integral over the reference cube of |A^{-T} grad_r u|^2 det A for
    u = sum_d p_d(rhat_d) + p3(r) p4(s) p5(t), by a numpy Gauss rule."""
    xg, wg = npleg.leggauss(npts)
    Ai = np.linalg.inv(A)
    dA = np.linalg.det(A)
    p = polys_sum
    dp = [pp.deriv() for pp in p]
    ref = 0.0
    for (a, ra), (bb, sb), (c, tc) in itertools.product(enumerate(xg), repeat=3):
        gr = np.array([dp[0](ra) + dp[3](ra) * p[4](sb) * p[5](tc),
                       dp[1](sb) + p[3](ra) * dp[4](sb) * p[5](tc),
                       dp[2](tc) + p[3](ra) * p[4](sb) * dp[5](tc)])
        gx = Ai.T @ gr
        ref += wg[a] * wg[bb] * wg[c] * (gx @ gx) * dA
    return ref


def _nodal(p, nodes):
    n = len(nodes)
    return np.array([p[0](nodes[i]) + p[1](nodes[j]) + p[2](nodes[k])
                     + p[3](nodes[i]) * p[4](nodes[j]) * p[5](nodes[k])
                     for k in range(n) for j in range(n) for i in range(n)])


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_affine_bp30_energy_is_exact_integral(N):
    """On an affine element the N+2 point Gauss rule integrates the stiffness
    integrand (degree <= 2N per direction) exactly, so q^T S q equals the
    exact Dirichlet energy of u for every u in Q^N (Section 4, BP3.0)."""
    rng = np.random.default_rng(7 + N)
    A = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    corners = np.array([[(-1.0, 1.0)[(c >> k) & 1] for k in range(3)] for c in range(8)])
    v = (corners @ A.T + rng.standard_normal(3))[None]
    b = oracle.Basis(N)
    p = [np.polynomial.Polynomial(rng.standard_normal(N + 1)) for _ in range(6)]
    q = _nodal(p, b.r)[None]
    G30, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    got = float(q[0] @ oracle.bp30(N, G30, 0.0, q)[0])
    ref = _grad_energy_ref(A, p, N)
    assert abs(got - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_box_bp35_energy_exact_for_additive_fields(N):
    """On an axis-aligned box G is diagonal and constant; for an additive
    field u = f(r) + g(s) + h(t) each term of the integrand has degree 2N-2
    in one direction and 0 in the others, which the GLL rule integrates
    exactly, so q^T S q is the exact Dirichlet energy (Section 4, BP3.5)."""
    rng = np.random.default_rng(17 + N)
    A = np.diag([0.3, 0.5, 0.2])
    corners = np.array([[(-1.0, 1.0)[(c >> k) & 1] for k in range(3)] for c in range(8)])
    v = (corners @ A.T + np.array([0.1, -0.2, 0.3]))[None]
    b = oracle.Basis(N)
    p = [np.polynomial.Polynomial(rng.standard_normal(N + 1)) for _ in range(3)]
    p += [np.polynomial.Polynomial([0.0])] * 3
    q = _nodal(p, b.r)[None]
    G35, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    got = float(q[0] @ oracle.bp35(N, G35, 0.0, q)[0])
    ref = _grad_energy_ref(A, p, N)
    assert abs(got - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("op", ["bp1", "bp35", "bp30"])
@pytest.mark.parametrize("N", [1, 3, 8])
def test_symmetry_and_positivity(op, N):
    v = _mesh(nx=2, jitter=0.2)
    E = v.shape[0]
    x = fem_synth.field(21, E, (N + 1) ** 3)
    y = fem_synth.field(22, E, (N + 1) ** 3)
    if op == "bp1":
        g, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
        f = lambda z: oracle.bp1(N, g, z)  # noqa: E731
    elif op == "bp35":
        g, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
        f = lambda z: oracle.bp35(N, g, 1.0, z)  # noqa: E731
    else:
        g, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
        f = lambda z: oracle.bp30(N, g, 1.0, z)  # noqa: E731
    Ax, Ay = f(x), f(y)
    # per element (the operator is block diagonal)
    lhs, rhs = np.sum(y * Ax, axis=1), np.sum(x * Ay, axis=1)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(Ax).max() * np.abs(y).sum(axis=1).max()
    assert np.all(np.sum(x * Ax, axis=1) > 0)


def test_block_diagonal():
    """Changing element e's input changes only element e's output
    (Section 4: the unassembled operator is block diagonal)."""
    N = 3
    v = _mesh(nx=2)
    E = v.shape[0]
    q = fem_synth.field(2, E, (N + 1) ** 3)
    g, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    base = oracle.bp30(N, g, 1.0, q)
    q2 = q.copy()
    q2[5] += 1.0
    out = oracle.bp30(N, g, 1.0, q2)
    changed = np.nonzero(np.abs(out - base).max(axis=1) > 0)[0]
    assert list(changed) == [5]
