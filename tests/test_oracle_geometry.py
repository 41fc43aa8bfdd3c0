"""Pins of the oracle's geometry (Section 4: trilinear element map, |J|,
the scaled metric G and the diagonal weight matrices G^e, J^e)."""
import itertools

import numpy as np
import pytest

import fem_synth
import oracle


def _fd_jacobian(v8, r, s, t, h=1e-3):
    """X by central differences of the map; exact up to rounding because the
    trilinear map is linear in each reference coordinate separately."""
    X = np.zeros((3, 3))
    for col, d in enumerate(np.eye(3)):
        xp, _ = oracle.trilinear(v8, r + h * d[0], s + h * d[1], t + h * d[2])
        xm, _ = oracle.trilinear(v8, r - h * d[0], s - h * d[1], t - h * d[2])
        X[:, col] = (xp - xm) / (2 * h)
    return X


def test_map_interpolates_vertices():
    v = fem_synth.box_mesh(3, jitter=0.1)[13]
    for c in range(8):
        r, s, t = [(-1.0, 1.0)[(c >> b) & 1] for b in range(3)]
        x, _ = oracle.trilinear(v, r, s, t)
        np.testing.assert_allclose(x, v[c], rtol=0, atol=1e-15)


def test_map_jacobian_matches_finite_differences():
    v = fem_synth.box_mesh(4, jitter=0.2)[21]
    rng = np.random.default_rng(0)
    for r, s, t in rng.uniform(-1, 1, size=(20, 3)):
        _, X = oracle.trilinear(v, r, s, t)
        np.testing.assert_allclose(X, _fd_jacobian(v, r, s, t), rtol=0, atol=1e-11)


@pytest.mark.parametrize("N", [1, 3, 7])
def test_unit_cube_closed_form(N):
    """Undistorted cube of side h: X = (h/2) Id, detJ = (h/2)^3,
    G = w (h/2) Id, wJ = w (h/2)^3."""
    nx = 8
    h = 1.0 / nx
    v = fem_synth.box_mesh(nx, jitter=0.0)
    b = oracle.Basis(N)
    for kind, (x, w) in ((oracle.KIND_BP35, (b.r, b.w)), (oracle.KIND_BP30, (b.rt, b.wt))):
        geo, mindet = oracle.geofacs(N, kind, v)
        q = len(x)
        W = np.einsum("c,b,a->cba", w, w, w).reshape(-1)
        assert abs(mindet - (h / 2) ** 3) < 1e-17
        for g, ref in zip(range(7), [h / 2, 0, 0, h / 2, 0, h / 2, (h / 2) ** 3]):
            np.testing.assert_allclose(geo[:, g, :], np.broadcast_to(W * ref, (v.shape[0], q ** 3)),
                                       rtol=1e-14, atol=1e-16)
    wj, _ = oracle.geofacs(N, oracle.KIND_BP1, v)
    W = np.einsum("c,b,a->cba", b.wt, b.wt, b.wt).reshape(-1)
    np.testing.assert_allclose(wj, np.broadcast_to(W * (h / 2) ** 3, wj.shape), rtol=1e-14)


def test_affine_element_metric_against_numpy_inverse():
    """Affine element x = A rhat + b: X = A everywhere and
    G = w detA A^{-1} A^{-T} (numpy.linalg for the inverse)."""
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    b0 = rng.standard_normal(3)
    v = np.array([A @ np.array([(-1.0, 1.0)[(c >> k) & 1] for k in range(3)]) + b0
                  for c in range(8)])[None]
    N = 4
    ob = oracle.Basis(N)
    geo, mindet = oracle.geofacs(N, oracle.KIND_BP35, v)
    Ai = np.linalg.inv(A)
    Gref = np.linalg.det(A) * Ai @ Ai.T
    W = np.einsum("c,b,a->cba", ob.w, ob.w, ob.w).reshape(-1)
    for g, (p, q) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        np.testing.assert_allclose(geo[0, g], W * Gref[p, q], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(geo[0, 6], W * np.linalg.det(A), rtol=1e-13)
    assert abs(mindet - np.linalg.det(A)) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 5])
def test_jittered_metric_against_finite_differences(N):
    """G / (w detJ) = X^{-1} X^{-T} with X from finite differences and
    numpy's determinant and inverse, at every quadrature point."""
    v = fem_synth.box_mesh(3, jitter=0.1)[:5]
    b = oracle.Basis(N)
    geo, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    q = N + 2
    for e in range(v.shape[0]):
        for c, bb, a in itertools.product(range(q), repeat=3):
            X = _fd_jacobian(v[e], b.rt[a], b.rt[bb], b.rt[c], h=0.25)
            det = np.linalg.det(X)
            Xi = np.linalg.inv(X)
            G = det * Xi @ Xi.T
            W = b.wt[a] * b.wt[bb] * b.wt[c]
            p = a + q * (bb + q * c)
            got = geo[e, :, p]
            ref = W * np.array([G[0, 0], G[0, 1], G[0, 2], G[1, 1], G[1, 2], G[2, 2], det])
            np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 15])
def test_total_volume(N):
    """sum of w detJ over all nodes = volume of the unit cube: Gauss rules
    always (detJ of a trilinear map has degree <= 2 per direction), GLL
    rules for N >= 2."""
    v = fem_synth.box_mesh(4, jitter=0.1)
    for kind in (oracle.KIND_BP1, oracle.KIND_BP30):
        geo, mindet = oracle.geofacs(N, kind, v)
        tot = geo.sum() if kind == oracle.KIND_BP1 else geo[:, 6].sum()
        assert abs(tot - 1.0) < 1e-13
        assert mindet > 0
    geo, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    if N >= 2:
        assert abs(geo[:, 6].sum() - 1.0) < 1e-13


def test_jittered_mesh_not_inverted():
    v = fem_synth.box_mesh(32, jitter=0.1)
    _, mindet = oracle.geofacs(1, oracle.KIND_BP30, v)
    h = 1.0 / 32
    assert mindet > 0.3 * (h / 2) ** 3
