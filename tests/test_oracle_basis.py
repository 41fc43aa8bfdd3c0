"""Pins of the oracle's 1D basis (Section 2 notation; Section 4: GLL and
Gauss rules, eq. interpolationOps and derivativeOps) against closed forms,
library routines and exactness properties -- never against itself."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.interpolate import BarycentricInterpolator

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_closed_forms.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, xs, ws = (p.strip() for p in line.split("|"))
        rule, npts = head.split()
        ev = lambda s: [eval(t, {"sqrt": math.sqrt}) for t in s.split(",")]  # noqa: E731
        rows.append((rule, int(npts), np.array(ev(xs)), np.array(ev(ws))))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[0]}{r[1]}")
def test_closed_form_rules(row):
    rule, npts, xs, ws = row
    x, w = oracle.gll(npts - 1) if rule == "gll" else oracle.gauss(npts)
    np.testing.assert_allclose(x, xs, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, ws, rtol=0, atol=4e-16)


@pytest.mark.parametrize("m", range(1, 21))
def test_gauss_matches_numpy_leggauss(m):
    x, w = oracle.gauss(m)
    xr, wr = npleg.leggauss(m)
    np.testing.assert_allclose(x, xr, rtol=0, atol=4e-16)
    np.testing.assert_allclose(w, wr, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("N", range(2, 17))
def test_gll_interior_are_roots_of_dPN(N):
    x, _ = oracle.gll(N)
    roots = np.sort(npleg.Legendre.basis(N).deriv().roots())
    np.testing.assert_allclose(x[1:-1], roots, rtol=0, atol=1e-13)
    assert x[0] == -1.0 and x[-1] == 1.0


def _mono_integral(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("N", range(1, 16))
def test_quadrature_exactness(N):
    x, w = oracle.gll(N)
    for k in range(0, 2 * N):  # GLL with N+1 points: exact to degree 2N-1
        assert abs(np.dot(w, x ** k) - _mono_integral(k)) < 1e-14
    # and not exact one degree higher (it is a rule with N+1 points)
    assert abs(np.dot(w, x ** (2 * N)) - _mono_integral(2 * N)) > 1e-11
    m = N + 2
    xg, wg = oracle.gauss(m)
    for k in range(0, 2 * m):  # Gauss with m points: exact to degree 2m-1
        assert abs(np.dot(wg, xg ** k) - _mono_integral(k)) < 1e-14


@pytest.mark.parametrize("N", range(1, 16))
def test_interpolation_matrix(N):
    b = oracle.Basis(N)
    n, m = N + 1, N + 2
    assert b.I.shape == (m, n)
    np.testing.assert_allclose(b.I.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    # exact on polynomials of degree <= N
    for k in range(N + 1):
        np.testing.assert_allclose(b.I @ b.r ** k, b.rt ** k, rtol=0, atol=1e-13)
    # centro-symmetry of I (Section 6, kernel 8): I[a][i] = I[m-1-a][n-1-i]
    np.testing.assert_allclose(b.I, b.I[::-1, ::-1], rtol=0, atol=1e-14)
    # against scipy's barycentric interpolation (a library routine)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        ref = BarycentricInterpolator(b.r, e)(b.rt)
        np.testing.assert_allclose(b.I[:, i], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", range(1, 16))
def test_differentiation_matrices(N):
    b = oracle.Basis(N)
    n, m = N + 1, N + 2
    # rows annihilate constants; exact derivative of x^k for k <= N (GLL) and
    # k <= N+1 (Gauss)
    np.testing.assert_allclose(b.D.sum(axis=1), 0.0, rtol=0, atol=1e-11)
    np.testing.assert_allclose(b.Dt.sum(axis=1), 0.0, rtol=0, atol=1e-11)
    for k in range(1, N + 1):
        ref = k * b.r ** (k - 1)
        np.testing.assert_allclose(b.D @ b.r ** k, ref, rtol=0, atol=2e-11 * max(1, N ** 2))
    for k in range(1, m):
        ref = k * b.rt ** (k - 1)
        np.testing.assert_allclose(b.Dt @ b.rt ** k, ref, rtol=0, atol=2e-11 * max(1, N ** 2))
    # anti-centro-symmetry
    np.testing.assert_allclose(b.D, -b.D[::-1, ::-1], rtol=0, atol=1e-12 * N ** 2)
    np.testing.assert_allclose(b.Dt, -b.Dt[::-1, ::-1], rtol=0, atol=1e-12 * N ** 2)
    # GLL corner entries: -N(N+1)/4 and +N(N+1)/4 (closed form)
    assert abs(b.D[0, 0] + N * (N + 1) / 4) < 1e-12 * N * N
    assert abs(b.D[N, N] - N * (N + 1) / 4) < 1e-12 * N * N
    # against the derivative of scipy's interpolant of each cardinal function
    # (compared through numpy's polynomial fit of the same cardinal data)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        c = npleg.legfit(b.r, e, N)  # exact interpolant in the Legendre basis
        ref = npleg.legval(b.r, npleg.legder(c))
        np.testing.assert_allclose(b.D[:, i], ref, rtol=0, atol=1e-9)
    for i in range(m):
        e = np.zeros(m)
        e[i] = 1.0
        c = npleg.legfit(b.rt, e, m - 1)
        ref = npleg.legval(b.rt, npleg.legder(c))
        np.testing.assert_allclose(b.Dt[:, i], ref, rtol=0, atol=1e-9)


def test_rejects_bad_degree():
    with pytest.raises(ValueError):
        oracle.Basis(0)
    with pytest.raises(ValueError):
        oracle.Basis(16)
