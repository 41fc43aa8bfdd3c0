"""Pins of the oracle's Jacobi preconditioner and PCG for the unassembled
BP3.5 screened-Poisson system (Algorithm 4's operator; the solver is the
textbook preconditioned conjugate gradient, Saad Algorithm 9.1)."""
import numpy as np
import pytest
from scipy.sparse.linalg import LinearOperator, cg

import fem_synth
import oracle


@pytest.mark.parametrize("N,lam", [(1, 1.0), (2, 0.5), (3, 1.0), (4, 0.0)])
def test_diagonal_equals_dense_matrix_diagonal(N, lam):
    v = fem_synth.box_mesh(2, jitter=0.2, seed=5)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    d = oracle.bp35_diag(N, G, lam)
    for e in range(v.shape[0]):
        A = oracle.dense_element(N, v[e], "gll", stiff=True, lam=lam)
        np.testing.assert_allclose(d[e], np.diag(A), rtol=1e-13, atol=0)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_manufactured_solution(N):
    """b = A u_I with u_I the nodal interpolant of sin(pi x) sin(pi y) sin(pi z):
    the exact discrete solution is u_I, so the solve error is known."""
    v = fem_synth.box_mesh(3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    X = oracle.gll_node_coordinates(N, v)
    u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    b = oracle.bp35(N, G, 1.0, u)
    x, it, rel = oracle.pcg_bp35(N, G, 1.0, b, tol=1e-12)
    assert rel <= 1e-12 and it > 0
    true_res = np.linalg.norm(b - oracle.bp35(N, G, 1.0, x)) / np.linalg.norm(b)
    assert true_res <= 1e-11
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= 1e-9


def test_matches_scipy_cg():
    """The same system through scipy's conjugate gradients with the same
    Jacobi preconditioner (a library implementation)."""
    N = 3
    v = fem_synth.box_mesh(2, jitter=0.15)
    E = v.shape[0]
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    b = fem_synth.field(9, E, (N + 1) ** 3)
    d = oracle.bp35_diag(N, G, 1.0).reshape(-1)
    n = b.size
    A = LinearOperator((n, n), matvec=lambda z: oracle.bp35(N, G, 1.0, z.reshape(E, -1)).reshape(-1))
    M = LinearOperator((n, n), matvec=lambda z: z / d)
    xs, info = cg(A, b.reshape(-1), rtol=1e-13, atol=0.0, M=M, maxiter=5000)
    assert info == 0
    xo, it, rel = oracle.pcg_bp35(N, G, 1.0, b, tol=1e-13)
    assert np.linalg.norm(xo.reshape(-1) - xs) / np.linalg.norm(xs) < 1e-10


def test_zero_rhs_and_warm_start():
    N = 2
    v = fem_synth.box_mesh(2)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    b = np.zeros((v.shape[0], 27))
    x, it, rel = oracle.pcg_bp35(N, G, 1.0, b)
    assert it == 0 and np.all(x == 0)
    # starting from the solution needs no iteration
    b = fem_synth.field(3, v.shape[0], 27)
    x1, _, _ = oracle.pcg_bp35(N, G, 1.0, b, tol=1e-13)
    x2, it2, rel2 = oracle.pcg_bp35(N, G, 1.0, b, x0=x1, tol=1e-10)
    assert it2 == 0 and rel2 <= 1e-10


@pytest.mark.parametrize("N,lam", [(1, 1.0), (2, 0.5), (3, 1.0), (4, 0.0)])
def test_bp30_diagonal_equals_dense_matrix_diagonal(N, lam):
    v = fem_synth.box_mesh(2, jitter=0.2, seed=6)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    d = oracle.bp30_diag(N, G, lam)
    for e in range(v.shape[0]):
        A = oracle.dense_element(N, v[e], "gauss", stiff=True, lam=lam)
        np.testing.assert_allclose(d[e], np.diag(A), rtol=1e-12, atol=0)


@pytest.mark.parametrize("N", [2, 4])
def test_bp30_manufactured_solution(N):
    v = fem_synth.box_mesh(3)
    G, _ = oracle.geofacs(N, oracle.KIND_BP30, v)
    X = oracle.gll_node_coordinates(N, v)
    u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    b = oracle.bp30(N, G, 1.0, u)
    x, it, rel = oracle.pcg_bp30(N, G, 1.0, b, tol=1e-12)
    assert rel <= 1e-12 and it > 0
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= 1e-9


def _rounded_factors(G, kind):
    """Factors rounded to binary16 after a power-of-two scaling that puts the
    largest below 2^14 (and back), or to FP32."""
    if kind == "fp32":
        return G.astype(np.float32).astype(np.float64)
    e = int(np.frexp(np.abs(G).max())[1])
    s = 2.0 ** (14 - e)
    return (G * s).astype(np.float16).astype(np.float64) / s


@pytest.mark.parametrize("kind", ["fp32", "fp16"])
def test_defect_correction_with_rounded_factors(kind):
    """FP64 defect correction whose inner PCG applies the operator with
    rounded factors (the inner operator of the mixed solver modes): every
    outer step reduces the FP64 residual by about the inner tolerance, with
    binary16 factors as with FP32 ones, and the outer loop reaches 1e-10."""
    N = 5
    v = fem_synth.box_mesh(4)
    G, _ = oracle.geofacs(N, oracle.KIND_BP35, v)
    X = oracle.gll_node_coordinates(N, v)
    u = np.sin(np.pi * X[..., 0]) * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    b = oracle.bp35(N, G, 1.0, u)
    Gl = _rounded_factors(G, kind)
    x = np.zeros_like(b)
    hist = []
    for _ in range(8):
        r = b - oracle.bp35(N, G, 1.0, x)
        hist.append(np.linalg.norm(r) / np.linalg.norm(b))
        if hist[-1] <= 1e-10:
            break
        d, _, _ = oracle.pcg_bp35(N, Gl, 1.0, r, tol=1e-3)
        x = x + d
    assert hist[-1] <= 1e-10 and len(hist) <= 5
    factors = [hist[k + 1] / hist[k] for k in range(len(hist) - 1)]
    assert max(factors) <= 3e-3
