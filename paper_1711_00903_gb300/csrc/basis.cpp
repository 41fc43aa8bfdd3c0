// Host FP64 basis of degree N (Section 2, Table of notation; Section 4):
// GLL and Gauss-Legendre rules, the interpolation matrix I and the
// differentiation matrices D (GLL) and Dt (Gauss).
//
// Route: nodes are eigenvalues of the symmetric tridiagonal Jacobi matrices
// of the Legendre (Gauss) and Jacobi(1,1) (GLL interior) polynomials
// (Golub & Welsch, Math. Comp. 23, 1969), found by Sturm-sequence bisection
// and polished by one Newton step on the orthonormal three-term recurrence.
// Gauss weights are the reciprocal Christoffel function 1 / sum_k p_k(x)^2 of
// the orthonormal Legendre polynomials; GLL weights solve the moment
// equations sum_j w_j P_k(x_j) = 2 delta_k0 (k = 0..N).  I, D and Dt use the
// barycentric Lagrange formulas (Berrut & Trefethen, SIAM Review 46, 2004).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "fem_internal.h"

namespace fem {
namespace {

// Number of eigenvalues below x of the M x M symmetric tridiagonal matrix
// with zero diagonal and off-diagonal b[1..M-1] (Sturm count of the LDL^T
// pivots).
int sturm_count(int M, const double *b, double x) {
    int cnt = 0;
    double d = -x;
    if (d < 0) cnt++;
    for (int k = 1; k < M; k++) {
        if (d == 0.0) d = 1e-300;
        d = -x - b[k] * b[k] / d;
        if (d < 0) cnt++;
    }
    return cnt;
}

// Ascending eigenvalues of that matrix, all inside (-1, 1).
void jacobi_eigenvalues(int M, const double *b, double *x) {
    for (int j = 0; j < M; j++) {
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(M, b, mid) > j)
                hi = mid;
            else
                lo = mid;
        }
        x[j] = 0.5 * (lo + hi);
    }
}

// Orthonormal polynomial p_M and its derivative from the recurrence
// x p_k = b_{k+1} p_{k+1} + b_k p_{k-1}, p_{-1} = 0, p_0 = 1.
void ortho_eval(int M, const double *b, double x, double *p, double *dp) {
    double pm = 0.0, pc = 1.0, dpm = 0.0, dpc = 0.0;
    for (int k = 0; k < M; k++) {
        double bk = (k == 0) ? 0.0 : b[k];
        double pn = (x * pc - bk * pm) / b[k + 1];
        double dpn = (pc + x * dpc - bk * dpm) / b[k + 1];
        pm = pc;
        pc = pn;
        dpm = dpc;
        dpc = dpn;
    }
    *p = pc;
    *dp = dpc;
}

void polish(int M, const double *b, double *x) {
    for (int j = 0; j < M; j++) {
        double p, dp;
        ortho_eval(M, b, x[j], &p, &dp);
        if (dp != 0.0) {
            double nx = x[j] - p / dp;
            if (std::fabs(nx - x[j]) < 1e-14) x[j] = nx;
        }
    }
    for (int j = 0; j < M / 2; j++) {  // enforce the mirror symmetry
        double s = 0.5 * (x[M - 1 - j] - x[j]);
        x[j] = -s;
        x[M - 1 - j] = s;
    }
    if (M % 2) x[M / 2] = 0.0;
}

// m-point Gauss-Legendre rule.
void gauss_rule(int m, double *x, double *w) {
    double b[kMaxQ + 2];
    for (int k = 1; k <= m; k++) b[k] = k / std::sqrt(4.0 * k * k - 1.0);
    jacobi_eigenvalues(m, b, x);
    polish(m, b, x);
    for (int j = 0; j < m; j++) {
        // Christoffel function of the orthonormal Legendre polynomials
        // phat_k = sqrt(k + 1/2) P_k.
        double pm = 0.0, pc = 1.0 / std::sqrt(2.0), s = pc * pc;
        for (int k = 0; k < m - 1; k++) {
            double bk = (k == 0) ? 0.0 : b[k];
            double pn = (x[j] * pc - bk * pm) / b[k + 1];
            pm = pc;
            pc = pn;
            s += pc * pc;
        }
        w[j] = 1.0 / s;
    }
}

// Solves A y = rhs (n x n, row-major, destroyed) by Gaussian elimination
// with partial pivoting.
void solve_dense(int n, double *A, double *rhs) {
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++)
            if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
        if (p != c) {
            for (int k = 0; k < n; k++) std::swap(A[c * n + k], A[p * n + k]);
            std::swap(rhs[c], rhs[p]);
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = n - 1; c >= 0; c--) {
        double s = rhs[c];
        for (int k = c + 1; k < n; k++) s -= A[c * n + k] * rhs[k];
        rhs[c] = s / A[c * n + c];
    }
}

// N+1 point Gauss-Lobatto-Legendre rule.
void gll_rule(int N, double *x, double *w) {
    int n = N + 1;
    x[0] = -1.0;
    x[N] = 1.0;
    if (N >= 2) {
        // interior nodes: zeros of the Jacobi(1,1) polynomial of degree N-1
        double b[kMaxQ + 2];
        for (int k = 1; k <= N - 1; k++)
            b[k] = std::sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
        jacobi_eigenvalues(N - 1, b, x + 1);
        polish(N - 1, b, x + 1);
    }
    // moments: sum_j w_j P_k(x_j) = integral of P_k = 2 delta_k0
    double A[kMaxQ * kMaxQ];
    for (int j = 0; j < n; j++) {
        double pm = 0.0, pc = 1.0;
        for (int k = 0; k < n; k++) {
            A[k * n + j] = pc;
            double pn = ((2.0 * k + 1.0) * x[j] * pc - k * pm) / (k + 1.0);
            pm = pc;
            pc = pn;
        }
    }
    for (int k = 0; k < n; k++) w[k] = (k == 0) ? 2.0 : 0.0;
    solve_dense(n, A, w);
    for (int j = 0; j < n / 2; j++) {
        double s = 0.5 * (w[j] + w[n - 1 - j]);
        w[j] = w[n - 1 - j] = s;
    }
}

void bary_weights(int n, const double *x, double *lam) {
    for (int j = 0; j < n; j++) {
        double p = 1.0;
        for (int k = 0; k < n; k++)
            if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
}

// Rows: evaluation points y (ny); columns: Lagrange basis on x (nx).
void bary_interp(int nx, const double *x, int ny, const double *y, double *out) {
    double lam[kMaxQ];
    bary_weights(nx, x, lam);
    for (int a = 0; a < ny; a++) {
        int hit = -1;
        for (int i = 0; i < nx; i++)
            if (y[a] == x[i]) hit = i;
        if (hit >= 0) {
            for (int i = 0; i < nx; i++) out[a * nx + i] = (i == hit) ? 1.0 : 0.0;
            continue;
        }
        double den = 0.0;
        for (int i = 0; i < nx; i++) den += lam[i] / (y[a] - x[i]);
        for (int i = 0; i < nx; i++) out[a * nx + i] = (lam[i] / (y[a] - x[i])) / den;
    }
}

// Collocation differentiation matrix on the nodes x (n x n).
void bary_diff(int n, const double *x, double *Dm) {
    double lam[kMaxQ];
    bary_weights(n, x, lam);
    for (int i = 0; i < n; i++) {
        double diag = 0.0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (x[i] - x[j]);
            Dm[i * n + j] = v;
            diag -= v;
        }
        Dm[i * n + i] = diag;
    }
}

}  // namespace

bool compute_basis(int N, HostBasis *hb) {
    if (N < 1 || N > kMaxN || !hb) return false;
    std::memset(hb, 0, sizeof(*hb));
    hb->N = N;
    hb->n = N + 1;
    hb->m = N + 2;
    gll_rule(N, hb->r, hb->w);
    gauss_rule(hb->m, hb->rt, hb->wt);
    bary_interp(hb->n, hb->r, hb->m, hb->rt, hb->I);
    bary_diff(hb->n, hb->r, hb->D);
    bary_diff(hb->m, hb->rt, hb->Dt);
    return true;
}

}  // namespace fem

// ---------------------------------------------------------------------------
// Folded operator table (see eo.cuh).
#include "fold_layout.h"

namespace fem {

void build_fold_block(int N, const double *I, const double *D, const double *Dt, double *out) {
    const int n = N + 1, m = N + 2;
    double IT[kMaxQ * kMaxQ], DT[kMaxQ * kMaxQ], DtT[kMaxQ * kMaxQ];
    for (int a = 0; a < m; a++)
        for (int i = 0; i < n; i++) IT[i * m + a] = I[a * n + i];
    for (int a = 0; a < n; a++)
        for (int i = 0; i < n; i++) DT[i * n + a] = D[a * n + i];
    for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) DtT[b * m + a] = Dt[a * m + b];
    const double *ops[kFoldCount] = {I, IT, D, DT, Dt, DtT};
    double *p = out;
    for (int op = 0; op < kFoldCount; op++) {
        const int P = fold_rows(op, n, m), Q = fold_cols(op, n, m);
        fold_matrix(P, Q, ops[op], p);
        p += fold_size(P, Q);
    }
}

}  // namespace fem

namespace fem {

const double *fold_table() {
    static std::vector<double> table;
    static std::once_flag once;
    std::call_once(once, [] {
        table.assign(kFoldTotal, 0.0);
        for (int N = 1; N <= kMaxN; N++) {
            HostBasis hb;
            compute_basis(N, &hb);
            build_fold_block(N, hb.I, hb.D, hb.Dt, table.data() + fold_degree_offset(N));
        }
    });
    return table.data();
}

}  // namespace fem
