// Host-side FP64 numerics used during setup: univariate splines (Sec. 2), Gauss rules,
// the univariate mass/stiffness matrices and knot-insertion transfers (Sec. 3), dense
// Cholesky / LU / symmetric eigensolvers for the piece-local smoothers and the coarse
// solver.  All matrices are dense row-major std::vector<double>.
#pragma once
#include <vector>

namespace igamg {

using Mat = std::vector<double>;  // row-major

// Open uniform knot vector with m intervals on [0,1] (p+1 repeated end knots).
std::vector<double> uniform_knots(int m, int p);
// Recognises an open uniform knot vector; returns m, or -1.
int uniform_intervals(const double* t, int num_knots, int p);

// Index `span` with t[span] <= x < t[span+1] (x = 1 maps to the last non-empty interval).
int find_span(const std::vector<double>& t, int p, double x);
// d^r/dx^r of the p+1 B-splines that do not vanish on `span`, r = 0..nd:
// out[r*(p+1) + j] = D^r B_{span-p+j}(x).
void nonzero_basis(const std::vector<double>& t, int p, int span, double x, int nd, double* out);

// nq-point Gauss-Legendre rule on [0,1] (Newton iteration on the Legendre polynomial).
void gauss_legendre(int nq, double* x, double* w);

// Univariate mass and stiffness matrices (n x n, n = m+p) on the open uniform knots.
void mass_stiffness_1d(int m, int p, Mat& M, Mat& K);

// Canonical embedding S_{p,1/mc} -> S_{p,1/(2mc)}: matrix (2mc+p) x (mc+p) obtained by
// interpolating the coarse B-splines at the fine Greville abscissae.
Mat prolongation_1d(int mc, int p);

// Threads the dense routines below may use when called from the current thread
// (OpenMP team size; 1 inside a pool of setup workers; n <= 0: every core).
void set_host_threads(int n);

// Dense linear algebra.
bool cholesky(int n, Mat& A);                               // A = L L^T, L in lower part
void cholesky_solve(int n, const Mat& L, double* b);         // in place
void cholesky_solve_many(int n, const Mat& L, Mat& B, int ncols);  // B n x ncols
bool lu_solve(int n, Mat A, Mat& B, int ncols);              // A X = B, partial pivoting
// Symmetric eigen-decomposition by cyclic Jacobi: A = V diag(lam) V^T (columns of V).
bool jacobi_eigen(int n, Mat A, std::vector<double>& lam, Mat& V);
// Generalised symmetric-definite K u = lam M u with U^T M U = I (columns of U).
bool generalized_eigen(int n, const Mat& K, const Mat& M, std::vector<double>& lam, Mat& U);

Mat submatrix(const Mat& A, int n, const std::vector<int>& idx);
Mat matmul(const Mat& A, const Mat& B, int m, int k, int n, bool ta = false, bool tb = false);

}  // namespace igamg
