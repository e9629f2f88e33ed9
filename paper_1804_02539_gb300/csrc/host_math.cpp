#include "host_math.h"

#include <omp.h>

#include <algorithm>
#include <cmath>

namespace igamg {

void set_host_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }


std::vector<double> uniform_knots(int m, int p) {
  std::vector<double> t;
  t.reserve(m + 2 * p + 1);
  for (int i = 0; i <= p; ++i) t.push_back(0.0);
  for (int i = 1; i < m; ++i) t.push_back(double(i) / m);
  for (int i = 0; i <= p; ++i) t.push_back(1.0);
  return t;
}

int uniform_intervals(const double* t, int num_knots, int p) {
  int m = num_knots - 2 * p - 1;
  if (m < 1) return -1;
  std::vector<double> u = uniform_knots(m, p);
  for (int i = 0; i < num_knots; ++i)
    if (std::fabs(u[i] - t[i]) > 1e-14) return -1;
  return m;
}

int find_span(const std::vector<double>& t, int p, double x) {
  int n = int(t.size()) - p - 1;
  if (x >= t[n]) return n - 1;  // right end belongs to the last non-empty interval
  int lo = p, hi = n;           // t[lo] <= x < t[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// Degree-by-degree table of the functions that live on `span`; values first, then the
// derivative recursion D B_{i,k} = k (B_{i,k-1}/(t_{i+k}-t_i) - B_{i+1,k-1}/(t_{i+k+1}-t_{i+1})).
void nonzero_basis(const std::vector<double>& t, int p, int span, double x, int nd, double* out) {
  // vals[k] holds B_{span-k+j, k}(x), j = 0..k
  std::vector<std::vector<double>> vals(p + 1);
  vals[0] = {1.0};
  for (int k = 1; k <= p; ++k) {
    vals[k].assign(k + 1, 0.0);
    for (int j = 0; j <= k; ++j) {
      int i = span - k + j;
      double v = 0.0;
      if (j > 0) {
        double d1 = t[i + k] - t[i];
        if (d1 > 0) v += (x - t[i]) / d1 * vals[k - 1][j - 1];
      }
      if (j < k) {
        double d2 = t[i + k + 1] - t[i + 1];
        if (d2 > 0) v += (t[i + k + 1] - x) / d2 * vals[k - 1][j];
      }
      vals[k][j] = v;
    }
  }
  for (int r = 0; r <= nd; ++r) {
    if (r > p) {
      for (int j = 0; j <= p; ++j) out[r * (p + 1) + j] = 0.0;
      continue;
    }
    std::vector<double> cur = vals[p - r];
    for (int k = p - r + 1; k <= p; ++k) {
      std::vector<double> nxt(k + 1, 0.0);
      for (int j = 0; j <= k; ++j) {
        int i = span - k + j;
        double v = 0.0;
        if (j > 0) {
          double d1 = t[i + k] - t[i];
          if (d1 > 0) v += k / d1 * cur[j - 1];
        }
        if (j < k) {
          double d2 = t[i + k + 1] - t[i + 1];
          if (d2 > 0) v -= k / d2 * cur[j];
        }
        nxt[j] = v;
      }
      cur.swap(nxt);
    }
    for (int j = 0; j <= p; ++j) out[r * (p + 1) + j] = cur[j];
  }
}

void gauss_legendre(int nq, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < nq; ++i) {
    double z = std::cos(pi * (i + 0.75) / (nq + 0.5));  // initial guess for root i
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // Legendre three-term recurrence
      for (int k = 2; k <= nq; ++k) {
        double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (nq == 1) { p1 = z; p0 = 1.0; }
      dp = nq * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= nq; ++k) {
        double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (nq == 1) { p1 = z; p0 = 1.0; }
      dp = nq * (z * p1 - p0) / (z * z - 1.0);
    }
    x[nq - 1 - i] = 0.5 * (1.0 + z);
    w[nq - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) scaled by 1/2
  }
}

void mass_stiffness_1d(int m, int p, Mat& M, Mat& K) {
  int n = m + p, nq = p + 1;
  M.assign(size_t(n) * n, 0.0);
  K.assign(size_t(n) * n, 0.0);
  std::vector<double> t = uniform_knots(m, p), xq(nq), wq(nq), d(2 * (p + 1));
  gauss_legendre(nq, xq.data(), wq.data());
  for (int e = 0; e < m; ++e) {
    double a = double(e) / m, h = 1.0 / m;
    for (int q = 0; q < nq; ++q) {
      double x = a + h * xq[q], w = h * wq[q];
      int span = p + e;
      nonzero_basis(t, p, span, x, 1, d.data());
      for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) {
          M[size_t(e + i) * n + (e + j)] += w * d[i] * d[j];
          K[size_t(e + i) * n + (e + j)] += w * d[p + 1 + i] * d[p + 1 + j];
        }
    }
  }
}

Mat prolongation_1d(int mc, int p) {
  int nc = mc + p, mf = 2 * mc, nf = mf + p;
  std::vector<double> tc = uniform_knots(mc, p), tf = uniform_knots(mf, p);
  Mat Bf(size_t(nf) * nf, 0.0), Bc(size_t(nf) * nc, 0.0);
  std::vector<double> d(p + 1);
  for (int i = 0; i < nf; ++i) {
    double g = 0.0;  // Greville abscissa of fine basis function i
    for (int k = 1; k <= p; ++k) g += tf[i + k];
    g /= p;
    int sf = find_span(tf, p, g), sc = find_span(tc, p, g);
    nonzero_basis(tf, p, sf, g, 0, d.data());
    for (int j = 0; j <= p; ++j) Bf[size_t(i) * nf + sf - p + j] = d[j];
    nonzero_basis(tc, p, sc, g, 0, d.data());
    for (int j = 0; j <= p; ++j) Bc[size_t(i) * nc + sc - p + j] = d[j];
  }
  lu_solve(nf, Bf, Bc, nc);
  for (double& v : Bc)
    if (std::fabs(v) < 1e-15) v = 0.0;  // exact zeros outside the stencil
  return Bc;
}

bool cholesky(int n, Mat& A) {
  // right-looking column Cholesky; the update of the trailing rows is parallel
  for (int j = 0; j < n; ++j) {
    const double diag = A[size_t(j) * n + j];
    double s = diag;
    for (int k = 0; k < j; ++k) s -= A[size_t(j) * n + k] * A[size_t(j) * n + k];
    if (!(s > 1e-13 * diag)) return false;  // not positive definite to working accuracy
    double ljj = std::sqrt(s);
    A[size_t(j) * n + j] = ljj;
    const double* rj = &A[size_t(j) * n];
#pragma omp parallel for schedule(static) if (n - j > 256)
    for (int i = j + 1; i < n; ++i) {
      double* ri = &A[size_t(i) * n];
      double v = ri[j];
      for (int k = 0; k < j; ++k) v -= ri[k] * rj[k];
      ri[j] = v / ljj;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[size_t(i) * n + j] = 0.0;
  return true;
}

void cholesky_solve(int n, const Mat& L, double* b) {
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    const double* ri = &L[size_t(i) * n];
    for (int k = 0; k < i; ++k) v -= ri[k] * b[k];
    b[i] = v / ri[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < n; ++k) v -= L[size_t(k) * n + i] * b[k];
    b[i] = v / L[size_t(i) * n + i];
  }
}

void cholesky_solve_many(int n, const Mat& L, Mat& B, int ncols) {
  // independent right-hand sides in parallel; the back substitution uses L^T stored by rows
  Mat LT(size_t(n) * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k <= i; ++k) LT[size_t(k) * n + i] = L[size_t(i) * n + k];
#pragma omp parallel
  {
    std::vector<double> col(n);
#pragma omp for schedule(dynamic, 8)
    for (int c = 0; c < ncols; ++c) {
      for (int i = 0; i < n; ++i) col[i] = B[size_t(i) * ncols + c];
      for (int i = 0; i < n; ++i) {
        double v = col[i];
        const double* ri = &L[size_t(i) * n];
        for (int k = 0; k < i; ++k) v -= ri[k] * col[k];
        col[i] = v / ri[i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double v = col[i];
        const double* ri = &LT[size_t(i) * n];
        for (int k = i + 1; k < n; ++k) v -= ri[k] * col[k];
        col[i] = v / ri[i];
      }
      for (int i = 0; i < n; ++i) B[size_t(i) * ncols + c] = col[i];
    }
  }
}

bool lu_solve(int n, Mat A, Mat& B, int ncols) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int r = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[size_t(i) * n + k]) > std::fabs(A[size_t(r) * n + k])) r = i;
    if (A[size_t(r) * n + k] == 0.0) return false;
    if (r != k) {
      for (int j = 0; j < n; ++j) std::swap(A[size_t(k) * n + j], A[size_t(r) * n + j]);
      for (int j = 0; j < ncols; ++j) std::swap(B[size_t(k) * ncols + j], B[size_t(r) * ncols + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[size_t(i) * n + k] / A[size_t(k) * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[size_t(i) * n + j] -= f * A[size_t(k) * n + j];
      for (int j = 0; j < ncols; ++j) B[size_t(i) * ncols + j] -= f * B[size_t(k) * ncols + j];
    }
  }
  for (int i = n - 1; i >= 0; --i)
    for (int j = 0; j < ncols; ++j) {
      double v = B[size_t(i) * ncols + j];
      for (int k = i + 1; k < n; ++k) v -= A[size_t(i) * n + k] * B[size_t(k) * ncols + j];
      B[size_t(i) * ncols + j] = v / A[size_t(i) * n + i];
    }
  return true;
}

bool jacobi_eigen(int n, Mat A, std::vector<double>& lam, Mat& V) {
  V.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  lam.assign(n, 0.0);
  if (n == 0) return true;
  double scale = 0.0;
  for (double v : A) scale = std::max(scale, std::fabs(v));
  if (scale == 0.0) return true;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[size_t(i) * n + j] * A[size_t(i) * n + j];
    if (std::sqrt(off) <= 1e-17 * scale * n) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[size_t(p) * n + q];
        if (std::fabs(apq) <= 1e-300) continue;
        double app = A[size_t(p) * n + p], aqq = A[size_t(q) * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < n; ++k) {  // rotate columns p, q
          double akp = A[size_t(k) * n + p], akq = A[size_t(k) * n + q];
          A[size_t(k) * n + p] = c * akp - s * akq;
          A[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rotate rows p, q
          double apk = A[size_t(p) * n + k], aqk = A[size_t(q) * n + k];
          A[size_t(p) * n + k] = c * apk - s * aqk;
          A[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
          V[size_t(k) * n + p] = c * vkp - s * vkq;
          V[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[size_t(i) * n + i];
  for (double l : lam)
    if (!std::isfinite(l)) return false;
  return true;
}

bool generalized_eigen(int n, const Mat& K, const Mat& M, std::vector<double>& lam, Mat& U) {
  Mat L = M;
  if (!cholesky(n, L)) return false;
  // C = L^{-1} K L^{-T}
  Mat C = K;
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {  // X = L^{-1} K (column by column)
    for (int i = 0; i < n; ++i) {
      double v = C[size_t(i) * n + c];
      for (int k = 0; k < i; ++k) v -= L[size_t(i) * n + k] * C[size_t(k) * n + c];
      C[size_t(i) * n + c] = v / L[size_t(i) * n + i];
    }
  }
  for (int r = 0; r < n; ++r) {  // C = X L^{-T}: solve L y = X[r,:]^T
    for (int i = 0; i < n; ++i) {
      double v = C[size_t(r) * n + i];
      for (int k = 0; k < i; ++k) v -= L[size_t(i) * n + k] * C[size_t(r) * n + k];
      C[size_t(r) * n + i] = v / L[size_t(i) * n + i];
    }
  }
  for (int i = 0; i < n; ++i)  // symmetrise against rounding
    for (int j = i + 1; j < n; ++j) {
      double a = 0.5 * (C[size_t(i) * n + j] + C[size_t(j) * n + i]);
      C[size_t(i) * n + j] = C[size_t(j) * n + i] = a;
    }
  Mat V;
  if (!jacobi_eigen(n, C, lam, V)) return false;
  // U = L^{-T} V
  U = V;
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double v = U[size_t(i) * n + c];
      for (int k = i + 1; k < n; ++k) v -= L[size_t(k) * n + i] * U[size_t(k) * n + c];
      U[size_t(i) * n + c] = v / L[size_t(i) * n + i];
    }
  return true;
}

Mat submatrix(const Mat& A, int n, const std::vector<int>& idx) {
  int s = int(idx.size());
  Mat B(size_t(s) * s);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) B[size_t(i) * s + j] = A[size_t(idx[i]) * n + idx[j]];
  return B;
}

Mat matmul(const Mat& A, const Mat& B, int m, int k, int n, bool ta, bool tb) {
  Mat C(size_t(m) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      double a = ta ? A[size_t(l) * m + i] : A[size_t(i) * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[size_t(i) * n + j] += a * (tb ? B[size_t(j) * k + l] : B[size_t(l) * n + j]);
    }
  return C;
}

}  // namespace igamg
