"""The library's host-side setup numerics (paper_1804_02539_gb300/csrc/host_math.cpp: Gauss
rules, B-spline values and derivatives, univariate mass/stiffness, the two-grid embedding,
dense Cholesky / LU / eigensolvers) compiled into a small host program and compared with
the oracle and with NumPy/SciPy.  Host compiler only, no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

from oracle import bspline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_02539_gb300", "csrc")

CASES_MP = [(1, 1), (4, 2), (8, 3), (5, 4), (16, 5), (3, 6)]
XS = [0.0, 0.03, 0.2, 0.25, 0.5, 0.61, 0.999, 1.0]

DRIVER = r"""
#include <cstdio>
#include <string>
#include <vector>
#include "host_math.h"
using namespace igamg;
static void pr(const std::string& key, const std::vector<double>& v) {
  std::printf("%s", key.c_str());
  for (double x : v) std::printf(" %.17g", x);
  std::printf("\n");
}
int main() {
  for (int nq = 1; nq <= 10; ++nq) {
    std::vector<double> x(nq), w(nq);
    gauss_legendre(nq, x.data(), w.data());
    pr("gx " + std::to_string(nq), x);
    pr("gw " + std::to_string(nq), w);
  }
  const int mp[][2] = {%CASES%};
  const double xs[] = {%XS%};
  for (const auto& c : mp) {
    const int m = c[0], p = c[1], n = m + p;
    const std::string tag = std::to_string(m) + "_" + std::to_string(p);
    std::vector<double> t = uniform_knots(m, p);
    pr("knots " + tag, t);
    for (double x : xs) {
      const int span = find_span(t, p, x);
      std::vector<double> out(3 * (p + 1));
      nonzero_basis(t, p, span, x, 2, out.data());
      out.insert(out.begin(), double(span));
      pr("basis " + tag + " " + std::to_string(x), out);
    }
    Mat M, K;
    mass_stiffness_1d(m, p, M, K);
    pr("mass " + tag, M);
    pr("stiff " + tag, K);
    pr("prol " + tag, prolongation_1d(m, p));
    std::vector<double> lam;
    Mat U;
    if (generalized_eigen(n, K, M, lam, U)) {
      pr("glam " + tag, lam);
      pr("gvec " + tag, U);
    }
    Mat L = M;
    if (cholesky(n, L)) {
      std::vector<double> b(n);
      for (int i = 0; i < n; ++i) b[i] = 1.0 + 0.5 * i;
      cholesky_solve(n, L, b.data());
      pr("chol " + tag, b);
    }
    Mat A = K, B(n);
    for (int i = 0; i < n; ++i) { A[i * n + i] += 1.0 + 0.1 * i; A[i * n + (n - 1 - i)] += 0.3; B[i] = 1.0 - 0.2 * i; }
    if (lu_solve(n, A, B, 1)) pr("lu " + tag, B);
    std::vector<double> jl;
    Mat V;
    if (jacobi_eigen(n, M, jl, V)) pr("jlam " + tag, jl);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def host_out(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("host_math")
    src = DRIVER.replace("%CASES%", ", ".join("{%d, %d}" % c for c in CASES_MP))
    src = src.replace("%XS%", ", ".join(repr(x) for x in XS))
    (d / "driver.cpp").write_text(src)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, str(d / "driver.cpp"),
                    os.path.join(CSRC, "host_math.cpp"), "-o", str(exe)], check=True)
    out = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        parts = line.split()
        nkey = 3 if parts[0] == "basis" else 2
        out[" ".join(parts[:nkey])] = np.array([float(v) for v in parts[nkey:]])
    return out


def test_gauss_rules(host_out):
    for nq in range(1, 11):
        x, w = bspline.gauss_legendre(nq)
        np.testing.assert_allclose(host_out[f"gx {nq}"], x, rtol=0, atol=2e-15)
        np.testing.assert_allclose(host_out[f"gw {nq}"], w, rtol=0, atol=2e-15)


def test_knots_and_basis_derivatives(host_out):
    for m, p in CASES_MP:
        t = bspline.uniform_knots(m, p)
        np.testing.assert_array_equal(host_out[f"knots {m}_{p}"], t)
        for x in XS:
            v = host_out[f"basis {m}_{p} {x:f}"]
            span = int(v[0])
            vals = v[1:].reshape(3, p + 1)
            for r in range(min(2, p) + 1):
                full = bspline.basis(t, p, [x], r)[0]
                ref = full[span - p:span + 1]
                scale = max(1.0, np.abs(full).max())
                np.testing.assert_allclose(vals[r], ref, rtol=0, atol=1e-12 * scale, err_msg=f"{m},{p},{x},{r}")
                # every other B-spline vanishes there
                rest = np.delete(full, np.arange(span - p, span + 1))
                assert np.all(rest == 0)


def test_mass_stiffness_and_embedding(host_out):
    for m, p in CASES_MP:
        n = m + p
        M, K = bspline.mass_stiffness_1d(bspline.uniform_knots(m, p), p)
        np.testing.assert_allclose(host_out[f"mass {m}_{p}"].reshape(n, n), M, rtol=0, atol=1e-15)
        np.testing.assert_allclose(host_out[f"stiff {m}_{p}"].reshape(n, n), K, rtol=0, atol=1e-11 * np.abs(K).max())
        P = host_out[f"prol {m}_{p}"].reshape(2 * m + p, n)
        np.testing.assert_allclose(P, bspline.prolongation_1d(m, p), rtol=0, atol=1e-13)


def test_dense_solvers(host_out):
    for m, p in CASES_MP:
        n = m + p
        M, K = bspline.mass_stiffness_1d(bspline.uniform_knots(m, p), p)
        # generalised eigenproblem K u = lam M u, U^T M U = I
        lam = host_out[f"glam {m}_{p}"]
        U = host_out[f"gvec {m}_{p}"].reshape(n, n)
        ref = scipy.linalg.eigh(K, M, eigvals_only=True)
        np.testing.assert_allclose(np.sort(lam), ref, rtol=1e-10, atol=1e-9 * ref.max())
        np.testing.assert_allclose(U.T @ M @ U, np.eye(n), rtol=0, atol=1e-10)
        np.testing.assert_allclose(K @ U, M @ U * lam[None, :], rtol=0, atol=1e-8 * np.abs(K).max())
        b = 1.0 + 0.5 * np.arange(n)
        np.testing.assert_allclose(host_out[f"chol {m}_{p}"], np.linalg.solve(M, b), rtol=1e-9)
        A = K.copy()
        for i in range(n):
            A[i, i] += 1.0 + 0.1 * i
            A[i, n - 1 - i] += 0.3
        np.testing.assert_allclose(host_out[f"lu {m}_{p}"], np.linalg.solve(A, 1.0 - 0.2 * np.arange(n)),
                                   rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(np.sort(host_out[f"jlam {m}_{p}"]), np.linalg.eigvalsh(M), rtol=1e-10,
                                   atol=1e-15)
