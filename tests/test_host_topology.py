"""The library's multi-patch topology (paper_1804_02539_gb300/csrc/topology.cpp: parsing, dof
identification across patches, Dirichlet elimination, the pieces of the additive smoother)
compiled into a small host program and compared with the oracle's space on every level:
the same dofs up to numbering (a bijection that keeps the eliminated nodes), and the same
partition into interior, face, edge and vertex pieces.  Host compiler only, no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads
from oracle import multipatch
from paper_1804_02539_gb300.igamg import Problem

from helpers import permutation

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_02539_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "topology.h"
using namespace igamg;
template <class T> static std::vector<T> rd(FILE* f, size_t n) {
  std::vector<T> v(n);
  for (auto& x : v) { double d; if (std::fscanf(f, "%lf", &d) != 1) throw 1; x = T(d); }
  return v;
}
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "r");
  int dim, K, levels;
  if (std::fscanf(f, "%d %d %d", &dim, &K, &levels) != 3) return 2;
  auto deg = rd<int>(f, K * dim);
  auto nk = rd<int>(f, K * dim);
  size_t total = 0;
  for (int v : nk) total += v;
  auto kn = rd<double>(f, total);
  auto ctrl = rd<double>(f, size_t(K) * (1 << dim) * dim);
  auto bc = rd<int>(f, size_t(K) * 2 * dim);
  std::vector<int> gd(K * dim, 1), gn(K * dim, 2);
  ProblemDesc pd;
  int code = 0;
  std::string e = parse_problem(dim, K, deg.data(), nk.data(), kn.data(), gd.data(), gn.data(), ctrl.data(),
                                bc.data(), levels, pd, &code);
  if (!e.empty()) { std::printf("error %s\n", e.c_str()); return 3; }
  for (int l = 0; l < levels; ++l) {
    LevelTopo t;
    e = build_level(pd, l, t, &code);
    if (!e.empty()) { std::printf("error %s\n", e.c_str()); return 4; }
    std::printf("level %d %lld %lld\n", l, (long long)t.N, (long long)t.T);
    std::printf("off");
    for (auto v : t.off) std::printf(" %lld", (long long)v);
    std::printf("\nn");
    for (auto v : t.n) std::printf(" %d", v);
    std::printf("\nl2g");
    for (auto v : t.l2g) std::printf(" %lld", (long long)v);
    std::printf("\n");
    for (const auto& in : t.interiors)
      std::printf("interior %d %d %d %d %d %d %d\n", in.k, in.lo[0], in.lo[1], in.lo[2], in.len[0], in.len[1],
                  in.len[2]);
    for (const auto& p : t.ifaces)
      std::printf("iface %d %d %d %d %d %lld\n", p.kind, p.k, p.ndir, p.len[0], p.len[1], (long long)p.first);
    std::printf("igid");
    for (auto v : t.iface_gid) std::printf(" %lld", (long long)v);
    std::printf("\n");
  }
  return 0;
}
"""

CASES = {
    "square_p2_m8": lambda: workloads.unit_square_quadrants(8, 2, 4),
    "grid3x3_p3_m16": lambda: workloads.perturbed_grid_2d(3, 3, 16, 4, 31),
    "grid2x2_p5_m32": lambda: workloads.perturbed_grid_2d(2, 5, 32, 3, 7),
    "single_patch_p2_m16": lambda: workloads.perturbed_grid_2d(1, 2, 16, 3, 3),
    "grid2x2_p1_m8": lambda: workloads.perturbed_grid_2d(2, 1, 8, 3, 5),
    "rect3x3_p3_m8_mixed_bc": lambda: workloads.perturbed_grid_2d(3, 3, 8, 3, 31, amp=0.0),
    "cube_p2_m4": lambda: workloads.perturbed_cube_3d(2, 2, 4, 3, 3),
    "cube_p3_m8": lambda: workloads.perturbed_cube_3d(2, 3, 8, 3, 3),
    "fichera_p2_m4": lambda: workloads.fichera_corner(1, 2, 4, 3),
    "cube_p4_m4_single": lambda: workloads.perturbed_cube_3d(1, 4, 4, 2, 5),
}


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("topology")
    (d / "driver.cpp").write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O2", "-fopenmp", "-I", CSRC, str(d / "driver.cpp"),
                    os.path.join(CSRC, "topology.cpp"), os.path.join(CSRC, "host_math.cpp"), "-o", str(exe)],
                   check=True)
    return d, exe


def run_driver(driver, pr, name):
    d, exe = driver
    P = Problem(pr)
    K, dim = np.asarray(pr.degree).shape
    vals = [f"{dim} {K} {int(pr.num_levels)}", " ".join(map(str, P._deg)), " ".join(map(str, P._nk)),
            " ".join(repr(float(v)) for v in P._kn), " ".join(repr(float(v)) for v in P._ctrl),
            " ".join(map(str, P._bc))]
    f = d / f"{name}.txt"
    f.write_text("\n".join(vals) + "\n")
    out = subprocess.run([str(exe), str(f)], check=True, capture_output=True, text=True).stdout
    levels = []
    for line in out.splitlines():
        w = line.split()
        if w[0] == "level":
            levels.append({"N": int(w[2]), "T": int(w[3]), "interiors": [], "ifaces": []})
        elif w[0] in ("off", "n", "l2g", "igid"):
            levels[-1][w[0]] = np.array([int(v) for v in w[1:]], dtype=np.int64)
        elif w[0] == "interior":
            levels[-1]["interiors"].append([int(v) for v in w[1:]])
        elif w[0] == "iface":
            levels[-1]["ifaces"].append([int(v) for v in w[1:]])
    return levels


@pytest.mark.parametrize("name", sorted(CASES))
def test_topology_matches_oracle(driver, name):
    pr = CASES[name]()
    levels = run_driver(driver, pr, name)
    K, dim = np.asarray(pr.degree).shape
    assert len(levels) == pr.num_levels
    for l, L in enumerate(levels):
        sp = multipatch.build_space(pr, l)
        assert L["N"] == sp.N and L["T"] == sum(a.size for a in sp.l2g)
        n = L["n"].reshape(K, dim)
        assert np.array_equal(n, np.asarray(sp.n)), (name, l)
        perm = permutation(sp, L["l2g"])  # oracle id -> library id, a bijection
        inv = np.empty_like(perm)
        inv[perm] = np.arange(sp.N)
        # library pieces as sets of oracle ids
        lib_pieces = []
        for k, lo0, lo1, lo2, n0, n1, n2 in L["interiors"]:
            lo, ln = [lo0, lo1, lo2][:dim], [n0, n1, n2][:dim]
            idx = np.ix_(*[np.arange(lo[j], lo[j] + ln[j]) for j in range(dim)])
            tile = L["l2g"][L["off"][k]:L["off"][k + 1]].reshape(tuple(n[k]))
            g = tile[idx].ravel()
            assert np.all(g >= 0)
            lib_pieces.append(("interior", frozenset(inv[g].tolist())))
        kinds = {0: "vertex", 1: "edge", 2: "face"}
        for kind, k, ndir, a, b, first in L["ifaces"]:
            cnt = 1 if ndir == 0 else (a if ndir == 1 else a * b)
            g = L["igid"][first:first + cnt]
            lib_pieces.append((kinds[kind], frozenset(inv[g].tolist())))
        ora_pieces = [(pc.kind, frozenset(np.asarray(pc.ids).ravel().tolist())) for pc in sp.pieces]
        assert sorted(map(len, (s for _, s in lib_pieces))) == sorted(map(len, (s for _, s in ora_pieces)))
        assert set(lib_pieces) == set(ora_pieces), (name, l)
        # the pieces partition the dofs
        allids = np.concatenate([np.fromiter(s, dtype=np.int64) for _, s in lib_pieces])
        assert np.array_equal(np.sort(allids), np.arange(sp.N))
