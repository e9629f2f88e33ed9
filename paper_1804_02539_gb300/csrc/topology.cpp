#include "topology.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>

#include "host_math.h"

namespace igamg {

namespace {
const int ERR_ARG = 1, ERR_GEOMETRY = 2, ERR_UNSUPPORTED = 3;

std::string fail(int* code, int c, const std::string& msg) {
  *code = c;
  return msg;
}

// Local corners (c = sum_j c_j 2^j) of the cube entity whose fixed directions sit at the
// given ends; fixed_mask bit j set = direction j fixed at end bit j of fixed_end.
void entity_corners(int dim, int fixed_mask, int fixed_end, std::vector<int>& out) {
  out.clear();
  for (int c = 0; c < (1 << dim); ++c)
    if ((c & fixed_mask) == (fixed_end & fixed_mask)) out.push_back(c);
}

double det_jacobian(int dim, const double* cr, const double* xi) {
  double J[3][3] = {{0}};
  for (int c = 0; c < (1 << dim); ++c)
    for (int j = 0; j < dim; ++j) {
      double w = ((c >> j) & 1) ? 1.0 : -1.0;
      for (int i = 0; i < dim; ++i)
        if (i != j) w *= ((c >> i) & 1) ? xi[i] : 1.0 - xi[i];
      for (int a = 0; a < dim; ++a) J[a][j] += w * cr[c * dim + a];
    }
  if (dim == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}
}  // namespace

std::string parse_problem(int dim, int K, const int* degree, const int* num_knots,
                          const double* knots, const int* geo_degree, const int* geo_num_ctrl,
                          const double* geo_ctrl, const int* side_bc, int num_levels,
                          ProblemDesc& pd, int* code) {
  *code = 0;
  if (dim != 2 && dim != 3) return fail(code, ERR_ARG, "dim must be 2 or 3");
  if (K < 1) return fail(code, ERR_ARG, "num_patches must be >= 1");
  if (num_levels < 1 || num_levels > 20) return fail(code, ERR_ARG, "num_levels out of range");
  if (!degree || !num_knots || !knots || !geo_degree || !geo_num_ctrl || !geo_ctrl || !side_bc)
    return fail(code, ERR_ARG, "NULL array in problem");
  pd = ProblemDesc();
  pd.dim = dim;
  pd.K = K;
  pd.levels = num_levels;
  pd.p.assign(degree, degree + K * dim);
  pd.m.assign(K * dim, 0);
  const double* t = knots;
  for (int i = 0; i < K * dim; ++i) {
    int p = degree[i];
    if (p < 1 || p > 12) return fail(code, ERR_UNSUPPORTED, "degree must be in 1..12");
    if (geo_degree[i] != 1 || geo_num_ctrl[i] != 2)
      return fail(code, ERR_UNSUPPORTED, "only multilinear geometry maps are supported");
    int m = uniform_intervals(t, num_knots[i], p);
    if (m < 1) return fail(code, ERR_UNSUPPORTED, "knot vectors must be open uniform on [0,1]");
    if (m % (1 << (num_levels - 1)))
      return fail(code, ERR_ARG, "finest intervals must be divisible by 2^(num_levels-1)");
    pd.m[i] = m;
    t += num_knots[i];
  }
  int nc = 1 << dim;
  pd.corners.assign(geo_ctrl, geo_ctrl + size_t(K) * nc * dim);
  pd.side_bc.assign(side_bc, side_bc + K * 2 * dim);
  for (int v : pd.side_bc)
    if (v < 0 || v > 2) return fail(code, ERR_ARG, "side tag out of range");
  // bijectivity check: det J of one sign at the corners and the centre
  for (int k = 0; k < K; ++k) {
    double sgn = 0;
    for (int c = 0; c <= nc; ++c) {
      double xi[3];
      for (int j = 0; j < dim; ++j) xi[j] = c < nc ? double((c >> j) & 1) : 0.5;
      double d = det_jacobian(dim, &pd.corners[size_t(k) * nc * dim], xi);
      if (!std::isfinite(d) || d == 0.0 || (sgn != 0 && d * sgn < 0))
        return fail(code, ERR_GEOMETRY, "geometry map of patch " + std::to_string(k) + " is not bijective");
      sgn = d;
    }
  }
  // global vertex ids by coordinate matching
  double scale = 1.0;
  for (double v : pd.corners) scale = std::max(scale, std::fabs(v));
  double tol = 1e-9 * scale;
  std::vector<int> rep;  // representative corner index of every vertex id
  pd.vid.assign(K * nc, -1);
  for (int i = 0; i < K * nc; ++i) {
    const double* x = &pd.corners[size_t(i) * dim];
    int found = -1;
    for (size_t r = 0; r < rep.size() && found < 0; ++r) {
      const double* y = &pd.corners[size_t(rep[r]) * dim];
      bool same = true;
      for (int a = 0; a < dim; ++a) same = same && std::fabs(x[a] - y[a]) <= tol;
      if (same) found = int(r);
    }
    if (found < 0) {
      found = int(rep.size());
      rep.push_back(i);
    }
    pd.vid[i] = found;
  }
  // sides: interface if another patch has the same corner set
  std::map<std::vector<int>, std::vector<int>> sides;  // sorted vids -> k*2dim+s
  std::vector<int> cs;
  for (int k = 0; k < K; ++k)
    for (int s = 0; s < 2 * dim; ++s) {
      int j = s / 2, e = s % 2;
      entity_corners(dim, 1 << j, e << j, cs);
      std::vector<int> key;
      for (int c : cs) key.push_back(pd.vid[k * nc + c]);
      std::sort(key.begin(), key.end());
      sides[key].push_back(k * 2 * dim + s);
    }
  pd.side.assign(K * 2 * dim, SIDE_DIRICHLET);
  for (auto& kv : sides) {
    if (kv.second.size() > 2) return fail(code, ERR_GEOMETRY, "a side is shared by more than two patches");
    for (int ks : kv.second) {
      int tag = pd.side_bc[ks];
      if (kv.second.size() == 2) {
        if (tag != 0) return fail(code, ERR_GEOMETRY, "interface side must be tagged AUTO");
        pd.side[ks] = SIDE_INTERFACE;
      } else {
        pd.side[ks] = (tag == 2) ? SIDE_NEUMANN : SIDE_DIRICHLET;
      }
    }
  }
  return "";
}

namespace {
struct KeyInfo {
  int64_t id = -1;
  bool dirichlet = false;
  std::vector<int64_t> copies;  // tile offsets, in patch order
  int first_k = -1;
  int first_fixed_mask = 0, first_fixed_end = 0;
  std::vector<int> first_free_sorted;  // patch-local directions in canonical order
};
}  // namespace

std::string build_level(const ProblemDesc& pd, int level, LevelTopo& L, int* code) {
  *code = 0;
  const int d = pd.dim, K = pd.K, nc = 1 << d;
  const int shift = pd.levels - 1 - level;
  L = LevelTopo();
  L.level = level;
  L.n.resize(K * d);
  L.off.assign(K + 1, 0);
  for (int k = 0; k < K; ++k) {
    int64_t cnt = 1;
    for (int j = 0; j < d; ++j) {
      L.n[k * d + j] = (pd.m[k * d + j] >> shift) + pd.p[k * d + j];
      cnt *= L.n[k * d + j];
    }
    L.off[k + 1] = L.off[k] + cnt;
  }
  L.T = L.off[K];

  std::map<std::vector<int64_t>, KeyInfo> keys;
  std::vector<const std::vector<int64_t>*> node_key(L.T, nullptr);
  std::vector<int> ec;
  for (int k = 0; k < K; ++k) {
    const int* nk = &L.n[k * d];
    int64_t cnt = L.off[k + 1] - L.off[k];
    for (int64_t li = 0; li < cnt; ++li) {
      int idx[3] = {0, 0, 0};
      int64_t r = li;
      for (int j = d - 1; j >= 0; --j) {
        idx[j] = int(r % nk[j]);
        r /= nk[j];
      }
      int fmask = 0, fend = 0;
      for (int j = 0; j < d; ++j) {
        if (idx[j] == 0) fmask |= 1 << j;
        else if (idx[j] == nk[j] - 1) { fmask |= 1 << j; fend |= 1 << j; }
      }
      if (!fmask) continue;
      entity_corners(d, fmask, fend, ec);
      int o = ec[0];
      for (int c : ec)
        if (pd.vid[k * nc + c] < pd.vid[k * nc + o]) o = c;
      std::vector<std::pair<int, int>> pos;  // (neighbour vid, index from origin)
      std::vector<std::pair<int, int>> dirs;
      for (int j = 0; j < d; ++j) {
        if (fmask & (1 << j)) continue;
        int nb = pd.vid[k * nc + (o ^ (1 << j))];
        int q = ((o >> j) & 1) ? nk[j] - 1 - idx[j] : idx[j];
        pos.push_back({nb, q});
        dirs.push_back({nb, j});
      }
      std::sort(pos.begin(), pos.end());
      std::sort(dirs.begin(), dirs.end());
      std::vector<int64_t> key;
      std::vector<int64_t> vs;
      for (int c : ec) vs.push_back(pd.vid[k * nc + c]);
      std::sort(vs.begin(), vs.end());
      key.push_back(int64_t(vs.size()));
      key.insert(key.end(), vs.begin(), vs.end());
      for (auto& pq : pos) key.push_back(pq.second);
      auto it = keys.find(key);
      if (it == keys.end()) {
        it = keys.emplace(key, KeyInfo()).first;
        it->second.first_k = k;
        it->second.first_fixed_mask = fmask;
        it->second.first_fixed_end = fend;
        for (auto& dj : dirs) it->second.first_free_sorted.push_back(dj.second);
      }
      KeyInfo& ki = it->second;
      ki.copies.push_back(L.off[k] + li);
      for (int s = 0; s < 2 * d; ++s) {
        int j = s / 2, e = s % 2;
        if (pd.side[k * 2 * d + s] == SIDE_DIRICHLET && idx[j] == (e ? nk[j] - 1 : 0)) ki.dirichlet = true;
      }
      node_key[L.off[k] + li] = &it->first;
    }
  }

  // interior boxes and piece-major numbering
  L.l2g.assign(L.T, -1);
  int64_t next = 0;
  for (int k = 0; k < K; ++k) {
    Interior in;
    in.k = k;
    const int* nk = &L.n[k * d];
    int64_t box = 1;
    for (int j = 0; j < 3; ++j) { in.lo[j] = 0; in.len[j] = 1; in.drop_lo[j] = in.drop_hi[j] = false; }
    for (int j = 0; j < d; ++j) {
      in.drop_lo[j] = pd.side[k * 2 * d + 2 * j] != SIDE_NEUMANN;
      in.drop_hi[j] = pd.side[k * 2 * d + 2 * j + 1] != SIDE_NEUMANN;
      in.lo[j] = in.drop_lo[j] ? 1 : 0;
      in.len[j] = nk[j] - in.lo[j] - (in.drop_hi[j] ? 1 : 0);
      if (in.len[j] < 0) return fail(code, ERR_UNSUPPORTED, "patch interior is ill-formed");
      box *= in.len[j];
    }
    for (int64_t b = 0; b < box; ++b) {
      int idx[3] = {0, 0, 0};
      int64_t r = b;
      for (int j = d - 1; j >= 0; --j) {
        idx[j] = in.lo[j] + int(r % in.len[j]);
        r /= in.len[j];
      }
      int64_t li = 0;
      for (int j = 0; j < d; ++j) li = li * nk[j] + idx[j];
      int64_t t = L.off[k] + li;
      if (node_key[t]) {
        KeyInfo& ki = keys[*node_key[t]];
        if (ki.dirichlet || ki.copies.size() != 1)
          return fail(code, ERR_UNSUPPORTED, "patch interior touches a shared or Dirichlet dof");
        ki.id = next;
      }
      L.l2g[t] = next++;
    }
    L.interiors.push_back(in);
  }
  // interface pieces, grouped by entity (sorted corner vids), canonical node order
  std::map<std::vector<int64_t>, std::vector<std::map<std::vector<int64_t>, KeyInfo>::iterator>> ents;
  for (auto it = keys.begin(); it != keys.end(); ++it) {
    KeyInfo& ki = it->second;
    if (ki.dirichlet) continue;
    if (ki.copies.size() < 2) {
      if (ki.id < 0) return fail(code, ERR_GEOMETRY, "non-matching discretisation on an interface");
      continue;
    }
    const std::vector<int64_t>& key = it->first;
    std::vector<int64_t> ent(key.begin(), key.begin() + 1 + key[0]);
    ents[ent].push_back(it);  // map order over keys = canonical index order within an entity
  }
  for (auto& kv : ents) {
    auto& lst = kv.second;
    KeyInfo& k0 = lst[0]->second;
    IfacePiece pc;
    int ncorner = int(kv.first[0]);
    pc.kind = ncorner == 1 ? PIECE_VERTEX : (ncorner == 2 ? PIECE_EDGE : PIECE_FACE);
    pc.k = k0.first_k;
    pc.ndir = int(k0.first_free_sorted.size());
    pc.dirs[0] = pc.dirs[1] = -1;
    pc.len[0] = pc.len[1] = 1;
    int64_t cnt = 1;
    for (int a = 0; a < pc.ndir; ++a) {
      pc.dirs[a] = k0.first_free_sorted[a];
      pc.len[a] = L.n[pc.k * d + pc.dirs[a]] - 2;
      cnt *= pc.len[a];
    }
    if (int64_t(lst.size()) != cnt) return fail(code, ERR_GEOMETRY, "incomplete interface piece");
    pc.first = int64_t(L.iface_gid.size());
    for (auto it : lst) {
      it->second.id = next++;
      L.iface_gid.push_back(it->second.id);
    }
    L.ifaces.push_back(pc);
  }
  L.N = next;
  for (int64_t t = 0; t < L.T; ++t)
    if (node_key[t]) {
      const KeyInfo& ki = keys[*node_key[t]];
      L.l2g[t] = ki.dirichlet ? -1 : ki.id;
    }
  // copies of every global dof in tile order
  L.g2t_ptr.assign(L.N + 1, 0);
  for (int64_t t = 0; t < L.T; ++t)
    if (L.l2g[t] >= 0) L.g2t_ptr[L.l2g[t] + 1]++;
  for (int64_t g = 0; g < L.N; ++g) L.g2t_ptr[g + 1] += L.g2t_ptr[g];
  L.g2t.assign(L.g2t_ptr[L.N], 0);
  std::vector<int64_t> fill(L.g2t_ptr.begin(), L.g2t_ptr.end() - 1);
  for (int64_t t = 0; t < L.T; ++t)
    if (L.l2g[t] >= 0) L.g2t[fill[L.l2g[t]]++] = t;
  for (int64_t g = 0; g < L.N; ++g)
    if (L.g2t_ptr[g + 1] == L.g2t_ptr[g]) return fail(code, ERR_GEOMETRY, "dof without a copy");
  return "";
}

}  // namespace igamg
