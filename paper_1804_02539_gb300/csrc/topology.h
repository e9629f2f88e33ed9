// Multi-patch topology, dof numbering and piece decomposition of V_l (Sec. 2, Eq. vh;
// Sec. 3, Eq. additive), built on the host during setup.
//
// Tile layout ("patch-local", the accumulated/distributed vectors of Sec. 4 on one
// device): level l stores, for every patch k, its full tensor basis as a tile of
// prod_j n_kj values in C order (last direction fastest); tiles are concatenated in patch
// order.  A global dof shared by several patches has one copy in each owner's tile.
//
// Global numbering of the library (piece-major): the patch-interior pieces in patch order
// (each in C order), then the interface pieces (edges / faces / vertices) in the order of
// their sorted corner-vertex ids, each in its canonical node order.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace igamg {

enum SideType { SIDE_INTERFACE = 0, SIDE_DIRICHLET = 1, SIDE_NEUMANN = 2 };
enum PieceKind { PIECE_VERTEX = 0, PIECE_EDGE = 1, PIECE_FACE = 2 };

struct ProblemDesc {  // validated copy of igamg_problem
  int dim = 0, K = 0, levels = 0;
  std::vector<int> p;        // [K*dim]
  std::vector<int> m;        // [K*dim] finest intervals
  std::vector<double> corners;  // [K * 2^dim * dim]
  std::vector<int> side_bc;  // [K*2*dim] input tags
  std::vector<int> side;     // [K*2*dim] resolved SideType
  std::vector<int> vid;      // [K*2^dim] global vertex ids
};

struct Interior {          // patch-interior piece: tensor box of a tile
  int k;
  int lo[3], len[3];       // first index and length per direction
  bool drop_lo[3], drop_hi[3];
};

struct IfacePiece {        // edge / face / vertex piece shared by >= 2 patches
  int kind;                // PieceKind
  int k;                   // first owner patch (its 1D data is used)
  int ndir;                // 0, 1 or 2 free directions
  int dirs[2];             // patch-k directions of the piece axes (canonical order)
  int len[2];              // nodes per axis (n - 2 each)
  int64_t first;           // index of its first node in the interface node list
};

struct LevelTopo {
  int level = 0;
  std::vector<int> n;           // [K*dim]
  std::vector<int64_t> off;     // [K+1] tile offsets
  int64_t T = 0;                // total tile nodes
  int64_t N = 0;                // active dofs
  std::vector<int64_t> l2g;     // [T]
  std::vector<int64_t> g2t_ptr; // [N+1] copies of every dof (tile offsets), patch order
  std::vector<int64_t> g2t;
  std::vector<Interior> interiors;
  std::vector<IfacePiece> ifaces;
  std::vector<int64_t> iface_gid;  // global id of every interface node, piece by piece
};

// Parses and validates; returns "" on success or an error message with *code set.
std::string parse_problem(int dim, int K, const int* degree, const int* num_knots,
                          const double* knots, const int* geo_degree, const int* geo_num_ctrl,
                          const double* geo_ctrl, const int* side_bc, int num_levels,
                          ProblemDesc& out, int* code);

std::string build_level(const ProblemDesc& pd, int level, LevelTopo& out, int* code);

}  // namespace igamg
