// Internal data structures of libnesa (host side).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nesa.h"

namespace nesa {

// Status carried as an exception inside the library; converted at the ABI boundary.
struct Error {
  int status;
  std::string what;
};
[[noreturn]] void fail(int status, const std::string &what);
// message returned by nesa_last_error on this host thread
void set_last_error(const std::string &what);

// Everything the host computes from the mesh and the parameters (integer structure,
// geometry of the points and of the equivalent-source spheres).  Built by
// build_host_model (nesa_host.cpp), then uploaded by nesa_build.
struct HostLevel {
  int q = 0;                        // Q_l (l >= l0)
  double width = 0.0;               // box side w_l
  std::vector<uint64_t> key;        // Morton keys of the occupied boxes, ascending
  std::vector<int32_t> ijk;         // [nbox][3] integer coordinates
  std::vector<int32_t> parent;      // index of the parent box at level l-1 (-1 at level 0)
  std::vector<int32_t> octant;      // child bits (x | y<<1 | z<<2) relative to the parent
  std::vector<int32_t> child_ptr;   // [nbox+1] children (at level l+1) are contiguous
  // interaction lists (l >= l0), CSR by target box
  std::vector<int32_t> il_ptr, il_src, il_slot;
  std::vector<int32_t> offsets;     // [noff][3] distinct offsets (target - source), sorted
  std::vector<double> eq_pts;       // [q][3] equivalent points about the origin
  std::vector<double> test_pts;     // [2q][3] test points about the origin
};

struct HostModel {
  // mesh
  int64_t nv = 0, nt = 0;
  std::vector<double> verts;        // [nv][3]
  std::vector<int32_t> tris;        // [nt][3]
  // RWG functions (ABI order)
  int64_t n = 0;
  std::vector<int32_t> rwg_edge;    // [n][2]
  std::vector<int32_t> rwg_tri;     // [n][2] T+, T-
  std::vector<int32_t> rwg_free;    // [n][2] local free vertex in T+, T-
  std::vector<int32_t> tri_rwg;     // [nt][3] RWG of the edge opposite local vertex c, or -1
  std::vector<double> tri_sl;       // [nt][3] sign * length
  // quadrature points (point 7t+i)
  int64_t np = 0;
  std::vector<double> pts;          // [np][3]
  std::vector<int32_t> pt_leaf_ijk; // [np][3]
  std::vector<int32_t> pt_leaf;     // [np] leaf index
  // tree
  int L = 0, l0 = 0;
  double origin[3] = {0, 0, 0};
  std::vector<HostLevel> lev;       // [L+1]
  std::vector<int32_t> leaf_pt_ptr; // [nleaf+1] points grouped by leaf
  std::vector<int32_t> leaf_pt;     // point ids, ascending within a leaf
  // V columns: RWG functions touching each leaf (ascending), CSR by leaf
  std::vector<int32_t> vc_ptr, vc_rwg;
  // reception map: for each RWG the global V columns it owns, CSR by RWG
  std::vector<int32_t> rx_ptr, rx_col;
  // triangles with a point in each leaf (CSR by leaf, ascending) and the touching leaves
  // of each leaf, itself included (CSR by leaf)
  std::vector<int32_t> leaf_tri_ptr, leaf_tri, nl_ptr, nl;
  // near field: triangle pairs (CSR by outer triangle, ascending inner) and the RWG
  // pattern (CSR by row, ascending columns)
  std::vector<int64_t> tp_ptr;
  std::vector<int32_t> tp_col;
  std::vector<int64_t> nz_ptr;
  std::vector<int32_t> nz_col;
};

void build_host_model(const nesa_mesh &mesh, double k, const nesa_params &p, HostModel &m);
// The stages of build_host_model, in order (nesa_build replaces host_tree by its device
// counterpart, which fills the same fields):
//   host_mesh     mesh copy, validation, RWG functions
//   host_tree     quadrature points, octree levels, leaf point lists, l0, interaction
//                 lists, leaf triangle lists, leaf near lists
//   host_level_q  Q, equivalent and test points per far level
//   host_patterns V columns, reception map, near triangle pairs, RWG near pattern
void host_mesh(const nesa_mesh &mesh, HostModel &m);
void host_tree(const nesa_params &p, HostModel &m);
void host_level_q(double k, const nesa_params &p, HostModel &m);
void host_patterns(HostModel &m);
// root cube of the tree (sets m.L and m.origin from the vertex bounding box lo, hi, which
// it fills); m.pts must hold the quadrature points when p.points_per_leaf > 0
double host_root(const nesa_params &p, HostModel &m, double lo[3], double hi[3]);
// Morton key of integer box coordinates (bits of i, j, k interleaved, i lowest)
uint64_t morton_key(int32_t i, int32_t j, int32_t k);
// Radon's 7-point rule: barycentric coordinates of the nodes [7][3]
void rule7_nodes(double bary[7][3]);
// shared pieces of host_tree and its device counterpart
void decode_keys(HostLevel &lv);
int coarsest_far_level(const HostModel &m, const double lo[3], const double hi[3]);
void finish_interactions(HostLevel &lv, const std::vector<int32_t> &tgt, const std::vector<int32_t> &src,
                         const std::vector<int32_t> &off);

// Q of one level (NESA_Q_FIXED / NESA_Q_AUTO rule).
int q_for_level(double k, double width, const nesa_params &p);

}  // namespace nesa
