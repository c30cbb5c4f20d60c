// Host-side structure of the NESA operator: RWG functions, quadrature points, octree,
// interaction lists and sparsity patterns.  Integer and geometry work only; all
// matrix values are filled on the device (nesa_build.cu).
//
// Compiled with -ffp-contract=off: the quadrature points and their leaf indices are
// evaluated in a fixed operation order, so that a point lying exactly on a box face
// always lands in the same leaf.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "nesa_internal.h"

namespace nesa {

void fail(int status, const std::string &what) { throw Error{status, what}; }

// Rows 0..n-1 of a CSR pattern computed in parallel: row_fn(r, out, mark) appends row r
// to out.  Rows are computed in contiguous chunks on the host threads and concatenated
// in row order, so the result does not depend on the number of threads.  mark is the
// thread's scratch of mark_size entries, -1 at the start; a thread meets its rows in
// ascending order, so a row may use its own index as the mark value.
template <typename PtrT, typename RowFn>
static void parallel_rows(int64_t n, int64_t mark_size, std::vector<PtrT> &ptr, std::vector<int32_t> &col,
                          RowFn row_fn) {
  const int nth = (int)std::max<unsigned>(1, std::min<unsigned>(32, std::thread::hardware_concurrency()));
  const int nchunk = (int)std::min<int64_t>(std::max<int64_t>(n, 1), 4 * nth);
  std::vector<std::vector<int32_t>> cols(nchunk);
  std::vector<std::vector<PtrT>> lens(nchunk);
  std::vector<char> failed(nchunk, 0);
  std::vector<std::string> what(nchunk);
  std::vector<int> status(nchunk, 0);
  auto work = [&](int t) {
    std::vector<int32_t> mark(std::max<int64_t>(mark_size, 0), -1);
    for (int ch = t; ch < nchunk; ch += nth) {
      const int64_t r0 = n * ch / nchunk, r1 = n * (ch + 1) / nchunk;
      try {
        for (int64_t r = r0; r < r1; ++r) {
          const size_t before = cols[ch].size();
          row_fn(r, cols[ch], mark);
          lens[ch].push_back((PtrT)(cols[ch].size() - before));
        }
      } catch (const Error &e) {
        failed[ch] = 1;
        status[ch] = e.status;
        what[ch] = e.what;
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) pool.emplace_back(work, t);
  for (auto &th : pool) th.join();
  for (int ch = 0; ch < nchunk; ++ch)
    if (failed[ch]) fail(status[ch], what[ch]);
  ptr.assign(n + 1, 0);
  size_t total = 0;
  for (auto &c : cols) total += c.size();
  col.clear();
  col.reserve(total);
  int64_t r = 0;
  for (int ch = 0; ch < nchunk; ++ch) {
    for (PtrT len : lens[ch]) {
      ptr[r + 1] = ptr[r] + len;
      ++r;
    }
    col.insert(col.end(), cols[ch].begin(), cols[ch].end());
    std::vector<int32_t>().swap(cols[ch]);
  }
}

// Radon's 7-point degree-5 rule (Stroud T2:5-1): centroid, and the orbits (a, b, b)
// with a = (9 -+ 2 sqrt15)/21, b = (6 +- sqrt15)/21.
static void rule7(double bary[7][3]) {
  const double s15 = std::sqrt(15.0);
  const double a1 = (9.0 - 2.0 * s15) / 21.0, b1 = (6.0 + s15) / 21.0;
  const double a2 = (9.0 + 2.0 * s15) / 21.0, b2 = (6.0 - s15) / 21.0;
  const double t = 1.0 / 3.0;
  const double B[7][3] = {{t, t, t}, {a1, b1, b1}, {b1, a1, b1}, {b1, b1, a1},
                          {a2, b2, b2}, {b2, a2, b2}, {b2, b2, a2}};
  std::memcpy(bary, B, sizeof(B));
}

int q_for_level(double k, double width, const nesa_params &p) {
  if (p.q_mode == NESA_Q_FIXED) return p.q_fixed;
  double kr = k * std::sqrt(3.0) / 2.0 * width;
  double nl = std::ceil(kr + 1.8 * std::pow(p.q_digits, 2.0 / 3.0) * std::cbrt(kr));
  long q = (long)(nl + 1) * (long)(nl + 1);
  return (int)std::max<long>(p.q_fixed, q);
}

static uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}
static uint64_t morton(int32_t i, int32_t j, int32_t k) {
  return spread3((uint64_t)i) | (spread3((uint64_t)j) << 1) | (spread3((uint64_t)k) << 2);
}
uint64_t morton_key(int32_t i, int32_t j, int32_t k) { return morton(i, j, k); }
void rule7_nodes(double bary[7][3]) { rule7(bary); }

static void fibonacci_sphere(int n, double radius, std::vector<double> &out) {
  out.resize((size_t)n * 3);
  const double ga = M_PI * (3.0 - std::sqrt(5.0));
  for (int i = 0; i < n; ++i) {
    double z = 1.0 - (2.0 * i + 1.0) / n;
    double s = std::sqrt(std::max(0.0, 1.0 - z * z));
    double ph = i * ga;
    out[3 * i + 0] = radius * s * std::cos(ph);
    out[3 * i + 1] = radius * s * std::sin(ph);
    out[3 * i + 2] = radius * z;
  }
}

static int find_box(const HostLevel &lv, uint64_t key) {
  auto it = std::lower_bound(lv.key.begin(), lv.key.end(), key);
  if (it == lv.key.end() || *it != key) return -1;
  return (int)(it - lv.key.begin());
}

static inline bool touch(const int32_t *a, const int32_t *b) {
  return std::abs(a[0] - b[0]) <= 1 && std::abs(a[1] - b[1]) <= 1 && std::abs(a[2] - b[2]) <= 1;
}

static void build_rwg(HostModel &m) {
  struct E {
    int32_t a, b, t, c;
  };
  std::vector<E> e;
  e.reserve((size_t)m.nt * 3);
  for (int64_t t = 0; t < m.nt; ++t)
    for (int c = 0; c < 3; ++c) {
      int32_t a = m.tris[3 * t + (c + 1) % 3], b = m.tris[3 * t + (c + 2) % 3];
      e.push_back({std::min(a, b), std::max(a, b), (int32_t)t, c});
    }
  std::sort(e.begin(), e.end(), [](const E &x, const E &y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    return x.t < y.t;
  });
  m.tri_rwg.assign((size_t)m.nt * 3, -1);
  m.tri_sl.assign((size_t)m.nt * 3, 0.0);
  size_t i = 0;
  while (i < e.size()) {
    size_t j = i;
    while (j < e.size() && e[j].a == e[i].a && e[j].b == e[i].b) ++j;
    if (j - i > 2) fail(NESA_ERR_MESH, "non-manifold edge shared by more than two triangles");
    if (j - i == 2) {
      int32_t id = (int32_t)m.n++;
      m.rwg_edge.push_back(e[i].a);
      m.rwg_edge.push_back(e[i].b);
      const double *va = &m.verts[3 * (size_t)e[i].a], *vb = &m.verts[3 * (size_t)e[i].b];
      double d0 = vb[0] - va[0], d1 = vb[1] - va[1], d2 = vb[2] - va[2];
      double len = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      for (int s = 0; s < 2; ++s) {
        const E &x = e[i + s];  // sorted by triangle: T+ first
        m.rwg_tri.push_back(x.t);
        m.rwg_free.push_back(x.c);
        m.tri_rwg[3 * (size_t)x.t + x.c] = id;
        m.tri_sl[3 * (size_t)x.t + x.c] = (s == 0 ? 1.0 : -1.0) * len;
      }
    }
    i = j;
  }
  if (m.n == 0) fail(NESA_ERR_MESH, "mesh has no interior edge");
}

// Integer coordinates of the boxes of a level from their Morton keys.
void decode_keys(HostLevel &lv) {
  lv.ijk.resize(lv.key.size() * 3);
  for (size_t b = 0; b < lv.key.size(); ++b) {
    uint64_t kk = lv.key[b];
    int32_t c[3] = {0, 0, 0};
    for (int bit = 0; bit < 21; ++bit)
      for (int x = 0; x < 3; ++x) c[x] |= (int32_t)((kk >> (3 * bit + x)) & 1ULL) << bit;
    for (int x = 0; x < 3; ++x) lv.ijk[3 * b + x] = c[x];
  }
}

// Coarsest far level (Sec. 3): the coarsest level with at least 4 occupied boxes along
// the longest extent of the vertex bounding box (the leaf level if none).
int coarsest_far_level(const HostModel &m, const double lo[3], const double hi[3]) {
  int axis = 0;
  for (int x = 1; x < 3; ++x)
    if (hi[x] - lo[x] > hi[axis] - lo[axis]) axis = x;
  for (int l = 0; l <= m.L; ++l) {
    std::vector<int32_t> c;
    for (size_t b = 0; b < m.lev[l].key.size(); ++b) c.push_back(m.lev[l].ijk[3 * b + axis]);
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    if (c.size() >= 4) return l;
  }
  return m.L;
}

// Interaction list of a level from its pairs in list order (targets ascending): CSR by
// target, and the slot of every pair's offset among the level's distinct offsets
// (target - source, sorted lexicographically).
void finish_interactions(HostLevel &lv, const std::vector<int32_t> &tgt, const std::vector<int32_t> &src,
                         const std::vector<int32_t> &off) {
  const size_t nbx = lv.key.size();
  std::vector<std::array<int32_t, 3>> offs;
  for (size_t e = 0; e < tgt.size(); ++e) offs.push_back({off[3 * e], off[3 * e + 1], off[3 * e + 2]});
  std::sort(offs.begin(), offs.end());
  offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
  lv.offsets.clear();
  for (auto &o : offs) lv.offsets.insert(lv.offsets.end(), o.begin(), o.end());
  lv.il_ptr.assign(nbx + 1, 0);
  for (int32_t a : tgt) lv.il_ptr[a + 1]++;
  for (size_t a = 0; a < nbx; ++a) lv.il_ptr[a + 1] += lv.il_ptr[a];
  lv.il_src.resize(tgt.size());
  lv.il_slot.resize(tgt.size());
  for (size_t e = 0; e < tgt.size(); ++e) {  // tgt is ascending already
    std::array<int32_t, 3> o = {off[3 * e], off[3 * e + 1], off[3 * e + 2]};
    lv.il_src[e] = src[e];
    lv.il_slot[e] = (int32_t)(std::lower_bound(offs.begin(), offs.end(), o) - offs.begin());
  }
}

// Mesh copy, validation and RWG functions.
void host_mesh(const nesa_mesh &mesh, HostModel &m) {
  m.nv = mesh.n_vertices;
  m.nt = mesh.n_triangles;
  m.verts.assign(mesh.vertices, mesh.vertices + 3 * m.nv);
  m.tris.assign(mesh.triangles, mesh.triangles + 3 * m.nt);
  for (int64_t t = 0; t < m.nt; ++t) {
    const int32_t *tv = &m.tris[3 * t];
    for (int c = 0; c < 3; ++c)
      if (tv[c] < 0 || tv[c] >= m.nv) fail(NESA_ERR_MESH, "triangle vertex index out of range");
    if (tv[0] == tv[1] || tv[1] == tv[2] || tv[0] == tv[2]) fail(NESA_ERR_MESH, "degenerate triangle");
    const double *a = &m.verts[3 * (size_t)tv[0]], *b = &m.verts[3 * (size_t)tv[1]], *c = &m.verts[3 * (size_t)tv[2]];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    // zero area, or an area at the rounding level of its edges (sine of the angle at a
    // below 1e-12): the RWG functions would divide by it
    const double c2 = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
    const double l1 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], l2 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    if (!(c2 > 1e-24 * l1 * l2)) fail(NESA_ERR_MESH, "degenerate triangle");
  }
  build_rwg(m);
}

// Bounding box of the vertices and the root cube: sets m.L and m.origin, returns the root
// side.  Needs the quadrature points (m.pts) only for the points_per_leaf rule.
double host_root(const nesa_params &p, HostModel &m, double lo[3], double hi[3]) {
  // root cube
  for (int x = 0; x < 3; ++x) {
    lo[x] = hi[x] = m.verts[x];
    for (int64_t v = 1; v < m.nv; ++v) {
      lo[x] = std::min(lo[x], m.verts[3 * v + x]);
      hi[x] = std::max(hi[x], m.verts[3 * v + x]);
    }
  }
  const double extent = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  if (!(extent > 0.0)) fail(NESA_ERR_MESH, "mesh has no extent");
  double root = 0.0;
  if (p.points_per_leaf > 0) {
    // Sec. 3: subdivide while the groups hold at least P sources on average.  The root
    // is the bounding cube; the leaf level is the deepest l <= 19 whose occupied boxes
    // average >= P points.  Boxes of level l are the depth-19 keys shifted by 3 (19 - l)
    // (dividing by a power of two is exact, so these are the level's own coordinates).
    constexpr int DMAX = NESA_MAX_LEVELS - 1;
    root = extent;
    double org[3];
    for (int x = 0; x < 3; ++x) org[x] = 0.5 * (lo[x] + hi[x]) - 0.5 * root;
    const double wd = root / std::ldexp(1.0, DMAX);
    const int32_t nbd = 1 << DMAX;
    std::vector<uint64_t> kd(m.np);
    for (int64_t q = 0; q < m.np; ++q) {
      int32_t c[3];
      for (int x = 0; x < 3; ++x) {
        double f = std::floor((m.pts[3 * q + x] - org[x]) / wd);
        c[x] = f < 0.0 ? 0 : (f > nbd - 1 ? nbd - 1 : (int32_t)f);
      }
      kd[q] = morton(c[0], c[1], c[2]);
    }
    std::sort(kd.begin(), kd.end());
    m.L = 0;
    for (int l = 0; l <= DMAX; ++l) {
      const int sh = 3 * (DMAX - l);
      int64_t nbox = 0;
      for (int64_t q = 0; q < m.np; ++q)
        if (q == 0 || (kd[q] >> sh) != (kd[q - 1] >> sh)) ++nbox;
      if ((double)m.np >= (double)p.points_per_leaf * (double)nbox)
        m.L = l;
      else
        break;
    }
  } else {
    if (p.n_levels > 0) {
      m.L = p.n_levels - 1;
    } else {  // the fewest levels whose root cube spans the bounding box
      m.L = 0;
      while (m.L < NESA_MAX_LEVELS - 1 && p.leaf_size * std::ldexp(1.0, m.L) < extent) ++m.L;
    }
    root = p.leaf_size * std::ldexp(1.0, m.L);
  }
  for (int x = 0; x < 3; ++x) m.origin[x] = 0.5 * (lo[x] + hi[x]) - 0.5 * root;
  return root;
}

// Quadrature points, octree, leaf point lists, coarsest far level, interaction lists,
// leaf triangle lists and leaf near lists (the part nesa_build runs on the device).
void host_tree(const nesa_params &p, HostModel &m) {
  // quadrature points, lambda0 v0 + lambda1 v1 + lambda2 v2 evaluated left to right
  double B[7][3];
  rule7(B);
  m.np = 7 * m.nt;
  m.pts.resize((size_t)m.np * 3);
  for (int64_t t = 0; t < m.nt; ++t)
    for (int i = 0; i < 7; ++i)
      for (int x = 0; x < 3; ++x) {
        double v0 = m.verts[3 * (size_t)m.tris[3 * t + 0] + x];
        double v1 = m.verts[3 * (size_t)m.tris[3 * t + 1] + x];
        double v2 = m.verts[3 * (size_t)m.tris[3 * t + 2] + x];
        double r = B[i][0] * v0 + B[i][1] * v1;
        m.pts[(7 * t + i) * 3 + x] = r + B[i][2] * v2;
      }

  double lo[3], hi[3];
  const double root = host_root(p, m, lo, hi);
  const double wl = root / std::ldexp(1.0, m.L);
  const int32_t nb = 1 << m.L;
  m.pt_leaf_ijk.resize((size_t)m.np * 3);
  std::vector<uint64_t> pkey(m.np);
  for (int64_t q = 0; q < m.np; ++q) {
    int32_t c[3];
    for (int x = 0; x < 3; ++x) {
      double f = std::floor((m.pts[3 * q + x] - m.origin[x]) / wl);
      int32_t i = f < 0.0 ? 0 : (f > nb - 1 ? nb - 1 : (int32_t)f);
      c[x] = i;
      m.pt_leaf_ijk[3 * q + x] = i;
    }
    pkey[q] = morton(c[0], c[1], c[2]);
  }

  // levels: occupied boxes, sorted Morton keys
  m.lev.assign(m.L + 1, HostLevel());
  {
    std::vector<uint64_t> keys(pkey);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (int l = m.L; l >= 0; --l) {
      HostLevel &lv = m.lev[l];
      lv.width = root / std::ldexp(1.0, l);
      if (l == m.L) {
        lv.key = keys;
      } else {
        lv.key.clear();
        for (uint64_t kk : m.lev[l + 1].key) {
          uint64_t pk = kk >> 3;
          if (lv.key.empty() || lv.key.back() != pk) lv.key.push_back(pk);
        }
      }
      decode_keys(lv);
    }
    for (int l = 0; l <= m.L; ++l) {
      HostLevel &lv = m.lev[l];
      size_t nbx = lv.key.size();
      lv.parent.assign(nbx, -1);
      lv.octant.assign(nbx, 0);
      if (l > 0)
        for (size_t b = 0; b < nbx; ++b) {
          lv.parent[b] = find_box(m.lev[l - 1], lv.key[b] >> 3);
          lv.octant[b] = (int32_t)(lv.key[b] & 7ULL);
        }
      lv.child_ptr.assign(nbx + 1, 0);
      if (l < m.L) {
        const HostLevel &ch = m.lev[l + 1];
        size_t c = 0;
        for (size_t b = 0; b < nbx; ++b) {
          lv.child_ptr[b] = (int32_t)c;
          while (c < ch.key.size() && (ch.key[c] >> 3) == lv.key[b]) ++c;
        }
        lv.child_ptr[nbx] = (int32_t)c;
      }
    }
  }

  m.l0 = coarsest_far_level(m, lo, hi);

  // points per leaf
  const HostLevel &leaves = m.lev[m.L];
  const int64_t nleaf = (int64_t)leaves.key.size();
  m.pt_leaf.resize(m.np);
  for (int64_t q = 0; q < m.np; ++q) m.pt_leaf[q] = find_box(leaves, pkey[q]);
  m.leaf_pt_ptr.assign(nleaf + 1, 0);
  for (int64_t q = 0; q < m.np; ++q) m.leaf_pt_ptr[m.pt_leaf[q] + 1]++;
  for (int64_t b = 0; b < nleaf; ++b) m.leaf_pt_ptr[b + 1] += m.leaf_pt_ptr[b];
  m.leaf_pt.resize(m.np);
  {
    std::vector<int32_t> fill(m.leaf_pt_ptr.begin(), m.leaf_pt_ptr.end() - 1);
    for (int64_t q = 0; q < m.np; ++q) m.leaf_pt[fill[m.pt_leaf[q]]++] = (int32_t)q;
  }

  // interaction lists
  for (int l = m.l0; l <= m.L; ++l) {
    HostLevel &lv = m.lev[l];
    const size_t nbx = lv.key.size();
    std::vector<int32_t> tgt, src, off;
    for (size_t a = 0; a < nbx; ++a) {
      const int32_t *ca = &lv.ijk[3 * a];
      auto add = [&](size_t b) {
        const int32_t *cb = &lv.ijk[3 * b];
        if (touch(ca, cb)) return;
        tgt.push_back((int32_t)a);
        src.push_back((int32_t)b);
        off.push_back(ca[0] - cb[0]);
        off.push_back(ca[1] - cb[1]);
        off.push_back(ca[2] - cb[2]);
      };
      if (l == m.l0) {
        for (size_t b = 0; b < nbx; ++b) add(b);
      } else {
        const HostLevel &pl = m.lev[l - 1];
        int32_t P = lv.parent[a];
        const int32_t *cp = &pl.ijk[3 * P];
        std::vector<int32_t> cand;
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              int32_t x = cp[0] + dx, y = cp[1] + dy, z = cp[2] + dz;
              if (x < 0 || y < 0 || z < 0) continue;
              int nb2 = find_box(pl, morton(x, y, z));
              if (nb2 >= 0) cand.push_back(nb2);
            }
        std::sort(cand.begin(), cand.end());
        for (int32_t P2 : cand)
          for (int32_t b = pl.child_ptr[P2]; b < pl.child_ptr[P2 + 1]; ++b) add((size_t)b);
      }
    }
    finish_interactions(lv, tgt, src, off);
  }
  // triangles with a point in each leaf, and near leaves (touching, incl. itself) of each leaf
  {
    std::vector<int32_t> &leaf_tri_ptr = m.leaf_tri_ptr, &leaf_tri = m.leaf_tri;
    leaf_tri_ptr.assign(nleaf + 1, 0);
    leaf_tri.clear();
    {
      std::vector<std::pair<int32_t, int32_t>> lt;
      lt.reserve(m.np);
      for (int64_t q = 0; q < m.np; ++q) lt.push_back({m.pt_leaf[q], (int32_t)(q / 7)});
      std::sort(lt.begin(), lt.end());
      lt.erase(std::unique(lt.begin(), lt.end()), lt.end());
      for (auto &x : lt) leaf_tri_ptr[x.first + 1]++;
      for (int64_t b = 0; b < nleaf; ++b) leaf_tri_ptr[b + 1] += leaf_tri_ptr[b];
      leaf_tri.resize(lt.size());
      for (size_t i = 0; i < lt.size(); ++i) leaf_tri[i] = lt[i].second;
    }
    // near leaves of every leaf
    std::vector<int32_t> &nl_ptr = m.nl_ptr, &nl = m.nl;
    nl_ptr.assign(nleaf + 1, 0);
    nl.clear();
    for (int64_t b = 0; b < nleaf; ++b) {
      const int32_t *c = &leaves.ijk[3 * b];
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            int32_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
            if (x < 0 || y < 0 || z < 0 || x >= nb || y >= nb || z >= nb) continue;
            int nb2 = find_box(leaves, morton(x, y, z));
            if (nb2 >= 0) nl.push_back(nb2);
          }
      nl_ptr[b + 1] = (int32_t)nl.size();
    }
  }
}

// Equivalent and test points of every far level (Q per level by the q_mode rule).
void host_level_q(double k, const nesa_params &p, HostModel &m) {
  for (int l = m.l0; l <= m.L; ++l) {
    HostLevel &lv = m.lev[l];
    lv.q = q_for_level(k, lv.width, p);
    if (lv.q <= 0 || lv.q > 16384) fail(NESA_ERR_INVALID_ARG, "number of equivalent sources out of range");
    double R = std::sqrt(3.0) / 2.0 * lv.width;
    fibonacci_sphere(lv.q, p.rho_eq * R, lv.eq_pts);
    fibonacci_sphere(2 * lv.q, p.rho_test * R, lv.test_pts);
  }
}

// V columns and reception map, near triangle pairs (with the check that every pair of
// triangles sharing a vertex is near) and the RWG near pattern.
void host_patterns(HostModel &m) {
  const int64_t nleaf = (int64_t)m.lev[m.L].key.size();
  // V columns: RWG functions with a point in each leaf
  {
    m.vc_ptr.assign(nleaf + 1, 0);
    m.vc_rwg.clear();
    std::vector<int32_t> cols;
    for (int64_t b = 0; b < nleaf; ++b) {
      cols.clear();
      for (int32_t e = m.leaf_pt_ptr[b]; e < m.leaf_pt_ptr[b + 1]; ++e) {
        int32_t t = m.leaf_pt[e] / 7;
        for (int c = 0; c < 3; ++c)
          if (m.tri_rwg[3 * (size_t)t + c] >= 0) cols.push_back(m.tri_rwg[3 * (size_t)t + c]);
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      m.vc_rwg.insert(m.vc_rwg.end(), cols.begin(), cols.end());
      m.vc_ptr[b + 1] = (int32_t)m.vc_rwg.size();
    }
    m.rx_ptr.assign(m.n + 1, 0);
    for (int32_t r : m.vc_rwg) m.rx_ptr[r + 1]++;
    for (int64_t r = 0; r < m.n; ++r) m.rx_ptr[r + 1] += m.rx_ptr[r];
    m.rx_col.resize(m.vc_rwg.size());
    std::vector<int32_t> fill(m.rx_ptr.begin(), m.rx_ptr.end() - 1);
    for (size_t g = 0; g < m.vc_rwg.size(); ++g) m.rx_col[fill[m.vc_rwg[g]]++] = (int32_t)g;
  }

  // near triangle pairs: inner triangles with a point in a leaf touching a leaf of the
  // outer triangle's points
  {
    const std::vector<int32_t> &leaf_tri_ptr = m.leaf_tri_ptr, &leaf_tri = m.leaf_tri, &nl_ptr = m.nl_ptr, &nl = m.nl;
    // near triangles of triangle t (ascending): every triangle with a point in a leaf
    // touching a leaf of one of t's points; rows computed in parallel
    {
      parallel_rows(m.nt, m.nt, m.tp_ptr, m.tp_col, [&](int64_t t, std::vector<int32_t> &out,
                                                         std::vector<int32_t> &mark) {
        const size_t at = out.size();
        for (int i = 0; i < 7; ++i) {
          int32_t lf = m.pt_leaf[7 * t + i];
          for (int32_t e = nl_ptr[lf]; e < nl_ptr[lf + 1]; ++e) {
            int32_t b = nl[e];
            for (int32_t f = leaf_tri_ptr[b]; f < leaf_tri_ptr[b + 1]; ++f) {
              int32_t t2 = leaf_tri[f];
              if (mark[t2] != t) {
                mark[t2] = (int32_t)t;
                out.push_back(t2);
              }
            }
          }
        }
        std::sort(out.begin() + at, out.end());
      });
    }
    // every pair of triangles sharing a vertex must be a near pair
    {
      std::vector<int32_t> vt_ptr(m.nv + 1, 0), vt(3 * m.nt);
      for (int64_t t = 0; t < m.nt; ++t)
        for (int c = 0; c < 3; ++c) vt_ptr[m.tris[3 * t + c] + 1]++;
      for (int64_t v = 0; v < m.nv; ++v) vt_ptr[v + 1] += vt_ptr[v];
      {
        std::vector<int32_t> fill(vt_ptr.begin(), vt_ptr.end() - 1);
        for (int64_t t = 0; t < m.nt; ++t)
          for (int c = 0; c < 3; ++c) vt[fill[m.tris[3 * t + c]]++] = (int32_t)t;
      }
      std::vector<int64_t> dummy_ptr;
      std::vector<int32_t> dummy_col;
      parallel_rows(m.nt, 0, dummy_ptr, dummy_col, [&](int64_t t, std::vector<int32_t> &, std::vector<int32_t> &) {
        for (int c = 0; c < 3; ++c) {
          const int32_t v = m.tris[3 * t + c];
          for (int32_t e = vt_ptr[v]; e < vt_ptr[v + 1]; ++e)
            if (!std::binary_search(m.tp_col.begin() + m.tp_ptr[t], m.tp_col.begin() + m.tp_ptr[t + 1], vt[e]))
              fail(NESA_ERR_MESH, "triangles sharing a vertex lie in non-touching leaves: leaf too small");
        }
      });
    }
    // RWG pattern: union over the supports of m of the RWG functions of near triangles
    {
      parallel_rows(m.n, m.n, m.nz_ptr, m.nz_col, [&](int64_t r, std::vector<int32_t> &out,
                                                       std::vector<int32_t> &mk) {
        const size_t at = out.size();
        for (int s = 0; s < 2; ++s) {
          int32_t t = m.rwg_tri[2 * r + s];
          for (int64_t e = m.tp_ptr[t]; e < m.tp_ptr[t + 1]; ++e) {
            int32_t t2 = m.tp_col[e];
            for (int c = 0; c < 3; ++c) {
              int32_t r2 = m.tri_rwg[3 * (size_t)t2 + c];
              if (r2 >= 0 && mk[r2] != r) {
                mk[r2] = (int32_t)r;
                out.push_back(r2);
              }
            }
          }
        }
        std::sort(out.begin() + at, out.end());
      });
    }
  }
}

void build_host_model(const nesa_mesh &mesh, double k, const nesa_params &p, HostModel &m) {
  host_mesh(mesh, m);
  host_tree(p, m);
  host_level_q(k, p, m);
  host_patterns(m);
}

}  // namespace nesa
