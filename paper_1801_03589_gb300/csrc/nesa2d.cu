// The 2D model problem of Sec. 3: the potential of N charges on a curve in the plane,
// phi_i = sum_{j != i} -log|x_i - x_j| q_j (Eq. 8), by the NESA product (Eqs. 9-14).
//
// Host (build): quadtree, near and interaction lists, the near-field blocks and the
// operators V, C, D in FP64 (readings in include/nesa2d.h).  Device (product), one
// kernel per stage and level, real FP64, every output element written by one thread
// (owner computes; deterministic):
//   k2_perm_in     q in the internal order (points sorted by leaf)
//   k2_near        y_a = sum_{b near a} Z_ab q_b                       (Eq. 9)
//   k2_radiate     s_b = V_b q_b                                       (Eq. 10)
//   k2_upward      s_P = sum_children C(quadrant) s_child              (Eq. 11)
//   k2_translate   o_a = C(quadrant)^T o_P(a) + sum_{b in IL(a)} D(a - b) s_b
//                                                                      (Eqs. 13, 12)
//   k2_receive     y_a += V_a^T o_a                                    (Eq. 14)
//   k2_perm_out    phi in the caller's order
// Layouts: internal vectors [nrhs][n]; s_l, o_l = [box][nrhs][Q]; V_b is Q x |b|
// column-major at Q * (first point of b); C and D are Q x Q column-major; the near
// block (a, b) is |a| x |b| column-major.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nesa2d.h"
#include "nesa_internal.h"

namespace nesa2d_impl {
// near-field kernel shape (k2_near): 8 warps, 2 rows per lane, tiles of 64 rows (leaves average P or
// more points, so a 64-row tile leaves few lanes idle)
constexpr int NEAR_WARPS = 8, NEAR_RB = 2, NEAR_TROWS = 32 * NEAR_RB;

using nesa::Error;
using nesa::fail;

constexpr int MAX_LEVEL = 30;  // Morton keys of 2 x 30 bits
constexpr double PI = 3.14159265358979323846;

struct Level {
  double w = 0.0;
  int64_t nbox = 0;
  std::vector<int64_t> key;                 // Morton keys of the occupied boxes, ascending
  std::vector<int32_t> ij;                  // [nbox][2]
  std::vector<int32_t> parent, quad;        // parent at l-1, quadrant bits (x | y << 1)
  std::vector<int32_t> child_ptr;           // [nbox+1] children at l+1 (l < L)
  std::vector<int32_t> il_ptr, il_src, il_slot;
  std::vector<int32_t> offsets;             // [noff][2] target - source, sorted
  // device
  double *D = nullptr, *C = nullptr, *Ct = nullptr, *s = nullptr, *o = nullptr;  // Ct: C transposed per quadrant
  int32_t *d_parent = nullptr, *d_quad = nullptr, *d_child_ptr = nullptr;
  int32_t *d_il_ptr = nullptr, *d_il_src = nullptr, *d_il_slot = nullptr;
};

}  // namespace nesa2d_impl

struct nesa2d_ctx {
  int64_t n = 0;
  int P = 0, Q = 0;
  double pinv_eps = 1e-9;
  int l0 = 2, L = 2;
  double lo[2] = {0, 0}, side = 0.0;
  cudaStream_t stream = nullptr;
  nesa2d_impl::Level lev[NESA2D_MAX_LEVELS];
  std::vector<int32_t> perm;      // internal index -> caller index
  std::vector<int32_t> leaf_ptr;  // [nleaf+1] internal point ranges of the leaves
  int64_t nleaf = 0, near_entries = 0;
  // device
  int32_t *d_perm = nullptr, *d_leaf_ptr = nullptr, *d_nptr = nullptr, *d_nleaf = nullptr;
  int32_t *d_pt_leaf = nullptr;  // [n] leaf of each internal point
  int64_t *d_noff = nullptr;
  int2 *d_tiles = nullptr;  // near-field row tiles (leaf, first row)
  int64_t ntile = 0;
  double *d_Z = nullptr, *d_V = nullptr, *d_qp = nullptr, *d_yp = nullptr;
  int nrhs_cap = 0;
  std::vector<void *> allocs;
  size_t device_bytes = 0;
};

namespace nesa2d_impl {

static void *dalloc(nesa2d_ctx *c, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    fail(NESA_ERR_OOM, "nesa2d: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  c->allocs.push_back(p);
  c->device_bytes += bytes;
  return p;
}

template <typename T>
static T *upload(nesa2d_ctx *c, const std::vector<T> &v) {
  T *d = (T *)dalloc(c, sizeof(T) * v.size());
  if (!v.empty() && cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    fail(NESA_ERR_CUDA, "nesa2d: upload failed");
  return d;
}

static void free_ctx(nesa2d_ctx *c) {
  if (!c) return;
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

static int64_t morton(int64_t i, int64_t j) {
  int64_t k = 0;
  for (int b = 0; b < MAX_LEVEL; ++b) k |= ((i >> b) & 1) << (2 * b + 1) | ((j >> b) & 1) << (2 * b);
  return k;
}

// -log|a - b|
static inline double g2(double ax, double ay, double bx, double by) {
  const double dx = ax - bx, dy = ay - by;
  return -0.5 * std::log(dx * dx + dy * dy);
}

// Tikhonov pseudo-inverse K = (A^T A + eps^2 I)^-1 A^T of A (m x nq, column-major,
// m >= nq), eps = pinv_eps ||A||_F: Householder QR of [A; eps I] = Q R, then
// K = R^-1 (Q^T [I_m; 0]) restricted to its first nq rows.  K is nq x m column-major.
static std::vector<double> tikhonov_pinv(const std::vector<double> &A, int m, int nq, double pinv_eps) {
  double fro = 0.0;
  for (double v : A) fro += v * v;
  const double eps = pinv_eps * std::sqrt(fro);
  const int mm = m + nq;
  std::vector<double> M((size_t)mm * nq, 0.0), B((size_t)mm * m, 0.0);
  for (int j = 0; j < nq; ++j) {
    for (int i = 0; i < m; ++i) M[(size_t)j * mm + i] = A[(size_t)j * m + i];
    M[(size_t)j * mm + m + j] = eps;
  }
  for (int j = 0; j < m; ++j) B[(size_t)j * mm + j] = 1.0;
  std::vector<double> v(mm);
  for (int k = 0; k < nq; ++k) {
    double nx = 0.0;
    for (int i = k; i < mm; ++i) nx += M[(size_t)k * mm + i] * M[(size_t)k * mm + i];
    nx = std::sqrt(nx);
    if (nx == 0.0) fail(NESA_ERR_NUMERIC, "nesa2d: rank-deficient fit matrix");
    const double x0 = M[(size_t)k * mm + k];
    const double alpha = x0 >= 0.0 ? -nx : nx;
    for (int i = k; i < mm; ++i) v[i] = M[(size_t)k * mm + i];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < mm; ++i) vv += v[i] * v[i];
    const double beta = vv > 0.0 ? 2.0 / vv : 0.0;
    auto apply = [&](double *col) {
      double sdot = 0.0;
      for (int i = k; i < mm; ++i) sdot += v[i] * col[i];
      sdot *= beta;
      for (int i = k; i < mm; ++i) col[i] -= sdot * v[i];
    };
    for (int j = k; j < nq; ++j) apply(&M[(size_t)j * mm]);
    for (int j = 0; j < m; ++j) apply(&B[(size_t)j * mm]);
  }
  std::vector<double> K((size_t)nq * m);
  for (int j = 0; j < m; ++j) {  // back substitution R x = B[0:nq, j]
    for (int i = nq - 1; i >= 0; --i) {
      double acc = B[(size_t)j * mm + i];
      for (int t = i + 1; t < nq; ++t) acc -= M[(size_t)t * mm + i] * K[(size_t)j * nq + t];
      K[(size_t)j * nq + i] = acc / M[(size_t)i * mm + i];
    }
  }
  return K;
}

// out (nq x cols, column-major) = K (nq x m) * G (m x cols); each entry summed over t
// in ascending order
static void matmul(const std::vector<double> &K, int nq, int m, const double *G, int cols, double *out) {
  for (int j = 0; j < cols; ++j) {
    double *o = out + (size_t)j * nq;
    for (int i = 0; i < nq; ++i) o[i] = 0.0;
    for (int t = 0; t < m; ++t) {
      const double gt = G[(size_t)j * m + t];
      const double *kt = &K[(size_t)t * nq];
      for (int i = 0; i < nq; ++i) o[i] += kt[i] * gt;
    }
  }
}

static void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)> &f) {
  const int nth = (int)std::max<unsigned>(1, std::min<unsigned>(16, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) pool.emplace_back(f, n * t / nth, n * (t + 1) / nth);
  for (auto &th : pool) th.join();
}

static void build(nesa2d_ctx *c, const double *x) {
  const int64_t n = c->n;
  for (int64_t i = 0; i < 2 * n; ++i)
    if (!std::isfinite(x[i])) fail(NESA_ERR_INVALID_ARG, "nesa2d: non-finite point");
  double hi[2] = {x[0], x[1]};
  c->lo[0] = x[0];
  c->lo[1] = x[1];
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 2; ++d) {
      c->lo[d] = std::min(c->lo[d], x[2 * i + d]);
      hi[d] = std::max(hi[d], x[2 * i + d]);
    }
  c->side = std::max(hi[0] - c->lo[0], hi[1] - c->lo[1]);
  if (!(c->side > 0.0)) fail(NESA_ERR_INVALID_ARG, "nesa2d: all points coincide");
  // integer coordinates of every point at level l, and the occupied boxes
  auto coords = [&](int l, std::vector<int64_t> &ci) {
    const int64_t nb = (int64_t)1 << l;
    const double w = c->side / (double)nb;
    ci.resize(2 * n);
    for (int64_t i = 0; i < n; ++i)
      for (int d = 0; d < 2; ++d) {
        int64_t v = (int64_t)std::floor((x[2 * i + d] - c->lo[d]) / w);
        ci[2 * i + d] = std::min(std::max<int64_t>(v, 0), nb - 1);
      }
  };
  auto occupied = [&](int l) {
    std::vector<int64_t> ci;
    coords(l, ci);
    std::vector<int64_t> keys(n);
    for (int64_t i = 0; i < n; ++i) keys[i] = morton(ci[2 * i], ci[2 * i + 1]);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    return keys;
  };
  c->l0 = 2;
  int L = c->l0;
  while (L < MAX_LEVEL && (double)n / (double)occupied(L + 1).size() >= (double)c->P) ++L;
  c->L = L;
  for (int l = c->l0; l <= L; ++l) {
    Level &lv = c->lev[l];
    lv.w = c->side / (double)((int64_t)1 << l);
    lv.key = occupied(l);
    lv.nbox = (int64_t)lv.key.size();
    lv.ij.resize(2 * lv.nbox);
    for (int64_t b = 0; b < lv.nbox; ++b) {
      int64_t i = 0, j = 0;
      for (int t = 0; t < MAX_LEVEL; ++t) {
        i |= ((lv.key[b] >> (2 * t + 1)) & 1) << t;
        j |= ((lv.key[b] >> (2 * t)) & 1) << t;
      }
      lv.ij[2 * b] = (int32_t)i;
      lv.ij[2 * b + 1] = (int32_t)j;
    }
  }
  auto find = [&](int l, int64_t i, int64_t j) -> int64_t {
    const int64_t nb = (int64_t)1 << l;
    if (i < 0 || j < 0 || i >= nb || j >= nb) return -1;
    const auto &k = c->lev[l].key;
    auto it = std::lower_bound(k.begin(), k.end(), morton(i, j));
    return (it != k.end() && *it == morton(i, j)) ? (int64_t)(it - k.begin()) : -1;
  };
  auto near = [&](int l, int64_t b, std::vector<int64_t> &out) {  // ascending box index
    out.clear();
    const int32_t *ij = &c->lev[l].ij[2 * b];
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        const int64_t f = find(l, ij[0] + di, ij[1] + dj);
        if (f >= 0) out.push_back(f);
      }
    std::sort(out.begin(), out.end());
  };
  // parents, quadrants, children
  for (int l = c->l0; l <= L; ++l) {
    Level &lv = c->lev[l];
    lv.parent.assign(lv.nbox, -1);
    lv.quad.assign(lv.nbox, 0);
    for (int64_t b = 0; b < lv.nbox; ++b) {
      lv.quad[b] = (lv.ij[2 * b] & 1) | ((lv.ij[2 * b + 1] & 1) << 1);
      if (l > c->l0) lv.parent[b] = (int32_t)find(l - 1, lv.ij[2 * b] >> 1, lv.ij[2 * b + 1] >> 1);
    }
    if (l > c->l0) {
      Level &pl = c->lev[l - 1];
      pl.child_ptr.assign(pl.nbox + 1, 0);
      for (int64_t b = 0; b < lv.nbox; ++b) pl.child_ptr[lv.parent[b] + 1]++;
      for (int64_t p = 0; p < pl.nbox; ++p) pl.child_ptr[p + 1] += pl.child_ptr[p];
    }
  }
  // interaction lists: at l0 every non-near box; below, children of the parent's near
  // boxes that are not near (offsets target - source)
  std::vector<int64_t> nb1, nb2;
  for (int l = c->l0; l <= L; ++l) {
    Level &lv = c->lev[l];
    std::vector<std::pair<int32_t, int32_t>> pairs;  // (target, source)
    for (int64_t a = 0; a < lv.nbox; ++a) {
      near(l, a, nb1);
      std::vector<int64_t> cand;
      if (l == c->l0) {
        for (int64_t b = 0; b < lv.nbox; ++b) cand.push_back(b);
      } else {
        near(l - 1, lv.parent[a], nb2);
        const Level &pl = c->lev[l - 1];
        for (int64_t pb : nb2)
          for (int32_t ch = pl.child_ptr[pb]; ch < pl.child_ptr[pb + 1]; ++ch) cand.push_back(ch);
        std::sort(cand.begin(), cand.end());
      }
      for (int64_t b : cand)
        if (!std::binary_search(nb1.begin(), nb1.end(), b)) pairs.push_back({(int32_t)a, (int32_t)b});
    }
    std::map<std::pair<int32_t, int32_t>, int32_t> slot;
    for (auto &p : pairs)
      slot[{lv.ij[2 * p.first] - lv.ij[2 * p.second], lv.ij[2 * p.first + 1] - lv.ij[2 * p.second + 1]}] = 0;
    int32_t k = 0;
    lv.offsets.clear();
    for (auto &s : slot) {
      s.second = k++;
      lv.offsets.push_back(s.first.first);
      lv.offsets.push_back(s.first.second);
    }
    lv.il_ptr.assign(lv.nbox + 1, 0);
    for (auto &p : pairs) lv.il_ptr[p.first + 1]++;
    for (int64_t a = 0; a < lv.nbox; ++a) lv.il_ptr[a + 1] += lv.il_ptr[a];
    lv.il_src.resize(pairs.size());
    lv.il_slot.resize(pairs.size());
    for (size_t e = 0; e < pairs.size(); ++e) {  // pairs are grouped by target already
      lv.il_src[e] = pairs[e].second;
      lv.il_slot[e] = slot[{lv.ij[2 * pairs[e].first] - lv.ij[2 * pairs[e].second],
                            lv.ij[2 * pairs[e].first + 1] - lv.ij[2 * pairs[e].second + 1]}];
    }
  }
  // points in the internal order: by leaf (Morton), then by caller index
  const Level &leaf = c->lev[L];
  std::vector<int64_t> ci;
  coords(L, ci);
  std::vector<int64_t> pleaf(n);
  for (int64_t i = 0; i < n; ++i) pleaf[i] = find(L, ci[2 * i], ci[2 * i + 1]);
  c->perm.resize(n);
  for (int64_t i = 0; i < n; ++i) c->perm[i] = (int32_t)i;
  std::stable_sort(c->perm.begin(), c->perm.end(), [&](int32_t a, int32_t b) { return pleaf[a] < pleaf[b]; });
  c->nleaf = leaf.nbox;
  c->leaf_ptr.assign(c->nleaf + 1, 0);
  for (int64_t i = 0; i < n; ++i) c->leaf_ptr[pleaf[i] + 1]++;
  for (int64_t b = 0; b < c->nleaf; ++b) c->leaf_ptr[b + 1] += c->leaf_ptr[b];
  std::vector<double> xp(2 * n);
  for (int64_t i = 0; i < n; ++i) {
    xp[2 * i] = x[2 * c->perm[i]];
    xp[2 * i + 1] = x[2 * c->perm[i] + 1];
  }
  // near-field blocks (Eq. 9): |a| x |b| column-major per near pair, K_ii = 0
  std::vector<int32_t> nptr(c->nleaf + 1, 0), nlist;
  std::vector<int64_t> noff;
  int64_t tot = 0;
  for (int64_t a = 0; a < c->nleaf; ++a) {
    near(L, a, nb1);
    for (int64_t b : nb1) {
      nlist.push_back((int32_t)b);
      noff.push_back(tot);
      tot += (int64_t)(c->leaf_ptr[a + 1] - c->leaf_ptr[a]) * (c->leaf_ptr[b + 1] - c->leaf_ptr[b]);
    }
    nptr[a + 1] = (int32_t)nlist.size();
  }
  c->near_entries = tot;
  std::vector<double> Z(std::max<int64_t>(tot, 1));
  std::atomic<bool> coincident{false};
  parallel_for(c->nleaf, [&](int64_t a0, int64_t a1) {
    for (int64_t a = a0; a < a1; ++a)
      for (int32_t e = nptr[a]; e < nptr[a + 1]; ++e) {
        const int64_t b = nlist[e];
        const int32_t ra = c->leaf_ptr[a], na = c->leaf_ptr[a + 1] - ra;
        const int32_t rb = c->leaf_ptr[b], nbb = c->leaf_ptr[b + 1] - rb;
        double *blk = &Z[noff[e]];
        for (int32_t j = 0; j < nbb; ++j)
          for (int32_t i = 0; i < na; ++i) {
            const int64_t pi = ra + i, pj = rb + j;
            double v = 0.0;
            if (pi != pj) {
              const double dx = xp[2 * pi] - xp[2 * pj], dy = xp[2 * pi + 1] - xp[2 * pj + 1];
              const double r2 = dx * dx + dy * dy;
              if (r2 == 0.0) coincident.store(true);
              v = -0.5 * std::log(r2);
            }
            blk[(int64_t)j * na + i] = v;
          }
      }
  });
  if (coincident.load()) fail(NESA_ERR_INVALID_ARG, "nesa2d: coincident points");
  // equivalent and test points, K_l, and the operators (Eqs. 10-12)
  const int Q = c->Q;
  std::vector<std::vector<double>> E(L + 1), T(L + 1), K(L + 1);
  for (int l = c->l0; l <= L; ++l) {
    const double w = c->lev[l].w, R = w / std::sqrt(2.0), rt = (2.0 - 1.0 / std::sqrt(2.0)) * w;
    E[l].resize(2 * Q);
    T[l].resize(4 * Q);
    for (int j = 0; j < Q; ++j) {
      const double t = 2.0 * PI * (j + 0.5) / Q;
      E[l][2 * j] = R * std::cos(t);
      E[l][2 * j + 1] = R * std::sin(t);
    }
    for (int j = 0; j < 2 * Q; ++j) {
      const double t = 2.0 * PI * j / (2 * Q);
      T[l][2 * j] = rt * std::cos(t);
      T[l][2 * j + 1] = rt * std::sin(t);
    }
    std::vector<double> A((size_t)2 * Q * Q);
    for (int j = 0; j < Q; ++j)
      for (int i = 0; i < 2 * Q; ++i) A[(size_t)j * 2 * Q + i] = g2(T[l][2 * i], T[l][2 * i + 1], E[l][2 * j], E[l][2 * j + 1]);
    K[l] = tikhonov_pinv(A, 2 * Q, Q, c->pinv_eps);
  }
  // V_b = K_L G(T_L + c_b, X_b), stored at Q * (first point of b)
  std::vector<double> V((size_t)Q * n);
  parallel_for(c->nleaf, [&](int64_t b0, int64_t b1) {
    std::vector<double> G;
    for (int64_t b = b0; b < b1; ++b) {
      const int32_t r0 = c->leaf_ptr[b], nbp = c->leaf_ptr[b + 1] - r0;
      const double cx = c->lo[0] + (leaf.ij[2 * b] + 0.5) * leaf.w, cy = c->lo[1] + (leaf.ij[2 * b + 1] + 0.5) * leaf.w;
      G.assign((size_t)2 * Q * nbp, 0.0);
      for (int32_t j = 0; j < nbp; ++j)
        for (int i = 0; i < 2 * Q; ++i)
          G[(size_t)j * 2 * Q + i] = g2(T[L][2 * i] + cx, T[L][2 * i + 1] + cy, xp[2 * (r0 + j)], xp[2 * (r0 + j) + 1]);
      matmul(K[L], Q, 2 * Q, G.data(), nbp, &V[(size_t)Q * r0]);
    }
  });
  for (int l = c->l0; l <= L; ++l) {
    Level &lv = c->lev[l];
    const int64_t noffs = (int64_t)lv.offsets.size() / 2;
    std::vector<double> D((size_t)std::max<int64_t>(noffs, 1) * Q * Q);
    for (int64_t s = 0; s < noffs; ++s)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i)
          D[((size_t)s * Q + j) * Q + i] = g2(E[l][2 * i] + lv.offsets[2 * s] * lv.w,
                                              E[l][2 * i + 1] + lv.offsets[2 * s + 1] * lv.w, E[l][2 * j], E[l][2 * j + 1]);
    lv.D = upload(c, D);
    if (l > c->l0) {  // C_l(quadrant) = K_{l-1} G(T_{l-1}, E_l + delta)
      std::vector<double> Cm((size_t)4 * Q * Q), G((size_t)2 * Q * Q);
      for (int qd = 0; qd < 4; ++qd) {
        const double dx = ((qd & 1) - 0.5) * lv.w, dy = (((qd >> 1) & 1) - 0.5) * lv.w;
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < 2 * Q; ++i)
            G[(size_t)j * 2 * Q + i] = g2(T[l - 1][2 * i], T[l - 1][2 * i + 1], E[l][2 * j] + dx, E[l][2 * j + 1] + dy);
        matmul(K[l - 1], Q, 2 * Q, G.data(), Q, &Cm[(size_t)qd * Q * Q]);
      }
      lv.C = upload(c, Cm);
      std::vector<double> Ctm(Cm.size());  // B = C^T of every quadrant, column-major
      for (int qd = 0; qd < 4; ++qd)
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < Q; ++i) Ctm[(size_t)qd * Q * Q + (size_t)j * Q + i] = Cm[(size_t)qd * Q * Q + (size_t)i * Q + j];
      lv.Ct = upload(c, Ctm);
    }
    lv.d_parent = upload(c, lv.parent);
    lv.d_quad = upload(c, lv.quad);
    if (l < L) lv.d_child_ptr = upload(c, lv.child_ptr);
    lv.d_il_ptr = upload(c, lv.il_ptr);
    lv.d_il_src = upload(c, lv.il_src);
    lv.d_il_slot = upload(c, lv.il_slot);
  }
  c->d_perm = upload(c, c->perm);
  c->d_leaf_ptr = upload(c, c->leaf_ptr);
  {
    std::vector<int32_t> pt_leaf(std::max<int64_t>(c->n, 1), 0);
    for (int64_t a = 0; a < c->nleaf; ++a)
      for (int32_t i = c->leaf_ptr[a]; i < c->leaf_ptr[a + 1]; ++i) pt_leaf[i] = (int32_t)a;
    c->d_pt_leaf = upload(c, pt_leaf);
  }
  c->d_nptr = upload(c, nptr);
  c->d_nleaf = upload(c, nlist);
  c->d_noff = upload(c, noff);
  {  // row tiles of the near-field kernel
    std::vector<int2> tiles;
    for (int64_t a = 0; a < c->nleaf; ++a)
      for (int32_t r0 = 0; r0 < c->leaf_ptr[a + 1] - c->leaf_ptr[a]; r0 += NEAR_TROWS)
        tiles.push_back(make_int2((int32_t)a, r0));
    c->ntile = (int64_t)tiles.size();
    c->d_tiles = upload(c, tiles);
  }
  c->d_Z = upload(c, Z);
  c->d_V = upload(c, V);
}

// ------------------------------------------------------------------ kernels
__global__ void k2_perm_in(double *qp, const double *q, const int32_t *perm, int64_t n, int nrhs) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, i = t % n;
    qp[t] = q[r * n + perm[i]];
  }
}

__global__ void k2_perm_out(double *phi, const double *yp, const int32_t *perm, int64_t n, int nrhs) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, i = t % n;
    phi[r * n + perm[i]] = yp[t];
  }
}

// Eq. 9.  The near blocks of a leaf a are stored one after the other, each column-major
// |a| x |b|, so together they form one column-major panel of |a| rows.  A CTA owns a tile
// of NEAR_TROWS rows of one leaf (work list `tiles`: leaf, first row); its 8 warps split
// the columns of every block between them (warp w: columns [w nb / 8, (w+1) nb / 8)), each
// lane accumulating NEAR_RB rows 32 apart, so that every column is one coalesced 256-byte
// load per row group and the panel is streamed once.  The 8 partial sums of a row are
// added in warp order (deterministic).  Rows past |a| are skipped.
__global__ void __launch_bounds__(32 * NEAR_WARPS) k2_near(double *__restrict__ yp, const double *__restrict__ qp,
                                                          int64_t n, int nrhs, const int32_t *__restrict__ leaf_ptr,
                                                          const int32_t *__restrict__ nptr,
                                                          const int32_t *__restrict__ nleaf,
                                                          const int64_t *__restrict__ noff,
                                                          const double *__restrict__ Z, const int2 *__restrict__ tiles,
                                                          int on) {
  __shared__ double red[NEAR_WARPS][NEAR_TROWS];
  const int2 tl = tiles[blockIdx.x];
  const int32_t a = tl.x, row0 = tl.y;
  const int32_t ra = leaf_ptr[a], na = leaf_ptr[a + 1] - ra;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = 0; r < nrhs; ++r) {
    double acc[NEAR_RB];
#pragma unroll
    for (int rr = 0; rr < NEAR_RB; ++rr) acc[rr] = 0.0;
    if (on)
      for (int32_t e = nptr[a]; e < nptr[a + 1]; ++e) {
        const int32_t b = nleaf[e], rb = leaf_ptr[b], nb = leaf_ptr[b + 1] - rb;
        const double *__restrict__ col = Z + noff[e] + row0 + lane;
        const double *__restrict__ xb = qp + (int64_t)r * n + rb;
        const int32_t j0 = (int32_t)((int64_t)warp * nb / NEAR_WARPS);
        const int32_t j1 = (int32_t)((int64_t)(warp + 1) * nb / NEAR_WARPS);
#pragma unroll 4
        for (int32_t j = j0; j < j1; ++j) {
          const double xj = __ldg(xb + j);
          const double *cj = col + (int64_t)j * na;
#pragma unroll
          for (int rr = 0; rr < NEAR_RB; ++rr)
            if (row0 + lane + 32 * rr < na) acc[rr] = fma(__ldcs(cj + 32 * rr), xj, acc[rr]);
        }
      }
#pragma unroll
    for (int rr = 0; rr < NEAR_RB; ++rr) red[warp][lane + 32 * rr] = acc[rr];
    __syncthreads();
    if (threadIdx.x < NEAR_TROWS && row0 + (int32_t)threadIdx.x < na) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < NEAR_WARPS; ++w) sum += red[w][threadIdx.x];
      yp[(int64_t)r * n + ra + row0 + threadIdx.x] = sum;
    }
    __syncthreads();
  }
}

// Far-field kernels (Eqs. 10-14 in 2D).  Each output block of Q values (a group's
// equivalent charges or potentials) is a sum of column-major matrix columns times
// scalars: a CTA owns the block, its 16 warps split the columns of every matrix between
// them, each lane accumulates the rows k0 + lane + 32 rr (FAR_KR rows, chunks of
// FAR_TROWS rows for larger Q), and the 16 partial sums are added in warp order
// (deterministic).  Every column is one coalesced load per row group.
constexpr int FAR_WARPS = 16, FAR_KR = 4, FAR_TROWS = 32 * FAR_KR;

__device__ __forceinline__ void far_col(double (&acc)[FAR_KR], const double *__restrict__ col, double xj, int k0,
                                        int q, int lane) {
#pragma unroll
  for (int rr = 0; rr < FAR_KR; ++rr) {
    const int k = k0 + lane + 32 * rr;
    if (k < q) acc[rr] = fma(__ldg(col + k), xj, acc[rr]);
  }
}

// columns [w len / 8, (w+1) len / 8) of a q x len panel M (column-major) times x
__device__ __forceinline__ void far_panel(double (&acc)[FAR_KR], const double *__restrict__ M,
                                          const double *__restrict__ x, int len, int k0, int q) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = (int)((int64_t)warp * len / FAR_WARPS), j1 = (int)((int64_t)(warp + 1) * len / FAR_WARPS);
#pragma unroll 4
  for (int j = j0; j < j1; ++j) far_col(acc, M + (int64_t)j * q, __ldg(x + j), k0, q, lane);
}

__device__ __forceinline__ void far_store(double (&acc)[FAR_KR], double (*red)[FAR_TROWS], double *__restrict__ out,
                                          int k0, int q) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int rr = 0; rr < FAR_KR; ++rr) red[warp][lane + 32 * rr] = acc[rr];
  __syncthreads();
  if (threadIdx.x < FAR_TROWS && k0 + (int)threadIdx.x < q) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < FAR_WARPS; ++w) sum += red[w][threadIdx.x];
    out[k0 + threadIdx.x] = sum;
  }
  __syncthreads();
}

// Eq. 10: CTA = leaf b; columns = the leaf's points (V_b is q x |b|, column j at point j)
__global__ void __launch_bounds__(32 * FAR_WARPS) k2_radiate(double *sL, const double *V, const double *qp, int64_t n,
                                                            int nrhs, const int32_t *leaf_ptr, int q) {
  __shared__ double red[FAR_WARPS][FAR_TROWS];
  const int64_t b = blockIdx.x;
  const int32_t r0 = leaf_ptr[b], nb = leaf_ptr[b + 1] - r0;
  const double *Vb = V + (int64_t)q * r0;
  for (int r = 0; r < nrhs; ++r)
    for (int k0 = 0; k0 < q; k0 += FAR_TROWS) {
      double acc[FAR_KR] = {};
      far_panel(acc, Vb, qp + (int64_t)r * n + r0, nb, k0, q);
      far_store(acc, red, sL + (b * nrhs + r) * q, k0, q);
    }
}

// Eq. 11: CTA = parent p at level l-1; columns = every child's q columns of C(quadrant)
__global__ void __launch_bounds__(32 * FAR_WARPS) k2_upward(double *sp, const double *sc, const double *C,
                                                           const int32_t *child_ptr, const int32_t *quad, int nrhs,
                                                           int q) {
  __shared__ double red[FAR_WARPS][FAR_TROWS];
  const int64_t p = blockIdx.x;
  for (int r = 0; r < nrhs; ++r)
    for (int k0 = 0; k0 < q; k0 += FAR_TROWS) {
      double acc[FAR_KR] = {};
      for (int32_t ch = child_ptr[p]; ch < child_ptr[p + 1]; ++ch)
        far_panel(acc, C + (int64_t)quad[ch] * q * q, sc + ((int64_t)ch * nrhs + r) * q, q, k0, q);
      far_store(acc, red, sp + (p * nrhs + r) * q, k0, q);
    }
}

// Eqs. 13 and 12: CTA = box a at level l; columns = B = C^T of its quadrant (stored
// transposed, Ct) on the parent's potentials, then D(offset) on each source of the list
__global__ void __launch_bounds__(32 * FAR_WARPS) k2_translate(double *o, const double *s, const double *D,
                                                              const int32_t *il_ptr, const int32_t *il_src,
                                                              const int32_t *il_slot, const double *op,
                                                              const double *Ct, const int32_t *parent,
                                                              const int32_t *quad, int nrhs, int q) {
  __shared__ double red[FAR_WARPS][FAR_TROWS];
  const int64_t a = blockIdx.x;
  for (int r = 0; r < nrhs; ++r)
    for (int k0 = 0; k0 < q; k0 += FAR_TROWS) {
      double acc[FAR_KR] = {};
      if (op) far_panel(acc, Ct + (int64_t)quad[a] * q * q, op + ((int64_t)parent[a] * nrhs + r) * q, q, k0, q);
      for (int32_t e = il_ptr[a]; e < il_ptr[a + 1]; ++e)
        far_panel(acc, D + (int64_t)il_slot[e] * q * q, s + ((int64_t)il_src[e] * nrhs + r) * q, q, k0, q);
      far_store(acc, red, o + (a * nrhs + r) * q, k0, q);
    }
}

// Eq. 14: 8 lanes per point i: y_i += V(:, i) . o_a (U = V^T, a the leaf of i), the 8
// lanes over the point's q values (contiguous, k = sub + 8 t) and a shuffle reduction in
// fixed order.  The grid runs over all points (32 per CTA), not one CTA per leaf, so
// that enough loads are in flight on every SM; o_a (q values) comes through L1.
__global__ void __launch_bounds__(256) k2_receive(double *__restrict__ yp, const double *__restrict__ oL,
                                                 const double *__restrict__ V, int64_t n, int nrhs,
                                                 const int32_t *__restrict__ pt_leaf, int q) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  const int sub = threadIdx.x & 7;
  const bool on = i < n;
  const int64_t ic = on ? i : 0;
  const double *Vi = V + (int64_t)q * ic;
  const int64_t a = pt_leaf[ic];
  for (int r = 0; r < nrhs; ++r) {
    const double *o = oL + (a * nrhs + r) * q;
    double acc = 0.0;
#pragma unroll 4
    for (int k = sub; k < q; k += 8) acc = fma(__ldg(Vi + k), __ldg(o + k), acc);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, 8);
    if (sub == 0 && on) yp[(int64_t)r * n + i] += acc;
  }
}

static unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 16)); }

static void check(cudaError_t e, const char *what) {
  if (e != cudaSuccess) fail(NESA_ERR_CUDA, std::string("nesa2d: ") + what + ": " + cudaGetErrorString(e));
}

static void ensure_workspace(nesa2d_ctx *c, int nrhs) {
  if (nrhs <= c->nrhs_cap) return;
  auto drop = [&](void *&p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
    p = nullptr;
  };
  drop((void *&)c->d_qp);
  drop((void *&)c->d_yp);
  c->d_qp = (double *)dalloc(c, sizeof(double) * (size_t)c->n * nrhs);
  c->d_yp = (double *)dalloc(c, sizeof(double) * (size_t)c->n * nrhs);
  for (int l = c->l0; l <= c->L; ++l) {
    Level &lv = c->lev[l];
    drop((void *&)lv.s);
    drop((void *&)lv.o);
    lv.s = (double *)dalloc(c, sizeof(double) * (size_t)lv.nbox * nrhs * c->Q);
    lv.o = (double *)dalloc(c, sizeof(double) * (size_t)lv.nbox * nrhs * c->Q);
  }
  c->nrhs_cap = nrhs;
}

static void matvec(nesa2d_ctx *c, const double *q, double *phi, int nrhs, int parts) {
  ensure_workspace(c, nrhs);
  cudaStream_t st = c->stream;
  const int Q = c->Q, L = c->L, l0 = c->l0;
  k2_perm_in<<<grid_of(c->n * nrhs), 256, 0, st>>>(c->d_qp, q, c->d_perm, c->n, nrhs);
  k2_near<<<(unsigned)c->ntile, 32 * NEAR_WARPS, 0, st>>>(c->d_yp, c->d_qp, c->n, nrhs, c->d_leaf_ptr, c->d_nptr,
                                                          c->d_nleaf, c->d_noff, c->d_Z, c->d_tiles,
                                                          (parts & NESA2D_PART_NEAR) ? 1 : 0);
  if (parts & NESA2D_PART_FAR) {
    k2_radiate<<<(unsigned)c->nleaf, 32 * FAR_WARPS, 0, st>>>(c->lev[L].s, c->d_V, c->d_qp, c->n, nrhs,
                                                              c->d_leaf_ptr, Q);
    for (int l = L; l > l0; --l)
      k2_upward<<<(unsigned)c->lev[l - 1].nbox, 32 * FAR_WARPS, 0, st>>>(c->lev[l - 1].s, c->lev[l].s, c->lev[l].C,
                                                             c->lev[l - 1].d_child_ptr, c->lev[l].d_quad, nrhs, Q);
    for (int l = l0; l <= L; ++l) {
      const Level &lv = c->lev[l];
      k2_translate<<<(unsigned)lv.nbox, 32 * FAR_WARPS, 0, st>>>(lv.o, lv.s, lv.D, lv.d_il_ptr, lv.d_il_src,
                                                                 lv.d_il_slot, l > l0 ? c->lev[l - 1].o : nullptr,
                                                                 lv.Ct, lv.d_parent, lv.d_quad, nrhs, Q);
    }
    k2_receive<<<(unsigned)((c->n * 8 + 255) / 256), 256, 0, st>>>(c->d_yp, c->lev[L].o, c->d_V, c->n, nrhs,
                                                                    c->d_pt_leaf, Q);
  }
  k2_perm_out<<<grid_of(c->n * nrhs), 256, 0, st>>>(phi, c->d_yp, c->d_perm, c->n, nrhs);
  check(cudaGetLastError(), "product launch");
}

}  // namespace nesa2d_impl

using namespace nesa2d_impl;

extern "C" {

int nesa2d_build(const double *points, int64_t n, int P, int Q, double pinv_eps, nesa2d_ctx **out) {
  if (!out) return NESA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!points || n < 2 || n > INT32_MAX || P < 1 || Q < 1 || Q > 1024) return NESA_ERR_INVALID_ARG;
  nesa2d_ctx *c = new nesa2d_ctx();
  c->n = n;
  c->P = P;
  c->Q = Q;
  c->pinv_eps = pinv_eps > 0.0 ? pinv_eps : 1e-9;
  try {
    build(c, points);
    check(cudaDeviceSynchronize(), "build");
  } catch (const Error &e) {
    nesa::set_last_error(e.what);
    free_ctx(c);
    return e.status;
  } catch (const std::bad_alloc &) {
    nesa::set_last_error("nesa2d_build: host allocation failed");
    free_ctx(c);
    return NESA_ERR_OOM;
  }
  *out = c;
  return NESA_OK;
}

int nesa2d_set_stream(nesa2d_ctx *c, void *stream) {
  if (!c) return NESA_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return NESA_OK;
}

int nesa2d_get_info(const nesa2d_ctx *c, nesa2d_info *info) {
  if (!c || !info) return NESA_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n_points = c->n;
  info->l0 = c->l0;
  info->L = c->L;
  info->q = c->Q;
  for (int l = c->l0; l <= c->L; ++l) {
    info->n_boxes[l] = c->lev[l].nbox;
    info->n_interactions[l] = (int64_t)c->lev[l].il_src.size();
    info->n_offsets[l] = (int64_t)c->lev[l].offsets.size() / 2;
  }
  info->near_entries = c->near_entries;
  info->device_bytes = (int64_t)c->device_bytes;
  return NESA_OK;
}

int nesa2d_matvec(nesa2d_ctx *c, const double *q, double *phi, int nrhs, int parts) {
  if (!c || !q || !phi || nrhs < 1 || nrhs > 64 || (parts & NESA2D_PART_ALL) == 0 ||
      (parts & ~NESA2D_PART_ALL) != 0 || q == phi)
    return NESA_ERR_INVALID_ARG;
  try {
    matvec(c, q, phi, nrhs, parts);
  } catch (const Error &e) {
    nesa::set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    nesa::set_last_error("nesa2d_matvec: host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

void nesa2d_destroy(nesa2d_ctx *c) { free_ctx(c); }

}  // extern "C"
