// nesa_build and the operator fills (device), plus the small ABI helpers.
//
// What is filled (paper Sec. 2, Eqs. 1-7; Sec. 3, Eqs. 9-14):
//   near field   Z^near_mn = -i eta k sum over the 2x2 triangle pairs of m and n of
//                s s' l l' M_ij(T,T'),   M_ij = sum_{p,q near} w_p w_q g(r_p,r_q)
//                [(r_p - v_i).(r_q - v'_j)/4 - 1/k^2]   (7-point rule per triangle);
//                triangle pairs sharing a vertex take g = (g - 1/(4 pi R)) + 1/(4 pi R)
//                with the 1/R part integrated over T' in closed form;
//   K_l          Tikhonov pseudo-inverse of G(test points, equivalent points);
//   V (radiation) per leaf and RWG column: K_L G(T_L + c, x_p) times the channel
//                coefficients of the points (x, y, z current components and charge);
//   C_l(octant)  K_{l-1} G(T_{l-1}, E_l + delta)  (source transfer; B = C^T);
//   D_l(offset)  G(E_l + offset w_l, E_l)           (translation).
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "nesa_device.cuh"

namespace nesa {

void check_cuda(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) fail(NESA_ERR_OOM, what);
  if (e != cudaSuccess) fail(NESA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
static void check_blas(cublasStatus_t s, const char *what) {
  if (s != CUBLAS_STATUS_SUCCESS) fail(NESA_ERR_CUDA, std::string("cublas ") + what);
}
static void check_solver(cusolverStatus_t s, const char *what) {
  if (s != CUSOLVER_STATUS_SUCCESS) fail(NESA_ERR_CUDA, std::string("cusolver ") + what);
}

void *dalloc(nesa_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  check_cuda(cudaMalloc(&p, bytes), "cudaMalloc");
  c->device_bytes += bytes;
  c->allocs.push_back(p);
  return p;
}

template <typename T>
static T *upload(nesa_ctx *c, const std::vector<T> &v) {
  T *p = (T *)dalloc(c, v.size() * sizeof(T));
  if (!v.empty()) check_cuda(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return p;
}

// Radon's 7-point rule weights (sum to one per triangle).
__constant__ double c_w7[7];

static void set_weights() {
  const double s15 = std::sqrt(15.0);
  double w[7] = {9.0 / 40.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0,
                 (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0};
  check_cuda(cudaMemcpyToSymbol(c_w7, w, sizeof(w)), "weights");
}

// ---------------------------------------------------------------- Green's matrices
// out[a + b*lda] = g(|A_a + shiftA - B_b - shiftB|)   (column-major, rows = observation)
__global__ void k_green_matrix(cplx *out, int64_t lda, const double *A, int na, const double *B, int nb, double k,
                               double sax, double say, double saz, double sbx, double sby, double sbz) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)na * nb) return;
  int a = (int)(idx % na), b = (int)(idx / na);
  double R = dist3(A[3 * a] + sax, A[3 * a + 1] + say, A[3 * a + 2] + saz, B[3 * b] + sbx, B[3 * b + 1] + sby,
                   B[3 * b + 2] + sbz);
  out[a + b * lda] = green(k, R);
}

// D[(s*q + j)*q + i] = g(|e_i + off_s * w - e_j|)
__global__ void k_translation_fill(cplx *D, const double *E, int q, const int32_t *offs, int64_t noff, double w,
                                   double k) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = noff * q * (int64_t)q;
  if (idx >= total) return;
  int i = (int)(idx % q);
  int j = (int)((idx / q) % q);
  int64_t s = idx / ((int64_t)q * q);
  double R = dist3(E[3 * i] + offs[3 * s] * w, E[3 * i + 1] + offs[3 * s + 1] * w, E[3 * i + 2] + offs[3 * s + 2] * w,
                   E[3 * j], E[3 * j + 1], E[3 * j + 2]);
  D[idx] = green(k, R);
}

// Augmented matrix [A; eps I] (3q x q, column-major) from A (2q x q).
__global__ void k_augment(cplx *aug, const cplx *A, int q, double eps) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= 3LL * q * q) return;
  int r = (int)(idx % (3 * q)), c = (int)(idx / (3 * q));
  cplx v = r < 2 * q ? A[r + (int64_t)c * 2 * q] : make_double2(r - 2 * q == c ? eps : 0.0, 0.0);
  aug[idx] = v;
}

// out (cols x rows) = conj(in(rows x cols))^T restricted to the first `rows` rows of in (ld_in)
__global__ void k_conj_transpose(cplx *out, const cplx *in, int rows, int cols, int ld_in) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int r = (int)(idx % rows), c = (int)(idx / rows);
  cplx v = in[r + (int64_t)c * ld_in];
  out[c + (int64_t)r * cols] = make_double2(v.x, -v.y);
}

// out (cols x rows) = in(rows x cols)^T, both column-major
__global__ void k_transpose(cplx *out, const cplx *in, int rows, int cols) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cols) return;
  int r = (int)(idx % rows), c = (int)(idx / rows);
  out[c + (int64_t)r * cols] = in[idx];
}

// copy the upper triangle of the leading q x q block of a (lda) into R (q x q), zero below
__global__ void k_take_r(cplx *R, const cplx *a, int q, int lda) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)q * q) return;
  int r = (int)(idx % q), c = (int)(idx / q);
  R[idx] = r <= c ? a[r + (int64_t)c * lda] : make_double2(0.0, 0.0);
}

// G_all[a + col*2q] = g(|t_a + c_leaf - x_p|), p = leaf_pt[col]
__global__ void k_radiation_green(cplx *G, const double *T, int q2, const double *pts, const int32_t *leaf_pt,
                                  const int32_t *pt_leaf, const double *centers, int64_t ncol, double k) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)q2 * ncol) return;
  int a = (int)(idx % q2);
  int64_t col = idx / q2;
  int32_t p = leaf_pt[col];
  int32_t lf = pt_leaf[p];
  const double *c = centers + 3 * (int64_t)lf;
  double R = dist3(T[3 * a] + c[0], T[3 * a + 1] + c[1], T[3 * a + 2] + c[2], pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]);
  G[idx] = green(k, R);
}

// V[(4g + ch)*q + i] = sum over points p of leaf(g) on a triangle of rwg(g) of P[i + pos(p)*q] a_ch(p)
// a_{x,y,z}(p) = w_p sl (r_p - v_free)/2,  a_rho(p) = w_p sl
__global__ void k_v_fill(cplx *V, const cplx *P, int q, const int32_t *vc_rwg, const int32_t *vc_leaf,
                         const int32_t *leaf_pt_ptr, const int32_t *leaf_pt, const int32_t *rwg_tri,
                         const int32_t *rwg_free, const int32_t *tris, const double *verts, const double *tri_sl,
                         const double *pts) {
  int64_t g = blockIdx.x;
  int32_t n = vc_rwg[g];
  int32_t lf = vc_leaf[g];
  int32_t t0 = rwg_tri[2 * n], t1 = rwg_tri[2 * n + 1];
  for (int i = threadIdx.x; i < q; i += blockDim.x) {
    cplx acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int32_t e = leaf_pt_ptr[lf]; e < leaf_pt_ptr[lf + 1]; ++e) {
      int32_t p = leaf_pt[e];
      int32_t t = p / 7;
      int side = t == t0 ? 0 : (t == t1 ? 1 : -1);
      if (side < 0) continue;
      int fr = rwg_free[2 * n + side];
      double sl = tri_sl[3 * t + fr];
      const double *v = verts + 3 * (int64_t)tris[3 * t + fr];
      double wsl = c_w7[p % 7] * sl;
      cplx pv = P[i + (int64_t)e * q];
      for (int x = 0; x < 3; ++x) {
        double a = 0.5 * wsl * (pts[3 * p + x] - v[x]);
        acc[x].x += pv.x * a;
        acc[x].y += pv.y * a;
      }
      acc[3].x += pv.x * wsl;
      acc[3].y += pv.y * wsl;
    }
    for (int ch = 0; ch < 4; ++ch) V[(4 * g + ch) * q + i] = acc[ch];
  }
}

// ---------------------------------------------------------------- near-field pair matrices
// Closed-form integrals over the flat triangle (p0, p1, p2) seen from r:
//   *I1 = int 1/R dS',  Iv = int (r' - r)/R dS'   (Wilton et al. 1984, Graglia 1993)
__device__ void tri_potentials(const double *p0, const double *p1, const double *p2, const double *r, double *I1,
                               double *Iv) {
  const double *P[3] = {p0, p1, p2};
  double e1[3], e2[3], nrm[3];
  for (int x = 0; x < 3; ++x) {
    e1[x] = p1[x] - p0[x];
    e2[x] = p2[x] - p0[x];
  }
  nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
  nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
  nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double inv = rsqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
  for (int x = 0; x < 3; ++x) nrm[x] *= inv;
  double h = nrm[0] * (r[0] - p0[0]) + nrm[1] * (r[1] - p0[1]) + nrm[2] * (r[2] - p0[2]);
  double ah = fabs(h);
  double rho[3] = {r[0] - h * nrm[0], r[1] - h * nrm[1], r[2] - h * nrm[2]};
  double size2 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
  double sum1 = 0.0, sv[3] = {0.0, 0.0, 0.0};
  for (int ed = 0; ed < 3; ++ed) {
    const double *a = P[ed], *b = P[(ed + 1) % 3];
    double tv[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double il = rsqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]);
    for (int x = 0; x < 3; ++x) tv[x] *= il;
    double u[3] = {tv[1] * nrm[2] - tv[2] * nrm[1], tv[2] * nrm[0] - tv[0] * nrm[2], tv[0] * nrm[1] - tv[1] * nrm[0]};
    double da[3] = {a[0] - rho[0], a[1] - rho[1], a[2] - rho[2]};
    double db[3] = {b[0] - rho[0], b[1] - rho[1], b[2] - rho[2]};
    double sA = da[0] * tv[0] + da[1] * tv[1] + da[2] * tv[2];
    double sB = db[0] * tv[0] + db[1] * tv[1] + db[2] * tv[2];
    double t0 = da[0] * u[0] + da[1] * u[1] + da[2] * u[2];
    double r0sq = t0 * t0 + h * h;
    double RA = sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2] + h * h);
    double RB = sqrt(db[0] * db[0] + db[1] * db[1] + db[2] * db[2] + h * h);
    double lg = 0.0;
    if (r0sq > 1e-28 * size2) {
      if (sA >= 0.0)
        lg = log((RB + sB) / (RA + sA));
      else if (sB <= 0.0)
        lg = log((RA - sA) / (RB - sB));
      else
        lg = log((RB + sB) * (RA - sA) / r0sq);
    }
    double bet = atan2(t0 * sB, r0sq + ah * RB) - atan2(t0 * sA, r0sq + ah * RA);
    sum1 += t0 * lg - ah * bet;
    double cf = 0.5 * (r0sq * lg + sB * RB - sA * RA);
    for (int x = 0; x < 3; ++x) sv[x] += cf * u[x];
  }
  *I1 = sum1;
  for (int x = 0; x < 3; ++x) Iv[x] = sv[x] - h * nrm[x] * sum1;
}

__device__ __forceinline__ bool leaves_touch(const int32_t *a, const int32_t *b) {
  return abs(a[0] - b[0]) <= 1 && abs(a[1] - b[1]) <= 1 && abs(a[2] - b[2]) <= 1;
}

// M[9] (row-major over free vertices of the outer triangle ta and the inner tb).
// singular: extraction of 1/(4 pi R) with the inner integral in closed form.
// must_near: the pair shares a vertex, so all 49 point pairs must lie in touching leaves.
__device__ void pair_block(int32_t ta, int32_t tb, bool singular, bool must_near, const int32_t *tris,
                           const double *verts, const double *pts, const int32_t *pt_ijk, double k, cplx M[9],
                           int *bad) {
  const double *va[3], *vb[3];
  for (int c = 0; c < 3; ++c) {
    va[c] = verts + 3 * (int64_t)tris[3 * ta + c];
    vb[c] = verts + 3 * (int64_t)tris[3 * tb + c];
  }
  // coordinates relative to the first vertex of the outer triangle
  const double o[3] = {va[0][0], va[0][1], va[0][2]};
  double A[3][3], B[3][3];
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) {
      A[c][x] = va[c][x] - o[x];
      B[c][x] = vb[c][x] - o[x];
    }
  // accumulate S = sum ww g, Sp = sum ww g rp, Sq = sum ww g rq, Spq = sum ww g rp.rq
  cplx S = {0, 0}, Spq = {0, 0}, Sp[3] = {{0, 0}, {0, 0}, {0, 0}}, Sq[3] = {{0, 0}, {0, 0}, {0, 0}};
  int nnear = 0;
  for (int p = 0; p < 7; ++p) {
    const double *rp = pts + 3 * (7 * (int64_t)ta + p);
    const int32_t *cp = pt_ijk + 3 * (7 * (int64_t)ta + p);
    double xp[3] = {rp[0] - o[0], rp[1] - o[1], rp[2] - o[2]};
    for (int qq = 0; qq < 7; ++qq) {
      const double *rq = pts + 3 * (7 * (int64_t)tb + qq);
      const int32_t *cq = pt_ijk + 3 * (7 * (int64_t)tb + qq);
      bool near = leaves_touch(cp, cq);
      nnear += near;
      if (!singular && !near) continue;
      double xq[3] = {rq[0] - o[0], rq[1] - o[1], rq[2] - o[2]};
      double R = sqrt((xp[0] - xq[0]) * (xp[0] - xq[0]) + (xp[1] - xq[1]) * (xp[1] - xq[1]) +
                      (xp[2] - xq[2]) * (xp[2] - xq[2]));
      cplx g;
      if (singular) {  // bounded part (exp(-ikR) - 1)/(4 pi R), value -ik/(4 pi) at R = 0
        if (R == 0.0) {
          g = make_double2(0.0, -k * 0.07957747154594767);
        } else {
          double s, c, sh = sin(0.5 * k * R);
          sincos(k * R, &s, &c);
          double f = 0.07957747154594767 / R;
          g = make_double2(-2.0 * sh * sh * f, -s * f);
        }
      } else {
        g = green(k, R);
      }
      double ww = c_w7[p] * c_w7[qq];
      g.x *= ww;
      g.y *= ww;
      S = cadd(S, g);
      double d = xp[0] * xq[0] + xp[1] * xq[1] + xp[2] * xq[2];
      Spq.x += g.x * d;
      Spq.y += g.y * d;
      for (int x = 0; x < 3; ++x) {
        Sp[x].x += g.x * xp[x];
        Sp[x].y += g.y * xp[x];
        Sq[x].x += g.x * xq[x];
        Sq[x].y += g.y * xq[x];
      }
    }
  }
  if (must_near && nnear != 49) atomicExch(bad, 1);
  const double ik2 = 1.0 / (k * k);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // sum ww g (xp - A_i).(xq - B_j) = Spq - A_i.Sq - B_j.Sp + (A_i.B_j) S
      double ab = A[i][0] * B[j][0] + A[i][1] * B[j][1] + A[i][2] * B[j][2];
      cplx v = Spq;
      for (int x = 0; x < 3; ++x) {
        v.x -= A[i][x] * Sq[x].x + B[j][x] * Sp[x].x;
        v.y -= A[i][x] * Sq[x].y + B[j][x] * Sp[x].y;
      }
      v.x += ab * S.x;
      v.y += ab * S.y;
      M[3 * i + j] = make_double2(0.25 * v.x - ik2 * S.x, 0.25 * v.y - ik2 * S.y);
    }
  if (!singular) return;
  // static part: sum_p w_p [ (r_p - a_i).(Iv + (r_p - b_j) I1)/(16 pi A') - I1/(4 pi k^2 A') ]
  double e1[3], e2[3];
  for (int x = 0; x < 3; ++x) {
    e1[x] = B[1][x] - B[0][x];
    e2[x] = B[2][x] - B[0][x];
  }
  double cr0 = e1[1] * e2[2] - e1[2] * e2[1], cr1 = e1[2] * e2[0] - e1[0] * e2[2], cr2 = e1[0] * e2[1] - e1[1] * e2[0];
  double areaB = 0.5 * sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
  const double inv16 = 1.0 / (16.0 * 3.14159265358979323846 * areaB);
  const double inv4k = ik2 / (4.0 * 3.14159265358979323846 * areaB);
  for (int p = 0; p < 7; ++p) {
    const double *rp = pts + 3 * (7 * (int64_t)ta + p);
    double xp[3] = {rp[0] - o[0], rp[1] - o[1], rp[2] - o[2]};
    double I1, Iv[3];
    tri_potentials(B[0], B[1], B[2], xp, &I1, Iv);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int x = 0; x < 3; ++x) acc += (xp[x] - A[i][x]) * (Iv[x] + (xp[x] - B[j][x]) * I1);
        M[3 * i + j].x += c_w7[p] * (acc * inv16 - I1 * inv4k);
      }
  }
}

__device__ __forceinline__ bool share_vertex(const int32_t *a, const int32_t *b) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (a[i] == b[j]) return true;
  return false;
}

// one thread per near triangle pair (CSR by outer triangle)
__global__ void k_pair_matrices(cplx *out, const int64_t *tp_ptr, const int32_t *tp_col, int64_t nt,
                                const int32_t *tris, const double *verts, const double *pts, const int32_t *pt_ijk,
                                double k, int self_only, int *bad) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= tp_ptr[nt]) return;
  // outer triangle: last t with tp_ptr[t] <= e
  int64_t lo = 0, hi = nt;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) / 2;
    if (tp_ptr[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  int32_t ta = (int32_t)lo, tb = tp_col[e];
  // triangles sharing a vertex: singular (extraction) unless only self pairs are
  const bool touching = share_vertex(tris + 3 * ta, tris + 3 * tb);
  const bool sing = touching && (!self_only || ta == tb);
  cplx M[9];
  if (sing && ta > tb) {
    // computed with the lower-numbered triangle outside, then transposed: exact symmetry
    cplx Mt[9];
    pair_block(tb, ta, true, true, tris, verts, pts, pt_ijk, k, Mt, bad);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[3 * i + j] = Mt[3 * j + i];
  } else {
    pair_block(ta, tb, sing, touching, tris, verts, pts, pt_ijk, k, M, bad);
    if (sing && ta == tb)
      for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) {
          cplx s = make_double2(0.5 * (M[3 * i + j].x + M[3 * j + i].x), 0.5 * (M[3 * i + j].y + M[3 * j + i].y));
          M[3 * i + j] = s;
          M[3 * j + i] = s;
        }
  }
  for (int x = 0; x < 9; ++x) out[9 * e + x] = M[x];
}

__device__ __forceinline__ int64_t find_pair(const int64_t *tp_ptr, const int32_t *tp_col, int32_t ta, int32_t tb) {
  int64_t lo = tp_ptr[ta], hi = tp_ptr[ta + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    int32_t v = tp_col[mid];
    if (v == tb) return mid;
    if (v < tb)
      lo = mid + 1;
    else
      hi = mid;
  }
  return -1;
}

// Z^near values: one warp per RWG row, lanes over the row's columns
__global__ void k_near_values(cplx *val, const int64_t *nz_ptr, const int32_t *nz_col, int64_t n,
                              const int32_t *rwg_tri, const int32_t *rwg_free, const double *tri_sl,
                              const int64_t *tp_ptr, const int32_t *tp_col, const cplx *pairM, double pref_im) {
  int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x & 31;
  if (m >= n) return;
  int32_t ta[2] = {rwg_tri[2 * m], rwg_tri[2 * m + 1]};
  int fa[2] = {rwg_free[2 * m], rwg_free[2 * m + 1]};
  for (int64_t e = nz_ptr[m] + lane; e < nz_ptr[m + 1]; e += 32) {
    int32_t c = nz_col[e];
    cplx acc = {0, 0};
    for (int s = 0; s < 2; ++s)
      for (int s2 = 0; s2 < 2; ++s2) {
        int32_t tb = rwg_tri[2 * c + s2];
        int fb = rwg_free[2 * c + s2];
        int64_t pi = find_pair(tp_ptr, tp_col, ta[s], tb);
        if (pi < 0) continue;
        double f = tri_sl[3 * ta[s] + fa[s]] * tri_sl[3 * tb + fb];
        cplx v = pairM[9 * pi + 3 * fa[s] + fb];
        acc.x += f * v.x;
        acc.y += f * v.y;
      }
    // times -i eta k
    val[e] = make_double2(pref_im * acc.y, -pref_im * acc.x);
  }
}

static inline unsigned grid_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Tikhonov pseudo-inverse K (q x 2q) of A = G(T, E) (2q x q), through the QR
// factorisation of [A; eps I]:  K = R^-1 Q1^H.
static void compute_k(nesa_ctx *c, cublasHandle_t hb, cusolverDnHandle_t hs, const cplx *A, int q, double pinv_eps,
                      cplx *K) {
  double fro = 0.0;
  check_blas(cublasDznrm2(hb, 2 * q * q, (const cuDoubleComplex *)A, 1, &fro), "dznrm2");
  double eps = pinv_eps * fro;
  cplx *aug, *tau, *R, *q1h;
  int *info;
  check_cuda(cudaMalloc(&aug, sizeof(cplx) * 3 * (size_t)q * q), "aug");
  check_cuda(cudaMalloc(&tau, sizeof(cplx) * q), "tau");
  check_cuda(cudaMalloc(&R, sizeof(cplx) * (size_t)q * q), "R");
  check_cuda(cudaMalloc(&q1h, sizeof(cplx) * 2 * (size_t)q * q), "q1h");
  check_cuda(cudaMalloc(&info, sizeof(int)), "info");
  k_augment<<<grid_for(3LL * q * q, 256), 256, 0, c->stream>>>(aug, A, q, eps);
  int lw1 = 0, lw2 = 0;
  check_solver(cusolverDnZgeqrf_bufferSize(hs, 3 * q, q, (cuDoubleComplex *)aug, 3 * q, &lw1), "geqrf size");
  check_solver(cusolverDnZungqr_bufferSize(hs, 3 * q, q, q, (cuDoubleComplex *)aug, 3 * q, (cuDoubleComplex *)tau,
                                           &lw2),
               "ungqr size");
  cplx *work;
  int lw = lw1 > lw2 ? lw1 : lw2;
  check_cuda(cudaMalloc(&work, sizeof(cplx) * (size_t)(lw > 0 ? lw : 1)), "work");
  check_solver(cusolverDnZgeqrf(hs, 3 * q, q, (cuDoubleComplex *)aug, 3 * q, (cuDoubleComplex *)tau,
                                (cuDoubleComplex *)work, lw, info),
               "geqrf");
  k_take_r<<<grid_for((int64_t)q * q, 256), 256, 0, c->stream>>>(R, aug, q, 3 * q);
  check_solver(cusolverDnZungqr(hs, 3 * q, q, q, (cuDoubleComplex *)aug, 3 * q, (cuDoubleComplex *)tau,
                                (cuDoubleComplex *)work, lw, info),
               "ungqr");
  // Q1^H: (q x 2q) from the top 2q rows of the 3q x q orthonormal factor
  k_conj_transpose<<<grid_for(2LL * q * q, 256), 256, 0, c->stream>>>(q1h, aug, 2 * q, q, 3 * q);
  cuDoubleComplex one = {1.0, 0.0};
  check_blas(cublasZtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, q, 2 * q,
                         &one, (const cuDoubleComplex *)R, q, (cuDoubleComplex *)q1h, q),
             "ztrsm");
  check_cuda(cudaMemcpyAsync(K, q1h, sizeof(cplx) * 2 * (size_t)q * q, cudaMemcpyDeviceToDevice, c->stream), "K");
  int hinfo = 0;
  check_cuda(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "info");
  check_cuda(cudaStreamSynchronize(c->stream), "sync");
  cudaFree(aug);
  cudaFree(tau);
  cudaFree(R);
  cudaFree(q1h);
  cudaFree(info);
  cudaFree(work);
  if (hinfo != 0) fail(NESA_ERR_NUMERIC, "QR of the equivalent-source fit failed");
}

static void build_device(nesa_ctx *c, const nesa_params &p) {
  HostModel &h = c->h;
  check_cuda(cudaGetDevice(&c->device), "current device");
  c->n = h.n;
  c->nt = h.nt;
  c->np = h.np;
  c->L = h.L;
  c->l0 = h.l0;
  c->nleaf = (int64_t)h.lev[h.L].key.size();
  set_weights();
  cudaStream_t st = c->stream;
  cublasHandle_t hb = nullptr;
  cusolverDnHandle_t hs = nullptr;
  check_blas(cublasCreate(&hb), "create");
  check_solver(cusolverDnCreate(&hs), "create");
  check_blas(cublasSetStream(hb, st), "stream");
  check_solver(cusolverDnSetStream(hs, st), "stream");
  try {
    if (!c->d_pts) c->d_pts = upload(c, h.pts);  // the device tree uploaded these already
    if (!c->d_verts) c->d_verts = upload(c, h.verts);
    if (!c->d_tris) c->d_tris = upload(c, h.tris);
    c->d_tri_rwg = upload(c, h.tri_rwg);
    c->d_tri_sl = upload(c, h.tri_sl);
    c->d_rwg_tri = upload(c, h.rwg_tri);
    c->d_rwg_free = upload(c, h.rwg_free);
    int32_t *d_pt_ijk = upload(c, h.pt_leaf_ijk);

    // ---- near field
    int64_t ntp = h.tp_ptr[h.nt];
    int64_t *d_tp_ptr = upload(c, h.tp_ptr);
    int32_t *d_tp_col = upload(c, h.tp_col);
    cplx *pairM = nullptr;
    check_cuda(cudaMalloc(&pairM, sizeof(cplx) * 9 * (size_t)ntp), "pair matrices");
    int *d_bad = nullptr;
    check_cuda(cudaMalloc(&d_bad, sizeof(int)), "flag");
    check_cuda(cudaMemsetAsync(d_bad, 0, sizeof(int), st), "flag");
    k_pair_matrices<<<grid_for(ntp, 128), 128, 0, st>>>(pairM, d_tp_ptr, d_tp_col, h.nt, c->d_tris, c->d_verts,
                                                        c->d_pts, d_pt_ijk, c->k,
                                                        p.singular_mode == NESA_SINGULAR_SELF ? 1 : 0, d_bad);
    check_cuda(cudaGetLastError(), "pair kernel");
    c->d_nz_ptr = upload(c, h.nz_ptr);
    c->d_nz_col = upload(c, h.nz_col);
    int64_t nnz = h.nz_ptr[h.n];
    c->d_nz_val = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nnz);
    k_near_values<<<grid_for(h.n * 32, 256), 256, 0, st>>>(c->d_nz_val, c->d_nz_ptr, c->d_nz_col, h.n, c->d_rwg_tri,
                                                           c->d_rwg_free, c->d_tri_sl, d_tp_ptr, d_tp_col, pairM,
                                                           c->eta * c->k);
    check_cuda(cudaGetLastError(), "near values kernel");
    int bad = 0;
    check_cuda(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
    check_cuda(cudaStreamSynchronize(st), "near fill");
    cudaFree(pairM);
    cudaFree(d_bad);
    if (bad) fail(NESA_ERR_MESH, "triangles sharing a vertex straddle non-touching leaves: leaf too small");

    // ---- far field structure
    for (int l = 0; l <= h.L; ++l) {
      const HostLevel &hl = h.lev[l];
      DevLevel &dl = c->lev[l];
      dl.nbox = (int64_t)hl.key.size();
      dl.width = hl.width;
      dl.parent = upload(c, hl.parent);
      dl.octant = upload(c, hl.octant);
      dl.child_ptr = upload(c, hl.child_ptr);
      if (l < h.l0) continue;
      dl.q = hl.q;
      dl.nil = (int64_t)hl.il_src.size();
      dl.noff = (int64_t)hl.offsets.size() / 3;
      dl.il_ptr = upload(c, hl.il_ptr);
      dl.il_src = upload(c, hl.il_src);
      dl.il_slot = upload(c, hl.il_slot);
      const int q = hl.q;
      double *d_E = upload(c, hl.eq_pts);
      double *d_T = upload(c, hl.test_pts);
      // K_l
      cplx *A = (cplx *)dalloc(c, sizeof(cplx) * 2 * (size_t)q * q);
      k_green_matrix<<<grid_for(2LL * q * q, 256), 256, 0, st>>>(A, 2 * q, d_T, 2 * q, d_E, q, c->k, 0, 0, 0, 0, 0, 0);
      dl.K = (cplx *)dalloc(c, sizeof(cplx) * 2 * (size_t)q * q);
      compute_k(c, hb, hs, A, q, p.pinv_eps, dl.K);
      // D_l for every offset in use: stored, or generated by the products (Eq. 12's
      // matrices are Green's-function matrices between equivalent points)
      int32_t *d_off = upload(c, hl.offsets);
      const double table_bytes = sizeof(cplx) * (double)dl.noff * q * q;
      dl.gen = c->tables_mode == NESA_TABLES_GENERATED || (c->tables_mode == NESA_TABLES_AUTO && table_bytes > 6e9);
      if (!dl.gen) {
        dl.D = (cplx *)dalloc(c, sizeof(cplx) * (size_t)dl.noff * q * q);
        k_translation_fill<<<grid_for(dl.noff * q * (int64_t)q, 256), 256, 0, st>>>(dl.D, d_E, q, d_off, dl.noff,
                                                                                     hl.width, c->k);
        check_cuda(cudaGetLastError(), "translation fill");
        dl.Ds = (double *)dalloc(c, sizeof(double) * (size_t)dl.noff * q * q);
        plane_sum(c, dl.Ds, dl.D, dl.noff * q * (int64_t)q);
      } else {
        dl.E = d_E;
        dl.offs = d_off;
        // chunks of offset slots whose tables fit a ~1.5 GB work buffer (at most 64)
        const double per_slot = sizeof(cplx) * (double)q * q;
        dl.chunk_slots = (int)std::max<double>(1.0, std::min<double>(64.0, std::floor(1.5e9 / per_slot)));
        dl.chunk_slots = (int)std::min<int64_t>(dl.chunk_slots, std::max<int64_t>(1, dl.noff));
        dl.nchunk = (int)((dl.noff + dl.chunk_slots - 1) / dl.chunk_slots);
        std::vector<int32_t> cptr((size_t)dl.nchunk * (dl.nbox + 1)), csrc(dl.nil), cslot(dl.nil);
        int64_t at = 0;
        for (int ch = 0; ch < dl.nchunk; ++ch) {
          const int32_t s0 = ch * dl.chunk_slots, s1 = s0 + dl.chunk_slots;
          int32_t *ptr = cptr.data() + (size_t)ch * (dl.nbox + 1);
          for (int64_t a = 0; a < dl.nbox; ++a) {
            ptr[a] = (int32_t)at;
            for (int32_t e = hl.il_ptr[a]; e < hl.il_ptr[a + 1]; ++e)
              if (hl.il_slot[e] >= s0 && hl.il_slot[e] < s1) {
                csrc[at] = hl.il_src[e];
                cslot[at] = hl.il_slot[e] - s0;
                ++at;
              }
          }
          ptr[dl.nbox] = (int32_t)at;
        }
        if (at != dl.nil) fail(NESA_ERR_INVALID_ARG, "translation chunks do not cover the interaction lists");
        dl.cil_ptr = upload(c, cptr);
        dl.cil_src = upload(c, csrc);
        dl.cil_slot = upload(c, cslot);
        dl.Dw = (cplx *)dalloc(c, sizeof(cplx) * (size_t)dl.chunk_slots * q * q);
        dl.Dws = (double *)dalloc(c, sizeof(double) * (size_t)dl.chunk_slots * q * q);
      }
      // C_l (l > l0): K_{l-1} G(T_{l-1}, E_l + delta)
      if (l > h.l0) {
        const int qp = h.lev[l - 1].q;
        DevLevel &pl = c->lev[l - 1];
        double *d_Tp = upload(c, h.lev[l - 1].test_pts);
        dl.C = (cplx *)dalloc(c, sizeof(cplx) * 8 * (size_t)qp * q);
        dl.Ct = (cplx *)dalloc(c, sizeof(cplx) * 8 * (size_t)qp * q);
        cplx *G = (cplx *)dalloc(c, sizeof(cplx) * 2 * (size_t)qp * q);
        for (int oc = 0; oc < 8; ++oc) {
          double dx = ((oc & 1) - 0.5) * hl.width, dy = (((oc >> 1) & 1) - 0.5) * hl.width,
                 dz = (((oc >> 2) & 1) - 0.5) * hl.width;
          k_green_matrix<<<grid_for(2LL * qp * q, 256), 256, 0, st>>>(G, 2 * qp, d_Tp, 2 * qp, d_E, q, c->k, 0, 0, 0,
                                                                       dx, dy, dz);
          cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
          cplx *Cm = dl.C + (size_t)oc * qp * q;
          check_blas(cublasZgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, qp, q, 2 * qp, &one, (const cuDoubleComplex *)pl.K, qp,
                                 (const cuDoubleComplex *)G, 2 * qp, &zero, (cuDoubleComplex *)Cm, qp),
                     "zgemm C");
          k_transpose<<<grid_for((int64_t)qp * q, 256), 256, 0, st>>>(dl.Ct + (size_t)oc * qp * q, Cm, qp, q);
        }
        dl.Cs = (double *)dalloc(c, sizeof(double) * 8 * (size_t)qp * q);
        dl.Cts = (double *)dalloc(c, sizeof(double) * 8 * (size_t)qp * q);
        plane_sum(c, dl.Cs, dl.C, 8LL * qp * q);
        plane_sum(c, dl.Cts, dl.Ct, 8LL * qp * q);
        check_cuda(cudaStreamSynchronize(st), "transfer fill");
      }
    }

    // ---- radiation matrices V (leaf level)
    {
      const HostLevel &hl = h.lev[h.L];
      const int q = hl.q;
      std::vector<double> centers(c->nleaf * 3);
      for (int64_t b = 0; b < c->nleaf; ++b)
        for (int x = 0; x < 3; ++x) centers[3 * b + x] = h.origin[x] + (hl.ijk[3 * b + x] + 0.5) * hl.width;
      double *d_centers = upload(c, centers);
      double *d_T = upload(c, hl.test_pts);
      int32_t *d_leaf_pt = upload(c, h.leaf_pt);
      int32_t *d_leaf_pt_ptr = upload(c, h.leaf_pt_ptr);
      int32_t *d_pt_leaf = upload(c, h.pt_leaf);
      c->d_vc_ptr = upload(c, h.vc_ptr);
      for (int64_t b = 0; b < c->nleaf; ++b) c->max_leaf_cols = std::max(c->max_leaf_cols, h.vc_ptr[b + 1] - h.vc_ptr[b]);
      c->d_vc_rwg = upload(c, h.vc_rwg);
      std::vector<int32_t> vc_leaf(h.vc_rwg.size());
      for (int64_t b = 0; b < c->nleaf; ++b)
        for (int32_t g = h.vc_ptr[b]; g < h.vc_ptr[b + 1]; ++g) vc_leaf[g] = (int32_t)b;
      c->d_vc_leaf = upload(c, vc_leaf);
      c->d_rx_ptr = upload(c, h.rx_ptr);
      c->d_rx_col = upload(c, h.rx_col);
      int64_t ncol = (int64_t)h.vc_rwg.size();
      c->d_V = (cplx *)dalloc(c, sizeof(cplx) * 4 * (size_t)ncol * q);
      // points in chunks of leaves so that the temporary G and P stay bounded
      const int64_t chunk_pts = std::max<int64_t>(1, (int64_t)(1LL << 27) / (3LL * q));
      cplx *G = nullptr, *P = nullptr;
      check_cuda(cudaMalloc(&G, sizeof(cplx) * 2 * (size_t)q * std::min<int64_t>(chunk_pts, h.np)), "G");
      check_cuda(cudaMalloc(&P, sizeof(cplx) * (size_t)q * std::min<int64_t>(chunk_pts, h.np)), "P");
      int64_t b0 = 0;
      while (b0 < c->nleaf) {
        int64_t b1 = b0;
        while (b1 < c->nleaf && (h.leaf_pt_ptr[b1 + 1] - h.leaf_pt_ptr[b0]) <= chunk_pts) ++b1;
        if (b1 == b0) fail(NESA_ERR_INVALID_ARG, "leaf holds too many points");
        int64_t p0 = h.leaf_pt_ptr[b0], p1 = h.leaf_pt_ptr[b1];
        int64_t npc = p1 - p0;
        k_radiation_green<<<grid_for(2LL * q * npc, 256), 256, 0, st>>>(G, d_T, 2 * q, c->d_pts, d_leaf_pt + p0,
                                                                         d_pt_leaf, d_centers, npc, c->k);
        cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
        check_blas(cublasZgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, q, (int)npc, 2 * q, &one,
                               (const cuDoubleComplex *)c->lev[h.L].K, q, (const cuDoubleComplex *)G, 2 * q, &zero,
                               (cuDoubleComplex *)P, q),
                   "zgemm P");
        // V columns of these leaves; P is indexed relative to p0
        int64_t g0 = h.vc_ptr[b0], g1 = h.vc_ptr[b1];
        if (g1 > g0) {
          // shift the leaf point pointers so that positions index P
          std::vector<int32_t> lp(h.leaf_pt_ptr.begin(), h.leaf_pt_ptr.end());
          for (auto &x : lp) x -= (int32_t)p0;
          int32_t *d_lp = nullptr;
          check_cuda(cudaMalloc(&d_lp, sizeof(int32_t) * lp.size()), "lp");
          check_cuda(cudaMemcpy(d_lp, lp.data(), sizeof(int32_t) * lp.size(), cudaMemcpyHostToDevice), "lp");
          k_v_fill<<<(unsigned)(g1 - g0), 128, 0, st>>>(c->d_V + 4 * g0 * q, P, q, c->d_vc_rwg + g0,
                                                        c->d_vc_leaf + g0, d_lp, d_leaf_pt + p0, c->d_rwg_tri,
                                                        c->d_rwg_free, c->d_tris, c->d_verts, c->d_tri_sl, c->d_pts);
          check_cuda(cudaGetLastError(), "v fill");
          check_cuda(cudaStreamSynchronize(st), "v fill");
          cudaFree(d_lp);
        }
        b0 = b1;
      }
      cudaFree(G);
      cudaFree(P);
    }
    check_cuda(cudaStreamSynchronize(st), "build");
  } catch (...) {
    cublasDestroy(hb);
    cusolverDnDestroy(hs);
    throw;
  }
  cublasDestroy(hb);
  cusolverDnDestroy(hs);
}

}  // namespace nesa

using namespace nesa;

extern "C" {

void nesa_default_params(nesa_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->leaf_size = 0.25;
  p->n_levels = 3;
  p->q_mode = NESA_Q_AUTO;
  p->q_fixed = 100;
  p->precision = NESA_FP64;
  p->q_digits = 5.0;
  p->rho_eq = 1.0;
  p->rho_test = (2.0 - std::sqrt(3.0) / 2.0) / (std::sqrt(3.0) / 2.0);
  p->pinv_eps = 1e-9;
}

const char *nesa_status_str(int s) {
  switch (s) {
    case NESA_OK: return "ok";
    case NESA_ERR_INVALID_ARG: return "invalid argument";
    case NESA_ERR_MESH: return "invalid mesh";
    case NESA_ERR_CUDA: return "CUDA error";
    case NESA_ERR_OOM: return "out of memory";
    case NESA_ERR_NOT_CONVERGED: return "not converged";
    case NESA_ERR_TIMEOUT: return "device wait timed out";
    case NESA_ERR_NUMERIC: return "numerical breakdown";
    default: return "unknown status";
  }
}

static thread_local std::string g_last_error;
const char *nesa_last_error(void) { return g_last_error.c_str(); }
}  // extern "C"

void nesa::set_last_error(const std::string &what) { g_last_error = what; }

extern "C" {

static void free_ctx(nesa_ctx *c) {
  if (!c) return;
  nesa_free_solve_work(c);
  tc_free(c);
  precond_free(c);
  for (void *p : c->allocs) cudaFree(p);
  for (auto &p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  delete c;
}

static bool build_args_ok(const nesa_mesh *mesh, double k, const nesa_params *params) {
  if (!mesh || !params || !mesh->vertices || !mesh->triangles || mesh->n_vertices < 3 || mesh->n_triangles < 1)
    return false;
  // leaf_size > 0 with n_levels in 1..MAX (or 0: the fewest levels spanning the mesh), or
  // leaf_size = 0 with points_per_leaf > 0 (the depth rule of Sec. 3)
  const bool by_size = params->leaf_size > 0.0 && params->points_per_leaf == 0 && params->n_levels >= 0 &&
                       params->n_levels <= NESA_MAX_LEVELS;
  const bool by_points = params->leaf_size == 0.0 && params->points_per_leaf > 0;
  return (k > 0.0) && (by_size || by_points) &&
         (params->singular_mode == NESA_SINGULAR_TOUCHING || params->singular_mode == NESA_SINGULAR_SELF) &&
         params->translation_tables >= NESA_TABLES_AUTO && params->translation_tables <= NESA_TABLES_GENERATED &&
         (params->q_mode == NESA_Q_FIXED || params->q_mode == NESA_Q_AUTO) && params->q_fixed >= 1 &&
         (params->precision == NESA_FP64 || params->precision == NESA_MIXED) && params->translate >= 0 &&
         params->translate <= 1 &&
         (params->tile_n == 0 || params->tile_n == 64 || params->tile_n == 128 || params->tile_n == 256) &&
         (params->rho_eq > 0.0) && (params->rho_test > params->rho_eq) && (params->pinv_eps >= 0.0) &&
         mesh->n_triangles <= (1LL << 28);
}

// the sizes nesa_info reports that the host model alone determines
static void host_info(const HostModel &h, nesa_info &I) {
  I.n_unknowns = h.n;
  I.n_triangles = h.nt;
  I.n_points = h.np;
  I.n_levels = h.L + 1;
  I.l0 = h.l0;
  for (int l = 0; l <= h.L; ++l) {
    I.q[l] = h.lev[l].q;
    I.n_boxes[l] = (int64_t)h.lev[l].key.size();
    I.n_interactions[l] = (int64_t)h.lev[l].il_src.size();
    I.n_offsets[l] = (int64_t)h.lev[l].offsets.size() / 3;
  }
  I.near_nnz = h.nz_ptr.empty() ? 0 : h.nz_ptr.back();
  I.near_tri_pairs = h.tp_ptr.empty() ? 0 : h.tp_ptr.back();
  I.v_columns = (int64_t)h.vc_rwg.size();
  I.max_leaf_columns = 0;
  for (size_t b = 0; b + 1 < h.vc_ptr.size(); ++b)
    I.max_leaf_columns = std::max<int64_t>(I.max_leaf_columns, h.vc_ptr[b + 1] - h.vc_ptr[b]);
}

int nesa_plan(const nesa_mesh *mesh, double k, const nesa_params *params, nesa_info *info) {
  if (!info || !build_args_ok(mesh, k, params)) return NESA_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  try {
    HostModel h;
    build_host_model(*mesh, k, *params, h);
    std::memset(info, 0, sizeof(*info));
    host_info(h, *info);
  } catch (const Error &e) {
    g_last_error = e.what;
    return e.status;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return NESA_ERR_OOM;
  }
  info->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return NESA_OK;
}

int nesa_build(const nesa_mesh *mesh, double k, const nesa_params *params, nesa_ctx **out) {
  if (!out) return NESA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!build_args_ok(mesh, k, params)) return NESA_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  nesa_ctx *c = new nesa_ctx();
  c->k = k;
  c->tables_mode = params->translation_tables;
  c->translate_engine = params->translate;
  c->eta = 4e-7 * 3.14159265358979323846 * 299792458.0;
  try {
    // the host model with its octree and box lists built on the device
    const auto th0 = std::chrono::steady_clock::now();
    host_mesh(*mesh, c->h);
    check_cuda(cudaGetDevice(&c->device), "current device");
    const auto th1 = std::chrono::steady_clock::now();
    device_tree(c, *params, c->h);
    const auto th2 = std::chrono::steady_clock::now();
    host_level_q(k, *params, c->h);
    host_patterns(c->h);
    const auto th3 = std::chrono::steady_clock::now();
    c->build_split[0] = std::chrono::duration<double>(th1 - th0).count();
    c->build_split[1] = std::chrono::duration<double>(th2 - th1).count();
    c->build_split[2] = std::chrono::duration<double>(th3 - th2).count();
    c->info.near_tri_pairs = c->h.tp_ptr.empty() ? 0 : c->h.tp_ptr.back();
    build_device(c, *params);
    c->build_split[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - th3).count();
    // drop the host arrays that the device copies replace
    c->h.tp_ptr.clear();
    c->h.tp_col.clear();
    c->h.nz_ptr.clear();
    c->h.nz_col.clear();
    c->h.tp_ptr.shrink_to_fit();
    c->h.tp_col.shrink_to_fit();
    c->h.nz_ptr.shrink_to_fit();
    c->h.nz_col.shrink_to_fit();
  } catch (const Error &e) {
    g_last_error = e.what;
    free_ctx(c);
    return e.status;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    free_ctx(c);
    return NESA_ERR_OOM;
  }
  nesa_info &I = c->info;
  I.n_unknowns = c->n;
  I.n_triangles = c->nt;
  I.n_points = c->np;
  I.n_levels = c->L + 1;
  I.l0 = c->l0;
  for (int l = 0; l <= c->L; ++l) {
    I.q[l] = c->lev[l].q;
    I.n_boxes[l] = c->lev[l].nbox;
    I.n_interactions[l] = c->lev[l].nil;
    I.n_offsets[l] = c->lev[l].noff;
  }
  {
    int64_t nnz = 0;
    cudaMemcpy(&nnz, c->d_nz_ptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost);
    I.near_nnz = nnz;
  }
  I.v_columns = (int64_t)c->h.vc_rwg.size();
  I.max_leaf_columns = c->max_leaf_cols;
  if (params->precision == NESA_MIXED) {
    try {
      build_mixed(c);
      if (params->translate == NESA_TRANSLATE_TENSOR) {
        c->autotune = params->tile_n == 0;
        c->fixed_tn = params->tile_n;
        tc_build(c);
      }
    } catch (const Error &e) {
      g_last_error = e.what;
      free_ctx(c);
      return e.status;
    } catch (const std::bad_alloc &) {
      g_last_error = "host allocation failed";
      free_ctx(c);
      return NESA_ERR_OOM;
    }
  }
  I.device_bytes = (int64_t)c->device_bytes;
  I.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < 4; ++i) I.build_split[i] = c->build_split[i];
  *out = c;
  return NESA_OK;
}

void nesa_destroy(nesa_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

int nesa_set_stream(nesa_ctx *c, void *stream) {
  if (!c) return NESA_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return NESA_OK;
}

int nesa_num_unknowns(const nesa_ctx *c, int64_t *n) {
  if (!c || !n) return NESA_ERR_INVALID_ARG;
  *n = c->n;
  return NESA_OK;
}

int nesa_get_info(const nesa_ctx *c, nesa_info *info) {
  if (!c || !info) return NESA_ERR_INVALID_ARG;
  *info = c->info;
  info->device_bytes = (int64_t)c->device_bytes;
  return NESA_OK;
}

int nesa_export(const nesa_ctx *c, int which, void *buf, size_t bytes) {
  if (!c || !buf) return NESA_ERR_INVALID_ARG;
  if (which == NESA_EXPORT_POINT_LEAF) {
    if (bytes != c->h.pt_leaf_ijk.size() * sizeof(int32_t)) return NESA_ERR_INVALID_ARG;
    std::memcpy(buf, c->h.pt_leaf_ijk.data(), bytes);
    return NESA_OK;
  }
  if (which == NESA_EXPORT_RWG) {
    if (bytes != (size_t)c->n * 4 * sizeof(int32_t)) return NESA_ERR_INVALID_ARG;
    int32_t *o = (int32_t *)buf;
    for (int64_t m = 0; m < c->n; ++m) {
      o[4 * m + 0] = c->h.rwg_edge[2 * m];
      o[4 * m + 1] = c->h.rwg_edge[2 * m + 1];
      o[4 * m + 2] = c->h.rwg_tri[2 * m];
      o[4 * m + 3] = c->h.rwg_tri[2 * m + 1];
    }
    return NESA_OK;
  }
  return NESA_ERR_INVALID_ARG;
}

int nesa_export_op(const nesa_ctx *c, int which, int level, int index, void *buf, size_t bytes) {
  if (!c || !buf || index < 0) return NESA_ERR_INVALID_ARG;
  if (level < c->l0 || level > c->L) return NESA_ERR_INVALID_ARG;
  const DevLevel &d = c->lev[level];
  const cplx *src = nullptr;
  size_t need = 0;
  if (which == NESA_OP_D || which == NESA_OP_OFFSET) {
    if (index >= d.noff) return NESA_ERR_INVALID_ARG;
    if (which == NESA_OP_OFFSET) {
      if (bytes != 3 * sizeof(int32_t)) return NESA_ERR_INVALID_ARG;
      std::memcpy(buf, c->h.lev[level].offsets.data() + 3 * (size_t)index, bytes);
      return NESA_OK;
    }
    need = sizeof(cplx) * (size_t)d.q * d.q;
    if (d.gen) {  // generated level: fill the one block into a temporary buffer
      if (bytes != need) return NESA_ERR_INVALID_ARG;
      cplx *tmp = nullptr;
      if (cudaMalloc(&tmp, need) != cudaSuccess) return NESA_ERR_OOM;
      int st = NESA_OK;
      try {
        fill_translations(const_cast<nesa_ctx *>(c), level, index, 1, tmp);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaMemcpy(buf, tmp, need, cudaMemcpyDeviceToHost) != cudaSuccess)
          st = NESA_ERR_CUDA;
      } catch (const Error &e) {
        st = e.status;
      }
      cudaFree(tmp);
      return st;
    }
    src = d.D + (int64_t)index * d.q * d.q;
  } else if (which == NESA_OP_C) {
    if (level == c->l0 || index >= 8) return NESA_ERR_INVALID_ARG;
    const int qp = c->lev[level - 1].q;
    src = d.C + (int64_t)index * qp * d.q;
    need = sizeof(cplx) * (size_t)qp * d.q;
  } else {
    return NESA_ERR_INVALID_ARG;
  }
  if (bytes != need) return NESA_ERR_INVALID_ARG;
  if (need == 0) return NESA_OK;
  if (cudaMemcpy(buf, src, need, cudaMemcpyDeviceToHost) != cudaSuccess) return NESA_ERR_CUDA;
  return NESA_OK;
}

}  // extern "C"
