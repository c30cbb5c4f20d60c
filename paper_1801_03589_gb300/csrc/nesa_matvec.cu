// The NESA matrix-vector product y = Z~ x on the device.
//
// Stages (paper Sec. 3), one kernel launch each (per level where the stage is per level):
//   k_radiate      s_beta = V_beta x_beta                      (Eq. 10)
//   k_upward       s_P    = sum_children C_l(octant) s_child   (Eq. 11, l = L..l0+1)
//   k_translate    o_a    = C_l(octant)^T o_P(a) + sum_{b in IL(a)} D_l(a - b) s_b
//                                                              (Eq. 13 and Eq. 12, l = l0..L)
//   k_near_receive y_m    = sum_n Z^near_mn x_n                (Eq. 9)
//                         + (-i eta k) sum_ch gamma_ch V^T o   (Eq. 14; U = V^T)
// The mixed product with 32 or more right-hand sides splits the last stage in two:
// k_receive_leaf (Eq. 14 per leaf and V column, for 64 right-hand sides at a time) and
// k_near_group (Eq. 9 for four rows at a time, two right-hand sides per lane, plus the
// rows' reception values).
// Every output element is owned by one thread or one warp (no atomics), so the
// product is deterministic.  The kernels are templated on the complex type of the
// operator: complex128 (the FP64 product, bound by the FP64 pipe: a complex
// multiply-add is four FP64 FMAs against 16 bytes of matrix data) and complex64
// (the mixed product's copy, FP32 arithmetic).  x and y are complex128 in both.
//
// Workspace layout per level l >= l0: s_l, o_l = [nbox][4*nrhs][Q_l], column 4r + ch
// holds channel ch (x, y, z, rho) of right-hand side r.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "nesa_device.cuh"

namespace nesa {

void dfree(nesa_ctx *c, void *p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFree(p);
}

// A context captured in a batch keeps its work buffers: products on it use the batch's
// number of right-hand sides until the batch is destroyed.
static void check_batch(const nesa_ctx *c, int nrhs) {
  if (c->batch_refs > 0 && nrhs != c->batch_nrhs)
    fail(NESA_ERR_INVALID_ARG, "context is a member of a batch captured with " + std::to_string(c->batch_nrhs) +
                                   " right-hand sides; destroy the batch before using " + std::to_string(nrhs));
}

int ensure_workspace(nesa_ctx *c, int nrhs) {
  if (nrhs > c->nrhs_cap) {
    check_batch(c, nrhs);
    for (int l = c->l0; l <= c->L; ++l) {
      DevLevel &d = c->lev[l];
      dfree(c, d.s);
      dfree(c, d.o);
      d.s = d.o = nullptr;
      size_t bytes = sizeof(cplx) * (size_t)d.nbox * 4 * nrhs * d.q;
      d.s = (cplx *)dalloc(c, bytes);
      d.o = (cplx *)dalloc(c, bytes);
    }
    c->nrhs_cap = nrhs;
  }
  return NESA_OK;
}

static void build_near_groups(nesa_ctx *c);
// from this many right-hand sides the mixed product's near field and reception run in
// the grouped and per-leaf forms (k_near_group, k_receive_leaf; 16 per CTA below 32)
constexpr int WIDE_MIN_RHS = 16;

static void free_near_groups(nesa_ctx *c) {
  for (void **p : {(void **)&c->d_ng_ptr, (void **)&c->d_ng_loc, (void **)&c->d_ng_val, (void **)&c->d_ng_row,
                   (void **)&c->d_ng_cbp, (void **)&c->d_ng_cb, (void **)&c->d_nb_ptr, (void **)&c->d_nb_col,
                   (void **)&c->d_vc_int}) {
    dfree(c, *p);
    *p = nullptr;
  }
  c->n_group = 0;
}

static void ensure_workspace32(nesa_ctx *c, int nrhs) {
  if (nrhs >= WIDE_MIN_RHS && c->n_group == 0 && c->n > 0) {  // n_group is set last: a failed build leaves it 0
    try {
      build_near_groups(c);
    } catch (...) {
      free_near_groups(c);
      throw;
    }
  }
  if (nrhs <= c->nrhs_cap32) return;
  dfree(c, c->d_xp);
  dfree(c, c->d_rcv);
  c->d_rcv = nullptr;
  // (nrhs + 1) & ~1: the row stride of the wide layout
  c->d_xp = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)std::max<int64_t>(1, c->n * ((nrhs + 1) & ~1)));
  if (nrhs >= WIDE_MIN_RHS) c->d_rcv = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)c->info.v_columns * nrhs);
  for (int l = c->l0; l <= c->L; ++l) {
    DevLevel &d = c->lev[l];
    dfree(c, d.s32);
    dfree(c, d.o32);
    d.s32 = d.o32 = nullptr;
    size_t bytes = sizeof(cplxf) * (size_t)d.nbox * 4 * nrhs * d.q;
    d.s32 = (cplxf *)dalloc(c, bytes);
    d.o32 = (cplxf *)dalloc(c, bytes);
  }
  c->nrhs_cap32 = nrhs;
}

template <typename CT>
__device__ __forceinline__ CT from64(double2 v);
template <>
__device__ __forceinline__ double2 from64<double2>(double2 v) {
  return v;
}
template <>
__device__ __forceinline__ float2 from64<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

// Row tiling of a (Q rows x 4 channels) block: ntile tiles of tr rows, 4*tr threads.
struct Tiling {
  int ntile, tr, threads;
};
static Tiling tiling(int q, int maxt = 512) {
  int ntile = (4 * q + maxt - 1) / maxt;
  int tr = (q + ntile - 1) / ntile;
  int threads = ((4 * tr + 31) / 32) * 32;
  return {ntile, tr, threads};
}
// Row tiling of the FP64 transfers and translations: smaller tiles where a level has
// few boxes, so that the grid holds at least four CTAs per SM (152 SMs); every tile
// stages the whole source column, which costs little against its Q-long row sums.
static Tiling tiling_fp64(int q, int64_t nbox) {
  for (int maxt : {512, 256}) {
    const Tiling t = tiling(q, maxt);
    if (nbox * t.ntile >= 4 * 152) return t;
  }
  return tiling(q, 128);
}

// Source columns pass through shared memory in chunks of JC values per channel, so any
// Q fits (the summation order over j is the same as with the whole column).
constexpr int JC = 512;

// ------------------------------------------------------------------ radiation (Eq. 10)
// Right-hand sides in blocks of RB: every V value is loaded once per block (the x values
// of the block's columns, jc at a time, sit in shared memory as [jc][RB]).  Per
// right-hand side the summation order over the columns is that of one at a time.
template <typename CT, int RB>
__global__ void __launch_bounds__(512) k_radiate(CT *__restrict__ s, const CT *__restrict__ V,
                                                 const int32_t *__restrict__ vc_ptr, const int32_t *__restrict__ vc_rwg,
                                                 const cplx *__restrict__ x, int64_t n, int nrhs, int q, int tr,
                                                 int jc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT *xs = (CT *)smem_raw;  // [jc][RB]
  const int32_t b = blockIdx.x;
  const int tile = blockIdx.y;
  const int ch = threadIdx.x / tr;
  const int i = tile * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < q;
  const int32_t g0 = vc_ptr[b], ns = vc_ptr[b + 1] - g0;
  const CT *Vb = V + (int64_t)4 * g0 * q;
  if constexpr (RB == 1) {  // one right-hand side at a time
    for (int r = 0; r < nrhs; ++r) {
      CT acc = {0, 0};
      for (int j0 = 0; j0 < ns; j0 += jc) {
        const int len = min(jc, ns - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < len; j += blockDim.x)
          xs[j] = from64<CT>(x[(int64_t)r * n + vc_rwg[g0 + j0 + j]]);
        __syncthreads();
        if (!active) continue;
        const CT *vp = Vb + (int64_t)4 * j0 * q + (int64_t)ch * q + i;
#pragma unroll 4
        for (int j = 0; j < len; ++j) cfma(acc, vp[(int64_t)4 * j * q], xs[j]);
      }
      if (active) s[((int64_t)b * 4 * nrhs + 4 * r + ch) * q + i] = acc;
    }
    return;
  }
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int rb = min(RB, nrhs - r0);
    CT acc[RB] = {};
    for (int j0 = 0; j0 < ns; j0 += jc) {
      const int len = min(jc, ns - j0);
      __syncthreads();
      for (int t = threadIdx.x; t < len * RB; t += blockDim.x) {
        const int j = t / RB, rr = t % RB;
        xs[t] = rr < rb ? from64<CT>(x[(int64_t)(r0 + rr) * n + vc_rwg[g0 + j0 + j]]) : CT{};
      }
      __syncthreads();
      if (!active) continue;
      const CT *vp = Vb + (int64_t)4 * j0 * q + (int64_t)ch * q + i;
#pragma unroll 4
      for (int j = 0; j < len; ++j) {
        const CT v = vp[(int64_t)4 * j * q];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr) cfma(acc[rr], v, xs[j * RB + rr]);
      }
    }
    if (active)
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
        if (rr < rb) s[((int64_t)b * 4 * nrhs + 4 * (r0 + rr) + ch) * q + i] = acc[rr];
  }
}

// Radiation of the mixed product with Q even: every thread owns two consecutive rows
// i, i+1 of one channel, so each V access is one 16-byte load (same order over j).
__global__ void __launch_bounds__(512) k_radiate2(cplxf *__restrict__ s, const cplxf *__restrict__ V,
                                                  const int32_t *__restrict__ vc_ptr,
                                                  const int32_t *__restrict__ vc_rwg, const cplx *__restrict__ x,
                                                  int64_t n, int nrhs, int q, int tr2, int jc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplxf *xs = (cplxf *)smem_raw;  // [jc]
  const int32_t b = blockIdx.x;
  const int ch = threadIdx.x / tr2;
  const int i = 2 * (blockIdx.y * tr2 + threadIdx.x % tr2);
  const bool active = ch < 4 && i < q;
  const int32_t g0 = vc_ptr[b], ns = vc_ptr[b + 1] - g0;
  const cplxf *Vb = V + (int64_t)4 * g0 * q;
  for (int r = 0; r < nrhs; ++r) {
    cplxf a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f};
    for (int j0 = 0; j0 < ns; j0 += jc) {
      const int len = min(jc, ns - j0);
      __syncthreads();
      for (int j = threadIdx.x; j < len; j += blockDim.x) {
        const cplx v = x[(int64_t)r * n + vc_rwg[g0 + j0 + j]];
        xs[j] = make_float2((float)v.x, (float)v.y);
      }
      __syncthreads();
      if (!active) continue;
      const cplxf *vp = Vb + (int64_t)4 * j0 * q + (int64_t)ch * q + i;
#pragma unroll 4
      for (int j = 0; j < len; ++j) {
        const float4 v2 = __ldcs((const float4 *)(vp + (int64_t)4 * j * q));
        const cplxf xj = xs[j];
        cfma(a0, make_float2(v2.x, v2.y), xj);
        cfma(a1, make_float2(v2.z, v2.w), xj);
      }
    }
    if (active)
      *(float4 *)(s + ((int64_t)b * 4 * nrhs + 4 * r + ch) * q + i) = make_float4(a0.x, a0.y, a1.x, a1.y);
  }
}

// Radiation of the mixed product with Q even and 8 or more right-hand sides: every
// thread owns two consecutive rows i, i+1 of one channel and RB right-hand sides, so a
// 16-byte V load serves 2 RB complex FMAs and the x values of a column come from shared
// memory as RB/2 16-byte broadcasts (one row per thread took one 8-byte V load per RB
// FMAs).  Per right-hand side the summation order over the columns is that of one at a
// time.
template <int RB>
__global__ void __launch_bounds__(512) k_radiate2w(cplxf *__restrict__ s, const cplxf *__restrict__ V,
                                                   const int32_t *__restrict__ vc_ptr,
                                                   const int32_t *__restrict__ vc_rwg, const cplx *__restrict__ x,
                                                   int64_t n, int nrhs, int q, int tr2, int jc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplxf *xs = (cplxf *)smem_raw;  // [jc][RB]
  const int32_t b = blockIdx.x;
  const int ch = threadIdx.x / tr2;
  const int i = 2 * (blockIdx.y * tr2 + threadIdx.x % tr2);
  const bool active = ch < 4 && i < q;
  const int32_t g0 = vc_ptr[b], ns = vc_ptr[b + 1] - g0;
  const cplxf *Vb = V + (int64_t)4 * g0 * q;
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int rb = min(RB, nrhs - r0);
    cplxf a0[RB], a1[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) a0[rr] = a1[rr] = make_float2(0.0f, 0.0f);
    for (int j0 = 0; j0 < ns; j0 += jc) {
      const int len = min(jc, ns - j0);
      __syncthreads();
      for (int t = threadIdx.x; t < len * RB; t += blockDim.x) {
        const int j = t / RB, rr = t % RB;
        cplxf v = make_float2(0.0f, 0.0f);
        if (rr < rb) {
          const cplx xv = x[(int64_t)(r0 + rr) * n + vc_rwg[g0 + j0 + j]];
          v = make_float2((float)xv.x, (float)xv.y);
        }
        xs[t] = v;
      }
      __syncthreads();
      if (!active) continue;
      const cplxf *vp = Vb + (int64_t)4 * j0 * q + (int64_t)ch * q + i;
#pragma unroll 2
      for (int j = 0; j < len; ++j) {
        const float4 v2 = *(const float4 *)(vp + (int64_t)4 * j * q);
        const cplxf va = make_float2(v2.x, v2.y), vb = make_float2(v2.z, v2.w);
        const float4 *xj = (const float4 *)(xs + j * RB);
#pragma unroll
        for (int h = 0; h < RB / 2; ++h) {
          const float4 x2 = xj[h];
          const cplxf xa = make_float2(x2.x, x2.y), xb = make_float2(x2.z, x2.w);
          cfma(a0[2 * h], va, xa);
          cfma(a1[2 * h], vb, xa);
          cfma(a0[2 * h + 1], va, xb);
          cfma(a1[2 * h + 1], vb, xb);
        }
      }
    }
    if (active)
#pragma unroll
      for (int rr = 0; rr < RB; ++rr)
        if (rr < rb)
          *(float4 *)(s + ((int64_t)b * 4 * nrhs + 4 * (r0 + rr) + ch) * q + i) =
              make_float4(a0[rr].x, a0[rr].y, a1[rr].x, a1[rr].y);
  }
}

// Radiation of the mixed product for many right-hand sides (nrhs >= 32) as a small
// complex product per leaf, s_b = V_b X_b (Eq. 10): a CTA owns 64 of the leaf's 4Q
// rows (ch Q + i) and 64 right-hand sides; thread (warp w, lane l) owns rows 8w .. 8w+7
// of the tile and right-hand sides 2l, 2l + 1.  The leaf's columns pass through shared
// memory RL_KC at a time: V as [column][64 rows] (512 contiguous bytes per column, every
// V value read once per 64 right-hand sides) and x as [column][64 right-hand sides]
// from the permuted complex64 copy xw (512 contiguous bytes per column).  Per column a
// lane reads its x pair with one 16-byte load and its eight V values with four
// broadcast loads, and does 64 FP32 FMAs.  Per output the summation order over the
// columns is that of one column at a time.
constexpr int RL_KC = 32, RL_ROWS = 64;
__global__ void __launch_bounds__(256) k_radiate_leaf(cplxf *__restrict__ s, const cplxf *__restrict__ V,
                                                      const int32_t *__restrict__ vc_ptr,
                                                      const int32_t *__restrict__ vc_int,
                                                      const cplxf *__restrict__ xw, int ldx, int nrhs, int q) {
  __shared__ __align__(16) cplxf Vs[RL_KC][RL_ROWS];
  __shared__ __align__(16) float4 Xs[RL_KC][32];
  const int32_t b = blockIdx.x;
  const int k0 = blockIdx.y * RL_ROWS;  // first row (ch Q + i) of the tile
  const int rb = blockIdx.z * 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q4 = 4 * q;
  const int32_t g0 = vc_ptr[b], ns = vc_ptr[b + 1] - g0;
  cplxf acc[8][2];
#pragma unroll
  for (int m = 0; m < 8; ++m) acc[m][0] = acc[m][1] = make_float2(0.0f, 0.0f);
  for (int j0 = 0; j0 < ns; j0 += RL_KC) {
    const int len = min(RL_KC, ns - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < RL_KC * RL_ROWS; t += blockDim.x) {
      const int j = t / RL_ROWS, rr = t % RL_ROWS;
      Vs[j][rr] = j < len && k0 + rr < q4 ? V[(int64_t)(g0 + j0 + j) * q4 + k0 + rr] : make_float2(0.0f, 0.0f);
    }
    for (int t = threadIdx.x; t < RL_KC * 32; t += blockDim.x) {
      const int j = t >> 5, pc = t & 31;
      Xs[j][pc] = j < len && rb + 2 * pc < ldx
                      ? *(const float4 *)(xw + (int64_t)vc_int[g0 + j0 + j] * ldx + rb + 2 * pc)
                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll 2
    for (int j = 0; j < len; ++j) {
      const float4 x2 = Xs[j][lane];
      const cplxf xa = make_float2(x2.x, x2.y), xb = make_float2(x2.z, x2.w);
      const float4 *vr = (const float4 *)&Vs[j][8 * warp];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 v2 = vr[h];
        const cplxf va = make_float2(v2.x, v2.y), vb = make_float2(v2.z, v2.w);
        cfma(acc[2 * h][0], va, xa);
        cfma(acc[2 * h][1], va, xb);
        cfma(acc[2 * h + 1][0], vb, xa);
        cfma(acc[2 * h + 1][1], vb, xb);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k = k0 + 8 * warp + m;
    if (k >= q4) break;
    const int ch = k / q, i = k % q;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int r = rb + 2 * lane + jj;
      if (r < nrhs) s[((int64_t)b * 4 * nrhs + 4 * r + ch) * q + i] = acc[m][jj];
    }
  }
}

// acc += M[i + j*ld] * col(ch)[j] over j < kdim, with the column (4 channels of kdim
// values at src, channel stride kdim) staged through shared memory in chunks of JC
template <typename CT>
__device__ __forceinline__ void matvec_chunked(CT &acc, CT *col, const CT *__restrict__ src,
                                               const CT *__restrict__ M, int64_t ld, int kdim, int ch, bool active) {
  for (int j0 = 0; j0 < kdim; j0 += JC) {
    const int len = min(JC, kdim - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * len; t += blockDim.x) col[t] = src[(int64_t)(t / len) * kdim + j0 + t % len];
    __syncthreads();
    if (!active) continue;
    const CT *Mj = M + (int64_t)j0 * ld;
    const CT *cs = col + ch * len;
#pragma unroll 4
    for (int j = 0; j < len; ++j) cfma(acc, Mj[(int64_t)j * ld], cs[j]);
  }
}

// ------------------------------------------------------------------ source transfer (Eq. 11)
// parent P at level l-1 (rows qp) gathers its children at level l (rows q)
template <typename CT>
__global__ void __launch_bounds__(512) k_upward(CT *__restrict__ sp, const CT *__restrict__ sc,
                                                const CT *__restrict__ C, const int32_t *__restrict__ child_ptr,
                                                const int32_t *__restrict__ octant, int nrhs, int qp, int q, int tr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT *col = (CT *)smem_raw;  // [4][JC]
  const int32_t P = blockIdx.x;
  const int tile = blockIdx.y;
  const int ch = threadIdx.x / tr;
  const int i = tile * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < qp;
  const int32_t c0 = child_ptr[P], c1 = child_ptr[P + 1];
  for (int r = 0; r < nrhs; ++r) {
    CT acc = {0, 0};
    for (int32_t cb = c0; cb < c1; ++cb)
      matvec_chunked(acc, col, sc + ((int64_t)cb * 4 * nrhs + 4 * r) * q, C + (int64_t)octant[cb] * qp * q + i,
                     qp, q, ch, active);
    if (active) sp[((int64_t)P * 4 * nrhs + 4 * r + ch) * qp + i] = acc;
  }
}

// ------------------------------------------------------------------ translation + potential transfer
template <typename CT>
__global__ void __launch_bounds__(512) k_translate(CT *__restrict__ o, const CT *__restrict__ s,
                                                   const CT *__restrict__ D, const int32_t *__restrict__ il_ptr,
                                                   const int32_t *__restrict__ il_src,
                                                   const int32_t *__restrict__ il_slot, const CT *__restrict__ op,
                                                   const CT *__restrict__ Ct, const int32_t *__restrict__ parent,
                                                   const int32_t *__restrict__ octant, int nrhs, int q, int qp,
                                                   int tr, int accum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT *col = (CT *)smem_raw;  // [4][JC]
  const int32_t a = blockIdx.x;
  const int tile = blockIdx.y;
  const int ch = threadIdx.x / tr;
  const int i = tile * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < q;
  const int32_t e0 = il_ptr[a], e1 = il_ptr[a + 1];
  if (accum && e0 == e1) return;  // a later chunk of offsets without pairs of this box
  for (int r = 0; r < nrhs; ++r) {
    CT acc = {0, 0};
    if (accum && active) acc = o[((int64_t)a * 4 * nrhs + 4 * r + ch) * q + i];  // earlier chunks
    if (op)  // potential transfer from the parent (Eq. 13): o_a += C^T o_P
      matvec_chunked(acc, col, op + ((int64_t)parent[a] * 4 * nrhs + 4 * r) * qp,
                     Ct + (int64_t)octant[a] * q * qp + i, q, qp, ch, active);
    for (int32_t e = e0; e < e1; ++e)  // translations (Eq. 12)
      matvec_chunked(acc, col, s + ((int64_t)il_src[e] * 4 * nrhs + 4 * r) * q, D + (int64_t)il_slot[e] * q * q + i,
                     q, q, ch, active);
    if (active) o[((int64_t)a * 4 * nrhs + 4 * r + ch) * q + i] = acc;
  }
}

// FP64 source transfer, translation and potential transfer with every complex product
// in the 3M (Gauss) form.  For a matrix M = A + iB and a source column u + iv,
//   Re(M x) = A u - B v,   Im(M x) = (A + B)(u + v) - A u - B v,
// so with the sums S = A + B stored beside M (one FP64 plane per matrix, made at build
// time) an entry costs three FMAs per channel instead of the four of the direct form,
// on kernels bound by the FP64 pipe.  Thread (channel ch, row i) as in k_translate (4Q
// threads per box, so nearly every lane works at Q = 100); the source columns pass
// through shared memory as (u, v) and u + v per channel, JC3 columns at a time.  The
// three sums per channel run over the columns in order and are combined once at the end.
constexpr int JC3 = 256;
constexpr size_t SMEM3 = (sizeof(double2) + sizeof(double)) * 4 * JC3;
// (p0, p1, p2) += (A u, B v, S (u + v)) over the kdim columns of M (column j at M + j ld,
// M and MS already offset to this thread's row) and the 4 channels of src (stride kdim)
__device__ __forceinline__ void mv3_chunked(double &p0, double &p1, double &p2, unsigned char *smem,
                                            const double2 *__restrict__ src, const double2 *__restrict__ M,
                                            const double *__restrict__ MS, int64_t ld, int kdim, int ch, bool active) {
  double2 *col = (double2 *)smem;                           // [4][JC3] (u, v)
  double *colw = (double *)(smem + sizeof(double2) * 4 * JC3);  // [4][JC3] u + v
  for (int j0 = 0; j0 < kdim; j0 += JC3) {
    const int len = min(JC3, kdim - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * len; t += blockDim.x) {
      const double2 v = src[(int64_t)(t / len) * kdim + j0 + t % len];
      col[t] = v;
      colw[t] = v.x + v.y;
    }
    __syncthreads();
    if (!active) continue;
    const double2 *cs = col + ch * len;
    const double *cw = colw + ch * len;
    const double2 *Mj = M + (int64_t)j0 * ld;
    const double *Sj = MS + (int64_t)j0 * ld;
#pragma unroll 4
    for (int j = 0; j < len; ++j) {
      const double2 m = Mj[(int64_t)j * ld];
      const double sm = Sj[(int64_t)j * ld];
      const double2 x = cs[j];
      p0 = fma(m.x, x.x, p0);
      p1 = fma(m.y, x.y, p1);
      p2 = fma(sm, cw[j], p2);
    }
  }
}

// Eq. 11: parent P at level l-1 (rows qp) gathers its children at level l (rows q)
__global__ void __launch_bounds__(512) k_upward64(double2 *__restrict__ sp, const double2 *__restrict__ sc,
                                                  const double2 *__restrict__ C, const double *__restrict__ CS,
                                                  const int32_t *__restrict__ child_ptr,
                                                  const int32_t *__restrict__ octant, int nrhs, int qp, int q, int tr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int32_t P = blockIdx.x;
  const int ch = threadIdx.x / tr;
  const int i = blockIdx.y * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < qp;
  const int32_t c0 = child_ptr[P], c1 = child_ptr[P + 1];
  for (int r = 0; r < nrhs; ++r) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (int32_t cb = c0; cb < c1; ++cb)
      mv3_chunked(p0, p1, p2, smem_raw, sc + ((int64_t)cb * 4 * nrhs + 4 * r) * q,
                  C + (int64_t)octant[cb] * qp * q + i, CS + (int64_t)octant[cb] * qp * q + i, qp, q, ch, active);
    if (active) sp[((int64_t)P * 4 * nrhs + 4 * r + ch) * qp + i] = make_double2(p0 - p1, p2 - p0 - p1);
  }
}

// Eqs. 13 and 12: o_a = C^T o_P + sum over the interaction list of D(offset) s_b; a later
// chunk of generated offsets adds its result to o
__global__ void __launch_bounds__(512) k_translate64(double2 *__restrict__ o, const double2 *__restrict__ s,
                                                     const double2 *__restrict__ D, const double *__restrict__ DS,
                                                     const int32_t *__restrict__ il_ptr,
                                                     const int32_t *__restrict__ il_src,
                                                     const int32_t *__restrict__ il_slot, const double2 *__restrict__ op,
                                                     const double2 *__restrict__ Ct, const double *__restrict__ CtS,
                                                     const int32_t *__restrict__ parent,
                                                     const int32_t *__restrict__ octant, int nrhs, int q, int qp, int tr,
                                                     int accum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int32_t a = blockIdx.x;
  const int ch = threadIdx.x / tr;
  const int i = blockIdx.y * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < q;
  const int32_t e0 = il_ptr[a], e1 = il_ptr[a + 1];
  if (accum && e0 == e1) return;  // a later chunk of offsets without pairs of this box
  for (int r = 0; r < nrhs; ++r) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    if (op)  // potential transfer from the parent (Eq. 13): o_a += C^T o_P
      mv3_chunked(p0, p1, p2, smem_raw, op + ((int64_t)parent[a] * 4 * nrhs + 4 * r) * qp,
                  Ct + (int64_t)octant[a] * q * qp + i, CtS + (int64_t)octant[a] * q * qp + i, q, qp, ch, active);
    for (int32_t e = e0; e < e1; ++e)  // translations (Eq. 12)
      mv3_chunked(p0, p1, p2, smem_raw, s + ((int64_t)il_src[e] * 4 * nrhs + 4 * r) * q,
                  D + (int64_t)il_slot[e] * q * q + i, DS + (int64_t)il_slot[e] * q * q + i, q, q, ch, active);
    if (active) {
      double2 *dst = o + ((int64_t)a * 4 * nrhs + 4 * r + ch) * q + i;
      double2 v = make_double2(p0 - p1, p2 - p0 - p1);
      if (accum) {  // earlier chunks
        const double2 w = *dst;
        v = make_double2(w.x + v.x, w.y + v.y);
      }
      *dst = v;
    }
  }
}

// S = Re + Im of every entry (the 3M sums of the FP64 translations)
__global__ void k_plane_sum(double *__restrict__ S, const double2 *__restrict__ D, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    S[e] = D[e].x + D[e].y;
}
void plane_sum(nesa_ctx *c, double *S, const cplx *D, int64_t count) {
  if (count <= 0) return;
  k_plane_sum<<<(unsigned)std::min<int64_t>((count + 255) / 256, 1 << 16), 256, 0, c->stream>>>(S, D, count);
  check_cuda(cudaGetLastError(), "plane sum");
}

// ------------------------------------------------------------------ near field + reception
// One warp per row m.  Right-hand sides go through in blocks of RB, so each near value,
// column index and V column is read once per block; each lane keeps two near entries in
// flight.  The channel weight gamma (1, 1, 1, -1/k^2) is folded into the V value.
template <typename CT, int RB>
__global__ void __launch_bounds__(256) k_near_receive(cplx *__restrict__ y, const cplx *__restrict__ x, int64_t n,
                                                      int nrhs, const int64_t *__restrict__ nz_ptr,
                                                      const int32_t *__restrict__ nz_col,
                                                      const CT *__restrict__ nz_val, const int32_t *__restrict__ rx_ptr,
                                                      const int32_t *__restrict__ rx_col,
                                                      const int32_t *__restrict__ vc_leaf, const CT *__restrict__ V,
                                                      const CT *__restrict__ oL, int q, double eta_k, double inv_k2,
                                                      int parts) {
  using RT = decltype(CT{}.x);
  const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (m >= n) return;
  const int64_t z0 = nz_ptr[m], z1 = nz_ptr[m + 1];
  const int32_t f0 = rx_ptr[m], f1 = rx_ptr[m + 1];
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int rb = min(RB, nrhs - r0);
    CT near[RB] = {}, far[RB] = {};
    if (parts & NESA_PART_NEAR) {
      const cplx *xr = x + (int64_t)r0 * n;
      int64_t e = z0 + lane;
      for (; e + 32 < z1; e += 64) {
        const CT v0 = nz_val[e], v1 = nz_val[e + 32];
        const int32_t k0 = nz_col[e], k1 = nz_col[e + 32];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < rb) {
            cfma(near[rr], v0, from64<CT>(xr[(int64_t)rr * n + k0]));
            cfma(near[rr], v1, from64<CT>(xr[(int64_t)rr * n + k1]));
          }
      }
      if (e < z1) {
        const CT v0 = nz_val[e];
        const int32_t k0 = nz_col[e];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < rb) cfma(near[rr], v0, from64<CT>(xr[(int64_t)rr * n + k0]));
      }
    }
    if (parts & NESA_PART_FAR) {
      for (int32_t e = f0; e < f1; ++e) {
        const int32_t g = rx_col[e];
        const int32_t lf = vc_leaf[g];
        const CT *vg = V + (int64_t)4 * g * q;
        const CT *ol = oL + ((int64_t)lf * 4 * nrhs + 4 * r0) * q;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
          const RT gam = ch < 3 ? (RT)1 : (RT)(-inv_k2);
          for (int i = lane; i < q; i += 32) {
            CT v = vg[ch * q + i];
            v.x *= gam;
            v.y *= gam;
#pragma unroll
            for (int rr = 0; rr < RB; ++rr)
              if (rr < rb) cfma(far[rr], v, ol[(int64_t)(4 * rr + ch) * q + i]);
          }
        }
      }
    }
    // y = near - i eta k far, summed over the warp in FP64
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
      double2 v = make_double2((double)near[rr].x + eta_k * (double)far[rr].y,
                               (double)near[rr].y - eta_k * (double)far[rr].x);
      for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, off);
        v.y += __shfl_down_sync(0xffffffffu, v.y, off);
      }
      if (lane == 0 && rr < rb) y[(int64_t)(r0 + rr) * n + m] = v;
    }
  }
}

// Near field + reception of the mixed product.  Warp r handles the internal row r
// (ABI row m = perm[r]): the near part runs over the padded complex64 CSR with four
// entries per lane and step (16- and 32-byte streaming loads) and gathers x from its
// internal-order complex64 copy xp; reception reads each V column and the leaf's
// outgoing field as contiguous 4Q-value blocks, two values per lane and load.
template <int RB>
__global__ void __launch_bounds__(256) k_near_receive_v(cplx *__restrict__ y, const cplxf *__restrict__ xp, int64_t n,
                                                        int nrhs, const int32_t *__restrict__ perm,
                                                        const int64_t *__restrict__ nz_ptr,
                                                        const int32_t *__restrict__ nz_col,
                                                        const cplxf *__restrict__ nz_val,
                                                        const int32_t *__restrict__ rx_ptr,
                                                        const int32_t *__restrict__ rx_col,
                                                        const int32_t *__restrict__ vc_leaf,
                                                        const cplxf *__restrict__ V, const cplxf *__restrict__ oL,
                                                        int q, double eta_k, double inv_k2, int parts) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const int32_t m = perm[r];
  const int64_t z0 = nz_ptr[r], z1 = nz_ptr[r + 1];
  const int32_t f0 = rx_ptr[m], f1 = rx_ptr[m + 1];
  const int q4 = 4 * q;
  const float mk2 = (float)(-inv_k2);
  for (int r0 = 0; r0 < nrhs; r0 += RB) {
    const int rb = min(RB, nrhs - r0);
    cplxf near[RB] = {}, far[RB] = {};
    if (parts & NESA_PART_NEAR) {
      const cplxf *xr = xp + (int64_t)r0 * n;
      for (int64_t e = z0 + 4 * lane; e < z1; e += 128) {
        const int4 k = __ldcs((const int4 *)(nz_col + e));
        const float4 va = __ldcs((const float4 *)(nz_val + e));
        const float4 vb = __ldcs((const float4 *)(nz_val + e + 2));
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
          if (rr < rb) {
            const cplxf *xq = xr + (int64_t)rr * n;
            cfma(near[rr], make_float2(va.x, va.y), xq[k.x]);
            cfma(near[rr], make_float2(va.z, va.w), xq[k.y]);
            cfma(near[rr], make_float2(vb.x, vb.y), xq[k.z]);
            cfma(near[rr], make_float2(vb.z, vb.w), xq[k.w]);
          }
      }
    }
    if (parts & NESA_PART_FAR) {
      for (int32_t e = f0; e < f1; ++e) {
        const int32_t g = rx_col[e];
        const cplxf *vg = V + (int64_t)g * q4;  // [ch][i]
        const cplxf *ol = oL + ((int64_t)vc_leaf[g] * 4 * nrhs + 4 * r0) * q;
        for (int j = 2 * lane; j < q4; j += 64) {  // values j, j+1 (q4 is even)
          const float4 v2 = __ldcs((const float4 *)(vg + j));
          const float g0 = j < 3 * q ? 1.0f : mk2, g1 = j + 1 < 3 * q ? 1.0f : mk2;
          const cplxf v0 = make_float2(g0 * v2.x, g0 * v2.y), v1 = make_float2(g1 * v2.z, g1 * v2.w);
#pragma unroll
          for (int rr = 0; rr < RB; ++rr)
            if (rr < rb) {
              const float4 o2 = *(const float4 *)(ol + (int64_t)rr * q4 + j);
              cfma(far[rr], v0, make_float2(o2.x, o2.y));
              cfma(far[rr], v1, make_float2(o2.z, o2.w));
            }
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
      double2 v = make_double2((double)near[rr].x + eta_k * (double)far[rr].y,
                               (double)near[rr].y - eta_k * (double)far[rr].x);
      for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, off);
        v.y += __shfl_down_sync(0xffffffffu, v.y, off);
      }
      if (lane == 0 && rr < rb) y[(int64_t)(r0 + rr) * n + m] = v;
    }
  }
}

// Reception of the mixed product for many right-hand sides (nrhs >= 16), one leaf b and
// one group of RW right-hand sides per block, as a small complex product per leaf:
//   R[g][r] = sum_{ch,i} gamma_ch V[g][ch][i] o_b[r][ch][i]       (Eq. 14, U = V^T)
// for the leaf's V columns g (an RWG function has one column per leaf that holds one of
// its triangles; k_near_group adds its columns up).  V and o go through shared memory in
// stages of RC_COLS columns x RC_KC of the 4Q values, copied asynchronously with the next
// stage in flight while this one is used: V as [column][k] (16-byte loads of two k
// values), o as [k][right-hand side] with rows padded by two values (a lane reads its
// two right-hand sides with one 16-byte load; gamma is applied to these o values).
// RW = 64 (32 or more right-hand sides): lane l owns right-hand sides 2l, 2l + 1 and
// warp w the columns w, w + 8, ... (every lane of a warp reads the same V values).
// RW = 16: lane l owns right-hand sides 2 (l mod 8), + 1 and, with the warp, the columns
// 4w + l / 8 + 32 j (four columns per warp at a time; V rows padded by two values so
// that they fall in different banks).  Per pair of k values a lane does 16 FMAs per
// column (RW = 64) or 8 (RW = 16).  FP32 sums in the order k = 0 .. 4Q-1.
constexpr int RC_KC = 32, RC_COLS = 64;
template <int RW>
struct RcShape {
  static constexpr int OPAD = RW + 2, VLD = RW == 64 ? RC_KC : RC_KC + 2;  // row strides of o and V
  static constexpr int VS = RC_COLS * VLD, OS = RC_KC * OPAD;              // complex64 values per stage
  static constexpr int SMEM = 2 * (VS + OS) * 8;
  static constexpr int CPW = RW == 64 ? RC_COLS / 8 : RC_COLS / 32;        // columns per lane per block
};
__device__ __forceinline__ void rc_cp16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void rc_cp8(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
template <int RW>
__global__ void __launch_bounds__(256) k_receive_leaf(cplxf *__restrict__ R, const cplxf *__restrict__ V,
                                                      const cplxf *__restrict__ oL, const int32_t *__restrict__ vc_ptr,
                                                      int nrhs, int q, float mk2) {
  using SH = RcShape<RW>;
  extern __shared__ __align__(16) cplxf rsm[];  // [2][SH::VS + SH::OS]
  const int64_t b = blockIdx.x;
  const int r0 = blockIdx.y * RW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t g0 = vc_ptr[b], ns = vc_ptr[b + 1] - g0;
  const int q4 = 4 * q, q3 = 3 * q;
  const cplxf *ob = oL + b * nrhs * (int64_t)q4;  // o_b[r][ch][i] at ob + r * 4Q + ch * Q + i
  const int pl = RW == 64 ? lane : (lane & 7);    // this lane's right-hand-side pair
  const int ra = r0 + 2 * pl;                     // this lane's right-hand sides ra, ra + 1
  // this lane's first column in a block and the step between its columns
  const int cfirst = RW == 64 ? warp : 4 * warp + (lane >> 3), cstep = RW == 64 ? 8 : 32;
  const int nkc = (q4 + RC_KC - 1) / RC_KC, ncb = (ns + RC_COLS - 1) / RC_COLS, nst = ncb * nkc;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(rsm);
  auto stage = [&](int st) {  // stage st (column block st / nkc, k chunk st % nkc) into buffer st & 1
    const int c0 = (st / nkc) * RC_COLS, k0 = (st % nkc) * RC_KC;
    const int nc = min(RC_COLS, ns - c0), kn = min(RC_KC, q4 - k0);  // kn even (q4 and k0 are)
    cplxf *Vs = rsm + (st & 1) * (SH::VS + SH::OS), *Os = Vs + SH::VS;
    for (int t = threadIdx.x; t < RC_COLS * (RC_KC / 2); t += blockDim.x) {
      const int cc = t / (RC_KC / 2), pc = t % (RC_KC / 2);
      cplxf *dst = Vs + cc * SH::VLD + 2 * pc;
      if (cc < nc && 2 * pc < kn)
        rc_cp16(sbase + (uint32_t)((dst - rsm) * 8), V + (int64_t)(g0 + c0 + cc) * q4 + k0 + 2 * pc);
      else
        *(float4 *)dst = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    for (int t = threadIdx.x; t < RW * RC_KC; t += blockDim.x) {  // coalesced along k
      const int rr = t / RC_KC, kk = t % RC_KC;
      cplxf *dst = Os + kk * SH::OPAD + rr;
      if (r0 + rr < nrhs && kk < kn)
        rc_cp8(sbase + (uint32_t)((dst - rsm) * 8), ob + (int64_t)(r0 + rr) * q4 + k0 + kk);
      else
        *dst = make_float2(0.0f, 0.0f);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  cplxf acc[SH::CPW][2];
  if (nst > 0) stage(0);
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) {
      stage(st + 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const int cb = st / nkc, kc = st % nkc;
    const int c0 = cb * RC_COLS, k0 = kc * RC_KC;
    const int nc = min(RC_COLS, ns - c0);
    const int jn = nc > cfirst ? (nc - cfirst + cstep - 1) / cstep : 0;  // this lane's columns in the block
    if (kc == 0)
#pragma unroll
      for (int j = 0; j < SH::CPW; ++j) acc[j][0] = acc[j][1] = make_float2(0.0f, 0.0f);
    const cplxf *Vs = rsm + (st & 1) * (SH::VS + SH::OS), *Os = Vs + SH::VS;
#pragma unroll 2
    for (int kk = 0; kk < RC_KC; kk += 2) {  // zeros past kn
      const float ga = k0 + kk < q3 ? 1.0f : mk2, gb = k0 + kk + 1 < q3 ? 1.0f : mk2;
      const float4 oa = *(const float4 *)&Os[kk * SH::OPAD + 2 * pl];
      const float4 obk = *(const float4 *)&Os[(kk + 1) * SH::OPAD + 2 * pl];
      const cplxf oa0 = make_float2(ga * oa.x, ga * oa.y), oa1 = make_float2(ga * oa.z, ga * oa.w);
      const cplxf ob0 = make_float2(gb * obk.x, gb * obk.y), ob1 = make_float2(gb * obk.z, gb * obk.w);
#pragma unroll
      for (int j = 0; j < SH::CPW; ++j)
        if (j < jn) {
          const float4 v2 = *(const float4 *)&Vs[(cfirst + cstep * j) * SH::VLD + kk];
          const cplxf va = make_float2(v2.x, v2.y), vb = make_float2(v2.z, v2.w);
          cfma(acc[j][0], va, oa0);
          cfma(acc[j][1], va, oa1);
          cfma(acc[j][0], vb, ob0);
          cfma(acc[j][1], vb, ob1);
        }
    }
    if (kc == nkc - 1)
#pragma unroll
      for (int j = 0; j < SH::CPW; ++j)
        if (j < jn) {
          cplxf *Rg = R + (int64_t)(g0 + c0 + cfirst + cstep * j) * nrhs;
          if (ra < nrhs) Rg[ra] = acc[j][0];
          if (ra + 1 < nrhs) Rg[ra + 1] = acc[j][1];
        }
    __syncthreads();  // every warp is done with this buffer before it is refilled
  }
}

// Near field and reception sum of the mixed product for many right-hand sides
// (nrhs >= 16).  The internal rows come in groups of four whose columns are the union
// of the four rows' columns (a row's value is 0 at a column it lacks), and the groups in
// blocks of eight (one CTA, one warp per group) whose x columns are the union of the
// eight groups' columns.  A CTA serves RW right-hand sides: with RW = 64 (32 or more)
// lane l owns right-hand sides 2l, 2l + 1 and all four rows; with RW = 16 lane l owns
// row l / 8 and right-hand sides 2 (l mod 8), + 1.  The CTA works through its column
// union NS_CH columns at a time; for each chunk it copies into shared memory,
// asynchronously and one chunk ahead of use, the x rows of the chunk's columns (8 RW
// contiguous bytes per column) and, per warp, the values and the in-chunk positions of
// its group's slots in the chunk (their ranges per chunk are precomputed).  Every
// operand of the inner loop then comes from shared memory: per slot a broadcast
// position, a 16-byte x load, the values (two broadcast 16-byte loads, or one 8-byte
// load of the lane's row) and 32 (RW = 64) or 8 (RW = 16) FP32 FMAs.  FP32 sums in slot
// order, converted to FP64; the far part adds the reception values R of the row's V
// columns (k_receive_leaf) times -i eta k.
constexpr int NG_ROWS = 4, NS_GROUPS = 8, NS_CH = 32, NS_VS = NS_CH + 2;
constexpr int NS_VB = NS_GROUPS * NS_VS * 32, NS_LB = NS_GROUPS * NS_VS * 4;
template <int RW>
struct NsShape {
  static constexpr int XB = NS_CH * (RW / 2) * 16;  // x bytes per stage
  static constexpr int SMEM = 2 * (XB + NS_VB + NS_LB);
  static constexpr int RPL = RW == 64 ? NG_ROWS : 1;  // rows per lane
};
__device__ __forceinline__ void ns_cp16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void ns_cp4(uint32_t dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
template <int RW>
__global__ void __launch_bounds__(256) k_near_group(cplx *__restrict__ y, const cplxf *__restrict__ xw, int ldx,
                                                    int64_t n, int nrhs, int64_t n_group,
                                                    const int64_t *__restrict__ g_ptr,
                                                    const int32_t *__restrict__ g_loc,
                                                    const float4 *__restrict__ g_val,
                                                    const int32_t *__restrict__ g_row,
                                                    const int64_t *__restrict__ g_cbp,
                                                    const int32_t *__restrict__ g_cb,
                                                    const int64_t *__restrict__ b_ptr,
                                                    const int32_t *__restrict__ b_col,
                                                    const int32_t *__restrict__ rx_ptr,
                                                    const int32_t *__restrict__ rx_col, const cplxf *__restrict__ R,
                                                    double eta_k, int parts) {
  using SH = NsShape<RW>;
  constexpr int PCS = RW / 2;  // 16-byte pieces of x per column
  extern __shared__ __align__(16) unsigned char nsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t blk = blockIdx.x;
  const int64_t g = blk * NS_GROUPS + warp;
  const bool gon = g < n_group;
  const int rb = blockIdx.y * RW;
  const int pl = RW == 64 ? lane : (lane & 7);  // this lane's right-hand-side pair
  const int il = RW == 64 ? 0 : (lane >> 3);    // this lane's first row in the group
  const int r0 = rb + 2 * pl;                   // this lane's right-hand sides r0, r0 + 1
  cplxf acc[SH::RPL][2];
#pragma unroll
  for (int i = 0; i < SH::RPL; ++i) acc[i][0] = acc[i][1] = make_float2(0.0f, 0.0f);
  if (parts & NESA_PART_NEAR) {
    const int64_t c0 = b_ptr[blk], nu = b_ptr[blk + 1] - c0;
    const int nch = (int)((nu + NS_CH - 1) / NS_CH);
    const int64_t e0 = gon ? g_ptr[g] : 0;
    const int32_t *cb = g_cb + (gon ? g_cbp[g] : 0);  // slot offsets of the chunks' starts, nch + 1
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(nsm);
    // stage k: buffer k & 1 holds x at [buf * XB], values at 2 XB + buf * NS_VB,
    // positions at 2 (XB + NS_VB) + buf * NS_LB
    int cnt0 = 0, cnt1 = 0;                          // slots of this warp's group in buffers 0 and 1
    int32_t nb_c = gon ? cb[0] : 0, nb_n = (gon && nch >= 1) ? cb[1] : 0;  // next chunk to stage
    auto stage = [&](int c) {
      const int buf = c & 1;
      for (int t = threadIdx.x; t < NS_CH * PCS; t += blockDim.x) {
        const int j = t / PCS, pc = t % PCS;  // column j of the chunk, right-hand sides rb + 2 pc, + 1
        const int64_t jj = (int64_t)c * NS_CH + j;
        const uint32_t off = (uint32_t)(buf * SH::XB + (j * PCS + pc) * 16);
        if (jj < nu && rb + 2 * pc < ldx)
          ns_cp16(sbase + off, xw + (int64_t)b_col[c0 + jj] * ldx + rb + 2 * pc);
        else
          *(float4 *)(nsm + off) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
      if (gon) {
        const int cnt = nb_n - nb_c;  // at most NS_CH + 1
        const int64_t sl = e0 + nb_c;
        const uint32_t voff = (uint32_t)(2 * SH::XB + buf * NS_VB + warp * NS_VS * 32);
        const uint32_t loff = (uint32_t)(2 * (SH::XB + NS_VB) + buf * NS_LB + warp * NS_VS * 4);
        for (int t = lane; t < 2 * cnt; t += 32) ns_cp16(sbase + voff + t * 16, g_val + 2 * sl + t);
        for (int t = lane; t < cnt; t += 32) ns_cp4(sbase + loff + t * 4, g_loc + sl + t);
        if (buf)
          cnt1 = cnt;
        else
          cnt0 = cnt;
        nb_c = nb_n;
        nb_n = c + 2 <= nch ? cb[c + 2] : nb_n;  // used by the next stage
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (nch > 0) stage(0);
    for (int c = 0; c < nch; ++c) {
      if (c + 1 < nch) {
        stage(c + 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const int buf = c & 1;
      const int cnt = buf ? cnt1 : cnt0;
      const float4 *xb = (const float4 *)(nsm + buf * SH::XB) + pl;
      const float4 *vb = (const float4 *)(nsm + 2 * SH::XB + buf * NS_VB + warp * NS_VS * 32);
      const int32_t *lb = (const int32_t *)(nsm + 2 * (SH::XB + NS_VB) + buf * NS_LB + warp * NS_VS * 4);
      const int cbase = c * NS_CH;
#pragma unroll 2
      for (int u = 0; u < cnt; ++u) {
        const float4 x2 = xb[(lb[u] - cbase) * PCS];
        const cplxf xa = make_float2(x2.x, x2.y), xb2 = make_float2(x2.z, x2.w);
        if constexpr (RW == 64) {
          const float4 v0 = vb[2 * u], v1 = vb[2 * u + 1];
          const cplxf va[NG_ROWS] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                     make_float2(v1.z, v1.w)};
#pragma unroll
          for (int i = 0; i < NG_ROWS; ++i) {
            cfma(acc[i][0], va[i], xa);
            cfma(acc[i][1], va[i], xb2);
          }
        } else {
          const cplxf v = ((const cplxf *)vb)[NG_ROWS * u + il];
          cfma(acc[0][0], v, xa);
          cfma(acc[0][1], v, xb2);
        }
      }
      __syncthreads();  // every warp is done with this buffer before it is refilled
    }
  }
  if (!gon) return;
  const bool on0 = r0 < nrhs, on1 = r0 + 1 < nrhs;
#pragma unroll
  for (int i = 0; i < SH::RPL; ++i) {
    const int32_t m = g_row[NG_ROWS * g + il + i];
    if (m < 0) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int rr = r0 + j;
      const int rc = rr < nrhs ? rr : 0;
      double2 v = make_double2((double)acc[i][j].x, (double)acc[i][j].y);
      if (parts & NESA_PART_FAR) {
        double fx = 0.0, fy = 0.0;
        for (int32_t e = rx_ptr[m]; e < rx_ptr[m + 1]; ++e) {
          const cplxf f = R[(int64_t)rx_col[e] * nrhs + rc];
          fx += f.x;
          fy += f.y;
        }
        v.x += eta_k * fy;
        v.y -= eta_k * fx;
      }
      if (j == 0 ? on0 : on1) y[(int64_t)rr * n + m] = v;
    }
  }
}

// xw[i][r] = complex64(x[r][perm[i]]) for r < nrhs, 0 for nrhs <= r < ldx   (right-hand
// sides innermost, rows ldx apart, for k_near_group)
__global__ void k_perm_x_wide(cplxf *__restrict__ xw, const cplx *__restrict__ x, const int32_t *__restrict__ perm,
                              int64_t n, int nrhs, int ldx) {
  const int64_t total = n * ldx;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldx, r = t % ldx;  // consecutive threads write consecutive xw
    if (r < nrhs) {
      const cplx v = x[r * n + perm[i]];
      xw[t] = make_float2((float)v.x, (float)v.y);
    } else {
      xw[t] = make_float2(0.0f, 0.0f);
    }
  }
}

// xp[r][i] = complex64(x[r][perm[i]])
__global__ void k_perm_x(cplxf *__restrict__ xp, const cplx *__restrict__ x, const int32_t *__restrict__ perm,
                         int64_t n, int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, i = t % n;
    const cplx v = x[r * n + perm[i]];
    xp[t] = make_float2((float)v.x, (float)v.y);
  }
}

// val4[e] = complex64(val[src[e]]), 0 where src[e] < 0
__global__ void k_gather_near(cplxf *__restrict__ val4, const int64_t *__restrict__ src, const cplx *__restrict__ val,
                              int64_t nnz4) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz4; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = src[e];
    val4[e] = s >= 0 ? make_float2((float)val[s].x, (float)val[s].y) : make_float2(0.0f, 0.0f);
  }
}

static inline unsigned grid_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ generated translations
// D[(s q + j) q + i] = g(|E_i + o_{slot0+s} w - E_j|) for s < ns (Eq. 12), evaluated in FP64
template <typename CT>
__global__ void k_fill_translations(CT *__restrict__ D, const double *__restrict__ E, int q,
                                    const int32_t *__restrict__ offs, int64_t ns, double w, double k) {
  const int64_t total = ns * q * (int64_t)q;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % q);
    const int j = (int)((idx / q) % q);
    const int64_t sl = idx / ((int64_t)q * q);
    const double R = dist3(E[3 * i] + offs[3 * sl] * w, E[3 * i + 1] + offs[3 * sl + 1] * w,
                           E[3 * i + 2] + offs[3 * sl + 2] * w, E[3 * j], E[3 * j + 1], E[3 * j + 2]);
    D[idx] = from64<CT>(green(k, R));
  }
}

template <typename CT>
static void fill_translations_t(nesa_ctx *c, int level, int64_t slot0, int64_t ns, CT *D) {
  const DevLevel &d = c->lev[level];
  if (!d.E || !d.offs) fail(NESA_ERR_INVALID_ARG, "level has no generation data");
  const int64_t total = ns * d.q * (int64_t)d.q;
  k_fill_translations<CT><<<(unsigned)std::min<int64_t>((total + 255) / 256, 1 << 20), 256, 0, c->stream>>>(
      D, d.E, d.q, d.offs + 3 * slot0, ns, d.width, c->k);
  check_cuda(cudaGetLastError(), "fill translations");
}
void fill_translations(nesa_ctx *c, int level, int64_t slot0, int64_t ns, cplx *D) {
  fill_translations_t<cplx>(c, level, slot0, ns, D);
}
void fill_translations(nesa_ctx *c, int level, int64_t slot0, int64_t ns, cplxf *D) {
  fill_translations_t<cplxf>(c, level, slot0, ns, D);
}

// Stage timing: an event before and after a launch when profiling is on.
cudaEvent_t take_event(nesa_ctx *c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  check_cuda(cudaEventCreate(&e), "event");
  return e;
}
struct StageScope {
  nesa_ctx *c;
  int stage;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  StageScope(nesa_ctx *c_, int s, double f, double b) : c(c_), stage(s), flops(f), bytes(b) {
    if (c->profiling) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~StageScope() {
    if (!c->profiling) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({stage, a, b, flops, bytes});
  }
};

// One precision of the product.  Arrays: near values, V, and per level s, o, C, Ct, D.
template <typename CT>
struct OpView {
  const CT *nz_val, *V;
  CT *s[NESA_MAX_LEVELS], *o[NESA_MAX_LEVELS];
  const CT *C[NESA_MAX_LEVELS], *Ct[NESA_MAX_LEVELS], *D[NESA_MAX_LEVELS];
};

template <typename CT>
static void run_product(nesa_ctx *c, const OpView<CT> &op, const cplx *x, cplx *y, int nrhs, int parts) {
  cudaStream_t st = c->stream;
  const int L = c->L, l0 = c->l0;
  const double B = sizeof(CT);
  const double ncol = (double)c->info.v_columns;
  if constexpr (std::is_same<CT, cplxf>::value) {
    if (nrhs >= WIDE_MIN_RHS) {  // x permuted to complex64 [n][ldx] for the near field (and radiation)
      const int ldx = (nrhs + 1) & ~1;
      k_perm_x_wide<<<(unsigned)std::min<int64_t>((c->n * ldx + 255) / 256, 1 << 16), 256, 0, st>>>(
          c->d_xp, x, c->d_perm, c->n, nrhs, ldx);
    }
  }
  if (parts & NESA_PART_FAR) {
    {  // radiation
      DevLevel &d = c->lev[L];
      Tiling t = tiling(d.q);
      const int rbk = nrhs >= 8 ? 8 : 1;  // right-hand sides per V pass
      const int jc = std::min(JC, (int)(32768 / (rbk * sizeof(CT))));
      size_t smem = sizeof(CT) * rbk * (size_t)std::min(jc, std::max(1, c->max_leaf_cols));
      StageScope sc(c, 0, 32.0 * nrhs * ncol * d.q,
                    B * (4.0 * ncol * d.q + 4.0 * nrhs * d.nbox * d.q) + 16.0 * nrhs * c->n);
      bool done = false;
      if constexpr (std::is_same<CT, cplxf>::value) {
        if (nrhs >= 32) {  // per-leaf product on the permuted complex64 x (made before the far part)
          k_radiate_leaf<<<dim3((unsigned)d.nbox, (unsigned)((4 * d.q + RL_ROWS - 1) / RL_ROWS),
                                (unsigned)((nrhs + 63) / 64)),
                           256, 0, st>>>(op.s[L], op.V, c->d_vc_ptr, c->d_vc_int, c->d_xp, (nrhs + 1) & ~1, nrhs,
                                         d.q);
          done = true;
        } else if (d.q % 2 == 0) {  // two rows per thread, 16-byte V loads
          Tiling t2 = tiling(d.q / 2);
          if (rbk == 1)
            k_radiate2<<<dim3((unsigned)d.nbox, t2.ntile), t2.threads, smem, st>>>(
                op.s[L], op.V, c->d_vc_ptr, c->d_vc_rwg, x, c->n, nrhs, d.q, t2.tr, jc);
          else
            k_radiate2w<8><<<dim3((unsigned)d.nbox, t2.ntile), t2.threads, smem, st>>>(
                op.s[L], op.V, c->d_vc_ptr, c->d_vc_rwg, x, c->n, nrhs, d.q, t2.tr, jc);
          done = true;
        }
      }
      if (!done) {
        auto rad = rbk == 8 ? k_radiate<CT, 8> : k_radiate<CT, 1>;
        rad<<<dim3((unsigned)d.nbox, t.ntile), t.threads, smem, st>>>(op.s[L], op.V, c->d_vc_ptr, c->d_vc_rwg, x,
                                                                      c->n, nrhs, d.q, t.tr, jc);
      }
    }
    for (int l = L; l > l0; --l) {  // source transfer
      DevLevel &d = c->lev[l], &p = c->lev[l - 1];
      Tiling t = tiling(p.q);
      size_t smem = sizeof(CT) * 4 * (size_t)std::min(JC, d.q);
      StageScope sc(c, 1, 32.0 * nrhs * d.nbox * (double)p.q * d.q,
                    B * (8.0 * p.q * d.q + 4.0 * nrhs * ((double)d.nbox * d.q + (double)p.nbox * p.q)));
      if constexpr (std::is_same<CT, cplxf>::value) {
        if (c->tc_enabled) {
          tc_upward_level(c, l, op.s[l], op.s[l - 1], nrhs);
          continue;
        }
      }
      if constexpr (std::is_same<CT, cplx>::value) {  // FP64: the 3M form
        const Tiling t3 = tiling_fp64(p.q, p.nbox);
        k_upward64<<<dim3((unsigned)p.nbox, t3.ntile), t3.threads, SMEM3, st>>>(
            op.s[l - 1], op.s[l], op.C[l], d.Cs, p.child_ptr, d.octant, nrhs, p.q, d.q, t3.tr);
      } else
        k_upward<CT><<<dim3((unsigned)p.nbox, t.ntile), t.threads, smem, st>>>(op.s[l - 1], op.s[l], op.C[l],
                                                                               p.child_ptr, d.octant, nrhs, p.q, d.q,
                                                                               t.tr);
    }
    for (int l = l0; l <= L; ++l) {  // translation and potential transfer
      DevLevel &d = c->lev[l];
      Tiling t = tiling(d.q);
      const bool down = l > l0;
      const int qp = down ? c->lev[l - 1].q : 0;
      size_t smem = sizeof(CT) * 4 * (size_t)std::min(JC, std::max(d.q, qp));
      double fl = 32.0 * nrhs * ((double)d.nil * d.q * d.q + (down ? (double)d.nbox * d.q * qp : 0.0));
      double by = B * ((double)d.noff * d.q * d.q + (down ? 8.0 * d.q * qp : 0.0) +
                       4.0 * nrhs * (2.0 * d.nbox * d.q + (down ? (double)c->lev[l - 1].nbox * qp : 0.0)));
      StageScope sc(c, 2, fl, by);
      // FP64: k_translate64 (3M form with the stored sums); complex64 (the CUDA-core
      // engine of the mixed product): k_translate
      auto translate = [&](const CT *Dm, const double *DSm, const int32_t *ptr, const int32_t *src,
                           const int32_t *slot, bool with_parent, int accum) {
        if constexpr (std::is_same<CT, cplx>::value) {
          const Tiling t3 = tiling_fp64(d.q, d.nbox);
          k_translate64<<<dim3((unsigned)d.nbox, t3.ntile), t3.threads, SMEM3, st>>>(
              op.o[l], op.s[l], Dm, DSm, ptr, src, slot, with_parent ? op.o[l - 1] : nullptr,
              with_parent ? op.Ct[l] : nullptr, with_parent ? d.Cts : nullptr, d.parent, d.octant, nrhs, d.q, qp,
              t3.tr, accum);
        } else {
          k_translate<CT><<<dim3((unsigned)d.nbox, t.ntile), t.threads, smem, st>>>(
              op.o[l], op.s[l], Dm, ptr, src, slot, with_parent ? op.o[l - 1] : nullptr,
              with_parent ? op.Ct[l] : nullptr, d.parent, d.octant, nrhs, d.q, qp, t.tr, accum);
        }
      };
      if constexpr (std::is_same<CT, cplxf>::value) {
        if (c->tc_enabled) {
          tc_translate_level(c, l, op.s[l], op.o[l], down ? op.o[l - 1] : nullptr, down ? op.Ct[l] : nullptr, nrhs);
          continue;
        }
      }
      if (d.gen) {  // translation matrices built chunk by chunk into the work buffer
        CT *Dw = nullptr;
        if constexpr (std::is_same<CT, cplx>::value)
          Dw = d.Dw;
        else
          Dw = d.Dw32;
        if (!Dw) fail(NESA_ERR_INVALID_ARG, "generated level without a work buffer for this precision");
        for (int chk = 0; chk < d.nchunk; ++chk) {
          const int64_t slot0 = (int64_t)chk * d.chunk_slots, ns = std::min<int64_t>(d.chunk_slots, d.noff - slot0);
          fill_translations(c, l, slot0, ns, Dw);
          if constexpr (std::is_same<CT, cplx>::value) plane_sum(c, d.Dws, Dw, ns * d.q * (int64_t)d.q);
          translate(Dw, d.Dws, d.cil_ptr + (int64_t)chk * (d.nbox + 1), d.cil_src, d.cil_slot, down && chk == 0,
                    chk > 0 ? 1 : 0);
        }
        continue;
      }
      translate(op.D[l], d.Ds, d.il_ptr, d.il_src, d.il_slot, down, 0);
    }
  }
  const DevLevel &dL = c->lev[L];
  const double nnz = (double)c->info.near_nnz;
  double fl = ((parts & NESA_PART_NEAR) ? 8.0 * nrhs * nnz : 0.0) +
              ((parts & NESA_PART_FAR) ? 32.0 * nrhs * ncol * dL.q : 0.0);
  double by = ((parts & NESA_PART_NEAR) ? (B + 4.0) * nnz + 8.0 * (c->n + 1) : 0.0) +
              ((parts & NESA_PART_FAR) ? B * 4.0 * ncol * dL.q + B * 4.0 * nrhs * dL.nbox * dL.q : 0.0) +
              16.0 * 2.0 * nrhs * c->n;
  StageScope sc(c, 3, fl, by);
  if constexpr (std::is_same<CT, cplxf>::value) {
    const unsigned pgrid = (unsigned)std::min<int64_t>((c->n * nrhs + 255) / 256, 1 << 16);
    if (nrhs >= WIDE_MIN_RHS) {  // many right-hand sides: groups of four rows, two right-hand sides per lane
      const int ldx = (nrhs + 1) & ~1;  // xw was made before the far part
      const float mk2 = (float)(-1.0 / (c->k * c->k));
      if (parts & NESA_PART_FAR) {
        if (nrhs >= 32)
          k_receive_leaf<64><<<dim3((unsigned)c->nleaf, (unsigned)((nrhs + 63) / 64)), 256, RcShape<64>::SMEM, st>>>(
              c->d_rcv, op.V, op.o[L], c->d_vc_ptr, nrhs, dL.q, mk2);
        else
          k_receive_leaf<16><<<dim3((unsigned)c->nleaf, (unsigned)((nrhs + 15) / 16)), 256, RcShape<16>::SMEM, st>>>(
              c->d_rcv, op.V, op.o[L], c->d_vc_ptr, nrhs, dL.q, mk2);
      }
      if (c->n_group > 0) {
        const int rw = nrhs >= 32 ? 64 : 16;
        const dim3 grid((unsigned)((c->n_group + NS_GROUPS - 1) / NS_GROUPS), (unsigned)((nrhs + rw - 1) / rw));
        auto kern = nrhs >= 32 ? k_near_group<64> : k_near_group<16>;
        kern<<<grid, 32 * NS_GROUPS, nrhs >= 32 ? NsShape<64>::SMEM : NsShape<16>::SMEM, st>>>(
            y, c->d_xp, ldx, c->n, nrhs, c->n_group, c->d_ng_ptr, c->d_ng_loc, (const float4 *)c->d_ng_val,
            c->d_ng_row, c->d_ng_cbp, c->d_ng_cb, c->d_nb_ptr, c->d_nb_col, c->d_rx_ptr, c->d_rx_col, c->d_rcv,
            c->eta * c->k, parts);
      }
    } else {
      if (parts & NESA_PART_NEAR) k_perm_x<<<pgrid, 256, 0, st>>>(c->d_xp, x, c->d_perm, c->n, nrhs);
      auto near = nrhs == 1 ? k_near_receive_v<1> : k_near_receive_v<4>;
      near<<<grid_for(c->n * 32, 256), 256, 0, st>>>(y, c->d_xp, c->n, nrhs, c->d_perm, c->d_nz_ptr4, c->d_nz_col4,
                                                    op.nz_val, c->d_rx_ptr, c->d_rx_col, c->d_vc_leaf, op.V, op.o[L],
                                                    dL.q, c->eta * c->k, 1.0 / (c->k * c->k), parts);
    }
  } else {
    auto near = nrhs == 1 ? k_near_receive<CT, 1> : k_near_receive<CT, 4>;
    near<<<grid_for(c->n * 32, 256), 256, 0, st>>>(y, x, c->n, nrhs, c->d_nz_ptr, c->d_nz_col, op.nz_val,
                                                  c->d_rx_ptr, c->d_rx_col, c->d_vc_leaf, op.V, op.o[L], dL.q,
                                                  c->eta * c->k, 1.0 / (c->k * c->k), parts);
  }
}

// Launch the product on the context's stream.
void launch_matvec(nesa_ctx *c, const cplx *x, cplx *y, int nrhs, int parts) {
  check_batch(c, nrhs);
  if (parts & NESA_PART_MIXED) {
    if (!c->mixed) fail(NESA_ERR_INVALID_ARG, "context was not built with NESA_MIXED");
    ensure_workspace32(c, nrhs);
    OpView<cplxf> op{};
    op.nz_val = c->d_nz_val32;
    op.V = c->d_V32;
    for (int l = c->l0; l <= c->L; ++l) {
      op.s[l] = c->lev[l].s32;
      op.o[l] = c->lev[l].o32;
      op.C[l] = c->lev[l].C32;
      op.Ct[l] = c->lev[l].Ct32;
      op.D[l] = c->lev[l].D32;
    }
    run_product<cplxf>(c, op, x, y, nrhs, parts & NESA_PART_ALL);
    return;
  }
  OpView<cplx> op{};
  op.nz_val = c->d_nz_val;
  op.V = c->d_V;
  for (int l = c->l0; l <= c->L; ++l) {
    op.s[l] = c->lev[l].s;
    op.o[l] = c->lev[l].o;
    op.C[l] = c->lev[l].C;
    op.Ct[l] = c->lev[l].Ct;
    op.D[l] = c->lev[l].D;
  }
  run_product<cplx>(c, op, x, y, nrhs, parts & NESA_PART_ALL);
}

// ------------------------------------------------------------------ mixed-precision copies
__global__ void k_to_c64(cplxf *dst, const cplx *src, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    cplx v = src[e];
    dst[e] = make_float2((float)v.x, (float)v.y);
  }
}

static cplxf *copy_c64(nesa_ctx *c, const cplx *src, int64_t n) {
  cplxf *d = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)std::max<int64_t>(n, 1));
  if (n > 0) k_to_c64<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65536), 256, 0, c->stream>>>(d, src, n);
  return d;
}

// Near field of the mixed product in the internal order: RWG functions sorted (stably)
// by the leaf of their first quadrature point, leaves in Morton order, so that the
// near columns of a row form a few contiguous runs and neighbouring rows share them.
// Rows are padded to multiples of 4 entries; columns are renumbered and sorted.
static void build_near_internal(nesa_ctx *c) {
  const HostModel &h = c->h;
  const int64_t n = c->n;
  // the near pattern lives on the device only (the host copy is released after upload)
  std::vector<int64_t> nz_ptr(n + 1);
  check_cuda(cudaMemcpy(nz_ptr.data(), c->d_nz_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost), "near ptr");
  std::vector<int32_t> nz_col(std::max<int64_t>(nz_ptr[n], 1));
  check_cuda(cudaMemcpy(nz_col.data(), c->d_nz_col, sizeof(int32_t) * nz_ptr[n], cudaMemcpyDeviceToHost), "near col");
  std::vector<int32_t> perm(n), inv(n);
  for (int64_t m = 0; m < n; ++m) perm[m] = (int32_t)m;
  auto leaf_of = [&](int32_t m) { return h.pt_leaf[7 * (int64_t)h.rwg_tri[2 * (int64_t)m]]; };
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return leaf_of(a) < leaf_of(b); });
  for (int64_t r = 0; r < n; ++r) inv[perm[r]] = (int32_t)r;
  std::vector<int64_t> ptr4(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    const int32_t m = perm[r];
    ptr4[r + 1] = ptr4[r] + ((nz_ptr[m + 1] - nz_ptr[m] + 3) / 4) * 4;
  }
  const int64_t nnz4 = std::max<int64_t>(ptr4[n], 4);
  std::vector<int32_t> col4(nnz4, 0);
  std::vector<int64_t> src(nnz4, -1);
  auto fill_rows = [&](int64_t r_begin, int64_t r_end) {
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int64_t r = r_begin; r < r_end; ++r) {
      const int32_t m = perm[r];
      const int64_t s0 = nz_ptr[m], len = nz_ptr[m + 1] - s0;
      row.resize(len);
      for (int64_t j = 0; j < len; ++j) row[j] = {inv[nz_col[s0 + j]], s0 + j};
      std::sort(row.begin(), row.end());
      const int64_t p = ptr4[r];
      for (int64_t j = 0; j < len; ++j) {
        col4[p + j] = row[j].first;
        src[p + j] = row[j].second;
      }
      const int32_t last = len > 0 ? row[len - 1].first : (int32_t)r;
      for (int64_t j = len; j < ptr4[r + 1] - p; ++j) col4[p + j] = last;
    }
  };
  const int nth = (int)std::max<unsigned>(1, std::min<unsigned>(16, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t) pool.emplace_back(fill_rows, n * t / nth, n * (t + 1) / nth);
  for (auto &th : pool) th.join();
  c->d_perm = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<int64_t>(n, 1));
  c->d_nz_ptr4 = (int64_t *)dalloc(c, sizeof(int64_t) * (n + 1));
  c->d_nz_col4 = (int32_t *)dalloc(c, sizeof(int32_t) * nnz4);
  c->d_nz_val32 = (cplxf *)dalloc(c, sizeof(cplxf) * nnz4);
  int64_t *d_src = (int64_t *)dalloc(c, sizeof(int64_t) * nnz4);
  check_cuda(cudaMemcpy(c->d_perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice), "near order");
  check_cuda(cudaMemcpy(c->d_nz_ptr4, ptr4.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice), "near order");
  check_cuda(cudaMemcpy(c->d_nz_col4, col4.data(), sizeof(int32_t) * nnz4, cudaMemcpyHostToDevice), "near order");
  check_cuda(cudaMemcpy(d_src, src.data(), sizeof(int64_t) * nnz4, cudaMemcpyHostToDevice), "near order");
  k_gather_near<<<(unsigned)std::min<int64_t>((nnz4 + 255) / 256, 1 << 16), 256, 0, c->stream>>>(
      c->d_nz_val32, d_src, c->d_nz_val, nnz4);
  check_cuda(cudaStreamSynchronize(c->stream), "near order");
  dfree(c, d_src);
}

// dst[e] = src[idx[e]], 0 where idx[e] < 0
__global__ void k_gather_c64(cplxf *__restrict__ dst, const int64_t *__restrict__ idx, const cplxf *__restrict__ src,
                             int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx[e];
    dst[e] = s >= 0 ? src[s] : make_float2(0.0f, 0.0f);
  }
}

// The near field of the mixed product regrouped for many right-hand sides (k_near_group).
// Within the internal rows of one leaf (rows whose first quadrature point lies in it),
// rows are ordered by their column lists, so that rows with the same list (RWG functions
// whose quadrature points lie in the same leaves) sit next to each other; then every
// four consecutive rows form a group over the union of their columns, and every eight
// consecutive groups a block over the union of the groups' columns.  A slot stores the
// position of its column in the block's union.  The values are the complex64 values of
// the padded CSR, gathered on the device; the zeros a row gets at columns it lacks
// change none of its sums.
static void build_near_groups(nesa_ctx *c) {
  const HostModel &h = c->h;
  const int64_t n = c->n;
  std::vector<int64_t> ptr4(n + 1);
  std::vector<int32_t> perm(std::max<int64_t>(n, 1));
  check_cuda(cudaMemcpy(ptr4.data(), c->d_nz_ptr4, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost), "near groups");
  check_cuda(cudaMemcpy(perm.data(), c->d_perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost), "near groups");
  {  // internal index of each V column's RWG function (the radiation's x rows)
    std::vector<int32_t> inv(std::max<int64_t>(n, 1)), vint(std::max<size_t>(h.vc_rwg.size(), 1));
    for (int64_t r = 0; r < n; ++r) inv[perm[r]] = (int32_t)r;
    for (size_t g = 0; g < h.vc_rwg.size(); ++g) vint[g] = inv[h.vc_rwg[g]];
    c->d_vc_int = (int32_t *)dalloc(c, sizeof(int32_t) * vint.size());
    check_cuda(cudaMemcpy(c->d_vc_int, vint.data(), sizeof(int32_t) * vint.size(), cudaMemcpyHostToDevice),
               "near groups");
  }
  const int64_t nnz4 = ptr4[n];
  std::vector<int32_t> col4(std::max<int64_t>(nnz4, 1));
  if (nnz4 > 0)
    check_cuda(cudaMemcpy(col4.data(), c->d_nz_col4, sizeof(int32_t) * nnz4, cudaMemcpyDeviceToHost), "near groups");
  // a row's true length: its padded tail repeats the last column
  auto row_len = [&](int64_t r) {
    int64_t e = ptr4[r + 1];
    while (e - 1 > ptr4[r] && col4[e - 1] == col4[e - 2]) --e;
    return e - ptr4[r];
  };
  // order the rows of each leaf by their column lists
  std::vector<int64_t> order(n);
  for (int64_t r = 0; r < n; ++r) order[r] = r;
  auto leaf_of = [&](int64_t r) { return h.pt_leaf[7 * (int64_t)h.rwg_tri[2 * (int64_t)perm[r]]]; };
  for (int64_t r0 = 0; r0 < n;) {
    int64_t r1 = r0 + 1;
    while (r1 < n && leaf_of(r1) == leaf_of(r0)) ++r1;
    std::stable_sort(order.begin() + r0, order.begin() + r1, [&](int64_t a, int64_t b) {
      const int32_t *pa = col4.data() + ptr4[a], *pb = col4.data() + ptr4[b];
      return std::lexicographical_compare(pa, pa + row_len(a), pb, pb + row_len(b));
    });
    r0 = r1;
  }
  const int64_t ng = (n + NG_ROWS - 1) / NG_ROWS;
  // union of each group's columns (ascending), padded to an even count
  std::vector<std::vector<int32_t>> ucol(ng);
  auto unions = [&](int64_t g0, int64_t g1) {
    for (int64_t g = g0; g < g1; ++g) {
      std::vector<int32_t> &u = ucol[g];
      for (int i = 0; i < NG_ROWS && g * NG_ROWS + i < n; ++i) {
        const int64_t r = order[g * NG_ROWS + i];
        u.insert(u.end(), col4.begin() + ptr4[r], col4.begin() + ptr4[r] + row_len(r));
      }
      std::sort(u.begin(), u.end());
      u.erase(std::unique(u.begin(), u.end()), u.end());
      if (u.empty()) u.push_back(0);
      if (u.size() & 1) u.push_back(u.back());
    }
  };
  const int nth = (int)std::max<unsigned>(1, std::min<unsigned>(16, std::thread::hardware_concurrency()));
  auto run_threads = [&](auto &&fn, int64_t count) {
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t) pool.emplace_back(fn, count * t / nth, count * (t + 1) / nth);
    for (auto &th : pool) th.join();
  };
  run_threads(unions, ng);
  std::vector<int64_t> gptr(ng + 1, 0);
  for (int64_t g = 0; g < ng; ++g) gptr[g + 1] = gptr[g] + (int64_t)ucol[g].size();
  const int64_t nslot = gptr[ng];
  std::vector<int32_t> gcol(std::max<int64_t>(nslot, 1)), grow(std::max<int64_t>(ng * NG_ROWS, 1), -1);
  for (int64_t g = 0; g < ng; ++g) {
    std::copy(ucol[g].begin(), ucol[g].end(), gcol.begin() + gptr[g]);
    for (int i = 0; i < NG_ROWS && g * NG_ROWS + i < n; ++i) grow[g * NG_ROWS + i] = perm[order[g * NG_ROWS + i]];
  }
  // blocks of NS_GROUPS groups: the union of their columns, and every slot's position in it
  const int64_t nb = (ng + NS_GROUPS - 1) / NS_GROUPS;
  std::vector<std::vector<int32_t>> bcol(nb);
  std::vector<int32_t> gloc(std::max<int64_t>(nslot, 1));
  auto blocks = [&](int64_t b0, int64_t b1) {
    for (int64_t b = b0; b < b1; ++b) {
      std::vector<int32_t> &u = bcol[b];
      const int64_t g0 = b * NS_GROUPS, g1 = std::min<int64_t>(ng, g0 + NS_GROUPS);
      u.assign(gcol.begin() + gptr[g0], gcol.begin() + gptr[g1]);
      std::sort(u.begin(), u.end());
      u.erase(std::unique(u.begin(), u.end()), u.end());
      for (int64_t sl = gptr[g0]; sl < gptr[g1]; ++sl)
        gloc[sl] = (int32_t)(std::lower_bound(u.begin(), u.end(), gcol[sl]) - u.begin());
    }
  };
  run_threads(blocks, nb);
  std::vector<int64_t> bptr(nb + 1, 0);
  for (int64_t b = 0; b < nb; ++b) bptr[b + 1] = bptr[b] + (int64_t)bcol[b].size();
  // per group, for each chunk c of NS_CH union positions of its block, the first slot
  // (relative to the group's first) whose position is >= c NS_CH; the last entry is the
  // group's slot count
  std::vector<int64_t> cbp(std::max<int64_t>(ng, 1), 0);
  for (int64_t g = 0, at = 0; g < ng; ++g) {
    cbp[g] = at;
    const int64_t b = g / NS_GROUPS;
    at += (bptr[b + 1] - bptr[b] + NS_CH - 1) / NS_CH + 1;
    if (g + 1 == ng) cbp.push_back(at);
  }
  std::vector<int32_t> cbv(std::max<int64_t>(ng > 0 ? cbp[ng] : 1, 1), 0);
  auto bounds = [&](int64_t ga, int64_t gb) {
    for (int64_t g = ga; g < gb; ++g) {
      const int64_t b = g / NS_GROUPS, nch = (bptr[b + 1] - bptr[b] + NS_CH - 1) / NS_CH;
      int64_t sl = gptr[g];
      for (int64_t c = 0; c <= nch; ++c) {
        while (sl < gptr[g + 1] && gloc[sl] < c * NS_CH) ++sl;
        cbv[cbp[g] + c] = (int32_t)(sl - gptr[g]);
      }
      cbv[cbp[g] + nch] = (int32_t)(gptr[g + 1] - gptr[g]);
    }
  };
  run_threads(bounds, ng);
  c->d_ng_cbp = (int64_t *)dalloc(c, sizeof(int64_t) * std::max<int64_t>(ng, 1));
  c->d_ng_cb = (int32_t *)dalloc(c, sizeof(int32_t) * cbv.size());
  check_cuda(cudaMemcpy(c->d_ng_cbp, cbp.data(), sizeof(int64_t) * std::max<int64_t>(ng, 1), cudaMemcpyHostToDevice),
             "near groups");
  check_cuda(cudaMemcpy(c->d_ng_cb, cbv.data(), sizeof(int32_t) * cbv.size(), cudaMemcpyHostToDevice), "near groups");
  std::vector<int32_t> bflat(std::max<int64_t>(bptr[nb], 1));
  for (int64_t b = 0; b < nb; ++b) std::copy(bcol[b].begin(), bcol[b].end(), bflat.begin() + bptr[b]);
  std::vector<std::vector<int32_t>>().swap(bcol);
  std::vector<std::vector<int32_t>>().swap(ucol);
  c->d_nb_ptr = (int64_t *)dalloc(c, sizeof(int64_t) * (nb + 1));
  c->d_nb_col = (int32_t *)dalloc(c, sizeof(int32_t) * bflat.size());
  check_cuda(cudaMemcpy(c->d_nb_ptr, bptr.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice), "near groups");
  check_cuda(cudaMemcpy(c->d_nb_col, bflat.data(), sizeof(int32_t) * bflat.size(), cudaMemcpyHostToDevice),
             "near groups");
  check_cuda(cudaFuncSetAttribute(k_near_group<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, NsShape<64>::SMEM),
             "near groups");
  check_cuda(cudaFuncSetAttribute(k_near_group<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, NsShape<16>::SMEM),
             "near groups");
  check_cuda(cudaFuncSetAttribute(k_receive_leaf<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, RcShape<64>::SMEM),
             "near groups");
  check_cuda(cudaFuncSetAttribute(k_receive_leaf<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, RcShape<16>::SMEM),
             "near groups");
  c->d_ng_ptr = (int64_t *)dalloc(c, sizeof(int64_t) * (ng + 1));
  c->d_ng_loc = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<int64_t>(nslot, 1));
  c->d_ng_row = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<int64_t>(ng * NG_ROWS, 1));
  c->d_ng_val = (cplxf *)dalloc(c, sizeof(cplxf) * std::max<int64_t>(nslot * NG_ROWS, 1));
  check_cuda(cudaMemcpy(c->d_ng_ptr, gptr.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice), "near groups");
  if (nslot > 0)
    check_cuda(cudaMemcpy(c->d_ng_loc, gloc.data(), sizeof(int32_t) * nslot, cudaMemcpyHostToDevice), "near groups");
  if (ng > 0)
    check_cuda(cudaMemcpy(c->d_ng_row, grow.data(), sizeof(int32_t) * ng * NG_ROWS, cudaMemcpyHostToDevice),
               "near groups");
  // source index in the padded CSR of every (slot, row) value, -1 for the zeros; built
  // and gathered in chunks of groups to bound the host index array (a single group has
  // at most n + 1 slots)
  const int64_t chunk_slots = (int64_t)1 << 24;
  std::vector<int64_t> src;
  int64_t *d_src = (int64_t *)dalloc(
      c, sizeof(int64_t) * (size_t)std::min<int64_t>(std::max<int64_t>(nslot, 1) * NG_ROWS,
                                                     (chunk_slots + 2 * (int64_t)n + 2) * NG_ROWS));
  for (int64_t g0 = 0; g0 < ng;) {
    int64_t g1 = g0 + 1;
    while (g1 < ng && gptr[g1 + 1] - gptr[g0] <= chunk_slots) ++g1;
    const int64_t s0 = gptr[g0], cnt = (gptr[g1] - s0) * NG_ROWS;
    src.assign(cnt, -1);
    auto fill = [&](int64_t a, int64_t b) {
      for (int64_t g = g0 + a; g < g0 + b; ++g)
        for (int i = 0; i < NG_ROWS && g * NG_ROWS + i < n; ++i) {
          const int64_t r = order[g * NG_ROWS + i], e0 = ptr4[r], len = row_len(r);
          int64_t e = e0;  // both lists ascending: walk them together
          for (int64_t sl = gptr[g]; sl < gptr[g + 1] && e < e0 + len; ++sl)
            if (gcol[sl] == col4[e]) {  // a repeated last slot stays 0: e has moved on
              src[(sl - s0) * NG_ROWS + i] = e;
              ++e;
            }
        }
    };
    run_threads(fill, g1 - g0);
    check_cuda(cudaMemcpy(d_src, src.data(), sizeof(int64_t) * cnt, cudaMemcpyHostToDevice), "near groups");
    k_gather_c64<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 1 << 16), 256, 0, c->stream>>>(
        c->d_ng_val + s0 * NG_ROWS, d_src, c->d_nz_val32, cnt);
    check_cuda(cudaStreamSynchronize(c->stream), "near groups");
    g0 = g1;
  }
  dfree(c, d_src);
  c->n_group = ng;
}

void build_mixed(nesa_ctx *c) {
  build_near_internal(c);
  c->d_V32 = copy_c64(c, c->d_V, 4 * c->info.v_columns * (int64_t)c->lev[c->L].q);
  for (int l = c->l0; l <= c->L; ++l) {
    DevLevel &d = c->lev[l];
    if (!d.gen)
      d.D32 = copy_c64(c, d.D, d.noff * (int64_t)d.q * d.q);
    else if (c->translate_engine == NESA_TRANSLATE_FP32)  // complex64 work buffer of the CUDA-core engine
      d.Dw32 = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)d.chunk_slots * d.q * d.q);
    if (l > c->l0) {
      const int64_t cn = 8LL * c->lev[l - 1].q * d.q;
      d.C32 = copy_c64(c, d.C, cn);
      d.Ct32 = copy_c64(c, d.Ct, cn);
    }
  }
  check_cuda(cudaGetLastError(), "mixed copies");
  check_cuda(cudaStreamSynchronize(c->stream), "mixed copies");
  c->mixed = true;
}

// ------------------------------------------------------------------ plane-wave excitation
// b_m = -sum_{T in supp m} sum_p w_p sl (r_p - v)/2 . pol exp(-i k khat.r_p)
__global__ void k_rhs_planewave(cplx *b, int64_t n, int nrhs, const double *khat, const cplx *pol,
                                const int32_t *rwg_tri, const int32_t *rwg_free, const int32_t *tris,
                                const double *verts, const double *tri_sl, const double *pts, const double *w7,
                                double k) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  int64_t m = idx % n;
  int r = (int)(idx / n);
  const double *kh = khat + 3 * r;
  const cplx *pl = pol + 3 * r;
  cplx acc = {0.0, 0.0};
  for (int s = 0; s < 2; ++s) {
    int32_t t = rwg_tri[2 * m + s];
    int fr = rwg_free[2 * m + s];
    double sl = tri_sl[3 * t + fr];
    const double *v = verts + 3 * (int64_t)tris[3 * t + fr];
    for (int p = 0; p < 7; ++p) {
      const double *rp = pts + 3 * (7 * (int64_t)t + p);
      double ph = -k * (kh[0] * rp[0] + kh[1] * rp[1] + kh[2] * rp[2]);
      double sn, cs;
      sincos(ph, &sn, &cs);
      double f = 0.5 * w7[p] * sl;
      cplx dp = {0.0, 0.0};
      for (int x = 0; x < 3; ++x) {
        double a = f * (rp[x] - v[x]);
        dp.x += a * pl[x].x;
        dp.y += a * pl[x].y;
      }
      acc = cadd(acc, cmul(dp, make_double2(cs, sn)));
    }
  }
  b[(int64_t)r * n + m] = make_double2(-acc.x, -acc.y);
}

}  // namespace nesa

using namespace nesa;

extern "C" {

int nesa_profile_enable(nesa_ctx *c, int enable) {
  if (!c) return NESA_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  for (auto &p : c->pending) {
    c->event_pool.push_back(p.a);
    c->event_pool.push_back(p.b);
  }
  c->pending.clear();
  c->prof = nesa_profile{};
  c->profiling = enable != 0;
  return NESA_OK;
}

int nesa_profile_read(nesa_ctx *c, nesa_profile *out) {
  if (!c || !out) return NESA_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NESA_ERR_CUDA;
  for (auto &p : c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return NESA_ERR_CUDA;
    c->prof.launches[p.stage] += 1;
    c->prof.ms[p.stage] += ms;
    c->prof.flops[p.stage] += p.flops;
    c->prof.bytes[p.stage] += p.bytes;
    c->event_pool.push_back(p.a);
    c->event_pool.push_back(p.b);
  }
  c->pending.clear();
  *out = c->prof;
  return NESA_OK;
}

int nesa_matvec_parts(nesa_ctx *c, const nesa_c128 *x, nesa_c128 *y, int nrhs, int parts) {
  if (!c || !x || !y || nrhs < 1 || nrhs > 64 || (parts & NESA_PART_ALL) == 0 ||
      (parts & ~(NESA_PART_ALL | NESA_PART_MIXED)) != 0)
    return NESA_ERR_INVALID_ARG;
  try {
    ensure_workspace(c, nrhs);
    launch_matvec(c, (const cplx *)x, (cplx *)y, nrhs, parts);
    check_cuda(cudaGetLastError(), "matvec launch");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_device_status(nesa_ctx *c) {
  if (!c) return NESA_ERR_INVALID_ARG;
  try {
    check_cuda(cudaStreamSynchronize(c->stream), "sync");
    if (tc_take_error(c)) return NESA_ERR_TIMEOUT;
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_inject_stall(nesa_ctx *c, int stall, uint32_t wait_limit) {
  if (!c || (stall != 0 && stall != 1)) return NESA_ERR_INVALID_ARG;
  c->tc_stall = stall;
  c->tc_wait_limit = wait_limit ? wait_limit : (1u << 20);
  return NESA_OK;
}

int nesa_matvec(nesa_ctx *c, const nesa_c128 *x, nesa_c128 *y, int nrhs) {
  return nesa_matvec_parts(c, x, y, nrhs, NESA_PART_ALL);
}

int nesa_matvec_host(nesa_ctx *c, const nesa_c128 *xh, nesa_c128 *yh, int nrhs, int parts) {
  if (!c || !xh || !yh || nrhs < 1 || nrhs > 64 || (parts & NESA_PART_ALL) == 0 ||
      (parts & ~(NESA_PART_ALL | NESA_PART_MIXED)) != 0)
    return NESA_ERR_INVALID_ARG;
  try {
    if (nrhs > c->hbuf_cap) {
      dfree(c, c->d_hx);
      dfree(c, c->d_hy);
      c->d_hx = (cplx *)dalloc(c, sizeof(cplx) * (size_t)c->n * nrhs);
      c->d_hy = (cplx *)dalloc(c, sizeof(cplx) * (size_t)c->n * nrhs);
      c->hbuf_cap = nrhs;
    }
    size_t bytes = sizeof(cplx) * (size_t)c->n * nrhs;
    check_cuda(cudaMemcpyAsync(c->d_hx, xh, bytes, cudaMemcpyHostToDevice, c->stream), "H2D");
    ensure_workspace(c, nrhs);
    launch_matvec(c, c->d_hx, c->d_hy, nrhs, parts);
    check_cuda(cudaGetLastError(), "matvec launch");
    check_cuda(cudaMemcpyAsync(yh, c->d_hy, bytes, cudaMemcpyDeviceToHost, c->stream), "D2H");
    check_cuda(cudaStreamSynchronize(c->stream), "sync");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_rhs_planewave(nesa_ctx *c, const double *khat, const nesa_c128 *pol, int nrhs, nesa_c128 *b) {
  if (!c || !khat || !pol || !b || nrhs < 1 || nrhs > 4096) return NESA_ERR_INVALID_ARG;
  try {
    // one device buffer: polarisations first (16-byte aligned complex), then the
    // directions and the 7 rule weights (doubles)
    const double s15 = std::sqrt(15.0);
    std::vector<double> buf(6 * (size_t)nrhs + 3 * (size_t)nrhs + 7);
    std::memcpy(buf.data(), pol, sizeof(nesa_c128) * 3 * nrhs);
    std::copy(khat, khat + 3 * nrhs, buf.begin() + 6 * nrhs);
    double w[7] = {9.0 / 40.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0,
                   (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0};
    std::copy(w, w + 7, buf.begin() + 9 * nrhs);
    double *d = (double *)dalloc(c, sizeof(double) * buf.size());
    check_cuda(cudaMemcpyAsync(d, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, c->stream), "H2D");
    k_rhs_planewave<<<grid_for(c->n * nrhs, 256), 256, 0, c->stream>>>(
        (cplx *)b, c->n, nrhs, d + 6 * nrhs, (const cplx *)d, c->d_rwg_tri, c->d_rwg_free, c->d_tris, c->d_verts,
        c->d_tri_sl, c->d_pts, d + 9 * nrhs, c->k);
    check_cuda(cudaGetLastError(), "rhs launch");
    check_cuda(cudaStreamSynchronize(c->stream), "rhs");
    dfree(c, d);
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

}  // extern "C"
