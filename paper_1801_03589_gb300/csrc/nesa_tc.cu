// Mixed-precision translation on the tensor cores (NESA_TRANSLATE_TENSOR).
//
// Per level l (Eq. 12 and Eq. 13):
//   k_split_s      s_l (complex64) -> BF16 hi/lo planes [box][4r+ch][Re s; Im s; 0]
//   k_tc_translate for every offset slot o: C = A(o) B(pairs with offset o) on tcgen05
//                  (nesa_tc.cuh), one FP32 column of 2Q values per pair and column
//   k_pair_reduce  o_a = C^T o_P(a) + sum over the pairs of a of their columns
// The reduction runs over each target's own pairs in a fixed order (owner computes),
// so the product is deterministic.
#include <algorithm>
#include <vector>

#include "nesa_device.cuh"
#include "nesa_tc.cuh"

namespace nesa {

struct TcLevel {
  int kp = 0, nmt = 0;
  __nv_bfloat16 *A_hi = nullptr, *A_lo = nullptr;  // [noff][nmt][kp/32][4096]
  int32_t *slot_ptr = nullptr, *slot_pair = nullptr;
  std::vector<int32_t> h_slot_npairs;
  // per-nrhs state
  int nrhs = 0;
  tc::Work *work = nullptr;
  int64_t nwork = 0;
  __nv_bfloat16 *s_hi = nullptr, *s_lo = nullptr;  // [nbox][4 nrhs][kp]
  float *P = nullptr;                              // [nil][4 nrhs][2q]
};

struct TcState {
  TcLevel lev[NESA_MAX_LEVELS];
  int *err = nullptr;
};

// A(o) for every offset slot, split and tiled in the shared-memory layout
__global__ void k_prep_A(__nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, const cplx *D, int64_t noff, int q, int kp,
                         int nmt) {
  const int nkc = kp / tc::TK;
  const int64_t total = noff * nmt * nkc * (int64_t)tc::TILE_ELEMS;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % tc::TILE_ELEMS);
    int64_t rest = idx / tc::TILE_ELEMS;
    const int kc = (int)(rest % nkc);
    rest /= nkc;
    const int mt = (int)(rest % nmt);
    const int64_t slot = rest / nmt;
    // inverse of tc::tile_offset
    const int b = 2 * t;
    const int kgrp = b / tc::LBO, rem = b % tc::LBO;
    const int rgrp = rem / tc::SBO, rem2 = rem % tc::SBO;
    const int m = mt * tc::TM + rgrp * 8 + rem2 / 16;
    const int k = kc * tc::TK + kgrp * 8 + (rem2 % 16) / 2;
    double v = 0.0;
    if (m < 2 * q && k < 2 * q) {
      const cplx *Dm = D + slot * (int64_t)q * q;
      const int i = m < q ? m : m - q, j = k < q ? k : k - q;
      const cplx d = Dm[i + (int64_t)j * q];
      if (m < q)
        v = k < q ? d.x : -d.y;
      else
        v = k < q ? d.y : d.x;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
    A_hi[idx] = hi;
    A_lo[idx] = lo;
  }
}

// s (complex64, [box][ccol][q]) -> hi/lo planes [box][ccol][kp] of [Re; Im; 0]
__global__ void k_split_s(__nv_bfloat16 *s_hi, __nv_bfloat16 *s_lo, const cplxf *s, int64_t ncolumns, int q,
                          int kp) {
  const int64_t total = ncolumns * kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % kp);
    const int64_t col = idx / kp;
    float v = 0.0f;
    if (k < q)
      v = s[col * q + k].x;
    else if (k < 2 * q)
      v = s[col * q + (k - q)].y;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    s_hi[idx] = hi;
    s_lo[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// o_a = C^T o_P (Eq. 13) + sum of the translated columns of a's pairs (Eq. 12)
__global__ void __launch_bounds__(512) k_pair_reduce(cplxf *__restrict__ o, const float *__restrict__ P,
                                                     const int32_t *__restrict__ il_ptr, const cplxf *__restrict__ op,
                                                     const cplxf *__restrict__ Ct, const int32_t *__restrict__ parent,
                                                     const int32_t *__restrict__ octant, int nrhs, int q, int qp,
                                                     int tr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplxf *col = (cplxf *)smem_raw;
  const int32_t a = blockIdx.x;
  const int tile = blockIdx.y;
  const int ch = threadIdx.x / tr;
  const int i = tile * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < q;
  const int ccol = 4 * nrhs;
  const int32_t e0 = il_ptr[a], e1 = il_ptr[a + 1];
  for (int r = 0; r < nrhs; ++r) {
    cplxf acc = {0.0f, 0.0f};
    if (op) {
      __syncthreads();
      const int32_t Pp = parent[a];
      const cplxf *src = op + ((int64_t)Pp * ccol + 4 * r) * qp;
      for (int j = threadIdx.x; j < 4 * qp; j += blockDim.x) col[j] = src[j];
      __syncthreads();
      if (active) {
        const cplxf *Bm = Ct + (int64_t)octant[a] * q * qp + i;
        const cplxf *cs = col + ch * qp;
#pragma unroll 4
        for (int j = 0; j < qp; ++j) cfma(acc, Bm[(int64_t)j * q], cs[j]);
      }
    }
    if (active) {
      for (int32_t e = e0; e < e1; ++e) {
        const float *pc = P + ((int64_t)e * ccol + 4 * r + ch) * 2 * q;
        acc.x += pc[i];
        acc.y += pc[q + i];
      }
      o[((int64_t)a * ccol + 4 * r + ch) * q + i] = acc;
    }
  }
}

static TcState *state(nesa_ctx *c) { return (TcState *)c->tc_state; }

void tc_build(nesa_ctx *c) {
  TcState *S = new TcState();
  c->tc_state = S;
  S->err = (int *)dalloc(c, sizeof(int));
  check_cuda(cudaMemset(S->err, 0, sizeof(int)), "tc flag");
  for (int l = c->l0; l <= c->L; ++l) {
    DevLevel &d = c->lev[l];
    TcLevel &t = S->lev[l];
    const HostLevel &hl = c->h.lev[l];
    t.kp = ((2 * d.q + tc::TK - 1) / tc::TK) * tc::TK;
    t.nmt = (2 * d.q + tc::TM - 1) / tc::TM;
    const int64_t nel = d.noff * t.nmt * (int64_t)(t.kp / tc::TK) * tc::TILE_ELEMS;
    t.A_hi = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * nel);
    t.A_lo = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * nel);
    k_prep_A<<<(unsigned)std::min<int64_t>((nel + 255) / 256, 1 << 20), 256, 0, c->stream>>>(t.A_hi, t.A_lo, d.D,
                                                                                           d.noff, d.q, t.kp, t.nmt);
    check_cuda(cudaGetLastError(), "prep A");
    // pairs grouped by offset slot (stable: ascending target within a slot)
    std::vector<int32_t> ptr(d.noff + 1, 0), pairs(hl.il_slot.size());
    for (int32_t sl : hl.il_slot) ptr[sl + 1]++;
    for (int64_t s = 0; s < d.noff; ++s) ptr[s + 1] += ptr[s];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t e = 0; e < hl.il_slot.size(); ++e) pairs[fill[hl.il_slot[e]]++] = (int32_t)e;
    t.h_slot_npairs.resize(d.noff);
    for (int64_t s = 0; s < d.noff; ++s) t.h_slot_npairs[s] = ptr[s + 1] - ptr[s];
    t.slot_ptr = (int32_t *)dalloc(c, sizeof(int32_t) * ptr.size());
    t.slot_pair = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<size_t>(1, pairs.size()));
    check_cuda(cudaMemcpy(t.slot_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice), "slots");
    if (!pairs.empty())
      check_cuda(cudaMemcpy(t.slot_pair, pairs.data(), sizeof(int32_t) * pairs.size(), cudaMemcpyHostToDevice),
                 "pairs");
  }
  check_cuda(cudaStreamSynchronize(c->stream), "tc build");
  c->tc_enabled = true;
}

static void tc_prepare_nrhs(nesa_ctx *c, TcLevel &t, const DevLevel &d, int nrhs) {
  if (t.nrhs == nrhs) return;
  dfree(c, t.work);
  dfree(c, t.s_hi);
  dfree(c, t.s_lo);
  dfree(c, t.P);
  const int ccol = 4 * nrhs;
  std::vector<tc::Work> w;
  for (int64_t s = 0; s < d.noff; ++s) {
    const int64_t ncols = (int64_t)t.h_slot_npairs[s] * ccol;
    const int nnt = (int)((ncols + tc::TN - 1) / tc::TN);
    for (int mt = 0; mt < t.nmt; ++mt)
      for (int nt = 0; nt < nnt; ++nt) w.push_back({(int32_t)s, mt, nt, 0});
  }
  t.nwork = (int64_t)w.size();
  t.work = (tc::Work *)dalloc(c, sizeof(tc::Work) * std::max<size_t>(1, w.size()));
  if (!w.empty())
    check_cuda(cudaMemcpy(t.work, w.data(), sizeof(tc::Work) * w.size(), cudaMemcpyHostToDevice), "work");
  t.s_hi = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * ccol * t.kp);
  t.s_lo = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * ccol * t.kp);
  t.P = (float *)dalloc(c, sizeof(float) * (size_t)std::max<int64_t>(1, d.nil) * ccol * 2 * d.q);
  t.nrhs = nrhs;
}

// Translation + potential transfer of level l on the tensor cores (mixed product).
void tc_translate_level(nesa_ctx *c, int l, const cplxf *s, cplxf *o, const cplxf *op, const cplxf *Ct, int nrhs,
                        int tr, int ntile, int threads) {
  TcState *S = state(c);
  TcLevel &t = S->lev[l];
  const DevLevel &d = c->lev[l];
  tc_prepare_nrhs(c, t, d, nrhs);
  cudaStream_t st = c->stream;
  const int ccol = 4 * nrhs;
  const int64_t ncolumns = d.nbox * ccol;
  k_split_s<<<(unsigned)std::min<int64_t>((ncolumns * t.kp + 255) / 256, 1 << 20), 256, 0, st>>>(t.s_hi, t.s_lo, s,
                                                                                                  ncolumns, d.q, t.kp);
  if (t.nwork > 0) {
    static bool attr_set = false;
    if (!attr_set) {
      check_cuda(cudaFuncSetAttribute(tc::k_tc_translate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc::SMEM_BYTES),
                 "smem attribute");
      attr_set = true;
    }
    tc::k_tc_translate<<<(unsigned)t.nwork, 128, tc::SMEM_BYTES, st>>>(t.work, t.A_hi, t.A_lo, t.s_hi, t.s_lo,
                                                                       t.slot_ptr, t.slot_pair, d.il_src, t.P, d.q,
                                                                       t.kp, t.nmt, ccol, S->err);
  }
  const int qp = op ? c->lev[l - 1].q : 0;
  size_t smem = sizeof(cplxf) * 4 * (size_t)std::max(qp, 1);
  k_pair_reduce<<<dim3((unsigned)d.nbox, ntile), threads, smem, st>>>(o, t.P, d.il_ptr, op, Ct, d.parent, d.octant,
                                                                      nrhs, d.q, qp, tr);
}

int tc_take_error(nesa_ctx *c) {
  TcState *S = state(c);
  if (!S) return 0;
  int h = 0;
  check_cuda(cudaMemcpy(&h, S->err, sizeof(int), cudaMemcpyDeviceToHost), "tc flag");
  if (h) check_cuda(cudaMemset(S->err, 0, sizeof(int)), "tc flag");
  return h;
}

void tc_free(nesa_ctx *c) {
  delete state(c);
  c->tc_state = nullptr;
}

}  // namespace nesa
