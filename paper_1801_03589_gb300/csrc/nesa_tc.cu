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
  int tn = 128;          // column-tile width of the GEMM (autotuned)
  int tuned_nrhs = 0;    // number of right-hand sides the width was tuned for
  float tune_ms[3] = {0, 0, 0};  // measured times for widths 64, 128, 256
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
    const int kgrp = b / tc::LBO_A, rem = b % tc::LBO_A;
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
// (columns col0 .. col0+cchunk-1 of every box; s has ctotal columns per box)
__global__ void k_split_s(__nv_bfloat16 *s_hi, __nv_bfloat16 *s_lo, const cplxf *s, int64_t nbox, int ctotal,
                          int col0, int cchunk, int q, int kp) {
  const int64_t total = nbox * cchunk * (int64_t)kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % kp);
    const int64_t oc = idx / kp;
    const int64_t col = (oc / cchunk) * ctotal + col0 + oc % cchunk;
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

// o_a = C^T o_P (Eq. 13) + sum of the translated columns of a's pairs (Eq. 12), for the
// right-hand sides r0 .. r0+rc-1 (P holds 4 rc columns per pair; o, op hold 4 nrhs)
__global__ void __launch_bounds__(512) k_pair_reduce(cplxf *__restrict__ o, const float *__restrict__ P,
                                                     const int32_t *__restrict__ il_ptr, const cplxf *__restrict__ op,
                                                     const cplxf *__restrict__ Ct, const int32_t *__restrict__ parent,
                                                     const int32_t *__restrict__ octant, int nrhs, int r0, int rc,
                                                     int q, int qp, int tr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplxf *col = (cplxf *)smem_raw;
  const int32_t a = blockIdx.x;
  const int tile = blockIdx.y;
  const int ch = threadIdx.x / tr;
  const int i = tile * tr + threadIdx.x % tr;
  const bool active = ch < 4 && i < q;
  const int ccol = 4 * nrhs, pcol = 4 * rc;
  const int32_t e0 = il_ptr[a], e1 = il_ptr[a + 1];
  for (int r = r0; r < r0 + rc; ++r) {
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
        const float *pc = P + ((int64_t)e * pcol + 4 * (r - r0) + ch) * 2 * q;
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
  check_cuda(cudaFuncSetAttribute(tc::k_tc_translate<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::smem_bytes<64>()),
             "smem attribute");
  check_cuda(cudaFuncSetAttribute(tc::k_tc_translate<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::smem_bytes<128>()),
             "smem attribute");
  check_cuda(cudaFuncSetAttribute(tc::k_tc_translate<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::smem_bytes<256>()),
             "smem attribute");
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

// work list of the GEMM for a column-tile width tn
static void tc_make_work(nesa_ctx *c, TcLevel &t, const DevLevel &d, int nrhs, int tn) {
  dfree(c, t.work);
  t.work = nullptr;
  const int ccol = 4 * nrhs;
  std::vector<tc::Work> w;
  for (int64_t s = 0; s < d.noff; ++s) {
    const int64_t ncols = (int64_t)t.h_slot_npairs[s] * ccol;
    const int nnt = (int)((ncols + tn - 1) / tn);
    for (int mt = 0; mt < t.nmt; ++mt)
      for (int nt = 0; nt < nnt; ++nt) w.push_back({(int32_t)s, mt, nt, 0});
  }
  t.nwork = (int64_t)w.size();
  t.work = (tc::Work *)dalloc(c, sizeof(tc::Work) * std::max<size_t>(1, w.size()));
  if (!w.empty())
    check_cuda(cudaMemcpy(t.work, w.data(), sizeof(tc::Work) * w.size(), cudaMemcpyHostToDevice), "work");
  t.tn = tn;
}

static void tc_gemm(nesa_ctx *c, TcLevel &t, const DevLevel &d, int nrhs) {
  TcState *S = state(c);
  const int ccol = 4 * nrhs;
  cudaStream_t st = c->stream;
  switch (t.tn) {
    case 64:
      tc::k_tc_translate<64><<<(unsigned)t.nwork, 128, tc::smem_bytes<64>(), st>>>(
          t.work, t.A_hi, t.A_lo, t.s_hi, t.s_lo, t.slot_ptr, t.slot_pair, d.il_src, t.P, d.q, t.kp, t.nmt, ccol,
          S->err);
      break;
    case 256:
      tc::k_tc_translate<256><<<(unsigned)t.nwork, 128, tc::smem_bytes<256>(), st>>>(
          t.work, t.A_hi, t.A_lo, t.s_hi, t.s_lo, t.slot_ptr, t.slot_pair, d.il_src, t.P, d.q, t.kp, t.nmt, ccol,
          S->err);
      break;
    default:
      tc::k_tc_translate<128><<<(unsigned)t.nwork, 128, tc::smem_bytes<128>(), st>>>(
          t.work, t.A_hi, t.A_lo, t.s_hi, t.s_lo, t.slot_ptr, t.slot_pair, d.il_src, t.P, d.q, t.kp, t.nmt, ccol,
          S->err);
  }
}

// Autotuner of the column-tile width: every candidate runs three times on the level's
// current operands (timed with CUDA events on the context's stream), the fastest is
// kept for this level and number of right-hand sides.  Synchronous: it runs at the
// first mixed product with a new number of right-hand sides (or from nesa_autotune).
static void tc_autotune(nesa_ctx *c, TcLevel &t, const DevLevel &d, int nrhs) {
  const int cand[3] = {64, 128, 256};
  float best = 1e30f;
  int best_tn = 128;
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  for (int tn : cand) {
    tc_make_work(c, t, d, nrhs, tn);
    if (t.nwork == 0) continue;
    tc_gemm(c, t, d, nrhs);  // warm-up
    check_cuda(cudaEventRecord(e0, c->stream), "event");
    for (int r = 0; r < 3; ++r) tc_gemm(c, t, d, nrhs);
    check_cuda(cudaEventRecord(e1, c->stream), "event");
    check_cuda(cudaEventSynchronize(e1), "autotune");
    float ms = 0.0f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event");
    t.tune_ms[tn == 64 ? 0 : (tn == 128 ? 1 : 2)] = ms / 3.0f;
    if (ms < best) {
      best = ms;
      best_tn = tn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tc_make_work(c, t, d, nrhs, best_tn);
  t.tuned_nrhs = nrhs;
}

static void tc_prepare_nrhs(nesa_ctx *c, TcLevel &t, const DevLevel &d, int nrhs) {
  if (t.nrhs == nrhs) return;
  dfree(c, t.s_hi);
  dfree(c, t.s_lo);
  dfree(c, t.P);
  const int ccol = 4 * nrhs;
  t.s_hi = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * ccol * t.kp);
  t.s_lo = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * ccol * t.kp);
  t.P = (float *)dalloc(c, sizeof(float) * (size_t)std::max<int64_t>(1, d.nil) * ccol * 2 * d.q);
  tc_make_work(c, t, d, nrhs, t.tn);
  t.nrhs = nrhs;
}

// Translation + potential transfer of level l on the tensor cores (mixed product).
void tc_translate_level(nesa_ctx *c, int l, const cplxf *s, cplxf *o, const cplxf *op, const cplxf *Ct, int nrhs,
                        int tr, int ntile, int threads) {
  TcState *S = state(c);
  TcLevel &t = S->lev[l];
  const DevLevel &d = c->lev[l];
  cudaStream_t st = c->stream;
  // right-hand sides go through in equal chunks of rc, so that the per-pair output P
  // stays within about 1 GB (rc = the largest divisor of nrhs that fits)
  const double per_rhs = 4.0 * 2.0 * d.q * 4.0 * (double)std::max<int64_t>(1, d.nil);
  int rc = (int)std::max(1.0, std::min((double)nrhs, 1.0e9 / per_rhs));
  while (nrhs % rc) --rc;
  tc_prepare_nrhs(c, t, d, rc);
  const int pcol = 4 * rc;
  const int qp = op ? c->lev[l - 1].q : 0;
  for (int r0 = 0; r0 < nrhs; r0 += rc) {
    k_split_s<<<(unsigned)std::min<int64_t>((d.nbox * pcol * (int64_t)t.kp + 255) / 256, 1 << 20), 256, 0, st>>>(
        t.s_hi, t.s_lo, s, d.nbox, 4 * nrhs, 4 * r0, pcol, d.q, t.kp);
    if (t.nwork > 0) {
      if (t.tuned_nrhs != rc && c->autotune) tc_autotune(c, t, d, rc);
      cudaEvent_t ev0 = nullptr;
      if (c->profiling) {
        ev0 = take_event(c);
        cudaEventRecord(ev0, st);
      }
      tc_gemm(c, t, d, rc);
      if (c->profiling) {  // stage 4: the GEMM launch alone; algorithmic complex flops, operand bytes
        cudaEvent_t ev1 = take_event(c);
        cudaEventRecord(ev1, st);
        const double fl = 32.0 * rc * (double)d.nil * d.q * d.q;
        const double by = 2.0 * 2.0 * (double)d.noff * t.nmt * t.kp * tc::TM +
                          2.0 * 2.0 * (double)d.nil * pcol * t.kp + 4.0 * (double)d.nil * pcol * 2 * d.q;
        c->pending.push_back({4, ev0, ev1, fl, by});
      }
    }
    size_t smem = sizeof(cplxf) * 4 * (size_t)std::max(qp, 1);
    k_pair_reduce<<<dim3((unsigned)d.nbox, ntile), threads, smem, st>>>(o, t.P, d.il_ptr, op, Ct, d.parent, d.octant,
                                                                        nrhs, r0, rc, d.q, qp, tr);
  }
}

// tile widths chosen per level (0 where the level has no tensor work), for nesa_get_tuning
void tc_tuning(nesa_ctx *c, int32_t *tn, float *ms) {
  TcState *S = state(c);
  for (int l = 0; l < NESA_MAX_LEVELS; ++l) {
    tn[l] = 0;
    for (int k = 0; k < 3; ++k) ms[3 * l + k] = 0.0f;
  }
  if (!S) return;
  for (int l = c->l0; l <= c->L; ++l) {
    tn[l] = S->lev[l].tn;
    for (int k = 0; k < 3; ++k) ms[3 * l + k] = S->lev[l].tune_ms[k];
  }
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
