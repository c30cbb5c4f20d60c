// Mixed-precision translation and potential transfer on the tensor cores
// (NESA_TRANSLATE_TENSOR).
//
// Per level l, for each chunk of rc right-hand sides (Eq. 12 and Eq. 13):
//   k_split        s_l (complex64) -> BF16 hi/lo column-group blocks (nesa_tc.cuh)
//   k_tc_gemm      translations: one GEMM per offset slot, D(o) [s_b ...]; every pair
//                  (a, b) gets its own block of P
//   k_split        o_{l-1} -> BF16 blocks (l > l0)
//   k_tc_gemm      potential transfer: one GEMM per octant, C_l(octant)^T [o_P ...];
//                  every box a gets the block nil + a of P
//   k_pair_reduce  o_a = P[nil + a] + sum over the pairs of a of P[pair]
// The reduction runs over each target's own blocks in a fixed order (owner computes),
// so the product is deterministic.
//
// With many right-hand sides (nrhs >= SEG_MIN_RHS) the same GEMMs run target-grouped
// instead: a work item is (target box, 32 right-hand sides, M tile) and its K loop runs
// over the target's whole list (interaction list, parent, or children), one segment per
// entry, into one TMEM accumulator, in list order.  The result goes straight to o_l (or
// s_P), with no per-pair blocks and no reduction; the A tiles and source blocks read per
// item are the same as in the offset-grouped form, whose column tiles then hold about
// two right-hand-side groups of each pair.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nesa_device.cuh"
#include "nesa_tc.cuh"

namespace nesa {

// One family of equal-shaped GEMMs (all offsets of a level, or its eight octants).
struct TcGemm {
  int q = 0, kdim = 0;  // complex rows and columns of each matrix
  // translations generated in the GEMM's producers instead of read from A (see GemmArgs)
  bool gen = false;
  float4 *gen_E = nullptr, *gen_S = nullptr;
  float2 *gen_P = nullptr;
  float gen_kap = 0.0f;
  int nk16 = 0, nkc = 0, nmt = 0;
  int64_t nslot = 0, nent = 0;
  __nv_bfloat16 *A = nullptr;  // [slot][nmt][nkc][2][4096]: hi then lo plane of every tile
  std::vector<int32_t> h_ptr, h_dst, h_src;         // entries (output block, source box) by slot
  int tn = 128;                   // column-tile width (autotuned)
  int tuned_rc = 0;               // chunk size the width was tuned for
  float tune_ms[3] = {0, 0, 0};   // measured times for widths 64, 128, 256
  tc::Work *work = nullptr;       // work list for (work_tn, work_rc)
  int32_t *wsrc = nullptr, *wdst = nullptr;
  int64_t nwork = 0;
  int work_tn = 0, work_rc = 0;
  // target-grouped form: per target its entries (slot, source box) in list order
  std::vector<int32_t> t_ptr, t_slot, t_src;
  int64_t ntarget = 0, nsource = 0;
  bool any_empty = false;          // some target has no entry (its output is not written)
  tc::Work *swork = nullptr;       // work list for swork_rc right-hand sides
  int32_t *swdst = nullptr;
  int2 *sseg = nullptr;
  int64_t snwork = 0;
  int swork_rc = 0;
};

constexpr int SEG_MIN_RHS = 32;  // products with at least this many right-hand sides
constexpr int SEG_TN = 256;      // run target-grouped, 32 right-hand sides per column tile

struct TcLevel {
  TcGemm tr, dn, up;  // translations (Eq. 12); potential transfer (Eq. 13) and source
                      // transfer to the parent level (Eq. 11), both for l > l0
  int rc = 0;         // right-hand sides per chunk the buffers below are sized for
  __nv_bfloat16 *s_hi = nullptr, *s_lo = nullptr;  // [nbox][rc][tr.nkc][256]
  __nv_bfloat16 *o_hi = nullptr, *o_lo = nullptr;  // [parent boxes][rc][dn.nkc][256]
  cplxf *P = nullptr;                              // [nil + nbox][4 rc][q]
  cplxf *P_up = nullptr;                           // [nbox][4 rc][q of the parent level]
  bool has_P = false;                              // P and P_up exist (offset-grouped form)
  bool s_split = false;  // s_hi/s_lo hold the split of all right-hand sides of the current
                         // product (set by the source transfer, used by the translation)
};

struct TcState {
  TcLevel lev[NESA_MAX_LEVELS];
  int *err = nullptr;
  int nsm = 0;
};

static TcState *state(nesa_ctx *c) { return (TcState *)c->tc_state; }

// Real A tiles of nslot complex matrices M (q x kdim, column-major, complex128): row 2i
// of A is Re M(i,:), row 2i+1 is Im M(i,:); rows >= 2q and columns >= kdim are zero.
// Each value v is split as hi = bf16(v), lo = bf16(v - hi).
__global__ void k_prep_A(__nv_bfloat16 *A, const cplx *M, int64_t nslot, int q, int kdim, int nmt, int nkc) {
  const int64_t total = nslot * nmt * nkc * (int64_t)tc::TILE_ELEMS;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx % tc::TILE_ELEMS);  // (row, k) with k fastest
    int64_t rest = idx / tc::TILE_ELEMS;
    const int kc = (int)(rest % nkc);
    rest /= nkc;
    const int mt = (int)(rest % nmt);
    const int64_t slot = rest / nmt;
    const int rloc = e / tc::TK, kloc = e % tc::TK;
    const int row = mt * tc::TM + rloc, k = kc * tc::TK + kloc;
    const int i = row >> 1;
    double v = 0.0;
    if (i < q && k < kdim) {
      const cplx m = M[slot * (int64_t)q * kdim + i + (int64_t)k * q];
      v = (row & 1) ? m.y : m.x;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
    const int64_t out = ((slot * nmt + mt) * nkc + kc) * 2 * tc::TILE_ELEMS + tc::a_tile_elem(rloc, kloc);
    A[out] = hi;
    A[out + tc::TILE_ELEMS] = lo;
  }
}

// x (complex64, [box][4 nrhs][q], column 4r + ch) -> hi/lo blocks [box][rc][nkc][256]
// for the right-hand sides r0 .. r0+rc-1: block (box, r, kc) holds the 8 columns
// 2ch + part (part 0: Re x_ch, 1: Im x_ch) at K = 32 kc .. 32 kc + 31 (zero past q).
// One thread per 16-byte row of a core matrix: 8 consecutive K of one column.
__global__ void k_split(__nv_bfloat16 *x_hi, __nv_bfloat16 *x_lo, const cplxf *x, int64_t nbox, int nrhs, int r0,
                        int rc, int q, int nkc) {
  const int64_t total = nbox * rc * nkc * 32;  // (kq, column) rows per block
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(idx % 32);  // kq * 8 + column
    int64_t rest = idx / 32;
    const int kc = (int)(rest % nkc);
    rest /= nkc;
    const int r = (int)(rest % rc);
    const int64_t box = rest / rc;
    const int kq = row >> 3, col = row & 7, k0 = kc * tc::TK + kq * 8;
    const cplxf *src = x + (box * 4 * nrhs + 4 * (r0 + r) + (col >> 1)) * q;
    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int k = k0 + kk;
      float v = 0.0f;
      if (k < q) {
        const cplxf z = src[k];
        v = (col & 1) ? z.y : z.x;
      }
      hi[kk] = __float2bfloat16_rn(v);
      lo[kk] = __float2bfloat16_rn(v - __bfloat162float(hi[kk]));
    }
    const int64_t out = ((box * rc + r) * nkc + kc) * tc::GROUP_ELEMS + tc::b_group_elem(col, kq * 8);
    *(uint4 *)(x_hi + out) = *(const uint4 *)hi;
    *(uint4 *)(x_lo + out) = *(const uint4 *)lo;
  }
}

// o_a (right-hand sides r0 .. r0+rc-1) = P[down + a] (when down >= 0) + sum of the
// pair blocks of a in list order; P blocks are [4 rc][q] complex64
__global__ void __launch_bounds__(256) k_pair_reduce(cplxf *__restrict__ o, const cplxf *__restrict__ P,
                                                     const int32_t *__restrict__ il_ptr, int64_t down, int nrhs,
                                                     int r0, int rc, int q) {
  const int32_t a = blockIdx.x;
  const int64_t blk = 4 * (int64_t)rc * q;
  const int64_t j = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
  if (j >= blk) return;
  cplxf acc = down >= 0 ? P[(down + a) * blk + j] : make_float2(0.0f, 0.0f);
  const int32_t e0 = il_ptr[a], e1 = il_ptr[a + 1];
  for (int32_t e = e0; e < e1; ++e) {
    const cplxf v = P[(int64_t)e * blk + j];
    acc.x += v.x;
    acc.y += v.y;
  }
  o[((int64_t)a * 4 * nrhs + 4 * r0) * q + j] = acc;
}

// A tiles and entry lists of one GEMM family; M = nslot matrices q x kdim (complex128)
static void gemm_setup(nesa_ctx *c, TcGemm &g, const cplx *M, int64_t nslot, int q, int kdim,
                       const std::vector<int32_t> &ent_slot, const std::vector<int32_t> &dst,
                       const std::vector<int32_t> &src) {
  g.q = q;
  g.kdim = kdim;
  g.nk16 = (kdim + 15) / 16;
  g.nkc = (g.nk16 + 1) / 2;
  g.nmt = (2 * q + tc::TM - 1) / tc::TM;
  g.nslot = nslot;
  g.nent = (int64_t)ent_slot.size();
  if (M) {  // stored A tiles (a generated family has none)
    const int64_t nel = nslot * g.nmt * (int64_t)g.nkc * tc::TILE_ELEMS;
    g.A = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * 2 * nel);
    k_prep_A<<<(unsigned)std::min<int64_t>((nel + 255) / 256, 1 << 20), 256, 0, c->stream>>>(g.A, M, nslot, q, kdim,
                                                                                           g.nmt, g.nkc);
    check_cuda(cudaGetLastError(), "prep A");
  }
  // entries grouped by slot (stable: ascending entry order within a slot)
  g.h_ptr.assign(nslot + 1, 0);
  g.h_dst.resize(g.nent);
  g.h_src.resize(g.nent);
  for (int32_t sl : ent_slot) g.h_ptr[sl + 1]++;
  for (int64_t s = 0; s < nslot; ++s) g.h_ptr[s + 1] += g.h_ptr[s];
  std::vector<int32_t> fill(g.h_ptr.begin(), g.h_ptr.end() - 1);
  for (int64_t e = 0; e < g.nent; ++e) {
    const int32_t at = fill[ent_slot[e]]++;
    g.h_dst[at] = dst[e];
    g.h_src[at] = src[e];
  }
}

// Target lists of a family for the target-grouped form: entry e (in ascending order)
// belongs to target tgt[e] and reads A matrix slot[e] and source box src[e].
static void seg_setup(TcGemm &g, int64_t ntarget, int64_t nsource, const std::vector<int32_t> &tgt,
                      const std::vector<int32_t> &slot, const std::vector<int32_t> &src) {
  g.ntarget = ntarget;
  g.nsource = nsource;
  g.t_ptr.assign(ntarget + 1, 0);
  for (int32_t t : tgt) g.t_ptr[t + 1]++;
  for (int64_t t = 0; t < ntarget; ++t) g.t_ptr[t + 1] += g.t_ptr[t];
  g.t_slot.resize(tgt.size());
  g.t_src.resize(tgt.size());
  std::vector<int32_t> fill(g.t_ptr.begin(), g.t_ptr.end() - 1);
  for (size_t e = 0; e < tgt.size(); ++e) {
    const int32_t at = fill[tgt[e]]++;
    g.t_slot[at] = slot[e];
    g.t_src[at] = src[e];
  }
  g.any_empty = false;
  for (int64_t t = 0; t < ntarget; ++t) g.any_empty |= g.t_ptr[t + 1] == g.t_ptr[t];
}

template <int TN, bool SEG, bool GEN>
static void set_smem() {
  check_cuda(cudaFuncSetAttribute(tc::k_tc_gemm<TN, SEG, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::smem_bytes<TN>()),
             "smem attribute");
}

// Generation data of the translation family of a level (Eq. 12 in the producers):
// equivalent points about the box centre in FP32, and per offset slot s = o w as
// (2 s, |s|) in FP32 with the phase exp(-i k |s|) evaluated in FP64.
static void gen_setup(nesa_ctx *c, TcGemm &g, const HostLevel &hl) {
  const int q = hl.q;
  std::vector<float4> E(q);
  for (int i = 0; i < q; ++i)
    E[i] = make_float4((float)hl.eq_pts[3 * i], (float)hl.eq_pts[3 * i + 1], (float)hl.eq_pts[3 * i + 2], 0.0f);
  const int64_t ns = (int64_t)hl.offsets.size() / 3;
  std::vector<float4> S(std::max<int64_t>(1, ns));
  std::vector<float2> P(std::max<int64_t>(1, ns));
  for (int64_t o = 0; o < ns; ++o) {
    const double sx = hl.offsets[3 * o] * hl.width, sy = hl.offsets[3 * o + 1] * hl.width,
                 sz = hl.offsets[3 * o + 2] * hl.width;
    const double R0 = std::sqrt(sx * sx + sy * sy + sz * sz);
    S[o] = make_float4((float)(2.0 * sx), (float)(2.0 * sy), (float)(2.0 * sz), (float)R0);
    P[o] = make_float2((float)std::cos(c->k * R0), (float)-std::sin(c->k * R0));
  }
  g.gen_E = (float4 *)dalloc(c, sizeof(float4) * E.size());
  g.gen_S = (float4 *)dalloc(c, sizeof(float4) * S.size());
  g.gen_P = (float2 *)dalloc(c, sizeof(float2) * P.size());
  check_cuda(cudaMemcpy(g.gen_E, E.data(), sizeof(float4) * E.size(), cudaMemcpyHostToDevice), "gen E");
  check_cuda(cudaMemcpy(g.gen_S, S.data(), sizeof(float4) * S.size(), cudaMemcpyHostToDevice), "gen S");
  check_cuda(cudaMemcpy(g.gen_P, P.data(), sizeof(float2) * P.size(), cudaMemcpyHostToDevice), "gen P");
  g.gen_kap = (float)(c->k / (2.0 * 3.14159265358979323846));
  g.gen = true;
}

void tc_build(nesa_ctx *c) {
  TcState *S = new TcState();
  c->tc_state = S;
  set_smem<64, false, false>();
  set_smem<128, false, false>();
  set_smem<256, false, false>();
  set_smem<SEG_TN, true, false>();
  set_smem<64, false, true>();
  set_smem<128, false, true>();
  set_smem<256, false, true>();
  set_smem<SEG_TN, true, true>();
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "device");
  check_cuda(cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  S->err = (int *)dalloc(c, sizeof(int));
  check_cuda(cudaMemset(S->err, 0, sizeof(int)), "tc flag");
  for (int l = c->l0; l <= c->L; ++l) {
    DevLevel &d = c->lev[l];
    TcLevel &t = S->lev[l];
    const HostLevel &hl = c->h.lev[l];
    // translations: entry = pair e, slot = its offset, source = il_src[e]
    std::vector<int32_t> dst(hl.il_slot.size());
    for (size_t e = 0; e < dst.size(); ++e) dst[e] = (int32_t)e;
    // translations generated in the producers where the level has no stored FP64 table
    // (automatic: tables too large to store) or where the context asks for it.  Measured
    // on the r = 3 sphere (1 RHS), generating a level's tiles costs about twice streaming
    // them from DRAM (0.35 against 0.17 ms at Q = 576), so it is used for memory only.
    const bool gen = d.gen || c->tables_mode == NESA_TABLES_GENERATED;
    gemm_setup(c, t.tr, gen ? nullptr : d.D, d.noff, d.q, d.q, hl.il_slot, dst, hl.il_src);
    if (gen) gen_setup(c, t.tr, hl);
    std::vector<int32_t> il_tgt(hl.il_slot.size());  // pair e belongs to target box a
    for (int64_t a = 0; a < d.nbox; ++a)
      for (int32_t e = hl.il_ptr[a]; e < hl.il_ptr[a + 1]; ++e) il_tgt[e] = (int32_t)a;
    seg_setup(t.tr, d.nbox, d.nbox, il_tgt, hl.il_slot, hl.il_src);
    if (l > c->l0) {  // potential transfer: entry = box a, slot = octant, source = parent
      std::vector<int32_t> bd(d.nbox), id(d.nbox);
      for (int64_t a = 0; a < d.nbox; ++a) {
        bd[a] = (int32_t)(d.nil + a);
        id[a] = (int32_t)a;
      }
      gemm_setup(c, t.dn, d.Ct, 8, d.q, c->lev[l - 1].q, hl.octant, bd, hl.parent);
      seg_setup(t.dn, d.nbox, c->lev[l - 1].nbox, id, hl.octant, hl.parent);
      // source transfer: entry = child box a, slot = octant, source = a, block a of P_up
      gemm_setup(c, t.up, d.C, 8, c->lev[l - 1].q, d.q, hl.octant, id, id);
      seg_setup(t.up, c->lev[l - 1].nbox, d.nbox, hl.parent, hl.octant, id);
    }
  }
  if (c->fixed_tn)
    for (int l = c->l0; l <= c->L; ++l) S->lev[l].tr.tn = S->lev[l].dn.tn = S->lev[l].up.tn = c->fixed_tn;
  check_cuda(cudaStreamSynchronize(c->stream), "tc build");
  c->tc_enabled = true;
}

// Work list (slot-major, so that CTAs running together share the slot's A tiles) and,
// per work item, the source block (box * rc + r) and output column (block * 4 rc + 4 r)
// of each of its tn/8 column groups (-1 past the slot's last group).
static void make_work(nesa_ctx *c, TcGemm &g, int rc, int tn) {
  if (g.work && g.work_tn == tn && g.work_rc == rc) return;
  dfree(c, g.work);
  dfree(c, g.wsrc);
  dfree(c, g.wdst);
  g.work = nullptr;
  g.wsrc = g.wdst = nullptr;
  std::vector<tc::Work> w;
  std::vector<int32_t> ws, wd;
  const int gt = tn / 8;
  for (int64_t s = 0; s < g.nslot; ++s) {
    const int32_t e0 = g.h_ptr[s];
    const int64_t ngroups = (int64_t)(g.h_ptr[s + 1] - e0) * rc;
    const int nnt = (int)((ngroups + gt - 1) / gt);
    for (int mt = 0; mt < g.nmt; ++mt)
      for (int nt = 0; nt < nnt; ++nt) {
        const int nvalid = (int)std::min<int64_t>(gt, ngroups - (int64_t)nt * gt);
        w.push_back({(int32_t)s, mt, nvalid, 0});
        for (int j = 0; j < gt; ++j) {
          const int64_t G = (int64_t)nt * gt + j;
          if (j < nvalid) {
            const int32_t e = e0 + (int32_t)(G / rc), r = (int32_t)(G % rc);
            ws.push_back(g.h_src[e] * rc + r);
            wd.push_back(g.h_dst[e] * 4 * rc + 4 * r);
          } else {
            ws.push_back(-1);
            wd.push_back(-1);
          }
        }
      }
  }
  g.nwork = (int64_t)w.size();
  g.work = (tc::Work *)dalloc(c, sizeof(tc::Work) * std::max<size_t>(1, w.size()));
  g.wsrc = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<size_t>(1, ws.size()));
  g.wdst = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<size_t>(1, wd.size()));
  if (!w.empty()) {
    check_cuda(cudaMemcpy(g.work, w.data(), sizeof(tc::Work) * w.size(), cudaMemcpyHostToDevice), "work");
    check_cuda(cudaMemcpy(g.wsrc, ws.data(), sizeof(int32_t) * ws.size(), cudaMemcpyHostToDevice), "work");
    check_cuda(cudaMemcpy(g.wdst, wd.data(), sizeof(int32_t) * wd.size(), cudaMemcpyHostToDevice), "work");
  }
  g.work_tn = tn;
  g.work_rc = rc;
}

static void launch_gemm(nesa_ctx *c, const TcGemm &g, const __nv_bfloat16 *B_hi, const __nv_bfloat16 *B_lo,
                        cplxf *P, int rc) {
  TcState *S = state(c);
  if (g.nwork == 0) return;
  (void)rc;
  tc::GemmArgs a{g.work, g.wsrc, g.wdst, g.nwork, g.A, B_hi, B_lo, P, g.q, g.nk16, g.nmt, S->err};
  a.wait_limit = c->tc_wait_limit;
  a.stall = c->tc_stall;
  a.gen_E = g.gen_E;
  a.gen_S = g.gen_S;
  a.gen_P = g.gen_P;
  a.gen_kap = g.gen_kap;
  const unsigned grid = (unsigned)std::min<int64_t>(g.nwork, S->nsm);
  cudaStream_t st = c->stream;
  constexpr int T0 = tc::Roles<false>::THREADS, T1 = tc::Roles<true>::THREADS;
  switch (g.work_tn * 2 + (g.gen ? 1 : 0)) {
    case 128:
      tc::k_tc_gemm<64, false, false><<<grid, T0, tc::smem_bytes<64>(), st>>>(a);
      break;
    case 129:
      tc::k_tc_gemm<64, false, true><<<grid, T1, tc::smem_bytes<64>(), st>>>(a);
      break;
    case 512:
      tc::k_tc_gemm<256, false, false><<<grid, T0, tc::smem_bytes<256>(), st>>>(a);
      break;
    case 513:
      tc::k_tc_gemm<256, false, true><<<grid, T1, tc::smem_bytes<256>(), st>>>(a);
      break;
    case 257:
      tc::k_tc_gemm<128, false, true><<<grid, T1, tc::smem_bytes<128>(), st>>>(a);
      break;
    default:
      tc::k_tc_gemm<128, false, false><<<grid, T0, tc::smem_bytes<128>(), st>>>(a);
  }
}

// Target-grouped work list for rc right-hand sides: per target with entries, per group
// of SEG_TN/8 right-hand sides r0.., its segments (slot, source block src * rc + r0) and
// one item per M tile; the output column of group j is target * 4 rc + 4 (r0 + j).
static void make_seg_work(nesa_ctx *c, TcGemm &g, int rc) {
  if (g.swork && g.swork_rc == rc) return;
  dfree(c, g.swork);
  dfree(c, g.swdst);
  dfree(c, g.sseg);
  g.swork = nullptr;
  g.swdst = nullptr;
  g.sseg = nullptr;
  std::vector<tc::Work> w;
  std::vector<int32_t> wd;
  std::vector<int2> sg;
  const int gt = SEG_TN / 8;
  for (int64_t t = 0; t < g.ntarget; ++t) {
    const int32_t e0 = g.t_ptr[t], e1 = g.t_ptr[t + 1];
    if (e0 == e1) continue;
    for (int r0 = 0; r0 < rc; r0 += gt) {
      const int nvalid = std::min(gt, rc - r0);
      const int32_t sb = (int32_t)sg.size();
      for (int32_t e = e0; e < e1; ++e) {
        if (g.t_slot[e] < 0 || g.t_slot[e] >= g.nslot || g.t_src[e] < 0 || g.t_src[e] >= g.nsource)
          fail(NESA_ERR_INVALID_ARG, "target-grouped work list: entry out of range");
        sg.push_back(make_int2(g.t_slot[e], g.t_src[e] * rc + r0));
      }
      const int32_t se = (int32_t)sg.size();
      for (int mt = 0; mt < g.nmt; ++mt) {
        w.push_back({sb, mt, nvalid, se});
        for (int j = 0; j < gt; ++j) wd.push_back(j < nvalid ? (int32_t)(t * 4 * rc + 4 * (r0 + j)) : -1);
      }
    }
  }
  if ((int64_t)sg.size() >= INT32_MAX || g.ntarget * 4 * (int64_t)rc >= INT32_MAX ||
      g.nsource * (int64_t)rc >= INT32_MAX)
    fail(NESA_ERR_INVALID_ARG, "target-grouped work list: index range");
  g.snwork = (int64_t)w.size();
  g.swork = (tc::Work *)dalloc(c, sizeof(tc::Work) * std::max<size_t>(1, w.size()));
  g.swdst = (int32_t *)dalloc(c, sizeof(int32_t) * std::max<size_t>(1, wd.size()));
  g.sseg = (int2 *)dalloc(c, sizeof(int2) * std::max<size_t>(1, sg.size()));
  if (!w.empty()) {
    check_cuda(cudaMemcpy(g.swork, w.data(), sizeof(tc::Work) * w.size(), cudaMemcpyHostToDevice), "work");
    check_cuda(cudaMemcpy(g.swdst, wd.data(), sizeof(int32_t) * wd.size(), cudaMemcpyHostToDevice), "work");
    check_cuda(cudaMemcpy(g.sseg, sg.data(), sizeof(int2) * sg.size(), cudaMemcpyHostToDevice), "work");
  }
  g.swork_rc = rc;
}

// out[target][4 rc][q] (+)= sum over the target's entries of A(slot) B(source).
static void launch_gemm_seg(nesa_ctx *c, const TcGemm &g, const __nv_bfloat16 *B_hi, const __nv_bfloat16 *B_lo,
                            cplxf *out, bool accum) {
  TcState *S = state(c);
  if (g.snwork == 0) return;
  // about 32 K steps of 16 per TMEM accumulation, as many as the largest translation
  // matrix of the offset-grouped form; the chunks are added in FP32 by the epilogue
  const int chunk = std::max(1, 32 / g.nk16);
  tc::GemmArgs a{g.swork, nullptr, g.swdst, g.snwork, g.A, B_hi, B_lo, out, g.q, g.nk16, g.nmt, S->err,
                 g.sseg, accum ? 1 : 0, chunk};
  a.wait_limit = c->tc_wait_limit;
  a.stall = c->tc_stall;
  a.gen_E = g.gen_E;
  a.gen_S = g.gen_S;
  a.gen_P = g.gen_P;
  a.gen_kap = g.gen_kap;
  const unsigned grid = (unsigned)std::min<int64_t>(g.snwork, S->nsm);
  if (g.gen)
    tc::k_tc_gemm<SEG_TN, true, true><<<grid, tc::Roles<true>::THREADS, tc::smem_bytes<SEG_TN>(), c->stream>>>(a);
  else
    tc::k_tc_gemm<SEG_TN, true, false><<<grid, tc::Roles<false>::THREADS, tc::smem_bytes<SEG_TN>(), c->stream>>>(a);
}

// Autotuner of the column-tile width: every candidate runs three times on the current
// operands (timed with CUDA events on the context's stream), the fastest is kept for
// this GEMM family and chunk size.  Synchronous: it runs at the first mixed product
// with a new chunk size (never inside a graph capture: the eager product comes first).
static void autotune(nesa_ctx *c, TcGemm &g, const __nv_bfloat16 *B_hi, const __nv_bfloat16 *B_lo, cplxf *P,
                     int rc) {
  const int cand[3] = {64, 128, 256};
  float best = 1e30f;
  int best_tn = 128;
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  for (int k = 0; k < 3; ++k) {
    make_work(c, g, rc, cand[k]);
    launch_gemm(c, g, B_hi, B_lo, P, rc);  // warm-up
    check_cuda(cudaEventRecord(e0, c->stream), "event");
    for (int r = 0; r < 3; ++r) launch_gemm(c, g, B_hi, B_lo, P, rc);
    check_cuda(cudaEventRecord(e1, c->stream), "event");
    check_cuda(cudaEventSynchronize(e1), "autotune");
    float ms = 0.0f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event");
    g.tune_ms[k] = ms / 3.0f;
    if (ms < best) {
      best = ms;
      best_tn = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  make_work(c, g, rc, best_tn);
  g.tn = best_tn;
  g.tuned_rc = rc;
}

static void prepare_rc(nesa_ctx *c, TcLevel &t, int l, int rc, bool with_P = true) {
  if (t.rc == rc && t.has_P == with_P) return;
  const DevLevel &d = c->lev[l];
  dfree(c, t.s_hi);
  dfree(c, t.s_lo);
  dfree(c, t.o_hi);
  dfree(c, t.o_lo);
  dfree(c, t.P);
  dfree(c, t.P_up);
  t.o_hi = t.o_lo = nullptr;
  t.P_up = nullptr;
  t.s_hi = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * rc * t.tr.nkc * tc::GROUP_ELEMS);
  t.s_lo = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)d.nbox * rc * t.tr.nkc * tc::GROUP_ELEMS);
  int64_t nblk = d.nil;
  if (l > c->l0) {
    const int64_t np = c->lev[l - 1].nbox;
    t.o_hi = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)np * rc * t.dn.nkc * tc::GROUP_ELEMS);
    t.o_lo = (__nv_bfloat16 *)dalloc(c, sizeof(__nv_bfloat16) * (size_t)np * rc * t.dn.nkc * tc::GROUP_ELEMS);
    nblk += d.nbox;
    if (with_P) t.P_up = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)d.nbox * 4 * rc * c->lev[l - 1].q);
  }
  t.P = with_P ? (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)std::max<int64_t>(1, nblk) * 4 * rc * d.q) : nullptr;
  t.rc = rc;
  t.has_P = with_P;
}

// Right-hand sides per chunk at level l: the largest divisor of nrhs for which the
// per-pair output P stays within about 4 GB.
static int level_rc(nesa_ctx *c, int l, int nrhs) {
  const DevLevel &d = c->lev[l];
  const bool down = l > c->l0;
  const double per_rhs = 4.0 * 8.0 * d.q * (double)std::max<int64_t>(1, d.nil + (down ? d.nbox : 0));
  int rc = (int)std::max(1.0, std::min((double)nrhs, 4.0e9 / per_rhs));
  while (nrhs % rc) --rc;
  return rc;
}

static inline unsigned grid_of(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 1 << 20); }

// Translation + potential transfer of level l on the tensor cores (mixed product).
void tc_translate_level(nesa_ctx *c, int l, const cplxf *s, cplxf *o, const cplxf *op, const cplxf *Ct, int nrhs) {
  (void)Ct;
  TcState *S = state(c);
  TcLevel &t = S->lev[l];
  const DevLevel &d = c->lev[l];
  cudaStream_t st = c->stream;
  const bool down = op != nullptr && l > c->l0;
  if (nrhs >= SEG_MIN_RHS) {  // target-grouped: o_l written by the GEMMs themselves
    prepare_rc(c, t, l, nrhs, false);
    if (!t.s_split)
      k_split<<<grid_of(d.nbox * nrhs * t.tr.nkc * (int64_t)32), 256, 0, st>>>(t.s_hi, t.s_lo, s, d.nbox, nrhs, 0,
                                                                                nrhs, d.q, t.tr.nkc);
    if (down) {
      const DevLevel &p = c->lev[l - 1];
      k_split<<<grid_of(p.nbox * nrhs * t.dn.nkc * (int64_t)32), 256, 0, st>>>(t.o_hi, t.o_lo, op, p.nbox, nrhs, 0,
                                                                                nrhs, p.q, t.dn.nkc);
      make_seg_work(c, t.dn, nrhs);
    }
    make_seg_work(c, t.tr, nrhs);
    const bool zero_first = !down && t.tr.any_empty;  // boxes without pairs still get o = 0
    if (zero_first)
      check_cuda(cudaMemsetAsync(o, 0, sizeof(cplxf) * (size_t)d.nbox * 4 * nrhs * d.q, st), "clear o");
    cudaEvent_t ev0 = nullptr;
    if (c->profiling) {
      ev0 = take_event(c);
      cudaEventRecord(ev0, st);
    }
    if (down) launch_gemm_seg(c, t.dn, t.o_hi, t.o_lo, o, false);  // o_a = C^T o_P(a)
    launch_gemm_seg(c, t.tr, t.s_hi, t.s_lo, o, down || zero_first);  // o_a += sum_b D s_b
    if (c->profiling) {
      cudaEvent_t ev1 = take_event(c);
      cudaEventRecord(ev1, st);
      double fl = 32.0 * nrhs * (double)d.nil * d.q * d.q;
      double by = (t.tr.gen ? 0.0 : 4.0 * (double)d.noff * t.tr.nmt * t.tr.nkc * tc::TILE_ELEMS) +
                  4.0 * (double)d.nil * nrhs * t.tr.nkc * tc::GROUP_ELEMS + 8.0 * (double)d.nbox * 4 * nrhs * d.q;
      if (down) {
        const int qp = c->lev[l - 1].q;
        fl += 32.0 * nrhs * (double)d.nbox * d.q * qp;
        by += 4.0 * 8 * t.dn.nmt * t.dn.nkc * tc::TILE_ELEMS + 4.0 * (double)d.nbox * nrhs * t.dn.nkc * tc::GROUP_ELEMS +
              16.0 * (double)d.nbox * 4 * nrhs * d.q;
      }
      c->pending.push_back({4, ev0, ev1, fl, by});
    }
    t.s_split = false;
    return;
  }
  const int rc = level_rc(c, l, nrhs);  // right-hand sides go through in equal chunks
  prepare_rc(c, t, l, rc);
  for (int r0 = 0; r0 < nrhs; r0 += rc) {
    if (!(t.s_split && rc == nrhs))
      k_split<<<grid_of(d.nbox * rc * t.tr.nkc * (int64_t)32), 256, 0, st>>>(t.s_hi, t.s_lo, s, d.nbox,
                                                                                         nrhs, r0, rc, d.q, t.tr.nkc);
    if (down) {
      const DevLevel &p = c->lev[l - 1];
      k_split<<<grid_of(p.nbox * rc * t.dn.nkc * (int64_t)32), 256, 0, st>>>(
          t.o_hi, t.o_lo, op, p.nbox, nrhs, r0, rc, p.q, t.dn.nkc);
    }
    if (c->autotune) {
      if (t.tr.tuned_rc != rc) autotune(c, t.tr, t.s_hi, t.s_lo, t.P, rc);
      if (down && t.dn.tuned_rc != rc) autotune(c, t.dn, t.o_hi, t.o_lo, t.P, rc);
    }
    make_work(c, t.tr, rc, t.tr.tn);
    if (down) make_work(c, t.dn, rc, t.dn.tn);
    cudaEvent_t ev0 = nullptr;
    if (c->profiling) {
      ev0 = take_event(c);
      cudaEventRecord(ev0, st);
    }
    launch_gemm(c, t.tr, t.s_hi, t.s_lo, t.P, rc);
    if (down) launch_gemm(c, t.dn, t.o_hi, t.o_lo, t.P, rc);
    if (c->profiling) {  // stage 4: the GEMM launches alone; algorithmic complex flops, operand bytes
      cudaEvent_t ev1 = take_event(c);
      cudaEventRecord(ev1, st);
      double fl = 32.0 * rc * (double)d.nil * d.q * d.q;
      double by = (t.tr.gen ? 0.0 : 4.0 * (double)d.noff * t.tr.nmt * t.tr.nkc * tc::TILE_ELEMS) +
                  4.0 * (double)d.nil * rc * t.tr.nkc * tc::GROUP_ELEMS + 32.0 * (double)d.nil * rc * d.q;
      if (down) {
        const int qp = c->lev[l - 1].q;
        fl += 32.0 * rc * (double)d.nbox * d.q * qp;
        by += 4.0 * 8 * t.dn.nmt * t.dn.nkc * tc::TILE_ELEMS + 4.0 * (double)d.nbox * rc * t.dn.nkc * tc::GROUP_ELEMS +
              32.0 * (double)d.nbox * rc * d.q;
      }
      c->pending.push_back({4, ev0, ev1, fl, by});
    }
    k_pair_reduce<<<dim3((unsigned)d.nbox, (unsigned)((4 * rc * d.q + 255) / 256)), 256, 0, st>>>(
        o, t.P, d.il_ptr, down ? d.nil : -1, nrhs, r0, rc, d.q);
  }
  t.s_split = false;
}

// Source transfer from level l to its parent level on the tensor cores (Eq. 11):
// s_P = sum over the children a of P of C_l(octant of a) s_a.
void tc_upward_level(nesa_ctx *c, int l, const cplxf *s, cplxf *sp, int nrhs) {
  TcState *S = state(c);
  TcLevel &t = S->lev[l];
  const DevLevel &d = c->lev[l], &p = c->lev[l - 1];
  cudaStream_t st = c->stream;
  if (nrhs >= SEG_MIN_RHS) {  // target-grouped: s_P written by the GEMM itself
    prepare_rc(c, t, l, nrhs, false);
    k_split<<<grid_of(d.nbox * nrhs * t.tr.nkc * (int64_t)32), 256, 0, st>>>(t.s_hi, t.s_lo, s, d.nbox, nrhs, 0,
                                                                              nrhs, d.q, t.tr.nkc);
    make_seg_work(c, t.up, nrhs);
    if (t.up.any_empty)
      check_cuda(cudaMemsetAsync(sp, 0, sizeof(cplxf) * (size_t)p.nbox * 4 * nrhs * p.q, st), "clear s");
    launch_gemm_seg(c, t.up, t.s_hi, t.s_lo, sp, t.up.any_empty);
    t.s_split = true;  // the translation of this level reuses the split
    return;
  }
  const int rc = level_rc(c, l, nrhs);
  prepare_rc(c, t, l, rc);
  for (int r0 = 0; r0 < nrhs; r0 += rc) {
    k_split<<<grid_of(d.nbox * rc * t.tr.nkc * (int64_t)32), 256, 0, st>>>(t.s_hi, t.s_lo, s, d.nbox,
                                                                                       nrhs, r0, rc, d.q, t.tr.nkc);
    if (c->autotune && t.up.tuned_rc != rc) autotune(c, t.up, t.s_hi, t.s_lo, t.P_up, rc);
    make_work(c, t.up, rc, t.up.tn);
    launch_gemm(c, t.up, t.s_hi, t.s_lo, t.P_up, rc);
    k_pair_reduce<<<dim3((unsigned)p.nbox, (unsigned)((4 * rc * p.q + 255) / 256)), 256, 0, st>>>(
        sp, t.P_up, p.child_ptr, -1, nrhs, r0, rc, p.q);
  }
  t.s_split = rc == nrhs;  // one chunk: the translation of this level can reuse the split
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
    tn[l] = S->lev[l].tr.tn;
    for (int k = 0; k < 3; ++k) ms[3 * l + k] = S->lev[l].tr.tune_ms[k];
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
