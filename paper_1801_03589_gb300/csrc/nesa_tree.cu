// The octree and its box lists on the device (Sec. 2 and Sec. 3): the part of the host
// model that nesa_build computes on the GPU.  It fills the same HostModel fields as
// host_tree (nesa_host.cpp), bit for bit:
//
//   k_points        quadrature points (lambda0 v0 + lambda1 v1) + lambda2 v2, every
//                   product and sum rounded separately, as on the host
//   k_leaf_keys     leaf coordinates floor((x - origin) / w_L), clamped, and Morton keys
//   radix_sort      stable LSD radix sort of (key, point id), 4 bits per pass
//   k_flags/scan    occupied boxes of every level (sorted unique keys), the points of each
//                   leaf (ascending id), parent links, octants and child ranges
//   k_il_*          interaction lists: at l0 every non-touching box, below it the children
//                   of the parent's neighbours that do not touch the box (count, then fill)
//   k_near_leaves   touching leaves of each leaf (itself included)
//   k_leaf_tri      the triangles with a point in each leaf (ascending)
//
// The small per-level steps (decoding keys to coordinates, the coarsest far level, the
// distinct offsets of an interaction list) reuse the host functions on the downloaded
// arrays.  Determinism: every output position is computed from prefix sums in a fixed
// order; no atomics decide an order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nesa_device.cuh"

namespace nesa {
namespace tree {

__constant__ double c_bary[7][3];

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}
__device__ __forceinline__ uint64_t morton(int32_t i, int32_t j, int32_t k) {
  return spread3((uint64_t)i) | (spread3((uint64_t)j) << 1) | (spread3((uint64_t)k) << 2);
}

// point 7t + i of triangle t, coordinate x: (B_i0 v0 + B_i1 v1) + B_i2 v2, each operation
// rounded on its own (no fused multiply-add), as the host evaluates it
__global__ void k_points(double *__restrict__ pts, const double *__restrict__ verts, const int32_t *__restrict__ tris,
                         int64_t nt) {
  const int64_t n = 7 * nt * 3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % 3);
    const int64_t q = idx / 3;
    const int64_t t = q / 7;
    const int i = (int)(q % 7);
    const double v0 = verts[3 * (int64_t)tris[3 * t + 0] + x];
    const double v1 = verts[3 * (int64_t)tris[3 * t + 1] + x];
    const double v2 = verts[3 * (int64_t)tris[3 * t + 2] + x];
    const double r = __dadd_rn(__dmul_rn(c_bary[i][0], v0), __dmul_rn(c_bary[i][1], v1));
    pts[idx] = __dadd_rn(r, __dmul_rn(c_bary[i][2], v2));
  }
}

// leaf coordinates floor((x - origin) / w) clamped to [0, nb - 1], Morton key, point id
__global__ void k_leaf_keys(int32_t *__restrict__ ijk, uint64_t *__restrict__ key, int32_t *__restrict__ pid,
                            const double *__restrict__ pts, int64_t np, double ox, double oy, double oz, double w,
                            int32_t nb) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
    const double o[3] = {ox, oy, oz};
    int32_t c[3];
    for (int x = 0; x < 3; ++x) {
      const double f = floor(__ddiv_rn(__dsub_rn(pts[3 * q + x], o[x]), w));
      c[x] = f < 0.0 ? 0 : (f > nb - 1 ? nb - 1 : (int32_t)f);
      ijk[3 * q + x] = c[x];
    }
    key[q] = morton(c[0], c[1], c[2]);
    pid[q] = (int32_t)q;
  }
}

// ------------------------------------------------------------------ inclusive scan (int32)
constexpr int SCAN_BS = 1024;

__device__ __forceinline__ int32_t block_inclusive_scan(int32_t v, int32_t *warp_sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  if (lane == 31) warp_sums[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += u;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  if (warp > 0) v += warp_sums[warp - 1];
  return v;
}

__global__ void k_scan_blocks(int32_t *__restrict__ out, const int32_t *__restrict__ in, int64_t n,
                              int32_t *__restrict__ block_sums) {
  __shared__ int32_t ws[32];
  const int64_t i = blockIdx.x * (int64_t)SCAN_BS + threadIdx.x;
  const int32_t v = block_inclusive_scan(i < n ? in[i] : 0, ws);
  if (i < n) out[i] = v;
  if (threadIdx.x == SCAN_BS - 1) block_sums[blockIdx.x] = v;
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ block_prefix) {
  const int64_t i = blockIdx.x * (int64_t)SCAN_BS + threadIdx.x;
  if (blockIdx.x > 0 && i < n) out[i] += block_prefix[blockIdx.x - 1];
}

// out = inclusive prefix sums of in (n entries; the total must fit int32)
static void inclusive_scan(int32_t *out, const int32_t *in, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t nb = (n + SCAN_BS - 1) / SCAN_BS;
  int32_t *sums = nullptr;
  check_cuda(cudaMalloc(&sums, sizeof(int32_t) * nb), "scan sums");
  k_scan_blocks<<<(unsigned)nb, SCAN_BS, 0, st>>>(out, in, n, sums);
  check_cuda(cudaGetLastError(), "scan");
  if (nb > 1) {
    inclusive_scan(sums, sums, nb, st);
    k_scan_add<<<(unsigned)nb, SCAN_BS, 0, st>>>(out, n, sums);
    check_cuda(cudaGetLastError(), "scan add");
  }
  check_cuda(cudaStreamSynchronize(st), "scan");
  cudaFree(sums);
}

// ------------------------------------------------------------------ stable radix sort
// (key, value) pairs by the low `bits` bits of the key, 4 bits per pass.  Each block sorts
// RS_ITEMS consecutive pairs per thread; the counts per (digit, block) are scanned digit
// by digit and block by block, and each thread's pairs go out in their input order, so
// equal keys keep their order.
constexpr int RS_BS = 256, RS_ITEMS = 8, RS_TILE = RS_BS * RS_ITEMS, RS_DIGITS = 16;

__global__ void k_rs_count(const uint64_t *__restrict__ key, int64_t n, int shift, int32_t *__restrict__ counts,
                           int64_t nblocks) {
  __shared__ int32_t cnt[RS_DIGITS];
  if (threadIdx.x < RS_DIGITS) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_BS) {
    const int64_t i = base + k;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 15], 1);  // a count: the order of the adds does not matter
  }
  __syncthreads();
  if (threadIdx.x < RS_DIGITS) counts[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(uint64_t *__restrict__ key_out, int32_t *__restrict__ val_out,
                             const uint64_t *__restrict__ key_in, const int32_t *__restrict__ val_in, int64_t n,
                             int shift, const int32_t *__restrict__ incl, int64_t nblocks) {
  __shared__ int32_t tc[RS_DIGITS][RS_BS];  // per-thread digit counts, then their exclusive prefix over threads
  __shared__ int32_t ws[32];
  const int64_t base = blockIdx.x * (int64_t)RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  int32_t my[RS_DIGITS];
#pragma unroll
  for (int d = 0; d < RS_DIGITS; ++d) my[d] = 0;
  uint64_t k[RS_ITEMS];
  int32_t v[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t i = base + j;
    k[j] = i < n ? key_in[i] : 0;
    v[j] = i < n ? val_in[i] : 0;
    if (i < n) my[(k[j] >> shift) & 15]++;
  }
  for (int d = 0; d < RS_DIGITS; ++d) {
    const int32_t incl_t = block_inclusive_scan(my[d], ws);
    tc[d][threadIdx.x] = incl_t - my[d];
    __syncthreads();
  }
  int32_t pos[RS_DIGITS];
#pragma unroll
  for (int d = 0; d < RS_DIGITS; ++d) {
    const int64_t slot = (int64_t)d * nblocks + blockIdx.x;
    const int32_t before = slot > 0 ? incl[slot - 1] : 0;  // all earlier (digit, block) counts
    pos[d] = before + tc[d][threadIdx.x];
  }
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t i = base + j;
    if (i < n) {
      const int d = (int)((k[j] >> shift) & 15);
      key_out[pos[d]] = k[j];
      val_out[pos[d]] = v[j];
      pos[d]++;
    }
  }
}

// sorts (key, val) in place by the low `bits` bits of the keys
static void radix_sort(uint64_t *key, int32_t *val, int64_t n, int bits, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return;
  const int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
  uint64_t *k2 = nullptr;
  int32_t *v2 = nullptr, *counts = nullptr;
  check_cuda(cudaMalloc(&k2, sizeof(uint64_t) * n), "sort keys");
  check_cuda(cudaMalloc(&v2, sizeof(int32_t) * n), "sort values");
  check_cuda(cudaMalloc(&counts, sizeof(int32_t) * RS_DIGITS * nblocks), "sort counts");
  uint64_t *ka = key, *kb = k2;
  int32_t *va = val, *vb = v2;
  for (int shift = 0; shift < bits; shift += 4) {
    k_rs_count<<<(unsigned)nblocks, RS_BS, 0, st>>>(ka, n, shift, counts, nblocks);
    check_cuda(cudaGetLastError(), "sort count");
    inclusive_scan(counts, counts, RS_DIGITS * nblocks, st);
    k_rs_scatter<<<(unsigned)nblocks, RS_BS, 0, st>>>(kb, vb, ka, va, n, shift, counts, nblocks);
    check_cuda(cudaGetLastError(), "sort scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != key) {
    check_cuda(cudaMemcpyAsync(key, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st), "sort copy");
    check_cuda(cudaMemcpyAsync(val, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st), "sort copy");
  }
  check_cuda(cudaStreamSynchronize(st), "sort");
  cudaFree(k2);
  cudaFree(v2);
  cudaFree(counts);
}

// ------------------------------------------------------------------ boxes
// flag[i] = 1 where (key[i] >> shift) starts a new run of the sorted keys
__global__ void k_flags(int32_t *__restrict__ flag, const uint64_t *__restrict__ key, int64_t n, int shift) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1 : 0;
}

// run starts: box key and first position; every element's box index (run - 1)
__global__ void k_compact(uint64_t *__restrict__ box_key, int32_t *__restrict__ box_start,
                          int32_t *__restrict__ box_of, const uint64_t *__restrict__ key, const int32_t *__restrict__ flag,
                          const int32_t *__restrict__ run, int64_t n, int shift) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = run[i] - 1;
    if (box_of) box_of[i] = b;
    if (flag[i]) {
      box_key[b] = key[i] >> shift;
      box_start[b] = (int32_t)i;
    }
  }
}

__global__ void k_scatter_leaf(int32_t *__restrict__ pt_leaf, const int32_t *__restrict__ pid,
                               const int32_t *__restrict__ box_of, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pt_leaf[pid[i]] = box_of[i];
}

// ------------------------------------------------------------------ lists
__device__ __forceinline__ int32_t find_key(const uint64_t *__restrict__ keys, int32_t n, uint64_t k) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (keys[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < n && keys[lo] == k) ? lo : -1;
}

__device__ __forceinline__ bool touch(const int32_t *a, const int32_t *b) {
  return abs(a[0] - b[0]) <= 1 && abs(a[1] - b[1]) <= 1 && abs(a[2] - b[2]) <= 1;
}

// Interaction list of box a at level l (ascending sources): count (out == nullptr) or fill.
// At l0 (pkeys == nullptr) every non-touching box; below, the children of the parent's
// neighbours (ascending parent index) that do not touch a.
__global__ void k_il(int32_t *__restrict__ count, const int32_t *__restrict__ ptr, int32_t *__restrict__ tgt,
                     int32_t *__restrict__ src, int32_t *__restrict__ off, const int32_t *__restrict__ ijk,
                     int32_t nbox, const int32_t *__restrict__ parent, const uint64_t *__restrict__ pkeys,
                     const int32_t *__restrict__ pijk, int32_t npbox, const int32_t *__restrict__ child_ptr) {
  const int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nbox) return;
  const int32_t *ca = ijk + 3 * a;
  int32_t c = 0, at = ptr ? ptr[a] : 0;
  auto add = [&](int32_t b) {
    const int32_t *cb = ijk + 3 * b;
    if (touch(ca, cb)) return;
    if (ptr) {
      tgt[at] = a;
      src[at] = b;
      off[3 * at + 0] = ca[0] - cb[0];
      off[3 * at + 1] = ca[1] - cb[1];
      off[3 * at + 2] = ca[2] - cb[2];
      ++at;
    }
    ++c;
  };
  if (!pkeys) {
    for (int32_t b = 0; b < nbox; ++b) add(b);
  } else {
    const int32_t *cp = pijk + 3 * parent[a];
    int32_t cand[27];
    int nc = 0;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          const int32_t x = cp[0] + dx, y = cp[1] + dy, z = cp[2] + dz;
          if (x < 0 || y < 0 || z < 0) continue;
          const int32_t p2 = find_key(pkeys, npbox, morton(x, y, z));
          if (p2 >= 0) cand[nc++] = p2;
        }
    for (int i = 1; i < nc; ++i)  // ascending parent index
      for (int j = i; j > 0 && cand[j - 1] > cand[j]; --j) {
        const int32_t t = cand[j];
        cand[j] = cand[j - 1];
        cand[j - 1] = t;
      }
    for (int i = 0; i < nc; ++i)
      for (int32_t b = child_ptr[cand[i]]; b < child_ptr[cand[i] + 1]; ++b) add(b);
  }
  if (!ptr) count[a] = c;
}

// touching leaves of every leaf (itself included), in (dx, dy, dz) order: count or fill
__global__ void k_near_leaves(int32_t *__restrict__ count, const int32_t *__restrict__ ptr, int32_t *__restrict__ nl,
                              const int32_t *__restrict__ ijk, const uint64_t *__restrict__ keys, int32_t nleaf,
                              int32_t nb) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nleaf) return;
  const int32_t *c = ijk + 3 * b;
  int32_t n = 0, at = ptr ? ptr[b] : 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        const int32_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
        if (x < 0 || y < 0 || z < 0 || x >= nb || y >= nb || z >= nb) continue;
        const int32_t f = find_key(keys, nleaf, morton(x, y, z));
        if (f < 0) continue;
        if (ptr) nl[at++] = f;
        ++n;
      }
  if (!ptr) count[b] = n;
}

// triangles of the points sorted by (leaf, point id): a new entry where the leaf or the
// triangle changes
__global__ void k_leaf_tri_flags(int32_t *__restrict__ flag, const int32_t *__restrict__ box_of,
                                 const int32_t *__restrict__ pid, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || box_of[i] != box_of[i - 1] || pid[i] / 7 != pid[i - 1] / 7) ? 1 : 0;
}
__global__ void k_leaf_tri(int32_t *__restrict__ tri, int32_t *__restrict__ leaf_start, const int32_t *__restrict__ flag,
                           const int32_t *__restrict__ run, const int32_t *__restrict__ box_of,
                           const int32_t *__restrict__ pid, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      const int32_t e = run[i] - 1;
      tri[e] = pid[i] / 7;
      if (i == 0 || box_of[i] != box_of[i - 1]) leaf_start[box_of[i]] = e;
    }
}

static inline unsigned grid_of(int64_t n, int bs = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + bs - 1) / bs, 1 << 20));
}

template <typename T>
static std::vector<T> download(const T *d, int64_t n) {
  std::vector<T> h(std::max<int64_t>(n, 0));
  if (n > 0) check_cuda(cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost), "download");
  return h;
}

template <typename T>
struct DevBuf {  // temporary device buffer, freed on scope exit
  T *p = nullptr;
  explicit DevBuf(int64_t n) { check_cuda(cudaMalloc(&p, sizeof(T) * std::max<int64_t>(n, 1)), "tree buffer"); }
  ~DevBuf() { cudaFree(p); }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
};

// CSR from per-row counts (counts has n entries): ptr[0] = 0, ptr[i + 1] = sum of counts[0..i]
static std::vector<int32_t> csr_from_counts(int32_t *d_counts, int64_t n, cudaStream_t st, int32_t *d_ptr) {
  inclusive_scan(d_ptr + 1, d_counts, n, st);
  check_cuda(cudaMemsetAsync(d_ptr, 0, sizeof(int32_t), st), "ptr");
  return download(d_ptr, n + 1);
}

}  // namespace tree

void device_tree(nesa_ctx *c, const nesa_params &p, HostModel &m) {
  using namespace tree;
  cudaStream_t st = c->stream;
  {
    double B[7][3];
    rule7_nodes(B);
    check_cuda(cudaMemcpyToSymbol(c_bary, B, sizeof(B)), "nodes");
  }
  m.np = 7 * m.nt;
  const int64_t np = m.np;
  if (np >= INT32_MAX) fail(NESA_ERR_INVALID_ARG, "too many quadrature points for the device tree");
  // mesh on the device (kept by the context) and the quadrature points
  c->d_verts = (double *)dalloc(c, sizeof(double) * 3 * (size_t)m.nv);
  c->d_tris = (int32_t *)dalloc(c, sizeof(int32_t) * 3 * (size_t)m.nt);
  check_cuda(cudaMemcpy(c->d_verts, m.verts.data(), sizeof(double) * 3 * m.nv, cudaMemcpyHostToDevice), "verts");
  check_cuda(cudaMemcpy(c->d_tris, m.tris.data(), sizeof(int32_t) * 3 * m.nt, cudaMemcpyHostToDevice), "tris");
  c->d_pts = (double *)dalloc(c, sizeof(double) * 3 * (size_t)np);
  k_points<<<grid_of(3 * np), 256, 0, st>>>(c->d_pts, c->d_verts, c->d_tris, m.nt);
  check_cuda(cudaGetLastError(), "points");
  m.pts = download(c->d_pts, 3 * np);

  double lo[3], hi[3];
  const double root = host_root(p, m, lo, hi);
  const double wl = root / std::ldexp(1.0, m.L);
  const int32_t nb = 1 << m.L;

  // leaf coordinates, keys, sort by (key, point id)
  DevBuf<int32_t> ijk(3 * np), pid(np), flag(np), run(np), box_of(np);
  DevBuf<uint64_t> key(np);
  k_leaf_keys<<<grid_of(np), 256, 0, st>>>(ijk.p, key.p, pid.p, c->d_pts, np, m.origin[0], m.origin[1],
                                           m.origin[2], wl, nb);
  check_cuda(cudaGetLastError(), "leaf keys");
  m.pt_leaf_ijk = download(ijk.p, 3 * np);
  radix_sort(key.p, pid.p, np, 3 * m.L, st);

  // leaves: runs of equal keys
  k_flags<<<grid_of(np), 256, 0, st>>>(flag.p, key.p, np, 0);
  inclusive_scan(run.p, flag.p, np, st);
  int32_t nleaf = 0;
  check_cuda(cudaMemcpy(&nleaf, run.p + np - 1, sizeof(int32_t), cudaMemcpyDeviceToHost), "leaf count");
  m.lev.assign(m.L + 1, HostLevel());
  std::vector<DevBuf<uint64_t> *> lkeys(m.L + 1, nullptr);
  std::vector<DevBuf<int32_t> *> lijk(m.L + 1, nullptr), lchild(m.L + 1, nullptr), lparent(m.L + 1, nullptr);
  auto cleanup = [&]() {
    for (auto *x : lkeys) delete x;
    for (auto *x : lijk) delete x;
    for (auto *x : lchild) delete x;
    for (auto *x : lparent) delete x;
  };
  try {
    {
      lkeys[m.L] = new DevBuf<uint64_t>(nleaf);
      DevBuf<int32_t> start(nleaf + 1);
      k_compact<<<grid_of(np), 256, 0, st>>>(lkeys[m.L]->p, start.p, box_of.p, key.p, flag.p, run.p, np, 0);
      check_cuda(cudaGetLastError(), "leaves");
      m.leaf_pt_ptr = download(start.p, nleaf);
      m.leaf_pt_ptr.push_back((int32_t)np);
      m.leaf_pt = download(pid.p, np);
      DevBuf<int32_t> ptl(np);
      k_scatter_leaf<<<grid_of(np), 256, 0, st>>>(ptl.p, pid.p, box_of.p, np);
      check_cuda(cudaGetLastError(), "point leaves");
      m.pt_leaf = download(ptl.p, np);
    }
    // coarser levels: runs of key >> 3 among the keys of the level below
    for (int l = m.L; l >= 0; --l) {
      HostLevel &lv = m.lev[l];
      lv.width = root / std::ldexp(1.0, l);
      const int32_t n = l == m.L ? nleaf : (int32_t)m.lev[l].key.size();
      if (l < m.L) {
        const int32_t nc = (int32_t)m.lev[l + 1].key.size();
        DevBuf<int32_t> f(nc), r(nc), start(nc);
        k_flags<<<grid_of(nc), 256, 0, st>>>(f.p, lkeys[l + 1]->p, nc, 3);
        inclusive_scan(r.p, f.p, nc, st);
        int32_t np_l = 0;
        check_cuda(cudaMemcpy(&np_l, r.p + nc - 1, sizeof(int32_t), cudaMemcpyDeviceToHost), "boxes");
        lkeys[l] = new DevBuf<uint64_t>(np_l);
        lparent[l + 1] = new DevBuf<int32_t>(nc);
        k_compact<<<grid_of(nc), 256, 0, st>>>(lkeys[l]->p, start.p, lparent[l + 1]->p, lkeys[l + 1]->p, f.p, r.p, nc,
                                               3);
        check_cuda(cudaGetLastError(), "levels");
        std::vector<int32_t> cp = download(start.p, np_l);
        cp.push_back(nc);
        lchild[l] = new DevBuf<int32_t>(np_l + 1);
        check_cuda(cudaMemcpy(lchild[l]->p, cp.data(), sizeof(int32_t) * cp.size(), cudaMemcpyHostToDevice), "children");
        lv.child_ptr = cp;
        m.lev[l + 1].parent = download(lparent[l + 1]->p, nc);
        lv.key = download(lkeys[l]->p, np_l);
      } else {
        lv.key = download(lkeys[l]->p, n);
        lv.child_ptr.assign(n + 1, 0);
      }
      decode_keys(lv);
      lijk[l] = new DevBuf<int32_t>(3 * (int64_t)lv.key.size());
      check_cuda(cudaMemcpy(lijk[l]->p, lv.ijk.data(), sizeof(int32_t) * lv.ijk.size(), cudaMemcpyHostToDevice), "ijk");
    }
    for (int l = 0; l <= m.L; ++l) {
      HostLevel &lv = m.lev[l];
      lv.octant.assign(lv.key.size(), 0);
      if (l == 0) {
        lv.parent.assign(lv.key.size(), -1);
      } else {
        for (size_t b = 0; b < lv.key.size(); ++b) lv.octant[b] = (int32_t)(lv.key[b] & 7ULL);
      }
    }
    m.l0 = coarsest_far_level(m, lo, hi);

    // interaction lists of the far levels
    for (int l = m.l0; l <= m.L; ++l) {
      HostLevel &lv = m.lev[l];
      const int32_t n = (int32_t)lv.key.size();
      const bool top = l == m.l0;
      DevBuf<int32_t> cnt(n), ptr(n + 1);
      const int32_t npb = top ? 0 : (int32_t)m.lev[l - 1].key.size();
      k_il<<<grid_of(n, 128), 128, 0, st>>>(cnt.p, nullptr, nullptr, nullptr, nullptr, lijk[l]->p, n,
                                            top ? nullptr : lparent[l]->p, top ? nullptr : lkeys[l - 1]->p,
                                            top ? nullptr : lijk[l - 1]->p, npb, top ? nullptr : lchild[l - 1]->p);
      check_cuda(cudaGetLastError(), "interaction count");
      std::vector<int32_t> hp = csr_from_counts(cnt.p, n, st, ptr.p);
      const int64_t ne = hp[n];
      DevBuf<int32_t> tgt(ne), src(ne), off(3 * ne);
      k_il<<<grid_of(n, 128), 128, 0, st>>>(nullptr, ptr.p, tgt.p, src.p, off.p, lijk[l]->p, n,
                                            top ? nullptr : lparent[l]->p, top ? nullptr : lkeys[l - 1]->p,
                                            top ? nullptr : lijk[l - 1]->p, npb, top ? nullptr : lchild[l - 1]->p);
      check_cuda(cudaGetLastError(), "interaction fill");
      finish_interactions(lv, download(tgt.p, ne), download(src.p, ne), download(off.p, 3 * ne));
    }

    // touching leaves of every leaf, and the triangles of every leaf
    {
      DevBuf<int32_t> cnt(nleaf), ptr(nleaf + 1);
      k_near_leaves<<<grid_of(nleaf, 128), 128, 0, st>>>(cnt.p, nullptr, nullptr, lijk[m.L]->p, lkeys[m.L]->p, nleaf,
                                                          nb);
      check_cuda(cudaGetLastError(), "near leaves");
      m.nl_ptr = csr_from_counts(cnt.p, nleaf, st, ptr.p);
      DevBuf<int32_t> nl(m.nl_ptr[nleaf]);
      k_near_leaves<<<grid_of(nleaf, 128), 128, 0, st>>>(nullptr, ptr.p, nl.p, lijk[m.L]->p, lkeys[m.L]->p, nleaf, nb);
      check_cuda(cudaGetLastError(), "near leaves");
      m.nl = download(nl.p, m.nl_ptr[nleaf]);
    }
    {
      k_leaf_tri_flags<<<grid_of(np), 256, 0, st>>>(flag.p, box_of.p, pid.p, np);
      inclusive_scan(run.p, flag.p, np, st);
      int32_t ne = 0;
      check_cuda(cudaMemcpy(&ne, run.p + np - 1, sizeof(int32_t), cudaMemcpyDeviceToHost), "leaf triangles");
      DevBuf<int32_t> tri(ne), start(nleaf);
      k_leaf_tri<<<grid_of(np), 256, 0, st>>>(tri.p, start.p, flag.p, run.p, box_of.p, pid.p, np);
      check_cuda(cudaGetLastError(), "leaf triangles");
      m.leaf_tri = download(tri.p, ne);
      m.leaf_tri_ptr = download(start.p, nleaf);
      m.leaf_tri_ptr.push_back(ne);
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

}  // namespace nesa
