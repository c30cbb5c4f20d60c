// Preconditioners for nesa_solve: block-Jacobi on the near field and a learned
// correction of it.
//
// Block-Jacobi (fallback).  Every RWG function belongs to the leaf that holds the
// centroid of its T+ ("home leaf"); the group of a leaf is its RWG functions in
// ascending order.  The diagonal block of Z^near over a group is inverted once
// (Gauss-Jordan with partial pivoting, FP64) and BJ r applies the inverses.
//
// Learned preconditioner.  M u = a1 * u + a2 * (BJ u) + a3 * (BJ N BJ u), with N the
// near-field product and a1..a3 complex coefficients per RWG function given by a small
// network with weights shared by all functions:
//     features x (8) -> tanh(W1 x + b1) (32) -> tanh(W2 h1 + b2) (32) -> W3 h2 + b3 (6)
// The features are local and static: k l, A+/l^2, A-/l^2, the phase and the relative
// magnitude of Z_mm, the relative near-row length and group size.  The network starts
// at a = (0, 1, 0), i.e. block-Jacobi.  It is trained on the GPU by the kernels below
// (forward, backward, Adam) to minimise  sum_s ||M(Z v_s) - v_s||^2 / sum_s ||v_s||^2
// over the Arnoldi vectors v_s that block-Jacobi GMRES produces for the training
// right-hand sides.  Once trained, a is fixed, so M is linear and right-preconditioned
// GMRES applies.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_fp16.h>
#include <cusolverDn.h>

#include <unordered_map>

#include "nesa_device.cuh"

namespace nesa {

constexpr int NF = 8, NH = 32, NO = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;  // 1542
static_assert(NPARAM == NESA_LEARN_PARAMS, "parameter count");

struct Precond {
  bool ready = false;
  // overlapping block-Jacobi (restricted additive Schwarz): rows of group g of the
  // inverse of the near-field block over E_g = functions whose home leaf touches g's
  bool ras_ready = false;
  int emax = 0;
  int32_t *e_ptr = nullptr, *e_rwg = nullptr;  // extended sets (CSR by group)
  int64_t *r_off = nullptr;                    // offset of R_g ([|g|][|E_g|] row-major)
  cplxf *R = nullptr;
  std::vector<int32_t> h_gptr, h_grwg, h_gleaf;  // host copies of the groups, leaf of each
  int64_t ngroup = 0;
  int smax = 0;
  int32_t *g_ptr = nullptr, *g_rwg = nullptr;  // groups (CSR), RWG ids
  int64_t *g_off = nullptr;                    // offset of each block (S^2 entries)
  cplx *inv = nullptr;                         // inverted blocks, column-major
  float *feat = nullptr;                       // [n][8]
  // network
  bool trained = false;
  float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr, *gpart = nullptr;
  __half *theta16 = nullptr;                   // inference copy of the weights
  float *coef = nullptr;                       // [n][6] coefficients a (re, im) x 3
  float *h1 = nullptr, *h2 = nullptr;          // [n][32] activations (training)
  float *ga = nullptr;                         // [n][6] dL/da
  double *lpart = nullptr;                     // loss partial sums
  cplx *t1 = nullptr, *t2 = nullptr;           // scratch vectors [cap][n]
  int tcap = 0;
  double vn2 = 1.0;                            // sum of |v_s|^2 of the training samples
  std::vector<float> h_theta;
};

static Precond *P_(nesa_ctx *c) { return (Precond *)c->precond; }

// ------------------------------------------------------------------ block-Jacobi
// near-field diagonal block of group g into blk + 2 g_off[g] (the left half of the
// S x 2S Gauss-Jordan work matrix, column-major with leading dimension S)
__global__ void k_group_blocks(cplx *blk, const int64_t *g_off, const int32_t *g_ptr, const int32_t *g_rwg,
                               const int64_t *nz_ptr, const int32_t *nz_col, const cplx *nz_val) {
  const int64_t g = blockIdx.x;
  const int32_t p0 = g_ptr[g], S = g_ptr[g + 1] - p0;
  cplx *B = blk + 2 * g_off[g];
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e % S, j = e / S;
    const int32_t m = g_rwg[p0 + i], n = g_rwg[p0 + j];
    int64_t lo = nz_ptr[m], hi = nz_ptr[m + 1];
    cplx v = make_double2(0.0, 0.0);
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      const int32_t cc = nz_col[mid];
      if (cc == n) {
        v = nz_val[mid];
        break;
      }
      if (cc < n)
        lo = mid + 1;
      else
        hi = mid;
    }
    B[i + (int64_t)j * S] = v;
  }
}

// Gauss-Jordan with partial pivoting on [A | I] (S x 2S, column-major, in global
// memory), one block per group; the right half becomes A^-1 and is copied to inv.
__global__ void k_block_invert(cplx *inv, cplx *work, const int64_t *g_off, const int32_t *g_ptr, int *bad) {
  const int64_t g = blockIdx.x;
  const int S = g_ptr[g + 1] - g_ptr[g];
  cplx *A = work + 2 * g_off[g];  // S x 2S
  const int ld = S;
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e % S, j = e / S;
    A[i + (int64_t)(S + j) * ld] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __shared__ int piv;
  __shared__ double pmax[256];
  __shared__ int pidx[256];
  __syncthreads();
  for (int k = 0; k < S; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < S; i += blockDim.x) {
      const cplx v = A[i + (int64_t)k * ld];
      const double a = v.x * v.x + v.y * v.y;
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    pmax[threadIdx.x] = best;
    pidx[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int ii = k;
      for (int t = 0; t < (int)blockDim.x; ++t)
        if (pmax[t] > b) {
          b = pmax[t];
          ii = pidx[t];
        }
      piv = ii;
      if (!(b > 0.0)) atomicExch(bad, 1);
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = threadIdx.x; j < 2 * S; j += blockDim.x) {
        const cplx t = A[k + (int64_t)j * ld];
        A[k + (int64_t)j * ld] = A[p + (int64_t)j * ld];
        A[p + (int64_t)j * ld] = t;
      }
    __syncthreads();
    const cplx d = A[k + (int64_t)k * ld];
    const double dd = d.x * d.x + d.y * d.y;
    const cplx di = dd > 0.0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0.0, 0.0);
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * S; j += blockDim.x) A[k + (int64_t)j * ld] = cmul(A[k + (int64_t)j * ld], di);
    __syncthreads();
    // eliminate column k from every other row
    for (int e = threadIdx.x; e < S * 2 * S; e += blockDim.x) {
      const int i = e % S, j = e / S;
      if (i == k || j == k) continue;
      const cplx f = A[i + (int64_t)k * ld];
      const cplx r = A[k + (int64_t)j * ld];
      A[i + (int64_t)j * ld] = make_double2(A[i + (int64_t)j * ld].x - (f.x * r.x - f.y * r.y),
                                            A[i + (int64_t)j * ld].y - (f.x * r.y + f.y * r.x));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S; i += blockDim.x)
      if (i != k) A[i + (int64_t)k * ld] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  cplx *I = inv + g_off[g];
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e % S, j = e / S;
    I[i + (int64_t)j * S] = A[i + (int64_t)(S + j) * ld];
  }
}

// z = BJ r for nrhs columns (grid: groups x nrhs)
__global__ void k_bj_apply(cplx *z, const cplx *r, int64_t n, const int64_t *g_off, const int32_t *g_ptr,
                           const int32_t *g_rwg, const cplx *inv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx *rs = (cplx *)smem_raw;
  const int64_t g = blockIdx.x;
  const int col = blockIdx.y;
  const int32_t p0 = g_ptr[g], S = g_ptr[g + 1] - p0;
  const cplx *rr = r + (int64_t)col * n;
  for (int j = threadIdx.x; j < S; j += blockDim.x) rs[j] = rr[g_rwg[p0 + j]];
  __syncthreads();
  const cplx *I = inv + g_off[g];
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    cplx acc = make_double2(0.0, 0.0);
    for (int j = 0; j < S; ++j) cfma(acc, I[i + (int64_t)j * S], rs[j]);
    z[(int64_t)col * n + g_rwg[p0 + i]] = acc;
  }
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ void mlp_forward(const float *th, const float *x, float *h1, float *h2, float *a) {
  for (int i = 0; i < NH; ++i) {
    float s = th[OFF_B1 + i];
    for (int j = 0; j < NF; ++j) s = fmaf(th[OFF_W1 + i * NF + j], x[j], s);
    h1[i] = tanhf(s);
  }
  for (int i = 0; i < NH; ++i) {
    float s = th[OFF_B2 + i];
    for (int j = 0; j < NH; ++j) s = fmaf(th[OFF_W2 + i * NH + j], h1[j], s);
    h2[i] = tanhf(s);
  }
  for (int i = 0; i < NO; ++i) {
    float s = th[OFF_B3 + i];
    for (int j = 0; j < NH; ++j) s = fmaf(th[OFF_W3 + i * NH + j], h2[j], s);
    a[i] = s;
  }
}

// inference: coefficients of every RWG function from the FP16 weights (FP32 arithmetic)
__global__ void k_mlp_infer(float *coef, const float *feat, const __half *th16, int64_t n) {
  __shared__ float th[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) th[i] = __half2float(th16[i]);
  __syncthreads();
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= n) return;
  float h1[NH], h2[NH], a[NO];
  mlp_forward(th, feat + m * NF, h1, h2, a);
  for (int i = 0; i < NO; ++i) coef[m * NO + i] = a[i];
}

// training forward: coefficients and activations with the FP32 weights
__global__ void k_mlp_train_forward(float *coef, float *H1, float *H2, const float *feat, const float *theta,
                                    int64_t n) {
  __shared__ float th[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= n) return;
  float a[NO];
  mlp_forward(th, feat + m * NF, H1 + m * NH, H2 + m * NH, a);
  for (int i = 0; i < NO; ++i) coef[m * NO + i] = a[i];
}

// z = a1 u + a2 f2 + a3 f3 per RWG function and column
__global__ void k_combine(cplx *z, const cplx *u, const cplx *f2, const cplx *f3, const float *coef, int64_t n,
                          int nrhs) {
  const int64_t total = n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e % n;
    const float *a = coef + m * NO;
    cplx acc = cmul(make_double2(a[0], a[1]), u[e]);
    acc = cadd(acc, cmul(make_double2(a[2], a[3]), f2[e]));
    acc = cadd(acc, cmul(make_double2(a[4], a[5]), f3[e]));
    z[e] = acc;
  }
}

// loss and dL/da over ns samples: e = sum_k a_k f_k - v; L = sum |e|^2 / vnorm2
// features of sample s: f1 = U[s], f2 = F2[s], f3 = F3[s]; target V[s]
__global__ void k_loss_grad_a(float *ga, double *lpart, const float *coef, const cplx *U, const cplx *F2,
                              const cplx *F3, const cplx *V, int64_t n, int ns, double inv_vnorm2) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double loss = 0.0;
  if (m < n) {
    const float *a = coef + m * NO;
    const cplx a1 = make_double2(a[0], a[1]), a2 = make_double2(a[2], a[3]), a3 = make_double2(a[4], a[5]);
    cplx G[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int s = 0; s < ns; ++s) {
      const int64_t e = (int64_t)s * n + m;
      const cplx f1 = U[e], f2 = F2[e], f3 = F3[e], v = V[e];
      cplx r = cadd(cadd(cmul(a1, f1), cmul(a2, f2)), cmul(a3, f3));
      r.x -= v.x;
      r.y -= v.y;
      loss += r.x * r.x + r.y * r.y;
      const cplx cr = make_double2(r.x, -r.y);
      G[0] = cadd(G[0], cmul(cr, f1));
      G[1] = cadd(G[1], cmul(cr, f2));
      G[2] = cadd(G[2], cmul(cr, f3));
    }
    for (int k = 0; k < 3; ++k) {
      ga[m * NO + 2 * k] = (float)(2.0 * G[k].x * inv_vnorm2);
      ga[m * NO + 2 * k + 1] = (float)(-2.0 * G[k].y * inv_vnorm2);
    }
  }
  // block sum of the loss
  __shared__ double sh[256];
  sh[threadIdx.x] = loss * inv_vnorm2;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = sh[0];
}

// backward through the network; per-block partial gradients gpart[block][NPARAM]
__global__ void __launch_bounds__(256) k_mlp_backward(float *gpart, const float *ga, const float *H1, const float *H2,
                                                      const float *feat, const float *theta, int64_t n) {
  __shared__ float th[NPARAM];
  __shared__ float acc[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    th[i] = theta[i];
    acc[i] = 0.0f;
  }
  __syncthreads();
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = m < n;
  float x[NF], h1[NH], h2[NH], g[NO], gz2[NH], gz1[NH];
  for (int i = 0; i < NF; ++i) x[i] = act ? feat[m * NF + i] : 0.0f;
  for (int i = 0; i < NH; ++i) {
    h1[i] = act ? H1[m * NH + i] : 0.0f;
    h2[i] = act ? H2[m * NH + i] : 0.0f;
  }
  for (int i = 0; i < NO; ++i) g[i] = act ? ga[m * NO + i] : 0.0f;
  for (int j = 0; j < NH; ++j) {
    float s = 0.0f;
    for (int i = 0; i < NO; ++i) s = fmaf(th[OFF_W3 + i * NH + j], g[i], s);
    gz2[j] = s * (1.0f - h2[j] * h2[j]);
  }
  for (int j = 0; j < NH; ++j) {
    float s = 0.0f;
    for (int i = 0; i < NH; ++i) s = fmaf(th[OFF_W2 + i * NH + j], gz2[i], s);
    gz1[j] = s * (1.0f - h1[j] * h1[j]);
  }
  // sum the per-function outer products over the warp, then over the block
  auto add = [&](int p, float v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[p], v);
  };
  for (int i = 0; i < NO; ++i) {
    add(OFF_B3 + i, g[i]);
    for (int j = 0; j < NH; ++j) add(OFF_W3 + i * NH + j, g[i] * h2[j]);
  }
  for (int i = 0; i < NH; ++i) {
    add(OFF_B2 + i, gz2[i]);
    for (int j = 0; j < NH; ++j) add(OFF_W2 + i * NH + j, gz2[i] * h1[j]);
  }
  for (int i = 0; i < NH; ++i) {
    add(OFF_B1 + i, gz1[i]);
    for (int j = 0; j < NF; ++j) add(OFF_W1 + i * NF + j, gz1[i] * x[j]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) gpart[(int64_t)blockIdx.x * NPARAM + i] = acc[i];
}

// grad[p] = sum over blocks (fixed order)
__global__ void k_grad_reduce(float *grad, const float *gpart, int nblocks) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float s = 0.0f;
  for (int b = 0; b < nblocks; ++b) s += gpart[(int64_t)b * NPARAM + p];
  grad[p] = s;
}

__global__ void k_adam(float *theta, float *m, float *v, const float *grad, float lr, float b1, float b2, float eps,
                       int t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float gr = grad[p];
  m[p] = b1 * m[p] + (1.0f - b1) * gr;
  v[p] = b2 * v[p] + (1.0f - b2) * gr * gr;
  const float mh = m[p] / (1.0f - powf(b1, (float)t)), vh = v[p] / (1.0f - powf(b2, (float)t));
  theta[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_to_half(__half *dst, const float *src, int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) dst[p] = __float2half_rn(src[p]);
}

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// diagonal Z^near_mm of every row (0 if absent)
__global__ void k_diag(cplx *d, const int64_t *nz_ptr, const int32_t *nz_col, const cplx *nz_val, int64_t n) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= n) return;
  int64_t lo = nz_ptr[m], hi = nz_ptr[m + 1];
  cplx v = make_double2(0.0, 0.0);
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    const int32_t cc = nz_col[mid];
    if (cc == m) {
      v = nz_val[mid];
      break;
    }
    if (cc < m)
      lo = mid + 1;
    else
      hi = mid;
  }
  d[m] = v;
}

// initial weights: small deterministic pseudo-random hidden layers, zero output layer
// and output bias (0,0, 1,0, 0,0) so that M = BJ
static void init_theta(std::vector<float> &th, uint32_t seed) {
  th.assign(NPARAM, 0.0f);
  uint64_t s = 0x9E3779B97F4A7C15ull ^ (uint64_t)seed;
  auto rnd = [&]() {  // splitmix64 -> uniform in [-1, 1)
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((double)(z >> 11) / 9007199254740992.0 * 2.0 - 1.0);
  };
  for (int i = 0; i < NH * NF; ++i) th[OFF_W1 + i] = rnd() / std::sqrt((float)NF);
  for (int i = 0; i < NH * NH; ++i) th[OFF_W2 + i] = rnd() / std::sqrt((float)NH);
  th[OFF_B3 + 2] = 1.0f;
}

static void ensure_scratch(nesa_ctx *c, Precond *P, int cols) {
  if (cols <= P->tcap) return;
  dfree(c, P->t1);
  dfree(c, P->t2);
  P->t1 = (cplx *)dalloc(c, sizeof(cplx) * (size_t)cols * c->n);
  P->t2 = (cplx *)dalloc(c, sizeof(cplx) * (size_t)cols * c->n);
  P->tcap = cols;
}

static void setup(nesa_ctx *c) {
  if (c->precond && P_(c)->ready) return;
  if (!c->precond) c->precond = new Precond();
  Precond *P = P_(c);
  const HostModel &h = c->h;
  const int64_t n = c->n;
  // groups by home leaf (leaf of the centroid of T+, quadrature node 0 of T+)
  const int64_t nleaf = c->nleaf;
  std::vector<int32_t> gp(nleaf + 1, 0), grwg(n);
  for (int64_t m = 0; m < n; ++m) gp[h.pt_leaf[7 * (int64_t)h.rwg_tri[2 * m]] + 1]++;
  for (int64_t b = 0; b < nleaf; ++b) gp[b + 1] += gp[b];
  {
    std::vector<int32_t> fill(gp.begin(), gp.end() - 1);
    for (int64_t m = 0; m < n; ++m) grwg[fill[h.pt_leaf[7 * (int64_t)h.rwg_tri[2 * m]]]++] = (int32_t)m;
  }
  // drop empty groups
  std::vector<int32_t> ptr{0};
  P->h_gleaf.clear();
  for (int64_t b = 0; b < nleaf; ++b)
    if (gp[b + 1] > gp[b]) {
      ptr.push_back(gp[b + 1]);
      P->h_gleaf.push_back((int32_t)b);
    }
  P->h_gptr = ptr;
  P->h_grwg = grwg;
  P->ngroup = (int64_t)ptr.size() - 1;
  std::vector<int64_t> off(P->ngroup + 1, 0);
  std::vector<int> gsize(n);
  double gsum = 0.0;
  for (int64_t g = 0; g < P->ngroup; ++g) {
    const int S = ptr[g + 1] - ptr[g];
    P->smax = std::max(P->smax, S);
    off[g + 1] = off[g] + (int64_t)S * S;
    for (int i = ptr[g]; i < ptr[g + 1]; ++i) gsize[grwg[i]] = S;
    gsum += (double)S * S;
  }
  P->g_ptr = (int32_t *)dalloc(c, sizeof(int32_t) * ptr.size());
  P->g_rwg = (int32_t *)dalloc(c, sizeof(int32_t) * n);
  P->g_off = (int64_t *)dalloc(c, sizeof(int64_t) * off.size());
  check_cuda(cudaMemcpy(P->g_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice), "groups");
  check_cuda(cudaMemcpy(P->g_rwg, grwg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice), "groups");
  check_cuda(cudaMemcpy(P->g_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice), "groups");
  const int64_t tot = off[P->ngroup];
  P->inv = (cplx *)dalloc(c, sizeof(cplx) * (size_t)std::max<int64_t>(1, tot));
  cplx *work = nullptr;
  check_cuda(cudaMalloc(&work, sizeof(cplx) * (size_t)std::max<int64_t>(1, 2 * tot)), "bj work");
  int *bad = nullptr;
  check_cuda(cudaMalloc(&bad, sizeof(int)), "flag");
  check_cuda(cudaMemset(bad, 0, sizeof(int)), "flag");
  // the blocks are written into the left half of the work matrices ([A | I], ld = S)
  k_group_blocks<<<(unsigned)P->ngroup, 256, 0, c->stream>>>(work, P->g_off, P->g_ptr, P->g_rwg, c->d_nz_ptr,
                                                               c->d_nz_col, c->d_nz_val);
  k_block_invert<<<(unsigned)P->ngroup, 256, 0, c->stream>>>(P->inv, work, P->g_off, P->g_ptr, bad);
  check_cuda(cudaGetLastError(), "bj invert");
  int hbad = 0;
  check_cuda(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag");
  check_cuda(cudaStreamSynchronize(c->stream), "bj");
  cudaFree(work);
  cudaFree(bad);
  if (hbad) fail(NESA_ERR_NUMERIC, "singular near-field diagonal block");

  // static features (host, FP64, then FP32)
  std::vector<int64_t> nzp(n + 1);
  check_cuda(cudaMemcpy(nzp.data(), c->d_nz_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost), "nz ptr");
  std::vector<cplx> diag(n);
  {
    cplx *dd = nullptr;
    check_cuda(cudaMalloc(&dd, sizeof(cplx) * n), "diag");
    k_diag<<<nblk(n, 256), 256, 0, c->stream>>>(dd, c->d_nz_ptr, c->d_nz_col, c->d_nz_val, n);
    check_cuda(cudaMemcpyAsync(diag.data(), dd, sizeof(cplx) * n, cudaMemcpyDeviceToHost, c->stream), "diag");
    check_cuda(cudaStreamSynchronize(c->stream), "diag");
    cudaFree(dd);
  }
  double mag_mean = 0.0, nnz_mean = 0.0, gs_mean = 0.0;
  for (int64_t m = 0; m < n; ++m) {
    if (!(std::hypot(diag[m].x, diag[m].y) > 0.0)) fail(NESA_ERR_NUMERIC, "zero diagonal entry");
    mag_mean += std::hypot(diag[m].x, diag[m].y);
    nnz_mean += (double)(nzp[m + 1] - nzp[m]);
    gs_mean += gsize[m];
  }
  mag_mean /= n;
  nnz_mean /= n;
  gs_mean /= n;
  std::vector<float> feat((size_t)n * NF);
  auto area = [&](int32_t t) {
    const double *a = &h.verts[3 * (size_t)h.tris[3 * t]], *b = &h.verts[3 * (size_t)h.tris[3 * t + 1]],
                 *cc = &h.verts[3 * (size_t)h.tris[3 * t + 2]];
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
    const double x = e1[1] * e2[2] - e1[2] * e2[1], y = e1[2] * e2[0] - e1[0] * e2[2], z = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * std::sqrt(x * x + y * y + z * z);
  };
  for (int64_t m = 0; m < n; ++m) {
    const int32_t tp = h.rwg_tri[2 * m], tm = h.rwg_tri[2 * m + 1];
    const double l = std::fabs(h.tri_sl[3 * (size_t)tp + h.rwg_free[2 * m]]);
    const double mag = std::hypot(diag[m].x, diag[m].y);
    const double f[NF] = {c->k * l, area(tp) / (l * l), area(tm) / (l * l), diag[m].x / mag, diag[m].y / mag,
                          std::log(mag / mag_mean), (double)(nzp[m + 1] - nzp[m]) / nnz_mean, gsize[m] / gs_mean};
    for (int i = 0; i < NF; ++i) feat[(size_t)m * NF + i] = (float)f[i];
  }
  P->feat = (float *)dalloc(c, sizeof(float) * feat.size());
  check_cuda(cudaMemcpy(P->feat, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice), "features");
  // network state
  init_theta(P->h_theta, 1801);
  P->theta = (float *)dalloc(c, sizeof(float) * NPARAM);
  P->adam_m = (float *)dalloc(c, sizeof(float) * NPARAM);
  P->adam_v = (float *)dalloc(c, sizeof(float) * NPARAM);
  P->grad = (float *)dalloc(c, sizeof(float) * NPARAM);
  P->theta16 = (__half *)dalloc(c, sizeof(__half) * NPARAM);
  P->coef = (float *)dalloc(c, sizeof(float) * NO * (size_t)n);
  P->h1 = (float *)dalloc(c, sizeof(float) * NH * (size_t)n);
  P->h2 = (float *)dalloc(c, sizeof(float) * NH * (size_t)n);
  P->ga = (float *)dalloc(c, sizeof(float) * NO * (size_t)n);
  P->gpart = (float *)dalloc(c, sizeof(float) * NPARAM * (size_t)nblk(n, 256));
  P->lpart = (double *)dalloc(c, sizeof(double) * (size_t)nblk(n, 256));
  check_cuda(cudaMemcpy(P->theta, P->h_theta.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "theta");
  P->ready = true;
}

void precond_bj(nesa_ctx *c, const cplx *r, cplx *z, int nrhs) {
  Precond *P = P_(c);
  k_bj_apply<<<dim3((unsigned)P->ngroup, nrhs), 128, sizeof(cplx) * P->smax, c->stream>>>(z, r, c->n, P->g_off,
                                                                                         P->g_ptr, P->g_rwg, P->inv);
}

// ------------------------------------------------------------------ overlapping block-Jacobi
// near-field block over the extended set E (ne functions), column-major, complex64
__global__ void k_ext_block(cplxf *A, const int32_t *E, int ne, const int64_t *nz_ptr, const int32_t *nz_col,
                            const cplx *nz_val) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)ne * ne;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % ne), j = (int)(idx / ne);
    const int32_t m = E[i], nn = E[j];
    int64_t lo = nz_ptr[m], hi = nz_ptr[m + 1];
    cplxf v = make_float2(0.0f, 0.0f);
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      const int32_t cc = nz_col[mid];
      if (cc == nn) {
        v = make_float2((float)nz_val[mid].x, (float)nz_val[mid].y);
        break;
      }
      if (cc < nn)
        lo = mid + 1;
      else
        hi = mid;
    }
    A[idx] = v;
  }
}

// unit columns: B[:, j] = e_{pos[j]} (ne x s, column-major)
__global__ void k_unit_cols(cplxf *B, const int32_t *pos, int ne, int s) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ne * s; idx += gridDim.x * blockDim.x) {
    const int e = idx % ne, j = idx / ne;
    B[idx] = make_float2(e == pos[j] ? 1.0f : 0.0f, 0.0f);
  }
}

// R[i][e] = X[e][i]  (R: s x ne row-major, X: ne x s column-major)
__global__ void k_take_rows(cplxf *R, const cplxf *X, int ne, int s) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ne * s; idx += gridDim.x * blockDim.x) {
    const int e = idx % ne, i = idx / ne;
    R[(int64_t)i * ne + e] = X[e + (int64_t)i * ne];
  }
}

// z = RAS r: grid (groups, nrhs); one warp per row of R_g
__global__ void k_ras_apply(cplx *z, const cplx *r, int64_t n, const int32_t *g_ptr, const int32_t *g_rwg,
                            const int32_t *e_ptr, const int32_t *e_rwg, const int64_t *r_off, const cplxf *R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplxf *re = (cplxf *)smem_raw;
  const int64_t g = blockIdx.x;
  const int col = blockIdx.y;
  const int32_t e0 = e_ptr[g], ne = e_ptr[g + 1] - e0, p0 = g_ptr[g], S = g_ptr[g + 1] - p0;
  const cplx *rr = r + (int64_t)col * n;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const cplx v = rr[e_rwg[e0 + e]];
    re[e] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const cplxf *Rg = R + r_off[g];
  for (int i = warp; i < S; i += nw) {
    cplxf acc = make_float2(0.0f, 0.0f);
    for (int e = lane; e < ne; e += 32) cfma(acc, Rg[(int64_t)i * ne + e], re[e]);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) z[(int64_t)col * n + g_rwg[p0 + i]] = make_double2(acc.x, acc.y);
  }
}

static void ras_setup(nesa_ctx *c) {
  setup(c);
  Precond *P = P_(c);
  if (P->ras_ready) return;
  const HostModel &h = c->h;
  const HostLevel &lv = h.lev[h.L];
  // group of every leaf, leaf of a coordinate triple
  std::unordered_map<uint64_t, int32_t> group_of;  // packed leaf coordinates -> group
  auto pack = [](int32_t i, int32_t j, int32_t k) {
    return (uint64_t)(uint32_t)i | ((uint64_t)(uint32_t)j << 21) | ((uint64_t)(uint32_t)k << 42);
  };
  const int64_t ng = P->ngroup;
  for (int64_t g = 0; g < ng; ++g) {
    const int32_t *ijk = &lv.ijk[3 * (size_t)P->h_gleaf[g]];
    group_of[pack(ijk[0], ijk[1], ijk[2])] = (int32_t)g;
  }
  std::vector<int32_t> eptr{0}, erwg, gpos;
  std::vector<int64_t> roff{0};
  for (int64_t g = 0; g < ng; ++g) {
    const int32_t *ijk = &lv.ijk[3 * (size_t)P->h_gleaf[g]];
    std::vector<int32_t> E;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          const int32_t x = ijk[0] + dx, y = ijk[1] + dy, z = ijk[2] + dz;
          if (x < 0 || y < 0 || z < 0) continue;
          auto it = group_of.find(pack(x, y, z));
          if (it == group_of.end()) continue;
          const int32_t g2 = it->second;
          E.insert(E.end(), P->h_grwg.begin() + P->h_gptr[g2], P->h_grwg.begin() + P->h_gptr[g2 + 1]);
        }
    std::sort(E.begin(), E.end());
    for (int32_t i = P->h_gptr[g]; i < P->h_gptr[g + 1]; ++i)
      gpos.push_back((int32_t)(std::lower_bound(E.begin(), E.end(), P->h_grwg[i]) - E.begin()));
    erwg.insert(erwg.end(), E.begin(), E.end());
    eptr.push_back((int32_t)erwg.size());
    roff.push_back(roff.back() + (int64_t)(P->h_gptr[g + 1] - P->h_gptr[g]) * (int64_t)E.size());
    P->emax = std::max(P->emax, (int)E.size());
  }
  P->e_ptr = (int32_t *)dalloc(c, sizeof(int32_t) * eptr.size());
  P->e_rwg = (int32_t *)dalloc(c, sizeof(int32_t) * erwg.size());
  P->r_off = (int64_t *)dalloc(c, sizeof(int64_t) * roff.size());
  P->R = (cplxf *)dalloc(c, sizeof(cplxf) * (size_t)roff.back());
  check_cuda(cudaMemcpy(P->e_ptr, eptr.data(), sizeof(int32_t) * eptr.size(), cudaMemcpyHostToDevice), "ras");
  check_cuda(cudaMemcpy(P->e_rwg, erwg.data(), sizeof(int32_t) * erwg.size(), cudaMemcpyHostToDevice), "ras");
  check_cuda(cudaMemcpy(P->r_off, roff.data(), sizeof(int64_t) * roff.size(), cudaMemcpyHostToDevice), "ras");
  int32_t *d_pos = nullptr;
  check_cuda(cudaMalloc(&d_pos, sizeof(int32_t) * gpos.size()), "ras pos");
  check_cuda(cudaMemcpy(d_pos, gpos.data(), sizeof(int32_t) * gpos.size(), cudaMemcpyHostToDevice), "ras pos");
  // per group: LU of the extended block (complex64, cuSOLVER), solve A^T X = unit columns
  // of g's positions, keep R_g = X^T.  The groups are independent: they go round-robin
  // over NS streams, each with its own solver handle and buffers, started behind an
  // event on the context's stream; the host waits for all of them before returning.
  constexpr int NS = 8;
  const int emax = P->emax, smax = P->smax;
  struct Lane {
    cudaStream_t st = nullptr;
    cusolverDnHandle_t hs = nullptr;
    cplxf *A = nullptr, *X = nullptr, *work = nullptr;
    int *ipiv = nullptr;
  } lane[NS];
  int *dinfo = nullptr;
  cudaEvent_t ev_start = nullptr;
  auto release = [&]() {
    for (Lane &q : lane) {
      if (q.st) cudaStreamSynchronize(q.st);
      cudaFree(q.A);
      cudaFree(q.X);
      cudaFree(q.work);
      cudaFree(q.ipiv);
      if (q.hs) cusolverDnDestroy(q.hs);
      if (q.st) cudaStreamDestroy(q.st);
    }
    cudaFree(dinfo);
    cudaFree(d_pos);
    if (ev_start) cudaEventDestroy(ev_start);
  };
  try {
    check_cuda(cudaMalloc(&dinfo, sizeof(int) * (ng + NS)), "ras info");  // getrf per group; getrs per lane
    check_cuda(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming), "ras event");
    check_cuda(cudaEventRecord(ev_start, c->stream), "ras event");
    for (Lane &q : lane) {
      check_cuda(cudaStreamCreateWithFlags(&q.st, cudaStreamNonBlocking), "ras stream");
      check_cuda(cudaStreamWaitEvent(q.st, ev_start, 0), "ras wait");
      if (cusolverDnCreate(&q.hs) != CUSOLVER_STATUS_SUCCESS) fail(NESA_ERR_CUDA, "cusolver create");
      cusolverDnSetStream(q.hs, q.st);
      int lwork = 0;
      check_cuda(cudaMalloc(&q.A, sizeof(cplxf) * (size_t)emax * emax), "ras A");
      check_cuda(cudaMalloc(&q.X, sizeof(cplxf) * (size_t)emax * smax), "ras X");
      check_cuda(cudaMalloc(&q.ipiv, sizeof(int) * emax), "ras piv");
      if (cusolverDnCgetrf_bufferSize(q.hs, emax, emax, (cuComplex *)q.A, emax, &lwork) != CUSOLVER_STATUS_SUCCESS)
        fail(NESA_ERR_CUDA, "cusolver getrf size");
      check_cuda(cudaMalloc(&q.work, sizeof(cplxf) * (size_t)std::max(1, lwork)), "ras work");
    }
    for (int64_t g = 0; g < ng; ++g) {
      Lane &q = lane[g % NS];
      const int ne = eptr[g + 1] - eptr[g], s = P->h_gptr[g + 1] - P->h_gptr[g];
      k_ext_block<<<nblk((int64_t)ne * ne, 256), 256, 0, q.st>>>(q.A, P->e_rwg + eptr[g], ne, c->d_nz_ptr,
                                                                  c->d_nz_col, c->d_nz_val);
      if (cusolverDnCgetrf(q.hs, ne, ne, (cuComplex *)q.A, ne, (cuComplex *)q.work, q.ipiv, dinfo + g) !=
          CUSOLVER_STATUS_SUCCESS)
        fail(NESA_ERR_CUDA, "cusolver getrf");
      k_unit_cols<<<nblk((int64_t)ne * s, 256), 256, 0, q.st>>>(q.X, d_pos + P->h_gptr[g], ne, s);
      if (cusolverDnCgetrs(q.hs, CUBLAS_OP_T, ne, s, (const cuComplex *)q.A, ne, q.ipiv, (cuComplex *)q.X, ne,
                           dinfo + ng + g % NS) != CUSOLVER_STATUS_SUCCESS)
        fail(NESA_ERR_CUDA, "cusolver getrs");
      k_take_rows<<<nblk((int64_t)ne * s, 256), 256, 0, q.st>>>(P->R + roff[g], q.X, ne, s);
    }
    check_cuda(cudaGetLastError(), "ras setup");
    for (Lane &q : lane) check_cuda(cudaStreamSynchronize(q.st), "ras setup");
    std::vector<int> info(ng);
    check_cuda(cudaMemcpy(info.data(), dinfo, sizeof(int) * ng, cudaMemcpyDeviceToHost), "info");
    for (int v : info)
      if (v != 0) fail(NESA_ERR_NUMERIC, "singular extended near-field block");
  } catch (...) {
    release();
    throw;
  }
  release();
  P->ras_ready = true;
}

void precond_ras(nesa_ctx *c, const cplx *r, cplx *z, int nrhs) {
  Precond *P = P_(c);
  k_ras_apply<<<dim3((unsigned)P->ngroup, nrhs), 256, sizeof(cplxf) * (size_t)P->emax, c->stream>>>(
      z, r, c->n, P->g_ptr, P->g_rwg, P->e_ptr, P->e_rwg, P->r_off, P->R);
}

// features f2 = S u and f3 = S N S u (S: overlapping block-Jacobi) into (f2, f3); t is
// scratch of the same size
static void features_of(nesa_ctx *c, const cplx *u, cplx *f2, cplx *f3, cplx *t, int cols) {
  precond_ras(c, u, f2, cols);
  for (int c0 = 0; c0 < cols; c0 += 64) {
    const int nc = std::min(64, cols - c0);
    launch_matvec(c, f2 + (size_t)c0 * c->n, t + (size_t)c0 * c->n, nc, NESA_PART_NEAR);
  }
  precond_ras(c, t, f3, cols);
}

static void refresh_coef(nesa_ctx *c) {
  Precond *P = P_(c);
  k_to_half<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(P->theta16, P->theta, NPARAM);
  k_mlp_infer<<<nblk(c->n, 128), 128, 0, c->stream>>>(P->coef, P->feat, P->theta16, c->n);
}

// z = M r (learned); nrhs columns.  Uses scratch t1 (f2) and t2 (f3 / N f2).
void precond_learned(nesa_ctx *c, const cplx *r, cplx *z, int nrhs) {
  Precond *P = P_(c);
  ensure_workspace(c, std::min(nrhs, 64));
  ensure_scratch(c, P, 2 * nrhs);
  cplx *f2 = P->t1, *f3 = P->t2, *tmp = P->t1 + (size_t)nrhs * c->n;
  precond_ras(c, r, f2, nrhs);
  for (int c0 = 0; c0 < nrhs; c0 += 64) {
    const int nc = std::min(64, nrhs - c0);
    launch_matvec(c, f2 + (size_t)c0 * c->n, tmp + (size_t)c0 * c->n, nc, NESA_PART_NEAR);
  }
  precond_ras(c, tmp, f3, nrhs);
  k_combine<<<nblk(c->n * nrhs, 256), 256, 0, c->stream>>>(z, r, f2, f3, P->coef, c->n, nrhs);
}

void precond_apply(nesa_ctx *c, int kind, const cplx *r, cplx *z, int nrhs) {
  if (kind == NESA_PRECOND_BLOCK_JACOBI) {
    precond_bj(c, r, z, nrhs);
  } else if (kind == NESA_PRECOND_OVERLAP || !P_(c)->trained) {
    precond_ras(c, r, z, nrhs);
  } else {
    precond_learned(c, r, z, nrhs);
  }
}

void precond_ready(nesa_ctx *c, int kind) {
  setup(c);
  if (kind == NESA_PRECOND_OVERLAP || kind == NESA_PRECOND_LEARNED) ras_setup(c);
}

void precond_free(nesa_ctx *c) {
  delete P_(c);
  c->precond = nullptr;
}

// loss and gradient for samples (u_s = Z v_s, v_s), ns columns each of length n
static double loss_grad(nesa_ctx *c, const cplx *U, const cplx *V, int ns, bool backward) {
  Precond *P = P_(c);
  const int64_t n = c->n;
  ensure_scratch(c, P, 2 * ns);
  cplx *F2 = P->t1, *F3 = P->t2, *T = P->t1 + (size_t)ns * n;
  (void)T;
  // features of the samples: F2 = BJ U, F3 = BJ N BJ U (scratch: second half of t1)
  features_of(c, U, F2, F3, P->t1 + (size_t)ns * n, ns);
  // V norm
  std::vector<cplx> hv((size_t)ns * n);
  check_cuda(cudaMemcpyAsync(hv.data(), V, sizeof(cplx) * hv.size(), cudaMemcpyDeviceToHost, c->stream), "v");
  check_cuda(cudaStreamSynchronize(c->stream), "v");
  double vn2 = 0.0;
  for (const cplx &x : hv) vn2 += x.x * x.x + x.y * x.y;
  if (!(vn2 > 0.0)) fail(NESA_ERR_INVALID_ARG, "training targets are zero");
  P->vn2 = vn2;
  const unsigned nb = nblk(n, 256);
  k_mlp_train_forward<<<nblk(n, 128), 128, 0, c->stream>>>(P->coef, P->h1, P->h2, P->feat, P->theta, n);
  k_loss_grad_a<<<nb, 256, 0, c->stream>>>(P->ga, P->lpart, P->coef, U, F2, F3, V, n, ns, 1.0 / vn2);
  if (backward) {
    k_mlp_backward<<<nb, 256, 0, c->stream>>>(P->gpart, P->ga, P->h1, P->h2, P->feat, P->theta, n);
    k_grad_reduce<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(P->grad, P->gpart, (int)nb);
  }
  std::vector<double> lp(nb);
  check_cuda(cudaMemcpyAsync(lp.data(), P->lpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream), "loss");
  check_cuda(cudaStreamSynchronize(c->stream), "loss");
  double L = 0.0;
  for (double x : lp) L += x;
  return L;
}

}  // namespace nesa

using namespace nesa;

// Arnoldi vectors of block-Jacobi GMRES for the training right-hand sides (declared
// in nesa_solve.cu): ns vectors per right-hand side into V (ns * nrhs columns)
int nesa_collect_krylov(nesa_ctx *c, const cplx *b, int nrhs, int ns, cplx *V);
double nesa_precond_validate(nesa_ctx *c, const cplx *b, int iters);

extern "C" {

int nesa_precond_setup(nesa_ctx *c) {
  if (!c) return NESA_ERR_INVALID_ARG;
  try {
    setup(c);
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_precond_apply(nesa_ctx *c, int kind, const nesa_c128 *r, nesa_c128 *z, int nrhs) {
  if (!c || !r || !z || nrhs < 1 || nrhs > 64 ||
      (kind != NESA_PRECOND_BLOCK_JACOBI && kind != NESA_PRECOND_LEARNED && kind != NESA_PRECOND_OVERLAP))
    return NESA_ERR_INVALID_ARG;
  try {
    precond_ready(c, kind);
    precond_apply(c, kind, (const cplx *)r, (cplx *)z, nrhs);
    check_cuda(cudaGetLastError(), "precond");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_precond_params(nesa_ctx *c, int set, float *host) {
  if (!c || !host) return NESA_ERR_INVALID_ARG;
  try {
    setup(c);
    Precond *P = P_(c);
    if (set) {
      check_cuda(cudaMemcpy(P->theta, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "theta");
      refresh_coef(c);
      P->trained = true;
    } else {
      check_cuda(cudaMemcpy(host, P->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "theta");
    }
    check_cuda(cudaStreamSynchronize(c->stream), "params");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_precond_features(nesa_ctx *c, float *host) {
  if (!c || !host) return NESA_ERR_INVALID_ARG;
  try {
    setup(c);
    check_cuda(cudaMemcpy(host, P_(c)->feat, sizeof(float) * NF * (size_t)c->n, cudaMemcpyDeviceToHost), "features");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

int nesa_precond_loss_grad(nesa_ctx *c, const nesa_c128 *u, const nesa_c128 *v, int ns, double *loss, float *grad) {
  if (!c || !u || !v || ns < 1 || ns > 4096 || !loss) return NESA_ERR_INVALID_ARG;
  try {
    precond_ready(c, NESA_PRECOND_LEARNED);
    *loss = loss_grad(c, (const cplx *)u, (const cplx *)v, ns, grad != nullptr);
    if (grad) check_cuda(cudaMemcpy(grad, P_(c)->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "grad");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  return NESA_OK;
}

void nesa_default_learn_opts(nesa_learn_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->samples = 48;
  o->steps = 300;
  o->lr = 3e-3f;
  o->val_iters = 100;
}

int nesa_precond_train(nesa_ctx *c, const nesa_c128 *b, int nrhs, const nesa_learn_opts *opts, nesa_learn_info *info) {
  if (!c || !b || nrhs < 1 || nrhs > 64) return NESA_ERR_INVALID_ARG;
  nesa_learn_opts o;
  nesa_default_learn_opts(&o);
  if (opts) o = *opts;
  if (o.samples < 2 || o.samples > 512 || o.steps < 0 || !(o.lr > 0.0f) || o.val_iters < 0 || o.val_iters > 1000)
    return NESA_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  nesa_learn_info I;
  std::memset(&I, 0, sizeof(I));
  try {
    precond_ready(c, NESA_PRECOND_LEARNED);
    Precond *P = P_(c);
    const int64_t n = c->n;
    const int ns = o.samples * nrhs;
    cplx *V = (cplx *)dalloc(c, sizeof(cplx) * (size_t)ns * n);
    cplx *U = (cplx *)dalloc(c, sizeof(cplx) * (size_t)ns * n);
    // training pairs: Arnoldi vectors v of block-Jacobi GMRES and u = Z v (FP64)
    int st = nesa_collect_krylov(c, (const cplx *)b, nrhs, o.samples, V);
    if (st != NESA_OK) fail(st, "collecting Arnoldi vectors failed");
    ensure_workspace(c, std::min(64, ns));  // the product's work vectors hold up to 64 columns
    for (int c0 = 0; c0 < ns; c0 += 64) {
      const int nc = std::min(64, ns - c0);
      launch_matvec(c, V + (size_t)c0 * n, U + (size_t)c0 * n, nc, NESA_PART_ALL);
    }
    I.samples = ns;
    // training starts from the initial weights (M = S)
    std::vector<float> th0;
    init_theta(th0, 1801);
    check_cuda(cudaMemcpy(P->theta, th0.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "theta");
    check_cuda(cudaMemset(P->adam_m, 0, sizeof(float) * NPARAM), "adam");
    check_cuda(cudaMemset(P->adam_v, 0, sizeof(float) * NPARAM), "adam");
    // the features of the samples do not depend on the weights: computed once inside
    // the first loss_grad call and kept in t1/t2 (ns columns each)
    double L = loss_grad(c, U, V, ns, true);
    I.loss_initial = L;
    for (int t = 1; t <= o.steps; ++t) {
      k_adam<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(P->theta, P->adam_m, P->adam_v, P->grad, o.lr, 0.9f, 0.999f,
                                                        1e-8f, t);
      const unsigned nb = nblk(n, 256);
      k_mlp_train_forward<<<nblk(n, 128), 128, 0, c->stream>>>(P->coef, P->h1, P->h2, P->feat, P->theta, n);
      k_loss_grad_a<<<nb, 256, 0, c->stream>>>(P->ga, P->lpart, P->coef, U, P->t1, P->t2, V, n, ns, 1.0 / P->vn2);
      k_mlp_backward<<<nb, 256, 0, c->stream>>>(P->gpart, P->ga, P->h1, P->h2, P->feat, P->theta, n);
      k_grad_reduce<<<nblk(NPARAM, 256), 256, 0, c->stream>>>(P->grad, P->gpart, (int)nb);
    }
    // final loss with the trained weights
    I.loss_final = loss_grad(c, U, V, ns, false);
    I.steps = o.steps;
    dfree(c, V);
    dfree(c, U);
    refresh_coef(c);
    P->trained = true;
    if (o.val_iters > 0) {
      // validation on the last training right-hand side: trained weights against the
      // initial ones; the lower true residual after val_iters GMRES steps wins
      const cplx *bv = (const cplx *)b + (size_t)(nrhs - 1) * n;
      std::vector<float> th_trained(NPARAM);
      check_cuda(cudaMemcpy(th_trained.data(), P->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "theta");
      I.val_iters = o.val_iters;
      I.val_res_learned = nesa_precond_validate(c, bv, o.val_iters);
      check_cuda(cudaMemcpy(P->theta, th0.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "theta");
      refresh_coef(c);
      I.val_res_base = nesa_precond_validate(c, bv, o.val_iters);
      if (I.val_res_learned < I.val_res_base) {
        check_cuda(cudaMemcpy(P->theta, th_trained.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice),
                   "theta");
        refresh_coef(c);
      } else {
        I.fallback = 1;
      }
    }
    check_cuda(cudaStreamSynchronize(c->stream), "train");
  } catch (const Error &e) {
    set_last_error(e.what);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return NESA_ERR_OOM;
  }
  I.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = I;
  return NESA_OK;
}

}  // extern "C"
