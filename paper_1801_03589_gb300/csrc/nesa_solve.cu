// nesa_solve: restarted GMRES(m) on the device for Z~ x = b (paper Sec. 2 names GMRES
// as the iterative solver; the algorithm is Saad & Schultz 1986).
//
// Readings: x0 = 0; Arnoldi with classical Gram-Schmidt applied twice (CGS2), which
// keeps the basis orthogonal to working precision with two reductions per step;
// Givens rotations on the Hessenberg column; stop when the relative residual estimate
// |g_{j+1}| / ||b|| <= tol, and recompute the true residual b - Z~ x at every restart.
// Right-hand sides advance in lock step (one product of nrhs columns per step) but
// keep their own Krylov spaces; a column that has converged stops updating its
// Hessenberg column and its step count.
//
// Every step of the iteration runs in kernels; the host only launches them and reads
// back one flag per right-hand side after each Arnoldi step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "nesa_device.cuh"

namespace nesa {

// Solver workspace of a context (grown on demand).
struct SolveWork {
  int m = 0, nrhs = 0;
  cplx *V = nullptr;     // [m+1][nrhs][n] basis
  cplx *w = nullptr;     // [nrhs][n]
  cplx *r = nullptr;     // [nrhs][n]
  cplx *H = nullptr;     // [nrhs][m+1][m] Hessenberg (column-major per rhs: H[(r*(m+1)) + i + j*(m+1)])
  cplx *h = nullptr;     // [nrhs][m+1] projections of the current step
  cplx *cs = nullptr;    // [nrhs][m]
  cplx *sn = nullptr;    // [nrhs][m]
  cplx *g = nullptr;     // [nrhs][m+1]
  cplx *y = nullptr;     // [nrhs][m]
  double *part = nullptr;  // partial sums [nrhs][m+1][nchunk] (complex as 2 doubles)
  double *nrm = nullptr;   // [nrhs] norms
  double *nrm0 = nullptr;  // [nrhs] norm of Z v_j before the projections
  int *flag = nullptr;     // [nrhs] 1: second projection pass needed
  double *bnorm = nullptr; // [nrhs]
  int *steps = nullptr;    // [nrhs] Arnoldi steps in this cycle
  int *state = nullptr;    // [nrhs] 0 running, 1 converged, 2 breakdown (lucky), 3 numeric
  double *est = nullptr;   // [nrhs] residual estimate
  int *h_state = nullptr;  // pinned host mirror of state
  double *h_est = nullptr; // pinned host mirror of est
  cplx *ro = nullptr;      // [nrhs][n] FP64 residual of the refinement loop
  cplx *dx = nullptr;      // [nrhs][n] correction from the inner solve
  double *onrm = nullptr;  // [nrhs] norms of the refinement loop
  cplx *zt = nullptr;      // [nrhs][n] preconditioned vector M v_j / V y
  cplx *zt2 = nullptr;     // [nrhs][n] M (V y)
};

static const int kChunk = 2048;  // vector elements per partial-sum block

// part[(r*ni + i)*nchunk + c] = sum over chunk c of conj(V_i[r]) w[r]   (i < ni).
// Grid (chunk, tile of kDotTile vectors, column r): every thread reads w once per
// element and keeps kDotTile complex sums in registers.  Per vector the order of the
// additions is the same as one dot at a time (thread strides, warp tree, warps in order).
static const int kDotTile = 8;
__global__ void __launch_bounds__(256) k_dots(double2 *part, const cplx *V, const cplx *w, int ni, int64_t n,
                                              int nrhs, int nchunk, const int *flag) {
  const int c = blockIdx.x, i0 = blockIdx.y * kDotTile, r = blockIdx.z;
  if (flag && !flag[r]) return;  // second pass not needed for this column
  const int nt = min(kDotTile, ni - i0);
  const int64_t lo = (int64_t)c * kChunk, hi = min(n, lo + kChunk);
  __shared__ double sre[8][kDotTile], sim[8][kDotTile];
  const cplx *wr = w + (int64_t)r * n;
  double re[kDotTile], im[kDotTile];
#pragma unroll
  for (int t = 0; t < kDotTile; ++t) re[t] = im[t] = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const cplx b = wr[e];
#pragma unroll
    for (int t = 0; t < kDotTile; ++t)
      if (t < nt) {
        const cplx a = V[((int64_t)(i0 + t) * nrhs + r) * n + e];
        re[t] = fma(a.x, b.x, re[t]);
        re[t] = fma(a.y, b.y, re[t]);
        im[t] = fma(a.x, b.y, im[t]);
        im[t] = fma(-a.y, b.x, im[t]);
      }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kDotTile; ++t) {
    for (int off = 16; off > 0; off >>= 1) {
      re[t] += __shfl_down_sync(0xffffffffu, re[t], off);
      im[t] += __shfl_down_sync(0xffffffffu, im[t], off);
    }
    if (lane == 0) {
      sre[wid][t] = re[t];
      sim[wid][t] = im[t];
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nt) {
    const int t = threadIdx.x;
    double a = 0.0, bb = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sre[k][t];
      bb += sim[k][t];
    }
    part[((int64_t)r * ni + i0 + t) * nchunk + c] = make_double2(a, bb);
  }
}

// h[r][i] (+)= sum_c part (accumulate when add != 0); y[r][i] = the same sum
__global__ void k_dots_reduce(cplx *h, int ldh, cplx *y, int ldy, const double2 *part, int ni, int nchunk, int add,
                              const int *flag) {
  const int i = blockIdx.x, r = blockIdx.y;
  if (flag && !flag[r]) return;
  double re = 0.0, im = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
    double2 v = part[((int64_t)r * ni + i) * nchunk + c];
    re += v.x;
    im += v.y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  if (threadIdx.x == 0) {
    cplx &o = h[(int64_t)r * ldh + i];
    if (add) {
      o.x += re;
      o.y += im;
    } else {
      o = make_double2(re, im);
    }
    y[(int64_t)r * ldy + i] = make_double2(re, im);
  }
}

// w[r] -= sum_{i<ni} V_i[r] * coef[r][i]   (four FP64 FMAs per term: the pass is bound
// by the FP64 pipe)
__global__ void k_subtract(cplx *w, const cplx *V, const cplx *coef, int ldc, int ni, int64_t n, int nrhs,
                           const int *flag) {
  const int r = blockIdx.y;
  if (flag && !flag[r]) return;
  const cplx *cr = coef + (int64_t)r * ldc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    cplx acc = w[(int64_t)r * n + e];
#pragma unroll 4
    for (int i = 0; i < ni; ++i) {
      const cplx v = V[((int64_t)i * nrhs + r) * n + e];
      const cplx c = cr[i];
      acc.x = fma(-v.x, c.x, acc.x);
      acc.x = fma(v.y, c.y, acc.x);
      acc.y = fma(-v.x, c.y, acc.y);
      acc.y = fma(-v.y, c.x, acc.y);
    }
    w[(int64_t)r * n + e] = acc;
  }
}

// second CGS pass only where the first one removed most of w: |w| after < eta |w| before
// ("twice is enough": one more pass restores orthogonality to working precision)
__global__ void k_reorth_flag(int *flag, const double *after, const double *before, double eta, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) flag[r] = after[r] < eta * before[r] ? 1 : 0;
}

// x[r] += sum_{i<k_r} V_i[r] y[r][i]
__global__ void k_update_x(cplx *x, const cplx *V, const cplx *y, int ldy, const int *steps, int64_t n, int nrhs) {
  const int r = blockIdx.y;
  const int k = steps[r];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    cplx acc = x[(int64_t)r * n + e];
#pragma unroll 4
    for (int i = 0; i < k; ++i) cfma(acc, V[((int64_t)i * nrhs + r) * n + e], y[(int64_t)r * ldy + i]);
    x[(int64_t)r * n + e] = acc;
  }
}

// partial sums of |v|^2 per column (columns with flag 0 skipped when flag is given)
__global__ void k_norm2(double2 *part, const cplx *v, int64_t n, int nchunk, const int *flag) {
  const int c = blockIdx.x, r = blockIdx.y;
  if (flag && !flag[r]) return;
  const int64_t lo = (int64_t)c * kChunk, hi = min(n, lo + kChunk);
  double s = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    cplx a = v[(int64_t)r * n + e];
    s = fma(a.x, a.x, s);
    s = fma(a.y, a.y, s);
  }
  __shared__ double sh[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    part[(int64_t)r * nchunk + c] = make_double2(t, 0.0);
  }
}

__global__ void k_norm_reduce(double *out, const double2 *part, int nchunk, const int *flag) {
  const int r = blockIdx.x;
  if (flag && !flag[r]) return;
  double s = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) s += part[(int64_t)r * nchunk + c].x;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) out[r] = sqrt(s);
}

// dst[r] = a * src[r] / scale[r]   (scale NULL: 1)
__global__ void k_scale(cplx *dst, const cplx *src, const double *scale, int64_t n, int nrhs) {
  const int r = blockIdx.y;
  const double f = scale ? (scale[r] > 0.0 ? 1.0 / scale[r] : 0.0) : 1.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    cplx a = src[(int64_t)r * n + e];
    dst[(int64_t)r * n + e] = make_double2(a.x * f, a.y * f);
  }
}

// x += d
__global__ void k_add(cplx *x, const cplx *d, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    cplx a = x[e], b = d[e];
    x[e] = make_double2(a.x + b.x, a.y + b.y);
  }
}

// r = b - r   (r holds Z~ x on entry)
__global__ void k_residual(cplx *r, const cplx *b, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    cplx z = r[e], bb = b[e];
    r[e] = make_double2(bb.x - z.x, bb.y - z.y);
  }
}

// start of a cycle: g = (beta, 0, ...), steps = 0, state from beta
__global__ void k_cycle_start(cplx *g, int m, const double *beta, const double *bnorm, int *steps, int *state,
                              double *est, double tol, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  for (int i = 0; i <= m; ++i) g[(int64_t)r * (m + 1) + i] = make_double2(i == 0 ? beta[r] : 0.0, 0.0);
  steps[r] = 0;
  // a NaN/Inf in b or in the residual stops the right-hand side with a numeric error
  // (a NaN norm would otherwise fail the test bnorm > 0 and read as a zero residual)
  if (!isfinite(bnorm[r]) || !isfinite(beta[r])) {
    est[r] = NAN;
    state[r] = 3;
    return;
  }
  const double e = bnorm[r] > 0.0 ? beta[r] / bnorm[r] : 0.0;
  est[r] = e;
  state[r] = (e <= tol) ? 1 : (isfinite(e) ? 0 : 3);
}

// Arnoldi step j: Hessenberg column from h (projections) and hn (norm of the
// orthogonalised vector); previous rotations, new rotation, residual estimate.
__global__ void k_givens(cplx *H, const cplx *h, const double *hn, cplx *cs, cplx *sn, cplx *g, int *steps,
                         int *state, double *est, const double *bnorm, int j, int m, double tol, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || state[r] != 0) return;
  cplx *Hr = H + (int64_t)r * (m + 1) * m;
  cplx *col = Hr + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h[(int64_t)r * (m + 1) + i];
  col[j + 1] = make_double2(hn[r], 0.0);
  cplx *c = cs + (int64_t)r * m, *s = sn + (int64_t)r * m, *gr = g + (int64_t)r * (m + 1);
  for (int i = 0; i < j; ++i) {
    // [c s; -conj(s) c] with c real
    cplx a = col[i], b = col[i + 1];
    double ci = c[i].x;
    cplx si = s[i];
    col[i] = make_double2(ci * a.x + si.x * b.x - si.y * b.y, ci * a.y + si.x * b.y + si.y * b.x);
    col[i + 1] = make_double2(-(si.x * a.x + si.y * a.y) + ci * b.x, -(si.x * a.y - si.y * a.x) + ci * b.y);
  }
  cplx a = col[j], b = col[j + 1];
  double na = hypot(a.x, a.y), nb = hypot(b.x, b.y);
  double den = hypot(na, nb);
  double cj;
  cplx sj;
  if (den == 0.0 || !isfinite(den)) {
    state[r] = 3;
    return;
  }
  if (na == 0.0) {
    cj = 0.0;
    sj = make_double2(b.x / nb, -b.y / nb);  // conj(b)/|b|
  } else {
    cj = na / den;
    // (a/|a|) conj(b) / den
    cplx ua = make_double2(a.x / na, a.y / na);
    sj = make_double2((ua.x * b.x + ua.y * b.y) / den, (ua.y * b.x - ua.x * b.y) / den);
  }
  c[j] = make_double2(cj, 0.0);
  s[j] = sj;
  col[j] = make_double2(cj * a.x + sj.x * b.x - sj.y * b.y, cj * a.y + sj.x * b.y + sj.y * b.x);
  col[j + 1] = make_double2(0.0, 0.0);
  cplx gj = gr[j];
  gr[j + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));
  gr[j] = make_double2(cj * gj.x, cj * gj.y);
  steps[r] = j + 1;
  const double e = hypot(gr[j + 1].x, gr[j + 1].y) / bnorm[r];
  est[r] = e;
  if (!isfinite(e))
    state[r] = 3;
  else if (e <= tol)
    state[r] = 1;
  else if (hn[r] == 0.0)
    state[r] = 2;  // the Krylov space is invariant: the solution is exact in it
}

// y = R^-1 g (upper triangular R = rotated H, size steps[r])
__global__ void k_backsolve(cplx *y, const cplx *H, const cplx *g, const int *steps, int m, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int k = steps[r];
  const cplx *Hr = H + (int64_t)r * (m + 1) * m;
  const cplx *gr = g + (int64_t)r * (m + 1);
  cplx *yr = y + (int64_t)r * m;
  for (int i = k - 1; i >= 0; --i) {
    cplx acc = gr[i];
    for (int t = i + 1; t < k; ++t) {
      cplx hv = Hr[i + (int64_t)t * (m + 1)], yv = yr[t];
      acc.x -= hv.x * yv.x - hv.y * yv.y;
      acc.y -= hv.x * yv.y + hv.y * yv.x;
    }
    cplx d = Hr[i + (int64_t)i * (m + 1)];
    double dd = d.x * d.x + d.y * d.y;
    yr[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
  }
}

static inline unsigned blocks_for(int64_t n, int bs, int cap) {
  int64_t b = (n + bs - 1) / bs;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace nesa

using namespace nesa;

static SolveWork *get_work(nesa_ctx *c, int m, int nrhs) {
  static_assert(sizeof(SolveWork) > 0, "");
  if (!c->solve_work) c->solve_work = new SolveWork();
  SolveWork *W = (SolveWork *)c->solve_work;
  if (W->m >= m && W->nrhs >= nrhs) return W;
  void *old[] = {W->V, W->w, W->r, W->H, W->h, W->cs, W->sn, W->g, W->y, W->part, W->nrm, W->nrm0, W->flag,
                 W->bnorm, W->steps, W->state, W->est, W->ro, W->dx, W->onrm, W->zt, W->zt2};
  for (void *p : old) dfree(c, p);
  if (W->h_state) cudaFreeHost(W->h_state);
  if (W->h_est) cudaFreeHost(W->h_est);
  *W = SolveWork();
  const int64_t n = c->n;
  const int nchunk = (int)((n + kChunk - 1) / kChunk);
  W->m = m;
  W->nrhs = nrhs;
  W->V = (cplx *)dalloc(c, sizeof(cplx) * (size_t)(m + 1) * nrhs * n);
  W->w = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->r = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->H = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * (m + 1) * m);
  W->h = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * (m + 1));
  W->cs = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * m);
  W->sn = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * m);
  W->g = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * (m + 1));
  W->y = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * m);
  W->part = (double *)dalloc(c, sizeof(double2) * (size_t)nrhs * (m + 1) * nchunk);
  W->nrm = (double *)dalloc(c, sizeof(double) * nrhs);
  W->nrm0 = (double *)dalloc(c, sizeof(double) * nrhs);
  W->flag = (int *)dalloc(c, sizeof(int) * nrhs);
  W->bnorm = (double *)dalloc(c, sizeof(double) * nrhs);
  W->steps = (int *)dalloc(c, sizeof(int) * nrhs);
  W->state = (int *)dalloc(c, sizeof(int) * nrhs);
  W->est = (double *)dalloc(c, sizeof(double) * nrhs);
  W->zt = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->zt2 = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->ro = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->dx = (cplx *)dalloc(c, sizeof(cplx) * (size_t)nrhs * n);
  W->onrm = (double *)dalloc(c, sizeof(double) * nrhs);
  check_cuda(cudaMallocHost(&W->h_state, sizeof(int) * nrhs), "pinned");
  check_cuda(cudaMallocHost(&W->h_est, sizeof(double) * nrhs), "pinned");
  return W;
}

void nesa_free_solve_work(nesa_ctx *c) {
  SolveWork *W = (SolveWork *)c->solve_work;
  if (!W) return;
  if (W->h_state) cudaFreeHost(W->h_state);
  if (W->h_est) cudaFreeHost(W->h_est);
  delete W;
  c->solve_work = nullptr;
}

// GMRES from x0 = 0 on the product selected by `parts`.  Throws Error on CUDA
// failures.  Returns NESA_OK, NESA_ERR_NOT_CONVERGED or NESA_ERR_NUMERIC; adds to the
// counters of I and fills its true residuals.
static int gmres_run(nesa_ctx *c, const cplx *b, cplx *x, int nrhs, double tol, int m, int max_iters, int parts,
                     int precond, nesa_solve_info &I) {
  int status = NESA_OK;
  if (precond != NESA_PRECOND_NONE) precond_ready(c, precond);
  {
    SolveWork *W = get_work(c, m, nrhs);
    ensure_workspace(c, nrhs);
    cudaStream_t st = c->stream;
    const int64_t n = c->n;
    const int nchunk = (int)((n + kChunk - 1) / kChunk);
    const dim3 vgrid(blocks_for(n, 256, 4096), nrhs);
    auto norms = [&](const cplx *v, double *out, const int *flag = nullptr) {
      k_norm2<<<dim3(nchunk, nrhs), 256, 0, st>>>((double2 *)W->part, v, n, nchunk, flag);
      k_norm_reduce<<<nrhs, 32, 0, st>>>(out, (const double2 *)W->part, nchunk, flag);
    };
    norms(b, W->bnorm);
    check_cuda(cudaMemsetAsync(x, 0, sizeof(cplx) * (size_t)nrhs * n, st), "x0");
    check_cuda(cudaMemcpyAsync(W->r, b, sizeof(cplx) * (size_t)nrhs * n, cudaMemcpyDeviceToDevice, st), "r0");
    int total = 0;
    while (true) {
      // r holds the residual; start a cycle
      norms(W->r, W->nrm);
      k_cycle_start<<<(nrhs + 63) / 64, 64, 0, st>>>(W->g, m, W->nrm, W->bnorm, W->steps, W->state, W->est, tol,
                                                     nrhs);
      check_cuda(cudaMemcpyAsync(W->h_state, W->state, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st), "state");
      check_cuda(cudaMemcpyAsync(W->h_est, W->est, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st), "est");
      check_cuda(cudaStreamSynchronize(st), "cycle start");
      bool running = false;
      for (int r = 0; r < nrhs; ++r) running |= W->h_state[r] == 0;
      for (int r = 0; r < nrhs; ++r)
        if (W->h_state[r] == 3) status = NESA_ERR_NUMERIC;
      if (!running || status != NESA_OK || total >= max_iters) break;
      k_scale<<<vgrid, 256, 0, st>>>(W->V, W->r, W->nrm, n, nrhs);
      I.restarts += total > 0;
      int j = 0;
      for (; j < m && total < max_iters; ++j) {
        cplx *Vj = W->V + (size_t)j * nrhs * n;
        cplx *Vn = W->V + (size_t)(j + 1) * nrhs * n;
        if (precond != NESA_PRECOND_NONE) {  // right preconditioning: w = Z (M v_j)
          precond_apply(c, precond, Vj, W->zt, nrhs);
          launch_matvec(c, W->zt, W->w, nrhs, parts);
        } else {
          launch_matvec(c, Vj, W->w, nrhs, parts);
        }
        I.matvecs += 1;
        // classical Gram-Schmidt onto V_0..V_j; a second pass for the columns whose
        // norm fell below 0.7 of its value before (CGS2 where needed; the projections
        // are bound by the FP64 pipe, so the pass is skipped on the device elsewhere)
        norms(W->w, W->nrm0);
        for (int pass = 0; pass < 2; ++pass) {
          const int *fl = pass ? W->flag : nullptr;
          k_dots<<<dim3(nchunk, (j + kDotTile) / kDotTile, nrhs), 256, 0, st>>>((double2 *)W->part, W->V, W->w,
                                                                               j + 1, n, nrhs, nchunk, fl);
          // h accumulates both passes; y holds this pass's coefficients for the subtraction
          k_dots_reduce<<<dim3(j + 1, nrhs), 32, 0, st>>>(W->h, m + 1, W->y, m, (const double2 *)W->part, j + 1,
                                                           nchunk, pass, fl);
          k_subtract<<<vgrid, 256, 0, st>>>(W->w, W->V, W->y, m, j + 1, n, nrhs, fl);
          norms(W->w, W->nrm, fl);
          if (pass == 0) k_reorth_flag<<<(nrhs + 63) / 64, 64, 0, st>>>(W->flag, W->nrm, W->nrm0, 0.7, nrhs);
        }
        k_givens<<<(nrhs + 63) / 64, 64, 0, st>>>(W->H, W->h, W->nrm, W->cs, W->sn, W->g, W->steps, W->state, W->est,
                                                  W->bnorm, j, m, tol, nrhs);
        k_scale<<<vgrid, 256, 0, st>>>(Vn, W->w, W->nrm, n, nrhs);
        ++total;
        check_cuda(cudaMemcpyAsync(W->h_state, W->state, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st), "state");
        check_cuda(cudaStreamSynchronize(st), "arnoldi step");
        bool any = false;
        for (int r = 0; r < nrhs; ++r) any |= W->h_state[r] == 0;
        if (!any) break;
      }
      // x += V y for the steps each column took in this cycle
      k_backsolve<<<(nrhs + 63) / 64, 64, 0, st>>>(W->y, W->H, W->g, W->steps, m, nrhs);
      if (precond != NESA_PRECOND_NONE) {  // x += M (V y)
        check_cuda(cudaMemsetAsync(W->zt, 0, sizeof(cplx) * (size_t)nrhs * n, st), "zt");
        k_update_x<<<vgrid, 256, 0, st>>>(W->zt, W->V, W->y, m, W->steps, n, nrhs);
        precond_apply(c, precond, W->zt, W->zt2, nrhs);
        k_add<<<blocks_for((int64_t)nrhs * n, 256, 4096), 256, 0, st>>>(x, W->zt2, (int64_t)nrhs * n);
      } else {
        k_update_x<<<vgrid, 256, 0, st>>>(x, W->V, W->y, m, W->steps, n, nrhs);
      }
      // true residual
      launch_matvec(c, x, W->r, nrhs, parts);
      I.matvecs += 1;
      k_residual<<<blocks_for((int64_t)nrhs * n, 256, 4096), 256, 0, st>>>(W->r, b, (int64_t)nrhs * n);
      check_cuda(cudaGetLastError(), "gmres launch");
      if (total >= max_iters) {
        norms(W->r, W->nrm);
        break;
      }
    }
    // final true residuals
    norms(W->r, W->nrm);
    std::vector<double> rn(nrhs), bn(nrhs);
    check_cuda(cudaMemcpyAsync(rn.data(), W->nrm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st), "res");
    check_cuda(cudaMemcpyAsync(bn.data(), W->bnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st), "bn");
    check_cuda(cudaStreamSynchronize(st), "solve");
    I.iterations += total;
    for (int r = 0; r < nrhs; ++r) {
      double rr = bn[r] > 0.0 ? rn[r] / bn[r] : 0.0;
      if (!std::isfinite(bn[r]) || !std::isfinite(rn[r])) rr = NAN;
      I.rel_residual[r] = rr;
      if (!std::isfinite(rr)) status = NESA_ERR_NUMERIC;
      // the true residual decides convergence (the estimate can be slightly optimistic)
      if (rr <= tol * (1.0 + 1e-6)) I.converged += 1;
    }
    if (status == NESA_OK && I.converged < nrhs) status = NESA_ERR_NOT_CONVERGED;
  }
  return status;
}

// x += d
__global__ void k_axpy(cplx *x, const cplx *d, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    cplx a = x[e], b = d[e];
    x[e] = make_double2(a.x + b.x, a.y + b.y);
  }
}

// FP64 iterative refinement: r = b - Z~ x with the FP64 product, an inner GMRES on the
// low-precision product solves Z~_mixed d = r to inner_tol, x += d.
static int refine_run(nesa_ctx *c, const cplx *b, cplx *x, int nrhs, double tol, const nesa_solve_opts &o,
                      nesa_solve_info &I) {
  if (!c->mixed) fail(NESA_ERR_INVALID_ARG, "mixed solve needs a context built with NESA_MIXED");
  SolveWork *W = get_work(c, o.restart, nrhs);
  cudaStream_t st = c->stream;
  const int64_t n = c->n, total = n * nrhs;
  const int nchunk = (int)((n + kChunk - 1) / kChunk);
  auto norms = [&](const cplx *v, double *out_dev, std::vector<double> &host) {
    k_norm2<<<dim3(nchunk, nrhs), 256, 0, st>>>((double2 *)W->part, v, n, nchunk, nullptr);
    k_norm_reduce<<<nrhs, 32, 0, st>>>(out_dev, (const double2 *)W->part, nchunk, nullptr);
    host.resize(nrhs);
    check_cuda(cudaMemcpyAsync(host.data(), out_dev, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st), "norm");
    check_cuda(cudaStreamSynchronize(st), "norm");
  };
  std::vector<double> bn, rn;
  norms(b, W->onrm, bn);
  check_cuda(cudaMemsetAsync(x, 0, sizeof(cplx) * (size_t)total, st), "x0");
  check_cuda(cudaMemcpyAsync(W->ro, b, sizeof(cplx) * (size_t)total, cudaMemcpyDeviceToDevice, st), "r0");
  int status = NESA_OK;
  for (int it = 0;; ++it) {
    norms(W->ro, W->onrm, rn);
    bool done = true;
    double emax = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      double e = bn[r] > 0.0 ? rn[r] / bn[r] : 0.0;
      if (!std::isfinite(bn[r]) || !std::isfinite(rn[r]) || !std::isfinite(e)) {
        I.rel_residual[r] = NAN;
        return NESA_ERR_NUMERIC;
      }
      done &= e <= tol;
      emax = std::max(emax, e);
    }
    if (done || it >= o.max_refine || I.iterations >= o.max_iters) break;
    // the inner solve reduces the residual by inner_tol, or only by what is left to
    // reach half the target when that is less
    const double inner = std::min(0.5, std::max(o.inner_tol, 0.5 * tol / emax));
    nesa_solve_info Ii;
    std::memset(&Ii, 0, sizeof(Ii));
    int si = gmres_run(c, W->ro, W->dx, nrhs, inner, o.restart, o.max_iters - I.iterations,
                       NESA_PART_ALL | NESA_PART_MIXED, o.precond, Ii);
    I.iterations += Ii.iterations;
    I.matvecs += Ii.matvecs;
    I.restarts += Ii.restarts;
    if (si == NESA_ERR_NUMERIC) return si;
    k_axpy<<<blocks_for(total, 256, 4096), 256, 0, st>>>(x, W->dx, total);
    launch_matvec(c, x, W->ro, nrhs, NESA_PART_ALL);
    I.fp64_matvecs += 1;
    k_residual<<<blocks_for(total, 256, 4096), 256, 0, st>>>(W->ro, b, total);
    check_cuda(cudaGetLastError(), "refinement launch");
    I.refinements += 1;
  }
  I.converged = 0;
  for (int r = 0; r < nrhs; ++r) {
    double e = bn[r] > 0.0 ? rn[r] / bn[r] : 0.0;
    I.rel_residual[r] = e;
    if (e <= tol) I.converged += 1;
  }
  if (I.converged < nrhs) status = NESA_ERR_NOT_CONVERGED;
  return status;
}

// Arnoldi vectors v_0..v_{ns-1} of block-Jacobi-preconditioned GMRES (one cycle of ns
// steps from x0 = 0) for each of the nrhs right-hand sides, into V [nrhs * ns][n]
// (right-hand side major).  Columns past a breakdown are zero.
// True relative residual after `iters` steps of GMRES(iters) with the learned
// preconditioner on one right-hand side (the mixed product when it was built);
// used to validate trained weights.  Throws Error on CUDA failures.
double nesa_precond_validate(nesa_ctx *c, const cplx *b, int iters) {
  SolveWork *W = get_work(c, iters, 1);
  nesa_solve_info I;
  std::memset(&I, 0, sizeof(I));
  const int parts = NESA_PART_ALL | (c->mixed ? NESA_PART_MIXED : 0);
  int st = gmres_run(c, b, W->dx, 1, 0.0, iters, iters, parts, NESA_PRECOND_LEARNED, I);
  if (st == NESA_ERR_NUMERIC) return INFINITY;
  const double r = I.rel_residual[0];
  return std::isfinite(r) ? r : INFINITY;
}

int nesa_collect_krylov(nesa_ctx *c, const cplx *b, int nrhs, int ns, cplx *V) {
  SolveWork *W = get_work(c, ns, nrhs);
  nesa_solve_info I;
  std::memset(&I, 0, sizeof(I));
  int st = gmres_run(c, b, W->dx, nrhs, 1e-300, ns, ns, NESA_PART_ALL, NESA_PRECOND_OVERLAP, I);
  if (st == NESA_ERR_NUMERIC) return st;
  std::vector<int> steps(nrhs);
  check_cuda(cudaMemcpy(steps.data(), W->steps, sizeof(int) * nrhs, cudaMemcpyDeviceToHost), "steps");
  const int64_t n = c->n;
  for (int r = 0; r < nrhs; ++r)
    for (int j = 0; j < ns; ++j) {
      cplx *dst = V + ((size_t)r * ns + j) * n;
      if (j <= steps[r] && j < ns)
        check_cuda(cudaMemcpyAsync(dst, W->V + ((size_t)j * nrhs + r) * n, sizeof(cplx) * n,
                                   cudaMemcpyDeviceToDevice, c->stream),
                   "krylov copy");
      else
        check_cuda(cudaMemsetAsync(dst, 0, sizeof(cplx) * n, c->stream), "krylov zero");
    }
  check_cuda(cudaStreamSynchronize(c->stream), "krylov");
  return NESA_OK;
}

extern "C" {

void nesa_default_solve_opts(nesa_solve_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->restart = 50;
  o->max_iters = 1000;
  o->mixed = 0;
  o->max_refine = 10;
  o->inner_tol = 3e-3;
}

int nesa_solve(nesa_ctx *c, const nesa_c128 *b_dev, nesa_c128 *x_dev, int nrhs, double tol,
               const nesa_solve_opts *opts, nesa_solve_info *info) {
  if (!c || !b_dev || !x_dev || nrhs < 1 || nrhs > 64 || !(tol > 0.0)) return NESA_ERR_INVALID_ARG;
  nesa_solve_opts o;
  nesa_default_solve_opts(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 1000 || o.max_iters < 1 || (o.mixed != 0 && o.mixed != 1) ||
      o.max_refine < 0 || !(o.inner_tol > 0.0 && o.inner_tol < 1.0) || o.precond < NESA_PRECOND_NONE ||
      o.precond > NESA_PRECOND_OVERLAP)
    return NESA_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  nesa_solve_info I;
  std::memset(&I, 0, sizeof(I));
  int status = NESA_OK;
  try {
    if (o.mixed) {
      status = refine_run(c, (const cplx *)b_dev, (cplx *)x_dev, nrhs, tol, o, I);
    } else {
      status = gmres_run(c, (const cplx *)b_dev, (cplx *)x_dev, nrhs, tol, o.restart, o.max_iters, NESA_PART_ALL,
                         o.precond, I);
      I.fp64_matvecs = I.matvecs;
    }
  } catch (const Error &e) {
    status = e.status;
    set_last_error(e.what);
  } catch (const std::bad_alloc &) {
    status = NESA_ERR_OOM;
    set_last_error("host allocation failed");
  }
  I.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = I;
  return status;
}

}  // extern "C"
