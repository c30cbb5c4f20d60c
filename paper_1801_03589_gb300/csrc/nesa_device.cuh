// Device-side types and helpers shared by the libnesa kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "nesa_internal.h"

namespace nesa {

typedef double2 cplx;  // (re, im)

__host__ __device__ inline cplx cmk(double re, double im) { return make_double2(re, im); }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b with four fused multiply-adds
__device__ __forceinline__ void cfma(cplx &acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// free-space Green's function exp(-i k R)/(4 pi R) (time convention exp(+i w t))
__device__ __forceinline__ cplx green(double k, double R) {
  double s, c;
  sincos(k * R, &s, &c);
  double f = 0.07957747154594767 / R;  // 1/(4 pi R)
  return make_double2(c * f, -s * f);
}

// Distances between points given as separate coordinates.
__device__ __forceinline__ double dist3(double ax, double ay, double az, double bx, double by, double bz) {
  double dx = ax - bx, dy = ay - by, dz = az - bz;
  return sqrt(dx * dx + dy * dy + dz * dz);
}

typedef float2 cplxf;  // complex64 (mixed-precision operator)

__device__ __forceinline__ void cfma(cplxf &acc, cplxf a, cplxf b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// Per-level device arrays of the far-field structure.
struct DevLevel {
  // complex64 copies for the mixed-precision product (NESA_MIXED)
  cplxf *D32 = nullptr, *C32 = nullptr, *Ct32 = nullptr, *s32 = nullptr, *o32 = nullptr;
  int q = 0;           // Q_l
  int64_t nbox = 0;
  int64_t nil = 0;     // interaction pairs
  int64_t noff = 0;    // distinct offsets
  double width = 0.0;
  int32_t *parent = nullptr, *octant = nullptr, *child_ptr = nullptr;
  int32_t *il_ptr = nullptr, *il_src = nullptr, *il_slot = nullptr;
  cplx *D = nullptr;   // [noff][q][q] column-major per offset
  double *Ds = nullptr;  // [noff][q][q] Re + Im of D (the FP64 product's 3M sums)
  cplx *C = nullptr;   // [8][q_{l-1}][q] column-major (rows: parent's sources)
  cplx *Ct = nullptr;  // [8][q][q_{l-1}] column-major (transpose of C)
  double *Cs = nullptr, *Cts = nullptr;  // Re + Im of C and Ct (the FP64 product's 3M sums)
  cplx *K = nullptr;   // [q][2q] column-major
  // generated translations (D == nullptr): equivalent points and offsets on the device,
  // and the pairs grouped in chunks of chunk_slots offset slots: chunk c's pairs by
  // target in cil_ptr[c (nbox + 1) ..], slots relative to the chunk's first slot; D of a
  // chunk is filled into Dw (FP64 product) or Dw32 (complex64 engine) before use
  bool gen = false;
  double *E = nullptr;
  int32_t *offs = nullptr;
  int chunk_slots = 0, nchunk = 0;
  int32_t *cil_ptr = nullptr, *cil_src = nullptr, *cil_slot = nullptr;
  cplx *Dw = nullptr;
  double *Dws = nullptr;  // Re + Im of Dw
  cplxf *Dw32 = nullptr;
  cplx *s = nullptr;   // workspace [nbox][4*nrhs][q] outgoing equivalent sources
  cplx *o = nullptr;   // workspace [nbox][4*nrhs][q] incoming field at the equivalent points
};

}  // namespace nesa

// The context behind the opaque ABI handle.
struct nesa_ctx {
  nesa::HostModel h;
  cudaStream_t stream = nullptr;
  int device = -1;               // CUDA device current at nesa_build (holds all device memory)
  // build time split (seconds): mesh and RWG functions (host), octree and box lists
  // (device), near pattern and V lists (host threads), operator fill (device)
  double build_split[4] = {0, 0, 0, 0};
  double k = 0.0, eta = 0.0;
  int64_t n = 0, nt = 0, np = 0, nleaf = 0;
  int L = 0, l0 = 0;
  nesa_info info{};
  // mesh and basis on the device
  double *d_pts = nullptr;       // [np][3]
  double *d_verts = nullptr;     // [nv][3]
  int32_t *d_tris = nullptr;     // [nt][3]
  int32_t *d_tri_rwg = nullptr;  // [nt][3]
  double *d_tri_sl = nullptr;    // [nt][3]
  int32_t *d_rwg_tri = nullptr;  // [n][2]
  int32_t *d_rwg_free = nullptr; // [n][2]
  // radiation / reception
  int32_t *d_vc_ptr = nullptr, *d_vc_rwg = nullptr, *d_vc_leaf = nullptr;
  int32_t *d_rx_ptr = nullptr, *d_rx_col = nullptr;
  nesa::cplx *d_V = nullptr;     // [ncol][4][q_L]
  // near field (CSR by RWG row)
  int64_t *d_nz_ptr = nullptr;
  int32_t *d_nz_col = nullptr;
  nesa::cplx *d_nz_val = nullptr;
  // complex64 copies (NESA_MIXED)
  bool mixed = false;
  // near field of the mixed product in the internal order (RWG functions sorted by the
  // leaf of their first quadrature point): padded CSR, rows start at multiples of 4,
  // columns ascending in the internal order, padding repeats the last column with value 0
  nesa::cplxf *d_nz_val32 = nullptr;
  int64_t *d_nz_ptr4 = nullptr;
  int32_t *d_nz_col4 = nullptr;
  int32_t *d_perm = nullptr;           // internal index -> ABI index
  nesa::cplxf *d_xp = nullptr;         // x in the internal order, complex64 [nrhs][n], or
                                       // [n][ldx] with nrhs >= 32 (ldx = nrhs rounded up to even)
  nesa::cplxf *d_rcv = nullptr;        // reception per V column, [ncol][nrhs] (nrhs >= 32)
  // the same near field for 32 or more right-hand sides (built by the first such
  // product): internal rows in groups of four, a group's columns the union of its
  // rows' columns, a row's value 0 at the columns it lacks; groups in blocks of eight
  // whose x columns are the union of the eight groups' columns
  int64_t n_group = 0;
  int64_t *d_ng_ptr = nullptr;         // [n_group + 1] first column slot of each group
  int32_t *d_ng_loc = nullptr;         // [slot] position of the slot's column in its block's union
  nesa::cplxf *d_ng_val = nullptr;     // [slot][4] the four rows' values at that column
  int32_t *d_ng_row = nullptr;         // [n_group][4] ABI row of each group member, -1 past the end
  int64_t *d_ng_cbp = nullptr;         // [n_group] start of each group's chunk boundaries in d_ng_cb
  int32_t *d_ng_cb = nullptr;          // per group and chunk of 32 union positions: first slot (relative)
  int64_t *d_nb_ptr = nullptr;         // [n_block + 1] start of each block's union in d_nb_col
  int32_t *d_nb_col = nullptr;         // internal columns of the blocks' unions, ascending per block
  int32_t *d_vc_int = nullptr;         // [ncol] internal index of each V column's RWG function
  nesa::cplxf *d_V32 = nullptr;
  int nrhs_cap32 = 0;
  // levels
  nesa::DevLevel lev[NESA_MAX_LEVELS];
  int nrhs_cap = 0;              // capacity of the s/o workspaces
  // batches holding this context in their graphs, and the right-hand sides they were
  // captured with: while one exists, no product may reallocate what the graph uses
  int batch_refs = 0, batch_nrhs = 0;
  int max_leaf_cols = 0;         // largest number of V columns of one leaf
  // host-pointer product buffers
  nesa::cplx *d_hx = nullptr, *d_hy = nullptr;
  int hbuf_cap = 0;
  size_t device_bytes = 0;
  // stage timing (nesa_profile_enable)
  bool profiling = false;
  struct Pending {
    int stage;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  nesa_profile prof{};
  void *solve_work = nullptr;    // GMRES workspace (nesa_solve.cu)
  void *tc_state = nullptr;      // tensor-core translation state (nesa_tc.cu)
  void *precond = nullptr;       // preconditioner state (nesa_precond.cu)
  bool tc_enabled = false;
  int tables_mode = NESA_TABLES_AUTO; // nesa_params.translation_tables
  int translate_engine = NESA_TRANSLATE_FP32;  // nesa_params.translate
  int tc_stall = 0;                   // failure-detection hook (nesa_inject_stall)
  uint32_t tc_wait_limit = 1u << 20;  // try-wait iterations of the tensor GEMM's bounded waits
  bool autotune = true;          // tune the GEMM tile width at the first product per chunk size
  int fixed_tn = 0;              // tile width used when the autotuner is off
  std::vector<void *> allocs;    // every device allocation owned by the context
};

namespace nesa {
// device allocation with accounting; throws Error on failure
void *dalloc(nesa_ctx *c, size_t bytes);
void dfree(nesa_ctx *c, void *p);
void check_cuda(cudaError_t e, const char *what);
void launch_matvec(nesa_ctx *c, const cplx *x, cplx *y, int nrhs, int parts);
// converted copies of the operator for the mixed-precision product
void build_mixed(nesa_ctx *c);
// the octree, its leaf lists and box lists on the device (nesa_tree.cu); fills the fields
// of c->h that host_tree fills, identically, and leaves the mesh and the quadrature
// points on the device (c->d_verts, c->d_tris, c->d_pts)
void device_tree(nesa_ctx *c, const nesa_params &p, HostModel &m);
// D_l(o) for the offset slots slot0 .. slot0 + ns - 1 of a generated level, into D
// ([ns][q][q] column-major, complex128 or complex64), on the context's stream
void fill_translations(nesa_ctx *c, int level, int64_t slot0, int64_t ns, cplx *D);
void fill_translations(nesa_ctx *c, int level, int64_t slot0, int64_t ns, cplxf *D);
// S[e] = D[e].x + D[e].y for e < count, on the context's stream (FP64 translations' 3M sums)
void plane_sum(nesa_ctx *c, double *S, const cplx *D, int64_t count);
// an event from the context's pool (stage timing)
cudaEvent_t take_event(nesa_ctx *c);
// tensor-core translations of the mixed product (nesa_tc.cu)
void tc_build(nesa_ctx *c);
void tc_translate_level(nesa_ctx *c, int l, const cplxf *s, cplxf *o, const cplxf *op, const cplxf *Ct, int nrhs);
void tc_upward_level(nesa_ctx *c, int l, const cplxf *s, cplxf *sp, int nrhs);
int tc_take_error(nesa_ctx *c);
void tc_free(nesa_ctx *c);
void tc_tuning(nesa_ctx *c, int32_t *tn, float *ms);
// preconditioners (nesa_precond.cu): z = M r
void precond_ready(nesa_ctx *c, int kind);
void precond_apply(nesa_ctx *c, int kind, const cplx *r, cplx *z, int nrhs);
void precond_free(nesa_ctx *c);
int ensure_workspace(nesa_ctx *c, int nrhs);
}  // namespace nesa
void nesa_free_solve_work(nesa_ctx *c);
namespace nesa {
}  // namespace nesa
