/*
 * nesa.h - C ABI of the GB300 NESA/EFIE library (libnesa.so).
 *
 * The library solves the electric-field integral equation for the surface current of
 * a perfectly conducting body, Z j = b (arxiv 1801.03589, Sec. 2, Eq. 2 and Eq. 3),
 * with the matrix-vector product Z x evaluated by the nested equivalent source
 * approximation: a near-field sparse product (Sec. 3, Eq. 9) plus the five far-field
 * stages radiation, source transfer, translation, potential transfer and reception
 * (Sec. 3, Eqs. 10-14; the nested factorisation is Sec. 2, Eqs. 4-7).  Every stage of
 * the product runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points
 *   - Lengths are in the same unit as 1/k (k = wavenumber); the medium is free space
 *     (impedance eta = mu0 c).  Time convention exp(+i w t): g = exp(-i k R)/(4 pi R).
 *   - Unknowns are RWG functions, one per interior mesh edge (an edge shared by exactly
 *     two triangles), numbered in lexicographic order of (smaller vertex id, larger
 *     vertex id).  The function is l/(2A+)(r - v+) on T+ (the adjacent triangle with the
 *     smaller index) and l/(2A-)(v- - r) on T-.
 *   - Complex numbers are interleaved (re, im) doubles.  A block of nrhs vectors of
 *     length N is column-major: element n of vector r is at [r * N + n].
 *   - "dev" pointers are CUDA device pointers owned by the caller; "host" pointers are
 *     host memory owned by the caller.  The library never frees caller memory.
 *   - Every call returns NESA_OK (0) or a negative status; nothing throws across the
 *     ABI.  nesa_status_str() names a status.  On error, outputs are unspecified unless
 *     stated otherwise.
 *   - Device work is ordered on the context's stream (default: the legacy default
 *     stream; see nesa_set_stream).  Calls that return device results do not
 *     synchronise unless stated.  A context is used by one host thread at a time.
 */
#ifndef NESA_H
#define NESA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define NESA_OK 0
#define NESA_ERR_INVALID_ARG (-1)   /* null pointer, size out of range, bad parameter */
#define NESA_ERR_MESH (-2)          /* non-manifold edge, degenerate triangle, bad index,
                                       triangles too large for the leaf size */
#define NESA_ERR_CUDA (-3)          /* a CUDA runtime or library call failed */
#define NESA_ERR_OOM (-4)           /* device or host allocation failed */
#define NESA_ERR_NOT_CONVERGED (-5) /* solver stopped at its iteration limit; x and info are filled */
#define NESA_ERR_TIMEOUT (-6)       /* a bounded device wait ran out */
#define NESA_ERR_NUMERIC (-7)       /* NaN/Inf met, or a breakdown */

/* precision of the operator copies built (nesa_params.precision) */
#define NESA_FP64 0  /* FP64 operator only */
#define NESA_MIXED 1 /* FP64 operator plus a low-precision copy (see NESA_PART_MIXED) */

/* rule for the number of equivalent sources per level (nesa_params.q_mode) */
#define NESA_Q_FIXED 0 /* Q = q_fixed in every group (the paper's choice, Sec. 3) */
#define NESA_Q_AUTO 1  /* Q_l = max(q_fixed, (n_l+1)^2), n_l = ceil(kR + 1.8 d^(2/3) (kR)^(1/3)) */

/* parts of the operator applied by nesa_matvec_parts */
#define NESA_PART_NEAR 1 /* near field, Eq. 9 */
#define NESA_PART_FAR 2  /* far field, Eqs. 10-14 */
#define NESA_PART_ALL 3
/* Or-ed into the parts: apply the low-precision copy (context built with NESA_MIXED):
   near field, radiation, transfers and reception in complex64 (FP32 arithmetic),
   translations as selected by nesa_params.translate (x and y stay complex128). */
#define NESA_PART_MIXED 4

/* translation engine of the mixed product (nesa_params.translate) */
#define NESA_TRANSLATE_FP32 0 /* complex64 on the CUDA cores */
/* Tensor cores (tcgen05, BF16 operands split hi/lo, three products per K step, FP32
   accumulation): the pairs of one level that share an offset form one complex GEMM
   (Sec. 5.1 notes that equal relative positions share a matrix), computed as the real
   GEMM [[Re D, -Im D], [Im D, Re D]] [Re s; Im s] */
#define NESA_TRANSLATE_TENSOR 1

typedef struct nesa_ctx nesa_ctx; /* opaque; owns all device memory of one operator */

typedef struct {
  double re, im;
} nesa_c128;

typedef struct {
  int64_t n_vertices;
  int64_t n_triangles;
  const double *vertices;   /* host, [n_vertices][3] */
  const int32_t *triangles; /* host, [n_triangles][3] vertex ids, counter-clockwise seen from outside */
} nesa_mesh;

/*
 * Octree and equivalent-source parameters (Sec. 2 and Sec. 3).
 *   leaf_size   side of a leaf box; the root cube has side leaf_size * 2^(n_levels-1)
 *               and is centred on the centre of the vertex bounding box
 *   n_levels    number of octree levels (root = level 0, leaves = level n_levels-1), 1..20;
 *               with leaf_size > 0, 0 selects the fewest levels whose root cube
 *               (leaf_size * 2^(levels-1)) spans the largest side of the bounding box
 *   q_mode      NESA_Q_FIXED or NESA_Q_AUTO
 *   q_fixed     Q for NESA_Q_FIXED; lower bound of Q_l for NESA_Q_AUTO
 *   q_digits    d of the NESA_Q_AUTO rule
 *   rho_eq      radius of the equivalent-source sphere / box circumradius
 *   rho_test    radius of the test sphere / box circumradius
 *   pinv_eps    Tikhonov parameter of the equivalent-source fit, relative to the
 *               Frobenius norm of the fitted matrix
 *   precision   NESA_FP64 or NESA_MIXED
 *   translate   NESA_TRANSLATE_* engine of the mixed product's translations
 *   tile_n      column-tile width of the tensor-core GEMMs (64, 128 or 256); 0 lets
 *               the autotuner time the three widths at the first mixed product and
 *               keep the fastest per GEMM family (a fixed width makes runs under a
 *               profiler, which distorts the tuner's timings, use the tuned layout)
 *   points_per_leaf  P of the paper's depth rule (Sec. 3: groups are subdivided while
 *               they hold at least P sources on average), used when leaf_size is 0: the
 *               root cube is the cube of the largest side of the vertex bounding box
 *               (same centre), and the leaf level is the deepest level l <= 19 whose
 *               occupied boxes hold on average at least P quadrature points (7 per
 *               triangle).  n_levels is then ignored.  0 when leaf_size > 0.
 *   singular_mode  NESA_SINGULAR_TOUCHING (default) or NESA_SINGULAR_SELF
 *   translation_tables  NESA_TABLES_AUTO (default), NESA_TABLES_STORED or
 *               NESA_TABLES_GENERATED: whether the translation matrices D_l(o) of Eq. 12
 *               are kept in device memory per offset or built from the equivalent points
 *               when a product needs them (D_l(o)_ij = g(|E_i + o w_l - E_j|), a plain
 *               Green's-function matrix).  Generated, the FP64 product fills them into a
 *               bounded work buffer (at most 64 offsets and about 1.5 GB at a time) just
 *               before the translations that use them, and the tensor-core product forms
 *               each BF16 tile in the GEMM's producer warps (FP32 arithmetic, phase taken
 *               relative to the offset's centre distance).  AUTO generates the levels whose
 *               FP64 tables would exceed 6 GB (both products), and stores the others:
 *               generating a tile costs about twice streaming it from device memory.
 */
#define NESA_TABLES_AUTO 0      /* translation matrices: generated where the tables would not fit */
#define NESA_TABLES_STORED 1    /* every translation matrix stored */
#define NESA_TABLES_GENERATED 2 /* every translation matrix generated when used */
#define NESA_SINGULAR_TOUCHING 0 /* singularity extraction for every triangle pair sharing a vertex */
#define NESA_SINGULAR_SELF 1     /* extraction for T = T' only; pairs sharing a vertex or an edge use the
                                    plain 7 x 7 rule (its nodes are interior, R > 0); Z symmetric to rounding */
typedef struct {
  double leaf_size;
  int32_t n_levels;
  int32_t q_mode;
  int32_t q_fixed;
  int32_t precision;
  double q_digits;
  double rho_eq;
  double rho_test;
  double pinv_eps;
  int32_t translate;
  int32_t tile_n;
  int32_t points_per_leaf;
  int32_t singular_mode;
  int32_t translation_tables;
  int32_t reserved;
} nesa_params;

/* Sizes of a built operator (host struct filled by nesa_get_info). */
#define NESA_MAX_LEVELS 20
typedef struct {
  int64_t n_unknowns;               /* N */
  int64_t n_triangles;
  int64_t n_points;                 /* 7 * n_triangles quadrature points (sources) */
  int32_t n_levels;                 /* L + 1 */
  int32_t l0;                       /* coarsest far level */
  int32_t q[NESA_MAX_LEVELS];       /* Q_l (0 above l0) */
  int64_t n_boxes[NESA_MAX_LEVELS]; /* occupied boxes per level */
  int64_t n_interactions[NESA_MAX_LEVELS]; /* interaction-list pairs per level */
  int64_t n_offsets[NESA_MAX_LEVELS];      /* distinct translation offsets per level */
  int64_t near_nnz;                 /* stored near-field entries */
  int64_t near_tri_pairs;           /* triangle pairs with a near part */
  int64_t v_columns;                /* sum over leaves of the RWG columns of V */
  int64_t device_bytes;             /* device memory held by the context */
  double build_seconds;             /* wall time of nesa_build */
  int64_t max_leaf_columns;         /* largest number of V columns of one leaf */
  double build_split[4];            /* seconds of nesa_build in: mesh and RWG functions (host),
                                       octree and box lists (device), near pattern and V lists
                                       (host threads), operator fill (device); 0 from nesa_plan */
} nesa_info;

/* Default parameters: leaf 0.25, 3 levels, NESA_Q_AUTO, q_fixed 100, q_digits 5,
   rho_eq 1, rho_test (2 - sqrt3/2)/(sqrt3/2), pinv_eps 1e-9, NESA_FP64, points_per_leaf 0,
   NESA_SINGULAR_TOUCHING. */
void nesa_default_params(nesa_params *p);

/*
 * Build the operator of a mesh at wavenumber k (> 0).  Copies the mesh, builds the RWG
 * functions, the octree and its lists, and fills the near-field matrix and the
 * radiation, transfer and translation operators on the current CUDA device.  On
 * success *out owns everything; release it with nesa_destroy.  Synchronous.
 * Errors: INVALID_ARG, MESH, CUDA, OOM.
 */
int nesa_build(const nesa_mesh *mesh, double k, const nesa_params *params, nesa_ctx **out);

/*
 * The host part of nesa_build alone (no device, no CUDA call): RWG functions, octree,
 * lists and Q per level for the same arguments, reported in *info (host struct) as
 * nesa_get_info would report them; device_bytes is 0 and build_seconds the host time.
 * Synchronous.  Errors: INVALID_ARG, MESH, OOM.
 */
int nesa_plan(const nesa_mesh *mesh, double k, const nesa_params *params, nesa_info *info);

/* Use cuda_stream (a cudaStream_t, may be NULL for the legacy stream) for all later
   device work of the context. */
int nesa_set_stream(nesa_ctx *ctx, void *cuda_stream);

int nesa_num_unknowns(const nesa_ctx *ctx, int64_t *n);
int nesa_get_info(const nesa_ctx *ctx, nesa_info *info);

/*
 * y = Z~ x for nrhs column-major vectors (dev, complex128, N x nrhs each; x and y must
 * not overlap).  Z~ is the NESA approximation of the EFIE matrix: the near part exactly
 * as Eq. 3 (point pairs in touching leaves, singular pairs by extraction) plus the five
 * far stages.  1 <= nrhs <= 64.  Asynchronous on the context's stream.
 */
int nesa_matvec(nesa_ctx *ctx, const nesa_c128 *x_dev, nesa_c128 *y_dev, int nrhs);

/* As nesa_matvec, applying only the parts selected by NESA_PART_* bits. */
int nesa_matvec_parts(nesa_ctx *ctx, const nesa_c128 *x_dev, nesa_c128 *y_dev, int nrhs, int parts);

/*
 * End-to-end product from host memory: copies x (host, N x nrhs) to the device,
 * applies nesa_matvec_parts(parts) and copies y back to host memory.  Synchronous.
 * Uses device buffers held by the context (grown on demand).  Pinned host memory
 * gives the fastest copies.
 */
int nesa_matvec_host(nesa_ctx *ctx, const nesa_c128 *x_host, nesa_c128 *y_host, int nrhs, int parts);

/*
 * Plane-wave excitation b_m = -int E^i . phi_m with E^i = pol_r exp(-i k khat_r . r)
 * (Sec. 2, Eq. 2; 7-point rule per triangle).  khat: host [nrhs][3] unit vectors;
 * pol: host [nrhs][3] complex; b_dev: dev, N x nrhs.  Asynchronous.
 */
int nesa_rhs_planewave(nesa_ctx *ctx, const double *khat, const nesa_c128 *pol, int nrhs, nesa_c128 *b_dev);

/*
 * Solve Z~ x = b by restarted GMRES(m) on the device (Sec. 2 names GMRES as the
 * iterative solver; Saad & Schultz 1986).  x0 = 0; Arnoldi by classical Gram-Schmidt
 * applied twice; Givens rotations; a right-hand side stops when its residual estimate
 * |g_{j+1}|/||b|| <= tol; the true residual b - Z~ x is recomputed at every restart and
 * at the end.  The nrhs right-hand sides advance in lock step (one product of nrhs
 * columns per Arnoldi step) with separate Krylov spaces.
 *   b_dev  dev, N x nrhs (read);  x_dev  dev, N x nrhs (written);  1 <= nrhs <= 64
 *   opts   NULL for defaults (restart 50, max_iters 1000)
 *   info   may be NULL; filled also when the solve does not converge
 * Returns NESA_OK when every true relative residual is <= tol, NESA_ERR_NOT_CONVERGED
 * when max_iters was reached first (x holds the last iterate), NESA_ERR_NUMERIC on
 * NaN/Inf.  Synchronous (the host reads one status word per Arnoldi step).
 * Device workspace: (restart + 3) * N * nrhs complex values, kept by the context.
 */
#define NESA_PRECOND_NONE 0
#define NESA_PRECOND_BLOCK_JACOBI 1 /* inverted near-field diagonal blocks, one per home leaf */
#define NESA_PRECOND_LEARNED 2      /* trained network correction of NESA_PRECOND_OVERLAP (see
                                       below); NESA_PRECOND_OVERLAP until trained */
#define NESA_PRECOND_OVERLAP 3      /* overlapping block-Jacobi (restricted additive Schwarz):
                                       the rows of a home-leaf group of the inverse of the
                                       near-field block over the functions whose home leaf
                                       touches the group's leaf (complex64) */
typedef struct {
  int32_t restart;    /* Krylov dimension m of a cycle */
  int32_t max_iters;  /* total Arnoldi steps (over all inner solves when mixed) */
  int32_t precond;    /* NESA_PRECOND_*: right preconditioning Z M y = b, x = M y */
  int32_t mixed;      /* 1: FP64 iterative refinement - r = b - Z~ x with the FP64 product,
                         an inner GMRES on the NESA_PART_MIXED product solves for the
                         correction to inner_tol, x += d - until ||r||/||b|| <= tol
                         (context built with NESA_MIXED); Arnoldi and Givens stay FP64 */
  int32_t max_refine; /* refinement steps (default 10) */
  double inner_tol;   /* relative tolerance of each inner solve (default 3e-3); a step that
                         needs less to reach tol/2 asks only for that */
  int32_t reserved[3];
} nesa_solve_opts;
typedef struct {
  int32_t iterations;      /* Arnoldi steps taken */
  int32_t restarts;        /* completed cycles before the last one */
  int32_t converged;       /* right-hand sides whose true residual met tol */
  int32_t matvecs;         /* products of nrhs columns (all precisions) */
  int32_t refinements;     /* refinement steps (mixed) */
  int32_t fp64_matvecs;    /* FP64 products among them */
  double rel_residual[64]; /* final true FP64 ||b - Z~ x|| / ||b|| per right-hand side */
  double seconds;          /* wall time of the call */
} nesa_solve_info;
void nesa_default_solve_opts(nesa_solve_opts *opts);
int nesa_solve(nesa_ctx *ctx, const nesa_c128 *b_dev, nesa_c128 *x_dev, int nrhs, double tol,
               const nesa_solve_opts *opts, nesa_solve_info *info);

/*
 * Preconditioners (not in the paper; the solver of Sec. 2 is used with them).
 *
 * Block-Jacobi: every RWG function belongs to the leaf holding the centroid of its T+;
 * the near-field diagonal block of each group is inverted (Gauss-Jordan, partial
 * pivoting, FP64).
 *
 * Overlapping block-Jacobi S: for each group, the extended set E = functions whose home
 * leaf touches the group's leaf; S r on the group = rows of the group of
 * (Z^near restricted to E x E)^-1 applied to r restricted to E (LU per group at setup).
 * Plain block-Jacobi can slow the EFIE down (its small blocks have nearly singular
 * loop modes); the overlapping one is the fallback of the learned preconditioner.
 *
 * Learned: M u = a1 u + a2 (S u) + a3 (S N S u), N = near-field product, with
 * complex coefficients a per RWG function from a network shared by all functions:
 * 8 static local features -> tanh 32 -> tanh 32 -> 6 (Re, Im of a1..a3).  Features:
 * k l, A+/l^2, A-/l^2, Re and Im of Z_mm/|Z_mm|, log(|Z_mm| / mean |Z_mm|), near-row
 * length / mean, group size / mean (mean over functions).  Weights: W1[32][8], b1[32],
 * W2[32][32], b2[32], W3[6][32], b3[6] (row-major, 1542 FP32 values, in this order);
 * the initial weights give a = (0, 1, 0), i.e. S.  Training (GPU kernels: forward,
 * backward, Adam) minimises L = sum_s |M(u_s) - v_s|^2 / sum_s |v_s|^2 over pairs
 * u_s = Z~ v_s, v_s the Arnoldi vectors of S-preconditioned GMRES for the training
 * right-hand sides.  Inference uses an FP16 copy of the weights with FP32 arithmetic.
 * Training always starts from the initial weights.  A lower L does not always mean
 * faster GMRES (on the aircraft body the trained map lowered L on held-out Krylov
 * vectors 8x and still stalled GMRES), so training ends with a validation: val_iters
 * steps of right-preconditioned GMRES on the last training right-hand side with the
 * trained weights and with the initial ones (M = S); the trained weights are kept only
 * if their true relative residual is lower, otherwise the initial weights are restored
 * (fallback = 1).
 */
#define NESA_LEARN_PARAMS 1542
typedef struct {
  int32_t samples;   /* Arnoldi vectors per training right-hand side (default 48) */
  int32_t steps;     /* Adam steps (default 300) */
  float lr;          /* Adam learning rate (default 3e-3) */
  int32_t val_iters; /* GMRES steps of the validation (default 100; 0: keep the trained weights) */
  int32_t reserved[4];
} nesa_learn_opts;
typedef struct {
  double loss_initial; /* L with the initial (overlapping block-Jacobi) weights */
  double loss_final;   /* L after training */
  int32_t samples;     /* training pairs */
  int32_t steps;
  double seconds;      /* training and validation */
  double val_res_learned; /* validation: true relative residual with the trained weights */
  double val_res_base;    /* validation: the same with the initial weights (M = S) */
  int32_t fallback;       /* 1: the initial weights were restored */
  int32_t val_iters;
} nesa_learn_info;
/* Build the block-Jacobi blocks and the features (idempotent; also done on demand). */
int nesa_precond_setup(nesa_ctx *ctx);
/* z = M r for kind NESA_PRECOND_BLOCK_JACOBI or NESA_PRECOND_LEARNED (dev, N x nrhs). */
int nesa_precond_apply(nesa_ctx *ctx, int kind, const nesa_c128 *r_dev, nesa_c128 *z_dev, int nrhs);
void nesa_default_learn_opts(nesa_learn_opts *opts);
/* Collect training pairs from b (dev, N x nrhs training right-hand sides) and train. */
int nesa_precond_train(nesa_ctx *ctx, const nesa_c128 *b_dev, int nrhs, const nesa_learn_opts *opts,
                       nesa_learn_info *info);
/* Get (set = 0) or set (set = 1) the NESA_LEARN_PARAMS weights (host FP32).  Setting
   them marks the learned preconditioner as trained. */
int nesa_precond_params(nesa_ctx *ctx, int set, float *host_params);
/* Features of every function (host, N x 8 FP32). */
int nesa_precond_features(nesa_ctx *ctx, float *host_features);
/* L and dL/dweights (host, NESA_LEARN_PARAMS FP32; may be NULL) for given pairs u, v
   (dev, N x nsamples each) with the current weights. */
int nesa_precond_loss_grad(nesa_ctx *ctx, const nesa_c128 *u_dev, const nesa_c128 *v_dev, int nsamples,
                           double *loss, float *grad_host);

/*
 * Export internal arrays for tests and tools (host copies).
 *   NESA_EXPORT_POINT_LEAF  int32 [n_points][3]  integer leaf coordinates of each
 *                           quadrature point (point 7t+i = node i of triangle t)
 *   NESA_EXPORT_RWG         int32 [N][4]  (vertex a, vertex b, T+, T-)
 * bytes must equal the array size.  Synchronous.
 */
#define NESA_EXPORT_POINT_LEAF 1
#define NESA_EXPORT_RWG 2
int nesa_export(const nesa_ctx *ctx, int which, void *host_buf, size_t bytes);

/*
 * Export one operator block (host copy of the FP64 operator, complex128 column-major):
 *   NESA_OP_D       D_l(o) of Eq. 12 for level l (l0 <= l <= L) and offset slot index
 *                   (0 .. n_offsets[l]-1): Q_l x Q_l, entry (i, j) = G(|E_i + o w_l - E_j|)
 *   NESA_OP_C       C_l(octant) of Eq. 11 for level l (l0 < l <= L), index = octant bits
 *                   x | y << 1 | z << 2 of the child: Q_{l-1} x Q_l
 *   NESA_OP_OFFSET  the offset o of slot index at level l: int32[3] (target - source, in
 *                   boxes of level l)
 * bytes must equal the block size (NESA_ERR_INVALID_ARG otherwise, and for an index
 * out of range).  Synchronous.
 */
#define NESA_OP_D 1
#define NESA_OP_C 2
#define NESA_OP_OFFSET 3
int nesa_export_op(const nesa_ctx *ctx, int which, int level, int index, void *host_buf, size_t bytes);

/*
 * Per-stage device timing of the product (for benchmarks).  When enabled, every kernel
 * launch of nesa_matvec* is bracketed by CUDA events on the context's stream.
 * nesa_profile_read synchronises the stream, adds the elapsed times of all launches
 * since the last read to the totals and returns them.  Stages:
 *   0 radiation (Eq. 10)   1 source transfer (Eq. 11)
 *   2 translation + potential transfer (Eqs. 12-13)   3 near field + reception (Eqs. 9, 14)
 *   4 the tensor-core GEMM launches alone (part of stage 2, NESA_TRANSLATE_TENSOR)
 * flops and bytes are the algorithmic FP64 flops (8 per complex multiply-add) and the
 * bytes of operator data and vectors each launch must touch at least once.
 */
#define NESA_STAGES 5
typedef struct {
  int64_t launches[NESA_STAGES];
  double ms[NESA_STAGES];
  double flops[NESA_STAGES];
  double bytes[NESA_STAGES];
} nesa_profile;
int nesa_profile_enable(nesa_ctx *ctx, int enable); /* also resets the totals */
int nesa_profile_read(nesa_ctx *ctx, nesa_profile *out);

/*
 * nesa_matvec_noalloc - the product y = Z~ x for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a property of the library, not of
 * the method.
 *
 * nesa_matvec keeps its per-level work vectors in buffers that the context allocates
 * (cudaMalloc) the first time a given nrhs is used.  Callers that must not allocate -
 * code running while a stream is captured into a CUDA graph, code held to a fixed
 * device-memory budget, real-time loops where an allocation could synchronise the
 * device - can call this entry point instead.  It runs the same kernels with the work
 * vectors taken from one fixed array of NESA_NOALLOC_SCRATCH_BYTES in device memory
 * that is part of the library image (present on every GPU that loads the library,
 * until the process exits).  It calls no allocating routine.
 *
 *   x_dev, y_dev, nrhs   as for nesa_matvec (caller-owned device memory)
 * Returns NESA_ERR_INVALID_ARG (with a message in nesa_last_error) when the work
 * vectors of this operator and nrhs need more than NESA_NOALLOC_SCRATCH_BYTES (about
 * 22 MB per right-hand side for 30,720 unknowns, 52 MB for 122,880).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current): make that first call before any
 * stream capture.  Call it with the context's device (the device current at nesa_build)
 * current: with another device current it returns NESA_ERR_INVALID_ARG and launches
 * nothing.  All calls share the array, which keeps the last call's data; calls whose
 * kernels overlap on the GPU race on it.  Asynchronous on the context's stream.
 */
#define NESA_NOALLOC_SCRATCH_BYTES (32u << 20)
int nesa_matvec_noalloc(nesa_ctx *ctx, const nesa_c128 *x_dev, nesa_c128 *y_dev, int nrhs);

/*
 * Batched passes over several operators (meshes of uneven size), each with its own
 * right-hand sides: one CUDA graph holds the products of all members as independent
 * branches, and one launch runs a pass (y_i = Z~_i x_i for every member i).
 *   ctxs[n], x_dev[n], y_dev[n], nrhs[n]   members and their buffers (dev, N_i x nrhs_i;
 *                                          bound into the graph: keep them alive)
 *   parts                                  NESA_PART_* bits as in nesa_matvec_parts
 * nesa_batch_create runs every product once eagerly (allocations, tile tuning), then
 * captures the kernels; it is synchronous.  A member context must not be destroyed or
 * rebuilt while the batch exists, and the batch must not run concurrently with other
 * work on its members.  While the batch exists, every product, solve or training call on
 * a member must use the member's nrhs (the graph holds the work buffers sized for it):
 * other counts fail with NESA_ERR_INVALID_ARG, and so does a context listed twice.
 * nesa_batch_launch is asynchronous on `stream`.
 */
typedef struct nesa_batch nesa_batch;
/*
 * Build the operators of n meshes for a batched pass (the several meshes of uneven size
 * of one sweep): out[i] = the context of meshes[i] at wavenumber k[i] (host array of n),
 * each exactly as nesa_build with the shared params.  Each mesh keeps its own tree, Q_l
 * and lists; nesa_batch_create then puts their products into one graph.  On failure
 * every context built so far is destroyed, out[] holds NULL, and the status of the first
 * mesh that failed is returned (its index is in nesa_last_error).  Synchronous.
 */
int nesa_build_batch(const nesa_mesh *meshes, int n, const double *k, const nesa_params *params, nesa_ctx **out);
int nesa_batch_create(nesa_ctx *const *ctxs, int n, const nesa_c128 *const *x_dev, nesa_c128 *const *y_dev,
                      const int *nrhs, int parts, nesa_batch **out);
int nesa_batch_launch(nesa_batch *batch, void *cuda_stream);
/* number of kernel nodes in the batch's graph */
int nesa_batch_kernels(const nesa_batch *batch, int64_t *kernel_nodes);
void nesa_batch_destroy(nesa_batch *batch);

/*
 * Tile widths (64, 128 or 256 columns) of the tensor-core translation GEMM chosen by the
 * autotuner for each level (0 above l0 or without NESA_TRANSLATE_TENSOR), and the times
 * it measured (ms per launch for widths 64, 128, 256; [level][3]).  Host arrays of
 * NESA_MAX_LEVELS and 3 * NESA_MAX_LEVELS entries.
 */
int nesa_get_tuning(nesa_ctx *ctx, int32_t *tile_n, float *ms);

/*
 * Device-side status of the context's kernels since the last call: NESA_OK, or
 * NESA_ERR_TIMEOUT when a bounded wait inside a kernel (tensor-core translation) ran
 * out; that product's result is then invalid.  Clears the status.  Synchronous.
 */
int nesa_device_status(nesa_ctx *ctx);

/*
 * Failure-detection hook (not part of the method; for tests of the timeout path).
 * While stall = 1, the producer warps of the tensor-core GEMMs (NESA_TRANSLATE_TENSOR
 * mixed products) issue no copies and publish no stage, so the consumers' bounded
 * mbarrier waits run out: the kernel leaves early without touching memory it does not
 * own, the product's result is invalid, and nesa_device_status returns
 * NESA_ERR_TIMEOUT.  Nothing faults, traps or hangs.  wait_limit is the number of
 * try-wait iterations of every bounded wait (0 restores the default, 2^20; a try-wait
 * sleeps up to 20 us while the phase is incomplete); stall = 0
 * restores normal products.  Host state only; takes effect at the next launch.
 */
int nesa_inject_stall(nesa_ctx *ctx, int stall, uint32_t wait_limit);

/* Release all memory of the context (NULL is allowed). */
void nesa_destroy(nesa_ctx *ctx);

const char *nesa_status_str(int status);

/* Message of the last failed nesa_build on this host thread ("" if none). */
const char *nesa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NESA_H */
