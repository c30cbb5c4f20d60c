/*
 * nesa2d.h - C ABI of the 2D model problem in libnesa.so (arxiv 1801.03589, Sec. 3).
 *
 * The potential of N charges q_j at points x_j in the plane, evaluated at the points,
 *     phi_i = sum_{j != i} -log|x_i - x_j| q_j                          (Eq. 8),
 * by the nested equivalent source approximation: the near field between neighbouring
 * finest-level groups (Eq. 9) and the five far-field stages radiation, source
 * transfer, translation, potential transfer and reception (Eqs. 10-14).  Real FP64;
 * every stage of the product runs in the library's own CUDA kernels.
 *
 * Construction (the readings of Sec. 3 this library takes):
 *   - Quadtree: the root square has the side of the largest extent of the points and
 *     its lower-left corner at their minimum; a point belongs to box
 *     floor((x - lo) / w_l), the last box on the upper edges.  The coarsest level is
 *     l0 = 2 (four groups along the longest dimension); the finest level L is the
 *     deepest whose occupied groups hold on average at least P points (L = l0 if none).
 *   - Near groups: the occupied 8-neighbours and the group itself, at level L.
 *     Interaction lists: at l0 all occupied groups that are not near; below, the
 *     occupied children of the parent's near groups that are not near.
 *   - Per level, Q equivalent points on the circle of radius R = w / sqrt(2) about the
 *     group centre at angles 2 pi (j + 1/2) / Q, and 2Q test points on the circle of
 *     radius (2 - 1/sqrt(2)) w at angles 2 pi j / (2Q).  K_l is the Tikhonov
 *     pseudo-inverse of G(T, E), G = -log|.|, regularised by pinv_eps ||G(T, E)||_F.
 *   - V = K_L G(T + c, X) (Eq. 10), C = K_{l-1} G(T_{l-1}, E_l + delta) (Eq. 11),
 *     D(off) = G(E + off w, E) (Eq. 12), B = C^T (Eq. 13), U = V^T (Eq. 14).
 *
 * Conventions: points are host memory, [n][2] doubles, copied at build.  Vectors are
 * device pointers owned by the caller: a block of nrhs vectors of length n is
 * column-major (element i of vector r at [r * n + i]), in the caller's point order.
 * Calls return NESA_OK (0) or a negative NESA_ERR_* status of nesa.h; device work is
 * ordered on the context's stream (set with nesa2d_set_stream; default the legacy
 * stream) and the product does not synchronise.
 */
#ifndef NESA2D_H
#define NESA2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nesa2d_ctx nesa2d_ctx;

/* Sizes of a built operator (host struct filled by nesa2d_get_info). */
#define NESA2D_MAX_LEVELS 32
typedef struct {
  int64_t n_points;
  int32_t l0, L;                              /* coarsest far level, finest level */
  int32_t q;                                  /* Q, equivalent points per group */
  int32_t reserved;
  int64_t n_boxes[NESA2D_MAX_LEVELS];         /* occupied groups per level */
  int64_t n_interactions[NESA2D_MAX_LEVELS];  /* interaction-list pairs per level */
  int64_t n_offsets[NESA2D_MAX_LEVELS];       /* distinct translation offsets per level */
  int64_t near_entries;                       /* stored near-field matrix entries */
  int64_t device_bytes;
} nesa2d_info;

/*
 * Build the operator for n points (host, [n][2]), group size P (>= 1) and Q (1..1024)
 * equivalent points per group; pinv_eps <= 0 selects 1e-9.  The near-field blocks and
 * every operator are filled on the host and copied to the current CUDA device.
 * Synchronous.  Errors: INVALID_ARG (n < 2, bad P or Q, non-finite or coincident
 * points), CUDA, OOM.
 */
int nesa2d_build(const double *points, int64_t n, int P, int Q, double pinv_eps, nesa2d_ctx **out);
int nesa2d_set_stream(nesa2d_ctx *ctx, void *cuda_stream);
int nesa2d_get_info(const nesa2d_ctx *ctx, nesa2d_info *info);

/* Which parts of the product to apply (or-ed): the near field (Eq. 9), the far field
   (Eqs. 10-14), or both. */
#define NESA2D_PART_NEAR 1
#define NESA2D_PART_FAR 2
#define NESA2D_PART_ALL 3

/*
 * phi = K~ q for nrhs (1..64) vectors q (dev, n x nrhs) into phi (dev, n x nrhs; may
 * not alias q).  Asynchronous on the context's stream; the work vectors are allocated
 * at the first call with a given nrhs.  Errors: INVALID_ARG, CUDA, OOM.
 */
int nesa2d_matvec(nesa2d_ctx *ctx, const double *q_dev, double *phi_dev, int nrhs, int parts);

void nesa2d_destroy(nesa2d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NESA2D_H */
