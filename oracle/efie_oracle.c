/*
 * EFIE oracle, C part.  TEST INFRASTRUCTURE ONLY: this file is compiled and called by
 * the oracle package (tests, the smoke check and the CPU baseline of the benchmark).
 * The library under paper_1801_03589_gb300/ never includes, links or calls it.
 *
 * Plain, slow, obviously correct FP64 loops; one triangle pair at a time.
 *
 * What it computes (paper Sec. 2, Eq. 1 and Eq. 3, with the gradient term moved onto
 * the testing function by integration by parts, valid for RWG functions):
 *
 *   Z_mn = -i eta k  int_T int_T' g(r,r') [ phi_m(r).phi_n(r') - k^-2 div phi_m div' phi_n ]
 *   g(r,r') = exp(-i k R) / (4 pi R),   R = |r - r'|
 *
 * For an RWG function supported on triangle T with free vertex v, edge length l,
 * area A and sign s (+1 on T+, -1 on T-):  phi = s l/(2A) (r - v),  div phi = s l / A.
 * Hence every RWG pair entry is a sum over its 2x2 triangle pairs of
 *   -i eta k  s s' l l'  M_ij(T, T')
 * with the 3x3 "pair matrix" over free vertices i of T and j of T'
 *   M_ij = sum_p sum_q w_p w_q g(r_p, r_q) [ (r_p - v_i).(r_q - v'_j)/4 - 1/k^2 ]
 * (7-point rule on each triangle, weights w summing to 1 per triangle; the areas
 * cancel against the 1/(2A) factors).
 *
 * Triangle pairs that share at least one vertex (including T = T') are "singular":
 * g = (exp(-ikR) - 1)/(4 pi R) + 1/(4 pi R).  The first (bounded) part uses the same
 * 7x7 rule; for the second, the inner integrals over T' of 1/R and (r'-r)/R are taken
 * in closed form (Wilton et al. 1984; Graglia 1993) and the outer one by the 7-point
 * rule.  The singular pair value is computed with the lower-numbered triangle as the
 * outer one and transposed for the mirrored pair; a self pair is symmetrised, so that
 * the assembled Z is exactly symmetric (reciprocity).
 *
 * singular_mode 1 ("self only") restricts the extraction to T = T': pairs that share
 * only a vertex or an edge then use the plain 7x7 rule (its nodes are interior, so R > 0),
 * and Z is symmetric to rounding only.  Touching pairs must still lie entirely in
 * touching leaves in the near-part mode (the leaf-size rule does not depend on the
 * integration rule).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double PI = 3.14159265358979323846;

static void sub3(const double *a, const double *b, double *c) { c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/*
 * Closed-form potential integrals over a flat triangle with vertices v[0..2] (each 3
 * doubles) seen from point r:
 *   I1    = int_T 1/|r - r'| dS'
 *   Iv[3] = int_T (r' - r)/|r - r'| dS'
 * Edge formulas: with n the unit normal, d = n.(r - v0) and rho the projection of r
 * on the plane, for edge i running from a to b (counter-clockwise about n), unit
 * tangent t, outward in-plane normal u = t x n, s- = (a - rho).t, s+ = (b - rho).t,
 * t0 = (a - rho).u, R0^2 = t0^2 + d^2, R- = |r - a|, R+ = |r - b|,
 *   f_i = ln((R+ + s+)/(R- + s-)),
 *   beta_i = atan(t0 s+/(R0^2 + |d| R+)) - atan(t0 s-/(R0^2 + |d| R-)),
 *   I1 = sum_i t0 f_i - |d| sum_i beta_i,
 *   int (rho' - rho)/R = 1/2 sum_i u_i [R0^2 f_i + s+ R+ - s- R-],
 * and (r' - r) = (rho' - rho) - d n on the plane.
 */
void orc_static_integrals(const double *v, const double *r, double *I1, double *Iv) {
  double e1[3], e2[3], n[3];
  sub3(v + 3, v, e1);
  sub3(v + 6, v, e2);
  cross3(e1, e2, n);
  double nn = norm3(n);
  n[0] /= nn; n[1] /= nn; n[2] /= nn;
  double rv[3];
  sub3(r, v, rv);
  double d = dot3(n, rv);
  double ad = fabs(d);
  double rho[3] = {r[0] - d * n[0], r[1] - d * n[1], r[2] - d * n[2]};
  double scale = norm3(e1) + norm3(e2);
  double i1 = 0.0, ip[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i) {
    const double *a = v + 3 * i;
    const double *b = v + 3 * ((i + 1) % 3);
    double ab[3];
    sub3(b, a, ab);
    double len = norm3(ab);
    double t[3] = {ab[0] / len, ab[1] / len, ab[2] / len};
    double u[3];
    cross3(t, n, u);
    double arho[3], brho[3];
    sub3(a, rho, arho);
    sub3(b, rho, brho);
    double sm = dot3(arho, t), sp = dot3(brho, t), t0 = dot3(arho, u);
    double R0sq = t0 * t0 + d * d;
    double ra[3], rb[3];
    sub3(r, a, ra);
    sub3(r, b, rb);
    double Rm = norm3(ra), Rp = norm3(rb);
    double f;
    if (R0sq < 1e-28 * scale * scale) {
      f = 0.0; /* r on the edge's line: every term below carries a factor t0 or R0^2 */
    } else if (sm >= 0.0 || sp >= 0.0) {
      /* (R + s) is well conditioned when s >= 0; for s < 0 use (R+ + s+)/(R- + s-) =
         (R- - s-)/(R+ - s+) which follows from (R+s)(R-s) = R0^2 */
      if (sm > 0.0 && sp > 0.0)
        f = log((Rp + sp) / (Rm + sm));
      else if (sm <= 0.0 && sp <= 0.0)
        f = log((Rm - sm) / (Rp - sp));
      else
        f = log((Rp + sp) * (Rm - sm) / R0sq);
    } else {
      f = log((Rm - sm) / (Rp - sp));
    }
    double beta = atan2(t0 * sp, R0sq + ad * Rp) - atan2(t0 * sm, R0sq + ad * Rm);
    i1 += t0 * f - ad * beta;
    double c = 0.5 * (R0sq * f + sp * Rp - sm * Rm);
    ip[0] += c * u[0];
    ip[1] += c * u[1];
    ip[2] += c * u[2];
  }
  *I1 = i1;
  Iv[0] = ip[0] - d * n[0] * i1;
  Iv[1] = ip[1] - d * n[1] * i1;
  Iv[2] = ip[2] - d * n[2] * i1;
}

static double tri_area(const double *v) {
  double e1[3], e2[3], c[3];
  sub3(v + 3, v, e1);
  sub3(v + 6, v, e2);
  cross3(e1, e2, c);
  return 0.5 * norm3(c);
}

/* exp(-ikR)/(4 pi R), or its bounded part (exp(-ikR) - 1)/(4 pi R) when smooth_only. */
static cplx green(double k, double R, int smooth_only) {
  if (!smooth_only) return cexp(-I * k * R) / (4.0 * PI * R);
  if (R == 0.0) return -I * k / (4.0 * PI);
  double h = sin(0.5 * k * R);
  return (-2.0 * h * h - I * sin(k * R)) / (4.0 * PI * R);
}

/*
 * Pair matrix M[i][j] (row-major 3x3) for outer triangle a (vertices va, 7 points qa,
 * weights w) and inner triangle b.  mask (7x7, may be NULL) keeps only the point pairs
 * with mask[p*7+q] != 0 (used for the near part of non-singular pairs).  singular:
 * use the extraction described above (the mask is then ignored).
 */
static void pair_matrix(const double *va, const double *qa, const double *vb, const double *qb,
                        const double *w, double k, int singular, const unsigned char *mask, cplx M[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = 0.0;
  double ik2 = 1.0 / (k * k);
  for (int p = 0; p < 7; ++p) {
    const double *rp = qa + 3 * p;
    for (int q = 0; q < 7; ++q) {
      if (!singular && mask && !mask[p * 7 + q]) continue;
      const double *rq = qb + 3 * q;
      double d[3];
      sub3(rp, rq, d);
      cplx g = green(k, norm3(d), singular) * (w[p] * w[q]);
      for (int i = 0; i < 3; ++i) {
        double a[3];
        sub3(rp, va + 3 * i, a);
        for (int j = 0; j < 3; ++j) {
          double b[3];
          sub3(rq, vb + 3 * j, b);
          M[i][j] += g * (0.25 * dot3(a, b) - ik2);
        }
      }
    }
  }
  if (!singular) return;
  double Ab = tri_area(vb);
  for (int p = 0; p < 7; ++p) {
    const double *rp = qa + 3 * p;
    double I1, Iv[3];
    orc_static_integrals(vb, rp, &I1, Iv);
    for (int i = 0; i < 3; ++i) {
      double a[3];
      sub3(rp, va + 3 * i, a);
      for (int j = 0; j < 3; ++j) {
        double b[3];
        sub3(rp, vb + 3 * j, b);
        double vec[3] = {Iv[0] + b[0] * I1, Iv[1] + b[1] * I1, Iv[2] + b[2] * I1};
        M[i][j] += w[p] * (dot3(a, vec) / (16.0 * PI * Ab) - I1 * ik2 / (4.0 * PI * Ab));
      }
    }
  }
}

static int share_vertex(const int32_t *ta, const int32_t *tb) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (ta[i] == tb[j]) return 1;
  return 0;
}

/* Pair matrix with the symmetry rules of the file header applied. */
static void pair_matrix_sym(int64_t ta, int64_t tb, const double *verts, const int32_t *tris,
                            const double *qpts, const double *w, double k, int singular,
                            const unsigned char *mask, cplx M[3][3]) {
  double va[9], vb[9];
  if (singular && ta > tb) {
    cplx Mt[3][3];
    pair_matrix_sym(tb, ta, verts, tris, qpts, w, k, singular, NULL, Mt);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = Mt[j][i];
    return;
  }
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) {
      va[3 * c + x] = verts[3 * tris[3 * ta + c] + x];
      vb[3 * c + x] = verts[3 * tris[3 * tb + c] + x];
    }
  pair_matrix(va, qpts + 21 * ta, vb, qpts + 21 * tb, w, k, singular, mask, M);
  if (singular && ta == tb) {
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j) {
        cplx s = 0.5 * (M[i][j] + M[j][i]);
        M[i][j] = s;
        M[j][i] = s;
      }
  }
}

/*
 * Rows of the EFIE matrix.
 *   verts [nv*3], tris [nt*3]             mesh
 *   qpts  [nt*7*3], w [7]                 7-point rule nodes per triangle and weights
 *   tri_rwg [nt*3]                        RWG index attached to the edge opposite local
 *                                          vertex c of triangle t, or -1
 *   tri_sl  [nt*3]                        sign * edge length of that RWG on t
 *   rwg_tri [n*2], rwg_free [n*2]         T+/T- of each RWG and the local index of its
 *                                          free vertex in each
 *   rows [nrows]                          requested RWG rows m
 *   mode 0: full matrix (dense MoM)
 *   mode 1: near part only: point pairs (p,q) whose leaves touch, leaf integer coordinates
 *           given per point in leaf_ijk [nt*7*3]; touching pairs must be entirely near
 *   singular_mode 0: extraction for every pair sharing a vertex; 1: for T = T' only
 *   out [nrows * n] complex (row-major)
 * Returns 0, or -1 if (mode 1) a singular pair has a point pair in non-touching leaves.
 */
int orc_efie_rows(int64_t nv, const double *verts, int64_t nt, const int32_t *tris, const double *qpts,
                  const double *w, int64_t n, const int32_t *tri_rwg, const double *tri_sl,
                  const int32_t *rwg_tri, const int32_t *rwg_free, double k, double eta,
                  int64_t nrows, const int64_t *rows, int mode, const int32_t *leaf_ijk, int singular_mode,
                  double complex *out) {
  (void)nv;
  (void)rwg_free;
  const cplx pref = -I * eta * k;
  int status = 0;
  memset(out, 0, sizeof(cplx) * (size_t)nrows * (size_t)n);
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t m = rows[r];
    cplx *zrow = out + r * n;
    for (int side = 0; side < 2; ++side) {
      int64_t ta = rwg_tri[2 * m + side];
      int ia = -1;
      for (int c = 0; c < 3; ++c)
        if (tri_rwg[3 * ta + c] == m) ia = c;
      double sla = tri_sl[3 * ta + ia];
      int lo[3], hi[3];
      if (mode == 1) {
        for (int x = 0; x < 3; ++x) { lo[x] = 1 << 30; hi[x] = -(1 << 30); }
        for (int p = 0; p < 7; ++p)
          for (int x = 0; x < 3; ++x) {
            int c = leaf_ijk[(ta * 7 + p) * 3 + x];
            if (c < lo[x]) lo[x] = c;
            if (c > hi[x]) hi[x] = c;
          }
      }
      for (int64_t tb = 0; tb < nt; ++tb) {
        int touching = share_vertex(tris + 3 * ta, tris + 3 * tb);
        int singular = touching && (singular_mode == 0 || ta == tb);
        unsigned char mask[49];
        const unsigned char *mp = NULL;
        if (mode == 1) {
          /* quick reject on the leaf coordinate ranges, then the exact per-pair mask */
          int any = 0;
          for (int q = 0; q < 7 && !any; ++q) {
            const int32_t *cq = leaf_ijk + (tb * 7 + q) * 3;
            if (cq[0] >= lo[0] - 1 && cq[0] <= hi[0] + 1 && cq[1] >= lo[1] - 1 && cq[1] <= hi[1] + 1 &&
                cq[2] >= lo[2] - 1 && cq[2] <= hi[2] + 1)
              any = 1;
          }
          if (!any && !touching) continue;
          int cnt = 0;
          for (int p = 0; p < 7; ++p)
            for (int q = 0; q < 7; ++q) {
              const int32_t *cp = leaf_ijk + (ta * 7 + p) * 3;
              const int32_t *cq = leaf_ijk + (tb * 7 + q) * 3;
              int near = abs(cp[0] - cq[0]) <= 1 && abs(cp[1] - cq[1]) <= 1 && abs(cp[2] - cq[2]) <= 1;
              mask[p * 7 + q] = (unsigned char)near;
              cnt += near;
            }
          if (touching && cnt != 49) status = -1;
          if (cnt == 0) continue;
          mp = mask;
        }
        cplx M[3][3];
        pair_matrix_sym(ta, tb, verts, tris, qpts, w, k, singular, mp, M);
        for (int jb = 0; jb < 3; ++jb) {
          int32_t nn = tri_rwg[3 * tb + jb];
          if (nn < 0) continue;
          zrow[nn] += pref * sla * tri_sl[3 * tb + jb] * M[ia][jb];
        }
      }
    }
  }
  return status;
}

/*
 * Plain 7-point-rule integral of f(r) = exp(-ik R)/(4 pi R) against nothing: helper for
 * the far-field check.  Green's function matrix G[i][j] = g(a_i, b_j) (row-major,
 * na x nb), R = 0 entries set to 0.
 */
void orc_green_matrix(double k, int64_t na, const double *a, int64_t nb, const double *b, double complex *G) {
  for (int64_t i = 0; i < na; ++i)
    for (int64_t j = 0; j < nb; ++j) {
      double d[3];
      sub3(a + 3 * i, b + 3 * j, d);
      double R = norm3(d);
      G[i * nb + j] = R > 0.0 ? cexp(-I * k * R) / (4.0 * PI * R) : 0.0;
    }
}
