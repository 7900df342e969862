/*
 * difvm_oracle.c -- plain, slow, FP64 CPU oracle of the DiFVM face-operator /
 * PISO path (arxiv 2603.15920, Sec. 2.3-2.6).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, constant or helper with the CUDA library; both are fed the same
 * seeded mesh arrays and nothing else.
 *
 * Every operator is the textbook face loop of the paper's message-passing form
 * (Sec. 2.4.1, Eqs. message/aggregate): visit faces in ascending face id,
 * compute the face quantity once, add it to the owner and subtract it from the
 * neighbour (sigma = +1 owner, -1 neighbour).  Boundary faces are edges from a
 * ghost node: they touch only their owner.  No blocking, fusion or reordering.
 *
 * Conventions
 *   mesh arrays: owner[nf], neighbour[nint], Sf/Cf [nf][3], V[nc], C[nc][3];
 *                boundary faces nint..nf-1 grouped by patch.
 *   fields:      component-major, phi[c*nc + i]; boundary values
 *                phib[c*nb + (f - nint)].
 *   bc[patch]:   0 fixed value (use phib), 1 zero gradient (use the owner
 *                value), 2 empty (face excluded from every sum).
 *   gradient:    grad[(c*3 + d)*nc + i] = d phi_c / d x_d.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   w_f  = S.(C_N - x_f) / S.(C_N - C_O)   owner weight of linear interpolation
 *   c_f  = |S|^2 / (S.d)                   |Delta_f|/|d| for the over-relaxed
 *                                          split Delta = (|S|/|S^.d^|) d^ (Eq. nonortho_flux;
 *                                          the minimum / orthogonal / no-correction
 *                                          splits of the same paragraph by om_mesh.nonorth)
 *   k_f  = S - c_f d                        non-orthogonal remainder
 *   boundary diffusion is orthogonal only, d = x_f - C_O.
 *   a boundary face carries its boundary-condition value for every scheme.
 *
 * Parity pins: see tests/test_oracle_*.py (closed forms, invariants, dense
 * solves, the manufactured Poisson solution of Sec. 3.1.1; the adjoint of a
 * PISO step against central differences of the forward step).
 * The interpolation weight w_f is a reading (the paper says only "linear
 * interpolation"); its computation is pinned by its defining property (the
 * interpolated value of a linear field is the field where the segment C_O-C_N
 * pierces the face plane, on jittered tetrahedra) and by w = 1/2 on uniform
 * hexes.  What stays open is the reading itself, not its implementation.
 *
 * Multi-core build (compiled with -fopenmp; only the all-cores CPU baseline
 * uses it): the Krylov vector loops run on all threads, the LDU apply visits
 * each cell's faces in ascending face id through a cell-to-face table (the
 * same additions in the same order as the face loop, so bitwise the same y),
 * and inner products add fixed blocks of OM_DOT_BLOCK entries and then the
 * block sums in order (the result does not depend on the thread count; it
 * differs from the single-thread sum by rounding only).  Everything else is
 * the code above, unchanged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nc, nint, nf, npatch;
  const int *owner, *neighbour;
  const double *Sf, *Cf, *V, *C;
  const int *patch_start, *patch_size, *patch_type;
  int nonorth;   /* split of S_f in Eq. nonortho_flux: NO_OVERRELAXED .. NO_NONE */
} om_mesh;

enum { BC_FIXED = 0, BC_ZEROGRAD = 1, BC_EMPTY = 2 };
enum { PT_WALL = 0, PT_INLET = 1, PT_OUTLET = 2, PT_EMPTY = 3 };
enum { DIV_UPWIND = 0, DIV_LINEAR = 1 };
enum { WK_EXACT = 0, WK_FE = 1, WK_BE = 2 };
enum { NO_OVERRELAXED = 0, NO_MINIMUM = 1, NO_ORTHOGONAL = 2, NO_NONE = 3 };
enum { CONV_UPWIND = 0, CONV_SOU = 1 };
enum { TIME_BE = 0, TIME_CN = 1 };

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static int patch_of_face(const om_mesh *m, int f) {
  for (int p = 0; p < m->npatch; ++p)
    if (f >= m->patch_start[p] && f < m->patch_start[p] + m->patch_size[p]) return p;
  return -1;
}

/* bc kind of the velocity / pressure fields implied by a patch type */
static int bc_of_U(int pt) { return pt == PT_EMPTY ? BC_EMPTY : (pt == PT_OUTLET ? BC_ZEROGRAD : BC_FIXED); }
static int bc_of_p(int pt) { return pt == PT_EMPTY ? BC_EMPTY : (pt == PT_OUTLET ? BC_FIXED : BC_ZEROGRAD); }

/* Limited explicit non-orthogonal correction ("limited corrected psi" of
 * OpenFOAM, used where the plain over-relaxed correction of Eq. nonortho_flux
 * is unstable): the correction is capped at psi/(1-psi) times the magnitude of
 * the orthogonal part of the same face flux; psi >= 1 leaves it unlimited. */
static double limit_corr(double corr, double orth, double psi) {
  if (psi >= 1.0) return corr;
  double cap = psi / (1.0 - psi) * fabs(orth);
  if (fabs(corr) > cap) return corr > 0.0 ? cap : -cap;
  return corr;
}

/* ---------------------------------------------------------------- geometry */
/* |Delta_f| / |d| for the split S = Delta + k of Eq. nonortho_flux, Delta
 * along d (Sec. 2.3.2, the paragraph on non-orthogonality correction):
 *   over-relaxed  Delta = (|S| / |S^.d^|) d^   ->  |S|^2 / (S.d)
 *   minimum       Delta = (S.d^) d^            ->  (S.d) / |d|^2
 *   orthogonal    Delta = |S| d^               ->  |S| / |d|
 *   none          the two-point flux of Eq. diff_ortho: |S| / |d|, k = 0 */
static double split_coeff(int scheme, const double *S, const double *d) {
  switch (scheme) {
    case NO_MINIMUM: return dot3(S, d) / dot3(d, d);
    case NO_ORTHOGONAL:
    case NO_NONE: return sqrt(dot3(S, S)) / sqrt(dot3(d, d));
    default: return dot3(S, S) / dot3(S, d);
  }
}

/* Derived face coefficients (Sec. 2.3.2): w[nint], c[nf], k[nint*3] with
 * k = S - Delta = S - c d (0 for the scheme without correction).  The splits
 * are defined along the cell-to-cell vector d_ij; a boundary face has none and
 * keeps the orthogonal-only boundary flux of the readings above. */
void om_face_coeffs(const om_mesh *m, double *w, double *c, double *k) {
  for (int f = 0; f < m->nf; ++f) {
    const double *S = m->Sf + 3 * f, *xf = m->Cf + 3 * f, *CO = m->C + 3 * m->owner[f];
    double d[3];
    if (f < m->nint) {
      const double *CN = m->C + 3 * m->neighbour[f];
      double dN[3] = {CN[0] - xf[0], CN[1] - xf[1], CN[2] - xf[2]};
      for (int a = 0; a < 3; ++a) d[a] = CN[a] - CO[a];
      w[f] = dot3(S, dN) / dot3(S, d);
      c[f] = split_coeff(m->nonorth, S, d);
      for (int a = 0; a < 3; ++a) k[3 * f + a] = m->nonorth == NO_NONE ? 0.0 : S[a] - c[f] * d[a];
    } else {   /* no cell on the other side: every scheme keeps |S|^2 / (S.d), d = x_f - C_O */
      for (int a = 0; a < 3; ++a) d[a] = xf[a] - CO[a];
      c[f] = split_coeff(NO_OVERRELAXED, S, d);
    }
  }
}

/* Geometry checks: V > 0, S.d > 0 on every face, and the closure residual
 * max_i |sum sigma S_f| / (sum |S_f|) over cells with no empty faces.
 * Returns the number of violations; *closure gets the worst residual. */
int om_check_geometry(const om_mesh *m, const int *bcU, double *closure) {
  int bad = 0;
  double *r = calloc((size_t)m->nc * 3, sizeof(double));
  double *a = calloc((size_t)m->nc, sizeof(double));
  char *hasempty = calloc((size_t)m->nc, 1);
  for (int i = 0; i < m->nc; ++i) bad += !(m->V[i] > 0);
  for (int f = 0; f < m->nf; ++f) {
    const double *S = m->Sf + 3 * f, *CO = m->C + 3 * m->owner[f];
    double d[3];
    int O = m->owner[f];
    if (f < m->nint) {
      int N = m->neighbour[f];
      for (int q = 0; q < 3; ++q) d[q] = m->C[3 * N + q] - CO[q];
      for (int q = 0; q < 3; ++q) { r[3 * O + q] += S[q]; r[3 * N + q] -= S[q]; }
      a[O] += sqrt(dot3(S, S)); a[N] += sqrt(dot3(S, S));
    } else {
      for (int q = 0; q < 3; ++q) d[q] = m->Cf[3 * f + q] - CO[q];
      for (int q = 0; q < 3; ++q) r[3 * O + q] += S[q];
      a[O] += sqrt(dot3(S, S));
      if (bcU && bcU[patch_of_face(m, f)] == BC_EMPTY) hasempty[O] = 1;
    }
    bad += !(dot3(S, d) > 0);
  }
  double worst = 0;
  for (int i = 0; i < m->nc; ++i) {
    if (hasempty[i]) continue;
    double e = sqrt(dot3(r + 3 * i, r + 3 * i)) / a[i];
    if (e > worst) worst = e;
  }
  *closure = worst;
  free(r); free(a); free(hasempty);
  return bad;
}

/* ------------------------------------------------------- face interpolation */
/* Face value of component `comp` on face f (Sec. 2.3.2, linear interpolation;
 * boundary faces take their boundary-condition value).  Returns 0 if the face
 * is empty (excluded), 1 otherwise. */
static int face_value(const om_mesh *m, const double *w, const int *bc, const double *phi,
                      const double *phib, int f, double *out) {
  int O = m->owner[f];
  if (f < m->nint) {
    int N = m->neighbour[f];
    *out = w[f] * phi[O] + (1.0 - w[f]) * phi[N];
    return 1;
  }
  int kind = bc[patch_of_face(m, f)];
  if (kind == BC_EMPTY) return 0;
  *out = (kind == BC_FIXED) ? phib[f - m->nint] : phi[O];
  return 1;
}

/* -------------------------------------------------------------- Gauss grad */
/* (grad phi)_i = (1/V_i) sum_f sigma phi_f S_f   (Eq. gauss_green) */
void om_grad_gauss(const om_mesh *m, const int *bc, int ncomp, const double *phi,
                   const double *phib, double *grad) {
  int nc = m->nc, nb = m->nf - m->nint;
  double *w = malloc(sizeof(double) * (m->nint + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (m->nint + 1));
  om_face_coeffs(m, w, c, k);
  memset(grad, 0, sizeof(double) * (size_t)ncomp * 3 * nc);
  for (int q = 0; q < ncomp; ++q) {
    const double *ph = phi + (size_t)q * nc, *pb = phib ? phib + (size_t)q * nb : NULL;
    double *g = grad + (size_t)q * 3 * nc;
    for (int f = 0; f < m->nf; ++f) {
      double pf;
      if (!face_value(m, w, bc, ph, pb, f, &pf)) continue;
      const double *S = m->Sf + 3 * f;
      int O = m->owner[f];
      for (int d = 0; d < 3; ++d) g[d * nc + O] += pf * S[d];
      if (f < m->nint) {
        int N = m->neighbour[f];
        for (int d = 0; d < 3; ++d) g[d * nc + N] -= pf * S[d];
      }
    }
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < nc; ++i) g[d * nc + i] /= m->V[i];
  }
  free(w); free(c); free(k);
}

/* ------------------------------------------------------------- convection */
/* R_i = sum_f sigma m_f phi_f   (Eq. conv_face_flux; upwind Eq. upwind with
 * m_f >= 0 taking the owner value; linear = central interpolation) */
void om_div_flux(const om_mesh *m, const int *bc, int scheme, int ncomp, const double *mf,
                 const double *phi, const double *phib, double *out) {
  int nc = m->nc, nb = m->nf - m->nint;
  double *w = malloc(sizeof(double) * (m->nint + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (m->nint + 1));
  om_face_coeffs(m, w, c, k);
  memset(out, 0, sizeof(double) * (size_t)ncomp * nc);
  for (int q = 0; q < ncomp; ++q) {
    const double *ph = phi + (size_t)q * nc, *pb = phib ? phib + (size_t)q * nb : NULL;
    double *r = out + (size_t)q * nc;
    for (int f = 0; f < m->nf; ++f) {
      double pf;
      int O = m->owner[f];
      if (f < m->nint) {
        int N = m->neighbour[f];
        if (scheme == DIV_UPWIND) pf = (mf[f] >= 0.0) ? ph[O] : ph[N];
        else pf = w[f] * ph[O] + (1.0 - w[f]) * ph[N];
        r[O] += mf[f] * pf;
        r[N] -= mf[f] * pf;
      } else {
        if (!face_value(m, w, bc, ph, pb, f, &pf)) continue;
        r[O] += mf[f] * pf;
      }
    }
  }
  free(w); free(c); free(k);
}

/* -------------------------------------------------------------- diffusion */
/* R_i = sum_f sigma gamma [ c_f (phi_N - phi_O) + (grad phi)_f . k_f ]
 * (Eq. nonortho_flux, over-relaxed), boundary fixed value: gamma c_f (phi_b - phi_O),
 * zero gradient and empty: 0.  grad == NULL gives the orthogonal part only. */
void om_laplacian(const om_mesh *m, const int *bc, int ncomp, double gamma, const double *phi,
                  const double *phib, const double *grad, double *out) {
  int nc = m->nc, nb = m->nf - m->nint;
  double *w = malloc(sizeof(double) * (m->nint + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (m->nint + 1));
  om_face_coeffs(m, w, c, k);
  memset(out, 0, sizeof(double) * (size_t)ncomp * nc);
  for (int q = 0; q < ncomp; ++q) {
    const double *ph = phi + (size_t)q * nc, *pb = phib ? phib + (size_t)q * nb : NULL;
    const double *g = grad ? grad + (size_t)q * 3 * nc : NULL;
    double *r = out + (size_t)q * nc;
    for (int f = 0; f < m->nf; ++f) {
      int O = m->owner[f];
      if (f < m->nint) {
        int N = m->neighbour[f];
        double F = gamma * c[f] * (ph[N] - ph[O]);
        if (g) {
          double gf[3];
          for (int d = 0; d < 3; ++d) gf[d] = w[f] * g[d * nc + O] + (1.0 - w[f]) * g[d * nc + N];
          F += gamma * dot3(gf, k + 3 * f);
        }
        r[O] += F;
        r[N] -= F;
      } else {
        int kind = bc[patch_of_face(m, f)];
        if (kind == BC_FIXED) r[O] += gamma * c[f] * (pb[f - m->nint] - ph[O]);
      }
    }
  }
  free(w); free(c); free(k);
}

/* ------------------------------------------------------------- LDU apply */
/* y_i = D_i x_i + sum_{f: O=i} U_f x_N + sum_{f: N=i} L_f x_O   (Eq. Ap_H).
 * U == NULL means symmetric (U = L).  Swapping L and U gives A^T. */
#ifdef _OPENMP
/* cell -> internal-face table of the last mesh seen, faces ascending per cell */
static struct { const int *owner; int nc, nint; int *ptr, *ent; } om_csr;
static void om_csr_build(const om_mesh *m) {
  if (om_csr.owner == m->owner && om_csr.nc == m->nc && om_csr.nint == m->nint) return;
  free(om_csr.ptr); free(om_csr.ent);
  int *ptr = calloc((size_t)m->nc + 1, sizeof(int)), *ent = malloc(sizeof(int) * (2 * (size_t)m->nint + 1));
  for (int f = 0; f < m->nint; ++f) { ptr[m->owner[f] + 1]++; ptr[m->neighbour[f] + 1]++; }
  for (int i = 0; i < m->nc; ++i) ptr[i + 1] += ptr[i];
  int *fill = malloc(sizeof(int) * ((size_t)m->nc + 1));
  memcpy(fill, ptr, sizeof(int) * (size_t)m->nc);
  for (int f = 0; f < m->nint; ++f) {        /* entry = face << 1 | (1 if the cell is the neighbour) */
    ent[fill[m->owner[f]]++] = f << 1;
    ent[fill[m->neighbour[f]]++] = (f << 1) | 1;
  }
  free(fill);
  om_csr.owner = m->owner; om_csr.nc = m->nc; om_csr.nint = m->nint;
  om_csr.ptr = ptr; om_csr.ent = ent;
}
#endif

void om_ldu_apply(const om_mesh *m, int ncomp, const double *D, const double *L,
                  const double *U, const double *x, double *y) {
  int nc = m->nc;
  if (!U) U = L;
#ifdef _OPENMP
  om_csr_build(m);
  for (int q = 0; q < ncomp; ++q) {
    const double *xq = x + (size_t)q * nc;
    double *yq = y + (size_t)q * nc;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nc; ++i) {
      double acc = D[i] * xq[i];
      for (int e = om_csr.ptr[i]; e < om_csr.ptr[i + 1]; ++e) {
        int f = om_csr.ent[e] >> 1;
        if (om_csr.ent[e] & 1) acc += L[f] * xq[m->owner[f]];
        else acc += U[f] * xq[m->neighbour[f]];
      }
      yq[i] = acc;
    }
  }
  return;
#endif
  for (int q = 0; q < ncomp; ++q) {
    const double *xq = x + (size_t)q * nc;
    double *yq = y + (size_t)q * nc;
    for (int i = 0; i < nc; ++i) yq[i] = D[i] * xq[i];
    for (int f = 0; f < m->nint; ++f) {
      int O = m->owner[f], N = m->neighbour[f];
      yq[O] += U[f] * xq[N];
      yq[N] += L[f] * xq[O];
    }
  }
}

/* ---------------------------------------------------------------- Krylov */
#ifdef _OPENMP
#define OM_DOT_BLOCK 4096
static double vdot(int n, const double *a, const double *b) {
  int nblk = (n + OM_DOT_BLOCK - 1) / OM_DOT_BLOCK;
  double *part = malloc(sizeof(double) * (nblk > 0 ? nblk : 1));
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nblk; ++k) {
    double s = 0.0;
    int e = (k + 1) * OM_DOT_BLOCK < n ? (k + 1) * OM_DOT_BLOCK : n;
    for (int i = k * OM_DOT_BLOCK; i < e; ++i) s += a[i] * b[i];
    part[k] = s;
  }
  double s = 0.0;
  for (int k = 0; k < nblk; ++k) s += part[k];
  free(part);
  return s;
}
#else
static double vdot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
#endif

/* number of threads the multi-core build uses (1 in the single-thread build) */
int om_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void om_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

typedef struct { int iters; double res0, res, bnorm; int status; } om_info;

/* Jacobi-preconditioned conjugate gradient (SPD pressure system, Sec. 2.6.1).
 * Stops when ||b - A x||_2 (recursive residual) <= max(tol_rel ||b||_2, tol_abs).
 * status 0 converged, 3 not converged, 5 non-finite. */
int om_pcg(const om_mesh *m, const double *D, const double *L, const double *U, const double *b,
           double *x, double tol_rel, double tol_abs, int maxit, om_info *info) {
  int n = m->nc;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
  double bn = sqrt(vdot(n, b, b));
  info->bnorm = bn; info->iters = 0; info->status = 0;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->res0 = info->res = 0.0;
    free(r); free(z); free(p); free(q);
    return 0;
  }
  double tol = fmax(tol_rel * bn, tol_abs);
  om_ldu_apply(m, 1, D, L, U, x, q);
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rn = sqrt(vdot(n, r, r));
  info->res0 = rn;
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) { z[i] = r[i] / D[i]; p[i] = z[i]; }
  double rz = vdot(n, r, z);
  int it = 0;
  while (rn > tol && it < maxit) {
    om_ldu_apply(m, 1, D, L, U, p, q);
    double alpha = rz / vdot(n, p, q);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    ++it;
    rn = sqrt(vdot(n, r, r));
    if (!isfinite(rn)) { info->status = 5; break; }
    if (rn <= tol) break;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) z[i] = r[i] / D[i];
    double rz1 = vdot(n, r, z);
    double beta = rz1 / rz;
    rz = rz1;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  info->iters = it; info->res = rn;
  if (info->status == 0 && rn > tol) info->status = 3;
  free(r); free(z); free(p); free(q);
  return info->status;
}

/* Diagonal incomplete Cholesky (the CG preconditioner the paper names, Sec. 2.6.1,
 * in its DIC form for a symmetric LDU matrix: D diagonal, L[f] the off-diagonal of
 * internal face f).  Cells are eliminated in the order rank[i] (the library uses its
 * RCM numbering); for face f, lo(f) / hi(f) are its cells of lower / higher rank.
 *   d_i = D_i - sum_{f: hi(f)=i} L_f^2 / d_lo(f)          in increasing rank
 * M = (Dd + Lo) Dd^-1 (Dd + Lo^T) with Dd = diag(d), Lo the strictly lower part:
 * diag(M) = diag(A) and M = A on the matrix's sparsity pattern (fill-in dropped).
 * d[nc] out. */
static void dic_sides(const om_mesh *m, const int *rank, int f, int *lo, int *hi) {
  int O = m->owner[f], N = m->neighbour[f];
  if (rank[O] < rank[N]) { *lo = O; *hi = N; } else { *lo = N; *hi = O; }
}

/* faces of each cell (CSR over cells) and the cells in rank order */
static void dic_tables(const om_mesh *m, const int *rank, int **fptr, int **fidx, int **byrank) {
  int nc = m->nc, ni = m->nint;
  int *ptr = calloc((size_t)nc + 1, sizeof(int)), *idx = malloc(sizeof(int) * 2 * (ni + 1));
  for (int f = 0; f < ni; ++f) { ptr[m->owner[f] + 1]++; ptr[m->neighbour[f] + 1]++; }
  for (int i = 0; i < nc; ++i) ptr[i + 1] += ptr[i];
  int *fill = malloc(sizeof(int) * nc);
  for (int i = 0; i < nc; ++i) fill[i] = ptr[i];
  for (int f = 0; f < ni; ++f) { idx[fill[m->owner[f]]++] = f; idx[fill[m->neighbour[f]]++] = f; }
  int *br = malloc(sizeof(int) * nc);
  for (int i = 0; i < nc; ++i) br[rank[i]] = i;
  free(fill);
  *fptr = ptr; *fidx = idx; *byrank = br;
}

void om_dic_factor(const om_mesh *m, const double *D, const double *L, const int *rank, double *d) {
  int *ptr, *idx, *br;
  dic_tables(m, rank, &ptr, &idx, &br);
  for (int k = 0; k < m->nc; ++k) {
    int i = br[k];
    double s = D[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (hi == i) s -= L[f] * L[f] / d[lo];
    }
    d[i] = s;
  }
  free(ptr); free(idx); free(br);
}

/* z = M^-1 r: forward (Dd + Lo) y = r, then backward (I + Dd^-1 Lo^T) z = y */
static void dic_apply(const om_mesh *m, const int *rank, const int *ptr, const int *idx,
                      const int *br, const double *d, const double *L, const double *r, double *z) {
  int nc = m->nc;
  for (int k = 0; k < nc; ++k) {
    int i = br[k];
    double s = r[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (hi == i) s -= L[f] * z[lo];
    }
    z[i] = s / d[i];
  }
  for (int k = nc - 1; k >= 0; --k) {
    int i = br[k];
    double s = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (lo == i) s += L[f] * z[hi];
    }
    z[i] -= s / d[i];
  }
}

/* CG preconditioned by DIC in the elimination order rank; same stopping rule as om_pcg */
int om_pcg_dic(const om_mesh *m, const double *D, const double *L, const int *rank, const double *b,
               double *x, double tol_rel, double tol_abs, int maxit, om_info *info) {
  int n = m->nc;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
  double *d = malloc(sizeof(double) * n);
  int *ptr, *idx, *br;
  dic_tables(m, rank, &ptr, &idx, &br);
  om_dic_factor(m, D, L, rank, d);
  double bn = sqrt(vdot(n, b, b));
  info->bnorm = bn; info->iters = 0; info->status = 0;
  int it = 0;
  double rn = 0.0;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->res0 = 0.0;
  } else {
    double tol = fmax(tol_rel * bn, tol_abs);
    om_ldu_apply(m, 1, D, L, NULL, x, q);
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    rn = sqrt(vdot(n, r, r));
    info->res0 = rn;
    dic_apply(m, rank, ptr, idx, br, d, L, r, z);
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = vdot(n, r, z);
    while (rn > tol && it < maxit) {
      om_ldu_apply(m, 1, D, L, NULL, p, q);
      double alpha = rz / vdot(n, p, q);
      for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      ++it;
      rn = sqrt(vdot(n, r, r));
      if (!isfinite(rn)) { info->status = 5; break; }
      if (rn <= tol) break;
      dic_apply(m, rank, ptr, idx, br, d, L, r, z);
      double rz1 = vdot(n, r, z);
      double beta = rz1 / rz;
      rz = rz1;
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (info->status == 0 && rn > tol) info->status = 3;
  }
  info->iters = it; info->res = rn;
  free(r); free(z); free(p); free(q); free(d); free(ptr); free(idx); free(br);
  return info->status;
}

/* Diagonal incomplete LU (DILU): the same factorisation for the non-symmetric
 * momentum matrix (Sec. 2.6.1 names ILU for the solvers).  Row O of an internal
 * face holds U_f in column N and row N holds L_f in column O (as om_ldu_apply);
 * in the elimination order rank, a(hi,lo) is the face's entry below the
 * diagonal and a(lo,hi) the one above it.  With Dd = diag(d), Lo / Up the
 * strictly lower / upper parts of A in that order,
 *   M = (Dd + Lo) Dd^-1 (Dd + Up),   d_i = D_i - sum_{f: hi(f)=i} L_f U_f / d_lo(f)
 * (the product a(hi,lo) a(lo,hi) is L_f U_f whichever side is lower):
 * diag(M) = diag(A) and M = A on the matrix's sparsity pattern.  U == L (or
 * NULL) gives the DIC factor. */
static double dilu_lower(const om_mesh *m, const int *rank, int f, const double *L, const double *U) {
  return rank[m->owner[f]] < rank[m->neighbour[f]] ? L[f] : U[f];   /* a(hi,lo) */
}
static double dilu_upper(const om_mesh *m, const int *rank, int f, const double *L, const double *U) {
  return rank[m->owner[f]] < rank[m->neighbour[f]] ? U[f] : L[f];   /* a(lo,hi) */
}

void om_dilu_factor(const om_mesh *m, const double *D, const double *L, const double *U, const int *rank,
                    double *d) {
  int *ptr, *idx, *br;
  if (!U) U = L;
  dic_tables(m, rank, &ptr, &idx, &br);
  for (int k = 0; k < m->nc; ++k) {
    int i = br[k];
    double s = D[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (hi == i) s -= L[f] * U[f] / d[lo];
    }
    d[i] = s;
  }
  free(ptr); free(idx); free(br);
}

/* z = M^-1 r: forward (Dd + Lo) y = r, then backward (I + Dd^-1 Up) z = y */
static void dilu_apply(const om_mesh *m, const int *rank, const int *ptr, const int *idx, const int *br,
                       const double *d, const double *L, const double *U, const double *r, double *z) {
  int nc = m->nc;
  for (int k = 0; k < nc; ++k) {
    int i = br[k];
    double s = r[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (hi == i) s -= dilu_lower(m, rank, f, L, U) * z[lo];
    }
    z[i] = s / d[i];
  }
  for (int k = nc - 1; k >= 0; --k) {
    int i = br[k];
    double s = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      int f = idx[e], lo, hi;
      dic_sides(m, rank, f, &lo, &hi);
      if (lo == i) s += dilu_upper(m, rank, f, L, U) * z[hi];
    }
    z[i] -= s / d[i];
  }
}

void om_dilu_apply(const om_mesh *m, const double *D, const double *L, const double *U, const int *rank,
                   const double *r, double *z) {
  int *ptr, *idx, *br;
  if (!U) U = L;
  double *d = malloc(sizeof(double) * m->nc);
  om_dilu_factor(m, D, L, U, rank, d);
  dic_tables(m, rank, &ptr, &idx, &br);
  dilu_apply(m, rank, ptr, idx, br, d, L, U, r, z);
  free(d); free(ptr); free(idx); free(br);
}

/* BiCGStab right-preconditioned by DILU in the elimination order rank: the
 * steps of om_bicgstab below with y = M^-1 p and z = M^-1 s in place of the
 * Jacobi scalings; same stopping rule. */
int om_bicgstab_dilu(const om_mesh *m, const double *D, const double *L, const double *U, const int *rank,
                     const double *b, double *x, double tol_rel, double tol_abs, int maxit, om_info *info) {
  int n = m->nc;
  if (!U) U = L;
  double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n);
  double *p = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
  double *y = malloc(sizeof(double) * n), *s = malloc(sizeof(double) * n);
  double *z = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
  double *d = malloc(sizeof(double) * n);
  int *ptr, *idx, *br;
  dic_tables(m, rank, &ptr, &idx, &br);
  om_dilu_factor(m, D, L, U, rank, d);
  double bn = sqrt(vdot(n, b, b));
  info->bnorm = bn; info->iters = 0; info->status = 0;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->res0 = info->res = 0.0;
    goto done;
  }
  double tol = fmax(tol_rel * bn, tol_abs);
  om_ldu_apply(m, 1, D, L, U, x, t);
  for (int i = 0; i < n; ++i) { r[i] = b[i] - t[i]; rh[i] = r[i]; }
  double rn = sqrt(vdot(n, r, r));
  info->res0 = rn;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  while (rn > tol && it < maxit) {
    double rho1 = vdot(n, rh, r);
    if (rho1 == 0.0 || omega == 0.0) { info->status = 4; break; }
    double beta = (rho1 / rho) * (alpha / omega);
    rho = rho1;
    for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    dilu_apply(m, rank, ptr, idx, br, d, L, U, p, y);
    om_ldu_apply(m, 1, D, L, U, y, v);
    alpha = rho / vdot(n, rh, v);
    for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    ++it;
    double sn = sqrt(vdot(n, s, s));
    if (sn <= tol) {
      for (int i = 0; i < n; ++i) x[i] += alpha * y[i];
      rn = sn;
      break;
    }
    dilu_apply(m, rank, ptr, idx, br, d, L, U, s, z);
    om_ldu_apply(m, 1, D, L, U, z, t);
    double tt = vdot(n, t, t);
    omega = tt > 0.0 ? vdot(n, t, s) / tt : 0.0;
    for (int i = 0; i < n; ++i) { x[i] += alpha * y[i] + omega * z[i]; r[i] = s[i] - omega * t[i]; }
    rn = sqrt(vdot(n, r, r));
    if (!isfinite(rn)) { info->status = 5; break; }
  }
  info->iters = it; info->res = rn;
  if (info->status == 0 && rn > tol) info->status = 3;
done:
  free(r); free(rh); free(p); free(v); free(y); free(s); free(z); free(t); free(d);
  free(ptr); free(idx); free(br);
  return info->status;
}

/* Right-Jacobi-preconditioned BiCGStab (van der Vorst 1992) for the
 * non-symmetric momentum system (Sec. 2.6.1).  Same stopping rule as om_pcg. */
int om_bicgstab(const om_mesh *m, const double *D, const double *L, const double *U,
                const double *b, double *x, double tol_rel, double tol_abs, int maxit, om_info *info) {
  int n = m->nc;
  double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n);
  double *p = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
  double *y = malloc(sizeof(double) * n), *s = malloc(sizeof(double) * n);
  double *z = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
  double bn = sqrt(vdot(n, b, b));
  info->bnorm = bn; info->iters = 0; info->status = 0;
  if (bn == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    info->res0 = info->res = 0.0;
    goto done;
  }
  double tol = fmax(tol_rel * bn, tol_abs);
  om_ldu_apply(m, 1, D, L, U, x, t);
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) { r[i] = b[i] - t[i]; rh[i] = r[i]; }
  double rn = sqrt(vdot(n, r, r));
  info->res0 = rn;
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  while (rn > tol && it < maxit) {
    double rho1 = vdot(n, rh, r);
    if (rho1 == 0.0 || omega == 0.0) { info->status = 4; break; }
    double beta = (rho1 / rho) * (alpha / omega);
    rho = rho1;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) y[i] = p[i] / D[i];
    om_ldu_apply(m, 1, D, L, U, y, v);
    alpha = rho / vdot(n, rh, v);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    ++it;
    double sn = sqrt(vdot(n, s, s));
    if (sn <= tol) {
      #pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) x[i] += alpha * y[i];
      rn = sn;
      break;
    }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) z[i] = s[i] / D[i];
    om_ldu_apply(m, 1, D, L, U, z, t);
    double tt = vdot(n, t, t);
    omega = tt > 0.0 ? vdot(n, t, s) / tt : 0.0;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) { x[i] += alpha * y[i] + omega * z[i]; r[i] = s[i] - omega * t[i]; }
    rn = sqrt(vdot(n, r, r));
    if (!isfinite(rn)) { info->status = 5; break; }
  }
  info->iters = it; info->res = rn;
  if (info->status == 0 && rn > tol) info->status = 3;
done:
  free(r); free(rh); free(p); free(v); free(y); free(s); free(z); free(t);
  return info->status;
}

/* ------------------------------------------------------------ Windkessel */
/* One RCR step per outlet (Eqs. windkessel_ode, windkessel_discrete):
 *   exact: p_c <- p_c e + R_d Q (1 - e),  e = exp(-dt/(R_d C))
 *   FE:    p_c <- p_c + dt (Q - p_c/R_d)/C
 *   BE:    p_c <- (p_c + dt Q/C) / (1 + dt/(R_d C))
 * then p_o = p_c + R_p Q. */
void om_windkessel_update(int n, int scheme, const double *Rp, const double *Cc, const double *Rd,
                          const double *Q, double dt, double *pc, double *pout) {
  for (int o = 0; o < n; ++o) {
    if (scheme == WK_EXACT) {
      double e = exp(-dt / (Rd[o] * Cc[o]));
      pc[o] = pc[o] * e + Rd[o] * Q[o] * (1.0 - e);
    } else if (scheme == WK_FE) {
      pc[o] = pc[o] + dt * (Q[o] - pc[o] / Rd[o]) / Cc[o];
    } else {
      pc[o] = (pc[o] + dt * Q[o] / Cc[o]) / (1.0 + dt / (Rd[o] * Cc[o]));
    }
    pout[o] = pc[o] + Rp[o] * Q[o];
  }
}

/* --------------------------------------------------- momentum assembly */
/* Backward-Euler, implicit upwind convection with the current face flux m,
 * implicit orthogonal diffusion, explicit non-orthogonal correction from
 * gradU (may be NULL).  Rows:  D_i U_i + sum offdiag = b_i  with
 *   D_i  = V_i/dt + sum_{O=i}(max(m,0) + nu c) + sum_{N=i}(max(-m,0) + nu c) + bnd
 *   Up_f = min(m,0) - nu c   (row O, column N)
 *   Lo_f = -max(m,0) - nu c  (row N, column O)
 *   b_i  = V_i/dt U^n_i + sigma nu (gradU)_f . k_f + bnd   (correction limited by psi)
 * boundary fixed U: D += nu c, b += (nu c - m) U_b;  zero gradient: D += m.
 * gradS (may be NULL): second-order upwind by deferred correction (Eqs.
 * deferred_correction, sou): on every internal face the explicit part
 *   t_f = m (gradS)_C . (x_f - x_C),  C = O if m >= 0 else N   (Eq. upwind)
 * leaves the upwind cell's row: b_O -= t_f, b_N += t_f.  Boundary faces keep
 * their boundary-condition face value. */
void om_momentum_assemble(const om_mesh *m, const int *bcU, double nu, double dt,
                          const double *mf, const double *Uold, const double *Ub,
                          const double *gradU, const double *gradS, double psi, double *D,
                          double *Lo, double *Up, double *b) {
  int nc = m->nc, nb = m->nf - m->nint;
  double *w = malloc(sizeof(double) * (m->nint + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (m->nint + 1));
  om_face_coeffs(m, w, c, k);
  for (int i = 0; i < nc; ++i) {
    D[i] = m->V[i] / dt;
    for (int q = 0; q < 3; ++q) b[q * nc + i] = m->V[i] / dt * Uold[q * nc + i];
  }
  for (int f = 0; f < m->nf; ++f) {
    int O = m->owner[f];
    double mm = mf[f];
    if (f < m->nint) {
      int N = m->neighbour[f];
      double a = nu * c[f];
      D[O] += fmax(mm, 0.0) + a;
      D[N] += fmax(-mm, 0.0) + a;
      Up[f] = fmin(mm, 0.0) - a;
      Lo[f] = -fmax(mm, 0.0) - a;
      if (gradU) {
        for (int q = 0; q < 3; ++q) {
          const double *g = gradU + (size_t)q * 3 * nc;
          double gf[3];
          for (int d = 0; d < 3; ++d) gf[d] = w[f] * g[d * nc + O] + (1.0 - w[f]) * g[d * nc + N];
          double orth = c[f] * (Uold[q * nc + N] - Uold[q * nc + O]);
          double corr = nu * limit_corr(dot3(gf, k + 3 * f), orth, psi);
          b[q * nc + O] += corr;
          b[q * nc + N] -= corr;
        }
      }
      if (gradS) {
        int Cu = mm >= 0.0 ? O : N;
        double dC[3];
        for (int a = 0; a < 3; ++a) dC[a] = m->Cf[3 * f + a] - m->C[3 * Cu + a];
        for (int q = 0; q < 3; ++q) {
          const double *g = gradS + (size_t)q * 3 * nc;
          double gC[3] = {g[Cu], g[nc + Cu], g[2 * nc + Cu]};
          double t = mm * dot3(gC, dC);
          b[q * nc + O] -= t;
          b[q * nc + N] += t;
        }
      }
    } else {
      int kind = bcU[patch_of_face(m, f)];
      int bf = f - m->nint;
      if (kind == BC_FIXED) {
        double a = nu * c[f];
        D[O] += a;
        for (int q = 0; q < 3; ++q) b[q * nc + O] += (a - mm) * Ub[q * nb + bf];
      } else if (kind == BC_ZEROGRAD) {
        D[O] += mm;
      }
    }
  }
  free(w); free(c); free(k);
}

/* Crank-Nicolson form of the momentum rows (Sec. 3 time schemes, second order):
 * with the backward-Euler rows D = V/dt + D_cd, off-diagonals Lo/Up and b = V/dt U^n + b_cd
 * of om_momentum_assemble, the spatial operator A_cd U - b_cd is averaged between the two
 * time levels: (V/dt + A_cd/2) U* = V/dt U^n + b_cd - A_cd U^n / 2.  Transforms D, Lo, Up,
 * b in place (A_cd U^n with the backward-Euler coefficients). */
void om_momentum_cn(const om_mesh *m, double dt, const double *Uold, double *D, double *Lo,
                    double *Up, double *b) {
  int nc = m->nc;
  for (int q = 0; q < 3; ++q) {
    const double *u = Uold + (size_t)q * nc;
    double *a = calloc((size_t)nc, sizeof(double));
    for (int i = 0; i < nc; ++i) a[i] = (D[i] - m->V[i] / dt) * u[i];
    for (int f = 0; f < m->nint; ++f) {
      a[m->owner[f]] += Up[f] * u[m->neighbour[f]];
      a[m->neighbour[f]] += Lo[f] * u[m->owner[f]];
    }
    for (int i = 0; i < nc; ++i) b[q * nc + i] -= 0.5 * a[i];
    free(a);
  }
  for (int i = 0; i < nc; ++i) D[i] = m->V[i] / dt + 0.5 * (D[i] - m->V[i] / dt);
  for (int f = 0; f < m->nint; ++f) { Lo[f] *= 0.5; Up[f] *= 0.5; }
}

/* H_i = b_i - sum_{f:O=i} Up_f U_N - sum_{f:N=i} Lo_f U_O  (Eq. Ap_H off-diagonal part) */
void om_H(const om_mesh *m, const double *Lo, const double *Up, const double *b,
          const double *U, double *H) {
  int nc = m->nc;
  for (int q = 0; q < 3; ++q) {
    const double *u = U + (size_t)q * nc;
    double *h = H + (size_t)q * nc;
    for (int i = 0; i < nc; ++i) h[i] = b[q * nc + i];
    for (int f = 0; f < m->nint; ++f) {
      int O = m->owner[f], N = m->neighbour[f];
      h[O] -= Up[f] * u[N];
      h[N] -= Lo[f] * u[O];
    }
  }
}

/* --------------------------------------------------- pressure assembly */
/* Pressure equation of one PISO corrector (Eqs. pressure_poisson, velocity_correction):
 *   phiHbyA_f = HbyA_f . S_f   (boundary: fixed U -> U_b.S, zero-gradient U -> HbyA_O.S)
 *   a_f       = rAU_f c_f,   rAU_f = w rAU_O + (1-w) rAU_N  (boundary fixed p: rAU_O c_f)
 *   nonorth_f = rAU_f (grad p)_f . k_f   (lagged from plag, limited by psi; gradp may be NULL)
 * SPD form  Dp p - sum a_f p_other = -div(phiHbyA) + div(nonorth) + sum_bnd a_f p_b
 * with Dp_i = sum a_f, Lp_f = -a_f.  af[nf] and nonorth[nint] are returned for the
 * flux correction. */
void om_pressure_assemble(const om_mesh *m, const int *bcU, const int *bcp, const double *rAU,
                          const double *HbyA, const double *Ub, const double *pb,
                          const double *gradp, const double *plag, double psi, double *Dp,
                          double *Lp, double *bp, double *phiHbyA, double *af, double *nonorth) {
  int nc = m->nc, nb = m->nf - m->nint;
  double *w = malloc(sizeof(double) * (m->nint + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (m->nint + 1));
  om_face_coeffs(m, w, c, k);
  for (int i = 0; i < nc; ++i) { Dp[i] = 0.0; bp[i] = 0.0; }
  for (int f = 0; f < m->nf; ++f) {
    const double *S = m->Sf + 3 * f;
    int O = m->owner[f];
    if (f < m->nint) {
      int N = m->neighbour[f];
      double hf[3];
      for (int d = 0; d < 3; ++d) hf[d] = w[f] * HbyA[d * nc + O] + (1.0 - w[f]) * HbyA[d * nc + N];
      phiHbyA[f] = dot3(hf, S);
      double rf = w[f] * rAU[O] + (1.0 - w[f]) * rAU[N];
      af[f] = rf * c[f];
      nonorth[f] = 0.0;
      if (gradp) {
        double gf[3];
        for (int d = 0; d < 3; ++d) gf[d] = w[f] * gradp[d * nc + O] + (1.0 - w[f]) * gradp[d * nc + N];
        nonorth[f] = rf * limit_corr(dot3(gf, k + 3 * f), c[f] * (plag[N] - plag[O]), psi);
      }
      Dp[O] += af[f];
      Dp[N] += af[f];
      Lp[f] = -af[f];
      bp[O] += -phiHbyA[f] + nonorth[f];
      bp[N] -= -phiHbyA[f] + nonorth[f];
    } else {
      int p = patch_of_face(m, f), bf = f - m->nint;
      int ku = bcU[p], kp = bcp[p];
      if (ku == BC_EMPTY) { phiHbyA[f] = 0.0; af[f] = 0.0; continue; }
      if (ku == BC_FIXED) {
        double ub[3] = {Ub[bf], Ub[nb + bf], Ub[2 * nb + bf]};
        phiHbyA[f] = dot3(ub, S);
      } else {
        double h[3] = {HbyA[O], HbyA[nc + O], HbyA[2 * nc + O]};
        phiHbyA[f] = dot3(h, S);
      }
      bp[O] += -phiHbyA[f];
      if (kp == BC_FIXED) {
        af[f] = rAU[O] * c[f];
        Dp[O] += af[f];
        bp[O] += af[f] * pb[bf];
      } else {
        af[f] = 0.0;
      }
    }
  }
  free(w); free(c); free(k);
}

/* ------------------------------------------------------------------ PISO */
typedef struct {
  double nu, dt;
  int ncorr, nonorth;           /* explicit non-orthogonal corrections: bit 0 momentum, bit 1 pressure */
  double tolU, tolp, tol_abs;
  int maxitU, maxitp;
  int pref_cell;                /* pinned cell when no patch fixes p */
  int wk_scheme;
  int n_out;                    /* Windkessel outlets */
  const int *wk_patch;          /* [n_out] patch ids */
  const double *Rp, *Cw, *Rd;   /* [n_out] */
  double psi;                   /* non-orthogonal limiter coefficient (1 = unlimited) */
  int conv;                     /* momentum convection: CONV_UPWIND or CONV_SOU (deferred correction) */
  int time;                     /* momentum time scheme: TIME_BE or TIME_CN */
} om_piso_opts;

typedef struct { int itU[3], itp[4], status; double Q[8], po[8]; } om_piso_info;

/* One PISO step (Sec. 2.4.2): Windkessel outlet update, momentum predictor
 * (BiCGStab per component), then ncorr pressure correctors (PCG) with the
 * Rhie-Chow flux correction and the velocity correction.  U[3][nc], p[nc],
 * phi[nf] are updated in place; Ub[3][nb] and pb[nb] hold the boundary values
 * at the new time level (pb is overwritten on Windkessel outlets); pc[n_out]
 * is the capacitor pressure, updated in place. */
int om_piso_step(const om_mesh *m, const om_piso_opts *o, double *U, double *p, double *phi,
                 const double *Ub, double *pb, double *pc, om_piso_info *info) {
  int nc = m->nc, nf = m->nf, ni = m->nint, nb = nf - ni;
  int *bcU = malloc(sizeof(int) * m->npatch), *bcp = malloc(sizeof(int) * m->npatch);
  int has_fixed_p = 0;
  for (int q = 0; q < m->npatch; ++q) {
    bcU[q] = bc_of_U(m->patch_type[q]);
    bcp[q] = bc_of_p(m->patch_type[q]);
    if (bcp[q] == BC_FIXED) has_fixed_p = 1;
  }
  memset(info, 0, sizeof(*info));
  /* 1. Windkessel outlets: Q from the current face flux, p_o imposed on the patch */
  for (int j = 0; j < o->n_out; ++j) {
    int q = o->wk_patch[j];
    double Q = 0.0;
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) Q += phi[f];
    double po;
    om_windkessel_update(1, o->wk_scheme, o->Rp + j, o->Cw + j, o->Rd + j, &Q, o->dt, pc + j, &po);
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) pb[f - ni] = po;
    if (j < 8) { info->Q[j] = Q; info->po[j] = po; }
  }
  double *gradp = malloc(sizeof(double) * 3 * nc), *gradU = malloc(sizeof(double) * 9 * nc);
  double *D = malloc(sizeof(double) * nc), *Lo = malloc(sizeof(double) * (ni + 1));
  double *Up = malloc(sizeof(double) * (ni + 1)), *b = malloc(sizeof(double) * 3 * nc);
  double *rhs = malloc(sizeof(double) * nc), *rAU = malloc(sizeof(double) * nc);
  double *H = malloc(sizeof(double) * 3 * nc), *HbyA = malloc(sizeof(double) * 3 * nc);
  double *Dp = malloc(sizeof(double) * nc), *Lp = malloc(sizeof(double) * (ni + 1));
  double *bp = malloc(sizeof(double) * nc), *phiHbyA = malloc(sizeof(double) * nf);
  double *af = malloc(sizeof(double) * nf), *nonorth = malloc(sizeof(double) * (ni + 1));
  om_info si;
  /* 2. momentum predictor: A U* = b - V grad p^n */
  om_grad_gauss(m, bcp, 1, p, pb, gradp);
  if ((o->nonorth & 1) || o->conv == CONV_SOU) om_grad_gauss(m, bcU, 3, U, Ub, gradU);
  om_momentum_assemble(m, bcU, o->nu, o->dt, phi, U, Ub, (o->nonorth & 1) ? gradU : NULL,
                       o->conv == CONV_SOU ? gradU : NULL, o->psi, D, Lo, Up, b);
  if (o->time == TIME_CN) om_momentum_cn(m, o->dt, U, D, Lo, Up, b);
  for (int q = 0; q < 3; ++q) {
    for (int i = 0; i < nc; ++i) rhs[i] = b[q * nc + i] - m->V[i] * gradp[q * nc + i];
    int st = om_bicgstab(m, D, Lo, Up, rhs, U + (size_t)q * nc, o->tolU, o->tol_abs, o->maxitU, &si);
    info->itU[q] = si.iters;
    if (st > info->status) info->status = st;
  }
  for (int i = 0; i < nc; ++i) rAU[i] = m->V[i] / D[i];
  /* 3. pressure correctors */
  for (int corr = 0; corr < o->ncorr; ++corr) {
    om_H(m, Lo, Up, b, U, H);
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < nc; ++i) HbyA[q * nc + i] = H[q * nc + i] / D[i];
    if (o->nonorth & 2) om_grad_gauss(m, bcp, 1, p, pb, gradp);
    om_pressure_assemble(m, bcU, bcp, rAU, HbyA, Ub, pb, (o->nonorth & 2) ? gradp : NULL, p,
                         o->psi, Dp, Lp, bp, phiHbyA, af, nonorth);
    if (!has_fixed_p) Dp[o->pref_cell] += Dp[o->pref_cell];   /* p_ref = 0 */
    int st = om_pcg(m, Dp, Lp, NULL, bp, p, o->tolp, o->tol_abs, o->maxitp, &si);
    if (corr < 4) info->itp[corr] = si.iters;
    if (st > info->status) info->status = st;
    /* Rhie-Chow flux correction */
    for (int f = 0; f < nf; ++f) {
      if (f < ni) {
        phi[f] = phiHbyA[f] - af[f] * (p[m->neighbour[f]] - p[m->owner[f]]) - nonorth[f];
      } else if (bcp[patch_of_face(m, f)] == BC_FIXED) {
        phi[f] = phiHbyA[f] - af[f] * (pb[f - ni] - p[m->owner[f]]);
      } else {
        phi[f] = phiHbyA[f];
      }
    }
    /* velocity correction U = HbyA - rAU grad p */
    om_grad_gauss(m, bcp, 1, p, pb, gradp);
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < nc; ++i) U[q * nc + i] = HbyA[q * nc + i] - rAU[i] * gradp[q * nc + i];
  }
  (void)nb;
  free(bcU); free(bcp); free(gradp); free(gradU); free(D); free(Lo); free(Up); free(b);
  free(rhs); free(rAU); free(H); free(HbyA); free(Dp); free(Lp); free(bp); free(phiHbyA);
  free(af); free(nonorth);
  return info->status;
}

/* Initial face flux from a cell velocity: phi_f = U_f . S_f with linear
 * interpolation; boundary: U_b.S (fixed U), U_O.S (zero gradient), 0 (empty). */
void om_flux_from_U(const om_mesh *m, const double *U, const double *Ub, double *phi) {
  int nc = m->nc, ni = m->nint, nb = m->nf - ni;
  int *bcU = malloc(sizeof(int) * m->npatch);
  for (int q = 0; q < m->npatch; ++q) bcU[q] = bc_of_U(m->patch_type[q]);
  double *w = malloc(sizeof(double) * (ni + 1));
  double *c = malloc(sizeof(double) * (m->nf + 1));
  double *k = malloc(sizeof(double) * 3 * (ni + 1));
  om_face_coeffs(m, w, c, k);
  for (int f = 0; f < m->nf; ++f) {
    double uf[3];
    int ok = 1;
    for (int q = 0; q < 3; ++q)
      ok &= face_value(m, w, bcU, U + (size_t)q * nc, Ub ? Ub + (size_t)q * nb : NULL, f, &uf[q]);
    phi[f] = ok ? dot3(uf, m->Sf + 3 * f) : 0.0;
  }
  free(bcU); free(w); free(c); free(k);
}

/* ======================================================= adjoint of a step */
/* Reverse-mode derivative of om_piso_step (Sec. 2.5, Eq. vjp): given the
 * adjoints of the step's outputs, return those of its inputs.  Each stage of
 * the forward step above is a plain function of its inputs; its adjoint is
 * written out here stage by stage, last stage first.  The two linear solves
 * are differentiated implicitly (Eq. implicit_diff): for x = A^{-1} r,
 *   r_bar = A^{-T} x_bar,   A_bar_ij = -r_bar_i x_j,
 * with A^{-T} applied by the same Krylov method on the transposed matrix
 * (lower and upper swapped; the pressure matrix is symmetric).  The upwind
 * switch max(m, 0) and the limiter take the derivative of the branch the
 * forward step took (max(0, 0) counts as the zero branch). */

/* G^T of om_grad_gauss for one component: phib_bar may be NULL */
static void grad_gauss_T(const om_mesh *m, const double *w, const int *bc, const double *gbar,
                         double *phibar, double *phibbar) {
  int nc = m->nc;
  for (int f = 0; f < m->nf; ++f) {
    const double *S = m->Sf + 3 * f;
    int O = m->owner[f];
    double gO[3], t;
    for (int d = 0; d < 3; ++d) gO[d] = gbar[d * nc + O] / m->V[O];
    if (f < m->nint) {
      int N = m->neighbour[f];
      double gN[3];
      for (int d = 0; d < 3; ++d) gN[d] = gbar[d * nc + N] / m->V[N];
      t = dot3(gO, S) - dot3(gN, S);          /* adjoint of the face value phi_f */
      phibar[O] += w[f] * t;
      phibar[N] += (1.0 - w[f]) * t;
    } else {
      int kind = bc[patch_of_face(m, f)];
      if (kind == BC_EMPTY) continue;
      t = dot3(gO, S);
      if (kind == BC_FIXED) { if (phibbar) phibbar[f - m->nint] += t; }
      else phibar[O] += t;
    }
  }
}

/* adjoint of limit_corr(corr, orth, psi) * 1: returns d/dcorr, sets *dorth */
static double limit_corr_d(double corr, double orth, double psi, double *dorth) {
  *dorth = 0.0;
  if (psi >= 1.0) return 1.0;
  double cap = psi / (1.0 - psi) * fabs(orth);
  if (fabs(corr) > cap) {
    double sc = corr > 0.0 ? 1.0 : -1.0, so = orth > 0.0 ? 1.0 : (orth < 0.0 ? -1.0 : 0.0);
    *dorth = sc * psi / (1.0 - psi) * so;
    return 0.0;
  }
  return 1.0;
}

/* Inputs: the step's inputs U, p, phi, Ub, pb, pc exactly as om_piso_step takes
 * them (they are not modified).  In/out: Ubar[3][nc], pbar[nc], phibar[nf],
 * pbbar[nb], pcbar[n_out] hold the adjoints of the step's outputs on entry and
 * those of its inputs on return.  Accumulated: Ubbar[3][nb], *nubar and the
 * Windkessel parameter adjoints Rpbar, Cbar, Rdbar[n_out].  Returns the worst
 * status of the forward replay and the adjoint solves. */
int om_piso_step_bwd(const om_mesh *m, const om_piso_opts *o, const double *U_in,
                     const double *p_in, const double *phi_in, const double *Ub,
                     const double *pb_in, const double *pc_in, double *Ubar, double *pbar,
                     double *phibar, double *pbbar, double *pcbar, double *Ubbar, double *nubar,
                     double *Rpbar, double *Cbar, double *Rdbar) {
  const int nc = m->nc, nf = m->nf, ni = m->nint, nb = nf - ni, K = o->ncorr;
  const int nonU = (o->nonorth & 1) != 0, nonP = (o->nonorth & 2) != 0, sou = o->conv == CONV_SOU;
  int status = 0;
  int *bcU = malloc(sizeof(int) * m->npatch), *bcp = malloc(sizeof(int) * m->npatch);
  int has_fixed_p = 0;
  for (int q = 0; q < m->npatch; ++q) {
    bcU[q] = bc_of_U(m->patch_type[q]);
    bcp[q] = bc_of_p(m->patch_type[q]);
    if (bcp[q] == BC_FIXED) has_fixed_p = 1;
  }
  double *w = malloc(sizeof(double) * (ni + 1)), *c = malloc(sizeof(double) * (nf + 1));
  double *k = malloc(sizeof(double) * 3 * (ni + 1));
  om_face_coeffs(m, w, c, k);
  om_info si;

  /* ---- forward replay, keeping what the reverse sweep reads ---- */
  double *pb = malloc(sizeof(double) * (nb + 1));   /* boundary p after the Windkessel */
  memcpy(pb, pb_in, sizeof(double) * nb);
  double *Qw = calloc(o->n_out + 1, sizeof(double));
  for (int j = 0; j < o->n_out; ++j) {
    int q = o->wk_patch[j];
    double Q = 0.0, pc = pc_in[j], po;
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) Q += phi_in[f];
    om_windkessel_update(1, o->wk_scheme, o->Rp + j, o->Cw + j, o->Rd + j, &Q, o->dt, &pc, &po);
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) pb[f - ni] = po;
    Qw[j] = Q;
  }
  double *gradU = malloc(sizeof(double) * 9 * nc);
  double *D = malloc(sizeof(double) * nc), *Lo = malloc(sizeof(double) * (ni + 1));
  double *Up = malloc(sizeof(double) * (ni + 1)), *b = malloc(sizeof(double) * 3 * nc);
  double *rhs = malloc(sizeof(double) * nc), *rAU = malloc(sizeof(double) * nc);
  double *Dp = malloc(sizeof(double) * nc), *Lp = malloc(sizeof(double) * (ni + 1));
  double *bp = malloc(sizeof(double) * nc), *phiH = malloc(sizeof(double) * nf);
  double *af = malloc(sizeof(double) * nf), *nonorth = malloc(sizeof(double) * (ni + 1));
  /* Us[s] = U_s (U_0 = predicted velocity), ps[s] = p_s (p_0 = p^n), gp[s] = grad p_s,
   * HbyA[s] of corrector s */
  double *Us = malloc(sizeof(double) * 3 * nc * (K + 1)), *ps = malloc(sizeof(double) * nc * (K + 1));
  double *gp = malloc(sizeof(double) * 3 * nc * (K + 1)), *HbyA = malloc(sizeof(double) * 3 * nc * K);
  double *H = malloc(sizeof(double) * 3 * nc);
  memcpy(ps, p_in, sizeof(double) * nc);
  om_grad_gauss(m, bcp, 1, p_in, pb, gp);
  if (nonU || sou) om_grad_gauss(m, bcU, 3, U_in, Ub, gradU);
  om_momentum_assemble(m, bcU, o->nu, o->dt, phi_in, U_in, Ub, nonU ? gradU : NULL,
                       sou ? gradU : NULL, o->psi, D, Lo, Up, b);
  if (o->time == TIME_CN) om_momentum_cn(m, o->dt, U_in, D, Lo, Up, b);
  memcpy(Us, U_in, sizeof(double) * 3 * nc);
  for (int q = 0; q < 3; ++q) {
    for (int i = 0; i < nc; ++i) rhs[i] = b[q * nc + i] - m->V[i] * gp[q * nc + i];
    int st = om_bicgstab(m, D, Lo, Up, rhs, Us + (size_t)q * nc, o->tolU, o->tol_abs, o->maxitU, &si);
    if (st > status) status = st;
  }
  for (int i = 0; i < nc; ++i) rAU[i] = m->V[i] / D[i];
  for (int s = 0; s < K; ++s) {
    double *Uk = Us + (size_t)3 * nc * s, *Un = Uk + 3 * nc, *Hk = HbyA + (size_t)3 * nc * s;
    double *pk = ps + (size_t)nc * s, *pn = pk + nc;
    om_H(m, Lo, Up, b, Uk, H);
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < nc; ++i) Hk[q * nc + i] = H[q * nc + i] / D[i];
    om_pressure_assemble(m, bcU, bcp, rAU, Hk, Ub, pb, nonP ? gp + (size_t)3 * nc * s : NULL, pk,
                         o->psi, Dp, Lp, bp, phiH, af, nonorth);
    if (!has_fixed_p) Dp[o->pref_cell] += Dp[o->pref_cell];
    memcpy(pn, pk, sizeof(double) * nc);
    int st = om_pcg(m, Dp, Lp, NULL, bp, pn, o->tolp, o->tol_abs, o->maxitp, &si);
    if (st > status) status = st;
    om_grad_gauss(m, bcp, 1, pn, pb, gp + (size_t)3 * nc * (s + 1));
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < nc; ++i)
        Un[q * nc + i] = Hk[q * nc + i] - rAU[i] * gp[(size_t)3 * nc * (s + 1) + q * nc + i];
  }
  /* Dp and af are the same in every corrector (they depend on rAU only) */

  /* ---- reverse sweep ---- */
  double *Ucur = malloc(sizeof(double) * 3 * nc), *pcur = malloc(sizeof(double) * nc);
  double *phio = malloc(sizeof(double) * nf);
  memcpy(Ucur, Ubar, sizeof(double) * 3 * nc);
  memcpy(pcur, pbar, sizeof(double) * nc);
  memcpy(phio, phibar, sizeof(double) * nf);
  double *pbb = calloc(nb + 1, sizeof(double));          /* adjoint of pb after the Windkessel */
  double *Db = calloc(nc, sizeof(double)), *bb = calloc(3 * nc, sizeof(double));
  double *Lob = calloc(ni + 1, sizeof(double)), *Upb = calloc(ni + 1, sizeof(double));
  double *rAUb = calloc(nc, sizeof(double)), *HAb = malloc(sizeof(double) * 3 * nc);
  double *gnext = calloc(3 * nc, sizeof(double)), *gb = malloc(sizeof(double) * 3 * nc);
  double *lam = malloc(sizeof(double) * nc), *phiHb = malloc(sizeof(double) * nf);
  double *afb = malloc(sizeof(double) * nf), *nob = malloc(sizeof(double) * (ni + 1));
  for (int s = K - 1; s >= 0; --s) {
    const double *Uk = Us + (size_t)3 * nc * s, *Hk = HbyA + (size_t)3 * nc * s;
    const double *pk = ps + (size_t)nc * s, *pn = pk + nc;
    const double *gk = gp + (size_t)3 * nc * s, *gn = gk + 3 * nc;
    /* U_{s+1} = HbyA_s - rAU grad p_{s+1} */
    for (int i = 0; i < nc; ++i)
      for (int q = 0; q < 3; ++q) {
        HAb[q * nc + i] = Ucur[q * nc + i];
        rAUb[i] -= Ucur[q * nc + i] * gn[q * nc + i];
        gb[q * nc + i] = gnext[q * nc + i] - rAU[i] * Ucur[q * nc + i];
      }
    /* grad p_{s+1} */
    grad_gauss_T(m, w, bcp, gb, pcur, pbb);
    /* Rhie-Chow flux correction; only the last corrector's flux leaves the step */
    for (int f = 0; f < nf; ++f) { phiHb[f] = 0.0; afb[f] = 0.0; }
    for (int f = 0; f < ni; ++f) nob[f] = 0.0;
    if (s == K - 1) {
      for (int f = 0; f < nf; ++f) {
        double g = phio[f];
        int O = m->owner[f];
        phiHb[f] = g;
        if (f < ni) {
          int N = m->neighbour[f];
          afb[f] -= g * (pn[N] - pn[O]);
          nob[f] -= g;
          pcur[N] -= af[f] * g;
          pcur[O] += af[f] * g;
        } else if (bcp[patch_of_face(m, f)] == BC_FIXED) {
          afb[f] -= g * (pb[f - ni] - pn[O]);
          pbb[f - ni] -= af[f] * g;
          pcur[O] += af[f] * g;
        }
      }
    }
    /* pressure solve: lam = Dp^{-T} p_bar_{s+1} (the matrix is symmetric) */
    for (int i = 0; i < nc; ++i) lam[i] = 0.0;
    int st = om_pcg(m, Dp, Lp, NULL, pcur, lam, o->tolp, o->tol_abs, o->maxitp, &si);
    if (st > status) status = st;
    for (int i = 0; i < nc; ++i) pcur[i] = 0.0;      /* from here on: adjoint of p_s */
    /* pressure assembly: Dp (with the pinned cell doubled), Lp = -a_f, bp */
    for (int f = 0; f < nf; ++f) {
      int O = m->owner[f];
      double mO = (!has_fixed_p && O == o->pref_cell) ? 2.0 : 1.0;
      double DpbO = -lam[O] * pn[O] * mO;             /* d/d(sum of a_f) at the owner */
      if (f < ni) {
        int N = m->neighbour[f];
        double mN = (!has_fixed_p && N == o->pref_cell) ? 2.0 : 1.0;
        double DpbN = -lam[N] * pn[N] * mN;
        double Lpb = -(lam[O] * pn[N] + lam[N] * pn[O]);
        afb[f] += DpbO + DpbN - Lpb;
        double qb = lam[O] - lam[N];                  /* adjoint of -phiHbyA + nonorth */
        phiHb[f] -= qb;
        nob[f] += qb;
      } else {
        int p = patch_of_face(m, f);
        if (bcU[p] == BC_EMPTY) continue;
        phiHb[f] -= lam[O];
        if (bcp[p] == BC_FIXED) {
          afb[f] += DpbO + lam[O] * pb[f - ni];
          pbb[f - ni] += lam[O] * af[f];
        }
      }
    }
    /* face quantities phiHbyA, a_f, nonorth of om_pressure_assemble */
    for (int i = 0; i < 3 * nc; ++i) gnext[i] = 0.0;  /* collects the adjoint of grad p_s */
    for (int f = 0; f < nf; ++f) {
      const double *S = m->Sf + 3 * f;
      int O = m->owner[f];
      if (f < ni) {
        int N = m->neighbour[f];
        for (int d = 0; d < 3; ++d) {
          HAb[d * nc + O] += w[f] * phiHb[f] * S[d];
          HAb[d * nc + N] += (1.0 - w[f]) * phiHb[f] * S[d];
        }
        double rf = w[f] * rAU[O] + (1.0 - w[f]) * rAU[N];
        double rfb = afb[f] * c[f];
        if (nonP) {
          double gf[3];
          for (int d = 0; d < 3; ++d) gf[d] = w[f] * gk[d * nc + O] + (1.0 - w[f]) * gk[d * nc + N];
          double corr = dot3(gf, k + 3 * f), orth = c[f] * (pk[N] - pk[O]), dorth;
          rfb += nob[f] * limit_corr(corr, orth, o->psi);
          double dcorr = limit_corr_d(corr, orth, o->psi, &dorth);
          double lb = nob[f] * rf;
          for (int d = 0; d < 3; ++d) {
            gnext[d * nc + O] += w[f] * lb * dcorr * k[3 * f + d];
            gnext[d * nc + N] += (1.0 - w[f]) * lb * dcorr * k[3 * f + d];
          }
          pcur[N] += lb * dorth * c[f];
          pcur[O] -= lb * dorth * c[f];
        }
        rAUb[O] += w[f] * rfb;
        rAUb[N] += (1.0 - w[f]) * rfb;
      } else {
        int p = patch_of_face(m, f), bf = f - ni;
        if (bcU[p] == BC_EMPTY) continue;
        if (bcU[p] == BC_FIXED) {
          for (int d = 0; d < 3; ++d) Ubbar[d * nb + bf] += phiHb[f] * S[d];
        } else {
          for (int d = 0; d < 3; ++d) HAb[d * nc + O] += phiHb[f] * S[d];
        }
        if (bcp[p] == BC_FIXED) rAUb[O] += afb[f] * c[f];
      }
    }
    /* HbyA_s = H(U_s)/D,  H = b - offdiag U_s */
    for (int i = 0; i < 3 * nc; ++i) Ucur[i] = 0.0;      /* from here on: adjoint of U_s */
    for (int q = 0; q < 3; ++q)
      for (int i = 0; i < nc; ++i) {
        double hb = HAb[q * nc + i] / D[i];
        Db[i] -= hb * Hk[q * nc + i];
        bb[q * nc + i] += hb;
        HAb[q * nc + i] = hb;                            /* now the adjoint of H */
      }
    for (int f = 0; f < ni; ++f) {
      int O = m->owner[f], N = m->neighbour[f];
      for (int q = 0; q < 3; ++q) {
        Ucur[q * nc + N] -= Up[f] * HAb[q * nc + O];
        Ucur[q * nc + O] -= Lo[f] * HAb[q * nc + N];
        Upb[f] -= HAb[q * nc + O] * Uk[q * nc + N];
        Lob[f] -= HAb[q * nc + N] * Uk[q * nc + O];
      }
    }
  }
  /* rAU = V/D */
  for (int i = 0; i < nc; ++i) Db[i] -= rAUb[i] * m->V[i] / (D[i] * D[i]);
  /* momentum predictor: U_0 = A^{-1}(b - V grad p^n), solved per component on A^T */
  const double *U0 = Us;
  for (int q = 0; q < 3; ++q) {
    double *lq = gb + (size_t)q * nc;                     /* gb reused for lambda_U */
    for (int i = 0; i < nc; ++i) lq[i] = 0.0;
    int st = om_bicgstab(m, D, Up, Lo, Ucur + (size_t)q * nc, lq, o->tolU, o->tol_abs, o->maxitU, &si);
    if (st > status) status = st;
  }
  for (int q = 0; q < 3; ++q) {
    const double *lq = gb + (size_t)q * nc, *u = U0 + (size_t)q * nc;
    for (int i = 0; i < nc; ++i) {
      Db[i] -= lq[i] * u[i];
      bb[q * nc + i] += lq[i];
      gnext[q * nc + i] -= m->V[i] * lq[i];               /* adjoint of grad p^n */
    }
    for (int f = 0; f < ni; ++f) {
      int O = m->owner[f], N = m->neighbour[f];
      Lob[f] -= lq[N] * u[O];
      Upb[f] -= lq[O] * u[N];
    }
  }
  /* grad p^n (predictor, and the corrector-0 non-orthogonal term) */
  grad_gauss_T(m, w, bcp, gnext, pcur, pbb);
  /* momentum assembly */
  double *Un_b = malloc(sizeof(double) * 3 * nc), *phin_b = calloc(nf, sizeof(double));
  double *gUb = calloc(9 * nc, sizeof(double));
  double nub = 0.0;
  for (int q = 0; q < 3; ++q)
    for (int i = 0; i < nc; ++i) Un_b[q * nc + i] = m->V[i] / o->dt * bb[q * nc + i];
  if (o->time == TIME_CN) {
    /* Crank-Nicolson transform backwards: D, Lo, Up hold the halved rows; the
     * backward-Euler coefficients are twice their off-time parts */
    for (int i = 0; i < nc; ++i) {
      double Dcd = 2.0 * (D[i] - m->V[i] / o->dt), s = 0.0;
      for (int q = 0; q < 3; ++q) {
        s += bb[q * nc + i] * U_in[q * nc + i];
        Un_b[q * nc + i] -= 0.5 * Dcd * bb[q * nc + i];
      }
      Db[i] = 0.5 * Db[i] - 0.5 * s;
    }
    for (int f = 0; f < ni; ++f) {
      int O = m->owner[f], N = m->neighbour[f];
      double sl = 0.0, su = 0.0;
      for (int q = 0; q < 3; ++q) {
        sl += bb[q * nc + N] * U_in[q * nc + O];
        su += bb[q * nc + O] * U_in[q * nc + N];
        Un_b[q * nc + O] -= 0.5 * (2.0 * Lo[f]) * bb[q * nc + N];
        Un_b[q * nc + N] -= 0.5 * (2.0 * Up[f]) * bb[q * nc + O];
      }
      Lob[f] = 0.5 * Lob[f] - 0.5 * sl;
      Upb[f] = 0.5 * Upb[f] - 0.5 * su;
    }
  }
  for (int f = 0; f < nf; ++f) {
    int O = m->owner[f];
    double mm = phi_in[f];
    if (f < ni) {
      int N = m->neighbour[f];
      double hp = mm > 0.0 ? 1.0 : 0.0, hn = mm < 0.0 ? 1.0 : 0.0;
      phin_b[f] += Db[O] * hp - Db[N] * hn + Upb[f] * hn - Lob[f] * hp;
      nub += c[f] * (Db[O] + Db[N] - Upb[f] - Lob[f]);
      if (nonU) {
        for (int q = 0; q < 3; ++q) {
          const double *g = gradU + (size_t)q * 3 * nc;
          double gf[3];
          for (int d = 0; d < 3; ++d) gf[d] = w[f] * g[d * nc + O] + (1.0 - w[f]) * g[d * nc + N];
          double corr = dot3(gf, k + 3 * f);
          double orth = c[f] * (U_in[q * nc + N] - U_in[q * nc + O]), dorth;
          double cb = bb[q * nc + O] - bb[q * nc + N];
          nub += cb * limit_corr(corr, orth, o->psi);
          double dcorr = limit_corr_d(corr, orth, o->psi, &dorth);
          double lb = o->nu * cb;
          double *gq = gUb + (size_t)q * 3 * nc;
          for (int d = 0; d < 3; ++d) {
            gq[d * nc + O] += w[f] * lb * dcorr * k[3 * f + d];
            gq[d * nc + N] += (1.0 - w[f]) * lb * dcorr * k[3 * f + d];
          }
          Un_b[q * nc + N] += lb * dorth * c[f];
          Un_b[q * nc + O] -= lb * dorth * c[f];
        }
      }
      if (sou) {   /* t_f = m (gradU)_C . d_Cf enters b_O with -1, b_N with +1 */
        int Cu = mm >= 0.0 ? O : N;
        double dC[3];
        for (int a = 0; a < 3; ++a) dC[a] = m->Cf[3 * f + a] - m->C[3 * Cu + a];
        for (int q = 0; q < 3; ++q) {
          const double *g = gradU + (size_t)q * 3 * nc;
          double gC[3] = {g[Cu], g[nc + Cu], g[2 * nc + Cu]};
          double tb = bb[q * nc + N] - bb[q * nc + O];
          phin_b[f] += tb * dot3(gC, dC);
          double *gq = gUb + (size_t)q * 3 * nc;
          for (int d = 0; d < 3; ++d) gq[d * nc + Cu] += tb * mm * dC[d];
        }
      }
    } else {
      int kind = bcU[patch_of_face(m, f)], bf = f - ni;
      if (kind == BC_FIXED) {
        double a = o->nu * c[f], s = 0.0;
        for (int q = 0; q < 3; ++q) {
          s += bb[q * nc + O] * Ub[q * nb + bf];
          Ubbar[q * nb + bf] += (a - mm) * bb[q * nc + O];
        }
        nub += c[f] * (Db[O] + s);
        phin_b[f] -= s;
      } else if (kind == BC_ZEROGRAD) {
        phin_b[f] += Db[O];
      }
    }
  }
  if (nonU || sou)
    for (int q = 0; q < 3; ++q)
      grad_gauss_T(m, w, bcU, gUb + (size_t)q * 3 * nc, Un_b + (size_t)q * nc, Ubbar + (size_t)q * nb);
  /* Windkessel: pb on an outlet patch is p_o, both inside the step and in its output */
  for (int bf = 0; bf < nb; ++bf) pbb[bf] += pbbar[bf];
  for (int j = 0; j < o->n_out; ++j) {
    int q = o->wk_patch[j];
    double pob = 0.0;
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) {
      pob += pbb[f - ni];
      pbb[f - ni] = 0.0;
    }
    double Rp = o->Rp[j], Cw = o->Cw[j], Rd = o->Rd[j], Q = Qw[j], p0 = pc_in[j], dt = o->dt;
    double dp0, dQ, dRd, dC;    /* partial derivatives of the new p_c */
    if (o->wk_scheme == WK_EXACT) {
      double e = exp(-dt / (Rd * Cw));
      double de_dRd = e * dt / (Rd * Rd * Cw), de_dC = e * dt / (Rd * Cw * Cw);
      dp0 = e;
      dQ = Rd * (1.0 - e);
      dRd = Q * (1.0 - e) + (p0 - Rd * Q) * de_dRd;
      dC = (p0 - Rd * Q) * de_dC;
    } else if (o->wk_scheme == WK_FE) {
      dp0 = 1.0 - dt / (Rd * Cw);
      dQ = dt / Cw;
      dRd = dt * p0 / (Cw * Rd * Rd);
      dC = -dt * (Q - p0 / Rd) / (Cw * Cw);
    } else {
      double den = 1.0 + dt / (Rd * Cw), num = p0 + dt * Q / Cw;
      dp0 = 1.0 / den;
      dQ = dt / (Cw * den);
      dRd = num / (den * den) * dt / (Rd * Rd * Cw);
      dC = -dt * Q / (Cw * Cw * den) + num / (den * den) * dt / (Rd * Cw * Cw);
    }
    double G = pcbar[j] + pob;                       /* adjoint of the new p_c */
    double Qb = G * dQ + pob * Rp;
    Rpbar[j] += pob * Q;
    Cbar[j] += G * dC;
    Rdbar[j] += G * dRd;
    pcbar[j] = G * dp0;
    for (int f = m->patch_start[q]; f < m->patch_start[q] + m->patch_size[q]; ++f) phin_b[f] += Qb;
  }
  memcpy(Ubar, Un_b, sizeof(double) * 3 * nc);
  memcpy(pbar, pcur, sizeof(double) * nc);
  memcpy(phibar, phin_b, sizeof(double) * nf);
  memcpy(pbbar, pbb, sizeof(double) * nb);
  *nubar += nub;
  free(bcU); free(bcp); free(w); free(c); free(k); free(pb); free(Qw); free(gradU); free(D);
  free(Lo); free(Up); free(b); free(rhs); free(rAU); free(Dp); free(Lp); free(bp); free(phiH);
  free(af); free(nonorth); free(Us); free(ps); free(gp); free(HbyA); free(H); free(Ucur);
  free(pcur); free(phio); free(pbb); free(Db); free(bb); free(Lob); free(Upb); free(rAUb);
  free(HAb); free(gnext); free(gb); free(lam); free(phiHb); free(afb); free(nob); free(Un_b);
  free(phin_b); free(gUb);
  return status;
}
