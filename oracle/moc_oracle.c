/*
 * Plain FP64 CPU oracle for the planar flat-source Method of Characteristics (MOC) on 2D
 * triangle meshes.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference the CUDA library is checked
 * against. Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may
 * build, load or call it. It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (each step cites the paper's section / equation):
 *  - modular (cyclic) rays over the bounding box of the whole domain (Sec. 3.1, the modular ray
 *    approach applied to the domain's bounding box rather than to pins or assemblies);
 *  - ray-mesh intersection: per-ray segment lengths and element ids, computed once (Sec. 3.1).
 *    Here every (ray, triangle) pair whose projections overlap is clipped exactly
 *    (Cyrus-Beck half-plane clipping), and the pieces are sorted along the ray. This is a
 *    deliberately different algorithm from the half-edge walk the library uses;
 *  - the multigroup source of the element-wise equation (Eq. MGNTE / MGNTE_element, isotropic
 *    scattering, L = 0): q = [sum_g' Sigma_s,g'->g phi_g' + chi_g/k sum_g' nuSigma_f,g' phi_g' + S_g]/(4 pi);
 *  - the flat-source characteristic solution along each segment (Eq. MOC_sol):
 *    psi_out = psi_in e^{-tau} + (q/Sigma_t)(1 - e^{-tau}), tau = Sigma_t * l / sin(theta_p);
 *  - the scalar flux by angular integration over all discrete directions (Sec. 2.1, text after
 *    Eq. MOC_sol): phi = 4 pi q/Sigma_t + sum_k W_k (psi_in - psi_out)_k / (Sigma_t A_i);
 *  - k-eigenvalue power iteration (the fine-mesh MOC solve of Alg. 1, without its HFEM step; the
 *    CMFD step optional), one transport sweep per outer, Jacobi in energy and in boundary flux.
 *  - DGMOC (Sec. 2.2, Alg. 2): the planar tracks extruded through axial planes, a linear
 *    discontinuous-Galerkin expansion in z on every characteristic (see the DGMOC block below).
 *
 * Readings where the paper is silent (all also listed in the design notes):
 *  - A azimuths cover [0, 2 pi); for the first quadrant phi_a = 2 pi (a + 1/2)/A,
 *    nx = floor(W sin(phi_a)/delta) + 1, ny = floor(H cos(phi_a)/delta) + 1, corrected angle
 *    atan(H nx/(W ny)), effective spacing (W/nx) sin(corrected angle); the other quadrants mirror it.
 *    Ray starts sit at (i + 1/2) W/nx on the bottom edge and (j + 1/2) H/ny on the side edge.
 *  - azimuthal weight of direction a: (phi_{a+1} - phi_{a-1})/(4 pi) over the sorted 2 pi set.
 *  - direction weight W_{a,p} = 4 pi omega_a w_p delta_a sin(theta_p); polar weights cover one
 *    hemisphere (2D symmetry psi(theta) = psi(pi - theta)).
 *  - region area: the tracked area A_i = sum over the 2 pi set of omega_a delta_a (sum of l in i).
 *  - pieces shorter than 1e-12 cm are dropped; a gap longer than 1e-9 cm along a ray (outside a
 *    non-rectangular mesh) splits the ray into separate tracks with vacuum ends.
 *  - reflective ends link to the ray end that starts at the same wall point with the mirrored
 *    direction; vacuum ends have zero incoming flux.
 *  - convergence: |k' - k| <= tol_k and max_i |f'_i - f_i|/f'_i <= tol_f over regions with
 *    f'_i > 0, f_i = sum_g nuSigma_f,g phi_i,g, flux normalised to sum_i A_i f_i = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
  /* mesh */
  int n_vert, n_tri;
  double *xy;      /* [V][2] */
  int32_t *tri;    /* [R][3] */
  int32_t *mat;    /* [R] */
  double xmin, xmax, ymin, ymax;
  int bc[4];       /* x-, x+, y-, y+ ; 0 vacuum 1 reflective */
  /* quadrature */
  int n_azim;      /* over 2 pi */
  int n_dir;       /* n_azim/2 directions in [0, pi) */
  double *phi_a, *delta_a, *omega_a;  /* [n_dir] */
  int *nx_a, *ny_a;                    /* [n_dir] */
  int layout;                          /* 0 cyclic modular rays over the box, 1 back projection */
  int n_polar;
  double *sin_theta, *polar_w;        /* [P] */
  /* tracks */
  int64_t n_tracks, n_seg;
  int32_t *track_dir;  /* [T] direction index */
  double *track_xy;    /* [T][4] start x,y end x,y */
  int64_t *seg_off;    /* [T+1] */
  int32_t *seg_reg;    /* [S] */
  double *seg_len;     /* [S] */
  int64_t *link;       /* [T][2]: end (t,d) feeds incoming (t',d') encoded 2t'+d', -1 vacuum */
  double *area;        /* [R] tracked area */
  /* cross sections */
  int n_mat, G;
  double *st, *nsf, *chi, *ss;   /* [M][G], [M][G], [M][G], [M][G][G] */
  double *ext;                    /* [R][G] fixed volumetric source or NULL */
  /* state */
  double *phi;      /* [R][G] */
  double *q;        /* [R][G] source per steradian */
  double *tally;    /* [R][G] */
  double *psi_in;   /* [T][2][P][G] incoming angular flux */
  double *psi_next; /* [T][2][P][G] */
  double *leak;     /* [G] outgoing W*psi at vacuum ends during the last sweep */
  double k;
  int n_threads;
  /* anisotropic scattering of order L (Legendre expansion of the scattering kernel, Sec. 2):
   * per-direction sources from the region-average angular flux of the previous outer */
  int L;              /* 0: isotropic */
  int ND;             /* directions m = (j * 2 + sense) * P + p, j over [0, pi) */
  double *ssl;        /* [L][M][G][G] Sigma_s,l g' -> g for l = 1..L */
  double *kern;       /* [L][ND][ND] 4 pi omega' w' (P_l(Om . Om'+) + P_l(Om . Om'-)) / 2 */
  double *qdir;       /* [R][ND][G] source per steradian per direction */
  double *tdir;       /* [R][ND][G] per-direction tally: sum of delta sin(theta) (psi_in - psi_out) */
  double *pbar;       /* [R][ND][G] region-average angular flux (state of the anisotropic source) */
  /* coarse-mesh finite difference acceleration (Alg. 1), partial-current form */
  int cmfd, n_cells, n_if, cm_outer, cm_inner, n_colors;
  double cm_omega;    /* over-relaxation factor of the coarse sweeps */
  int32_t *cell;      /* [R] */
  int32_t *color;     /* [n_cells] greedy colouring: no two cells of one interface share a colour */
  int32_t *nb_off, *nb_cell, *nb_in;  /* per cell, its neighbours in interface order and the
                                         slot of the current from each neighbour into it */
  uint64_t *pairs;    /* [n_if] sorted (min cell << 32 | max cell) */
  double *cur;        /* [2 n_if][G]: slot 2e a->b (a the lower id), 2e+1 b->a */
  double *cleak;      /* [n_cells][G] net current out of the domain boundary: out at every track end
                         (vacuum or reflective) minus in at every track start */
  /* DGMOC: the planar tracks extruded through nz axial planes (0: the planar 2D method) */
  int nz;
  int bcz[2];         /* bottom, top: 0 vacuum 1 reflective */
  double *dz;         /* [nz] plane heights */
  int32_t *mat3;      /* [nz][R] material of each region in each plane */
  double *phi3;       /* [nz][R][2][G] scalar flux moments: plane average, linear (xi) coefficient */
  double *q3;         /* [nz][R][2][G] source moments per steradian */
  double *tal3;       /* [nz][R][2][G] sum over segments of W * (segment integral of the moments) */
  double *psi3_in, *psi3_next;  /* [T][2 sense][2 down/up][nz][P][2][G] radial boundary flux moments */
  double *ztop;       /* [S][2 sense][P][G] upward top-face trace of the last sweep (reflective top) */
  double *leak3;      /* [3][G] leakage of the last sweep: radial, bottom, top */
  /* axial coarse-mesh acceleration of DGMOC: coarse cells = planes */
  int dgcm, dgcm_outer, dgcm_inner;
  double dgcm_omega;
  double *jz;         /* [2][nz-1][G]: partial currents up (plane z -> z+1) and down (z+1 -> z) */
  double *zleak;      /* [nz][G]: net current out of each plane through the domain boundary
                         (radial track ends, bottom and top faces): out minus in */
  char err[256];
} orc_t;

static void *xcalloc(size_t n, size_t sz) {
  void *p = calloc(n ? n : 1, sz);
  if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
  return p;
}

const char *orc_error(orc_t *h) { return h->err; }

void orc_destroy(orc_t *h) {
  if (!h) return;
  free(h->xy); free(h->tri); free(h->mat);
  free(h->phi_a); free(h->delta_a); free(h->omega_a); free(h->nx_a); free(h->ny_a);
  free(h->sin_theta); free(h->polar_w);
  free(h->track_dir); free(h->track_xy); free(h->seg_off); free(h->seg_reg); free(h->seg_len);
  free(h->link); free(h->area);
  free(h->st); free(h->nsf); free(h->chi); free(h->ss); free(h->ext);
  free(h->phi); free(h->q); free(h->tally); free(h->psi_in); free(h->psi_next); free(h->leak);
  free(h->cell); free(h->pairs); free(h->cur); free(h->cleak); free(h->color);
  free(h->nb_off); free(h->nb_cell); free(h->nb_in);
  free(h->ssl); free(h->kern); free(h->qdir); free(h->tdir); free(h->pbar);
  free(h->dz); free(h->mat3); free(h->phi3); free(h->q3); free(h->tal3); free(h->psi3_in); free(h->psi3_next);
  free(h->ztop); free(h->leak3); free(h->jz); free(h->zleak);
  free(h);
}

/* ---------------------------------------------------------------- quadrature ---- */
/* smallest and largest of v . x over the mesh vertices */
static void vertex_extent(const orc_t *h, double vx, double vy, double *lo, double *hi) {
  *lo = INFINITY; *hi = -INFINITY;
  for (int k = 0; k < h->n_vert; ++k) {
    double c = vx * h->xy[2 * k] + vy * h->xy[2 * k + 1];
    if (c < *lo) *lo = c;
    if (c > *hi) *hi = c;
  }
}

static int build_quadrature(orc_t *h, double spacing) {
  int A = h->n_azim, nq = A / 4;
  double W = h->xmax - h->xmin, H = h->ymax - h->ymin;
  h->n_dir = A / 2;
  h->phi_a = xcalloc(h->n_dir, sizeof(double));
  h->delta_a = xcalloc(h->n_dir, sizeof(double));
  h->omega_a = xcalloc(h->n_dir, sizeof(double));
  h->nx_a = xcalloc(h->n_dir, sizeof(int));
  h->ny_a = xcalloc(h->n_dir, sizeof(int));
  if (h->layout == 1) {
    /* back projection: nominal angles; per direction ceil(extent / spacing) rays spread evenly
     * over the projection of the mesh on the normal (stored as nx, with ny = 0) */
    for (int j = 0; j < h->n_dir; ++j) {
      double phi = 2.0 * ORC_PI * (j + 0.5) / A, lo, hi;
      vertex_extent(h, -sin(phi), cos(phi), &lo, &hi);
      int n = (int)ceil((hi - lo) / spacing);
      if (n < 1) n = 1;
      h->phi_a[j] = phi;
      h->delta_a[j] = (hi - lo > 0.0) ? (hi - lo) / n : spacing;
      h->nx_a[j] = n; h->ny_a[j] = 0;
    }
    nq = 0;
  }
  for (int a = 0; a < nq; ++a) {
    double phi = 2.0 * ORC_PI * (a + 0.5) / A;
    int nx = (int)floor(W * sin(phi) / spacing) + 1;
    int ny = (int)floor(H * cos(phi) / spacing) + 1;
    double pc = atan((H * nx) / (W * ny));
    double d = (W / nx) * sin(pc);
    /* first quadrant direction a, second quadrant mirror at index n_dir-1-a */
    h->phi_a[a] = pc; h->delta_a[a] = d; h->nx_a[a] = nx; h->ny_a[a] = ny;
    int b = h->n_dir - 1 - a;
    h->phi_a[b] = ORC_PI - pc; h->delta_a[b] = d; h->nx_a[b] = nx; h->ny_a[b] = ny;
  }
  /* full sorted set over [0, 2 pi): directions j and j + pi */
  double *full = xcalloc(A, sizeof(double));
  for (int j = 0; j < h->n_dir; ++j) { full[j] = h->phi_a[j]; full[j + h->n_dir] = h->phi_a[j] + ORC_PI; }
  for (int j = 1; j < A; ++j)
    if (!(full[j] > full[j - 1])) { snprintf(h->err, sizeof h->err, "azimuthal angles not increasing"); free(full); return -1; }
  for (int j = 0; j < h->n_dir; ++j) {
    double lo = (j == 0) ? full[A - 1] - 2.0 * ORC_PI : full[j - 1];
    double hi = full[j + 1];
    h->omega_a[j] = (hi - lo) / (4.0 * ORC_PI);
  }
  free(full);
  return 0;
}

/* ---------------------------------------------------------------- tracks ---- */
typedef struct { double s0, s1; int32_t tri; } piece_t;

static int cmp_piece(const void *a, const void *b) {
  const piece_t *x = a, *y = b;
  if (x->s0 < y->s0) return -1;
  if (x->s0 > y->s0) return 1;
  return (x->tri < y->tri) ? -1 : (x->tri > y->tri);
}

typedef struct { double c; int idx; } offs_t;
static int cmp_offs(const void *a, const void *b) {
  const offs_t *x = a, *y = b;
  return (x->c < y->c) ? -1 : (x->c > y->c);
}

/* Clip the line p0 + s u, s in [0, L], against CCW triangle t. Returns 1 and the interval if
 * the intersection has positive length. Each edge's side test is evaluated from its lower-id
 * vertex (and negated for the other orientation), so the two triangles of an edge see exactly
 * opposite values and a line along a shared edge belongs to exactly one of them. */
static int clip_triangle(const double *xy, const int32_t *tri, int t, const double *p0, const double *u, double L,
                         double *s_in, double *s_out) {
  double lo = 0.0, hi = L;
  for (int e = 0; e < 3; ++e) {
    int ia = tri[3 * t + e], ib = tri[3 * t + (e + 1) % 3], fwd = ia < ib;
    const double *a = xy + 2 * (int64_t)(fwd ? ia : ib), *b = xy + 2 * (int64_t)(fwd ? ib : ia);
    double sg = fwd ? 1.0 : -1.0;
    double nx = -(b[1] - a[1]), ny = b[0] - a[0];           /* inward normal of the CCW edge, */
    double f0 = nx * (p0[0] - a[0]) + ny * (p0[1] - a[1]);  /* up to the orientation sign sg */
    double fu = nx * u[0] + ny * u[1];
    nx *= sg; ny *= sg; f0 *= sg; fu *= sg;
    if (fu == 0.0) {
      /* ray parallel to this edge: outside if on the outer side; a ray running exactly along
       * the edge belongs to the triangle on its left only */
      if (f0 < 0.0) return 0;
      if (f0 == 0.0 && (nx * (-u[1]) + ny * u[0]) <= 0.0) return 0;
      continue;
    }
    double s = -f0 / fu;
    if (fu > 0.0) { if (s > lo) lo = s; } else { if (s < hi) hi = s; }
  }
  if (hi - lo <= 0.0) return 0;
  *s_in = lo; *s_out = hi;
  return 1;
}

/* exit parameter of the ray p0 + s u from the box */
static double box_exit(const orc_t *h, const double *p0, const double *u) {
  double s = INFINITY;
  if (u[0] > 0) s = fmin(s, (h->xmax - p0[0]) / u[0]);
  if (u[0] < 0) s = fmin(s, (h->xmin - p0[0]) / u[0]);
  if (u[1] > 0) s = fmin(s, (h->ymax - p0[1]) / u[1]);
  if (u[1] < 0) s = fmin(s, (h->ymin - p0[1]) / u[1]);
  return s;
}

/* wall id of a boundary point: 0 x-, 1 x+, 2 y-, 3 y+ ; -1 if interior */
static int wall_of(const orc_t *h, double x, double y, double tol) {
  if (fabs(x - h->xmin) <= tol) return 0;
  if (fabs(x - h->xmax) <= tol) return 1;
  if (fabs(y - h->ymin) <= tol) return 2;
  if (fabs(y - h->ymax) <= tol) return 3;
  return -1;
}

typedef struct { int key; double c; int64_t e; } inc_t;
static int cmp_inc(const void *a, const void *b) {
  const inc_t *x = a, *y = b;
  if (x->key != y->key) return (x->key < y->key) ? -1 : 1;
  if (x->c != y->c) return (x->c < y->c) ? -1 : 1;
  return (x->e < y->e) ? -1 : (x->e > y->e);
}

static int build_tracks(orc_t *h) {
  double W = h->xmax - h->xmin, H = h->ymax - h->ymin;
  const double sliver = 1e-12, gap = 1e-9;
  /* 1. rays over the bounding box, per direction */
  int64_t n_rays = 0;
  for (int j = 0; j < h->n_dir; ++j) n_rays += h->nx_a[j] + h->ny_a[j];
  double *ray = xcalloc(n_rays * 5, sizeof(double));   /* x0 y0 ux uy L */
  int32_t *ray_dir = xcalloc(n_rays, sizeof(int32_t));
  int64_t r = 0;
  for (int j = 0; j < h->n_dir; ++j) {
    double ph = h->phi_a[j], u[2] = {cos(ph), sin(ph)};
    int nx = h->nx_a[j], ny = h->ny_a[j];
    if (h->layout == 1) {
      /* ray i: the line nrm . x = lo + (i + 1/2) delta, over the bounding box's extent along u */
      double nrm[2] = {-sin(ph), cos(ph)}, lo, hi, corner[4][2] = {{h->xmin, h->ymin}, {h->xmax, h->ymin},
                                                                     {h->xmin, h->ymax}, {h->xmax, h->ymax}};
      vertex_extent(h, nrm[0], nrm[1], &lo, &hi);
      double t0 = INFINITY, t1 = -INFINITY;
      for (int k = 0; k < 4; ++k) {
        double t = u[0] * corner[k][0] + u[1] * corner[k][1];
        if (t < t0) t0 = t;
        if (t > t1) t1 = t;
      }
      for (int i = 0; i < nx; ++i) {
        double c = lo + (i + 0.5) * h->delta_a[j];
        ray[5 * r] = c * nrm[0] + t0 * u[0]; ray[5 * r + 1] = c * nrm[1] + t0 * u[1];
        ray[5 * r + 2] = u[0]; ray[5 * r + 3] = u[1]; ray[5 * r + 4] = t1 - t0; ray_dir[r] = j; ++r;
      }
      continue;
    }
    for (int i = 0; i < nx; ++i) {        /* bottom edge starts */
      double p0[2] = {h->xmin + (i + 0.5) * W / nx, h->ymin};
      ray[5 * r] = p0[0]; ray[5 * r + 1] = p0[1]; ray[5 * r + 2] = u[0]; ray[5 * r + 3] = u[1];
      ray[5 * r + 4] = box_exit(h, p0, u); ray_dir[r] = j; ++r;
    }
    for (int i = 0; i < ny; ++i) {        /* side edge starts: left for ux>0, right for ux<0 */
      double p0[2] = {(u[0] > 0) ? h->xmin : h->xmax, h->ymin + (i + 0.5) * H / ny};
      ray[5 * r] = p0[0]; ray[5 * r + 1] = p0[1]; ray[5 * r + 2] = u[0]; ray[5 * r + 3] = u[1];
      ray[5 * r + 4] = box_exit(h, p0, u); ray_dir[r] = j; ++r;
    }
  }
  /* 2. clip every (ray, triangle) pair whose projections on the ray normal overlap */
  int64_t *cnt = xcalloc(n_rays, sizeof(int64_t));
  int64_t *cap = xcalloc(n_rays, sizeof(int64_t));
  piece_t **pcs = xcalloc(n_rays, sizeof(piece_t *));
  int64_t r0 = 0;
  for (int j = 0; j < h->n_dir; ++j) {
    int nr = h->nx_a[j] + h->ny_a[j];
    double ph = h->phi_a[j], nrm[2] = {-sin(ph), cos(ph)};
    offs_t *off = xcalloc(nr, sizeof(offs_t));
    for (int i = 0; i < nr; ++i) {
      off[i].c = nrm[0] * ray[5 * (r0 + i)] + nrm[1] * ray[5 * (r0 + i) + 1];
      off[i].idx = i;
    }
    qsort(off, nr, sizeof(offs_t), cmp_offs);
    for (int t = 0; t < h->n_tri; ++t) {
      const double *v[3];
      double cmin = INFINITY, cmax = -INFINITY;
      for (int k = 0; k < 3; ++k) {
        v[k] = h->xy + 2 * (int64_t)h->tri[3 * t + k];
        double c = nrm[0] * v[k][0] + nrm[1] * v[k][1];
        if (c < cmin) cmin = c;
        if (c > cmax) cmax = c;
      }
      /* widened by a rounding margin: a ray along an edge of the triangle is a candidate even
       * when the projections round to just outside it; the clip decides */
      cmin -= 1e-9 * fmax(W, H);
      cmax += 1e-9 * fmax(W, H);
      /* first ray with offset >= cmin */
      int lo = 0, hi = nr;
      while (lo < hi) { int m = (lo + hi) / 2; if (off[m].c < cmin) lo = m + 1; else hi = m; }
      for (int q = lo; q < nr && off[q].c <= cmax; ++q) {
        int64_t rr = r0 + off[q].idx;
        double s0, s1;
        if (!clip_triangle(h->xy, h->tri, t, ray + 5 * rr, ray + 5 * rr + 2, ray[5 * rr + 4], &s0, &s1)) continue;
        if (s1 - s0 < sliver) continue;
        if (cnt[rr] == cap[rr]) {
          cap[rr] = cap[rr] ? 2 * cap[rr] : 16;
          pcs[rr] = realloc(pcs[rr], cap[rr] * sizeof(piece_t));
          if (!pcs[rr]) abort();
        }
        pcs[rr][cnt[rr]].s0 = s0; pcs[rr][cnt[rr]].s1 = s1; pcs[rr][cnt[rr]].tri = t;
        cnt[rr]++;
      }
    }
    free(off);
    r0 += nr;
  }
  /* 3. sort pieces along each ray; split at gaps into tracks */
  int64_t n_tr = 0, n_sg = 0;
  for (int64_t q = 0; q < n_rays; ++q) {
    if (!cnt[q]) continue;
    qsort(pcs[q], cnt[q], sizeof(piece_t), cmp_piece);
    n_tr++;
    for (int64_t k = 1; k < cnt[q]; ++k)
      if (pcs[q][k].s0 - pcs[q][k - 1].s1 > gap) n_tr++;
    n_sg += cnt[q];
  }
  h->n_tracks = n_tr; h->n_seg = n_sg;
  h->track_dir = xcalloc(n_tr, sizeof(int32_t));
  h->track_xy = xcalloc(4 * n_tr, sizeof(double));
  h->seg_off = xcalloc(n_tr + 1, sizeof(int64_t));
  h->seg_reg = xcalloc(n_sg, sizeof(int32_t));
  h->seg_len = xcalloc(n_sg, sizeof(double));
  int64_t t = 0, s = 0;
  for (int64_t q = 0; q < n_rays; ++q) {
    if (!cnt[q]) continue;
    const double *p0 = ray + 5 * q, *u = ray + 5 * q + 2;
    int64_t k = 0;
    while (k < cnt[q]) {
      int64_t k1 = k + 1;
      while (k1 < cnt[q] && pcs[q][k1].s0 - pcs[q][k1 - 1].s1 <= gap) k1++;
      h->track_dir[t] = ray_dir[q];
      h->seg_off[t] = s;
      double sa = pcs[q][k].s0, sb = pcs[q][k1 - 1].s1;
      h->track_xy[4 * t] = p0[0] + sa * u[0]; h->track_xy[4 * t + 1] = p0[1] + sa * u[1];
      h->track_xy[4 * t + 2] = p0[0] + sb * u[0]; h->track_xy[4 * t + 3] = p0[1] + sb * u[1];
      for (int64_t m = k; m < k1; ++m) {
        h->seg_reg[s] = pcs[q][m].tri;
        h->seg_len[s] = pcs[q][m].s1 - pcs[q][m].s0;
        s++;
      }
      t++;
      k = k1;
    }
    free(pcs[q]);
  }
  h->seg_off[t] = s;
  free(pcs); free(cnt); free(cap); free(ray); free(ray_dir);

  /* 4. links: each outgoing end (t,d) -> the incoming end starting at the same wall point with
   *    the mirrored direction, if that wall is reflective */
  double tol = 1e-9 * fmax(W, H);
  h->link = xcalloc(2 * h->n_tracks, sizeof(int64_t));
  /* index incoming ends by (direction-in-2pi, wall, coordinate along the wall), sorted */
  int64_t ne = 2 * h->n_tracks;
  inc_t *inc = xcalloc(ne, sizeof(inc_t));
  for (int64_t tt = 0; tt < h->n_tracks; ++tt) {
    for (int d = 0; d < 2; ++d) {
      /* incoming end of (tt,d): forward enters at the start point, backward at the end point */
      double x = h->track_xy[4 * tt + (d ? 2 : 0)], y = h->track_xy[4 * tt + (d ? 3 : 1)];
      int w = wall_of(h, x, y, tol);
      int dir2pi = h->track_dir[tt] + d * h->n_dir;
      inc[2 * tt + d].key = (w < 0) ? -1 : dir2pi * 4 + w;
      inc[2 * tt + d].c = (w == 0 || w == 1) ? y : x;
      inc[2 * tt + d].e = 2 * tt + d;
    }
  }
  qsort(inc, ne, sizeof(inc_t), cmp_inc);
  for (int64_t e = 0; e < ne; ++e) h->link[e] = -1;
  for (int64_t tt = 0; tt < h->n_tracks; ++tt) {
    for (int d = 0; d < 2; ++d) {
      /* outgoing end of (tt,d): forward leaves at the end point, backward at the start point */
      double x = h->track_xy[4 * tt + (d ? 0 : 2)], y = h->track_xy[4 * tt + (d ? 1 : 3)];
      int w = wall_of(h, x, y, tol);
      if (w < 0 || h->bc[w] == 0) continue;   /* interior gap end or vacuum wall */
      double ph = h->phi_a[h->track_dir[tt]] + d * ORC_PI;
      double ux = cos(ph), uy = sin(ph);
      if (w <= 1) ux = -ux; else uy = -uy;
      double pr = atan2(uy, ux);
      if (pr < 0) pr += 2.0 * ORC_PI;
      /* direction index (over 2 pi) of the reflected angle */
      int best = -1; double bd = 1e300;
      for (int j = 0; j < 2 * h->n_dir; ++j) {
        double pj = h->phi_a[j % h->n_dir] + (j >= h->n_dir ? ORC_PI : 0.0);
        double dd = fabs(pj - pr);
        if (dd > ORC_PI) dd = 2.0 * ORC_PI - dd;
        if (dd < bd) { bd = dd; best = j; }
      }
      if (bd > 1e-9) { snprintf(h->err, sizeof h->err, "reflected direction not in the set"); free(inc); return -1; }
      int key = best * 4 + w;
      double c = (w <= 1) ? y : x;
      /* first entry with (key, coordinate) >= (key, c - tol) */
      int64_t lo = 0, hi = ne;
      while (lo < hi) {
        int64_t m = (lo + hi) / 2;
        if (inc[m].key < key || (inc[m].key == key && inc[m].c < c - tol)) lo = m + 1; else hi = m;
      }
      if (lo >= ne || inc[lo].key != key || fabs(inc[lo].c - c) > tol) {
        snprintf(h->err, sizeof h->err, "no reflective partner for track %lld end %d", (long long)tt, d);
        free(inc); return -1;
      }
      h->link[2 * tt + d] = inc[lo].e;
    }
  }
  free(inc);
  /* 5. tracked areas */
  h->area = xcalloc(h->n_tri, sizeof(double));
  for (int64_t tt = 0; tt < h->n_tracks; ++tt) {
    int j = h->track_dir[tt];
    double wgt = 2.0 * h->omega_a[j] * h->delta_a[j];
    for (int64_t s2 = h->seg_off[tt]; s2 < h->seg_off[tt + 1]; ++s2) h->area[h->seg_reg[s2]] += wgt * h->seg_len[s2];
  }
  return 0;
}

orc_t *orc_create(int n_vert, const double *xy, int n_tri, const int32_t *tri, const int32_t *mat,
                  const double *bbox, const int32_t *bc, int n_azim, double spacing, int n_polar,
                  const double *sin_theta, const double *polar_w, int layout, char *err_out) {
  orc_t *h = xcalloc(1, sizeof(orc_t));
  h->n_vert = n_vert; h->n_tri = n_tri;
  h->xy = xcalloc(2 * (size_t)n_vert, sizeof(double)); memcpy(h->xy, xy, 2 * (size_t)n_vert * sizeof(double));
  h->tri = xcalloc(3 * (size_t)n_tri, sizeof(int32_t)); memcpy(h->tri, tri, 3 * (size_t)n_tri * sizeof(int32_t));
  h->mat = xcalloc(n_tri, sizeof(int32_t)); memcpy(h->mat, mat, (size_t)n_tri * sizeof(int32_t));
  h->xmin = bbox[0]; h->xmax = bbox[1]; h->ymin = bbox[2]; h->ymax = bbox[3];
  for (int i = 0; i < 4; ++i) h->bc[i] = bc[i];
  h->n_azim = n_azim; h->n_polar = n_polar;
  h->sin_theta = xcalloc(n_polar, sizeof(double)); memcpy(h->sin_theta, sin_theta, n_polar * sizeof(double));
  h->polar_w = xcalloc(n_polar, sizeof(double)); memcpy(h->polar_w, polar_w, n_polar * sizeof(double));
  h->n_threads = 1;
  h->k = 1.0;
  h->layout = layout;
  if (n_azim < 4 || n_azim % 4 || spacing <= 0 || n_polar < 1 || layout < 0 || layout > 1) {
    snprintf(err_out, 256, "bad quadrature arguments"); orc_destroy(h); return NULL;
  }
  if (layout == 1 && (bc[0] || bc[1] || bc[2] || bc[3])) {
    snprintf(err_out, 256, "back-projected rays need vacuum on every boundary"); orc_destroy(h); return NULL;
  }
  if (build_quadrature(h, spacing) || build_tracks(h)) {
    snprintf(err_out, 256, "%s", h->err); orc_destroy(h); return NULL;
  }
  return h;
}

void orc_set_threads(orc_t *h, int n) { h->n_threads = n > 0 ? n : 1; }

void orc_counts(const orc_t *h, int64_t *n_tracks, int64_t *n_seg, int *n_dir) {
  *n_tracks = h->n_tracks; *n_seg = h->n_seg; *n_dir = h->n_dir;
}

void orc_get_quadrature(const orc_t *h, double *phi, double *delta, double *omega, int32_t *nx, int32_t *ny) {
  for (int j = 0; j < h->n_dir; ++j) {
    phi[j] = h->phi_a[j]; delta[j] = h->delta_a[j]; omega[j] = h->omega_a[j];
    nx[j] = h->nx_a[j]; ny[j] = h->ny_a[j];
  }
}

void orc_get_tracks(const orc_t *h, int64_t *seg_off, int32_t *seg_reg, double *seg_len,
                    int32_t *track_dir, double *track_xy, int64_t *link) {
  memcpy(seg_off, h->seg_off, (h->n_tracks + 1) * sizeof(int64_t));
  memcpy(seg_reg, h->seg_reg, h->n_seg * sizeof(int32_t));
  memcpy(seg_len, h->seg_len, h->n_seg * sizeof(double));
  memcpy(track_dir, h->track_dir, h->n_tracks * sizeof(int32_t));
  memcpy(track_xy, h->track_xy, 4 * h->n_tracks * sizeof(double));
  memcpy(link, h->link, 2 * h->n_tracks * sizeof(int64_t));
}

void orc_get_areas(const orc_t *h, double *area) { memcpy(area, h->area, h->n_tri * sizeof(double)); }

/* ---------------------------------------------------------------- CMFD set-up ---- */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x < y) ? -1 : (x > y);
}

/* slot of the current from cell a to cell b */
static int64_t cmfd_slot(const orc_t *h, int a, int b) {
  uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a), key = (lo << 32) | hi;
  int64_t l = 0, r = h->n_if;
  while (l < r) { int64_t m = (l + r) / 2; if (h->pairs[m] < key) l = m + 1; else r = m; }
  return 2 * l + (a > b ? 1 : 0);
}

/* ---------------------------------------------------------------- physics ---- */
int orc_set_xs(orc_t *h, int n_mat, int G, const double *st, const double *nsf, const double *chi,
               const double *ss) {
  free(h->st); free(h->nsf); free(h->chi); free(h->ss);
  free(h->phi); free(h->q); free(h->tally); free(h->psi_in); free(h->psi_next); free(h->leak);
  free(h->ext); h->ext = NULL;
  free(h->ssl); free(h->kern); free(h->qdir); free(h->tdir); free(h->pbar);
  h->ssl = h->kern = h->qdir = h->tdir = h->pbar = NULL; h->L = 0;
  free(h->cell); free(h->pairs); free(h->cur); free(h->cleak); free(h->color);
  free(h->nb_off); free(h->nb_cell); free(h->nb_in);
  h->cell = NULL; h->pairs = NULL; h->cur = NULL; h->cleak = NULL; h->color = NULL; h->cmfd = 0;
  h->nb_off = h->nb_cell = h->nb_in = NULL;
  free(h->dz); free(h->mat3); free(h->phi3); free(h->q3); free(h->tal3); free(h->psi3_in); free(h->psi3_next);
  free(h->ztop); free(h->leak3); free(h->jz); free(h->zleak);
  h->dz = h->phi3 = h->q3 = h->tal3 = h->psi3_in = h->psi3_next = h->ztop = h->leak3 = h->jz = h->zleak = NULL;
  h->mat3 = NULL; h->nz = 0; h->dgcm = 0;
  h->n_mat = n_mat; h->G = G;
  h->st = xcalloc((size_t)n_mat * G, sizeof(double)); memcpy(h->st, st, (size_t)n_mat * G * sizeof(double));
  h->nsf = xcalloc((size_t)n_mat * G, sizeof(double)); memcpy(h->nsf, nsf, (size_t)n_mat * G * sizeof(double));
  h->chi = xcalloc((size_t)n_mat * G, sizeof(double)); memcpy(h->chi, chi, (size_t)n_mat * G * sizeof(double));
  h->ss = xcalloc((size_t)n_mat * G * G, sizeof(double)); memcpy(h->ss, ss, (size_t)n_mat * G * G * sizeof(double));
  for (int i = 0; i < h->n_tri; ++i)
    if (h->mat[i] < 0 || h->mat[i] >= n_mat) { snprintf(h->err, sizeof h->err, "material id out of range"); return -1; }
  size_t RG = (size_t)h->n_tri * G, PB = (size_t)h->n_tracks * 2 * h->n_polar * G;
  h->phi = xcalloc(RG, sizeof(double));
  h->q = xcalloc(RG, sizeof(double));
  h->tally = xcalloc(RG, sizeof(double));
  h->psi_in = xcalloc(PB, sizeof(double));
  h->psi_next = xcalloc(PB, sizeof(double));
  h->leak = xcalloc(G, sizeof(double));
  for (size_t i = 0; i < RG; ++i) h->phi[i] = 1.0;
  h->k = 1.0;
  return 0;
}

/* Enable the acceleration on the coarse cells `cell` [R] (NULL disables). Interfaces are the
 * pairs of cells that consecutive segments of some track cross between. Cells are coloured
 * greedily in ascending id (each takes the smallest colour none of its lower-id neighbours has),
 * so cells of one colour share no interface and their over-relaxed updates are independent.
 * Call after orc_set_xs. */
int orc_set_cmfd(orc_t *h, const int32_t *cell, int n_cells, int n_outer, int n_inner, double omega) {
  free(h->cell); free(h->pairs); free(h->cur); free(h->cleak); free(h->color);
  free(h->nb_off); free(h->nb_cell); free(h->nb_in);
  h->cell = NULL; h->pairs = NULL; h->cur = NULL; h->cleak = NULL; h->color = NULL; h->cmfd = 0;
  h->nb_off = h->nb_cell = h->nb_in = NULL;
  if (!cell) return 0;
  if (h->L) { snprintf(h->err, sizeof h->err, "CMFD with anisotropic scattering is not supported"); return -1; }
  if (h->nz) { snprintf(h->err, sizeof h->err, "CMFD with DGMOC is not supported"); return -1; }
  h->cell = xcalloc(h->n_tri, sizeof(int32_t));
  memcpy(h->cell, cell, h->n_tri * sizeof(int32_t));
  int64_t np = 0;
  for (int64_t t = 0; t < h->n_tracks; ++t)
    for (int64_t s2 = h->seg_off[t]; s2 + 1 < h->seg_off[t + 1]; ++s2)
      if (cell[h->seg_reg[s2]] != cell[h->seg_reg[s2 + 1]]) np++;
  uint64_t *pr = xcalloc(np, sizeof(uint64_t));
  np = 0;
  for (int64_t t = 0; t < h->n_tracks; ++t)
    for (int64_t s2 = h->seg_off[t]; s2 + 1 < h->seg_off[t + 1]; ++s2) {
      int a = cell[h->seg_reg[s2]], b = cell[h->seg_reg[s2 + 1]];
      if (a == b) continue;
      uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
      pr[np++] = (lo << 32) | hi;
    }
  qsort(pr, np, sizeof(uint64_t), cmp_u64);
  int64_t nu = 0;
  for (int64_t k = 0; k < np; ++k) if (nu == 0 || pr[k] != pr[nu - 1]) pr[nu++] = pr[k];
  h->pairs = pr; h->n_if = (int)nu;
  h->n_cells = n_cells; h->cm_outer = n_outer; h->cm_inner = n_inner;
  h->cur = xcalloc(2 * (size_t)nu * h->G, sizeof(double));
  h->cleak = xcalloc((size_t)(n_cells > 1 ? n_cells : 1) * h->G, sizeof(double));
  h->cm_omega = omega;
  /* neighbour lists */
  h->nb_off = xcalloc((size_t)n_cells + 1, sizeof(int32_t));
  h->nb_cell = xcalloc(2 * (size_t)nu + 1, sizeof(int32_t));
  h->nb_in = xcalloc(2 * (size_t)nu + 1, sizeof(int32_t));
  for (int e = 0; e < h->n_if; ++e) {
    h->nb_off[(int)(h->pairs[e] >> 32) + 1]++;
    h->nb_off[(int)(h->pairs[e] & 0xffffffffu) + 1]++;
  }
  for (int i = 0; i < n_cells; ++i) h->nb_off[i + 1] += h->nb_off[i];
  int32_t *fill = xcalloc((size_t)n_cells + 1, sizeof(int32_t));
  for (int e = 0; e < h->n_if; ++e) {
    int a = (int)(h->pairs[e] >> 32), b = (int)(h->pairs[e] & 0xffffffffu);
    /* slot 2e runs a -> b, slot 2e + 1 runs b -> a */
    int qa = h->nb_off[a] + fill[a]++, qb = h->nb_off[b] + fill[b]++;
    h->nb_cell[qa] = b; h->nb_in[qa] = 2 * e + 1;
    h->nb_cell[qb] = a; h->nb_in[qb] = 2 * e;
  }
  free(fill);
  /* greedy colouring over the interface graph */
  h->color = xcalloc(n_cells > 1 ? n_cells : 1, sizeof(int32_t));
  int *used = xcalloc((size_t)n_cells + 1, sizeof(int));  /* used[c] == i + 1: colour c taken for cell i */
  h->n_colors = 0;
  for (int i = 0; i < n_cells; ++i) {
    for (int q = h->nb_off[i]; q < h->nb_off[i + 1]; ++q) {
      int j = h->nb_cell[q];
      if (j < i) used[h->color[j]] = i + 1;
    }
    int c = 0;
    while (used[c] == i + 1) ++c;
    h->color[i] = c;
    if (c + 1 > h->n_colors) h->n_colors = c + 1;
  }
  free(used);
  h->cmfd = 1;
  return 0;
}

/* Legendre polynomial P_l(x) by the three-term recurrence */
double orc_legendre(int l, double x) {
  double p0 = 1.0, p1 = x;
  if (l == 0) return p0;
  for (int n = 1; n < l; ++n) {
    double p2 = ((2.0 * n + 1.0) * x * p1 - n * p0) / (n + 1.0);
    p0 = p1; p1 = p2;
  }
  return p1;
}

/* the direction of index m: azimuth phi_j (+ pi for the reverse sense), polar sin/cos (upper
 * hemisphere) */
static void direction_of(const orc_t *h, int m, double *om) {
  int P = h->n_polar, p = m % P, jd = m / P, j = jd / 2, d = jd % 2;
  double ph = h->phi_a[j] + d * ORC_PI, st = h->sin_theta[p], ct = sqrt(1.0 - st * st);
  om[0] = st * cos(ph); om[1] = st * sin(ph); om[2] = ct;
}

static void init_pbar(orc_t *h) {
  for (int i = 0; i < h->n_tri; ++i)
    for (int m = 0; m < h->ND; ++m)
      for (int g = 0; g < h->G; ++g)
        h->pbar[((size_t)i * h->ND + m) * h->G + g] = h->phi[(size_t)i * h->G + g] / (4.0 * ORC_PI);
}

/* Anisotropic scattering of order L (0 restores isotropic scattering): ssl [L][M][G][G] holds
 * Sigma_s,l for l = 1..L. The scattering source of direction Om is
 *   sum_l (2l+1)/(4 pi) sum_g' Sigma_s,l g'->g  int P_l(Om . Om') psi_g'(Om') dOm',
 * the integral taken with the discrete quadrature (both hemispheres of each polar angle) over the
 * region-average angular flux of the previous outer. Call after orc_set_xs. */
int orc_set_scattering(orc_t *h, int L, const double *ssl) {
  free(h->ssl); free(h->kern); free(h->qdir); free(h->tdir); free(h->pbar);
  h->ssl = h->kern = h->qdir = h->tdir = h->pbar = NULL; h->L = 0;
  if (L <= 0 || !ssl) return 0;
  if (h->cmfd) { snprintf(h->err, sizeof h->err, "anisotropic scattering with CMFD is not supported"); return -1; }
  if (h->nz) { snprintf(h->err, sizeof h->err, "anisotropic scattering with DGMOC is not supported"); return -1; }
  int G = h->G, M = h->n_mat, P = h->n_polar;
  h->L = L;
  h->ND = 2 * h->n_dir * P;
  int ND = h->ND;
  h->ssl = xcalloc((size_t)L * M * G * G, sizeof(double));
  memcpy(h->ssl, ssl, (size_t)L * M * G * G * sizeof(double));
  h->kern = xcalloc((size_t)L * ND * ND, sizeof(double));
  for (int m = 0; m < ND; ++m) {
    double om[3];
    direction_of(h, m, om);
    for (int m2 = 0; m2 < ND; ++m2) {
      double o2[3];
      direction_of(h, m2, o2);
      int j2 = (m2 / P) / 2, p2 = m2 % P;
      double w = 4.0 * ORC_PI * h->omega_a[j2] * h->polar_w[p2];
      double cp = om[0] * o2[0] + om[1] * o2[1] + om[2] * o2[2];
      double cm = om[0] * o2[0] + om[1] * o2[1] - om[2] * o2[2];
      for (int l = 1; l <= L; ++l)
        h->kern[((size_t)(l - 1) * ND + m) * ND + m2] = w * 0.5 * (orc_legendre(l, cp) + orc_legendre(l, cm));
    }
  }
  h->qdir = xcalloc((size_t)h->n_tri * ND * G, sizeof(double));
  h->tdir = xcalloc((size_t)h->n_tri * ND * G, sizeof(double));
  h->pbar = xcalloc((size_t)h->n_tri * ND * G, sizeof(double));
  init_pbar(h);
  return 0;
}

void orc_set_fixed_source(orc_t *h, const double *S) {
  free(h->ext); h->ext = NULL;
  if (S) {
    h->ext = xcalloc((size_t)h->n_tri * h->G, sizeof(double));
    memcpy(h->ext, S, (size_t)h->n_tri * h->G * sizeof(double));
  }
}

static void dg_set_state(orc_t *h, const double *phi3, double k);
static double dg_outer(orc_t *h, int eigen);
static double dg_fission_total(const orc_t *h, const double *phi3);

/* F = sum_i A_i sum_g nuSigma_f phi */
static double fission_total(const orc_t *h, const double *phi) {
  double F = 0.0;
  for (int i = 0; i < h->n_tri; ++i) {
    const double *nf = h->nsf + (size_t)h->mat[i] * h->G;
    double f = 0.0;
    for (int g = 0; g < h->G; ++g) f += nf[g] * phi[(size_t)i * h->G + g];
    F += h->area[i] * f;
  }
  return F;
}

void orc_set_state(orc_t *h, const double *phi, double k, const double *psi) {
  if (h->nz) { dg_set_state(h, phi, k); return; }   /* phi: [nz][R][2][G]; psi not used */
  size_t RG = (size_t)h->n_tri * h->G, PB = (size_t)h->n_tracks * 2 * h->n_polar * h->G;
  if (phi) memcpy(h->phi, phi, RG * sizeof(double)); else for (size_t i = 0; i < RG; ++i) h->phi[i] = 1.0;
  if (psi) memcpy(h->psi_in, psi, PB * sizeof(double)); else memset(h->psi_in, 0, PB * sizeof(double));
  /* vacuum boundary: an incoming end that no outgoing end feeds has zero inflow */
  char *fed = xcalloc(2 * h->n_tracks, 1);
  for (int64_t e = 0; e < 2 * h->n_tracks; ++e) if (h->link[e] >= 0) fed[h->link[e]] = 1;
  size_t per = (size_t)h->n_polar * h->G;
  for (int64_t e = 0; e < 2 * h->n_tracks; ++e) if (!fed[e]) memset(h->psi_in + e * per, 0, per * sizeof(double));
  free(fed);
  h->k = k;
  if (h->L) init_pbar(h);   /* the anisotropic state restarts from an isotropic angular flux */
}

void orc_get_state(const orc_t *h, double *phi, double *k, double *psi) {
  size_t RG = (size_t)h->n_tri * h->G, PB = (size_t)h->n_tracks * 2 * h->n_polar * h->G;
  if (phi) memcpy(phi, h->phi, RG * sizeof(double));
  if (k) *k = h->k;
  if (psi) memcpy(psi, h->psi_in, PB * sizeof(double));
}

void orc_get_q(const orc_t *h, double *q) { memcpy(q, h->q, (size_t)h->n_tri * h->G * sizeof(double)); }
void orc_get_tally(const orc_t *h, double *t) { memcpy(t, h->tally, (size_t)h->n_tri * h->G * sizeof(double)); }
void orc_get_leakage(const orc_t *h, double *l) { memcpy(l, h->leak, h->G * sizeof(double)); }

/* Eq. MGNTE_element source, isotropic (per steradian) */
static void update_source(orc_t *h, int eigen) {
  int G = h->G;
  for (int i = 0; i < h->n_tri; ++i) {
    int m = h->mat[i];
    const double *ph = h->phi + (size_t)i * G;
    double fis = 0.0;
    for (int gp = 0; gp < G; ++gp) fis += h->nsf[(size_t)m * G + gp] * ph[gp];
    for (int g = 0; g < G; ++g) {
      double sc = 0.0;
      for (int gp = 0; gp < G; ++gp) sc += h->ss[((size_t)m * G + gp) * G + g] * ph[gp];
      double src = sc;
      if (eigen) src += h->chi[(size_t)m * G + g] / h->k * fis;
      if (h->ext) src += h->ext[(size_t)i * G + g];
      h->q[(size_t)i * G + g] = src / (4.0 * ORC_PI);
    }
    if (h->L) {
      int ND = h->ND;
      double *v = xcalloc(ND, sizeof(double));
      for (int mdir = 0; mdir < ND; ++mdir)
        for (int g = 0; g < G; ++g) h->qdir[((size_t)i * ND + mdir) * G + g] = h->q[(size_t)i * G + g];
      for (int l = 1; l <= h->L; ++l) {
        const double *K = h->kern + (size_t)(l - 1) * ND * ND;
        for (int gp = 0; gp < G; ++gp) {
          /* v_m = int P_l(Om_m . Om') psi_g'(Om') dOm' */
          for (int mdir = 0; mdir < ND; ++mdir) {
            double a = 0.0;
            for (int m2 = 0; m2 < ND; ++m2) a += K[(size_t)mdir * ND + m2] * h->pbar[((size_t)i * ND + m2) * G + gp];
            v[mdir] = a;
          }
          for (int g = 0; g < G; ++g) {
            double sl = h->ssl[(((size_t)(l - 1) * h->n_mat + m) * G + gp) * G + g];
            if (sl == 0.0) continue;
            double c = (2.0 * l + 1.0) / (4.0 * ORC_PI) * sl;
            for (int mdir = 0; mdir < ND; ++mdir) h->qdir[((size_t)i * ND + mdir) * G + g] += c * v[mdir];
          }
        }
      }
      free(v);
    }
  }
}

/* One transport sweep of every track, both directions, every polar angle and group (Eq. MOC_sol),
 * tallying W (psi_in - psi_out) per segment into its region; outgoing fluxes are routed to the
 * linked incoming ends for the next sweep (Jacobi in boundary flux).
 *
 * Parallel in a fixed order: groups one after another; within a group the tracks are cut into
 * n_chunks fixed ranges of track indices (a function of the problem, never of the thread count),
 * each chunk sums its own partial tallies and currents, and the partials are added in chunk order.
 * The result is therefore the same for any thread count. */
static int sweep_chunks(const orc_t *h) {
  int64_t nc = h->n_tracks / 64;
  int cap = h->L ? 4 : 32;   /* per-direction tallies make a chunk's partials large */
  if (nc < 1) nc = 1;
  if (nc > cap) nc = cap;
  return (int)nc;
}

static void transport_sweep(orc_t *h) {
  const int G = h->G, P = h->n_polar, R = h->n_tri, ND = h->L ? h->ND : 0;
  const int NC = sweep_chunks(h);
  const size_t PB = (size_t)h->n_tracks * 2 * P * G;
  const size_t n_cur = h->cmfd ? 2 * (size_t)h->n_if : 0, n_cl = h->cmfd ? (size_t)h->n_cells : 0;
  /* per-chunk partials of one group: tally [R], per-direction tally [R][ND], currents, leakage */
  const size_t per = (size_t)R + (size_t)R * ND + n_cur + n_cl + 1;
  double *part = xcalloc((size_t)NC * per, sizeof(double));
  memset(h->psi_next, 0, PB * sizeof(double));
  for (int g = 0; g < G; ++g) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(h->n_threads)
    for (int c = 0; c < NC; ++c) {
      double *tal = part + (size_t)c * per, *tdir = tal + R, *cur = tdir + (size_t)R * ND, *cleak = cur + n_cur;
      double *lk = cleak + n_cl;
      const int64_t t0 = h->n_tracks * c / NC, t1 = h->n_tracks * (c + 1) / NC;
      for (int64_t t = t0; t < t1; ++t) {
        int j = h->track_dir[t];
        int64_t s0 = h->seg_off[t], s1 = h->seg_off[t + 1];
        for (int d = 0; d < 2; ++d) {
          for (int p = 0; p < P; ++p) {
            double Wt = 4.0 * ORC_PI * h->omega_a[j] * h->polar_w[p] * h->delta_a[j] * h->sin_theta[p];
            double psi = h->psi_in[((size_t)(2 * t + d) * P + p) * G + g];
            if (h->cmfd) {
              /* current entering the domain at this start (zero at vacuum starts) */
              int64_t s_first = d ? (s1 - 1) : s0;
              cleak[h->cell[h->seg_reg[s_first]]] -= Wt * psi;
            }
            int mdir = (j * 2 + d) * P + p;
            for (int64_t n = 0; n < s1 - s0; ++n) {
              int64_t s = d ? (s1 - 1 - n) : (s0 + n);
              int i = h->seg_reg[s];
              double sig = h->st[(size_t)h->mat[i] * G + g];
              double qi = h->L ? h->qdir[((size_t)i * h->ND + mdir) * G + g] : h->q[(size_t)i * G + g];
              double tau = sig * h->seg_len[s] / h->sin_theta[p];
              double delta = (psi - qi / sig) * (-expm1(-tau));
              tal[i] += Wt * delta;
              if (h->L) tdir[(size_t)i * ND + mdir] += h->delta_a[j] * h->sin_theta[p] * delta;
              psi -= delta;
              if (h->cmfd && n + 1 < s1 - s0) {
                /* partial current W psi into the next cell along the track, if the cell changes */
                int64_t sn = d ? (s - 1) : (s + 1);
                int a = h->cell[i], b = h->cell[h->seg_reg[sn]];
                if (a != b) cur[cmfd_slot(h, a, b)] += Wt * psi;
              }
            }
            int64_t e = h->link[2 * t + d];
            if (e >= 0) h->psi_next[((size_t)e * P + p) * G + g] = psi;
            else *lk += Wt * psi;
            if (h->cmfd) {
              /* current leaving the domain at this end, vacuum or reflective */
              int64_t s_last = d ? s0 : (s1 - 1);
              cleak[h->cell[h->seg_reg[s_last]]] += Wt * psi;
            }
          }
        }
      }
    }
    /* the chunks' partials in chunk order (and cleared for the next group) */
#pragma omp parallel for schedule(static) num_threads(h->n_threads)
    for (int i = 0; i < R; ++i) {
      double a = 0.0;
      for (int c = 0; c < NC; ++c) {
        double *v = part + (size_t)c * per + i;
        a += *v;
        *v = 0.0;
      }
      h->tally[(size_t)i * G + g] = a;
      for (int m = 0; m < ND; ++m) {
        double b = 0.0;
        for (int c = 0; c < NC; ++c) {
          double *v = part + (size_t)c * per + R + (size_t)i * ND + m;
          b += *v;
          *v = 0.0;
        }
        h->tdir[((size_t)i * ND + m) * G + g] = b;
      }
    }
    const size_t tail = (size_t)R + (size_t)R * ND;
    for (size_t x = 0; x < n_cur + n_cl + 1; ++x) {
      double a = 0.0;
      for (int c = 0; c < NC; ++c) {
        double *v = part + (size_t)c * per + tail + x;
        a += *v;
        *v = 0.0;
      }
      if (x < n_cur) h->cur[x * G + g] = a;
      else if (x < n_cur + n_cl) h->cleak[(x - n_cur) * G + g] = a;
      else h->leak[g] = a;
    }
  }
  free(part);
}

/* scalar flux from source and tallies */
static void finalize_flux(const orc_t *h, double *phi_new, double *pbar_new) {
  int G = h->G, P = h->n_polar, ND = h->ND;
  for (int i = 0; i < h->n_tri; ++i) {
    for (int g = 0; g < G; ++g) {
      double sig = h->st[(size_t)h->mat[i] * G + g];
      size_t ig = (size_t)i * G + g;
      double v;
      if (h->L) {
        /* angular integration of the flat-source part over the discrete directions, and the
         * region-average angular flux of every direction for the next source */
        v = 0.0;
        for (int m = 0; m < ND; ++m) {
          int j = (m / P) / 2, p = m % P;
          double qm = h->qdir[((size_t)i * ND + m) * G + g];
          v += 4.0 * ORC_PI * h->omega_a[j] * h->polar_w[p] * qm / sig;
          double pb = qm / sig;
          if (h->area[i] > 0.0) pb += h->tdir[((size_t)i * ND + m) * G + g] / (sig * h->area[i]);
          pbar_new[((size_t)i * ND + m) * G + g] = pb;
        }
      } else {
        v = 4.0 * ORC_PI * h->q[ig] / sig;
      }
      if (h->area[i] > 0.0) v += h->tally[ig] / (sig * h->area[i]);
      phi_new[ig] = v;
    }
  }
}

/* The coarse step on the normalised new flux phi_new (currents already divided by the same
 * normalisation): homogenise per cell, coarse balance with partial-current coefficients, a fixed
 * number of coarse power iterations (Gauss-Seidel in energy, over-relaxed Gauss-Seidel sweeps in
 * space, colour by colour), then scale phi_new
 * and the boundary flux for the next sweep by the coarse/fine ratio of their cell and take the
 * coarse k. */
static void cmfd_step(orc_t *h, double *phi_new) {
  int G = h->G, N = h->n_cells, P = h->n_polar;
  double *cphi = xcalloc((size_t)N * G, sizeof(double)), *TV = xcalloc((size_t)N * G, sizeof(double));
  double *FV = xcalloc((size_t)N * G, sizeof(double)), *CH = xcalloc((size_t)N * G, sizeof(double));
  double *SV = xcalloc((size_t)N * G * G, sizeof(double)), *V = xcalloc(N, sizeof(double));
  /* homogenisation, regions of each cell in ascending order */
  for (int r = 0; r < h->n_tri; ++r) {
    int i = h->cell[r], m = h->mat[r];
    double A = h->area[r], f = 0.0;
    V[i] += A;
    for (int g = 0; g < G; ++g) f += h->nsf[(size_t)m * G + g] * phi_new[(size_t)r * G + g];
    for (int g = 0; g < G; ++g) {
      double a = A * phi_new[(size_t)r * G + g];
      cphi[(size_t)i * G + g] += a;
      TV[(size_t)i * G + g] += h->st[(size_t)m * G + g] * a;
      FV[(size_t)i * G + g] += h->nsf[(size_t)m * G + g] * a;
      CH[(size_t)i * G + g] += h->chi[(size_t)m * G + g] * A * f;
      for (int gg = 0; gg < G; ++gg) SV[((size_t)i * G + g) * G + gg] += h->ss[((size_t)m * G + g) * G + gg] * a;
    }
  }
  for (int i = 0; i < N; ++i) {
    double chs = 0.0;
    for (int g = 0; g < G; ++g) chs += CH[(size_t)i * G + g];
    for (int g = 0; g < G; ++g) {
      size_t x = (size_t)i * G + g;
      double raw = cphi[x];
      if (raw > 0.0) {
        TV[x] = TV[x] * V[i] / raw;
        FV[x] = FV[x] * V[i] / raw;
        for (int gg = 0; gg < G; ++gg) SV[x * G + gg] = SV[x * G + gg] * V[i] / raw;
      } else {
        TV[x] = FV[x] = 0.0;
        for (int gg = 0; gg < G; ++gg) SV[x * G + gg] = 0.0;
      }
      cphi[x] = (V[i] > 0.0) ? raw / V[i] : 0.0;
      CH[x] = (chs > 0.0) ? CH[x] / chs : 0.0;
    }
  }
  /* coefficients: out of cell i through interface e (cell i side s): D = J(out)/phi_i; in: J(in)/phi_j */
  double *diag = xcalloc((size_t)N * G, sizeof(double));
  double *phic = xcalloc((size_t)N * G, sizeof(double));
  double *fis = xcalloc(N, sizeof(double));
  for (int i = 0; i < N; ++i)
    for (int g = 0; g < G; ++g) {
      size_t x = (size_t)i * G + g;
      double pi = cphi[x], dg = TV[x] - SV[x * G + g];
      if (pi > 0.0) dg += h->cleak[x] / pi;
      diag[x] = dg;
      phic[x] = pi;
    }
  for (int e = 0; e < h->n_if; ++e) {
    int a = (int)(h->pairs[e] >> 32), b = (int)(h->pairs[e] & 0xffffffffu);
    for (int g = 0; g < G; ++g) {
      double pa = cphi[(size_t)a * G + g], pb = cphi[(size_t)b * G + g];
      if (pa > 0.0) diag[(size_t)a * G + g] += h->cur[(size_t)(2 * e) * G + g] / pa;
      if (pb > 0.0) diag[(size_t)b * G + g] += h->cur[(size_t)(2 * e + 1) * G + g] / pb;
    }
  }
  double kc = h->k;
  for (int it = 0; it < h->cm_outer; ++it) {
    double F_old = 0.0;
    for (int i = 0; i < N; ++i) {
      double f = 0.0;
      for (int g = 0; g < G; ++g) f += FV[(size_t)i * G + g] * phic[(size_t)i * G + g];
      fis[i] = f;
      F_old += f;
    }
    for (int g = 0; g < G; ++g) {
      /* n_inner over-relaxed Gauss-Seidel sweeps, colour by colour (cells of one colour are
       * independent): x_i <- x_i + omega (rhs_i / diag_i - x_i), rhs_i = fission and other groups'
       * scattering into g + inflow from the neighbours at their current values */
      for (int j = 0; j < h->cm_inner; ++j) {
        for (int c = 0; c < h->n_colors; ++c) {
          for (int i = 0; i < N; ++i) {
            if (h->color[i] != c) continue;
            size_t x = (size_t)i * G + g;
            double rhs = CH[x] * fis[i] / kc;
            for (int gg = 0; gg < G; ++gg)
              if (gg != g) rhs += SV[((size_t)i * G + gg) * G + g] * phic[(size_t)i * G + gg];
            for (int q = h->nb_off[i]; q < h->nb_off[i + 1]; ++q) {
              int nb = h->nb_cell[q];
              double pn = cphi[(size_t)nb * G + g];
              if (pn > 0.0) rhs += h->cur[(size_t)h->nb_in[q] * G + g] / pn * phic[(size_t)nb * G + g];
            }
            if (diag[x] > 0.0) phic[x] += h->cm_omega * (rhs / diag[x] - phic[x]);
          }
        }
      }
    }
    double F_new = 0.0;
    for (int i = 0; i < N; ++i)
      for (int g = 0; g < G; ++g) F_new += FV[(size_t)i * G + g] * phic[(size_t)i * G + g];
    if (F_new > 0.0 && F_old > 0.0) kc = kc * F_new / F_old;
  }
  /* prolongation of the flux and of the incoming boundary flux of the next sweep */
  for (int r = 0; r < h->n_tri; ++r)
    for (int g = 0; g < G; ++g) {
      size_t x = (size_t)h->cell[r] * G + g;
      double ratio = (cphi[x] > 0.0 && phic[x] > 0.0) ? phic[x] / cphi[x] : 1.0;
      phi_new[(size_t)r * G + g] *= ratio;
    }
  for (int64_t t = 0; t < h->n_tracks; ++t)
    for (int d = 0; d < 2; ++d) {
      int r = h->seg_reg[d ? h->seg_off[t + 1] - 1 : h->seg_off[t]];
      for (int g = 0; g < G; ++g) {
        size_t x = (size_t)h->cell[r] * G + g;
        double ratio = (cphi[x] > 0.0 && phic[x] > 0.0) ? phic[x] / cphi[x] : 1.0;
        for (int p = 0; p < P; ++p) h->psi_next[((size_t)(2 * t + d) * P + p) * G + g] *= ratio;
      }
    }
  h->k = kc;
  free(cphi); free(TV); free(FV); free(CH); free(SV); free(V); free(diag); free(phic); free(fis);
}

/* One outer iteration: source, sweep, flux, and (eigen mode) k update + normalisation.
 * Returns the residual. */
double orc_outer(orc_t *h, int eigen) {
  if (h->nz) return dg_outer(h, eigen);
  int G = h->G;
  size_t RG = (size_t)h->n_tri * G, PB = (size_t)h->n_tracks * 2 * h->n_polar * G;
  double *phi_new = xcalloc(RG, sizeof(double));
  size_t RD = h->L ? (size_t)h->n_tri * h->ND * G : 0;
  double *pbar_new = h->L ? xcalloc(RD, sizeof(double)) : NULL;
  update_source(h, eigen);
  transport_sweep(h);
  finalize_flux(h, phi_new, pbar_new);
  double resid = 0.0;
  if (eigen) {
    double F_old = fission_total(h, h->phi);
    double F_new = fission_total(h, phi_new);
    h->k = h->k * F_new / F_old;
    for (size_t i = 0; i < RG; ++i) phi_new[i] /= F_new;
    for (size_t i = 0; i < RD; ++i) pbar_new[i] /= F_new;
    for (size_t i = 0; i < PB; ++i) h->psi_next[i] /= F_new;
    for (int g = 0; g < G; ++g) h->leak[g] /= F_new;
    for (int i = 0; i < h->n_tri; ++i) {
      const double *nf = h->nsf + (size_t)h->mat[i] * G;
      double fo = 0.0, fn = 0.0;
      for (int g = 0; g < G; ++g) { fo += nf[g] * h->phi[(size_t)i * G + g] / F_old; fn += nf[g] * phi_new[(size_t)i * G + g]; }
      if (fn > 0.0) { double r = fabs(fn - fo) / fn; if (r > resid) resid = r; }
    }
    if (h->cmfd) {
      /* currents in the same normalisation as phi_new */
      for (size_t x = 0; x < 2 * (size_t)h->n_if * G; ++x) h->cur[x] /= F_new;
      for (size_t x = 0; x < (size_t)h->n_cells * G; ++x) h->cleak[x] /= F_new;
      cmfd_step(h, phi_new);
      double F2 = fission_total(h, phi_new);
      for (size_t i = 0; i < RG; ++i) phi_new[i] /= F2;
      for (size_t i = 0; i < PB; ++i) h->psi_next[i] /= F2;
    }
  } else {
    for (size_t i = 0; i < RG; ++i)
      if (phi_new[i] > 0.0) { double r = fabs(phi_new[i] - h->phi[i]) / phi_new[i]; if (r > resid) resid = r; }
  }
  memcpy(h->phi, phi_new, RG * sizeof(double));
  if (h->L) { memcpy(h->pbar, pbar_new, RD * sizeof(double)); free(pbar_new); }
  double *tmp = h->psi_in; h->psi_in = h->psi_next; h->psi_next = tmp;
  free(phi_new);
  return resid;
}

/* Normalise the current state so that F = 1 (eigen mode). */
void orc_normalise(orc_t *h) {
  if (h->nz) {
    double F3 = dg_fission_total(h, h->phi3);
    size_t n3 = (size_t)h->nz * h->n_tri * 2 * h->G;
    size_t nb = (size_t)h->n_tracks * 2 * 2 * h->nz * h->n_polar * 2 * h->G;
    size_t nt = (size_t)h->n_seg * 2 * h->n_polar * h->G;
    if (F3 > 0.0) {
      for (size_t i = 0; i < n3; ++i) h->phi3[i] /= F3;
      for (size_t i = 0; i < nb; ++i) h->psi3_in[i] /= F3;
      for (size_t i = 0; i < nt; ++i) h->ztop[i] /= F3;
    }
    return;
  }
  double F = fission_total(h, h->phi);
  size_t RG = (size_t)h->n_tri * h->G, PB = (size_t)h->n_tracks * 2 * h->n_polar * h->G;
  if (F > 0.0) {
    for (size_t i = 0; i < RG; ++i) h->phi[i] /= F;
    for (size_t i = 0; i < PB; ++i) h->psi_in[i] /= F;
    if (h->L)
      for (size_t i = 0; i < (size_t)h->n_tri * h->ND * h->G; ++i) h->pbar[i] /= F;
  }
}

/* Power iteration (eigen=1) or fixed-source iteration (eigen=0). Returns 0 if converged. */
int orc_iterate(orc_t *h, int eigen, double tol_k, double tol_f, int max_outer, double *k_out,
                int *n_out, double *resid_out) {
  if (eigen) orc_normalise(h);
  int n = 0;
  double resid = INFINITY;
  int conv = 0;
  while (n < max_outer) {
    double k_old = h->k;
    resid = orc_outer(h, eigen);
    n++;
    if ((!eigen || fabs(h->k - k_old) <= tol_k) && resid <= tol_f) { conv = 1; break; }
  }
  *k_out = h->k; *n_out = n; *resid_out = resid;
  return conv ? 0 : 1;
}

/* ============================================================================================
 * DGMOC (Sec. 2.2 "DGMOC formulation", Eq. DGMOC_expansion, DGMOC_weak, DGMOC_weak_up; the plane
 * by plane upward/downward march of Alg. 2).
 *
 * The planar tracks are extruded through nz axial planes of heights dz. In plane i the angular
 * flux along a track and the source are expanded in the Legendre basis u_1 = 1, u_2 = xi, with xi
 * running from -1 at the plane's bottom to +1 at its top (n = 2 basis functions, first order, as
 * in the paper). For an upward direction (polar cosine mu > 0, in-plane component sin(theta)),
 * testing the transport equation with 1 and with xi over the plane, integrating the axial
 * derivative by parts and taking the bottom-face value from the plane below (upwinding) gives,
 * along the planar track coordinate s, with psi = a + b xi, q = q0 + q1 xi and c = mu / dz:
 *     sin(theta) a' = q0 - Sigma_t a -   c (a + b - psi_in)
 *     sin(theta) b' = q1 - Sigma_t b - 3 c (b - a + psi_in)
 * i.e. y' = r - K y with y = (a, b), K = (Sigma_t I + c [[1, 1], [-3, 3]]) / sin(theta) and
 * r = (q0 + c psi_in, q1 - 3 c psi_in) / sin(theta): a 2 x 2 matrix-exponential system on every
 * segment. A downward direction is the mirror image xi -> -xi: the same system for (a, -b) with
 * q1 negated, its inflow on the top face.
 *
 * Readings (where the paper is silent; also listed in the design notes):
 *  - the inflow psi_in of a segment in plane i is the segment average of the outflow face trace
 *    (a + b for upward travel) of the same segment in the plane upwind of it, computed earlier in
 *    the same march (Alg. 2: the axial interface source of the next plane is formed after each
 *    plane's ray tracing); flat along the segment, like the flat source;
 *  - axial boundaries: vacuum (no inflow) or reflective. Each (track, sense, polar angle, group)
 *    marches downward first (top plane to bottom), then upward. A reflective bottom feeds the
 *    upward march with the downward march's bottom traces of the same sweep; a reflective top
 *    feeds the downward march with the upward top traces of the previous sweep (lagged like the
 *    radial boundary flux);
 *  - radial boundary flux: both moments of every plane and both marches, routed through the
 *    planar links (a reflection in x-y keeps mu), Jacobi-lagged as in the planar method;
 *  - direction weight 2 pi omega_a w_p delta_a for each of the up and down copies of a polar
 *    angle; the scalar flux moments are phi_m = sum over segments of W * integral of the
 *    m-th coefficient / A_i (A_i the tracked area); the source moments are
 *    q_m = [Sigma_s phi_m + chi/k nuSigma_f phi_m (+ S for m = 0)] / (4 pi);
 *  - fission total F = sum over planes and regions of dz A_i sum_g nuSigma_f phi_0; the residual
 *    is the planar one over (plane, region) elements.
 * The per-segment system is solved from its definition: E = exp(-K l) by scaling and squaring a
 * Taylor series, y_inf = K^{-1} r, y(l) = y_inf + E (y0 - y_inf) and the segment integral
 * l y_inf + K^{-1} (y0 - y(l)).
 * ============================================================================================ */

/* exp(M) of a 2 x 2 matrix (row-major) by scaling and squaring a truncated Taylor series */
void orc_expm2(const double *M, double *E) {
  double nrm = fmax(fabs(M[0]) + fabs(M[1]), fabs(M[2]) + fabs(M[3]));
  int sq = 0;
  while (nrm > 0.25 && sq < 1100) { nrm *= 0.5; ++sq; }
  double A[4];
  double f = ldexp(1.0, -sq);
  for (int i = 0; i < 4; ++i) A[i] = M[i] * f;
  double S[4] = {1.0, 0.0, 0.0, 1.0}, T[4] = {1.0, 0.0, 0.0, 1.0};
  for (int n = 1; n <= 24; ++n) {
    double U[4] = {T[0] * A[0] + T[1] * A[2], T[0] * A[1] + T[1] * A[3],
                   T[2] * A[0] + T[3] * A[2], T[2] * A[1] + T[3] * A[3]};
    for (int i = 0; i < 4; ++i) { T[i] = U[i] / n; S[i] += T[i]; }
  }
  for (int k = 0; k < sq; ++k) {
    double U[4] = {S[0] * S[0] + S[1] * S[2], S[0] * S[1] + S[1] * S[3],
                   S[2] * S[0] + S[3] * S[2], S[2] * S[1] + S[3] * S[3]};
    memcpy(S, U, sizeof U);
  }
  memcpy(E, S, sizeof S);
}

static void solve2(const double *K, const double *v, double *x) {
  double det = K[0] * K[3] - K[1] * K[2];
  x[0] = (K[3] * v[0] - K[1] * v[1]) / det;
  x[1] = (K[0] * v[1] - K[2] * v[0]) / det;
}

/* One segment of one plane: y0 = (a, b) entering (b signed along the march, i.e. -b for a
 * downward march), psi_in the axial inflow, q1s the linear source coefficient with the same
 * sign convention. Returns y at the segment's end and the segment integral of y. */
void orc_dg_segment(const double *y0, double psi_in, double len, double sin_theta, double mu, double h,
                    double sig, double q0, double q1s, double *y1, double *yint) {
  double c = mu / h;
  double K[4] = {(sig + c) / sin_theta, c / sin_theta, -3.0 * c / sin_theta, (sig + 3.0 * c) / sin_theta};
  double r[2] = {(q0 + c * psi_in) / sin_theta, (q1s - 3.0 * c * psi_in) / sin_theta};
  double mK[4] = {-K[0] * len, -K[1] * len, -K[2] * len, -K[3] * len};
  double E[4], yinf[2], d[2], w[2];
  orc_expm2(mK, E);
  solve2(K, r, yinf);
  d[0] = y0[0] - yinf[0];
  d[1] = y0[1] - yinf[1];
  y1[0] = yinf[0] + E[0] * d[0] + E[1] * d[1];
  y1[1] = yinf[1] + E[2] * d[0] + E[3] * d[1];
  double dy[2] = {y0[0] - y1[0], y0[1] - y1[1]};
  solve2(K, dy, w);
  yint[0] = len * yinf[0] + w[0];
  yint[1] = len * yinf[1] + w[1];
}

/* Switch to DGMOC on nz planes (call after orc_set_xs; mat3 [nz][R] or NULL for the planar
 * materials in every plane). The state restarts flat: phi_0 = 1, phi_1 = 0, zero boundary flux. */
int orc_set_axial(orc_t *h, int nz, const double *dz, const int32_t *mat3, int bc_bottom, int bc_top) {
  free(h->dz); free(h->mat3); free(h->phi3); free(h->q3); free(h->tal3); free(h->psi3_in); free(h->psi3_next);
  free(h->ztop); free(h->leak3); free(h->jz); free(h->zleak);
  h->dz = h->phi3 = h->q3 = h->tal3 = h->psi3_in = h->psi3_next = h->ztop = h->leak3 = h->jz = h->zleak = NULL;
  h->mat3 = NULL; h->nz = 0; h->dgcm = 0;
  if (nz <= 0) return 0;
  if (h->cmfd || h->L) { snprintf(h->err, sizeof h->err, "DGMOC with CMFD or anisotropic scattering is not supported"); return -1; }
  if (!h->st) { snprintf(h->err, sizeof h->err, "set_axial before set_xs"); return -1; }
  for (int z = 0; z < nz; ++z)
    if (!(dz[z] > 0.0)) { snprintf(h->err, sizeof h->err, "plane heights must be > 0"); return -1; }
  size_t R = h->n_tri, G = h->G, P = h->n_polar;
  h->mat3 = xcalloc((size_t)nz * R, sizeof(int32_t));
  for (int z = 0; z < nz; ++z)
    for (size_t i = 0; i < R; ++i) {
      int32_t m = mat3 ? mat3[(size_t)z * R + i] : h->mat[i];
      if (m < 0 || m >= h->n_mat) { snprintf(h->err, sizeof h->err, "material id out of range"); free(h->mat3); h->mat3 = NULL; return -1; }
      h->mat3[(size_t)z * R + i] = m;
    }
  h->nz = nz;
  h->bcz[0] = bc_bottom ? 1 : 0;
  h->bcz[1] = bc_top ? 1 : 0;
  h->dz = xcalloc(nz, sizeof(double));
  memcpy(h->dz, dz, nz * sizeof(double));
  size_t n3 = (size_t)nz * R * 2 * G;
  h->phi3 = xcalloc(n3, sizeof(double));
  h->q3 = xcalloc(n3, sizeof(double));
  h->tal3 = xcalloc(n3, sizeof(double));
  size_t nb = (size_t)h->n_tracks * 2 * 2 * nz * P * 2 * G;
  h->psi3_in = xcalloc(nb, sizeof(double));
  h->psi3_next = xcalloc(nb, sizeof(double));
  h->ztop = xcalloc((size_t)h->n_seg * 2 * P * G, sizeof(double));
  h->leak3 = xcalloc(3 * G, sizeof(double));
  h->jz = xcalloc(2 * (size_t)(nz > 1 ? nz - 1 : 1) * G, sizeof(double));
  h->zleak = xcalloc((size_t)nz * G, sizeof(double));
  dg_set_state(h, NULL, 1.0);
  return 0;
}

/* Axial coarse-mesh acceleration of DGMOC (the CMFD step of Alg. 1 with the planes as coarse
 * cells): n_outer coarse power iterations of n_inner over-relaxed (omega) Gauss-Seidel sweeps per
 * group, odd and even planes as the two colours. n_outer = 0 switches it off. */
int orc_set_dg_cmfd(orc_t *h, int n_outer, int n_inner, double omega) {
  h->dgcm = 0;
  if (n_outer <= 0) return 0;
  if (!h->nz) { snprintf(h->err, sizeof h->err, "DGMOC acceleration needs set_axial first"); return -1; }
  if (n_inner <= 0 || !(omega > 0.0 && omega < 2.0)) { snprintf(h->err, sizeof h->err, "bad acceleration parameters"); return -1; }
  h->dgcm = 1; h->dgcm_outer = n_outer; h->dgcm_inner = n_inner; h->dgcm_omega = omega;
  return 0;
}

static void dg_set_state(orc_t *h, const double *phi3, double k) {
  size_t n3 = (size_t)h->nz * h->n_tri * 2 * h->G;
  if (phi3) memcpy(h->phi3, phi3, n3 * sizeof(double));
  else
    for (size_t x = 0; x < n3; ++x) h->phi3[x] = (x / h->G) % 2 == 0 ? 1.0 : 0.0;
  memset(h->psi3_in, 0, (size_t)h->n_tracks * 2 * 2 * h->nz * h->n_polar * 2 * h->G * sizeof(double));
  memset(h->ztop, 0, (size_t)h->n_seg * 2 * h->n_polar * h->G * sizeof(double));
  h->k = k;
}

void orc_get_flux3(const orc_t *h, double *phi3, double *k) {
  if (phi3) memcpy(phi3, h->phi3, (size_t)h->nz * h->n_tri * 2 * h->G * sizeof(double));
  if (k) *k = h->k;
}

void orc_get_leakage3(const orc_t *h, double *l) { memcpy(l, h->leak3, 3 * (size_t)h->G * sizeof(double)); }

static double dg_fission_total(const orc_t *h, const double *phi3) {
  int G = h->G;
  double F = 0.0;
  for (int z = 0; z < h->nz; ++z)
    for (int i = 0; i < h->n_tri; ++i) {
      const double *nf = h->nsf + (size_t)h->mat3[(size_t)z * h->n_tri + i] * G;
      const double *ph = phi3 + ((size_t)z * h->n_tri + i) * 2 * G;
      double f = 0.0;
      for (int g = 0; g < G; ++g) f += nf[g] * ph[g];
      F += h->dz[z] * h->area[i] * f;
    }
  return F;
}

/* source moments of every element */
static void dg_source(orc_t *h, int eigen) {
  int G = h->G;
  for (int z = 0; z < h->nz; ++z)
    for (int i = 0; i < h->n_tri; ++i) {
      int m = h->mat3[(size_t)z * h->n_tri + i];
      size_t e = ((size_t)z * h->n_tri + i) * 2 * G;
      for (int mo = 0; mo < 2; ++mo) {
        const double *ph = h->phi3 + e + (size_t)mo * G;
        double fis = 0.0;
        for (int gp = 0; gp < G; ++gp) fis += h->nsf[(size_t)m * G + gp] * ph[gp];
        for (int g = 0; g < G; ++g) {
          double src = 0.0;
          for (int gp = 0; gp < G; ++gp) src += h->ss[((size_t)m * G + gp) * G + g] * ph[gp];
          if (eigen) src += h->chi[(size_t)m * G + g] / h->k * fis;
          if (mo == 0 && h->ext) src += h->ext[(size_t)i * G + g];
          h->q3[e + (size_t)mo * G + g] = src / (4.0 * ORC_PI);
        }
      }
    }
}

/* One DGMOC sweep: every track, sense, polar angle and group marches down through the planes,
 * then up (Alg. 2), each plane a planar sweep of its segments with the axial inflow of the
 * plane upwind. */
static void dg_sweep(orc_t *h) {
  int G = h->G, P = h->n_polar, nz = h->nz;
  size_t R = h->n_tri;
  memset(h->tal3, 0, (size_t)nz * R * 2 * G * sizeof(double));
  memset(h->psi3_next, 0, (size_t)h->n_tracks * 2 * 2 * nz * P * 2 * G * sizeof(double));
  size_t nif = nz > 1 ? nz - 1 : 1;
  memset(h->jz, 0, 2 * nif * G * sizeof(double));
  memset(h->zleak, 0, (size_t)nz * G * sizeof(double));
  int64_t maxn = 0;
  for (int64_t t = 0; t < h->n_tracks; ++t)
    if (h->seg_off[t + 1] - h->seg_off[t] > maxn) maxn = h->seg_off[t + 1] - h->seg_off[t];
  double *lk = xcalloc(3 * (size_t)G, sizeof(double));
#pragma omp parallel for schedule(static) num_threads(h->n_threads)
  for (int g = 0; g < G; ++g) {
    double *face = xcalloc(maxn ? maxn : 1, sizeof(double));
    for (int64_t t = 0; t < h->n_tracks; ++t) {
      int j = h->track_dir[t];
      int64_t s0 = h->seg_off[t], ns = h->seg_off[t + 1] - s0;
      for (int d = 0; d < 2; ++d)
        for (int p = 0; p < P; ++p) {
          double st = h->sin_theta[p], mu = sqrt(1.0 - st * st);
          double W = 2.0 * ORC_PI * h->omega_a[j] * h->polar_w[p] * h->delta_a[j];
          for (int ud = 0; ud < 2; ++ud) {      /* 0: downward march, 1: upward */
            double sg = ud ? 1.0 : -1.0;        /* sign of xi along the march */
            /* axial inflow of the first plane of the march */
            for (int64_t n = 0; n < ns; ++n) {
              int64_t s = d ? (s0 + ns - 1 - n) : (s0 + n);
              if (ud == 0) face[n] = h->bcz[1] ? h->ztop[((size_t)s * 2 + d) * P * G + (size_t)p * G + g] : 0.0;
              else if (!h->bcz[0]) face[n] = 0.0;   /* reflective bottom: keep the downward traces */
              /* current entering the first plane of the march through the top or bottom face */
              h->zleak[(size_t)(ud ? 0 : nz - 1) * G + g] -= W * mu * h->seg_len[s] * face[n];
            }
            for (int zi = 0; zi < nz; ++zi) {
              int z = ud ? zi : nz - 1 - zi;
              size_t bidx = ((((size_t)(2 * t + d) * 2 + ud) * nz + z) * P + p) * 2 * G;
              double y[2] = {h->psi3_in[bidx + g], h->psi3_in[bidx + G + g]};
              h->zleak[(size_t)z * G + g] -= W * st * h->dz[z] * y[0];   /* radial current in at the start */
              for (int64_t n = 0; n < ns; ++n) {
                int64_t s = d ? (s0 + ns - 1 - n) : (s0 + n);
                int i = h->seg_reg[s];
                int m = h->mat3[(size_t)z * R + i];
                size_t e = ((size_t)z * R + i) * 2 * G;
                double y1[2], yi[2];
                orc_dg_segment(y, face[n], h->seg_len[s], st, mu, h->dz[z], h->st[(size_t)m * G + g],
                               h->q3[e + g], sg * h->q3[e + G + g], y1, yi);
                h->tal3[e + g] += W * yi[0];
                h->tal3[e + G + g] += W * sg * yi[1];
                face[n] = (yi[0] + yi[1]) / h->seg_len[s];   /* outflow face trace, segment average */
                y[0] = y1[0];
                y[1] = y1[1];
              }
              int64_t el = h->link[2 * t + d];
              if (el >= 0) {
                size_t o = ((((size_t)el * 2 + ud) * nz + z) * P + p) * 2 * G;
                h->psi3_next[o + g] = y[0];
                h->psi3_next[o + G + g] = y[1];
              } else {
                lk[g] += W * st * h->dz[z] * y[0];
              }
              h->zleak[(size_t)z * G + g] += W * st * h->dz[z] * y[0];   /* radial current out at the end */
              /* the plane's outflow through its downwind face: into the next plane of the march,
               * or out of the domain */
              double J = 0.0;
              for (int64_t n = 0; n < ns; ++n) {
                int64_t s = d ? (s0 + ns - 1 - n) : (s0 + n);
                J += W * mu * h->seg_len[s] * face[n];
              }
              if (ud == 1 && z < nz - 1) h->jz[(size_t)z * G + g] += J;
              else if (ud == 0 && z > 0) h->jz[(nif + (size_t)(z - 1)) * G + g] += J;
              else h->zleak[(size_t)z * G + g] += J;
            }
            /* the march's last face: bottom (downward) or top (upward) */
            for (int64_t n = 0; n < ns; ++n) {
              int64_t s = d ? (s0 + ns - 1 - n) : (s0 + n);
              double J = W * mu * h->seg_len[s] * face[n];
              if (ud == 0) { if (!h->bcz[0]) lk[(size_t)G + g] += J; }
              else {
                h->ztop[((size_t)s * 2 + d) * P * G + (size_t)p * G + g] = face[n];
                if (!h->bcz[1]) lk[2 * (size_t)G + g] += J;
              }
            }
          }
        }
    }
    free(face);
  }
  memcpy(h->leak3, lk, 3 * (size_t)G * sizeof(double));
  free(lk);
}

/* The coarse step with the planes as coarse cells, on the normalised new moments pn (currents
 * normalised alike): flux-volume homogenisation per plane, coarse balance
 *   (Sigma_t V - Sigma_s,gg V + J_out/phi_z + L_z/phi_z) phi_z
 *     = sum_{g' != g} Sigma_s,g'g V phi_z,g' + chi/k nuSigma_f V phi + J_in from each neighbour
 * with D = J / phi of the current iterate (a fixed point at the transport solution), a fixed
 * number of coarse power iterations (Gauss-Seidel in energy, over-relaxed Gauss-Seidel over the
 * planes, even planes then odd), then both moments of every element, the radial boundary flux of
 * every plane and the stored top traces scaled by their plane's coarse/fine ratio; k = coarse k. */
static void dg_cmfd_step(orc_t *h, double *pn) {
  int G = h->G, nz = h->nz;
  size_t R = h->n_tri, nif = nz > 1 ? nz - 1 : 1;
  double *cphi = xcalloc((size_t)nz * G, sizeof(double)), *TV = xcalloc((size_t)nz * G, sizeof(double));
  double *FV = xcalloc((size_t)nz * G, sizeof(double)), *CH = xcalloc((size_t)nz * G, sizeof(double));
  double *SV = xcalloc((size_t)nz * G * G, sizeof(double)), *V = xcalloc(nz, sizeof(double));
  for (int z = 0; z < nz; ++z)
    for (size_t r = 0; r < R; ++r) {
      int m = h->mat3[(size_t)z * R + r];
      double A = h->area[r] * h->dz[z], f = 0.0;
      const double *ph = pn + ((size_t)z * R + r) * 2 * G;
      V[z] += A;
      for (int g = 0; g < G; ++g) f += h->nsf[(size_t)m * G + g] * ph[g];
      for (int g = 0; g < G; ++g) {
        double a = A * ph[g];
        cphi[(size_t)z * G + g] += a;
        TV[(size_t)z * G + g] += h->st[(size_t)m * G + g] * a;
        FV[(size_t)z * G + g] += h->nsf[(size_t)m * G + g] * a;
        CH[(size_t)z * G + g] += h->chi[(size_t)m * G + g] * A * f;
        for (int gg = 0; gg < G; ++gg) SV[((size_t)z * G + g) * G + gg] += h->ss[((size_t)m * G + g) * G + gg] * a;
      }
    }
  for (int z = 0; z < nz; ++z) {
    double chs = 0.0;
    for (int g = 0; g < G; ++g) chs += CH[(size_t)z * G + g];
    for (int g = 0; g < G; ++g) {
      size_t x = (size_t)z * G + g;
      double raw = cphi[x];
      if (raw > 0.0) {
        TV[x] = TV[x] * V[z] / raw;
        FV[x] = FV[x] * V[z] / raw;
        for (int gg = 0; gg < G; ++gg) SV[x * G + gg] = SV[x * G + gg] * V[z] / raw;
      } else {
        TV[x] = FV[x] = 0.0;
        for (int gg = 0; gg < G; ++gg) SV[x * G + gg] = 0.0;
      }
      cphi[x] = V[z] > 0.0 ? raw / V[z] : 0.0;
      CH[x] = chs > 0.0 ? CH[x] / chs : 0.0;
    }
  }
  const double *jup = h->jz, *jdn = h->jz + nif * G;
  double *diag = xcalloc((size_t)nz * G, sizeof(double)), *phic = xcalloc((size_t)nz * G, sizeof(double));
  double *fis = xcalloc(nz, sizeof(double));
  for (int z = 0; z < nz; ++z)
    for (int g = 0; g < G; ++g) {
      size_t x = (size_t)z * G + g;
      double pz = cphi[x], dg = TV[x] - SV[x * G + g];
      if (pz > 0.0) {
        dg += h->zleak[x] / pz;
        if (z < nz - 1) dg += jup[(size_t)z * G + g] / pz;
        if (z > 0) dg += jdn[(size_t)(z - 1) * G + g] / pz;
      }
      diag[x] = dg;
      phic[x] = pz;
    }
  double kc = h->k;
  for (int it = 0; it < h->dgcm_outer; ++it) {
    double F_old = 0.0;
    for (int z = 0; z < nz; ++z) {
      double f = 0.0;
      for (int g = 0; g < G; ++g) f += FV[(size_t)z * G + g] * phic[(size_t)z * G + g];
      fis[z] = f;
      F_old += f;
    }
    for (int g = 0; g < G; ++g)
      for (int j = 0; j < h->dgcm_inner; ++j)
        for (int c = 0; c < 2; ++c)
          for (int z = c; z < nz; z += 2) {
            size_t x = (size_t)z * G + g;
            double rhs = CH[x] * fis[z] / kc;
            for (int gg = 0; gg < G; ++gg)
              if (gg != g) rhs += SV[((size_t)z * G + gg) * G + g] * phic[(size_t)z * G + gg];
            if (z > 0 && cphi[x - G] > 0.0) rhs += jup[(size_t)(z - 1) * G + g] / cphi[x - G] * phic[x - G];
            if (z < nz - 1 && cphi[x + G] > 0.0) rhs += jdn[(size_t)z * G + g] / cphi[x + G] * phic[x + G];
            if (diag[x] > 0.0) phic[x] += h->dgcm_omega * (rhs / diag[x] - phic[x]);
          }
    double F_new = 0.0;
    for (int z = 0; z < nz; ++z)
      for (int g = 0; g < G; ++g) F_new += FV[(size_t)z * G + g] * phic[(size_t)z * G + g];
    if (F_new > 0.0 && F_old > 0.0) kc = kc * F_new / F_old;
  }
  double *ratio = xcalloc((size_t)nz * G, sizeof(double));
  for (size_t x = 0; x < (size_t)nz * G; ++x) ratio[x] = (cphi[x] > 0.0 && phic[x] > 0.0) ? phic[x] / cphi[x] : 1.0;
  for (int z = 0; z < nz; ++z)
    for (size_t r = 0; r < R; ++r)
      for (int mo = 0; mo < 2; ++mo)
        for (int g = 0; g < G; ++g) pn[(((size_t)z * R + r) * 2 + mo) * G + g] *= ratio[(size_t)z * G + g];
  int P = h->n_polar;
  for (int64_t e = 0; e < 2 * h->n_tracks; ++e)
    for (int ud = 0; ud < 2; ++ud)
      for (int z = 0; z < nz; ++z)
        for (int p = 0; p < P; ++p)
          for (int mo = 0; mo < 2; ++mo)
            for (int g = 0; g < G; ++g)
              h->psi3_next[(((((size_t)e * 2 + ud) * nz + z) * P + p) * 2 + mo) * G + g] *= ratio[(size_t)z * G + g];
  for (size_t x = 0; x < (size_t)h->n_seg * 2 * P * G; ++x) h->ztop[x] *= ratio[(size_t)(nz - 1) * G + x % G];
  h->k = kc;
  free(cphi); free(TV); free(FV); free(CH); free(SV); free(V); free(diag); free(phic); free(fis); free(ratio);
}

static double dg_outer(orc_t *h, int eigen) {
  int G = h->G, nz = h->nz;
  size_t R = h->n_tri, n3 = (size_t)nz * R * 2 * G;
  size_t nb = (size_t)h->n_tracks * 2 * 2 * nz * h->n_polar * 2 * G;
  size_t nt = (size_t)h->n_seg * 2 * h->n_polar * G;
  dg_source(h, eigen);
  dg_sweep(h);
  double *pn = xcalloc(n3, sizeof(double));
  for (int z = 0; z < nz; ++z)
    for (size_t i = 0; i < R; ++i) {
      int m = h->mat3[(size_t)z * R + i];
      size_t e = ((size_t)z * R + i) * 2 * G;
      for (int mo = 0; mo < 2; ++mo)
        for (int g = 0; g < G; ++g) {
          size_t x = e + (size_t)mo * G + g;
          pn[x] = h->area[i] > 0.0 ? h->tal3[x] / h->area[i] : 4.0 * ORC_PI * h->q3[x] / h->st[(size_t)m * G + g];
        }
    }
  double resid = 0.0;
  if (eigen) {
    double F_old = dg_fission_total(h, h->phi3), F_new = dg_fission_total(h, pn);
    h->k = h->k * F_new / F_old;
    for (size_t x = 0; x < n3; ++x) pn[x] /= F_new;
    for (size_t x = 0; x < nb; ++x) h->psi3_next[x] /= F_new;
    for (size_t x = 0; x < nt; ++x) h->ztop[x] /= F_new;
    for (int x = 0; x < 3 * G; ++x) h->leak3[x] /= F_new;
    for (size_t x = 0; x < 2 * (size_t)(nz > 1 ? nz - 1 : 1) * G; ++x) h->jz[x] /= F_new;
    for (size_t x = 0; x < (size_t)nz * G; ++x) h->zleak[x] /= F_new;
    for (int z = 0; z < nz; ++z)
      for (size_t i = 0; i < R; ++i) {
        const double *nf = h->nsf + (size_t)h->mat3[(size_t)z * R + i] * G;
        size_t e = ((size_t)z * R + i) * 2 * G;
        double fo = 0.0, fn = 0.0;
        for (int g = 0; g < G; ++g) { fo += nf[g] * h->phi3[e + g] / F_old; fn += nf[g] * pn[e + g]; }
        if (fn > 0.0) { double r = fabs(fn - fo) / fn; if (r > resid) resid = r; }
      }
    if (h->dgcm) {
      dg_cmfd_step(h, pn);
      double F2 = dg_fission_total(h, pn);
      for (size_t x = 0; x < n3; ++x) pn[x] /= F2;
      for (size_t x = 0; x < nb; ++x) h->psi3_next[x] /= F2;
      for (size_t x = 0; x < nt; ++x) h->ztop[x] /= F2;
    }
  } else {
    for (int z = 0; z < nz; ++z)
      for (size_t i = 0; i < R; ++i)
        for (int g = 0; g < G; ++g) {
          size_t x = ((size_t)z * R + i) * 2 * G + g;
          if (pn[x] > 0.0) { double r = fabs(pn[x] - h->phi3[x]) / pn[x]; if (r > resid) resid = r; }
        }
  }
  memcpy(h->phi3, pn, n3 * sizeof(double));
  free(pn);
  double *tmp = h->psi3_in; h->psi3_in = h->psi3_next; h->psi3_next = tmp;
  return resid;
}

/* One flat-source characteristic along a sequence of segments, one group and polar angle:
 * returns psi after each segment (used to pin Eq. MOC_sol against the exact path integral). */
void orc_track_sweep(int n, const double *sig, const double *qr, const double *len, double sin_theta,
                     double psi_in, double *psi_after) {
  double psi = psi_in;
  for (int k = 0; k < n; ++k) {
    double tau = sig[k] * len[k] / sin_theta;
    psi -= (psi - qr[k]) * (-expm1(-tau));
    psi_after[k] = psi;
  }
}

/* ------------------------------------------------------------------ sampled regions ---- */
/* Scalar flux after one fixed-source outer (Q from phi0 and S, one sweep from psi0) for a sample of
 * regions, without segmenting the whole problem: only rays crossing a sampled region are laid down
 * and clipped (same laydown, clipping and weights as above, restated for a subset). For a
 * rectangular mesh the ray index equals the track index of the full track list, so psi0 is indexed
 * [ray][2][P][G]. A mesh that does not fill its box (non-rectangular, or with holes) is accepted
 * when every wall is vacuum: each maximal in-mesh chord of a ray is then a track with zero inflow
 * (the reading of Sec. 3.1's modular rays on such meshes used throughout) and psi0 is not read.
 * Returns 0 on success, -2 for a gap along a ray when some wall is reflective. */
typedef struct { double cmin, cmax; int t; } proj_t;
static int cmp_proj(const void *a, const void *b) {
  const proj_t *x = a, *y = b;
  if (x->cmin != y->cmin) return (x->cmin < y->cmin) ? -1 : 1;
  return (x->t < y->t) ? -1 : (x->t > y->t);
}

int orc_sample_fixed_source(int n_vert, const double *xy, int n_tri, const int32_t *tri, const int32_t *mat,
                            const double *bbox, const int32_t *bc, int n_azim, double spacing, int n_polar, const double *sin_theta,
                            const double *polar_w, int n_mat, int G, const double *st, const double *ss,
                            const double *S, const double *phi0, const double *psi0, int n_sample,
                            const int32_t *sample, double *phi_out, double *area_out) {
  orc_t h0;
  memset(&h0, 0, sizeof h0);
  orc_t *h = &h0;
  h->n_vert = n_vert; h->n_tri = n_tri; h->xy = (double *)xy; h->tri = (int32_t *)tri; h->mat = (int32_t *)mat;
  h->xmin = bbox[0]; h->xmax = bbox[1]; h->ymin = bbox[2]; h->ymax = bbox[3];
  h->n_azim = n_azim; h->n_polar = n_polar;
  if (build_quadrature(h, spacing)) return -1;
  double W = h->xmax - h->xmin, H = h->ymax - h->ymin;
  const int allvac = bc[0] == 0 && bc[1] == 0 && bc[2] == 0 && bc[3] == 0;
  /* sample lookup */
  int *slot = xcalloc(n_tri, sizeof(int));
  for (int i = 0; i < n_tri; ++i) slot[i] = -1;
  for (int q = 0; q < n_sample; ++q) slot[sample[q]] = q;
  double *tal = xcalloc((size_t)n_sample * G, sizeof(double));
  double *area = xcalloc(n_sample, sizeof(double));
  /* directions run in parallel, each into its own tally; the partial tallies are summed in
   * direction order afterwards, so the result does not depend on the thread count */
  int64_t *base = xcalloc(h->n_dir + 1, sizeof(int64_t));
  for (int j = 0; j < h->n_dir; ++j) base[j + 1] = base[j] + h->nx_a[j] + h->ny_a[j];
  double *tal_d = xcalloc((size_t)h->n_dir * n_sample * G, sizeof(double));
  double *area_d = xcalloc((size_t)h->n_dir * n_sample, sizeof(double));
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < h->n_dir; ++j) {
    double *tal_j = tal_d + (size_t)j * n_sample * G, *area_j = area_d + (size_t)j * n_sample;
    int64_t ray_base = base[j];
    double ph = h->phi_a[j], u[2] = {cos(ph), sin(ph)}, nrm[2] = {-sin(ph), cos(ph)};
    int nx = h->nx_a[j], ny = h->ny_a[j], nr = nx + ny;
    /* offsets of all rays of this direction, and which rays cross a sampled region */
    double *p0 = xcalloc(2 * (size_t)nr, sizeof(double));
    for (int i = 0; i < nx; ++i) { p0[2 * i] = h->xmin + (i + 0.5) * W / nx; p0[2 * i + 1] = h->ymin; }
    for (int i = 0; i < ny; ++i) { p0[2 * (nx + i)] = (u[0] > 0) ? h->xmin : h->xmax; p0[2 * (nx + i) + 1] = h->ymin + (i + 0.5) * H / ny; }
    char *need = xcalloc(nr, 1);
    for (int q = 0; q < n_sample; ++q) {
      int t = sample[q];
      double cmin = INFINITY, cmax = -INFINITY;
      for (int k = 0; k < 3; ++k) {
        const double *v = xy + 2 * (int64_t)tri[3 * t + k];
        double c = nrm[0] * v[0] + nrm[1] * v[1];
        if (c < cmin) cmin = c;
        if (c > cmax) cmax = c;
      }
      for (int r = 0; r < nr; ++r) {
        double c = nrm[0] * p0[2 * r] + nrm[1] * p0[2 * r + 1];
        if (c >= cmin && c <= cmax) need[r] = 1;
      }
    }
    /* triangle projection intervals of this direction, sorted, for the per-ray candidate search */
    proj_t *pj = xcalloc(n_tri, sizeof(proj_t));
    double wmax = 0.0;
    for (int t = 0; t < n_tri; ++t) {
      double cmin = INFINITY, cmax = -INFINITY;
      for (int k = 0; k < 3; ++k) {
        const double *v = xy + 2 * (int64_t)tri[3 * t + k];
        double cc = nrm[0] * v[0] + nrm[1] * v[1];
        if (cc < cmin) cmin = cc;
        if (cc > cmax) cmax = cc;
      }
      /* rounding margin, as in build_tracks */
      pj[t].cmin = cmin - 1e-9 * fmax(h->xmax - h->xmin, h->ymax - h->ymin);
      pj[t].cmax = cmax + 1e-9 * fmax(h->xmax - h->xmin, h->ymax - h->ymin);
      pj[t].t = t;
      if (cmax - cmin > wmax) wmax = cmax - cmin;
    }
    qsort(pj, n_tri, sizeof(proj_t), cmp_proj);
    for (int r = 0; r < nr; ++r) {
      if (!need[r]) continue;
      double c = nrm[0] * p0[2 * r] + nrm[1] * p0[2 * r + 1];
      double L = box_exit(h, p0 + 2 * r, u);
      int cap = 64, cnt = 0;
      piece_t *pc = xcalloc(cap, sizeof(piece_t));
      int lo = 0, hi = n_tri;
      while (lo < hi) { int m = (lo + hi) / 2; if (pj[m].cmin < c - wmax) lo = m + 1; else hi = m; }
      for (int q2 = lo; q2 < n_tri && pj[q2].cmin <= c; ++q2) {
        if (pj[q2].cmax < c) continue;
        int t = pj[q2].t;
        double s0, s1;
        if (!clip_triangle(xy, tri, t, p0 + 2 * r, u, L, &s0, &s1)) continue;
        if (s1 - s0 < 1e-12) continue;
        if (cnt == cap) { cap *= 2; pc = realloc(pc, cap * sizeof(piece_t)); if (!pc) abort(); }
        pc[cnt].s0 = s0; pc[cnt].s1 = s1; pc[cnt].tri = t; cnt++;
      }
      qsort(pc, cnt, sizeof(piece_t), cmp_piece);
      /* brk[k]: a gap precedes piece k, so piece k starts a new chord of this ray. Each maximal
       * in-mesh chord is its own track with vacuum inflow (the exterior absorbs); that is only
       * consistent with the caller's psi0 (one track per ray) when every wall is vacuum */
      char *brk = xcalloc(cnt + 1, 1);
      for (int k = 1; k < cnt; ++k)
        if (pc[k].s0 - pc[k - 1].s1 > 1e-9) {
          brk[k] = 1;
          if (!allvac) fail = 1;   /* a gap in a mesh with a reflective wall: not supported */
        }
      int64_t tr = ray_base + r;
      for (int d = 0; d < 2; ++d) {
        /* entry point of this sense; inflow through a vacuum wall is zero */
        double ex = d ? p0[2 * r] + L * u[0] : p0[2 * r], ey = d ? p0[2 * r + 1] + L * u[1] : p0[2 * r + 1];
        int w = wall_of(h, ex, ey, 1e-9 * fmax(W, H));
        int vac = allvac || (w >= 0 && bc[w] == 0);
        for (int p = 0; p < n_polar; ++p) {
          double Wt = 4.0 * ORC_PI * h->omega_a[j] * polar_w[p] * h->delta_a[j] * sin_theta[p];
          for (int g = 0; g < G; ++g) {
            double psi = vac ? 0.0 : psi0[((size_t)(2 * tr + d) * n_polar + p) * G + g];
            for (int n = 0; n < cnt; ++n) {
              int k = d ? (cnt - 1 - n) : n;
              /* entering a new chord (backward travel crosses the gap after piece k) */
              if (n > 0 && (d ? brk[k + 1] : brk[k])) psi = 0.0;
              int i = pc[k].tri, m = mat[i];
              double sig = st[(size_t)m * G + g];
              /* Eq. MGNTE_element source of region i from phi0 (fixed source, no fission) */
              double sc = 0.0;
              for (int gp = 0; gp < G; ++gp) sc += ss[((size_t)m * G + gp) * G + g] * phi0[(size_t)i * G + gp];
              double qi = (sc + S[(size_t)i * G + g]) / (4.0 * ORC_PI);
              double len = pc[k].s1 - pc[k].s0;
              double delta = (psi - qi / sig) * (-expm1(-sig * len / sin_theta[p]));
              if (slot[i] >= 0) tal_j[(size_t)slot[i] * G + g] += Wt * delta;
              psi -= delta;
            }
          }
        }
      }
      for (int n = 0; n < cnt; ++n)
        if (slot[pc[n].tri] >= 0) area_j[slot[pc[n].tri]] += 2.0 * h->omega_a[j] * h->delta_a[j] * (pc[n].s1 - pc[n].s0);
      free(brk);
      free(pc);
    }
    free(pj);
    free(need);
    free(p0);
  }
  for (int j = 0; j < h->n_dir; ++j) {
    for (size_t q = 0; q < (size_t)n_sample * G; ++q) tal[q] += tal_d[(size_t)j * n_sample * G + q];
    for (int q = 0; q < n_sample; ++q) area[q] += area_d[(size_t)j * n_sample + q];
  }
  free(tal_d); free(area_d); free(base);
  if (fail) { free(h->phi_a); free(h->delta_a); free(h->omega_a); free(h->nx_a); free(h->ny_a); free(slot); free(tal); free(area); return -2; }
  for (int q = 0; q < n_sample; ++q) {
    int i = sample[q], m = mat[i];
    area_out[q] = area[q];
    for (int g = 0; g < G; ++g) {
      double sig = st[(size_t)m * G + g], sc = 0.0;
      for (int gp = 0; gp < G; ++gp) sc += ss[((size_t)m * G + gp) * G + g] * phi0[(size_t)i * G + gp];
      double qi = (sc + S[(size_t)i * G + g]) / (4.0 * ORC_PI);
      double v = 4.0 * ORC_PI * qi / sig;
      if (area[q] > 0.0) v += tal[(size_t)q * G + g] / (sig * area[q]);
      phi_out[(size_t)q * G + g] = v;
    }
  }
  free(h->phi_a); free(h->delta_a); free(h->omega_a); free(h->nx_a); free(h->ny_a);
  free(slot); free(tal); free(area);
  return 0;
}
