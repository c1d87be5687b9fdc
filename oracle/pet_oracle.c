/*
 * FP64 CPU oracle for RDP-regularised PET reconstruction with preconditioned
 * stochastic gradients (Ehrhardt, Kereta, Schramm, "Fast PET Reconstruction with
 * Variance Reduction and Prior-Aware Preconditioning").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow and written to be checked
 * against the paper by eye.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the product path never does.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every quantity is double precision.  Loops follow the definitions literally:
 * no blocking, fusion or reordering beyond what the definitions state.
 *
 * Parity status: every function below is pinned by the "not gpu" tests
 * (adjointness, closed-form line integrals, dense-matrix transpose, TOF partition
 * of unity, KL identities, RDP finite differences and homogeneity, MLEM identity
 * and monotonicity, estimator special cases, KKT at convergence, Table 1).  The
 * NRMSE normalisation (Sec. 3.1) is a reading, not a derived quantity, and is
 * marked "parity unpinned" in its own comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Scanner / image description (problem statement Sec. 1.1, eq. 1; simulation  */
/* setup Sec. 3.1).  Image voxel (ix,iy,iz) is stored at (iz*ny+iy)*nx+ix and  */
/* its centre is ((i-(n-1)/2)*d) per axis.  Sinogram bin (v,p,r,b) is stored   */
/* at ((v*nplane+p)*nrad+r)*ntof+b.                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  int nrad, nview, nplane, ntof;
  double drad, rdet;
  const double *z1, *z2; /* per plane: axial position (mm) of endpoint 1 and 2 */
  double tof_sigma;      /* TOF Gaussian sigma along the LOR (mm) */
  double tof_bin;        /* TOF bin width (mm) */
  double res_fwhm;       /* image-space Gaussian resolution model, FWHM (mm); 0 = none */
} og_geom;

/* ------------------------------------------------------------------------- */
/* Image-space resolution model (Sec. 3.1: an isotropic Gaussian kernel of     */
/* 4 mm models the limited spatial resolution): P is replaced by P G, where G  */
/* convolves with a Gaussian of the given FWHM, sigma = FWHM / (2 sqrt(2 ln 2)). */
/* Per axis the kernel is sampled at the voxel offsets k*delta, |k| <= R =     */
/* ceil(3 sigma / delta), and normalised to unit sum; voxels outside the image */
/* count as zero.  The axial pass is skipped for single-slice images.  With a  */
/* symmetric kernel and zero padding, G is its own adjoint, so the            */
/* backprojector applies the same G after P^T.                                 */
/* ------------------------------------------------------------------------- */
static int gauss_taps(double fwhm, double delta, double *w) {
  double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  int R = (int)ceil(3.0 * sigma / delta);
  double sum = 0.0;
  for (int k = -R; k <= R; k++) {
    w[k + R] = exp(-(k * delta) * (k * delta) / (2.0 * sigma * sigma));
    sum += w[k + R];
  }
  for (int k = 0; k <= 2 * R; k++) w[k] /= sum;
  return R;
}

/* out = G in (out may not alias in). */
void o_gauss_filter(int nx, int ny, int nz, double dx, double dy, double dz, double fwhm,
                    const double *in, double *out) {
  size_t N = (size_t)nx * ny * nz;
  if (!(fwhm > 0)) { memcpy(out, in, sizeof(double) * N); return; }
  int n[3] = {nx, ny, nz};
  double del[3] = {dx, dy, dz};
  size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
  double *a = malloc(sizeof(double) * N), *b = malloc(sizeof(double) * N);
  memcpy(a, in, sizeof(double) * N);
  for (int ax = 0; ax < 3; ax++) {
    if (ax == 2 && nz == 1) continue;
    int Rmax = (int)ceil(3.0 * fwhm / (2.0 * sqrt(2.0 * log(2.0))) / del[ax]);
    double *w = malloc(sizeof(double) * (2 * Rmax + 1));
    int R = gauss_taps(fwhm, del[ax], w);
    for (int iz = 0; iz < nz; iz++)
      for (int iy = 0; iy < ny; iy++)
        for (int ix = 0; ix < nx; ix++) {
          int i3[3] = {ix, iy, iz};
          size_t c = (size_t)iz * stride[2] + (size_t)iy * stride[1] + ix;
          double acc = 0.0;
          for (int k = -R; k <= R; k++) {
            int j = i3[ax] + k;
            if (j < 0 || j >= n[ax]) continue;
            acc += w[k + R] * a[c + (long)k * (long)stride[ax]];
          }
          b[c] = acc;
        }
    free(w);
    double *t = a; a = b; b = t;
  }
  memcpy(out, a, sizeof(double) * N);
  free(a); free(b);
}

/* x itself, or G x in a new buffer (to be freed) when the geometry has a resolution model. */
static const double *resolved_input(const og_geom *g, const double *x, double **owned) {
  *owned = NULL;
  if (!(g->res_fwhm > 0)) return x;
  size_t N = (size_t)g->nx * g->ny * g->nz;
  *owned = malloc(sizeof(double) * N);
  o_gauss_filter(g->nx, g->ny, g->nz, g->dx, g->dy, g->dz, g->res_fwhm, x, *owned);
  return *owned;
}

/* LOR endpoints on the detector cylinder.  View v has angle v*pi/V, radial bin r
 * sits at signed distance s=(r-(R-1)/2)*drad from the axis, the in-plane
 * direction is u=(-sin phi, cos phi), endpoint 1 is the "minus u" end. */
static void lor_endpoints(const og_geom *g, int v, int p, int r, double e1[3], double e2[3]) {
  double phi = (double)v * M_PI / (double)g->nview;
  double c = cos(phi), s = sin(phi);
  double sr = ((double)r - 0.5 * (double)(g->nrad - 1)) * g->drad;
  double h = sqrt(g->rdet * g->rdet - sr * sr);
  double mx = sr * c, my = sr * s;
  double ux = -s, uy = c;
  e1[0] = mx - h * ux;
  e1[1] = my - h * uy;
  e1[2] = g->z1[p];
  e2[0] = mx + h * ux;
  e2[1] = my + h * uy;
  e2[2] = g->z2[p];
}

/* Driving axis of a view: the in-plane axis k maximising |u_k|/delta_k.  For
 * square pixels this is an exact integer test on the view index (an exact 45
 * degree view drives along x); otherwise a direct comparison. */
int o_driving_axis(const og_geom *g, int v) {
  if (g->dx == g->dy) {
    int V = g->nview;
    return (4 * v >= V && 4 * v <= 3 * V) ? 0 : 1;
  }
  double phi = (double)v * M_PI / (double)g->nview;
  return fabs(sin(phi)) * g->dy >= fabs(cos(phi)) * g->dx ? 0 : 1;
}

/* Joseph's method: for every voxel-centre plane along the driving axis,
 * intersect the LOR and bilinearly interpolate in the two other axes; a
 * neighbour outside the image counts as zero.  Each sample is weighted by the
 * ray length between consecutive planes.  Writes one entry per in-image
 * neighbour: voxel index, weight (interpolation weight x step length, mm) and
 * the sample position t along the LOR, measured from the LOR midpoint towards
 * endpoint 2 (mm).  Returns the number of entries, or -1 if the axial axis would
 * drive the ray (not supported by this geometry). */
int o_lor_entries(const og_geom *g, int v, int p, int r, int *vox, double *wt, double *tpos) {
  double e1[3], e2[3];
  lor_endpoints(g, v, p, r, e1, e2);
  double d[3] = {e2[0] - e1[0], e2[1] - e1[1], e2[2] - e1[2]};
  double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  int n[3] = {g->nx, g->ny, g->nz};
  double del[3] = {g->dx, g->dy, g->dz};
  int k = o_driving_axis(g, v);
  if (fabs(d[2]) / del[2] > fabs(d[k]) / del[k]) return -1;
  int a = (k == 0) ? 1 : 0; /* transverse in-plane axis */
  int b = 2;                /* axial axis */
  double step = del[k] * len / fabs(d[k]);
  int ne = 0;
  for (int i = 0; i < n[k]; i++) {
    double ck = ((double)i - 0.5 * (double)(n[k] - 1)) * del[k];
    double lam = (ck - e1[k]) / d[k];
    double pa = e1[a] + lam * d[a];
    double pb = e1[b] + lam * d[b];
    double fa = pa / del[a] + 0.5 * (double)(n[a] - 1);
    double fb = pb / del[b] + 0.5 * (double)(n[b] - 1);
    double fa0 = floor(fa), fb0 = floor(fb);
    double wa = fa - fa0, wb = fb - fb0;
    double t = (lam - 0.5) * len;
    for (int ja = 0; ja < 2; ja++) {
      for (int jb = 0; jb < 2; jb++) {
        double ia = fa0 + ja, ib = fb0 + jb;
        if (ia < 0 || ia >= n[a] || ib < 0 || ib >= n[b]) continue;
        double w = (ja ? wa : 1.0 - wa) * (jb ? wb : 1.0 - wb);
        if (w == 0.0) continue;
        int idx[3];
        idx[k] = i;
        idx[a] = (int)ia;
        idx[b] = (int)ib;
        vox[ne] = (idx[2] * g->ny + idx[1]) * g->nx + idx[0];
        wt[ne] = w * step;
        tpos[ne] = t;
        ne++;
      }
    }
  }
  return ne;
}

/* TOF bin weight of a point at position t on the LOR: the mass that a Gaussian
 * of standard deviation sigma centred at t, truncated at +-3 sigma and
 * renormalised, puts into bin b = [c_b - w/2, c_b + w/2], c_b = (b-(T-1)/2)*w.
 * The truncation is a reading (the paper only gives the 390 ps resolution); it
 * keeps the weight continuous in t and exactly zero beyond 3 sigma + w/2. */
double o_tof_weight(const og_geom *g, int b, double t) {
  double amax = 3.0 / sqrt(2.0);
  double cb = ((double)b - 0.5 * (double)(g->ntof - 1)) * g->tof_bin;
  double uhi = (cb + 0.5 * g->tof_bin - t) / (sqrt(2.0) * g->tof_sigma);
  double ulo = (cb - 0.5 * g->tof_bin - t) / (sqrt(2.0) * g->tof_sigma);
  if (uhi > amax) uhi = amax;
  if (uhi < -amax) uhi = -amax;
  if (ulo > amax) ulo = amax;
  if (ulo < -amax) ulo = -amax;
  return (erf(uhi) - erf(ulo)) / (2.0 * erf(amax));
}

static int max_entries(const og_geom *g) {
  int m = g->nx > g->ny ? g->nx : g->ny;
  if (g->nz > m) m = g->nz;
  return 4 * m + 4;
}

/* Views of subset s (0-based) out of n: every n-th view, s, s+n, ... (Sec. 3.1). */
int o_subset_views(int nview, int nsub, int s, int *views) {
  int c = 0;
  for (int v = s; v < nview; v += nsub) views[c++] = v;
  return c;
}

/* Geometric projection P x over the listed views (no multiplicative factors):
 * out[j][p][r][b] for j over the listed views. Returns 0 or -1 (bad geometry). */
int o_project(const og_geom *g, const int *views, int nviews, const double *x_in, double *out) {
  double *owned;
  const double *x = resolved_input(g, x_in, &owned);
  int me = max_entries(g);
  int *vox = malloc(sizeof(int) * me);
  double *wt = malloc(sizeof(double) * me), *tp = malloc(sizeof(double) * me);
  int T = g->ntof > 1 ? g->ntof : 1;
  int rc = 0;
  for (int j = 0; j < nviews; j++)
    for (int p = 0; p < g->nplane; p++)
      for (int r = 0; r < g->nrad; r++) {
        double *o = out + (((size_t)j * g->nplane + p) * g->nrad + r) * T;
        int ne = o_lor_entries(g, views[j], p, r, vox, wt, tp);
        if (ne < 0) { rc = -1; ne = 0; }
        for (int b = 0; b < T; b++) {
          double acc = 0.0;
          for (int e = 0; e < ne; e++) {
            double tw = (T > 1) ? o_tof_weight(g, b, tp[e]) : 1.0;
            acc += wt[e] * tw * x[vox[e]];
          }
          o[b] = acc;
        }
      }
  free(vox); free(wt); free(tp); free(owned);
  return rc;
}

/* Geometric projection of an explicit list of LORs (v, p, r triples): out[l][b]. */
int o_project_lors(const og_geom *g, const int *vpr, int nl, const double *x_in, double *out) {
  double *owned;
  const double *x = resolved_input(g, x_in, &owned);
  int me = max_entries(g);
  int *vox = malloc(sizeof(int) * me);
  double *wt = malloc(sizeof(double) * me), *tp = malloc(sizeof(double) * me);
  int T = g->ntof > 1 ? g->ntof : 1;
  int rc = 0;
  for (int l = 0; l < nl; l++) {
    int ne = o_lor_entries(g, vpr[3 * l], vpr[3 * l + 1], vpr[3 * l + 2], vox, wt, tp);
    if (ne < 0) { rc = -1; ne = 0; }
    for (int b = 0; b < T; b++) {
      double acc = 0.0;
      for (int e = 0; e < ne; e++) {
        double tw = (T > 1) ? o_tof_weight(g, b, tp[e]) : 1.0;
        acc += wt[e] * tw * x[vox[e]];
      }
      out[(size_t)l * T + b] = acc;
    }
  }
  free(vox); free(wt); free(tp); free(owned);
  return rc;
}

/* Literal transpose of o_project: img = P^T q (img is overwritten). */
int o_backproject(const og_geom *g, const int *views, int nviews, const double *q, double *img) {
  int me = max_entries(g);
  int *vox = malloc(sizeof(int) * me);
  double *wt = malloc(sizeof(double) * me), *tp = malloc(sizeof(double) * me);
  int T = g->ntof > 1 ? g->ntof : 1;
  size_t N = (size_t)g->nx * g->ny * g->nz;
  memset(img, 0, sizeof(double) * N);
  int rc = 0;
  for (int j = 0; j < nviews; j++)
    for (int p = 0; p < g->nplane; p++)
      for (int r = 0; r < g->nrad; r++) {
        const double *qq = q + (((size_t)j * g->nplane + p) * g->nrad + r) * T;
        int ne = o_lor_entries(g, views[j], p, r, vox, wt, tp);
        if (ne < 0) { rc = -1; ne = 0; }
        for (int e = 0; e < ne; e++)
          for (int b = 0; b < T; b++) {
            double tw = (T > 1) ? o_tof_weight(g, b, tp[e]) : 1.0;
            img[vox[e]] += wt[e] * tw * qq[b];
          }
      }
  if (g->res_fwhm > 0) { /* (P G)^T = G P^T */
    double *t = malloc(sizeof(double) * N);
    o_gauss_filter(g->nx, g->ny, g->nz, g->dx, g->dy, g->dz, g->res_fwhm, img, t);
    memcpy(img, t, sizeof(double) * N);
    free(t);
  }
  free(vox); free(wt); free(tp);
  return rc;
}

/* Multiplicative factors m = sens * exp(-P_nonTOF mu) for every LOR of the full
 * sinogram, [V][P][R] (forward model A includes sensitivities and attenuation,
 * Sec. 1.1; water attenuation, Sec. 3.1).  sens may be NULL (= 1), mu may be
 * NULL (no attenuation). */
int o_multiplicative(const og_geom *g, const double *mu, const double *sens, double *m) {
  size_t nl = (size_t)g->nview * g->nplane * g->nrad;
  og_geom g1 = *g;
  g1.ntof = 1;
  g1.res_fwhm = 0.0; /* attenuation: line integrals of mu through the object itself */
  int rc = 0;
  if (mu) {
    int *views = malloc(sizeof(int) * g->nview);
    for (int v = 0; v < g->nview; v++) views[v] = v;
    rc = o_project(&g1, views, g->nview, mu, m);
    free(views);
    for (size_t l = 0; l < nl; l++) m[l] = exp(-m[l]);
  } else {
    for (size_t l = 0; l < nl; l++) m[l] = 1.0;
  }
  if (sens)
    for (size_t l = 0; l < nl; l++) m[l] *= sens[l];
  return rc;
}

/* KL data term d(s,t) of Sec. 1.2. */
double o_kl_term(double s, double t) {
  if (t > 0 && s > 0) return s - t + t * log(t / s);
  if (t == 0 && s >= 0) return s;
  return INFINITY;
}

/* Subset data term D_s(x) = sum_{j in S_s} d(A_j x + r_j, y_j) and its gradient
 * A_s^T (1 - y/(A_s x + r)) (eq. 2 and the definition of f_i in eq. 5).  A = m P.
 * m: [V][P][R], r and y: full sinogram [V][P][R][T].  s = -1 means all views.
 * grad (may be NULL) is overwritten.  Returns the data term value. */
double o_data_grad(const og_geom *g, int nsub, int s, const double *x, const double *m,
                   const double *rr, const double *y, double *grad) {
  int T = g->ntof > 1 ? g->ntof : 1;
  int *views = malloc(sizeof(int) * g->nview);
  int nv = (s < 0) ? o_subset_views(g->nview, 1, 0, views) : o_subset_views(g->nview, nsub, s, views);
  size_t per_view = (size_t)g->nplane * g->nrad * T;
  double *px = malloc(sizeof(double) * nv * per_view);
  double *q = malloc(sizeof(double) * nv * per_view);
  o_project(g, views, nv, x, px);
  double val = 0.0;
  for (int j = 0; j < nv; j++)
    for (int p = 0; p < g->nplane; p++)
      for (int r = 0; r < g->nrad; r++) {
        size_t lor = ((size_t)views[j] * g->nplane + p) * g->nrad + r;
        size_t loc = ((size_t)j * g->nplane + p) * g->nrad + r;
        for (int b = 0; b < T; b++) {
          double ybar = m[lor] * px[loc * T + b] + rr[lor * T + b];
          double yy = y[lor * T + b];
          val += o_kl_term(ybar, yy);
          /* d/ds d(s,t) = 1 - t/s for t > 0 and d/ds d(s,0) = 1 (d(s,0) = s, also at
             s = 0); chain rule through A = m P */
          q[loc * T + b] = m[lor] * (yy > 0 ? 1.0 - yy / ybar : 1.0);
        }
      }
  if (grad) o_backproject(g, views, nv, q, grad);
  free(views); free(px); free(q);
  return val;
}

/* The same data term and gradient (eq. 5, KL of Sec. 1.2) over an explicit list of
 * views whose data are given in compact layout: m_c [j][P][R], r_c and y_c
 * [j][P][R][T] for j over the listed views.  With the plane list of g restricted to a
 * subset of the scanner's planes this evaluates the share of those LORs, so a large
 * subset can be split into pieces whose values and gradients add up.  grad (may be
 * NULL) is overwritten.  Returns the data term value, or NAN if a LOR cannot be
 * represented (axial driving axis). */
double o_data_grad_views(const og_geom *g, const int *views, int nv, const double *x, const double *m_c,
                         const double *r_c, const double *y_c, double *grad) {
  int T = g->ntof > 1 ? g->ntof : 1;
  size_t nl = (size_t)nv * g->nplane * g->nrad;
  double *px = malloc(sizeof(double) * nl * T);
  double *q = malloc(sizeof(double) * nl * T);
  int rc = o_project(g, views, nv, x, px);
  double val = 0.0;
  for (size_t l = 0; l < nl; l++)
    for (int b = 0; b < T; b++) {
      double ybar = m_c[l] * px[l * T + b] + r_c[l * T + b];
      double yy = y_c[l * T + b];
      val += o_kl_term(ybar, yy);
      q[l * T + b] = m_c[l] * (yy > 0 ? 1.0 - yy / ybar : 1.0);
    }
  if (grad && o_backproject(g, views, nv, q, grad) != 0) rc = -1;
  free(px); free(q);
  return rc == 0 ? val : NAN;
}

/* Sensitivity A_s^T 1 (all TOF bins) for subset s (s=-1: all views). */
void o_sensitivity(const og_geom *g, int nsub, int s, const double *m, double *sens_img) {
  int T = g->ntof > 1 ? g->ntof : 1;
  int *views = malloc(sizeof(int) * g->nview);
  int nv = (s < 0) ? o_subset_views(g->nview, 1, 0, views) : o_subset_views(g->nview, nsub, s, views);
  size_t per_view = (size_t)g->nplane * g->nrad * T;
  double *q = malloc(sizeof(double) * nv * per_view);
  for (int j = 0; j < nv; j++)
    for (int p = 0; p < g->nplane; p++)
      for (int r = 0; r < g->nrad; r++) {
        size_t lor = ((size_t)views[j] * g->nplane + p) * g->nrad + r;
        size_t loc = ((size_t)j * g->nplane + p) * g->nrad + r;
        for (int b = 0; b < T; b++) q[loc * T + b] = m[lor];
      }
  o_backproject(g, views, nv, q, sens_img);
  free(views); free(q);
}

/* ------------------------------------------------------------------------- */
/* Relative difference prior, eq. 3, with derivatives from Appendix A.1.       */
/* Neighbourhood: the 26 voxels around i (8 in-plane when nz = 1); neighbours  */
/* outside the image are omitted.  w_ij = min(d)/||o*d|| for integer offset o. */
/* kappa may be NULL (= 1).                                                    */
/* ------------------------------------------------------------------------- */
static double rdp_weight(int ox, int oy, int oz, double dx, double dy, double dz) {
  double dmin = dx < dy ? dx : dy;
  if (dz < dmin) dmin = dz;
  double dist = sqrt((ox * dx) * (ox * dx) + (oy * dy) * (oy * dy) + (oz * dz) * (oz * dz));
  return dmin / dist;
}

/* Returns S(x); grad and hdiag (each may be NULL) receive dS/dx_i and d2S/dx_i^2. */
double o_rdp(int nx, int ny, int nz, double dx, double dy, double dz, double gamma, double eps,
             const double *kappa, const double *x, double *grad, double *hdiag) {
  double S = 0.0;
  for (int iz = 0; iz < nz; iz++)
    for (int iy = 0; iy < ny; iy++)
      for (int ix = 0; ix < nx; ix++) {
        size_t i = ((size_t)iz * ny + iy) * nx + ix;
        double gi = 0.0, hi = 0.0;
        for (int oz = -1; oz <= 1; oz++)
          for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
              if (ox == 0 && oy == 0 && oz == 0) continue;
              int jx = ix + ox, jy = iy + oy, jz = iz + oz;
              if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
              size_t j = ((size_t)jz * ny + jy) * nx + jx;
              double w = rdp_weight(ox, oy, oz, dx, dy, dz);
              double kk = kappa ? kappa[i] * kappa[j] : 1.0;
              double d = x[i] - x[j];
              double s = x[i] + x[j];
              double phi = s + gamma * fabs(d) + eps;
              S += 0.5 * w * kk * d * d / phi;
              gi += w * kk * d * (2.0 * phi - (d + gamma * fabs(d))) / (phi * phi);
              hi += 2.0 * w * kk * (s - d + eps) * (s - d + eps) / (phi * phi * phi);
            }
        if (grad) grad[i] = gi;
        if (hdiag) hdiag[i] = hi;
      }
  return S;
}

/* ------------------------------------------------------------------------- */
/* Preconditioners, Sec. 2.3.                                                  */
/* kind 0: D_MLEM = (x+delta)/A^T1.                                            */
/* kind 1: harmonic, eq. 8: (x+delta)/(A^T1 + alpha*diag(H_{beta S})(x+delta)). */
/* hdiag_betaS is the diagonal of the Hessian of beta*S.  Where the            */
/* denominator is zero the entry is zero.                                      */
/* ------------------------------------------------------------------------- */
void o_precond(size_t N, int kind, const double *x, const double *sens, const double *hdiag_betaS,
               double alpha, double delta, double *D) {
  for (size_t i = 0; i < N; i++) {
    double num = x[i] + delta;
    double den = sens[i];
    if (kind == 1) den += alpha * hdiag_betaS[i] * num;
    D[i] = den > 0 ? num / den : 0.0;
  }
}

/* ------------------------------------------------------------------------- */
/* Subset sampling: splitmix64 (Steele, Lea, Flood 2014) drives a Fisher-Yates */
/* shuffle; one fresh permutation per epoch (Sec. 2.4, "without replacement"). */
/* ------------------------------------------------------------------------- */
uint64_t o_splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Subset index for each of niter iterations: epoch e (iterations e*n .. e*n+n-1)
 * takes a permutation of 0..n-1 obtained by shuffling the identity with draws
 * j = next() mod (i+1), i = n-1..1; the generator state runs on across epochs. */
void o_subset_order(uint64_t seed, int nsub, int niter, int *order) {
  uint64_t st = seed;
  int *perm = malloc(sizeof(int) * nsub);
  for (int k = 0; k < niter; k++) {
    if (k % nsub == 0) {
      for (int i = 0; i < nsub; i++) perm[i] = i;
      for (int i = nsub - 1; i >= 1; i--) {
        int j = (int)(o_splitmix64(&st) % (uint64_t)(i + 1));
        int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
      }
    }
    order[k] = perm[k % nsub];
  }
  free(perm);
}

/* ------------------------------------------------------------------------- */
/* Subset sampling rules of Sec. 2.4.                                          */
/* ------------------------------------------------------------------------- */
enum { O_SAMPLE_PERM = 0, O_SAMPLE_REPLACE = 1, O_SAMPLE_HM = 2, O_SAMPLE_COFACTOR = 3,
       O_SAMPLE_IMPORTANCE = 4 };

/* Output number k (0-based) of the splitmix64 stream started at state seed, i.e.
 * the value of the (k+1)-th call of o_splitmix64. */
uint64_t o_splitmix64_at(uint64_t seed, long k) {
  uint64_t st = seed;
  uint64_t z = 0;
  for (long c = 0; c <= k; c++) z = o_splitmix64(&st);
  return z;
}

/* Herman-Meyer order: n = p1 p2 ... pm with the prime factors ascending; iteration j
 * of an epoch writes j in mixed radix with digit d1 (base p1) least significant,
 * then d2 (base p2), ..., and visits subset d1 n/p1 + d2 n/(p1 p2) + ... +
 * dm n/(p1...pm).  For n = 2^m this is the bit reversal of j. */
static void herman_meyer(int n, int *out) {
  int f[64], m = 0, r = n;
  for (int q = 2; q <= r; q++)
    while (r % q == 0) { f[m++] = q; r /= q; }
  for (int j = 0; j < n; j++) {
    int rest = j, w = n, idx = 0;
    for (int t = 0; t < m; t++) {
      w /= f[t];
      idx += (rest % f[t]) * w;
      rest /= f[t];
    }
    out[j] = idx;
  }
}

static int gcd_int(int a, int b) {
  while (b) { int t = a % b; a = b; b = t; }
  return a;
}

/* Cofactor order: the generators of the cyclic group Z_n (1 <= g < n, gcd(g, n) = 1)
 * ranked by their distance to the nearer of 0.3 n and 0.7 n (ties: smaller g first;
 * distances compared as the integers |10 g - 3 n|, |10 g - 7 n|).  Epoch e uses the
 * (e mod count)-th generator g and visits 0, g, 2g, ... (mod n).  Returns the number
 * of generators written to gens (n - 1 at most). */
int o_cofactor_generators(int n, int *gens) {
  int c = 0;
  for (int g = 1; g < n; g++)
    if (gcd_int(g, n) == 1) gens[c++] = g;
  for (int a = 1; a < c; a++) { /* insertion sort by (distance, g) */
    int g = gens[a], b = a - 1;
    int dg = abs(10 * g - 3 * n) < abs(10 * g - 7 * n) ? abs(10 * g - 3 * n) : abs(10 * g - 7 * n);
    while (b >= 0) {
      int h = gens[b];
      int dh = abs(10 * h - 3 * n) < abs(10 * h - 7 * n) ? abs(10 * h - 3 * n) : abs(10 * h - 7 * n);
      if (dh < dg || (dh == dg && h < g)) break;
      gens[b + 1] = h;
      b--;
    }
    gens[b + 1] = g;
  }
  return c;
}

/* Subset index for each of niter iterations under the rules of Sec. 2.4:
 *   O_SAMPLE_PERM      uniformly at random without replacement (o_subset_order);
 *   O_SAMPLE_REPLACE   uniformly at random with replacement: iteration k takes
 *                      ((z_k >> 32) n) >> 32 with z_k = o_splitmix64_at(seed, k);
 *   O_SAMPLE_HM        Herman-Meyer order, repeated every epoch;
 *   O_SAMPLE_COFACTOR  cofactor order (o_cofactor_generators).
 * Returns 0, or -1 for an unknown kind (importance sampling depends on the iterates
 * and is drawn inside o_solve). */
int o_subset_order_kind(int kind, uint64_t seed, int nsub, int niter, int *order) {
  if (kind == O_SAMPLE_PERM) { o_subset_order(seed, nsub, niter, order); return 0; }
  if (kind == O_SAMPLE_REPLACE) {
    uint64_t st = seed;
    for (int k = 0; k < niter; k++) order[k] = (int)(((o_splitmix64(&st) >> 32) * (uint64_t)nsub) >> 32);
    return 0;
  }
  if (kind == O_SAMPLE_HM) {
    int *hm = malloc(sizeof(int) * nsub);
    herman_meyer(nsub, hm);
    for (int k = 0; k < niter; k++) order[k] = hm[k % nsub];
    free(hm);
    return 0;
  }
  if (kind == O_SAMPLE_COFACTOR) {
    int *gens = malloc(sizeof(int) * (nsub > 1 ? nsub : 1));
    int c = o_cofactor_generators(nsub, gens);
    for (int k = 0; k < niter; k++) {
      int e = k / nsub, j = k % nsub;
      int g = c > 0 ? gens[e % c] : 0;
      order[k] = (int)(((long)j * g) % nsub);
    }
    free(gens);
    return 0;
  }
  return -1;
}

/* Importance draw (Sec. 2.4): the smallest i with u < p_0 + ... + p_i (cumulative sum in
 * index order, FP64), or the last i with p_i > 0 when rounding leaves u above the sum. */
int o_draw_index(const double *p, int n, double u) {
  double c = 0.0;
  int last = 0;
  for (int i = 0; i < n; i++) {
    if (p[i] > 0) last = i;
    c += p[i];
    if (p[i] > 0 && u < c) return i;
  }
  return last;
}

/* ------------------------------------------------------------------------- */
/* Stepsize rules, Sec. 2.2 and Table 1.                                       */
/* ------------------------------------------------------------------------- */
enum { O_STEP_CONST = 0, O_STEP_VANISH = 1, O_STEP_ALG1 = 2, O_STEP_BB = 3, O_STEP_ALG2 = 4 };

/* Piecewise ALG1 rule of Table 1. */
double o_step_alg1(long k) {
  if (k < 10) return 3.0;
  if (k < 100) return 2.0;
  if (k < 200) return 1.5;
  if (k < 300) return 1.0;
  return 0.5;
}

/* ALG2/ALG3 cap of Table 1 applied to a BB step. */
double o_step_alg2(long k, int nsub, double tau_bb) {
  double cap = (k < 10) ? 3.0 : (k < 2L * nsub ? 2.2 : 1.0);
  return tau_bb < cap ? tau_bb : cap;
}

/* ------------------------------------------------------------------------- */
/* Preconditioned proximal stochastic gradient methods, eq. 6 with the SGD,    */
/* SAGA (eq. 7) and SVRG (eq. 9, Algorithm 1) estimators.                      */
/* f_i(x) = D_i(x) + (beta/n) S(x)  (eq. 5); prox = max(0, .) (eq. 6).         */
/* ------------------------------------------------------------------------- */
typedef struct {
  int algo;          /* 0 SGD, 1 SAGA, 2 SVRG */
  int nsub;          /* n */
  long niter;        /* iterations to run */
  int omega;         /* SVRG snapshot period in epochs */
  int step_rule;     /* O_STEP_* */
  double tau0, eta;  /* constant/vanishing parameters; BB start value */
  int precond_kind;  /* 0 MLEM, 1 harmonic */
  double alpha;      /* harmonic weight */
  double delta_rel;  /* delta = delta_rel * max(x) at each preconditioner update */
  const long *pc_iters; int n_pc;  /* iterations at which D is recomputed */
  double beta, gamma, eps;         /* RDP */
  const double *kappa;             /* may be NULL */
  const int *order;                /* subset index per iteration (length niter) */
  int sampling;                    /* O_SAMPLE_IMPORTANCE draws inside (SVRG); else order */
  uint64_t sample_seed;            /* importance draws: u_k from o_splitmix64_at(seed, k) */
  int *subsets_out;                /* may be NULL: subset used by each non-refresh iteration */
  long bb_until;                   /* BB step recomputed only at refreshes k <= bb_until
                                      (0: at every refresh); later it stays fixed */
} og_opts;

/* Gradient of f_i at x: data gradient of subset i plus (beta/n) grad S. */
static void subset_objective_grad(const og_geom *g, const og_opts *o, int i, const double *x,
                                  const double *m, const double *rr, const double *y, double *out,
                                  double *tmp) {
  size_t N = (size_t)g->nx * g->ny * g->nz;
  o_data_grad(g, o->nsub, i, x, m, rr, y, out);
  o_rdp(g->nx, g->ny, g->nz, g->dx, g->dy, g->dz, o->gamma, o->eps, o->kappa, x, tmp, NULL);
  for (size_t v = 0; v < N; v++) out[v] += (o->beta / o->nsub) * tmp[v];
}

/* Runs the method from x (overwritten with the final iterate).  tau_out (may be
 * NULL) receives the stepsize of each iteration.  snap (may be NULL) receives x
 * after every snap_every iterations (snap[j] after iteration (j+1)*snap_every). */
int o_solve(const og_geom *g, const og_opts *o, const double *m, const double *rr, const double *y,
            const double *sens, double *x, double *tau_out, double *snap, long snap_every) {
  size_t N = (size_t)g->nx * g->ny * g->nz;
  int n = o->nsub;
  double *D = calloc(N, sizeof(double));
  double *dir = malloc(sizeof(double) * N);
  double *gi = malloc(sizeof(double) * N);
  double *tmp = malloc(sizeof(double) * N);
  double *H = malloc(sizeof(double) * N);
  double *table = NULL, *G = NULL, *xhat_old = NULL, *G_old = NULL;
  if (o->algo >= 1) {
    table = malloc(sizeof(double) * N * n);
    G = calloc(N, sizeof(double));
  }
  if (o->algo == 2) {
    xhat_old = malloc(sizeof(double) * N);
    G_old = malloc(sizeof(double) * N);
  }
  int have_bb = 0, have_snapshot = 0;
  double tau_bb = o->tau0;
  /* importance sampling (Sec. 2.4, SVRG): p_i proportional to ||grad f_i(xhat)||,
   * recomputed at every snapshot refresh */
  const int importance = o->algo == 2 && o->sampling == O_SAMPLE_IMPORTANCE;
  double *prob = malloc(sizeof(double) * n);
  for (int i = 0; i < n; i++) prob[i] = 1.0 / n;
  /* SAGA table initialisation: all g_i = grad f_i(x^0) (a reading; the paper is
   * silent).  It takes no step. */
  if (o->algo == 1) {
    for (int i = 0; i < n; i++) {
      subset_objective_grad(g, o, i, x, m, rr, y, table + (size_t)i * N, tmp);
      for (size_t v = 0; v < N; v++) G[v] += table[(size_t)i * N + v];
    }
  }
  long snap_j = 0;
  for (long k = 0; k < o->niter; k++) {
    /* Algorithm 1: preconditioner update at the listed iterations. */
    for (int c = 0; c < o->n_pc; c++)
      if (o->pc_iters[c] == k) {
        double xmax = 0.0;
        for (size_t v = 0; v < N; v++) if (x[v] > xmax) xmax = x[v];
        double delta = o->delta_rel * xmax;
        if (o->precond_kind == 1) {
          o_rdp(g->nx, g->ny, g->nz, g->dx, g->dy, g->dz, o->gamma, o->eps, o->kappa, x, NULL, H);
          for (size_t v = 0; v < N; v++) H[v] *= o->beta; /* diag Hessian of beta*S */
        }
        o_precond(N, o->precond_kind, x, sens, H, o->alpha, delta, D);
      }
    if (o->subsets_out) o->subsets_out[k] = -1; /* refresh iterations use no subset */
    if (o->algo == 0) { /* SGD: n grad f_i */
      int i = o->order[k];
      if (o->subsets_out) o->subsets_out[k] = i;
      subset_objective_grad(g, o, i, x, m, rr, y, gi, tmp);
      for (size_t v = 0; v < N; v++) dir[v] = n * gi[v];
    } else if (o->algo == 1) { /* SAGA, eq. 7 */
      int i = o->order[k];
      if (o->subsets_out) o->subsets_out[k] = i;
      subset_objective_grad(g, o, i, x, m, rr, y, gi, tmp);
      double *Ti = table + (size_t)i * N;
      for (size_t v = 0; v < N; v++) {
        dir[v] = n * (gi[v] - Ti[v]) + G[v];
        G[v] += gi[v] - Ti[v];
        Ti[v] = gi[v];
      }
    } else { /* SVRG, eq. 9 / Algorithm 1 */
      if (k % ((long)o->omega * n) == 0) {
        for (size_t v = 0; v < N; v++) G[v] = 0.0;
        for (int i = 0; i < n; i++) {
          subset_objective_grad(g, o, i, x, m, rr, y, table + (size_t)i * N, tmp);
          for (size_t v = 0; v < N; v++) G[v] += table[(size_t)i * N + v];
        }
        /* short BB step from consecutive snapshots (Sec. 2.2: computed when the full
         * gradient is recomputed), taken in the metric of the preconditioner: the
         * gradient-descent form p'q / q'q applied to the variables D^(-1/2) x, i.e.
         * p'q / q'Dq.  This reading makes the step dimensionless, on the scale of the
         * Table 1 caps (3, 2.2, 1) and of the ALG1 steps that also multiply D grad. */
        if (have_snapshot && (o->bb_until <= 0 || k <= o->bb_until)) {
          double pq = 0.0, qq = 0.0;
          for (size_t v = 0; v < N; v++) {
            double pv = x[v] - xhat_old[v], qv = G[v] - G_old[v];
            pq += pv * qv;
            qq += qv * D[v] * qv;
          }
          if (qq > 0) { tau_bb = pq / qq; have_bb = 1; }
        }
        memcpy(xhat_old, x, sizeof(double) * N);
        memcpy(G_old, G, sizeof(double) * N);
        have_snapshot = 1;
        if (importance) {
          double tot = 0.0;
          for (int i = 0; i < n; i++) {
            double s2 = 0.0;
            for (size_t v = 0; v < N; v++) s2 += table[(size_t)i * N + v] * table[(size_t)i * N + v];
            prob[i] = sqrt(s2);
            tot += prob[i];
          }
          for (int i = 0; i < n; i++) prob[i] = tot > 0 ? prob[i] / tot : 1.0 / n;
        }
        for (size_t v = 0; v < N; v++) dir[v] = G[v];
      } else {
        int i;
        double w = n; /* uniform sampling: 1/p_i = n */
        if (importance) {
          /* with probabilities p the unbiased estimator weights the correction by 1/p_i */
          double u = (double)(o_splitmix64_at(o->sample_seed, k) >> 11) * (1.0 / 9007199254740992.0);
          i = o_draw_index(prob, n, u);
          w = 1.0 / prob[i];
        } else {
          i = o->order[k];
        }
        if (o->subsets_out) o->subsets_out[k] = i;
        subset_objective_grad(g, o, i, x, m, rr, y, gi, tmp);
        double *Ti = table + (size_t)i * N;
        for (size_t v = 0; v < N; v++) dir[v] = w * (gi[v] - Ti[v]) + G[v];
      }
    }
    double tau;
    switch (o->step_rule) {
      case O_STEP_CONST: tau = o->tau0; break;
      case O_STEP_VANISH: tau = o->tau0 / (1.0 + o->eta * (double)k / (double)n); break;
      case O_STEP_ALG1: tau = o_step_alg1(k); break;
      case O_STEP_BB: tau = have_bb ? tau_bb : o->tau0; break;
      default: tau = o_step_alg2(k, n, have_bb ? tau_bb : o->tau0); break;
    }
    if (tau_out) tau_out[k] = tau;
    /* eq. 6: x <- prox(x - tau D dir), prox = max(0, .) */
    for (size_t v = 0; v < N; v++) {
      double xn = x[v] - tau * D[v] * dir[v];
      x[v] = xn > 0 ? xn : 0.0;
    }
    if (snap && snap_every > 0 && (k + 1) % snap_every == 0) {
      memcpy(snap + (size_t)snap_j * N, x, sizeof(double) * N);
      snap_j++;
    }
  }
  (void)have_bb;
  free(prob);
  free(D); free(dir); free(gi); free(tmp); free(H);
  free(table); free(G); free(xhat_old); free(G_old);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* OSEM / MLEM (Sec. 2.3 names MLEM; Sec. 3.1 initialises every run with one   */
/* OSEM epoch):  x <- x / (A_s^T 1) * A_s^T (y_s / (A_s x + r_s)).             */
/* Voxels with A_s^T 1 = 0 keep their value.                                   */
/* ------------------------------------------------------------------------- */
void o_em_update(const og_geom *g, int nsub, int s, const double *m, const double *rr,
                 const double *y, double *x) {
  int T = g->ntof > 1 ? g->ntof : 1;
  size_t N = (size_t)g->nx * g->ny * g->nz;
  int *views = malloc(sizeof(int) * g->nview);
  int nv = o_subset_views(g->nview, nsub, s, views);
  size_t per_view = (size_t)g->nplane * g->nrad * T;
  double *px = malloc(sizeof(double) * nv * per_view);
  double *q = malloc(sizeof(double) * nv * per_view);
  double *bp = malloc(sizeof(double) * N);
  double *se = malloc(sizeof(double) * N);
  o_project(g, views, nv, x, px);
  for (int j = 0; j < nv; j++)
    for (int p = 0; p < g->nplane; p++)
      for (int r = 0; r < g->nrad; r++) {
        size_t lor = ((size_t)views[j] * g->nplane + p) * g->nrad + r;
        size_t loc = ((size_t)j * g->nplane + p) * g->nrad + r;
        for (int b = 0; b < T; b++) {
          double ybar = m[lor] * px[loc * T + b] + rr[lor * T + b];
          /* bins with y = 0 add nothing to A^T (y / ybar), also where ybar = 0 */
          q[loc * T + b] = y[lor * T + b] > 0 ? m[lor] * y[lor * T + b] / ybar : 0.0;
        }
      }
  o_backproject(g, views, nv, q, bp);
  o_sensitivity(g, nsub, s, m, se);
  for (size_t v = 0; v < N; v++)
    if (se[v] > 0) x[v] = x[v] / se[v] * bp[v];
  free(views); free(px); free(q); free(bp); free(se);
}

/* ------------------------------------------------------------------------- */
/* NRMSE against a reference image, Sec. 3.1: root mean square difference over */
/* the evaluation mask, divided by the mean of the reference over the          */
/* background mask.  Parity unpinned: the paper describes the masks only in   */
/* words (leave out the cold surroundings of the phantom, normalise by the     */
/* largest background region); these masks are a reading of that.             */
/* ------------------------------------------------------------------------- */
double o_nrmse(size_t N, const double *x, const double *ref, const unsigned char *mask,
               const unsigned char *bg) {
  double se = 0.0, sb = 0.0;
  size_t nm = 0, nb = 0;
  for (size_t i = 0; i < N; i++) {
    if (mask[i]) { se += (x[i] - ref[i]) * (x[i] - ref[i]); nm++; }
    if (bg[i]) { sb += ref[i]; nb++; }
  }
  return sqrt(se / (double)nm) / (sb / (double)nb);
}
