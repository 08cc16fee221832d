/*
 * CPU oracle of the hexahedral Lagrangian-hydro element update whose
 * equation-of-state call is the approximated region (TEST INFRASTRUCTURE ONLY).
 *
 * The paper approximates kernels of LULESH (Table 1; Section 4.1) but prints
 * no hydro equations, so this restates a textbook staggered-grid scheme:
 * nodes carry position and velocity, elements energy, pressure, viscosity and
 * relative volume. The volume of a trilinear hexahedron is its plain
 * definition, the integral of det J over the reference cube, evaluated with the
 * 2 x 2 x 2 Gauss-Legendre rule (exact: det J has degree at most 2 in each
 * reference coordinate). Its gradient with respect to a node position is the
 * derivative of that same sum, the cofactor form
 *   d(det J)/d x_c = dN_c/dxi (X_eta x X_zeta) + dN_c/deta (X_zeta x X_xi)
 *                  + dN_c/dzeta (X_xi x X_eta).
 * Nothing here is shared with the CUDA library.
 *
 * Mesh: n^3 elements on [0,1]^3, node (i,j,k) at ((k(n+1) + j)(n+1) + i),
 * element (i,j,k) at ((k n + j) n + i); element corners in lexicographic order
 * c = a + 2b + 4d for node (i+a, j+b, k+d).
 *
 * One time step (fixed dt):
 *  1. corner forces f_c = (p + q) dV/dx_c at x^n; node force = sum over the
 *     adjacent elements (fixed order: k, then j, then i ascending);
 *  2. u^{n+1} = u^n + dt F / m_node, symmetry planes x = 0, y = 0, z = 0 hold
 *     the normal velocity at 0; x^{n+1} = x^n + dt u^{n+1};
 *  3. V = volume(x^{n+1}), v1 = V / V0, dv = v1 - v, L = cbrt(V), rho = 1/v1,
 *     c_s = sqrt(gamma max(p,0) v1), du = L dv / (v1 dt),
 *     q = rho (c_q^2 du^2 + c_l c_s |du|) in compression (dv < 0), else 0;
 *  4. EOS region on (e, v1, dv, q) -> p (exactly, or under TAF / iACT);
 *  5. e = p v1 / (gamma - 1), v = v1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* from hpac_oracle.c (same library) */
typedef struct {
  int32_t kind, dtype;
  int64_t n;
  int32_t n_in, n_out;
  int64_t in_stride, out_stride;
  int64_t threads;
  int32_t block;
  double param;
  int32_t arg, pad;
  const float *aux;
} orc_region;
int orc_run_exact(const orc_region *R, const void *in, void *out);
int orc_run_taf(const orc_region *R, const void *in, int32_t hsize, int32_t psize, double thr,
                int32_t level, int32_t reset, void *out, uint8_t *mask, void *stat,
                int64_t *counters);
int orc_run_iact(const orc_region *R, const void *in, int32_t tsize, int32_t tperwarp,
                 double thr, int32_t level, const double *in_scale, void *out, uint8_t *mask,
                 void *stat, int64_t *counters);
int orc_run_taf_persist(const orc_region *R, const void *in, int32_t hsize, int32_t psize,
                        double thr, int32_t level, int32_t reset, double *st_vals,
                        int32_t *st_cnt, int32_t *st_pred, void *out, uint8_t *mask, void *stat,
                        int64_t *counters);
int orc_run_iact_persist(const orc_region *R, const void *in, int32_t tsize, int32_t tperwarp,
                         double thr, int32_t level, const double *in_scale, float *st_z,
                         double *st_y, int32_t *st_valid, int32_t *st_rr, void *out,
                         uint8_t *mask, void *stat, int64_t *counters);

#define HYDRO_CQ 2.0
#define HYDRO_CL 0.5

static const double GP[2] = {0.21132486540518711775, 0.78867513459481288225}; /* (1 -+ 1/sqrt3)/2 */

/* shape-function derivatives of corner c at (xi, eta, zeta) */
static void dshape(int c, double xi, double eta, double ze, double *dxi, double *deta, double *dze) {
  int a = c & 1, b = (c >> 1) & 1, d = (c >> 2) & 1;
  double fa = a ? xi : 1.0 - xi, fb = b ? eta : 1.0 - eta, fd = d ? ze : 1.0 - ze;
  double ga = a ? 1.0 : -1.0, gb = b ? 1.0 : -1.0, gd = d ? 1.0 : -1.0;
  *dxi = ga * fb * fd;
  *deta = fa * gb * fd;
  *dze = fa * fb * gd;
}

static void cross(const double *u, const double *v, double *w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

/* Volume and (optionally) its gradient for one hexahedron (corners X, Y, Z). */
static double hex_vol_grad(const double *X, const double *Y, const double *Z, double *gX,
                           double *gY, double *gZ) {
  double V = 0.0;
  if (gX)
    for (int c = 0; c < 8; ++c) gX[c] = gY[c] = gZ[c] = 0.0;
  for (int g = 0; g < 8; ++g) {
    double xi = GP[g & 1], eta = GP[(g >> 1) & 1], ze = GP[(g >> 2) & 1];
    double w = 0.125;
    double Jx[3] = {0, 0, 0}, Je[3] = {0, 0, 0}, Jz[3] = {0, 0, 0};
    double dn[8][3];
    for (int c = 0; c < 8; ++c) {
      dshape(c, xi, eta, ze, &dn[c][0], &dn[c][1], &dn[c][2]);
      double p[3] = {X[c], Y[c], Z[c]};
      for (int k = 0; k < 3; ++k) {
        Jx[k] += p[k] * dn[c][0];
        Je[k] += p[k] * dn[c][1];
        Jz[k] += p[k] * dn[c][2];
      }
    }
    double ez[3], zx[3], xe[3];
    cross(Je, Jz, ez);
    cross(Jz, Jx, zx);
    cross(Jx, Je, xe);
    V += w * (Jx[0] * ez[0] + Jx[1] * ez[1] + Jx[2] * ez[2]);
    if (gX) {
      for (int c = 0; c < 8; ++c) {
        gX[c] += w * (dn[c][0] * ez[0] + dn[c][1] * zx[0] + dn[c][2] * xe[0]);
        gY[c] += w * (dn[c][0] * ez[1] + dn[c][1] * zx[1] + dn[c][2] * xe[1]);
        gZ[c] += w * (dn[c][0] * ez[2] + dn[c][1] * zx[2] + dn[c][2] * xe[2]);
      }
    }
  }
  return V;
}

double orc_hex_volume(const double *X, const double *Y, const double *Z) {
  return hex_vol_grad(X, Y, Z, NULL, NULL, NULL);
}

void orc_hex_volume_grad(const double *X, const double *Y, const double *Z, double *gX, double *gY,
                         double *gZ) {
  hex_vol_grad(X, Y, Z, gX, gY, gZ);
}

static void gather(int n, int64_t e, const double *x, const double *y, const double *z, double *X,
                   double *Y, double *Zc) {
  int64_t n1 = n + 1;
  int64_t i = e % n, j = (e / n) % n, k = e / ((int64_t)n * n);
  for (int c = 0; c < 8; ++c) {
    int64_t nd = ((k + ((c >> 2) & 1)) * n1 + (j + ((c >> 1) & 1))) * n1 + (i + (c & 1));
    X[c] = x[nd];
    Y[c] = y[nd];
    Zc[c] = z[nd];
  }
}

/* Reference volumes V0 (element mass = V0 at unit reference density) and node
 * masses (an eighth of each adjacent element's mass). */
int orc_hydro_init(int32_t n, const double *x, const double *y, const double *z, double *V0,
                   double *mnode, double *unused) {
  (void)unused;
  if (n < 1) return 1;
  int64_t E = (int64_t)n * n * n, n1 = n + 1, Nn = n1 * n1 * n1;
  int64_t e;
#pragma omp parallel for schedule(static)
  for (e = 0; e < E; ++e) {
    double X[8], Y[8], Z[8];
    gather(n, e, x, y, z, X, Y, Z);
    V0[e] = hex_vol_grad(X, Y, Z, NULL, NULL, NULL);
  }
  int64_t nd;
#pragma omp parallel for schedule(static)
  for (nd = 0; nd < Nn; ++nd) {
    int64_t i = nd % n1, j = (nd / n1) % n1, k = nd / (n1 * n1);
    double m = 0.0;
    for (int64_t ek = k - 1; ek <= k; ++ek)
      for (int64_t ej = j - 1; ej <= j; ++ej)
        for (int64_t ei = i - 1; ei <= i; ++ei) {
          if (ei < 0 || ej < 0 || ek < 0 || ei >= n || ej >= n || ek >= n) continue;
          m += 0.125 * V0[(ek * n + ej) * n + ei];
        }
    mnode[nd] = m;
  }
  return 0;
}

/* EOS technique for step 4: mode 0 exact, 1 TAF, 2 iACT. */
typedef struct {
  int32_t mode;
  int32_t hsize, psize;     /* TAF */
  int32_t tsize, tperwarp;  /* iACT */
  int32_t level;
  double thresh;
  int64_t threads;          /* T for the EOS region */
  int32_t block;
  int32_t reserved;
  double in_scale[4];       /* iACT */
  /* State kept across steps (NULL: each step's call starts empty, as the
   * paper's kernel-scoped state). TAF: st[0] window values (double, [h][T]),
   * st[1] fill counts, st[2] owed predictions (int32, [T]); iACT: st[0] scaled
   * inputs (float), st[1] outputs (double), st[2] valid flags, st[3]
   * round-robin slots (int32), laid out as orc_run_iact_persist reads them. */
  void *st[4];
} orc_eos_knobs;

/* One time step. eos_in: scratch of 4E doubles (left holding the EOS inputs
 * of this step); mask: E bytes or NULL; counters[4] as for the techniques. */
int orc_hydro_step(int32_t n, double dt, double gamma, double *x, double *y, double *z, double *u,
                   double *v, double *w, double *e, double *p, double *q, double *vrel,
                   const double *V0, const double *mnode, int32_t use_knobs,
                   const orc_eos_knobs *K, double *eos_in, uint8_t *mask, int64_t *counters) {
  if (n < 1 || !(dt > 0.0)) return 1;
  const int64_t E = (int64_t)n * n * n, n1 = n + 1, Nn = n1 * n1 * n1;
  double *G = (double *)malloc(sizeof(double) * 24 * E);
  if (!G) return 2;
  int64_t el;
  /* 1. volume gradients at x^n */
#pragma omp parallel for schedule(static)
  for (el = 0; el < E; ++el) {
    double X[8], Y[8], Z[8];
    gather(n, el, x, y, z, X, Y, Z);
    hex_vol_grad(X, Y, Z, G + 24 * el, G + 24 * el + 8, G + 24 * el + 16);
  }
  /* 2. node forces, velocity and position update */
  int64_t nd;
#pragma omp parallel for schedule(static)
  for (nd = 0; nd < Nn; ++nd) {
    int64_t i = nd % n1, j = (nd / n1) % n1, k = nd / (n1 * n1);
    double F[3] = {0.0, 0.0, 0.0};
    for (int64_t ek = k - 1; ek <= k; ++ek)
      for (int64_t ej = j - 1; ej <= j; ++ej)
        for (int64_t ei = i - 1; ei <= i; ++ei) {
          if (ei < 0 || ej < 0 || ek < 0 || ei >= n || ej >= n || ek >= n) continue;
          int64_t eid = (ek * n + ej) * n + ei;
          int c = (int)((i - ei) + 2 * (j - ej) + 4 * (k - ek));
          double pq = p[eid] + q[eid];
          F[0] += pq * G[24 * eid + c];
          F[1] += pq * G[24 * eid + 8 + c];
          F[2] += pq * G[24 * eid + 16 + c];
        }
    double inv_m = 1.0 / mnode[nd];
    double un = u[nd] + dt * F[0] * inv_m;
    double vn = v[nd] + dt * F[1] * inv_m;
    double wn = w[nd] + dt * F[2] * inv_m;
    if (i == 0) un = 0.0;
    if (j == 0) vn = 0.0;
    if (k == 0) wn = 0.0;
    u[nd] = un;
    v[nd] = vn;
    w[nd] = wn;
  }
#pragma omp parallel for schedule(static)
  for (nd = 0; nd < Nn; ++nd) {
    x[nd] += dt * u[nd];
    y[nd] += dt * v[nd];
    z[nd] += dt * w[nd];
  }
  free(G);
  /* 3. new volume, viscosity and the EOS inputs */
#pragma omp parallel for schedule(static)
  for (el = 0; el < E; ++el) {
    double X[8], Y[8], Z[8];
    gather(n, el, x, y, z, X, Y, Z);
    double V = hex_vol_grad(X, Y, Z, NULL, NULL, NULL);
    double v1 = V / V0[el];
    double dv = v1 - vrel[el];
    double qn = 0.0;
    if (dv < 0.0) {
      double L = cbrt(V);
      double rho = 1.0 / v1;
      double pp = p[el] > 0.0 ? p[el] : 0.0;
      double cs = sqrt(gamma * pp * v1);
      double du = L * dv / (v1 * dt);
      qn = rho * (HYDRO_CQ * HYDRO_CQ * du * du + HYDRO_CL * cs * fabs(du));
    }
    eos_in[el] = e[el];
    eos_in[E + el] = v1;
    eos_in[2 * E + el] = dv;
    eos_in[3 * E + el] = qn;
  }
  /* 4. the EOS region */
  orc_region R;
  memset(&R, 0, sizeof(R));
  R.kind = 1;
  R.dtype = 1;
  R.n = E;
  R.n_in = 4;
  R.n_out = 1;
  R.in_stride = E;
  R.out_stride = E;
  R.threads = use_knobs ? K->threads : 0;
  R.block = use_knobs ? K->block : 256;
  R.param = gamma;
  double *pn = (double *)malloc(sizeof(double) * E);
  if (!pn) return 2;
  int rc = 0;
  int mode = use_knobs ? K->mode : 0;
  if (mode == 0) {
    rc = orc_run_exact(&R, eos_in, pn);
    if (mask) memset(mask, 0, (size_t)E);
    if (counters) counters[0] = E, counters[1] = counters[2] = counters[3] = 0;
  } else if (mode == 1) {
    if (K->st[0])
      rc = orc_run_taf_persist(&R, eos_in, K->hsize, K->psize, K->thresh, K->level, 0,
                               (double *)K->st[0], (int32_t *)K->st[1], (int32_t *)K->st[2], pn,
                               mask, NULL, counters);
    else
      rc = orc_run_taf(&R, eos_in, K->hsize, K->psize, K->thresh, K->level, 0, pn, mask, NULL,
                       counters);
  } else {
    if (K->st[0])
      rc = orc_run_iact_persist(&R, eos_in, K->tsize, K->tperwarp, K->thresh, K->level,
                                K->in_scale, (float *)K->st[0], (double *)K->st[1],
                                (int32_t *)K->st[2], (int32_t *)K->st[3], pn, mask, NULL,
                                counters);
    else
      rc = orc_run_iact(&R, eos_in, K->tsize, K->tperwarp, K->thresh, K->level, K->in_scale, pn,
                        mask, NULL, counters);
  }
  if (rc) {
    free(pn);
    return 3;
  }
  /* 5. energy from the new pressure; state advance */
#pragma omp parallel for schedule(static)
  for (el = 0; el < E; ++el) {
    double v1 = eos_in[E + el];
    p[el] = pn[el];
    e[el] = pn[el] * v1 / (gamma - 1.0);
    q[el] = eos_in[3 * E + el];
    vrel[el] = v1;
  }
  free(pn);
  return 0;
}
