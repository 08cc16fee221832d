/*
 * CPU oracle of the LavaMD-style neighbour-box force region (Table 1, LavaMD:
 * particle potential and forces from the particles of the neighbouring boxes;
 * Section 5 approximates the force calculation for a neighbouring box with TAF
 * and iACT, at thread and warp level, Figure 9).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU legs,
 * never by the library. It shares no code with the CUDA path. Compiled with
 * -ffp-contract=off, so every operation below is one IEEE-rounded operation in
 * the written order.
 *
 * Space: B x B x B boxes, box b = (bz B + by) B + bx, NP particles per box,
 * particle p = b NP + m. Inputs rq: 4 rows of P = B^3 NP doubles (x, y, z,
 * charge q; row stride P). Output fv: 4 rows of P doubles (potential, force
 * x, y, z).
 *
 * Region (one invocation): the contribution of box b to particle p,
 *   y(p, b) = sum over the NP particles j of b, in order, of
 *             (q_j v, q_j (fs dx), q_j (fs dy), q_j (fs dz)),
 *   d = r_p - r_j, r2 = dx dx + dy dy + dz dz, v = exp(-(a2 r2)), fs = 2 v.
 * The neighbour sequence of home box h: h itself, then the boxes at offsets
 * (dx, dy, dz) in {-1, 0, 1}^3 \ {0} in the order dz, dy, dx (dx fastest)
 * that lie inside the grid; nn(h) of them (1..27). Particle p accumulates the
 * outputs of its nn invocations in that order: fv_p = sum_k y_k.
 *
 * Schedule: one logical block per home box, its NP particles on lanes
 * 0..NP-1 of ceil(NP/32) warps; all lanes of a block share the neighbour
 * sequence and advance one invocation k at a time. Invocation (p, k) has the
 * mask index k P + p.
 *
 * TAF (Section 2.3, per particle): the window holds the last hsize accurate
 * outputs (all four components); its statistic is the RSD (population
 * moments, sigma / |mu|, 0/0 = 0) of their potentials. A prediction repeats
 * all four components of the newest accurate output. Decisions at thread,
 * warp or block level follow the majority rule of the other regions: among
 * the group's lanes that computed exactly at this step, if more than half want
 * to predict, every one of them with a full window predicts the next psize
 * invocations.
 *
 * iACT (Section 2.3, tables shared within a warp, Section 3.1.4): the inputs
 * of invocation (p, b) are the particle's coordinates (x_p, y_p, z_p), scaled
 * to single precision z_d = (float)(s_d x_d); a table slot holds z and the
 * four outputs. The box is not an input: a hit reuses the force that some box
 * exerted on a particle near p. With one private table per lane a particle's
 * own entry lies at distance 0, so every invocation after its first exact one
 * hits for any thr > 0; shared tables hold the entries of the lanes that lie
 * farthest from them (the write rule below), a spread sample of positions. Read,
 * decide, execute and write phases as the other regions' iACT: nearest valid
 * slot by single-precision Euclidean distance (ties to the lowest slot),
 * majority rule over the group's active lanes at warp or block level, and per
 * table one write per step by the lane that computed exactly and lies
 * farthest from its table (+inf when the table is empty; ties to the lowest
 * lane) into the round-robin slot.
 *
 * Parity status: pinned by tests that do not reuse this code (a numpy brute
 * force over all particle pairs of neighbouring boxes, closed forms for one
 * and two particles, the TAF and iACT limits thr = 0 and thr = +inf, and the
 * one-lane group that makes warp and block level the thread level).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { LMD_EXACT = 0, LMD_TAF = 1, LMD_IACT = 2 };
enum { LMD_THREAD = 0, LMD_WARP = 1, LMD_BLOCK = 2 };
enum { LMD_MASK_EXACT = 0, LMD_MASK_APPROX = 1 };
#define LMD_BORDER_REL 1e-6

/* Boxes of the neighbour sequence of home box h (returns nn). */
static int neighbours(int B, int64_t h, int64_t nb[27]) {
  const int hx = (int)(h % B), hy = (int)((h / B) % B), hz = (int)(h / ((int64_t)B * B));
  int nn = 0;
  nb[nn++] = h;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int x = hx + dx, y = hy + dy, z = hz + dz;
        if (x < 0 || y < 0 || z < 0 || x >= B || y >= B || z >= B) continue;
        nb[nn++] = ((int64_t)z * B + y) * B + x;
      }
  return nn;
}

/* y(p, b): the contribution of box b's particles to particle p. */
static void box_force(const double *rq, int64_t P, int NP, double a2, int64_t p, int64_t b,
                      double y[4]) {
  const double xp = rq[p], yp = rq[P + p], zp = rq[2 * P + p];
  double pot = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
  for (int m = 0; m < NP; ++m) {
    const int64_t j = b * NP + m;
    const double dx = xp - rq[j], dy = yp - rq[P + j], dz = zp - rq[2 * P + j];
    const double q = rq[3 * P + j];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double v = exp(-(a2 * r2));
    const double fs = 2.0 * v;
    pot = pot + q * v;
    fx = fx + q * (fs * dx);
    fy = fy + q * (fs * dy);
    fz = fz + q * (fs * dz);
  }
  y[0] = pot;
  y[1] = fx;
  y[2] = fy;
  y[3] = fz;
}

/* RSD of the h potentials win[(head + j) % h][0], oldest first. */
static double window_rsd(const double *win, int head, int h) {
  double sum = 0.0;
  for (int j = 0; j < h; ++j) sum = sum + win[((head + j) % h) * 4];
  const double mu = sum / h;
  double acc = 0.0;
  for (int j = 0; j < h; ++j) {
    const double d = win[((head + j) % h) * 4] - mu;
    acc = acc + d * d;
  }
  const double var = acc / h;
  const double sd = sqrt(var);
  const double amu = fabs(mu);
  if (amu == 0.0) return var == 0.0 ? 0.0 : INFINITY;
  return sd / amu;
}

static int borderline(double s, double thr) {
  if (isinf(thr) || isnan(s)) return 0;
  return fabs(s - thr) <= LMD_BORDER_REL * thr;
}

/* technique: LMD_EXACT / LMD_TAF / LMD_IACT; level: LMD_THREAD / WARP /
 * BLOCK. TAF knobs hsize 1..64, psize >= 0, thr >= 0, reset 0/1; iACT knobs
 * tsize 1..64, tperwarp dividing 32, thr >= 0, in_scale (3 doubles or NULL).
 * mask (nullable, 27 P bytes): written at k P + p for k < nn. counters
 * (nullable): [0] invocations, [1] approximated, [2] 0, [3] borderline. */
int orc_lavamd(int32_t B, int32_t NP, double a2, const double *rq, double *fv, int32_t technique,
               int32_t level, int32_t hsize, int32_t psize, double thr, int32_t reset,
               int32_t tsize, int32_t tperwarp, const double *in_scale, uint8_t *mask,
               int64_t *counters) {
  if (B < 0 || NP < 1 || NP > 1024 || technique < LMD_EXACT || technique > LMD_IACT) return 1;
  if (level < LMD_THREAD || level > LMD_BLOCK) return 1;
  if (technique == LMD_TAF && (hsize < 1 || hsize > 64 || psize < 0 || !(thr >= 0.0))) return 1;
  if (technique == LMD_IACT &&
      (tsize < 1 || tsize > 64 || tperwarp < 1 || tperwarp > 32 || 32 % tperwarp != 0 ||
       !(thr >= 0.0)))
    return 1;
  const int64_t nbox = (int64_t)B * B * B, P = nbox * NP;
  const int NL = (NP + 31) / 32 * 32; /* lanes of a block */
  const int h = hsize, L = technique == LMD_IACT ? 32 / tperwarp : 32;
  const int ntab = technique == LMD_IACT ? (NL / 32) * tperwarp : 0;
  const float thr_f = (float)thr;
  const int thr_inf = isinf(thr);
  double sc[3] = {1.0, 1.0, 1.0};
  if (in_scale)
    for (int d = 0; d < 3; ++d) sc[d] = in_scale[d];
  int64_t n_inv = 0, n_apx = 0, n_border = 0;
  int64_t hb;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_inv, n_apx, n_border)
  for (hb = 0; hb < nbox; ++hb) {
    int64_t nb[27];
    const int nn = neighbours(B, hb, nb);
    double *acc = (double *)calloc((size_t)NL * 4, sizeof(double));
    double *y = (double *)calloc((size_t)NL * 4, sizeof(double));
    int *act = (int *)calloc(NL, sizeof(int));
    int *decided = (int *)calloc(NL, sizeof(int));
    int *wants = (int *)calloc(NL, sizeof(int));
    int *own = (int *)calloc(NL, sizeof(int));
    int *apx = (int *)calloc(NL, sizeof(int));
    /* TAF state */
    double *win = (double *)calloc((size_t)NL * (technique == LMD_TAF ? h : 1) * 4, sizeof(double));
    int *head = (int *)calloc(NL, sizeof(int));
    int *cnt = (int *)calloc(NL, sizeof(int));
    int64_t *pred = (int64_t *)calloc(NL, sizeof(int64_t));
    /* iACT state */
    const int ts = technique == LMD_IACT ? tsize : 1;
    float *tz = (float *)calloc((size_t)(ntab ? ntab : 1) * ts * 3, sizeof(float));
    double *ty = (double *)calloc((size_t)(ntab ? ntab : 1) * ts * 4, sizeof(double));
    int *tvalid = (int *)calloc((size_t)(ntab ? ntab : 1) * ts, sizeof(int));
    int *rr = (int *)calloc(ntab ? ntab : 1, sizeof(int));
    int *has = (int *)calloc(NL, sizeof(int));
    int *near = (int *)calloc(NL, sizeof(int));
    float *dmin = (float *)calloc(NL, sizeof(float));
    float *z = (float *)calloc((size_t)NL * 3, sizeof(float));
    for (int l = 0; l < NL; ++l) act[l] = l < NP;

    for (int k = 0; k < nn; ++k) {
      const int64_t b = nb[k];
      if (technique == LMD_EXACT) {
        for (int l = 0; l < NP; ++l) {
          const int64_t p = hb * NP + l;
          box_force(rq, P, NP, a2, p, b, y + 4 * l);
          if (mask) mask[(int64_t)k * P + p] = LMD_MASK_EXACT;
          n_inv++;
        }
      } else if (technique == LMD_TAF) {
        /* per-lane path */
        for (int l = 0; l < NP; ++l) {
          const int64_t p = hb * NP + l;
          double *w = win + (size_t)l * h * 4;
          decided[l] = wants[l] = 0;
          n_inv++;
          if (pred[l] > 0) {
            const int newest = (head[l] + cnt[l] - 1) % h;
            for (int c = 0; c < 4; ++c) y[4 * l + c] = w[newest * 4 + c];
            if (mask) mask[(int64_t)k * P + p] = LMD_MASK_APPROX;
            pred[l] -= 1;
            n_apx++;
            if (reset && pred[l] == 0) cnt[l] = 0;
            continue;
          }
          box_force(rq, P, NP, a2, p, b, y + 4 * l);
          if (mask) mask[(int64_t)k * P + p] = LMD_MASK_EXACT;
          decided[l] = 1;
          int slot;
          if (cnt[l] < h) {
            slot = (head[l] + cnt[l]) % h;
            cnt[l] += 1;
          } else {
            slot = head[l];
            head[l] = (head[l] + 1) % h;
          }
          for (int c = 0; c < 4; ++c) w[slot * 4 + c] = y[4 * l + c];
          if (cnt[l] == h) {
            const double s = window_rsd(w, head[l], h);
            n_border += borderline(s, thr);
            wants[l] = thr_inf || s < thr;
          }
        }
        /* decision at the requested level */
        for (int l = 0; l < NL; ++l) own[l] = 0;
        if (level == LMD_THREAD) {
          for (int l = 0; l < NP; ++l) own[l] = decided[l] && wants[l];
        } else {
          const int gsize = level == LMD_WARP ? 32 : NL;
          for (int g0 = 0; g0 < NL; g0 += gsize) {
            int n_dec = 0, n_want = 0;
            for (int l = g0; l < g0 + gsize; ++l) {
              n_dec += decided[l];
              n_want += decided[l] && wants[l];
            }
            if (2 * n_want > n_dec)
              for (int l = g0; l < g0 + gsize; ++l) own[l] = decided[l] && cnt[l] == h;
          }
        }
        for (int l = 0; l < NP; ++l)
          if (own[l]) pred[l] = psize;
      } else {
        /* iACT read phase */
        for (int l = 0; l < NP; ++l) {
          const int64_t p = hb * NP + l;
          const int tab = (l / 32) * tperwarp + (l % 32) / L;
          for (int d = 0; d < 3; ++d) z[3 * l + d] = (float)(sc[d] * rq[(int64_t)d * P + p]);
          has[l] = wants[l] = 0;
          near[l] = -1;
          dmin[l] = INFINITY;
          float best = INFINITY;
          for (int j = 0; j < tsize; ++j) {
            const size_t s = (size_t)tab * tsize + j;
            if (!tvalid[s]) continue;
            float a = 0.0f;
            for (int d = 0; d < 3; ++d) {
              const float df = z[3 * l + d] - tz[s * 3 + d];
              const float sq = df * df;
              a = a + sq;
            }
            if (!has[l] || a < best) {
              best = a;
              near[l] = j;
            }
            has[l] = 1;
          }
          if (has[l]) {
            dmin[l] = sqrtf(best);
            wants[l] = dmin[l] < thr_f;
            n_border += borderline((double)dmin[l], thr);
          }
        }
        /* decision */
        if (level == LMD_THREAD) {
          for (int l = 0; l < NL; ++l) apx[l] = act[l] && wants[l];
        } else {
          const int gsize = level == LMD_WARP ? 32 : NL;
          for (int g0 = 0; g0 < NL; g0 += gsize) {
            int n_act = 0, n_want = 0;
            for (int l = g0; l < g0 + gsize; ++l) {
              n_act += act[l];
              n_want += act[l] && wants[l];
            }
            const int maj = 2 * n_want > n_act;
            for (int l = g0; l < g0 + gsize; ++l) apx[l] = maj && act[l] && has[l];
          }
        }
        /* execute */
        for (int l = 0; l < NP; ++l) {
          const int64_t p = hb * NP + l;
          const int tab = (l / 32) * tperwarp + (l % 32) / L;
          n_inv++;
          if (apx[l]) {
            for (int c = 0; c < 4; ++c) y[4 * l + c] = ty[((size_t)tab * tsize + near[l]) * 4 + c];
            if (mask) mask[(int64_t)k * P + p] = LMD_MASK_APPROX;
            n_apx++;
          } else {
            box_force(rq, P, NP, a2, p, b, y + 4 * l);
            if (mask) mask[(int64_t)k * P + p] = LMD_MASK_EXACT;
          }
        }
        /* write phase */
        for (int tab = 0; tab < ntab; ++tab) {
          const int l0 = (tab / tperwarp) * 32 + (tab % tperwarp) * L;
          int writer = -1;
          for (int l = l0; l < l0 + L; ++l) {
            if (!act[l] || apx[l]) continue;
            if (writer < 0 || dmin[l] > dmin[writer]) writer = l;
          }
          if (writer < 0) continue;
          const size_t s = (size_t)tab * tsize + rr[tab];
          for (int d = 0; d < 3; ++d) tz[s * 3 + d] = z[3 * writer + d];
          for (int c = 0; c < 4; ++c) ty[s * 4 + c] = y[4 * writer + c];
          tvalid[s] = 1;
          rr[tab] = (rr[tab] + 1) % tsize;
        }
      }
      for (int l = 0; l < NP; ++l)
        for (int c = 0; c < 4; ++c) acc[4 * l + c] = acc[4 * l + c] + y[4 * l + c];
    }
    for (int l = 0; l < NP; ++l)
      for (int c = 0; c < 4; ++c) fv[(int64_t)c * P + hb * NP + l] = acc[4 * l + c];
    free(acc); free(y); free(act); free(decided); free(wants); free(own); free(apx);
    free(win); free(head); free(cnt); free(pred);
    free(tz); free(ty); free(tvalid); free(rr); free(has); free(near); free(dmin); free(z);
  }
  if (counters) {
    counters[0] = n_inv;
    counters[1] = n_apx;
    counters[2] = 0;
    counters[3] = n_border;
  }
  return 0;
}
