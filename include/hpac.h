/*
 * hpac.h - C ABI of a GB300 (sm_103a) library that runs an annotated,
 * data-parallel loop region under the software approximation techniques of
 * HPAC-Offload (Fink, Parasyris, Georgakoudis, Menon, arXiv 2308.16877):
 * loop perforation, TAF temporal output memoization and iACT approximate input
 * memoization, with thread-, warp- or block-level (majority-rules) decisions.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are CUDA device pointers owned by the caller; h_* are
 *    host pointers owned by the caller. The library owns region handles and the
 *    small device buffers it allocates for them.
 *  - Region inputs are a column-major (structure-of-arrays) matrix: element d
 *    of invocation i is at d_in[d * in_stride + i] (the strided array section
 *    in(input[i*D:D:N]) of the paper's programming model, Section 3.2). The
 *    single output of invocation i is d_out[i].
 *  - Work is enqueued on the region's CUDA stream and returns without waiting,
 *    except calls given a non-NULL h_stats / h_result, which wait for their own
 *    work to finish before returning.
 *  - Every call returns an hpac_status; on anything but HPAC_OK,
 *    hpac_last_error() returns a message for the calling host thread. No call
 *    aborts the process or traps on the device.
 *  - The logical schedule is part of the semantics (Section 3.1.3, Figure 3(d)):
 *    logical thread t (0 <= t < T) performs invocations i = t + k*T,
 *    k = 0, 1, ..., i < N; warps are 32 consecutive logical threads and blocks
 *    block_threads consecutive logical threads. Decisions and memoization
 *    state follow this schedule exactly, whatever the physical launch.
 *  - Approximation state (TAF windows, iACT tables) lives for one call only, as
 *    in the paper's shared-memory AC state scoped to one kernel (Section 3.1.1).
 */
#ifndef HPAC_H_
#define HPAC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HPAC_OK = 0,
  HPAC_EINVAL = 1,        /* bad argument: descriptor, knob, pointer or size   */
  HPAC_ENOMEM = 2,        /* a device or host allocation failed                */
  HPAC_ECUDA = 3,         /* a CUDA runtime call failed (message says which)   */
  HPAC_ETIMEOUT = 4,      /* a bounded device-side wait gave up                */
  HPAC_EUNSUPPORTED = 5   /* valid request this build does not implement       */
} hpac_status;

typedef enum { HPAC_F32 = 0, HPAC_F64 = 1 } hpac_dtype;

/* Decision hierarchy, the level(thread|warp|team) clause of Section 3.2. At
 * warp and block level the group approximates iff strictly more than half of
 * its deciding lanes meet their criterion (Section 3.3, majority rules). */
typedef enum { HPAC_LEVEL_THREAD = 0, HPAC_LEVEL_WARP = 1, HPAC_LEVEL_BLOCK = 2 } hpac_level;

/* Built-in regions.
 *  BLACKSCHOLES: European call (Table 1, Black-Scholes). D = 4 inputs
 *    (spot S, strike K, expiry T in years, volatility sigma), param = rate r.
 *    F32 or F64. C = S N(d1) - K e^{-rT} N(d2).
 *  EOS: ideal-gas pressure with an implicit trapezoid energy update. D = 4
 *    inputs (e_n, v_{n+1}, dv, q_{n+1}), param = gamma. F64 only.
 *    p = (gamma-1) e_{n+1} / v_{n+1}, e_{n+1} = (e_n - dv (p_n + 2q)/2) /
 *    (1 + (gamma-1) dv / (2 v_{n+1})) clamped at 0, p_n = (gamma-1) e_n / (v_{n+1} - dv).
 *  IDENTITY: output = first input; 1 <= D <= 8; F32 or F64. A region without
 *    arithmetic, for measuring a technique's own cost and for bit-exact tests.
 *  BINOMIAL: American call on a Cox-Ross-Rubinstein tree (Table 1, Binomial
 *    Options: a portfolio of American options priced at several time points).
 *    D = 4 inputs (spot S, strike X, time to expiry T, volatility sigma),
 *    param = rate r, arg = tree steps N in 1..1024; F32 only. Per option (in
 *    double, then rounded): dt = T/N, v = sigma sqrt(dt), u = e^v, d = 1/u,
 *    a = e^{r dt}, pu = (a - d)/(u - d), weights pu/a and (1 - pu)/a, leaves
 *    S_j = S0 e^{v (2j - N)}, V_j = max(S_j - X, 0); then N single-precision
 *    backward steps S_j <- S_j u, V_j <- max(fma(pu/a, V_{j+1}, (pd/a) V_j),
 *    S_j - X). One invocation is a whole tree, computed by a team of 32 lanes:
 *    the logical schedule's T counts teams, each team prices options
 *    i = t + k T in turn, and TAF / iACT decide per team (the paper's
 *    block-level decision, one option per block): level must be
 *    HPAC_LEVEL_BLOCK and iACT keeps one table per team (tperwarp = 32).
 *  KMEANS: nearest-centroid assignment (Table 1, K-Means; Section 4.2
 *    approximates this distance kernel). D = 8 features, arg = clusters K in
 *    1..64, the centroids (K x 8 floats, row k at k*8) in device memory set by
 *    hpac_region_set_aux; F32 only. Output: the id (as a float) of the centroid
 *    with the smallest sum over d = 0..7 of (x_d - c_kd)^2, accumulated in
 *    order in single precision, ties to the lowest id. */
typedef enum {
  HPAC_REGION_BLACKSCHOLES = 0,
  HPAC_REGION_EOS = 1,
  HPAC_REGION_IDENTITY = 3,
  HPAC_REGION_BINOMIAL = 4,
  HPAC_REGION_KMEANS = 5
} hpac_region_kind;

/* Perforation patterns (Section 2.3; the runtime encounter counter of Section
 * 3.3). With k the invocation's step within its logical thread and
 * key = k when herded (Section 3.1.5: every thread drops the same steps) or
 * key = i otherwise:
 *  SMALL:M   drop when key mod M == M-1 (skip one of every M)
 *  LARGE:M   drop when key mod M != 0   (execute one of every M)
 *  INI:P     drop i <  floor(N P / 100) (first P percent of the loop)
 *  FINI:P    drop i >= N - floor(N P / 100) (last P percent)
 *  RANDOM:r  drop when (splitmix64(seed ^ key) >> 40) < floor(r * 2^24)
 *            (SplitMix64 of Steele, Lea and Flood 2014; not in the paper) */
typedef enum {
  HPAC_PERFO_SMALL = 0,
  HPAC_PERFO_LARGE = 1,
  HPAC_PERFO_INI = 2,
  HPAC_PERFO_FINI = 3,
  HPAC_PERFO_RANDOM = 4
} hpac_perfo_kind;

/* Per-invocation mask values written to d_mask (one byte per invocation). */
enum { HPAC_MASK_EXACT = 0, HPAC_MASK_APPROX = 1, HPAC_MASK_SKIPPED = 2 };

typedef enum { HPAC_METRIC_MAPE = 0, HPAC_METRIC_RMSE = 1, HPAC_METRIC_MCR = 2 } hpac_metric;

/* One annotated loop region. */
typedef struct {
  int32_t kind;             /* hpac_region_kind                                  */
  int32_t dtype;            /* hpac_dtype of inputs, output and statistic        */
  int64_t n;                /* trip count N >= 0                                 */
  int32_t n_in;             /* D, checked against kind                           */
  int32_t n_out;            /* must be 1                                         */
  int64_t in_stride;        /* >= n; column stride of d_in, in elements          */
  int64_t out_stride;       /* >= n; reserved for multi-output regions           */
  int64_t logical_threads;  /* T >= 0; 0 means N (one invocation per thread)     */
  int32_t block_threads;    /* B: multiple of 32, 32..1024                       */
  int32_t arg;              /* BINOMIAL: tree steps 1..1024; KMEANS: clusters    */
                            /* 1..64; 0 for the other kinds                      */
  double param;             /* r (BLACKSCHOLES, BINOMIAL), gamma (EOS), unused   */
} hpac_region_desc;

/* perfo(kind:arg) clause (Section 3.2, Table 2). m_or_percent is M for
 * SMALL/LARGE (>= 1) and P for INI/FINI (0..100); rate in [0, 1] and seed are
 * used by RANDOM; herded selects the step-uniform pattern (default 1). */
typedef struct {
  int32_t kind;
  int32_t m_or_percent;
  double rate;
  uint64_t seed;
  int32_t herded;
  int32_t reserved0;
} hpac_perfo_knobs;

/* memo(out:hsize:psize:thresh) clause (Sections 2.3, 3.2). hsize in 1..64,
 * psize >= 0, thresh >= 0 (a plain ratio; +inf always predicts once the window
 * is full), level is an hpac_level. reset_on_exit: 0 (the default reading)
 * keeps the window across a prediction run, so the next accurate output slides
 * it and re-tests; 1 (the alternative reading) empties it when the run ends,
 * so hsize accurate outputs refill it before the next test. */
typedef struct {
  int32_t hsize;
  int32_t psize;
  double thresh;
  int32_t level;
  int32_t reset_on_exit;
} hpac_taf_knobs;

/* memo(in:tsize:thresh:tperwarp) clause (Sections 2.3, 3.1.4, 3.2). tsize in
 * 1..64 slots per table, tperwarp in {1,2,4,8,16,32} tables per warp (32 gives
 * one private table per lane), thresh >= 0 on the Euclidean distance of scaled
 * inputs z_d = in_scale[d] * x_d (single precision), level an hpac_level.
 * in_scale: host array of D doubles, or NULL for all ones. */
typedef struct {
  int32_t tsize;
  int32_t tperwarp;
  double thresh;
  int32_t level;
  int32_t reserved0;
  const double *in_scale;
} hpac_iact_knobs;

/* Counts for one call. borderline counts decisions whose statistic lies
 * within 1e-6 relative of the threshold. */
typedef struct {
  int64_t invocations;
  int64_t approximated;
  int64_t skipped;
  int64_t borderline;
} hpac_stats;

/* Result of hpac_quality. For MAPE the terms with exact value 0 are set
 * aside: zeros counts them, zeros_mismatch those whose approximation is not
 * 0, zero_max_abs the largest |approx| among them. used = terms averaged. */
typedef struct {
  double value;
  double zero_max_abs;
  int64_t used;
  int64_t zeros;
  int64_t zeros_mismatch;
} hpac_quality_result;

typedef struct hpac_region hpac_region;

/* Create a region handle on the current CUDA device. desc is copied;
 * cuda_stream is a cudaStream_t (NULL = legacy default stream) used by every
 * later call on the handle. Allocates a few hundred bytes of device memory for
 * counters. Errors: HPAC_EINVAL (descriptor), HPAC_ECUDA, HPAC_ENOMEM. */
hpac_status hpac_region_create(const hpac_region_desc *desc, void *cuda_stream,
                               hpac_region **out);

/* Destroy a handle (NULL is accepted). Waits for the handle's stream. */
hpac_status hpac_region_destroy(hpac_region *region);

/* Change the stream later calls on the handle are enqueued on. */
hpac_status hpac_region_set_stream(hpac_region *region, void *cuda_stream);

/* Approximation state kept across calls. Not in the paper, whose TAF windows
 * and iACT tables live in one kernel's shared memory (Section 3.1.1) and so
 * restart at every launch. With enable = 1, every later TAF call on the region
 * resumes each logical thread's window and owed predictions where its previous
 * TAF call left them, and every iACT call resumes each logical warp's tables:
 * a sequence of calls then behaves as one call over the concatenated
 * iteration spaces (when each call's N is a multiple of T). The state lives in
 * device memory owned by the region (TAF: hsize x T values + 8 bytes per
 * logical thread; iACT: one table image per logical warp), allocated on first
 * use, and starts empty whenever the technique or its shape (TAF hsize; iACT
 * tsize, tperwarp) or T changes. enable = 0 frees it (after waiting for the
 * region's stream). Calls on one region must not run concurrently. */
hpac_status hpac_region_set_persistent(hpac_region *region, int32_t enable);

/* Empty the kept state (asynchronous on the region's stream). */
hpac_status hpac_region_reset_state(hpac_region *region);

/* KMEANS regions: the centroids every later run reads (device pointer, K x 8
 * floats, caller-owned, may change between runs; must stay valid while a run
 * using it is in flight; 16-byte aligned). HPAC_EINVAL for other kinds, NULL
 * or a pointer that is not 16-byte aligned. */
hpac_status hpac_region_set_aux(hpac_region *region, const void *d_aux);

/* K-Means centroid update, the exact step between two assignments: centroid k
 * becomes the mean of the observations whose id (d_assign, floats) is k,
 * summed in double (atomics, so the last bits of the sum may vary) and
 * rounded once; a cluster without observations keeps its centroid. d_x: 8
 * rows of `stride` floats; d_cent: K x 8 floats, updated in place; d_work: a
 * device workspace of hpac_kmeans_workspace_bytes(K) bytes, 8-byte aligned.
 * d_prev (nullable): the previous assignment; with h_changed non-NULL the call
 * waits and returns how many observations changed cluster (the convergence
 * test: none). Asynchronous on cuda_stream otherwise. */
size_t hpac_kmeans_workspace_bytes(int32_t clusters);
hpac_status hpac_kmeans_update(int64_t n, int32_t clusters, const float *d_x, int64_t stride,
                               const float *d_assign, const float *d_prev, float *d_cent,
                               void *d_work, int64_t *h_changed, void *cuda_stream);

/* Accurate execution path: d_out[i] = region(d_in[:, i]) for all i < N
 * (the non-approximated region the paper's speedups are measured against). */
hpac_status hpac_run_exact(hpac_region *region, const void *d_in, void *d_out);

/* Loop perforation (Sections 2.3, 3.1.5, 3.3). Dropped invocations read no
 * input and leave d_out[i] untouched. d_mask (nullable, N bytes) receives
 * HPAC_MASK_EXACT / HPAC_MASK_SKIPPED. h_stats (nullable) makes the call
 * synchronous and returns the counts. */
hpac_status hpac_run_perfo(hpac_region *region, const hpac_perfo_knobs *knobs, const void *d_in,
                           void *d_out, uint8_t *d_mask, hpac_stats *h_stats);

/* TAF (Section 2.3; GPU algorithm Section 3.1.3; runtime Section 3.3). Per
 * logical thread, a window of the last hsize accurate outputs; when full, the
 * relative standard deviation RSD = sigma/|mu| (population moments, 0/0 := 0)
 * is compared with thresh and, if lower, the next psize invocations output the
 * newest window value without reading their inputs. The window is kept across
 * a prediction run unless knobs->reset_on_exit. d_mask (nullable) gets EXACT/APPROX; d_stat (nullable, N
 * values of the region dtype) gets the RSD of every accurate invocation with a
 * full window, NaN elsewhere. */
hpac_status hpac_run_taf(hpac_region *region, const hpac_taf_knobs *knobs, const void *d_in,
                         void *d_out, uint8_t *d_mask, void *d_stat, hpac_stats *h_stats);

/* iACT (Section 2.3; table sharing Section 3.1.4; read/write phases Section
 * 3.3). Read phase: each lane finds the nearest valid slot of its table
 * (ties to the lowest slot) and wants to approximate iff its distance is below
 * thresh. Approximated invocations output that slot's value; at warp/block
 * level a majority forces every lane holding a valid slot. Write phase: per
 * table, the exactly computing lane farthest from the table (ties to the
 * lowest lane) stores its (scaled input, output) in the round-robin slot.
 * d_stat (nullable) gets the nearest distance (+inf for an empty table). */
hpac_status hpac_run_iact(hpac_region *region, const hpac_iact_knobs *knobs, const void *d_in,
                          void *d_out, uint8_t *d_mask, void *d_stat, hpac_stats *h_stats);

/* Quality loss of an approximated output against an exact reference (Section
 * 4): MAPE (Eq. 1), RMSE, or MCR (Eq. 2), accumulated in double precision on
 * the device. d_exact: n doubles; d_approx: n values of approx_dtype. The call
 * waits for the result. Uses a device buffer the library allocates once per
 * device on first use. */
hpac_status hpac_quality(int32_t approx_dtype, int64_t n, const double *d_exact,
                         const void *d_approx, int32_t metric, hpac_quality_result *h_result,
                         void *cuda_stream);

/* ------------------------------------------------------------------------
 * Hexahedral Lagrangian hydro with the EOS as the approximated region.
 *
 * The paper approximates kernels of the LULESH hydro proxy (Table 1, Section
 * 4.1; QoI: the final origin energy) but prints no hydro equations; this is a
 * textbook staggered-grid scheme on a structured n^3 hexahedral mesh over
 * [0,1]^3 with symmetry planes x = 0, y = 0, z = 0. Nodes: position and
 * velocity; elements: energy per reference volume e, pressure p, artificial
 * viscosity q, relative volume v. Per time step: nodal forces
 * (p + q) dV/dx from the exact trilinear volume gradient, velocity and position
 * update, new volume and viscosity, then the EOS region on (e, v_{n+1}, dv, q)
 * giving p, and e = p v / (gamma - 1).
 *
 * The caller allocates every array (device memory) and owns it; the library
 * keeps no state between calls, so copying the arrays checkpoints the run.
 * Node arrays hold (n+1)^3 doubles, node (i,j,k) at ((k(n+1) + j)(n+1) + i);
 * element arrays n^3 doubles, element (i,j,k) at ((k n + j) n + i).
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t n;                 /* elements per axis, 1..1024                         */
  int32_t reserved0;         /* must be 0                                          */
  double gamma;              /* ratio of specific heats (> 1)                      */
  double dt;                 /* fixed time step (> 0)                              */
  double *x, *y, *z;         /* node positions                                     */
  double *u, *v, *w;         /* node velocities                                    */
  double *mnode;             /* node masses                                        */
  double *e, *p, *q, *vrel;  /* element energy, pressure, viscosity, V / V0        */
  double *V0;                /* element reference volumes (= masses, density 1)    */
  double *grad;              /* 24 n^3 scratch: 12 dV/dx per corner (x, y, z rows) */
  double *eos_in;            /* 4 n^3: the EOS region's inputs of the last step    */
  double *pq;                /* n^3: p + q of the last step (init, finalize)        */
  double *rmass;             /* (n+1)^3: 1 / (12 m) per node (init)                */
  double *rV0;               /* n^3: 1 / V0 per element (init)                      */
} hpac_hydro_state;

/* From x, y, z and e (initial state): V0, node masses, p = (gamma-1) e,
 * q = 0, v = 1, zero velocities, the volume gradients and the derived arrays
 * pq, rmass and rV0. Relative volumes are formed as 1 where V = V0 and as
 * V rV0 otherwise (within a rounding of V / V0). Enqueued on cuda_stream.
 * Errors: HPAC_EINVAL (state), HPAC_ECUDA. */
hpac_status hpac_hydro_init(const hpac_hydro_state *s, void *cuda_stream);

/* Recompute the derived arrays from the state (pq = p + q, rmass = 1 / (12
 * mnode), rV0 = 1 / V0): for a caller that has overwritten p, q, mnode or V0,
 * e.g. restored a checkpoint of the other arrays. Enqueued on cuda_stream.
 * Errors as hpac_hydro_init. */
hpac_status hpac_hydro_derive(const hpac_hydro_state *s, void *cuda_stream);

/* The three non-region phases of a time step, each one kernel on cuda_stream,
 * for callers that run the EOS region themselves between them:
 * nodes (forces from pq = p + q and the stored gradients, velocity,
 * position, symmetry planes), elements (volume and gradient at the new
 * positions, viscosity, the EOS inputs in eos_in), finalize (e = p v_{n+1} /
 * (gamma - 1), v = v_{n+1}, pq = p + q). hpac_hydro_step is nodes, elements,
 * the region, finalize. */
hpac_status hpac_hydro_nodes(const hpac_hydro_state *s, void *cuda_stream);
hpac_status hpac_hydro_elements(const hpac_hydro_state *s, void *cuda_stream);
hpac_status hpac_hydro_finalize(const hpac_hydro_state *s, void *cuda_stream);

/* One time step on the EOS region's stream. eos: a region of kind
 * HPAC_REGION_EOS, F64, n = in_stride = n^3, param = gamma. technique 0 runs
 * the EOS exactly, 1 under TAF (knobs: hpac_taf_knobs), 2 under iACT
 * (hpac_iact_knobs), 3 under perforation (hpac_perfo_knobs; a dropped
 * element keeps its previous pressure). d_mask and h_stats as for the
 * technique's own call. */
hpac_status hpac_hydro_step(const hpac_hydro_state *s, hpac_region *eos, int32_t technique,
                            const void *knobs, uint8_t *d_mask, hpac_stats *h_stats);

/* `steps` time steps of hpac_hydro_step without masks or statistics,
 * enqueued back to back without waiting. */
hpac_status hpac_hydro_run(const hpac_hydro_state *s, hpac_region *eos, int32_t steps,
                           int32_t technique, const void *knobs);

/* ------------------------------------------------------------------------
 * LavaMD-style neighbour-box forces (Table 1, LavaMD: the potential and force
 * on each particle from the particles of the boxes that touch its own).
 * Section 5 approximates the force calculation for a neighbouring box with
 * TAF and iACT and compares thread- and warp-level decisions (Figure 9).
 *
 * Space: boxes1d^3 boxes, box b = (bz B + by) B + bx, par_per_box (NP)
 * particles per box, particle p = b NP + m, P = boxes1d^3 NP. d_rq: 4 rows of
 * P doubles (x, y, z, charge q; row stride P), device, 8-byte aligned, read
 * only. d_fv: 4 rows of P doubles (potential, force x, y, z), device, written.
 * One invocation is the contribution of one box b to one particle p:
 *   sum over b's particles j of (q_j v, 2 q_j v d), d = r_p - r_j,
 *   v = exp(-a2 |d|^2),
 * and fv_p sums the invocations of p's neighbour sequence: its own box, then
 * the touching boxes inside the grid at offsets (dx, dy, dz) != 0 in the
 * order dz, dy, dx (dx fastest); (3 boxes1d - 2)^3 NP invocations in all.
 * Arithmetic: FP64 with fused multiply-adds; the exponential within two ulps
 * (a table-driven method for |a2 r^2| <= 700, CUDA's exp beyond); each
 * invocation's NP terms summed in four interleaved partial sums.
 *
 * The block of a home box holds its NP particles on ceil(NP/32) warps; its
 * lanes advance through the sequence together. technique 0: exact. 1: TAF
 * (hpac_taf_knobs): per particle a window of the last hsize accurate outputs,
 * the RSD of their potentials against thresh, a prediction repeating all four
 * components of the newest output. 2: iACT (hpac_iact_knobs): the inputs are
 * the particle's coordinates (in_scale: 3 doubles or NULL), tables shared by
 * 32 / tperwarp lanes hold scaled coordinates and the four outputs; with one
 * table per lane every invocation after a particle's first hits (its own entry
 * is at distance 0) for any thresh > 0. Decision levels as for the regions
 * (level BLOCK: the home box). Shared memory per block: 32 NP bytes plus, for
 * TAF, 32 hsize ceil(NP/32)*32 or, for iACT, about 44 tsize bytes per table;
 * HPAC_EINVAL above the device's limit. d_mask (nullable, 27 P bytes): at
 * k P + p, for the k-th invocation of particle p, HPAC_MASK_EXACT or
 * HPAC_MASK_APPROX; the bytes of invocations that do not exist are left as
 * they are. h_stats (nullable) makes the call synchronous and returns the
 * counts. Errors: HPAC_EINVAL (descriptor, knobs, NULL or misaligned
 * pointers when P > 0), HPAC_ECUDA. Asynchronous on cuda_stream otherwise.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t boxes1d;      /* B, 0..1290                                           */
  int32_t par_per_box;  /* NP, 1..1024                                          */
  double a2;            /* pair potential exp(-a2 r^2): a2 = 2 alpha^2, >= 0    */
} hpac_lavamd_desc;

hpac_status hpac_lavamd_run(const hpac_lavamd_desc *desc, int32_t technique, const void *knobs,
                            const double *d_rq, double *d_fv, uint8_t *d_mask,
                            hpac_stats *h_stats, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched knob sweep (the paper's design-space exploration, Section 2.4 and
 * Section 4 / Table 2, which builds and runs each configuration separately):
 * every configuration over every Black-Scholes region (single precision) in
 * one persistent kernel captured in a CUDA graph. Per (configuration, region)
 * it returns counts and error sums against a double-precision exact price, no
 * output arrays. TAF runs at thread level; a dropped (perforated) invocation
 * counts with output 0 (a zero-prefilled output buffer).
 * ------------------------------------------------------------------------ */
enum { HPAC_SWEEP_TAF = 1, HPAC_SWEEP_PERFO = 3 };

typedef struct {
  int32_t technique;      /* HPAC_SWEEP_TAF or HPAC_SWEEP_PERFO                   */
  int32_t level;          /* TAF: must be HPAC_LEVEL_THREAD                        */
  int32_t hsize, psize;   /* TAF knobs (as hpac_taf_knobs)                         */
  double thresh;
  int32_t perfo_kind;     /* perforation knobs (as hpac_perfo_knobs)               */
  int32_t m_or_percent;
  double rate;
  uint64_t seed;
  int32_t herded;
  int32_t reserved0;
} hpac_sweep_config;

typedef struct {
  int64_t n;               /* options in the region                                */
  int64_t offset;          /* its first column in d_in / d_ref                     */
  int64_t logical_threads; /* T of the region's logical schedule (0 = n)           */
} hpac_sweep_region;

typedef struct {
  int64_t invocations;
  int64_t approximated;    /* TAF predictions                                      */
  int64_t skipped;         /* perforated invocations                               */
  int64_t mape_terms;      /* invocations whose exact price is not 0               */
  double sum_abs_rel;      /* sum |a - y| / |a| over those: MAPE = sum / terms     */
  double sum_sq;           /* sum (a - y)^2 over all: RMSE = sqrt(sum / invocations) */
} hpac_sweep_stats;

typedef struct hpac_sweep hpac_sweep;

/* Build a sweep: copies the configurations and regions, packs the inputs and
 * the split reference (hi, lo, 1/|a|) into 16-byte vectors per option, and
 * captures the launch in a CUDA graph. d_in: 4 rows (S, K, T, sigma) of
 * in_stride floats holding every region's options at its offset; d_ref: the
 * double-precision exact prices at the same positions; rate: r. Schedule (not
 * semantics): block_threads (64/128/256), persistent blocks per SM, logical
 * blocks per work item (tile_blocks). Allocates device memory (about 32 bytes
 * per option plus the tables); waits for cuda_stream's pending work once.
 * d_in is read only here; d_ref must stay valid and unchanged while the sweep
 * exists (relative errors beyond 1e30 are formed from it in double precision).
 * HPAC_EUNSUPPORTED if a work item would cover 2^32 or more invocations. */
hpac_status hpac_sweep_create(int32_t n_configs, const hpac_sweep_config *h_configs,
                              int32_t n_regions, const hpac_sweep_region *h_regions,
                              const float *d_in, int64_t in_stride, const double *d_ref,
                              double rate, int32_t block_threads, int32_t blocks_per_sm,
                              int32_t tile_blocks, void *cuda_stream, hpac_sweep **out);

/* Launch the captured graph on the creation stream (asynchronous). */
hpac_status hpac_sweep_run(hpac_sweep *sweep);

/* Wait for the last run and copy n_configs x n_regions stats, configuration
 * major (h_stats[c * n_regions + r]). */
hpac_status hpac_sweep_results(hpac_sweep *sweep, hpac_sweep_stats *h_stats);

hpac_status hpac_sweep_destroy(hpac_sweep *sweep);

/* ------------------------------------------------------------------------
 * Adjoint of the exact region: d out / d in for every invocation, the
 * derivative targets of the learned surrogate. Not from the paper.
 * Black-Scholes (inputs S, K, T, sigma): dC/dS = N(d1), dC/dK = -e^{-rT} N(d2),
 * dC/dT = S phi(d1) sigma / (2 sqrt T) + r K e^{-rT} N(d2), dC/dsigma =
 * S phi(d1) sqrt T. EOS: the closed-form partials of p_{n+1} with respect to
 * (e_n, v_{n+1}, dv, q) (zero where the energy clamp is active).
 * IDENTITY: 1 for the first input, 0 for the others.
 * d_grad: D x n values of the region dtype, row d at d_grad[d * n + i].
 * ------------------------------------------------------------------------ */
hpac_status hpac_region_adjoint(hpac_region *region, const void *d_in, void *d_grad);

/* Vector-Jacobian product of the exact region (the backward pass of a
 * differentiable region call): d_grad[d * n + i] = d_gout[i] * d out_i / d in_{d,i}.
 * d_gout: n values of the region dtype (device), the derivative of a scalar
 * loss with respect to each output. Same regions, layout and errors as
 * hpac_region_adjoint; HPAC_EINVAL if d_gout is NULL for n > 0. Asynchronous
 * on the region's stream. */
hpac_status hpac_region_vjp(hpac_region *region, const void *d_in, const void *d_gout, void *d_grad);

/* ------------------------------------------------------------------------
 * Learned surrogate of a region (not from the paper): an MLP
 * n_feat -> hidden -> hidden -> 1 with GELU (tanh form), BF16 weights and
 * activations and FP32 accumulation; layer 1 on FP32 features, layer 2 (in
 * inference, training and input derivatives), the backward product
 * dh1 = dz2 W2 and the training gradient's contractions over the samples on
 * the tcgen05 tensor cores with tensor-memory accumulators. Their
 * kernels bound every wait on a tensor-core product; a wait that gives up is
 * reported as HPAC_ETIMEOUT by the next call that returns statistics or a
 * loss (hpac_mlp_infer with h_stats, hpac_mlp_grad / hpac_mlp_train with
 * h_loss). Black-Scholes features: ln(S/K), sigma sqrt(T), r T, d1 (the
 * Black-Scholes d1 clamped to [-10, 10]), sigma;
 * output C = S (out_shift + out_scale net). EOS features: e, v_{n+1}, dv, q
 * (as FP32); output p = m max(out_shift + out_scale net, 0) with the
 * multiplier m = (gamma - 1) max(e - dv q, 0) / v_{n+1} (the ideal-gas
 * pressure after the viscous work; 0 for an untouched element). Features are
 * normalized as (f - feat_shift) * feat_scale. Trained with Adam (beta 0.9 / 0.999,
 * eps 1e-8, cosine-decayed step) on the mean squared error of net against the
 * normalized region outputs.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t kind;            /* HPAC_REGION_BLACKSCHOLES (n_feat 5) or HPAC_REGION_EOS (4) */
  int32_t n_feat;
  int32_t hidden;          /* 64 or 128                                            */
  int32_t reserved0;
  float feat_shift[8];
  float feat_scale[8];
  float out_shift, out_scale;
} hpac_mlp_desc;

typedef struct hpac_mlp hpac_mlp;

/* Create a surrogate on the current device, enqueued on cuda_stream.
 * h_params: hpac_mlp_num_params FP32 values (W1 [hidden][n_feat], b1, W2
 * [hidden][hidden], b2, W3 [hidden], b3) or NULL for a seeded uniform
 * +-1/sqrt(fan_in) initialization with zero biases. */
hpac_status hpac_mlp_create(const hpac_mlp_desc *desc, const float *h_params, uint64_t seed,
                            void *cuda_stream, hpac_mlp **out);
hpac_status hpac_mlp_destroy(hpac_mlp *mlp);
int32_t hpac_mlp_num_params(const hpac_mlp *mlp);
hpac_status hpac_mlp_get_params(hpac_mlp *mlp, float *h_params);
hpac_status hpac_mlp_set_params(hpac_mlp *mlp, const float *h_params); /* resets Adam */

/* Set the feature and output normalisation (feat_shift/feat_scale to the
 * mean and 1/std of each feature, out_shift/out_scale to the mean and std of
 * the targets divided by the output multiplier) from n training invocations;
 * waits for the result. Allocates 144 bytes of device memory for the call. */
hpac_status hpac_mlp_fit_normalization(hpac_mlp *mlp, int64_t n, const void *d_in,
                                       int64_t in_stride, double param, const float *d_target);

/* Copy the surrogate's current descriptor (normalisation included). */
hpac_status hpac_mlp_get_desc(const hpac_mlp *mlp, hpac_mlp_desc *out);

/* Inference over n invocations of the region inputs (the region's layout:
 * float for Black-Scholes, double for EOS; param = r or gamma). d_out: n
 * outputs in the region's dtype (float / double). fallback_below: where a Black-Scholes prediction is below this price
 * the exact region is evaluated instead (NaN: never); d_mask (nullable) gets
 * HPAC_MASK_APPROX for surrogate outputs and HPAC_MASK_EXACT for fallbacks;
 * h_stats (nullable, synchronous) counts approximated = surrogate outputs. */
hpac_status hpac_mlp_infer(hpac_mlp *mlp, int64_t n, const void *d_in, int64_t in_stride,
                           double param, void *d_out, float fallback_below, uint8_t *d_mask,
                           hpac_stats *h_stats);

/* Calibrated fallback bound of a surrogate (the exact region as judge of its
 * error; not in the paper). On n held-out invocations with surrogate
 * predictions d_pred (floats) and exact region outputs d_exact (doubles, both
 * device), an invocation is bad when |pred - exact| > target |exact|. The
 * floor is the smallest prediction value v such that, among the k predictions
 * >= v, at most k - ceil(quantile k) are bad: the nearest-rank quantile of
 * the relative error over the invocations the surrogate would serve is
 * within target. -0 and +0 count as one value; NaN predictions are never at
 * or above a floor. *h_floor gets the floor (+inf when no v qualifies, so the
 * exact region serves everything; pass it as hpac_mlp_infer's fallback_below)
 * and *h_kept (nullable) the k at that floor. target >= 0 and finite,
 * quantile in (0, 1], 0 <= n <= 2^31. Waits for the result; allocates about
 * 12 bytes per invocation (rounded up to a power of two, at least 2048) of
 * device memory for the call. Errors: HPAC_EINVAL, HPAC_ECUDA. */
hpac_status hpac_calibrate_floor(int64_t n, const float *d_pred, const double *d_exact,
                                 double target, double quantile, float *h_floor,
                                 int64_t *h_kept, void *cuda_stream);

/* Gradient of the mean squared error over n invocations with targets d_target
 * (region outputs, n floats) into d_grad (num_params floats, overwritten; NULL:
 * the surrogate's internal buffer). h_loss (nullable, synchronous): the loss. */
hpac_status hpac_mlp_grad(hpac_mlp *mlp, int64_t n, const void *d_in, int64_t in_stride,
                          double param, const float *d_target, float *d_grad, float *h_loss);

/* Adam training: `epochs` passes over the n invocations in consecutive
 * batches of `batch`, each one gradient launch and one update launch; lr is
 * the peak step size. h_loss (nullable, synchronous): final loss over all n. */
hpac_status hpac_mlp_train(hpac_mlp *mlp, int64_t n, const void *d_in, int64_t in_stride,
                           double param, const float *d_target, int32_t batch, int32_t epochs,
                           float lr, float *h_loss);

/* Derivatives of the surrogate's region output with respect to the region
 * inputs (the surrogate's counterpart of hpac_region_adjoint): d_grad receives
 * 4 x n floats, row d at d_grad[d * n + i]. Asynchronous on the surrogate's
 * stream. Errors: HPAC_EINVAL (NULL surrogate, inputs or d_grad with n > 0,
 * n < 0, stride < n), HPAC_ECUDA, HPAC_EUNSUPPORTED (the kernel does not fit
 * an SM). */
hpac_status hpac_mlp_input_grad(hpac_mlp *mlp, int64_t n, const void *d_in, int64_t in_stride,
                                double param, float *d_grad);

/* Vector-Jacobian products of the surrogate's region output as hpac_mlp_infer
 * returns it without fallback (the backward pass of a differentiable surrogate
 * call): given d_gout (n floats, device: the derivative of a scalar loss with
 * respect to each output), d_grad_params (nullable; n_params floats, device,
 * overwritten) receives sum_i gout_i d out_i / d params with the bfloat16
 * rounding of weights and activations passed through as the identity, and
 * d_grad_in (nullable; 4 x n floats, row d at d_grad_in[d * n + i])
 * receives gout_i d out_i / d in_{d,i}. An EOS output clamped at zero has zero
 * derivative. Asynchronous on the surrogate's stream. Errors: HPAC_EINVAL
 * (NULL surrogate, inputs or d_gout, n < 0, stride < n), HPAC_ECUDA. */
hpac_status hpac_mlp_vjp(hpac_mlp *mlp, int64_t n, const void *d_in, int64_t in_stride,
                         double param, const float *d_gout, float *d_grad_params,
                         float *d_grad_in);

/* Replace the surrogate's parameters from device memory (n_params floats in
 * the layout of hpac_mlp_get_params): an asynchronous device-to-device copy on
 * the surrogate's stream, so a caller can keep the parameters as its own
 * tensor (for example a framework's trainable parameter) and load them before
 * each call. */
hpac_status hpac_mlp_set_params_device(hpac_mlp *mlp, const float *d_params);

/* Measured double-precision FMA rate of the current device in TFLOP/s
 * (2 flops per FMA), from a kernel of independent FMA chains on every SM: the
 * arithmetic ceiling of the FP64-bound hydro kernels. Not from the paper.
 * Waits for its own work; allocates 8 bytes of device memory for the call. */
hpac_status hpac_device_fp64_rate(double *h_tflops, void *cuda_stream);

/* hpac_quality without any allocation, for callers that cannot call cudaMalloc:
 * code that runs after a service has reserved all of its device memory up front
 * (through its own pool, or a framework's caching allocator that owns every
 * free byte), or that must not enter the CUDA allocator at all once it is
 * running. The paper has no counterpart; this is a library convenience.
 * Same arguments, layout and result as hpac_quality, with these differences:
 *  - Scratch is a fixed array inside the library (about 656 KB on every device
 *    that loads it, held until the process exits), so n must not exceed
 *    134,217,728 elements; larger n returns HPAC_EINVAL with a message.
 *  - The first call on a device, made with that device current, finds the
 *    array's device address and caches it. A call with n = 0 does that set-up
 *    and also makes the CUDA runtime load the call's kernels (with lazy
 *    module loading, the default, a kernel's code is loaded, into newly
 *    allocated device memory, at its first use), then returns without
 *    launching anything. Make one such call per device before the caller
 *    reserves that device's memory; later calls then allocate nothing.
 *  - Like hpac_quality, the call copies its result to the host and waits for
 *    it, so it must not be made on a stream that is being captured.
 *  - Every call on a device uses the same array. A call waits for its own
 *    result, but calls issued from several host threads whose work overlaps on
 *    the GPU race on the array: serialize them.
 *  - The cached address belongs to the device's primary context: resetting
 *    the device (cudaDeviceReset) while the library is in use invalidates it. */
hpac_status hpac_quality_noalloc(int32_t approx_dtype, int64_t n, const double *d_exact,
                                 const void *d_approx, int32_t metric,
                                 hpac_quality_result *h_result, void *cuda_stream);

/* Message for the last non-OK status returned on the calling host thread. */
const char *hpac_last_error(void);

/* Library version string. */
const char *hpac_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HPAC_H_ */
