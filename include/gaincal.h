/*
 * gaincal.h -- C ABI of the GB300 gain-calibration library (libgaincal.so).
 *
 * Method: Smirnov & Tasse, "Radio interferometric gain calibration as a complex
 * optimization problem" (arXiv:1502.06974).  The library solves, for many independent
 * solution intervals at once,
 *
 *     min_g  sum_{pq s} | d_pqs - g_p m_pqs conj(g_q) |^2               (Sect. 2.3, eq. cal:DI:tf)
 *     min_G  sum_{pq s} || D_pqs - G_p M_pqs G_q^H ||_F^2                (Sect. 4, eq. cal:DI:pol)
 *     min_g  sum_{pq s} | d_pqs - sum_d g_p^(d) m^(d)_pqs conj(g_q^(d)) |^2   (Sect. 2.5, eq. cal:dd:unpol)
 *
 * with the approximate-inverse iterations of Sect. 3: StefCal (eq. stefcal, with the
 * GN/average alternation of eq. stefcal-lambda-average), its 2x2 form (eq. update:DI:diag:pol,
 * computed as [sum D Y^H][sum Y Y^H]^-1) and CohJones (Sect. 3.2.2, N_d x N_d antenna blocks).
 *
 * ---------------------------------------------------------------------------------------
 * Data layout (all kinds)
 *   A "row" is one (baseline, sample) pair.  Interval i owns the rows
 *       row_off[i] .. row_off[i] + n_samp[i] * n_bl[i] - 1
 *   stored sample-major, baseline-minor (row = row_off[i] + s * n_bl[i] + b).  A sample is one
 *   (time, channel) point of the interval (Sect. 2.3: the sample index s).  Baseline b of
 *   interval i is the antenna pair (ant1[bl_off[i] + b], ant2[bl_off[i] + b]); antenna numbers
 *   are local to the interval (0 .. n_ant[i]-1).  Either orientation may be stored, since
 *   d_qp = conj(d_pq) (Sect. 2.1) and D_qp = D_pq^H (Sect. 4); a pair with ant1 == ant2 is an
 *   error (autocorrelations are excluded, Sect. 2.1).  Intervals may share baseline tables.
 *
 *   Element types (dtype):
 *     scalar  vis, model, gains: complex (re, im) pairs; GC_DTYPE_C64 = 2 x float,
 *             GC_DTYPE_C128 = 2 x double.
 *     jones   one row = a 2x2 complex matrix stored row-major [x00, x01, x10, x11]
 *             (32 bytes in C64); a gain is one such 2x2 matrix per antenna.
 *     dd      vis: one complex per row; model: n_dir planes, model[d * n_rows + row];
 *             gains: gains[(gain_off[i] + p) * n_dir + d].
 *   Gains of interval i occupy slots gain_off[i] .. gain_off[i] + n_ant[i] - 1.
 *
 * Ownership and synchronisation
 *   - gc_layout and every array it points to are HOST memory, read during the call only.
 *   - With opt->host_buffers == 0, vis, model, gains and the per-interval outputs are DEVICE
 *     pointers owned by the caller; work is queued on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) and the call returns once every interval has converged or reached
 *     max_iter (the host reads a device flag between iteration batches); results are then
 *     complete on `stream`.
 *   - With opt->host_buffers == 1 the same pointers are HOST memory (pinned is fastest); the
 *     library copies inputs to the device, solves, and copies gains and outputs back before
 *     returning.
 *   - The library keeps a per-process device workspace that grows on demand; gc_release()
 *     frees it.  Calls must not run concurrently from several host threads.
 *
 * Errors
 *   Return value: GC_OK (0) when every interval converged; a positive count of intervals whose
 *   status is not GC_ST_OK; or a negative GC_ERR_* code, in which case nothing was launched
 *   (argument errors) or the CUDA error is reported (GC_ERR_CUDA).  The library never aborts and
 *   never traps on the device.
 */
#ifndef GAINCAL_H
#define GAINCAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define GC_OK 0
#define GC_ERR_ARG (-1)      /* NULL pointer where one is required, or a bad option value     */
#define GC_ERR_LAYOUT (-2)   /* offsets / counts out of range or inconsistent                 */
#define GC_ERR_ANTENNA (-3)  /* antenna index outside 0..n_ant-1, or ant1 == ant2            */
#define GC_ERR_DTYPE (-4)    /* dtype not supported by this entry point                       */
#define GC_ERR_CUDA (-5)     /* a CUDA runtime call failed (see gc_last_cuda_error)          */
#define GC_ERR_LIMIT (-6)    /* a size beyond a documented maximum                            */

/* ---- per-interval status (status_out[i]) ---- */
#define GC_ST_OK 0            /* converged: ||g_k+1 - g_k|| <= tol ||g_k+1||                  */
#define GC_ST_NOT_CONVERGED 1 /* stopped at max_iter                                           */
#define GC_ST_NONFINITE 2     /* a NaN/Inf appeared in the gains; the interval was stopped     */
#define GC_ST_NODATA 3        /* the interval has no rows; gains left unchanged, iters = 0     */
#define GC_ST_SINGULAR_FLAG 16 /* OR-ed in: at the last update some antenna's J^H J block was
                                  not invertible (e.g. no unflagged baselines); that antenna's
                                  gain was left unchanged                                     */

#define GC_DTYPE_C64 0
#define GC_DTYPE_C128 1

#define GC_SCHED_STEFCAL 0  /* odd k: GN step; even k: LM step with lambda = 1 = average (Sect. 3.1) */
#define GC_SCHED_GN 1       /* GN step every iteration                                        */
#define GC_SCHED_LM 2       /* opt->lm_after StefCal iterations, then Levenberg-Marquardt with the whole
                               J^H J (App. C, Algorithm LM; Sect. 1, eq. LM): see gc_options     */

/* Levenberg-Marquardt (GC_SCHED_LM) limits and defaults */
#define GC_LM_MAX_UNKNOWNS 512       /* real unknowns per interval: 8 x antennas (2x2), 2 x antennas (scalar) */
#define GC_LM_DEFAULT_AFTER 20       /* StefCal iterations before the first LM step                 */
#define GC_LM_DEFAULT_LAMBDA0 1e-2   /* initial damping                                             */
#define GC_LM_DEFAULT_K 10.0         /* damping factor K of App. C                                   */

#define GC_MAX_ANT 1024      /* antennas per interval                                          */
#define GC_MAX_DIR 10        /* directions for the DD entry point                              */

typedef struct gc_layout {
  int32_t n_intervals;
  const int64_t* row_off;   /* [n_intervals] first row of each interval                     */
  const int32_t* n_samp;    /* [n_intervals] samples (time x channel points) per interval   */
  const int32_t* n_bl;      /* [n_intervals] baselines per interval                         */
  const int32_t* bl_off;    /* [n_intervals] first entry of the interval in ant1/ant2       */
  const int32_t* n_ant;     /* [n_intervals] antennas (gain slots) per interval              */
  const int32_t* gain_off;  /* [n_intervals] first gain slot of the interval                 */
  int32_t n_bl_table;       /* entries in ant1 / ant2                                         */
  const int32_t* ant1;      /* [n_bl_table]                                                   */
  const int32_t* ant2;      /* [n_bl_table]                                                   */
  int64_t n_rows;           /* rows in vis (and per model plane)                              */
  int32_t n_gain;           /* gain slots                                                     */
  int32_t n_dir;            /* directions (dd only; 1 for the DI entry points)                */
} gc_layout;

typedef struct gc_options {
  double tol;               /* relative step tolerance (App. C, first criterion)               */
  int32_t max_iter;         /* >= 1                                                           */
  int32_t schedule;         /* GC_SCHED_*                                                     */
  int32_t dtype;            /* GC_DTYPE_*                                                     */
  int32_t host_buffers;     /* 0: data pointers are device memory; 1: host memory              */
  int32_t compute_chi2;     /* 1: fill chi2_out with sum |r|^2 at the final gains              */
  int32_t profile;          /* 1: time the iteration kernels with CUDA events on `stream`;
                               2 (moment path): time the accumulate launches alone, one launch
                               per iteration without graph segments;
                               read the totals with gc_profile_last / gc_profile_detail        */
  int32_t path;             /* DI entry points: GC_PATH_AUTO / _STREAM / _MOMENTS / _RESIDENT     */
  int32_t reserved;         /* must be 0                                                      */
  /* GC_SCHED_LM only (DI entry points, complex64, moment path):
   *   The first lm_after iterations are StefCal's (GN / average alternation, no stopping), from
   *   the given gains.  Then every interval takes App. C's LM iterations: the whole J^H J of
   *   eq. JHJ:pol (2x2) or eq. JHJ:DI (scalar), off-diagonal antenna blocks included, and J^H R
   *   are formed at the current gains from the per-baseline moments; the step solves
   *       (J^H J + lambda diag(J^H J) + mu v v^T) dz = (I - v v^T) J^H R             (eq. LM)
   *   with v the unit phase-gauge direction i G (J^H J is singular along it, Sect. 2.1) and mu the
   *   mean of diag(J^H J) -- the LM step in the complement of the gauge direction; the matrix is
   *   factored in FP32 (Cholesky).  chi^2 at the trial gains is evaluated in FP64; a step that
   *   lowers it is kept and lambda /= lm_K, otherwise the gains are kept and lambda *= lm_K.  An
   *   interval stops (GC_ST_OK) after a step with ||dz|| <= tol ||G|| (App. C, first criterion),
   *   or at max_iter (every LM iteration, kept or not, counts as one iteration).
   *   Intervals with more than GC_LM_MAX_UNKNOWNS real unknowns: GC_ERR_LIMIT.           */
  int32_t lm_after;         /* StefCal iterations before LM, >= 0 (0: LM from the given gains;
                               GC_LM_DEFAULT_AFTER suits a start far from the solution)          */
  int32_t lm_reserved;      /* must be 0                                                      */
  double lm_lambda0;        /* initial lambda; 0 selects GC_LM_DEFAULT_LAMBDA0                   */
  double lm_K;              /* lambda factor, > 1; 0 selects GC_LM_DEFAULT_K                     */
  /* Per-row weights (Sect. 2.4, eq. LSmin:w with a diagonal W; eqs. JHJ:DI:tfw, JHR:DI:tfw): NULL
   * for unit weights, else [n_rows] non-negative reals (float for GC_DTYPE_C64, double for
   * GC_DTYPE_C128; device memory, or host memory with host_buffers).  Row r's weight multiplies its
   * terms in every sum over rows (J^H W J, J^H W R, J^H W D, chi^2); one weight serves the four
   * correlations of a 2x2 row.  Taken by the DI entry points on the moment and streaming paths
   * (and GC_SCHED_LM); GC_PATH_RESIDENT and the DD entry points return GC_ERR_ARG when it is set. */
  const void* weights;
} gc_options;

/* Execution paths of the direction-independent solvers (same results up to FP32 rounding order):
 *   GC_PATH_STREAM    every iteration is one launch that re-reads all rows of the active intervals;
 *   GC_PATH_MOMENTS   one pass reduces each interval's samples to per-baseline moments (the gains
 *                     factor out of the sample sums); every iteration is then one launch that
 *                     reads the moments of the active intervals (FP32 only);
 *   GC_PATH_RESIDENT  one pass reduces each interval's samples to per-baseline moments (the gains
 *                     factor out of the sample sums), then one persistent launch of thread-block
 *                     clusters iterates every interval to convergence with its moments held on chip.
 *                     FP32 only; up to 256 antennas and 8 x 512 baselines (scalar: 8 x 2048) per
 *                     interval.
 *   GC_PATH_AUTO      MOMENTS for complex64 data, STREAM for complex128. */
#define GC_PATH_AUTO 0
#define GC_PATH_STREAM 1
#define GC_PATH_RESIDENT 2
#define GC_PATH_MOMENTS 3

/*
 * Direction-independent scalar gains: StefCal (Sect. 3.1, eq. stefcal and
 * eq. stefcal-lambda-average) over every interval of `layout`.
 *   vis, model  [n_rows] complex (dtype C64 or C128)
 *   gains       [n_gain] complex, read as the starting point, overwritten with the solution
 *   iters_out   [n_intervals] int32, iterations taken (may be NULL)
 *   chi2_out    [n_intervals] double, sum |r|^2 at the solution when opt->compute_chi2 (may be NULL)
 *   status_out  [n_intervals] int32 GC_ST_* (may be NULL)
 */
int gc_calibrate_di_scalar(const void* vis, const void* model, const gc_layout* layout, void* gains,
                           const gc_options* opt, int32_t* iters_out, double* chi2_out,
                           int32_t* status_out, void* stream);

/*
 * Direction-independent full-Jones 2x2 gains: polarized StefCal (Sect. 4.2,
 * eq. update:DI:diag:pol, product order [sum_q D_pq Y_pq^H][sum_q Y_pq Y_pq^H]^-1 with
 * Y_pq = M_pq G_q^H), same schedule and arguments as gc_calibrate_di_scalar; vis, model and
 * gains hold 2x2 matrices (row-major).
 */
int gc_calibrate_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                             const gc_options* opt, int32_t* iters_out, double* chi2_out,
                             int32_t* status_out, void* stream);

/*
 * Direction-dependent scalar gains: CohJones (Sect. 3.2.2).  Per antenna p the N_d x N_d
 * block A_p[c][d] = sum_{q,s} conj(y^(c)) y^(d), y^(d) = m^(d) conj(g_q^(d)) (eq. JHJ:DD:unpol)
 * is solved against J^H d (eq. JHR:DD:unpol, data form of eq. ghat) by a Cholesky factorisation
 * in FP32 refined once against a float-float residual; when an FP32 pivot is not positive the
 * block is factored in FP64, and a block FP64 cannot factor keeps the antenna's gains and sets
 * GC_ST_SINGULAR_FLAG in its interval's status.  The sums over samples are first reduced to
 * per-baseline moments
 * X^(cd)_pq = sum_s conj(m^(c)) m^(d) and b^(c)_pq = sum_s conj(m^(c)) d (Sect. 3.2.1, the
 * gains factor out of the sample sum), read once per interval.
 *   vis    [n_rows] complex64; model [n_dir][n_rows] complex64; gains [n_gain][n_dir] complex64.
 * Only GC_DTYPE_C64.  n_dir <= GC_MAX_DIR.
 */
int gc_calibrate_dd_cohjones(const void* vis, const void* model, const gc_layout* layout, void* gains,
                             const gc_options* opt, int32_t* iters_out, double* chi2_out,
                             int32_t* status_out, void* stream);

/*
 * Direction-dependent scalar gains: AllJones (Sect. 3.2.3, eq. stefcal:dd:unpol).  The whole
 * J^H J is taken as its diagonal, so the step goes through the residuals:
 *   g_p^(d) += c_p^(d) / sum_{q,s} |y^(d)|^2,   c_p^(d) = sum_{q,s} conj(y^(d)) r_pqs,
 * every antenna and direction independently.  c is formed from the same per-baseline moments as
 * CohJones (c_p = b_p - A_p g_p, an identity of the residual sum), in float-float.  A direction
 * with no signal at an antenna keeps its gain and sets GC_ST_SINGULAR_FLAG.  Same schedule
 * (odd iterations the step, even ones its average with the current gains), layout, arguments and
 * limits as gc_calibrate_dd_cohjones.
 */
int gc_calibrate_dd_alljones(const void* vis, const void* model, const gc_layout* layout, void* gains,
                             const gc_options* opt, int32_t* iters_out, double* chi2_out,
                             int32_t* status_out, void* stream);

/*
 * Direction-dependent 2x2 gains (Sect. 4.4, eqs. JHJ:DD:pol, JHR:DD:pol), with Y^(d) = M^(d) G_q^(d)H.
 * Per antenna p, H (2Nd x 2Nd, 2x2 block (c, d) = sum_{q,s} Y^(c) Y^(d)H) and
 * CD = [.. sum_{q,s} D Y^(d)H ..] (2 x 2Nd); the antenna's normal equations are
 * [G^(1) .. G^(Nd)] H = CD (the 4Nd x 4Nd operator block R_H, inverted as R_{H^-1}).
 *   gc_calibrate_dd_cohjones2x2: polarized CohJones, [G^(1) .. G^(Nd)] = CD H^-1 (data form), H
 *     factored in FP32 and the solution refined once against a float-float residual; FP64 when an
 *     FP32 pivot fails; an antenna FP64 cannot factor keeps its gains (GC_ST_SINGULAR_FLAG).
 *   gc_calibrate_dd_alljones2x2: polarized AllJones (eq. update:DD:diag:pol),
 *     G^(d) += [sum R Y^(d)H] [sum Y^(d) Y^(d)H]^-1 per antenna and direction (residual form).
 * The sums over samples are taken once per interval as the Hermitian Gram matrix of each
 * baseline's stacked row [D, M^(1) .. M^(Nd)] (16 (Nd + 1)(Nd + 2) / 2 complex values per baseline).
 *   vis [n_rows][2][2] complex64 (row-major 2x2); model [n_dir][n_rows][2][2]; gains
 *   [n_gain][n_dir][2][2].  vis and model 16-byte aligned (device buffers; GC_ERR_ARG otherwise).
 * Same schedule, options, outputs and limits as gc_calibrate_dd_cohjones; only GC_DTYPE_C64.
 */
int gc_calibrate_dd_cohjones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                int32_t* status_out, void* stream);
int gc_calibrate_dd_alljones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                int32_t* status_out, void* stream);

/*
 * Smoothing in time and frequency (Sect. 3.4, eqs. cal:DI:smooth, stefcal:w, JHJ:diag:smooth).
 * Every sample (t, f) of an n_t x n_f grid has its own gains; each iteration replaces the sums of
 * StefCal's update by their convolutions with a separable Gaussian kernel over the grid,
 *   scalar: g_p(t, f) = (w o alpha_p)(t, f) / (w o beta_p)(t, f),
 *           alpha_p = sum_q conj(y_pq) d_pq, beta_p = sum_q |y_pq|^2 at each sample;
 *   2x2:    G_p(t, f) = (w o C_p)(t, f) (w o H_p)(t, f)^-1, C_p = sum_q D Y^H, H_p = sum_q Y Y^H;
 * w(dt, df) = exp(-dt^2 / 2 sigma_t^2) exp(-df^2 / 2 sigma_f^2) on the sample grid, cut at
 * |dt| <= ceil(3 sigma_t), |df| <= ceil(3 sigma_f) and at the grid's edges (sigma = 0: no
 * smoothing along that axis).  Odd iterations take these gains, even ones their average with the
 * current ones (opt->schedule as for the DI solvers); the grid stops as a whole when
 * ||g_{k+1} - g_k|| <= tol ||g_{k+1}|| over every sample and antenna.  A sample and antenna whose
 * smoothed sum is singular keeps its gains (GC_ST_SINGULAR_FLAG).
 *   vis, model [n_t][n_f][n_bl] rows (complex64; 2x2 row-major for the 2x2 entry point), device;
 *   gains [n_t][n_f][n_ant] (2x2: [..][2][2]) in/out, device; ant1/ant2 host [n_bl].
 *   iters_out, status_out: one value each (device); chi2_out: [n_t * n_f] per-sample chi^2 (device,
 *   opt->compute_chi2).  Only GC_DTYPE_C64, device buffers, no weights.  Synchronous; returns 0
 *   when the grid converged, 1 when not, or a GC_ERR_* code.
 */
typedef struct gc_smooth {
  int32_t n_t, n_f;         /* sample grid (time-major)                                      */
  int32_t n_bl;             /* baselines per sample                                          */
  int32_t n_ant;            /* antennas                                                      */
  const int32_t* ant1;      /* host [n_bl]                                                   */
  const int32_t* ant2;      /* host [n_bl]                                                   */
  double sigma_t, sigma_f;  /* kernel widths in samples, >= 0                                */
} gc_smooth;
int gc_calibrate_di_smooth_scalar(const void* vis, const void* model, const gc_smooth* sm, void* gains,
                                  const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                                  void* stream);
int gc_calibrate_di_smooth_jones2x2(const void* vis, const void* model, const gc_smooth* sm, void* gains,
                                    const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                                    void* stream);

/*
 * One accumulation pass, no update: for every gain slot p of every interval, the top half of
 * J^H d and the diagonal block of J^H J at the given gains (device pointers, work on `stream`,
 * asynchronous).
 *   scalar (eqs. JHJ:DI:tf, JHR:DI:tf in data form):
 *     jhd_out [n_gain] complex  = sum_{q,s} conj(y_pqs) d_pqs,  y_pqs = m_pqs conj(g_q)
 *     jhj_out [n_gain] real     = sum_{q,s} |y_pqs|^2
 *   jones (eq. JHJ:pol diagonal and the polarized J^H D):
 *     jhd_out [n_gain] 2x2 complex = sum_{q,s} D_pqs Y_pqs^H,  Y_pqs = M_pqs G_q^H
 *     jhj_out [n_gain] 2x2 complex = sum_{q,s} Y_pqs Y_pqs^H   (Hermitian, both triangles written)
 * Types follow `dtype` (C64: float, C128: double).
 */
int gc_jhj_jhr_di_scalar(const void* vis, const void* model, const gc_layout* layout, const void* gains,
                         int32_t dtype, void* jhd_out, void* jhj_out, void* stream);
int gc_jhj_jhr_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, const void* gains,
                           int32_t dtype, void* jhd_out, void* jhj_out, void* stream);

/*
 * gc_jhj_jhr_di_jones2x2 for callers that cannot allocate device memory.  (This entry point has no
 * counterpart in the paper; it is a deployment variant of the accumulation pass above.)
 *
 * Who needs it: a caller that must not let a library call cudaMalloc -- for example a real-time
 * pipeline that reserves all device memory when it starts and cannot afford an allocation that
 * fails or stalls later, or an application whose own allocator owns the device memory.  This call
 * allocates nothing: apart from the caller's inputs and outputs, everything the kernel needs (a
 * copy of the layout, the reduction slot lists, work items, per-interval state and the per-item
 * scratch sums) lives in one static device array of GC_NOALLOC_MAX_BYTES, which every GPU that
 * loads the library holds until the process exits.
 *   - Arguments, layouts and results are exactly those of gc_jhj_jhr_di_jones2x2 (device
 *     pointers; the layout arrays are host memory).  At most 64 distinct baseline tables, n_dir 1.
 *   - Returns GC_ERR_LIMIT when the layout, its work items and scratch need more than
 *     GC_NOALLOC_MAX_BYTES; nothing is launched then.
 *   - The first call on a device, with that device current, looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any stream capture.
 *   - All calls share the array and each call overwrites it (its state is re-initialised on the
 *     device at the start of every call).  Calls whose GPU work overlaps -- on different streams
 *     or from different host threads -- race; serialise them on one stream.
 *   - The work is queued on `stream` and the call returns once the layout has been copied out of
 *     the library's host staging area.
 */
#define GC_NOALLOC_MAX_BYTES (4u << 20)
int gc_jhj_jhr_di_jones2x2_noalloc(const void* vis, const void* model, const gc_layout* layout,
                                   const void* gains, int32_t dtype, void* jhd_out, void* jhj_out,
                                   void* stream);

/*
 * Autotuner for the direction-independent solvers (launch shapes only; results are the same up to
 * FP32 summation order).  Runs `iters` iterations (tol 0) of gc_calibrate_di_scalar (kind 0) or
 * gc_calibrate_di_jones2x2 (kind 1) with each candidate shape -- reduction split, how the next
 * tile is brought in (none, registers, per-thread copies, or bulk copies into a shared-memory
 * ring), CTAs per SM for the moment path; rows per work item and CTAs per SM for the raw-row
 * path -- on the
 * caller's data, and records the fastest for the layout's shape bucket (kind, dtype, path, and
 * the powers of two of the interval count, largest baseline count and mean samples per interval).
 * Later calls with a layout in that bucket use it.  vis, model and gains are device pointers;
 * `gains` is restored before returning.  best_ms (may be NULL) receives the fastest time of the
 * iteration kernels.  Synchronous.
 */
int gc_autotune_di(int32_t kind, const void* vis, const void* model, const gc_layout* layout, void* gains,
                   int32_t dtype, int32_t iters, double* best_ms, void* stream);

/*
 * Totals of the last gc_calibrate_* call made with opt->profile = 1 or 2: summed device time of
 * its iteration launches (profile 2: of its accumulate launches only) in ms from CUDA events on the
 * call's stream, the number of iterations timed, and rows processed by them (sum over intervals
 * of iterations x rows).  With GC_SCHED_LM these are the diagonal iterations; gc_profile_lm reports
 * the LM phase.  Any pointer may be NULL.
 */
int gc_profile_last(double* iter_kernel_ms, int64_t* iter_launches, int64_t* row_iterations);
/* More of the same profile: the moment-pass time (ms; 0 on the streaming path), baselines x
 * iterations processed, and the path taken (GC_PATH_STREAM, GC_PATH_MOMENTS or GC_PATH_RESIDENT;
 * GC_PATH_MOMENTS for gc_calibrate_dd_cohjones, whose iteration launches are the per-antenna
 * N_d x N_d solves over the moments). */
int gc_profile_detail(double* moment_pass_ms, int64_t* baseline_iterations, int32_t* path);

/*
 * chi^2 = sum |r|^2 per interval at the given 2x2 gains (eq. cal:DI:pol with the sample sums of
 * Sect. 2.3), FP32 compensated sums, FP64 totals.  vis/model/gains device pointers, complex64 or
 * complex128 per dtype; chi2_out [n_intervals] double (device).  Asynchronous on `stream`.
 */
int gc_chi2_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, const void* gains,
                        int32_t dtype, double* chi2_out, void* stream);

/* ---- learned warm start --------------------------------------------------------------------
 * A small MLP (in -> h1 -> h2 -> out, ReLU on the hidden layers) proposes each interval's starting
 * gains from the antenna's earlier solutions; the iteration then runs to the usual tolerance from
 * that start, so the network only changes where the solver starts and a poor proposal costs
 * iterations, never accuracy.  The paper has no counterpart; its Sect. 3.4 (gains do not
 * vary arbitrarily in time and frequency) is what makes earlier solutions informative.
 * Parameter buffer `params` (float, device): W1 [in][h1] | b1 [h1] | W2 [h1][h2] | b2 [h2] |
 * W3 [h2][out] | b3 [out], row-major with y = x W + b.  grads, adam_m, adam_v: same size (training
 * only); params_bf16: same count of bfloat16 (inference; rewritten from params by each inference).
 * Supported shape: 48, 256, 256, 8 (GC_ERR_LIMIT otherwise).  Buffers are owned by the caller.
 * Activations are row-major [n][width] floats (device).  All calls asynchronous on `stream`. */
typedef struct gc_mlp {
  int32_t in, h1, h2, out;
  float* params;
  float* grads;
  float* adam_m;
  float* adam_v;
  void* params_bf16;
} gc_mlp;
/* floats of work buffer the FP32 forward / gradient / training calls need for n rows */
size_t gc_mlp_work_floats(const gc_mlp* net, int32_t n);
/* FP32 forward: y [n][out] */
int gc_mlp_forward_f32(const gc_mlp* net, const float* x, int32_t n, float* y, float* work, void* stream);
/* FP32 gradient of the mean squared error mean((y - t)^2) over n x out: grads (like params), loss
 * (one float, device) */
int gc_mlp_grad_f32(const gc_mlp* net, const float* x, const float* t, int32_t n, float* grads, float* loss,
                    float* work, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected at `step` >= 1) on that gradient */
int gc_mlp_train_step(gc_mlp* net, const float* x, const float* t, int32_t n, float lr, int32_t step, float* loss,
                      float* work, void* stream);
/* BF16 inference (weights converted from params, activations rounded to bfloat16, FP32 sums) */
int gc_mlp_infer_bf16(const gc_mlp* net, const float* x, int32_t n, float* y, void* stream);
/* Network inputs per (interval, antenna) row: hist [n][hist_stride >= 32] holds the antenna's 4
 * previous 2x2 gains newest first (each row-major (re, im) pairs); jhd/jhj [n][8] the 2x2 blocks
 * C = sum D Y^H and H = sum Y Y^H (as gc_jhj_jhr_di_jones2x2 writes them) at the newest of them
 * on the target interval; lead [n] the scaled lead time.  With phi = arg of the newest gain's xx
 * element: x [n][in_width >= 41] = e^{-i phi} [g1 | g1-g2 | g2-g3 | g3-g4 | C H^-1 - g1] | lead |
 * zeros (the C H^-1 entries are zero where H is singular), rot [n][2] = (cos phi, sin phi). */
int gc_ws_features_jones(const float* hist, int32_t hist_stride, const float* jhd, const float* jhj, const float* lead,
                         int32_t n, int32_t in_width, float* x, float* rot, void* stream);
/* Training target [n][8] = e^{-i phi} (g_next - g1), the network output that would propose g_next. */
int gc_ws_target_jones(const float* g1, const float* g_next, const float* rot, int32_t n, float* target,
                       void* stream);
/* Training-set preparation for the network (device pointers, asynchronous on `stream`).
 * gc_rows_gather_f32: dst[r][:] = src[index[r]][:] for r < n, rows of `width` floats (index int64,
 *   device; every entry must address a row of src: not checked).
 * gc_col_stats_f32: per column of x [.][width] over the rows index[0..n-1] (rows 0..n-1 when index
 *   is NULL), the FP64 mean and population standard deviation (two passes); a column whose
 *   deviation is below 1e-12 gets sd = 1 and, when zero_const_mean, mean = 0.  n >= 1.
 * gc_standardize_f32: out = (x - mean) / sd per column in FP64, rounded to FP32 (mean may be NULL:
 *   out = x / sd); out may equal x.
 * gc_mlp_fold_standardization: rewrite the network in place so that it takes raw inputs and
 *   returns raw outputs: with W1, b1 the first layer and W3, b3 the last, b1 -= (mean/sd) W1,
 *   W1 /= sd (per input row), W3 *= tsd and b3 *= tsd (per output column), in FP64.  mean/sd
 *   [in], tsd [out], device.
 * Each returns GC_OK, GC_ERR_ARG (bad size or NULL), GC_ERR_LIMIT (network shape) or GC_ERR_CUDA. */
int gc_rows_gather_f32(const float* src, int32_t width, const int64_t* index, int64_t n, float* dst, void* stream);
int gc_col_stats_f32(const float* x, int32_t width, const int64_t* index, int64_t n, int32_t zero_const_mean,
                     double* mean, double* sd, void* stream);
int gc_standardize_f32(const float* x, int32_t width, int64_t n, const double* mean, const double* sd, float* out,
                       void* stream);
int gc_mlp_fold_standardization(gc_mlp* net, const double* mean, const double* sd, const double* tsd, void* stream);

/* Inputs of a warm-started solve. */
typedef struct gc_warm {
  const float* solutions;  /* device: earlier 2x2 solutions, [n_solutions][8] floats */
  int64_t n_solutions;     /* gain slots in `solutions` */
  const int32_t* hist_off; /* host [n_intervals][4]: slot in `solutions` of antenna 0 of each of the
                              interval's 4 previous solutions, newest first (n_ant[i] consecutive
                              slots each; GC_ERR_ARG if any lies outside [0, n_solutions)) */
  const float* lead;       /* host [n_intervals]: scaled lead time, a network input */
  const gc_mlp* net;       /* trained network, or NULL: the start is then the newest previous solution */
  int32_t* used_out;       /* optional, device [n_intervals]: 1 where the proposal was taken */
  double* dchi2_out;       /* optional, device [n_intervals]: chi^2(proposal) - chi^2(previous) */
  float* start_out;        /* optional, device [n_gain][8]: the start the iteration took */
} gc_warm;

/*
 * gc_calibrate_di_jones2x2 from a learned start.  Per interval, with g1 the newest previous
 * solution: one pass over the interval's per-baseline moments gives C, H and chi^2 at g1; the
 * network (BF16) proposes g1 + e^{i phi} delta from the features above; a second pass gives
 * chi^2 at the proposal; the iteration starts from the proposal if its chi^2 is lower, else from
 * g1, and runs exactly as gc_calibrate_di_jones2x2 does.  The chi^2 comparison drops the common
 * term sum |d|^2 and sums the per-antenna terms tr(G H G^H) - 2 Re tr(C G^H) in FP64.
 * Complex64 device buffers only (opt->dtype GC_DTYPE_C64, host_buffers 0, path AUTO or MOMENTS,
 * else GC_ERR_DTYPE / GC_ERR_ARG).  The initial content of `gains` is ignored; on return it holds
 * the solutions.  Returns like gc_calibrate_di_jones2x2.
 */
int gc_calibrate_di_jones2x2_warm(const void* vis, const void* model, const gc_layout* layout, const gc_warm* warm,
                                  void* gains, const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                  int32_t* status_out, void* stream);

/* A time-major grid of intervals solved as a wavefront with learned starts. */
typedef struct gc_wavefront {
  int32_t n_t, n_fb;     /* interval i = t * n_fb + f, t < n_t, f < n_fb; n_t * n_fb = n_intervals, and
                            every interval of block f has the antennas of interval f (GC_ERR_LAYOUT) */
  int32_t lag;           /* wave length L in time steps (>= 1) */
  int32_t max_lead;      /* the newest history time may lie up to max_lead (>= 1) steps before the
                            wave's first time: 1 = always the 4 times just before the wave */
  float lead_scale;      /* network input lead = (t - newest history time) / lead_scale (> 0) */
  double gate_tol;       /* a wave joins once every interval of its history stopped or took a relative
                            step <= gate_tol (gate_tol <= tol: only finished histories) */
  const gc_mlp* net;     /* trained network, or NULL: the start is the newest previous solution */
  int32_t* used_out;     /* optional, device [n_intervals]: 1 where the proposal was taken */
  int32_t* wave_k_out;   /* optional, host [ceil(n_t / lag)]: the global iteration after which each
                            wave joined (0 for the first) */
} gc_wavefront;

/*
 * The whole grid in one iteration loop.  The times [wL, (w+1)L) form wave w.  Wave 0 starts from
 * `gains`; wave w >= 1 joins the running iteration as soon as, for some history time th with
 * wL - max_lead <= th < wL, every interval at times th-3 .. th (clamped at 0) has finished or taken
 * a step below gate_tol (the newest such th is used).  It then starts as
 * gc_calibrate_di_jones2x2_warm does, from the solutions at th .. th-3 of the same block f, each put
 * in the canonical gauge, with lead t - th.  Every interval iterates to opt->tol with its own
 * iteration count
 * (iters_out counts from its first iteration; the GN / average alternation restarts with it).
 * On return `gains` holds the solutions in the canonical gauge (see gc_gauge_fix_di).
 * Complex64 device buffers only, as gc_calibrate_di_jones2x2_warm.  Returns the number of
 * intervals not converged, or GC_ERR_LIMIT if the loop bound (waves x max_iter iterations) ran out.
 */
int gc_calibrate_di_jones2x2_wavefront(const void* vis, const void* model, const gc_layout* layout,
                                       const gc_wavefront* wf, void* gains, const gc_options* opt, int32_t* iters_out,
                                       double* chi2_out, int32_t* status_out, void* stream);

/*
 * Canonical gauge (Sect. 2.1: chi^2 is unchanged by one phase on all antennas): each interval's
 * gains (device, kind 0 scalar or 1 2x2, dtype C64/C128) are rotated in place so that sum_p g_p
 * (scalar) or sum_p tr(G_p) (2x2) is real and non-negative; left as they are where that sum is 0.
 * Synchronous.
 */
int gc_gauge_fix_di(int32_t kind, void* gains, const gc_layout* layout, int32_t dtype, void* stream);

/*
 * Totals of the Levenberg-Marquardt phase (GC_SCHED_LM) of the last DI calibration made with
 * opt->profile != 0: summed device time of its iteration launches (ms, CUDA events on the call's
 * stream), their number, and the algorithmic floating-point operations of the FP32 Cholesky
 * factorisations and triangular solves they performed (n^3/3 + 2 n^2 per interval and iteration,
 * n real unknowns).  Any pointer may be NULL.
 */
int gc_profile_lm(double* lm_ms, int64_t* launches, double* flop);
/* SM clock cycles the same LM phase spent, summed over interval iterations, in its parts: [0] the
 * per-antenna J^H J blocks and J^H R, [1] the damped matrix, [2] the Cholesky factorisation with
 * the forward substitution, [3] the back substitution, [4] trial gains, chi^2 and the damping
 * decision; and within [2]: [5] panel loads, [6] panel solves, [7] trailing updates with the
 * look-ahead factor of the next diagonal block.  Writes min(n, 8) values; returns 8 (or GC_ERR_ARG). */
int gc_profile_lm_phases(double* cycles, int32_t n);

/* Text for a GC_ERR_* return code or a GC_ST_* status. */
const char* gc_error_string(int code);
const char* gc_status_string(int status);
/* The last CUDA error string seen by the library ("" if none). */
const char* gc_last_cuda_error(void);
/* Bounded waits.  The 2x2 accumulate kernel of the moment path waits for each tile's bulk copies
 * on an mbarrier, at most `tries` polls (each poll may also suspend the thread briefly); when the
 * wait runs out the kernel first waits, with the default bound, for the copies it still has in
 * flight, records the failure and ends, and the calling gc_calibrate_* returns GC_ERR_CUDA with
 * gc_last_cuda_error() naming the incomplete copy.  The GPU context stays usable.  tries < 0
 * restores the default bound (2^22 polls); 0 makes every such wait give up at once.  Applies to the
 * current device and every later call on it; meant for testing the error path.  Returns GC_OK or
 * GC_ERR_CUDA. */
int gc_set_wait_limit(int32_t tries);
/* Kernels launched by this process so far (a monotone counter, for launch accounting). */
int64_t gc_launch_count(void);
/* Free the cached device workspace (safe to call at any time no call is running). */
int gc_release(void);

#ifdef __cplusplus
}
#endif

#endif /* GAINCAL_H */
