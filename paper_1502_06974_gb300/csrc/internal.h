// Host/device shared definitions of the gain-calibration library (not part of the public ABI).
#pragma once

#include <stdint.h>

#include "../../include/gaincal.h"

namespace gc {

constexpr int kDIThreads = 256;  // CTA size of the direction-independent kernels
constexpr int kSubChain = 16;    // samples a thread sums in registers before an antenna reduction

// Arguments of the direction-independent kernels (all pointers device memory).
struct DIArgs {
  const void* vis;
  const void* model;
  void* gains;
  // layout
  const int64_t* row_off;
  const int32_t* n_samp;
  const int32_t* n_bl;
  const int32_t* bl_off;
  const int32_t* n_ant;
  const int32_t* gain_off;
  const int32_t* ant1;
  const int32_t* ant2;
  // antenna-reduction plan: per baseline table and tile of kDIThreads baselines, the list of
  // partial-sum slots (offsets into the CTA's partials array) that belong to each antenna
  const int32_t* itab;      // [n_int] table of each interval
  const int32_t* tab_base;  // [n_tab] first csr_off entry of the table
  const int32_t* tab_nant;  // [n_tab] antennas the table spans
  const int32_t* csr_off;   // per table: tiles x (tab_nant + 1) offsets into csr_ent
  const int32_t* csr_ent;   // slot offsets
  // work items: (interval, sample range); items of one interval are consecutive
  const int32_t* item_int;
  const int32_t* item_s0;
  const int32_t* item_s1;
  const int64_t* item_scr;  // scratch offset (elements) of the item's per-antenna partials
  const int32_t* n_chunks;  // [n_int] items per interval
  const int32_t* first_item;
  int32_t n_items;
  int32_t na_max;
  // iteration state
  int32_t* active;
  int32_t* iters;
  int32_t* status;
  int32_t* counters;  // [n_int] chunk arrival counters (reset by the last arrival)
  int32_t* n_active;  // intervals still iterating
  int32_t* qhead;     // [2] work-queue heads, used alternately by consecutive launches
  void* scratch;
  double tol;
  int32_t max_iter;
  int32_t schedule;
  int32_t k;  // iteration number, 1-based
  // accumulate-only outputs
  void* jhd_out;
  void* jhj_out;
  // moment-stream path: per-baseline moments and each interval's first baseline in them
  const float* moments;
  const int64_t* mom_off;
  // compacted work lists (moment-stream path): iteration k takes items from list[k % 3], appends
  // the items of intervals that stay active to list[(k + 1) % 3], and clears list (k + 2) % 3
  int32_t* ilist;    // [3][n_items]
  int32_t* icount;   // [3]
  int32_t* kbase;    // iteration base added to k (graph-captured iteration segments); may be NULL
  float* aux;        // [n_gain][AW] per-antenna auxiliaries of the current gains (moment path)
  float* gnew;       // [n_gain][GW] staged new gains (moment path)
  // intervals that join a running iteration (wavefront solve): interval i counts its own
  // iterations from k - k0[i]; gate[i] records the first of them whose relative step fell below
  // gate_tol (0 = not yet).  Both may be NULL (every interval starts at k = 1, no gate).
  int32_t* k0;
  int32_t* gate;
  double gate_tol;
  // an accumulate launch with xcount > 0 takes the items xbegin .. xbegin + xcount - 1 instead of
  // its iteration's work list (and leaves the work lists alone)
  int32_t xbegin;
  int32_t xcount;
  // single-launch iteration (di_mstep1_kernel): per-interval publication flags, and the work list
  // the init launch fills (0 = list 1, the two-launch scheme's first list)
  int32_t* flag;
  int32_t first_list;
  // bulk-copy accumulate (di_macc_bulk_kernel): per item three int4 descriptors
  //   {moment float index lo, hi, baselines in the tile, static block offset (ints)},
  //   {static block length (ints), antennas of the table, first gain, antennas of the interval},
  //   {scratch offset lo, hi, 0, 0};
  // per (table, tile) one static block of ints, 16-byte aligned: ant1 and ant2 of the tile's slots
  // [kDIThreads each], the reduction offsets [tab_nant + 1, padded to 4] and slot entries [padded
  // to 4]; tblk_max the longest block; err set when a copy's wait gives up.
  const int4* item_desc;
  const int32_t* tblk;
  int32_t tblk_max;
  int32_t* err;
  // per-row weights (Sect. 2.4; T of the kernel's dtype, [n_rows]) or NULL for unit weights
  const void* weights;
};
// DIArgs goes to the kernels by value: every translation unit, host and device pass, must agree on
// its layout.  A field added here changes this size and must be added in the same build of every
// object that uses it (the library build recompiles all of them together).
static_assert(sizeof(DIArgs) == 424, "DIArgs layout changed: rebuild every translation unit and update this size");

// Launchers implemented in di_kernels.cu.  kind: 0 scalar, 1 jones.  Return cudaError_t as int.
int di_smem_bytes(int kind, int dtype, int na_max);
int di_max_blocks_per_sm(int kind, int dtype, int acc_only, int smem, int* out);
int di_launch_iter(int kind, int dtype, int acc_only, const DIArgs& a, int grid, int smem, void* stream);
int di_launch_init(const DIArgs& a, int n_int, int n_active0, void* stream);
int di_macc_smem(int kind, int na_max, int red_chunks, int prefetch);
int di_macc_bulk_smem(int kind, int na_max, int tblk_max);
// Smoothing in time and frequency (smooth.cu): per-sample per-antenna sums (one CTA per sample; the
// antennas' (baseline, side) lists ant_off / ent sorted by baseline, a12 the pairs [n_bl][2]);
// separable convolution along one axis of a
// [n_outer][n_axis][inner] float array with 2R + 1 taps; the update of every sample (phase
// alignment, schedule, canonical gauge) and the grid-wide stopping rule (state [4] ints: done,
// iterations, status, apply; partials 3 doubles per sample), then the staged gains copied over the
// current ones when the step is kept.
int sm_launch_conv(const float* in, float* out, int64_t n_outer, int n_axis, int64_t inner, const float* taps, int R,
                   const int* state, void* stream);
// Baselines per tile of the per-sample accumulation of this kind; tent [n_tiles + 1][n_ant]: the
// index in ent of antenna p's first entry with a baseline of tile t or later.
int sm_tile_rows(int kind);
int sm_launch_acc(int kind, const float* vis, const float* model, const float* gains, int n_s, int n_bl, int n_ant,
                  const int32_t* ant_off, const int32_t* ent, const int32_t* a12, const int32_t* tent,
                  const int* state, float* sums, void* stream);
int sm_launch_update(int kind, const float* sums, const float* gains, float* gnew, int n_s, int n_ant, int k,
                     int schedule, int max_iter, double tol, int* state, double* partials, void* stream);
int sm_launch_init(int* state, void* stream);
// Tries of the bulk-copy accumulate kernel's first wait per tile on the current device (< 0: the
// default bound).  Returns cudaError_t as int.
int di_set_bulk_wait_tries(int tries);
int di_macc_max_blocks_per_sm(int kind, int smem, int red_chunks, int prefetch, int* out);
// one iteration: the accumulate launch, then the solve launch
int di_launch_mstep(int kind, const DIArgs& a, int grid, int smem, int n_int, int red_chunks, int prefetch,
                    void* stream);
int di_launch_msolve(int kind, const DIArgs& a, int n_int, void* stream);
// one iteration in one cooperative launch: the update of the previous iteration and, interval by
// interval as each update is published, the accumulate of this one (*err set if a wait timed out)
int di_mstep1_smem(int kind, int na_max, int red_chunks);
int di_mstep1_max_grid(int kind, int smem, int red_chunks, int prefetch, int* out);
int di_launch_mstep1(int kind, const DIArgs& a, int grid, int smem, int n_int, int red_chunks, int prefetch, int* err,
                     void* stream);
int di_launch_advance(int* kbase, int by, void* stream);
// persistent iteration loop (cooperative launch): up to S iterations from *kbase + 1, stops early
// when no interval is active; bar = 2 zeroed words, *err set if a grid barrier timed out
int di_mloop_smem(int kind, int na_max, int red_chunks);
int di_mloop_max_grid(int kind, int smem, int red_chunks, int prefetch, int* out);
int di_launch_mloop(int kind, const DIArgs& a, int grid, int smem, int n_int, int S, int red_chunks, int prefetch,
                    unsigned* bar, int* err, void* stream);
// accumulate launch alone (iteration a.k's work list) and the per-interval combine without a solve
int di_launch_macc(int kind, const DIArgs& a, int grid, int smem, int red_chunks, int prefetch, void* stream);
int di_launch_msum(int kind, const DIArgs& a, int i_lo, int n, float* tot_out, double* e_out, void* stream);
// wavefront solve: hold every interval from i_hold on (pending) after the init launch; activate
// the intervals [i_lo, i_lo + n) so that they join at iteration *kbase + 1
int di_launch_wf_hold(const DIArgs& a, int n_int, int i_hold, int n_active0, void* stream);
int di_launch_wf_activate(const DIArgs& a, int i_lo, int n, void* stream);
int di_launch_maux(int kind, const float* gains, float* aux, int n_gain, void* stream);
// moment pass (resident.cu): per-baseline moments of every interval; items are (interval, 32 baselines);
// ns_max, the most samples of any interval, picks one thread per baseline (few samples) or sample
// lanes with a compensated shared-memory reduction
int moment_pass(int kind, const float* vis, const float* model, float* moments, const int64_t* row_off,
                const int64_t* mom_off, const int32_t* n_samp, const int32_t* n_bl, const int32_t* item_int,
                const int32_t* item_tile, int n_items, int ns_max, void* stream, const float* weights);
int moment_chi2(int kind, const float* vis, const float* model, const float* gains, const int64_t* row_off,
                const int32_t* n_samp, const int32_t* n_bl, const int32_t* bl_off, const int32_t* gain_off,
                const int32_t* ant1, const int32_t* ant2, const int32_t* item_int, const int32_t* item_tile,
                int n_items, const int32_t* first, const int32_t* count, double* item_chi2, double* out, int n_int,
                void* stream, const float* weights);
int di_launch_chi2(int kind, int dtype, const DIArgs& a, double* item_chi2, double* chi2_out, int n_int,
                   int grid, void* stream);

// learned warm start (mlp.cu)
int mlp_check(const gc_mlp* net);
int mlp_infer(const gc_mlp* net, const float* x, int n, float* y, void* stream);
int ws_gather(const float* sol, const int32_t* hoff, const float* lead, const int32_t* gain_off, const int32_t* n_ant,
              int i_lo, int n, int64_t gbase, int canon, float* hbuf, float* g1, float* lead_row, void* stream);
int ws_features_packed(const float* hbuf, const float* tot, const float* lead_row, int n, float* x, float* rot,
                       void* stream);
int ws_propose(const float* hbuf, const float* delta, const float* rot, int n, float* gains, void* stream);
int ws_choose(const float* g1, const double* e_prev, const double* e_prop, const int32_t* gain_off,
              const int32_t* n_ant, int i_lo, int n, int64_t gbase, float* gains, int32_t* used, double* dchi2,
              void* stream);
int gauge_fix(int kind, int dtype, void* gains, const int32_t* gain_off, const int32_t* n_ant, int n_int,
              void* stream);

// Levenberg-Marquardt polish with the whole J^H J (lm.cu), run after the diagonal iterations of the
// moment path: vis / model the rows, row_off / n_samp / moments / mom_off / ant1 / ant2 the caller's
// plan, gains / iters / status its device state.  lm_limit_ok: every interval has at most GC_LM_MAX_UNKNOWNS real unknowns.
int lm_limit_ok(int kind, const gc_layout* L);
int lm_run(int kind, const gc_layout* L, const float* vis, const float* model, const int64_t* row_off,
           const int32_t* n_samp, const float* moments, const int64_t* mom_off, const int32_t* ant1,
           const int32_t* ant2, float* gains, int32_t* iters, int32_t* status, const gc_options* opt, void* stream,
           const float* weights);
// time of the last profiled polish's iteration launches (CUDA events), their count, and the
// algorithmic flops of its factorisations and triangular solves
int lm_profile(double* ms, int64_t* launches, double* flop);
// SM cycles the last profiled polish spent per phase (summed over interval iterations); returns the
// number of phases
int lm_profile_phases(double* cycles, int n);

}  // namespace gc
