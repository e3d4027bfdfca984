// Shared definitions of the direction-dependent solvers (scalar and 2x2 gains): kernel
// arguments, the per-antenna Hermitian solvers, the per-call plan and its builder.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gc {

constexpr int kIterThreads = 256;

struct DDArgs {
  const float* vis;
  const float* model;  // [n_dir][n_rows] complex
  float* gains;        // [n_gain][n_dir] complex
  int64_t n_rows;
  const int64_t* row_off;
  const int32_t* n_samp;
  const int32_t* n_bl;
  const int32_t* bl_off;
  const int32_t* n_ant;
  const int32_t* gain_off;
  const int32_t* ant1;
  const int32_t* ant2;
  const int64_t* mom_off;    // [n_int] first moment (complex index) of the interval
  // moment items
  const int32_t* mitem_int;
  const int32_t* mitem_tile;
  int32_t n_mitems;
  // iteration items (interval, antenna) and per-table antenna -> (baseline, side) lists
  const int32_t* iitem_int;
  const int32_t* iitem_ant;
  int32_t n_iitems;
  const int32_t* ent;        // baseline * 2 + side (side 1: the antenna is ant2 of the stored pair)
  const int32_t* entq;       // the other antenna of each entry's baseline
  const int32_t* iitem_e0;   // per iteration item: its antenna's entries [e0, e1) in ent / entq
  const int32_t* iitem_e1;
  // state
  float2* moments;
  float* gnew;               // [n_gain][n_dir] complex GN gains of this iteration
  int32_t* sing;             // [n_gain]
  int32_t* active;
  int32_t* iters;
  int32_t* status;
  int32_t* counters;
  int32_t* n_active;
  int32_t* kbase;            // iterations before this launch's segment (advanced on the device)
  double tol;
  int32_t max_iter;
  int32_t schedule;
  int32_t k;                 // position within the segment: the iteration is *kbase + k
  int32_t na_max;
  int32_t method;            // 0 CohJones (antenna-block inverse), 1 AllJones (diagonal, residual form)
  // scalar DD iteration state: iterates by parity ([2][n_gain][n_dir] complex; g^(k) at k & 1) and
  // per-antenna convergence partials (float-float |dg|^2, |g|^2) and flags (bit 0 non-finite,
  // bit 1 singular), [2][n_gain] each, read by the next launch
  float* gbuf;
  float4* conv;
  int32_t* cflag;
  int64_t n_gain;
  int32_t* stopk;  // [n_int] the launch that took the interval's stop decision (0: none yet)
};

// Component index -> (c, d) for the upper triangle, row-major: (0,0) (0,1) .. (0,ND-1) (1,1) ..
__host__ __device__ inline void upper_cd(int nd, int comp, int& c, int& d) {
  int r = 0, base = 0;
  while (comp >= base + (nd - r)) { base += nd - r; ++r; }
  c = r;
  d = r + (comp - base);
}

// ------------------------------------------------------------------------------------ FP64 solve
// Cholesky A = L L^H of the Hermitian ND x ND block (upper triangle given) and solve A x = b, in
// FP64, by one warp (right-looking: at column k one lane takes the square root of the pivot, the
// lanes scale the column below it and update the trailing lower triangle in parallel; then the
// two triangular solves, column by column).  Am: [ND][ND] double2 and dinv: [ND] double of shared
// memory.  Every lane of the warp calls it and gets the same result; false when a pivot is not
// positive (the block is not numerically positive definite).
template <int ND>
__device__ bool chol_solve_warp(const double2* Aup, const double2* b, double2* x, double2* Am, double* dinv,
                                int* ok_s) {
  const int lane = threadIdx.x & 31;
  auto au = [](int r, int c) { return r * ND - r * (r - 1) / 2 + (c - r); };  // upper entry (r <= c)
  for (int e = lane; e < ND * ND; e += 32) {  // lower triangle of A (conjugates of the upper entries)
    const int r = e / ND, c = e % ND;
    if (c <= r) {
      double2 v = Aup[au(c, r)];
      v.y = -v.y;
      Am[e] = v;
    }
  }
  for (int r = lane; r < ND; r += 32) x[r] = b[r];
  if (lane == 0) *ok_s = 1;
  __syncwarp();
  for (int k = 0; k < ND; ++k) {
    if (lane == 0) {
      const double akk = Am[k * ND + k].x;
      if (!(akk > 0.0) || !isfinite(akk)) {
        *ok_s = 0;
      } else {
        const double l = sqrt(akk);
        Am[k * ND + k] = make_double2(l, 0.0);
        dinv[k] = 1.0 / l;
      }
    }
    __syncwarp();
    if (!*ok_s) return false;
    for (int i = k + 1 + lane; i < ND; i += 32) {
      const double2 v = Am[i * ND + k];
      Am[i * ND + k] = make_double2(v.x * dinv[k], v.y * dinv[k]);
    }
    __syncwarp();
    // A[i][j] -= L[i][k] conj(L[j][k]) for k < j <= i
    const int m = ND - 1 - k;
    for (int t = lane; t < m * (m + 1) / 2; t += 32) {
      int i = 0;
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      const int j = t - i * (i + 1) / 2;
      const int ii = k + 1 + i, jj = k + 1 + j;
      const double2 p = Am[ii * ND + k], q = Am[jj * ND + k];
      double2 v = Am[ii * ND + jj];
      v.x -= p.x * q.x + p.y * q.y;
      v.y -= p.y * q.x - p.x * q.y;
      Am[ii * ND + jj] = v;
    }
    __syncwarp();
  }
  for (int k = 0; k < ND; ++k) {  // L y = b (y in x)
    if (lane == 0) x[k] = make_double2(x[k].x * dinv[k], x[k].y * dinv[k]);
    __syncwarp();
    for (int i = k + 1 + lane; i < ND; i += 32) {
      const double2 p = Am[i * ND + k], q = x[k];
      x[i].x -= p.x * q.x - p.y * q.y;
      x[i].y -= p.x * q.y + p.y * q.x;
    }
    __syncwarp();
  }
  for (int k = ND - 1; k >= 0; --k) {  // L^H x = y
    if (lane == 0) x[k] = make_double2(x[k].x * dinv[k], x[k].y * dinv[k]);
    __syncwarp();
    for (int i = lane; i < k; i += 32) {  // x[i] -= conj(L[k][i]) x[k]
      const double2 p = Am[k * ND + i], q = x[k];
      x[i].x -= p.x * q.x + p.y * q.y;
      x[i].y -= p.x * q.y - p.y * q.x;
    }
    __syncwarp();
  }
  return true;
}

// The factorisation in FP32 followed by one step of iterative refinement (Moler's
// mixed-precision scheme): the residual r = b - A x0 in float-float against the float-float
// block, then the correction solved with the FP32 factor; one step takes the error from about
// kappa(A) u_32 to about (kappa(A) u_32)^2.  Ah + Al is the upper triangle of A and bh + bl the
// right-hand side, each an unevaluated float-float sum.  Called by one whole warp: lane r keeps
// row r of the block in registers and the columns are factored right-looking with shuffles (lanes
// r >= ND shadow row ND - 1 and store nothing).  False when an FP32 pivot is not positive: the
// caller then runs the FP64 factorisation, which alone decides singularity.
// Ls: [ND][ND] of shared memory (the factor, rows); the solution goes to x.
template <int ND, int NR = 1>
__device__ bool chol_solve_warp_mixed(const Cx<float>* Ah, const Cx<float>* Al, const Cx<float>* bh,
                                      const Cx<float>* bl, Cx<float>* x, Cx<float>* Ls) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int r = lane < ND ? lane : ND - 1;
  auto au = [](int i, int j) { return i * ND - i * (i - 1) / 2 + (j - i); };  // upper entry (i <= j)
  auto shfl = [&](Cx<float> v, int src) {
    return cx<float>(__shfl_sync(kAll, v.x, src), __shfl_sync(kAll, v.y, src));
  };
  float dinv[ND];
  {
    Cx<float> L[ND];  // row r: A[r][j], becoming L[r][j] for j <= r
#pragma unroll
    for (int j = 0; j < ND; ++j) L[j] = r <= j ? Ah[au(r, j)] : conj_(Ah[au(j, r)]);
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const float akk = __shfl_sync(kAll, L[k].x, k);
      if (!(akk > 0.f) || !isfinite(akk)) return false;  // the same pivot in every lane
      const float l = sqrtf(akk);
      dinv[k] = __frcp_rn(l);
      if (r == k) L[k] = cx<float>(l, 0.f);
      else if (r > k) L[k] = scale_(L[k], dinv[k]);
#pragma unroll
      for (int j = k + 1; j < ND; ++j) {  // A[r][j] -= L[r][k] conj(L[j][k]) for j <= r
        const Cx<float> ljk = shfl(L[k], j);
        if (r >= j) L[j] = sub_(L[j], mulc_(L[k], ljk));
      }
    }
    if (lane < ND) {
#pragma unroll
      for (int j = 0; j < ND; ++j)
        if (j <= r) Ls[r * ND + j] = L[j];
    }
  }
  __syncwarp();
  // L L^H v = w for the w held by lane r: forward with row r of L, backward with column r
  auto subst = [&](Cx<float> v) {
    Cx<float> row[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) row[k] = k < r ? Ls[r * ND + k] : cx<float>(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      if (r == k) v = scale_(v, dinv[k]);
      const Cx<float> vk = shfl(v, k);
      if (r > k) v = sub_(v, mul_(row[k], vk));
    }
    Cx<float> col[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) col[k] = k > r ? Ls[k * ND + r] : cx<float>(0.f, 0.f);
#pragma unroll
    for (int k = ND - 1; k >= 0; --k) {
      if (r == k) v = scale_(v, dinv[k]);
      const Cx<float> vk = shfl(v, k);
      if (r < k) v = sub_(v, cmul_(col[k], vk));  // v_r -= conj(L[k][r]) v_k
    }
    return v;
  };
  for (int rr = 0; rr < NR; ++rr) {  // right-hand sides [NR][ND], one factorisation
  const Cx<float>* bhr = bh + rr * ND;
  const Cx<float>* blr = bl + rr * ND;
  const Cx<float> x0 = subst(bhr[r]);
  // residual in float-float: r_r = b_r - sum_j A[r][j] x0_j, two interleaved partial sums per part
  FF rx0{bhr[r].x, blr[r].x}, ry0{bhr[r].y, blr[r].y}, rx1{0.f, 0.f}, ry1{0.f, 0.f};
  float lox = 0.f, loy = 0.f;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int u = r <= j ? au(r, j) : au(j, r);
    Cx<float> h = Ah[u], lo = Al[u];
    if (r > j) { h.y = -h.y; lo.y = -lo.y; }
    const Cx<float> xj = shfl(x0, j);
    FF& ax = (j & 1) ? rx1 : rx0;
    FF& ay = (j & 1) ? ry1 : ry0;
    ax = ff_sub_prod(ax, h.x, xj.x);
    ax = ff_sub_prod(ax, -h.y, xj.y);
    ay = ff_sub_prod(ay, h.x, xj.y);
    ay = ff_sub_prod(ay, h.y, xj.x);
    lox = fmaf(lo.x, xj.x, fmaf(-lo.y, xj.y, lox));
    loy = fmaf(lo.x, xj.y, fmaf(lo.y, xj.x, loy));
  }
  const FF rx = ff_add(rx0, rx1), ry = ff_add(ry0, ry1);
  const Cx<float> dres = cx<float>(rx.hi + (rx.lo - lox), ry.hi + (ry.lo - loy));
  const Cx<float> d = subst(dres);
  if (lane < ND) x[rr * ND + lane] = add_(x0, d);
  }
  __syncwarp();
  return true;
}

static __global__ void dd_init_kernel(DDArgs a, int n_int, int n_active0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { *a.n_active = n_active0; *a.kbase = 0; }
  if (i < n_int) {
    const int64_t rows = (int64_t)a.n_samp[i] * a.n_bl[i];
    a.active[i] = rows > 0 ? 1 : 0;
    a.iters[i] = 0;
    a.status[i] = rows > 0 ? GC_ST_NOT_CONVERGED : GC_ST_NODATA;
    a.counters[i] = 0;
    if (a.stopk) a.stopk[i] = 0;
  }
}

// Schedule and convergence test of interval i (odd k or the GN schedule: the new gains; even k:
// their average with the current ones), run by the whole CTA of the interval's last antenna to
// finish its update.  W complex gain values per antenna; gs holds the interval's current gains in
// shared memory; red >= 160 floats of shared memory.
__device__ inline void dd_interval_update(const DDArgs& a, int i, int k, int na, int64_t go, int W, Cx<float>* gs,
                                          float* red) {
  const int tid = threadIdx.x;
  const bool gn_step = (a.schedule == GC_SCHED_GN) || (k & 1);
  FF d2{0.f, 0.f}, n2{0.f, 0.f};  // float-float sums (the FP64 pipe of GB300 is narrow)
  int nonfin = 0, sing = 0;
  for (int x = tid; x < na * W; x += blockDim.x) {
    const Cx<float> old = gs[x];
    const Cx<float> gn = cx<float>(__ldcg(a.gnew + 2 * (go * W + x)), __ldcg(a.gnew + 2 * (go * W + x) + 1));
    const Cx<float> nw = gn_step ? gn : cx<float>(0.5f * (old.x + gn.x), 0.5f * (old.y + gn.y));
    d2 = ff_add_f(d2, abs2_(sub_(nw, old)));
    n2 = ff_add_f(n2, abs2_(nw));
    if (!isfinite(nw.x) || !isfinite(nw.y)) nonfin = 1;
    gs[x] = nw;  // stage; written below unless non-finite
  }
  for (int x = tid; x < na; x += blockDim.x) sing |= __ldcg(a.sing + go + x);
  block_reduce_step_ff(d2, n2, nonfin, sing, red, (int)blockDim.x);
  const double D2 = ff_value(d2), N2 = ff_value(n2);
  if (!nonfin)
    for (int x = tid; x < na * W; x += blockDim.x) {
      a.gains[2 * (go * W + x)] = gs[x].x;
      a.gains[2 * (go * W + x) + 1] = gs[x].y;
    }
  if (tid == 0) {
    a.counters[i] = 0;
    int st = -1;
    if (nonfin) st = GC_ST_NONFINITE;
    else if (D2 <= a.tol * a.tol * N2) st = GC_ST_OK;
    else if (k >= a.max_iter) st = GC_ST_NOT_CONVERGED;
    if (st >= 0) {
      a.active[i] = 0;
      a.iters[i] = k;
      a.status[i] = st | (sing ? GC_ST_SINGULAR_FLAG : 0);
      atomicSub(a.n_active, 1);
    }
  }
}

// ------------------------------------------------------------------------------------ host side
extern std::atomic<long long> g_launches;
int ws_get(const char* name, size_t bytes, void** out);
int pinned_flag(int** out);
int validate_layout(const gc_layout* L, int n_dir_max);
uint64_t layout_hash(const gc_layout* L, uint64_t salt);
int set_cuda_error(cudaError_t e, const char* what);

struct DDPlan {
  uint64_t key = 0;
  void* dev = nullptr;
  size_t dev_bytes = 0;
  DDArgs args{};
  int n_int = 0, n_active0 = 0, nd = 1;
  int64_t n_mom = 0;
  cudaGraphExec_t gexec = nullptr;  // the captured iteration segment
  DDArgs gargs{};
  int gS = 0, gnd = 0;
  int32_t* chi2_first = nullptr;
  int32_t* chi2_count = nullptr;
  double* chi2_items = nullptr;
  double* chi2_out = nullptr;
};

// Per-call plan of a DD solve: moment items of mom_tile baselines (interval, tile), iteration
// items (interval, antenna) with each antenna's (baseline, side) entries, per-interval moment
// offsets (mom_per_bl complex values per baseline), state arrays; one device allocation.
int build_dd_plan(const gc_layout* L, DDPlan& P, cudaStream_t s, int64_t mom_per_bl, int mom_tile);

#define DD_CUDA(call)                                             \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return set_cuda_error(e__, #call);    \
  } while (0)

void profile_record(double iter_ms, int64_t launches, int64_t row_iters, double moment_ms, int64_t bl_iters, int path);

// opt->profile: the moment pass and every iteration launch bracketed by CUDA events on `s`
struct DDTimer {
  bool on;
  std::vector<cudaEvent_t> ev;
  int used = 0;
  double ms = 0.0;
  int64_t launches = 0;
  explicit DDTimer(bool on_, int cap) : on(on_) {
    if (on)
      for (int i = 0; i < 2 * cap; ++i) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        ev.push_back(e);
      }
  }
  ~DDTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  void before(cudaStream_t s) {
    if (on) cudaEventRecord(ev[2 * used], s);
  }
  void after(cudaStream_t s) {
    if (on) { cudaEventRecord(ev[2 * used + 1], s); ++used; }
  }
  void drain() {  // after a synchronize of the stream
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      ms += t;
    }
    launches += used;
    used = 0;
  }
};

}  // namespace gc
