// Smoothing in time and frequency (Sect. 3.4): every sample of a time x frequency grid has its own
// gains, updated by the ratio of two kernel convolutions (eq. JHJ:diag:smooth),
//     scalar: g_p = (w o alpha_p) / (w o beta_p),  2x2: G_p = (w o C_p) (w o H_p)^-1,
// with alpha_p, beta_p (C_p, H_p) the per-sample sums of StefCal's update: a per-sample
// accumulation, the separable convolution along one axis of the grid, the update with the
// schedule and the phase conventions, and the convergence test over the whole grid.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace gc {

// out[o][a0][e] = sum_{|a - a0| <= R, 0 <= a < n_axis} taps[a - a0 + R] in[o][a][e]; arrays
// [n_outer][n_axis][inner] floats, one thread per output value.
__global__ void sm_conv_kernel(const float* __restrict__ in, float* __restrict__ out, int n_axis, int64_t inner,
                               const float* __restrict__ taps, int R, int64_t total, const int* state) {
  if (state[0]) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t e = idx % inner;
  const int64_t oa = idx / inner;
  const int a0 = (int)(oa % n_axis);
  const int64_t base = (oa - a0) * inner + e;  // o * n_axis * inner + e
  const int lo = max(0, a0 - R), hi = min(n_axis - 1, a0 + R);
  float s = 0.f;
  for (int a = lo; a <= hi; ++a) s = fmaf(taps[a - a0 + R], in[base + (int64_t)a * inner], s);
  out[idx] = s;
}

// The same convolution with the inputs staged once: a CTA takes kCvE consecutive inner columns and
// kCvA consecutive outputs along the axis of one outer slice, copies the kCvA + 2R inputs they need
// (coalesced rows of kCvE floats) and the taps into shared memory, and each thread forms outputs
// of one column with the same terms in the same order as sm_conv_kernel (identical results).
constexpr int kCvE = 32, kCvA = 64, kCvThreads = 256;
__global__ void __launch_bounds__(kCvThreads) sm_conv_tiled_kernel(const float* __restrict__ in,
                                                                  float* __restrict__ out, int n_axis, int64_t inner,
                                                                  const float* __restrict__ taps, int R,
                                                                  const int* state) {
  if (state[0]) return;
  extern __shared__ __align__(16) float cv_smem[];
  float* st = cv_smem;                                  // taps [2R + 1]
  float* tile = cv_smem + (2 * R + 1 + 3) / 4 * 4;      // [(kCvA + 2R)][kCvE]
  const int64_t o = blockIdx.z;
  const int64_t e0 = (int64_t)blockIdx.x * kCvE;
  const int a_0 = (int)blockIdx.y * kCvA;
  const int lo_in = max(0, a_0 - R), hi_in = min(n_axis - 1, a_0 + kCvA - 1 + R);
  const int nin = hi_in - lo_in + 1;
  for (int x = threadIdx.x; x < 2 * R + 1; x += blockDim.x) st[x] = taps[x];
  const int ec = threadIdx.x % kCvE, ar = threadIdx.x / kCvE;
  constexpr int kRows = kCvThreads / kCvE;
  const int64_t e = e0 + ec;
  const bool ev = e < inner;
  const float* src = in + o * n_axis * inner;
  for (int r = ar; r < nin; r += kRows) tile[r * kCvE + ec] = ev ? src[(int64_t)(lo_in + r) * inner + e] : 0.f;
  __syncthreads();
  float* dst = out + o * n_axis * inner;
  const int a_end = min(n_axis, a_0 + kCvA);
  for (int a0 = a_0 + ar; a0 < a_end; a0 += kRows) {
    const int lo = max(0, a0 - R), hi = min(n_axis - 1, a0 + R);
    float s = 0.f;
    for (int a = lo; a <= hi; ++a) s = fmaf(st[a - a0 + R], tile[(a - lo_in) * kCvE + ec], s);
    if (ev) dst[(int64_t)a0 * inner + e] = s;
  }
}

// One side of a row's contribution to StefCal's per-antenna sums, in the component order K::solve
// reads (scalar [Re c, Im c, A]; 2x2 [C (8), H00, H11, Re H01, Im H01]).  Stored row (p, q), antenna
// p: y = m conj(g_q), c += conj(y) d, A += |y|^2 (2x2: Y = M G_q^H, C += D Y^H, H += Y Y^H).
// Conjugate row, antenna q: w = g_p m, c += w conj(d), A += |w|^2 (2x2: W = G_p M, C += D^H W,
// H += W^H W).  o: the other antenna's gain.
template <class K> struct SmoothRow;
template <> struct SmoothRow<ScalarKind<float>> {
  static GC_DEV void add(const float* vis, const float* mod, int64_t r, const Cx<float>& o, bool conj_side,
                         float* v) {
    const Cx<float> d = Vec<float>::ld1(vis + 2 * r), m = Vec<float>::ld1(mod + 2 * r);
    if (!conj_side) {
      const Cx<float> y = mulc_(m, o);
      v[0] = fmaf(y.x, d.x, fmaf(y.y, d.y, 0.f));
      v[1] = fmaf(y.x, d.y, -y.y * d.x);
      v[2] = abs2_(y);
    } else {
      const Cx<float> w = mul_(o, m);
      v[0] = fmaf(w.x, d.x, w.y * d.y);
      v[1] = fmaf(w.y, d.x, -w.x * d.y);
      v[2] = abs2_(w);
    }
  }
};
template <> struct SmoothRow<JonesKind<float>> {
  static GC_DEV void add(const float* vis, const float* mod, int64_t r, const M2<float>& o, bool conj_side,
                         float* v) {
    const M2<float> D = Vec<float>::ld4(vis + 8 * r), M = Vec<float>::ld4(mod + 8 * r);
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = 0.f;
    if (!conj_side) {
      const M2<float> Y = mmh_(M, o);
      fmac2(v[0], v[1], D.a, Y.a); fmac2(v[0], v[1], D.b, Y.b);
      fmac2(v[2], v[3], D.a, Y.c); fmac2(v[2], v[3], D.b, Y.d);
      fmac2(v[4], v[5], D.c, Y.a); fmac2(v[4], v[5], D.d, Y.b);
      fmac2(v[6], v[7], D.c, Y.c); fmac2(v[6], v[7], D.d, Y.d);
      v[8] = abs2_(Y.a) + abs2_(Y.b);
      v[9] = abs2_(Y.c) + abs2_(Y.d);
      fmac2(v[10], v[11], Y.a, Y.c); fmac2(v[10], v[11], Y.b, Y.d);
    } else {
      const M2<float> W = mm_(o, M);
      cfma2(v[0], v[1], D.a, W.a); cfma2(v[0], v[1], D.c, W.c);
      cfma2(v[2], v[3], D.a, W.b); cfma2(v[2], v[3], D.c, W.d);
      cfma2(v[4], v[5], D.b, W.a); cfma2(v[4], v[5], D.d, W.c);
      cfma2(v[6], v[7], D.b, W.b); cfma2(v[6], v[7], D.d, W.d);
      v[8] = abs2_(W.a) + abs2_(W.c);
      v[9] = abs2_(W.b) + abs2_(W.d);
      cfma2(v[10], v[11], W.a, W.b); cfma2(v[10], v[11], W.c, W.d);
    }
  }
};

// Per-sample sums: one CTA per sample.  The sample's baselines are taken in tiles of TB: every
// thread forms both sides of its baselines' contributions from coalesced row loads (each row read
// once) into shared memory; then kSmSplit threads per antenna add the tile's entries of its
// (baseline, side) list -- sorted by baseline, so each tile's entries are the next ones of the
// list, from tent -- each a fixed share, into compensated FP32 sums combined in a fixed order.
// The sample's gains are staged in shared memory.  sums [n_s][n_ant][NC].
template <class K> struct SmoothTile { static constexpr int TB = 1024; };
template <> struct SmoothTile<JonesKind<float>> { static constexpr int TB = 512; };
constexpr int kSmSplit = 4;  // threads per antenna in the per-antenna sums

template <class K>
__global__ void __launch_bounds__(256) sm_acc_kernel(const float* __restrict__ vis, const float* __restrict__ mod,
                                                     const float* __restrict__ gains, int n_bl, int n_ant,
                                                     const int32_t* __restrict__ ant_off,
                                                     const int32_t* __restrict__ ent, const int32_t* __restrict__ a12,
                                                     const int32_t* __restrict__ tent, const int* state,
                                                     float* __restrict__ sums) {
  constexpr int NC = K::NC, GW = K::GW, TB = SmoothTile<K>::TB;
  extern __shared__ __align__(16) float smem[];
  float* gs = smem;                        // [n_ant][GW]
  float* con = smem + n_ant * GW;          // [TB][2][NC] contributions of the tile's baselines
  if (state[0]) return;
  const int smp = blockIdx.x, tid = threadIdx.x;
  const int64_t g0 = (int64_t)smp * n_ant, r0 = (int64_t)smp * n_bl;
  for (int x = tid; x < n_ant * GW; x += blockDim.x) gs[x] = gains[g0 * GW + x];
  __syncthreads();
  // antenna p = pb + tid / kSmSplit, part j = tid % kSmSplit: the part's share of the antenna's
  // entries of every tile (entries j, j + kSmSplit, ..); the parts combine in a fixed order at the end
  const int j = tid % kSmSplit;
  for (int pb = 0; pb < n_ant; pb += blockDim.x / kSmSplit) {
    const int p = pb + tid / kSmSplit;
    float acc[NC], cmp[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = cmp[c] = 0.f;
    for (int b0 = 0, t = 0; b0 < n_bl; b0 += TB, ++t) {
      const int nb = min(TB, n_bl - b0);
      for (int bl = tid; bl < nb; bl += blockDim.x) {
        const int b = b0 + bl;
        const int2 pq = __ldg(reinterpret_cast<const int2*>(a12) + b);
        SmoothRow<K>::add(vis, mod, r0 + b, K::ld_gain(gs + GW * pq.y), false, con + (2 * bl) * NC);
        SmoothRow<K>::add(vis, mod, r0 + b, K::ld_gain(gs + GW * pq.x), true, con + (2 * bl + 1) * NC);
      }
      __syncthreads();
      // the tile's entries of the antenna are e .. e_end - 1
      const int e = p < n_ant ? __ldg(tent + (int64_t)t * n_ant + p) : 0;
      const int e_end = p < n_ant ? __ldg(tent + (int64_t)(t + 1) * n_ant + p) : 0;
      for (int x = e + j; x < e_end; x += kSmSplit) {
        const int en = __ldg(ent + x);
        const float* v = con + (2 * ((en >> 1) - b0) + (en & 1)) * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) kahan_add(acc[c], cmp[c], v[c]);
      }
      __syncthreads();
    }
    // combine the kSmSplit parts (consecutive lanes) in part order
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float v = acc[c] - cmp[c];
      float tot = 0.f;
#pragma unroll
      for (int q = 0; q < kSmSplit; ++q) tot += __shfl_sync(0xffffffffu, v, (threadIdx.x & 31 & ~(kSmSplit - 1)) + q);
      if (p < n_ant && j == 0) sums[(g0 + p) * NC + c] = tot;
    }
  }
}

// Complex sums over a sample's antennas for the phase conventions: scalar sum conj(a) b, 2x2
// sum tr(A^H B) (alignment); scalar sum g, 2x2 sum tr G (canonical gauge).
template <class K> struct SmoothPhase;
template <> struct SmoothPhase<ScalarKind<float>> {
  using G = Cx<float>;
  static GC_DEV Cx<float> inner(const G& a, const G& b) { return cmul_(a, b); }
  static GC_DEV Cx<float> trace(const G& g) { return g; }
  static GC_DEV G rot(const G& g, Cx<float> e) { return mul_(g, e); }
};
template <> struct SmoothPhase<JonesKind<float>> {
  using G = M2<float>;
  static GC_DEV Cx<float> inner(const G& a, const G& b) {
    Cx<float> s = cmul_(a.a, b.a);
    s = add_(s, cmul_(a.b, b.b));
    s = add_(s, cmul_(a.c, b.c));
    return add_(s, cmul_(a.d, b.d));
  }
  static GC_DEV Cx<float> trace(const G& g) { return add_(g.a, g.d); }
  static GC_DEV G rot(G g, Cx<float> e) {
    g.a = mul_(g.a, e); g.b = mul_(g.b, e); g.c = mul_(g.c, e); g.d = mul_(g.d, e);
    return g;
  }
};

// e^{-i arg z} (1 for z = 0); the sum is formed in FP64, the unit factor in FP32
GC_DEV Cx<float> unphase(double zx, double zy) {
  const float x = (float)zx, y = (float)zy;
  const float m2 = fmaf(x, x, y * y);
  if (!(m2 > 0.f)) return cx<float>(1.f, 0.f);
  const float r = rsqrtf(m2);
  return cx<float>(x * r, -y * r);
}

constexpr int kSmWarps = 8;  // samples per update CTA (one warp each)

GC_DEV double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per sample: for its antennas the GN gains from the smoothed sums, rotated by the common
// phase that best aligns them with the current gains; the schedule (odd k: those gains, even k:
// their average with the current ones); the result put in the canonical gauge (sum of the gains,
// 2x2 of their traces, real and non-negative) and staged in gnew; the sample's step norms, summed
// over the CTA's samples in warp order into one partial per CTA.
// state[0] done, [1] iterations, [2] status, [3] apply the staged gains.
// partials: per CTA {|dg|^2, |g|^2 (FP64), flags (bit 0 non-finite, bit 1 singular)}.
template <class K>
__global__ void __launch_bounds__(32 * kSmWarps) sm_update_kernel(const float* __restrict__ sums,
                                                                  const float* __restrict__ gains,
                                                                  float* __restrict__ gnew, int n_s, int n_ant, int k,
                                                                  int schedule, const int* state, double* partials) {
  using P = SmoothPhase<K>;
  __shared__ double red[kSmWarps][3];
  if (state[0]) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int smp = blockIdx.x * kSmWarps + w;
  double d2 = 0.0, n2 = 0.0;
  int fl = 0;
  if (smp < n_s) {  // warp-uniform
    const int64_t g0 = (int64_t)smp * n_ant;
    const bool gn_step = schedule == GC_SCHED_GN || (k & 1);
    int sing = 0;
    double ax = 0.0, ay = 0.0;
    for (int p = lane; p < n_ant; p += 32) {
      float v[K::NC];
#pragma unroll
      for (int c = 0; c < K::NC; ++c) v[c] = sums[(g0 + p) * K::NC + c];
      const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
      typename K::G gn;
      if (!K::solve(v, old, gn)) sing = 1;
      K::st_gain(gnew + K::GW * (g0 + p), gn);
      const Cx<float> t = P::inner(old, gn);
      ax += t.x; ay += t.y;
    }
    const Cx<float> ea = unphase(warp_sum_d(ax), warp_sum_d(ay));
    double sx = 0.0, sy = 0.0;
    for (int p = lane; p < n_ant; p += 32) {
      const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
      const typename K::G gn = P::rot(K::ld_gain(gnew + K::GW * (g0 + p)), ea);
      const typename K::G nw = gn_step ? gn : K::avg(old, gn);
      K::st_gain(gnew + K::GW * (g0 + p), nw);
      const Cx<float> t = P::trace(nw);
      sx += t.x; sy += t.y;
    }
    const Cx<float> ec = unphase(warp_sum_d(sx), warp_sum_d(sy));
    int nonfin = 0;
    for (int p = lane; p < n_ant; p += 32) {
      const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
      const typename K::G nw = P::rot(K::ld_gain(gnew + K::GW * (g0 + p)), ec);
      if (!K::finite(nw)) nonfin = 1;
      d2 += (double)K::dist2(nw, old);
      n2 += (double)K::norm2(nw);
      K::st_gain(gnew + K::GW * (g0 + p), nw);
    }
    d2 = warp_sum_d(d2);
    n2 = warp_sum_d(n2);
    fl = (__any_sync(0xffffffffu, nonfin) ? 1 : 0) | (__any_sync(0xffffffffu, sing) ? 2 : 0);
  }
  if (lane == 0) { red[w][0] = d2; red[w][1] = n2; red[w][2] = (double)fl; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double D = 0.0, N = 0.0;
    int f = 0;
    for (int j = 0; j < kSmWarps; ++j) { D += red[j][0]; N += red[j][1]; f |= (int)red[j][2]; }
    double* q = partials + 3 * blockIdx.x;
    q[0] = D; q[1] = N; q[2] = (double)f;
  }
}

// One CTA: the grid's step norms from the per-CTA partials of the update (each thread a fixed
// stride, then a fixed tree), the stopping rule, and whether the staged gains are applied.
__global__ void __launch_bounds__(256) sm_final_kernel(const double* partials, int n_s, int k, int max_iter,
                                                       double tol, int* state) {
  __shared__ double red[32];
  if (state[0]) return;
  double D2 = 0.0, N2 = 0.0;
  int fl = 0;
  for (int i = threadIdx.x; i < n_s; i += blockDim.x) {
    D2 += partials[3 * i];
    N2 += partials[3 * i + 1];
    fl |= (int)partials[3 * i + 2];
  }
  D2 = block_sum<double>(D2, red);
  N2 = block_sum<double>(N2, red);
  const int nf = __syncthreads_or(fl & 1), sg = __syncthreads_or(fl & 2);
  if (threadIdx.x != 0) return;
  const int sflag = sg ? GC_ST_SINGULAR_FLAG : 0;
  state[1] = k;
  if (nf) {  // non-finite gains: stop, keep the last finite ones
    state[0] = 1; state[2] = GC_ST_NONFINITE | sflag; state[3] = 0;
    return;
  }
  state[3] = 1;
  if (D2 <= tol * tol * N2) { state[0] = 1; state[2] = GC_ST_OK | sflag; }
  else if (k >= max_iter) { state[0] = 1; state[2] = GC_ST_NOT_CONVERGED | sflag; }
  else state[2] = GC_ST_NOT_CONVERGED | sflag;
}

__global__ void sm_apply_kernel(const float* __restrict__ gnew, float* __restrict__ gains, int64_t n, int* state) {
  if (!state[3]) return;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    gains[x] = gnew[x];
}

__global__ void sm_init_kernel(int* state) {
  if (threadIdx.x == 0 && blockIdx.x == 0) { state[0] = 0; state[1] = 0; state[2] = GC_ST_NOT_CONVERGED; state[3] = 0; }
}

int sm_launch_conv(const float* in, float* out, int64_t n_outer, int n_axis, int64_t inner, const float* taps, int R,
                   const int* state, void* stream) {
  const int64_t total = n_outer * n_axis * inner;
  if (total <= 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = sizeof(float) * (((size_t)2 * R + 1 + 3) / 4 * 4 + (size_t)(kCvA + 2 * R) * kCvE);
  const int64_t gx = (inner + kCvE - 1) / kCvE, gy = (n_axis + kCvA - 1) / kCvA;
  if (smem <= 96 * 1024 && n_outer <= 65535 && gy <= 65535 && gx <= 0x7fffffff) {
    cudaError_t e = cudaFuncSetAttribute(sm_conv_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    sm_conv_tiled_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)n_outer), kCvThreads, smem, s>>>(in, out, n_axis,
                                                                                                    inner, taps, R, state);
  } else {
    sm_conv_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(in, out, n_axis, inner, taps, R, total, state);
  }
  return (int)cudaGetLastError();
}

int sm_tile_rows(int kind) {
  return kind == 0 ? SmoothTile<ScalarKind<float>>::TB : SmoothTile<JonesKind<float>>::TB;
}

template <class K>
static int sm_launch_tiled(const float* vis, const float* model, const float* gains, int n_s, int n_bl, int n_ant,
                           const int32_t* ant_off, const int32_t* ent, const int32_t* a12, const int32_t* tent,
                           const int* state, float* sums, cudaStream_t s) {
  const size_t smem = sizeof(float) * ((size_t)n_ant * K::GW + (size_t)SmoothTile<K>::TB * 2 * K::NC);
  cudaError_t e = cudaFuncSetAttribute(sm_acc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  sm_acc_kernel<K><<<n_s, 256, smem, s>>>(vis, model, gains, n_bl, n_ant, ant_off, ent, a12, tent, state, sums);
  return 0;
}

int sm_launch_acc(int kind, const float* vis, const float* model, const float* gains, int n_s, int n_bl, int n_ant,
                  const int32_t* ant_off, const int32_t* ent, const int32_t* a12, const int32_t* tent,
                  const int* state, float* sums, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int rc = kind == 0 ? sm_launch_tiled<ScalarKind<float>>(vis, model, gains, n_s, n_bl, n_ant, ant_off, ent, a12,
                                                                tent, state, sums, s)
                           : sm_launch_tiled<JonesKind<float>>(vis, model, gains, n_s, n_bl, n_ant, ant_off, ent, a12,
                                                               tent, state, sums, s);
  if (rc) return rc;
  return (int)cudaGetLastError();
}

int sm_launch_update(int kind, const float* sums, const float* gains, float* gnew, int n_s, int n_ant, int k,
                     int schedule, int max_iter, double tol, int* state, double* partials, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (n_s + kSmWarps - 1) / kSmWarps;
  if (kind == 0)
    sm_update_kernel<ScalarKind<float>><<<nb, 32 * kSmWarps, 0, s>>>(sums, gains, gnew, n_s, n_ant, k, schedule, state,
                                                                     partials);
  else
    sm_update_kernel<JonesKind<float>><<<nb, 32 * kSmWarps, 0, s>>>(sums, gains, gnew, n_s, n_ant, k, schedule, state,
                                                                    partials);
  sm_final_kernel<<<1, 256, 0, s>>>(partials, nb, k, max_iter, tol, state);
  const int64_t nf = (int64_t)n_s * n_ant * (kind == 0 ? 2 : 8);
  sm_apply_kernel<<<(unsigned)std::min<int64_t>((nf + 255) / 256, 4 * 152), 256, 0, s>>>(gnew, const_cast<float*>(gains),
                                                                                        nf, state);
  return (int)cudaGetLastError();
}

int sm_launch_init(int* state, void* stream) {
  sm_init_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(state);
  return (int)cudaGetLastError();
}

}  // namespace gc
