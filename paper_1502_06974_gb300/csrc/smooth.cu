// Smoothing in time and frequency (Sect. 3.4): every sample of a time x frequency grid has its own
// gains, updated by the ratio of two kernel convolutions (eq. JHJ:diag:smooth),
//     scalar: g_p = (w o alpha_p) / (w o beta_p),  2x2: G_p = (w o C_p) (w o H_p)^-1,
// with alpha_p, beta_p (C_p, H_p) the per-sample sums of StefCal's update.  The per-sample sums come
// from the library's accumulation pass (every sample one solution interval); this file holds the
// separable convolution along one axis of the grid, the update with the schedule, and the
// convergence test over the whole grid.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace gc {

// out[o][a0][e] = sum_{|a - a0| <= R, 0 <= a < n_axis} taps[a - a0 + R] in[o][a][e]; arrays
// [n_outer][n_axis][inner] floats, one thread per output value.
__global__ void sm_conv_kernel(const float* __restrict__ in, float* __restrict__ out, int n_axis, int64_t inner,
                               const float* __restrict__ taps, int R, int64_t total) {
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

// The smoothed sums of every gain slot in the layout K::solve reads: scalar [Re c, Im c, A] from
// jhd (complex) and jhj (real); 2x2 [C (8), H00, H11, Re H01, Im H01] from jhd (C, 2x2 complex)
// and jhj (H, 2x2 complex).
template <class K> struct SmoothIn;
template <> struct SmoothIn<ScalarKind<float>> {
  static constexpr int JD = 2, JJ = 1;  // floats per slot in jhd, jhj
  static GC_DEV void load(const float* jd, const float* jj, int64_t x, float* v) {
    v[0] = jd[2 * x]; v[1] = jd[2 * x + 1]; v[2] = jj[x];
  }
};
template <> struct SmoothIn<JonesKind<float>> {
  static constexpr int JD = 8, JJ = 8;
  static GC_DEV void load(const float* jd, const float* jj, int64_t x, float* v) {
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = jd[8 * x + c];
    const float* h = jj + 8 * x;
    v[8] = h[0]; v[9] = h[6]; v[10] = h[2]; v[11] = h[3];
  }
};

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

// e^{-i arg z} (1 for z = 0)
GC_DEV Cx<float> unphase(double zx, double zy) {
  const double m = sqrt(zx * zx + zy * zy);
  return m > 0.0 ? cx<float>((float)(zx / m), (float)(-zy / m)) : cx<float>(1.f, 0.f);
}

// One CTA per sample: for its antennas the GN gains from the smoothed sums, rotated by the common
// phase that best aligns them with the current gains; the schedule (odd k: those gains, even k:
// their average with the current ones); the result put in the canonical gauge (sum of the gains,
// 2x2 of their traces, real and non-negative) and staged in gnew; the sample's step norms.
// state[0] done, [1] iterations, [2] status, [3] apply the staged gains.
// partials: per sample {|dg|^2, |g|^2 (FP64), flags (bit 0 non-finite, bit 1 singular)}.
template <class K>
__global__ void __launch_bounds__(64) sm_update_kernel(const float* __restrict__ jd, const float* __restrict__ jj,
                                                       const float* __restrict__ gains, float* __restrict__ gnew,
                                                       int n_ant, int k, int schedule, const int* state,
                                                       double* partials) {
  using P = SmoothPhase<K>;
  __shared__ double red[32];
  if (state[0]) return;
  const int smp = blockIdx.x, tid = threadIdx.x;
  const int64_t g0 = (int64_t)smp * n_ant;
  const bool gn_step = schedule == GC_SCHED_GN || (k & 1);
  int sing = 0;
  // GN gains and their alignment sum
  double ax = 0.0, ay = 0.0;
  for (int p = tid; p < n_ant; p += blockDim.x) {
    float v[K::NC];
    SmoothIn<K>::load(jd, jj, g0 + p, v);
    const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
    typename K::G gn;
    if (!K::solve(v, old, gn)) sing = 1;
    K::st_gain(gnew + K::GW * (g0 + p), gn);
    const Cx<float> t = P::inner(old, gn);
    ax += t.x; ay += t.y;
  }
  ax = block_sum<double>(ax, red);
  ay = block_sum<double>(ay, red);
  const Cx<float> ea = unphase(ax, ay);
  // aligned, scheduled gains and their canonical-gauge sum
  double sx = 0.0, sy = 0.0;
  for (int p = tid; p < n_ant; p += blockDim.x) {
    const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
    const typename K::G gn = P::rot(K::ld_gain(gnew + K::GW * (g0 + p)), ea);
    const typename K::G nw = gn_step ? gn : K::avg(old, gn);
    K::st_gain(gnew + K::GW * (g0 + p), nw);
    const Cx<float> t = P::trace(nw);
    sx += t.x; sy += t.y;
  }
  sx = block_sum<double>(sx, red);
  sy = block_sum<double>(sy, red);
  const Cx<float> ec = unphase(sx, sy);
  double d2 = 0.0, n2 = 0.0;
  int nonfin = 0;
  for (int p = tid; p < n_ant; p += blockDim.x) {
    const typename K::G old = K::ld_gain(gains + K::GW * (g0 + p));
    const typename K::G nw = P::rot(K::ld_gain(gnew + K::GW * (g0 + p)), ec);
    if (!K::finite(nw)) nonfin = 1;
    d2 += (double)K::dist2(nw, old);
    n2 += (double)K::norm2(nw);
    K::st_gain(gnew + K::GW * (g0 + p), nw);
  }
  d2 = block_sum<double>(d2, red);
  n2 = block_sum<double>(n2, red);
  const int fl = __syncthreads_or(nonfin) | (__syncthreads_or(sing) << 1);
  if (tid == 0) {
    double* q = partials + 3 * smp;
    q[0] = d2; q[1] = n2; q[2] = (double)fl;
  }
}

// One CTA: the grid's step norms from the per-sample partials (each thread a fixed stride, then a
// fixed tree), the stopping rule, and whether the staged gains are applied.
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
                   void* stream) {
  const int64_t total = n_outer * n_axis * inner;
  if (total <= 0) return 0;
  sm_conv_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, out, n_axis, inner, taps, R,
                                                                                    total);
  return (int)cudaGetLastError();
}

int sm_launch_update(int kind, const float* jd, const float* jj, const float* gains, float* gnew, int n_s, int n_ant,
                     int k, int schedule, int max_iter, double tol, int* state, double* partials, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0)
    sm_update_kernel<ScalarKind<float>><<<n_s, 64, 0, s>>>(jd, jj, gains, gnew, n_ant, k, schedule, state, partials);
  else
    sm_update_kernel<JonesKind<float>><<<n_s, 64, 0, s>>>(jd, jj, gains, gnew, n_ant, k, schedule, state, partials);
  sm_final_kernel<<<1, 256, 0, s>>>(partials, n_s, k, max_iter, tol, state);
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
