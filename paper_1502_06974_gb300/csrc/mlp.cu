// Learned warm start: a small MLP (IN -> 256 -> 256 -> OUT, ReLU) that proposes each interval's
// starting gains.  FP32 training (forward, backward, Adam) and BF16 inference, hand-written.
//
// Parameter buffer layout (floats, contiguous): W1 [IN][H1] | b1 [H1] | W2 [H1][H2] | b2 [H2] |
// W3 [H2][OUT] | b3 [OUT]; row-major, y = x W + b.  Activations are row-major [n][width].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "common.cuh"
#include "internal.h"

namespace gc {

extern std::atomic<long long> g_launches;
int set_cuda_error(cudaError_t e, const char* what);
int ws_get(const char* name, size_t bytes, void** out);

constexpr int kT = 32;  // GEMM tile

// C[M][N] = op(A) op(B) (+ bias[N]) (ReLU) with op(A) = A [M][K] or A^T (A stored [K][M]) and
// op(B) = B [K][N] or B^T (B stored [N][K]).  beta: C = beta * C + result.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                    float* __restrict__ Cm, const float* __restrict__ bias, int M,
                                                    int N, int K, int relu, float beta) {
  __shared__ float As[kT][kT + 1], Bs[kT][kT + 1];
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;  // 32 x 8 threads, 4 rows each
  const int row0 = blockIdx.y * kT, col = blockIdx.x * kT + tx;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += kT) {
    for (int r = ty; r < kT; r += 8) {
      const int gr = row0 + r, gk = k0 + tx;
      As[r][tx] = (gr < M && gk < K) ? (TA ? A[(size_t)gk * M + gr] : A[(size_t)gr * K + gk]) : 0.f;
      const int bk = k0 + r, bn = blockIdx.x * kT + tx;
      Bs[r][tx] = (bk < K && bn < N) ? (TB ? B[(size_t)bn * K + bk] : B[(size_t)bk * N + bn]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kT; ++kk) {
      const float b = Bs[kk][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(As[ty * 4 + j][kk], b, acc[j]);
    }
    __syncthreads();
  }
  if (col >= N) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = row0 + ty * 4 + j;
    if (r >= M) continue;
    float v = acc[j] + (bias ? bias[col] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    float* c = Cm + (size_t)r * N + col;
    *c = beta != 0.f ? beta * *c + v : v;
  }
}

static int sgemm(bool ta, bool tb, const float* A, const float* B, float* C, const float* bias, int M, int N, int K,
                 int relu, float beta, cudaStream_t s) {
  const dim3 grid((N + kT - 1) / kT, (M + kT - 1) / kT);
  if (!ta && !tb) sgemm_kernel<false, false><<<grid, 256, 0, s>>>(A, B, C, bias, M, N, K, relu, beta);
  else if (ta && !tb) sgemm_kernel<true, false><<<grid, 256, 0, s>>>(A, B, C, bias, M, N, K, relu, beta);
  else if (!ta && tb) sgemm_kernel<false, true><<<grid, 256, 0, s>>>(A, B, C, bias, M, N, K, relu, beta);
  else sgemm_kernel<true, true><<<grid, 256, 0, s>>>(A, B, C, bias, M, N, K, relu, beta);
  g_launches++;
  return (int)cudaGetLastError();
}

// d <- d * (h > 0)
__global__ void relu_mask_kernel(float* d, const float* h, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && !(h[i] > 0.f)) d[i] = 0.f;
}

// column sums of D [n][w] -> out[w] (fixed order per column)
__global__ void colsum_kernel(const float* D, int n, int w, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= w) return;
  float s = 0.f, cc = 0.f;
  for (int r = 0; r < n; ++r) kahan_add(s, cc, D[(size_t)r * w + c]);
  out[c] = s - cc;
}

// dy = 2 (y - t) / (n * out); per-row squared error into err[n]
__global__ void mse_grad_kernel(const float* y, const float* t, int n, int out, float* dy, float* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float sc = 2.f / ((float)n * out);
  float e = 0.f;
  for (int c = 0; c < out; ++c) {
    const float d = y[(size_t)r * out + c] - t[(size_t)r * out + c];
    dy[(size_t)r * out + c] = sc * d;
    e = fmaf(d, d, e);
  }
  err[r] = e;
}

__global__ void sum_kernel(const float* v, int n, float scale, float* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  s = block_sum<double>(s, red);
  if (threadIdx.x == 0) *out = (float)(s * scale);
}

// Adam (bias-corrected), step t >= 1
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* q, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

// dst[r][:] = src[index[r]][:], rows of w floats
__global__ void rows_gather_kernel(const float* src, int w, const int64_t* index, int64_t n, float* dst) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * w) return;
  const int64_t r = e / w;
  dst[e] = src[index[r] * w + (e - r * w)];
}

// Per column c of x [.][w] over the rows index[0 .. n-1] (all rows 0 .. n-1 when index is NULL):
// FP64 mean and population standard deviation, two passes (mean first, then the centred squares).
// A column whose deviation is below 1e-12 gets sd 1 (and mean 0 when zero_const_mean).
__global__ void col_stats_kernel(const float* x, int w, const int64_t* index, int64_t n, int zero_const_mean,
                                 double* mean, double* sd) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  if (c >= w) return;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += (double)x[(index ? index[r] : r) * w + c];
  const double mu = block_sum<double>(s, red) / (double)n;
  double q = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double d = (double)x[(index ? index[r] : r) * w + c] - mu;
    q = fma(d, d, q);
  }
  const double v = block_sum<double>(q, red) / (double)n;
  if (threadIdx.x == 0) {
    double sdv = sqrt(v), m = mu;
    if (sdv < 1e-12) {
      sdv = 1.0;
      if (zero_const_mean) m = 0.0;
    }
    mean[c] = m;
    sd[c] = sdv;
  }
}

// out = (x - mean) / sd per column, in FP64, rounded to FP32 (mean may be NULL: no centring)
__global__ void standardize_kernel(const float* x, int w, int64_t n, const double* mean, const double* sd, float* out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * w) return;
  const int c = (int)(e % w);
  out[e] = (float)(((double)x[e] - (mean ? mean[c] : 0.0)) / sd[c]);
}

// Fold x -> (x - mean) / sd into the first layer and y -> y * tsd into the last, in place:
// b1[h] -= sum_i (mean_i / sd_i) W1[i][h], W1[i][h] /= sd_i, W3[.][o] *= tsd_o, b3[o] *= tsd_o (FP64).
// One thread per first-layer unit h (it alone touches column h of W1 and b1[h]) and, after them,
// one per last-layer weight or bias.
__global__ void fold_standardization_kernel(float* p, int in, int h1, int h2, int out, const double* mean,
                                            const double* sd, const double* tsd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < h1) {
    double b = p[(size_t)in * h1 + t];
    for (int i = 0; i < in; ++i) {
      const double wv = p[(size_t)i * h1 + t];
      b -= (mean[i] / sd[i]) * wv;
      p[(size_t)i * h1 + t] = (float)(wv / sd[i]);
    }
    p[(size_t)in * h1 + t] = (float)b;
    return;
  }
  const int u = t - h1;
  const size_t o3 = (size_t)in * h1 + h1 + (size_t)h1 * h2 + h2;
  if (u < h2 * out) p[o3 + u] = (float)((double)p[o3 + u] * tsd[u % out]);
  else if (u < h2 * out + out) p[o3 + u] = (float)((double)p[o3 + u] * tsd[u - h2 * out]);
}

// BF16 inference: weights and activations in BF16, products accumulated in FP32.  One CTA holds
// all weights in shared memory and runs rows in tiles of kRows; thread j owns hidden unit j.
constexpr int kRows = 16;
template <int IN, int H1, int H2, int OUT>
__global__ void __launch_bounds__(256) mlp_infer_bf16_kernel(const __nv_bfloat16* __restrict__ w, const float* x,
                                                             int n, float* y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* b1 = W1 + IN * H1;
  __nv_bfloat16* W2 = b1 + H1;
  __nv_bfloat16* b2 = W2 + H1 * H2;
  __nv_bfloat16* W3 = b2 + H2;
  __nv_bfloat16* b3 = W3 + H2 * OUT;
  __nv_bfloat16* xs = b3 + OUT + 8;                 // [kRows][IN]
  __nv_bfloat16* h1 = xs + kRows * IN;              // [kRows][H1]
  __nv_bfloat16* h2 = h1 + kRows * H1;              // [kRows][H2]
  constexpr int NP = IN * H1 + H1 + H1 * H2 + H2 + H2 * OUT + OUT;
  for (int i = threadIdx.x; i < NP; i += blockDim.x) W1[i] = w[i];
  __syncthreads();
  for (int r0 = blockIdx.x * kRows; r0 < n; r0 += gridDim.x * kRows) {
    const int nr = min(kRows, n - r0);
    for (int i = threadIdx.x; i < kRows * IN; i += blockDim.x)
      xs[i] = __float2bfloat16_rn(i / IN < nr ? x[(size_t)r0 * IN + i] : 0.f);
    __syncthreads();
    for (int j = threadIdx.x; j < H1; j += blockDim.x) {
      float acc[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r] = __bfloat162float(b1[j]);
      for (int k = 0; k < IN; ++k) {
        const float wk = __bfloat162float(W1[k * H1 + j]);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = fmaf(__bfloat162float(xs[r * IN + k]), wk, acc[r]);
      }
#pragma unroll
      for (int r = 0; r < kRows; ++r) h1[r * H1 + j] = __float2bfloat16_rn(fmaxf(acc[r], 0.f));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < H2; j += blockDim.x) {
      float acc[kRows];
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r] = __bfloat162float(b2[j]);
      for (int k = 0; k < H1; ++k) {
        const float wk = __bfloat162float(W2[k * H2 + j]);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = fmaf(__bfloat162float(h1[r * H1 + k]), wk, acc[r]);
      }
#pragma unroll
      for (int r = 0; r < kRows; ++r) h2[r * H2 + j] = __float2bfloat16_rn(fmaxf(acc[r], 0.f));
    }
    __syncthreads();
    for (int o = threadIdx.x; o < kRows * OUT; o += blockDim.x) {
      const int r = o / OUT, c = o - r * OUT;
      float acc = __bfloat162float(b3[c]);
      for (int k = 0; k < H2; ++k) acc = fmaf(__bfloat162float(h2[r * H2 + k]), __bfloat162float(W3[k * OUT + c]), acc);
      if (r < nr) y[(size_t)(r0 + r) * OUT + c] = acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------ features
// Per antenna of each target interval, in the frame where the newest previous gain's xx element is
// real and non-negative (rotation e^{-i phi}, phi = arg g1_xx; the problem is unchanged by a global
// phase, Sect. 2.1, and this per-antenna frame makes the network's input phase-free):
//   [g1 (8) | g1-g2 (8) | g2-g3 (8) | g3-g4 (8) | step (8) | lead (1) | zero pad]
// gk: the k-th previous 2x2 gain (row-major re, im); step = C H^-1 - g1, the GN step of the 2x2
// update (eq. update:DI:diag:pol) at g1 on the target interval (C = sum D Y^H, H = sum Y Y^H;
// zero where H is singular).  H is read either as a 2x2 complex matrix (hfmt 0, 8 reals) or as
// the packed (h00, h11, Re h01, Im h01) of the partial-sum order (hfmt 1).  rot [n][2] receives
// (cos phi, sin phi).
__global__ void ws_features_kernel(const float* hist, int hist_stride, const float* jhd, int jhd_stride,
                                   const float* jhj, int jhj_stride, int hfmt, const float* lead, int n, int in_w,
                                   float* x, float* rot) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float* h = hist + (size_t)r * hist_stride;  // 4 consecutive 2x2 gains, newest first
  float* o = x + (size_t)r * in_w;
  const float ar = h[0], ai = h[1];
  const float mag = sqrtf(ar * ar + ai * ai);
  const float c = mag > 0.f ? ar / mag : 1.f, sn = mag > 0.f ? ai / mag : 0.f;
  rot[2 * r] = c;
  rot[2 * r + 1] = sn;
  // multiply a complex pair by e^{-i phi}
  auto rotc = [&](float re, float im, float* dst) {
    dst[0] = re * c + im * sn;
    dst[1] = im * c - re * sn;
  };
  for (int e = 0; e < 4; ++e) {
    const int k = 2 * e;
    rotc(h[k], h[k + 1], o + k);
    rotc(h[k] - h[8 + k], h[k + 1] - h[9 + k], o + 8 + k);
    rotc(h[8 + k] - h[16 + k], h[9 + k] - h[17 + k], o + 16 + k);
    rotc(h[16 + k] - h[24 + k], h[17 + k] - h[25 + k], o + 24 + k);
  }
  const float* C = jhd + (size_t)r * jhd_stride;
  const float* H = jhj + (size_t)r * jhj_stride;
  float h00, h11;
  Cx<float> h01;
  if (hfmt == 0) { h00 = H[0]; h11 = H[6]; h01 = cx<float>(H[2], H[3]); }
  else { h00 = H[0]; h11 = H[1]; h01 = cx<float>(H[2], H[3]); }
  const float det = h00 * h11 - abs2_(h01);
  float st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (det > 0.f && h00 > 0.f) {
    const float inv = 1.f / det;
    const Cx<float> C00 = cx<float>(C[0], C[1]), C01 = cx<float>(C[2], C[3]), C10 = cx<float>(C[4], C[5]),
                    C11 = cx<float>(C[6], C[7]);
    const Cx<float> g00 = scale_(sub_(scale_(C00, h11), mulc_(C01, h01)), inv);
    const Cx<float> g01 = scale_(sub_(scale_(C01, h00), mul_(C00, h01)), inv);
    const Cx<float> g10 = scale_(sub_(scale_(C10, h11), mulc_(C11, h01)), inv);
    const Cx<float> g11 = scale_(sub_(scale_(C11, h00), mul_(C10, h01)), inv);
    const float gn[8] = {g00.x, g00.y, g01.x, g01.y, g10.x, g10.y, g11.x, g11.y};
    for (int k = 0; k < 8; ++k) st[k] = gn[k] - h[k];
  }
  for (int e = 0; e < 4; ++e) rotc(st[2 * e], st[2 * e + 1], o + 32 + 2 * e);
  o[40] = lead[r];
  for (int k = 41; k < in_w; ++k) o[k] = 0.f;
}

// proposal = g1 + e^{i phi} delta (delta predicted in the rotated frame); g1 has stride g1_stride
__global__ void ws_propose_kernel(const float* g1, int g1_stride, const float* delta, const float* rot, int n,
                                  float* prop) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float c = rot[2 * r], sn = rot[2 * r + 1];
  const float* g = g1 + (size_t)r * g1_stride;
  for (int e = 0; e < 4; ++e) {
    const float dr = delta[8 * r + 2 * e], di = delta[8 * r + 2 * e + 1];
    prop[8 * r + 2 * e] = g[2 * e] + dr * c - di * sn;
    prop[8 * r + 2 * e + 1] = g[2 * e + 1] + dr * sn + di * c;
  }
}

// training target = e^{-i phi} (g_next - g1)
__global__ void ws_target_kernel(const float* g1, const float* gnext, const float* rot, int n, float* t) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float c = rot[2 * r], sn = rot[2 * r + 1];
  for (int e = 0; e < 4; ++e) {
    const float dr = gnext[8 * r + 2 * e] - g1[8 * r + 2 * e], di = gnext[8 * r + 2 * e + 1] - g1[8 * r + 2 * e + 1];
    t[8 * r + 2 * e] = dr * c + di * sn;
    t[8 * r + 2 * e + 1] = di * c - dr * sn;
  }
}

// One CTA per target interval i = i_lo + b: the 4 previous solutions of each antenna (newest
// first) into hbuf [.][32], the newest also into g1 [.][8], and the interval's lead into each row;
// rows are the interval's gain slots minus gbase.  With canon != 0 each previous solution is first
// put in the canonical gauge (sum over the interval's antennas of tr(G) real, non-negative).
__global__ void ws_gather_kernel(const float* sol, const int32_t* hoff, const float* lead, const int32_t* gain_off,
                                 const int32_t* n_ant, int i_lo, int n, int64_t gbase, int canon, float* hbuf,
                                 float* g1, float* lead_row) {
  __shared__ double red[32];
  __shared__ float rc[4][2];
  const int b = blockIdx.x;
  if (b >= n) return;
  const int i = i_lo + b;
  const int na = n_ant[i];
  const int64_t go = gain_off[i] - gbase;
  if (threadIdx.x < 8) rc[threadIdx.x / 2][threadIdx.x % 2] = threadIdx.x % 2 ? 0.f : 1.f;
  __syncthreads();
  if (canon)
    for (int j = 0; j < 4; ++j) {
      const float* h = sol + (int64_t)hoff[4 * b + j] * 8;
      double sr = 0.0, si = 0.0;
      for (int an = threadIdx.x; an < na; an += blockDim.x) {
        sr += (double)h[an * 8] + (double)h[an * 8 + 6];
        si += (double)h[an * 8 + 1] + (double)h[an * 8 + 7];
      }
      sr = block_sum<double>(sr, red);
      si = block_sum<double>(si, red);
      const double m = sqrt(sr * sr + si * si);
      if (threadIdx.x == 0 && m > 0.0) {
        rc[j][0] = (float)(sr / m);
        rc[j][1] = (float)(-si / m);
      }
    }
  __syncthreads();
  for (int x = threadIdx.x; x < na * 16; x += blockDim.x) {  // complex entries: antenna, solution, element
    const int an = x / 16, j = (x / 4) & 3, e = x & 3;
    const float* src = sol + ((int64_t)hoff[4 * b + j] + an) * 8 + 2 * e;
    const float re = src[0], im = src[1], c = rc[j][0], sn = rc[j][1];
    const float vr = re * c - im * sn, vi = re * sn + im * c;
    float* dst = hbuf + (go + an) * 32 + 8 * j + 2 * e;
    dst[0] = vr;
    dst[1] = vi;
    if (j == 0) {
      g1[(go + an) * 8 + 2 * e] = vr;
      g1[(go + an) * 8 + 2 * e + 1] = vi;
    }
  }
  for (int an = threadIdx.x; an < na; an += blockDim.x) lead_row[go + an] = lead[b];
}

// Per interval i = i_lo + b: keep the proposal (already in gains) if e_prop < e_prev, else restore
// g1 (rows relative to gbase).
__global__ void ws_choose_kernel(const float* g1, const double* e_prev, const double* e_prop, const int32_t* gain_off,
                                 const int32_t* n_ant, int i_lo, int n, int64_t gbase, float* gains, int32_t* used,
                                 double* dchi2) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const int i = i_lo + b;
  const bool take = e_prop[b] < e_prev[b];
  if (threadIdx.x == 0) {
    if (used) used[i] = take ? 1 : 0;
    if (dchi2) dchi2[i] = e_prop[b] - e_prev[b];
  }
  if (take) return;
  const int64_t go = gain_off[i] - gbase;
  for (int x = threadIdx.x; x < n_ant[i] * 8; x += blockDim.x) gains[(int64_t)gain_off[i] * 8 + x] = g1[go * 8 + x];
}

// Canonical gauge per interval: gains rotated so that sum_p tr(G_p) (or sum_p g_p) is real and
// non-negative (chi^2 is unchanged by one phase on all antennas, Sect. 2.1).  Left as is when the
// sum is zero.
template <typename T, int GW>
__global__ void gauge_fix_kernel(T* gains, const int32_t* gain_off, const int32_t* n_ant, int n_int) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  if (i >= n_int) return;
  const int na = n_ant[i];
  T* g = gains + (int64_t)gain_off[i] * GW;
  double sr = 0.0, si = 0.0;
  for (int an = threadIdx.x; an < na; an += blockDim.x) {
    sr += (double)g[an * GW];
    si += (double)g[an * GW + 1];
    if (GW == 8) { sr += (double)g[an * GW + 6]; si += (double)g[an * GW + 7]; }
  }
  sr = block_sum<double>(sr, red);
  si = block_sum<double>(si, red);
  const double m = sqrt(sr * sr + si * si);
  if (!(m > 0.0)) return;
  const T c = (T)(sr / m), sn = (T)(-si / m);  // multiply by conj(s) / |s|
  for (int x = threadIdx.x; x < na * GW / 2; x += blockDim.x) {
    const T re = g[2 * x], im = g[2 * x + 1];
    g[2 * x] = re * c - im * sn;
    g[2 * x + 1] = re * sn + im * c;
  }
}

// ------------------------------------------------------------------------------------ host side
struct MlpDims {
  int in, h1, h2, out;
  size_t np() const { return (size_t)in * h1 + h1 + (size_t)h1 * h2 + h2 + (size_t)h2 * out + out; }
};

static int check_dims(const MlpDims& d) {
  if (d.in != 48 || d.h1 != 256 || d.h2 != 256 || d.out != 8) return GC_ERR_LIMIT;
  return GC_OK;
}

// work buffer: h1 [n][H1] | h2 [n][H2] | y [n][OUT] | d2 [n][H2] | d1 [n][H1] | dy [n][OUT] | err [n] | loss
static size_t work_floats(const MlpDims& d, int n) {
  return (size_t)n * (2 * d.h1 + 2 * d.h2 + 2 * d.out + 1) + 8;
}

static int forward(const MlpDims& d, const float* p, const float* x, int n, float* work, cudaStream_t s) {
  const float *W1 = p, *b1 = W1 + d.in * d.h1, *W2 = b1 + d.h1, *b2 = W2 + d.h1 * d.h2, *W3 = b2 + d.h2,
              *b3 = W3 + d.h2 * d.out;
  float *h1 = work, *h2 = h1 + (size_t)n * d.h1, *y = h2 + (size_t)n * d.h2;
  int rc;
  if ((rc = sgemm(false, false, x, W1, h1, b1, n, d.h1, d.in, 1, 0.f, s))) return rc;
  if ((rc = sgemm(false, false, h1, W2, h2, b2, n, d.h2, d.h1, 1, 0.f, s))) return rc;
  return sgemm(false, false, h2, W3, y, b3, n, d.out, d.h2, 0, 0.f, s);
}

static int backward(const MlpDims& d, const float* p, const float* x, const float* t, int n, float* g, float* work,
                    float* loss, cudaStream_t s) {
  const float *W2 = p + d.in * d.h1 + d.h1, *W3 = W2 + d.h1 * d.h2 + d.h2;
  float *gW1 = g, *gb1 = gW1 + d.in * d.h1, *gW2 = gb1 + d.h1, *gb2 = gW2 + d.h1 * d.h2, *gW3 = gb2 + d.h2,
        *gb3 = gW3 + d.h2 * d.out;
  float *h1 = work, *h2 = h1 + (size_t)n * d.h1, *y = h2 + (size_t)n * d.h2, *d2 = y + (size_t)n * d.out,
        *d1 = d2 + (size_t)n * d.h2, *dy = d1 + (size_t)n * d.h1, *err = dy + (size_t)n * d.out;
  int rc;
  mse_grad_kernel<<<(n + 255) / 256, 256, 0, s>>>(y, t, n, d.out, dy, err);
  sum_kernel<<<1, 256, 0, s>>>(err, n, 1.f / ((float)n * d.out), loss);
  g_launches += 2;
  if ((rc = sgemm(true, false, h2, dy, gW3, nullptr, d.h2, d.out, n, 0, 0.f, s))) return rc;  // h2^T dy
  colsum_kernel<<<(d.out + 255) / 256, 256, 0, s>>>(dy, n, d.out, gb3);
  if ((rc = sgemm(false, true, dy, W3, d2, nullptr, n, d.h2, d.out, 0, 0.f, s))) return rc;  // dy W3^T
  relu_mask_kernel<<<(unsigned)(((size_t)n * d.h2 + 255) / 256), 256, 0, s>>>(d2, h2, (size_t)n * d.h2);
  if ((rc = sgemm(true, false, h1, d2, gW2, nullptr, d.h1, d.h2, n, 0, 0.f, s))) return rc;  // h1^T d2
  colsum_kernel<<<(d.h2 + 255) / 256, 256, 0, s>>>(d2, n, d.h2, gb2);
  if ((rc = sgemm(false, true, d2, W2, d1, nullptr, n, d.h1, d.h2, 0, 0.f, s))) return rc;  // d2 W2^T
  relu_mask_kernel<<<(unsigned)(((size_t)n * d.h1 + 255) / 256), 256, 0, s>>>(d1, h1, (size_t)n * d.h1);
  if ((rc = sgemm(true, false, x, d1, gW1, nullptr, d.in, d.h1, n, 0, 0.f, s))) return rc;  // x^T d1
  colsum_kernel<<<(d.h1 + 255) / 256, 256, 0, s>>>(d1, n, d.h1, gb1);
  g_launches += 5;
  return (int)cudaGetLastError();
}

}  // namespace gc

using namespace gc;

extern "C" {

size_t gc_mlp_work_floats(const gc_mlp* net, int32_t n) {
  if (!net) return 0;
  return work_floats(MlpDims{net->in, net->h1, net->h2, net->out}, n);
}

int gc_mlp_forward_f32(const gc_mlp* net, const float* x, int32_t n, float* y, float* work, void* stream) {
  if (!net || n < 0) return GC_ERR_ARG;
  const MlpDims d{net->in, net->h1, net->h2, net->out};
  int rc = check_dims(d);
  if (rc) return rc;
  if (n == 0) return GC_OK;
  if (!net->params || !x || !y || !work) return GC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = forward(d, net->params, x, n, work, s))) return set_cuda_error((cudaError_t)rc, "mlp forward");
  const float* yw = work + (size_t)n * (d.h1 + d.h2);
  cudaError_t e = cudaMemcpyAsync(y, yw, (size_t)n * d.out * sizeof(float), cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "mlp forward copy");
}

int gc_mlp_grad_f32(const gc_mlp* net, const float* x, const float* t, int32_t n, float* grads, float* loss,
                    float* work, void* stream) {
  if (!net || !x || !t || !grads || !loss || !work || n < 1) return GC_ERR_ARG;
  const MlpDims d{net->in, net->h1, net->h2, net->out};
  int rc = check_dims(d);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = forward(d, net->params, x, n, work, s))) return set_cuda_error((cudaError_t)rc, "mlp forward");
  if ((rc = backward(d, net->params, x, t, n, grads, work, loss, s))) return set_cuda_error((cudaError_t)rc, "mlp backward");
  return GC_OK;
}

int gc_mlp_train_step(gc_mlp* net, const float* x, const float* t, int32_t n, float lr, int32_t step, float* loss,
                      float* work, void* stream) {
  if (!net || !net->grads || !net->adam_m || !net->adam_v || step < 1) return GC_ERR_ARG;
  int rc = gc_mlp_grad_f32(net, x, t, n, net->grads, loss, work, stream);
  if (rc) return rc;
  const MlpDims d{net->in, net->h1, net->h2, net->out};
  const size_t np = d.np();
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, (cudaStream_t)stream>>>(net->params, net->grads, net->adam_m,
                                                                              net->adam_v, np, lr, b1, b2, 1e-8f, c1, c2);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "adam");
}

int gc_mlp_infer_bf16(const gc_mlp* net, const float* x, int32_t n, float* y, void* stream) {
  if (!net || n < 0) return GC_ERR_ARG;
  const MlpDims d{net->in, net->h1, net->h2, net->out};
  int rc = check_dims(d);
  if (rc) return rc;
  if (n == 0) return GC_OK;
  if (!net->params || !net->params_bf16 || !x || !y) return GC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t np = d.np();
  __nv_bfloat16* wq = reinterpret_cast<__nv_bfloat16*>(net->params_bf16);
  to_bf16_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(net->params, wq, np);
  const size_t smem = sizeof(__nv_bfloat16) * (np + 8 + (size_t)kRows * (d.in + d.h1 + d.h2));
  cudaError_t e = cudaFuncSetAttribute(mlp_infer_bf16_kernel<48, 256, 256, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_cuda_error(e, "mlp infer attribute");
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int grid = (n + kRows - 1) / kRows;
  if (grid > nsm) grid = nsm;
  mlp_infer_bf16_kernel<48, 256, 256, 8><<<grid, 256, smem, s>>>(wq, x, n, y);
  g_launches += 2;
  e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "mlp infer");
}

int gc_ws_features_jones(const float* hist, int32_t hist_stride, const float* jhd, const float* jhj, const float* lead,
                         int32_t n, int32_t in_width, float* x, float* rot, void* stream) {
  if (n < 0 || in_width < 41 || hist_stride < 32) return GC_ERR_ARG;
  if (n == 0) return GC_OK;
  if (!hist || !jhd || !jhj || !lead || !x || !rot) return GC_ERR_ARG;
  ws_features_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(hist, hist_stride, jhd, 8, jhj, 8, 0, lead, n,
                                                                       in_width, x, rot);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "features");
}

int gc_ws_target_jones(const float* g1, const float* g_next, const float* rot, int32_t n, float* target,
                       void* stream) {
  if (n < 0) return GC_ERR_ARG;
  if (n == 0) return GC_OK;
  if (!g1 || !g_next || !rot || !target) return GC_ERR_ARG;
  ws_target_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(g1, g_next, rot, n, target);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "target");
}

int gc_rows_gather_f32(const float* src, int32_t width, const int64_t* index, int64_t n, float* dst, void* stream) {
  if (width < 1 || n < 0) return GC_ERR_ARG;
  if (n == 0) return GC_OK;
  if (!src || !index || !dst) return GC_ERR_ARG;
  const int64_t ne = n * width;
  rows_gather_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src, width, index, n, dst);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "rows gather");
}

int gc_col_stats_f32(const float* x, int32_t width, const int64_t* index, int64_t n, int32_t zero_const_mean,
                     double* mean, double* sd, void* stream) {
  if (width < 1 || n < 1 || !x || !mean || !sd) return GC_ERR_ARG;
  col_stats_kernel<<<width, 256, 0, (cudaStream_t)stream>>>(x, width, index, n, zero_const_mean, mean, sd);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "column statistics");
}

int gc_standardize_f32(const float* x, int32_t width, int64_t n, const double* mean, const double* sd, float* out,
                       void* stream) {
  if (width < 1 || n < 0) return GC_ERR_ARG;
  if (n == 0) return GC_OK;
  if (!x || !sd || !out) return GC_ERR_ARG;
  const int64_t ne = n * width;
  standardize_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, width, n, mean, sd, out);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "standardize");
}

int gc_mlp_fold_standardization(gc_mlp* net, const double* mean, const double* sd, const double* tsd, void* stream) {
  if (!net || !net->params || !mean || !sd || !tsd) return GC_ERR_ARG;
  const MlpDims d{net->in, net->h1, net->h2, net->out};
  int rc = check_dims(d);
  if (rc) return rc;
  const int nt = d.h1 + d.h2 * d.out + d.out;
  fold_standardization_kernel<<<(nt + 255) / 256, 256, 0, (cudaStream_t)stream>>>(net->params, d.in, d.h1, d.h2,
                                                                                   d.out, mean, sd, tsd);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GC_OK : set_cuda_error(e, "fold standardization");
}

}  // extern "C"

namespace gc {

int mlp_check(const gc_mlp* net) {
  if (!net || !net->params || !net->params_bf16) return GC_ERR_ARG;
  return check_dims(MlpDims{net->in, net->h1, net->h2, net->out});
}

int ws_gather(const float* sol, const int32_t* hoff, const float* lead, const int32_t* gain_off, const int32_t* n_ant,
              int i_lo, int n, int64_t gbase, int canon, float* hbuf, float* g1, float* lead_row, void* stream) {
  if (n <= 0) return 0;
  ws_gather_kernel<<<n, 256, 0, (cudaStream_t)stream>>>(sol, hoff, lead, gain_off, n_ant, i_lo, n, gbase, canon, hbuf,
                                                        g1, lead_row);
  return (int)cudaGetLastError();
}

int ws_features_packed(const float* hbuf, const float* tot, const float* lead_row, int n, float* x, float* rot,
                       void* stream) {
  ws_features_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(hbuf, 32, tot, 12, tot + 8, 12, 1, lead_row,
                                                                       n, 48, x, rot);
  return (int)cudaGetLastError();
}

int ws_propose(const float* hbuf, const float* delta, const float* rot, int n, float* gains, void* stream) {
  ws_propose_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(hbuf, 32, delta, rot, n, gains);
  return (int)cudaGetLastError();
}

int ws_choose(const float* g1, const double* e_prev, const double* e_prop, const int32_t* gain_off,
              const int32_t* n_ant, int i_lo, int n, int64_t gbase, float* gains, int32_t* used, double* dchi2,
              void* stream) {
  if (n <= 0) return 0;
  ws_choose_kernel<<<n, 128, 0, (cudaStream_t)stream>>>(g1, e_prev, e_prop, gain_off, n_ant, i_lo, n, gbase, gains,
                                                        used, dchi2);
  return (int)cudaGetLastError();
}

int mlp_infer(const gc_mlp* net, const float* x, int n, float* y, void* stream) {
  return gc_mlp_infer_bf16(net, x, n, y, stream);
}

int gauge_fix(int kind, int dtype, void* gains, const int32_t* gain_off, const int32_t* n_ant, int n_int,
              void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0) {
    if (dtype == GC_DTYPE_C64) gauge_fix_kernel<float, 2><<<n_int, 128, 0, s>>>((float*)gains, gain_off, n_ant, n_int);
    else gauge_fix_kernel<double, 2><<<n_int, 128, 0, s>>>((double*)gains, gain_off, n_ant, n_int);
  } else {
    if (dtype == GC_DTYPE_C64) gauge_fix_kernel<float, 8><<<n_int, 128, 0, s>>>((float*)gains, gain_off, n_ant, n_int);
    else gauge_fix_kernel<double, 8><<<n_int, 128, 0, s>>>((double*)gains, gain_off, n_ant, n_int);
  }
  return (int)cudaGetLastError();
}

}  // namespace gc
