// Levenberg-Marquardt with the whole J^H J (App. C, Algorithm LM; Sect. 1, eq. LM) for the
// direction-independent solvers, run on the per-baseline moments of each interval.
//
// StefCal (Sect. 3.1) drops the off-diagonal antenna blocks of J^H J.  On 2x2 problems with a weakly
// polarized sky it then crawls along the near-unitary directions G_p -> G_p U, contracting by a
// factor close to 1 per iteration.  This file takes the other option Sect. 4.3 names: substitute
// the 4x4 forms of the operators (App. B) into eq. JHJ:pol and solve the whole system.
//
// Unknowns.  Real coordinates of the gains in their storage order: per antenna the entries of G_p
// (2x2: G00, G01, G10, G11; scalar: g) as (re, im) pairs, n = 8 N_ant (scalar 2 N_ant) reals.  The
// GN model of chi^2 = sum ||D - G_p M G_q^H||^2 around G is x^T H x - 2 x^T g with
//   g       = J^H R per antenna (eq. JHR for 2x2 with the product order R Y^H; eq. JHR:DI),
//   H[p][p] = the map d -> d sum_q Y_pq Y_pq^H   (eq. JHJ:pol top-left, eq. JHJ:DI A),
//   H[p][q] = the map d_q -> G_p Phi_pq(d_q^H G_q) (eq. JHJ:pol top-right R_{Y^H_pq} L_{Y^H_qp};
//             scalar: d_q -> g_p g_q Q_pq conj(d_q), eq. JHJ:DI B),
// Phi_pq(X) = sum_s M X M^H.  Everything is computed from the moments of the interval (P_pq =
// sum_s conj(M) kron D, R_pq = Phi_pq on Hermitian coordinates; scalar B_pq = sum conj(m) d,
// Q_pq = sum |m|^2), since the gains factor out of the sample sums.
//
// One LM iteration per interval (App. C): H and g at the current gains; the step solves
//   (H + lambda diag(H) + mu v v^T) x = (I - v v^T) g,
// v the unit vector of the phase-gauge direction i G (chi^2 is unchanged by G -> G e^{i phi},
// Sect. 2.1, so J^H J is singular along v) and mu the mean of diag(H): the step is taken in the
// complement of the gauge direction, and the matrix stays well conditioned however small lambda
// gets.  The factorisation is an FP32 blocked Cholesky in global memory (panels of 32 columns in
// shared memory, warp-tiled rank-32 trailing updates); chi^2 at the trial gains is summed in FP64
// from the FP32 residuals of the interval's rows; lambda is updated in FP64: divided by K after a
// step that lowered chi^2, multiplied by K (gains kept) after one that did not.  An interval stops
// when a step is below tol ||G|| (App. C, first criterion).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace gc {

extern std::atomic<long long> g_launches;
int ws_get(const char* name, size_t bytes, void** out);
int set_cuda_error(cudaError_t e, const char* what);
int pinned_flag(int** out);
uint64_t layout_hash(const gc_layout* L, uint64_t salt);

constexpr int kLMThreads = 256;
constexpr int kNB = 32;  // Cholesky panel width

struct LMArgs {
  const float* vis;         // the rows (complex64; 2x2 row-major for the 2x2 kind)
  const float* model;
  const float* weights;     // per-row weights (Sect. 2.4) or NULL
  const int64_t* row_off;   // [n_int] first row of the interval
  const int32_t* n_samp;    // [n_int] samples per baseline
  const float* moments;
  const int64_t* mom_off;   // [n_int] baseline slot of the interval's first moment tile
  float* gains;
  const int32_t* ant1;      // baseline tables
  const int32_t* ant2;
  const int4* iinfo;        // [n_int] {table, n_ant, gain_off, n_bl}
  const int4* tinfo;        // [n_tab] {first pair_off entry, first ant_off entry, bl_off, antennas spanned}
  const int32_t* pair_off;  // per table and antenna pair P > Q (index P(P-1)/2 + Q): offsets into pair_ent
  const int32_t* pair_ent;  // baseline * 2 + (1 if the baseline's first antenna is P)
  const int32_t* ant_off;   // per table and antenna: offsets into ant_ent
  const int32_t* ant_ent;   // baseline * 2 + (1 if the antenna is the baseline's second)
  double* lam;              // [n_int] damping
  double* chi;              // [n_int] chi^2 at the current gains
  int32_t* iters;
  int32_t* status;
  int32_t* list;            // [3][n_int] active intervals: iteration k reads list k % 3, appends to (k+1) % 3
  int32_t* cnt;             // [0..2] list lengths, [3..5] work heads
  float* work;              // per CTA: npad_max^2 floats (the damped J^H J, factored in place)
  int64_t work_stride;
  double lam0;
  double tol;
  double K;
  int32_t max_iter;
  int32_t k;
  int32_t n_int;
  double* flop;             // optional: algorithmic flops of the factorisations and solves, summed
  unsigned long long* phase;  // optional [kLMPhases]: SM cycles per phase, summed over intervals
};

// Phases of one LM iteration of an interval (profile only): per-antenna sums, the matrix, the
// factorisation with the forward substitution, the back substitution, trial gains and chi^2; then,
// inside the factorisation, the panel loads, the panel solves and the trailing updates.
constexpr int kLMPhases = 8;

GC_DEV void lm_mark(unsigned long long* phase, int ph, long long& t0) {
  if (phase && threadIdx.x == 0) {
    const long long t = clock64();
    atomicAdd(phase + ph, (unsigned long long)(t - t0));
    t0 = t;
  }
}

// ------------------------------------------------------------------------------------------
// Per-kind pieces.  Gains: GW floats per antenna, (re, im) pairs in storage order.
// ------------------------------------------------------------------------------------------
struct LMJones {
  static constexpr int GW = 8, NM = 48, AW = 4;
  using RK = JonesKind<float>;
  static GC_DEV void ld_mom(const float* mom, int64_t moff, int b, float* m) {
#pragma unroll
    for (int c = 0; c < NM; c += 4) {
      const float4 v = *reinterpret_cast<const float4*>(mom + mom_index(moff, b, c, NM));
      m[c] = v.x; m[c + 1] = v.y; m[c + 2] = v.z; m[c + 3] = v.w;
    }
  }
  // G^H G as (a00, a11, Re a01, Im a01)
  static GC_DEV void aux(const float* g, float* a) {
    a[0] = g[0] * g[0] + g[1] * g[1] + g[4] * g[4] + g[5] * g[5];
    a[1] = g[2] * g[2] + g[3] * g[3] + g[6] * g[6] + g[7] * g[7];
    // conj(G00) G01 + conj(G10) G11
    a[2] = g[0] * g[2] + g[1] * g[3] + g[4] * g[6] + g[5] * g[7];
    a[3] = g[0] * g[3] - g[1] * g[2] + g[4] * g[7] - g[5] * g[6];
  }
  static GC_DEV float diag_sum(const float* A) { return 4.f * (A[0] + A[1]); }
  static GC_DEV bool no_data(const float* A) { return !(A[0] + A[1] > 0.f); }

  // One baseline's contribution to antenna `me` (other antenna `o`): the diagonal block
  // Hb = sum Y Y^H (4 Hermitian coordinates) and J^H R = C - G_me Hb with C = sum D Y^H.
  //   side 0 (me first):  C = unvec(P vec G_o),   Hb = R a_o
  //   side 1 (me second): C = unvec(P^H vec G_o), Hb = R' a_o, R' = W^-1 R^T W, W = diag(1, 1, 2, 2)
  static GC_DEV void side(const float* m, const float* gme, const float* go, const float* ao, int sd, float* A,
                          float* gr, float* gc) {
    const Cx<float> vo[4] = {cx<float>(go[0], go[1]), cx<float>(go[4], go[5]), cx<float>(go[2], go[3]),
                             cx<float>(go[6], go[7])};
    Cx<float> c[4];
    float h[4];
    const float* R = m + 32;
    if (sd == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        c[r] = cx<float>(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) fma_(c[r], cx<float>(m[2 * (r * 4 + k)], m[2 * (r * 4 + k) + 1]), vo[k]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) s = fmaf(R[i * 4 + j], ao[j], s);
        h[i] = s;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[k] = cx<float>(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) cfma_(c[k], cx<float>(m[2 * (r * 4 + k)], m[2 * (r * 4 + k) + 1]), vo[r]);
      }
      const float w[4] = {1.f, 1.f, 2.f, 2.f};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) s = fmaf(R[j * 4 + i] * (w[j] / w[i]), ao[j], s);
        h[i] = s;
      }
    }
    // G_me herm(h), herm(h) = [[h0, h2 + i h3], [h2 - i h3, h1]]; C row-major = (c0, c2, c1, c3)
    const Cx<float> h01 = cx<float>(h[2], h[3]), h10 = cx<float>(h[2], -h[3]);
    const Cx<float> ga = cx<float>(gme[0], gme[1]), gb = cx<float>(gme[2], gme[3]);
    const Cx<float> gc_ = cx<float>(gme[4], gme[5]), gd = cx<float>(gme[6], gme[7]);
    Cx<float> t00 = scale_(ga, h[0]); fma_(t00, gb, h10);
    Cx<float> t01 = scale_(gb, h[1]); fma_(t01, ga, h01);
    Cx<float> t10 = scale_(gc_, h[0]); fma_(t10, gd, h10);
    Cx<float> t11 = scale_(gd, h[1]); fma_(t11, gc_, h01);
    const float d[8] = {c[0].x - t00.x, c[0].y - t00.y, c[2].x - t01.x, c[2].y - t01.y,
                        c[1].x - t10.x, c[1].y - t10.y, c[3].x - t11.x, c[3].y - t11.y};
#pragma unroll
    for (int e = 0; e < 8; ++e) kahan_add(gr[e], gc[e], d[e]);
#pragma unroll
    for (int i = 0; i < 4; ++i) A[i] += h[i];
  }

  // Block of J^H J coupling the step of antenna s into the equations of antenna f, for a stored
  // baseline (f, s): d_s -> G_f Phi(d_s^H G_s).  Column (i, j, re|im) of the 8x8 real block is
  // realify(Z_ij) | realify(-i Z_ij), Z_ij = G_f unvec(w_ij), w_ij = G_s[i][0] F[:, j] + G_s[i][1] F[:, 2 + j]
  // with F the complex 4x4 matrix of Phi on vec X, rebuilt from R (Phi(E_00), Phi(E_11) are Hermitian
  // with coordinates R[:, 0], R[:, 1]; Phi(E_01) = (R[:, 2] - i R[:, 3]) / 2, Phi(E_10) = (R[:, 2] + i R[:, 3]) / 2).
  // tr: add the transposed block (the equations of s, step of f).
  static GC_DEV void cross(const float* m, const float* gf, const float* gs, bool tr, float* blk) {
    const float* R = m + 32;
    // vec of the Hermitian matrix with coordinates (h0, h1, h2, h3): (h0, h2 - i h3, h2 + i h3, h1)
    auto hv = [&](int c, Cx<float>* v) {
      v[0] = cx<float>(R[0 * 4 + c], 0.f);
      v[1] = cx<float>(R[2 * 4 + c], -R[3 * 4 + c]);
      v[2] = cx<float>(R[2 * 4 + c], R[3 * 4 + c]);
      v[3] = cx<float>(R[1 * 4 + c], 0.f);
    };
    Cx<float> u2[4], u3[4];
    hv(2, u2);
    hv(3, u3);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      Cx<float> Fa[4], Fb[4];
      if (j == 0) {
        hv(0, Fa);
#pragma unroll
        for (int r = 0; r < 4; ++r) Fb[r] = cx<float>(0.5f * (u2[r].x + u3[r].y), 0.5f * (u2[r].y - u3[r].x));
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) Fa[r] = cx<float>(0.5f * (u2[r].x - u3[r].y), 0.5f * (u2[r].y + u3[r].x));
        hv(1, Fb);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const Cx<float> s0 = cx<float>(gs[4 * i + 0], gs[4 * i + 1]), s1 = cx<float>(gs[4 * i + 2], gs[4 * i + 3]);
        Cx<float> w[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) { w[r] = mul_(s0, Fa[r]); fma_(w[r], s1, Fb[r]); }
        // unvec: [[w0, w2], [w1, w3]]; Z = G_f W
        const Cx<float> fa = cx<float>(gf[0], gf[1]), fb = cx<float>(gf[2], gf[3]);
        const Cx<float> fc = cx<float>(gf[4], gf[5]), fd = cx<float>(gf[6], gf[7]);
        Cx<float> Z[4];
        Z[0] = mul_(fa, w[0]); fma_(Z[0], fb, w[1]);
        Z[1] = mul_(fa, w[2]); fma_(Z[1], fb, w[3]);
        Z[2] = mul_(fc, w[0]); fma_(Z[2], fd, w[1]);
        Z[3] = mul_(fc, w[2]); fma_(Z[3], fd, w[3]);
        const int k = 2 * (2 * i + j);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float re[2] = {Z[e].x, Z[e].y}, im[2] = {Z[e].y, -Z[e].x};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 2 * e + h;
            if (!tr) { blk[r * 8 + k] += re[h]; blk[r * 8 + k + 1] += im[h]; }
            else { blk[k * 8 + r] += re[h]; blk[(k + 1) * 8 + r] += im[h]; }
          }
        }
      }
    }
  }

  // The antenna's own block: d -> d herm(A) (the same 4x4 for both rows of d) plus lambda diag.
  static GC_DEV void diag(const float* A, float lam, float* blk) {
    const float a0 = A[0] * (1.f + lam), a1 = A[1] * (1.f + lam), a2 = A[2], a3 = A[3];
    const float T[16] = {a0, 0.f, a2, a3,   0.f, a0, -a3, a2,   a2, -a3, a1, 0.f,   a3, a2, 0.f, a1};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) blk[r * 8 + c] = ((r >> 2) == (c >> 2)) ? T[(r & 3) * 4 + (c & 3)] : 0.f;
  }
};

struct LMScalar {
  static constexpr int GW = 2, NM = 4, AW = 1;
  using RK = ScalarKind<float>;
  static GC_DEV void ld_mom(const float* mom, int64_t moff, int b, float* m) {
    const float4 v = *reinterpret_cast<const float4*>(mom + mom_index(moff, b, 0, NM));
    m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
  }
  static GC_DEV void aux(const float* g, float* a) { a[0] = g[0] * g[0] + g[1] * g[1]; }
  static GC_DEV float diag_sum(const float* A) { return 2.f * A[0]; }
  static GC_DEV bool no_data(const float* A) { return !(A[0] > 0.f); }
  // side 0: c = g_o B, side 1: c = g_o conj(B); Hb = |g_o|^2 Q; J^H r = c - g_me Hb
  static GC_DEV void side(const float* m, const float* gme, const float* go, const float* ao, int sd, float* A,
                          float* gr, float* gc) {
    const Cx<float> B = cx<float>(m[0], sd ? -m[1] : m[1]);
    const Cx<float> c = mul_(cx<float>(go[0], go[1]), B);
    const float h = ao[0] * m[2];
    kahan_add(gr[0], gc[0], c.x - gme[0] * h);
    kahan_add(gr[1], gc[1], c.y - gme[1] * h);
    A[0] += h;
  }
  // d_s -> b conj(d_s), b = g_f g_s Q (eq. JHJ:DI B); the real 2x2 block is symmetric
  static GC_DEV void cross(const float* m, const float* gf, const float* gs, bool, float* blk) {
    const Cx<float> b = scale_(mul_(cx<float>(gf[0], gf[1]), cx<float>(gs[0], gs[1])), m[2]);
    blk[0] += b.x; blk[1] += b.y; blk[2] += b.y; blk[3] -= b.x;
  }
  static GC_DEV void diag(const float* A, float lam, float* blk) {
    blk[0] = A[0] * (1.f + lam); blk[1] = 0.f; blk[2] = 0.f; blk[3] = A[0] * (1.f + lam);
  }
};

// ------------------------------------------------------------------------------------------
// Shared-memory layout of one CTA (one interval at a time); NP = largest padded n, NA = NP / GW.
// ------------------------------------------------------------------------------------------
template <class T>
struct LMSmem {
  static __host__ __device__ size_t union_bytes(int NP) {
    const size_t panel = (size_t)kNB * NP * 4;
    const size_t pass1 = (size_t)kLMThreads * (4 * 4 + T::GW * 4);
    size_t u = panel > pass1 ? panel : pass1;
    u = u > (size_t)8 * 32 * 4 ? u : (size_t)8 * 32 * 4;
    return (u + 15) & ~(size_t)15;
  }
  static __host__ __device__ size_t bytes(int NP) {
    const int NA = NP / T::GW;
    return union_bytes(NP) + (size_t)NP * 4 /*rhs*/ + (size_t)NP * 4 /*gains*/ + (size_t)NA * 4 * 4 /*aux*/ +
           (size_t)NA * 4 * 4 /*A*/;
  }
};

GC_DEV void lm_pair_decode(int idx, int& P, int& Q) {
  int p = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
  while ((p + 1) * (p + 2) / 2 <= idx) ++p;
  while (p * (p + 1) / 2 > idx) --p;
  P = p;
  Q = idx - p * (p + 1) / 2;
}

// Rank-32 update of the trailing lower triangle: H[k0+32.., k0+32..] -= Lp Lp^T, Lp = panel rows
// 32..m-1 (in Ps, column-major [32][m]).  Warp-tiled: a warp takes one 32x32 block at a time from a
// shared counter (warps that arrive late -- warp 0 after its look-ahead -- take fewer), each lane an
// 8x4 tile (lanes 4 x 8), operands read from shared memory as float4; the next block's values are
// loaded while the current one is computed.  Blocks from 1 on (block 0 is the next diagonal block,
// which the look-ahead updates).  *next must be 0 before the first warp arrives.
GC_DEV void lm_syrk(float* H, int npad, int k0, int m, const float* Ps, int* next) {
  const int t = m - kNB;
  if (t <= 0) return;
  const int T = t / 32;
  const int nblk = T * (T + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int ly = lane >> 3, lx = lane & 7;
  const unsigned full = 0xffffffffu;
  auto grab = [&]() {
    int b = 0;
    if (lane == 0) b = 1 + atomicAdd(next, 1);
    return __shfl_sync(full, b, 0);
  };
  // block order: (1, 0), (2, 0), .. (T-1, 0) -- the next panel, which the next step loads first --
  // then the rest, (1, 1), (2, 1), (2, 2), ..
  auto decode = [&](int b, int& bi, int& bj) {
    if (b < T) { bi = b; bj = 0; return; }
    int p, q;
    lm_pair_decode(b - T, p, q);       // (bi - 1, bj - 1) over the lower triangle of T - 1 blocks
    bi = p + 1; bj = q + 1;
  };
  int bidx = grab();
  if (bidx >= nblk) return;
  int bi, bj;
  decode(bidx, bi, bj);
  float4 cv[8];
  {
    const int r0 = kNB + bi * 32 + ly * 8, c0 = kNB + bj * 32 + lx * 4;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
      cv[rr] = *reinterpret_cast<const float4*>(H + (int64_t)(k0 + r0 + rr) * npad + k0 + c0);
  }
  while (true) {
    const int r0 = kNB + bi * 32 + ly * 8;
    const int c0 = kNB + bj * 32 + lx * 4;
    float acc[8][4];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = 0.f;
#pragma unroll 4
    for (int c = 0; c < kNB; ++c) {
      const float* col = Ps + c * m;
      const float4 a0 = *reinterpret_cast<const float4*>(col + r0);
      const float4 a1 = *reinterpret_cast<const float4*>(col + r0 + 4);
      const float4 b = *reinterpret_cast<const float4*>(col + c0);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = fmaf(av[rr], bv[cc], acc[rr][cc]);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      float4 v = cv[rr];
      v.x -= acc[rr][0]; v.y -= acc[rr][1]; v.z -= acc[rr][2]; v.w -= acc[rr][3];
      *reinterpret_cast<float4*>(H + (int64_t)(k0 + r0 + rr) * npad + k0 + c0) = v;
    }
    bidx = grab();
    if (bidx >= nblk) break;
    decode(bidx, bi, bj);
    const int nr0 = kNB + bi * 32 + ly * 8, nc0 = kNB + bj * 32 + lx * 4;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
      cv[rr] = *reinterpret_cast<const float4*>(H + (int64_t)(k0 + nr0 + rr) * npad + k0 + nc0);
  }
}

// Factor of one 32 x 32 diagonal block, by one warp (lane r holds row r of the block in x): L_kk^-1
// in Linv ([t][c] = L_kk^-1[c][t]) and in H in place of the block (rows / columns k0.., row-major,
// zeros above the diagonal: only the inverse is needed afterwards), y_k = L_kk^-1 rhs_k in
// rhs[k0..] and yk.  *fail is set when a pivot is not positive.
GC_DEV void lm_diag_block(float (&x)[kNB], float* H, int npad, int k0, float* rhs, float* Linv, float* yk,
                          float* stage, int* fail) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  int bad = 0;
  float dl = 0.f;   // 1 / L[lane][lane] (kept apart: indexing x by the lane would move x to local memory)
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    const float piv = __shfl_sync(full, x[j], j);
    bad |= !(piv > 0.f);
    const float d = sqrtf(fmaxf(piv, 1e-30f)), inv = 1.f / d;
    if (lane == j) { x[j] = d; dl = inv; }
    if (lane > j) x[j] *= inv;
    const float lj = x[j];
#pragma unroll
    for (int c = 1; c < kNB; ++c) {
      if (c > j) {   // a fixed trip count keeps every index a compile-time constant after unrolling
        const float lc = __shfl_sync(full, x[j], c);
        if (lane >= c) x[c] = fmaf(-lj, lc, x[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c) stage[c * kNB + lane] = c <= lane ? x[c] : 0.f;
  __syncwarp();
  // row `lane` of L_kk^-1: row t is final once divided by L[t][t]; it then updates the rows below
  float w[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) w[c] = c == lane ? 1.f : 0.f;
#pragma unroll
  for (int t = 0; t < kNB; ++t) {
    if (lane == t) {
#pragma unroll
      for (int c = 0; c <= t; ++c) w[c] *= dl;
    }
    const float lrt = stage[t * kNB + lane];
#pragma unroll
    for (int c = 0; c <= t; ++c) {
      const float v = __shfl_sync(full, w[c], t);
      if (lane > t) w[c] = fmaf(-lrt, v, w[c]);
    }
  }
  const float tr = rhs[k0 + lane];
  float y = 0.f;
  float* row = H + (int64_t)(k0 + lane) * npad + k0;   // row `lane` of L_kk^-1 replaces L_kk in H
#pragma unroll
  for (int c = 0; c < kNB; c += 4)
    *reinterpret_cast<float4*>(row + c) = make_float4(c <= lane ? w[c] : 0.f, c + 1 <= lane ? w[c + 1] : 0.f,
                                                      c + 2 <= lane ? w[c + 2] : 0.f, c + 3 <= lane ? w[c + 3] : 0.f);
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    Linv[c * kNB + lane] = c <= lane ? w[c] : 0.f;
    y = fmaf(w[c], __shfl_sync(full, tr, c), y);
  }
  rhs[k0 + lane] = y;
  yk[lane] = y;
  if (lane == 0 && bad) *fail = 1;
}

// In-place blocked Cholesky H = L L^T (lower triangle of the row-major npad x npad matrix) with the
// forward substitution L y = rhs carried along (rhs holds y on return).  Per panel of 32 columns,
// its diagonal block already factored (L_kk^-1 in Linv, y_k in yk):
//   (a) the panel rows below the diagonal block into shared memory (Ps, column-major [32][m]);
//   (c) those rows solve x L_kk^T = a as the product x = a L_kk^-T (a warp-tiled 32-column GEMM,
//       no dependent chain per row) and update rhs_r -= x . y_k;
//   (d) the panel goes back to H;
//   (e) look-ahead: warp 0 applies the rank-32 update to the next diagonal block and factors it
//       (lm_diag_block) while the other warps apply it to the rest of the trailing matrix; warp 0
//       then takes its share of what remains.
// Returns 1 when a pivot is not positive (nothing more is computed then).  Linv, stage: 32 x 32
// floats of shared memory; yk: 32 floats.
GC_DEV int lm_cholesky_solve(float* H, int npad, float* rhs, float* Ps, float* Linv, float* yk, float* stage,
                             int* fail, int* next, unsigned long long* phase) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned full = 0xffffffffu;
  long long tc = phase ? clock64() : 0;
  if (warp == 0) {
    float x[kNB];
    const float* row = H + (int64_t)lane * npad;
#pragma unroll
    for (int c = 0; c < kNB; c += 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + c);
      x[c] = v.x; x[c + 1] = v.y; x[c + 2] = v.z; x[c + 3] = v.w;
    }
    lm_diag_block(x, H, npad, 0, rhs, Linv, yk, stage, fail);
  }
  __syncthreads();
  if (*fail) return 1;
  for (int k0 = 0; k0 < npad; k0 += kNB) {
    const int m = npad - k0;
    if (m == kNB) break;
    // (a) rows 32..m-1; a warp takes 32 consecutive rows of one 4-column group
    const int mr = m - kNB;
    for (int idx = tid; idx < mr * 8; idx += kLMThreads) {
      const int cg = idx / mr, r = kNB + idx - cg * mr;
      const float4 v = *reinterpret_cast<const float4*>(H + (int64_t)(k0 + r) * npad + k0 + 4 * cg);
      Ps[(4 * cg + 0) * m + r] = v.x;
      Ps[(4 * cg + 1) * m + r] = v.y;
      Ps[(4 * cg + 2) * m + r] = v.z;
      Ps[(4 * cg + 3) * m + r] = v.w;
    }
    __syncthreads();
    lm_mark(phase, 5, tc);
    // (c) warp w takes 32-row blocks of the rows below; lane (ly, lx) an 8 x 4 tile
    {
      const int ly = lane >> 3, lx = lane & 7;
      const int nbr = mr / 32;
      for (int bi = warp; bi < nbr; bi += kLMThreads / 32) {
        const int r0 = kNB + bi * 32 + ly * 8, c0 = lx * 4;
        float acc[8][4];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = 0.f;
#pragma unroll 4
        for (int t = 0; t < kNB; ++t) {
          const float4 a0 = *reinterpret_cast<const float4*>(Ps + t * m + r0);
          const float4 a1 = *reinterpret_cast<const float4*>(Ps + t * m + r0 + 4);
          const float4 b = *reinterpret_cast<const float4*>(Linv + t * kNB + c0);
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = fmaf(av[rr], bv[cc], acc[rr][cc]);
        }
        __syncwarp();   // every lane of the warp has read its 32 rows before any is overwritten
        float part[8];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          part[rr] = 0.f;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) part[rr] = fmaf(acc[rr][cc], yk[c0 + cc], part[rr]);
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          *reinterpret_cast<float4*>(Ps + (c0 + cc) * m + r0) =
              make_float4(acc[0][cc], acc[1][cc], acc[2][cc], acc[3][cc]);
          *reinterpret_cast<float4*>(Ps + (c0 + cc) * m + r0 + 4) =
              make_float4(acc[4][cc], acc[5][cc], acc[6][cc], acc[7][cc]);
        }
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
#pragma unroll
          for (int o = 1; o < 8; o <<= 1) part[rr] += __shfl_xor_sync(full, part[rr], o);
        }
        if (lx == 0) {
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) rhs[k0 + r0 + rr] -= part[rr];
        }
      }
    }
    __syncthreads();
    lm_mark(phase, 6, tc);
    // (d) the solved rows back to H (the back substitution reads them)
    for (int idx = tid; idx < mr * 8; idx += kLMThreads) {
      const int cg = idx / mr, r = kNB + idx - cg * mr;
      float4 v;
      v.x = Ps[(4 * cg + 0) * m + r];
      v.y = Ps[(4 * cg + 1) * m + r];
      v.z = Ps[(4 * cg + 2) * m + r];
      v.w = Ps[(4 * cg + 3) * m + r];
      *reinterpret_cast<float4*>(H + (int64_t)(k0 + r) * npad + k0 + 4 * cg) = v;
    }
    // (e) next diagonal block: rows / columns k0+32..k0+63 minus the panel's rank-32 update, then
    // its factor (warp 0); the rest of the trailing matrix by warps 1..
    if (warp == 0) {
      const int kn = k0 + kNB;
      float x[kNB];
      const float* row = H + (int64_t)(kn + lane) * npad + kn;
#pragma unroll
      for (int c = 0; c < kNB; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(row + c);
        x[c] = v.x; x[c + 1] = v.y; x[c + 2] = v.z; x[c + 3] = v.w;
      }
#pragma unroll 4
      for (int t = 0; t < kNB; ++t) {
        const float* col = Ps + t * m + kNB;
        const float a = col[lane];
#pragma unroll
        for (int c = 0; c < kNB; c += 4) {
          const float4 b = *reinterpret_cast<const float4*>(col + c);
          x[c] = fmaf(-a, b.x, x[c]); x[c + 1] = fmaf(-a, b.y, x[c + 1]);
          x[c + 2] = fmaf(-a, b.z, x[c + 2]); x[c + 3] = fmaf(-a, b.w, x[c + 3]);
        }
      }
      lm_diag_block(x, H, npad, kn, rhs, Linv, yk, stage, fail);
    }
    lm_syrk(H, npad, k0, m, Ps, next);
    __syncthreads();
    if (tid == 0) *next = 0;
    lm_mark(phase, 7, tc);
    if (*fail) return 1;
  }
  return 0;
}

GC_DEV void lm_cp16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// L^T x = y for the factor left in H by lm_cholesky_solve (each diagonal block holding L_kk^-1);
// rhs holds x on return.  Last block first: the slab of 32 rows below which x_k's contributions
// are removed, H[k0..k0+31][0..k0), is copied to shared memory (cp.async, into `slab`) while warp 0
// forms x_k = L_kk^-T b_k (lane r sums column r of L_kk^-1 against b); then every thread removes
// x_k from its right-hand sides above, rhs_c -= sum_i L[k0+i][c] x_i.  `slab` holds 32 x (npad - 32)
// floats.
GC_DEV void lm_back_substitute(const float* H, int npad, float* rhs, float* slab) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned full = 0xffffffffu;
  for (int k0 = npad - kNB; k0 >= 0; k0 -= kNB) {
    const int q4 = k0 / 4;   // float4 groups per slab row
    for (int idx = tid; idx < kNB * q4; idx += kLMThreads) {
      const int i = idx / q4, c4 = idx - i * q4;
      lm_cp16(slab + i * k0 + 4 * c4, H + (int64_t)(k0 + i) * npad + 4 * c4);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0) {
      float li[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c) li[c] = H[(int64_t)(k0 + c) * npad + k0 + lane];   // L_kk^-1[c][lane]
      const float b = rhs[k0 + lane];
      float x = 0.f;
#pragma unroll
      for (int c = 0; c < kNB; ++c) x = fmaf(li[c], __shfl_sync(full, b, c), x);
      rhs[k0 + lane] = x;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int c = tid; c < k0; c += kLMThreads) {
      float acc = 0.f;
#pragma unroll 8
      for (int i = 0; i < kNB; ++i) acc = fmaf(slab[i * k0 + c], rhs[k0 + i], acc);
      rhs[c] -= acc;
    }
    __syncthreads();
  }
}

// chi^2 of interval i at the gains in gs (shared memory): sum over its rows of the squared residual
// ||D - G_p M G_q^H||^2 (eq. cal:DI:pol / eq. cal:DI:tf), residuals in FP32, each thread's sum
// compensated, the block total in FP64; every thread returns it.  Computing the residuals from the
// rows keeps chi^2 free of the cancellation against sum |D|^2 that a moment-space form suffers:
// near convergence chi^2 is ~1e-6 of sum |D|^2, and the damping decision compares two such values.
template <class T>
GC_DEV double lm_chi(const LMArgs& a, int i, int bo, int nb, const float* gs, double* red) {
  using RK = typename T::RK;
  const int tid = threadIdx.x;
  const int64_t r0 = a.row_off[i];
  const int ns = a.n_samp[i];
  float sum = 0.f, comp = 0.f;
  for (int b = tid; b < nb; b += kLMThreads) {
    const typename RK::G gp = RK::ld_gain(gs + T::GW * a.ant1[bo + b]);
    const typename RK::G gq = RK::ld_gain(gs + T::GW * a.ant2[bo + b]);
#pragma unroll 4
    for (int smp = 0; smp < ns; ++smp)
      kahan_add(sum, comp, row_w(a.weights, r0 + (int64_t)smp * nb + b) *
                               RK::resid2(a.vis, a.model, r0 + (int64_t)smp * nb + b, gp, gq));
  }
  return block_sum((double)sum - (double)comp, red);
}

// Start of the polish: chi^2 at the current gains, lambda = lambda0, every interval that has data
// and finite gains on list 1.  One CTA per interval.
template <class T>
__global__ void __launch_bounds__(kLMThreads) lm_init_kernel(const LMArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  const int i = blockIdx.x, tid = threadIdx.x;
  const int4 inf = a.iinfo[i];
  const int4 tb = a.tinfo[inf.x];
  const int N = inf.y, nb = inf.w;
  const int st = a.status[i] & 15;
  if (st == GC_ST_NODATA || st == GC_ST_NONFINITE || nb == 0) return;
  float* gs = reinterpret_cast<float*>(smem);
  for (int e = tid; e < T::GW * N; e += kLMThreads) gs[e] = a.gains[(int64_t)inf.z * T::GW + e];
  __syncthreads();
  const double chi = lm_chi<T>(a, i, tb.z, nb, gs, red);
  if (tid == 0) {
    a.chi[i] = chi;
    a.lam[i] = a.lam0;
    a.status[i] = GC_ST_NOT_CONVERGED | (a.status[i] & GC_ST_SINGULAR_FLAG);
    if (a.iters[i] < a.max_iter) {
      const int at = atomicAdd(&a.cnt[1], 1);
      a.list[1 * a.n_int + at] = i;
    }
  }
}

// One LM iteration for every interval on list k % 3 (persistent CTAs, one interval at a time).
template <class T>
__global__ void __launch_bounds__(kLMThreads, 2) lm_iter_kernel(const LMArgs a, int NP) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ __align__(16) float Linv[kNB * kNB];
  __shared__ __align__(16) float stage[kNB * kNB];
  __shared__ __align__(16) float yk[kNB];
  __shared__ int s_i, s_fail, s_acc, s_next;
  const int tid = threadIdx.x;
  const int lin = a.k % 3, lout = (a.k + 1) % 3, lclr = (a.k + 2) % 3;
  if (blockIdx.x == 0 && tid == 0) { a.cnt[lclr] = 0; a.cnt[3 + lclr] = 0; }
  float* H = a.work + (int64_t)blockIdx.x * a.work_stride;
  const int NA = NP / T::GW;
  unsigned char* U = smem;
  float* rhs = reinterpret_cast<float*>(smem + LMSmem<T>::union_bytes(NP));
  float* gs = rhs + NP;
  float* auxs = gs + NP;
  float* As = auxs + 4 * NA;
  for (;;) {
    if (tid == 0) {
      const int idx = atomicAdd(&a.cnt[3 + lin], 1);
      s_i = idx < a.cnt[lin] ? a.list[lin * a.n_int + idx] : -1;
      s_fail = 0;
      s_next = 0;
    }
    __syncthreads();
    const int i = s_i;
    if (i < 0) break;
    long long tclk = a.phase ? clock64() : 0;
    auto mark = [&](int ph) {
      if (a.phase && threadIdx.x == 0) {
        const long long t = clock64();
        atomicAdd(a.phase + ph, (unsigned long long)(t - tclk));
        tclk = t;
      }
    };
    const int4 inf = a.iinfo[i];
    const int4 tb = a.tinfo[inf.x];
    const int N = inf.y, nb = inf.w, bo = tb.z, nat = tb.w;
    const int n = T::GW * N, npad = (n + kNB - 1) & ~(kNB - 1);
    const int64_t moff = a.mom_off[i];
    for (int e = tid; e < n; e += kLMThreads) gs[e] = a.gains[(int64_t)inf.z * T::GW + e];
    __syncthreads();
    for (int p = tid; p < N; p += kLMThreads) T::aux(gs + T::GW * p, auxs + 4 * p);
    __syncthreads();
    // ---- pass 1: per antenna (S threads each, fixed order) its block of J^H J and J^H R
    {
      const int S = N >= kLMThreads ? 1 : kLMThreads / N;
      float* pA = reinterpret_cast<float*>(U);
      float* pg = pA + (size_t)kLMThreads * 4;
      for (int t = tid; t < N * S; t += kLMThreads) {
        const int p = t / S, part = t - p * S;
        float A[4] = {0.f, 0.f, 0.f, 0.f};
        float g[T::GW], gc[T::GW];   // compensated sums of J^H R
#pragma unroll
        for (int c = 0; c < T::GW; ++c) { g[c] = 0.f; gc[c] = 0.f; }
        if (p < nat) {
          const int e0 = a.ant_off[tb.y + p], e1 = a.ant_off[tb.y + p + 1];
          float m[T::NM];
          for (int e = e0 + part; e < e1; e += S) {
            const int ent = a.ant_ent[e], b = ent >> 1, sd = ent & 1;
            const int o = sd ? a.ant1[bo + b] : a.ant2[bo + b];
            T::ld_mom(a.moments, moff, b, m);
            T::side(m, gs + T::GW * p, gs + T::GW * o, auxs + 4 * o, sd, A, g, gc);
          }
        }
        // N * S <= kLMThreads: slot t is this thread's own
#pragma unroll
        for (int c = 0; c < 4; ++c) pA[4 * t + c] = A[c];
#pragma unroll
        for (int c = 0; c < T::GW; ++c) pg[T::GW * t + c] = g[c] - gc[c];
      }
      __syncthreads();
      double dsum = 0.0, gn2 = 0.0;
      for (int p = tid; p < N; p += kLMThreads) {
        float A[4] = {0.f, 0.f, 0.f, 0.f};
        float g[T::GW], gc[T::GW];
#pragma unroll
        for (int c = 0; c < T::GW; ++c) { g[c] = 0.f; gc[c] = 0.f; }
        for (int part = 0; part < S; ++part) {
#pragma unroll
          for (int c = 0; c < 4; ++c) A[c] += pA[4 * (p * S + part) + c];
#pragma unroll
          for (int c = 0; c < T::GW; ++c) kahan_add(g[c], gc[c], pg[T::GW * (p * S + part) + c]);
        }
#pragma unroll
        for (int c = 0; c < T::GW; ++c) g[c] -= gc[c];
        const bool nd = T::no_data(A);
#pragma unroll
        for (int c = 0; c < 4; ++c) As[4 * p + c] = A[c];
#pragma unroll
        for (int c = 0; c < T::GW; ++c) {
          rhs[T::GW * p + c] = nd ? 0.f : (float)g[c];
          gn2 += (double)gs[T::GW * p + c] * gs[T::GW * p + c];
        }
        dsum += nd ? 0.0 : (double)T::diag_sum(A);
      }
      for (int r = n + tid; r < npad; r += kLMThreads) rhs[r] = 0.f;
      dsum = block_sum(dsum, red);
      gn2 = block_sum(gn2, red);
      const float mu = (float)(dsum / n);
      const double vnorm = gn2 > 0.0 ? 1.0 / sqrt(gn2) : 0.0;
      // project the right-hand side off the gauge direction v = i G / ||G||
      double vg = 0.0;
      for (int e = tid; e < n / 2; e += kLMThreads)
        vg += (-(double)gs[2 * e + 1] * rhs[2 * e] + (double)gs[2 * e] * rhs[2 * e + 1]) * vnorm;
      vg = block_sum(vg, red);
      bool finite = true;
      for (int e = tid; e < n / 2; e += kLMThreads) {
        rhs[2 * e] = (float)(rhs[2 * e] + (double)gs[2 * e + 1] * vnorm * vg);
        rhs[2 * e + 1] = (float)(rhs[2 * e + 1] - (double)gs[2 * e] * vnorm * vg);
        finite = finite && isfinite(rhs[2 * e]) && isfinite(rhs[2 * e + 1]);
      }
      if (!finite) s_fail = 2;
      mark(0);
      // ---- pass 2: the damped, gauge-fixed matrix, block (P, Q), P >= Q, one thread each
      const float lam = (float)a.lam[i];
      const float vs = (float)vnorm;
      const int nblk = N * (N + 1) / 2;
      constexpr int B2 = T::GW * T::GW;
      for (int idx = tid; idx < nblk; idx += kLMThreads) {
        int P, Q;
        lm_pair_decode(idx, P, Q);
        float blk[B2];
#pragma unroll
        for (int e = 0; e < B2; ++e) blk[e] = 0.f;
        if (P == Q) {
          if (T::no_data(As + 4 * P)) {
#pragma unroll
            for (int e = 0; e < T::GW; ++e) blk[e * T::GW + e] = 1.f;
          } else {
            T::diag(As + 4 * P, lam, blk);
          }
        } else if (P < nat) {
          const int tri = P * (P - 1) / 2 + Q;
          const int e0 = a.pair_off[tb.x + tri], e1 = a.pair_off[tb.x + tri + 1];
          float m[T::NM];
          for (int e = e0; e < e1; ++e) {
            const int ent = a.pair_ent[e], b = ent >> 1;
            const bool firstP = ent & 1;
            T::ld_mom(a.moments, moff, b, m);
            if (firstP) T::cross(m, gs + T::GW * P, gs + T::GW * Q, false, blk);
            else T::cross(m, gs + T::GW * Q, gs + T::GW * P, true, blk);
          }
        }
        // + mu v_P v_Q^T, v = i G / ||G||: per complex entry (re, im) -> (-im, re)
        float vP[T::GW], vQ[T::GW];
#pragma unroll
        for (int e = 0; e < T::GW / 2; ++e) {
          vP[2 * e] = -gs[T::GW * P + 2 * e + 1] * vs; vP[2 * e + 1] = gs[T::GW * P + 2 * e] * vs;
          vQ[2 * e] = -gs[T::GW * Q + 2 * e + 1] * vs; vQ[2 * e + 1] = gs[T::GW * Q + 2 * e] * vs;
        }
#pragma unroll
        for (int r = 0; r < T::GW; ++r)
#pragma unroll
          for (int c = 0; c < T::GW; ++c) blk[r * T::GW + c] = fmaf(mu * vP[r], vQ[c], blk[r * T::GW + c]);
#pragma unroll
        for (int r = 0; r < T::GW; ++r) {
          float* row = H + (int64_t)(T::GW * P + r) * npad + T::GW * Q;
          if (T::GW == 8) {
            *reinterpret_cast<float4*>(row) = make_float4(blk[r * T::GW], blk[r * T::GW + 1], blk[r * T::GW + 2],
                                                          blk[r * T::GW + 3]);
            *reinterpret_cast<float4*>(row + 4) = make_float4(blk[r * T::GW + 4], blk[r * T::GW + 5],
                                                              blk[r * T::GW + 6], blk[r * T::GW + 7]);
          } else {
            *reinterpret_cast<float2*>(row) = make_float2(blk[r * T::GW], blk[r * T::GW + 1]);
          }
        }
      }
      // padding rows: identity
      for (int e = tid; e < (npad - n) * npad; e += kLMThreads) {
        const int r = n + e / npad, c = e % npad;
        H[(int64_t)r * npad + c] = r == c ? 1.f : 0.f;
      }
      __syncthreads();
    }
    mark(1);
    // ---- factor and solve (skipped if the right-hand side is not finite)
    if (s_fail == 0)
      lm_cholesky_solve(H, npad, rhs, reinterpret_cast<float*>(U), Linv, yk, stage, &s_fail, &s_next, a.phase);
    __syncthreads();
    mark(2);
    if (s_fail == 0) lm_back_substitute(H, npad, rhs, reinterpret_cast<float*>(U));
    mark(3);
    // ---- trial gains, their chi^2 (FP64), the damping decision (App. C)
    double dx2 = 0.0, gn2 = 0.0;
    const bool solved = s_fail == 0;
    if (solved) {
      for (int e = tid; e < n; e += kLMThreads) {
        const float v = gs[e] + rhs[e];
        dx2 += (double)rhs[e] * rhs[e];
        gn2 += (double)v * v;
        gs[e] = v;
      }
    }
    dx2 = block_sum(dx2, red);
    gn2 = block_sum(gn2, red);
    double chi = 0.0;
    const bool finite = solved && isfinite(dx2) && isfinite(gn2);
    if (finite) chi = lm_chi<T>(a, i, bo, nb, gs, red);
    if (tid == 0) {
      const double chi0 = a.chi[i];
      double lam = a.lam[i];
      const bool acc = finite && chi < chi0;
      const bool small = finite && dx2 <= a.tol * a.tol * gn2;
      const int it = a.iters[i] + 1;
      a.iters[i] = it;
      if (acc) { a.chi[i] = chi; lam /= a.K; }
      else lam *= a.K;
      a.lam[i] = lam;
      const int keep = a.status[i] & GC_ST_SINGULAR_FLAG;
      bool done = true;
      if (s_fail == 2 || (solved && !finite)) a.status[i] = GC_ST_NONFINITE | keep;
      else if (small) a.status[i] = GC_ST_OK | keep;
      else if (it >= a.max_iter) a.status[i] = GC_ST_NOT_CONVERGED | keep;
      else done = false;
      if (!done) {
        const int at = atomicAdd(&a.cnt[lout], 1);
        a.list[lout * a.n_int + at] = i;
      }
      s_acc = acc;
      // algorithmic work of this interval's step: Cholesky n^3/3 flops, two triangular solves n^2 each
      if (a.flop && s_fail != 2) atomicAdd(a.flop, (double)n * n * n / 3.0 + 2.0 * (double)n * n);
    }
    __syncthreads();
    if (s_acc)
      for (int e = tid; e < n; e += kLMThreads) a.gains[(int64_t)inf.z * T::GW + e] = gs[e];
    __syncthreads();
    mark(4);
  }
}

// ------------------------------------------------------------------------------------------
// Host side: per-layout plan (tables, antenna and pair lists), the init launch and the iteration loop.
// ------------------------------------------------------------------------------------------
struct LMPlan {
  uint64_t key = 0;
  int n_int = 0, np_max = 0, n_lm = 0;
  void* dev = nullptr;
  size_t bytes = 0;
  const int4* iinfo = nullptr;
  const int4* tinfo = nullptr;
  const int32_t *pair_off = nullptr, *pair_ent = nullptr, *ant_off = nullptr, *ant_ent = nullptr;
};
static LMPlan g_lm_plan[2];

static int lm_build_plan(int kind, const gc_layout* L, LMPlan& P, cudaStream_t s) {
  const int GW = kind == 0 ? 2 : 8;
  const int n = L->n_intervals;
  std::map<std::pair<int, int>, int> tabs;
  std::vector<int4> iinfo(n), tinfo;
  std::vector<int32_t> pair_off, pair_ent, ant_off, ant_ent;
  int np_max = kNB;
  for (int i = 0; i < n; ++i) {
    const auto key = std::make_pair((int)L->bl_off[i], (int)L->n_bl[i]);
    auto f = tabs.find(key);
    int t;
    if (f != tabs.end()) {
      t = f->second;
    } else {
      t = (int)tinfo.size();
      tabs[key] = t;
      const int bo = key.first, nb = key.second;
      int nat = 0;
      for (int b = 0; b < nb; ++b) nat = std::max(nat, std::max(L->ant1[bo + b], L->ant2[bo + b]) + 1);
      tinfo.push_back(make_int4((int)pair_off.size(), (int)ant_off.size(), bo, nat));
      // antenna -> (baseline, side), baselines in increasing order
      std::vector<std::vector<int>> al(nat);
      for (int b = 0; b < nb; ++b) {
        al[L->ant1[bo + b]].push_back(2 * b);
        al[L->ant2[bo + b]].push_back(2 * b + 1);
      }
      for (int p = 0; p < nat; ++p) {
        ant_off.push_back((int)ant_ent.size());
        ant_ent.insert(ant_ent.end(), al[p].begin(), al[p].end());
      }
      ant_off.push_back((int)ant_ent.size());
      // unordered pair (P > Q) -> baselines
      const int npair = nat * (nat - 1) / 2;
      std::vector<std::vector<int>> pl(npair > 0 ? npair : 1);
      for (int b = 0; b < nb; ++b) {
        const int p = L->ant1[bo + b], q = L->ant2[bo + b];
        const int P = std::max(p, q), Q = std::min(p, q);
        pl[P * (P - 1) / 2 + Q].push_back(2 * b + (p == P ? 1 : 0));
      }
      for (int x = 0; x < npair; ++x) {
        pair_off.push_back((int)pair_ent.size());
        pair_ent.insert(pair_ent.end(), pl[x].begin(), pl[x].end());
      }
      pair_off.push_back((int)pair_ent.size());
    }
    iinfo[i] = make_int4(t, L->n_ant[i], L->gain_off[i], L->n_bl[i]);
    const int np = (GW * L->n_ant[i] + kNB - 1) / kNB * kNB;
    np_max = std::max(np_max, np);
  }
  if (pair_ent.empty()) pair_ent.push_back(0);
  if (ant_ent.empty()) ant_ent.push_back(0);
  if (tinfo.empty()) tinfo.push_back(make_int4(0, 0, 0, 0));
  auto al16 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_ii = 0, o_ti = o_ii + al16(iinfo.size() * 16), o_po = o_ti + al16(tinfo.size() * 16);
  const size_t o_pe = o_po + al16(pair_off.size() * 4), o_ao = o_pe + al16(pair_ent.size() * 4);
  const size_t o_ae = o_ao + al16(ant_off.size() * 4), total = o_ae + al16(ant_ent.size() * 4);
  std::vector<unsigned char> host(total, 0);
  memcpy(host.data() + o_ii, iinfo.data(), iinfo.size() * 16);
  memcpy(host.data() + o_ti, tinfo.data(), tinfo.size() * 16);
  memcpy(host.data() + o_po, pair_off.data(), pair_off.size() * 4);
  memcpy(host.data() + o_pe, pair_ent.data(), pair_ent.size() * 4);
  memcpy(host.data() + o_ao, ant_off.data(), ant_off.size() * 4);
  memcpy(host.data() + o_ae, ant_ent.data(), ant_ent.size() * 4);
  if (P.dev && P.bytes < total) { cudaFree(P.dev); P.dev = nullptr; P.bytes = 0; }
  if (!P.dev) {
    const cudaError_t e = cudaMalloc(&P.dev, total);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (LM plan)");
    P.bytes = total;
  }
  cudaError_t e = cudaMemcpyAsync(P.dev, host.data(), total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(e, "copy of the LM plan");
  unsigned char* d = static_cast<unsigned char*>(P.dev);
  P.iinfo = reinterpret_cast<const int4*>(d + o_ii);
  P.tinfo = reinterpret_cast<const int4*>(d + o_ti);
  P.pair_off = reinterpret_cast<const int32_t*>(d + o_po);
  P.pair_ent = reinterpret_cast<const int32_t*>(d + o_pe);
  P.ant_off = reinterpret_cast<const int32_t*>(d + o_ao);
  P.ant_ent = reinterpret_cast<const int32_t*>(d + o_ae);
  P.n_int = n;
  P.np_max = np_max;
  return GC_OK;
}

int lm_limit_ok(int kind, const gc_layout* L) {
  const int GW = kind == 0 ? 2 : 8;
  for (int i = 0; i < L->n_intervals; ++i)
    if (GW * L->n_ant[i] > GC_LM_MAX_UNKNOWNS) return 0;
  return 1;
}

struct LMProfile {
  double ms = 0.0, flop = 0.0;
  int64_t launches = 0;
  double phase[kLMPhases] = {};
};
static LMProfile g_lm_prof;

template <class T>
static int lm_launch_all(LMArgs& a, int n_int, int np_max, int max_lm, bool prof, cudaStream_t s) {
  const size_t ish = (size_t)np_max * 4;
  lm_init_kernel<T><<<n_int, kLMThreads, ish, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error(e, "lm_init_kernel");
  g_launches++;
  const size_t sh = LMSmem<T>::bytes(np_max);
  e = cudaFuncSetAttribute(lm_iter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute (lm_iter_kernel)");
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lm_iter_kernel<T>, kLMThreads, sh);
  if (e != cudaSuccess) return set_cuda_error(e, "occupancy (lm_iter_kernel)");
  if (per < 1) return GC_ERR_LIMIT;
  const int grid = std::min(n_int, per * nsm);
  void* w = nullptr;
  int rc = ws_get("lm_work", (size_t)grid * np_max * np_max * sizeof(float), &w);
  if (rc) return rc;
  a.work = static_cast<float*>(w);
  a.work_stride = (int64_t)np_max * np_max;
  int* flag = nullptr;
  if ((rc = pinned_flag(&flag))) return rc;
  std::vector<cudaEvent_t> ev;
  for (int k = 1; k <= max_lm; ++k) {
    a.k = k;
    if (prof) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      ev.push_back(e0);
      ev.push_back(e1);
      cudaEventRecord(e0, s);
    }
    lm_iter_kernel<T><<<grid, kLMThreads, sh, s>>>(a, np_max);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, "lm_iter_kernel");
    if (prof) cudaEventRecord(ev.back(), s);
    g_launches++;
    if (k % 4 == 0 || k == max_lm) {
      e = cudaMemcpyAsync(flag + 8, a.cnt + (k + 1) % 3, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return set_cuda_error(e, "LM active count");
      if (flag[8] <= 0) break;
    }
  }
  if (prof) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "LM profile");
    double ms = 0.0;
    for (size_t j = 0; j + 1 < ev.size(); j += 2) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[j], ev[j + 1]);
      ms += t;
      cudaEventDestroy(ev[j]);
      cudaEventDestroy(ev[j + 1]);
    }
    g_lm_prof.ms = ms;
    g_lm_prof.launches = (int64_t)(ev.size() / 2);
  }
  return GC_OK;
}

// The polish after the diagonal iterations: gains, iters and status are device arrays of the
// calling solver (iters already counts the diagonal iterations); ant1 / ant2 / mom_off are the
// device copies of the baseline tables and moment offsets of the calling solver's plan.
int lm_run(int kind, const gc_layout* L, const float* vis, const float* model, const int64_t* row_off,
           const int32_t* n_samp, const float* moments, const int64_t* mom_off, const int32_t* ant1,
           const int32_t* ant2, float* gains, int32_t* iters, int32_t* status, const gc_options* opt, void* stream,
           const float* weights) {
  cudaStream_t s = (cudaStream_t)stream;
  const int n = L->n_intervals;
  if (n == 0) return GC_OK;
  LMPlan& P = g_lm_plan[kind == 0 ? 0 : 1];
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t key = layout_hash(L, 0x4c4d0000ull + (uint64_t)kind) ^ ((uint64_t)dev << 40);
  if (P.key != key || P.n_int != n || !P.dev) {
    P.key = 0;
    int rc = lm_build_plan(kind, L, P, s);
    if (rc != GC_OK) return rc;
    P.key = key;
  }
  void* st = nullptr;
  int rc = ws_get("lm_state", 2 * sizeof(double) + kLMPhases * sizeof(unsigned long long) + (size_t)n * 2 * sizeof(double) +
                                  (size_t)(3 * n + 8) * sizeof(int32_t), &st);
  if (rc) return rc;
  LMArgs a{};
  a.vis = vis;
  a.model = model;
  a.weights = weights;
  a.row_off = row_off;
  a.n_samp = n_samp;
  a.moments = moments;
  a.mom_off = mom_off;
  a.gains = gains;
  a.ant1 = ant1;
  a.ant2 = ant2;
  a.iinfo = P.iinfo;
  a.tinfo = P.tinfo;
  a.pair_off = P.pair_off;
  a.pair_ent = P.pair_ent;
  a.ant_off = P.ant_off;
  a.ant_ent = P.ant_ent;
  // state: [flop counter, 2 doubles][phase counters][lambda n][chi n][lists 3n ints][counters 8 ints]
  double* flop_slot = static_cast<double*>(st);
  unsigned long long* phase_slot = reinterpret_cast<unsigned long long*>(flop_slot + 2);
  a.lam = reinterpret_cast<double*>(phase_slot + kLMPhases);
  a.chi = a.lam + n;
  a.list = reinterpret_cast<int32_t*>(a.chi + n);
  a.cnt = a.list + 3 * n;
  a.iters = iters;
  a.status = status;
  a.lam0 = opt->lm_lambda0 > 0.0 ? opt->lm_lambda0 : GC_LM_DEFAULT_LAMBDA0;
  a.K = opt->lm_K > 1.0 ? opt->lm_K : GC_LM_DEFAULT_K;
  a.tol = opt->tol;
  a.max_iter = opt->max_iter;
  a.n_int = n;
  cudaError_t e = cudaMemsetAsync(a.cnt, 0, 8 * sizeof(int32_t), s);
  if (e != cudaSuccess) return set_cuda_error(e, "LM counters");
  const bool prof = opt->profile != 0;
  g_lm_prof = LMProfile{};
  if (prof) {
    a.flop = flop_slot;
    a.phase = phase_slot;
    e = cudaMemsetAsync(a.flop, 0, sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.phase, 0, kLMPhases * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_cuda_error(e, "LM profile counter");
  }
  rc = kind == 0 ? lm_launch_all<LMScalar>(a, n, P.np_max, opt->max_iter, prof, s)
                 : lm_launch_all<LMJones>(a, n, P.np_max, opt->max_iter, prof, s);
  if (rc != GC_OK || !prof) return rc;
  unsigned long long ph[kLMPhases];
  e = cudaMemcpy(&g_lm_prof.flop, a.flop, sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ph, a.phase, sizeof(ph), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_cuda_error(e, "LM profile counter");
  for (int j = 0; j < kLMPhases; ++j) g_lm_prof.phase[j] = (double)ph[j];
  return GC_OK;
}

int lm_profile_phases(double* cycles, int n) {
  for (int j = 0; j < n && j < kLMPhases; ++j) cycles[j] = g_lm_prof.phase[j];
  return kLMPhases;
}

int lm_profile(double* ms, int64_t* launches, double* flop) {
  if (ms) *ms = g_lm_prof.ms;
  if (launches) *launches = g_lm_prof.launches;
  if (flop) *flop = g_lm_prof.flop;
  return GC_OK;
}

}  // namespace gc
