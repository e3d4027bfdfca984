// Direction-dependent 2x2 (fully polarized) gains, Sect. 4.4: polarized CohJones (each antenna's
// 2Nd x 2Nd system, eqs. JHJ:DD:pol / JHR:DD:pol with the antenna blocks only) and polarized
// AllJones (eq. update:DD:diag:pol, per antenna and direction, through the residuals).
//
// Moments.  Within an interval the gains do not depend on the sample, so every sum over samples
// the iterations need is an entry of one Hermitian matrix per baseline: the Gram matrix of the
// stacked row v_s = [D, M^(1), .., M^(Nd)] (each 2x2 row-major, K = 4 (Nd + 1) complex entries),
//     Gm[e1][e2] = sum_s conj(v_s[e1]) v_s[e2],
// kept as its upper triangle of 4x4 tiles (tile (r, c), r <= c: the entries of block r against
// block c; diagonal tiles whole).  With Y^(d) = M^(d) G_q^(d)H and the element indices of the
// row-major blocks,
//   stored row (p, q), antenna p (X = G_q^(c)H G_q^(d)):
//     [sum_s Y^(c) Y^(d)H][i][a] = sum_{j,b} Gm[(d, a, b)][(c, i, j)] X[j][b]
//     [sum_s D Y^(d)H][i][a]     = sum_{j,b} Gm[(d, a, b)][(D, i, j)] G_q^(d)[j][b]
//   conjugate row (q, p), antenna q (D_qp = D^H, M_qp = M^H, X' = G_p^(c)H G_p^(d)):
//     [sum_s Y^(c) Y^(d)H][i][a] = sum_{j,b} Gm[(c, j, i)][(d, b, a)] X'[j][b]
//     [sum_s D Y^(d)H][i][a]     = sum_{j,b} Gm[(D, j, i)][(d, b, a)] G_p^(d)[j][b].
// Per antenna these give the Hermitian H (2Nd x 2Nd, block (c, d) = sum Y^(c) Y^(d)H) and
// CD = [.. sum D Y^(d)H ..] (2 x 2Nd); the antenna's normal equations are X H = CD with
// X = [G^(1) .. G^(Nd)] (the 4Nd x 4Nd operator block of eq. JHJ:DD:pol is R_H, inverted as
// R_{H^-1}, App. B).  CohJones solves H X^H = CD^H (two right-hand sides, FP32 Cholesky with one
// float-float refinement step); AllJones forms the residual sums C = CD - X H in float-float and
// takes G^(d) += C^(d) H[d, d]^-1.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "dd.h"
#include "dd_common.cuh"

namespace gc {

constexpr int kPolBl = 4;      // baselines per moment CTA
constexpr int kPolSps = 4;     // samples per staging slot (one block barrier per slot)
constexpr int kPolNst = 3;     // staging slots (two in flight while one is read)
constexpr int kPolChain = 16;  // samples summed in plain FP32 before a compensated add

template <int ND>
struct PolShape {
  static constexpr int T = ND + 1;            // 2x2 blocks in the stacked row: D, M^(1) .. M^(Nd)
  static constexpr int NT = T * (T + 1) / 2;  // upper 4x4 tiles of the Gram matrix
  static constexpr int NO = NT * 16;          // complex moments per baseline
  static constexpr int MTHR = (kPolBl * NT + 31) / 32 * 32;  // moment CTA size
  static constexpr int NBH = ND * (ND + 1) / 2;              // upper 2x2 blocks of H
  static constexpr int NOUT = 4 * (NBH + ND);                // accumulated entries per antenna
  static constexpr int ITHR = NOUT > 256 ? (NOUT + 31) / 32 * 32 : 256;  // iteration CTA size
  static constexpr int LANES = ITHR / NOUT;                  // entry lanes per accumulated value
  static constexpr int N2 = 2 * ND;                          // order of H
  static constexpr int NU2 = N2 * (N2 + 1) / 2;              // packed upper triangle of H
};

// Complex offset of Gram entry (e1, e2) within a baseline's moments, and whether the stored value
// is its conjugate (e1 in a later block than e2: the mirror entry of the Hermitian matrix).
__host__ __device__ inline int pol_gram_off(int T, int e1, int e2, int* conj_flag) {
  int r = e1 >> 2, c = e2 >> 2, u = e1 & 3, v = e2 & 3;
  *conj_flag = 0;
  if (r > c) {
    const int t = r; r = c; c = t;
    const int w = u; u = v; v = w;
    *conj_flag = 1;
  }
  return (r * T - r * (r - 1) / 2 + (c - r)) * 16 + u * 4 + v;
}

__device__ __forceinline__ void pol_cp16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void pol_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void pol_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------------------------ moments
// One CTA per (interval, tile of kPolBl baselines); thread (baseline, Gram tile).  Rows arrive in
// shared memory by per-thread 16-byte asynchronous copies, kPolSps samples per slot and two slots
// ahead: for one sample the kPolBl baselines of a plane (vis, or model d) are 4 x 32 contiguous
// bytes.  Each thread multiplies the conjugated 4 entries of its tile's row block by the 4 of its
// column block (16 complex products per sample), sums kPolChain samples in FP32 and adds the chain
// into a compensated total.
template <int ND>
__global__ void __launch_bounds__(PolShape<ND>::MTHR) ddpol_moment_kernel(const DDArgs a) {
  using S = PolShape<ND>;
  constexpr int T = S::T, NT = S::NT, NO = S::NO;
  constexpr int CH = T * kPolBl * 2;  // 16-byte chunks per sample
  __shared__ __align__(16) float4 stage[kPolNst][kPolSps][T][kPolBl][2];
  const int it = blockIdx.x;
  if (it >= a.n_mitems) return;
  const int i = a.mitem_int[it], tile = a.mitem_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i];
  const int b0 = tile * kPolBl;
  const int nbt = min(kPolBl, nb - b0);
  const int tid = threadIdx.x;
  const int bl = tid / NT, tt = tid - (tid / NT) * NT;
  int tr = 0, tc = 0;
  upper_cd(T, tt, tr, tc);
  const bool live = bl < nbt;
  const int64_t r0 = a.row_off[i] + b0;
  const int nslots = (ns + kPolSps - 1) / kPolSps;
  auto issue = [&](int slot, int sbase) {
    for (int c = tid; c < kPolSps * CH; c += blockDim.x) {
      const int sj = c / CH, rem = c - sj * CH;
      const int pl = rem / (kPolBl * 2), rb = rem - pl * (kPolBl * 2);
      const int b = rb >> 1, h = rb & 1;
      const int s = sbase + sj;
      float4* dst = &stage[slot][sj][pl][b][h];
      if (s < ns && b < nbt) {
        const int64_t r = r0 + (int64_t)s * nb + b;
        const float* src = pl == 0 ? a.vis + 8 * r : a.model + 8 * ((int64_t)(pl - 1) * a.n_rows + r);
        pol_cp16(dst, src + 4 * h);
      } else {
        *dst = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    pol_commit();
  };
#pragma unroll
  for (int j = 0; j < kPolNst - 1; ++j) {
    if (j < nslots) issue(j, j * kPolSps);
    else pol_commit();
  }
  float ar[16], ai[16], tr_[16], ti_[16], cr[16], ci[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) ar[e] = ai[e] = tr_[e] = ti_[e] = cr[e] = ci[e] = 0.f;
  constexpr int SLOTS_PER_CHAIN = kPolChain / kPolSps;
  for (int j = 0; j < nslots; ++j) {
    pol_wait<kPolNst - 2>();
    __syncthreads();  // slot j is complete for every thread; slot j - 1 is free
    {
      const int nx = j + kPolNst - 1;
      if (nx < nslots) issue(nx % kPolNst, nx * kPolSps);
      else pol_commit();
    }
    if (live) {
      const int slot = j % kPolNst;
#pragma unroll
      for (int sj = 0; sj < kPolSps; ++sj) {
        const float4 u0 = stage[slot][sj][tr][bl][0], u1 = stage[slot][sj][tr][bl][1];
        const float4 w0 = stage[slot][sj][tc][bl][0], w1 = stage[slot][sj][tc][bl][1];
        const float ur[4] = {u0.x, u0.z, u1.x, u1.z}, ui[4] = {u0.y, u0.w, u1.y, u1.w};
        const float wr[4] = {w0.x, w0.z, w1.x, w1.z}, wi[4] = {w0.y, w0.w, w1.y, w1.w};
#pragma unroll
        for (int e1 = 0; e1 < 4; ++e1)
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {  // += conj(u) w
            const int e = e1 * 4 + e2;
            ar[e] = fmaf(ur[e1], wr[e2], fmaf(ui[e1], wi[e2], ar[e]));
            ai[e] = fmaf(ur[e1], wi[e2], fmaf(-ui[e1], wr[e2], ai[e]));
          }
      }
    }
    if ((j + 1) % SLOTS_PER_CHAIN == 0 || j + 1 == nslots) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        kahan_add(tr_[e], cr[e], ar[e]);
        kahan_add(ti_[e], ci[e], ai[e]);
        ar[e] = ai[e] = 0.f;
      }
    }
  }
  pol_wait<0>();
  if (live) {
    float2* out = reinterpret_cast<float2*>(a.moments) + a.mom_off[i] + (int64_t)(b0 + bl) * NO + tt * 16;
#pragma unroll
    for (int e = 0; e < 16; ++e) out[e] = make_float2(tr_[e] - cr[e], ti_[e] - ci[e]);
  }
}

// ------------------------------------------------------------------------------------ iteration
// Polarized AllJones update of one antenna, by one warp: lane m < 2Nd takes column m of the
// residual sums C = CD - X H (rows k = 0, 1; X = [G^(1) .. G^(Nd)] the antenna's current gains),
// formed in float-float against the float-float H and CD; then direction d = m / 2 solves its
// 2x2 block, G^(d) += C^(d) H[d, d]^-1, the two lanes of a direction exchanging their columns by
// shuffles.  A direction whose block is not positive definite keeps its gains and sets *sing.
// Hh/Hl: packed upper triangle of H (hi, lo); Ch/Cl: [2][2Nd] of CD (hi, lo); g: the antenna's
// gains [Nd][4]; x: the new gains [Nd][4].
template <int ND>
__device__ void ddpol_alljones_warp(const Cx<float>* Hh, const Cx<float>* Hl, const Cx<float>* Ch,
                                    const Cx<float>* Cl, const Cx<float>* g, Cx<float>* x, int* sing) {
  constexpr int N2 = 2 * ND;
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int m = lane < N2 ? lane : N2 - 1;
  auto au = [](int r, int c) { return r * N2 - r * (r - 1) / 2 + (c - r); };  // r <= c
  Cx<float> res[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    FF rx{Ch[k * N2 + m].x, Cl[k * N2 + m].x}, ry{Ch[k * N2 + m].y, Cl[k * N2 + m].y};
    float lox = 0.f, loy = 0.f;
#pragma unroll
    for (int n = 0; n < N2; ++n) {  // C[k][m] -= X[k][n] H[n][m]
      const int u = n <= m ? au(n, m) : au(m, n);
      Cx<float> h = Hh[u], lo = Hl[u];
      if (n > m) { h.y = -h.y; lo.y = -lo.y; }
      const Cx<float> xv = g[(n >> 1) * 4 + 2 * k + (n & 1)];
      rx = ff_sub_prod(rx, xv.x, h.x);
      rx = ff_sub_prod(rx, -xv.y, h.y);
      ry = ff_sub_prod(ry, xv.x, h.y);
      ry = ff_sub_prod(ry, xv.y, h.x);
      lox = fmaf(xv.x, lo.x, fmaf(-xv.y, lo.y, lox));
      loy = fmaf(xv.x, lo.y, fmaf(xv.y, lo.x, loy));
    }
    res[k] = cx<float>(rx.hi + (rx.lo - lox), ry.hi + (ry.lo - loy));
  }
  // direction d = m / 2, column a = m & 1; the partner lane holds the other column
  const int d = m >> 1, a = m & 1;
  Cx<float> oth[2];
#pragma unroll
  for (int k = 0; k < 2; ++k)
    oth[k] = cx<float>(__shfl_xor_sync(kAll, res[k].x, 1), __shfl_xor_sync(kAll, res[k].y, 1));
  const Cx<float> h00 = add_(Hh[au(2 * d, 2 * d)], Hl[au(2 * d, 2 * d)]);
  const Cx<float> h11 = add_(Hh[au(2 * d + 1, 2 * d + 1)], Hl[au(2 * d + 1, 2 * d + 1)]);
  const Cx<float> h01 = add_(Hh[au(2 * d, 2 * d + 1)], Hl[au(2 * d, 2 * d + 1)]);
  const float det = h00.x * h11.x - abs2_(h01);
  if (lane >= N2) return;
  if (!(det > 0.f) || !(h00.x > 0.f)) {
    x[d * 4 + 0 + a] = g[d * 4 + 0 + a];
    x[d * 4 + 2 + a] = g[d * 4 + 2 + a];
    atomicOr(sing, 1);
    return;
  }
  const float inv = 1.f / det;
  // Hd^-1 = [[h11, -h01], [-conj(h01), h00]] / det; column a of it
  const Cx<float> i0a = a == 0 ? cx<float>(h11.x * inv, 0.f) : scale_(h01, -inv);           // row 0
  const Cx<float> i1a = a == 0 ? scale_(conj_(h01), -inv) : cx<float>(h00.x * inv, 0.f);    // row 1
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const Cx<float> c0 = a == 0 ? res[k] : oth[k], c1 = a == 0 ? oth[k] : res[k];
    Cx<float> dl = mul_(c0, i0a);
    fma_(dl, c1, i1a);
    x[d * 4 + 2 * k + a] = add_(g[d * 4 + 2 * k + a], dl);
  }
}

// One CTA per (interval, antenna): the antenna's H (upper 2x2 blocks) and CD from the moments of
// its baselines, summed with compensation per thread and in float-float across lanes; then the
// CohJones solve (method 0) or the AllJones step (method 1) by one warp; the interval's last
// antenna applies the schedule and the convergence test.  Registers are capped for three CTAs per
// SM (80 per thread; the solver spills a little): unbounded, the kernel takes 121 and fits two,
// and the 744 CTAs of the 62-antenna 9-direction workload then need three rounds instead of two.
template <int ND>
__global__ void __launch_bounds__(PolShape<ND>::ITHR, 3) ddpol_iter_kernel(const DDArgs a) {
  using S = PolShape<ND>;
  constexpr int T = S::T, NO = S::NO, NBH = S::NBH, NOUT = S::NOUT, LANES = S::LANES, N2 = S::N2,
                NU2 = S::NU2, W = 4 * ND;
  constexpr int ITHR = S::ITHR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<float>* gs = reinterpret_cast<Cx<float>*>(smem_raw);        // [n_ant][ND][4]
  float4* red = reinterpret_cast<float4*>(gs + (size_t)a.na_max * W);  // [LANES][NOUT]
  __shared__ Cx<float> Hh[NU2], Hl[NU2], Ch[2 * N2], Cl[2 * N2], xs[W], rh[2 * N2], rl[2 * N2], xv[2 * N2];
  __shared__ Cx<float> Ls[N2 * N2];
  __shared__ int s_last, s_sing, s_nf;
  __shared__ double s_red[80];
  __shared__ int2 s_ent[ITHR];
  const int it = blockIdx.x;
  if (it >= a.n_iitems) return;
  const int i = a.iitem_int[it];
  const int k = *a.kbase + a.k;
  if (a.active[i] == 0 || k > a.max_iter) return;
  const int p = a.iitem_ant[it];
  const int na = a.n_ant[i];
  const int64_t go = a.gain_off[i];
  const int tid = threadIdx.x;
  for (int x = tid; x < na * W; x += blockDim.x)
    gs[x] = cx<float>(a.gains[2 * (go * W + x)], a.gains[2 * (go * W + x) + 1]);
  // this thread's accumulated value: block blk (H block (c, d) for blk < NBH, else CD block d),
  // element (ii, aa); Gram offsets of its 4 terms for each side
  const int comp = tid % NOUT, lane = tid / NOUT;
  const bool worker = lane < LANES;
  const int blk = comp >> 2, ii = (comp >> 1) & 1, aa = comp & 1;
  int c = 0, d = 0;
  const bool isH = blk < NBH;
  if (isH) upper_cd(ND, blk, c, d);
  else d = blk - NBH;
  int offp[4], offq[4], cjp[4], cjq[4];  // stored side (antenna = ant1) and conjugate side
#pragma unroll
  for (int jb = 0; jb < 4; ++jb) {
    const int j = jb >> 1, b = jb & 1;
    const int ep1 = 4 * (1 + d) + 2 * aa + b, ep2 = isH ? 4 * (1 + c) + 2 * ii + j : 2 * ii + j;
    const int eq1 = isH ? 4 * (1 + c) + 2 * j + ii : 2 * j + ii, eq2 = 4 * (1 + d) + 2 * b + aa;
    offp[jb] = pol_gram_off(T, ep1, ep2, &cjp[jb]);
    offq[jb] = pol_gram_off(T, eq1, eq2, &cjq[jb]);
  }
  float sx = 0.f, sxc = 0.f, sy = 0.f, syc = 0.f;
  const float2* mom = reinterpret_cast<const float2*>(a.moments) + a.mom_off[i];
  const int e0 = a.iitem_e0[it], e1 = a.iitem_e1[it];
  for (int base = e0; base < e1; base += ITHR) {
    const int n = min(ITHR, e1 - base);
    if (tid < n) s_ent[tid] = make_int2(a.ent[base + tid], a.entq[base + tid]);
    __syncthreads();
    if (worker) {
      constexpr int U = 4;
      for (int j0 = lane; j0 < n; j0 += U * LANES) {
        float2 v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = j0 + u * LANES;
          const int en = idx < n ? s_ent[idx].x : 0;
          const float2* mb = mom + (int64_t)(en >> 1) * NO;
          const bool side = en & 1;
#pragma unroll
          for (int jb = 0; jb < 4; ++jb) {
            v[u][jb] = idx < n ? mb[side ? offq[jb] : offp[jb]] : make_float2(0.f, 0.f);
            if (side ? cjq[jb] : cjp[jb]) v[u][jb].y = -v[u][jb].y;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = j0 + u * LANES;
          if (idx >= n) continue;
          const int q = s_ent[idx].y;
          const Cx<float>* gq = gs + (size_t)q * W;
          Cx<float> z[4];  // Z[j][b]
          if (isH) {       // X = G^(c)H G^(d) of the other antenna
#pragma unroll
            for (int jb = 0; jb < 4; ++jb) {
              const int j = jb >> 1, b = jb & 1;
              Cx<float> t = cmul_(gq[c * 4 + j], gq[d * 4 + b]);
              fma_(t, conj_(gq[c * 4 + 2 + j]), gq[d * 4 + 2 + b]);
              z[jb] = t;
            }
          } else {
#pragma unroll
            for (int jb = 0; jb < 4; ++jb) z[jb] = gq[d * 4 + jb];
          }
          Cx<float> t = mul_(cx<float>(v[u][0].x, v[u][0].y), z[0]);
#pragma unroll
          for (int jb = 1; jb < 4; ++jb) fma_(t, cx<float>(v[u][jb].x, v[u][jb].y), z[jb]);
          kahan_add(sx, sxc, t.x);
          kahan_add(sy, syc, t.y);
        }
      }
    }
    __syncthreads();  // before the next chunk replaces the staged entries
  }
  if (e1 <= e0) __syncthreads();  // the gains are staged even for an antenna without baselines
  if (worker) red[lane * NOUT + comp] = make_float4(sx, -sxc, sy, -syc);  // Kahan: the sum is s - c
  if (tid == 0) { s_nf = 0; s_sing = 0; }
  __syncthreads();
  for (int o = tid; o < NOUT; o += blockDim.x) {
    FF re{0.f, 0.f}, im{0.f, 0.f};
    for (int l = 0; l < LANES; ++l) {
      const float4 v = red[l * NOUT + o];
      re = ff_add(re, ff_two_sum(v.x, v.y));
      im = ff_add(im, ff_two_sum(v.z, v.w));
    }
    if (!isfinite(re.hi) || !isfinite(im.hi)) atomicOr(&s_nf, 1);  // sums overflowed: the gains diverged
    const int bk = o >> 2, i2 = (o >> 1) & 1, a2 = o & 1;
    if (bk < NBH) {  // H[2c + i2][2d + a2], upper triangle only
      int cc = 0, dd = 0;
      upper_cd(ND, bk, cc, dd);
      const int r = 2 * cc + i2, col = 2 * dd + a2;
      if (r <= col) {
        const int u = r * N2 - r * (r - 1) / 2 + (col - r);
        Hh[u] = cx<float>(re.hi, im.hi);
        Hl[u] = cx<float>(re.lo, im.lo);
      }
    } else {         // CD[k = i2][2d + a2]
      const int dd = bk - NBH;
      Ch[i2 * N2 + 2 * dd + a2] = cx<float>(re.hi, im.hi);
      Cl[i2 * N2 + 2 * dd + a2] = cx<float>(re.lo, im.lo);
    }
  }
  __syncthreads();
  if (a.method == 1) {
    if (tid < 32) ddpol_alljones_warp<ND>(Hh, Hl, Ch, Cl, gs + (size_t)p * W, xs, &s_sing);
  } else if (tid < 32) {
    // CohJones: H X^H = CD^H, one right-hand side per row k of X, one FP32 factorisation
    for (int u = tid; u < 2 * N2; u += 32) {
      rh[u] = conj_(Ch[u]);
      rl[u] = conj_(Cl[u]);
    }
    __syncwarp();
    bool ok = chol_solve_warp_mixed<N2, 2>(Hh, Hl, rh, rl, xv, Ls);
    for (int kk = 0; kk < 2 && !ok; ++kk) {  // rare: not positive definite in FP32; FP64 decides
      __shared__ double2 Ad[NU2], bd[N2], xd[N2], Am[N2 * N2];
      __shared__ double dinv[N2];
      __shared__ int s_ok;
      for (int u = tid; u < NU2; u += 32)
        Ad[u] = make_double2((double)Hh[u].x + (double)Hl[u].x, (double)Hh[u].y + (double)Hl[u].y);
      for (int r = tid; r < N2; r += 32)
        bd[r] = make_double2((double)rh[kk * N2 + r].x + (double)rl[kk * N2 + r].x,
                             (double)rh[kk * N2 + r].y + (double)rl[kk * N2 + r].y);
      __syncwarp();
      const bool ok64 = chol_solve_warp<N2>(Ad, bd, xd, Am, dinv, &s_ok);
      for (int r = tid; r < N2; r += 32) xv[kk * N2 + r] = cx<float>((float)xd[r].x, (float)xd[r].y);
      __syncwarp();
      if (!ok64) { if (tid == 0) s_sing = 1; break; }
      if (kk == 1) ok = true;
    }
    if (ok)
      for (int u = tid; u < 2 * N2; u += 32) {
        const int kk = u / N2, r = u - kk * N2;
        xs[(r >> 1) * 4 + 2 * kk + (r & 1)] = conj_(xv[u]);
      }
    __syncwarp();
  }
  __syncthreads();
  for (int x = tid; x < W; x += blockDim.x) {
    Cx<float> g = (s_sing && a.method != 1) ? gs[(size_t)p * W + x] : xs[x];
    if (s_nf) g = cx<float>(__int_as_float(0x7fc00000), 0.f);  // reported as non-finite gains
    a.gnew[2 * ((go + p) * W + x)] = g.x;
    a.gnew[2 * ((go + p) * W + x) + 1] = g.y;
  }
  if (tid == 0) a.sing[go + p] = s_sing;
  // the last antenna of the interval to finish applies the schedule and the convergence test
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&a.counters[i], 1) == na - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  dd_interval_update(a, i, k, na, go, W, gs, reinterpret_cast<float*>(s_red));
}

// chi^2 per moment item (interval, kPolBl baselines) over all its rows, then per interval:
// sum ||D - sum_d G_p^(d) M^(d) G_q^(d)H||_F^2, compensated per thread, FP64 across threads.
template <int ND>
__global__ void __launch_bounds__(256) ddpol_chi2_kernel(const DDArgs a, double* item_chi2) {
  __shared__ double red[64];
  const int it = blockIdx.x;
  if (it >= a.n_mitems) return;
  const int i = a.mitem_int[it], tile = a.mitem_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i], bo = a.bl_off[i];
  const int64_t go = a.gain_off[i];
  const int nbt = min(kPolBl, nb - tile * kPolBl);
  auto ldg = [&](int ant, int d) {
    const float* g = a.gains + 8 * ((go + ant) * ND + d);
    M2<float> m;
    m.a = cx<float>(g[0], g[1]); m.b = cx<float>(g[2], g[3]);
    m.c = cx<float>(g[4], g[5]); m.d = cx<float>(g[6], g[7]);
    return m;
  };
  float s = 0.f, c = 0.f;
  for (int u = threadIdx.x; u < nbt * ns; u += blockDim.x) {
    const int sl = u / nbt, bl = u - sl * nbt;
    const int b = tile * kPolBl + bl;
    const int p = a.ant1[bo + b], q = a.ant2[bo + b];
    const int64_t r = a.row_off[i] + (int64_t)sl * nb + b;
    M2<float> R = Vec<float>::ld4(a.vis + 8 * r);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const M2<float> M = Vec<float>::ld4(a.model + 8 * ((int64_t)d * a.n_rows + r));
      const M2<float> V = mmh_(mm_(ldg(p, d), M), ldg(q, d));
      R.a = sub_(R.a, V.a); R.b = sub_(R.b, V.b); R.c = sub_(R.c, V.c); R.d = sub_(R.d, V.d);
    }
    kahan_add(s, c, abs2_(R.a) + abs2_(R.b) + abs2_(R.c) + abs2_(R.d));
  }
  const double tot = block_sum<double>((double)s - (double)c, red);
  if (threadIdx.x == 0) item_chi2[it] = tot;
}

static __global__ void ddpol_chi2_final(const int32_t* first, const int32_t* count, const double* item_chi2,
                                        double* out, int n_int) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  double s = 0.0;
  for (int j = 0; j < count[i]; ++j) s += item_chi2[first[i] + j];
  out[i] = s;
}

// ------------------------------------------------------------------------------------ host side
static DDPlan g_ddpol;

template <int ND>
static int ddpol_run_nd(DDPlan& P, const gc_options* opt, cudaStream_t s, int* flag, double* prof_ms) {
  using S = PolShape<ND>;
  DDArgs& a = P.args;
  const size_t ismem = (size_t)a.na_max * 4 * ND * sizeof(Cx<float>) + (size_t)S::LANES * S::NOUT * sizeof(float4) + 16;
  DD_CUDA(cudaFuncSetAttribute(ddpol_iter_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
  dd_init_kernel<<<(P.n_int + 255) / 256, 256, 0, s>>>(a, P.n_int, P.n_active0);
  g_launches++;
  const char* ce = getenv("GAINCAL_CHECK_EVERY");
  const int SEG = ce && atoi(ce) > 0 ? atoi(ce) : 8;
  DDTimer mt(opt->profile != 0, 1), it(opt->profile != 0, 1);
  if (a.n_mitems > 0) {
    mt.before(s);
    ddpol_moment_kernel<ND><<<a.n_mitems, S::MTHR, 0, s>>>(a);
    mt.after(s);
    g_launches++;
  }
  DD_CUDA(cudaGetLastError());
  if (a.n_iitems > 0) {
    // iteration segments of SEG launches captured once per argument set (as for the scalar DD path)
    DDArgs ga = a;
    ga.k = 0;
    ga.vis = ga.model = nullptr;
    if (!P.gexec || P.gS != SEG || P.gnd != ND || memcmp(&P.gargs, &ga, sizeof(DDArgs)) != 0) {
      if (P.gexec) { cudaGraphExecDestroy(P.gexec); P.gexec = nullptr; }
      cudaStream_t cs = nullptr;
      DD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaError_t ce2 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      int crc = ce2 == cudaSuccess ? 0 : (int)ce2;
      for (int j = 1; j <= SEG && !crc; ++j) {
        DDArgs x = ga;
        x.k = j;
        ddpol_iter_kernel<ND><<<a.n_iitems, S::ITHR, ismem, cs>>>(x);
        crc = (int)cudaGetLastError();
      }
      if (!crc) crc = di_launch_advance(a.kbase, SEG, cs);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = ce2 == cudaSuccess ? cudaStreamEndCapture(cs, &g) : ce2;
      cudaStreamDestroy(cs);
      cudaError_t ie = cudaSuccess;
      if (!crc && ee == cudaSuccess) ie = cudaGraphInstantiate(&P.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (crc || ee != cudaSuccess || ie != cudaSuccess) {
        if (P.gexec) { cudaGraphExecDestroy(P.gexec); P.gexec = nullptr; }
        return set_cuda_error(crc ? (cudaError_t)crc : (ee != cudaSuccess ? ee : ie),
                              "capture of the polarized DD iteration segment");
      }
      P.gargs = ga;
      P.gS = SEG;
      P.gnd = ND;
    }
    for (int k0 = 0; k0 < opt->max_iter; k0 += SEG) {
      it.before(s);
      DD_CUDA(cudaGraphLaunch(P.gexec, s));
      it.after(s);
      g_launches += SEG + 1;
      DD_CUDA(cudaMemcpyAsync(flag, a.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      DD_CUDA(cudaStreamSynchronize(s));
      if (it.on) it.drain();
      if (*flag <= 0) break;
    }
  }
  if (opt->profile) {
    DD_CUDA(cudaStreamSynchronize(s));
    it.drain();
    mt.drain();
    prof_ms[0] = it.ms;
    prof_ms[1] = (double)it.launches * SEG;
    prof_ms[2] = mt.ms;
  }
  if (opt->compute_chi2 && a.n_mitems > 0) {
    ddpol_chi2_kernel<ND><<<a.n_mitems, 256, 0, s>>>(a, P.chi2_items);
    ddpol_chi2_final<<<(P.n_int + 255) / 256, 256, 0, s>>>(P.chi2_first, P.chi2_count, P.chi2_items, P.chi2_out,
                                                           P.n_int);
    g_launches += 2;
    DD_CUDA(cudaGetLastError());
  }
  return GC_OK;
}

void ddpol_release() {
  if (g_ddpol.gexec) cudaGraphExecDestroy(g_ddpol.gexec);
  if (g_ddpol.dev) cudaFree(g_ddpol.dev);
  g_ddpol = DDPlan{};
}

static int run_ddpol(const void* vis, const void* model, const gc_layout* L, void* gains, const gc_options* opt,
                     int32_t* iters_out, double* chi2_out, int32_t* status_out, void* stream, int method) {
  if (!opt || !L) return GC_ERR_ARG;
  if (opt->dtype != GC_DTYPE_C64) return GC_ERR_DTYPE;
  if (opt->max_iter < 1 || !(opt->tol >= 0.0) || (opt->schedule != GC_SCHED_STEFCAL && opt->schedule != GC_SCHED_GN))
    return GC_ERR_ARG;
  if ((opt->host_buffers != 0 && opt->host_buffers != 1) || opt->reserved || opt->weights) return GC_ERR_ARG;
  int rc = validate_layout(L, GC_MAX_DIR);
  if (rc != GC_OK) return rc;
  if (L->n_intervals == 0) return GC_OK;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && !gains)) return GC_ERR_ARG;
  // rows are copied in 16-byte units
  if (!opt->host_buffers && ((reinterpret_cast<uintptr_t>(vis) | reinterpret_cast<uintptr_t>(model)) & 15))
    return GC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  const int nd = L->n_dir;
  const int T = nd + 1;
  const int64_t NO = (int64_t)T * (T + 1) / 2 * 16;
  const uint64_t key = layout_hash(L, 0xDD2ull ^ ((uint64_t)dev << 40));
  if (g_ddpol.key != key || !g_ddpol.dev) {
    g_ddpol.key = 0;
    if ((rc = build_dd_plan(L, g_ddpol, s, NO, kPolBl))) return rc;
    g_ddpol.key = key;
  }
  DDPlan& P = g_ddpol;
  const size_t vb = (size_t)L->n_rows * 32, mb = (size_t)L->n_rows * nd * 32, gb = (size_t)L->n_gain * nd * 32;
  DDArgs& a = P.args;
  void* dg = nullptr;
  if ((rc = ws_get("ddpol_gains", gb > 0 ? gb : 8, &dg))) return rc;
  if (opt->host_buffers) {
    void *dv, *dm;
    if ((rc = ws_get("ddpol_h_vis", vb, &dv)) || (rc = ws_get("ddpol_h_model", mb, &dm))) return rc;
    if (vb) DD_CUDA(cudaMemcpyAsync(dv, vis, vb, cudaMemcpyHostToDevice, s));
    if (mb) DD_CUDA(cudaMemcpyAsync(dm, model, mb, cudaMemcpyHostToDevice, s));
    a.vis = (const float*)dv; a.model = (const float*)dm;
  } else {
    a.vis = (const float*)vis; a.model = (const float*)model;
  }
  if (gb)
    DD_CUDA(cudaMemcpyAsync(dg, gains, gb, opt->host_buffers ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  a.gains = (float*)dg;
  void *mom, *gnew;
  if ((rc = ws_get("ddpol_moments", (size_t)(P.n_mom > 0 ? P.n_mom : 1) * sizeof(float2), &mom))) return rc;
  if ((rc = ws_get("ddpol_gnew", gb > 0 ? gb : 8, &gnew))) return rc;
  a.moments = (float2*)mom;
  a.gnew = (float*)gnew;
  a.tol = opt->tol;
  a.max_iter = opt->max_iter;
  a.schedule = opt->schedule;
  a.method = method;
  int* flag = nullptr;
  if ((rc = pinned_flag(&flag))) return rc;
  double prof[3] = {0.0, 0.0, 0.0};
  switch (nd) {
    case 1: rc = ddpol_run_nd<1>(P, opt, s, flag, prof); break;
    case 2: rc = ddpol_run_nd<2>(P, opt, s, flag, prof); break;
    case 3: rc = ddpol_run_nd<3>(P, opt, s, flag, prof); break;
    case 4: rc = ddpol_run_nd<4>(P, opt, s, flag, prof); break;
    case 5: rc = ddpol_run_nd<5>(P, opt, s, flag, prof); break;
    case 6: rc = ddpol_run_nd<6>(P, opt, s, flag, prof); break;
    case 7: rc = ddpol_run_nd<7>(P, opt, s, flag, prof); break;
    case 8: rc = ddpol_run_nd<8>(P, opt, s, flag, prof); break;
    case 9: rc = ddpol_run_nd<9>(P, opt, s, flag, prof); break;
    case 10: rc = ddpol_run_nd<10>(P, opt, s, flag, prof); break;
    default: return GC_ERR_LIMIT;
  }
  if (rc) return rc;
  const cudaMemcpyKind dk = opt->host_buffers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (gb) DD_CUDA(cudaMemcpyAsync(gains, a.gains, gb, dk, s));
  if (iters_out) DD_CUDA(cudaMemcpyAsync(iters_out, a.iters, (size_t)P.n_int * 4, dk, s));
  if (status_out) DD_CUDA(cudaMemcpyAsync(status_out, a.status, (size_t)P.n_int * 4, dk, s));
  if (chi2_out && opt->compute_chi2) DD_CUDA(cudaMemcpyAsync(chi2_out, P.chi2_out, (size_t)P.n_int * 8, dk, s));
  std::vector<int32_t> stv(P.n_int), itv(P.n_int);
  DD_CUDA(cudaMemcpyAsync(stv.data(), a.status, (size_t)P.n_int * 4, cudaMemcpyDeviceToHost, s));
  if (opt->profile) DD_CUDA(cudaMemcpyAsync(itv.data(), a.iters, (size_t)P.n_int * 4, cudaMemcpyDeviceToHost, s));
  DD_CUDA(cudaStreamSynchronize(s));
  int bad = 0;
  for (int i = 0; i < P.n_int; ++i) bad += (stv[i] & 15) != GC_ST_OK;
  if (opt->profile) {
    int64_t ri = 0, bi = 0;
    for (int i = 0; i < P.n_int; ++i) {
      ri += (int64_t)itv[i] * L->n_samp[i] * L->n_bl[i];
      bi += (int64_t)itv[i] * L->n_bl[i];
    }
    profile_record(prof[0], (int64_t)prof[1], ri, prof[2], bi, GC_PATH_MOMENTS);
  }
  return bad;
}

}  // namespace gc

extern "C" int gc_calibrate_dd_cohjones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                           const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                           int32_t* status_out, void* stream) {
  return gc::run_ddpol(vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream, 0);
}
extern "C" int gc_calibrate_dd_alljones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                           const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                           int32_t* status_out, void* stream) {
  return gc::run_ddpol(vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream, 1);
}
