// Direction-dependent scalar gains: CohJones (Sect. 3.2.2) on the GPU.
//
// Per solution interval the sums over samples are taken once (moment pass), because the gains
// are constant over an interval and factor out of the sample sum (Sect. 3.2.1, the
// non-orthogonality terms X^(cd)):
//     X^(cd)_pq = sum_s conj(m^(c)_pqs) m^(d)_pqs        (Hermitian in (c, d); upper triangle kept)
//     B^(c)_pq  = sum_s conj(m^(c)_pqs) d_pqs
// Each iteration then forms, per antenna p, the N_d x N_d block and right-hand side of
// eqs. JHJ:DD:unpol / JHR:DD:unpol (data form, eq. ghat):
//     stored row (p, q):   A_p[c][d] += g_q^(c) conj(g_q^(d)) X^(cd)_pq,   b_p[c] += g_q^(c) B^(c)_pq
//     conjugate row (q, p): A_q[c][d] += g_p^(c) conj(g_p^(d)) conj(X^(cd)_pq), b_q[c] += g_p^(c) conj(B^(c)_pq)
// and solves A_p g_p = b_p by an FP64 Cholesky factorisation (the GN step with the antenna-block
// approximation of J^H J).  Odd iterations take the GN gains, even ones average them with the
// current gains (the approximate LM analogue of Sect. 3.2.2).  A streaming pass computes
// chi^2 = sum |d - sum_d g_p^(d) m^(d) conj(g_q^(d))|^2 at the end.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "dd.h"
#include "dd_common.cuh"

namespace gc {

constexpr int kMomBl = 32;      // baselines per moment CTA
constexpr int kMomLanes = 8;    // sample lanes per baseline in the moment CTA

template <int ND>
struct DDShape {
  static constexpr int NU = ND * (ND + 1) / 2;  // upper-triangle entries of X
  static constexpr int NO = NU + ND;            // moments per baseline
};

// ------------------------------------------------------------------------------------ moments
// Rows reach shared memory by cp.async, NST samples ahead of the arithmetic, so that the bytes in
// flight per SM do not depend on registers (the N_d = 9 accumulators already take most of them).
// Each thread reads back only the elements it copied itself, so a wait on its own copy groups is
// enough; the staging area is reused for the lane partials after the sample loop.
template <int ND>
struct DDMomStages {
  static constexpr int R = DDShape<ND>::NO / (ND + 1);  // stages that fit where the partials go
  static constexpr int N = R < 3 ? 3 : (R > 6 ? 6 : R);
};

__device__ __forceinline__ void dd_cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void dd_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void dd_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int ND>
constexpr size_t dd_moment_smem() {
  constexpr size_t part = (size_t)kMomLanes * kMomBl * DDShape<ND>::NO * sizeof(float2);
  constexpr size_t stage = (size_t)DDMomStages<ND>::N * (ND + 1) * kMomLanes * kMomBl * sizeof(float2);
  return part > stage ? part : stage;
}

template <int ND>
__global__ void __launch_bounds__(kMomBl * kMomLanes) dd_moment_kernel(const DDArgs a) {
  constexpr int NU = DDShape<ND>::NU, NO = DDShape<ND>::NO;
  constexpr int NST = DDMomStages<ND>::N, NP = ND + 1, NT = kMomBl * kMomLanes;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* part = reinterpret_cast<float2*>(smem_raw);   // [lanes][kMomBl][NO], after the sample loop
  float2* stage = reinterpret_cast<float2*>(smem_raw);  // [NST][NP][NT], during it
  const int it = blockIdx.x;
  if (it >= a.n_mitems) return;
  const int i = a.mitem_int[it];
  const int tile = a.mitem_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i];
  const int tid = threadIdx.x;
  const int bl = tid % kMomBl, lane = tid / kMomBl;
  const int b = tile * kMomBl + bl;
  const int chunk = (ns + kMomLanes - 1) / kMomLanes;
  const int s0 = lane * chunk, s1 = min(ns, s0 + chunk);
  Cx<float> X[NU], Bv[ND];
#pragma unroll
  for (int u = 0; u < NU; ++u) X[u] = cx<float>(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < ND; ++c) Bv[c] = cx<float>(0.f, 0.f);
  if (b < nb && s1 > s0) {
    const int64_t r0 = a.row_off[i] + b;
    const int cnt = s1 - s0;
    // sample j of this thread's chunk goes to stage slot j % NST: plane 0 is vis, plane 1 + c model c
    auto issue = [&](int j, int slot) {
      if (j < cnt) {
        const int64_t r = r0 + (int64_t)(s0 + j) * nb;
        float2* st = stage + (size_t)slot * NP * NT + tid;
        dd_cp_async8(st, a.vis + 2 * r);
#pragma unroll
        for (int c = 0; c < ND; ++c) dd_cp_async8(st + (c + 1) * NT, a.model + 2 * ((int64_t)c * a.n_rows + r));
      }
      dd_cp_commit();
    };
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) issue(j, j);
    int slot = 0;
    for (int j = 0; j < cnt; ++j) {
      // refill the slot read in the previous step (by this thread only) with sample j + NST - 1
      issue(j + NST - 1, slot == 0 ? NST - 1 : slot - 1);
      dd_cp_wait<NST - 1>();
      const float2* st = stage + (size_t)slot * NP * NT + tid;
      const Cx<float> d = cx<float>(st[0].x, st[0].y);
      Cx<float> m[ND];
#pragma unroll
      for (int c = 0; c < ND; ++c) m[c] = cx<float>(st[(c + 1) * NT].x, st[(c + 1) * NT].y);
      int u = 0;
#pragma unroll
      for (int c = 0; c < ND; ++c) {
#pragma unroll
        for (int e = c; e < ND; ++e) { cfma_(X[u], m[c], m[e]); ++u; }
        cfma_(Bv[c], m[c], d);
      }
      slot = slot + 1 == NST ? 0 : slot + 1;
    }
    dd_cp_wait<0>();
  }
  __syncthreads();  // every thread is done with the staging area
  float2* my = part + ((size_t)lane * kMomBl + bl) * NO;
#pragma unroll
  for (int u = 0; u < NU; ++u) my[u] = make_float2(X[u].x, X[u].y);
#pragma unroll
  for (int c = 0; c < ND; ++c) my[NU + c] = make_float2(Bv[c].x, Bv[c].y);
  __syncthreads();
  // compensated sum over the sample lanes, in lane order
  const int nbt = min(kMomBl, nb - tile * kMomBl);
  float2* out = a.moments + a.mom_off[i] + (int64_t)tile * kMomBl * NO;
  for (int x = threadIdx.x; x < nbt * NO; x += blockDim.x) {
    float sx = 0.f, cxs = 0.f, sy = 0.f, cys = 0.f;
    for (int l = 0; l < kMomLanes; ++l) {
      const float2 v = part[(size_t)l * kMomBl * NO + x];
      kahan_add(sx, cxs, v.x);
      kahan_add(sy, cys, v.y);
    }
    out[x] = make_float2(sx - cxs, sy - cys);
  }
}

// AllJones (Sect. 3.2.3, eq. stefcal:dd:unpol): J^H J taken as its diagonal, so the step goes
// through the residuals.  For antenna p, c_p[r] = sum conj(y^(r)) r equals b_p[r] - sum_j A_p[r][j]
// g_p^(j) exactly (the residual r = d - sum_j g_p^(j) y^(j) summed against conj(y^(r))), with A_p,
// b_p the CohJones block and data sums built from the moments; g_p^(r) += c_p[r] / A_p[r][r].
// c is formed in float-float against the float-float A and b (as the CohJones refinement
// residual).  One warp, lane r takes direction r; a direction with A_p[r][r] <= 0 (no signal)
// keeps its gain and sets *sing.
template <int ND>
__device__ void alljones_update_warp(const Cx<float>* Ah, const Cx<float>* Al, const Cx<float>* bh,
                                     const Cx<float>* bl, const Cx<float>* g, Cx<float>* x, int* sing) {
  const int r = threadIdx.x & 31;
  if (r >= ND) return;
  auto au = [](int i, int j) { return i * ND - i * (i - 1) / 2 + (j - i); };  // upper entry (i <= j)
  FF rx{bh[r].x, bl[r].x}, ry{bh[r].y, bl[r].y};
  float lox = 0.f, loy = 0.f;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int u = r <= j ? au(r, j) : au(j, r);
    Cx<float> h = Ah[u], lo = Al[u];
    if (r > j) { h.y = -h.y; lo.y = -lo.y; }
    const Cx<float> gj = g[j];
    rx = ff_sub_prod(rx, h.x, gj.x);
    rx = ff_sub_prod(rx, -h.y, gj.y);
    ry = ff_sub_prod(ry, h.x, gj.y);
    ry = ff_sub_prod(ry, h.y, gj.x);
    lox = fmaf(lo.x, gj.x, fmaf(-lo.y, gj.y, lox));
    loy = fmaf(lo.x, gj.y, fmaf(lo.y, gj.x, loy));
  }
  const Cx<float> c = cx<float>(rx.hi + (rx.lo - lox), ry.hi + (ry.lo - loy));
  const float arr = Ah[au(r, r)].x + Al[au(r, r)].x;
  if (arr > 0.f) {
    const float inv = 1.f / arr;
    x[r] = cx<float>(g[r].x + c.x * inv, g[r].y + c.y * inv);
  } else {
    x[r] = g[r];
    atomicOr(sing, 1);
  }
}

// ------------------------------------------------------------------------------------ iteration
// Stop decision on iteration kp of an interval from its na per-antenna partials cv (float-float
// |dg|^2, |g|^2) and flags cf (bit 0 non-finite, bit 1 singular): the status that ends the
// interval (GC_ST_NONFINITE, GC_ST_OK, GC_ST_NOT_CONVERGED at kp >= max_iter) or -1 to go on;
// *sing the OR of the singular flags.  Called by one whole warp: lane-strided float-float sums,
// a fixed tree to lane 0 and lane 0's result broadcast, so that every caller that reads the same
// slots takes the same decision.  GLOBAL: the slots are in global memory (read through L2).
template <bool GLOBAL>
__device__ inline int dd_decide(const float4* cv, const int32_t* cf, int na, double tol, int kp, int max_iter,
                                int* sing) {
  const int lane = threadIdx.x & 31;
  FF d2{0.f, 0.f}, n2{0.f, 0.f};
  int fl = 0;
  for (int q = lane; q < na; q += 32) {
    const float4 v = GLOBAL ? __ldcg(cv + q) : cv[q];
    d2 = ff_add(d2, FF{v.x, v.y});
    n2 = ff_add(n2, FF{v.z, v.w});
    fl |= GLOBAL ? __ldcg(cf + q) : cf[q];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const FF d{__shfl_down_sync(0xffffffffu, d2.hi, o), __shfl_down_sync(0xffffffffu, d2.lo, o)};
    const FF n{__shfl_down_sync(0xffffffffu, n2.hi, o), __shfl_down_sync(0xffffffffu, n2.lo, o)};
    if (lane + o < 32) { d2 = ff_add(d2, d); n2 = ff_add(n2, n); }
  }
  fl = __reduce_or_sync(0xffffffffu, fl);
  d2 = FF{__shfl_sync(0xffffffffu, d2.hi, 0), __shfl_sync(0xffffffffu, d2.lo, 0)};
  n2 = FF{__shfl_sync(0xffffffffu, n2.hi, 0), __shfl_sync(0xffffffffu, n2.lo, 0)};
  *sing = (fl >> 1) & 1;
  if (fl & 1) return GC_ST_NONFINITE;
  if (ff_value(d2) <= tol * tol * ff_value(n2)) return GC_ST_OK;
  if (kp >= max_iter) return GC_ST_NOT_CONVERGED;
  return -1;
}

constexpr int kIterEntries = 64;  // entries (baseline, side) of an antenna staged per chunk

template <int ND>
constexpr size_t dd_iter_smem(int na_max) {
  constexpr int NO = DDShape<ND>::NO, CS = (NO + 31) / 32 * 32;
  constexpr int LANES = kIterThreads / CS > 0 ? kIterThreads / CS : 1;
  return (size_t)na_max * ND * sizeof(Cx<float>) + (size_t)LANES * NO * sizeof(float4) +
         (size_t)kIterEntries * NO * sizeof(float2);
}

// One CTA per (interval, antenna p), launch k of the loop: iteration k of the interval, from
// g^(k-1) (gbuf parity (k-1) & 1) to g^(k) (parity k & 1).
//  * The antenna's entries and their moments (constant over the iterations) are fetched first,
//    before the wait on the previous launch (programmatic dependent launch), by cp.async.
//  * The interval's stop decision on iteration k - 1 comes next (dd_decide): a CTA of a finished
//    interval copies its antenna's final gains out (g^(k-1), or g^(k-2) after a non-finite
//    iteration) and the antenna-0 CTA records status, iterations and the deciding launch (stopk);
//    no CTA of the interval writes anything else.  Later launches skip the interval by stopk,
//    never by a flag written in the same launch.  The launch after max_iter only decides.
//  * Otherwise: the block sum from the moments (lane-strided compensated FP32, lanes combined in
//    float-float), the CohJones solve (FP32 Cholesky in registers by one warp, one float-float
//    refinement, FP64 when a pivot fails) or the AllJones step, the schedule for antenna p (odd k
//    or GN: the new gains; even k: their average with g^(k-1)), and the antenna's convergence
//    partials |g^(k) - g^(k-1)|^2, |g^(k)|^2 (float-float) and flags for the next launch.
// No CTA waits for another within a launch: the interval-wide test is deferred by one launch.
template <int ND>
__global__ void __launch_bounds__(kIterThreads, 5) dd_iter_kernel(const DDArgs a) {
  constexpr int NU = DDShape<ND>::NU, NO = DDShape<ND>::NO;
  constexpr int CS = (NO + 31) / 32 * 32;       // component slots per lane group
  constexpr int LANES = kIterThreads / CS > 0 ? kIterThreads / CS : 1;
  static_assert(kIterEntries % LANES == 0, "every chunk starts at lane 0");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<float>* gs = reinterpret_cast<Cx<float>*>(smem_raw);                       // [n_ant][ND]
  float4* red = reinterpret_cast<float4*>(gs + a.na_max * ND);                  // [LANES][NO]
  float2* smom = reinterpret_cast<float2*>(red + LANES * NO);                   // [kIterEntries][NO]
  __shared__ Cx<float> Ah[NU], Al[NU], bh[ND], bl[ND], xs[ND];
  __shared__ int s_sing, s_nf, s_st, s_sg;
  __shared__ int2 s_ent[kIterEntries];
  pdl_launch_dependents();
  const int it = blockIdx.x;
  if (it >= a.n_iitems) return;
  const int k = *a.kbase + a.k;
  if (k > a.max_iter + 1) return;
  const int i = a.iitem_int[it];
  const int p = a.iitem_ant[it];
  const int e0 = a.iitem_e0[it], e1 = a.iitem_e1[it];
  const int na = a.n_ant[i];
  const int64_t go = a.gain_off[i];
  const int tid = threadIdx.x;
  const int comp = tid % CS, lane = tid / CS;
  const bool worker = comp < NO && lane < LANES;
  const float2* mom = a.moments + a.mom_off[i];
  // entries base .. base + kIterEntries - 1 and their moments into shared memory (cp.async)
  auto stage = [&](int base) {
    const int m = min(kIterEntries, e1 - base);
    if (tid < m) s_ent[tid] = make_int2(a.ent[base + tid], a.entq[base + tid]);
    __syncthreads();
    if (worker)
      for (int idx = lane; idx < m; idx += LANES)
        dd_cp_async8(smom + idx * NO + comp, mom + (int64_t)(s_ent[idx].x >> 1) * NO + comp);
    dd_cp_commit();
    return m;
  };
  const int m0 = e1 > e0 ? stage(e0) : 0;
  pdl_wait();  // g^(k-1), the partials of iteration k - 1 and the flags come from the previous launch
  // the active flag, the decision on iteration k - 1 (warp 0) and g^(k-1) (the other warps) are
  // read at once; the gains are used only if the interval goes on
  const float* gcur = a.gbuf + (size_t)((k - 1) & 1) * a.n_gain * ND * 2;
  if (tid < 32) {
    int sg = 0;
    const size_t so = (size_t)((k - 1) & 1) * a.n_gain + go;  // the partials of iteration k - 1
    const int st = k >= 2 ? dd_decide<true>(a.conv + so, a.cflag + so, na, a.tol, k - 1, a.max_iter, &sg) : -1;
    // an interval decided by an earlier launch is left alone; one decided by this launch (its
    // antenna-0 CTA may already have recorded it) is decided again, identically, by every CTA
    if (tid == 0) {
      const int sk = __ldcg(a.stopk + i);
      s_st = (sk != 0 && sk < k) ? -2 : st;
      s_sg = sg;
    }
  } else {
    for (int x = tid - 32; x < na * ND; x += blockDim.x - 32)
      gs[x] = cx<float>(__ldcg(gcur + 2 * (go * ND + x)), __ldcg(gcur + 2 * (go * ND + x) + 1));
  }
  __syncthreads();
  if (s_st == -2) { dd_cp_wait<0>(); return; }  // finished in an earlier launch
  if (s_st >= 0) {
    const size_t src = (size_t)((s_st == GC_ST_NONFINITE ? k - 2 : k - 1) & 1) * a.n_gain * ND;
    if (tid < 2 * ND) a.gains[2 * ((go + p) * ND) + tid] = __ldcg(a.gbuf + 2 * (src + (go + p) * ND) + tid);
    if (p == 0 && tid == 0) {
      a.stopk[i] = k;
      a.active[i] = 0;
      a.iters[i] = k - 1;
      a.status[i] = s_st | (s_sg ? GC_ST_SINGULAR_FLAG : 0);
      atomicSub(a.n_active, 1);
    }
    dd_cp_wait<0>();
    return;
  }
  if (k > a.max_iter) { dd_cp_wait<0>(); return; }  // iteration max_iter was decided above
  int c = 0, d = 0;
  if (comp < NU) upper_cd(ND, comp, c, d);
  else c = comp - NU;
  float sx = 0.f, sxc = 0.f, sy = 0.f, syc = 0.f;
  // each lane takes entries lane, lane + LANES, ... of every chunk, in order
  for (int base = e0; base < e1; base += kIterEntries) {
    const int m = base == e0 ? m0 : stage(base);
    dd_cp_wait<0>();
    __syncthreads();  // every thread's copies visible
    if (worker)
      for (int idx = lane; idx < m; idx += LANES) {
        float2 v = smom[idx * NO + comp];
        const int2 e = s_ent[idx];
        if (e.x & 1) v.y = -v.y;  // conjugate baseline: conj(X), conj(B)
        const int q = e.y;
        Cx<float> t;
        if (comp < NU) t = mul_(mulc_(gs[q * ND + c], gs[q * ND + d]), cx<float>(v.x, v.y));
        else t = mul_(gs[q * ND + c], cx<float>(v.x, v.y));
        kahan_add(sx, sxc, t.x);
        kahan_add(sy, syc, t.y);
      }
    __syncthreads();  // before the next chunk replaces the staged entries and moments
  }
  if (worker) red[lane * NO + comp] = make_float4(sx, -sxc, sy, -syc);  // Kahan: the sum is s - c
  if (tid == 0) s_nf = 0;
  __syncthreads();
  if (tid < NO) {
    FF re{0.f, 0.f}, im{0.f, 0.f};
    for (int l = 0; l < LANES; ++l) {
      const float4 v = red[l * NO + tid];
      re = ff_add(re, ff_two_sum(v.x, v.y));
      im = ff_add(im, ff_two_sum(v.z, v.w));
    }
    if (tid < NU) { Ah[tid] = cx<float>(re.hi, im.hi); Al[tid] = cx<float>(re.lo, im.lo); }
    else { bh[tid - NU] = cx<float>(re.hi, im.hi); bl[tid - NU] = cx<float>(re.lo, im.lo); }
    if (!isfinite(re.hi) || !isfinite(im.hi)) atomicOr(&s_nf, 1);  // sums overflowed: the gains diverged
  }
  __syncthreads();
  if (a.method == 1) {  // AllJones
    if (tid == 0) s_sing = 0;
    __syncthreads();
    if (tid < 32) alljones_update_warp<ND>(Ah, Al, bh, bl, gs + p * ND, xs, &s_sing);
  } else if (tid < 32) {
    __shared__ Cx<float> Ls[ND * ND];
    __shared__ int s_ok;
    bool ok = chol_solve_warp_mixed<ND>(Ah, Al, bh, bl, xs, Ls);
    if (!ok) {  // rare: the block is not positive definite in FP32; FP64 decides
      __shared__ double2 Ad[NU], bd[ND], xd[ND], Am[ND * ND];
      __shared__ double dinv[ND];
      for (int u = tid; u < NU; u += 32)
        Ad[u] = make_double2((double)Ah[u].x + (double)Al[u].x, (double)Ah[u].y + (double)Al[u].y);
      for (int r = tid; r < ND; r += 32)
        bd[r] = make_double2((double)bh[r].x + (double)bl[r].x, (double)bh[r].y + (double)bl[r].y);
      __syncwarp();
      ok = chol_solve_warp<ND>(Ad, bd, xd, Am, dinv, &s_ok);
      for (int r = tid; r < ND; r += 32) xs[r] = cx<float>((float)xd[r].x, (float)xd[r].y);
      __syncwarp();
    }
    if (tid == 0) s_sing = ok ? 0 : 1;
  }
  __syncthreads();
  // schedule for antenna p, g^(k) out, and this antenna's convergence partials
  if (tid < 32) {
    FF d2{0.f, 0.f}, n2{0.f, 0.f};
    int nonfin = 0;
    if (tid < ND) {
      const Cx<float> old = gs[p * ND + tid];
      Cx<float> g = (s_sing && a.method != 1) ? old : xs[tid];
      if (s_nf) g = cx<float>(__int_as_float(0x7fc00000), 0.f);  // reported as non-finite gains
      const bool gn_step = (a.schedule == GC_SCHED_GN) || (k & 1);
      const Cx<float> nw = gn_step ? g : cx<float>(0.5f * (old.x + g.x), 0.5f * (old.y + g.y));
      float* gout = a.gbuf + (size_t)(k & 1) * a.n_gain * ND * 2 + 2 * ((go + p) * ND + tid);
      gout[0] = nw.x;
      gout[1] = nw.y;
      d2 = FF{abs2_(sub_(nw, old)), 0.f};
      n2 = FF{abs2_(nw), 0.f};
      nonfin = !isfinite(nw.x) || !isfinite(nw.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const FF dd{__shfl_down_sync(0xffffffffu, d2.hi, o), __shfl_down_sync(0xffffffffu, d2.lo, o)};
      const FF nn{__shfl_down_sync(0xffffffffu, n2.hi, o), __shfl_down_sync(0xffffffffu, n2.lo, o)};
      if (tid + o < 32) { d2 = ff_add(d2, dd); n2 = ff_add(n2, nn); }
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    if (tid == 0) {
      a.conv[(size_t)(k & 1) * a.n_gain + go + p] = make_float4(d2.hi, d2.lo, n2.hi, n2.lo);
      a.cflag[(size_t)(k & 1) * a.n_gain + go + p] = nonfin | (s_sing << 1);
    }
  }
}


// chi^2 per moment item (interval, 32-baseline tile) over all its rows, then per interval.
template <int ND>
__global__ void __launch_bounds__(256) dd_chi2_kernel(const DDArgs a, double* item_chi2) {
  __shared__ double red[64];
  const int it = blockIdx.x;
  if (it >= a.n_mitems) return;
  const int i = a.mitem_int[it], tile = a.mitem_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i], bo = a.bl_off[i];
  const int64_t go = a.gain_off[i];
  const int nbt = min(kMomBl, nb - tile * kMomBl);
  float s = 0.f, c = 0.f;
  for (int u = threadIdx.x; u < nbt * ns; u += blockDim.x) {
    const int sl = u / nbt, bl = u - sl * nbt;
    const int b = tile * kMomBl + bl;
    const int p = a.ant1[bo + b], q = a.ant2[bo + b];
    const int64_t r = a.row_off[i] + (int64_t)sl * nb + b;
    Cx<float> v = Vec<float>::ld1(a.vis + 2 * r);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const Cx<float> m = Vec<float>::ld1(a.model + 2 * ((int64_t)d * a.n_rows + r));
      const Cx<float> gp = cx<float>(a.gains[2 * ((go + p) * ND + d)], a.gains[2 * ((go + p) * ND + d) + 1]);
      const Cx<float> gq = cx<float>(a.gains[2 * ((go + q) * ND + d)], a.gains[2 * ((go + q) * ND + d) + 1]);
      v = sub_(v, mulc_(mul_(gp, m), gq));
    }
    kahan_add(s, c, abs2_(v));
  }
  const double tot = block_sum<double>((double)s - (double)c, red);
  if (threadIdx.x == 0) item_chi2[it] = tot;
}

__global__ void dd_chi2_final(const int32_t* first, const int32_t* count, const double* item_chi2, double* out,
                              int n_int) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  double s = 0.0;
  for (int j = 0; j < count[i]; ++j) s += item_chi2[first[i] + j];
  out[i] = s;
}

// ------------------------------------------------------------------------------------ host side
static DDPlan g_dd;

int build_dd_plan(const gc_layout* L, DDPlan& P, cudaStream_t s, int64_t mom_per_bl, int mom_tile) {
  const int n = L->n_intervals, nd = L->n_dir;
  const int64_t NO = mom_per_bl;
  std::vector<int64_t> mom_off(n);
  std::vector<int> mint, mtile, iint, iant, itab(n), tab_aoff, ant_off, ent, entq, cfirst(n), ccount(n);
  std::map<std::pair<int, int>, int> tabs;
  int64_t mo = 0;
  int n_active0 = 0, na_max = 1;
  for (int i = 0; i < n; ++i) {
    const int nb = L->n_bl[i], ns = L->n_samp[i], na = L->n_ant[i];
    na_max = na > na_max ? na : na_max;
    mom_off[i] = mo;
    mo += (int64_t)nb * NO;
    cfirst[i] = (int)mint.size();
    const bool has = (int64_t)nb * ns > 0;
    n_active0 += has;
    if (has)
      for (int t = 0; t < (nb + mom_tile - 1) / mom_tile; ++t) { mint.push_back(i); mtile.push_back(t); }
    ccount[i] = (int)mint.size() - cfirst[i];
    if (has)
      for (int p = 0; p < na; ++p) { iint.push_back(i); iant.push_back(p); }
    auto key = std::make_pair((int)L->bl_off[i], (int)nb);
    auto f = tabs.find(key);
    if (f != tabs.end()) { itab[i] = f->second; continue; }
    // antenna -> (baseline, side) lists for this table, sized for the interval's antenna count
    const int tid = (int)tab_aoff.size();
    tabs[key] = tid;
    itab[i] = tid;
    int nat = na;
    for (int b = 0; b < nb; ++b) {
      nat = L->ant1[key.first + b] + 1 > nat ? L->ant1[key.first + b] + 1 : nat;
      nat = L->ant2[key.first + b] + 1 > nat ? L->ant2[key.first + b] + 1 : nat;
    }
    std::vector<std::vector<std::pair<int, int>>> lists(nat);  // (baseline * 2 + side, other antenna)
    for (int b = 0; b < nb; ++b) {
      const int p1 = L->ant1[key.first + b], p2 = L->ant2[key.first + b];
      lists[p1].push_back({b * 2, p2});
      lists[p2].push_back({b * 2 + 1, p1});
    }
    tab_aoff.push_back((int)ant_off.size());
    for (int p = 0; p < nat; ++p) {
      ant_off.push_back((int)ent.size());
      for (auto& e : lists[p]) { ent.push_back(e.first); entq.push_back(e.second); }
    }
    ant_off.push_back((int)ent.size());
  }
  // a table shared by intervals with more antennas than it spans would index past its list:
  // extend every interval's reference to a table sized for it
  for (int i = 0; i < n; ++i) {
    const int tid = itab[i];
    const int next = tid + 1 < (int)tab_aoff.size() ? tab_aoff[tid + 1] : (int)ant_off.size();
    const int nat = next - tab_aoff[tid] - 1;
    if (nat < L->n_ant[i]) return GC_ERR_LAYOUT;
  }
  std::vector<int> ie0(iint.size()), ie1(iint.size());  // each iteration item's entry range
  for (size_t j = 0; j < iint.size(); ++j) {
    const int o = tab_aoff[itab[iint[j]]] + iant[j];
    ie0[j] = ant_off[o];
    ie1[j] = ant_off[o + 1];
  }
  if (ent.empty()) { ent.push_back(0); entq.push_back(0); }
  if (ie0.empty()) { ie0.push_back(0); ie1.push_back(0); }
  if (mint.empty()) { mint.push_back(0); mtile.push_back(0); }
  if (iint.empty()) { iint.push_back(0); iant.push_back(0); }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts;
  size_t off = 0;
  auto add = [&](const void* src, size_t bytes) { parts.push_back({src, bytes, off}); off += al(bytes ? bytes : 1); return parts.size() - 1; };
  const size_t p_row_off = add(L->row_off, (size_t)n * 8);
  const size_t p_mom_off = add(mom_off.data(), (size_t)n * 8);
  const size_t p_n_samp = add(L->n_samp, (size_t)n * 4);
  const size_t p_n_bl = add(L->n_bl, (size_t)n * 4);
  const size_t p_bl_off = add(L->bl_off, (size_t)n * 4);
  const size_t p_n_ant = add(L->n_ant, (size_t)n * 4);
  const size_t p_gain_off = add(L->gain_off, (size_t)n * 4);
  const size_t p_ant1 = add(L->ant1, (size_t)L->n_bl_table * 4);
  const size_t p_ant2 = add(L->ant2, (size_t)L->n_bl_table * 4);
  const size_t p_mint = add(mint.data(), mint.size() * 4);
  const size_t p_mtile = add(mtile.data(), mtile.size() * 4);
  const size_t p_iint = add(iint.data(), iint.size() * 4);
  const size_t p_iant = add(iant.data(), iant.size() * 4);
  const size_t p_ie0 = add(ie0.data(), ie0.size() * 4);
  const size_t p_ie1 = add(ie1.data(), ie1.size() * 4);
  const size_t p_ent = add(ent.data(), ent.size() * 4);
  const size_t p_entq = add(entq.data(), entq.size() * 4);
  const size_t p_cfirst = add(cfirst.data(), cfirst.size() * 4);
  const size_t p_ccount = add(ccount.data(), ccount.size() * 4);
  const size_t p_active = add(nullptr, (size_t)n * 4);
  const size_t p_iters = add(nullptr, (size_t)n * 4);
  const size_t p_status = add(nullptr, (size_t)n * 4);
  const size_t p_counters = add(nullptr, (size_t)n * 4);
  const size_t p_misc = add(nullptr, 64);
  const size_t p_sing = add(nullptr, (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 4);
  const size_t p_conv = add(nullptr, (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 2 * sizeof(float4));
  const size_t p_cflag = add(nullptr, (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 2 * 4);
  const size_t p_stopk = add(nullptr, (size_t)(n > 0 ? n : 1) * 4);
  const size_t p_chi2 = add(nullptr, mint.size() * 8);
  const size_t p_chi2o = add(nullptr, (size_t)(n > 0 ? n : 1) * 8);
  const size_t total = off;
  std::vector<unsigned char> host(total, 0);
  for (auto& pt : parts)
    if (pt.src && pt.bytes) memcpy(host.data() + pt.off, pt.src, pt.bytes);
  if (P.dev && P.dev_bytes < total) { cudaFree(P.dev); P.dev = nullptr; P.dev_bytes = 0; }
  if (!P.dev) { DD_CUDA(cudaMalloc(&P.dev, total)); P.dev_bytes = total; }
  DD_CUDA(cudaMemcpyAsync(P.dev, host.data(), total, cudaMemcpyHostToDevice, s));
  DD_CUDA(cudaStreamSynchronize(s));
  unsigned char* d = static_cast<unsigned char*>(P.dev);
  auto at = [&](size_t idx) { return (void*)(d + parts[idx].off); };
  DDArgs& a = P.args;
  a = DDArgs{};
  a.n_rows = L->n_rows;
  a.row_off = (const int64_t*)at(p_row_off);
  a.mom_off = (const int64_t*)at(p_mom_off);
  a.n_samp = (const int32_t*)at(p_n_samp);
  a.n_bl = (const int32_t*)at(p_n_bl);
  a.bl_off = (const int32_t*)at(p_bl_off);
  a.n_ant = (const int32_t*)at(p_n_ant);
  a.gain_off = (const int32_t*)at(p_gain_off);
  a.ant1 = (const int32_t*)at(p_ant1);
  a.ant2 = (const int32_t*)at(p_ant2);
  a.mitem_int = (const int32_t*)at(p_mint);
  a.mitem_tile = (const int32_t*)at(p_mtile);
  a.n_mitems = (int)(n_active0 > 0 ? mint.size() : 0);
  a.iitem_int = (const int32_t*)at(p_iint);
  a.iitem_ant = (const int32_t*)at(p_iant);
  a.n_iitems = (int)(n_active0 > 0 ? iint.size() : 0);
  a.iitem_e0 = (const int32_t*)at(p_ie0);
  a.iitem_e1 = (const int32_t*)at(p_ie1);
  a.ent = (const int32_t*)at(p_ent);
  a.entq = (const int32_t*)at(p_entq);
  a.active = (int32_t*)at(p_active);
  a.iters = (int32_t*)at(p_iters);
  a.status = (int32_t*)at(p_status);
  a.counters = (int32_t*)at(p_counters);
  a.n_active = (int32_t*)at(p_misc);
  a.kbase = a.n_active + 1;
  a.sing = (int32_t*)at(p_sing);
  a.conv = (float4*)at(p_conv);
  a.cflag = (int32_t*)at(p_cflag);
  a.stopk = (int32_t*)at(p_stopk);
  a.n_gain = L->n_gain;
  a.na_max = na_max;
  P.chi2_first = (int32_t*)at(p_cfirst);
  P.chi2_count = (int32_t*)at(p_ccount);
  P.chi2_items = (double*)at(p_chi2);
  P.chi2_out = (double*)at(p_chi2o);
  P.n_int = n;
  P.n_active0 = n_active0;
  P.nd = nd;
  P.n_mom = mo;
  return GC_OK;
}

template <int ND>
static int dd_run_nd(DDPlan& P, const gc_options* opt, cudaStream_t s, int* flag, double* prof_ms) {
  DDArgs& a = P.args;
  const size_t msmem = dd_moment_smem<ND>();
  const size_t ismem = dd_iter_smem<ND>(a.na_max);
  DD_CUDA(cudaFuncSetAttribute(dd_moment_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem));
  DD_CUDA(cudaFuncSetAttribute(dd_iter_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
  dd_init_kernel<<<(P.n_int + 255) / 256, 256, 0, s>>>(a, P.n_int, P.n_active0);
  g_launches++;
  const char* ce = getenv("GAINCAL_CHECK_EVERY");
  const int S = ce && atoi(ce) > 0 ? atoi(ce) : 8;
  DDTimer mt(opt->profile != 0, 1), it(opt->profile != 0, 1);
  if (a.n_mitems > 0) {
    mt.before(s);
    dd_moment_kernel<ND><<<a.n_mitems, kMomBl * kMomLanes, msmem, s>>>(a);
    mt.after(s);
    g_launches++;
  }
  DD_CUDA(cudaGetLastError());
  if (a.n_iitems > 0) {
    // One segment = S iteration launches (iterations *kbase + 1 .. *kbase + S) and the advance of
    // *kbase, captured once per argument set and relaunched until no interval is active.  A block
    // of a converged interval, or of an iteration past max_iter, returns at once.
    DDArgs ga = a;
    ga.k = 0;
    ga.vis = ga.model = nullptr;  // the iterations read only the moments
    if (!P.gexec || P.gS != S || P.gnd != ND || memcmp(&P.gargs, &ga, sizeof(DDArgs)) != 0) {
      if (P.gexec) { cudaGraphExecDestroy(P.gexec); P.gexec = nullptr; }
      cudaStream_t cs = nullptr;
      DD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaError_t ce2 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      int crc = ce2 == cudaSuccess ? 0 : (int)ce2;
      for (int j = 1; j <= S && !crc; ++j) {
        // programmatic dependent launches: launch j + 1 stages its entries and moments while
        // launch j finishes
        DDArgs x = ga;
        x.k = j;
        void* kargs[] = {&x};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.n_iitems);
        cfg.blockDim = dim3(kIterThreads);
        cfg.dynamicSmemBytes = ismem;
        cfg.stream = cs;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        crc = (int)cudaLaunchKernelExC(&cfg, (const void*)&dd_iter_kernel<ND>, kargs);
        if (!crc) crc = (int)cudaGetLastError();
      }
      if (!crc) crc = di_launch_advance(a.kbase, S, cs);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = ce2 == cudaSuccess ? cudaStreamEndCapture(cs, &g) : ce2;
      cudaStreamDestroy(cs);
      cudaError_t ie = cudaSuccess;
      if (!crc && ee == cudaSuccess) ie = cudaGraphInstantiate(&P.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (crc || ee != cudaSuccess || ie != cudaSuccess) {
        if (P.gexec) { cudaGraphExecDestroy(P.gexec); P.gexec = nullptr; }
        return set_cuda_error(crc ? (cudaError_t)crc : (ee != cudaSuccess ? ee : ie), "capture of the DD iteration segment");
      }
      P.gargs = ga;
      P.gS = S;
      P.gnd = ND;
    }
    // launch max_iter + 1 only takes the decision on iteration max_iter
    for (int k0 = 0; k0 <= opt->max_iter; k0 += S) {
      it.before(s);
      DD_CUDA(cudaGraphLaunch(P.gexec, s));
      it.after(s);
      g_launches += S + 1;
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
    prof_ms[1] = (double)it.launches * S;  // iteration launches (segments x S)
    prof_ms[2] = mt.ms;
  }
  if (opt->compute_chi2 && a.n_mitems > 0) {
    dd_chi2_kernel<ND><<<a.n_mitems, 256, 0, s>>>(a, P.chi2_items);
    dd_chi2_final<<<(P.n_int + 255) / 256, 256, 0, s>>>(P.chi2_first, P.chi2_count, P.chi2_items, P.chi2_out,
                                                         P.n_int);
    g_launches += 2;
    DD_CUDA(cudaGetLastError());
  }
  return GC_OK;
}

void dd_release() {
  if (g_dd.gexec) cudaGraphExecDestroy(g_dd.gexec);
  if (g_dd.dev) cudaFree(g_dd.dev);
  g_dd = DDPlan{};
}

int run_dd(const void* vis, const void* model, const gc_layout* L, void* gains, const gc_options* opt,
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
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  const uint64_t key = layout_hash(L, 0xDDull ^ ((uint64_t)dev << 40));
  if (g_dd.key != key || !g_dd.dev) {
    g_dd.key = 0;
    if ((rc = build_dd_plan(L, g_dd, s, (int64_t)L->n_dir * (L->n_dir + 1) / 2 + L->n_dir, kMomBl))) return rc;
    g_dd.key = key;
  }
  DDPlan& P = g_dd;
  const int nd = L->n_dir;
  const size_t vb = (size_t)L->n_rows * 8, mb = (size_t)L->n_rows * nd * 8, gb = (size_t)L->n_gain * nd * 8;
  DDArgs& a = P.args;
  // the iterations work on a copy of the gains in the workspace, so that the captured iteration
  // segment stays valid from call to call
  void* dg = nullptr;
  if ((rc = ws_get("dd_gains", gb > 0 ? gb : 8, &dg))) return rc;
  if (opt->host_buffers) {
    void *dv, *dm;
    if ((rc = ws_get("dd_h_vis", vb, &dv)) || (rc = ws_get("dd_h_model", mb, &dm))) return rc;
    if (vb) DD_CUDA(cudaMemcpyAsync(dv, vis, vb, cudaMemcpyHostToDevice, s));
    if (mb) DD_CUDA(cudaMemcpyAsync(dm, model, mb, cudaMemcpyHostToDevice, s));
    a.vis = (const float*)dv; a.model = (const float*)dm;
  } else {
    a.vis = (const float*)vis; a.model = (const float*)model;
  }
  if (gb) DD_CUDA(cudaMemcpyAsync(dg, gains, gb, opt->host_buffers ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  a.gains = (float*)dg;
  // iterates by parity; g^(0) = the starting gains
  void* gbuf = nullptr;
  if ((rc = ws_get("dd_gbuf", gb > 0 ? 2 * gb : 16, &gbuf))) return rc;
  if (gb) DD_CUDA(cudaMemcpyAsync(gbuf, dg, gb, cudaMemcpyDeviceToDevice, s));
  a.gbuf = (float*)gbuf;
  void *mom, *gnew;
  if ((rc = ws_get("dd_moments", (size_t)(P.n_mom > 0 ? P.n_mom : 1) * sizeof(float2), &mom))) return rc;
  if ((rc = ws_get("dd_gnew", gb > 0 ? gb : 8, &gnew))) return rc;
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
    case 1: rc = dd_run_nd<1>(P, opt, s, flag, prof); break;
    case 2: rc = dd_run_nd<2>(P, opt, s, flag, prof); break;
    case 3: rc = dd_run_nd<3>(P, opt, s, flag, prof); break;
    case 4: rc = dd_run_nd<4>(P, opt, s, flag, prof); break;
    case 5: rc = dd_run_nd<5>(P, opt, s, flag, prof); break;
    case 6: rc = dd_run_nd<6>(P, opt, s, flag, prof); break;
    case 7: rc = dd_run_nd<7>(P, opt, s, flag, prof); break;
    case 8: rc = dd_run_nd<8>(P, opt, s, flag, prof); break;
    case 9: rc = dd_run_nd<9>(P, opt, s, flag, prof); break;
    case 10: rc = dd_run_nd<10>(P, opt, s, flag, prof); break;
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

extern "C" int gc_calibrate_dd_cohjones(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                        const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                        int32_t* status_out, void* stream) {
  return gc::run_dd(vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream, 0);
}
extern "C" int gc_calibrate_dd_alljones(const void* vis, const void* model, const gc_layout* layout, void* gains,
                                        const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                        int32_t* status_out, void* stream) {
  return gc::run_dd(vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream, 1);
}
