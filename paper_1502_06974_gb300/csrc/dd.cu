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
template <int ND>
__global__ void __launch_bounds__(kIterThreads, 5) dd_iter_kernel(const DDArgs a) {
  constexpr int NU = DDShape<ND>::NU, NO = DDShape<ND>::NO;
  constexpr int CS = (NO + 31) / 32 * 32;       // component slots per lane group
  constexpr int LANES = kIterThreads / CS > 0 ? kIterThreads / CS : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<float>* gs = reinterpret_cast<Cx<float>*>(smem_raw);            // [n_ant][ND]
  float4* red = reinterpret_cast<float4*>(gs + a.na_max * ND);       // [LANES][NO] float-float (re, im)
  __shared__ Cx<float> Ah[NU], Al[NU], bh[ND], bl[ND], xs[ND];
  __shared__ int s_last, s_sing, s_nf;
  __shared__ double s_red[80];  // >= 160 floats for the end-of-update reduction
  __shared__ int2 s_ent[kIterThreads];
  const int it = blockIdx.x;
  if (it >= a.n_iitems) return;
  const int i = a.iitem_int[it];
  const int k = *a.kbase + a.k;
  if (a.active[i] == 0 || k > a.max_iter) return;
  const int p = a.iitem_ant[it];
  const int na = a.n_ant[i];
  const int64_t go = a.gain_off[i];
  const int tid = threadIdx.x;
  for (int x = tid; x < na * ND; x += blockDim.x)
    gs[x] = cx<float>(a.gains[2 * (go * ND + x)], a.gains[2 * (go * ND + x) + 1]);
  const int comp = tid % CS, lane = tid / CS;
  const bool worker = comp < NO && lane < LANES;
  int c = 0, d = 0;
  if (comp < NU) upper_cd(ND, comp, c, d);
  else c = comp - NU;
  float sx = 0.f, sxc = 0.f, sy = 0.f, syc = 0.f;
  const float2* mom = a.moments + a.mom_off[i];
  const int e0 = a.iitem_e0[it], e1 = a.iitem_e1[it];
  // the antenna's entries, kIterThreads at a time, staged in shared memory so that every moment
  // load's address is known at once; each lane takes entries lane, lane + LANES, ... in order
  for (int base = e0; base < e1; base += kIterThreads) {
    const int n = min(kIterThreads, e1 - base);
    if (tid < n) s_ent[tid] = make_int2(a.ent[base + tid], a.entq[base + tid]);
    __syncthreads();
    if (worker) {
      constexpr int U = 8;
      for (int j = lane; j < n; j += U * LANES) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = j + u * LANES;
          const int en = idx < n ? s_ent[idx].x : 0;
          v[u] = idx < n ? mom[(int64_t)(en >> 1) * NO + comp] : make_float2(0.f, 0.f);
          if (en & 1) v[u].y = -v[u].y;  // conjugate baseline: conj(X), conj(B)
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = j + u * LANES;
          if (idx >= n) continue;
          const int q = s_ent[idx].y;
          Cx<float> t;
          if (comp < NU) t = mul_(mulc_(gs[q * ND + c], gs[q * ND + d]), cx<float>(v[u].x, v[u].y));
          else t = mul_(gs[q * ND + c], cx<float>(v[u].x, v[u].y));
          kahan_add(sx, sxc, t.x);
          kahan_add(sy, syc, t.y);
        }
      }
    }
    __syncthreads();  // before the next chunk replaces the staged entries
  }
  if (e1 <= e0) __syncthreads();  // the gains are staged even for an antenna without baselines
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
  if (tid < ND) {
    Cx<float> g = (s_sing && a.method != 1) ? gs[p * ND + tid] : xs[tid];
    if (s_nf) g = cx<float>(__int_as_float(0x7fc00000), 0.f);  // reported as non-finite gains
    a.gnew[2 * ((go + p) * ND + tid)] = g.x;
    a.gnew[2 * ((go + p) * ND + tid) + 1] = g.y;
  }
  if (tid == 0) a.sing[go + p] = s_sing;
  // the last antenna of the interval to finish applies the schedule and the convergence test
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&a.counters[i], 1) == na - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  dd_interval_update(a, i, k, na, go, ND, gs, reinterpret_cast<float*>(s_red));
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
  constexpr int NO = DDShape<ND>::NO;
  constexpr int CS = (NO + 31) / 32 * 32;
  constexpr int LANES = kIterThreads / CS > 0 ? kIterThreads / CS : 1;
  DDArgs& a = P.args;
  const size_t msmem = dd_moment_smem<ND>();
  const size_t ismem = (size_t)a.na_max * ND * sizeof(Cx<float>) + (size_t)LANES * NO * sizeof(float4) + 16;
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
        DDArgs x = ga;
        x.k = j;
        dd_iter_kernel<ND><<<a.n_iitems, kIterThreads, ismem, cs>>>(x);
        crc = (int)cudaGetLastError();
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
    for (int k0 = 0; k0 < opt->max_iter; k0 += S) {
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
