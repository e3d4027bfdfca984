// Direction-independent StefCal kernels (scalar and 2x2 Jones), streaming form.
//
// One launch = one iteration k of Sect. 3.1 over every active solution interval:
//   1. accumulate, per antenna, the top half of J^H d and the diagonal block of J^H J over all
//      rows (baselines x samples) of the interval -- eqs. JHJ:DI:tf / JHR:DI:tf (scalar) and the
//      diagonal of eq. JHJ:pol with the polarized J^H D (2x2).  Every stored baseline (p, q)
//      feeds antenna p directly and antenna q through its conjugate row (Sect. 2.1, eq. JJ:di);
//   2. the CTA that completes an interval applies the GN step with the diagonal approximation
//      (eq. stefcal; 2x2: eq. update:DI:diag:pol read as [sum D Y^H][sum Y Y^H]^-1), averages it
//      with the current gains on even k (eq. stefcal-lambda-average, lambda = 1), and tests
//      ||g_k+1 - g_k|| <= tol ||g_k+1|| (App. C, first criterion).
//
// Work decomposition: a persistent grid pulls (interval, sample-range) items from an atomic
// queue.  Inside an item, thread t owns baseline b = tile*256 + t and sums its samples in
// registers (at most kSubChain at a time); the 256 per-thread partials are then reduced into
// per-antenna sums in shared memory in a fixed order given by a host-built slot list, with
// compensated (Kahan) addition.  Items of a multi-item interval write their per-antenna sums to
// scratch; the last one to arrive (atomic counter) combines them in item order.  Results are
// therefore bitwise reproducible run to run.
#include <cuda_runtime.h>

#include <cstdlib>
#include <type_traits>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace gc {

constexpr int kRedChunks = 4;  // chunk count of the optional split slot-list reduction (GAINCAL_RED_CHUNKS=4)

// Shared-memory carve-up (elements of T): partials [256][2 NC + 1] (padded: bank-conflict free) |
// acc [na_max][NC] | comp [na_max][NC] | gains [na_max][GW] | new gains [na_max][GW] |
// reduction buffer [64] | per-antenna auxiliaries [na_max][4] (moment path).
template <typename T, class K>
__host__ __device__ inline size_t di_smem_elems(int na_max) {
  return (size_t)kDIThreads * (2 * K::NC + 1) + 2 * (size_t)na_max * K::NC + 2 * (size_t)na_max * K::GW + 64 +
         4 * (size_t)na_max + (size_t)na_max * K::NC * kRedChunks;
}

template <typename T, class K, bool ACC_ONLY>
__global__ void __launch_bounds__(kDIThreads) di_iter_kernel(const DIArgs a) {
  constexpr int NC = K::NC, GW = K::GW, TB = kDIThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* part = reinterpret_cast<T*>(smem_raw);
  constexpr int PS = 2 * NC + 1;
  T* acc = part + TB * PS;
  T* cmp = acc + a.na_max * NC;
  T* gs = cmp + a.na_max * NC;
  T* ng = gs + a.na_max * GW;
  T* red = ng + a.na_max * GW;
  __shared__ int s_item, s_last;
  const int tid = threadIdx.x;
  const int k = a.k + (a.kbase ? *a.kbase : 0);
  const T* vis = static_cast<const T*>(a.vis);
  const T* mod = static_cast<const T*>(a.model);
  const T* wts = static_cast<const T*>(a.weights);
  T* gains = static_cast<T*>(a.gains);

  if (blockIdx.x == 0 && tid == 0) a.qhead[(k + 1) & 1] = 0;  // next launch's queue head

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.qhead[k & 1], 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    const int i = a.item_int[it];
    if (!ACC_ONLY && a.active[i] == 0) continue;

    const int nb = a.n_bl[i], na = a.n_ant[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int64_t r0 = a.row_off[i];
    const int s0 = a.item_s0[it], s1 = a.item_s1[it];
    const int tab = a.itab[i];
    const int nat = a.tab_nant[tab];
    const int* csr = a.csr_off + a.tab_base[tab];

    for (int x = tid; x < na * GW; x += TB) gs[x] = gains[go * GW + x];
    for (int x = tid; x < na * NC; x += TB) { acc[x] = T(0); cmp[x] = T(0); }
    __syncthreads();

    const int ntiles = (nb + TB - 1) / TB;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t * TB + tid;
      const bool have = b < nb;
      typename K::G gp{}, gq{};
      if (have) {
        const int p = a.ant1[bo + b], q = a.ant2[bo + b];
        gp = K::ld_gain(gs + p * GW);
        gq = K::ld_gain(gs + q * GW);
      }
      const int* off = csr + t * (nat + 1);
      for (int sc = s0; sc < s1; sc += kSubChain) {
        const int se = min(s1, sc + kSubChain);
        T pp[NC], pq[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { pp[c] = T(0); pq[c] = T(0); }
        if (have) {
          const int64_t rb = r0 + b;
#pragma unroll 4
          for (int s = sc; s < se; ++s) {
            const int64_t r = rb + (int64_t)s * nb;
            K::row(vis, mod, r, gp, gq, pp, pq, row_sw(wts, r));
          }
        }
        T* my = part + tid * PS;
#pragma unroll
        for (int c = 0; c < NC; ++c) { my[c] = pp[c]; my[NC + c] = pq[c]; }
        __syncthreads();
        for (int x = tid; x < nat * NC; x += TB) {
          const int an = x / NC, c = x - an * NC;
          T s = T(0);
          const int e1 = __ldg(off + an + 1);
          for (int e = __ldg(off + an); e < e1; ++e) s += part[__ldg(a.csr_ent + e) + c];
          kahan_add(acc[x], cmp[x], s);
        }
        __syncthreads();
      }
    }

    // Combine the items of a multi-item interval: the last arrival sums them in item order.
    bool finish = true;
    const int nch = a.n_chunks[i];
    if (nch > 1) {
      T* scr = static_cast<T*>(a.scratch) + a.item_scr[it];
      for (int x = tid; x < nat * NC; x += TB) scr[x] = acc[x] - cmp[x];
      __threadfence();
      __syncthreads();
      if (tid == 0) s_last = (atomicAdd(&a.counters[i], 1) == nch - 1);
      __syncthreads();
      finish = s_last;
      if (finish) {
        __threadfence();
        const int fi = a.first_item[i];
        for (int x = tid; x < nat * NC; x += TB) {
          T s = T(0), c = T(0);
          for (int j = 0; j < nch; ++j)
            kahan_add(s, c, __ldcg(static_cast<const T*>(a.scratch) + a.item_scr[fi + j] + x));
          acc[x] = s;
          cmp[x] = c;
        }
        if (tid == 0) a.counters[i] = 0;
        __syncthreads();
      }
    }
    if (!finish) continue;

    if (ACC_ONLY) {
      T* jhd = static_cast<T*>(a.jhd_out);
      T* jhj = static_cast<T*>(a.jhj_out);
      for (int an = tid; an < na; an += TB) {
        T v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = acc[an * NC + c] - cmp[an * NC + c];
        K::write_acc(v, jhd, jhj, go + an);
      }
      __syncthreads();
      continue;
    }

    // Update (eq. stefcal / eq. update:DI:diag:pol), schedule and convergence for interval i.
    T d2 = T(0), n2 = T(0);
    int sing = 0, nonfin = 0;
    const bool gn_step = (a.schedule == GC_SCHED_GN) || (k & 1);
    for (int an = tid; an < na; an += TB) {
      T v[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = acc[an * NC + c] - cmp[an * NC + c];
      const typename K::G old = K::ld_gain(gs + an * GW);
      typename K::G g;
      if (!K::solve(v, old, g)) sing = 1;
      const typename K::G nw = gn_step ? g : K::avg(old, g);
      d2 += K::dist2(nw, old);
      n2 += K::norm2(nw);
      if (!K::finite(nw)) nonfin = 1;
      K::st_gain(ng + an * GW, nw);
    }
    d2 = block_sum(d2, red);
    n2 = block_sum(n2, red);
    sing = block_or(sing, reinterpret_cast<int*>(red));
    nonfin = block_or(nonfin, reinterpret_cast<int*>(red));
    if (!nonfin)
      for (int x = tid; x < na * GW; x += TB) gains[go * GW + x] = ng[x];
    if (tid == 0) {
      int st = -1;
      if (nonfin) st = GC_ST_NONFINITE;
      else if ((double)d2 <= a.tol * a.tol * (double)n2) st = GC_ST_OK;
      else if (k >= a.max_iter) st = GC_ST_NOT_CONVERGED;
      if (st >= 0) {
        a.active[i] = 0;
        a.iters[i] = k;
        a.status[i] = st | (sing ? GC_ST_SINGULAR_FLAG : 0);
        atomicSub(a.n_active, 1);
      }
    }
    __syncthreads();
  }
}


// ------------------------------------------------------------------------------------------
// Moment-stream iteration, split in two launches per iteration.
//
// di_macc_kernel (accumulate): a grid-stride loop over the tiles (256 baselines) of the intervals
//   still iterating.  Each thread turns one baseline's moments (the sample sums with the gains
//   factored out, written once by the moment pass) into its p- and q-side contributions -- 48
//   coalesced loads and 160 FMA per 2x2 baseline -- and the CTA reduces the tile into per-antenna
//   partial sums (fixed-order slot lists), written to scratch.  No atomics, no fences: the tile
//   work is spread evenly over the grid.
// di_msolve_kernel (update): one CTA per interval; sums its tiles' partials in tile order with
//   compensation, applies the GN step / average, tests convergence, writes gains and the
//   per-antenna auxiliaries (G^H G) and, if the interval keeps iterating, appends its tiles to
//   the next iteration's list (lists rotate over three buffers: launch k reads list k % 3,
//   appends to (k + 1) % 3; the accumulate launch of k clears (k + 2) % 3).
// ------------------------------------------------------------------------------------------
// Device-scope acquire/release operations (cheaper than a sequentially consistent fence): an
// atomic add whose release side orders the CTA's earlier writes (made visible to this thread by a
// block barrier) before the add, and whose acquire side orders later reads after it.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Loads of data other CTAs of the same launch write (gains, auxiliaries, work lists) go through L2
// (ld.global.cg) in the persistent loop kernel, whose CTAs do not meet at a launch boundary.
template <bool COH>
__device__ __forceinline__ float ldc(const float* p) { return COH ? __ldcg(p) : *p; }
template <bool COH>
__device__ __forceinline__ int ldc(const int* p) { return COH ? __ldcg(p) : *p; }

template <class K, bool COH>
__device__ __forceinline__ typename K::G ld_gain_c(const float* g) {
  if constexpr (!COH) {
    return K::ld_gain(g);
  } else {
    float v[K::GW];
#pragma unroll
    for (int c = 0; c < K::GW; ++c) v[c] = __ldcg(g + c);
    return K::ld_gain(v);
  }
}

// An interval's tile partials summed in tile order with compensation, all (antenna, component)
// pairs in parallel; antennas the baseline table does not reach get zeros.  The interval's items
// are consecutive and so are their scratch blocks (nat * NC floats each), so every tile's address
// is known without loading it: eight tiles' loads are in flight at once.
template <int NC>
__device__ __forceinline__ void combine_tiles(const DIArgs& a, const float* scr, int na, int nat, int nch, int fi,
                                              float* tot) {
  const float* base = scr + a.item_scr[fi];
  const int64_t stride = (int64_t)nat * NC;
  for (int x = threadIdx.x; x < na * NC; x += blockDim.x) {
    float s = 0.f, cc = 0.f;
    if (x < nat * NC) {
      int j = 0;
      for (; j + 8 <= nch; j += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(base + (j + u) * stride + x);
#pragma unroll
        for (int u = 0; u < 8; ++u) kahan_add(s, cc, v[u]);
      }
      for (; j < nch; ++j) kahan_add(s, cc, __ldcg(base + j * stride + x));
    }
    tot[x] = s - cc;
  }
}

// Update of interval i at iteration k by one CTA (every thread calls it): its tiles' partials
// summed in tile order with compensation, the GN step / average, the convergence test, gains and
// auxiliaries written, and either the interval retired or its tiles appended to work list nxt.
// `tot` holds [na_max][NC] floats.
template <class MK, bool COH>
__device__ __forceinline__ void solve_interval(const DIArgs& a, int k, int i, float* tot, double* red, int nxt) {
  using K = typename MK::K;
  using G = typename K::G;
  constexpr int NC = K::NC, GW = K::GW, AW = MK::AW, TB = kDIThreads;
  const int tid = threadIdx.x;
  float* gains = static_cast<float*>(a.gains);
  const float* scr = static_cast<const float*>(a.scratch);
  const int na = a.n_ant[i];
  const int64_t go = a.gain_off[i];
  const int nat = a.tab_nant[a.itab[i]];
  const int nch = a.n_chunks[i], fi = a.first_item[i];
  combine_tiles<NC>(a, scr, na, nat, nch, fi, tot);
  __syncthreads();
  FF d2{0.f, 0.f}, n2{0.f, 0.f};  // float-float sums (the FP64 pipe of GB300 is narrow)
  int sing = 0, nonfin = 0;
  const int kl = k - (a.k0 ? ldc<COH>(a.k0 + i) : 0);  // the interval's own iteration number
  const bool gn_step = (a.schedule == GC_SCHED_GN) || (kl & 1);
  for (int an = tid; an < na; an += TB) {
    const G old = ld_gain_c<K, COH>(gains + (go + an) * GW);
    G g;
    if (!K::solve(tot + an * NC, old, g)) sing = 1;
    const G nw = gn_step ? g : K::avg(old, g);
    d2 = ff_add_f(d2, K::dist2(nw, old));
    n2 = ff_add_f(n2, K::norm2(nw));
    if (!K::finite(nw)) nonfin = 1;
    K::st_gain(a.gnew + (go + an) * GW, nw);   // staged until the interval's decision is known
  }
  block_reduce_step_ff(d2, n2, sing, nonfin, reinterpret_cast<float*>(red), na);  // antennas tid < na only
  if (!nonfin)
    for (int an = tid; an < na; an += TB) {
      const G nw = K::ld_gain(a.gnew + (go + an) * GW);
      K::st_gain(gains + (go + an) * GW, nw);
      MK::aux(nw, a.aux + (go + an) * AW);
    }
  if (tid == 0) {
    const double D2 = ff_value(d2), N2 = ff_value(n2);
    int st = -1;
    if (nonfin) st = GC_ST_NONFINITE;
    else if (D2 <= a.tol * a.tol * N2) st = GC_ST_OK;
    else if (kl >= a.max_iter) st = GC_ST_NOT_CONVERGED;
    if (a.gate && a.gate[i] == 0 && (st >= 0 || D2 <= a.gate_tol * a.gate_tol * N2)) a.gate[i] = kl;
    if (st >= 0) {
      a.active[i] = 0;
      a.iters[i] = kl;
      a.status[i] = st | (sing ? GC_ST_SINGULAR_FLAG : 0);
      atomicSub(a.n_active, 1);
    } else {
      const int base = atomicAdd(&a.icount[nxt], nch);
      for (int j = 0; j < nch; ++j) a.ilist[(size_t)nxt * a.n_items + base + j] = fi + j;
    }
  }
  __syncthreads();
}

// Solve phase of iteration k (see di_msolve_kernel): CTAs loop over the intervals.
template <class MK, bool COH>
__device__ __forceinline__ void msolve_phase(const DIArgs& a, int k, int n_int, float* tot, double* red) {
  for (int i = blockIdx.x; i < n_int; i += gridDim.x) {
    if (ldc<COH>(a.active + i) == 0) continue;
    solve_interval<MK, COH>(a, k, i, tot, red, (k + 1) % 3);
  }
}

// p-side contributions summed over each maximal run of lanes with the same antenna p inside a
// warp (an inclusive segmented scan, fixed shuffle order): the run's last lane then holds the
// run's sum, and the antenna's slot list names only run ends.  In a baseline table ordered by p
// a warp holds one or two runs, so the slot lists shrink from ~N_ant entries to a few per tile.
// Lanes past the last baseline pass p = -1 and zeros.  Every lane of the warp must call it.
template <int NC>
__device__ __forceinline__ void warp_run_scan(int p, float* v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int up = __shfl_up_sync(full, p, 1);
  const unsigned starts = __ballot_sync(full, lane == 0 || up != p);
  const int seg0 = 31 - __clz(starts & (full >> (31 - lane)));   // first lane of this lane's run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float u = __shfl_up_sync(full, v[c], o);
      if (lane - o >= seg0) v[c] += u;
    }
  }
}

// Accumulate phase of iteration k (see di_macc_kernel); `smem` holds [TB][2 NC + 1] partials and
// [na_max * NC * CH] chunk sums.
template <class MK, int CH, bool PF, bool COH>
__device__ __forceinline__ void macc_phase(const DIArgs& a, int k, float* smem) {
  using K = typename MK::K;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, AW = MK::AW, TB = kDIThreads, PS = 2 * NC + 1;
  float* part = smem;           // [TB][PS]
  float* ps = part + TB * PS;   // [na_max * NC * CH]
  const int tid = threadIdx.x;
  const int cur = k % 3;
  const bool fixed = a.xcount > 0;
  const int* list = a.ilist + (size_t)cur * a.n_items;
  const int n_list = fixed ? a.xcount : ldc<COH>(a.icount + cur);
  if (!fixed && blockIdx.x == 0 && tid == 0) a.icount[(k + 2) % 3] = 0;
  const float* gains = static_cast<const float*>(a.gains);
  // the moments of the next tile are requested while the current tile is being reduced
  float m[NM];
  auto item = [&](int slot) { return fixed ? a.xbegin + slot : ldc<COH>(list + slot); };
  auto fetch = [&](int slot) {
    const int it = item(slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    if (t * TB + tid < a.n_bl[i]) {
      // tile layout [NM / 4][TB][4] (see mom_index): one 16-byte load per 4 components
      const float4* src = reinterpret_cast<const float4*>(a.moments + (a.mom_off[i] + (int64_t)t * TB) * NM) + tid;
#pragma unroll
      for (int g = 0; g < NM / 4; ++g) {
        const float4 v = __ldg(src + g * TB);
        m[4 * g] = v.x; m[4 * g + 1] = v.y; m[4 * g + 2] = v.z; m[4 * g + 3] = v.w;
      }
    }
  };
  int slot = blockIdx.x;
  if (PF && slot < n_list) fetch(slot);
  while (slot < n_list) {
    if (!PF) fetch(slot);
    const int it = item(slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    const int nb = a.n_bl[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int b = t * TB + tid;
    float pp[NC], pq[NC];
    int p = -1;
#pragma unroll
    for (int c = 0; c < NC; ++c) pp[c] = pq[c] = 0.f;
    if (b < nb) {
      p = a.ant1[bo + b];
      const int q = a.ant2[bo + b];
      float ap[AW], aq[AW];
#pragma unroll
      for (int c = 0; c < AW; ++c) {
        ap[c] = ldc<COH>(a.aux + (go + p) * AW + c);
        aq[c] = ldc<COH>(a.aux + (go + q) * AW + c);
      }
      MK::partials(m, ld_gain_c<K, COH>(gains + (go + p) * GW), ld_gain_c<K, COH>(gains + (go + q) * GW), ap, aq,
                   pp, pq);
    }
    warp_run_scan<NC>(p, pp);
    if (b < nb) {
      float* my = part + tid * PS;
#pragma unroll
      for (int c = 0; c < NC; ++c) { my[c] = pp[c]; my[NC + c] = pq[c]; }
    }
    const int next = slot + gridDim.x;
    if (PF && next < n_list) fetch(next);
    __syncthreads();
    const int tab = a.itab[i];
    const int nat = a.tab_nant[tab];
    const int* off = a.csr_off + a.tab_base[tab] + t * (nat + 1);
    float* scr = static_cast<float*>(a.scratch) + a.item_scr[it];
    if (CH == 1) {
      for (int x = tid; x < nat * NC; x += TB) {
        const int an = x / NC, c = x - an * NC;
        const int e1 = __ldg(off + an + 1);
        float s = 0.f;
        for (int e = __ldg(off + an); e < e1; ++e) s += part[__ldg(a.csr_ent + e) + c];
        scr[x] = s;
      }
    } else {
      for (int x = tid; x < nat * NC * CH; x += TB) {
        const int ch = x % CH, r = x / CH, an = r / NC, c = r - an * NC;
        const int e0 = __ldg(off + an), len = __ldg(off + an + 1) - e0;
        const int b0 = e0 + (len * ch) / CH, b1 = e0 + (len * (ch + 1)) / CH;
        float s = 0.f;
        for (int e = b0; e < b1; ++e) s += part[__ldg(a.csr_ent + e) + c];
        ps[x] = s;
      }
      __syncthreads();
      for (int x = tid; x < nat * NC; x += TB) {
        float s = 0.f;
#pragma unroll
        for (int ch = 0; ch < CH; ++ch) s += ps[x * CH + ch];
        scr[x] = s;
      }
    }
    __syncthreads();
    slot = next;
  }
}

template <class MK, int CH, bool PF>
__global__ void __launch_bounds__(kDIThreads, PF ? 3 : 4) di_macc_kernel(const DIArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_launch_dependents();
  pdl_wait();  // gains, lists and the iteration base come from the previous launch
  macc_phase<MK, CH, PF, false>(a, a.k + (a.kbase ? *a.kbase : 0), reinterpret_cast<float*>(smem_raw));
}

// di_macc_staged_kernel: the accumulate launch with the moments staged through shared memory.
// Each thread copies its own baseline's moments of the CTA's next tile with 16-byte asynchronous
// copies (cp.async, no registers held) while the current tile is computed and reduced, so every
// CTA keeps one tile (48 KB for 2x2) in flight from HBM at all times.  Two stages of one tile
// each; the current stage is reused for the per-thread partials once its moments are in
// registers.  Same arithmetic and reduction order as di_macc_kernel (slot-list reduction, CH = 1).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class MK>
__global__ void __launch_bounds__(kDIThreads, 2) di_macc_staged_kernel(const DIArgs a) {
  pdl_launch_dependents();
  pdl_wait();  // gains, lists and the iteration base come from the previous launch
  using K = typename MK::K;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, NG = NM / 4, AW = MK::AW, TB = kDIThreads, PS = 2 * NC + 1;
  // a stage holds a tile's moments ([NG][TB] float4) and, after they are read, its partials
  // ([TB][PS] floats): SG float4 per thread
  constexpr int SG = (NM > PS ? NM : PS + 3) / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* stage0 = reinterpret_cast<float4*>(smem_raw);   // [2][SG][TB] float4
  const int tid = threadIdx.x;
  const int k = a.k + (a.kbase ? *a.kbase : 0);
  const int cur = k % 3;
  const bool fixed = a.xcount > 0;
  const int* list = a.ilist + (size_t)cur * a.n_items;
  const int n_list = fixed ? a.xcount : a.icount[cur];
  if (!fixed && blockIdx.x == 0 && tid == 0) a.icount[(k + 2) % 3] = 0;
  const float* gains = static_cast<const float*>(a.gains);
  const int G = gridDim.x;
  auto item = [&](int slot) { return fixed ? a.xbegin + slot : list[slot]; };
  // copies this thread's moments of the tile at `slot` into stage st
  auto issue = [&](int slot, int st) {
    const int it = item(slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    const float4* src = reinterpret_cast<const float4*>(a.moments + (a.mom_off[i] + (int64_t)t * TB) * NM) + tid;
    float4* dst = stage0 + (size_t)st * SG * TB + tid;
#pragma unroll
    for (int g = 0; g < NG; ++g) cp_async16(dst + g * TB, src + g * TB);
    cp_async_commit();
  };
  int slot = blockIdx.x, st = 0;
  if (slot < n_list) issue(slot, 0);
  for (; slot < n_list; slot += G, st ^= 1) {
    const int next = slot + G;
    if (next < n_list) issue(next, st ^ 1);   // that stage was released by the barrier ending the last tile
    const int it = item(slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    const int nb = a.n_bl[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int b = t * TB + tid;
    float pp[NC], pq[NC];
    int p = -1, q = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) pp[c] = pq[c] = 0.f;
    if (b < nb) { p = a.ant1[bo + b]; q = a.ant2[bo + b]; }
    // every thread waits for its own copies of this tile (also past the last baseline: the stage is
    // about to be overwritten with partials, so no copy into it may still be in flight)
    if (next < n_list) cp_async_wait<1>(); else cp_async_wait<0>();
    if (b < nb) {
      const typename K::G gp = K::ld_gain(gains + (go + p) * GW), gq = K::ld_gain(gains + (go + q) * GW);
      const float4* mine = stage0 + (size_t)st * SG * TB + tid;
      float m[NM];
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const float4 v = mine[g * TB];
        m[4 * g] = v.x; m[4 * g + 1] = v.y; m[4 * g + 2] = v.z; m[4 * g + 3] = v.w;
      }
      MK::partials(m, gp, gq, a.aux + (go + p) * AW, a.aux + (go + q) * AW, pp, pq);
    }
    warp_run_scan<NC>(p, pp);
    __syncthreads();                                   // every thread has its moments: reuse the stage
    float* part = reinterpret_cast<float*>(stage0 + (size_t)st * SG * TB);   // [TB][PS]
    if (b < nb) {
      float* my = part + tid * PS;
#pragma unroll
      for (int c = 0; c < NC; ++c) { my[c] = pp[c]; my[NC + c] = pq[c]; }
    }
    __syncthreads();
    const int tab = a.itab[i];
    const int nat = a.tab_nant[tab];
    const int* off = a.csr_off + a.tab_base[tab] + t * (nat + 1);
    float* scr = static_cast<float*>(a.scratch) + a.item_scr[it];
    for (int x = tid; x < nat * NC; x += TB) {
      const int an = x / NC, c = x - an * NC;
      const int e1 = __ldg(off + an + 1);
      float s = 0.f;
      for (int e = __ldg(off + an); e < e1; ++e) s += part[__ldg(a.csr_ent + e) + c];
      scr[x] = s;
    }
    __syncthreads();                                   // the stage is free for the copy after next
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------ bulk-copy accumulate
// di_macc_bulk_kernel: the accumulate launch fed by bulk asynchronous copies (cp.async.bulk, the
// one-dimensional form of the tensor memory accelerator) into a two-stage shared-memory ring per
// CTA.  Per tile, one thread copies four contiguous blocks whose addresses come from the item's
// descriptor alone: the tile's moments (48 KB for 2x2), its static block (the antenna pair of each
// slot and the slot lists of the reduction), and the interval's gains and auxiliaries; an mbarrier
// per stage counts the bytes in.  The next tile is in flight while the current one is computed and
// reduced from shared memory, so the only global loads on a tile's dependency chain are the
// work-list entry and the descriptor, which the copying thread fetches a tile further ahead.  Same
// arithmetic and reduction order as di_macc_kernel with CH = 1 (identical results).
constexpr int kBulkSpins = 1 << 22;  // bounded mbarrier waits: each try_wait also suspends briefly
// Tries of a tile's first wait (kBulkSpins unless di_set_bulk_wait_tries changed it).  Waits for
// copies still in flight after a failed one always take the full kBulkSpins: a CTA leaves only once
// its own copies have landed, or after that bound too.
__device__ int g_bulk_wait_tries = kBulkSpins;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int tries) {
  const unsigned addr = smem_u32(bar);
  for (int n = 0; n < tries; ++n) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <class MK>
struct BulkShape {
  using K = typename MK::K;
  static constexpr int PS = 2 * K::NC + 1;
  static constexpr int MW = MK::NM > PS ? MK::NM : PS;  // floats per slot in a stage's first region
  static_assert(MK::NM % 4 == 0 && K::GW % 4 == 0 && MK::AW % 4 == 0, "bulk copies move 16-byte units");
  // a stage: [MW][TB] moments (then [TB][PS] partials) | static block | gains | auxiliaries
  __host__ __device__ static size_t stage_floats(int na_max, int tblk_max) {
    return (size_t)MW * kDIThreads + (size_t)tblk_max + (size_t)na_max * (K::GW + MK::AW);
  }
};

template <class MK>
__global__ void __launch_bounds__(kDIThreads, 2) di_macc_bulk_kernel(const DIArgs a) {
  pdl_launch_dependents();
  pdl_wait();  // gains, lists and the iteration base come from the previous launch
  using K = typename MK::K;
  using Sh = BulkShape<MK>;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, NG = NM / 4, AW = MK::AW, TB = kDIThreads, PS = Sh::PS,
                MW = Sh::MW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ int4 hdr[2][2];  // per stage: {baselines, table antennas, scratch lo, hi}, {first gain, ...}
  const int tid = threadIdx.x;
  const int na_max = a.na_max, tbm = a.tblk_max;
  const size_t sf = Sh::stage_floats(na_max, tbm);
  const int tries = g_bulk_wait_tries;
  const int k = a.k + (a.kbase ? *a.kbase : 0);
  const int cur = k % 3;
  const bool fixed = a.xcount > 0;
  const int* list = a.ilist + (size_t)cur * a.n_items;
  const int n_list = fixed ? a.xcount : a.icount[cur];
  if (!fixed && blockIdx.x == 0 && tid == 0) a.icount[(k + 2) % 3] = 0;
  const int G = gridDim.x;
  if ((int)blockIdx.x >= n_list) return;  // the whole CTA: no tile for it
  const float* gains = static_cast<const float*>(a.gains);
  const bool gal = (reinterpret_cast<uintptr_t>(gains) & 15) == 0;  // gains copied in bulk when 16-byte aligned
  float* const stage0 = reinterpret_cast<float*>(smem_raw);
  // work-list entry and descriptor of a slot (thread 0); they are fetched a tile apart so that
  // neither load waits for the other
  auto item = [&](int slot) { return fixed ? a.xbegin + slot : list[slot]; };
  auto desc = [&](int it, int4* d) {
    const int4* p = a.item_desc + (size_t)it * 3;
    d[0] = p[0];
    d[1] = p[1];
    d[2] = p[2];
  };
  // copies of one tile into stage s (thread 0)
  auto issue = [&](int s, const int4* d) {
    float* st = stage0 + (size_t)s * sf;
    const int64_t mom = (int64_t)(((uint64_t)(unsigned)d[0].y << 32) | (unsigned)d[0].x);
    const int go = d[1].z, na = d[1].w;
    hdr[s][0] = make_int4(d[0].z, d[1].y, d[2].x, d[2].y);
    hdr[s][1] = make_int4(go, 0, 0, 0);
    const unsigned mb = (unsigned)(NM * TB * sizeof(float)), tb = (unsigned)d[1].x * 4u;
    const unsigned gb = gal ? (unsigned)(na * GW * sizeof(float)) : 0u, ab = (unsigned)(na * AW * sizeof(float));
    mbar_expect_tx(&full[s], mb + tb + gb + ab);
    bulk_g2s(st, a.moments + mom, mb, &full[s]);
    bulk_g2s(st + MW * TB, a.tblk + d[0].w, tb, &full[s]);
    if (gb) bulk_g2s(st + MW * TB + tbm, gains + (size_t)go * GW, gb, &full[s]);
    bulk_g2s(st + MW * TB + tbm + (size_t)na_max * GW, a.aux + (size_t)go * AW, ab, &full[s]);
  };
  int4 nd[3];          // thread 0: descriptor of the slot after the two in flight
  int nit = 0;         // thread 0: work-list entry of the slot after that
  bool pend[2] = {false, false};
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    int4 d[3];
    desc(item(blockIdx.x), d);
    issue(0, d);
    pend[0] = true;
    if ((int)blockIdx.x + G < n_list) {
      desc(item(blockIdx.x + G), d);
      issue(1, d);
      pend[1] = true;
    }
    if ((int)blockIdx.x + 2 * G < n_list) desc(item(blockIdx.x + 2 * G), nd);
    if ((int)blockIdx.x + 3 * G < n_list) nit = item(blockIdx.x + 3 * G);
  }
  int j = 0;
  for (int slot = blockIdx.x; slot < n_list; slot += G, ++j) {
    const int s = j & 1;
    const bool ok = mbar_wait(&full[s], (unsigned)(j >> 1) & 1u, tries);
    float* st = stage0 + (size_t)s * sf;
    const int4 h = hdr[s][0];
    const int nbt = h.x, nat = h.y, go = hdr[s][1].x;
    const int* tbk = reinterpret_cast<const int*>(st + MW * TB);
    const float* sg = st + MW * TB + tbm;
    const float* sa = sg + (size_t)na_max * GW;
    float pp[NC], pq[NC];
    int p = -1;
#pragma unroll
    for (int c = 0; c < NC; ++c) pp[c] = pq[c] = 0.f;
    if (ok && tid < nbt) {
      p = tbk[tid];
      const int q = tbk[TB + tid];
      float m[NM];
      const float4* mine = reinterpret_cast<const float4*>(st) + tid;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const float4 v = mine[g * TB];
        m[4 * g] = v.x; m[4 * g + 1] = v.y; m[4 * g + 2] = v.z; m[4 * g + 3] = v.w;
      }
      const typename K::G gp = gal ? K::ld_gain(sg + p * GW) : K::ld_gain(gains + ((int64_t)go + p) * GW);
      const typename K::G gq = gal ? K::ld_gain(sg + q * GW) : K::ld_gain(gains + ((int64_t)go + q) * GW);
      MK::partials(m, gp, gq, sa + p * AW, sa + q * AW, pp, pq);
    }
    warp_run_scan<NC>(p, pp);
    // the partials go over this thread's own moment slots (it alone read them), component c of
    // side h at float4 group (h NC + c) / 4: no barrier is needed before the stores
    static_assert(NC % 4 == 0 && 2 * NC / 4 <= NG, "partials fit the thread's moment slots");
    float4* my4 = reinterpret_cast<float4*>(st) + tid;
    if (tid < nbt) {
#pragma unroll
      for (int r = 0; r < NC / 4; ++r) {
        my4[r * TB] = make_float4(pp[4 * r], pp[4 * r + 1], pp[4 * r + 2], pp[4 * r + 3]);
        my4[(NC / 4 + r) * TB] = make_float4(pq[4 * r], pq[4 * r + 1], pq[4 * r + 2], pq[4 * r + 3]);
      }
    }
    // a copy that never landed ends the CTA (all threads agree), after a bounded wait for every
    // copy it still has in flight (this tile's and the next one's)
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(a.err, 1);
        for (int t = 0; t < 2; ++t)
          if (pend[t]) mbar_wait(&full[t], (unsigned)((t == s ? j : j + 1) >> 1) & 1u, kBulkSpins);
      }
      __syncthreads();
      return;
    }
    if (tid == 0) pend[s] = false;
    const float* part = st;  // slot s, component c of side h: [(h NC + c) / 4][TB][4]
    const int* off = tbk + 2 * TB;
    const int* ent = off + ((nat + 1 + 3) & ~3);
    float* scr = static_cast<float*>(a.scratch) + (int64_t)(((uint64_t)(unsigned)h.w << 32) | (unsigned)h.z);
    // a thread takes one antenna and CG consecutive components: the slot list is read once for
    // them and their sums (each in list order, as in the other variants) proceed side by side
    constexpr int CG = 3, NG3 = NC / CG;
    static_assert(NC % CG == 0, "components come in groups of CG");
    for (int x = tid; x < nat * NG3; x += TB) {
      const int an = x / NG3, c0 = (x - an * NG3) * CG;
      const int e1 = off[an + 1];
      float sum[CG];
#pragma unroll
      for (int u = 0; u < CG; ++u) sum[u] = 0.f;
      int co[CG];  // offset of component c0 + u from its slot's first component
#pragma unroll
      for (int u = 0; u < CG; ++u) co[u] = ((c0 + u) >> 2) * TB * 4 + ((c0 + u) & 3);
      for (int e = off[an]; e < e1; ++e) {
        const float* pe = part + ent[e];
#pragma unroll
        for (int u = 0; u < CG; ++u) sum[u] += pe[co[u]];
      }
#pragma unroll
      for (int u = 0; u < CG; ++u) scr[an * NC + c0 + u] = sum[u];
    }
    __syncthreads();  // the stage is free
    if (tid == 0 && slot + 2 * G < n_list) {
      // the stage was read and written through the generic proxy: order that before the copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(s, nd);
      pend[s] = true;
      if (slot + 3 * G < n_list) desc(nit, nd);
      if (slot + 4 * G < n_list) nit = item(slot + 4 * G);
    }
  }
}

template <class MK>
__global__ void __launch_bounds__(kDIThreads, 8) di_msolve_kernel(const DIArgs a, int n_int) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_launch_dependents();
  pdl_wait();  // the tile partials come from the accumulate launch
  __shared__ double red[96];
  msolve_phase<MK, false>(a, a.k + (a.kbase ? *a.kbase : 0), n_int, reinterpret_cast<float*>(smem_raw), red);
}

// di_mstep1_kernel: one launch per iteration (cooperative launch, so every CTA is resident).
//   Phase S: each CTA updates its intervals from the previous iteration's tile partials (the solve
//   of di_msolve_kernel), appends the survivors' tiles to work list (k-1) % 3, and publishes
//   flag[i] = k (release), or -k when the interval stopped.  An interval in its first iteration
//   is only published and listed.
//   Phase A: the accumulate of iteration k over the tiles of list (k+1) % 3 (the survivors of the
//   update before last, a superset of the current ones); a tile waits (acquire, bounded) for its
//   interval's flag, skips the interval if it stopped, and otherwise runs exactly the accumulate
//   of di_macc_kernel.  Tiles of intervals updated early start while other CTAs still solve.
//   Lists rotate over three buffers: launch k clears list k % 3 (read two launches ago).
//   Same arithmetic and order as the two-launch iteration, so the results are bitwise equal.
__device__ __forceinline__ int ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
constexpr unsigned kFlagSpins = 1u << 24;

template <class MK, int CH, bool PF>
__global__ void __launch_bounds__(kDIThreads, PF ? 3 : 4) di_mstep1_kernel(const DIArgs a, int n_int, int* err) {
  using K = typename MK::K;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, AW = MK::AW, TB = kDIThreads, PS = 2 * NC + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* part = reinterpret_cast<float*>(smem_raw);   // [TB][PS]
  float* ps = part + TB * PS;                           // [na_max * NC * CH]
  float* tot = ps + (size_t)a.na_max * NC * CH;         // [na_max][NC]
  __shared__ double red[96];
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  const int k = a.k + *a.kbase;
  if (blockIdx.x == 0 && tid == 0) a.icount[k % 3] = 0;
  // ---- phase S: the update of iteration k - 1
  const int ls = (k + 2) % 3;  // = (k - 1) % 3
  for (int i = blockIdx.x; i < n_int; i += gridDim.x) {
    if (__ldcg(a.active + i) == 0) {  // stopped earlier or without data: any tile of it is skipped
      if (tid == 0) st_release_i(a.flag + i, -k);
      continue;
    }
    const int kp = k - 1 - (a.k0 ? __ldcg(a.k0 + i) : 0);  // the interval's own number of the previous iteration
    if (kp >= 1) {
      solve_interval<MK, true>(a, k - 1, i, tot, red, ls);
    } else if (tid == 0) {
      const int nch = a.n_chunks[i], fi = a.first_item[i];
      const int base = atomicAdd(&a.icount[ls], nch);
      for (int j = 0; j < nch; ++j) a.ilist[(size_t)ls * a.n_items + base + j] = fi + j;
    }
    __syncthreads();
    if (tid == 0) st_release_i(a.flag + i, __ldcg(a.active + i) ? k : -k);
  }
  // ---- phase A: the accumulate of iteration k
  const int la = (k + 1) % 3;
  const int* list = a.ilist + (size_t)la * a.n_items;
  const int n_list = __ldcg(a.icount + la);
  const float* gains = static_cast<const float*>(a.gains);
  float m[NM];
  auto fetch = [&](int slot) {
    const int it = __ldcg(list + slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    if (t * TB + tid < a.n_bl[i]) {
      const float4* src = reinterpret_cast<const float4*>(a.moments + (a.mom_off[i] + (int64_t)t * TB) * NM) + tid;
#pragma unroll
      for (int g = 0; g < NM / 4; ++g) {
        const float4 v = __ldg(src + g * TB);
        m[4 * g] = v.x; m[4 * g + 1] = v.y; m[4 * g + 2] = v.z; m[4 * g + 3] = v.w;
      }
    }
  };
  int slot = blockIdx.x;
  if (PF && slot < n_list) fetch(slot);
  while (slot < n_list) {
    if (!PF) fetch(slot);
    const int it = __ldcg(list + slot);
    const int i = a.item_int[it], t = a.item_s0[it];
    const int next = slot + gridDim.x;
    if (tid == 0) {
      int f = ld_acquire_i(a.flag + i);
      unsigned n = 0;
      while (f != k && f != -k) {
        if (++n > kFlagSpins) { atomicExch(err, 1); f = 0; break; }
        __nanosleep(64);
        f = ld_acquire_i(a.flag + i);
      }
      s_flag = f;
    }
    __syncthreads();
    const int f = s_flag;
    if (f == 0) return;            // a wait timed out: the host reports the error
    if (f != k) {                  // the interval stopped at the last update
      if (PF && next < n_list) fetch(next);
      __syncthreads();
      slot = next;
      continue;
    }
    const int nb = a.n_bl[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int b = t * TB + tid;
    float pp[NC], pq[NC];
    int p = -1;
#pragma unroll
    for (int c = 0; c < NC; ++c) pp[c] = pq[c] = 0.f;
    if (b < nb) {
      p = a.ant1[bo + b];
      const int q = a.ant2[bo + b];
      float ap[AW], aq[AW];
#pragma unroll
      for (int c = 0; c < AW; ++c) {
        ap[c] = __ldcg(a.aux + (go + p) * AW + c);
        aq[c] = __ldcg(a.aux + (go + q) * AW + c);
      }
      MK::partials(m, ld_gain_c<K, true>(gains + (go + p) * GW), ld_gain_c<K, true>(gains + (go + q) * GW), ap,
                   aq, pp, pq);
    }
    warp_run_scan<NC>(p, pp);
    if (b < nb) {
      float* my = part + tid * PS;
#pragma unroll
      for (int c = 0; c < NC; ++c) { my[c] = pp[c]; my[NC + c] = pq[c]; }
    }
    if (PF && next < n_list) fetch(next);
    __syncthreads();
    const int tab = a.itab[i];
    const int nat = a.tab_nant[tab];
    const int* off = a.csr_off + a.tab_base[tab] + t * (nat + 1);
    float* scr = static_cast<float*>(a.scratch) + a.item_scr[it];
    if (CH == 1) {
      for (int x = tid; x < nat * NC; x += TB) {
        const int an = x / NC, c = x - an * NC;
        const int e1 = __ldg(off + an + 1);
        float s = 0.f;
        for (int e = __ldg(off + an); e < e1; ++e) s += part[__ldg(a.csr_ent + e) + c];
        scr[x] = s;
      }
    } else {
      for (int x = tid; x < nat * NC * CH; x += TB) {
        const int ch = x % CH, r = x / CH, an = r / NC, c = r - an * NC;
        const int e0 = __ldg(off + an), len = __ldg(off + an + 1) - e0;
        const int b0 = e0 + (len * ch) / CH, b1 = e0 + (len * (ch + 1)) / CH;
        float s = 0.f;
        for (int e = b0; e < b1; ++e) s += part[__ldg(a.csr_ent + e) + c];
        ps[x] = s;
      }
      __syncthreads();
      for (int x = tid; x < nat * NC; x += TB) {
        float s = 0.f;
#pragma unroll
        for (int ch = 0; ch < CH; ++ch) s += ps[x * CH + ch];
        scr[x] = s;
      }
    }
    __syncthreads();
    slot = next;
  }
}

// Grid-wide barrier of the persistent loop kernel (a cooperative launch, so every CTA is
// resident): arrival counter bar[0], generation bar[1].  The wait is bounded: after
// kBarrierSpins polls the CTA records the timeout in *err and the kernel returns, so a barrier
// that cannot complete ends the launch with an error status instead of hanging the GPU.
constexpr unsigned kBarrierSpins = 1u << 25;

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(bar + 1);
    int ok = 1;
    if (atom_add_acq_rel(bar, 1u) + 1u == gridDim.x) {
      st_relaxed(bar, 0u);
      atom_add_acq_rel(bar + 1, 1u);  // release: the reset and every arrival happen before the new generation
    } else {
      unsigned n = 0;
      while (ld_acquire(bar + 1) == gen) {
        if (++n > kBarrierSpins) { ok = 0; atomicExch(err, 1); break; }
        __nanosleep(32);
      }
    }
    *s_ok = ok && *(volatile int*)err == 0;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Persistent iteration loop: up to S iterations (k = *kbase + 1 ..) in one cooperative launch,
// the accumulate and solve phases separated by grid barriers; stops early once no interval is
// active and leaves *kbase at the last iteration done.  Same arithmetic, in the same order, as
// the two-launch iteration.
template <class MK, int CH, bool PF>
__global__ void __launch_bounds__(kDIThreads, PF ? 3 : 4) di_mloop_kernel(const DIArgs a, int n_int, int S,
                                                                          unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[96];
  __shared__ int s_ok;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int base = *a.kbase;
  int j = 1;
  for (; j <= S; ++j) {
    if (__ldcg(a.n_active) <= 0) break;
    macc_phase<MK, CH, PF, true>(a, base + j, sm);
    if (!grid_barrier(bar, err, &s_ok)) return;
    msolve_phase<MK, true>(a, base + j, n_int, sm, red);
    if (!grid_barrier(bar, err, &s_ok)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.kbase = base + j - 1;
}

// di_msum_kernel: after an accumulate launch at the current gains, per interval: the combined
//   per-antenna sums (tot_out [n_gain][NC], the partial-sum component order) and
//   e_out[i] = chi^2(g) - sum |d|^2 over the interval.  Each baseline feeds both of its antennas,
//   and both orientations of a row have the same residual norm, so the interval's chi^2 is half the
//   sum of the per-antenna energies plus the constant sum |d|^2, which cancels when two gain sets of
//   the same interval are compared.  Gains, flags and work lists are left untouched.
template <class MK>
__global__ void __launch_bounds__(kDIThreads) di_msum_kernel(const DIArgs a, int i_lo, int n, float* tot_out,
                                                             double* e_out) {
  using K = typename MK::K;
  constexpr int NC = K::NC, GW = K::GW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tot = reinterpret_cast<float*>(smem_raw);  // [na_max][NC]
  __shared__ double red[32];
  const float* gains = static_cast<const float*>(a.gains);
  const float* scr = static_cast<const float*>(a.scratch);
  const int64_t gbase = a.gain_off[i_lo];
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const int i = i_lo + j;
    const int na = a.n_ant[i];
    const int64_t go = a.gain_off[i] - gbase;  // tot_out rows start at the range's first gain slot
    if ((int64_t)a.n_samp[i] * a.n_bl[i] == 0) {
      for (int x = threadIdx.x; x < na * NC; x += blockDim.x) tot_out[go * NC + x] = 0.f;
      if (threadIdx.x == 0) e_out[j] = 0.0;
      continue;
    }
    combine_tiles<NC>(a, scr, na, a.tab_nant[a.itab[i]], a.n_chunks[i], a.first_item[i], tot);
    __syncthreads();
    for (int x = threadIdx.x; x < na * NC; x += blockDim.x) tot_out[go * NC + x] = tot[x];
    const float* gi = gains + (int64_t)a.gain_off[i] * GW;
    double e = 0.0;
    for (int an = threadIdx.x; an < na; an += blockDim.x) e += K::energy(tot + an * NC, K::ld_gain(gi + an * GW));
    e = block_sum<double>(e, red);
    if (threadIdx.x == 0) e_out[j] = 0.5 * e;
    __syncthreads();
  }
}

// Per-antenna auxiliaries (G^H G or |g|^2) of the starting gains.
template <class MK>
__global__ void di_maux_kernel(const float* gains, float* aux, int n_gain) {
  using K = typename MK::K;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n_gain) MK::aux(K::ld_gain(gains + (int64_t)x * K::GW), aux + (int64_t)x * MK::AW);
}

// Per-call state: active flags, statuses, counters.
__global__ void di_init_kernel(const DIArgs a, int n_int, int n_active0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *a.n_active = n_active0;
    if (a.kbase) *a.kbase = 0;
    if (a.err) *a.err = 0;
    a.qhead[0] = 0;
    a.qhead[1] = 0;
    if (a.icount) {
      a.icount[0] = a.icount[1] = a.icount[2] = 0;
      a.icount[a.first_list ? a.first_list : 1] = a.n_items;
    }
  }
  if (a.ilist)  // iteration 1 takes every item
    for (int j = i; j < a.n_items; j += gridDim.x * blockDim.x)
      a.ilist[(size_t)(a.first_list ? a.first_list : 1) * a.n_items + j] = j;
  if (i < n_int) {
    const int64_t rows = (int64_t)a.n_samp[i] * a.n_bl[i];
    if (a.flag) a.flag[i] = 0;
    a.active[i] = rows > 0 ? 1 : 0;
    a.iters[i] = 0;
    a.status[i] = rows > 0 ? GC_ST_NOT_CONVERGED : GC_ST_NODATA;
    a.counters[i] = 0;
  }
}

// chi^2 = sum |r|^2 per item (compensated sums in T, block total in double).
template <typename T, class K>
__global__ void __launch_bounds__(kDIThreads) di_chi2_kernel(const DIArgs a, double* item_chi2) {
  constexpr int GW = K::GW;
  __shared__ double red[64];
  const T* vis = static_cast<const T*>(a.vis);
  const T* mod = static_cast<const T*>(a.model);
  const T* wts = static_cast<const T*>(a.weights);
  const T* gains = static_cast<const T*>(a.gains);
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int i = a.item_int[it];
    const int nb = a.n_bl[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i], r0 = a.row_off[i];
    const int s0 = a.item_s0[it], s1 = a.item_s1[it];
    const int64_t n = (int64_t)(s1 - s0) * nb;
    T s = T(0), c = T(0);
    for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
      const int sl = (int)(u / nb), b = (int)(u - (int64_t)sl * nb);
      const int p = a.ant1[bo + b], q = a.ant2[bo + b];
      const typename K::G gp = K::ld_gain(gains + (go + p) * GW);
      const typename K::G gq = K::ld_gain(gains + (go + q) * GW);
      const int64_t r = r0 + (int64_t)(s0 + sl) * nb + b;
      kahan_add(s, c, row_w(wts, r) * K::resid2(vis, mod, r, gp, gq));
    }
    const double tot = block_sum<double>((double)s - (double)c, red);
    if (threadIdx.x == 0) item_chi2[it] = tot;
  }
}

__global__ void di_chi2_final_kernel(const DIArgs a, const double* item_chi2, double* out, int n_int) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  const int64_t rows = (int64_t)a.n_samp[i] * a.n_bl[i];
  double s = 0.0;
  if (rows > 0) {
    const int fi = a.first_item[i];
    for (int j = 0; j < a.n_chunks[i]; ++j) s += item_chi2[fi + j];
  }
  out[i] = s;
}

// ------------------------------------------------------------------------------------------ host
template <typename T, class K, bool ACC>
static void* kernel_ptr() { return reinterpret_cast<void*>(&di_iter_kernel<T, K, ACC>); }

static void* pick(int kind, int dtype, int acc_only) {
  if (kind == 0) {
    if (dtype == GC_DTYPE_C64) return acc_only ? kernel_ptr<float, ScalarKind<float>, true>() : kernel_ptr<float, ScalarKind<float>, false>();
    return acc_only ? kernel_ptr<double, ScalarKind<double>, true>() : kernel_ptr<double, ScalarKind<double>, false>();
  }
  if (dtype == GC_DTYPE_C64) return acc_only ? kernel_ptr<float, JonesKind<float>, true>() : kernel_ptr<float, JonesKind<float>, false>();
  return acc_only ? kernel_ptr<double, JonesKind<double>, true>() : kernel_ptr<double, JonesKind<double>, false>();
}

// prefetch: 0 none, 1 the next tile's moments into registers, 2 staged through shared memory
// (di_macc_staged_kernel, single-chunk reduction)
template <class MK>
static const void* pick_acc_k(int red_chunks, int prefetch) {
  const bool c4 = red_chunks == kRedChunks;
  if constexpr (std::is_same<MK, JonesMom>::value) {
    if (prefetch == 3) return (const void*)&di_macc_bulk_kernel<MK>;
  }
  if (prefetch == 2) return (const void*)&di_macc_staged_kernel<MK>;
  if (prefetch) return c4 ? (const void*)&di_macc_kernel<MK, kRedChunks, true> : (const void*)&di_macc_kernel<MK, 1, true>;
  return c4 ? (const void*)&di_macc_kernel<MK, kRedChunks, false> : (const void*)&di_macc_kernel<MK, 1, false>;
}

static const void* pick_acc(int kind, int red_chunks, int prefetch) {
  return kind == 0 ? pick_acc_k<ScalarMom>(red_chunks, prefetch) : pick_acc_k<JonesMom>(red_chunks, prefetch);
}

int di_macc_smem(int kind, int na_max, int red_chunks, int prefetch) {
  const int nc = kind == 0 ? 3 : 12, nm = kind == 0 ? 4 : 48;
  if (prefetch == 2) {
    const int ps = 2 * nc + 1, sg = (nm > ps ? nm : ps + 3) / 4;
    return (int)(sizeof(float) * 2 * 4 * (size_t)sg * kDIThreads);
  }
  const int ch = red_chunks == kRedChunks ? kRedChunks : 1;
  return (int)(sizeof(float) * ((size_t)kDIThreads * (2 * nc + 1) + (size_t)na_max * nc * ch + (size_t)na_max * nc));
}

int di_macc_bulk_smem(int kind, int na_max, int tblk_max) {
  if (kind != 1) return 1 << 30;
  return (int)(2 * sizeof(float) * BulkShape<JonesMom>::stage_floats(na_max, tblk_max));
}

int di_set_bulk_wait_tries(int tries) {
  const int v = tries < 0 ? kBulkSpins : tries;
  return (int)cudaMemcpyToSymbol(g_bulk_wait_tries, &v, sizeof(int));
}

int di_macc_max_blocks_per_sm(int kind, int smem, int red_chunks, int prefetch, int* out) {
  const void* f = pick_acc(kind, red_chunks, prefetch);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, kDIThreads, smem);
}

constexpr int kSolveGrid = 1216;  // 8 CTAs on each of 152 SMs

static const void* pick_loop(int kind, int red_chunks, int prefetch) {
  const bool c4 = red_chunks == kRedChunks, pf = prefetch == 1;
  if (kind == 0) {
    if (pf) return c4 ? (const void*)&di_mloop_kernel<ScalarMom, kRedChunks, true> : (const void*)&di_mloop_kernel<ScalarMom, 1, true>;
    return c4 ? (const void*)&di_mloop_kernel<ScalarMom, kRedChunks, false> : (const void*)&di_mloop_kernel<ScalarMom, 1, false>;
  }
  if (pf) return c4 ? (const void*)&di_mloop_kernel<JonesMom, kRedChunks, true> : (const void*)&di_mloop_kernel<JonesMom, 1, true>;
  return c4 ? (const void*)&di_mloop_kernel<JonesMom, kRedChunks, false> : (const void*)&di_mloop_kernel<JonesMom, 1, false>;
}

int di_mloop_smem(int kind, int na_max, int red_chunks) {
  const int nc = kind == 0 ? 3 : 12;
  return std::max(di_macc_smem(kind, na_max, red_chunks, 0), (int)(sizeof(float) * (size_t)na_max * nc));
}

int di_mloop_max_grid(int kind, int smem, int red_chunks, int prefetch, int* out) {
  const void* f = pick_loop(kind, red_chunks, prefetch);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0, dev = 0, nsm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kDIThreads, smem);
  if (e != cudaSuccess) return (int)e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  *out = per_sm * nsm;
  return 0;
}

int di_launch_mloop(int kind, const DIArgs& a, int grid, int smem, int n_int, int S, int red_chunks, int prefetch,
                    unsigned* bar, int* err, void* stream) {
  void* args[] = {const_cast<DIArgs*>(&a), &n_int, &S, &bar, &err};
  return (int)cudaLaunchCooperativeKernel(pick_loop(kind, red_chunks, prefetch), dim3(grid), dim3(kDIThreads), args,
                                          (size_t)smem, (cudaStream_t)stream);
}

static const void* pick_step1(int kind, int red_chunks, int prefetch) {
  const bool c4 = red_chunks == kRedChunks, pf = prefetch == 1;
  if (kind == 0) {
    if (pf) return c4 ? (const void*)&di_mstep1_kernel<ScalarMom, kRedChunks, true> : (const void*)&di_mstep1_kernel<ScalarMom, 1, true>;
    return c4 ? (const void*)&di_mstep1_kernel<ScalarMom, kRedChunks, false> : (const void*)&di_mstep1_kernel<ScalarMom, 1, false>;
  }
  if (pf) return c4 ? (const void*)&di_mstep1_kernel<JonesMom, kRedChunks, true> : (const void*)&di_mstep1_kernel<JonesMom, 1, true>;
  return c4 ? (const void*)&di_mstep1_kernel<JonesMom, kRedChunks, false> : (const void*)&di_mstep1_kernel<JonesMom, 1, false>;
}

int di_mstep1_smem(int kind, int na_max, int red_chunks) {
  return di_macc_smem(kind, na_max, red_chunks, 0);  // partials, chunk sums and the solve's [na_max][NC]
}

int di_mstep1_max_grid(int kind, int smem, int red_chunks, int prefetch, int* out) {
  const void* f = pick_step1(kind, red_chunks, prefetch);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0, dev = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kDIThreads, smem)) != cudaSuccess) return (int)e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  *out = per_sm * nsm;
  return 0;
}

// one iteration in one cooperative launch (the launch attribute keeps it capturable in a graph)
int di_launch_mstep1(int kind, const DIArgs& a, int grid, int smem, int n_int, int red_chunks, int prefetch, int* err,
                     void* stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kDIThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<DIArgs*>(&a), &n_int, &err};
  return (int)cudaLaunchKernelExC(&cfg, pick_step1(kind, red_chunks, prefetch), args);
}

// The accumulate and solve launches of an iteration go out with programmatic stream serialization
// (each kernel waits for its predecessor with griddepcontrol.wait before touching its data), so a
// launch is scheduled while the previous one drains.  GAINCAL_PDL=0 turns it off.
static bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("GAINCAL_PDL");
    return !(v && atoi(v) == 0);
  }();
  return on;
}

static cudaError_t launch_dep(const void* f, int grid, size_t smem, cudaStream_t s, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kDIThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, f, args);
}

static cudaError_t launch_msolve(int kind, const DIArgs& a, int n_int, cudaStream_t s) {
  int n = n_int;
  void* args[] = {const_cast<DIArgs*>(&a), &n};
  const int g2 = n_int < kSolveGrid ? n_int : kSolveGrid;  // CTAs loop over the intervals
  const size_t sm2 = sizeof(float) * (size_t)a.na_max * (kind == 0 ? 3 : 12);
  const void* f = kind == 0 ? (const void*)&di_msolve_kernel<ScalarMom> : (const void*)&di_msolve_kernel<JonesMom>;
  return launch_dep(f, g2, sm2, s, args);
}

int di_launch_msolve(int kind, const DIArgs& a, int n_int, void* stream) {
  return (int)launch_msolve(kind, a, n_int, (cudaStream_t)stream);
}

int di_launch_mstep(int kind, const DIArgs& a, int grid, int smem, int n_int, int red_chunks, int prefetch,
                    void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  void* args[] = {const_cast<DIArgs*>(&a)};
  cudaError_t e = launch_dep(pick_acc(kind, red_chunks, prefetch), grid, (size_t)smem, s, args);
  if (e != cudaSuccess) return (int)e;
  return (int)launch_msolve(kind, a, n_int, s);
}

int di_launch_macc(int kind, const DIArgs& a, int grid, int smem, int red_chunks, int prefetch, void* stream) {
  void* args[] = {const_cast<DIArgs*>(&a)};
  return (int)launch_dep(pick_acc(kind, red_chunks, prefetch), grid, (size_t)smem, (cudaStream_t)stream, args);
}

int di_launch_msum(int kind, const DIArgs& a, int i_lo, int n, float* tot_out, double* e_out, void* stream) {
  if (n <= 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const int g2 = n < 4096 ? n : 4096;
  const size_t sm2 = sizeof(float) * (size_t)a.na_max * (kind == 0 ? 3 : 12);
  if (kind == 0) di_msum_kernel<ScalarMom><<<g2, kDIThreads, sm2, s>>>(a, i_lo, n, tot_out, e_out);
  else di_msum_kernel<JonesMom><<<g2, kDIThreads, sm2, s>>>(a, i_lo, n, tot_out, e_out);
  return (int)cudaGetLastError();
}

// After the init launch: intervals from i_hold on wait (inactive, not in work list 1); every
// interval starts its own count at 0 and has no gate yet.  Items are numbered by interval, so the
// items of the first i_hold intervals are 0 .. first_item[i_hold] - 1.
__global__ void di_wf_hold_kernel(const DIArgs a, int n_int, int i_hold, int n_active0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *a.n_active = n_active0;
    a.icount[1] = i_hold < n_int ? a.first_item[i_hold] : a.n_items;
  }
  if (i < n_int) {
    a.k0[i] = 0;
    a.gate[i] = 0;
    if (i >= i_hold) a.active[i] = 0;
  }
}

int di_launch_wf_hold(const DIArgs& a, int n_int, int i_hold, int n_active0, void* stream) {
  const int g = (n_int + 255) / 256 > 0 ? (n_int + 255) / 256 : 1;
  di_wf_hold_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(a, n_int, i_hold, n_active0);
  return (int)cudaGetLastError();
}

// Intervals [i_lo, i_lo + n) join the running iteration: they take iteration *kbase + 1 as their
// first (k0 = *kbase) and their items go to that iteration's work list.
__global__ void di_wf_activate_kernel(const DIArgs a, int i_lo, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = i_lo + j;
  const int kb = *a.kbase;
  const int cur = (kb + 1) % 3;
  a.k0[i] = kb;
  a.gate[i] = 0;
  a.iters[i] = 0;
  a.counters[i] = 0;
  if ((int64_t)a.n_samp[i] * a.n_bl[i] == 0) {
    a.status[i] = GC_ST_NODATA;
    return;
  }
  a.status[i] = GC_ST_NOT_CONVERGED;
  a.active[i] = 1;
  const int nch = a.n_chunks[i], fi = a.first_item[i];
  const int base = atomicAdd(&a.icount[cur], nch);
  for (int c = 0; c < nch; ++c) a.ilist[(size_t)cur * a.n_items + base + c] = fi + c;
  atomicAdd(a.n_active, 1);
}

int di_launch_wf_activate(const DIArgs& a, int i_lo, int n, void* stream) {
  if (n <= 0) return 0;
  di_wf_activate_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(a, i_lo, n);
  return (int)cudaGetLastError();
}

__global__ void di_advance_kernel(int* kbase, int by) { *kbase += by; }

int di_launch_advance(int* kbase, int by, void* stream) {
  di_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(kbase, by);
  return (int)cudaGetLastError();
}

int di_launch_maux(int kind, const float* gains, float* aux, int n_gain, void* stream) {
  if (n_gain <= 0) return 0;
  const int g = (n_gain + 255) / 256;
  if (kind == 0) di_maux_kernel<ScalarMom><<<g, 256, 0, (cudaStream_t)stream>>>(gains, aux, n_gain);
  else di_maux_kernel<JonesMom><<<g, 256, 0, (cudaStream_t)stream>>>(gains, aux, n_gain);
  return (int)cudaGetLastError();
}

int di_smem_bytes(int kind, int dtype, int na_max) {
  size_t e;
  if (kind == 0) e = dtype == GC_DTYPE_C64 ? di_smem_elems<float, ScalarKind<float>>(na_max) * 4 : di_smem_elems<double, ScalarKind<double>>(na_max) * 8;
  else e = dtype == GC_DTYPE_C64 ? di_smem_elems<float, JonesKind<float>>(na_max) * 4 : di_smem_elems<double, JonesKind<double>>(na_max) * 8;
  return (int)e;
}

int di_max_blocks_per_sm(int kind, int dtype, int acc_only, int smem, int* out) {
  const void* f = pick(kind, dtype, acc_only);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, kDIThreads, smem);
}

int di_launch_iter(int kind, int dtype, int acc_only, const DIArgs& a, int grid, int smem, void* stream) {
  const void* f = pick(kind, dtype, acc_only);
  void* args[] = {const_cast<DIArgs*>(&a)};
  return (int)cudaLaunchKernel(f, dim3(grid), dim3(kDIThreads), args, (size_t)smem, (cudaStream_t)stream);
}

int di_launch_init(const DIArgs& a, int n_int, int n_active0, void* stream) {
  const int g = (n_int + 255) / 256 > 0 ? (n_int + 255) / 256 : 1;
  di_init_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(a, n_int, n_active0);
  return (int)cudaGetLastError();
}

int di_launch_chi2(int kind, int dtype, const DIArgs& a, double* item_chi2, double* chi2_out, int n_int, int grid,
                   void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0) {
    if (dtype == GC_DTYPE_C64) di_chi2_kernel<float, ScalarKind<float>><<<grid, kDIThreads, 0, s>>>(a, item_chi2);
    else di_chi2_kernel<double, ScalarKind<double>><<<grid, kDIThreads, 0, s>>>(a, item_chi2);
  } else {
    if (dtype == GC_DTYPE_C64) di_chi2_kernel<float, JonesKind<float>><<<grid, kDIThreads, 0, s>>>(a, item_chi2);
    else di_chi2_kernel<double, JonesKind<double>><<<grid, kDIThreads, 0, s>>>(a, item_chi2);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  di_chi2_final_kernel<<<(n_int + 255) / 256, 256, 0, s>>>(a, item_chi2, chi2_out, n_int);
  return (int)cudaGetLastError();
}

}  // namespace gc
