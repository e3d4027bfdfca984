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

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace gc {

// Shared-memory carve-up (elements of T): partials [256][2 NC + 1] (padded: bank-conflict free) |
// acc [na_max][NC] | comp [na_max][NC] | gains [na_max][GW] | new gains [na_max][GW] |
// reduction buffer [64] | per-antenna auxiliaries [na_max][4] (moment path).
template <typename T, class K>
__host__ __device__ inline size_t di_smem_elems(int na_max) {
  return (size_t)kDIThreads * (2 * K::NC + 1) + 2 * (size_t)na_max * K::NC + 2 * (size_t)na_max * K::GW + 64 +
         4 * (size_t)na_max;
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
  const int k = a.k;
  const T* vis = static_cast<const T*>(a.vis);
  const T* mod = static_cast<const T*>(a.model);
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
          for (int s = sc; s < se; ++s) K::row(vis, mod, rb + (int64_t)s * nb, gp, gq, pp, pq);
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
// Moment-stream iteration: the same per-iteration structure as di_iter_kernel, but each item is
// (interval, range of 256-baseline tiles) and each thread turns one baseline's moments (the sample
// sums with the gains factored out, written once by the moment pass) into its p- and q-side
// contributions -- 12 independent float4 loads and 160 FMA per 2x2 baseline per iteration.
// ------------------------------------------------------------------------------------------
template <class MK, bool ACC_ONLY>
__global__ void __launch_bounds__(kDIThreads) di_miter_kernel(const DIArgs a) {
  using K = typename MK::K;
  using G = typename K::G;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, AW = MK::AW, TB = kDIThreads, PS = 2 * NC + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* part = reinterpret_cast<float*>(smem_raw);
  float* acc = part + TB * PS;
  float* cmp = acc + a.na_max * NC;
  float* gs = cmp + a.na_max * NC;
  float* ng = gs + a.na_max * GW;
  float* red = ng + a.na_max * GW;
  float* ax = red + 64;
  __shared__ int s_item, s_last;
  const int tid = threadIdx.x;
  const int k = a.k;
  float* gains = static_cast<float*>(a.gains);

  const int cur = k % 3, nxt = (k + 1) % 3;
  const int* list = a.ilist + (size_t)cur * a.n_items;
  const int n_list = ACC_ONLY ? a.n_items : a.icount[cur];
  if (blockIdx.x == 0 && tid == 0) {
    a.qhead[(k + 1) & 1] = 0;
    if (!ACC_ONLY) a.icount[(k + 2) % 3] = 0;
  }
  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.qhead[k & 1], 1);
    __syncthreads();
    const int slot = s_item;
    __syncthreads();
    if (slot >= n_list) break;
    const int it = ACC_ONLY ? slot : list[slot];
    const int i = a.item_int[it];
    if (!ACC_ONLY && a.active[i] == 0) continue;
    const int nb = a.n_bl[i], na = a.n_ant[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int t0 = a.item_s0[it], t1 = a.item_s1[it];
    const int tab = a.itab[i];
    const int nat = a.tab_nant[tab];
    const int* csr = a.csr_off + a.tab_base[tab];
    const float* mom = a.moments + a.mom_off[i] * NM;
    for (int x = tid; x < na * GW; x += TB) gs[x] = gains[go * GW + x];
    for (int x = tid; x < na * NC; x += TB) { acc[x] = 0.f; cmp[x] = 0.f; }
    __syncthreads();
    for (int x = tid; x < na; x += TB) MK::aux(K::ld_gain(gs + x * GW), ax + x * AW);
    __syncthreads();
    for (int t = t0; t < t1; ++t) {
      const int b = t * TB + tid;
      if (b < nb) {
        float m[NM];
        const float4* src = reinterpret_cast<const float4*>(mom + (int64_t)b * NM);
#pragma unroll
        for (int c = 0; c < NM / 4; ++c) {
          const float4 v = __ldg(src + c);
          m[4 * c] = v.x; m[4 * c + 1] = v.y; m[4 * c + 2] = v.z; m[4 * c + 3] = v.w;
        }
        const int p = a.ant1[bo + b], q = a.ant2[bo + b];
        float pp[NC], pq[NC];
        MK::partials(m, K::ld_gain(gs + p * GW), K::ld_gain(gs + q * GW), ax + p * AW, ax + q * AW, pp, pq);
        float* my = part + tid * PS;
#pragma unroll
        for (int c = 0; c < NC; ++c) { my[c] = pp[c]; my[NC + c] = pq[c]; }
      }
      __syncthreads();
      const int* off = csr + t * (nat + 1);
      for (int x = tid; x < nat * NC; x += TB) {
        const int an = x / NC, c = x - an * NC;
        float s = 0.f;
        const int e1 = __ldg(off + an + 1);
        for (int e = __ldg(off + an); e < e1; ++e) s += part[__ldg(a.csr_ent + e) + c];
        kahan_add(acc[x], cmp[x], s);
      }
      __syncthreads();
    }
    bool finish = true;
    const int nch = a.n_chunks[i];
    if (nch > 1) {
      float* scr = static_cast<float*>(a.scratch) + a.item_scr[it];
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
          float s = 0.f, c = 0.f;
          for (int j = 0; j < nch; ++j)
            kahan_add(s, c, __ldcg(static_cast<const float*>(a.scratch) + a.item_scr[fi + j] + x));
          acc[x] = s;
          cmp[x] = c;
        }
        if (tid == 0) a.counters[i] = 0;
        __syncthreads();
      }
    }
    if (!finish) continue;
    if (ACC_ONLY) {
      float* jhd = static_cast<float*>(a.jhd_out);
      float* jhj = static_cast<float*>(a.jhj_out);
      for (int an = tid; an < na; an += TB) {
        float v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = acc[an * NC + c] - cmp[an * NC + c];
        K::write_acc(v, jhd, jhj, go + an);
      }
      __syncthreads();
      continue;
    }
    float d2 = 0.f, n2 = 0.f;
    int sing = 0, nonfin = 0;
    const bool gn_step = (a.schedule == GC_SCHED_GN) || (k & 1);
    for (int an = tid; an < na; an += TB) {
      float v[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = acc[an * NC + c] - cmp[an * NC + c];
      const G old = K::ld_gain(gs + an * GW);
      G g;
      if (!K::solve(v, old, g)) sing = 1;
      const G nw = gn_step ? g : K::avg(old, g);
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
      } else {  // still iterating: its items go to the next iteration's list
        const int base = atomicAdd(&a.icount[nxt], nch);
        const int fi = a.first_item[i];
        for (int j = 0; j < nch; ++j) a.ilist[(size_t)nxt * a.n_items + base + j] = fi + j;
      }
    }
    __syncthreads();
  }
}

// Per-call state: active flags, statuses, counters.
__global__ void di_init_kernel(const DIArgs a, int n_int, int n_active0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *a.n_active = n_active0;
    a.qhead[0] = 0;
    a.qhead[1] = 0;
    if (a.icount) { a.icount[1] = a.n_items; a.icount[2] = 0; a.icount[0] = 0; }
  }
  if (a.ilist)  // iteration 1 takes every item
    for (int j = i; j < a.n_items; j += gridDim.x * blockDim.x) a.ilist[(size_t)1 * a.n_items + j] = j;
  if (i < n_int) {
    const int64_t rows = (int64_t)a.n_samp[i] * a.n_bl[i];
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
      kahan_add(s, c, K::resid2(vis, mod, r0 + (int64_t)(s0 + sl) * nb + b, gp, gq));
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

static void* pick_m(int kind, int acc_only) {
  if (kind == 0)
    return acc_only ? reinterpret_cast<void*>(&di_miter_kernel<ScalarMom, true>)
                    : reinterpret_cast<void*>(&di_miter_kernel<ScalarMom, false>);
  return acc_only ? reinterpret_cast<void*>(&di_miter_kernel<JonesMom, true>)
                  : reinterpret_cast<void*>(&di_miter_kernel<JonesMom, false>);
}

int di_m_max_blocks_per_sm(int kind, int acc_only, int smem, int* out) {
  const void* f = pick_m(kind, acc_only);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, kDIThreads, smem);
}

int di_launch_miter(int kind, int acc_only, const DIArgs& a, int grid, int smem, void* stream) {
  const void* f = pick_m(kind, acc_only);
  void* args[] = {const_cast<DIArgs*>(&a)};
  return (int)cudaLaunchKernel(f, dim3(grid), dim3(kDIThreads), args, (size_t)smem, (cudaStream_t)stream);
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
