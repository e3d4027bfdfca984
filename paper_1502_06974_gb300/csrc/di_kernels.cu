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

namespace gc {

// ------------------------------------------------------------------------------------------
// Per-kind row arithmetic.  Partial-sum component order (per side):
//   scalar: [Re c, Im c, A]                              c = sum conj(y) d, A = sum |y|^2
//   jones : [C00, C01, C10, C11 (re,im each), H00, H11, Re H01, Im H01]
//           C = sum D Y^H, H = sum Y Y^H
// ------------------------------------------------------------------------------------------
template <typename T>
struct ScalarKind {
  static constexpr int NC = 3;  // components per side
  static constexpr int GW = 2;  // reals per gain
  using G = Cx<T>;
  static GC_DEV G ld_gain(const T* g) { return cx<T>(g[0], g[1]); }
  static GC_DEV void st_gain(T* g, const G& v) { g[0] = v.x; g[1] = v.y; }

  // Row (p, q, s): y = m conj(g_q) feeds antenna p; the conjugate row (q, p) has
  // y_qp = conj(m) conj(g_p) = conj(w) with w = g_p m and d_qp = conj(d).
  static GC_DEV void row(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq, T* pp, T* pq) {
    const Cx<T> d = Vec<T>::ld1(vis + 2 * r);
    const Cx<T> m = Vec<T>::ld1(mod + 2 * r);
    const Cx<T> y = mulc_(m, gq);
    const Cx<T> w = mul_(gp, m);
    pp[0] = fma(y.x, d.x, fma(y.y, d.y, pp[0]));   // conj(y) d
    pp[1] = fma(y.x, d.y, fma(-y.y, d.x, pp[1]));
    pp[2] = fma(y.x, y.x, fma(y.y, y.y, pp[2]));
    pq[0] = fma(w.x, d.x, fma(w.y, d.y, pq[0]));   // w conj(d)
    pq[1] = fma(w.y, d.x, fma(-w.x, d.y, pq[1]));
    pq[2] = fma(w.x, w.x, fma(w.y, w.y, pq[2]));
  }

  // |d - g_p m conj(g_q)|^2
  static GC_DEV T resid2(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq) {
    const Cx<T> d = Vec<T>::ld1(vis + 2 * r);
    const Cx<T> m = Vec<T>::ld1(mod + 2 * r);
    const Cx<T> v = mulc_(mul_(gp, m), gq);
    return abs2_(sub_(d, v));
  }

  // GN gain from the sums; returns false (and leaves out = old) when A is not positive.
  static GC_DEV bool solve(const T* v, const G& old, G& out) {
    const T A = v[2];
    if (!(A > T(0))) { out = old; return false; }
    const T inv = T(1) / A;
    out = cx<T>(v[0] * inv, v[1] * inv);
    return true;
  }
  static GC_DEV G avg(const G& a, const G& b) { return cx<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y + b.y)); }
  static GC_DEV T dist2(const G& a, const G& b) { return abs2_(sub_(a, b)); }
  static GC_DEV T norm2(const G& a) { return abs2_(a); }
  static GC_DEV bool finite(const G& a) { return isfinite(a.x) && isfinite(a.y); }
  static GC_DEV void write_acc(const T* v, T* jhd, T* jhj, int64_t slot) {
    jhd[2 * slot] = v[0]; jhd[2 * slot + 1] = v[1]; jhj[slot] = v[2];
  }
};

template <typename T>
struct JonesKind {
  static constexpr int NC = 12;
  static constexpr int GW = 8;
  using G = M2<T>;
  static GC_DEV G ld_gain(const T* g) {
    G m;
    m.a = cx<T>(g[0], g[1]); m.b = cx<T>(g[2], g[3]); m.c = cx<T>(g[4], g[5]); m.d = cx<T>(g[6], g[7]);
    return m;
  }
  static GC_DEV void st_gain(T* g, const G& m) {
    g[0] = m.a.x; g[1] = m.a.y; g[2] = m.b.x; g[3] = m.b.y;
    g[4] = m.c.x; g[5] = m.c.y; g[6] = m.d.x; g[7] = m.d.y;
  }

  // Row (p, q, s) with Y = M G_q^H feeds antenna p: C_p += D Y^H, H_p += Y Y^H.
  // Its conjugate row (q, p) has Y_qp = M^H G_p^H = W^H with W = G_p M and D_qp = D^H:
  //   C_q += D^H W,  H_q += W^H W.
  static GC_DEV void row(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq, T* pp, T* pq) {
    const M2<T> D = Vec<T>::ld4(vis + 8 * r);
    const M2<T> M = Vec<T>::ld4(mod + 8 * r);
    const M2<T> Y = mmh_(M, gq);
    const M2<T> W = mm_(gp, M);
    // p side
    fmac2(pp[0], pp[1], D.a, Y.a); fmac2(pp[0], pp[1], D.b, Y.b);
    fmac2(pp[2], pp[3], D.a, Y.c); fmac2(pp[2], pp[3], D.b, Y.d);
    fmac2(pp[4], pp[5], D.c, Y.a); fmac2(pp[4], pp[5], D.d, Y.b);
    fmac2(pp[6], pp[7], D.c, Y.c); fmac2(pp[6], pp[7], D.d, Y.d);
    pp[8] += abs2_(Y.a) + abs2_(Y.b);
    pp[9] += abs2_(Y.c) + abs2_(Y.d);
    fmac2(pp[10], pp[11], Y.a, Y.c); fmac2(pp[10], pp[11], Y.b, Y.d);
    // q side
    cfma2(pq[0], pq[1], D.a, W.a); cfma2(pq[0], pq[1], D.c, W.c);
    cfma2(pq[2], pq[3], D.a, W.b); cfma2(pq[2], pq[3], D.c, W.d);
    cfma2(pq[4], pq[5], D.b, W.a); cfma2(pq[4], pq[5], D.d, W.c);
    cfma2(pq[6], pq[7], D.b, W.b); cfma2(pq[6], pq[7], D.d, W.d);
    pq[8] += abs2_(W.a) + abs2_(W.c);
    pq[9] += abs2_(W.b) + abs2_(W.d);
    cfma2(pq[10], pq[11], W.a, W.b); cfma2(pq[10], pq[11], W.c, W.d);
  }

  // ||D - G_p M G_q^H||_F^2
  static GC_DEV T resid2(const T* vis, const T* mod, int64_t r, const G& gp, const G& gq) {
    const M2<T> D = Vec<T>::ld4(vis + 8 * r);
    const M2<T> M = Vec<T>::ld4(mod + 8 * r);
    const M2<T> V = mmh_(mm_(gp, M), gq);
    return abs2_(sub_(D.a, V.a)) + abs2_(sub_(D.b, V.b)) + abs2_(sub_(D.c, V.c)) + abs2_(sub_(D.d, V.d));
  }

  // G = C H^-1 with H = [[h00, h01], [conj h01, h11]]; false when det(H) is not positive.
  static GC_DEV bool solve(const T* v, const G& old, G& out) {
    const T h00 = v[8], h11 = v[9];
    const Cx<T> h01 = cx<T>(v[10], v[11]);
    const T det = h00 * h11 - abs2_(h01);
    if (!(det > T(0)) || !(h00 > T(0))) { out = old; return false; }
    const T inv = T(1) / det;
    const Cx<T> C00 = cx<T>(v[0], v[1]), C01 = cx<T>(v[2], v[3]), C10 = cx<T>(v[4], v[5]), C11 = cx<T>(v[6], v[7]);
    // [C00 C01; C10 C11] [h11 -h01; -conj(h01) h00] / det
    out.a = scale_(sub_(scale_(C00, h11), mulc_(C01, h01)), inv);
    out.b = scale_(sub_(scale_(C01, h00), mul_(C00, h01)), inv);
    out.c = scale_(sub_(scale_(C10, h11), mulc_(C11, h01)), inv);
    out.d = scale_(sub_(scale_(C11, h00), mul_(C10, h01)), inv);
    return true;
  }
  static GC_DEV G avg(const G& x, const G& y) {
    G r;
    r.a = scale_(add_(x.a, y.a), T(0.5)); r.b = scale_(add_(x.b, y.b), T(0.5));
    r.c = scale_(add_(x.c, y.c), T(0.5)); r.d = scale_(add_(x.d, y.d), T(0.5));
    return r;
  }
  static GC_DEV T dist2(const G& x, const G& y) {
    return abs2_(sub_(x.a, y.a)) + abs2_(sub_(x.b, y.b)) + abs2_(sub_(x.c, y.c)) + abs2_(sub_(x.d, y.d));
  }
  static GC_DEV T norm2(const G& x) { return abs2_(x.a) + abs2_(x.b) + abs2_(x.c) + abs2_(x.d); }
  static GC_DEV bool finite(const G& x) {
    return isfinite(x.a.x) && isfinite(x.a.y) && isfinite(x.b.x) && isfinite(x.b.y) && isfinite(x.c.x) &&
           isfinite(x.c.y) && isfinite(x.d.x) && isfinite(x.d.y);
  }
  static GC_DEV void write_acc(const T* v, T* jhd, T* jhj, int64_t slot) {
    for (int c = 0; c < 8; ++c) jhd[8 * slot + c] = v[c];
    T* h = jhj + 8 * slot;
    h[0] = v[8]; h[1] = 0; h[2] = v[10]; h[3] = v[11];
    h[4] = v[10]; h[5] = -v[11]; h[6] = v[9]; h[7] = 0;
  }
};

// Shared-memory carve-up (elements of T): partials [256][2][NC] | acc [na_max][NC] |
// comp [na_max][NC] | gains [na_max][GW] | new gains [na_max][GW] | reduction buffer [64].
template <typename T, class K>
__host__ __device__ inline size_t di_smem_elems(int na_max) {
  return (size_t)kDIThreads * 2 * K::NC + 2 * (size_t)na_max * K::NC + 2 * (size_t)na_max * K::GW + 64;
}

template <typename T, class K, bool ACC_ONLY>
__global__ void __launch_bounds__(kDIThreads) di_iter_kernel(const DIArgs a) {
  constexpr int NC = K::NC, GW = K::GW, TB = kDIThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* part = reinterpret_cast<T*>(smem_raw);
  T* acc = part + TB * 2 * NC;
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
        T* my = part + tid * 2 * NC;
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

// Per-call state: active flags, statuses, counters.
__global__ void di_init_kernel(const DIArgs a, int n_int, int n_active0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) { *a.n_active = n_active0; a.qhead[0] = 0; a.qhead[1] = 0; }
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
