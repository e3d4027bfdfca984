// Direction-independent StefCal with the sample sums taken once and the iterations kept on chip.
//
// Within a solution interval the gains do not depend on the sample index, so they factor out of
// the sample sums (the observation of Sect. 3.2.1 for the DD terms X^(cd), applied here to the DI
// blocks).  With vec stacking columns and vec(A X B) = (B^T kron A) vec X (App. B):
//   2x2, stored row (p, q):
//     sum_s D Y^H   = sum_s D G_q M^H           -> vec: P_pq vec(G_q),   P_pq = sum_s conj(M) kron D
//     sum_s Y Y^H   = sum_s M (G_q^H G_q) M^H   -> R_pq applied to A_q = G_q^H G_q
//   conjugate row (q, p) (D_qp = D^H, M_qp = M^H):
//     sum_s D^H G_p M          -> vec: P_pq^H vec(G_p)
//     sum_s M^H (G_p^H G_p) M  -> R'_pq applied to A_p
//   where R_pq is the real 4x4 matrix of A -> sum_s M A M^H on Hermitian A in the coordinates
//   (a00, a11, Re a01, Im a01), and R' = W^-1 R^T W, W = diag(1, 1, 2, 2), is its adjoint.
//   scalar: sum conj(y) d = g_q sum conj(m) d,  sum |y|^2 = |g_q|^2 sum |m|^2 (conjugate row: conj).
// These are exactly the sums of eq. JHJ:pol / eq. JHJ:DI:tf and the J^H d of eq. ghat, reordered.
//
// di_moment_kernel: one pass over vis and model (HBM-bound), per-baseline moments to global.
// di_resident_kernel: a persistent grid of thread-block clusters.  Each cluster pulls intervals
//   from an atomic queue; its CTAs split the interval's baselines and keep their moments in
//   registers.  Per iteration each CTA reduces its baselines' contributions into per-antenna sums
//   (fixed-order slot lists), the cluster exchanges those sums through distributed shared memory,
//   and every CTA then solves all antennas redundantly (identical arithmetic, so identical gains
//   in every CTA), applies the schedule and tests convergence.  The whole iteration loop of every
//   interval runs inside one launch; the only barriers are cluster and block barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "kinds.cuh"

namespace cg = cooperative_groups;

namespace gc {

constexpr int kResThreads = 512;
constexpr int kMomBl2 = 32, kMomLanes2 = 8;  // moment CTA: 32 baselines x 8 sample lanes

struct MomArgs {
  const float* vis;
  const float* model;
  float* moments;
  const int64_t* row_off;
  const int64_t* mom_off;  // per interval, in baselines
  const int32_t* n_samp;
  const int32_t* n_bl;
  const int32_t* item_int;
  const int32_t* item_tile;
  int32_t n_items;
  const float* weights;  // per-row weights or NULL (Sect. 2.4)
};

template <class MK>
__global__ void __launch_bounds__(kMomBl2 * kMomLanes2) di_moment_kernel(const MomArgs a) {
  constexpr int NM = MK::NM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* part = reinterpret_cast<float*>(smem_raw);  // [lanes][32][NM]
  const int it = blockIdx.x;
  if (it >= a.n_items) return;
  const int i = a.item_int[it], tile = a.item_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i];
  const int bl = threadIdx.x % kMomBl2, lane = threadIdx.x / kMomBl2;
  const int b = tile * kMomBl2 + bl;
  const int chunk = (ns + kMomLanes2 - 1) / kMomLanes2;
  const int s0 = lane * chunk, s1 = min(ns, s0 + chunk);
  float m[NM];
#pragma unroll
  for (int c = 0; c < NM; ++c) m[c] = 0.f;
  if (b < nb) {
    const int64_t r0 = a.row_off[i] + b;
    for (int s = s0; s < s1; ++s) {
      const int64_t r = r0 + (int64_t)s * nb;
      MK::accum(a.vis, a.model, r, m, row_sw(a.weights, r));
    }
  }
  float* my = part + ((size_t)lane * kMomBl2 + bl) * NM;
#pragma unroll
  for (int c = 0; c < NM; ++c) my[c] = m[c];
  __syncthreads();
  // tiled layout [NM / 4][256][4] (see mom_index): consecutive threads write consecutive words
  const int nbt = min(kMomBl2, nb - tile * kMomBl2);
  for (int x = threadIdx.x; x < nbt * NM; x += blockDim.x) {
    const int q = x >> 2, blx = q % nbt, c = (q / nbt) * 4 + (x & 3);
    float s = 0.f, cc = 0.f;
    for (int l = 0; l < kMomLanes2; ++l) kahan_add(s, cc, part[((size_t)l * kMomBl2 + blx) * NM + c]);
    a.moments[mom_index(a.mom_off[i], tile * kMomBl2 + blx, c, NM)] = s - cc;
  }
}

// di_moment_direct_kernel: the same moments for intervals with few samples per baseline (at most
// kDirectSamp): one warp per 32-baseline item, one thread per baseline summing its samples in
// order (plain FP32 sums of at most kDirectSamp terms), written straight into the tiled layout.
// With 8 sample lanes and a shared-memory reduction, a 4-sample interval would leave half the
// threads idle and spend most of its time in the reduction.
constexpr int kDirectSamp = 16;
template <class MK>
__global__ void __launch_bounds__(256, 3) di_moment_direct_kernel(const MomArgs a) {
  constexpr int NM = MK::NM;
  const int it = blockIdx.x * 8 + (int)(threadIdx.x >> 5);
  if (it >= a.n_items) return;
  const int i = a.item_int[it], tile = a.item_tile[it];
  const int nb = a.n_bl[i], ns = a.n_samp[i];
  const int b = tile * kMomBl2 + (int)(threadIdx.x & 31);
  if (b >= nb) return;
  float m[NM];
#pragma unroll
  for (int c = 0; c < NM; ++c) m[c] = 0.f;
  const int64_t r0 = a.row_off[i] + b;
#pragma unroll 2
  for (int s = 0; s < ns; ++s) {
    const int64_t r = r0 + (int64_t)s * nb;
    MK::accum(a.vis, a.model, r, m, row_sw(a.weights, r));
  }
  float4* out = reinterpret_cast<float4*>(a.moments);
#pragma unroll
  for (int g = 0; g < NM / 4; ++g)
    out[mom_index(a.mom_off[i], b, 4 * g, NM) / 4] = make_float4(m[4 * g], m[4 * g + 1], m[4 * g + 2], m[4 * g + 3]);
}

// ------------------------------------------------------------------------------------ resident
struct ResArgs {
  const float* moments;
  float* gains;
  const int64_t* mom_off;
  const int32_t* n_bl;
  const int32_t* n_ant;
  const int32_t* gain_off;
  const int32_t* bl_off;
  const int32_t* ant1;
  const int32_t* ant2;
  const int32_t* order;     // intervals in queue order
  const int32_t* itab;      // per interval: baseline table
  const int32_t* tab_soff;  // per (table, rank): offset of the slot-list offsets in soff
  const int32_t* soff;      // per (table, rank): nat + 1 offsets into sent (absolute)
  const int32_t* sent;      // slot-list entries: side * NC * S + local baseline
  const int32_t* tab_nat;
  int32_t* iters;
  int32_t* status;
  int32_t* queue;
  int32_t n_int;
  int32_t na_max;
  int32_t max_slots;  // largest per-rank slot-list length
  double tol;
  int32_t max_iter;
  int32_t schedule;
};

template <class MK>
__global__ void __launch_bounds__(kResThreads, 1) di_resident_kernel(const ResArgs a) {
  using K = typename MK::K;
  using G = typename K::G;
  constexpr int NC = K::NC, GW = K::GW, NM = MK::NM, AW = MK::AW, BPT = MK::BPT, T = kResThreads;
  constexpr int PS = 2 * NC + 1;  // padded partial-sum stride per slot (bank-conflict free)
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), C = (int)cluster.num_blocks();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* part = reinterpret_cast<float*>(smem_raw);        // [T * BPT][PS]
  float* acc = part + T * BPT * PS;                        // [2 parity][C ranks][na_max][NC]
  float* gsb = acc + 2 * C * a.na_max * NC;                // [2 parity][na_max][GW]
  float* axb = gsb + 2 * a.na_max * GW;                    // [2 parity][na_max][AW]
  int* sl_off = reinterpret_cast<int*>(axb + 2 * a.na_max * AW);  // [na_max + 1]
  int* sl_ent = sl_off + a.na_max + 1;                     // [max_slots]
  __shared__ int s_idx;
  __shared__ double red[96];
  const int tid = threadIdx.x;

  for (;;) {
    if (rank == 0 && tid == 0) {
      const int v = atomicAdd(a.queue, 1);
      for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&s_idx, r) = v;
    }
    cluster.sync();
    const int qi = s_idx;
    if (qi >= a.n_int) break;
    const int i = a.order[qi];
    const int nb = a.n_bl[i], na = a.n_ant[i], bo = a.bl_off[i];
    const int64_t go = a.gain_off[i];
    const int per = (nb + C - 1) / C;
    const int lb0 = rank * per, lbn = max(0, min(nb, lb0 + per) - lb0);
    const int tab = a.itab[i], nat = a.tab_nat[tab];
    const int so = a.tab_soff[tab * C + rank];
    for (int x = tid; x <= nat; x += T) sl_off[x] = a.soff[so + x] - a.soff[so];
    const int e0 = a.soff[so], ne = a.soff[so + nat] - e0;
    for (int x = tid; x < ne; x += T) sl_ent[x] = a.sent[e0 + x];
    for (int x = tid; x < na * GW; x += T) gsb[x] = a.gains[go * GW + x];
    float mom[BPT][NM];
    int pa[BPT], qa[BPT];
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      const int lb = j * T + tid;
      pa[j] = qa[j] = 0;
      if (lb < lbn) {
        const int b = lb0 + lb;
        pa[j] = a.ant1[bo + b];
        qa[j] = a.ant2[bo + b];
#pragma unroll
        for (int c = 0; c < NM; ++c) mom[j][c] = __ldcs(a.moments + mom_index(a.mom_off[i], b, c, NM));
      } else {
#pragma unroll
        for (int c = 0; c < NM; ++c) mom[j][c] = 0.f;
      }
    }
    __syncthreads();
    for (int x = tid; x < na; x += T) MK::aux(K::ld_gain(gsb + x * GW), axb + x * AW);
    __syncthreads();

    int k = 1, st = -1, sing = 0, cur = 0;
    for (;; ++k) {
      const float* gs = gsb + cur * a.na_max * GW;
      const float* ax = axb + cur * a.na_max * AW;
      // (A) per-baseline contributions of this CTA's baselines
#pragma unroll
      for (int j = 0; j < BPT; ++j) {
        const int lb = j * T + tid;
        if (lb < lbn) {
          float pp[NC], pq[NC];
          MK::partials(mom[j], K::ld_gain(gs + pa[j] * GW), K::ld_gain(gs + qa[j] * GW), ax + pa[j] * AW,
                       ax + qa[j] * AW, pp, pq);
          float* dst = part + lb * PS;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            dst[c] = pp[c];
            dst[NC + c] = pq[c];
          }
        }
      }
      __syncthreads();
      // (B) fixed-order sums into per-antenna partials, pushed into every CTA's slot for this rank
      float* accp = acc + (size_t)(k & 1) * C * a.na_max * NC;
      for (int x = tid; x < na * NC; x += T) {
        const int an = x / NC, c = x - an * NC;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
        if (an < nat) {
          const int ea = sl_off[an], eb = sl_off[an + 1], em = (ea + eb) >> 1;
          for (int e = ea, f = em; e < em || f < eb; ++e, ++f) {  // two independent chains
            if (e < em) kahan_add(s0, c0, part[sl_ent[e] + c]);
            if (f < eb) kahan_add(s1, c1, part[sl_ent[f] + c]);
          }
        }
        const float v = (s0 - c0) + (s1 - c1);
        for (int r = 0; r < C; ++r) *cluster.map_shared_rank(accp + ((size_t)rank * a.na_max * NC + x), r) = v;
      }
      cluster.sync();
      // (C) totals in rank order, update, schedule, convergence -- identical in every CTA
      const bool gn_step = (a.schedule == GC_SCHED_GN) || (k & 1);
      FF d2{0.f, 0.f}, n2{0.f, 0.f};
      int sg = 0, nonfin = 0;
      float* gn_out = gsb + (cur ^ 1) * a.na_max * GW;
      float* ax_out = axb + (cur ^ 1) * a.na_max * AW;
      for (int an = tid; an < na; an += T) {
        float v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = 0.f;
        for (int r = 0; r < C; ++r) {
          const float* src = accp + ((size_t)r * a.na_max + an) * NC;
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] += src[c];
        }
        const G old = K::ld_gain(gs + an * GW);
        G g;
        if (!K::solve(v, old, g)) sg = 1;
        const G nw = gn_step ? g : K::avg(old, g);
        d2 = ff_add_f(d2, K::dist2(nw, old));
        n2 = ff_add_f(n2, K::norm2(nw));
        if (!K::finite(nw)) nonfin = 1;
        K::st_gain(gn_out + an * GW, nw);
        MK::aux(nw, ax_out + an * AW);
      }
      block_reduce_step_ff(d2, n2, sg, nonfin, reinterpret_cast<float*>(red), (int)blockDim.x);
      sing = sg;
      if (nonfin) { st = GC_ST_NONFINITE; break; }
      cur ^= 1;
      if (ff_value(d2) <= a.tol * a.tol * ff_value(n2)) { st = GC_ST_OK; break; }
      if (k >= a.max_iter) { st = GC_ST_NOT_CONVERGED; break; }
    }
    if (rank == 0) {
      const float* gs = gsb + cur * a.na_max * GW;
      for (int x = tid; x < na * GW; x += T) a.gains[go * GW + x] = gs[x];
      if (tid == 0) {
        a.iters[i] = k;
        a.status[i] = st | (sing ? GC_ST_SINGULAR_FLAG : 0);
      }
    }
    __syncthreads();
  }
}

// chi^2 per moment item (interval, 32 baselines) over all samples.
template <class MK>
__global__ void __launch_bounds__(256) di_res_chi2_kernel(const float* vis, const float* model, const float* gains,
                                                          const int64_t* row_off, const int32_t* n_samp,
                                                          const int32_t* n_bl, const int32_t* bl_off,
                                                          const int32_t* gain_off, const int32_t* ant1,
                                                          const int32_t* ant2, const int32_t* item_int,
                                                          const int32_t* item_tile, int n_items, double* item_chi2,
                                                          const float* weights) {
  using K = typename MK::K;
  __shared__ double red[64];
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int i = item_int[it], tile = item_tile[it];
  const int nb = n_bl[i], ns = n_samp[i], bo = bl_off[i];
  const int64_t go = gain_off[i];
  const int nbt = min(kMomBl2, nb - tile * kMomBl2);
  float s = 0.f, c = 0.f;
  for (int u = threadIdx.x; u < nbt * ns; u += blockDim.x) {
    const int sl = u / nbt, b = tile * kMomBl2 + (u - sl * nbt);
    const int p = ant1[bo + b], q = ant2[bo + b];
    const int64_t r = row_off[i] + (int64_t)sl * nb + b;
    kahan_add(s, c, row_w(weights, r) * K::resid2(vis, model, r, K::ld_gain(gains + (go + p) * K::GW),
                                                  K::ld_gain(gains + (go + q) * K::GW)));
  }
  const double tot = block_sum<double>((double)s - (double)c, red);
  if (threadIdx.x == 0) item_chi2[it] = tot;
}

__global__ void res_chi2_final(const int32_t* first, const int32_t* count, const double* item_chi2, double* out,
                               int n_int) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_int) return;
  double s = 0.0;
  for (int j = 0; j < count[i]; ++j) s += item_chi2[first[i] + j];
  out[i] = s;
}

__global__ void res_init(int32_t* iters, int32_t* status, int32_t* queue, const int32_t* n_samp, const int32_t* n_bl,
                         int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *queue = 0;
  if (i < n) {
    iters[i] = 0;
    status[i] = ((int64_t)n_samp[i] * n_bl[i] > 0) ? GC_ST_NOT_CONVERGED : GC_ST_NODATA;
  }
}

// ------------------------------------------------------------------------------------ host side
extern std::atomic<long long> g_launches;
int ws_get(const char* name, size_t bytes, void** out);
int set_cuda_error(cudaError_t e, const char* what);
int validate_layout(const gc_layout* L, int n_dir_max);
uint64_t layout_hash(const gc_layout* L, uint64_t salt);
void profile_record(double iter_ms, int64_t launches, int64_t row_iters, double moment_ms, int64_t bl_iters, int path);

#define RS_CUDA(call)                                             \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return set_cuda_error(e__, #call);    \
  } while (0)

struct ResPlan {
  uint64_t key = 0;
  void* dev = nullptr;
  size_t dev_bytes = 0;
  int n_int = 0, n_items = 0, na_max = 1, C = 1, max_slots = 1, grid = 0, smem = 0, msmem = 0;
  int64_t n_mom_bl = 0;  // total baselines (moment rows)
  MomArgs m{};
  ResArgs r{};
  int32_t* chi2_first = nullptr;
  int32_t* chi2_count = nullptr;
  double* chi2_items = nullptr;
  double* chi2_out = nullptr;
  const int32_t* n_samp = nullptr;
  const int64_t* row_off = nullptr;
};
static ResPlan g_res[2];

template <class MK>
static int res_smem(int na_max, int max_slots, int C) {
  using K = typename MK::K;
  return (int)(sizeof(float) * ((2 * K::NC + 1) * kResThreads * MK::BPT + 2 * (size_t)C * na_max * K::NC +
                                2 * (size_t)na_max * K::GW + 2 * (size_t)na_max * MK::AW) +
               sizeof(int) * ((size_t)na_max + 1 + max_slots) + 16);
}

// Can the resident path take this layout?  (cluster of <= 8 CTAs, all moments in registers)
int res_supported(int kind, const gc_layout* L) {
  const int bpt = kind == 0 ? ScalarMom::BPT : JonesMom::BPT;
  for (int i = 0; i < L->n_intervals; ++i) {
    if (L->n_bl[i] > 8 * kResThreads * bpt) return 0;
    if (L->n_ant[i] > 256) return 0;
  }
  return 1;
}

template <class MK>
static int build_res_plan(int kind, const gc_layout* L, ResPlan& P, cudaStream_t s) {
  constexpr int NC = MK::K::NC;
  const int n = L->n_intervals;
  const int cap = kResThreads * MK::BPT;
  int nb_max = 0, na_max = 1;
  for (int i = 0; i < n; ++i) {
    nb_max = std::max(nb_max, (int)L->n_bl[i]);
    na_max = std::max(na_max, (int)L->n_ant[i]);
  }
  int C = 1;
  while (C * cap < nb_max) C *= 2;
  if (C > 8) return GC_ERR_LIMIT;
  const char* cenv = getenv("GAINCAL_CLUSTER");
  if (cenv) {
    const int want = atoi(cenv);
    if (want >= C && want <= 8 && (want & (want - 1)) == 0) C = want;
  }
  // tables and per-(table, rank) slot lists
  std::map<std::pair<int, int>, int> tabs;
  std::vector<int> itab(n), tab_nat, tab_soff, soff, sent;
  int max_slots = 1;
  for (int i = 0; i < n; ++i) {
    auto key = std::make_pair((int)L->bl_off[i], (int)L->n_bl[i]);
    auto f = tabs.find(key);
    if (f != tabs.end()) { itab[i] = f->second; continue; }
    const int t = (int)tab_nat.size();
    tabs[key] = t;
    itab[i] = t;
    const int bo = key.first, nb = key.second;
    int nat = 0;
    for (int b = 0; b < nb; ++b) nat = std::max(nat, std::max(L->ant1[bo + b], L->ant2[bo + b]) + 1);
    tab_nat.push_back(nat);
    const int per = (nb + C - 1) / C;
    for (int r = 0; r < C; ++r) {
      tab_soff.push_back((int)soff.size());
      const int lb0 = r * per, lbn = std::max(0, std::min(nb, lb0 + per) - lb0);
      std::vector<std::vector<int>> lists(nat);
      for (int lb = 0; lb < lbn; ++lb) {
        lists[L->ant1[bo + lb0 + lb]].push_back(lb * (2 * NC + 1));
        lists[L->ant2[bo + lb0 + lb]].push_back(lb * (2 * NC + 1) + NC);
      }
      const int base = (int)sent.size();
      for (int an = 0; an < nat; ++an) {
        soff.push_back((int)sent.size());
        sent.insert(sent.end(), lists[an].begin(), lists[an].end());
      }
      soff.push_back((int)sent.size());
      max_slots = std::max(max_slots, (int)sent.size() - base);
    }
  }
  if (sent.empty()) sent.push_back(0);
  // moment items and offsets; queue order: most rows first
  std::vector<int64_t> mom_off(n);
  std::vector<int> mint, mtile, cfirst(n), ccount(n), order(n);
  int64_t mo = 0;
  for (int i = 0; i < n; ++i) {
    mom_off[i] = mo;
    mo += (int64_t)(L->n_bl[i] + kMomTile - 1) / kMomTile * kMomTile;
    cfirst[i] = (int)mint.size();
    if ((int64_t)L->n_bl[i] * L->n_samp[i] > 0)
      for (int t = 0; t < (L->n_bl[i] + kMomBl2 - 1) / kMomBl2; ++t) { mint.push_back(i); mtile.push_back(t); }
    ccount[i] = (int)mint.size() - cfirst[i];
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (int64_t)L->n_bl[x] * L->n_samp[x] > (int64_t)L->n_bl[y] * L->n_samp[y];
  });
  // intervals without rows are not queued
  int nq = 0;
  for (int i = 0; i < n; ++i)
    if ((int64_t)L->n_bl[order[i]] * L->n_samp[order[i]] > 0) order[nq++] = order[i];
  if (mint.empty()) { mint.push_back(0); mtile.push_back(0); }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts;
  size_t off = 0;
  auto add = [&](const void* src, size_t bytes) { parts.push_back({src, bytes, off}); off += al(bytes ? bytes : 1); return parts.size() - 1; };
  const size_t p_row_off = add(L->row_off, (size_t)n * 8), p_mom_off = add(mom_off.data(), (size_t)n * 8);
  const size_t p_n_samp = add(L->n_samp, (size_t)n * 4), p_n_bl = add(L->n_bl, (size_t)n * 4);
  const size_t p_n_ant = add(L->n_ant, (size_t)n * 4), p_gain_off = add(L->gain_off, (size_t)n * 4);
  const size_t p_bl_off = add(L->bl_off, (size_t)n * 4);
  const size_t p_ant1 = add(L->ant1, (size_t)L->n_bl_table * 4), p_ant2 = add(L->ant2, (size_t)L->n_bl_table * 4);
  const size_t p_order = add(order.data(), (size_t)n * 4), p_itab = add(itab.data(), (size_t)n * 4);
  const size_t p_tsoff = add(tab_soff.data(), tab_soff.size() * 4), p_soff = add(soff.data(), soff.size() * 4);
  const size_t p_sent = add(sent.data(), sent.size() * 4), p_tnat = add(tab_nat.data(), tab_nat.size() * 4);
  const size_t p_mint = add(mint.data(), mint.size() * 4), p_mtile = add(mtile.data(), mtile.size() * 4);
  const size_t p_cfirst = add(cfirst.data(), (size_t)n * 4), p_ccount = add(ccount.data(), (size_t)n * 4);
  const size_t p_iters = add(nullptr, (size_t)n * 4), p_status = add(nullptr, (size_t)n * 4);
  const size_t p_misc = add(nullptr, 64), p_chi2 = add(nullptr, mint.size() * 8), p_chi2o = add(nullptr, (size_t)n * 8);
  const size_t total = off;
  std::vector<unsigned char> host(total, 0);
  for (auto& pt : parts)
    if (pt.src && pt.bytes) memcpy(host.data() + pt.off, pt.src, pt.bytes);
  if (P.dev && P.dev_bytes < total) { cudaFree(P.dev); P.dev = nullptr; P.dev_bytes = 0; }
  if (!P.dev) { RS_CUDA(cudaMalloc(&P.dev, total)); P.dev_bytes = total; }
  RS_CUDA(cudaMemcpyAsync(P.dev, host.data(), total, cudaMemcpyHostToDevice, s));
  RS_CUDA(cudaStreamSynchronize(s));
  unsigned char* d = static_cast<unsigned char*>(P.dev);
  auto at = [&](size_t idx) { return (void*)(d + parts[idx].off); };
  P.m = MomArgs{};
  P.m.row_off = (const int64_t*)at(p_row_off);
  P.m.mom_off = (const int64_t*)at(p_mom_off);
  P.m.n_samp = (const int32_t*)at(p_n_samp);
  P.m.n_bl = (const int32_t*)at(p_n_bl);
  P.m.item_int = (const int32_t*)at(p_mint);
  P.m.item_tile = (const int32_t*)at(p_mtile);
  P.m.n_items = (int)(mo > 0 && nq > 0 ? mint.size() : 0);
  P.r = ResArgs{};
  P.r.mom_off = P.m.mom_off;
  P.r.n_bl = P.m.n_bl;
  P.r.n_ant = (const int32_t*)at(p_n_ant);
  P.r.gain_off = (const int32_t*)at(p_gain_off);
  P.r.bl_off = (const int32_t*)at(p_bl_off);
  P.r.ant1 = (const int32_t*)at(p_ant1);
  P.r.ant2 = (const int32_t*)at(p_ant2);
  P.r.order = (const int32_t*)at(p_order);
  P.r.itab = (const int32_t*)at(p_itab);
  P.r.tab_soff = (const int32_t*)at(p_tsoff);
  P.r.soff = (const int32_t*)at(p_soff);
  P.r.sent = (const int32_t*)at(p_sent);
  P.r.tab_nat = (const int32_t*)at(p_tnat);
  P.r.iters = (int32_t*)at(p_iters);
  P.r.status = (int32_t*)at(p_status);
  P.r.queue = (int32_t*)at(p_misc);
  P.r.n_int = nq;
  P.r.na_max = na_max;
  P.r.max_slots = max_slots;
  P.chi2_first = (int32_t*)at(p_cfirst);
  P.chi2_count = (int32_t*)at(p_ccount);
  P.chi2_items = (double*)at(p_chi2);
  P.chi2_out = (double*)at(p_chi2o);
  P.n_samp = P.m.n_samp;
  P.row_off = P.m.row_off;
  P.n_int = n;
  P.n_items = P.m.n_items;
  P.na_max = na_max;
  P.C = C;
  P.max_slots = max_slots;
  P.n_mom_bl = mo;
  P.smem = res_smem<MK>(na_max, max_slots, C);
  P.msmem = (int)(sizeof(float) * kMomLanes2 * kMomBl2 * MK::NM);
  int dev = 0, max_smem = 0;
  RS_CUDA(cudaGetDevice(&dev));
  RS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (P.smem > max_smem) return GC_ERR_LIMIT;
  RS_CUDA(cudaFuncSetAttribute(di_resident_kernel<MK>, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem));
  RS_CUDA(cudaFuncSetAttribute(di_moment_kernel<MK>, cudaFuncAttributeMaxDynamicSharedMemorySize, P.msmem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = P.smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  RS_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, (void*)di_resident_kernel<MK>, &cfg));
  if (nclusters < 1) return GC_ERR_LIMIT;
  const char* genv = getenv("GAINCAL_RES_CLUSTERS");
  if (genv && atoi(genv) > 0 && atoi(genv) < nclusters) nclusters = atoi(genv);
  if (nclusters > nq) nclusters = nq > 0 ? nq : 1;
  P.grid = nclusters * C;
  (void)kind;
  return GC_OK;
}

template <class MK>
static int res_run(ResPlan& P, const void* vis, const void* model, void* gains, const gc_options* opt,
                   cudaStream_t s) {
  void* mom = nullptr;
  int rc;
  if ((rc = ws_get("res_moments", (size_t)(P.n_mom_bl > 0 ? P.n_mom_bl : 1) * MK::NM * sizeof(float), &mom))) return rc;
  P.m.vis = (const float*)vis;
  P.m.model = (const float*)model;
  P.m.moments = (float*)mom;
  P.r.moments = (const float*)mom;
  P.r.gains = (float*)gains;
  P.r.tol = opt->tol;
  P.r.max_iter = opt->max_iter;
  P.r.schedule = opt->schedule;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (opt->profile)
    for (auto& e : ev) RS_CUDA(cudaEventCreate(&e));
  res_init<<<(P.n_int + 255) / 256, 256, 0, s>>>(P.r.iters, P.r.status, P.r.queue, P.m.n_samp, P.m.n_bl, P.n_int);
  RS_CUDA(cudaGetLastError());
  if (opt->profile) RS_CUDA(cudaEventRecord(ev[0], s));
  if (P.m.n_items > 0) {
    di_moment_kernel<MK><<<P.m.n_items, kMomBl2 * kMomLanes2, P.msmem, s>>>(P.m);
    RS_CUDA(cudaGetLastError());
  }
  if (opt->profile) RS_CUDA(cudaEventRecord(ev[1], s));
  if (P.r.n_int > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(P.grid);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RS_CUDA(cudaLaunchKernelEx(&cfg, di_resident_kernel<MK>, P.r));
  }
  if (opt->profile) RS_CUDA(cudaEventRecord(ev[2], s));
  g_launches += 3;
  if (opt->compute_chi2 && P.m.n_items > 0) {
    di_res_chi2_kernel<MK><<<P.m.n_items, 256, 0, s>>>(
        (const float*)vis, (const float*)model, (const float*)gains, P.m.row_off, P.m.n_samp, P.m.n_bl, P.r.bl_off,
        P.r.gain_off, P.r.ant1, P.r.ant2, P.m.item_int, P.m.item_tile, P.m.n_items, P.chi2_items, nullptr);
    res_chi2_final<<<(P.n_int + 255) / 256, 256, 0, s>>>(P.chi2_first, P.chi2_count, P.chi2_items, P.chi2_out, P.n_int);
    RS_CUDA(cudaGetLastError());
    g_launches += 2;
  }
  if (opt->profile) {
    RS_CUDA(cudaEventSynchronize(ev[2]));
    float m_ms = 0.f, r_ms = 0.f;
    RS_CUDA(cudaEventElapsedTime(&m_ms, ev[0], ev[1]));
    RS_CUDA(cudaEventElapsedTime(&r_ms, ev[1], ev[2]));
    for (auto e : ev) cudaEventDestroy(e);
    // rows x iterations and baselines x iterations, from the per-interval iteration counts
    std::vector<int32_t> it(P.n_int), nsv(P.n_int), nbv(P.n_int);
    RS_CUDA(cudaMemcpy(it.data(), P.r.iters, (size_t)P.n_int * 4, cudaMemcpyDeviceToHost));
    RS_CUDA(cudaMemcpy(nsv.data(), P.m.n_samp, (size_t)P.n_int * 4, cudaMemcpyDeviceToHost));
    RS_CUDA(cudaMemcpy(nbv.data(), P.m.n_bl, (size_t)P.n_int * 4, cudaMemcpyDeviceToHost));
    int64_t ri = 0, bi = 0;
    for (int i = 0; i < P.n_int; ++i) {
      ri += (int64_t)it[i] * nsv[i] * nbv[i];
      bi += (int64_t)it[i] * nbv[i];
    }
    profile_record(r_ms, 1, ri, m_ms, bi, 2);
  }
  return GC_OK;
}

int moment_pass(int kind, const float* vis, const float* model, float* moments, const int64_t* row_off,
                const int64_t* mom_off, const int32_t* n_samp, const int32_t* n_bl, const int32_t* item_int,
                const int32_t* item_tile, int n_items, int ns_max, void* stream, const float* weights) {
  if (n_items <= 0) return 0;
  MomArgs m{vis, model, moments, row_off, mom_off, n_samp, n_bl, item_int, item_tile, n_items, weights};
  cudaStream_t s = (cudaStream_t)stream;
  if (ns_max <= kDirectSamp) {
    const int grid = (n_items + 7) / 8;
    if (kind == 0) di_moment_direct_kernel<ScalarMom><<<grid, 256, 0, s>>>(m);
    else di_moment_direct_kernel<JonesMom><<<grid, 256, 0, s>>>(m);
  } else if (kind == 0) {
    const int sm = (int)(sizeof(float) * kMomLanes2 * kMomBl2 * ScalarMom::NM);
    di_moment_kernel<ScalarMom><<<n_items, kMomBl2 * kMomLanes2, sm, s>>>(m);
  } else {
    const int sm = (int)(sizeof(float) * kMomLanes2 * kMomBl2 * JonesMom::NM);
    cudaError_t e = cudaFuncSetAttribute(di_moment_kernel<JonesMom>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return (int)e;
    di_moment_kernel<JonesMom><<<n_items, kMomBl2 * kMomLanes2, sm, s>>>(m);
  }
  return (int)cudaGetLastError();
}

int moment_chi2(int kind, const float* vis, const float* model, const float* gains, const int64_t* row_off,
                const int32_t* n_samp, const int32_t* n_bl, const int32_t* bl_off, const int32_t* gain_off,
                const int32_t* ant1, const int32_t* ant2, const int32_t* item_int, const int32_t* item_tile,
                int n_items, const int32_t* first, const int32_t* count, double* item_chi2, double* out, int n_int,
                void* stream, const float* weights) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n_items > 0) {
    if (kind == 0)
      di_res_chi2_kernel<ScalarMom><<<n_items, 256, 0, s>>>(vis, model, gains, row_off, n_samp, n_bl, bl_off,
                                                            gain_off, ant1, ant2, item_int, item_tile, n_items,
                                                            item_chi2, weights);
    else
      di_res_chi2_kernel<JonesMom><<<n_items, 256, 0, s>>>(vis, model, gains, row_off, n_samp, n_bl, bl_off,
                                                           gain_off, ant1, ant2, item_int, item_tile, n_items,
                                                           item_chi2, weights);
  }
  res_chi2_final<<<(n_int + 255) / 256, 256, 0, s>>>(first, count, item_chi2, out, n_int);
  return (int)cudaGetLastError();
}

// Entry used by run_di: kind 0 scalar, 1 jones (FP32 only).
int res_calibrate(int kind, const gc_layout* L, const void* vis, const void* model, void* gains,
                  const gc_options* opt, int32_t** iters_dev, int32_t** status_dev, double** chi2_dev,
                  cudaStream_t s) {
  ResPlan& P = g_res[kind];
  int dev = 0;
  RS_CUDA(cudaGetDevice(&dev));
  const char* cenv = getenv("GAINCAL_CLUSTER");
  const char* genv = getenv("GAINCAL_RES_CLUSTERS");
  const uint64_t key = layout_hash(L, 0x5E5ull ^ (uint64_t)kind ^ ((uint64_t)dev << 40) ^
                                          ((uint64_t)(cenv ? atoi(cenv) : 0) << 20) ^
                                          ((uint64_t)(genv ? atoi(genv) : 0) << 28));
  if (P.key != key || !P.dev) {
    P.key = 0;
    const int rc = kind == 0 ? build_res_plan<ScalarMom>(kind, L, P, s) : build_res_plan<JonesMom>(kind, L, P, s);
    if (rc != GC_OK) return rc;
    P.key = key;
  }
  const int rc = kind == 0 ? res_run<ScalarMom>(P, vis, model, gains, opt, s)
                           : res_run<JonesMom>(P, vis, model, gains, opt, s);
  if (rc != GC_OK) return rc;
  *iters_dev = P.r.iters;
  *status_dev = P.r.status;
  *chi2_dev = P.chi2_out;
  return GC_OK;
}

void res_release() {
  for (auto& p : g_res) {
    if (p.dev) cudaFree(p.dev);
    p = ResPlan{};
  }
}

}  // namespace gc
