// C ABI of the gain-calibration library: argument validation, plans (device copies of the layout
// and the per-antenna reduction slot lists), the cached workspace, and the iteration loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <string>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"
#include "dd.h"

namespace gc {

int res_supported(int kind, const gc_layout* L);
int res_calibrate(int kind, const gc_layout* L, const void* vis, const void* model, void* gains,
                  const gc_options* opt, int32_t** iters_dev, int32_t** status_dev, double** chi2_dev,
                  cudaStream_t s);
void res_release();

std::atomic<long long> g_launches{0};
static char g_cuda_err[256] = "";

static int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return GC_ERR_CUDA;
}
#define GC_CUDA(call)                                       \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call);   \
  } while (0)
#define GC_CUDA_I(call)                                            \
  do {                                                             \
    int e__ = (call);                                              \
    if (e__ != 0) return cuda_fail((cudaError_t)e__, #call);       \
  } while (0)

// ------------------------------------------------------------------------------------ workspace
// Grow-only device buffers, one per named slot.  The device they live on is recorded; a call on
// another device reallocates.
struct Slot {
  void* p = nullptr;
  size_t n = 0;
  int dev = -1;
};
static std::map<std::string, Slot> g_ws;
static int* g_pinned_flag = nullptr;

int ws_get(const char* name, size_t bytes, void** out) {
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  Slot& s = g_ws[name];
  if (s.p && (s.n < bytes || s.dev != dev)) {
    int cur = dev;
    if (s.dev != dev) cudaSetDevice(s.dev);
    cudaFree(s.p);
    if (s.dev != dev) cudaSetDevice(cur);
    s.p = nullptr;
    s.n = 0;
  }
  if (!s.p && bytes > 0) {
    size_t want = bytes + bytes / 8 + 256;
    GC_CUDA(cudaMalloc(&s.p, want));
    s.n = want;
    s.dev = dev;
  }
  *out = s.p;
  return GC_OK;
}

int pinned_flag(int** out) {
  if (!g_pinned_flag) GC_CUDA(cudaHostAlloc((void**)&g_pinned_flag, 64, cudaHostAllocDefault));
  *out = g_pinned_flag;
  return GC_OK;
}

const char* last_cuda_error() { return g_cuda_err; }

int set_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

// ------------------------------------------------------------------------------------ layout checks
int validate_layout(const gc_layout* L, int n_dir_required_max) {
  if (!L) return GC_ERR_ARG;
  if (L->n_intervals < 0 || L->n_bl_table < 0 || L->n_rows < 0 || L->n_gain < 0) return GC_ERR_LAYOUT;
  if (L->n_intervals == 0) return GC_OK;
  if (!L->row_off || !L->n_samp || !L->n_bl || !L->bl_off || !L->n_ant || !L->gain_off) return GC_ERR_ARG;
  if (L->n_bl_table > 0 && (!L->ant1 || !L->ant2)) return GC_ERR_ARG;
  if (L->n_dir < 1 || L->n_dir > n_dir_required_max) return GC_ERR_LIMIT;
  // per-table maximum antenna index (tables identified by (bl_off, n_bl))
  std::map<std::pair<int, int>, int> tab_max;
  for (int i = 0; i < L->n_intervals; ++i) {
    const int64_t ns = L->n_samp[i], nb = L->n_bl[i], na = L->n_ant[i];
    if (ns < 0 || nb < 0 || na < 1) return GC_ERR_LAYOUT;
    if (na > GC_MAX_ANT) return GC_ERR_LIMIT;
    if (L->row_off[i] < 0 || L->row_off[i] + ns * nb > L->n_rows) return GC_ERR_LAYOUT;
    if (L->bl_off[i] < 0 || (int64_t)L->bl_off[i] + nb > L->n_bl_table) return GC_ERR_LAYOUT;
    if (L->gain_off[i] < 0 || (int64_t)L->gain_off[i] + na > L->n_gain) return GC_ERR_LAYOUT;
    auto key = std::make_pair((int)L->bl_off[i], (int)nb);
    auto f = tab_max.find(key);
    int mx;
    if (f == tab_max.end()) {
      mx = -1;
      for (int b = 0; b < nb; ++b) {
        const int p = L->ant1[L->bl_off[i] + b], q = L->ant2[L->bl_off[i] + b];
        if (p < 0 || q < 0 || p == q) return GC_ERR_ANTENNA;
        mx = p > mx ? p : mx;
        mx = q > mx ? q : mx;
      }
      tab_max[key] = mx;
    } else {
      mx = f->second;
    }
    if (mx >= na) return GC_ERR_ANTENNA;
  }
  return GC_OK;
}

static uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}

uint64_t layout_hash(const gc_layout* L, uint64_t salt) {
  uint64_t h = 1469598103934665603ull ^ salt;
  const size_t n = (size_t)L->n_intervals;
  h = fnv(h, &L->n_intervals, sizeof(int32_t));
  h = fnv(h, &L->n_rows, sizeof(int64_t));
  h = fnv(h, &L->n_gain, sizeof(int32_t));
  h = fnv(h, &L->n_dir, sizeof(int32_t));
  h = fnv(h, &L->n_bl_table, sizeof(int32_t));
  if (n) {
    h = fnv(h, L->row_off, n * 8);
    h = fnv(h, L->n_samp, n * 4);
    h = fnv(h, L->n_bl, n * 4);
    h = fnv(h, L->bl_off, n * 4);
    h = fnv(h, L->n_ant, n * 4);
    h = fnv(h, L->gain_off, n * 4);
  }
  if (L->n_bl_table) {
    h = fnv(h, L->ant1, (size_t)L->n_bl_table * 4);
    h = fnv(h, L->ant2, (size_t)L->n_bl_table * 4);
  }
  return h;
}

// ------------------------------------------------------------------------------------ tunables
// Launch-shape choices of the DI solvers.  Defaults below; gc_autotune_di measures candidates on
// the caller's data and records the fastest per shape bucket; GAINCAL_* environment variables
// override both (for experiments).
struct Tune {
  int red_chunks = 1;     // moment path: per-antenna slot lists summed in 1 or 4 chunks
  int prefetch = 3;       // moment path: 0 none, 1 next tile's moments into registers while reducing this one,
                          // 2 staged in shared memory by cp.async, 3 bulk copies into a two-stage ring (2x2;
                          // scalar moments take 1)
  int bps = 0;            // CTAs per SM of the persistent grid (0 = as many as fit)
  int check_every = 64;   // iterations per graph segment / between host checks of the active count
  int target_rows = 0;    // raw-row path: rows per work item (0 = default)
  int graph = 1;          // capture iteration segments in a CUDA graph
  int step1 = 0;          // moment path: one cooperative launch per iteration (update + accumulate)
  int loop = 0;           // moment path: run segments in one persistent cooperative launch instead
                          // (grid barriers between the phases; measured slower than graph segments)
};
static std::map<uint64_t, Tune> g_tune;
static bool g_tune_override_on = false;
static Tune g_tune_override;

static int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) { v >>= 1; ++r; }
  return r;
}

static uint64_t tune_bucket(int kind, int dtype, int mode, const gc_layout* L) {
  int64_t nb_max = 0, rows = 0;
  for (int i = 0; i < L->n_intervals; ++i) {
    nb_max = std::max<int64_t>(nb_max, L->n_bl[i]);
    rows += (int64_t)L->n_bl[i] * L->n_samp[i];
  }
  const int64_t ms = L->n_intervals > 0 && nb_max > 0 ? rows / std::max<int64_t>(1, (int64_t)L->n_intervals * nb_max) : 0;
  return ((uint64_t)kind) | ((uint64_t)dtype << 2) | ((uint64_t)mode << 4) | ((uint64_t)ilog2(L->n_intervals) << 8) |
         ((uint64_t)ilog2(nb_max) << 16) | ((uint64_t)ilog2(ms) << 24);
}

static int env_int(const char* name, int dflt);

static Tune effective_tune(int kind, int dtype, int mode, const gc_layout* L) {
  Tune t;
  if (g_tune_override_on) {
    t = g_tune_override;
  } else {
    auto f = g_tune.find(tune_bucket(kind, dtype, mode, L));
    if (f != g_tune.end()) t = f->second;
  }
  t.red_chunks = env_int("GAINCAL_RED_CHUNKS", t.red_chunks);
  t.prefetch = env_int("GAINCAL_ACC_PREFETCH", t.prefetch);
  if (t.prefetch == 3 && (kind != 1 || mode != 1)) t.prefetch = 1;  // the bulk-copy kernel: 2x2 moments only
  t.bps = env_int("GAINCAL_BLOCKS_PER_SM", t.bps);
  t.check_every = std::max(1, env_int("GAINCAL_CHECK_EVERY", t.check_every));
  t.target_rows = env_int(kind == 0 ? "GAINCAL_TARGET_ROWS_SCALAR" : "GAINCAL_TARGET_ROWS_JONES", t.target_rows);
  t.graph = env_int("GAINCAL_GRAPH", t.graph);
  t.loop = env_int("GAINCAL_LOOP", t.loop);
  t.step1 = env_int("GAINCAL_STEP1", t.step1);
  return t;
}

static uint64_t tune_hash(const Tune& t) {
  return (uint64_t)t.red_chunks * 1000003ull ^ (uint64_t)t.prefetch * 7919ull ^ (uint64_t)t.bps * 104729ull ^
         (uint64_t)t.target_rows * 1299709ull ^ (uint64_t)t.check_every * 15485863ull ^ (uint64_t)t.loop * 32452843ull ^
         (uint64_t)t.step1 * 49979687ull;
}

// ------------------------------------------------------------------------------------ DI plan
struct DIPlan {
  uint64_t key = 0;
  int n_int = 0, n_items = 0, na_max = 1, n_active0 = 0;
  int64_t scr_elems = 0;
  // device copies, carved out of one buffer
  void* dev = nullptr;
  size_t dev_bytes = 0;
  DIArgs args{};  // layout / plan pointers filled in
  double* chi2_items = nullptr;
  double* chi2_out = nullptr;
  int grid = 0, smem = 0;
  int lgrid = 0, lsmem = 0;  // persistent loop kernel (moment mode): co-resident grid, shared memory
  int sgrid = 0, ssmem = 0;  // single-launch iteration kernel (moment mode)
  // moment-stream mode: moment-pass items (interval, 32 baselines), per-item chi^2 bookkeeping
  int mode = 0;
  int n_mitems = 0;
  int ns_max = 0;  // most samples per baseline of any interval
  int64_t n_mom_bl = 0;
  const int32_t* mitem_int = nullptr;
  const int32_t* mitem_tile = nullptr;
  const int32_t* mfirst = nullptr;
  const int32_t* mcount = nullptr;
  double* mchi2 = nullptr;
  Tune tune;
  // captured iteration segment (graph) and the arguments it was captured with
  cudaGraphExec_t gexec = nullptr;
  DIArgs gargs{};
  int gS = 0;
};

static DIPlan g_di_plan[2][2][2][2];  // [mode][kind][dtype][acc_only]
static int g_target_rows[2] = {32768, 8192};

static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v ? atoi(v) : dflt;
}

// Build the work items, baseline-table reduction lists and device copies for one layout.
static int build_di_plan(int mode, int kind, int dtype, int acc_only, const gc_layout* L, const Tune& tune, DIPlan& P,
                         void* stream) {
  const int nc = kind == 0 ? 3 : 12;
  const int TB = kDIThreads;
  const int n = L->n_intervals;
  // baseline tables
  std::map<std::pair<int, int>, int> tabs;
  std::vector<int> itab(n), tab_base, tab_nant, csr_off, csr_ent;
  std::vector<int> tblk;                                   // bulk-copy accumulate: static tile blocks
  std::vector<std::vector<std::pair<int, int>>> tblk_at;   // per table and tile: (offset, length) in ints
  int tblk_max = 4;
  auto pad4 = [](int x) { return (x + 3) & ~3; };
  for (int i = 0; i < n; ++i) {
    auto key = std::make_pair((int)L->bl_off[i], (int)L->n_bl[i]);
    auto f = tabs.find(key);
    if (f != tabs.end()) { itab[i] = f->second; continue; }
    const int t = (int)tab_base.size();
    tabs[key] = t;
    itab[i] = t;
    const int bo = key.first, nb = key.second;
    int nat = 0;
    for (int b = 0; b < nb; ++b) {
      nat = L->ant1[bo + b] + 1 > nat ? L->ant1[bo + b] + 1 : nat;
      nat = L->ant2[bo + b] + 1 > nat ? L->ant2[bo + b] + 1 : nat;
    }
    tab_base.push_back((int)csr_off.size());
    tab_nant.push_back(nat);
    tblk_at.emplace_back();
    const int ntiles = (nb + TB - 1) / TB;
    for (int tile = 0; tile < ntiles; ++tile) {
      std::vector<std::vector<int>> lists(nat);
      for (int s = 0; s < TB; ++s) {
        const int b = tile * TB + s;
        if (b >= nb) break;
        // p side of slot s; the moment kernels first sum each warp's runs of equal p, so there
        // only the last slot of a run is listed
        const bool run_end = s % 32 == 31 || b + 1 == nb || L->ant1[bo + b + 1] != L->ant1[bo + b];
        if (mode == 0 || run_end) lists[L->ant1[bo + b]].push_back(s * (2 * nc + 1));
        lists[L->ant2[bo + b]].push_back(s * (2 * nc + 1) + nc);   // q side of slot s
      }
      for (int a = 0; a < nat; ++a) {
        csr_off.push_back((int)csr_ent.size());
        csr_ent.insert(csr_ent.end(), lists[a].begin(), lists[a].end());
      }
      csr_off.push_back((int)csr_ent.size());
      if (mode == 1) {
        const int o = (int)tblk.size();
        tblk.resize(o + 2 * TB, -1);
        for (int s = 0; s < TB && tile * TB + s < nb; ++s) {
          tblk[o + s] = L->ant1[bo + tile * TB + s];
          tblk[o + TB + s] = L->ant2[bo + tile * TB + s];
        }
        const int oo = (int)tblk.size();
        tblk.resize(oo + pad4(nat + 1), 0);
        int ne = 0;
        for (int a = 0; a < nat; ++a) { tblk[oo + a] = ne; ne += (int)lists[a].size(); }
        tblk[oo + nat] = ne;
        // entries address the partials as the bulk-copy kernel stores them: slot s's components
        // c in float4 groups over the tile's moment area, [c / 4][TB][4] (q side from group nc / 4)
        const int eo = (int)tblk.size();
        tblk.resize(eo + pad4(ne), 0);
        int e = eo;
        for (int a = 0; a < nat; ++a)
          for (int v : lists[a]) {
            const int slot = v / (2 * nc + 1), q_side = v % (2 * nc + 1) == nc;
            tblk[e++] = slot * 4 + (q_side ? (nc / 4) * TB * 4 : 0);
          }
        const int len = (int)tblk.size() - o;
        tblk_at[t].push_back({o, len});
        tblk_max = len > tblk_max ? len : tblk_max;
      }
    }
  }
  if (csr_off.empty()) csr_off.push_back(0);
  if (csr_ent.empty()) csr_ent.push_back(0);
  // work items: (interval, sample range) for the raw-row kernel; (interval, tile range) for moments
  const int target = tune.target_rows > 0 ? tune.target_rows : g_target_rows[kind];
  const int tpi = 1;  // moment path: one item per 256-baseline tile
  std::vector<int> item_int, item_s0, item_s1, n_chunks(n), first_item(n);
  std::vector<int64_t> item_scr, mom_off(n);
  std::vector<int> mint, mtile, mfirst(n), mcount(n);
  int64_t scr = 0, mo = 0;
  int na_max = 1, n_active0 = 0;
  for (int i = 0; i < n; ++i) {
    const int ns = L->n_samp[i], nb = L->n_bl[i];
    na_max = L->n_ant[i] > na_max ? L->n_ant[i] : na_max;
    first_item[i] = (int)item_int.size();
    mom_off[i] = mo;
    mo += (int64_t)(nb + 255) / 256 * 256;   // tiled moment layout: whole 256-baseline tiles
    mfirst[i] = (int)mint.size();
    if ((int64_t)ns * nb > 0)
      for (int t = 0; t < (nb + 31) / 32; ++t) { mint.push_back(i); mtile.push_back(t); }
    mcount[i] = (int)mint.size() - mfirst[i];
    if ((int64_t)ns * nb == 0) { n_chunks[i] = 0; continue; }
    ++n_active0;
    int per, units;
    if (mode == 1) {
      units = (nb + TB - 1) / TB;
      per = tpi < units ? tpi : units;
    } else {
      units = ns;
      per = nb > 0 ? (target + nb - 1) / nb : ns;
      per = per < 1 ? 1 : (per > ns ? ns : per);
    }
    const int nch = (units + per - 1) / per;
    n_chunks[i] = nch;
    for (int c = 0; c < nch; ++c) {
      item_int.push_back(i);
      item_s0.push_back(c * per);
      item_s1.push_back((c + 1) * per < units ? (c + 1) * per : units);
      const int nat = tab_nant[itab[i]];
      if (nch > 1 || mode == 1) { item_scr.push_back(scr); scr += (int64_t)nat * nc; }
      else item_scr.push_back(-1);
    }
  }
  const int n_items = (int)item_int.size();
  std::vector<int4> idesc;  // bulk-copy accumulate descriptors, three per item
  if (mode == 1) {
    const int nm = kind == 0 ? 4 : 48;
    for (int it = 0; it < n_items; ++it) {
      const int i = item_int[it], t = item_s0[it];
      const int64_t mom = (mom_off[i] + (int64_t)t * TB) * nm, sc = item_scr[it];
      const int nbt = std::min(TB, L->n_bl[i] - t * TB);
      const std::pair<int, int> blk = tblk_at[itab[i]][t];
      idesc.push_back(make_int4((int)(mom & 0xffffffff), (int)(mom >> 32), nbt, blk.first));
      idesc.push_back(make_int4(blk.second, tab_nant[itab[i]], L->gain_off[i], L->n_ant[i]));
      idesc.push_back(make_int4((int)(sc & 0xffffffff), (int)(sc >> 32), 0, 0));
    }
  }
  if (tblk.empty()) tblk.assign(4, 0);
  if (idesc.empty()) idesc.assign(3, make_int4(0, 0, 0, 0));
  // pack into one device buffer: int64 arrays first
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  struct Part { const void* src; size_t bytes; size_t off; };
  std::vector<Part> parts;
  size_t off = 0;
  auto add = [&](const void* src, size_t bytes) { parts.push_back({src, bytes, off}); off += al(bytes > 0 ? bytes : 1); return parts.size() - 1; };
  const size_t p_row_off = add(L->row_off, (size_t)n * 8);
  const size_t p_item_scr = add(item_scr.data(), item_scr.size() * 8);
  const size_t p_n_samp = add(L->n_samp, (size_t)n * 4);
  const size_t p_n_bl = add(L->n_bl, (size_t)n * 4);
  const size_t p_bl_off = add(L->bl_off, (size_t)n * 4);
  const size_t p_n_ant = add(L->n_ant, (size_t)n * 4);
  const size_t p_gain_off = add(L->gain_off, (size_t)n * 4);
  const size_t p_ant1 = add(L->ant1, (size_t)L->n_bl_table * 4);
  const size_t p_ant2 = add(L->ant2, (size_t)L->n_bl_table * 4);
  const size_t p_itab = add(itab.data(), itab.size() * 4);
  const size_t p_tab_base = add(tab_base.data(), tab_base.size() * 4);
  const size_t p_tab_nant = add(tab_nant.data(), tab_nant.size() * 4);
  const size_t p_csr_off = add(csr_off.data(), csr_off.size() * 4);
  const size_t p_csr_ent = add(csr_ent.data(), csr_ent.size() * 4);
  const size_t p_item_int = add(item_int.data(), item_int.size() * 4);
  const size_t p_item_s0 = add(item_s0.data(), item_s0.size() * 4);
  const size_t p_item_s1 = add(item_s1.data(), item_s1.size() * 4);
  const size_t p_n_chunks = add(n_chunks.data(), n_chunks.size() * 4);
  const size_t p_first_item = add(first_item.data(), first_item.size() * 4);
  const size_t p_tblk = add(tblk.data(), tblk.size() * 4);
  const size_t p_idesc = add(idesc.data(), idesc.size() * sizeof(int4));
  if (mint.empty()) { mint.push_back(0); mtile.push_back(0); }
  const size_t p_mom_off = add(mom_off.data(), mom_off.size() * 8);
  const size_t p_mint = add(mint.data(), mint.size() * 4);
  const size_t p_mtile = add(mtile.data(), mtile.size() * 4);
  const size_t p_mfirst = add(mfirst.data(), mfirst.size() * 4);
  const size_t p_mcount = add(mcount.data(), mcount.size() * 4);
  const size_t p_mchi2 = add(nullptr, mint.size() * 8);
  const size_t p_ilist = add(nullptr, (size_t)3 * (n_items > 0 ? n_items : 1) * 4);
  const size_t p_icount = add(nullptr, 16);
  // per-call state
  const size_t p_active = add(nullptr, (size_t)n * 4);
  const size_t p_iters = add(nullptr, (size_t)n * 4);
  const size_t p_status = add(nullptr, (size_t)n * 4);
  const size_t p_counters = add(nullptr, (size_t)n * 4);
  const size_t p_misc = add(nullptr, 64);
  const size_t p_chi2 = add(nullptr, (size_t)(n_items > 0 ? n_items : 1) * 8);
  const size_t p_chi2o = add(nullptr, (size_t)(n > 0 ? n : 1) * 8);
  const size_t total = off;
  std::vector<unsigned char> host(total, 0);
  for (auto& pt : parts)
    if (pt.src && pt.bytes) memcpy(host.data() + pt.off, pt.src, pt.bytes);
  if (P.dev && P.dev_bytes < total) { cudaFree(P.dev); P.dev = nullptr; P.dev_bytes = 0; }
  if (!P.dev) { GC_CUDA(cudaMalloc(&P.dev, total)); P.dev_bytes = total; }
  GC_CUDA(cudaMemcpyAsync(P.dev, host.data(), total, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  GC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned char* d = static_cast<unsigned char*>(P.dev);
  auto at = [&](size_t idx) { return (void*)(d + parts[idx].off); };
  DIArgs& a = P.args;
  a = DIArgs{};
  a.row_off = (const int64_t*)at(p_row_off);
  a.item_scr = (const int64_t*)at(p_item_scr);
  a.n_samp = (const int32_t*)at(p_n_samp);
  a.n_bl = (const int32_t*)at(p_n_bl);
  a.bl_off = (const int32_t*)at(p_bl_off);
  a.n_ant = (const int32_t*)at(p_n_ant);
  a.gain_off = (const int32_t*)at(p_gain_off);
  a.ant1 = (const int32_t*)at(p_ant1);
  a.ant2 = (const int32_t*)at(p_ant2);
  a.itab = (const int32_t*)at(p_itab);
  a.tab_base = (const int32_t*)at(p_tab_base);
  a.tab_nant = (const int32_t*)at(p_tab_nant);
  a.csr_off = (const int32_t*)at(p_csr_off);
  a.csr_ent = (const int32_t*)at(p_csr_ent);
  a.item_int = (const int32_t*)at(p_item_int);
  a.item_s0 = (const int32_t*)at(p_item_s0);
  a.item_s1 = (const int32_t*)at(p_item_s1);
  a.n_chunks = (const int32_t*)at(p_n_chunks);
  a.first_item = (const int32_t*)at(p_first_item);
  a.active = (int32_t*)at(p_active);
  a.iters = (int32_t*)at(p_iters);
  a.status = (int32_t*)at(p_status);
  a.counters = (int32_t*)at(p_counters);
  a.n_active = (int32_t*)at(p_misc);
  a.qhead = (int32_t*)at(p_misc) + 4;
  a.kbase = (int32_t*)at(p_misc) + 8;
  a.err = (int32_t*)at(p_misc) + 12;
  a.tblk = (const int32_t*)at(p_tblk);
  a.item_desc = (const int4*)at(p_idesc);
  a.tblk_max = tblk_max;
  a.n_items = n_items;
  a.na_max = na_max;
  a.mom_off = (const int64_t*)at(p_mom_off);
  a.ilist = mode == 1 ? (int32_t*)at(p_ilist) : nullptr;
  a.icount = mode == 1 ? (int32_t*)at(p_icount) : nullptr;
  P.mode = mode;
  P.n_mitems = n_active0 > 0 ? (int)mint.size() : 0;
  P.n_mom_bl = mo;
  P.ns_max = 0;
  for (int i = 0; i < n; ++i) P.ns_max = std::max(P.ns_max, (int)L->n_samp[i]);
  P.mitem_int = (const int32_t*)at(p_mint);
  P.mitem_tile = (const int32_t*)at(p_mtile);
  P.mfirst = (const int32_t*)at(p_mfirst);
  P.mcount = (const int32_t*)at(p_mcount);
  P.mchi2 = (double*)at(p_mchi2);
  P.chi2_items = (double*)at(p_chi2);
  P.chi2_out = (double*)at(p_chi2o);
  P.n_int = n;
  P.n_items = n_items;
  P.na_max = na_max;
  P.n_active0 = n_active0;
  P.scr_elems = scr;
  P.smem = di_smem_bytes(kind, dtype, na_max);
  int dev = 0, nsm = 0, per_sm = 0, max_smem = 0;
  GC_CUDA(cudaGetDevice(&dev));
  GC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  GC_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (P.smem > max_smem) return GC_ERR_LIMIT;
  Tune tn = tune;
  // the bulk-copy kernel's ring must fit; otherwise the register-prefetch kernel takes its place
  if (mode == 1 && tn.prefetch == 3 && di_macc_bulk_smem(kind, na_max, tblk_max) > max_smem) tn.prefetch = 1;
  if (mode == 1) {
    P.smem = tn.prefetch == 3 ? di_macc_bulk_smem(kind, na_max, tblk_max)
                              : di_macc_smem(kind, na_max, tn.red_chunks, tn.prefetch);
    if (P.smem > max_smem) return GC_ERR_LIMIT;
    GC_CUDA_I(di_macc_max_blocks_per_sm(kind, P.smem, tn.red_chunks, tn.prefetch, &per_sm));
  } else {
    GC_CUDA_I(di_max_blocks_per_sm(kind, dtype, acc_only, P.smem, &per_sm));
  }
  if (per_sm < 1) return GC_ERR_LIMIT;
  if (tune.bps > 0 && tune.bps < per_sm) per_sm = tune.bps;
  P.tune = tn;
  P.grid = nsm * per_sm;
  if (P.grid > n_items) P.grid = n_items > 0 ? n_items : 1;
  if (mode == 1) {
    P.lsmem = di_mloop_smem(kind, na_max, tune.red_chunks);
    if (P.lsmem > max_smem) return GC_ERR_LIMIT;
    int cap = 0;
    GC_CUDA_I(di_mloop_max_grid(kind, P.lsmem, tune.red_chunks, tune.prefetch, &cap));
    if (tune.bps > 0 && tune.bps * nsm < cap) cap = tune.bps * nsm;
    P.lgrid = cap;
    P.ssmem = di_mstep1_smem(kind, na_max, tune.red_chunks);
    if (P.ssmem > max_smem) return GC_ERR_LIMIT;
    GC_CUDA_I(di_mstep1_max_grid(kind, P.ssmem, tune.red_chunks, tune.prefetch, &cap));
    if (tune.bps > 0 && tune.bps * nsm < cap) cap = tune.bps * nsm;
    P.sgrid = cap;
  }
  return GC_OK;
}

static int get_di_plan(int mode, int kind, int dtype, int acc_only, const gc_layout* L, DIPlan** out, void* stream) {
  DIPlan& P = g_di_plan[mode][kind][dtype][acc_only];
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  const Tune tune = effective_tune(kind, dtype, mode, L);
  const uint64_t key = layout_hash(L, (uint64_t)(kind * 131 + dtype * 7 + acc_only) ^ ((uint64_t)dev << 40) ^
                                          ((uint64_t)mode << 4) ^ tune_hash(tune));
  if (P.key != key || P.n_int != L->n_intervals || !P.dev) {
    P.key = 0;
    if (P.gexec) { cudaGraphExecDestroy(P.gexec); P.gexec = nullptr; }
    int rc = build_di_plan(mode, kind, dtype, acc_only, L, tune, P, stream);
    if (rc != GC_OK) return rc;
    P.key = key;
  }
  P.tune = tune;
  *out = &P;
  return GC_OK;
}

// Optional per-launch timing of the iteration kernels (opt->profile).
struct ProfileTotals {
  double ms = 0.0, moment_ms = 0.0;
  int64_t launches = 0, row_iters = 0, bl_iters = 0;
  int path = 0;
};
static ProfileTotals g_prof;

void profile_record(double iter_ms, int64_t launches, int64_t row_iters, double moment_ms, int64_t bl_iters,
                    int path) {
  g_prof.ms = iter_ms;
  g_prof.launches = launches;
  g_prof.row_iters = row_iters;
  g_prof.moment_ms = moment_ms;
  g_prof.bl_iters = bl_iters;
  g_prof.path = path;
}

struct Profiler {
  bool on;
  int cap, used = 0, weight = 1;  // weight: iterations per bracketed launch
  std::vector<cudaEvent_t> ev;
  double ms = 0.0;
  int64_t launches = 0;
  Profiler(bool on_, int cap_) : on(on_), cap(cap_ > 0 ? cap_ : 1) {}
  ~Profiler() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  int init() {
    if (!on) return GC_OK;
    ev.resize(2 * (size_t)cap, nullptr);
    for (auto& e : ev) GC_CUDA(cudaEventCreate(&e));
    return GC_OK;
  }
  int before(cudaStream_t s) {
    if (!on) return GC_OK;
    if (used == cap) { int rc = drain_sync(s); if (rc) return rc; }
    GC_CUDA(cudaEventRecord(ev[2 * used], s));
    return GC_OK;
  }
  int after(cudaStream_t s) {
    if (!on) return GC_OK;
    GC_CUDA(cudaEventRecord(ev[2 * used + 1], s));
    ++used;
    return GC_OK;
  }
  int drain_sync(cudaStream_t s) {
    GC_CUDA(cudaStreamSynchronize(s));
    return drain();
  }
  int drain() {
    if (!on) return GC_OK;
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      GC_CUDA(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
      ms += t;
    }
    launches += (int64_t)used * weight;
    used = 0;
    return GC_OK;
  }
  void finish(int64_t row_iters, int64_t bl_iters, double mom_ms, int path) {
    profile_record(ms, launches, row_iters, mom_ms, bl_iters, path);
  }
};

static size_t elem_bytes(int kind, int dtype) {
  const size_t r = dtype == GC_DTYPE_C64 ? 8 : 16;  // one complex
  return kind == 0 ? r : 4 * r;
}

// Stage host buffers on the device when opt->host_buffers is set.
struct Staged {
  const void* vis;
  const void* model;
  void* gains;
};

// Learned start for the intervals [i_lo, i_lo + n) (moment path, 2x2; the moments, the accumulate
// scratch and the init launch are in place, `a` holds the plan's pointers):
//   g1 = newest previous solution (from `sol` at the slots hoff [n][4], each put in the canonical
//   gauge first when canon != 0); tot, e1 = per-antenna sums and chi^2 - sum|d|^2 at g1 (one
//   accumulate launch over the range's moments); features -> BF16 MLP -> proposal; e2 at the
//   proposal; start = proposal where e2 < e1, else g1.  Without a network the start is g1.
//   The range's gains (and their per-antenna auxiliaries) end up holding the start.
static int warm_range(const gc_layout* L, DIPlan* P, DIArgs a, const float* sol, const int32_t* hoff,
                      const float* lead, const gc_mlp* net, int canon, int i_lo, int n, const int32_t* first_item_h,
                      float* gains, int32_t* used_out, double* dchi2_out, float* start_out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0) return GC_OK;
  const int64_t gbase = L->gain_off[i_lo];
  int64_t ng = 0;
  for (int i = i_lo; i < i_lo + n; ++i) ng = std::max<int64_t>(ng, (int64_t)L->gain_off[i] + L->n_ant[i] - gbase);
  void *meta = nullptr, *fb = nullptr, *eb = nullptr;
  int rc;
  if ((rc = ws_get("warm_meta", (size_t)n * 5 * sizeof(int32_t), &meta))) return rc;
  if ((rc = ws_get("warm_f", (size_t)(ng > 0 ? ng : 1) * (32 + 8 + 1 + 48 + 2 + 8 + 12) * sizeof(float), &fb)))
    return rc;
  if ((rc = ws_get("warm_e", (size_t)n * 2 * sizeof(double), &eb))) return rc;
  int32_t* d_hoff = (int32_t*)meta;
  float* d_lead = (float*)(d_hoff + 4 * (size_t)n);
  float* hbuf = (float*)fb;
  float* g1 = hbuf + ng * 32;
  float* lead_row = g1 + ng * 8;
  float* x = lead_row + ng;
  float* rot = x + ng * 48;
  float* delta = rot + ng * 2;
  float* tot = delta + ng * 8;
  double* e1 = (double*)eb;
  double* e2 = e1 + n;
  float* gr = gains + gbase * 8;  // the range's gain slots
  GC_CUDA(cudaMemcpyAsync(d_hoff, hoff, (size_t)n * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d_lead, lead, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
  GC_CUDA_I(ws_gather(sol, d_hoff, d_lead, a.gain_off, a.n_ant, i_lo, n, gbase, canon, hbuf, g1, lead_row, stream));
  GC_CUDA(cudaMemcpyAsync(gr, g1, (size_t)ng * 8 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  g_launches++;
  if (!net) {
    if (used_out) GC_CUDA(cudaMemsetAsync(used_out + i_lo, 0, (size_t)n * sizeof(int32_t), s));
    if (dchi2_out) GC_CUDA(cudaMemsetAsync(dchi2_out + i_lo, 0, (size_t)n * sizeof(double), s));
  } else {
    const Tune& tn = P->tune;
    DIArgs b = a;
    b.gains = gains;
    b.xbegin = first_item_h[i_lo];
    b.xcount = (i_lo + n < P->n_int ? first_item_h[i_lo + n] : P->n_items) - b.xbegin;
    GC_CUDA_I(di_launch_maux(1, gr, a.aux + gbase * 4, (int)ng, stream));
    if (b.xcount > 0) GC_CUDA_I(di_launch_macc(1, b, P->grid, P->smem, tn.red_chunks, tn.prefetch, stream));
    GC_CUDA_I(di_launch_msum(1, b, i_lo, n, tot, e1, stream));
    GC_CUDA_I(ws_features_packed(hbuf, tot, lead_row, (int)ng, x, rot, stream));
    if ((rc = mlp_infer(net, x, (int)ng, delta, stream))) return rc;
    GC_CUDA_I(ws_propose(hbuf, delta, rot, (int)ng, gr, stream));
    GC_CUDA_I(di_launch_maux(1, gr, a.aux + gbase * 4, (int)ng, stream));
    if (b.xcount > 0) GC_CUDA_I(di_launch_macc(1, b, P->grid, P->smem, tn.red_chunks, tn.prefetch, stream));
    GC_CUDA_I(di_launch_msum(1, b, i_lo, n, tot, e2, stream));
    GC_CUDA_I(ws_choose(g1, e1, e2, a.gain_off, a.n_ant, i_lo, n, gbase, gains, used_out, dchi2_out, stream));
    g_launches += 9;
  }
  GC_CUDA_I(di_launch_maux(1, gr, a.aux + gbase * 4, (int)ng, stream));
  g_launches++;
  if (start_out) GC_CUDA(cudaMemcpyAsync(start_out + gbase * 8, gr, (size_t)ng * 8 * sizeof(float),
                                         cudaMemcpyDeviceToDevice, s));
  return GC_OK;
}

// Two barrier words and an error flag for the persistent loop kernel, zeroed on `s`.
static int loop_barrier(unsigned** out, cudaStream_t s) {
  void* p = nullptr;
  int rc = ws_get("loop_barrier", 4 * sizeof(unsigned), &p);
  if (rc) return rc;
  GC_CUDA(cudaMemsetAsync(p, 0, 4 * sizeof(unsigned), s));
  *out = (unsigned*)p;
  return GC_OK;
}

static int first_items_host(DIPlan* P, std::vector<int32_t>& out, cudaStream_t s) {
  out.resize(P->n_int);
  GC_CUDA(cudaMemcpyAsync(out.data(), P->args.first_item, (size_t)P->n_int * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  return GC_OK;
}

// Learned warm start before the iteration of a whole batch (gc_calibrate_di_jones2x2_warm).
static int warm_prephase(const gc_warm* w, const gc_layout* L, DIPlan* P, DIArgs a, float* gains, void* stream) {
  std::vector<int32_t> fi;
  int rc = first_items_host(P, fi, (cudaStream_t)stream);
  if (rc) return rc;
  if ((rc = warm_range(L, P, a, w->solutions, w->hist_off, w->lead, w->net, 0, 0, P->n_int, fi.data(), gains,
                       w->used_out, w->dchi2_out, w->start_out, stream)))
    return rc;
  // the range's accumulate launches used fixed item ranges; reset the per-call state all the same
  GC_CUDA_I(di_launch_init(a, P->n_int, P->n_active0, stream));
  g_launches++;
  return GC_OK;
}

static int run_di(int kind, const void* vis, const void* model, const gc_layout* L, void* gains,
                  const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out, void* stream,
                  const gc_warm* warm = nullptr) {
  if (!opt || !L) return GC_ERR_ARG;
  if (opt->dtype != GC_DTYPE_C64 && opt->dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  if (opt->max_iter < 1 || !(opt->tol >= 0.0) ||
      (opt->schedule != GC_SCHED_STEFCAL && opt->schedule != GC_SCHED_GN && opt->schedule != GC_SCHED_LM))
    return GC_ERR_ARG;
  if (opt->host_buffers != 0 && opt->host_buffers != 1) return GC_ERR_ARG;
  if (opt->reserved || opt->path < GC_PATH_AUTO || opt->path > GC_PATH_MOMENTS) return GC_ERR_ARG;
  if (opt->profile < 0 || opt->profile > 2) return GC_ERR_ARG;
  const bool lm = opt->schedule == GC_SCHED_LM;
  if (opt->lm_reserved || opt->lm_after < 0 || !(opt->lm_lambda0 >= 0.0) || !(opt->lm_K == 0.0 || opt->lm_K > 1.0))
    return GC_ERR_ARG;
  if (lm && (opt->dtype != GC_DTYPE_C64)) return GC_ERR_DTYPE;
  if (lm && (opt->path == GC_PATH_STREAM || opt->path == GC_PATH_RESIDENT)) return GC_ERR_ARG;
  int rc = validate_layout(L, 1);
  if (rc != GC_OK) return rc;
  if (L->n_intervals == 0) return GC_OK;
  if (lm && !lm_limit_ok(kind, L)) return GC_ERR_LIMIT;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && !gains)) return GC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (opt->path == GC_PATH_RESIDENT && opt->weights) return GC_ERR_ARG;  // the resident path takes no weights
  const bool can_res = opt->dtype == GC_DTYPE_C64 && res_supported(kind, L);
  if (opt->path == GC_PATH_RESIDENT && !can_res) return GC_ERR_LIMIT;
  if (opt->path == GC_PATH_MOMENTS && opt->dtype != GC_DTYPE_C64) return GC_ERR_DTYPE;
  const bool resident = opt->path == GC_PATH_RESIDENT;
  const int mode = (opt->path == GC_PATH_MOMENTS || (opt->path == GC_PATH_AUTO && opt->dtype == GC_DTYPE_C64)) ? 1 : 0;
  DIPlan* P = nullptr;
  if (!resident) {
    rc = get_di_plan(mode, kind, opt->dtype, 0, L, &P, stream);
    if (rc != GC_OK) return rc;
  }
  const size_t eb = elem_bytes(kind, opt->dtype);
  Staged st{vis, model, gains};
  if (opt->host_buffers) {
    void *dv = nullptr, *dm = nullptr, *dg = nullptr;
    if ((rc = ws_get("h_vis", (size_t)L->n_rows * eb, &dv))) return rc;
    if ((rc = ws_get("h_model", (size_t)L->n_rows * eb, &dm))) return rc;
    if ((rc = ws_get("h_gains", (size_t)L->n_gain * eb, &dg))) return rc;
    if (L->n_rows) {
      GC_CUDA(cudaMemcpyAsync(dv, vis, (size_t)L->n_rows * eb, cudaMemcpyHostToDevice, s));
      GC_CUDA(cudaMemcpyAsync(dm, model, (size_t)L->n_rows * eb, cudaMemcpyHostToDevice, s));
    }
    GC_CUDA(cudaMemcpyAsync(dg, gains, (size_t)L->n_gain * eb, cudaMemcpyHostToDevice, s));
    st = Staged{dv, dm, dg};
  }
  // per-row weights (Sect. 2.4): real, of the dtype's precision, [n_rows]
  const void* wts = opt->weights;
  if (wts && opt->host_buffers && L->n_rows) {
    const size_t wb = (size_t)L->n_rows * (opt->dtype == GC_DTYPE_C64 ? 4 : 8);
    void* dw = nullptr;
    if ((rc = ws_get("h_weights", wb, &dw))) return rc;
    GC_CUDA(cudaMemcpyAsync(dw, wts, wb, cudaMemcpyHostToDevice, s));
    wts = dw;
  }
  if (resident) {
    int32_t *it_d = nullptr, *st_d = nullptr;
    double* c2_d = nullptr;
    rc = res_calibrate(kind, L, st.vis, st.model, st.gains, opt, &it_d, &st_d, &c2_d, s);
    if (rc != GC_OK) return rc;
    const cudaMemcpyKind dk = opt->host_buffers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int n = L->n_intervals;
    if (opt->host_buffers) GC_CUDA(cudaMemcpyAsync(gains, st.gains, (size_t)L->n_gain * eb, dk, s));
    if (iters_out) GC_CUDA(cudaMemcpyAsync(iters_out, it_d, (size_t)n * 4, dk, s));
    if (status_out) GC_CUDA(cudaMemcpyAsync(status_out, st_d, (size_t)n * 4, dk, s));
    if (chi2_out && opt->compute_chi2) GC_CUDA(cudaMemcpyAsync(chi2_out, c2_d, (size_t)n * 8, dk, s));
    std::vector<int32_t> stv(n);
    GC_CUDA(cudaMemcpyAsync(stv.data(), st_d, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    int bad = 0;
    for (int i = 0; i < n; ++i) bad += (stv[i] & 15) != GC_ST_OK;
    return bad;
  }
  DIArgs a = P->args;
  a.vis = st.vis;
  a.model = st.model;
  a.gains = st.gains;
  a.weights = wts;
  a.tol = opt->tol;
  a.max_iter = opt->max_iter;
  a.schedule = opt->schedule;
  // LM schedule: a fixed number of StefCal iterations first (no stopping), then lm_run
  const int lm_after = lm ? std::min(opt->max_iter, opt->lm_after) : 0;
  if (lm) {
    a.tol = 0.0;
    a.max_iter = lm_after;
    a.schedule = GC_SCHED_STEFCAL;
  }
  if (P->scr_elems > 0) {
    void* scr = nullptr;
    if ((rc = ws_get("di_scratch", (size_t)P->scr_elems * (opt->dtype == GC_DTYPE_C64 ? 4 : 8), &scr))) return rc;
    a.scratch = scr;
  }
  // single-launch iterations: publication flags, an error word, and work list 2 first
  const bool s1 = mode == 1 && P->tune.step1 && !P->tune.loop && P->sgrid > 0;
  int* s1err = nullptr;
  if (s1) {
    void* fv = nullptr;
    if ((rc = ws_get("di_flags", (size_t)(P->n_int + 4) * sizeof(int32_t), &fv))) return rc;
    a.flag = (int32_t*)fv;
    s1err = a.flag + P->n_int;
    GC_CUDA(cudaMemsetAsync(s1err, 0, sizeof(int32_t), s));
    a.first_list = 2;
  }
  GC_CUDA_I(di_launch_init(a, P->n_int, P->n_active0, stream));
  g_launches++;
  double mom_ms = 0.0;
  if (mode == 1) {
    void* mom = nullptr;
    const int nm = kind == 0 ? 4 : 48;
    if ((rc = ws_get("di_moments", (size_t)(P->n_mom_bl > 0 ? P->n_mom_bl : 1) * nm * sizeof(float), &mom))) return rc;
    a.moments = (const float*)mom;
    cudaEvent_t m0 = nullptr, m1 = nullptr;
    if (opt->profile) {
      GC_CUDA(cudaEventCreate(&m0));
      GC_CUDA(cudaEventCreate(&m1));
      GC_CUDA(cudaEventRecord(m0, s));
    }
    GC_CUDA_I(moment_pass(kind, (const float*)st.vis, (const float*)st.model, (float*)mom, a.row_off, a.mom_off,
                          a.n_samp, a.n_bl, P->mitem_int, P->mitem_tile, P->n_mitems, P->ns_max, stream,
                          (const float*)wts));
    void *aux = nullptr, *gnew = nullptr;
    if ((rc = ws_get("di_aux", (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 4 * sizeof(float), &aux))) return rc;
    if ((rc = ws_get("di_gnew", (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 8 * sizeof(float), &gnew))) return rc;
    a.aux = (float*)aux;
    a.gnew = (float*)gnew;
    if (warm && (rc = warm_prephase(warm, L, P, a, (float*)st.gains, stream))) return rc;
    GC_CUDA_I(di_launch_maux(kind, (const float*)st.gains, a.aux, L->n_gain, stream));
    g_launches += 2;
    if (opt->profile) {
      GC_CUDA(cudaEventRecord(m1, s));
      GC_CUDA(cudaEventSynchronize(m1));
      float t = 0.f;
      GC_CUDA(cudaEventElapsedTime(&t, m0, m1));
      mom_ms = t;
      cudaEventDestroy(m0);
      cudaEventDestroy(m1);
    }
  }
  int* flag = nullptr;
  if ((rc = pinned_flag(&flag))) return rc;
  const Tune& tn = P->tune;
  const int S = tn.check_every;
  const int per_iter = mode == 1 && !s1 ? 2 : 1;
  // the single-launch scheme updates iteration k in launch k + 1: one more launch at the end
  const int last_k = (lm ? lm_after : opt->max_iter) + (s1 ? 1 : 0);
  auto launch_iter = [&](const DIArgs& x, cudaStream_t st) -> int {
    if (s1) return di_launch_mstep1(kind, x, P->sgrid, P->ssmem, P->n_int, tn.red_chunks, tn.prefetch, s1err, st);
    return mode == 1 ? di_launch_mstep(kind, x, P->grid, P->smem, P->n_int, tn.red_chunks, tn.prefetch, st)
                     : di_launch_iter(kind, opt->dtype, 0, x, P->grid, P->smem, st);
  };
  auto check_s1 = [&]() -> int {
    if (!s1) return GC_OK;
    GC_CUDA(cudaMemcpyAsync(flag + 4, s1err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (flag[4]) return cuda_fail(cudaErrorLaunchTimeout, "wait for an interval's update timed out");
    return GC_OK;
  };
  Profiler prof(opt->profile != 0, S);
  if ((rc = prof.init())) return rc;
  // profile 2: the accumulate launches timed alone (moment path, two launches per iteration)
  const bool acc_prof = opt->profile == 2 && mode == 1 && !s1 && !(tn.loop && P->lgrid > 0);
  bool use_graph = tn.graph != 0 && !acc_prof;
  if (use_graph && !(mode == 1 && tn.loop && P->lgrid > 0)) {
    // One segment = S iterations captured once (k = *kbase + 1 .. *kbase + S) plus a node that
    // advances *kbase; segments are relaunched until no interval is active.  Iterations past
    // max_iter find no active interval and do nothing.
    DIArgs ga = a;
    ga.k = 0;
    if (mode == 1) ga.vis = ga.model = nullptr;  // the moment-space iterations never read the rows
    if (!P->gexec || P->gS != S || memcmp(&P->gargs, &ga, sizeof(DIArgs)) != 0) {
      if (P->gexec) { cudaGraphExecDestroy(P->gexec); P->gexec = nullptr; }
      cudaStream_t cs = nullptr;
      GC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      GC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int crc = 0;
      for (int j = 1; j <= S && !crc; ++j) {
        DIArgs x = ga;
        x.k = j;
        crc = launch_iter(x, cs);
      }
      if (!crc) crc = di_launch_advance(a.kbase, S, cs);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      cudaError_t ie = cudaSuccess;
      if (!crc && ee == cudaSuccess) ie = cudaGraphInstantiate(&P->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (crc || ee != cudaSuccess || ie != cudaSuccess) {
        if (P->gexec) { cudaGraphExecDestroy(P->gexec); P->gexec = nullptr; }
        if (!s1)
          return cuda_fail(crc ? (cudaError_t)crc : (ee != cudaSuccess ? ee : ie), "capture of the iteration segment");
        cudaGetLastError();  // a cooperative launch that cannot be captured: launch one by one instead
        use_graph = false;
      } else {
        P->gargs = ga;
        P->gS = S;
      }
    }
  }
  if (mode == 1 && tn.loop && P->lgrid > 0) {
    prof.weight = S;
    unsigned* bar = nullptr;
    if ((rc = loop_barrier(&bar, s))) return rc;
    int* err = (int*)(bar + 2);
    for (int k0 = 0; k0 < opt->max_iter; k0 += S) {
      if ((rc = prof.before(s))) return rc;
      GC_CUDA_I(di_launch_mloop(kind, a, P->lgrid, P->lsmem, P->n_int, S, tn.red_chunks, tn.prefetch, bar, err,
                                stream));
      if ((rc = prof.after(s))) return rc;
      g_launches++;
      GC_CUDA(cudaMemcpyAsync(flag, a.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(flag + 1, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaStreamSynchronize(s));
      if ((rc = prof.drain())) return rc;
      if (flag[1]) return cuda_fail(cudaErrorLaunchTimeout, "grid barrier of the iteration loop timed out");
      if (*flag <= 0) break;
    }
  } else if (use_graph) {
    prof.weight = S;
    for (int k0 = 0; k0 < last_k; k0 += S) {
      if ((rc = prof.before(s))) return rc;
      GC_CUDA(cudaGraphLaunch(P->gexec, s));
      if ((rc = prof.after(s))) return rc;
      g_launches += (int64_t)S * per_iter + 1;
      GC_CUDA(cudaMemcpyAsync(flag, a.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaStreamSynchronize(s));
      if ((rc = prof.drain())) return rc;
      if ((rc = check_s1())) return rc;
      if (*flag <= 0) break;
    }
  } else {
    for (int k = 1; k <= last_k; ++k) {
      a.k = k;
      if ((rc = prof.before(s))) return rc;
      if (acc_prof) {
        GC_CUDA_I(di_launch_macc(kind, a, P->grid, P->smem, tn.red_chunks, tn.prefetch, stream));
        if ((rc = prof.after(s))) return rc;
        GC_CUDA_I(di_launch_msolve(kind, a, P->n_int, stream));
      } else {
        GC_CUDA_I(launch_iter(a, s));
        if ((rc = prof.after(s))) return rc;
      }
      g_launches += per_iter;
      if (k % S == 0 || k == last_k) {
        GC_CUDA(cudaMemcpyAsync(flag, a.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if ((rc = prof.drain())) return rc;
        if ((rc = check_s1())) return rc;
        if (*flag <= 0) break;
      }
    }
  }
  if (lm && opt->max_iter > lm_after) {
    rc = lm_run(kind, L, (const float*)st.vis, (const float*)st.model, a.row_off, a.n_samp, a.moments, a.mom_off,
                a.ant1, a.ant2, (float*)st.gains, a.iters, a.status, opt, stream, (const float*)wts);
    if (rc != GC_OK) return rc;
  }
  if (opt->compute_chi2) {
    if (mode == 1)
      GC_CUDA_I(moment_chi2(kind, (const float*)st.vis, (const float*)st.model, (const float*)st.gains, a.row_off,
                            a.n_samp, a.n_bl, a.bl_off, a.gain_off, a.ant1, a.ant2, P->mitem_int, P->mitem_tile,
                            P->n_mitems, P->mfirst, P->mcount, P->mchi2, P->chi2_out, P->n_int, stream,
                            (const float*)wts));
    else
      GC_CUDA_I(di_launch_chi2(kind, opt->dtype, a, P->chi2_items, P->chi2_out, P->n_int, P->grid, stream));
    g_launches += 2;
  }
  const cudaMemcpyKind dk = opt->host_buffers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (opt->host_buffers) GC_CUDA(cudaMemcpyAsync(gains, st.gains, (size_t)L->n_gain * eb, dk, s));
  if (iters_out) GC_CUDA(cudaMemcpyAsync(iters_out, a.iters, (size_t)P->n_int * 4, dk, s));
  if (status_out) GC_CUDA(cudaMemcpyAsync(status_out, a.status, (size_t)P->n_int * 4, dk, s));
  if (chi2_out && opt->compute_chi2) GC_CUDA(cudaMemcpyAsync(chi2_out, P->chi2_out, (size_t)P->n_int * 8, dk, s));
  // count intervals not OK
  std::vector<int32_t> stv(P->n_int), itv(P->n_int);
  GC_CUDA(cudaMemcpyAsync(stv.data(), a.status, (size_t)P->n_int * 4, cudaMemcpyDeviceToHost, s));
  if (opt->profile) GC_CUDA(cudaMemcpyAsync(itv.data(), a.iters, (size_t)P->n_int * 4, cudaMemcpyDeviceToHost, s));
  if (mode == 1) GC_CUDA(cudaMemcpyAsync(flag + 5, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  if (mode == 1 && flag[5]) return cuda_fail(cudaErrorLaunchTimeout, "a bulk copy of an accumulate tile did not complete");
  int bad = 0;
  for (int i = 0; i < P->n_int; ++i) bad += (stv[i] & 15) != GC_ST_OK;
  if (opt->profile) {
    int64_t ri = 0, bi = 0;
    for (int i = 0; i < P->n_int; ++i) {
      // the profiled launches are the diagonal iterations only (the LM schedule's first lm_after)
      const int64_t k = lm ? std::min<int64_t>(itv[i], lm_after) : itv[i];
      ri += k * L->n_samp[i] * L->n_bl[i];
      bi += k * L->n_bl[i];
    }
    prof.finish(ri, bi, mom_ms, mode == 1 ? GC_PATH_MOMENTS : GC_PATH_STREAM);
  }
  return bad;
}

static int32_t* g_pinned_ints = nullptr;
static size_t g_pinned_ints_n = 0;

static int pinned_ints(size_t n, int32_t** out) {
  if (g_pinned_ints_n < n) {
    if (g_pinned_ints) cudaFreeHost(g_pinned_ints);
    g_pinned_ints = nullptr;
    g_pinned_ints_n = 0;
    GC_CUDA(cudaHostAlloc((void**)&g_pinned_ints, n * sizeof(int32_t), cudaHostAllocDefault));
    g_pinned_ints_n = n;
  }
  *out = g_pinned_ints;
  return GC_OK;
}

// Wavefront solve of a time-major grid of 2x2 intervals with learned starts (one iteration loop;
// waves join it as soon as their history has passed the gate).
static int run_wavefront(const void* vis, const void* model, const gc_layout* L, const gc_wavefront* wf, void* gains,
                         const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                         void* stream) {
  if (!wf || !opt || !L) return GC_ERR_ARG;
  if (opt->dtype != GC_DTYPE_C64) return GC_ERR_DTYPE;
  if (opt->max_iter < 1 || !(opt->tol >= 0.0) || (opt->schedule != GC_SCHED_STEFCAL && opt->schedule != GC_SCHED_GN))
    return GC_ERR_ARG;
  if (opt->host_buffers != 0 || opt->reserved || (opt->path != GC_PATH_AUTO && opt->path != GC_PATH_MOMENTS))
    return GC_ERR_ARG;
  if (wf->n_t < 1 || wf->n_fb < 1 || wf->lag < 1 || wf->max_lead < 1 || !(wf->lead_scale > 0.f) ||
      !(wf->gate_tol >= 0.0))
    return GC_ERR_ARG;
  int rc = validate_layout(L, 1);
  if (rc != GC_OK) return rc;
  if ((int64_t)wf->n_t * wf->n_fb != L->n_intervals) return GC_ERR_LAYOUT;
  for (int i = wf->n_fb; i < L->n_intervals; ++i)
    if (L->n_ant[i] != L->n_ant[i % wf->n_fb]) return GC_ERR_LAYOUT;  // a history slot must hold the same antennas
  if (wf->net && (rc = mlp_check(wf->net))) return rc;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && !gains)) return GC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DIPlan* P = nullptr;
  if ((rc = get_di_plan(1, 1, GC_DTYPE_C64, 0, L, &P, stream))) return rc;
  const int n_int = P->n_int, nfb = wf->n_fb, lag = wf->lag;
  DIArgs a = P->args;
  a.vis = vis;
  a.model = model;
  a.gains = gains;
  a.tol = opt->tol;
  a.max_iter = opt->max_iter;
  a.schedule = opt->schedule;
  void *scr = nullptr, *mom = nullptr, *aux = nullptr, *gnew = nullptr, *st = nullptr;
  if (P->scr_elems > 0) {
    if ((rc = ws_get("di_scratch", (size_t)P->scr_elems * 4, &scr))) return rc;
    a.scratch = scr;
  }
  if ((rc = ws_get("di_moments", (size_t)(P->n_mom_bl > 0 ? P->n_mom_bl : 1) * 48 * sizeof(float), &mom))) return rc;
  if ((rc = ws_get("di_aux", (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 4 * sizeof(float), &aux))) return rc;
  if ((rc = ws_get("di_gnew", (size_t)(L->n_gain > 0 ? L->n_gain : 1) * 8 * sizeof(float), &gnew))) return rc;
  if ((rc = ws_get("wf_state", (size_t)n_int * 2 * sizeof(int32_t), &st))) return rc;
  a.moments = (const float*)mom;
  a.aux = (float*)aux;
  a.gnew = (float*)gnew;
  a.k0 = (int32_t*)st;
  a.gate = a.k0 + n_int;
  a.gate_tol = wf->gate_tol;
  float* g = (float*)gains;
  GC_CUDA_I(di_launch_init(a, n_int, P->n_active0, stream));
  a.weights = opt->weights;
  GC_CUDA_I(moment_pass(1, (const float*)vis, (const float*)model, (float*)mom, a.row_off, a.mom_off, a.n_samp,
                        a.n_bl, P->mitem_int, P->mitem_tile, P->n_mitems, P->ns_max, stream,
                        (const float*)opt->weights));
  const int n_waves = (wf->n_t + lag - 1) / lag;
  auto wave_lo = [&](int w) { return std::min(w * lag, wf->n_t) * nfb; };
  int n0_active = 0;
  for (int i = 0; i < wave_lo(1); ++i) n0_active += (int64_t)L->n_samp[i] * L->n_bl[i] > 0;
  GC_CUDA_I(di_launch_wf_hold(a, n_int, wave_lo(1), n0_active, stream));
  GC_CUDA_I(di_launch_maux(1, g, a.aux, L->n_gain, stream));
  g_launches += 4;
  if (wf->used_out) GC_CUDA(cudaMemsetAsync(wf->used_out, 0, (size_t)n_int * sizeof(int32_t), s));
  std::vector<int32_t> fi;
  if ((rc = first_items_host(P, fi, s))) return rc;
  // the iteration segment: S iterations and the advance of *kbase, captured once per argument set
  const Tune& tn = P->tune;
  const int S = tn.check_every;
  const bool use_loop = tn.loop && P->lgrid > 0;
  if (!use_loop) {
    DIArgs ga = a;
    ga.k = 0;
    ga.vis = ga.model = nullptr;
    if (!P->gexec || P->gS != S || memcmp(&P->gargs, &ga, sizeof(DIArgs)) != 0) {
      if (P->gexec) { cudaGraphExecDestroy(P->gexec); P->gexec = nullptr; }
      cudaStream_t cs = nullptr;
      GC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      GC_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      int crc = 0;
      for (int j = 1; j <= S && !crc; ++j) {
        DIArgs x = ga;
        x.k = j;
        crc = di_launch_mstep(1, x, P->grid, P->smem, n_int, tn.red_chunks, tn.prefetch, cs);
      }
      if (!crc) crc = di_launch_advance(a.kbase, S, cs);
      cudaGraph_t gr = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &gr);
      cudaStreamDestroy(cs);
      if (crc) return cuda_fail((cudaError_t)crc, "capture of the iteration segment");
      if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
      const cudaError_t ie = cudaGraphInstantiate(&P->gexec, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
      P->gargs = ga;
      P->gS = S;
    }
  }
  // the host reads the state of the win = max_lead + 3 times before the next wave
  const int ml = wf->max_lead, win = ml + 3;
  const int gate_n = win * nfb;
  int32_t* hb = nullptr;
  if ((rc = pinned_ints((size_t)(3 + 2 * gate_n), &hb))) return rc;
  int32_t* h_act = hb + 3;
  int32_t* h_gate = hb + 3 + gate_n;
  std::vector<int32_t> hoff;
  std::vector<float> lead;
  int next = 1, kb = 0;
  const int64_t max_segments = (int64_t)n_waves * (opt->max_iter / S + 2) + 16;
  unsigned* bar = nullptr;
  if (use_loop && (rc = loop_barrier(&bar, s))) return rc;
  int* lerr = use_loop ? (int*)(bar + 2) : nullptr;
  for (int64_t seg = 0; seg < max_segments; ++seg) {
    if (use_loop) {
      GC_CUDA_I(di_launch_mloop(1, a, P->lgrid, P->lsmem, n_int, S, tn.red_chunks, tn.prefetch, bar, lerr, stream));
      g_launches++;
    } else {
      GC_CUDA(cudaGraphLaunch(P->gexec, s));
      g_launches += (int64_t)S * 2 + 1;
    }
    int t_lo = 0, tw = 0;
    if (next < n_waves) {
      tw = next * lag;
      t_lo = std::max(0, tw - win);
    }
    const int g_n = (tw - t_lo) * nfb;
    GC_CUDA(cudaMemcpyAsync(hb, a.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (use_loop) GC_CUDA(cudaMemcpyAsync(hb + 1, lerr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaMemcpyAsync(hb + 2, a.kbase, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (g_n > 0) {
      GC_CUDA(cudaMemcpyAsync(h_act, a.active + t_lo * nfb, (size_t)g_n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(h_gate, a.gate + t_lo * nfb, (size_t)g_n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    GC_CUDA(cudaStreamSynchronize(s));
    kb = hb[2];
    if (use_loop && hb[1]) return cuda_fail(cudaErrorLaunchTimeout, "grid barrier of the iteration loop timed out");
    const int n_active = hb[0];
    if (next < n_waves) {
      // every time before the wave belongs to a wave already running: it is done once all of its
      // blocks have stopped or passed the gate
      auto done = [&](int t) {
        for (int f = 0; f < nfb; ++f) {
          const int j = (t - t_lo) * nfb + f;
          if (!(h_act[j] == 0 || h_gate[j] > 0)) return false;
        }
        return true;
      };
      // the newest history time th (tw - max_lead <= th < tw) whose 4 solutions are all done
      int th = -1;
      for (int c = tw - 1; c >= std::max(0, tw - ml) && th < 0; --c) {
        bool ok = true;
        for (int j = 0; j < 4 && ok; ++j) ok = done(std::max(0, c - j));
        if (ok) th = c;
      }
      if (th >= 0) {
        const int i_lo = wave_lo(next), n = wave_lo(next + 1) - i_lo;
        hoff.resize((size_t)n * 4);
        lead.resize(n);
        for (int b = 0; b < n; ++b) {
          const int i = i_lo + b, t = i / nfb, f = i % nfb;
          for (int j = 0; j < 4; ++j) hoff[4 * b + j] = L->gain_off[std::max(0, th - j) * nfb + f];
          lead[b] = (float)(t - th) / wf->lead_scale;
        }
        if ((rc = warm_range(L, P, a, g, hoff.data(), lead.data(), wf->net, 1, i_lo, n, fi.data(), g, wf->used_out,
                             nullptr, nullptr, stream)))
          return rc;
        GC_CUDA_I(di_launch_wf_activate(a, i_lo, n, stream));
        g_launches++;
        if (wf->wave_k_out) wf->wave_k_out[next] = kb;
        ++next;
        continue;
      }
    }
    if (n_active <= 0 && next >= n_waves) break;
  }
  if (wf->wave_k_out) wf->wave_k_out[0] = 0;
  GC_CUDA_I(gauge_fix(1, GC_DTYPE_C64, gains, a.gain_off, a.n_ant, n_int, stream));
  g_launches++;
  if (opt->compute_chi2) {
    GC_CUDA_I(moment_chi2(1, (const float*)vis, (const float*)model, g, a.row_off, a.n_samp, a.n_bl, a.bl_off,
                          a.gain_off, a.ant1, a.ant2, P->mitem_int, P->mitem_tile, P->n_mitems, P->mfirst, P->mcount,
                          P->mchi2, P->chi2_out, n_int, stream, (const float*)opt->weights));
    g_launches += 2;
  }
  if (iters_out) GC_CUDA(cudaMemcpyAsync(iters_out, a.iters, (size_t)n_int * 4, cudaMemcpyDeviceToDevice, s));
  if (status_out) GC_CUDA(cudaMemcpyAsync(status_out, a.status, (size_t)n_int * 4, cudaMemcpyDeviceToDevice, s));
  if (chi2_out && opt->compute_chi2)
    GC_CUDA(cudaMemcpyAsync(chi2_out, P->chi2_out, (size_t)n_int * 8, cudaMemcpyDeviceToDevice, s));
  std::vector<int32_t> stv(n_int);
  GC_CUDA(cudaMemcpyAsync(stv.data(), a.status, (size_t)n_int * 4, cudaMemcpyDeviceToHost, s));
  int* berr = nullptr;
  if ((rc = pinned_flag(&berr))) return rc;
  GC_CUDA(cudaMemcpyAsync(berr + 5, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  if (berr[5]) return cuda_fail(cudaErrorLaunchTimeout, "a bulk copy of an accumulate tile did not complete");
  int bad = 0;
  for (int i = 0; i < n_int; ++i) bad += (stv[i] & 15) != GC_ST_OK;
  if (next < n_waves) return GC_ERR_LIMIT;  // the segment bound ran out before every wave joined
  return bad;
}

static int run_di_acc(int kind, const void* vis, const void* model, const gc_layout* L, const void* gains, int dtype,
                      void* jhd, void* jhj, void* stream) {
  if (!L) return GC_ERR_ARG;
  if (dtype != GC_DTYPE_C64 && dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  int rc = validate_layout(L, 1);
  if (rc != GC_OK) return rc;
  if (L->n_intervals == 0) return GC_OK;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && (!gains || !jhd || !jhj))) return GC_ERR_ARG;
  DIPlan* P = nullptr;
  rc = get_di_plan(0, kind, dtype, 1, L, &P, stream);
  if (rc != GC_OK) return rc;
  DIArgs a = P->args;
  a.kbase = nullptr;
  a.vis = vis;
  a.model = model;
  a.gains = const_cast<void*>(gains);
  a.jhd_out = jhd;
  a.jhj_out = jhj;
  a.k = 1;
  if (P->scr_elems > 0) {
    void* scr = nullptr;
    if ((rc = ws_get("di_scratch", (size_t)P->scr_elems * (dtype == GC_DTYPE_C64 ? 4 : 8), &scr))) return rc;
    a.scratch = scr;
  }
  // zero the outputs of antennas without data, then one pass
  const size_t eb = elem_bytes(kind, dtype);
  GC_CUDA(cudaMemsetAsync(jhd, 0, (size_t)L->n_gain * eb, (cudaStream_t)stream));
  GC_CUDA(cudaMemsetAsync(jhj, 0, (size_t)L->n_gain * (kind == 0 ? eb / 2 : eb), (cudaStream_t)stream));
  GC_CUDA_I(di_launch_init(a, P->n_int, P->n_active0, stream));
  GC_CUDA_I(di_launch_iter(kind, dtype, 1, a, P->grid, P->smem, stream));
  g_launches += 2;
  return GC_OK;
}

static int run_chi2(int kind, const void* vis, const void* model, const gc_layout* L, const void* gains, int dtype,
                    double* chi2_out, void* stream) {
  if (!L || !chi2_out) return GC_ERR_ARG;
  if (dtype != GC_DTYPE_C64 && dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  int rc = validate_layout(L, 1);
  if (rc != GC_OK) return rc;
  if (L->n_intervals == 0) return GC_OK;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && !gains)) return GC_ERR_ARG;
  DIPlan* P = nullptr;
  if ((rc = get_di_plan(0, kind, dtype, 1, L, &P, stream))) return rc;
  DIArgs a = P->args;
  a.kbase = nullptr;
  a.vis = vis;
  a.model = model;
  a.gains = const_cast<void*>(gains);
  GC_CUDA_I(di_launch_chi2(kind, dtype, a, P->chi2_items, chi2_out, P->n_int, P->grid, stream));
  g_launches += 2;
  return GC_OK;
}

// Smoothing (Sect. 3.4): every sample of the grid is one solution interval of one sample for the
// accumulation pass; its per-antenna sums are convolved along frequency, then time, and each
// sample's gains updated from the smoothed sums.
static int run_smooth(int kind, const void* vis, const void* model, const gc_smooth* sm, void* gains,
                      const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                      void* stream) {
  if (!sm || !opt) return GC_ERR_ARG;
  if (opt->dtype != GC_DTYPE_C64) return GC_ERR_DTYPE;
  if (opt->max_iter < 1 || !(opt->tol >= 0.0) || (opt->schedule != GC_SCHED_STEFCAL && opt->schedule != GC_SCHED_GN))
    return GC_ERR_ARG;
  if (opt->host_buffers || opt->reserved || opt->weights) return GC_ERR_ARG;
  if (sm->n_t < 1 || sm->n_f < 1 || sm->n_bl < 1 || sm->n_ant < 2 || !sm->ant1 || !sm->ant2) return GC_ERR_ARG;
  if (!(sm->sigma_t >= 0.0) || !(sm->sigma_f >= 0.0) || sm->sigma_t > 1e4 || sm->sigma_f > 1e4) return GC_ERR_ARG;
  if (!vis || !model || !gains) return GC_ERR_ARG;
  const int64_t n_s = (int64_t)sm->n_t * sm->n_f;
  if (n_s > INT32_MAX || n_s * sm->n_ant > INT32_MAX) return GC_ERR_LIMIT;
  const int n_int = (int)n_s;
  // the grid as one-sample intervals sharing one baseline table
  std::vector<int64_t> row_off(n_int);
  std::vector<int32_t> n_samp(n_int, 1), n_bl(n_int, sm->n_bl), bl_off(n_int, 0), n_ant(n_int, sm->n_ant),
      gain_off(n_int);
  for (int i = 0; i < n_int; ++i) {
    row_off[i] = (int64_t)i * sm->n_bl;
    gain_off[i] = i * sm->n_ant;
  }
  gc_layout L{n_int, row_off.data(), n_samp.data(), n_bl.data(), bl_off.data(), n_ant.data(), gain_off.data(),
              sm->n_bl, sm->ant1, sm->ant2, n_s * sm->n_bl, (int32_t)(n_s * sm->n_ant), 1};
  int rc = validate_layout(&L, 1);
  if (rc != GC_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // Gaussian taps exp(-x^2 / 2 sigma^2), |x| <= ceil(3 sigma) (one tap of 1 for sigma = 0)
  auto taps = [](double sigma, std::vector<float>& w) {
    const int R = sigma > 0.0 ? (int)std::ceil(3.0 * sigma) : 0;
    w.resize(2 * R + 1);
    for (int x = -R; x <= R; ++x) w[x + R] = sigma > 0.0 ? (float)std::exp(-0.5 * (x / sigma) * (x / sigma)) : 1.f;
    return R;
  };
  std::vector<float> wt, wf;
  const int Rt = taps(sm->sigma_t, wt), Rf = taps(sm->sigma_f, wf);
  // every antenna's (baseline * 2 + side) list in baseline order, the same for every sample, and
  // the baselines' antenna pairs
  std::vector<int32_t> ant_off(sm->n_ant + 1, 0), ent(2 * (size_t)sm->n_bl), a12(2 * (size_t)sm->n_bl);
  for (int b = 0; b < sm->n_bl; ++b) { ant_off[sm->ant1[b] + 1]++; ant_off[sm->ant2[b] + 1]++; }
  for (int p = 0; p < sm->n_ant; ++p) ant_off[p + 1] += ant_off[p];
  {
    std::vector<int32_t> fill(ant_off.begin(), ant_off.end() - 1);
    for (int b = 0; b < sm->n_bl; ++b) {
      const int p = sm->ant1[b], q = sm->ant2[b];
      ent[fill[p]++] = 2 * b;
      ent[fill[q]++] = 2 * b + 1;
      a12[2 * b] = p;
      a12[2 * b + 1] = q;
    }
  }
  // per tile of the accumulation, every antenna's first entry at or after the tile's first baseline
  const int TBr = sm_tile_rows(kind), n_tiles = (sm->n_bl + TBr - 1) / TBr;
  std::vector<int32_t> tent((size_t)(n_tiles + 1) * sm->n_ant);
  for (int p = 0; p < sm->n_ant; ++p) {
    int e = ant_off[p];
    for (int t = 0; t <= n_tiles; ++t) {
      while (e < ant_off[p + 1] && (ent[e] >> 1) < t * TBr) ++e;
      tent[(size_t)t * sm->n_ant + p] = e;
    }
  }
  const int64_t n_gain = n_s * sm->n_ant;
  const int NC = kind == 0 ? 3 : 12, GW = kind == 0 ? 2 : 8;
  void *sums = nullptr, *tmp = nullptr, *ssum = nullptr, *gnew = nullptr, *aux = nullptr;
  const size_t tb = (wt.size() + wf.size()) * sizeof(float);
  const size_t lb = (ant_off.size() + ent.size() + a12.size() + tent.size()) * sizeof(int32_t);
  if ((rc = ws_get("sm_sums", (size_t)n_gain * NC * 4, &sums)) || (rc = ws_get("sm_tmp", (size_t)n_gain * NC * 4, &tmp)) ||
      (rc = ws_get("sm_ssum", (size_t)n_gain * NC * 4, &ssum)) || (rc = ws_get("sm_gnew", (size_t)n_gain * GW * 4, &gnew)) ||
      (rc = ws_get("sm_aux", tb + 32 + (size_t)n_int * 3 * 8 + lb, &aux)))
    return rc;
  float* dtaps = (float*)aux;
  int* state = (int*)((char*)aux + ((tb + 15) & ~(size_t)15));
  double* partials = (double*)(state + 4);
  int32_t* d_a12 = (int32_t*)(partials + 3 * (size_t)n_int);  // 8-byte aligned: read as int2
  int32_t* d_off = d_a12 + a12.size();
  int32_t* d_ent = d_off + ant_off.size();
  int32_t* d_tent = d_ent + ent.size();
  GC_CUDA(cudaMemcpyAsync(dtaps, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(dtaps + wt.size(), wf.data(), wf.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d_off, ant_off.data(), ant_off.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d_ent, ent.data(), ent.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d_a12, a12.data(), a12.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d_tent, tent.data(), tent.size() * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA_I(sm_launch_init(state, stream));
  int* flag = nullptr;
  if ((rc = pinned_flag(&flag))) return rc;
  const int64_t inner = (int64_t)sm->n_ant * NC;  // floats per sample
  for (int k = 1; k <= opt->max_iter; ++k) {
    GC_CUDA_I(sm_launch_acc(kind, (const float*)vis, (const float*)model, (const float*)gains, n_int, sm->n_bl,
                            sm->n_ant, d_off, d_ent, d_a12, d_tent, state, (float*)sums, stream));
    // frequency, then time: [n_t][n_f][n_ant * NC]; an axis without smoothing (one tap of 1) is skipped
    const float* cur = (const float*)sums;
    if (Rf > 0) {
      GC_CUDA_I(sm_launch_conv(cur, (float*)tmp, sm->n_t, sm->n_f, inner, dtaps + wt.size(), Rf, state, stream));
      cur = (const float*)tmp;
      g_launches++;
    }
    if (Rt > 0) {
      GC_CUDA_I(sm_launch_conv(cur, (float*)ssum, 1, sm->n_t, (int64_t)sm->n_f * inner, dtaps, Rt, state, stream));
      cur = (const float*)ssum;
      g_launches++;
    }
    GC_CUDA_I(sm_launch_update(kind, cur, (const float*)gains, (float*)gnew, n_int, sm->n_ant, k, opt->schedule,
                               opt->max_iter, opt->tol, state, partials, stream));
    g_launches += 4;
    // the host looks at the state every kSmCheck iterations: once the grid is done every kernel of
    // the iterations launched after it returns at once (the apply kernel copies the same gains)
    constexpr int kSmCheck = 4;
    if (k % kSmCheck == 0 || k == opt->max_iter) {
      GC_CUDA(cudaMemcpyAsync(flag, state, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaStreamSynchronize(s));
      if (flag[0]) break;
    }
  }
  if (iters_out) GC_CUDA(cudaMemcpyAsync(iters_out, state + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (status_out) GC_CUDA(cudaMemcpyAsync(status_out, state + 2, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (chi2_out && opt->compute_chi2) {
    DIPlan* P = nullptr;
    if ((rc = get_di_plan(0, kind, GC_DTYPE_C64, 1, &L, &P, stream))) return rc;
    DIArgs a = P->args;
    a.kbase = nullptr;
    a.vis = vis;
    a.model = model;
    a.gains = gains;
    GC_CUDA_I(di_launch_chi2(kind, GC_DTYPE_C64, a, P->chi2_items, chi2_out, P->n_int, P->grid, stream));
    g_launches += 2;
  }
  GC_CUDA(cudaStreamSynchronize(s));
  return (flag[2] & 15) == GC_ST_OK ? 0 : 1;
}

// Time candidate launch shapes on the caller's data and record the fastest for this shape bucket.
static int autotune_di(int kind, const void* vis, const void* model, const gc_layout* L, void* gains, int dtype,
                       int iters, double* best_ms, void* stream) {
  if (!L || (kind != 0 && kind != 1) || iters < 1) return GC_ERR_ARG;
  if (dtype != GC_DTYPE_C64 && dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  int rc = validate_layout(L, 1);
  if (rc != GC_OK) return rc;
  if (L->n_intervals == 0 || L->n_gain == 0) return GC_OK;
  const int mode = dtype == GC_DTYPE_C64 ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t gb = (size_t)L->n_gain * elem_bytes(kind, dtype);
  void* saved = nullptr;
  if ((rc = ws_get("tune_gains", gb, &saved))) return rc;
  GC_CUDA(cudaMemcpyAsync(saved, gains, gb, cudaMemcpyDeviceToDevice, s));
  std::vector<Tune> cands;
  if (mode == 1) {
    for (int ch : {1, 4})
      for (int pf : {0, 1, 2, 3})
        for (int bps : {0, 2}) {
          if (pf >= 2 && ch != 1) continue;  // the staged and bulk-copy kernels reduce in one chunk
          if (pf == 3 && (kind != 1 || bps != 0)) continue;  // the bulk-copy kernel: 2x2 only
          Tune t;
          t.red_chunks = ch;
          t.prefetch = pf;
          t.bps = bps;
          cands.push_back(t);
        }
  } else {
    for (int tr : {4096, 8192, 16384, 32768})
      for (int bps : {0, 2}) {
        Tune t;
        t.target_rows = tr;
        t.bps = bps;
        cands.push_back(t);
      }
  }
  gc_options opt{};
  opt.tol = 0.0;
  opt.max_iter = iters;
  opt.dtype = dtype;
  opt.profile = 1;
  double best = 1e300;
  Tune best_t;
  for (const Tune& c : cands) {
    g_tune_override = c;
    g_tune_override_on = true;
    double t_c = 1e300;
    for (int rep = 0; rep < 2; ++rep) {  // the first run builds the plan and captures the graph
      GC_CUDA(cudaMemcpyAsync(gains, saved, gb, cudaMemcpyDeviceToDevice, s));
      rc = run_di(kind, vis, model, L, gains, &opt, nullptr, nullptr, nullptr, stream);
      if (rc < 0) break;
      t_c = g_prof.ms;
    }
    g_tune_override_on = false;
    if (rc == GC_ERR_CUDA) return rc;
    if (rc < 0) continue;  // shape not launchable (e.g. shared memory): skip
    if (t_c < best) { best = t_c; best_t = c; }
  }
  g_tune_override_on = false;
  GC_CUDA(cudaMemcpyAsync(gains, saved, gb, cudaMemcpyDeviceToDevice, s));
  GC_CUDA(cudaStreamSynchronize(s));
  if (best < 1e300) g_tune[tune_bucket(kind, dtype, mode, L)] = best_t;
  if (best_ms) *best_ms = best < 1e300 ? best : -1.0;
  return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" {

int gc_calibrate_di_scalar(const void* vis, const void* model, const gc_layout* layout, void* gains,
                           const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                           void* stream) {
  return run_di(0, vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream);
}

int gc_calibrate_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, void* gains,
                             const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                             void* stream) {
  return run_di(1, vis, model, layout, gains, opt, iters_out, chi2_out, status_out, stream);
}

int gc_calibrate_di_jones2x2_warm(const void* vis, const void* model, const gc_layout* layout, const gc_warm* warm,
                                  void* gains, const gc_options* opt, int32_t* iters_out, double* chi2_out,
                                  int32_t* status_out, void* stream) {
  if (!warm || !opt || !layout || !warm->solutions || !warm->hist_off || !warm->lead || warm->n_solutions < 0)
    return GC_ERR_ARG;
  if (opt->dtype != GC_DTYPE_C64) return GC_ERR_DTYPE;
  if (opt->host_buffers != 0 || (opt->path != GC_PATH_AUTO && opt->path != GC_PATH_MOMENTS)) return GC_ERR_ARG;
  int rc = validate_layout(layout, 1);
  if (rc != GC_OK) return rc;
  for (int i = 0; i < layout->n_intervals; ++i)
    for (int j = 0; j < 4; ++j) {
      const int64_t o = warm->hist_off[4 * i + j];
      if (o < 0 || o + layout->n_ant[i] > warm->n_solutions) return GC_ERR_ARG;
    }
  if (warm->net && (rc = mlp_check(warm->net))) return rc;
  gc_options o2 = *opt;
  o2.path = GC_PATH_MOMENTS;
  return run_di(1, vis, model, layout, gains, &o2, iters_out, chi2_out, status_out, stream, warm);
}

int gc_calibrate_di_jones2x2_wavefront(const void* vis, const void* model, const gc_layout* layout,
                                       const gc_wavefront* wf, void* gains, const gc_options* opt, int32_t* iters_out,
                                       double* chi2_out, int32_t* status_out, void* stream) {
  return run_wavefront(vis, model, layout, wf, gains, opt, iters_out, chi2_out, status_out, stream);
}

int gc_gauge_fix_di(int32_t kind, void* gains, const gc_layout* layout, int32_t dtype, void* stream) {
  if (!layout || (kind != 0 && kind != 1)) return GC_ERR_ARG;
  if (dtype != GC_DTYPE_C64 && dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  int rc = validate_layout(layout, 1);
  if (rc != GC_OK) return rc;
  const int n = layout->n_intervals;
  if (n == 0 || layout->n_gain == 0) return GC_OK;
  if (!gains) return GC_ERR_ARG;
  void* dv = nullptr;
  if ((rc = ws_get("gauge_meta", (size_t)n * 8, &dv))) return rc;
  int32_t* d = (int32_t*)dv;
  cudaStream_t s = (cudaStream_t)stream;
  GC_CUDA(cudaMemcpyAsync(d, layout->gain_off, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA(cudaMemcpyAsync(d + n, layout->n_ant, (size_t)n * 4, cudaMemcpyHostToDevice, s));
  GC_CUDA_I(gauge_fix(kind, dtype, gains, d, d + n, n, stream));
  g_launches++;
  GC_CUDA(cudaStreamSynchronize(s));
  return GC_OK;
}

int gc_jhj_jhr_di_scalar(const void* vis, const void* model, const gc_layout* layout, const void* gains, int32_t dtype,
                         void* jhd_out, void* jhj_out, void* stream) {
  return run_di_acc(0, vis, model, layout, gains, dtype, jhd_out, jhj_out, stream);
}

int gc_jhj_jhr_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, const void* gains,
                           int32_t dtype, void* jhd_out, void* jhj_out, void* stream) {
  return run_di_acc(1, vis, model, layout, gains, dtype, jhd_out, jhj_out, stream);
}

int gc_calibrate_di_smooth_scalar(const void* vis, const void* model, const gc_smooth* sm, void* gains,
                                  const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                                  void* stream) {
  return run_smooth(0, vis, model, sm, gains, opt, iters_out, chi2_out, status_out, stream);
}

int gc_calibrate_di_smooth_jones2x2(const void* vis, const void* model, const gc_smooth* sm, void* gains,
                                    const gc_options* opt, int32_t* iters_out, double* chi2_out, int32_t* status_out,
                                    void* stream) {
  return run_smooth(1, vis, model, sm, gains, opt, iters_out, chi2_out, status_out, stream);
}

int gc_chi2_di_jones2x2(const void* vis, const void* model, const gc_layout* layout, const void* gains,
                        int32_t dtype, double* chi2_out, void* stream) {
  return run_chi2(1, vis, model, layout, gains, dtype, chi2_out, stream);
}

int gc_autotune_di(int32_t kind, const void* vis, const void* model, const gc_layout* layout, void* gains,
                   int32_t dtype, int32_t iters, double* best_ms, void* stream) {
  return autotune_di(kind, vis, model, layout, gains, dtype, iters, best_ms, stream);
}

const char* gc_error_string(int code) {
  switch (code) {
    case GC_OK: return "ok";
    case GC_ERR_ARG: return "invalid argument";
    case GC_ERR_LAYOUT: return "inconsistent layout";
    case GC_ERR_ANTENNA: return "antenna index out of range or autocorrelation";
    case GC_ERR_DTYPE: return "unsupported dtype";
    case GC_ERR_CUDA: return "CUDA error";
    case GC_ERR_LIMIT: return "size beyond a library limit";
    default: return code > 0 ? "some intervals did not converge" : "unknown error";
  }
}

const char* gc_status_string(int status) {
  switch (status & 15) {
    case GC_ST_OK: return (status & GC_ST_SINGULAR_FLAG) ? "converged (singular antenna)" : "converged";
    case GC_ST_NOT_CONVERGED: return "not converged";
    case GC_ST_NONFINITE: return "non-finite gains";
    case GC_ST_NODATA: return "no data";
    default: return "unknown";
  }
}

const char* gc_last_cuda_error(void) { return gc::last_cuda_error(); }

int gc_set_wait_limit(int32_t tries) {
  GC_CUDA_I(gc::di_set_bulk_wait_tries(tries));
  return GC_OK;
}

int gc_profile_detail(double* moment_pass_ms, int64_t* baseline_iterations, int32_t* path) {
  if (moment_pass_ms) *moment_pass_ms = gc::g_prof.moment_ms;
  if (baseline_iterations) *baseline_iterations = gc::g_prof.bl_iters;
  if (path) *path = gc::g_prof.path;
  return GC_OK;
}

int gc_profile_last(double* iter_kernel_ms, int64_t* iter_launches, int64_t* row_iterations) {
  if (iter_kernel_ms) *iter_kernel_ms = gc::g_prof.ms;
  if (iter_launches) *iter_launches = gc::g_prof.launches;
  if (row_iterations) *row_iterations = gc::g_prof.row_iters;
  return GC_OK;
}

int64_t gc_launch_count(void) { return (int64_t)gc::g_launches.load(); }

int gc_profile_lm(double* lm_ms, int64_t* launches, double* flop) { return gc::lm_profile(lm_ms, launches, flop); }

int gc_profile_lm_phases(double* cycles, int32_t n) {
  if (!cycles || n < 0) return GC_ERR_ARG;
  return gc::lm_profile_phases(cycles, n);
}

int gc_release(void) {
  for (auto& kv : gc::g_ws) {
    if (kv.second.p) cudaFree(kv.second.p);
  }
  gc::g_ws.clear();
  for (auto& m : gc::g_di_plan)
    for (auto& a : m)
      for (auto& b : a)
        for (auto& c : b) {
          if (c.dev) cudaFree(c.dev);
          if (c.gexec) cudaGraphExecDestroy(c.gexec);
          c = gc::DIPlan{};
        }
  gc::dd_release();
  gc::ddpol_release();
  gc::res_release();
  gc::g_tune.clear();
  if (gc::g_pinned_flag) { cudaFreeHost(gc::g_pinned_flag); gc::g_pinned_flag = nullptr; }
  if (gc::g_pinned_ints) { cudaFreeHost(gc::g_pinned_ints); gc::g_pinned_ints = nullptr; gc::g_pinned_ints_n = 0; }
  return GC_OK;
}

}  // extern "C"
