// gc_jhj_jhr_di_jones2x2_noalloc: the 2x2 accumulation pass without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a streaming pipeline that reserves all of its
// device memory at start-up and must not fail or stall on an allocation later, or a host framework
// whose own allocator owns the device memory.  This entry point runs the same kernel as
// gc_jhj_jhr_di_jones2x2 but keeps everything that kernel needs besides the caller's inputs and
// outputs -- the layout copy, the reduction slot lists, the work items, the per-interval state and
// the per-item scratch partial sums -- in one file-scope __device__ array of GC_NOALLOC_MAX_BYTES.
// Every GPU that loads the library holds that array until the process exits.
//
// The host-side name of the array is only a stand-in; the device address is obtained once per
// device with cudaGetSymbolAddress, on the first call made with that device current.  All calls
// share the array: two calls whose work overlaps on the GPU (different streams, or different host
// threads) overwrite each other's state and race.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>

#include "internal.h"

namespace gc {

int set_cuda_error(cudaError_t e, const char* what);
extern std::atomic<long long> g_launches;

constexpr size_t kArenaBytes = GC_NOALLOC_MAX_BYTES;
constexpr int kArenaMaxTables = 64;   // distinct baseline tables per call
constexpr int kArenaMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_arena[kArenaBytes];
alignas(256) static unsigned char g_noalloc_image[kArenaBytes];  // host image of the metadata part
static void* g_arena_addr[kArenaMaxDevices];

static int arena_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kArenaMaxDevices) return GC_ERR_LIMIT;
  if (!g_arena_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_arena);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_arena)");
    g_arena_addr[dev] = p;
  }
  *out = g_arena_addr[dev];
  return GC_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static int noalloc_jones_acc(const void* vis, const void* model, const gc_layout* L, const void* gains, int dtype,
                             void* jhd, void* jhj, void* stream) {
  constexpr int NC = 12, TB = kDIThreads;
  if (!L) return GC_ERR_ARG;
  if (dtype != GC_DTYPE_C64 && dtype != GC_DTYPE_C128) return GC_ERR_DTYPE;
  const int n = L->n_intervals;
  if (n < 0 || L->n_bl_table < 0 || L->n_rows < 0 || L->n_gain < 0) return GC_ERR_LAYOUT;
  if (n == 0) return GC_OK;
  if (!L->row_off || !L->n_samp || !L->n_bl || !L->bl_off || !L->n_ant || !L->gain_off) return GC_ERR_ARG;
  if (L->n_bl_table > 0 && (!L->ant1 || !L->ant2)) return GC_ERR_ARG;
  if (L->n_dir != 1) return GC_ERR_LIMIT;
  if ((L->n_rows > 0 && (!vis || !model)) || (L->n_gain > 0 && (!gains || !jhd || !jhj))) return GC_ERR_ARG;

  // distinct baseline tables, validation, and sizes (no heap use: fixed-size tables)
  int tab_bo[kArenaMaxTables], tab_nb[kArenaMaxTables], tab_nat[kArenaMaxTables];
  int n_tab = 0;
  const char* tv = getenv("GAINCAL_TARGET_ROWS_JONES");
  const int target = tv ? atoi(tv) : 8192;
  size_t n_csr_off = 0, n_csr_ent = 0, n_items = 0, scr_elems = 0;
  int na_max = 1, n_active0 = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t ns = L->n_samp[i], nb = L->n_bl[i], na = L->n_ant[i];
    if (ns < 0 || nb < 0 || na < 1) return GC_ERR_LAYOUT;
    if (na > GC_MAX_ANT) return GC_ERR_LIMIT;
    if (L->row_off[i] < 0 || L->row_off[i] + ns * nb > L->n_rows) return GC_ERR_LAYOUT;
    if (L->bl_off[i] < 0 || (int64_t)L->bl_off[i] + nb > L->n_bl_table) return GC_ERR_LAYOUT;
    if (L->gain_off[i] < 0 || (int64_t)L->gain_off[i] + na > L->n_gain) return GC_ERR_LAYOUT;
    int t = 0;
    while (t < n_tab && !(tab_bo[t] == L->bl_off[i] && tab_nb[t] == nb)) ++t;
    if (t == n_tab) {
      if (n_tab == kArenaMaxTables) return GC_ERR_LIMIT;
      int nat = 0;
      for (int b = 0; b < nb; ++b) {
        const int p = L->ant1[L->bl_off[i] + b], q = L->ant2[L->bl_off[i] + b];
        if (p < 0 || q < 0 || p == q) return GC_ERR_ANTENNA;
        nat = p + 1 > nat ? p + 1 : nat;
        nat = q + 1 > nat ? q + 1 : nat;
      }
      tab_bo[t] = L->bl_off[i]; tab_nb[t] = (int)nb; tab_nat[t] = nat;
      ++n_tab;
      const int tiles = (int)((nb + TB - 1) / TB);
      n_csr_off += (size_t)tiles * (nat + 1);
      n_csr_ent += 2 * (size_t)nb;
    }
    if (tab_nat[t] > na) return GC_ERR_ANTENNA;
    na_max = na > na_max ? (int)na : na_max;
    if (ns * nb == 0) continue;
    ++n_active0;
    int per = (int)((target + nb - 1) / nb);
    per = per < 1 ? 1 : (per > ns ? (int)ns : per);
    const int nch = (int)((ns + per - 1) / per);
    n_items += nch;
    if (nch > 1) scr_elems += (size_t)nch * tab_nat[t] * NC;
  }
  // arena layout: metadata (uploaded from the host image), per-call state, scratch
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += up256(bytes ? bytes : 1); return o; };
  const size_t o_row_off = take((size_t)n * 8), o_item_scr = take(n_items * 8);
  const size_t o_n_samp = take((size_t)n * 4), o_n_bl = take((size_t)n * 4), o_bl_off = take((size_t)n * 4);
  const size_t o_n_ant = take((size_t)n * 4), o_gain_off = take((size_t)n * 4);
  const size_t o_ant1 = take((size_t)L->n_bl_table * 4), o_ant2 = take((size_t)L->n_bl_table * 4);
  const size_t o_itab = take((size_t)n * 4), o_tab_base = take((size_t)n_tab * 4), o_tab_nant = take((size_t)n_tab * 4);
  const size_t o_csr_off = take(n_csr_off * 4), o_csr_ent = take(n_csr_ent * 4);
  const size_t o_item_int = take(n_items * 4), o_item_s0 = take(n_items * 4), o_item_s1 = take(n_items * 4);
  const size_t o_n_chunks = take((size_t)n * 4), o_first = take((size_t)n * 4);
  const size_t meta_bytes = off;
  const size_t o_active = take((size_t)n * 4), o_iters = take((size_t)n * 4), o_status = take((size_t)n * 4);
  const size_t o_counters = take((size_t)n * 4), o_misc = take(64);
  const size_t o_scratch = take(scr_elems * (dtype == GC_DTYPE_C64 ? 4 : 8));
  if (off > kArenaBytes) return GC_ERR_LIMIT;

  // host image
  unsigned char* H = g_noalloc_image;
  auto i32 = [&](size_t o) { return reinterpret_cast<int32_t*>(H + o); };
  memcpy(H + o_row_off, L->row_off, (size_t)n * 8);
  memcpy(H + o_n_samp, L->n_samp, (size_t)n * 4);
  memcpy(H + o_n_bl, L->n_bl, (size_t)n * 4);
  memcpy(H + o_bl_off, L->bl_off, (size_t)n * 4);
  memcpy(H + o_n_ant, L->n_ant, (size_t)n * 4);
  memcpy(H + o_gain_off, L->gain_off, (size_t)n * 4);
  if (L->n_bl_table) {
    memcpy(H + o_ant1, L->ant1, (size_t)L->n_bl_table * 4);
    memcpy(H + o_ant2, L->ant2, (size_t)L->n_bl_table * 4);
  }
  // reduction slot lists per table and tile: for antenna a, the partial-sum slots of its p side
  // (ant1 == a) and q side (ant2 == a) in slot order
  int32_t* csr_off = i32(o_csr_off);
  int32_t* csr_ent = i32(o_csr_ent);
  size_t co = 0, ce = 0;
  for (int t = 0; t < n_tab; ++t) {
    i32(o_tab_base)[t] = (int32_t)co;
    i32(o_tab_nant)[t] = tab_nat[t];
    const int bo = tab_bo[t], nb = tab_nb[t], nat = tab_nat[t];
    const int tiles = (nb + TB - 1) / TB;
    for (int tile = 0; tile < tiles; ++tile) {
      const int s1 = nb - tile * TB < TB ? nb - tile * TB : TB;
      for (int a = 0; a < nat; ++a) {
        csr_off[co++] = (int32_t)ce;
        for (int s = 0; s < s1; ++s) {
          if (L->ant1[bo + tile * TB + s] == a) csr_ent[ce++] = s * (2 * NC + 1);
          if (L->ant2[bo + tile * TB + s] == a) csr_ent[ce++] = s * (2 * NC + 1) + NC;
        }
      }
      csr_off[co++] = (int32_t)ce;
    }
  }
  // work items (same policy as the allocating path)
  size_t it = 0;
  int64_t scr = 0;
  for (int i = 0; i < n; ++i) {
    int t = 0;
    while (!(tab_bo[t] == L->bl_off[i] && tab_nb[t] == L->n_bl[i])) ++t;
    i32(o_itab)[i] = t;
    const int ns = L->n_samp[i], nb = L->n_bl[i];
    i32(o_first)[i] = (int32_t)it;
    if ((int64_t)ns * nb == 0) { i32(o_n_chunks)[i] = 0; continue; }
    int per = (target + nb - 1) / nb;
    per = per < 1 ? 1 : (per > ns ? ns : per);
    const int nch = (ns + per - 1) / per;
    i32(o_n_chunks)[i] = nch;
    for (int c = 0; c < nch; ++c, ++it) {
      i32(o_item_int)[it] = i;
      i32(o_item_s0)[it] = c * per;
      i32(o_item_s1)[it] = (c + 1) * per < ns ? (c + 1) * per : ns;
      int64_t so = -1;
      if (nch > 1) { so = scr; scr += (int64_t)tab_nat[t] * NC; }
      reinterpret_cast<int64_t*>(H + o_item_scr)[it] = so;
    }
  }

  void* arena = nullptr;
  int rc = arena_address(&arena);
  if (rc != GC_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(arena, H, meta_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return set_cuda_error(e, "cudaMemcpyAsync(arena)");
  unsigned char* D = static_cast<unsigned char*>(arena);
  DIArgs a{};
  a.vis = vis;
  a.model = model;
  a.gains = const_cast<void*>(gains);
  a.row_off = (const int64_t*)(D + o_row_off);
  a.item_scr = (const int64_t*)(D + o_item_scr);
  a.n_samp = (const int32_t*)(D + o_n_samp);
  a.n_bl = (const int32_t*)(D + o_n_bl);
  a.bl_off = (const int32_t*)(D + o_bl_off);
  a.n_ant = (const int32_t*)(D + o_n_ant);
  a.gain_off = (const int32_t*)(D + o_gain_off);
  a.ant1 = (const int32_t*)(D + o_ant1);
  a.ant2 = (const int32_t*)(D + o_ant2);
  a.itab = (const int32_t*)(D + o_itab);
  a.tab_base = (const int32_t*)(D + o_tab_base);
  a.tab_nant = (const int32_t*)(D + o_tab_nant);
  a.csr_off = (const int32_t*)(D + o_csr_off);
  a.csr_ent = (const int32_t*)(D + o_csr_ent);
  a.item_int = (const int32_t*)(D + o_item_int);
  a.item_s0 = (const int32_t*)(D + o_item_s0);
  a.item_s1 = (const int32_t*)(D + o_item_s1);
  a.n_chunks = (const int32_t*)(D + o_n_chunks);
  a.first_item = (const int32_t*)(D + o_first);
  a.active = (int32_t*)(D + o_active);
  a.iters = (int32_t*)(D + o_iters);
  a.status = (int32_t*)(D + o_status);
  a.counters = (int32_t*)(D + o_counters);
  a.n_active = (int32_t*)(D + o_misc);
  a.qhead = (int32_t*)(D + o_misc) + 4;
  a.scratch = D + o_scratch;
  a.n_items = (int32_t)n_items;
  a.na_max = na_max;
  a.jhd_out = jhd;
  a.jhj_out = jhj;
  a.k = 1;
  const int smem = di_smem_bytes(1, dtype, na_max);
  int dev = 0, nsm = 0, max_smem = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return set_cuda_error(e, "cudaDeviceGetAttribute");
  if ((e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return set_cuda_error(e, "cudaDeviceGetAttribute");
  if (smem > max_smem) return GC_ERR_LIMIT;
  int ce2 = di_max_blocks_per_sm(1, dtype, 1, smem, &per_sm);
  if (ce2) return set_cuda_error((cudaError_t)ce2, "occupancy");
  if (per_sm < 1) return GC_ERR_LIMIT;
  int grid = nsm * per_sm;
  if ((size_t)grid > n_items) grid = n_items > 0 ? (int)n_items : 1;
  // outputs of antennas without data stay zero; the state (counters, queue heads) starts at zero
  const size_t eb = dtype == GC_DTYPE_C64 ? 32 : 64;
  if ((e = cudaMemsetAsync(jhd, 0, (size_t)L->n_gain * eb, s)) != cudaSuccess) return set_cuda_error(e, "memset");
  if ((e = cudaMemsetAsync(jhj, 0, (size_t)L->n_gain * eb, s)) != cudaSuccess) return set_cuda_error(e, "memset");
  int le = di_launch_init(a, n, n_active0, stream);
  if (le) return set_cuda_error((cudaError_t)le, "di_init_kernel");
  le = di_launch_iter(1, dtype, 1, a, grid, smem, stream);
  if (le) return set_cuda_error((cudaError_t)le, "di_iter_kernel");
  g_launches += 2;
  return GC_OK;
}

}  // namespace gc

extern "C" int gc_jhj_jhr_di_jones2x2_noalloc(const void* vis, const void* model, const gc_layout* layout,
                                               const void* gains, int32_t dtype, void* jhd_out, void* jhj_out,
                                               void* stream) {
  return gc::noalloc_jones_acc(vis, model, layout, gains, dtype, jhd_out, jhj_out, stream);
}
