// gwcp_analyze_noalloc: the whole analysis of a small trace without any allocation.
//
// Some callers cannot allocate device memory at the point where they want a trace
// analysed: code running while another component owns the memory pool, a runtime
// hook that must not call cudaMalloc/cudaFree (both can synchronise the device), or
// an embedding whose allocator is unavailable. This entry point takes the trace and
// the output buffer from the caller and carves every intermediate buffer out of one
// file-scope __device__ array of fixed size, so it calls no cudaMalloc, cudaFree or
// other allocating routine. It runs the same kernels as gwcp_compute_order.
//
// The scratch array is shared by every call in the process on a device and keeps the
// previous call's contents; each call clears what must start at zero. Calls that
// overlap on the GPU (on different streams, or from different threads) race on it.
// The array is reserved when this module is loaded on a device, which lazy module
// loading defers to the first call here (n = 0 is enough): callers make that call at
// initialisation, before any stream capture.
#include <algorithm>

#include "gwcp_internal.cuh"

namespace gwcp {
void phaseE_scan(const Bufs& b, const Sizes& z, cudaStream_t s, Prof& p);
void phaseF_deps(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
size_t check_chunks(uint32_t n_acc);
size_t check_group_count(uint32_t n_acc);
}  // namespace gwcp

using namespace gwcp;

namespace {

constexpr size_t kScratchBytes = size_t(96) << 20;  // 96 MiB per device
constexpr uint64_t kMaxEventsNoalloc = uint64_t(1) << 18;
constexpr uint32_t kMaxAgentsNoalloc = 256;

// Device-side scratch. In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array in the current device's context. Looked up on
// every call: an address belongs to a context, and a cached one would go stale after
// cudaDeviceReset or under another context on the same ordinal. The first lookup on a
// device loads this library's module there (lazy module loading), which is when the
// array is reserved; later lookups are cheap.
int scratch_base(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return GWCP_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return GWCP_OK;
}

struct Arena {
  unsigned char* base;
  size_t used = 0;
  bool full = false;
  template <typename T>
  T* take(size_t count) {
    const size_t bytes = ((count ? count : 1) * sizeof(T) + 255) & ~size_t(255);
    if (used + bytes > kScratchBytes) {
      full = true;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

__global__ void k_races_out(const uint64_t* keys, uint64_t n, gwcp_race* out) {
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = gwcp_race{keys[i] & 0xFFFFFFFFull, keys[i] >> 32};
}

// host reads of device scalars into host stack memory (synchronous, no allocation)
int read_back(cudaStream_t s, DevStatus* st_h, const DevStatus* st_d, uint32_t* vals,
              const uint32_t* const* ptrs, int n) {
  cudaMemcpyAsync(st_h, st_d, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  for (int i = 0; i < n; ++i) cudaMemcpyAsync(vals + i, ptrs[i], sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return GWCP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
}

int analyze(const Event* ev, uint64_t n, const Geo& g, gwcp_race* out, uint64_t cap, uint64_t* n_races,
            uint64_t* bad_index, cudaStream_t s, unsigned char* scratch) {
  Arena A{scratch};
  Bufs b{};
  Sizes z{};
  Prof prof;  // off
  DevStatus st{};
  uint32_t v[8] = {};
  z.N = n;
  z.TA = 2048;
  z.ntA = uint32_t((n + z.TA - 1) / z.TA);
  b.ev = ev;
  b.st = A.take<DevStatus>(1);
  b.hist_a = A.take<uint32_t>(size_t(g.W) * z.ntA + 1);
  b.tile_cnt = A.take<uint32_t>(3 * (size_t(z.ntA) + 1));
  const size_t scan_need = std::max({scan_tmp_need(size_t(g.W) * z.ntA + 1), radix_tmp_need(n + 1),
                                     scan_tmp_need(n + 1)}) + 64;
  uint32_t* scan1 = A.take<uint32_t>(scan_need);
  b.scan_tmp = scan1;
  if (A.full) return GWCP_ERR_UNSUPPORTED;
  DevStatus init{};
  init.bad_index = ~0ull;
  init.key_and = ~0ull;
  init.lock_and = ~0ull;
  cudaMemcpyAsync(b.st, &init, sizeof(init), cudaMemcpyHostToDevice, s);

  phaseA_count(b, g, z, s, prof);
  {
    const uint32_t* p[4] = {b.hist_a + size_t(g.W) * z.ntA, b.tile_cnt + z.ntA, b.tile_cnt + 2 * z.ntA + 1,
                            b.tile_cnt + 3 * z.ntA + 2};
    if (int rc = read_back(s, &st, b.st, v, p, 4)) return rc;
  }
  int code = st.code;
  if (code && code != GWCP_ERR_INVALID_TRACE) return code;
  z.nS = v[0];
  z.n_acc = v[1];
  z.n_acqrel = v[2];
  z.n_bar = v[3];
  z.n_sync = z.nS - z.n_acc;
  const uint64_t key_mask = st.key_or ^ st.key_and;
  const uint64_t lock_mask = st.lock_or ^ st.lock_and;
  const size_t ns1 = size_t(z.n_sync) + 1, na1 = size_t(z.n_acqrel) + 1;
  b.S = A.take<uint32_t>(z.nS);
  b.seg = A.take<uint32_t>(g.W + 1);
  b.acqrel = A.take<uint32_t>(z.n_acqrel);
  b.bar = A.take<uint32_t>(z.n_bar);
  b.acc_key = A.take<uint64_t>(z.n_acc);
  b.acc_idx = A.take<uint32_t>(z.n_acc);
  b.acc_key2 = A.take<uint64_t>(z.n_acc);
  b.acc_idx2 = A.take<uint32_t>(z.n_acc);
  b.sy_cnt = A.take<uint32_t>(z.nS / 512 + 2);
  uint32_t** sy[] = {&b.sy_spos, &b.sy_idx, &b.sy_kind, &b.sy_aux, &b.sy_N, &b.sy_depth, &b.sy_inner,
                     &b.sy_ver, &b.sy_match, &b.sy_relk, &b.sy_agent, &b.incs_cnt, &b.cs_of_sync};
  for (uint32_t** q : sy) *q = A.take<uint32_t>(ns1);
  z.d_shift = 8;
  while (uint64_t(g.W) * ((z.N >> z.d_shift) + 2) > (1ull << 23)) ++z.d_shift;
  z.d_nw = uint32_t((z.N >> z.d_shift) + 2);
  b.d_index = A.take<uint32_t>(size_t(g.W) * z.d_nw);
  b.sy_start = A.take<uint32_t>(g.W + 1);
  b.vcount = A.take<uint32_t>(g.W + 1);
  b.lk_key = A.take<uint64_t>(na1);
  b.lk_key2 = A.take<uint64_t>(na1);
  uint32_t** lk[] = {&b.lk_k, &b.lk_k2, &b.lk_flags, &b.lk_csid, &b.lk_rank, &b.cs_agent, &b.cs_sid,
                     &b.cs_epoch, &b.cs_rel_idx, &b.cs_rel_epoch, &b.cs_lock, &b.cs_parent, &b.acq_dep_off,
                     &b.acq_dep_cnt};
  for (uint32_t** q : lk) *q = A.take<uint32_t>(na1);
  b.lock_first = A.take<uint32_t>(na1 + 1);
  b.lock_cs_lo = A.take<uint32_t>(na1 + 1);
  if (A.full) return GWCP_ERR_UNSUPPORTED;

  phaseA_scatter(b, g, z, s, prof);
  phaseB_sync(b, g, z, s, prof);
  cudaMemsetAsync(b.vcount, 0, size_t(g.W + 1) * 4, s);
  cudaMemsetAsync(b.cs_of_sync, 0xFF, ns1 * 4, s);
  phaseC_walk(b, g, z, s, prof);
  phaseE_locks(b, g, z, lock_mask, s, prof);
  phaseE_scan(b, z, s, prof);
  {
    const uint32_t* p[5] = {b.incs_cnt + z.n_sync, b.vcount + g.W, b.lk_csid + z.n_acqrel, b.lk_flags + z.n_acqrel,
                            reinterpret_cast<const uint32_t*>(&b.st->spare[1])};
    if (int rc = read_back(s, &st, b.st, v, p, 5)) return rc;
  }
  code = st.code;
  if (code && code != GWCP_ERR_INVALID_TRACE) return code;
  z.n_incs = v[0];
  z.n_rows = v[1];
  z.n_cs = z.n_acqrel ? v[2] : 0;
  z.n_locks = z.n_acqrel ? v[3] : 0;
  z.n_exp = v[4];
  const uint32_t slots = std::min<uint32_t>(g.B + 1, lock_scope_cap(g.B));
  z.pool_cap = z.n_cs * slots + z.n_exp * 2 * slots + 64;
  b.dep_pool = A.take<uint32_t>(z.pool_cap);
  if (A.full) return GWCP_ERR_UNSUPPORTED;
  // the last validity check (W3) needs only the buffers carved so far: an invalid trace is
  // reported with its first bad index before the rest of the scratch is sized
  phaseE_walk(b, g, z, s, prof);
  if (int rc = read_back(s, &st, b.st, v, nullptr, 0)) return rc;
  if (st.code) {  // no later phase runs on an invalid trace or after an error
    if (bad_index) *bad_index = st.bad_index;
    return st.code;
  }
  const size_t ni1 = size_t(z.n_incs) + 1;
  const size_t ne1 = std::max<size_t>(size_t(z.n_exp), size_t(z.n_incs) * kMaxNest) + 1;
  b.acc_info = A.take<AccInfo>(z.N);
  uint32_t** inc[] = {&b.incs_idx, &b.incs_ver, &b.incs_k, &b.incs_wr, &b.exp_off};
  for (uint32_t** q : inc) *q = A.take<uint32_t>(ni1);
  b.incs_key = A.take<uint64_t>(ni1);
  b.ex_key = A.take<uint64_t>(ne1);
  b.ex_key2 = A.take<uint64_t>(ne1);
  uint32_t** ex[] = {&b.ex_val, &b.ex_val2, &b.ex_rec, &b.ex_cs, &b.ex_flags, &b.ex_dep_off, &b.ex_dep_cnt};
  for (uint32_t** q : ex) *q = A.take<uint32_t>(ne1);
  b.ex_group = A.take<uint32_t>(ne1 + 1);
  b.rows = A.take<uint32_t>(size_t(z.n_rows) * g.Wp);
  b.psnap = A.take<uint32_t>((size_t(z.n_cs) + 1) * g.Wp);
  b.hsnap = A.take<uint32_t>((size_t(z.n_cs) + 1) * g.Wp);
  b.done = A.take<uint32_t>(size_t(z.n_cs) + 1);
  b.plan = A.take<uint4>(2 * (size_t(z.n_sync) + z.n_incs) + 2);
  b.recmeta = A.take<uint4>(size_t(z.n_cs) + 1);
  b.flat_off = A.take<uint32_t>(ni1);
  b.flat = A.take<uint32_t>(z.pool_cap);
  b.cursor = A.take<uint32_t>(size_t(g.W) * (z.n_locks + 1));
  const size_t smem = size_t(2) * g.apb * 2 * g.Wp * 4;
  z.cta_barriers = g.apb <= 32 && smem <= 96 * 1024;
  const bool global_bars = !z.cta_barriers || g.gran == GWCP_GRAN_THREAD;
  b.bar_j = A.take<uint32_t>(global_bars ? size_t(z.n_bar) * 2 * g.Wp : 1);
  b.bar_cnt = A.take<uint32_t>(global_bars ? z.n_bar : 1);
  z.n_chunks = uint32_t(check_chunks(z.n_acc));
  const size_t ng = check_group_count(z.n_acc);
  b.tails = A.take<uint32_t>((size_t(z.n_chunks) + ng) * 4 * g.Wp * 2 + ng + 8);
  if (A.full) return GWCP_ERR_UNSUPPORTED;
  // races: the rest of the scratch, split in two sort buffers and their sort scratch
  const size_t left = kScratchBytes - A.used;
  z.race_cap = left / (2 * sizeof(uint64_t) + 8) > 4096 ? left / (2 * sizeof(uint64_t) + 8) - 4096 : 0;
  const size_t ex_bound = size_t(z.n_incs) * kMaxNest + 1;
  const size_t need2 = std::max({scan_need, radix_tmp_need(ex_bound), scan_tmp_need(ex_bound)}) + 64;
  if (need2 > scan_need) b.scan_tmp = A.take<uint32_t>(need2);
  size_t race_tmp_elems = radix_tmp_need(z.race_cap + 1) + 64;
  while (z.race_cap && A.used + 2 * ((z.race_cap * 8 + 255) & ~size_t(255)) + race_tmp_elems * 4 + 512 > kScratchBytes) {
    z.race_cap -= z.race_cap / 8 + 1;
    race_tmp_elems = radix_tmp_need(z.race_cap + 1) + 64;
  }
  b.races = A.take<uint64_t>(z.race_cap);
  b.races2 = A.take<uint64_t>(z.race_cap);
  uint32_t* race_tmp = A.take<uint32_t>(race_tmp_elems);
  if (A.full || !z.race_cap) return GWCP_ERR_UNSUPPORTED;

  cudaMemsetAsync(b.done, 0, (size_t(z.n_cs) + 1) * 4, s);
  cudaMemsetAsync(b.cursor, 0, size_t(g.W) * (z.n_locks + 1) * 4, s);
  if (global_bars && z.n_bar) {
    cudaMemsetAsync(b.bar_j, 0, size_t(z.n_bar) * 2 * g.Wp * 4, s);
    cudaMemsetAsync(b.bar_cnt, 0, size_t(z.n_bar) * 4, s);
  }
  phaseD_gaps(b, g, z, s, prof);
  phaseF_incs(b, g, z, key_mask, s, prof);
  phaseF_walk(b, g, z, key_mask, s, prof);
  z.n_groups = z.n_exp;
  phaseF_deps(b, g, z, s, prof);
  phaseH_sort(b, g, z, key_mask, b.scan_tmp, s, prof);
  if (int rc = phaseG_propagate(b, g, z, s, prof)) return rc;
  phaseI_carry(b, g, z, s, prof);
  phaseI_check(b, g, z, s, prof);
  if (int rc = read_back(s, &st, b.st, v, nullptr, 0)) return rc;
  if (st.code) {
    if (bad_index) *bad_index = st.bad_index;
    return st.code;
  }
  const uint64_t total = st.n_races;
  *n_races = total;
  if (total > z.race_cap) return GWCP_ERR_UNSUPPORTED;  // more races than the scratch holds
  b.scan_tmp = race_tmp;
  const bool second = phaseI_sort_races(b, z, total, s, prof);
  const uint64_t m = std::min<uint64_t>(total, cap);
  if (m) {
    k_races_out<<<uint32_t((m + 255) / 256), 256, 0, s>>>(second ? b.races2 : b.races, m, out);
    count_launch();
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GWCP_ERR_CUDA;
  return total > cap ? GWCP_ERR_CAPACITY : GWCP_OK;
}

}  // namespace

extern "C" int gwcp_analyze_noalloc(const gwcp_event* ev_dev, uint64_t n, const gwcp_geometry* geo,
                                    gwcp_race* races_dev, uint64_t races_cap, uint64_t* n_races,
                                    uint64_t* first_bad_index, void* cuda_stream) {
  if (!geo || !n_races || (n && !ev_dev) || (races_cap && !races_dev)) return GWCP_ERR_ARGS;
  *n_races = 0;
  if (first_bad_index) *first_bad_index = ~0ull;
  if (geo->num_agents == 0 || geo->agents_per_block == 0 || geo->reserved != 0 ||
      geo->num_agents % geo->agents_per_block != 0 || geo->granularity > 1)
    return GWCP_ERR_ARGS;
  if (n > kMaxEventsNoalloc || geo->num_agents > kMaxAgentsNoalloc) return GWCP_ERR_UNSUPPORTED;
  // set-up first, so that a zero-length call loads the module and reserves the array
  unsigned char* scratch = nullptr;
  if (int rc = scratch_base(&scratch)) return rc;
  if (n == 0) return GWCP_OK;
  Geo g{};
  g.W = geo->num_agents;
  g.apb = geo->agents_per_block;
  g.B = g.W / g.apb;
  g.gran = geo->granularity;
  uint32_t k = 1;
  while (k * 32 < g.W) k <<= 1;
  g.K = k;
  g.Wp = 32 * k;
  g.nT = 0;
  g.RW = g.Wp;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int rc = analyze(reinterpret_cast<const Event*>(ev_dev), n, g, races_dev, races_cap, n_races,
                         first_bad_index, s, scratch);
  // an early error return may leave work queued that writes the scratch: drain it, so that
  // a caller's next call (on any stream) does not overlap it
  if (rc != GWCP_OK && rc != GWCP_ERR_CAPACITY) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
  }
  return rc;
}
