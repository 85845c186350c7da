// C ABI of libgwcp (include/gwcp.h): context, trace loading, the analysis pipeline,
// race reporting, test hooks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "gwcp_internal.cuh"

namespace gwcp {
unsigned long long launch_count();
size_t check_chunks(uint32_t n_acc);
size_t check_group_count(uint32_t n_acc);
void phaseE_scan(const Bufs& b, const Sizes& z, cudaStream_t s, Prof& p);
void phaseF_deps(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);

cudaEvent_t Prof::ev() {
  if (used == pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool.push_back(e);
  }
  return pool[used++];
}
// Every phase is also an NVTX range on the host thread (profilers can filter launches
// by phase); the CUDA-event records are kept only with options.profile.
void Prof::begin(const char* name, double bytes, cudaStream_t on_stream) {
  nvtxRangePushA(name);
  if (!on) return;
  Rec r{name, ev(), ev(), bytes, on_stream ? on_stream : s};
  cudaEventRecord(r.a, r.s);
  recs.push_back(r);
}
void Prof::end() {
  nvtxRangePop();
  if (!on || recs.empty()) return;
  cudaEventRecord(recs.back().b, recs.back().s);
}
}  // namespace gwcp

using namespace gwcp;

struct gwcp_ctx {
  int device = 0;
  gwcp_options opt{};
  const Event* ev_dev = nullptr;
  Event* ev_own = nullptr;
  size_t ev_own_cap = 0;
  uint64_t n = 0;
  Geo g{};
  bool has_trace = false, computed = false;
  int compute_rc = GWCP_ERR_STATE;
  std::map<std::string, std::pair<void*, size_t>> allocs;
  Bufs b{};
  Sizes z{};
  DevStatus* st_host = nullptr;
  uint32_t* cnt_host = nullptr;  // pinned readback of sizes
  Prof prof;
  bool races_second = false;
  uint64_t n_races = 0;
  unsigned long long bad_index = ~0ull;
  uint64_t counters[GWCP_N_COUNTERS] = {};
  unsigned long long first_race_ns = 0;  // last compute: %globaltimer of its first race (0: none)
  uint64_t key_mask = 0;                 // last compute: location-key bits that vary
  bool acc_info_partial = false;         // last compute wrote the kept accesses' records only
  uint64_t clock_words[3] = {};  // last compute: tiles, pool words taken, words written
  uint64_t tile_cap_hint = 0;  // wide clocks: pool size that the last run needed
  bool compressed = false;     // GWCP_CLOCKS_COMPRESSED was in force at gwcp_load_trace
  uint64_t cv_cap_hint = 0;    // compressed versions: pool words that the last run needed
  uint64_t alloc_limit = 0;    // gwcp_debug_alloc_limit: cap on the cached buffers' bytes (0 = none)
  cudaStream_t side = nullptr;  // runs the access sort and grouping beside the main phases
  cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr;
  cudaEvent_t kept_ev = nullptr;  // the access sort's kept count has reached cnt_host[15]
  cudaEvent_t sync_ev = nullptr;  // options.blocking_sync: host waits sleep on this event
  cudaStream_t alloc_s = nullptr;  // stream that buffer (re)allocations are ordered on
  void* stage_host = nullptr;       // pinned staging for race copies into pageable memory
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  std::vector<float> rank_theta;  // gwcp_set_ranker: the MLP's parameters (empty = off)
  uint32_t clock_mode = GWCP_CLOCKS_AUTO;  // gwcp_set_clock_mode
  uint32_t check_mode = GWCP_CHECK_AUTO;   // gwcp_set_check_mode
  uint32_t n_chunks_timeline = 0; // chunks of the last check's timeline
  std::vector<float> prof_ms;
  std::vector<float> prof_start;  // ms from the first kernel's start
  std::vector<double> prof_bytes;
  std::vector<const char*> prof_names;
};

namespace {

const uint32_t kNoneHost = 0xFFFFFFFFu;
const int kRerun = 1;  // run() result: the tile or compressed-version pool was grown, run again
const uint64_t kCvMaxWords = (1ull << 31) - 1;  // compressed-version offsets have 31 bits

// Buffers come from the device's default memory pool, allocated and freed in stream
// order on the context's current stream (c->alloc_s): growing a buffer neither waits for
// the device nor blocks other streams, so contexts on other streams keep running.
template <typename T>
T* get(gwcp_ctx* c, const char* name, size_t count, bool* oom) {
  const size_t bytes = (count ? count : 1) * sizeof(T);
  auto& a = c->allocs[name];
  if (a.second < bytes) {
    if (c->alloc_limit) {  // injected memory limit: fail as an exhausted device would
      size_t held = 0;
      for (auto& kv : c->allocs) held += kv.second.second;
      if (held - a.second + bytes + bytes / 8 > c->alloc_limit) {
        *oom = true;
        return nullptr;
      }
    }
    if (a.first) cudaFreeAsync(a.first, c->alloc_s);
    a.first = nullptr;
    a.second = 0;
    const size_t want = bytes + bytes / 8;
    if (cudaMallocAsync(&a.first, want, c->alloc_s) != cudaSuccess) {
      cudaGetLastError();
      *oom = true;
      return nullptr;
    }
    a.second = want;
  }
  return static_cast<T*>(a.first);
}

// get<T> with the returned pointer aligned to `align` bytes (over-allocated by align)
template <typename T>
T* get_aligned(gwcp_ctx* c, const char* name, size_t count, size_t align, bool* oom) {
  unsigned char* p = get<unsigned char>(c, name, count * sizeof(T) + align, oom);
  if (!p) return nullptr;
  return reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(p) + align - 1) & ~uintptr_t(align - 1));
}

// Makes s the stream that buffer frees and allocations are ordered on; when the caller
// switched streams, the previous one is drained first so that no stream-ordered free can
// overtake work still queued there.
void use_stream(gwcp_ctx* c, cudaStream_t s) {
  if (c->alloc_s != s) {
    cudaStreamSynchronize(c->alloc_s);
    c->alloc_s = s;
  }
}

cudaError_t wait_stream(gwcp_ctx* c, cudaStream_t s);

constexpr size_t kStageChunk = size_t(8) << 20;  // bytes per staging half

// Device -> host copy of `bytes` into caller memory. Page-locked (or registered) memory
// takes one DMA. Pageable memory goes through the context's own two pinned halves, chunk
// by chunk (the next chunk's DMA overlaps the host copy of the previous one), instead of
// the driver's shared staging path.
int copy_to_host(gwcp_ctx* c, void* out, const void* dev, size_t bytes, cudaStream_t s) {
  cudaPointerAttributes at{};
  const bool pinned = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
                      (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (pinned || bytes <= 65536) {
    if (cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GWCP_ERR_CUDA;
    return wait_stream(c, s) == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
  }
  if (!c->stage_host) {
    if (cudaMallocHost(&c->stage_host, 2 * kStageChunk) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_ev[0], cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_ev[1], cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess) {
      cudaGetLastError();
      if (c->stage_host) cudaFreeHost(c->stage_host);
      c->stage_host = nullptr;
      if (cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GWCP_ERR_CUDA;
      return wait_stream(c, s) == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
    }
  }
  char* half[2] = {static_cast<char*>(c->stage_host), static_cast<char*>(c->stage_host) + kStageChunk};
  const size_t n = (bytes + kStageChunk - 1) / kStageChunk;
  for (size_t k = 0; k <= n; ++k) {
    if (k < n) {  // DMA of chunk k into half k % 2
      const size_t len = std::min(kStageChunk, bytes - k * kStageChunk);
      if (cudaMemcpyAsync(half[k & 1], static_cast<const char*>(dev) + k * kStageChunk, len,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaEventRecord(c->stage_ev[k & 1], s) != cudaSuccess)
        return GWCP_ERR_CUDA;
    }
    if (k > 0) {  // host copy of chunk k - 1
      const size_t j = k - 1;
      const size_t len = std::min(kStageChunk, bytes - j * kStageChunk);
      if (cudaEventSynchronize(c->stage_ev[j & 1]) != cudaSuccess) return GWCP_ERR_CUDA;
      std::memcpy(static_cast<char*>(out) + j * kStageChunk, half[j & 1], len);
    }
  }
  return GWCP_OK;
}

int cuda_rc() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
}

// waits for stream s: spinning (default) or, with options.blocking_sync, sleeping on an
// event so that many host threads can wait at once without occupying cores
cudaError_t wait_stream(gwcp_ctx* c, cudaStream_t s) {
  if (!c->sync_ev) return cudaStreamSynchronize(s);
  cudaError_t e = cudaEventRecord(c->sync_ev, s);
  return e != cudaSuccess ? e : cudaEventSynchronize(c->sync_ev);
}

int read_status(gwcp_ctx* c, cudaStream_t s, const uint32_t* const* extra, int n_extra) {
  cudaMemcpyAsync(c->st_host, c->b.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  for (int i = 0; i < n_extra; ++i)
    cudaMemcpyAsync(c->cnt_host + i, extra[i], sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (wait_stream(c, s) != cudaSuccess) return GWCP_ERR_CUDA;
  return cuda_rc();
}

// Once work is on the side stream, every exit from run() makes s wait for it, so that the
// next use of the context's buffers on s is ordered after it.
struct SideJoin {
  gwcp_ctx* c;
  cudaStream_t s;
  bool armed = false;
  void join() {
    if (!armed) return;
    cudaEventRecord(c->join, c->side);
    cudaStreamWaitEvent(s, c->join, 0);
    armed = false;
  }
  ~SideJoin() { join(); }
};

int run(gwcp_ctx* c, cudaStream_t s) {
  use_stream(c, s);
  c->first_race_ns = 0;
  Bufs& b = c->b;
  Sizes& z = c->z;
  const Geo& g = c->g;
  bool oom = false;
  z = Sizes{};
  z.N = c->n;
  z.hb_only = c->opt.hb_only != 0;
  z.pack_walkers = c->opt.pack_walkers != 0;
  z.compress = c->compressed && !g.nT;
  z.forced_barrier = c->opt.forced_barrier != 0 || z.compress;
  z.sparse_check = g.nT || z.compress || c->check_mode == GWCP_CHECK_SPARSE ||
                   (c->check_mode == GWCP_CHECK_AUTO && g.W >= kSparseCheckFromAgents);
  // many agents: S by a sort on the agent (a per-warp count table of Wp words would leave
  // phase A a few warps per SM)
  z.agent_sort = g.Wp > 2048;
  z.TA = g.Wp <= 256 || z.agent_sort ? 2048 : 8192;
  if (!z.agent_sort)
    while (uint64_t(g.W) * ((z.N + z.TA - 1) / z.TA) > (1ull << 26)) z.TA <<= 1;  // bounded agent histogram
  z.ntA = uint32_t((z.N + z.TA - 1) / z.TA);
  const size_t hist_words = z.agent_sort ? 1 : size_t(g.W) * z.ntA + 1;
  b.ev = c->ev_dev;
  b.st = get<DevStatus>(c, "st", 1, &oom);
  b.hist_a = get<uint32_t>(c, "hist_a", hist_words, &oom);
  b.tile_cnt = get<uint32_t>(c, "tile_cnt", 4 * (size_t(z.ntA) + 1), &oom);
  const size_t scan_need = std::max({scan_tmp_need(hist_words), radix_tmp_need(z.N + 1),
                                     scan_tmp_need(z.N + 1)}) + 64;
  b.scan_tmp = get<uint32_t>(c, "scan_tmp", scan_need, &oom);
  if (oom) return GWCP_ERR_OOM;
  DevStatus init{};
  init.bad_index = ~0ull;
  init.key_and = ~0ull;
  init.lock_and = ~0ull;
  cudaMemcpyAsync(b.st, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  c->prof.on = c->opt.profile != 0;
  c->prof.s = s;
  c->prof.recs.clear();
  c->prof.used = 0;

  // ---- A: counts, then sync 1 -------------------------------------------------------
  phaseA_count(b, g, z, s, c->prof);
  {
    const uint32_t* ex[4] = {z.agent_sort ? b.tile_cnt + 4 * z.ntA + 3 : b.hist_a + size_t(g.W) * z.ntA,
                             b.tile_cnt + z.ntA, b.tile_cnt + 2 * z.ntA + 1, b.tile_cnt + 3 * z.ntA + 2};
    int rc = read_status(c, s, ex, 4);
    if (rc) return rc;
  }
  int code = c->st_host->code;
  if (code && code != GWCP_ERR_INVALID_TRACE) return code;
  z.nS = c->cnt_host[0];
  z.n_acc = c->cnt_host[1];
  z.n_acqrel = c->cnt_host[2];
  z.n_bar = c->cnt_host[3];
  z.n_sync = z.nS - z.n_acc;
  const uint64_t key_mask = c->st_host->key_or ^ c->st_host->key_and;
  c->key_mask = key_mask;
  c->acc_info_partial = false;
  // grouped access order for the partner check (no ranker): the composite key (location,
  // class, agent) must fit 64 bits, i.e. the location's varying address bits at most 48
  uint64_t sort_mask = key_mask;
  if (z.sparse_check && c->rank_theta.empty()) {
    const uint64_t m = key_mask & ~(1ull << 63);
    const uint32_t lo = m ? uint32_t(__builtin_ctzll(m)) : 0u, hi = m ? uint32_t(63 - __builtin_clzll(m)) : 0u;
    const uint32_t span = m ? hi - lo + 1 : 1u;
    if (span + 1 + 15 <= 64) {
      z.grouped = true;
      z.comp_lo = lo;
      z.comp_span = span;
      uint32_t ab = 0;
      while ((1u << ab) < g.W) ++ab;
      sort_mask = (((m >> lo) | ((key_mask >> 63) << span)) << 15) | (3ull << 13) | ((1ull << ab) - 1);
      // written-location bitmap of about four bits per access
      z.wl_log2 = 16;
      while (z.wl_log2 < 31 && (1ull << z.wl_log2) < 4ull * z.n_acc) ++z.wl_log2;
    }
  }
  const uint64_t lock_mask = c->st_host->lock_or ^ c->st_host->lock_and;

  b.S = get<uint32_t>(c, "S", z.nS, &oom);
  b.seg = get<uint32_t>(c, "seg", g.W + 1, &oom);
  b.acqrel = get<uint32_t>(c, "acqrel", z.n_acqrel, &oom);
  b.bar = get<uint32_t>(c, "bar", z.n_bar, &oom);
  if (z.agent_sort) {
    b.s_key = get<uint64_t>(c, "s_key", z.nS, &oom);
    b.s_key2 = get<uint64_t>(c, "s_key2", z.nS, &oom);
    b.s_tmp = get<uint32_t>(c, "s_tmp", radix_tmp_need(size_t(z.nS) + 1) + 64, &oom);
  }
  b.acc_key = get<uint64_t>(c, "acc_key", z.n_acc, &oom);
  b.acc_idx = get<uint32_t>(c, "acc_idx", z.n_acc, &oom);
  b.acc_key2 = get<uint64_t>(c, "acc_key2", z.n_acc, &oom);
  b.acc_idx2 = get<uint32_t>(c, "acc_idx2", z.n_acc, &oom);
  // compressed versions keep local times in 31 bits; a local time is at most 1 + n_sync
  if (z.compress && z.n_sync >= kCvExpanded - 1) return GWCP_ERR_UNSUPPORTED;
  const size_t ns1 = size_t(z.n_sync) + 1;
  b.sy_cnt = get<uint32_t>(c, "sy_cnt", z.nS / 512 + 2, &oom);  // one count per 512-entry chunk of S
  b.sy_spos = get<uint32_t>(c, "sy_spos", ns1, &oom);
  b.sy_idx = get<uint32_t>(c, "sy_idx", ns1, &oom);
  b.sy_kind = get<uint32_t>(c, "sy_kind", ns1, &oom);
  b.sy_start = get<uint32_t>(c, "sy_start", g.W + 1, &oom);
  b.sy_aux = get<uint32_t>(c, "sy_aux", ns1, &oom);
  b.sy_N = get<uint32_t>(c, "sy_N", ns1, &oom);
  b.sy_depth = get<uint32_t>(c, "sy_depth", ns1, &oom);
  b.sy_inner = get<uint32_t>(c, "sy_inner", ns1, &oom);
  b.sy_ver = get<uint32_t>(c, "sy_ver", ns1, &oom);
  b.sy_match = get<uint32_t>(c, "sy_match", ns1, &oom);
  b.sy_relk = get<uint32_t>(c, "sy_relk", ns1, &oom);
  b.sy_agent = get<uint32_t>(c, "sy_agent", ns1, &oom);
  // phase D's index: windows of 2^d_shift events, at most 2^23 entries over all agents
  z.d_shift = 8;
  while (uint64_t(g.W) * ((z.N >> z.d_shift) + 2) > (1ull << 23)) ++z.d_shift;
  z.d_nw = uint32_t((z.N >> z.d_shift) + 2);
  b.d_index = get<uint32_t>(c, "d_index", size_t(g.W) * z.d_nw, &oom);
  b.incs_cnt = get<uint32_t>(c, "incs_cnt", ns1, &oom);
  b.vcount = get<uint32_t>(c, "vcount", g.W + 1, &oom);
  const size_t na1 = size_t(z.n_acqrel) + 1;
  b.lk_key = get<uint64_t>(c, "lk_key", na1, &oom);
  b.lk_k = get<uint32_t>(c, "lk_k", na1, &oom);
  b.lk_key2 = get<uint64_t>(c, "lk_key2", na1, &oom);
  b.lk_k2 = get<uint32_t>(c, "lk_k2", na1, &oom);
  b.lk_flags = get<uint32_t>(c, "lk_flags", na1, &oom);
  b.lk_csid = get<uint32_t>(c, "lk_csid", na1, &oom);
  b.lk_rank = get<uint32_t>(c, "lk_rank", na1, &oom);
  b.lock_first = get<uint32_t>(c, "lock_first", na1 + 1, &oom);
  b.lock_cs_lo = get<uint32_t>(c, "lock_cs_lo", na1 + 1, &oom);
  b.cs_of_sync = get<uint32_t>(c, "cs_of_sync", ns1, &oom);
  b.cs_agent = get<uint32_t>(c, "cs_agent", na1, &oom);
  b.cs_sid = get<uint32_t>(c, "cs_sid", na1, &oom);
  b.cs_epoch = get<uint32_t>(c, "cs_epoch", na1, &oom);
  b.cs_rel_idx = get<uint32_t>(c, "cs_rel_idx", na1, &oom);
  b.cs_rel_epoch = get<uint32_t>(c, "cs_rel_epoch", na1, &oom);
  b.cs_lock = get<uint32_t>(c, "cs_lock", na1, &oom);
  b.cs_parent = get<uint32_t>(c, "cs_parent", na1, &oom);
  b.acq_dep_off = get<uint32_t>(c, "acq_dep_off", na1, &oom);
  b.acq_dep_cnt = get<uint32_t>(c, "acq_dep_cnt", na1, &oom);
  if (z.forced_barrier) {
    const size_t nb1 = size_t(z.n_bar) + 1;
    b.fb_key = get<uint64_t>(c, "fb_key", nb1, &oom);
    b.fb_key2 = get<uint64_t>(c, "fb_key2", nb1, &oom);
    b.fb_val = get<uint32_t>(c, "fb_val", nb1, &oom);
    b.fb_val2 = get<uint32_t>(c, "fb_val2", nb1, &oom);
    b.fb_rank = get<uint32_t>(c, "fb_rank", nb1, &oom);
    b.fb_off = get<uint32_t>(c, "fb_off", nb1, &oom);
    b.fb_blo = get<uint32_t>(c, "fb_blo", size_t(g.B) + 1, &oom);
    b.fb_rec = get<uint4>(c, "fb_rec", ns1, &oom);
    b.fb_boff = get<uint32_t>(c, "fb_boff", ns1, &oom);
  }
  // scratch of the side stream's sorts and scans
  uint32_t* side_tmp = get<uint32_t>(
      c, "side_tmp", std::max(radix_tmp_need(size_t(z.n_acc) + 1), scan_tmp_need(size_t(z.n_acc) * 4 + 2)) + 64, &oom);
  if (z.wl_log2) {
    b.wl_bits = get<uint32_t>(c, "wl_bits", (size_t(1) << z.wl_log2) / 32, &oom);
    b.n_kept = get<uint32_t>(c, "n_kept", 1, &oom);
  }
  if (oom) return GWCP_ERR_OOM;

  phaseA_scatter(b, g, z, s, c->prof);
  // the access sort needs only the decoded accesses: it runs on the side stream beside the
  // main stream's other phases (measured on the 8192-warp workload: it overlaps them, and
  // the grouping ends before the propagation starts; with the side stream at a lower
  // priority the sort drifts into the propagation and slows its latency-bound walkers)
  SideJoin side{c, s};
  cudaEventRecord(c->fork, s);
  cudaStreamWaitEvent(c->side, c->fork, 0);
  side.armed = true;
  phaseH_sort(b, g, z, sort_mask, side_tmp, c->side, c->prof);
  if (z.grouped) {  // the kept count sizes the grouping and the check (read before they are enqueued)
    cudaMemcpyAsync(c->cnt_host + 15, b.n_kept, 4, cudaMemcpyDeviceToHost, c->side);
    cudaEventRecord(c->kept_ev, c->side);
  }
  phaseB_sync(b, g, z, s, c->prof);
  cudaMemsetAsync(b.vcount, 0, size_t(g.W + 1) * 4, s);
  cudaMemsetAsync(b.cs_of_sync, 0xFF, ns1 * 4, s);
  phaseC_walk(b, g, z, s, c->prof);
  // forced compression at barriers renumbers the local times; barriers are validated in
  // phase A, so an invalid trace skips it
  if (z.forced_barrier && code != GWCP_ERR_INVALID_TRACE) phaseC_forced(b, g, z, s, c->prof);
  phaseE_locks(b, g, z, lock_mask, s, c->prof);
  phaseE_scan(b, z, s, c->prof);
  {
    const uint32_t* ex[5] = {b.incs_cnt + z.n_sync, b.vcount + g.W, b.lk_csid + z.n_acqrel,
                             b.lk_flags + z.n_acqrel, reinterpret_cast<const uint32_t*>(&b.st->spare[1])};
    int rc = read_status(c, s, ex, 5);
    if (rc) return rc;
  }
  code = c->st_host->code;
  if (code && code != GWCP_ERR_INVALID_TRACE) return code;
  z.n_incs = c->cnt_host[0];
  z.n_rows = c->cnt_host[1];
  z.n_cs = z.n_acqrel ? c->cnt_host[2] : 0;
  z.n_locks = z.n_acqrel ? c->cnt_host[3] : 0;
  z.n_exp = c->cnt_host[4];
  const uint32_t slots = std::min<uint32_t>(g.B + 1, lock_scope_cap(g.B));
  z.pool_cap = z.n_cs * slots + z.n_exp * 2 * slots + 64;
  b.dep_pool = get<uint32_t>(c, "dep_pool", z.pool_cap, &oom);
  z.race_cap = c->opt.race_capacity ? c->opt.race_capacity : std::max<uint64_t>(1u << 20, z.N);
  // scratch for every later scan and sort (the stream is idle here, so it may move)
  const size_t ex_bound = size_t(z.n_incs) * kMaxNest + 1;
  const size_t need2 = std::max({scan_need, radix_tmp_need(ex_bound), radix_tmp_need(z.race_cap + 1),
                                 scan_tmp_need(ex_bound)}) + 64;
  b.scan_tmp = get<uint32_t>(c, "scan_tmp", need2, &oom);
  if (oom) return GWCP_ERR_OOM;
  phaseE_walk(b, g, z, s, c->prof);  // W3; runs on invalid traces too, for the first bad index
  {
    // the last validation (W3) and the acquires' dependency lists are done: no later phase
    // runs on an invalid trace or after an error (their inputs would be incomplete)
    int rc = read_status(c, s, nullptr, 0);
    if (rc) return rc;
  }
  code = c->st_host->code;
  if (code) {
    c->bad_index = c->st_host->bad_index;
    return code;
  }

  // ---- remaining buffers ------------------------------------------------------------
  const size_t ni1 = size_t(z.n_incs) + 1;
  b.acc_info = get<AccInfo>(c, "acc_info", z.N, &oom);
  b.incs_idx = get<uint32_t>(c, "incs_idx", ni1, &oom);
  b.incs_ver = get<uint32_t>(c, "incs_ver", ni1, &oom);
  b.incs_k = get<uint32_t>(c, "incs_k", ni1, &oom);
  b.incs_key = get<uint64_t>(c, "incs_key", ni1, &oom);
  b.incs_wr = get<uint32_t>(c, "incs_wr", ni1, &oom);
  b.exp_off = get<uint32_t>(c, "exp_off", ni1, &oom);
  // expanded records: sized by the bound (depth <= kMaxNest), sorted by the exact count
  const size_t ne1 = std::max<size_t>(size_t(z.n_exp), size_t(z.n_incs) * kMaxNest) + 1;
  b.ex_key = get<uint64_t>(c, "ex_key", ne1, &oom);
  b.ex_val = get<uint32_t>(c, "ex_val", ne1, &oom);
  b.ex_key2 = get<uint64_t>(c, "ex_key2", ne1, &oom);
  b.ex_val2 = get<uint32_t>(c, "ex_val2", ne1, &oom);
  b.ex_rec = get<uint32_t>(c, "ex_rec", ne1, &oom);
  b.ex_cs = get<uint32_t>(c, "ex_cs", ne1, &oom);
  b.ex_flags = get<uint32_t>(c, "ex_flags", ne1, &oom);
  b.ex_group = get<uint32_t>(c, "ex_group", ne1 + 1, &oom);
  b.ex_dep_off = get<uint32_t>(c, "ex_dep_off", ne1, &oom);
  b.ex_dep_cnt = get<uint32_t>(c, "ex_dep_cnt", ne1, &oom);
  b.rows = get<uint32_t>(c, "rows", size_t(z.n_rows) * (z.compress ? g.B : g.RW), &oom);
  if (z.compress) {
    // compressed versions: first sized at half a dense row per version plus every walker's
    // chunk; later runs take what the last one needed; grown and rerun on exhaustion
    const uint64_t want = uint64_t(z.n_rows) * (g.W / 2 + 1) + uint64_t(g.W) * kCvChunk + 65536;
    z.cv_cap = std::min<uint64_t>(c->cv_cap_hint ? c->cv_cap_hint : want, kCvMaxWords);
    b.cv_pool = get<uint32_t>(c, "cv_pool", z.cv_cap, &oom);
  }
  b.psnap = get<uint32_t>(c, "psnap", (size_t(z.n_cs) + 1) * g.RW, &oom);
  b.hsnap = get<uint32_t>(c, "hsnap", (size_t(z.n_cs) + 1) * g.RW, &oom);
  if (g.nT) {
    // tile pool: a few new tiles per clock version; grown and rerun on exhaustion
    const uint64_t want = 2ull * (uint64_t(z.n_rows) + z.n_cs) + uint64_t(z.n_bar) * (g.apb + 2) + 65536;
    z.tile_cap = std::max<uint64_t>(c->tile_cap_hint, want);
    // 2 MB aligned: the walkers' time depended by ~3% on where the pool landed after the
    // buffers allocated before it (77 vs 79.5 ms on the 8192-warp, 200M-event workload
    // when one earlier buffer grew by 1.4 MB); aligned, it is the faster placement whatever
    // came before
    b.tiles = get_aligned<uint32_t>(c, "tiles", size_t(z.tile_cap) * kTileW, size_t(2) << 20, &oom);
  }
  b.done = get<uint32_t>(c, "done", size_t(z.n_cs) + 1, &oom);
  b.plan = get<uint4>(c, "plan", 2 * (size_t(z.n_sync) + z.n_incs) + 2, &oom);
  b.recmeta = get<uint4>(c, "recmeta", size_t(z.n_cs) + 1, &oom);
  b.flat_off = get<uint32_t>(c, "flat_off", ni1, &oom);
  b.flat = get<uint32_t>(c, "flat", z.pool_cap, &oom);
  b.cursor = get<uint32_t>(c, "cursor", size_t(g.W) * (z.n_locks + 1), &oom);
  b.jsnap = g.nT ? get<uint32_t>(c, "jsnap", (size_t(z.n_cs) + 1) * g.RW, &oom) : nullptr;
  const size_t smem = size_t(2) * g.apb * 2 * g.Wp * 4;
  z.cta_barriers = g.nT ? true : (g.apb <= 32 && smem <= 96 * 1024);
  const bool global_bars = !z.cta_barriers || g.gran == GWCP_GRAN_THREAD;
  b.bar_j = get<uint32_t>(c, "bar_j", global_bars ? size_t(z.n_bar) * 2 * g.Wp : 1, &oom);
  b.bar_cnt = get<uint32_t>(c, "bar_cnt", global_bars ? z.n_bar : 1, &oom);
  if (z.sparse_check) {
    const size_t na = size_t(z.n_acc) + 1;
    b.wc_flag = get<uint32_t>(c, "wc_flag", na, &oom);
    b.wc_run = get<uint32_t>(c, "wc_run", na + 1, &oom);  // [n] runs, [n + 1] accesses kept by the regrouping
    if (!z.grouped) {  // the regrouping sort of the location order
      b.wc_key = get<uint64_t>(c, "wc_key", na, &oom);
      b.wc_val = get<uint32_t>(c, "wc_val", na, &oom);
      b.wc_key2 = get<uint64_t>(c, "wc_key2", na, &oom);
      b.wc_val2 = get<uint32_t>(c, "wc_val2", na, &oom);
    }
    b.wc_gflag = get<uint32_t>(c, "wc_gflag", na, &oom);
    b.wc_gexcl = get<uint32_t>(c, "wc_gexcl", na, &oom);
    b.wc_grp_lo = get<uint32_t>(c, "wc_grp_lo", na, &oom);
    b.wc_grp_agent = get<uint32_t>(c, "wc_grp_agent", na, &oom);
    b.wc_rc = get<uint32_t>(c, "wc_rc", 4 * na + 2, &oom);
    b.wc_who = get<uint32_t>(c, "wc_who", na, &oom);
    b.wc_row = get<uint32_t>(c, "wc_row", na, &oom);
    b.wc_ep = get<uint32_t>(c, "wc_ep", na, &oom);
  } else {
    z.n_chunks = uint32_t(check_chunks(z.n_acc));
    const size_t ng = check_group_count(z.n_acc);
    b.tails = get<uint32_t>(c, "tails", (size_t(z.n_chunks) + ng) * 4 * g.Wp * 2 + ng + 8, &oom);
  }
  b.races = get<uint64_t>(c, "races", z.race_cap, &oom);
  b.races2 = get<uint64_t>(c, "races2", z.race_cap, &oom);
  if (oom) return GWCP_ERR_OOM;
  cudaMemsetAsync(b.done, 0, (size_t(z.n_cs) + 1) * 4, s);
  if (g.nT) {  // tile 0 is the zero tile; ids are handed out from 1
    cudaMemsetAsync(b.tiles, 0, kTileW * 4, s);
    const unsigned long long one = 1;
    cudaMemcpyAsync(&b.st->spare[2], &one, sizeof(one), cudaMemcpyHostToDevice, s);
  }
  cudaMemsetAsync(b.cursor, 0, size_t(g.W) * (z.n_locks + 1) * 4, s);
  if (global_bars && z.n_bar) {
    cudaMemsetAsync(b.bar_j, 0, size_t(z.n_bar) * 2 * g.Wp * 4, s);
    cudaMemsetAsync(b.bar_cnt, 0, size_t(z.n_bar) * 4, s);
  }

  phaseD_gaps(b, g, z, s, c->prof);
  c->acc_info_partial = z.wl_log2 != 0;
  // the access grouping and the check's carries need the access records (phase D), not
  // clock values: they follow the sort on the side stream while the propagation runs on s
  cudaEventRecord(c->fork2, s);
  const bool ranked = !c->rank_theta.empty() && z.n_acc;
  RankIn rin{};
  uint32_t *rk_tmp = nullptr, *rk_nloc = nullptr, *rk_val = nullptr, *rk_val2 = nullptr;
  float *rk_feat = nullptr, *rk_score = nullptr, *rk_theta = nullptr;
  uint64_t *rk_lockey = nullptr, *rk_key = nullptr, *rk_key2 = nullptr;
  size_t rk_bits_words = size_t(z.N) / 32 + 2;
  if (ranked) {
    rk_tmp = get<uint32_t>(c, "rk_tmp", rank_tmp_words(z.n_acc), &oom);
    rin.bits = get<uint32_t>(c, "rk_bits", rk_bits_words, &oom);
    rk_feat = get<float>(c, "rk_feat", size_t(z.n_acc) * kRankFeatures, &oom);
    rk_lockey = get<uint64_t>(c, "rk_lockey", z.n_acc, &oom);
    rk_score = get<float>(c, "rk_score", z.n_acc, &oom);
    rk_nloc = get<uint32_t>(c, "rk_nloc", 1, &oom);
    rk_theta = get<float>(c, "rk_theta", kRankParams, &oom);
    rk_key = get<uint64_t>(c, "rk_key", z.n_acc, &oom);
    rk_key2 = get<uint64_t>(c, "rk_key2", z.n_acc, &oom);
    rk_val = get<uint32_t>(c, "rk_val", z.n_acc, &oom);
    rk_val2 = get<uint32_t>(c, "rk_val2", z.n_acc, &oom);
  }
  z.n_timeline = z.sparse_check ? sparse_check_blocks(z.n_acc) : z.n_chunks;
  if (c->opt.timeline) {
    b.chunk_ns = get<unsigned long long>(c, "chunk_ns", size_t(z.n_timeline) + 1, &oom);
    b.chunk_races = get<uint32_t>(c, "chunk_races", size_t(z.n_timeline) + 1, &oom);
  } else {
    b.chunk_ns = nullptr;
    b.chunk_races = nullptr;
  }
  if (oom) return GWCP_ERR_OOM;
  phaseF_incs(b, g, z, key_mask, s, c->prof);
  phaseF_walk(b, g, z, key_mask, s, c->prof);
  z.n_groups = z.n_exp;  // upper bound; the kernel reads the exact count on the device
  phaseF_deps(b, g, z, s, c->prof);
  cudaStreamWaitEvent(c->side, c->fork2, 0);
  if (z.grouped) {
    // the main stream has phases D-F queued; the sort has usually finished by now
    if (cudaEventSynchronize(c->kept_ev) != cudaSuccess) return GWCP_ERR_CUDA;
    z.n_kept = std::min(c->cnt_host[15], z.n_acc);
    z.n_timeline = sparse_check_blocks(z.n_kept);
  }
  if (ranked) {
    // the ranker's order of the check: location runs by descending score
    c->prof.begin("h_rank", double(z.n_acc) * (12 + 16 + 12 * 2 * 6 + 12), c->side);
    cudaMemcpyAsync(rk_theta, c->rank_theta.data(), kRankParams * 4, cudaMemcpyHostToDevice, c->side);
    rin.key = b.acc_key;
    rin.idx = b.acc_idx;
    rin.info = b.acc_info;
    rin.n_acc = z.n_acc;
    rin.incs_idx = b.incs_idx;
    rin.n_incs = z.n_incs;
    rin.acqrel = b.acqrel;
    rin.n_acqrel = z.n_acqrel;
    rin.bar = b.bar;
    rin.n_bar = z.n_bar;
    rank_features(rin, rk_tmp, rk_bits_words, rk_feat, rk_lockey, rk_nloc, side_tmp, c->side);
    rank_scores(rk_theta, rk_feat, rk_nloc, z.n_acc, rk_score, c->side);
    rank_order(rin, rk_tmp, rk_score, rk_key, rk_val, rk_key2, rk_val2, b.acc_key2, b.acc_idx2, side_tmp, c->side);
    std::swap(b.acc_key, b.acc_key2);
    std::swap(b.acc_idx, b.acc_idx2);
    c->prof.end();
  }
  if (z.sparse_check)
    z.grouped ? phaseI_grouped(b, g, z, side_tmp, c->side, c->prof)
              : phaseI_wide_group(b, g, z, side_tmp, c->side, c->prof);
  else
    phaseI_carry(b, g, z, c->side, c->prof);
  int prc = phaseG_propagate(b, g, z, s, c->prof);
  side.join();
  if (prc) return prc;
  if (b.chunk_ns) stamp_now(&b.st->spare[5], s);  // the check's start, for the timeline
  if (z.sparse_check)
    phaseI_wide_check(b, g, z, s, c->prof);
  else
    phaseI_check(b, g, z, s, c->prof);
  c->n_chunks_timeline = b.chunk_ns ? z.n_timeline : 0;
  {
    int rc = read_status(c, s, nullptr, 0);
    if (rc) return rc;
  }
  code = c->st_host->code;
  c->bad_index = c->st_host->bad_index;
  if (code == GWCP_ERR_OOM && g.nT && c->st_host->spare[2] > z.tile_cap) {
    c->tile_cap_hint = 2 * z.tile_cap;  // the tile pool ran out: the caller runs again
    return kRerun;
  }
  if (z.compress) {
    // the walkers count every chunk they took, also past the end of the pool; the next run
    // sizes the pool from the count (with room for the chunks' varying tails)
    const uint64_t used = c->st_host->spare[3];
    const uint64_t next = used + used / 8 + uint64_t(g.W) * kCvChunk;
    if (used > z.cv_cap) {
      if (z.cv_cap >= kCvMaxWords) return GWCP_ERR_UNSUPPORTED;
      c->cv_cap_hint = next;
      return kRerun;
    }
    c->cv_cap_hint = std::max(c->cv_cap_hint, next);
    // the propagation's algorithmic bytes: the compressed words written, not dense rows
    for (auto& r : c->prof.recs)
      if (!std::strcmp(r.name, "g_propagate"))
        r.bytes = 4.0 * double(c->st_host->spare[4]) + double(z.n_cs) * 2 * g.Wp * 4;
  }
  if (code) return code;
  c->n_races = c->st_host->n_races;
  if (c->n_races > z.race_cap && c->opt.race_capacity == 0) {
    // automatic capacity: the race buffer was too small (a location read by many agents
    // and written once races with each of them); grow it and run the check again, which
    // writes nothing but the races and two counters
    z.race_cap = c->n_races + c->n_races / 8;
    b.races = get<uint64_t>(c, "races", z.race_cap, &oom);
    b.races2 = get<uint64_t>(c, "races2", z.race_cap, &oom);
    b.scan_tmp = get<uint32_t>(c, "scan_tmp", std::max(need2, radix_tmp_need(z.race_cap + 1) + 64), &oom);
    if (oom) return GWCP_ERR_OOM;
    const unsigned long long tests = c->st_host->partner_tests;
    cudaMemsetAsync(&b.st->n_races, 0, sizeof(unsigned long long), s);
    if (z.sparse_check)
      phaseI_wide_check(b, g, z, s, c->prof);
    else
      phaseI_check(b, g, z, s, c->prof);
    int rc = read_status(c, s, nullptr, 0);
    if (rc) return rc;
    if (c->st_host->code) return c->st_host->code;
    c->n_races = c->st_host->n_races;
    c->st_host->partner_tests = tests;
  }
  c->races_second = phaseI_sort_races(b, z, c->n_races, s, c->prof);
  c->counters[0] = z.n_acc;
  c->counters[1] = z.n_sync;
  c->counters[2] = z.n_cs;
  c->counters[3] = z.n_incs;
  c->counters[4] = z.n_rows;
  c->counters[5] = c->st_host->partner_tests;
  c->counters[6] = c->st_host->loop_visits;
  c->counters[7] = c->st_host->joins;
  c->first_race_ns = c->st_host->first_race_ns;
  c->counters[8] = c->st_host->tiles_read;
  c->counters[9] = c->st_host->tiles_written;
  c->clock_words[0] = c->st_host->spare[2];  // tiles handed out
  c->clock_words[1] = c->st_host->spare[3];  // compressed-version pool words handed out
  c->clock_words[2] = c->st_host->spare[4];  // compressed-version words written
  return cuda_rc();
}

}  // namespace

namespace gwcp {
// device bytes the context holds (its cached buffers and its copy of the trace)
size_t ctx_device_bytes(const gwcp_ctx* c) {
  size_t t = c->ev_own_cap;
  for (auto& kv : c->allocs) t += kv.second.second;
  return t;
}
void ctx_set_pack_walkers(gwcp_ctx* c, bool pack) { c->opt.pack_walkers = pack ? 1u : 0u; }
// %globaltimer (ns) at which the last compute's check found its first race; 0 if none
unsigned long long ctx_first_race_ns(const gwcp_ctx* c) { return c->computed ? c->first_race_ns : 0; }
// false when the last compute found more races than the device race buffer holds
bool ctx_races_complete(const gwcp_ctx* c) { return c->n_races <= c->z.race_cap; }
// releases the cached buffers (the next compute allocates them again); the caller makes
// sure no work of this context is in flight
void ctx_trim(gwcp_ctx* c) {
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->alloc_s);
  for (auto& kv : c->allocs)
    if (kv.second.first) cudaFreeAsync(kv.second.first, c->alloc_s);
  c->allocs.clear();
  if (c->ev_own) cudaFreeAsync(c->ev_own, c->alloc_s);
  cudaStreamSynchronize(c->alloc_s);
  cudaMemPool_t mp;  // give the pool's unused reserve back to the device
  if (cudaDeviceGetDefaultMemPool(&mp, c->device) == cudaSuccess) cudaMemPoolTrimTo(mp, 0);
  c->ev_own = nullptr;
  c->ev_own_cap = 0;
  c->has_trace = false;
  c->computed = false;
}
}  // namespace gwcp

extern "C" {

int gwcp_create(gwcp_ctx** out, int device, const gwcp_options* opt) {
  if (!out) return GWCP_ERR_ARGS;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GWCP_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return GWCP_ERR_CUDA;
  {
    // freed buffers stay reserved in the device's default pool for the next allocation
    // instead of going back to the driver at every synchronisation
    cudaMemPool_t mp;
    uint64_t keep = ~0ull;
    if (cudaDeviceGetDefaultMemPool(&mp, device) == cudaSuccess)
      cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
  }
  auto* c = new gwcp_ctx();
  c->device = device;
  if (opt) c->opt = *opt;
  if (cudaMallocHost(&c->st_host, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->cnt_host, 16 * sizeof(uint32_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->kept_ev, cudaEventDisableTiming) != cudaSuccess ||
      (c->opt.blocking_sync &&
       cudaEventCreateWithFlags(&c->sync_ev, cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess)) {
    gwcp_destroy(c);
    return GWCP_ERR_OOM;
  }
  *out = c;
  return GWCP_OK;
}

int gwcp_load_trace(gwcp_ctx* c, const gwcp_event* ev, uint64_t n, const gwcp_geometry* geo, int ev_is_device,
                    void* stream) {
  if (!c || !geo || (!ev && n)) return GWCP_ERR_ARGS;
  if (n > kMaxEvents || geo->num_agents == 0 || geo->agents_per_block == 0 || geo->reserved != 0 ||
      geo->num_agents % geo->agents_per_block != 0 || geo->granularity > 1)
    return GWCP_ERR_ARGS;
  // clocks of more than kMaxAgents entries are tile tables: warp granularity, and a block
  // of agents fits one CTA of walkers
  const bool tiles_ok =
      geo->num_agents <= kMaxAgentsWide && geo->granularity == GWCP_GRAN_WARP && geo->agents_per_block <= 32;
  if (geo->num_agents > kMaxAgents && !tiles_ok) return GWCP_ERR_UNSUPPORTED;
  if (c->clock_mode == GWCP_CLOCKS_TILES && !tiles_ok) return GWCP_ERR_UNSUPPORTED;
  if (c->clock_mode == GWCP_CLOCKS_COMPRESSED && geo->num_agents > kMaxAgents) return GWCP_ERR_UNSUPPORTED;
  // automatic: tiles from kTilesFromAgents agents on (measured faster from there on GB300)
  const bool tiles = geo->num_agents > kMaxAgents || c->clock_mode == GWCP_CLOCKS_TILES ||
                     (c->clock_mode == GWCP_CLOCKS_AUTO && tiles_ok && geo->num_agents >= kTilesFromAgents);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  use_stream(c, s);
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
  if (tiles) {
    g.nT = (g.W + kTileW - 1) / kTileW;
    g.Wp = g.nT * kTileW;
    g.K = g.Wp / 32;
    g.RW = kTabW;
  }
  c->g = g;
  c->compressed = c->clock_mode == GWCP_CLOCKS_COMPRESSED;
  c->n = n;
  c->computed = false;
  c->compute_rc = GWCP_ERR_STATE;
  if (ev_is_device) {
    c->ev_dev = reinterpret_cast<const Event*>(ev);
  } else {
    const size_t bytes = (n ? n : 1) * sizeof(Event);
    if (c->ev_own_cap < bytes) {
      if (c->ev_own) cudaFreeAsync(c->ev_own, s);
      c->ev_own = nullptr;
      c->ev_own_cap = 0;
      if (cudaMallocAsync(&c->ev_own, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return GWCP_ERR_OOM;
      }
      c->ev_own_cap = bytes;
    }
    if (n && cudaMemcpyAsync(c->ev_own, ev, n * sizeof(Event), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return GWCP_ERR_CUDA;
    c->ev_dev = c->ev_own;
  }
  c->has_trace = true;
  return GWCP_OK;
}

int gwcp_compute_order(gwcp_ctx* c, void* stream) {
  if (!c) return GWCP_ERR_ARGS;
  if (!c->has_trace) return GWCP_ERR_STATE;
  cudaSetDevice(c->device);
  c->bad_index = ~0ull;
  c->n_races = 0;
  if (c->n == 0) {
    c->computed = true;
    c->compute_rc = GWCP_OK;
    c->z = Sizes{};
    std::memset(c->counters, 0, sizeof(c->counters));
    std::memset(c->clock_words, 0, sizeof(c->clock_words));
    return GWCP_OK;
  }
  int rc = run(c, static_cast<cudaStream_t>(stream));
  for (int attempt = 0; rc == kRerun && attempt < 6; ++attempt) rc = run(c, static_cast<cudaStream_t>(stream));
  if (rc == kRerun) rc = GWCP_ERR_OOM;
  c->computed = true;
  c->compute_rc = rc;
  return rc;
}

int gwcp_report_races(gwcp_ctx* c, gwcp_race* out, uint64_t cap, uint64_t* n_races, void* stream) {
  if (!c || !n_races || (cap && !out)) return GWCP_ERR_ARGS;
  if (!c->computed) return GWCP_ERR_STATE;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  use_stream(c, s);
  if (wait_stream(c, s) != cudaSuccess) return GWCP_ERR_CUDA;
  *n_races = 0;
  if (c->compute_rc) return c->compute_rc;
  *n_races = c->n_races;
  if (c->n_races > c->z.race_cap) return GWCP_ERR_CAPACITY;
  const uint64_t m = std::min<uint64_t>(cap, c->n_races);
  if (m) {
    // the sorted (later << 32 | earlier) words become gwcp_race records on the device; one
    // copy brings them to the caller
    bool oom = false;
    gwcp_race* dev = get<gwcp_race>(c, "races_out", m, &oom);
    if (oom) return GWCP_ERR_OOM;
    races_to_records(c->races_second ? c->b.races2 : c->b.races, m, dev, s);
    int rc = copy_to_host(c, out, dev, m * sizeof(gwcp_race), s);
    if (rc) return rc;
  }
  // profile of this compute
  c->prof_ms.clear();
  c->prof_start.clear();
  c->prof_bytes.clear();
  c->prof_names.clear();
  if (c->prof.on) {
    for (auto& r : c->prof.recs) {
      float ms = 0;
      cudaEventElapsedTime(&ms, r.a, r.b);
      c->prof_ms.push_back(ms);
      float at = 0;
      cudaEventElapsedTime(&at, c->prof.recs[0].a, r.a);
      c->prof_start.push_back(at);
      c->prof_bytes.push_back(r.bytes);
      c->prof_names.push_back(r.name);
    }
  }
  return cap < c->n_races ? GWCP_ERR_CAPACITY : GWCP_OK;
}

namespace {
// a published clock (Wp words, or a table of tile ids for wide clocks) into out[Wp]
void read_clock(gwcp_ctx* c, const uint32_t* src, uint32_t* out) {
  const Geo& g = c->g;
  if (!g.nT) {
    cudaMemcpy(out, src, size_t(g.Wp) * 4, cudaMemcpyDeviceToHost);
    return;
  }
  uint32_t ids[kTabW];
  cudaMemcpy(ids, src, sizeof(ids), cudaMemcpyDeviceToHost);
  for (uint32_t t = 0; t < g.nT; ++t)
    cudaMemcpy(out + size_t(t) * kTileW, c->b.tiles + size_t(ids[t]) * kTileW, kTileW * 4, cudaMemcpyDeviceToHost);
}

// clock version `row` into out[Wp]: a published clock, or a compressed version decoded
// (header word per block, then warp words, then lane values)
int read_version(gwcp_ctx* c, uint32_t row, uint32_t* out) {
  const Geo& g = c->g;
  if (!c->z.compress) {
    read_clock(c, c->b.rows + size_t(row) * g.RW, out);
    return GWCP_OK;
  }
  const uint32_t gs = cv_group(g.gran), nw = (g.apb + gs - 1) / gs;
  std::vector<uint32_t> hdr(g.B), wv(nw), lanes(32);
  cudaMemcpy(hdr.data(), c->b.rows + size_t(row) * g.B, size_t(g.B) * 4, cudaMemcpyDeviceToHost);
  std::fill(out, out + g.Wp, 0u);
  for (uint32_t b = 0; b < g.B; ++b) {
    uint32_t* o = out + size_t(b) * g.apb;
    if (!(hdr[b] & kCvExpanded)) {
      std::fill(o, o + g.apb, hdr[b]);
      continue;
    }
    const uint64_t at = hdr[b] & ~kCvExpanded;
    if (at + nw > c->z.cv_cap) return GWCP_ERR_STATE;
    cudaMemcpy(wv.data(), c->b.cv_pool + at, size_t(nw) * 4, cudaMemcpyDeviceToHost);
    for (uint32_t w = 0; w < nw; ++w) {
      const uint32_t lo = w * gs, hi = std::min(lo + gs, g.apb);
      if (!(wv[w] & kCvExpanded)) {
        std::fill(o + lo, o + hi, wv[w]);
        continue;
      }
      const uint64_t at2 = wv[w] & ~kCvExpanded;
      if (at2 + 32 > c->z.cv_cap) return GWCP_ERR_STATE;
      cudaMemcpy(lanes.data(), c->b.cv_pool + at2, 32 * 4, cudaMemcpyDeviceToHost);
      std::copy(lanes.begin(), lanes.begin() + (hi - lo), o + lo);
    }
  }
  return GWCP_OK;
}
}  // namespace

namespace {
// the records of every access (a grouped-order compute writes only the kept accesses')
int complete_acc_info(gwcp_ctx* c, cudaStream_t s) {
  if (!c->acc_info_partial) return GWCP_OK;
  phaseD_trace(c->b, c->g, c->z, s, false);
  c->acc_info_partial = false;
  return cudaStreamSynchronize(s) == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
}
}  // namespace

int gwcp_debug_clock(gwcp_ctx* c, uint64_t idx, int which, uint32_t* out) {
  if (!c || !out) return GWCP_ERR_ARGS;
  if (!c->computed || c->compute_rc) return GWCP_ERR_STATE;
  if (idx >= c->n) return GWCP_ERR_ARGS;
  cudaSetDevice(c->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return GWCP_ERR_CUDA;
  const Geo& g = c->g;
  const Bufs& b = c->b;
  Event e;
  cudaMemcpy(&e, c->ev_dev + idx, sizeof(e), cudaMemcpyDeviceToHost);
  std::vector<uint32_t> row(g.Wp);
  uint32_t own = 0;
  uint32_t version = kNoneHost;
  if (e.op <= GWCP_ATOMIC) {
    if (which != 0) return GWCP_ERR_UNSUPPORTED;
    if (int rc = complete_acc_info(c, nullptr)) return rc;
    AccInfo inf;
    cudaMemcpy(&inf, b.acc_info + idx, sizeof(inf), cudaMemcpyDeviceToHost);
    version = inf.row;
    own = inf.epoch;
  } else if (e.op == GWCP_ACQ || e.op == GWCP_REL) {
    uint32_t k0, k1;
    cudaMemcpy(&k0, b.sy_start + e.agent, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(&k1, b.sy_start + e.agent + 1, 4, cudaMemcpyDeviceToHost);
    std::vector<uint32_t> ids(k1 - k0);
    if (k1 > k0) cudaMemcpy(ids.data(), b.sy_idx + k0, size_t(k1 - k0) * 4, cudaMemcpyDeviceToHost);
    auto it = std::lower_bound(ids.begin(), ids.end(), uint32_t(idx));
    if (it == ids.end() || *it != idx) return GWCP_ERR_STATE;
    const uint32_t k = k0 + uint32_t(it - ids.begin());
    uint32_t N, ver, rb, cs;
    cudaMemcpy(&N, b.sy_N + k, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(&ver, b.sy_ver + k, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(&rb, b.vcount + e.agent, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(&cs, b.cs_of_sync + k, 4, cudaMemcpyDeviceToHost);
    own = e.op == GWCP_REL ? N - 1 : N;
    if (which == 0) {
      version = rb + ver;
    } else {
      if (e.op != GWCP_REL || cs == kNoneHost) return GWCP_ERR_UNSUPPORTED;
      read_clock(c, b.hsnap + size_t(cs) * g.RW, row.data());
      std::memcpy(out, row.data(), g.W * 4);
      return cuda_rc();
    }
  } else {
    return GWCP_ERR_UNSUPPORTED;
  }
  const int rc = read_version(c, version, row.data());
  if (rc) return rc;
  row[e.agent] = own;
  std::memcpy(out, row.data(), g.W * 4);
  return cuda_rc();
}

int gwcp_clock_bytes(const gwcp_ctx* c, uint64_t* out3) {
  if (!c || !out3) return GWCP_ERR_ARGS;
  if (!c->computed || c->compute_rc) return GWCP_ERR_STATE;
  const Geo& g = c->g;
  const Sizes& z = c->z;
  const uint64_t rows = z.n_rows;
  out3[0] = rows * g.Wp * 4;
  if (z.compress) {
    out3[1] = c->clock_words[2] * 4;
    out3[2] = (rows * g.B + c->clock_words[1]) * 4;
  } else if (g.nT) {
    const uint64_t tiles = c->clock_words[0];  // handed out, including the zero tile
    out3[1] = out3[2] = rows * kTabW * 4 + tiles * kTileW * 4;
  } else {
    out3[1] = out3[2] = out3[0];
  }
  return GWCP_OK;
}

int gwcp_set_check_mode(gwcp_ctx* c, uint32_t mode) {
  if (!c || mode > GWCP_CHECK_SPARSE) return GWCP_ERR_ARGS;
  c->check_mode = mode;
  return GWCP_OK;
}

int gwcp_set_clock_mode(gwcp_ctx* c, uint32_t mode) {
  if (!c || mode > GWCP_CLOCKS_COMPRESSED) return GWCP_ERR_ARGS;
  c->clock_mode = mode;
  return GWCP_OK;
}

int gwcp_set_ranker(gwcp_ctx* c, const float* theta) {
  if (!c) return GWCP_ERR_ARGS;
  if (!theta) {
    c->rank_theta.clear();
    return GWCP_OK;
  }
  c->rank_theta.assign(theta, theta + kRankParams);
  return GWCP_OK;
}

namespace {
// location order rebuilt from the trace (the grouped order leaves read-only locations
// out): the accesses' (location key, trace index) pairs in trace order, then a stable sort
__global__ void k_lf_flag(const Event* ev, uint64_t N, uint32_t* flag) {
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) flag[i] = ev[i].op <= GWCP_ATOMIC ? 1u : 0u;
}
__global__ void k_lf_acc(const Event* ev, uint64_t N, uint32_t apb, const uint32_t* flag, const uint32_t* pos,
                         uint64_t* k, uint32_t* v) {
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N && flag[i]) {
    k[pos[i]] = location_key(ev[i], apb);
    v[pos[i]] = uint32_t(i);
  }
}
}  // namespace

int gwcp_location_features(gwcp_ctx* c, float* feat, uint64_t* keys, uint64_t cap, uint64_t* n_loc, void* stream) {
  if (!c || !n_loc || (cap && (!feat || !keys))) return GWCP_ERR_ARGS;
  if (!c->computed || c->compute_rc) return GWCP_ERR_STATE;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  use_stream(c, s);
  *n_loc = 0;
  const Sizes& z = c->z;
  if (c->n == 0 || z.n_acc == 0) return GWCP_OK;
  bool oom = false;
  RankIn in{};
  const size_t bits_words = size_t(z.N) / 32 + 2;
  uint32_t* tmp = get<uint32_t>(c, "rk_tmp", rank_tmp_words(z.n_acc), &oom);
  in.bits = get<uint32_t>(c, "rk_bits", bits_words, &oom);
  float* f = get<float>(c, "rk_feat", size_t(z.n_acc) * kRankFeatures, &oom);
  uint64_t* k = get<uint64_t>(c, "rk_lockey", z.n_acc, &oom);
  uint32_t* nl = get<uint32_t>(c, "rk_nloc", 1, &oom);
  uint32_t* stmp = get<uint32_t>(c, "side_tmp", scan_tmp_need(size_t(z.n_acc) + 1) + 64, &oom);
  if (oom) return GWCP_ERR_OOM;
  const Bufs& b = c->b;
  in.key = b.acc_key;
  in.idx = b.acc_idx;
  if (z.grouped) {  // the check ran on the grouped order: rebuild the location order
    const size_t n = z.n_acc;
    uint64_t* k0 = get<uint64_t>(c, "lf_k0", n, &oom);
    uint64_t* k1 = get<uint64_t>(c, "lf_k1", n, &oom);
    uint32_t* v0 = get<uint32_t>(c, "lf_v0", n, &oom);
    uint32_t* v1 = get<uint32_t>(c, "lf_v1", n, &oom);
    uint32_t* flag = get<uint32_t>(c, "lf_flag", z.N, &oom);
    uint32_t* pos = get<uint32_t>(c, "lf_pos", z.N, &oom);
    uint32_t* st2 = get<uint32_t>(c, "lf_tmp", std::max(radix_tmp_need(n + 1), scan_tmp_need(z.N)) + 64, &oom);
    if (oom) return GWCP_ERR_OOM;
    const uint32_t nbN = uint32_t((z.N + 255) / 256);
    k_lf_flag<<<nbN, 256, 0, s>>>(b.ev, z.N, flag);
    count_launch();
    scan_exclusive(flag, pos, z.N, nullptr, st2, s);
    k_lf_acc<<<nbN, 256, 0, s>>>(b.ev, z.N, c->g.apb, flag, pos, k0, v0);
    count_launch();
    if (radix_sort_pairs(k0, v0, k1, v1, n, c->key_mask, st2, s)) {
      std::swap(k0, k1);
      std::swap(v0, v1);
    }
    in.key = k0;
    in.idx = v0;
  }
  if (int rc = complete_acc_info(c, s)) return rc;
  in.info = b.acc_info;
  in.n_acc = z.n_acc;
  in.incs_idx = b.incs_idx;
  in.n_incs = z.n_incs;
  in.acqrel = b.acqrel;
  in.n_acqrel = z.n_acqrel;
  in.bar = b.bar;
  in.n_bar = z.n_bar;
  rank_features(in, tmp, bits_words, f, k, nl, stmp, s);
  uint32_t n = 0;
  if (cudaMemcpyAsync(&n, nl, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || wait_stream(c, s) != cudaSuccess)
    return GWCP_ERR_CUDA;
  *n_loc = n;
  const uint64_t m = std::min<uint64_t>(cap, n);
  if (m && (cudaMemcpyAsync(feat, f, m * kRankFeatures * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(keys, k, m * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            wait_stream(c, s) != cudaSuccess))
    return GWCP_ERR_CUDA;
  return cap < n ? GWCP_ERR_CAPACITY : cuda_rc();
}

int gwcp_rank_scores(const float* theta, const float* feat, uint64_t n, float* scores, void* stream) {
  if ((n && (!theta || !feat || !scores)) || n > kMaxEvents) return GWCP_ERR_ARGS;
  if (!n) return GWCP_OK;
  rank_scores(theta, feat, nullptr, uint32_t(n), scores, static_cast<cudaStream_t>(stream));
  return cuda_rc();
}

int gwcp_rank_grad(const float* theta, const float* feat, const float* labels, uint64_t n, float pos_weight,
                   float* grad, float* loss, void* stream) {
  if (!theta || !grad || !loss || (n && (!feat || !labels)) || n > kMaxEvents) return GWCP_ERR_ARGS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(grad, 0, kRankParams * 4, s);
  cudaMemsetAsync(loss, 0, 4, s);
  if (!n) return cuda_rc();
  return rank_grad(theta, feat, labels, 0, uint32_t(n), pos_weight, 1.0f / float(n), grad, loss, s);
}

int gwcp_rank_train(float* theta, const float* feat, const float* labels, uint64_t n, const gwcp_train_options* o,
                    float* epoch_loss, void* stream) {
  if (!theta || !o || !o->epochs || !o->batch || (n && (!feat || !labels)) || n > kMaxEvents) return GWCP_ERR_ARGS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // optimizer state, gradient, loss accumulator, per-epoch losses, counters
  float* buf = nullptr;
  const size_t words = 3 * size_t(kRankParams) + 1 + o->epochs + 2;
  if (cudaMalloc(&buf, words * 4) != cudaSuccess) {
    cudaGetLastError();
    return GWCP_ERR_OOM;
  }
  float *m = buf, *v = buf + kRankParams, *g = buf + 2 * kRankParams, *acc = buf + 3 * kRankParams;
  float* losses = acc + 1;
  auto* ctr = reinterpret_cast<uint32_t*>(losses + o->epochs);
  cudaMemsetAsync(buf, 0, words * 4, s);
  int rc = GWCP_OK;
  if (n) {
    // one epoch's launches (a gradient and an Adam step per mini-batch) are captured once
    // as a CUDA graph and replayed for every epoch; without capture they are launched
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int erc = rank_epoch(theta, feat, labels, uint32_t(n), o->batch, o->lr, o->pos_weight, m, v, g, acc,
                                 losses, ctr, cs);
      if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || erc ||
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
    }
    cudaGetLastError();
    for (uint32_t e = 0; e < o->epochs && !rc; ++e) {
      if (exec)
        rc = cudaGraphLaunch(exec, s) == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
      else
        rc = rank_epoch(theta, feat, labels, uint32_t(n), o->batch, o->lr, o->pos_weight, m, v, g, acc, losses,
                        ctr, s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
  }
  if (!rc && epoch_loss &&
      cudaMemcpyAsync(epoch_loss, losses, size_t(o->epochs) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = GWCP_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = GWCP_ERR_CUDA;
  cudaFree(buf);
  return rc ? rc : cuda_rc();
}

int gwcp_check_timeline(gwcp_ctx* c, uint64_t* start_ns, uint64_t* chunk_end_ns, uint32_t* chunk_races, uint64_t cap,
                        uint64_t* n_chunks) {
  if (!c || !n_chunks || !start_ns || (cap && (!chunk_end_ns || !chunk_races))) return GWCP_ERR_ARGS;
  if (!c->computed || c->compute_rc) return GWCP_ERR_STATE;
  cudaSetDevice(c->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return GWCP_ERR_CUDA;
  *n_chunks = c->n_chunks_timeline;
  if (!c->n_chunks_timeline) return c->opt.timeline ? GWCP_OK : GWCP_ERR_STATE;
  cudaMemcpy(start_ns, &c->b.st->spare[5], 8, cudaMemcpyDeviceToHost);
  const uint64_t m = std::min<uint64_t>(cap, c->n_chunks_timeline);
  if (m) {
    cudaMemcpy(chunk_end_ns, c->b.chunk_ns, m * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(chunk_races, c->b.chunk_races, m * 4, cudaMemcpyDeviceToHost);
  }
  return cap < c->n_chunks_timeline ? GWCP_ERR_CAPACITY : cuda_rc();
}

int gwcp_debug_alloc_limit(gwcp_ctx* c, uint64_t bytes) {
  if (!c) return GWCP_ERR_ARGS;
  c->alloc_limit = bytes;
  return GWCP_OK;
}

int gwcp_debug_wait_timeout(int device, uint32_t spin_limit, int* status) {
  if (!status || spin_limit == 0) return GWCP_ERR_ARGS;
  if (cudaSetDevice(device) != cudaSuccess) return GWCP_ERR_CUDA;
  *status = GWCP_OK;
  return wait_probe(spin_limit, status);
}

uint64_t gwcp_first_bad_index(const gwcp_ctx* c) { return c ? c->bad_index : ~0ull; }

uint64_t gwcp_launch_count(void) { return gwcp::launch_count(); }

int gwcp_profile_get(const gwcp_ctx* c, int i, const char** name, float* ms, double* bytes) {
  if (!c || i < 0 || size_t(i) >= c->prof_ms.size()) return GWCP_ERR_ARGS;
  if (name) *name = c->prof_names[i];
  if (ms) *ms = c->prof_ms[i];
  if (bytes) *bytes = c->prof_bytes[i];
  return GWCP_OK;
}

int gwcp_profile_start(const gwcp_ctx* c, int i, float* start_ms) {
  if (!c || i < 0 || size_t(i) >= c->prof_start.size() || !start_ms) return GWCP_ERR_ARGS;
  *start_ms = c->prof_start[i];
  return GWCP_OK;
}

int gwcp_counters(const gwcp_ctx* c, uint64_t* out8) {
  if (!c || !out8) return GWCP_ERR_ARGS;
  std::memcpy(out8, c->counters, 8 * sizeof(uint64_t));
  return GWCP_OK;
}

int gwcp_counters_ex(const gwcp_ctx* c, uint64_t* out, uint32_t n) {
  if (!c || (n && !out)) return GWCP_ERR_ARGS;
  std::memcpy(out, c->counters, std::min<uint32_t>(n, GWCP_N_COUNTERS) * sizeof(uint64_t));
  return GWCP_OK;
}

void gwcp_destroy(gwcp_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->alloc_s);
  if (c->side) cudaStreamSynchronize(c->side);
  for (auto& kv : c->allocs)
    if (kv.second.first) cudaFreeAsync(kv.second.first, c->alloc_s);
  if (c->ev_own) cudaFreeAsync(c->ev_own, c->alloc_s);
  cudaStreamSynchronize(c->alloc_s);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->stage_host) cudaFreeHost(c->stage_host);
  for (auto e : c->stage_ev)
    if (e) cudaEventDestroy(e);
  if (c->cnt_host) cudaFreeHost(c->cnt_host);
  for (auto e : c->prof.pool) cudaEventDestroy(e);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->fork2) cudaEventDestroy(c->fork2);
  if (c->kept_ev) cudaEventDestroy(c->kept_ev);
  if (c->sync_ev) cudaEventDestroy(c->sync_ev);
  if (c->side) cudaStreamDestroy(c->side);
  delete c;
}

const char* gwcp_strerror(int code) {
  switch (code) {
    case GWCP_OK: return "ok";
    case GWCP_ERR_INVALID_TRACE: return "invalid trace (see gwcp_first_bad_index)";
    case GWCP_ERR_OOM: return "out of device memory";
    case GWCP_ERR_CUDA: return "CUDA error";
    case GWCP_ERR_CAPACITY: return "race buffer too small";
    case GWCP_ERR_TIMEOUT: return "a bounded device wait gave up";
    case GWCP_ERR_STATE: return "calls out of order";
    case GWCP_ERR_ARGS: return "invalid arguments";
    case GWCP_ERR_UNSUPPORTED: return "unsupported size or configuration";
    default: return "unknown error";
  }
}

}  // extern "C"
