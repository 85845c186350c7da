// Internal declarations of libgwcp (device buffers, kernels, launch helpers).
// Shared only among the library's own translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gwcp.h"

namespace gwcp {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int kMaxNest = 4;         // deepest lockset a valid trace may hold
constexpr uint32_t kMaxAgents = 1024;      // clocks held in registers
constexpr uint32_t kMaxAgentsWide = 8192;  // clocks as tables of copy-on-write tiles
constexpr uint32_t kTileW = 256;           // entries per clock tile
constexpr uint32_t kTabW = 32;             // words per published tile table (nT <= 32)
constexpr uint32_t kTilesFromAgents = 512;  // automatic clock mode: tiles from this width on
constexpr uint32_t kSparseCheckFromAgents = 1;  // automatic check mode: partner groups (measured faster)
constexpr uint32_t kMaxEvents = (1u << 30) - 1;
// distinct scope ids one lock may be used with: 64, or 320 when the trace has more than
// 63 blocks (a block-scoped lock may be used in every block)
constexpr int kLockScopesSmall = 64, kLockScopesLarge = 320;
__host__ __device__ inline uint32_t lock_scope_cap(uint32_t blocks) {
  return blocks + 1 <= uint32_t(kLockScopesSmall) ? kLockScopesSmall : kLockScopesLarge;
}

// S entry kinds (agent-sorted event stream), packed as (kind << 30) | trace index
enum : uint32_t { K_ACCESS = 0, K_ACQ = 1, K_REL = 2, K_BAR = 3 };
__host__ __device__ inline uint32_t s_kind(uint32_t s) { return s >> 30; }
__host__ __device__ inline uint32_t s_idx(uint32_t s) { return s & 0x3FFFFFFFu; }

// access classes
enum : uint32_t { C_READ = 0, C_WRITE = 1, C_ATOM_CTA = 2, C_ATOM_DEV = 3 };

struct Event {
  uint32_t agent;
  uint8_t op, scope, space, flags;
  uint64_t addr;
};

// Device-side status and counters (one per context).
struct DevStatus {
  int code;                      // GWCP_OK or a GWCP_ERR_*
  int pad;
  unsigned long long bad_index;  // first offending event (atomicMin)
  unsigned long long key_or, key_and;    // over access location keys
  unsigned long long lock_or, lock_and;  // over acquire/release lock ids
  unsigned long long n_races;            // races found (may exceed the buffer)
  unsigned long long dep_pool_used;
  unsigned long long partner_tests;
  unsigned long long loop_visits;
  unsigned long long joins;
  unsigned long long spare[6];
  unsigned long long tiles_read, tiles_written;  // wide clocks: 1 KB tiles the walkers read / wrote
  unsigned long long first_race_ns;              // %globaltimer when the check found its first race (0: none)
};

// %globaltimer (ns); the check stamps its first race with it
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Geo {
  uint32_t W, apb, B, gran, Wp, K;  // Wp = W rounded up to 32 * K, K = Wp / 32 (a power of two)
  uint32_t nT;  // wide clocks: tiles of kTileW entries (0: clocks in registers)
  uint32_t RW;  // words per published clock: Wp, or kTabW tile ids when nT > 0
};

// Per-access record consumed by the check (indexed by trace index).
struct AccInfo {
  uint32_t epoch;  // N_t of the access
  uint32_t row;    // global clock-version row holding P_t for the access
  uint32_t who;    // agent | class << 13 | block << 15 (agent, block < 8192)
  uint32_t pad;
};
__host__ __device__ inline uint32_t make_who(uint32_t agent, uint32_t cls, uint32_t block) {
  return agent | (cls << 13) | (block << 15);
}
__host__ __device__ inline uint32_t who_agent(uint32_t w) { return w & 0x1FFFu; }
__host__ __device__ inline uint32_t who_class(uint32_t w) { return (w >> 13) & 3u; }
__host__ __device__ inline uint32_t who_block(uint32_t w) { return w >> 15; }

// All device buffers of one analysis. Sizes in comments.
struct Bufs {
  const Event* ev = nullptr;  // [N]
  DevStatus* st = nullptr;
  // phase A: agent counting sort, trace-order compactions
  uint32_t* hist_a = nullptr;    // [W * ntA + 1]
  uint32_t* tile_cnt = nullptr;  // [3 * ntA + 3]: accesses, acq/rel, barriers per tile (+ S entries
                                 // per tile when S is built by sorting)
  uint32_t* d_index = nullptr;   // [W * d_nw] phase D: each agent's first sync entry per trace window
  uint64_t* s_key = nullptr;     // [nS] (agent << 32 | S entry), sorted by agent (+ alt)
  uint64_t* s_key2 = nullptr;
  uint32_t* s_tmp = nullptr;     // the agent sort's scratch
  uint32_t* S = nullptr;         // [nS]
  uint32_t* seg = nullptr;       // [W + 1] start of each agent's segment in S
  uint32_t* acqrel = nullptr;    // [n_acqrel] trace indices
  uint32_t* bar = nullptr;       // [n_bar] trace indices
  uint64_t* acc_key = nullptr;   // [n_acc] (+ alt)
  uint32_t* acc_idx = nullptr;   // [n_acc] (+ alt)
  uint64_t* acc_key2 = nullptr;
  uint32_t* acc_idx2 = nullptr;
  // phase B: sync list
  uint32_t* sy_cnt = nullptr;   // [ntS + 1]
  uint32_t* sy_spos = nullptr;  // [n_sync]
  uint32_t* sy_idx = nullptr;   // [n_sync]
  uint32_t* sy_kind = nullptr;  // [n_sync]
  uint32_t* sy_start = nullptr; // [W + 1]
  uint32_t* sy_aux = nullptr;   // [n_sync] barrier ordinal for barrier entries
  // phase C: per-agent sync walk
  uint32_t* sy_N = nullptr;      // epoch after the entry
  uint32_t* sy_depth = nullptr;  // lock depth after the entry
  uint32_t* sy_inner = nullptr;  // sync ordinal of the innermost open acquire after it
  uint32_t* sy_ver = nullptr;    // version index after the entry
  uint32_t* sy_match = nullptr;  // REL: its acquire; ACQ: the enclosing acquire
  uint32_t* sy_relk = nullptr;   // ACQ: the matching release (NONE if never released)
  uint32_t* sy_agent = nullptr;  // agent of the entry
  uint32_t* incs_cnt = nullptr;  // [n_sync + 1] in-section accesses in the gap after k
  uint32_t* vcount = nullptr;    // [W + 1] versions per agent -> row base (scanned)
  // phase D: accesses
  AccInfo* acc_info = nullptr;   // [N]
  uint32_t* incs_idx = nullptr;  // [n_incs]
  uint32_t* incs_ver = nullptr;
  uint32_t* incs_k = nullptr;    // sync ordinal of the gap the access lies in
  uint64_t* incs_key = nullptr;
  uint32_t* incs_wr = nullptr;
  // phase E: locks and critical sections
  uint64_t* lk_key = nullptr;  // [n_acqrel] (+ alt)
  uint32_t* lk_k = nullptr;
  uint64_t* lk_key2 = nullptr;
  uint32_t* lk_k2 = nullptr;
  uint32_t* lk_flags = nullptr;    // [n_acqrel + 1] scan scratch
  uint32_t* lk_csid = nullptr;     // [n_acqrel + 1]
  uint32_t* lk_rank = nullptr;     // [n_acqrel + 1]
  uint32_t* lock_first = nullptr;  // [n_locks + 1] first sorted entry of each lock
  uint32_t* lock_cs_lo = nullptr;  // [n_locks + 1]
  uint32_t* cs_of_sync = nullptr;  // [n_sync]
  uint32_t* cs_agent = nullptr;    // [n_cs]
  uint32_t* cs_sid = nullptr;
  uint32_t* cs_epoch = nullptr;
  uint32_t* cs_rel_idx = nullptr;
  uint32_t* cs_rel_epoch = nullptr;  // N of the releasing agent at the release
  uint32_t* cs_lock = nullptr;
  uint32_t* cs_parent = nullptr;
  uint32_t* acq_dep_off = nullptr;  // [n_cs]
  uint32_t* acq_dep_cnt = nullptr;
  uint32_t* dep_pool = nullptr;     // [pool_cap]
  // phase F: in-section dependencies
  uint32_t* exp_off = nullptr;   // [n_incs + 1]
  uint64_t* ex_key = nullptr;    // [n_exp] (+ alt)
  uint32_t* ex_val = nullptr;
  uint64_t* ex_key2 = nullptr;
  uint32_t* ex_val2 = nullptr;
  uint32_t* ex_rec = nullptr;    // [n_exp] in-section record of each expanded record
  uint32_t* ex_cs = nullptr;     // [n_exp] held critical section
  uint32_t* ex_flags = nullptr;  // [n_exp + 1]
  uint32_t* ex_group = nullptr;  // [n_groups + 1]
  uint32_t* ex_dep_off = nullptr;  // [n_exp]
  uint32_t* ex_dep_cnt = nullptr;
  // phase G: propagation
  uint4* plan = nullptr;        // [2 * (n_sync + n_incs)] one 32-byte entry per clock-changing step
  uint4* recmeta = nullptr;     // [n_cs + 1] (agent, acquire epoch, release index, scope id)
  uint32_t* flat_off = nullptr; // [n_incs + 1] dependency list of each in-section access
  uint32_t* flat = nullptr;     // [pool_cap]
  uint32_t* rows = nullptr;     // [n_rows * RW], or [n_rows * B] headers of compressed versions
  uint32_t* cv_pool = nullptr;  // compressed versions: [cv_cap] warp words and lane values
  uint32_t* psnap = nullptr;    // [n_cs * RW]
  uint32_t* hsnap = nullptr;    // [n_cs * RW]
  uint32_t* tiles = nullptr;    // wide clocks: [tile_cap * kTileW] tile pool, tile 0 = zeros
  uint32_t* done = nullptr;     // [n_cs]
  uint32_t* cursor = nullptr;   // [W * n_locks]
  uint32_t* jsnap = nullptr;    // wide clocks: [n_cs * RW] JN tables published at releases
  uint32_t* bar_j = nullptr;    // [n_bar * 2 * Wp] global-barrier joins
  uint32_t* bar_cnt = nullptr;  // [n_bar]
  // forced compression at barriers: barriers by block, their members' records, offsets
  uint64_t *fb_key = nullptr, *fb_key2 = nullptr;  // [n_bar]
  uint32_t *fb_val = nullptr, *fb_val2 = nullptr;  // [n_bar]
  uint32_t* fb_rank = nullptr;                     // [n_bar] barrier -> position by block
  uint32_t* fb_off = nullptr;                      // [n_bar + 1] member counts, then offsets
  uint32_t* fb_blo = nullptr;                      // [B + 1] each block's first position
  uint4* fb_rec = nullptr;                         // [n_sync] (entry, N before, member, count)
  uint32_t* fb_boff = nullptr;                     // [n_sync] offset from each barrier entry on
  // phase I: check
  uint32_t* tails = nullptr;    // [n_chunks * 4 * Wp * 2]
  // sparse check: accesses grouped by (location, class, agent)
  uint32_t* wc_flag = nullptr;   // [n_acc] location-run starts in key order
  uint32_t* wc_run = nullptr;    // [n_acc + 1] exclusive scan of wc_flag
  uint64_t* wc_key = nullptr;    // [n_acc] (run << 15 | class << 13 | agent) (+ alt)
  uint32_t* wc_val = nullptr;    // [n_acc] key-order position (+ alt)
  uint64_t* wc_key2 = nullptr;
  uint32_t* wc_val2 = nullptr;
  uint32_t* wc_gflag = nullptr;  // [n_acc] group starts
  uint32_t* wc_gexcl = nullptr;  // [n_acc + 1]
  uint32_t* wc_grp_lo = nullptr;     // [n_groups + 1]
  uint32_t* wc_grp_agent = nullptr;  // [n_groups]
  uint32_t* wc_rc = nullptr;     // [4 * n_acc + 2] first group of each (run, class)
  uint32_t* wc_who = nullptr;    // [n_acc] record fields in key order: who, version row, epoch
  uint32_t* wc_row = nullptr;
  uint32_t* wc_ep = nullptr;
  // grouped order: hashed bitmap of the locations with a write-class access, and the
  // number of accesses the filter keeps (those whose location's bit is set)
  uint32_t* wl_bits = nullptr;  // [2^wl_log2 / 32]
  uint32_t* n_kept = nullptr;   // [1]
  unsigned long long* chunk_ns = nullptr;  // [n_chunks] check timeline (options.timeline)
  uint32_t* chunk_races = nullptr;         // [n_chunks]
  uint64_t* races = nullptr;    // [race_cap] (later << 32) | earlier
  uint64_t* races2 = nullptr;
  // scan scratch
  uint32_t* scan_tmp = nullptr;
  size_t scan_tmp_elems = 0;
};

// ---- primitives (gwcp_prims.cu) ----------------------------------------------------
// Process-wide count of kernels this library has launched (gwcp_launch_count).
void count_launch();
// Exclusive scan of n u32 values (in may equal out); writes the total to *total_dev
// when non-null. tmp must hold scan_tmp_need(n) elements.
size_t scan_tmp_need(size_t n);
void scan_exclusive(const uint32_t* in, uint32_t* out, size_t n, uint32_t* total_dev, uint32_t* tmp,
                    cudaStream_t s);
// Stable LSD radix sort of (key, val) pairs on the bits set in `mask`, 8-bit digits.
// Ping-pongs between (k0, v0) and (k1, v1); returns true if the result is in (k1, v1).
// tmp must hold radix_tmp_need(n) u32. With n_dev, only the first min(n, *n_dev) pairs are
// sorted (a count known on the device only; n bounds it).
// With keep.bits, the first pass keeps only the pairs whose bit wl_bit(key >> keep.shift,
// keep.log2) is set in keep.bits (a stable filter folded into the sort); the kept count is
// written to keep.n_out and bounds the later passes.
struct RadixKeep {
  const uint32_t* bits = nullptr;
  uint32_t log2 = 0, shift = 0;
  uint32_t* n_out = nullptr;
};
size_t radix_tmp_need(size_t n);
bool radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, size_t n, uint64_t mask,
                      uint32_t* tmp, cudaStream_t s, const uint32_t* n_dev = nullptr, RadixKeep keep = {});
// Digit windows covering the bits of `mask` (low bit of each window).
std::vector<int> radix_windows(uint64_t mask);

// ---- device helpers -----------------------------------------------------------------
__device__ __forceinline__ void set_error(DevStatus* st, int code, unsigned long long idx) {
  atomicCAS(&st->code, 0, code);
  atomicMin(&st->bad_index, idx);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Location key of an access: shared memory is per block (reading of the paper's
// shared-memory paragraph): (1 << 63) | (block << 40) | addr.
__device__ __forceinline__ uint64_t location_key(const Event& e, uint32_t apb) {
  if (e.space == GWCP_SPACE_SHARED) return (1ull << 63) | (uint64_t(e.agent / apb) << 40) | e.addr;
  return e.addr;
}

__device__ __forceinline__ uint32_t access_class(const Event& e) {
  if (e.op == GWCP_READ) return C_READ;
  if (e.op == GWCP_WRITE) return C_WRITE;
  return e.scope == GWCP_SCOPE_DEVICE ? C_ATOM_DEV : C_ATOM_CTA;
}

// scope id of a lock use: 0 device, block + 1 block-scoped
__device__ __forceinline__ uint32_t scope_id(uint32_t agent, uint8_t scope, uint32_t apb) {
  return scope == GWCP_SCOPE_DEVICE ? 0u : agent / apb + 1u;
}
__host__ __device__ __forceinline__ bool scopes_overlap(uint32_t a, uint32_t b) {
  return a == 0 || b == 0 || a == b;
}

// Members of a barrier event: first member and count, contiguous except WARP masks at
// thread granularity (then `mask` has the lane bits relative to `first`).
struct BarMembers {
  uint32_t first, count, mask;  // mask == 0 means the contiguous range [first, first+count)
  bool ok;
};
__device__ __forceinline__ BarMembers barrier_members(const Event& e, const Geo& g) {
  BarMembers m{0, 0, 0, false};
  if (e.scope == GWCP_SCOPE_CTA) {
    if (e.addr >= g.B) return m;
    m.first = uint32_t(e.addr) * g.apb;
    m.count = g.apb;
    m.ok = true;
    return m;
  }
  if (e.scope == GWCP_SCOPE_WARP) {
    if (e.addr == 0 || e.addr > 0xffffffffull) return m;
    if (g.gran == GWCP_GRAN_WARP) {
      m.first = e.agent;
      m.count = 1;
      m.ok = true;
      return m;
    }
    uint32_t blk = e.agent / g.apb;
    uint32_t base = blk * g.apb + ((e.agent - blk * g.apb) / 32u) * 32u;
    uint32_t mask = uint32_t(e.addr);
    uint32_t hi = 31 - __clz(mask);
    if (base + hi >= (blk + 1) * g.apb) return m;
    m.first = base;
    m.count = __popc(mask);
    m.mask = mask;
    m.ok = true;
  }
  return m;
}

// ---- launchers (defined in the phase files) -----------------------------------------
// ---- compressed clock versions (section "Vector Clock Compression") ---------------
// The paper's blockVC / warpVC form of a vector clock: one header word per block, holding
// the block's common value (bit 31 clear) or kCvExpanded | the pool offset of the block's
// warp words; a warp word holds the warp's common value or kCvExpanded | the pool offset
// of its 32 lane values. At warp granularity a warp is one agent, so the warp words of an
// expanded block are the agents' values. Values must stay below 2^31: every clock entry
// is a local time, at most 1 + the number of synchronisation entries (forced compression
// raises a local time only to another member's), which the host bounds.
constexpr uint32_t kCvExpanded = 0x80000000u;
constexpr uint32_t kCvChunk = 2048;  // pool words a walker takes at a time
__host__ __device__ inline uint32_t cv_group(uint32_t gran) { return gran == GWCP_GRAN_WARP ? 1u : 32u; }

// Entry v of the compressed version whose headers start at hdr; offsets at or past cap
// (headers a failed walk left stale) read as zero.
__device__ __forceinline__ uint32_t cv_entry(const uint32_t* hdr, const uint32_t* pool, unsigned long long cap,
                                             uint32_t v, uint32_t apb, uint32_t gs) {
  const uint32_t h = __ldg(hdr + v / apb);
  if (!(h & kCvExpanded)) return h;
  const uint32_t l = v % apb;
  const unsigned long long o = (h & ~kCvExpanded) + l / gs;
  if (o >= cap) return 0u;
  const uint32_t w = __ldg(pool + o);
  if (!(w & kCvExpanded)) return w;
  const unsigned long long o2 = (w & ~kCvExpanded) + l % gs;
  return o2 < cap ? __ldg(pool + o2) : 0u;
}

struct Sizes {
  uint64_t N = 0;
  uint32_t ntA = 0, TA = 0;
  uint32_t nS = 0, n_acc = 0, n_acqrel = 0, n_bar = 0;
  uint32_t ntS = 0;
  uint32_t n_sync = 0, n_incs = 0, n_rows = 0, n_cs = 0, n_locks = 0, n_exp = 0, n_groups = 0;
  uint32_t pool_cap = 0;
  uint32_t n_chunks = 0;
  uint64_t race_cap = 0;
  uint64_t tile_cap = 0;      // wide clocks: tiles in the pool
  bool cta_barriers = false;  // every block fits one CTA of walkers
  bool hb_only = false;       // versions hold H_t: the check then tests scoped happens-before
  bool sparse_check = false;  // partner-group check (always with tile clocks)
  bool pack_walkers = false;  // tile walkers: two CTAs per SM where they fit
  uint32_t n_timeline = 0;    // check timeline entries (chunks or check blocks)
  bool forced_barrier = false;  // members leave a barrier at their highest local time
  bool compress = false;        // clock versions in the block/warp compressed form
  uint64_t cv_cap = 0;          // words of the compressed-version pool
  // grouped access order (partner check without a ranker): the access keys are the
  // composite (location, class, agent), one sort groups each location's accesses by class
  // and agent in trace order. The location part is the key's varying bits [comp_lo,
  // comp_lo + comp_span) and the shared-memory flag above them.
  bool grouped = false;
  uint32_t comp_lo = 0, comp_span = 0;
  uint32_t wl_log2 = 0;  // bits of the written-location bitmap (log2); 0 = no filter
  uint32_t n_kept = 0;   // grouped order: accesses the filter kept (read back after the sort)
  uint32_t d_shift = 0, d_nw = 0;  // phase D index: trace windows of 2^d_shift events, d_nw per agent
  // many agents: S is built by a stable sort of (agent, entry) keys instead of per-(agent,
  // tile) counting tables (which would limit phase A to a few warps per SM)
  bool agent_sort = false;
};

// bit of a location (the composite key without its class and agent) in the
// written-location bitmap of 2^log2 bits: the top bits of MurmurHash3's 64-bit finaliser
__host__ __device__ inline uint32_t wl_bit(uint64_t loc_part, uint32_t log2) {
  uint64_t x = loc_part;
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return uint32_t(x >> (64 - log2));
}

// composite access key of the grouped order (see Sizes::grouped)
__host__ __device__ inline uint64_t composite_key(uint64_t loc, uint32_t cls, uint32_t agent, uint32_t lo,
                                                 uint32_t span) {
  const uint64_t addr = ((loc & ~(1ull << 63)) >> lo) & ((1ull << span) - 1);
  return ((addr | ((loc >> 63) << span)) << 15) | (uint64_t(cls) << 13) | agent;
}

// profiling hook: records an event pair around each launch when enabled
struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
    double bytes;
    cudaStream_t s;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t ev();
  void begin(const char* name, double bytes, cudaStream_t on = nullptr);  // nullptr: the default stream s
  void end();
};

void phaseA_count(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseA_scatter(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseB_sync(const Bufs& b, const Geo& g, Sizes& z, cudaStream_t s, Prof& p);
void phaseC_walk(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseC_forced(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseD_gaps(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
// phase D's trace-order pass alone (filtered: the grouped order's kept accesses only; the
// records of the others are then left unwritten)
void phaseD_trace(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, bool filtered);
void phaseE_locks(Bufs& b, const Geo& g, const Sizes& z, uint64_t lock_mask, cudaStream_t s, Prof& p);
void phaseE_walk(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseF_incs(const Bufs& b, const Geo& g, const Sizes& z, uint64_t key_mask, cudaStream_t s, Prof& p);
void phaseF_walk(Bufs& b, const Geo& g, const Sizes& z, uint64_t key_mask, cudaStream_t s, Prof& p);
int phaseG_propagate(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
// failure detection test: the walkers' bounded wait on a row nothing completes
int wait_probe(uint32_t limit, int* code);
// access grouping; tmp is the sort scratch (it may run beside other work on stream s)
void phaseH_sort(Bufs& b, const Geo& g, const Sizes& z, uint64_t key_mask, uint32_t* tmp, cudaStream_t s, Prof& p);
// per-chunk carries of the check (needs the sorted accesses and AccInfo, not the clocks)
void phaseI_carry(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
void phaseI_check(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
bool phaseI_sort_races(const Bufs& b, const Sizes& z, uint64_t n_races, cudaStream_t s, Prof& p);
// address ranker (gwcp_rank.cu): features of the locations of a sorted access stream, the
// MLP's scores, and the ranked order of the stream (location runs by descending score)
constexpr int kRankParams = 5313, kRankFeatures = 16;
struct RankIn {
  const uint64_t* key;   // [n_acc] sorted so that each location's accesses are one run, in trace order
  const uint32_t* idx;   // [n_acc]
  const AccInfo* info;
  uint32_t n_acc;
  const uint32_t* incs_idx;  // [n_incs] accesses inside a critical section
  uint32_t n_incs;
  uint32_t* bits;            // [N / 32 + 1] scratch bitmap
  const uint32_t* acqrel;    // [n_acqrel] acquire/release trace indices, ascending
  uint32_t n_acqrel;
  const uint32_t* bar;       // [n_bar] barrier trace indices, ascending
  uint32_t n_bar;
};
size_t rank_tmp_words(uint32_t n_acc);
void rank_features(const RankIn& in, uint32_t* tmp, size_t bits_words, float* feat, uint64_t* loc_key,
                   uint32_t* n_loc_dev, uint32_t* scan_tmp, cudaStream_t s);
void rank_scores(const float* theta, const float* feat, const uint32_t* n_dev, uint32_t n_bound, float* score,
                 cudaStream_t s);
void rank_order(const RankIn& in, const uint32_t* tmp, const float* score, uint64_t* rkey, uint32_t* rval,
                uint64_t* rkey2, uint32_t* rval2, uint64_t* key_out, uint32_t* idx_out, uint32_t* sort_tmp,
                cudaStream_t s);
int rank_grad(const float* theta, const float* feat, const float* y, uint32_t lo, uint32_t hi, float pos_weight,
              float inv_b, float* grad, float* loss, cudaStream_t s);
void rank_adam(float* theta, float* m, float* v, float* grad, float lr, float c1, float c2, cudaStream_t s);
int rank_epoch(float* theta, const float* feat, const float* y, uint32_t n, uint32_t batch, float lr,
               float pos_weight, float* m, float* v, float* grad, float* loss_acc, float* losses, uint32_t* ctr,
               cudaStream_t s);
// sorted race words (later << 32 | earlier) -> gwcp_race records (gwcp_check.cu)
void races_to_records(const uint64_t* words, uint64_t n, gwcp_race* out, cudaStream_t s);
// check timeline: per chunk the globaltimer at its end and its race count (optional)
void stamp_now(unsigned long long* at, cudaStream_t s);

// wide clocks and the sparse check (gwcp_wide.cu): the walker over tile tables (after the
// plan is built), the grouping of accesses (on the side stream: the grouped order's groups,
// or with a ranker the regrouping of its location order) and the per-access partner check
int phaseG_wide(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s);
void phaseI_wide_group(Bufs& b, const Geo& g, Sizes& z, uint32_t* tmp, cudaStream_t s, Prof& p);
void phaseI_grouped(Bufs& b, const Geo& g, Sizes& z, uint32_t* tmp, cudaStream_t s, Prof& p);
void phaseI_wide_check(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p);
uint32_t sparse_check_blocks(uint32_t n_acc);  // timeline entries of the partner-group check

}  // namespace gwcp
