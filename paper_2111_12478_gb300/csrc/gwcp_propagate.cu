// Clock propagation of libgwcp (Algorithms 1 and 2 of the paper).
//
// One warp per agent walks the agent's clock-changing entries in trace order:
// acquires, releases, barrier participations and accesses made while holding a lock.
// The agent's P_t and H_t live in registers, blocked so that lane l holds entries
// [l*K, l*K+K) (K = Wp/32); every join is a 32-lane vector max over the whole clock
// width (64-, 128- or 256-bit loads). After each entry the warp stores P_t as the
// agent's next clock version; the race check reads those rows.
//
// Cross-agent values are snapshots written once: a release stores P_t and H_t (the
// paper's P_<l,s>, H_<l,s> and its Rel-queue entry) and then raises a completion flag
// with release semantics. An acquire waits (bounded) on the flags of the releases it
// joins - the latest release on every overlapping scope of the lock, precomputed per
// acquire. Because every dependence points backwards in trace order and each walker
// processes its own entries in trace order, the earliest unprocessed event can always
// proceed, so all waits end on a well-formed trace. All walkers are co-resident
// (cooperative launch). A barrier whose block fits in one CTA is a CTA barrier with a
// shared-memory join; other barriers use a per-barrier global join with atomics and a
// bounded wait. A wait that gives up sets GWCP_ERR_TIMEOUT and the walker continues
// without waiting, so no CTA barrier is left short of arrivals.
#include "gwcp_internal.cuh"

namespace gwcp {

namespace {

constexpr uint32_t kSpinLimit = 1u << 23;

struct PropArgs {
  Geo g;
  const Event* ev;
  DevStatus* st;
  const uint32_t *sy_start, *sy_idx, *sy_kind, *sy_N, *sy_ver, *sy_aux, *sy_agent;
  const uint32_t *incs_off, *incs_ver, *incs_k, *exp_off, *ex_dep_off, *ex_dep_cnt;
  const uint32_t* rowbase;
  const uint32_t *cs_of_sync, *cs_agent, *cs_sid, *cs_epoch, *cs_rel_idx, *cs_lock, *lock_cs_lo, *cs_rel_epoch;
  const uint32_t *acq_dep_off, *acq_dep_cnt, *pool;
  const uint32_t* flat;
  uint4* plan;
  uint4* recmeta;
  uint32_t hb_only;  // publish H_t instead of P_t as the clock versions the check reads
  uint32_t* rows;
  uint32_t *psnap, *hsnap, *done, *cursor;
  uint32_t *bar_j, *bar_cnt;
  uint32_t n_locks;
  int cta_barriers;
  uint32_t forced;  // forced compression at barriers: local times come from the plan
  // compressed clock versions: rows holds B header words per version
  uint32_t compress;
  uint32_t* cv_pool;
  unsigned long long cv_cap;
  unsigned long long *cv_used, *cv_words;  // pool words handed out; words written
};

// Clock rows another walker may still be writing: every word goes once from SENTINEL to
// its value, and a reader takes a row only when no word is SENTINEL, so relaxed gpu-scope
// accesses (each word single-copy atomic, no order between words needed) make the
// exchange race-free under the PTX memory model; they cost what .cg accesses cost.
template <int K>
__device__ __forceinline__ void load_row(const uint32_t* row, uint32_t (&x)[K]) {
  const int lane = threadIdx.x & 31;
  const uint32_t* p = row + lane * K;
  if constexpr (K == 1) {
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(x[0]) : "l"(p) : "memory");
  } else if constexpr (K == 2) {
    asm volatile("ld.relaxed.gpu.global.v2.u32 {%0, %1}, [%2];" : "=r"(x[0]), "=r"(x[1]) : "l"(p) : "memory");
  } else {
#pragma unroll
    for (int j = 0; j < K; j += 4)
      asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(x[j]), "=r"(x[j + 1]), "=r"(x[j + 2]), "=r"(x[j + 3])
                   : "l"(p + j)
                   : "memory");
  }
}

template <int K>
__device__ __forceinline__ void store_row(uint32_t* row, const uint32_t (&x)[K]) {
  const int lane = threadIdx.x & 31;
  uint32_t* p = row + lane * K;
  if constexpr (K == 1) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x[0]) : "memory");
  } else if constexpr (K == 2) {
    asm volatile("st.relaxed.gpu.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(x[0]), "r"(x[1]) : "memory");
  } else {
#pragma unroll
    for (int j = 0; j < K; j += 4)
      asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p + j), "r"(x[j]), "r"(x[j + 1]),
                   "r"(x[j + 2]), "r"(x[j + 3])
                   : "memory");
  }
}

// the same blocked layout in shared memory (plain stores: __stcg is for global memory)
template <int K>
__device__ __forceinline__ void store_row_shared(uint32_t* row, const uint32_t (&x)[K]) {
  uint32_t* p = row + (threadIdx.x & 31) * K;
#pragma unroll
  for (int j = 0; j < K; ++j) p[j] = x[j];
}

// Walker state of the compressed-version pool: the chunk being filled, words written.
struct CvState {
  unsigned long long cur, end, words;
};

// Stores the clock the warp left in `scratch` (its Wc shared words, entry e at e) as the
// compressed version `row` (the blockVC / warpVC form): B header words at rows + row * B;
// the words of expanded blocks go to the pool, from a chunk of kCvChunk words the walker
// takes at a time. A version that does not fit the pool gets zero headers, and the host
// runs again with a larger pool (cv_used keeps counting). Only the compressing walker
// instantiations contain it, out of line (the register path below is the common one).
__device__ __noinline__ CvState put_row_c(const PropArgs& a, uint32_t row, const uint32_t* scratch, CvState cs) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t apb = a.g.apb, nb = a.g.B, gs = cv_group(a.g.gran), nw = (apb + gs - 1) / gs;
  // pass 1: which of the lane's blocks (b = lane + 32 i) are uniform, and the words the
  // others need: nw warp words, plus 32 lane values per warp that is not uniform
  uint32_t need = 0, umask = 0;
  for (uint32_t b = lane, i = 0; b < nb; b += 32, ++i) {
    const uint32_t* q = scratch + b * apb;
    bool uni = true;
    uint32_t ew = 0;
    for (uint32_t w = 0; w < nw; ++w) {
      const uint32_t lo = w * gs, hi = min(lo + gs, apb), v = q[lo];
      bool wu = true;
      for (uint32_t e = lo; e < hi; ++e) wu &= q[e] == v;
      uni &= wu && v == q[0];
      ew += wu ? 0u : 1u;
    }
    if (uni)
      umask |= 1u << i;
    else
      need += nw + 32 * ew;
  }
  const uint32_t incl = warp_inclusive_scan(need);
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  if (total && cs.cur + total > cs.end) {
    unsigned long long base = 0;
    const unsigned long long take = max(total, kCvChunk);
    if (lane == 0) base = atomicAdd(a.cv_used, take);
    base = __shfl_sync(0xffffffffu, base, 0);
    cs.cur = base;
    cs.end = base + take;
  }
  unsigned long long o = cs.cur + (incl - need);
  cs.cur += total;
  cs.words += nb + total;
  const bool fits = cs.cur <= a.cv_cap;  // the whole version lies inside the pool
  uint32_t* hdr = a.rows + size_t(row) * nb;
  // pass 2: headers, warp words and lane values
  for (uint32_t b = lane, i = 0; b < nb; b += 32, ++i) {
    const uint32_t* q = scratch + b * apb;
    if ((umask >> i) & 1u) {
      __stcg(hdr + b, q[0]);
      continue;
    }
    if (!fits) {
      __stcg(hdr + b, 0u);
      continue;
    }
    __stcg(hdr + b, kCvExpanded | uint32_t(o));
    unsigned long long o2 = o + nw;
    for (uint32_t w = 0; w < nw; ++w) {
      const uint32_t lo = w * gs, hi = min(lo + gs, apb), v = q[lo];
      bool wu = true;
      for (uint32_t e = lo; e < hi; ++e) wu &= q[e] == v;
      if (wu) {
        __stcg(a.cv_pool + o + w, v);
      } else {
        __stcg(a.cv_pool + o + w, kCvExpanded | uint32_t(o2));
        for (uint32_t e = 0; e < 32; ++e) __stcg(a.cv_pool + o2 + e, lo + e < apb ? q[lo + e] : 0u);
        o2 += 32;
      }
    }
    o = o2;
  }
  __syncwarp();
  return cs;
}

// The same store from registers, for warp granularity with K dividing agents_per_block:
// a block is L = apb / K consecutive lanes, so its uniformity is one ballot and its
// expanded words are the lanes' own entries (one per agent, in agent order).
template <int K>
__device__ __forceinline__ CvState put_row_lanes(const PropArgs& a, uint32_t row, const uint32_t (&x)[K], CvState cs) {
  const uint32_t lane = threadIdx.x & 31, apb = a.g.apb, nb = a.g.B, L = apb / K;
  const uint32_t grp = lane / L, first = grp * L;
  const bool live = grp < nb;  // lanes past the last block hold padding
  bool same = true;
#pragma unroll
  for (int j = 0; j < K; ++j) same &= x[j] == x[0];
  const uint32_t head_v = __shfl_sync(0xffffffffu, x[0], live ? first : lane);
  const uint32_t ok = __ballot_sync(0xffffffffu, live && same && x[0] == head_v);
  const uint32_t gmask = live ? ((L == 32 ? 0xffffffffu : (1u << L) - 1u) << first) : 0u;
  const bool uni = live && (ok & gmask) == gmask;
  const bool head = live && lane == first;
  const uint32_t expm = __ballot_sync(0xffffffffu, head && !uni);  // bit at each expanded block's first lane
  const uint32_t total = __popc(expm) * apb;
  if (total && cs.cur + total > cs.end) {
    unsigned long long base = 0;
    const unsigned long long take = max(total, kCvChunk);
    if (lane == 0) base = atomicAdd(a.cv_used, take);
    base = __shfl_sync(0xffffffffu, base, 0);
    cs.cur = base;
    cs.end = base + take;
  }
  const unsigned long long o = cs.cur + (unsigned long long)apb * __popc(expm & ((1u << first) - 1u));
  cs.cur += total;
  cs.words += nb + total;
  const bool fits = cs.cur <= a.cv_cap;
  if (head) __stcg(a.rows + size_t(row) * nb + grp, uni ? x[0] : fits ? kCvExpanded | uint32_t(o) : 0u);
  if (live && !uni && fits) {
#pragma unroll
    for (int j = 0; j < K; ++j) __stcg(a.cv_pool + o + (lane - first) * K + j, x[j]);
  }
  return cs;
}

template <int K>
__device__ __forceinline__ void join_row(uint32_t (&x)[K], const uint32_t* row) {
  uint32_t y[K];
  load_row<K>(row, y);
#pragma unroll
  for (int j = 0; j < K; ++j) x[j] = max(x[j], y[j]);
}

// entry v of a blocked clock (owner lane v / K, register v % K), broadcast to the warp
template <int K>
__device__ __forceinline__ uint32_t get_entry(const uint32_t (&x)[K], uint32_t v) {
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (j == int(v % K)) r = x[j];
  return __shfl_sync(0xffffffffu, r, int(v / K));
}

template <int K>
__device__ __forceinline__ void set_entry(uint32_t (&x)[K], uint32_t v, uint32_t val) {
  if ((threadIdx.x & 31) == v / K) {
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j == int(v % K)) x[j] = val;
  }
}

constexpr uint32_t SENTINEL = 0xFFFFFFFFu;  // no clock entry ever takes this value
enum : uint32_t { P_ACQ = 0, P_REL = 1, P_BAR = 2, P_INCS = 3 };
enum : uint32_t { BAR_SINGLE = 0, BAR_CTA = 1, BAR_GLOBAL = 2 };

// Snapshot rows are written once by another walker. They start filled with SENTINEL;
// each 32-bit word is written exactly once, so a row with no SENTINEL word is complete.
// Rows are always read through L2 (ld.cg, cp.async.cg), never cached in L1. No flag or
// fence is involved.
template <int K>
__device__ __forceinline__ bool row_complete(const uint32_t (&y)[K]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < K; ++j) ok &= y[j] != SENTINEL;
  return __all_sync(0xffffffffu, ok);
}

// re-read from L2 until complete (bounded: after `limit` polls the wait gives up, sets
// GWCP_ERR_TIMEOUT and the walker carries on)
template <int K>
__device__ __noinline__ void wait_row(const uint32_t* row, uint32_t (&y)[K], bool& abort, DevStatus* st,
                                     uint32_t limit = kSpinLimit) {
  uint32_t it = 0;
  for (;;) {
    load_row<K>(row, y);
    if (row_complete<K>(y) || abort) return;
    if (++it > limit) {
      if ((threadIdx.x & 31) == 0) atomicCAS(&st->code, 0, GWCP_ERR_TIMEOUT);
      abort = true;
      return;
    }
    __nanosleep(32);
  }
}

// x |= the rows at base + ids[q] * Wp, all loads issued before any is used
template <int K, int M>
__device__ __forceinline__ void join_rows(uint32_t (&x)[K], const uint32_t* base, const uint32_t (&ids)[M], int n,
                                          uint32_t Wp, bool& abort, DevStatus* st) {
  uint32_t y[M][K];
#pragma unroll
  for (int q = 0; q < M; ++q)
    if (q < n) load_row<K>(base + size_t(ids[q]) * Wp, y[q]);
#pragma unroll
  for (int q = 0; q < M; ++q) {
    if (q < n) {
      if (!row_complete<K>(y[q])) wait_row<K>(base + size_t(ids[q]) * Wp, y[q], abort, st);
#pragma unroll
      for (int j = 0; j < K; ++j) x[j] = max(x[j], y[q][j]);
    }
  }
}

// x |= rows of base_x, y |= rows of base_y for the same ids: all loads issued first
template <int K, int M>
__device__ __forceinline__ void join_rows2(uint32_t (&x)[K], const uint32_t* base_x, uint32_t (&y)[K],
                                           const uint32_t* base_y, const uint32_t (&ids)[M], int n, uint32_t Wp,
                                           bool& abort, DevStatus* st) {
  uint32_t rx[M][K], ry[M][K];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    if (q < n) {
      load_row<K>(base_x + size_t(ids[q]) * Wp, rx[q]);
      load_row<K>(base_y + size_t(ids[q]) * Wp, ry[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < M; ++q) {
    if (q < n) {
      if (!row_complete<K>(rx[q])) wait_row<K>(base_x + size_t(ids[q]) * Wp, rx[q], abort, st);
      if (!row_complete<K>(ry[q])) wait_row<K>(base_y + size_t(ids[q]) * Wp, ry[q], abort, st);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        x[j] = max(x[j], rx[q][j]);
        y[j] = max(y[j], ry[q][j]);
      }
    }
  }
}

// P entry v of every lane's own agent index (lane-varying v), by K shuffles
template <int K>
__device__ __forceinline__ uint32_t lookup_entry(const uint32_t (&x)[K], uint32_t v) {
  uint32_t r = 0;
  const int src = int(min(v, 32u * K - 1) / K);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const uint32_t t = __shfl_sync(0xffffffffu, x[j], src);
    if (j == int(v % K)) r = t;
  }
  return r;
}

// cp.async (LDGSTS): 16-byte copy global -> shared through L2 only (no L1 line that
// could hold a row before its release wrote it)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// stage one clock row (Wc words) into shared memory: lane l copies 16-byte chunk l
template <int Wc>
__device__ __forceinline__ void stage_row(uint32_t* dst, const uint32_t* src) {
  const int lane = threadIdx.x & 31;
  if (lane < Wc / 4) cp_async16(dst + 4 * lane, src + 4 * lane);
}

template <int K>
__device__ __forceinline__ void read_row_shared(const uint32_t* row, uint32_t (&y)[K]) {
  const uint32_t* p = row + (threadIdx.x & 31) * K;
#pragma unroll
  for (int j = 0; j < K; ++j) y[j] = p[j];
}

// shared-memory words per ring slot: four rows, or 32 section records + one row; then
// a 4-word header (kind, staged cursor, row count)
template <int K>
__host__ __device__ constexpr int slot_words() {
  return (((4 * 32 * K > 128 + 32 * K) ? 4 * 32 * K : 128 + 32 * K) + 4 + 3) & ~3;
}

// One warp per agent walks the agent's plan (its clock-changing steps in trace order).
// R > 0: a ring of R shared-memory slots per warp; while entry p is processed, the
// copies for entry p + R - 1 are in flight (one commit group per entry).
// CV: clock versions stored compressed (a separate instantiation, so that the plain
// walkers' register allocation does not carry it).
template <int K, int R, int MAXT, bool CV>
__global__ void __launch_bounds__(MAXT, 1) k_propagate(PropArgs a) {
  constexpr int Wc = 32 * K;
  constexpr int SLOT = slot_words<K>();
  constexpr int RR = R > 0 ? R : 1;
  extern __shared__ __align__(16) uint32_t sm[];
  const Geo& g = a.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t u = a.cta_barriers ? blockIdx.x * g.apb + warp : blockIdx.x * 32 + warp;
  uint32_t* const xchg = sm;  // CTA barriers: [2 buffers][warps][C | H][Wp]
  const uint32_t xchg_words = a.cta_barriers ? 2u * nwarps * 2 * Wc : 0u;
  uint32_t* const ring = sm + xchg_words + (R > 0 ? size_t(warp) * RR * SLOT : 0);  // unused when R = 0
  // per-warp scratch for folding joined release epochs into jn (stale words never exceed jn)
  uint32_t* const jn_tmp = sm + xchg_words + (R > 0 ? size_t(nwarps) * RR * SLOT : 0) + size_t(warp) * Wc;
  // one read of the status per CTA, so all warps of a CTA agree on whether to run
  __shared__ int start_code;
  if (threadIdx.x == 0) start_code = *(volatile int*)&a.st->code;
  __syncthreads();
  if (start_code) return;
  const bool active = a.cta_barriers ? (uint32_t(warp) < g.apb) : (u < g.W);
  if (!active) return;
  for (int j = lane; j < Wc; j += 32) jn_tmp[j] = 0;
  __syncwarp();

  uint32_t P[K], H[K];
  // jn[v]: latest release epoch of agent v whose H snapshot is already joined into P.
  // H of one agent only grows along its timeline, so a release of v with epoch <= jn[v]
  // is dominated and its join is a no-op.
  uint32_t jn[K];
#pragma unroll
  for (int j = 0; j < K; ++j) P[j] = H[j] = jn[j] = 0;
  set_entry<K>(H, u, 1u);  // H_t = bottom{t := 1}
  uint32_t N = 1;          // N_t
  bool abort = false;
  uint64_t joins = 0, visits = 0;
  uint32_t nbar = 0;
  CvState cvs{0, 0, 0};  // compressed versions
  const bool cv_lanes = g.gran == GWCP_GRAN_WARP && g.apb % K == 0;
  auto put_version = [&](uint32_t r) {
    if constexpr (CV) {
      if (cv_lanes) {
        cvs = a.hb_only ? put_row_lanes<K>(a, r, H, cvs) : put_row_lanes<K>(a, r, P, cvs);
        return;
      }
      // the clock goes through the warp's jn scratch words, which are then left holding jn
      // (the release loop's rule: no word there exceeds jn)
      if (a.hb_only)
        store_row_shared<K>(jn_tmp, H);
      else
        store_row_shared<K>(jn_tmp, P);
      __syncwarp();
      cvs = put_row_c(a, r, jn_tmp, cvs);
      store_row_shared<K>(jn_tmp, jn);
      __syncwarp();
    } else if (a.hb_only) {
      store_row<K>(a.rows + size_t(r) * Wc, H);
    } else {
      store_row<K>(a.rows + size_t(r) * Wc, P);
    }
  };
  put_version(a.rowbase[u]);
  const uint32_t k0 = a.sy_start[u], k1 = a.sy_start[u + 1];
  const uint32_t pb = k0 + a.incs_off[k0], pe = k1 + a.incs_off[k1];
  uint32_t* const cursor_row = a.cursor + size_t(u) * a.n_locks;

  // plan entries in registers: the current batch of 32 and the next one; a release
  // entry's lane also holds its cursor (forwarded when an earlier release of the same
  // lock moves it)
  uint4 ea, eb, ea2, eb2;
  uint32_t pre, pre2;
  auto load_batch = [&](uint32_t b0, uint4& xa, uint4& xb, uint32_t& xp) {
    const uint32_t pi = b0 + lane;
    xa = make_uint4(0, 0, 0, 0);
    xb = make_uint4(0, 0, 0, 0);
    xp = 0;
    if (pi < pe) {
      xa = a.plan[2 * size_t(pi)];
      xb = a.plan[2 * size_t(pi) + 1];
      if ((xa.x & 0xFF) == P_REL) xp = __ldcg(cursor_row + xa.w);
    }
  };
  uint32_t base = pb;
  load_batch(base, ea, eb, pre);
  load_batch(base + 32, ea2, eb2, pre2);

  auto stage = [&](uint32_t p) {
    if constexpr (R > 0) {
      if (p < pe) {
        const bool second = p >= base + 32;
        const int src = int((p - base) & 31);
        const uint32_t t2 = __shfl_sync(0xffffffffu, second ? ea2.x : ea.x, src) & 0xFF;
        if (t2 == P_BAR) {  // a barrier stages nothing: an empty group, header kind 0
          if (lane == 0) (ring + (p % R) * SLOT)[SLOT - 4] = 0u;
          cp_async_commit();
          return;
        }
        const uint32_t w2 = __shfl_sync(0xffffffffu, second ? ea2.w : ea.w, src);
        const uint32_t x0 = __shfl_sync(0xffffffffu, second ? eb2.x : eb.x, src);
        const uint32_t x1 = __shfl_sync(0xffffffffu, second ? eb2.y : eb.y, src);
        const uint32_t x2 = __shfl_sync(0xffffffffu, second ? eb2.z : eb.z, src);
        const uint32_t x3 = __shfl_sync(0xffffffffu, second ? eb2.w : eb.w, src);
        const uint32_t pr = __shfl_sync(0xffffffffu, second ? pre2 : pre, src);
        uint32_t* slot = ring + (p % R) * SLOT;
        uint32_t kind = 0, nrows = 0, cur_staged = 0;
        if (t2 == P_ACQ && w2 >= 1 && w2 <= 2) {
          stage_row<Wc>(slot, a.psnap + size_t(x0) * Wc);
          stage_row<Wc>(slot + Wc, a.hsnap + size_t(x0) * Wc);
          if (w2 == 2) {
            stage_row<Wc>(slot + 2 * Wc, a.psnap + size_t(x1) * Wc);
            stage_row<Wc>(slot + 3 * Wc, a.hsnap + size_t(x1) * Wc);
          }
          kind = 1;
          nrows = 2 * w2;
        } else if (t2 == P_INCS && w2 >= 1 && w2 <= 4) {
          const uint32_t ids[4] = {x0, x1, x2, x3};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < int(w2)) stage_row<Wc>(slot + q * Wc, a.hsnap + size_t(ids[q]) * Wc);
          kind = 1;
          nrows = w2;
        } else if (t2 == P_REL) {
          const uint32_t lo = x0, hi = x1;
          cur_staged = pr;
          if (lo + pr + lane < hi) cp_async16(slot + 4 * lane, a.recmeta + lo + pr + lane);
          if (lo + pr < hi) stage_row<Wc>(slot + 128, a.hsnap + size_t(lo + pr) * Wc);
          kind = 2;
        }
        if (lane == 0) {
          slot[SLOT - 4] = kind;
          slot[SLOT - 3] = cur_staged;
          slot[SLOT - 2] = nrows;
        }
      }
      cp_async_commit();
    }
  };
  for (int q = 0; q < R - 1; ++q) stage(pb + q);

  for (uint32_t p = pb; p < pe; ++p) {
    const uint32_t i = p - base;
    __syncwarp();
    stage(p + R - 1);
    uint32_t skind = 0;
    const uint32_t* slot = ring + (R > 0 ? (p % RR) : 0) * SLOT;
    if constexpr (R > 0) {
      cp_async_wait<(R > 0 ? R - 1 : 0)>();
      __syncwarp();
      skind = slot[SLOT - 4];
    }
    const uint32_t t = __shfl_sync(0xffffffffu, ea.x, i) & 0xFF;
    const uint32_t row = __shfl_sync(0xffffffffu, ea.y, i);
    const uint32_t z = __shfl_sync(0xffffffffu, ea.z, i);
    const uint32_t w = __shfl_sync(0xffffffffu, ea.w, i);
    if ((t == P_ACQ || t == P_INCS) && skind == 1) {
      // staged rows: validate (an incomplete one is re-read from L2), then join
      const int nrows = int(slot[SLOT - 2]);
      const uint32_t ids[4] = {__shfl_sync(0xffffffffu, eb.x, i), __shfl_sync(0xffffffffu, eb.y, i),
                               __shfl_sync(0xffffffffu, eb.z, i), __shfl_sync(0xffffffffu, eb.w, i)};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < nrows) {
          uint32_t y[K];
          read_row_shared<K>(slot + q * Wc, y);
          const bool acq = t == P_ACQ;
          const uint32_t* src = acq ? ((q & 1) ? a.hsnap : a.psnap) + size_t(ids[q >> 1]) * Wc
                                    : a.hsnap + size_t(ids[q]) * Wc;
          if (!row_complete<K>(y)) wait_row<K>(src, y, abort, a.st);
          if (acq && (q & 1)) {
#pragma unroll
            for (int j = 0; j < K; ++j) H[j] = max(H[j], y[j]);
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) P[j] = max(P[j], y[j]);
          }
        }
      }
      joins += nrows;
    } else if (t == P_ACQ || t == P_INCS) {
      // acquire (Algorithm 1): P_t |= P_<l,s'>, H_t |= H_<l,s'> over the overlapping
      // scopes' latest releases; in-section access (Algorithm 2): P_t |= L^w (| L^r)
      const uint32_t* list = t == P_ACQ ? a.pool : a.flat;
      for (uint32_t q0 = 0; q0 < w; q0 += 4) {
        uint32_t ids[4];
        if (w <= 4) {
          ids[0] = __shfl_sync(0xffffffffu, eb.x, i);
          ids[1] = __shfl_sync(0xffffffffu, eb.y, i);
          ids[2] = __shfl_sync(0xffffffffu, eb.z, i);
          ids[3] = __shfl_sync(0xffffffffu, eb.w, i);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) ids[q] = q0 + q < w ? __ldcg(list + z + q0 + q) : 0;
        }
        const int n = int(min(4u, w - q0));
        if (t == P_ACQ) {
          join_rows2<K, 4>(P, a.psnap, H, a.hsnap, ids, n, Wc, abort, a.st);
          joins += 2 * n;
        } else {
          join_rows<K, 4>(P, a.hsnap, ids, n, Wc, abort, a.st);
          joins += n;
        }
      }
    } else if (t == P_REL) {
      // release (Algorithm 1): pop other agents' records on this lock while their
      // acquire is ordered before C_t; join the released ones whose scope overlaps.
      // Waves: every record before the first one failing the test against the current
      // P passes (P only grows), so their snapshots are joined together; the failing
      // record is tested again only if the wave changed P.
      const uint32_t c = z, L = w;
      const uint32_t lo = __shfl_sync(0xffffffffu, eb.x, i), hi = __shfl_sync(0xffffffffu, eb.y, i);
      const uint32_t s = __shfl_sync(0xffffffffu, eb.z, i), my_idx = __shfl_sync(0xffffffffu, eb.w, i);
      uint32_t cur = __shfl_sync(0xffffffffu, pre, i);
      bool staged = skind == 2 && slot[SLOT - 3] == cur;
      bool stop = false;
      while (!stop && lo + cur < hi) {
        const uint32_t rec = lo + cur + lane;
        const uint32_t nbr = min(32u, hi - (lo + cur));
        uint4 m = make_uint4(NONE, 0, NONE, 0);
        uint32_t spec[K];
        if (staged) {  // the first 32 records and the first one's snapshot are in the slot
          if (rec < hi) m = *reinterpret_cast<const uint4*>(slot + 4 * lane);
          read_row_shared<K>(slot + 128, spec);
        } else {
          if (rec < hi) m = __ldg(a.recmeta + rec);
          load_row<K>(a.hsnap + size_t(lo + cur) * Wc, spec);
        }
        staged = false;
        bool spec_live = true;
        const uint32_t mag = m.x == NONE ? NONE : (m.x & 0xFFFF);
        const uint32_t msid = m.x >> 16;
        const bool mine = mag == u;
        const bool joinable = !mine && m.z != NONE && m.z < my_idx && scopes_overlap(msid, s);
        uint32_t start = 0;
        while (start < nbr) {
          const uint32_t pv = lookup_entry<K>(P, mag);
          const uint32_t jv = lookup_entry<K>(jn, mag);
          const bool in = uint32_t(lane) >= start && uint32_t(lane) < nbr;
          const uint32_t fail = __ballot_sync(0xffffffffu, in && !mine && m.y > pv);
          const uint32_t f = fail ? uint32_t(__ffs(fail) - 1) : nbr;  // first failing record
          const uint32_t popped = __ballot_sync(0xffffffffu, in && uint32_t(lane) < f && joinable);
          // of the popped releases, join only those not dominated, and per agent only
          // the latest (records of one agent are in acquire order)
          const bool cand = ((popped >> lane) & 1u) && m.w > jv;
          const uint32_t same = __match_any_sync(0xffffffffu, cand ? mag : 0xFFFFFFFFu);
          const uint32_t wave = __ballot_sync(0xffffffffu, cand && (same >> lane) <= 1u);
          visits += __popc(__ballot_sync(0xffffffffu, in && uint32_t(lane) <= f && !mine));
          uint32_t wm = wave;
          if (wave) {  // record the joined releases' epochs: distinct agents scatter, owners fold
            if ((wave >> lane) & 1u) jn_tmp[mag] = m.w;
            __syncwarp();
#pragma unroll
            for (int j = 0; j < K; ++j) jn[j] = max(jn[j], jn_tmp[lane * K + j]);
            __syncwarp();
          }
          if (spec_live && (wm & 1u)) {  // record lo + cur: its row is already loaded
            if (!row_complete<K>(spec)) wait_row<K>(a.hsnap + size_t(lo + cur) * Wc, spec, abort, a.st);
#pragma unroll
            for (int j = 0; j < K; ++j) P[j] = max(P[j], spec[j]);
            ++joins;
            wm &= ~1u;
          }
          spec_live = false;
          while (wm) {
            uint32_t ids[4];
            int n = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              ids[q] = 0;
              if (wm) {
                ids[q] = lo + cur + (__ffs(wm) - 1);
                wm &= wm - 1;
                ++n;
              }
            }
            join_rows<K, 4>(P, a.hsnap, ids, n, Wc, abort, a.st);
            joins += n;
          }
          if (f == nbr) {
            start = nbr;
          } else if (wave) {
            start = f;  // P grew: test the failing record again
          } else {
            stop = true;  // P unchanged: the record stays unordered
            start = f;
            break;
          }
        }
        cur += start;
      }
      if (lane == 0) __stcg(cursor_row + L, cur);
      // later releases of L, in this batch and the next, start from the new cursor
      if (lane > int(i) && (ea.x & 0xFF) == P_REL && ea.w == L) pre = cur;
      if ((ea2.x & 0xFF) == P_REL && ea2.w == L) pre2 = cur;
      store_row<K>(a.psnap + size_t(c) * Wc, P);
      store_row<K>(a.hsnap + size_t(c) * Wc, H);
      set_entry<K>(H, u, N + 1);  // H_t[t]++ (H_t[t] = N_t)
      ++N;
    } else {
      // sync (Algorithm 1): join C_t and H_t over the barrier's scope
      const uint32_t mode = __shfl_sync(0xffffffffu, eb.x, i);
      // under forced compression at barriers the agent enters the join with the highest
      // N among the members (otherwise the plan holds N_t itself)
      if (a.forced) {
        const uint32_t Nb = __shfl_sync(0xffffffffu, eb.y, i);
        if (Nb != N) {
          N = Nb;
          set_entry<K>(H, u, N);
        }
      }
      uint32_t C[K];
#pragma unroll
      for (int j = 0; j < K; ++j) C[j] = P[j];
      set_entry<K>(C, u, N);
      if (mode == BAR_SINGLE) {
#pragma unroll
        for (int j = 0; j < K; ++j) P[j] = C[j];
      } else if (mode == BAR_CTA) {
        uint32_t* buf = xchg + size_t(nbar & 1) * nwarps * 2 * Wc;
        store_row_shared<K>(buf + size_t(warp) * 2 * Wc, C);
        store_row_shared<K>(buf + size_t(warp) * 2 * Wc + Wc, H);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) P[j] = H[j] = 0;
        for (int wv = 0; wv < nwarps; ++wv) {
          const uint32_t* srcp = buf + size_t(wv) * 2 * Wc + lane * K;
#pragma unroll
          for (int j = 0; j < K; ++j) {
            P[j] = max(P[j], srcp[j]);
            H[j] = max(H[j], srcp[Wc + j]);
          }
        }
        joins += 2;  // this member's C_t and H_t joined into the block's
        ++nbar;
      } else {
        const uint32_t bid = z, count = w;
        uint32_t* J = a.bar_j + size_t(bid) * 2 * Wc;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          atomicMax(J + lane * K + j, C[j]);
          atomicMax(J + Wc + lane * K + j, H[j]);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.bar_cnt + bid, 1u);
        if (!abort) {
          bool ok = true;
          if (lane == 0) {
            uint32_t it = 0;
            while (ld_acquire(a.bar_cnt + bid) < count) {
              if (++it > kSpinLimit) {
                ok = false;
                break;
              }
              __nanosleep(64);
            }
            if (!ok) atomicCAS(&a.st->code, 0, GWCP_ERR_TIMEOUT);
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          __syncwarp();
          if (!ok) abort = true;
        }
        load_row<K>(J, P);
        load_row<K>(J + Wc, H);
        joins += 2;
      }
      set_entry<K>(H, u, N + 1);
      ++N;
    }
    put_version(row);
    if (i == 31) {  // next batch
      base += 32;
      ea = ea2;
      eb = eb2;
      pre = pre2;
      load_batch(base + 32, ea2, eb2, pre2);
    }
  }
  if constexpr (R > 0) cp_async_wait<0>();
  if (lane == 0) {
    atomicAdd(&a.st->joins, (unsigned long long)joins);
    atomicAdd(&a.st->loop_visits, (unsigned long long)visits);
    if constexpr (CV) atomicAdd(a.cv_words, cvs.words);
  }
}

// ---- plan construction -------------------------------------------------------------


// section record as the release loop reads it: (agent | scope id << 16, acquire epoch,
// release index, release epoch)
__global__ void k_recmeta(uint32_t n_cs, const uint32_t* cs_agent, const uint32_t* cs_epoch,
                          const uint32_t* cs_rel_idx, const uint32_t* cs_sid, const uint32_t* cs_rel_epoch,
                          uint4* recmeta) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cs) recmeta[c] = make_uint4(cs_agent[c] | (cs_sid[c] << 16), cs_epoch[c], cs_rel_idx[c], cs_rel_epoch[c]);
}

// (both flattening kernels stand down after an error: the per-record lists are then
// incomplete)
__global__ void k_flatcount(uint32_t n_incs, const uint32_t* exp_off, const uint32_t* ex_dep_cnt, uint32_t* cnt,
                            const DevStatus* st) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_incs) return;
  if (st->code) {
    cnt[r] = 0;
    return;
  }
  uint32_t t = 0;
  for (uint32_t e = exp_off[r]; e < exp_off[r + 1]; ++e) t += ex_dep_cnt[e];
  cnt[r] = t;
}

__global__ void k_flatfill(uint32_t n_incs, const uint32_t* exp_off, const uint32_t* ex_dep_off,
                           const uint32_t* ex_dep_cnt, const uint32_t* pool, const uint32_t* flat_off,
                           uint32_t* flat, const DevStatus* st) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_incs || st->code) return;
  uint32_t o = flat_off[r];
  for (uint32_t e = exp_off[r]; e < exp_off[r + 1]; ++e)
    for (uint32_t q = 0; q < ex_dep_cnt[e]; ++q) flat[o++] = pool[ex_dep_off[e] + q];
}

__global__ void k_plan_sync(PropArgs a, const uint32_t* sy_kind_, const uint32_t* sy_ver, const uint32_t* sy_match,
                            uint32_t n_sync) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sync) return;
  const Geo& g = a.g;
  const uint32_t u = a.sy_agent[k];
  const uint32_t row = a.rowbase[u] + sy_ver[k];
  const uint32_t kind = sy_kind_[k];
  uint4 ea, eb = make_uint4(0, 0, 0, 0);
  if (kind == K_ACQ) {
    const uint32_t c = a.cs_of_sync[k];
    const uint32_t off = a.acq_dep_off[c], cnt = a.acq_dep_cnt[c];
    ea = make_uint4(P_ACQ, row, off, cnt);
    if (cnt <= 4)  // up to four dependency ids ride in the entry itself
      eb = make_uint4(cnt > 0 ? a.pool[off] : 0, cnt > 1 ? a.pool[off + 1] : 0, cnt > 2 ? a.pool[off + 2] : 0,
                      cnt > 3 ? a.pool[off + 3] : 0);
  } else if (kind == K_REL) {
    const uint32_t c = a.cs_of_sync[k];
    const uint32_t L = a.cs_lock[c];
    ea = make_uint4(P_REL, row, c, L);
    eb = make_uint4(a.lock_cs_lo[L], a.lock_cs_lo[L + 1], a.cs_sid[c], a.sy_idx[k]);
  } else {
    const Event e = a.ev[a.sy_idx[k]];
    const BarMembers bm = barrier_members(e, g);
    const uint32_t mode = bm.count == 1 ? BAR_SINGLE
                          : (a.cta_barriers && e.scope == GWCP_SCOPE_CTA) ? BAR_CTA
                                                                          : BAR_GLOBAL;
    ea = make_uint4(P_BAR, row, a.sy_aux[k], bm.count);
    eb.x = mode;
    eb.y = a.sy_N[k] - 1;  // N_t entering the join (after the barrier, N_t = eb.y + 1)
  }
  (void)sy_match;
  const size_t p = size_t(k) + a.incs_off[k];
  a.plan[2 * p] = ea;
  a.plan[2 * p + 1] = eb;
}

__global__ void k_plan_incs(PropArgs a, const uint32_t* incs_k, const uint32_t* incs_ver, const uint32_t* flat_off,
                            uint32_t n_incs) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_incs) return;
  const uint32_t k = incs_k[r];
  const uint32_t u = a.sy_agent[k];
  const size_t p = size_t(k) + 1 + r;
  const uint32_t off = flat_off[r], cnt = flat_off[r + 1] - off;
  a.plan[2 * p] = make_uint4(P_INCS, a.rowbase[u] + incs_ver[r], off, cnt);
  a.plan[2 * p + 1] = cnt <= 4 ? make_uint4(cnt > 0 ? a.flat[off] : 0, cnt > 1 ? a.flat[off + 1] : 0,
                                            cnt > 2 ? a.flat[off + 2] : 0, cnt > 3 ? a.flat[off + 3] : 0)
                               : make_uint4(0, 0, 0, 0);
}

template <int K, int R, int MAXT, bool CV = false>
int launch(const PropArgs& a, uint32_t grid, uint32_t threads, size_t smem_xchg, cudaStream_t s) {
  auto kern = k_propagate<K, R, MAXT, CV>;
  const size_t smem = smem_xchg + (R > 0 ? size_t(threads / 32) * R * slot_words<K>() * 4 : 0) +
                     size_t(threads / 32) * 32 * K * 4;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)))
    return GWCP_ERR_UNSUPPORTED;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, int(threads), smem) != cudaSuccess)
    return GWCP_ERR_CUDA;
  if (uint64_t(per_sm) * sms < grid) return GWCP_ERR_UNSUPPORTED;  // walkers must be co-resident
  PropArgs copy = a;
  void* args[] = {&copy};
  if (cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(grid), dim3(threads), args, smem, s) !=
      cudaSuccess)
    return GWCP_ERR_CUDA;
  count_launch();
  return GWCP_OK;
}

// ring depth: deepest that keeps a CTA's shared memory within budget
template <int K>
int launch_k(const PropArgs& a, uint32_t grid, uint32_t threads, size_t smem_xchg, cudaStream_t s) {
  const size_t per_slot = size_t(threads / 32) * slot_words<K>() * 4;
  const size_t kBudget = 160 * 1024 - size_t(threads / 32) * 32 * K * 4;
  // compressed versions: the same shapes, instantiated with the compressing store
  if constexpr (K <= 4) {
    if (threads <= 256 && smem_xchg + 8 * per_slot <= kBudget)
      return a.compress ? launch<K, 8, 256, true>(a, grid, threads, smem_xchg, s)
                        : launch<K, 8, 256>(a, grid, threads, smem_xchg, s);
    if (smem_xchg + 2 * per_slot <= kBudget)
      return a.compress ? launch<K, 2, 1024, true>(a, grid, threads, smem_xchg, s)
                        : launch<K, 2, 1024>(a, grid, threads, smem_xchg, s);
  }
  return a.compress ? launch<K, 0, 1024, true>(a, grid, threads, smem_xchg, s)
                    : launch<K, 0, 1024>(a, grid, threads, smem_xchg, s);
}

// failure-detection test: one warp waits, with the walkers' bounded wait, on a clock row
// that nothing completes
__global__ void k_wait_probe(const uint32_t* row, DevStatus* st, uint32_t limit) {
  uint32_t y[1];
  bool abort = false;
  wait_row<1>(row, y, abort, st, limit);
}

}  // namespace

int wait_probe(uint32_t limit, int* code) {
  // a 32-word row of SENTINEL words (never completed) and a status record
  void* mem = nullptr;
  if (cudaMalloc(&mem, 256 + sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return GWCP_ERR_OOM;
  }
  auto* row = static_cast<uint32_t*>(mem);
  auto* st = reinterpret_cast<DevStatus*>(static_cast<char*>(mem) + 256);
  cudaMemset(row, 0xFF, 256);
  cudaMemset(st, 0, sizeof(DevStatus));
  k_wait_probe<<<1, 32>>>(row, st, limit);
  count_launch();
  int rc = cudaDeviceSynchronize() == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
  if (!rc && cudaMemcpy(code, &st->code, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = GWCP_ERR_CUDA;
  cudaFree(mem);
  return rc;
}

int phaseG_propagate(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  PropArgs a{};
  a.g = g;
  a.ev = b.ev;
  a.st = b.st;
  a.sy_start = b.sy_start;
  a.sy_idx = b.sy_idx;
  a.sy_kind = b.sy_kind;
  a.sy_N = b.sy_N;
  a.sy_ver = b.sy_ver;
  a.sy_aux = b.sy_aux;
  a.sy_agent = b.sy_agent;
  a.incs_off = b.incs_cnt;
  a.incs_ver = b.incs_ver;
  a.incs_k = b.incs_k;
  a.exp_off = b.exp_off;
  a.ex_dep_off = b.ex_dep_off;
  a.ex_dep_cnt = b.ex_dep_cnt;
  a.rowbase = b.vcount;
  a.cs_of_sync = b.cs_of_sync;
  a.cs_agent = b.cs_agent;
  a.cs_sid = b.cs_sid;
  a.cs_epoch = b.cs_epoch;
  a.cs_rel_idx = b.cs_rel_idx;
  a.cs_lock = b.cs_lock;
  a.cs_rel_epoch = b.cs_rel_epoch;
  a.lock_cs_lo = b.lock_cs_lo;
  a.acq_dep_off = b.acq_dep_off;
  a.acq_dep_cnt = b.acq_dep_cnt;
  a.pool = b.dep_pool;
  a.rows = b.rows;
  a.psnap = b.psnap;
  a.hsnap = b.hsnap;
  a.done = b.done;
  a.cursor = b.cursor;
  a.bar_j = b.bar_j;
  a.bar_cnt = b.bar_cnt;
  a.n_locks = z.n_locks;
  a.cta_barriers = z.cta_barriers;
  a.flat = b.flat;
  a.plan = b.plan;
  a.recmeta = b.recmeta;
  a.hb_only = z.hb_only;
  a.forced = z.forced_barrier;
  a.compress = z.compress;
  a.cv_pool = b.cv_pool;
  a.cv_cap = z.cv_cap;
  a.cv_used = reinterpret_cast<unsigned long long*>(&b.st->spare[3]);
  a.cv_words = reinterpret_cast<unsigned long long*>(&b.st->spare[4]);
  // plan: per-agent stream of clock-changing steps with their static data resolved
  p.begin("g_plan", double(z.n_sync + z.n_incs) * 64 + double(z.n_cs) * 2 * g.RW * 4);
  if (z.n_cs) {
    k_recmeta<<<(z.n_cs + 255) / 256, 256, 0, s>>>(z.n_cs, b.cs_agent, b.cs_epoch, b.cs_rel_idx, b.cs_sid,
                                                    b.cs_rel_epoch, b.recmeta);
    count_launch();
    // snapshot rows start as SENTINEL: a reader accepts a row once none is left
    cudaMemsetAsync(b.psnap, 0xFF, size_t(z.n_cs) * g.RW * 4, s);
    cudaMemsetAsync(b.hsnap, 0xFF, size_t(z.n_cs) * g.RW * 4, s);
    if (g.nT) cudaMemsetAsync(b.jsnap, 0xFF, size_t(z.n_cs) * g.RW * 4, s);
  }
  if (z.n_incs) {
    k_flatcount<<<(z.n_incs + 255) / 256, 256, 0, s>>>(z.n_incs, b.exp_off, b.ex_dep_cnt, b.flat_off, b.st);
    count_launch();
    scan_exclusive(b.flat_off, b.flat_off, size_t(z.n_incs) + 1, nullptr, b.scan_tmp, s);
    k_flatfill<<<(z.n_incs + 255) / 256, 256, 0, s>>>(z.n_incs, b.exp_off, b.ex_dep_off, b.ex_dep_cnt, b.dep_pool,
                                                       b.flat_off, b.flat, b.st);
    count_launch();
    k_plan_incs<<<(z.n_incs + 255) / 256, 256, 0, s>>>(a, b.incs_k, b.incs_ver, b.flat_off, z.n_incs);
    count_launch();
  }
  if (z.n_sync) {
    k_plan_sync<<<(z.n_sync + 255) / 256, 256, 0, s>>>(a, b.sy_kind, b.sy_ver, b.sy_match, z.n_sync);
    count_launch();
  }
  p.end();
  if (g.nT) {
    // tile tables: each clock version and snapshot is a table (new tiles counted apart)
    p.begin("g_propagate", double(z.n_rows) * g.RW * 4 + double(z.n_cs) * 2 * g.RW * 4);
    const int rc = phaseG_wide(b, g, z, s);
    p.end();
    return rc;
  }
  uint32_t grid, threads;
  size_t smem = 0;
  if (z.cta_barriers) {
    grid = g.B;
    threads = g.apb * 32;
    smem = size_t(2) * g.apb * 2 * g.Wp * 4;
  } else {
    grid = (g.W + 31) / 32;
    threads = 1024;
  }
  // algorithmic bytes: each clock version written once, each join reads a row
  p.begin("g_propagate", double(z.n_rows) * g.Wp * 4 + double(z.n_cs) * 2 * g.Wp * 4);
  int rc;
  switch (g.K) {
    case 1: rc = launch_k<1>(a, grid, threads, smem, s); break;
    case 2: rc = launch_k<2>(a, grid, threads, smem, s); break;
    case 4: rc = launch_k<4>(a, grid, threads, smem, s); break;
    case 8: rc = launch_k<8>(a, grid, threads, smem, s); break;
    case 16: rc = launch_k<16>(a, grid, threads, smem, s); break;
    case 32: rc = launch_k<32>(a, grid, threads, smem, s); break;
    default: rc = GWCP_ERR_UNSUPPORTED;
  }
  p.end();
  return rc;
}

}  // namespace gwcp
