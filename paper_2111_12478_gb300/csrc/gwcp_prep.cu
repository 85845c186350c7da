// Preprocessing of libgwcp: everything the clock propagation and the race check need
// that does not depend on clock values.
//
//   A  decode + validate (W1), stable counting sort of events by agent (barriers are
//      expanded to one entry per member), trace-order compaction of accesses,
//      acquire/release events and barriers.
//   B  compaction of each agent's synchronisation entries (ACQ, REL, barrier).
//   C  per-agent walk over those entries (one warp per agent, warp scans): local time
//      N_t (incremented at each release and barrier, Algorithm 1), lock depth, matching
//      of releases to acquires (W2), innermost held section, clock-version numbering.
//   D  per-access epoch N(e), clock-version row, and the list of in-section accesses
//      (accesses made while the lockset is not empty, Algorithm 2).
//   E  per-lock walk in trace order: the acquire's joins (the latest release on every
//      overlapping scope of the lock, Algorithm 1 acquire), W3, the per-lock list of
//      critical-section records used by the release loop.
//   F  per (lock, location) walk: for every in-section access and held lock, the
//      releases whose L^r / L^w contribution it joins (Algorithm 2).
#include "gwcp_internal.cuh"

namespace gwcp {

namespace {

constexpr int A_WARPS = 4;  // warps per CTA of phase A while their histograms fit 48 KB

__device__ bool validate_w1(const Event& e, const Geo& g) {
  if (e.agent >= g.W || e.op > GWCP_FENCE || e.scope > GWCP_SCOPE_WARP || e.space > GWCP_SPACE_SHARED) return false;
  if (e.scope == GWCP_SCOPE_WARP && e.op != GWCP_BARRIER) return false;
  if (e.space == GWCP_SPACE_SHARED && e.op > GWCP_ATOMIC) return false;
  if (e.op <= GWCP_ATOMIC) {
    if (e.space == GWCP_SPACE_SHARED && e.addr >= (1ull << 40)) return false;
    if (e.space == GWCP_SPACE_GLOBAL && e.addr >= (1ull << 63)) return false;
  }
  if (e.op == GWCP_BARRIER) return barrier_members(e, g).ok;
  return true;
}

__device__ __forceinline__ uint32_t member_at(const BarMembers& m, uint32_t j) {
  if (!m.mask) return m.first + j;
  uint32_t mask = m.mask;
  for (uint32_t q = 0; q < j; ++q) mask &= mask - 1;  // drop the j lowest lanes
  return m.first + (__ffs(mask) - 1);
}

__device__ __forceinline__ uint32_t entry_kind(uint8_t op) {
  return op <= GWCP_ATOMIC ? K_ACCESS : op == GWCP_ACQ ? K_ACQ : op == GWCP_REL ? K_REL : K_BAR;
}

// Phase A walks each tile with one warp, 32 events a round; with many agents few warps fit
// an SM (each holds a per-agent count table in shared memory), so each lane loads the
// events of kAhead rounds before it processes them (4: without spills at four blocks per
// SM in the passes for many agents; 8 measured 0.85 ms slower per 200M events).
constexpr int kAhead = 4;

// event i; vec: the array is 16-byte aligned (one 128-bit load)
__device__ __forceinline__ Event load_event(const Event* ev, uint64_t i, bool vec) {
  if (!vec) return ev[i];
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(ev) + i);
  Event e;
  e.agent = v.x;
  e.op = uint8_t(v.y);
  e.scope = uint8_t(v.y >> 8);
  e.space = uint8_t(v.y >> 16);
  e.flags = uint8_t(v.y >> 24);
  e.addr = uint64_t(v.z) | (uint64_t(v.w) << 32);
  return e;
}

// Phase A, pass 1: per (agent, tile) entry counts and per-tile compaction counts.
__global__ void k_a_count(const Event* ev, uint64_t N, Geo g, uint32_t TA, uint32_t ntA, uint32_t* hist,
                          uint32_t* tile_cnt, DevStatus* st, bool vec) {
  extern __shared__ uint32_t sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + warp;
  uint32_t* cnt = sm + warp * g.Wp;
  for (uint32_t u = lane; u < g.Wp; u += 32) cnt[u] = 0;
  __syncwarp();
  if (tile >= ntA) return;
  const uint64_t lo = uint64_t(tile) * TA, hi = (lo + TA < N ? lo + TA : N);
  uint32_t n_acc = 0, n_ar = 0, n_bar = 0;
  uint64_t kor = 0, kand = ~0ull, lor = 0, land = ~0ull;
  for (uint64_t base0 = lo; base0 < hi; base0 += 32 * kAhead) {
    Event eb[kAhead];
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t i = base0 + r * 32 + lane;
      eb[r] = i < hi ? load_event(ev, i, vec) : Event{};
    }
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t base = base0 + r * 32;
      if (base >= hi) break;
      const uint64_t i = base + lane;
      const bool valid = i < hi;
      const Event e = eb[r];
      bool ok = !valid || validate_w1(e, g);
      if (!ok) set_error(st, GWCP_ERR_INVALID_TRACE, i);
      const bool acc = valid && ok && e.op <= GWCP_ATOMIC;
      const bool ar = valid && ok && (e.op == GWCP_ACQ || e.op == GWCP_REL);
      const bool bar = valid && ok && e.op == GWCP_BARRIER;
      if (acc || ar) atomicAdd(&cnt[e.agent], 1u);
      if (acc) {
        uint64_t k = location_key(e, g.apb);
        kor |= k;
        kand &= k;
      }
      if (ar) {
        lor |= e.addr;
        land &= e.addr;
      }
      if (bar) {
        BarMembers m = barrier_members(e, g);
        for (uint32_t j = 0; j < m.count; ++j) atomicAdd(&cnt[member_at(m, j)], 1u);
      }
      n_acc += __popc(__ballot_sync(0xffffffffu, acc));
      n_ar += __popc(__ballot_sync(0xffffffffu, ar));
      n_bar += __popc(__ballot_sync(0xffffffffu, bar));
    }
  }
  __syncwarp();
  for (uint32_t u = lane; u < g.W; u += 32) hist[size_t(u) * ntA + tile] = cnt[u];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kor |= __shfl_xor_sync(0xffffffffu, kor, o);
    kand &= __shfl_xor_sync(0xffffffffu, kand, o);
    lor |= __shfl_xor_sync(0xffffffffu, lor, o);
    land &= __shfl_xor_sync(0xffffffffu, land, o);
  }
  if (lane == 0) {
    tile_cnt[tile] = n_acc;
    tile_cnt[ntA + 1 + tile] = n_ar;
    tile_cnt[2 * (ntA + 1) + tile] = n_bar;
    if (n_acc) {
      atomicOr(&st->key_or, kor);
      atomicAnd(&st->key_and, kand);
    }
    if (n_ar) {
      atomicOr(&st->lock_or, lor);
      atomicAnd(&st->lock_and, land);
    }
  }
}

// Trace-order compactions of one round of 32 events (lane order is trace order): access
// keys and indices (with the written-location bitmap of the grouped order), acquire/release
// and barrier indices. Returns the barrier ballot of the round.
struct ACompact {
  uint64_t* acc_key;
  uint32_t* acc_idx;
  uint32_t* acqrel;
  uint32_t* bar;
  uint32_t comp_lo, comp_span;  // composite access keys when comp_span > 0
  uint32_t* wl_bits;
  uint32_t wl_log2;
};

__device__ __forceinline__ uint32_t a_compact(const ACompact& c, const Event& e, uint64_t i, bool acc, bool ar,
                                              bool isbar, const Geo& g, uint32_t lt, uint32_t& o_acc,
                                              uint32_t& o_ar, uint32_t& o_bar) {
  uint32_t m = __ballot_sync(0xffffffffu, acc);
  if (acc) {
    const uint32_t p = o_acc + __popc(m & lt);
    const uint64_t loc = location_key(e, g.apb);
    const uint32_t cls = access_class(e);
    const uint64_t key = c.comp_span ? composite_key(loc, cls, e.agent, c.comp_lo, c.comp_span) : loc;
    c.acc_key[p] = key;
    c.acc_idx[p] = uint32_t(i);
    if (c.wl_log2 && cls != C_READ) {  // a write-class access marks its location
      const uint32_t h = wl_bit(key >> 15, c.wl_log2);
      atomicOr(c.wl_bits + (h >> 5), 1u << (h & 31));
    }
  }
  o_acc += __popc(m);
  m = __ballot_sync(0xffffffffu, ar);
  if (ar) c.acqrel[o_ar + __popc(m & lt)] = uint32_t(i);
  o_ar += __popc(m);
  m = __ballot_sync(0xffffffffu, isbar);
  if (isbar) c.bar[o_bar + __popc(m & lt)] = uint32_t(i);
  o_bar += __popc(m);
  return m;
}

// Phase A, pass 2: stable scatter into the agent-sorted stream S and the trace-order
// compactions. Chunks with a barrier are processed one event at a time.
__global__ void k_a_scatter(const Event* ev, uint64_t N, Geo g, uint32_t TA, uint32_t ntA, const uint32_t* hist,
                            const uint32_t* tile_off, uint32_t* S, ACompact cpt, bool vec) {
  extern __shared__ uint32_t sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + warp;
  if (tile >= ntA) return;
  uint32_t* cnt = sm + warp * g.Wp;
  for (uint32_t u = lane; u < g.W; u += 32) cnt[u] = hist[size_t(u) * ntA + tile];
  __syncwarp();
  uint32_t o_acc = tile_off[tile], o_ar = tile_off[ntA + 1 + tile], o_bar = tile_off[2 * (ntA + 1) + tile];
  const uint32_t lt = lanemask_lt();
  const uint64_t lo = uint64_t(tile) * TA, hi = (lo + TA < N ? lo + TA : N);
  for (uint64_t base0 = lo; base0 < hi; base0 += 32 * kAhead) {
    Event eb[kAhead];
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t i = base0 + r * 32 + lane;
      eb[r] = i < hi ? load_event(ev, i, vec) : Event{};
    }
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t base = base0 + r * 32;
      if (base >= hi) break;
      const uint64_t i = base + lane;
      const bool valid = i < hi;
      const Event e = eb[r];
      // events that break W1 are left out, as in the counting pass
      const bool ok = valid && validate_w1(e, g);
      const bool acc = ok && e.op <= GWCP_ATOMIC;
      const bool ar = ok && (e.op == GWCP_ACQ || e.op == GWCP_REL);
      const bool isbar = ok && e.op == GWCP_BARRIER;
      const uint32_t kind = entry_kind(e.op);
      const uint32_t m = a_compact(cpt, e, i, acc, ar, isbar, g, lt, o_acc, o_ar, o_bar);
      // agent-sorted stream
      if (!m) {
        const bool in_s = acc || ar;
        const uint32_t key = in_s ? e.agent : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const uint32_t b0 = in_s ? cnt[e.agent] : 0;
        __syncwarp();
        if (in_s) {
          S[b0 + __popc(peers & lt)] = (kind << 30) | uint32_t(i);
          if (lane == __ffs(peers) - 1) cnt[e.agent] = b0 + __popc(peers);
        }
        __syncwarp();
      } else {
        for (int L = 0; L < 32; ++L) {
          const uint32_t eop = __shfl_sync(0xffffffffu, uint32_t(e.op), L);
          const uint32_t eagent = __shfl_sync(0xffffffffu, e.agent, L);
          const uint32_t escope = __shfl_sync(0xffffffffu, uint32_t(e.scope), L);
          const uint64_t eaddr = __shfl_sync(0xffffffffu, e.addr, L);
          const bool ev_valid = __shfl_sync(0xffffffffu, valid, L);
          const bool ev_ok = __shfl_sync(0xffffffffu, ok, L);
          if (!ev_valid) break;
          const uint32_t idx = uint32_t(base) + L;
          if (!ev_ok) continue;
          if (eop <= GWCP_REL) {
            if (lane == 0) S[cnt[eagent]++] = (entry_kind(uint8_t(eop)) << 30) | idx;
          } else if (eop == GWCP_BARRIER) {
            Event be{};
            be.agent = eagent;
            be.op = GWCP_BARRIER;
            be.scope = uint8_t(escope);
            be.addr = eaddr;
            BarMembers bm = barrier_members(be, g);
            for (uint32_t j = lane; j < bm.count; j += 32) {
              uint32_t mb = member_at(bm, j);
              S[cnt[mb]++] = (K_BAR << 30) | idx;
            }
          }
          __syncwarp();
        }
      }
    }
  }
}

// ---- Phase A with many agents: S from a stable sort on the agent ---------------------
// Pass 1, one warp per tile of TA events: per-tile counts of accesses, acquires/releases,
// barriers and S entries (an access or acquire/release is one entry of its agent, a
// barrier one entry per member), W1 and the key / lock bit summaries. Both passes run four
// 256-thread blocks per SM (64 registers; 80 allowed three): 0.9 ms faster per 200M events.
__global__ void __launch_bounds__(256, 4) k_aw_count(const Event* ev, uint64_t N, Geo g, uint32_t TA, uint32_t ntA, uint32_t* tile_cnt,
                           DevStatus* st, bool vec) {
  const int lane = threadIdx.x & 31;
  const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tile >= ntA) return;
  const uint64_t lo = uint64_t(tile) * TA, hi = (lo + TA < N ? lo + TA : N);
  uint32_t n_acc = 0, n_ar = 0, n_bar = 0, n_s = 0;
  uint64_t kor = 0, kand = ~0ull, lor = 0, land = ~0ull;
  for (uint64_t base0 = lo; base0 < hi; base0 += 32 * kAhead) {
    Event eb[kAhead];
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t i = base0 + r * 32 + lane;
      eb[r] = i < hi ? load_event(ev, i, vec) : Event{};
    }
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      if (base0 + r * 32 >= hi) break;
      const uint64_t i = base0 + r * 32 + lane;
      const bool valid = i < hi;
      const Event e = eb[r];
      const bool ok = !valid || validate_w1(e, g);
      if (!ok) set_error(st, GWCP_ERR_INVALID_TRACE, i);
      const bool acc = valid && ok && e.op <= GWCP_ATOMIC;
      const bool ar = valid && ok && (e.op == GWCP_ACQ || e.op == GWCP_REL);
      const bool bar = valid && ok && e.op == GWCP_BARRIER;
      const uint32_t ns = bar ? barrier_members(e, g).count : (acc || ar) ? 1u : 0u;
      if (acc) {
        const uint64_t k = location_key(e, g.apb);
        kor |= k;
        kand &= k;
      }
      if (ar) {
        lor |= e.addr;
        land &= e.addr;
      }
      n_acc += __popc(__ballot_sync(0xffffffffu, acc));
      n_ar += __popc(__ballot_sync(0xffffffffu, ar));
      n_bar += __popc(__ballot_sync(0xffffffffu, bar));
      n_s += __reduce_add_sync(0xffffffffu, ns);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kor |= __shfl_xor_sync(0xffffffffu, kor, o);
    kand &= __shfl_xor_sync(0xffffffffu, kand, o);
    lor |= __shfl_xor_sync(0xffffffffu, lor, o);
    land &= __shfl_xor_sync(0xffffffffu, land, o);
  }
  if (lane == 0) {
    tile_cnt[tile] = n_acc;
    tile_cnt[ntA + 1 + tile] = n_ar;
    tile_cnt[2 * (ntA + 1) + tile] = n_bar;
    tile_cnt[3 * (ntA + 1) + tile] = n_s;
    if (n_acc) {
      atomicOr(&st->key_or, kor);
      atomicAnd(&st->key_and, kand);
    }
    if (n_ar) {
      atomicOr(&st->lock_or, lor);
      atomicAnd(&st->lock_and, land);
    }
  }
}

// Pass 2: the trace-order compactions and the S keys (agent << 32 | S entry) in trace
// order, barrier members at the barrier's place; a stable sort on the agent bits then
// gives S (each agent's entries in trace order).
__global__ void __launch_bounds__(256, 4) k_aw_scatter(const Event* ev, uint64_t N, Geo g, uint32_t TA, uint32_t ntA, const uint32_t* tile_off,
                             uint64_t* skey, ACompact cpt, bool vec) {
  const int lane = threadIdx.x & 31;
  const uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tile >= ntA) return;
  uint32_t o_acc = tile_off[tile], o_ar = tile_off[ntA + 1 + tile], o_bar = tile_off[2 * (ntA + 1) + tile];
  uint32_t o_s = tile_off[3 * (ntA + 1) + tile];
  const uint32_t lt = lanemask_lt();
  const uint64_t lo = uint64_t(tile) * TA, hi = (lo + TA < N ? lo + TA : N);
  for (uint64_t base0 = lo; base0 < hi; base0 += 32 * kAhead) {
    Event eb[kAhead];
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      const uint64_t i = base0 + r * 32 + lane;
      eb[r] = i < hi ? load_event(ev, i, vec) : Event{};
    }
#pragma unroll
    for (int r = 0; r < kAhead; ++r) {
      if (base0 + r * 32 >= hi) break;
      const uint64_t i = base0 + r * 32 + lane;
      const Event e = eb[r];
      // events that break W1 are left out, as in the counting pass
      const bool ok = i < hi && validate_w1(e, g);
      const bool acc = ok && e.op <= GWCP_ATOMIC;
      const bool ar = ok && (e.op == GWCP_ACQ || e.op == GWCP_REL);
      const bool isbar = ok && e.op == GWCP_BARRIER;
      a_compact(cpt, e, i, acc, ar, isbar, g, lt, o_acc, o_ar, o_bar);
      BarMembers bm{0, 0, 0, false};
      uint32_t ns = (acc || ar) ? 1u : 0u;
      if (isbar) {
        bm = barrier_members(e, g);
        ns = bm.count;
      }
      const uint32_t incl = warp_inclusive_scan(ns);
      const uint32_t q = o_s + incl - ns;
      if (acc || ar) {
        skey[q] = (uint64_t(e.agent) << 32) | (entry_kind(e.op) << 30) | uint32_t(i);
      } else if (isbar) {
        for (uint32_t j = 0; j < bm.count; ++j)
          skey[q + j] = (uint64_t(member_at(bm, j)) << 32) | (K_BAR << 30) | uint32_t(i);
      }
      o_s += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

__global__ void k_aw_extract(const uint64_t* key, uint32_t n, uint32_t* S) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) S[p] = uint32_t(key[p]);
}

// seg[u]: the first S position of agent u (seg[W] = n)
__global__ void k_aw_seg(const uint64_t* key, uint32_t n, uint32_t W, uint32_t* seg) {
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > W) return;
  const uint64_t x = uint64_t(u) << 32;
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (key[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  seg[u] = lo;
}

__global__ void k_a_segments(const uint32_t* hist, uint32_t W, uint32_t ntA, uint32_t nS, uint32_t* seg) {
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < W) seg[u] = hist[size_t(u) * ntA];
  if (u == W) seg[W] = nS;
}

template <typename T>
__device__ __forceinline__ uint32_t lower_bound_dev(const T* a, uint32_t n, T x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Phase B: the synchronisation entries of S in S order. One warp per chunk of B_CHUNK
// consecutive S positions (its own offset from the counting pass, ballot ranks within a
// round of 32), so no warp waits for another.
constexpr int B_THREADS = 256, B_ROUNDS = 16, B_CHUNK = 32 * B_ROUNDS;

__global__ void k_b_count(const uint32_t* S, uint32_t nS, uint32_t n_chunks, uint32_t* cnt) {
  const uint32_t chunk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (chunk >= n_chunks) return;
  const uint32_t base = chunk * B_CHUNK;
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < B_ROUNDS; ++j) {
    const uint32_t p = base + j * 32 + lane;
    if (p < nS && s_kind(S[p]) != K_ACCESS) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) cnt[chunk] = c;
}

__global__ void k_b_scatter(const Event* ev, const uint32_t* S, uint32_t nS, uint32_t n_chunks, const uint32_t* off,
                            const uint32_t* bar, uint32_t n_bar, const uint32_t* acqrel, uint32_t n_acqrel,
                            uint32_t* sy_spos, uint32_t* sy_idx, uint32_t* sy_kind, uint32_t* sy_aux,
                            uint64_t* lk_key, uint32_t* lk_k) {
  const uint32_t chunk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (chunk >= n_chunks) return;
  const uint32_t base = chunk * B_CHUNK;
  uint32_t sv[B_ROUNDS];
#pragma unroll
  for (int j = 0; j < B_ROUNDS; ++j) {
    const uint32_t p = base + j * 32 + lane;
    sv[j] = p < nS ? S[p] : (K_ACCESS << 30);
  }
  uint32_t run = off[chunk];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < B_ROUNDS; ++j) {
    const uint32_t p = base + j * 32 + lane;
    const uint32_t s = sv[j];
    const bool sy = s_kind(s) != K_ACCESS;
    const uint32_t m = __ballot_sync(0xffffffffu, sy);
    if (sy) {
      const uint32_t k = run + __popc(m & lt);
      const uint32_t idx = s_idx(s), kind = s_kind(s);
      sy_spos[k] = p;
      sy_idx[k] = idx;
      sy_kind[k] = kind;
      sy_aux[k] = kind == K_BAR ? lower_bound_dev(bar, n_bar, idx) : NONE;
      if (kind != K_BAR) {
        uint32_t q = lower_bound_dev(acqrel, n_acqrel, idx);
        lk_key[q] = ev[idx].addr;
        lk_k[q] = k;
      }
    }
    run += __popc(m);
  }
}

__global__ void k_b_starts(const uint32_t* seg, uint32_t W, const uint32_t* sy_spos, uint32_t n_sync,
                           uint32_t* sy_start) {
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u <= W) sy_start[u] = lower_bound_dev(sy_spos, n_sync, seg[u]);
}

// Phase C: one warp per agent over its synchronisation entries.
__global__ void k_c_walk(const Event* ev, Geo g, const uint32_t* seg, const uint32_t* sy_start,
                         const uint32_t* sy_spos, const uint32_t* sy_idx, const uint32_t* sy_kind, uint32_t* sy_N,
                         uint32_t* sy_depth, uint32_t* sy_inner, uint32_t* sy_ver, uint32_t* sy_match,
                         uint32_t* sy_relk, uint32_t* incs_cnt, uint32_t* vcount, uint32_t* sy_agent,
                         DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= g.W) return;
  const uint32_t k0 = sy_start[u], k1 = sy_start[u + 1];
  int depth_c = 0;
  uint32_t N_c = 1, ver_c = 0;
  uint32_t prev_spos = seg[u] - 1;  // wraps for u's first entry at 0: only differences matter
  uint32_t stk[kMaxNest + 1];
  uint64_t stk_lock[kMaxNest + 1];
  uint32_t stk_sid[kMaxNest + 1];
#pragma unroll
  for (int d = 0; d <= kMaxNest; ++d) {
    stk[d] = NONE;
    stk_lock[d] = 0;
    stk_sid[d] = NONE;
  }
  const uint32_t lt = lanemask_lt(), le = lt | (1u << lane);
  for (uint32_t kb = k0; kb < k1; kb += 32) {
    const uint32_t k = kb + lane;
    const bool valid = k < k1;
    uint32_t kind = K_BAR, spos = 0, idx = 0;
    uint64_t lock = 0;
    uint32_t sid = NONE;
    if (valid) {
      kind = sy_kind[k];
      spos = sy_spos[k];
      idx = sy_idx[k];
      if (kind != K_BAR) {
        Event e = ev[idx];
        lock = e.addr;
        sid = scope_id(e.agent, e.scope, g.apb);
      }
    }
    const int delta = !valid ? 0 : kind == K_ACQ ? 1 : kind == K_REL ? -1 : 0;
    const int d_after = depth_c + warp_inclusive_scan(delta);
    const int d_before = d_after - delta;
    if (valid && kind == K_REL && d_before <= 0) set_error(st, GWCP_ERR_INVALID_TRACE, idx);
    if (valid && kind == K_ACQ && d_after > kMaxNest) set_error(st, GWCP_ERR_INVALID_TRACE, idx);
    const uint32_t N_after = N_c + warp_inclusive_scan(uint32_t(valid && kind != K_ACQ));
    uint32_t prev = __shfl_up_sync(0xffffffffu, spos, 1);
    if (lane == 0) prev = prev_spos;
    const uint32_t gap = spos - prev - 1;
    const uint32_t ic = (valid && d_before > 0) ? gap : 0;
    const uint32_t ver_after = ver_c + warp_inclusive_scan(valid ? ic + 1 : 0u);
    if (valid && k > k0) incs_cnt[k - 1] = ic;
    // expanded (access, held lock) records of the gap: ic accesses at depth d_before
    const uint32_t nexp = __reduce_add_sync(0xffffffffu, ic * uint32_t(max(d_before, 0)));
    if (lane == 0 && nexp) atomicAdd(&st->spare[1], (unsigned long long)nexp);
    // innermost acquire per level, matching, parents
    uint32_t inner = NONE, match = NONE;
    uint64_t mlock = 0;
    uint32_t msid = NONE;
    for (int d = 1; d <= kMaxNest; ++d) {
      const uint32_t md = __ballot_sync(0xffffffffu, valid && kind == K_ACQ && d_after == d);
      const uint32_t m_le = md & le, m_lt = md & lt;
      const int L_le = m_le ? 31 - __clz(m_le) : -1;
      const int L_lt = m_lt ? 31 - __clz(m_lt) : -1;
      const uint32_t k_le = __shfl_sync(0xffffffffu, k, L_le < 0 ? 0 : L_le);
      const uint32_t k_lt = __shfl_sync(0xffffffffu, k, L_lt < 0 ? 0 : L_lt);
      const uint64_t lock_lt = __shfl_sync(0xffffffffu, lock, L_lt < 0 ? 0 : L_lt);
      const uint32_t sid_lt = __shfl_sync(0xffffffffu, sid, L_lt < 0 ? 0 : L_lt);
      const uint32_t c_le = L_le >= 0 ? k_le : stk[d];
      const uint32_t c_lt = L_lt >= 0 ? k_lt : stk[d];
      if (d == d_after) inner = c_le;
      if (kind == K_REL && d == d_before) {
        match = c_lt;
        mlock = L_lt >= 0 ? lock_lt : stk_lock[d];
        msid = L_lt >= 0 ? sid_lt : stk_sid[d];
      }
      if (kind == K_ACQ && d == d_after - 1) match = c_lt;
      if (md) {
        const int L_hi = 31 - __clz(md);
        stk[d] = __shfl_sync(0xffffffffu, k, L_hi);
        stk_lock[d] = __shfl_sync(0xffffffffu, lock, L_hi);
        stk_sid[d] = __shfl_sync(0xffffffffu, sid, L_hi);
      }
    }
    if (valid) {
      if (kind == K_REL && d_before > 0 && (match == NONE || mlock != lock || msid != sid))
        set_error(st, GWCP_ERR_INVALID_TRACE, idx);
      sy_N[k] = N_after;
      sy_agent[k] = u;
      sy_depth[k] = uint32_t(max(d_after, 0));
      sy_inner[k] = d_after > 0 ? inner : NONE;
      sy_ver[k] = ver_after;
      sy_match[k] = match;
      if (kind == K_REL && match != NONE) sy_relk[match] = k;
    }
    const int last = (k1 - kb) >= 32 ? 31 : int(k1 - kb) - 1;
    depth_c = __shfl_sync(0xffffffffu, d_after, last);
    N_c = __shfl_sync(0xffffffffu, N_after, last);
    ver_c = __shfl_sync(0xffffffffu, ver_after, last);
    prev_spos = __shfl_sync(0xffffffffu, spos, last);
  }
  if (lane == 0) {
    uint32_t tail_ic = 0;
    if (k1 > k0) {
      tail_ic = depth_c > 0 ? seg[u + 1] - prev_spos - 1 : 0;
      incs_cnt[k1 - 1] = tail_ic;
      if (tail_ic) atomicAdd(&st->spare[1], (unsigned long long)tail_ic * uint32_t(depth_c));
    }
    vcount[u] = ver_c + tail_ic + 1;
  }
}

// Phase D, accesses outside critical sections, in trace order (coalesced reads of the
// events and writes of the records): the access's gap is the one after its agent's latest
// synchronisation entry before it (a binary search in the agent's entries, which are in
// trace order); all accesses of such a gap share the epoch and the clock version.
// Phase D's index: table[u * nw + w] is agent u's first synchronisation entry at or after
// trace position w << shift (sy_start[u + 1] when there is none), so an access at i
// searches only the entries of its own window, [table[w], table[w + 1]). One thread per
// entry fills the windows from after its predecessor's window up to its own.
__global__ void k_d_index(const uint32_t* sy_idx, const uint32_t* sy_agent, const uint32_t* sy_start, uint32_t n_sync,
                          uint32_t shift, uint32_t nw, uint32_t* table) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sync) return;
  const uint32_t u = sy_agent[k];
  const uint32_t wk = sy_idx[k] >> shift;
  const uint32_t w0 = k > sy_start[u] ? (sy_idx[k - 1] >> shift) + 1 : 0;
  uint32_t* row = table + size_t(u) * nw;
  for (uint32_t w = w0; w <= wk; ++w) row[w] = k;
}

// the windows after an agent's last entry (all of them when it has none): a warp per agent
__global__ void k_d_index_tail(const uint32_t* sy_idx, const uint32_t* sy_start, uint32_t W, uint32_t shift,
                               uint32_t nw, uint32_t* table) {
  const uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (u >= W) return;
  const uint32_t k0 = sy_start[u], k1 = sy_start[u + 1];
  const uint32_t w0 = k1 > k0 ? (sy_idx[k1 - 1] >> shift) + 1 : 0;
  uint32_t* row = table + size_t(u) * nw;
  for (uint32_t w = w0 + lane; w < nw; w += 32) row[w] = k1;
}

__global__ void k_d_trace(const Event* ev, uint64_t N, Geo g, const uint32_t* sy_start, const uint32_t* sy_idx,
                          const uint32_t* table, uint32_t shift, uint32_t nw, const uint32_t* sy_N,
                          const uint32_t* sy_depth, const uint32_t* sy_ver, const uint32_t* rowbase, AccInfo* acc_info,
                          const DevStatus* st, bool vec, const uint32_t* wl_bits, uint32_t wl_log2,
                          uint32_t comp_lo, uint32_t comp_span) {
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N || st->code) return;
  const Event e = load_event(ev, i, vec);
  if (e.op > GWCP_ATOMIC) return;
  const uint32_t u = e.agent, x = uint32_t(i);
  if (wl_log2) {  // grouped order: a location without write-class accesses is never checked
    const uint64_t ck = composite_key(location_key(e, g.apb), access_class(e), u, comp_lo, comp_span);
    const uint32_t h = wl_bit(ck >> 15, wl_log2);
    if (!((__ldg(wl_bits + (h >> 5)) >> (h & 31)) & 1u)) return;
  }
  const uint32_t k0 = sy_start[u];
  // the agent's first entry at or after i: among its entries in i's window, else the first
  // entry of a later window
  const uint32_t* row = table + size_t(u) * nw + (x >> shift);
  uint32_t a = row[0], b = row[1];
  while (a < b) {
    const uint32_t mid = (a + b) >> 1;
    if (sy_idx[mid] < x)
      a = mid + 1;
    else
      b = mid;
  }
  uint32_t epoch = 1, ver = 0;
  if (a > k0) {
    const uint32_t k = a - 1;
    if (sy_depth[k] > 0) return;  // in a critical section: the gap walk below
    epoch = sy_N[k];
    ver = sy_ver[k];
  }
  acc_info[i] = AccInfo{epoch, rowbase[u] + ver, make_who(u, access_class(e), u / g.apb), 0};
}

// Phase D, accesses inside critical sections: one warp per gap after a synchronisation
// entry at nesting depth > 0 (each access there has a clock version of its own).
__global__ void k_d_fill(const Event* ev, Geo g, uint32_t n_sync, const uint32_t* S, const uint32_t* seg,
                         const uint32_t* sy_start, const uint32_t* sy_agent, const uint32_t* sy_spos,
                         const uint32_t* sy_N,
                         const uint32_t* sy_depth, const uint32_t* sy_ver, const uint32_t* incs_off,
                         const uint32_t* rowbase, AccInfo* acc_info, uint32_t* incs_idx, uint32_t* incs_ver,
                         uint32_t* incs_k, uint64_t* incs_key, uint32_t* incs_wr, const DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const uint64_t gid = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (gid >= n_sync || st->code) return;
  const uint32_t k = uint32_t(gid);
  if (sy_depth[k] == 0) return;
  const uint32_t u = sy_agent[k];
  const uint32_t lo = sy_spos[k] + 1;
  const uint32_t hi = (k + 1 < sy_start[u + 1]) ? sy_spos[k + 1] : seg[u + 1];
  const uint32_t epoch = sy_N[k], vbase = sy_ver[k];
  const uint32_t rb = rowbase[u];
  for (uint32_t p = lo + lane; p < hi; p += 32) {
    const uint32_t j = p - lo + 1;
    const uint32_t idx = s_idx(S[p]);
    const Event e = ev[idx];
    const uint32_t cls = access_class(e);
    const uint32_t ver = vbase + j;
    acc_info[idx] = AccInfo{epoch, rb + ver, make_who(u, cls, u / g.apb), 0};
    const uint32_t r = incs_off[k] + j - 1;
    incs_idx[r] = idx;
    incs_ver[r] = ver;
    incs_k[r] = k;
    incs_key[r] = location_key(e, g.apb);
    incs_wr[r] = cls != C_READ;
  }
}

// Phase C': forced compression at barriers (section "Vector Clock Compression"). Every
// member leaves a barrier at the same local time, the highest N_t among the members; the
// join then gives every member one common value for all members' entries. Local times are
// the plain ones plus a per-agent offset that changes only at the agent's barriers. A
// block's barriers involve only its own agents, so one warp per block walks them in trace
// order: M = max over members of (N before + offset), then offset = M - N before. When
// every barrier of a block has all the block's agents as members (always so at warp
// granularity), each barrier leaves them all at M + 1, so M_i = M_(i-1) + the largest
// plain increase of a member since the previous barrier: a prefix sum instead of a walk.
// A barrier with one member changes no offset and is left out.

// barrier -> (its block, or B for a one-member barrier; its trace-order position)
__global__ void k_fb_keys(const Event* ev, Geo g, const uint32_t* bar, uint32_t n_bar, uint64_t* key,
                          uint32_t* val) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_bar) return;
  const Event e = ev[bar[i]];
  const bool single = barrier_members(e, g).count <= 1;
  key[i] = single ? g.B : e.scope == GWCP_SCOPE_CTA ? uint32_t(e.addr) : e.agent / g.apb;
  val[i] = i;
}

// position r of the block-sorted order: inverse map, member count, block starts
__global__ void k_fb_rank(const Event* ev, Geo g, const uint32_t* bar, const uint64_t* skey, const uint32_t* spos,
                          uint32_t n_bar, uint32_t* rank, uint32_t* cnt, uint32_t* blo) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > n_bar) return;
  const uint32_t blk = r < n_bar ? uint32_t(skey[r]) : g.B;
  const uint32_t prev = r > 0 ? uint32_t(skey[r - 1]) : 0u;
  if (r == 0) {
    for (uint32_t b = 0; b <= blk; ++b) blo[b] = 0;
  } else {
    for (uint32_t b = prev + 1; b <= blk; ++b) blo[b] = r;
  }
  if (r == n_bar) {
    cnt[r] = 0;
    return;
  }
  const uint32_t pos = spos[r];
  rank[pos] = r;
  cnt[r] = barrier_members(ev[bar[pos]], g).count;
}

// one record per barrier participation, grouped by barrier in block order
__global__ void k_fb_records(const Event* ev, Geo g, uint32_t n_sync, uint32_t n_bar, const uint32_t* sy_agent,
                             const uint32_t* sy_kind, const uint32_t* sy_idx, const uint32_t* sy_aux,
                             const uint32_t* sy_N, const uint32_t* rank, const uint32_t* off, uint4* rec) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sync || sy_kind[k] != K_BAR) return;
  const uint32_t u = sy_agent[k];
  const BarMembers m = barrier_members(ev[sy_idx[k]], g);
  const uint32_t d = u - m.first, pos = sy_aux[k];
  if (!m.ok || d >= (m.mask ? 32u : m.count) || pos >= n_bar) return;  // not on a validated trace
  const uint32_t j = m.mask ? __popc(m.mask & ((1u << d) - 1u)) : d;
  if (j < m.count) rec[off[rank[pos]] + j] = make_uint4(k, sy_N[k] - 1, u % g.apb, m.count);
}

constexpr uint32_t FB_STAGE = 1024;  // records staged in shared memory at a time

__global__ void __launch_bounds__(32) k_fb_walk(Geo g, uint32_t n_sync, const uint32_t* blo, const uint32_t* off,
                                                const uint4* rec, uint32_t* boff, DevStatus* st) {
  __shared__ uint32_t off_s[1024];  // per member of the block (agents_per_block <= 1024)
  __shared__ uint4 rec_s[FB_STAGE];
  const uint32_t lane = threadIdx.x, b = blockIdx.x;
  const uint32_t r0 = blo[b], r1 = blo[b + 1];
  bool partial = false;
  for (uint32_t r = r0 + lane; r < r1; r += 32) partial |= off[r + 1] - off[r] != g.apb;
  if (!__any_sync(0xffffffffu, partial)) {
    // whole-block barriers: d_i = max over members of (N before barrier i - N before
    // barrier i-1), d_r0 = max N before the first; M_i = sum of d up to i
    uint32_t carry = 0;
    for (uint32_t i0 = r0; i0 < r1; i0 += 32) {
      const uint32_t i = i0 + lane;
      uint32_t d = 0;
      if (i < r1) {
        const uint32_t o = off[i], op = i > r0 ? off[i - 1] : 0u;
        for (uint32_t j = 0; j < g.apb; ++j) d = max(d, rec[o + j].y - (i > r0 ? rec[op + j].y : 0u));
      }
      const uint32_t M = carry + warp_inclusive_scan(d);
      if (i < r1) {
        const uint32_t o = off[i];
        for (uint32_t j = 0; j < g.apb; ++j) {
          const uint4 r = rec[o + j];
          if (r.x < n_sync) boff[r.x] = M - r.y;
        }
      }
      carry = __shfl_sync(0xffffffffu, M, 31);
    }
    return;
  }
  for (uint32_t j = lane; j < g.apb; j += 32) off_s[j] = 0;
  const uint32_t pend = off[r1];
  uint32_t p = off[r0], lo = p, hi = p;
  auto stage = [&](uint32_t at) {
    __syncwarp();
    lo = at;
    hi = min(at + FB_STAGE, pend);
    for (uint32_t i = lane; i < hi - lo; i += 32) rec_s[i] = rec[lo + i];
    __syncwarp();
  };
  while (p < pend) {
    if (p >= hi) stage(p);
    const uint32_t c = rec_s[p - lo].w;
    if (c == 0 || c > pend - p) {  // cannot happen on a validated trace
      if (lane == 0) set_error(st, GWCP_ERR_INVALID_TRACE, 0);
      return;
    }
    if (p + c > hi && c <= FB_STAGE) stage(p);
    const bool staged = p + c <= hi;
    uint32_t M = 0;
    bool bad = false;
    for (uint32_t j = lane; j < c; j += 32) {
      const uint4 r = staged ? rec_s[p - lo + j] : rec[p + j];
      bad |= r.z >= g.apb || r.x >= n_sync;
      M = max(M, r.y + (r.z < g.apb ? off_s[r.z] : 0u));
    }
    M = __reduce_max_sync(0xffffffffu, M);
    if (__any_sync(0xffffffffu, bad)) {  // a record left unwritten: not on a validated trace
      if (lane == 0) set_error(st, GWCP_ERR_INVALID_TRACE, 0);
      return;
    }
    for (uint32_t j = lane; j < c; j += 32) {
      const uint4 r = staged ? rec_s[p - lo + j] : rec[p + j];
      off_s[r.z] = M - r.y;
      boff[r.x] = M - r.y;
    }
    __syncwarp();
    p += c;
  }
}

// N after each entry += the offset of the agent's latest barrier entry at or before it
__global__ void k_fb_apply(Geo g, const uint32_t* sy_start, const uint32_t* boff, uint32_t* sy_N) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (u >= g.W) return;
  const uint32_t k0 = sy_start[u], k1 = sy_start[u + 1];
  const uint32_t le = (2u << lane) - 1u;
  uint32_t carry = 0;
  for (uint32_t kb = k0; kb < k1; kb += 32) {
    const uint32_t k = kb + lane;
    const bool valid = k < k1;
    const uint32_t o = valid ? boff[k] : NONE;
    const uint32_t set = __ballot_sync(0xffffffffu, valid && o != NONE);
    const uint32_t m = set & le;
    const uint32_t from = __shfl_sync(0xffffffffu, o, m ? 31 - __clz(m) : 0);
    if (valid) sy_N[k] += m ? from : carry;
    if (set) carry = __shfl_sync(0xffffffffu, o, 31 - __clz(set));
  }
}

// Phase E
__global__ void k_e_flags(const uint64_t* key, const uint32_t* kk, uint32_t n, const uint32_t* sy_kind,
                          uint32_t* is_acq, uint32_t* is_new) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  is_acq[m] = sy_kind[kk[m]] == K_ACQ;
  is_new[m] = (m == 0 || key[m] != key[m - 1]);
}

__global__ void k_e_assign(const Event* ev, Geo g, const uint32_t* kk, uint32_t n, const uint32_t* is_new,
                           const uint32_t* csid, const uint32_t* newscan, const uint32_t* sy_kind,
                           const uint32_t* sy_idx, const uint32_t* sy_N, const uint32_t* sy_relk,
                           uint32_t* cs_of_sync, uint32_t* cs_agent, uint32_t* cs_sid, uint32_t* cs_epoch,
                           uint32_t* cs_rel_idx, uint32_t* cs_rel_epoch, uint32_t* cs_lock, uint32_t* lock_first,
                           uint32_t* lock_cs_lo) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const uint32_t k = kk[m];
  const uint32_t lr = newscan[m] + is_new[m] - 1;
  if (m == n - 1) {  // sentinels: one past the last lock
    lock_first[lr + 1] = n;
    lock_cs_lo[lr + 1] = csid[n];
  }
  if (is_new[m]) {
    lock_first[lr] = m;
    lock_cs_lo[lr] = csid[m];
  }
  if (sy_kind[k] != K_ACQ) return;
  const uint32_t c = csid[m];
  const Event e = ev[sy_idx[k]];
  cs_of_sync[k] = c;
  cs_agent[c] = e.agent;
  cs_sid[c] = scope_id(e.agent, e.scope, g.apb);
  cs_epoch[c] = sy_N[k];
  cs_lock[c] = lr;
  cs_rel_idx[c] = sy_relk[k] != NONE ? sy_idx[sy_relk[k]] : NONE;
  cs_rel_epoch[c] = sy_relk[k] != NONE ? sy_N[sy_relk[k]] - 1 : 0;  // N before the release's increment
}

__global__ void k_e_assign_rel(const uint32_t* kk, uint32_t n, const uint32_t* sy_kind, const uint32_t* sy_match,
                               uint32_t* cs_of_sync, uint32_t* cs_parent) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const uint32_t k = kk[m];
  const uint32_t mt = sy_match[k];
  if (sy_kind[k] == K_REL) {
    cs_of_sync[k] = mt != NONE ? cs_of_sync[mt] : NONE;
  } else {
    cs_parent[cs_of_sync[k]] = mt != NONE ? cs_of_sync[mt] : NONE;
  }
}

struct LockSlot {
  uint32_t sid, latest_cs, latest_rel, open;
};

// One thread per lock: acquire joins (the latest release on each overlapping scope),
// W3 (overlapping critical sections never interleave). A lock's scopes get slots in order
// of first use, found through a small open-addressing table. Device scope (0) overlaps
// every scope; a block scope overlaps itself and device scope. An acquire at block scope
// joins the latest critical section of its own scope and of device scope; one at device
// scope joins the latest of device scope and of every scope released since then (the
// `recent` list, emptied by each device-scope release).
template <int MAXS>
__global__ void k_e_walk(const uint32_t* kk, const uint32_t* lock_first, uint32_t n_locks, const uint32_t* csid,
                         const uint32_t* sy_kind, const uint32_t* sy_idx, const uint32_t* cs_of_sync,
                         const uint32_t* cs_sid, uint32_t* acq_dep_off, uint32_t* acq_dep_cnt, uint32_t* pool,
                         uint32_t pool_cap, DevStatus* st) {
  constexpr int HS = MAXS <= 64 ? 128 : 1024;  // power of two, at least twice MAXS
  uint32_t lr = blockIdx.x * blockDim.x + threadIdx.x;
  const int code = st->code;
  if (lr >= n_locks || (code && code != GWCP_ERR_INVALID_TRACE)) return;
  LockSlot sl[MAXS];
  uint16_t hslot[HS];    // slot + 1, 0 = empty
  uint16_t recent[MAXS];  // slots released since the latest device-scope release
  bool in_recent[MAXS];
  for (int h = 0; h < HS; ++h) hslot[h] = 0;
  int ns = 0, n_recent = 0, q0 = -1;
  uint32_t open_total = 0;
  auto slot = [&](uint32_t sid) -> int {
    uint32_t h = (sid * 0x9E3779B1u) >> 16;
    for (;; ++h) {
      const uint32_t e = hslot[h & (HS - 1)];
      if (e == 0) break;
      if (sl[e - 1].sid == sid) return int(e - 1);
    }
    if (ns == MAXS) return -1;
    sl[ns] = LockSlot{sid, NONE, NONE, 0};
    in_recent[ns] = false;
    hslot[h & (HS - 1)] = uint16_t(ns + 1);
    if (sid == 0) q0 = ns;
    return ns++;
  };
  for (uint32_t m = lock_first[lr]; m < lock_first[lr + 1]; ++m) {
    const uint32_t k = kk[m], idx = sy_idx[k];
    const uint32_t c = cs_of_sync[k];
    if (c == NONE) return;  // invalid trace, flagged by the agent walk
    const uint32_t sid = cs_sid[c];
    const int q = slot(sid);
    if (q < 0) {
      set_error(st, GWCP_ERR_UNSUPPORTED, idx);
      return;
    }
    if (sy_kind[k] == K_ACQ) {
      const bool clash = sid == 0 ? open_total > 0 : (sl[q].open > 0 || (q0 >= 0 && sl[q0].open > 0));
      if (clash) {
        set_error(st, GWCP_ERR_INVALID_TRACE, idx);
        return;
      }
      uint32_t deps[MAXS];
      uint32_t nd = 0;
      if (q0 >= 0 && sl[q0].latest_cs != NONE) deps[nd++] = sl[q0].latest_cs;
      if (sid == 0) {
        for (int r = 0; r < n_recent; ++r) deps[nd++] = sl[recent[r]].latest_cs;
      } else if (q != q0 && sl[q].latest_cs != NONE) {
        deps[nd++] = sl[q].latest_cs;
      }
      const uint32_t cid = csid[m];
      uint32_t off = 0;
      if (nd) {
        off = uint32_t(atomicAdd(&st->dep_pool_used, (unsigned long long)nd));
        if (off + nd > pool_cap) {
          set_error(st, GWCP_ERR_OOM, idx);
          return;
        }
        for (uint32_t j = 0; j < nd; ++j) pool[off + j] = deps[j];
      }
      acq_dep_off[cid] = off;
      acq_dep_cnt[cid] = nd;
      sl[q].open++;
      open_total++;
    } else {
      sl[q].open--;
      open_total--;
      sl[q].latest_cs = c;
      sl[q].latest_rel = idx;
      if (q == q0) {
        for (int r = 0; r < n_recent; ++r) in_recent[recent[r]] = false;
        n_recent = 0;
      } else if (!in_recent[q]) {
        in_recent[q] = true;
        recent[n_recent++] = uint16_t(q);
      }
    }
  }
}

// Phase F
__global__ void k_f_depths(const uint32_t* incs_k, uint32_t n_incs, const uint32_t* sy_depth, uint32_t* out) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_incs) out[r] = sy_depth[incs_k[r]];
}

__global__ void k_f_expand(const uint32_t* incs_k, const uint32_t* incs_idx, uint32_t n_incs,
                           const uint32_t* exp_off, const uint32_t* sy_inner, const uint32_t* cs_of_sync,
                           const uint32_t* cs_parent, uint32_t* ex_rec, uint32_t* ex_cs, uint64_t* key,
                           uint32_t* val) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_incs) return;
  uint32_t c = cs_of_sync[sy_inner[incs_k[r]]];
  for (uint32_t e = exp_off[r]; e < exp_off[r + 1]; ++e) {
    ex_rec[e] = r;
    ex_cs[e] = c;
    key[e] = incs_idx[r];
    val[e] = e;
    c = c != NONE ? cs_parent[c] : NONE;
  }
}

__global__ void k_f_rekey(const uint32_t* val, uint32_t n, int stage, const uint32_t* ex_rec, const uint32_t* ex_cs,
                          const uint64_t* incs_key, const uint32_t* cs_lock, uint64_t* key) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const uint32_t e = val[m];
  const uint32_t c = ex_cs[e];
  key[m] = stage == 1 ? incs_key[ex_rec[e]] : uint64_t(c != NONE ? cs_lock[c] : 0);
}

__global__ void k_f_groupflags(const uint32_t* val, uint32_t n, const uint32_t* ex_rec, const uint32_t* ex_cs,
                               const uint64_t* incs_key, const uint32_t* cs_lock, uint32_t* flags) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  bool nw = m == 0;
  if (!nw) {
    const uint32_t a = val[m - 1], b = val[m];
    const uint32_t ca = ex_cs[a], cb = ex_cs[b];
    nw = incs_key[ex_rec[a]] != incs_key[ex_rec[b]] || ca == NONE || cb == NONE || cs_lock[ca] != cs_lock[cb];
  }
  flags[m] = nw;
}

__global__ void k_f_groupstarts(const uint32_t* flags, const uint32_t* scan, uint32_t n, uint32_t* starts) {
  uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n && flags[m]) starts[scan[m]] = m;
  if (m == n - 1) starts[scan[m] + flags[m]] = n;  // one past the last group
}

struct ObjSlot {
  uint32_t sid, cur, cur_w, cur_r, prev_w, prev_r;
};

// One thread per (lock, location): in trace order, the releases whose L^w / L^r an
// in-section access joins, per overlapping scope (Algorithm 2). L^w_<l,s>,x is the
// join of H over earlier releases on <l,s> whose section wrote x; those H only grow
// along one scoped lock, so the latest such release is the whole join.
template <int MAXS>
__global__ void k_f_walk(const uint32_t* val, const uint32_t* starts, uint32_t max_groups, const uint32_t* ex_rec,
                         const uint32_t* ex_cs, const uint32_t* incs_wr, const uint32_t* cs_sid,
                         const uint32_t* cs_rel_idx, uint32_t* ex_dep_off, uint32_t* ex_dep_cnt, uint32_t* pool,
                         uint32_t pool_cap, DevStatus* st) {
  uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n_groups = uint32_t(st->spare[0]);  // exact count, written by the group scan
  if (gi >= max_groups || gi >= n_groups || st->code) return;
  ObjSlot sl[MAXS];
  int ns = 0;
  for (uint32_t m = starts[gi]; m < starts[gi + 1]; ++m) {
    const uint32_t e = val[m];
    const uint32_t c = ex_cs[e];
    if (c == NONE) return;
    const uint32_t s = cs_sid[c];
    const bool wr = incs_wr[ex_rec[e]] != 0;
    int q = -1;
    for (int r = 0; r < ns; ++r)
      if (sl[r].sid == s) q = r;
    if (q < 0) {
      if (ns == MAXS) {
        set_error(st, GWCP_ERR_UNSUPPORTED, 0);
        return;
      }
      q = ns++;
      sl[q] = ObjSlot{s, NONE, 0, 0, NONE, NONE};
    }
    if (sl[q].cur != c) {  // a new section on this scope: the previous one is complete
      if (sl[q].cur != NONE) {
        if (sl[q].cur_w) sl[q].prev_w = sl[q].cur;
        if (sl[q].cur_r) sl[q].prev_r = sl[q].cur;
      }
      sl[q].cur = c;
      sl[q].cur_w = sl[q].cur_r = 0;
    }
    uint32_t deps[2 * MAXS];
    uint32_t nd = 0;
    // latest completed section on scope slot r that wrote (w) or read (!w) x
    auto latest = [&](int r, bool w) -> uint32_t {
      if (sl[r].sid != s && sl[r].cur != NONE && (w ? sl[r].cur_w : sl[r].cur_r)) return sl[r].cur;
      return w ? sl[r].prev_w : sl[r].prev_r;
    };
    for (int kind = 0; kind < (wr ? 2 : 1); ++kind) {
      const bool w = kind == 0;  // reads join L^w; writes join L^w and L^r
      int q0 = -1;
      for (int r = 0; r < ns; ++r)
        if (sl[r].sid == 0) q0 = r;
      const uint32_t d0 = q0 >= 0 ? latest(q0, w) : NONE;
      if (d0 != NONE) deps[nd++] = d0;
      const uint32_t rel0 = d0 != NONE ? cs_rel_idx[d0] : NONE;
      for (int r = 0; r < ns; ++r) {
        if (r == q0) continue;
        if (s != 0 && sl[r].sid != s) continue;
        const uint32_t d = latest(r, w);
        if (d == NONE) continue;
        if (s == 0 && rel0 != NONE && cs_rel_idx[d] <= rel0) continue;
        deps[nd++] = d;
      }
    }
    uint32_t off = 0;
    if (nd) {
      off = uint32_t(atomicAdd(&st->dep_pool_used, (unsigned long long)nd));
      if (off + nd > pool_cap) {
        set_error(st, GWCP_ERR_OOM, 0);
        return;
      }
      for (uint32_t j = 0; j < nd; ++j) pool[off + j] = deps[j];
    }
    ex_dep_off[e] = off;
    ex_dep_cnt[e] = nd;
    if (wr)
      sl[q].cur_w = 1;
    else
      sl[q].cur_r = 1;
  }
}

inline uint32_t blocks(uint64_t n, uint32_t t) { return uint32_t((n + t - 1) / t); }

// phase A warps per CTA: each holds a Wp-word histogram in shared memory (<= 48 KB per CTA)
inline uint32_t a_warps(const Geo& g) {
  uint32_t w = A_WARPS;
  while (w > 1 && size_t(w) * g.Wp * 4 > 48 * 1024) w >>= 1;
  return w;
}

}  // namespace

void phaseA_count(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  p.begin("a_count", double(z.N) * 16);
  const bool vec = (reinterpret_cast<uintptr_t>(b.ev) & 15) == 0;
  if (z.agent_sort) {
    k_aw_count<<<blocks(z.ntA, 8), 256, 0, s>>>(b.ev, z.N, g, z.TA, z.ntA, b.tile_cnt, b.st, vec);
    count_launch();
    p.end();
    for (int q = 0; q < 4; ++q) {  // in-place exclusive scans of the per-tile counts
      uint32_t* t = b.tile_cnt + q * (z.ntA + 1);
      scan_exclusive(t, t, z.ntA, t + z.ntA, b.scan_tmp, s);
    }
    return;
  }
  const uint32_t aw = a_warps(g);
  k_a_count<<<blocks(z.ntA, aw), aw * 32, aw * g.Wp * 4, s>>>(b.ev, z.N, g, z.TA, z.ntA, b.hist_a,
                                                                          b.tile_cnt, b.st, vec);
  count_launch();
  p.end();
  // in-place exclusive scans: agent histogram and the three per-tile counts
  scan_exclusive(b.hist_a, b.hist_a, size_t(g.W) * z.ntA, b.hist_a + size_t(g.W) * z.ntA, b.scan_tmp, s);
  for (int q = 0; q < 3; ++q) {
    uint32_t* t = b.tile_cnt + q * (z.ntA + 1);
    scan_exclusive(t, t, z.ntA, t + z.ntA, b.scan_tmp, s);
  }
}

void phaseA_scatter(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  p.begin("a_scatter", double(z.N) * 16 + double(z.nS) * 4 + double(z.n_acc) * 12);
  if (z.wl_log2) cudaMemsetAsync(b.wl_bits, 0, (size_t(1) << z.wl_log2) / 8, s);
  const bool vec = (reinterpret_cast<uintptr_t>(b.ev) & 15) == 0;
  const ACompact cpt{b.acc_key, b.acc_idx, b.acqrel, b.bar, z.grouped ? z.comp_lo : 0u,
                     z.grouped ? z.comp_span : 0u, b.wl_bits, z.wl_log2};
  if (z.agent_sort) {
    k_aw_scatter<<<blocks(z.ntA, 8), 256, 0, s>>>(b.ev, z.N, g, z.TA, z.ntA, b.tile_cnt, b.s_key, cpt, vec);
    count_launch();
    uint32_t ab = 0;
    while ((1u << ab) < g.W) ++ab;
    const uint64_t mask = ((1ull << ab) - 1) << 32;
    const uint64_t* sorted =
        radix_sort_pairs(b.s_key, nullptr, b.s_key2, nullptr, z.nS, mask, b.s_tmp, s) ? b.s_key2 : b.s_key;
    if (z.nS) {
      k_aw_extract<<<blocks(z.nS, 256), 256, 0, s>>>(sorted, z.nS, b.S);
      count_launch();
    }
    k_aw_seg<<<blocks(g.W + 1, 256), 256, 0, s>>>(sorted, z.nS, g.W, b.seg);
    count_launch();
    p.end();
    return;
  }
  const uint32_t aw = a_warps(g);
  k_a_scatter<<<blocks(z.ntA, aw), aw * 32, aw * g.Wp * 4, s>>>(b.ev, z.N, g, z.TA, z.ntA, b.hist_a, b.tile_cnt,
                                                                b.S, cpt, vec);
  count_launch();
  k_a_segments<<<blocks(g.W + 1, 256), 256, 0, s>>>(b.hist_a, g.W, z.ntA, z.nS, b.seg);
  count_launch();
  p.end();
}

void phaseB_sync(const Bufs& b, const Geo& g, Sizes& z, cudaStream_t s, Prof& p) {
  z.ntS = blocks(z.nS, B_CHUNK);  // chunks of S, one warp each
  p.begin("b_sync", double(z.nS) * 8);
  if (z.ntS) {
    k_b_count<<<blocks(uint64_t(z.ntS) * 32, B_THREADS), B_THREADS, 0, s>>>(b.S, z.nS, z.ntS, b.sy_cnt);
    count_launch();
    scan_exclusive(b.sy_cnt, b.sy_cnt, z.ntS, b.sy_cnt + z.ntS, b.scan_tmp, s);
    k_b_scatter<<<blocks(uint64_t(z.ntS) * 32, B_THREADS), B_THREADS, 0, s>>>(
        b.ev, b.S, z.nS, z.ntS, b.sy_cnt, b.bar, z.n_bar, b.acqrel, z.n_acqrel, b.sy_spos, b.sy_idx, b.sy_kind,
        b.sy_aux, b.lk_key, b.lk_k);
    count_launch();
  }
  k_b_starts<<<blocks(g.W + 1, 256), 256, 0, s>>>(b.seg, g.W, b.sy_spos, z.n_sync, b.sy_start);
  count_launch();
  p.end();
}

void phaseC_walk(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  p.begin("c_walk", double(z.n_sync) * 40);
  cudaMemsetAsync(b.sy_relk, 0xFF, size_t(z.n_sync + 1) * 4, s);
  cudaMemsetAsync(b.incs_cnt, 0, size_t(z.n_sync + 1) * 4, s);
  k_c_walk<<<blocks(uint64_t(g.W) * 32, 128), 128, 0, s>>>(b.ev, g, b.seg, b.sy_start, b.sy_spos, b.sy_idx, b.sy_kind,
                                                           b.sy_N, b.sy_depth, b.sy_inner, b.sy_ver, b.sy_match,
                                                           b.sy_relk, b.incs_cnt, b.vcount, b.sy_agent, b.st);
  count_launch();
  p.end();
  scan_exclusive(b.incs_cnt, b.incs_cnt, z.n_sync + 1, nullptr, b.scan_tmp, s);
  scan_exclusive(b.vcount, b.vcount, g.W + 1, nullptr, b.scan_tmp, s);
}

void phaseC_forced(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  const uint32_t n = z.n_bar;
  if (!n) return;
  p.begin("c_forced", double(n) * 40 + double(z.n_sync) * 24);
  k_fb_keys<<<blocks(n, 256), 256, 0, s>>>(b.ev, g, b.bar, n, b.fb_key, b.fb_val);
  count_launch();
  uint64_t mask = 0;  // keys 0..B (B: one-member barriers, left out of the walk)
  while (mask < g.B) mask = (mask << 1) | 1;
  const bool second = radix_sort_pairs(b.fb_key, b.fb_val, b.fb_key2, b.fb_val2, n, mask, b.scan_tmp, s);
  const uint64_t* skey = second ? b.fb_key2 : b.fb_key;
  const uint32_t* spos = second ? b.fb_val2 : b.fb_val;
  k_fb_rank<<<blocks(uint64_t(n) + 1, 256), 256, 0, s>>>(b.ev, g, b.bar, skey, spos, n, b.fb_rank, b.fb_off,
                                                          b.fb_blo);
  count_launch();
  scan_exclusive(b.fb_off, b.fb_off, size_t(n) + 1, nullptr, b.scan_tmp, s);
  cudaMemsetAsync(b.fb_boff, 0xFF, size_t(z.n_sync + 1) * 4, s);
  k_fb_records<<<blocks(z.n_sync, 256), 256, 0, s>>>(b.ev, g, z.n_sync, n, b.sy_agent, b.sy_kind, b.sy_idx, b.sy_aux,
                                                     b.sy_N, b.fb_rank, b.fb_off, b.fb_rec);
  count_launch();
  k_fb_walk<<<g.B, 32, 0, s>>>(g, z.n_sync, b.fb_blo, b.fb_off, b.fb_rec, b.fb_boff, b.st);
  count_launch();
  k_fb_apply<<<blocks(uint64_t(g.W) * 32, 128), 128, 0, s>>>(g, b.sy_start, b.fb_boff, b.sy_N);
  count_launch();
  p.end();
}

// the trace-order pass of phase D; filtered: only accesses the grouped order keeps
void phaseD_trace(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, bool filtered) {
  k_d_trace<<<blocks(z.N, 256), 256, 0, s>>>(b.ev, z.N, g, b.sy_start, b.sy_idx, b.d_index, z.d_shift, z.d_nw,
                                              b.sy_N, b.sy_depth, b.sy_ver, b.vcount, b.acc_info, b.st,
                                              (reinterpret_cast<uintptr_t>(b.ev) & 15) == 0, b.wl_bits,
                                              filtered ? z.wl_log2 : 0u, z.comp_lo, z.comp_span);
  count_launch();
}

void phaseD_gaps(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  p.begin("d_gaps", double(z.n_acc) * (4 + 16 + 16), s);
  if (z.n_sync) {
    k_d_index<<<blocks(z.n_sync, 256), 256, 0, s>>>(b.sy_idx, b.sy_agent, b.sy_start, z.n_sync, z.d_shift, z.d_nw,
                                                    b.d_index);
    count_launch();
  }
  k_d_index_tail<<<blocks(uint64_t(g.W) * 32, 256), 256, 0, s>>>(b.sy_idx, b.sy_start, g.W, z.d_shift, z.d_nw,
                                                                 b.d_index);
  count_launch();
  phaseD_trace(b, g, z, s, true);
  if (z.n_sync) {
    k_d_fill<<<blocks(uint64_t(z.n_sync) * 32, 256), 256, 0, s>>>(
        b.ev, g, z.n_sync, b.S, b.seg, b.sy_start, b.sy_agent, b.sy_spos, b.sy_N, b.sy_depth, b.sy_ver, b.incs_cnt,
        b.vcount, b.acc_info, b.incs_idx, b.incs_ver, b.incs_k, b.incs_key, b.incs_wr, b.st);
    count_launch();
  }
  p.end();
}

void phaseE_locks(Bufs& b, const Geo& g, const Sizes& z, uint64_t lock_mask, cudaStream_t s, Prof& p) {
  (void)g;
  const uint32_t n = z.n_acqrel;
  if (!n) return;
  p.begin("e_sort", double(n) * 24);
  if (radix_sort_pairs(b.lk_key, b.lk_k, b.lk_key2, b.lk_k2, n, lock_mask, b.scan_tmp, s)) {
    std::swap(b.lk_key, b.lk_key2);
    std::swap(b.lk_k, b.lk_k2);
  }
  k_e_flags<<<blocks(n, 256), 256, 0, s>>>(b.lk_key, b.lk_k, n, b.sy_kind, b.lk_flags, b.lk_rank);
  count_launch();
  p.end();
}

// lk_csid = exclusive scan of the acquire flags (critical-section ids, grouped by lock
// and in acquire order within a lock); lk_flags then holds the scan of new-lock flags.
void phaseE_scan(const Bufs& b, const Sizes& z, cudaStream_t s, Prof& p) {
  const uint32_t n = z.n_acqrel;
  if (!n) return;
  p.begin("e_scan", double(n) * 16);
  scan_exclusive(b.lk_flags, b.lk_csid, n, b.lk_csid + n, b.scan_tmp, s);
  scan_exclusive(b.lk_rank, b.lk_flags, n, b.lk_flags + n, b.scan_tmp, s);
  p.end();
}

void phaseE_walk(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  const uint32_t n = z.n_acqrel;
  if (!n) return;
  p.begin("e_walk", double(n) * 32);
  const uint32_t* newflag = b.lk_rank;
  const uint32_t* newscan = b.lk_flags;
  k_e_assign<<<blocks(n, 256), 256, 0, s>>>(b.ev, g, b.lk_k, n, newflag, b.lk_csid, newscan, b.sy_kind, b.sy_idx,
                                            b.sy_N, b.sy_relk, b.cs_of_sync, b.cs_agent, b.cs_sid, b.cs_epoch,
                                            b.cs_rel_idx, b.cs_rel_epoch, b.cs_lock, b.lock_first, b.lock_cs_lo);
  count_launch();
  k_e_assign_rel<<<blocks(n, 256), 256, 0, s>>>(b.lk_k, n, b.sy_kind, b.sy_match, b.cs_of_sync, b.cs_parent);
  count_launch();
  auto ew = lock_scope_cap(g.B) == kLockScopesSmall ? k_e_walk<kLockScopesSmall> : k_e_walk<kLockScopesLarge>;
  ew<<<blocks(z.n_locks, 128), 128, 0, s>>>(b.lk_k, b.lock_first, z.n_locks, b.lk_csid, b.sy_kind, b.sy_idx,
                                            b.cs_of_sync, b.cs_sid, b.acq_dep_off, b.acq_dep_cnt, b.dep_pool,
                                            z.pool_cap, b.st);
  count_launch();
  p.end();
}

void phaseF_incs(const Bufs& b, const Geo& g, const Sizes& z, uint64_t key_mask, cudaStream_t s, Prof& p) {
  (void)g;
  (void)key_mask;
  if (!z.n_incs) return;
  p.begin("f_expand", double(z.n_incs) * 16);
  k_f_depths<<<blocks(z.n_incs, 256), 256, 0, s>>>(b.incs_k, z.n_incs, b.sy_depth, b.exp_off);
  count_launch();
  scan_exclusive(b.exp_off, b.exp_off, z.n_incs + 1, nullptr, b.scan_tmp, s);
  p.end();
}

void phaseF_walk(Bufs& bb, const Geo& g, const Sizes& z, uint64_t key_mask, cudaStream_t s, Prof& p) {
  (void)g;
  const Bufs& b = bb;
  const uint32_t n = z.n_exp;
  if (!n) return;
  p.begin("f_walk", double(n) * 64);
  k_f_expand<<<blocks(z.n_incs, 256), 256, 0, s>>>(b.incs_k, b.incs_idx, z.n_incs, b.exp_off, b.sy_inner,
                                                   b.cs_of_sync, b.cs_parent, b.ex_rec, b.ex_cs, bb.ex_key, bb.ex_val);
  count_launch();
  uint64_t idx_mask = 0;
  for (uint64_t v = z.N; v; v >>= 1) idx_mask = (idx_mask << 1) | 1;
  // stage 0: by trace index; stage 1: by location key; stage 2: by lock rank (LSD)
  for (int stage = 0; stage < 3; ++stage) {
    if (stage > 0) {
      k_f_rekey<<<blocks(n, 256), 256, 0, s>>>(bb.ex_val, n, stage, b.ex_rec, b.ex_cs, b.incs_key, b.cs_lock,
                                               bb.ex_key);
      count_launch();
    }
    uint64_t mask = stage == 0 ? idx_mask : stage == 1 ? key_mask : 0;
    if (stage == 2)
      for (uint64_t v = z.n_locks; v; v >>= 1) mask = (mask << 1) | 1;
    if (radix_sort_pairs(bb.ex_key, bb.ex_val, bb.ex_key2, bb.ex_val2, n, mask, bb.scan_tmp, s)) {
      std::swap(bb.ex_key, bb.ex_key2);
      std::swap(bb.ex_val, bb.ex_val2);
    }
  }
  k_f_groupflags<<<blocks(n, 256), 256, 0, s>>>(bb.ex_val, n, b.ex_rec, b.ex_cs, b.incs_key, b.cs_lock, b.ex_flags);
  count_launch();
  uint32_t* scan = bb.ex_val2;  // free after the sorts
  uint32_t* n_groups = reinterpret_cast<uint32_t*>(&b.st->spare[0]);
  scan_exclusive(b.ex_flags, scan, n, n_groups, b.scan_tmp, s);
  k_f_groupstarts<<<blocks(n, 256), 256, 0, s>>>(b.ex_flags, scan, n, b.ex_group);
  count_launch();
  p.end();
}

void phaseF_deps(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  if (!z.n_groups) return;
  p.begin("f_deps", double(z.n_exp) * 32);
  auto fw = lock_scope_cap(g.B) == kLockScopesSmall ? k_f_walk<kLockScopesSmall> : k_f_walk<kLockScopesLarge>;
  fw<<<blocks(z.n_groups, 128), 128, 0, s>>>(b.ex_val, b.ex_group, z.n_groups, b.ex_rec, b.ex_cs, b.incs_wr,
                                             b.cs_sid, b.cs_rel_idx, b.ex_dep_off, b.ex_dep_cnt, b.dep_pool,
                                             z.pool_cap, b.st);
  count_launch();
  p.end();
}

}  // namespace gwcp
