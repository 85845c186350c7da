// Access grouping and the per-location race check of libgwcp.
//
// Accesses are sorted by (location key, trace index) with the library's radix sort,
// then cut into fixed chunks of CH entries; one warp checks one chunk in order. The
// warp keeps, for every agent v (lane l owns agents [l*K, l*K+K)) and access class
// (read, write, block-scoped atomic, device-scoped atomic), the latest access by v to
// the current location as (index << 32 | epoch) - the R_x / W_x state of the paper's
// metadata, kept per agent. For an access b by u every lane forms, for each of its
// agents v != u, a* = the latest access of v that conflicts with b and is not exempt,
// and reports (a*, b) when N(a*) > C_b[v], reading C_b[v] from the clock-version row
// of b written by the propagation. A location that spans chunks carries the state in:
// per chunk the state of its last location is reduced, then a segmented max-scan over
// chunks (two levels) gives each chunk the state at its start.
#include "gwcp_internal.cuh"

namespace gwcp {

namespace {

constexpr uint32_t CH = 512;       // accesses per chunk (one warp)
constexpr uint32_t GRP = 32;       // chunks per first-level scan group
constexpr int CHK_WARPS = 4;

struct ChunkArgs {
  const uint64_t* key;
  const uint32_t* idx;
  const AccInfo* info;
  uint32_t n;
  uint32_t n_chunks;
  uint64_t* T;          // [n_chunks][4 * Wp] packed (index << 32 | epoch), 0 = none
  const uint32_t* rows;
  uint64_t* races;
  uint64_t race_cap;
  DevStatus* st;
  Geo g;
  unsigned long long* chunk_ns;  // optional timeline: globaltimer at each chunk's end
  uint32_t* chunk_races;         // and the races it found
};

__device__ __forceinline__ bool chunk_continues(const ChunkArgs& a, uint32_t c) {
  // the last location of chunk c goes on into chunk c + 1
  if (c + 1 >= a.n_chunks) return false;
  const uint32_t e = (c + 1) * CH;
  return a.key[e - 1] == a.key[e];
}

// last[cl][ag % K] := v on the lane that owns agent ag. One indexed store keeps the
// table in local memory (L1); measured faster than a select per register slot, which
// every lane executes for all 4 * K slots.
template <int K>
__device__ __forceinline__ void put_slot(uint64_t (&last)[4][K], int lane, uint32_t ag, uint32_t cl, uint64_t v) {
  if (uint32_t(lane) == ag / K) last[cl][ag % K] = v;
}

// State of the chunk's last location over the chunk's entries.
template <int K>
__global__ void k_tail(ChunkArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= a.n_chunks) return;
  const uint32_t Wp = a.g.Wp;
  uint64_t* T = a.T + size_t(c) * 4 * Wp;
  uint64_t last[4][K];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < K; ++j) last[q][j] = 0;
  if (chunk_continues(a, c)) {
    const uint32_t lo = c * CH, hi = min(lo + CH, a.n);
    const uint64_t tk = a.key[hi - 1];
    for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
      const uint32_t p = b0 + lane;
      bool mine = false;
      uint32_t ix = 0, ep = 0, who = 0;
      if (p < hi && a.key[p] == tk) {
        mine = true;
        ix = a.idx[p];
        const AccInfo inf = a.info[ix];
        ep = inf.epoch;
        who = inf.who;
      }
      uint32_t m = __ballot_sync(0xffffffffu, mine);
      while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t wb = __shfl_sync(0xffffffffu, who, i);
        const uint64_t v = (uint64_t(__shfl_sync(0xffffffffu, ix, i)) << 32) | __shfl_sync(0xffffffffu, ep, i);
        put_slot<K>(last, lane, who_agent(wb), who_class(wb), v);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < K; ++j) T[q * Wp + lane * K + j] = last[q][j];
}

// links for the segmented scan: chunk c folds in chunk c-1's prefix when chunk c-1
// continues into c and chunk c holds only that location
__device__ __forceinline__ bool linked(const ChunkArgs& a, uint32_t c) {
  if (c == 0 || !chunk_continues(a, c - 1)) return false;
  const uint32_t lo = c * CH, hi = min(lo + CH, a.n);
  return a.key[lo] == a.key[hi - 1];
}

__global__ void k_scan1(ChunkArgs a, uint64_t* gagg, uint32_t* gfull) {
  const uint32_t cols = 4 * a.g.Wp;
  const uint32_t g0 = blockIdx.x * GRP, g1 = min(g0 + GRP, a.n_chunks);
  const bool first_linked = linked(a, g0);
  bool full = first_linked;
  for (uint32_t c = g0 + 1; c < g1; ++c) full = full && linked(a, c);
  for (uint32_t col = threadIdx.x; col < cols; col += blockDim.x) {
    uint64_t acc = 0;
    for (uint32_t c = g0; c < g1; ++c) {
      uint64_t v = a.T[size_t(c) * cols + col];
      acc = (c > g0 && linked(a, c)) ? max(acc, v) : v;
      a.T[size_t(c) * cols + col] = acc;
    }
    gagg[size_t(blockIdx.x) * cols + col] = acc;
  }
  if (threadIdx.x == 0) gfull[blockIdx.x] = uint32_t(full) | (uint32_t(first_linked) << 1);
}

__global__ void k_scan2(ChunkArgs a, uint32_t ngroups, uint64_t* gagg, const uint32_t* gfull) {
  // gagg[g] becomes the carry into group g. The loads of a window of groups are issued
  // together; only the running value is carried from group to group.
  constexpr int U = 8;
  const uint32_t cols = 4 * a.g.Wp;
  const uint32_t col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  uint64_t prev_final = 0;
  for (uint32_t g0 = 0; g0 < ngroups; g0 += U) {
    uint64_t agg[U];
    uint32_t fl[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      agg[q] = g0 + q < ngroups ? gagg[size_t(g0 + q) * cols + col] : 0;
      fl[q] = g0 + q < ngroups ? gfull[g0 + q] : 0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (g0 + q >= ngroups) break;
      const uint64_t carry = (fl[q] & 2) ? prev_final : 0;  // group starts linked to the previous one
      prev_final = (fl[q] & 1) ? max(prev_final, agg[q]) : agg[q];
      gagg[size_t(g0 + q) * cols + col] = carry;
    }
  }
}

__global__ void k_scan3(ChunkArgs a, const uint64_t* gagg) {
  const uint32_t cols = 4 * a.g.Wp;
  const uint32_t g0 = blockIdx.x * GRP, g1 = min(g0 + GRP, a.n_chunks);
  for (uint32_t col = threadIdx.x; col < cols; col += blockDim.x) {
    const uint64_t carry = gagg[size_t(blockIdx.x) * cols + col];
    if (!carry) continue;
    for (uint32_t c = g0; c < g1 && linked(a, c); ++c) {
      uint64_t& v = a.T[size_t(c) * cols + col];
      v = max(v, carry);
    }
  }
}

// classes a later access of class cb conflicts with and is not exempt from, as a 4-bit
// mask over (read, write, block atomic, device atomic); `same` = the two agents share a
// block (then two block-scoped atomics are exempt)
__device__ __forceinline__ uint32_t conflict_mask(uint32_t cb, bool same) {
  switch (cb) {
    case C_READ: return 0b1110;
    case C_WRITE: return 0b1111;
    case C_ATOM_CTA: return same ? 0b0011 : 0b0111;
    default: return 0b0011;  // device atomic: exempt against every atomic
  }
}

template <int K>
__global__ void __launch_bounds__(CHK_WARPS * 32) k_check(ChunkArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= a.n_chunks) return;
  const Geo& g = a.g;
  const uint32_t Wp = g.Wp;
  const uint32_t lo = c * CH, hi = min(lo + CH, a.n);
  const uint32_t lt = lanemask_lt();
  uint64_t last[4][K];
  if (c > 0 && chunk_continues(a, c - 1)) {
    const uint64_t* T = a.T + size_t(c - 1) * 4 * Wp;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < K; ++j) last[q][j] = T[q * Wp + lane * K + j];
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int j = 0; j < K; ++j) last[q][j] = 0;
  }
  uint32_t myblk[K];
#pragma unroll
  for (int j = 0; j < K; ++j) myblk[j] = (lane * K + j) / g.apb;
  uint64_t prev_key = a.key[lo];  // the chunk's first location continues the carried state
  uint32_t tests = 0, found = 0;
  for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
    const uint32_t p = b0 + lane;
    uint64_t k = ~0ull;
    uint32_t ix = 0, ep = 0, rw = 0, who = 0;
    if (p < hi) {
      k = a.key[p];
      ix = a.idx[p];
      const AccInfo inf = a.info[ix];
      ep = inf.epoch;
      rw = inf.row;
      who = inf.who;
    }
    // accesses that start a new location in this round, found once for all 32
    uint64_t kprev = __shfl_up_sync(0xffffffffu, k, 1);
    if (lane == 0) kprev = prev_key;
    const uint32_t starts = __ballot_sync(0xffffffffu, p < hi && k != kprev);
    prev_key = __shfl_sync(0xffffffffu, k, 31);
    const uint32_t nb = min(32u, hi - b0);
    for (uint32_t i = 0; i < nb; ++i) {
      if ((starts >> i) & 1u) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < K; ++j) last[q][j] = 0;
      }
      const uint32_t ib = __shfl_sync(0xffffffffu, ix, i);
      const uint32_t eb = __shfl_sync(0xffffffffu, ep, i);
      const uint32_t rowb = __shfl_sync(0xffffffffu, rw, i);
      const uint32_t wb = __shfl_sync(0xffffffffu, who, i);
      const uint32_t ub = who_agent(wb), cb = who_class(wb), bu = who_block(wb);
      const uint32_t m_diff = conflict_mask(cb, false), m_same = conflict_mask(cb, true);
      uint64_t best[K];
      bool any = false;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const uint32_t m = myblk[j] == bu ? m_same : m_diff;
        uint64_t b = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) b = ((m >> q) & 1u) ? max(b, last[q][j]) : b;
        best[j] = (lane * K + j == ub) ? 0 : b;
        any |= best[j] != 0;
      }
      bool race[K];
#pragma unroll
      for (int j = 0; j < K; ++j) race[j] = false;
      if (any) {
        uint32_t cv[K];
        const uint32_t* row = a.rows + size_t(rowb) * Wp + lane * K;
#pragma unroll
        for (int j = 0; j < K; ++j) cv[j] = __ldg(row + j);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          tests += best[j] != 0;
          race[j] = best[j] != 0 && uint32_t(best[j]) > cv[j];  // N(a*) > C_b[v]
        }
      }
      // emit (a*, b) pairs: one ballot per register slot, positions by popcount
      uint32_t cnt = 0, bal[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        bal[j] = __ballot_sync(0xffffffffu, race[j]);
        cnt += __popc(bal[j]);
      }
      found += cnt;
      if (cnt) {
        unsigned long long base = 0;
        if (lane == 0) {
          base = atomicAdd(&a.st->n_races, (unsigned long long)cnt);
          if (base == 0 && cnt) atomicCAS(&a.st->first_race_ns, 0ull, global_ns());  // the first races found
        }
        base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          if (race[j]) {
            const unsigned long long pos = base + __popc(bal[j] & lt);
            if (pos < a.race_cap) a.races[pos] = (uint64_t(ib) << 32) | (best[j] >> 32);
          }
          base += __popc(bal[j]);
        }
      }
      put_slot<K>(last, lane, ub, cb, (uint64_t(ib) << 32) | eb);
    }
  }
  tests = __reduce_add_sync(0xffffffffu, tests);
  if (lane == 0 && tests) atomicAdd(&a.st->partner_tests, (unsigned long long)tests);
  if (a.chunk_ns && lane == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    a.chunk_ns[c] = t;
    a.chunk_races[c] = found;
  }
}

inline uint32_t blocks(uint64_t n, uint32_t t) { return uint32_t((n + t - 1) / t); }

template <int K>
void run_carry(const ChunkArgs& a, uint64_t* gagg, uint32_t* gfull, cudaStream_t s, Prof& p) {
  const uint32_t nw = a.n_chunks;
  const uint32_t cols = 4 * a.g.Wp;
  const uint32_t ng = blocks(nw, GRP);
  p.begin("i_carry", double(nw) * cols * 8 * 3, s);
  k_tail<K><<<blocks(uint64_t(nw) * 32, CHK_WARPS * 32), CHK_WARPS * 32, 0, s>>>(a);
  count_launch();
  k_scan1<<<ng, 256, 0, s>>>(a, gagg, gfull);
  count_launch();
  k_scan2<<<blocks(cols, 256), 256, 0, s>>>(a, ng, gagg, gfull);
  count_launch();
  k_scan3<<<ng, 256, 0, s>>>(a, gagg);
  count_launch();
  p.end();
}

template <int K>
void run_check(const ChunkArgs& a, cudaStream_t s, Prof& p, double bytes_per) {
  const uint32_t nw = a.n_chunks;
  p.begin("i_check", double(a.n) * bytes_per, s);
  k_check<K><<<blocks(uint64_t(nw) * 32, CHK_WARPS * 32), CHK_WARPS * 32, 0, s>>>(a);
  count_launch();
  p.end();
}

}  // namespace

size_t check_chunks(uint32_t n_acc) { return (n_acc + CH - 1) / CH; }
size_t check_group_count(uint32_t n_acc) { return (check_chunks(n_acc) + GRP - 1) / GRP; }

void phaseH_sort(Bufs& b, const Geo& g, const Sizes& z, uint64_t key_mask, uint32_t* tmp, cudaStream_t s, Prof& p) {
  (void)g;
  p.begin("h_sort", double(z.n_acc) * 12 * 3 * radix_windows(key_mask).size(), s);
  RadixKeep keep;
  if (z.wl_log2) {  // the written-location filter of the grouped order, in the first pass
    keep.bits = b.wl_bits;
    keep.log2 = z.wl_log2;
    keep.shift = 15;
    keep.n_out = b.n_kept;
  }
  if (radix_sort_pairs(b.acc_key, b.acc_idx, b.acc_key2, b.acc_idx2, z.n_acc, key_mask, tmp, s, nullptr, keep)) {
    std::swap(b.acc_key, b.acc_key2);
    std::swap(b.acc_idx, b.acc_idx2);
  }
  p.end();
}

static ChunkArgs chunk_args(const Bufs& b, const Geo& g, const Sizes& z) {
  ChunkArgs a{};
  a.key = b.acc_key;
  a.idx = b.acc_idx;
  a.info = b.acc_info;
  a.n = z.n_acc;
  a.n_chunks = z.n_chunks;
  a.T = reinterpret_cast<uint64_t*>(b.tails);
  a.rows = b.rows;
  a.races = b.races;
  a.race_cap = z.race_cap;
  a.st = b.st;
  a.g = g;
  a.chunk_ns = b.chunk_ns;
  a.chunk_races = b.chunk_races;
  return a;
}

void phaseI_carry(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  if (!z.n_acc) return;
  const ChunkArgs a = chunk_args(b, g, z);
  uint64_t* gagg = a.T + size_t(z.n_chunks) * 4 * g.Wp;
  uint32_t* gfull = reinterpret_cast<uint32_t*>(gagg + size_t(check_group_count(z.n_acc)) * 4 * g.Wp);
  switch (g.K) {
    case 1: run_carry<1>(a, gagg, gfull, s, p); break;
    case 2: run_carry<2>(a, gagg, gfull, s, p); break;
    case 4: run_carry<4>(a, gagg, gfull, s, p); break;
    case 8: run_carry<8>(a, gagg, gfull, s, p); break;
    case 16: run_carry<16>(a, gagg, gfull, s, p); break;
    case 32: run_carry<32>(a, gagg, gfull, s, p); break;
  }
}

void phaseI_check(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  if (!z.n_acc) return;
  const ChunkArgs a = chunk_args(b, g, z);
  // per access: sorted key + index (12 B), its record (16 B), its clock-version row
  const double per = 12.0 + 16.0 + 4.0 * g.Wp;
  switch (g.K) {
    case 1: run_check<1>(a, s, p, per); break;
    case 2: run_check<2>(a, s, p, per); break;
    case 4: run_check<4>(a, s, p, per); break;
    case 8: run_check<8>(a, s, p, per); break;
    case 16: run_check<16>(a, s, p, per); break;
    case 32: run_check<32>(a, s, p, per); break;
  }
}

namespace {
__global__ void k_race_records(const uint64_t* w, uint64_t n, gwcp_race* out) {
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = gwcp_race{w[i] & 0xFFFFFFFFull, w[i] >> 32};
}
}  // namespace

void races_to_records(const uint64_t* words, uint64_t n, gwcp_race* out, cudaStream_t s) {
  if (!n) return;
  k_race_records<<<unsigned((n + 255) / 256), 256, 0, s>>>(words, n, out);
  count_launch();
}

bool phaseI_sort_races(const Bufs& b, const Sizes& z, uint64_t n_races, cudaStream_t s, Prof& p) {
  const uint64_t n = n_races < z.race_cap ? n_races : z.race_cap;
  if (n <= 1) return false;
  uint64_t mask = 0;
  for (uint64_t v = z.N; v; v >>= 1) mask = (mask << 1) | 1;
  mask |= mask << 32;
  p.begin("i_race_sort", double(n) * 8 * 2);
  bool second = radix_sort_pairs(b.races, nullptr, b.races2, nullptr, n, mask, b.scan_tmp, s);
  p.end();
  return second;
}

}  // namespace gwcp
