// Wide clocks (W > 1024 agents, up to 8192): clock propagation and race check over
// copy-on-write clock tiles.
//
// A clock of width W is cut into nT = ceil(W / 256) tiles of 256 u32 entries. Tiles live
// in one pool and are immutable once written; a clock is a table of nT tile ids (id 0 is
// the all-zero tile). A warp walks one agent as in the register-resident walker, but
// lane T holds the ids of tile T of P_t and H_t instead of the entries themselves. A join
// P_t |= X (Algorithms 1-2) compares ids tile by tile: an equal or zero tile costs
// nothing, a differing one is merged by the whole warp (8 entries per lane) and the
// result keeps an input's id when it equals that input, else it is written as a new
// tile. Clocks shared after a barrier or an acquire therefore share their tiles, and a
// clock version (the row the check reads) is a 128-byte table. A release snapshot is
// two tables. H_t[t] = N_t is kept implicit: the walker holds N_t in a register and the
// table's own entry may lag, so an increment copies no tile; the release snapshot of H_t
// writes the entry out (one tile copy), and a barrier raises every member's own entry to
// its local time while it joins the members' tables, as it does for C_t.
//
// Publication: a writer fences after writing new tiles and before storing a table that
// refers to them; tables are written once over SENTINEL words, so a reader accepts a
// table once none of its nT words is SENTINEL. All waits are bounded (GWCP_ERR_TIMEOUT).
// Pool exhaustion sets GWCP_ERR_OOM; the walker then keeps its old tile (the host grows
// the pool and runs the analysis again).
//
// The check for wide clocks enumerates partners per access instead of holding a W-wide
// table: accesses sorted by location are re-sorted stably by (location, class, agent);
// for access b every (class, agent) group of its location whose class conflicts with b
// is searched for its latest access before b, and an agent is tested once, against its
// latest conflicting non-exempt access a*: race iff N(a*) > C_b[v] (the paper's check).
#include <algorithm>

#include "gwcp_internal.cuh"

namespace gwcp {

namespace {

constexpr uint32_t kSpinLimitW = 1u << 23;
constexpr uint32_t SENT = 0xFFFFFFFFu;
enum : uint32_t { P_ACQ = 0, P_REL = 1, P_BAR = 2, P_INCS = 3 };
enum : uint32_t { BAR_SINGLE = 0, BAR_CTA = 1, BAR_GLOBAL = 2 };

struct WideArgs {
  Geo g;
  DevStatus* st;
  const uint32_t *sy_start, *incs_off, *rowbase;
  const uint4* plan;
  const uint4* recmeta;
  const uint32_t *pool, *flat;
  uint32_t *rows, *psnap, *hsnap, *jsnap, *cursor;
  uint32_t* tiles;
  unsigned long long* tile_ctr;
  unsigned long long tile_cap;
  uint32_t n_locks;
  uint32_t hb_only;  // publish H_t instead of P_t as the clock versions
};

__device__ __forceinline__ uint4 max4(uint4 x, uint4 y) {
  return make_uint4(max(x.x, y.x), max(x.y, y.y), max(x.z, y.z), max(x.w, y.w));
}
__device__ __forceinline__ bool eq4(uint4 x, uint4 y) { return x.x == y.x && x.y == y.y && x.z == y.z && x.w == y.w; }

// Tiles are immutable once written and a tile id becomes known to a walker only through a
// table published after the tile (or through its own CTA after a barrier), so no L1 line
// can hold a tile's address before the tile is written (L1 starts clean each launch):
// tile reads may go through L1, and a merge first prefetches every tile it will read.
__device__ __forceinline__ void prefetch_tile(const WideArgs& a, uint32_t id) {
  const char* p = reinterpret_cast<const char*>(a.tiles + size_t(id) * kTileW);
#pragma unroll
  for (int q = 0; q < 8; ++q) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + q * 128));
}
// the tiles a merge of `src` into the table `my` will read (lane T: tile T of each)
__device__ __forceinline__ void prefetch_merge(const WideArgs& a, uint32_t my, uint32_t src) {
  if ((threadIdx.x & 31) < int(a.g.nT) && src != 0 && src != my && my != 0) {
    prefetch_tile(a, my);
    prefetch_tile(a, src);
  }
}

__device__ __forceinline__ const uint4* tile_src(const WideArgs& a, uint32_t id) {
  return reinterpret_cast<const uint4*>(a.tiles + size_t(id) * kTileW) + (threadIdx.x & 31) * 2;
}
__device__ __forceinline__ uint4* tile_dst(const WideArgs& a, uint32_t id) {
  return reinterpret_cast<uint4*>(a.tiles + size_t(id) * kTileW) + (threadIdx.x & 31) * 2;
}

// A lane holds 8 consecutive entries of a tile as (x0, x1). These update entry c (0..7)
// with register selects only, so the pair is never addressed through memory.
__device__ __forceinline__ uint32_t sel_raise(uint32_t x, bool hit, uint32_t val, bool& up) {
  const bool h = hit && x < val;
  up |= h;
  return h ? val : x;
}
__device__ __forceinline__ bool raise8(uint4& x0, uint4& x1, uint32_t c, uint32_t val) {
  bool up = false;
  x0.x = sel_raise(x0.x, c == 0, val, up);
  x0.y = sel_raise(x0.y, c == 1, val, up);
  x0.z = sel_raise(x0.z, c == 2, val, up);
  x0.w = sel_raise(x0.w, c == 3, val, up);
  x1.x = sel_raise(x1.x, c == 4, val, up);
  x1.y = sel_raise(x1.y, c == 5, val, up);
  x1.z = sel_raise(x1.z, c == 6, val, up);
  x1.w = sel_raise(x1.w, c == 7, val, up);
  return up;
}
__device__ __forceinline__ void set8(uint4& x0, uint4& x1, uint32_t c, uint32_t val) {
  x0.x = c == 0 ? val : x0.x;
  x0.y = c == 1 ? val : x0.y;
  x0.z = c == 2 ? val : x0.z;
  x0.w = c == 3 ? val : x0.w;
  x1.x = c == 4 ? val : x1.x;
  x1.y = c == 5 ? val : x1.y;
  x1.z = c == 6 ? val : x1.z;
  x1.w = c == 7 ? val : x1.w;
}

// Tile ids are handed to each warp kTileChunk at a time (one atomic per chunk instead of
// one per tile on a single counter); the warp-uniform state lives in the walker.
constexpr uint32_t kTileChunk = 8;
struct TileAlloc {
  uint32_t next = 0, end = 0;  // ids [next, end) are the warp's; both clamped to the pool size
  uint32_t* cnt = nullptr;     // shared words: tiles read, tiles written (lane 0 adds)
  __device__ __forceinline__ void count(uint32_t rd, uint32_t wr) const {
    if ((threadIdx.x & 31) == 0) {
      cnt[0] += rd;
      cnt[1] += wr;
    }
  }
};

// a fresh tile id (warp-uniform); 0 when the pool is exhausted (GWCP_ERR_OOM set)
__device__ __forceinline__ uint32_t alloc_tile(const WideArgs& a, TileAlloc& ta) {
  if (ta.next == ta.end) {
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(a.tile_ctr, (unsigned long long)kTileChunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    ta.next = uint32_t(min(base, a.tile_cap));
    ta.end = uint32_t(min(base + kTileChunk, a.tile_cap));
    if (ta.next == ta.end) {
      if ((threadIdx.x & 31) == 0) atomicCAS(&a.st->code, 0, GWCP_ERR_OOM);
      return 0;
    }
  }
  return ta.next++;
}

// my |= src, tile by tile (lane T < nT holds the ids of tile T)
__device__ __noinline__ void merge_table(const WideArgs& a, uint32_t& my, uint32_t src, bool& dirty, TileAlloc& ta) {
  const int lane = threadIdx.x & 31;
  bool need = lane < int(a.g.nT) && src != 0 && src != my;
  if (need && my == 0) {
    my = src;
    need = false;
  }
  if (need) {
    prefetch_tile(a, my);
    prefetch_tile(a, src);
  }
  uint32_t m = __ballot_sync(0xffffffffu, need);
  while (m) {
    const int T = __ffs(m) - 1;
    m &= m - 1;
    const uint32_t ia = __shfl_sync(0xffffffffu, my, T), ib = __shfl_sync(0xffffffffu, src, T);
    const uint4* pa = tile_src(a, ia);
    const uint4* pb = tile_src(a, ib);
    const uint4 x0 = __ldca(pa), x1 = __ldca(pa + 1), y0 = __ldca(pb), y1 = __ldca(pb + 1);
    const uint4 r0 = max4(x0, y0), r1 = max4(x1, y1);
    uint32_t nid;
    if (__all_sync(0xffffffffu, eq4(r0, x0) && eq4(r1, x1))) {
      nid = ia;
      ta.count(2, 0);
    } else if (__all_sync(0xffffffffu, eq4(r0, y0) && eq4(r1, y1))) {
      nid = ib;
      ta.count(2, 0);
    } else {
      nid = alloc_tile(a, ta);
      ta.count(2, 1);
      if (nid) {
        uint4* d = tile_dst(a, nid);
        d[0] = r0;
        d[1] = r1;
        dirty = true;
      } else {
        nid = ia;
      }
    }
    if (lane == T) my = nid;
  }
}

// copy of tile `id` with entry e set to val; returns the new id (warp-uniform)
__device__ __forceinline__ uint32_t cow_set(const WideArgs& a, uint32_t id, uint32_t e, uint32_t val, bool& dirty, TileAlloc& ta) {
  const int lane = threadIdx.x & 31;
  const uint4* p = tile_src(a, id);
  uint4 x0 = __ldca(p), x1 = __ldca(p + 1);
  if (lane == int(e >> 3)) set8(x0, x1, e & 7, val);
  const uint32_t nid = alloc_tile(a, ta);
  ta.count(1, 1);
  if (!nid) return id;
  uint4* d = tile_dst(a, nid);
  d[0] = x0;
  d[1] = x1;
  dirty = true;
  return nid;
}

// entry t of the table held by the warp := val (copy of the tile holding t)
__device__ __forceinline__ void set_entry_w(const WideArgs& a, uint32_t& my, uint32_t t, uint32_t val, bool& dirty,
                                            TileAlloc& ta) {
  const uint32_t T = t / kTileW;
  const uint32_t id = __shfl_sync(0xffffffffu, my, T);
  const uint32_t nid = cow_set(a, id, t % kTileW, val, dirty, ta);
  if ((threadIdx.x & 31) == int(T)) my = nid;
}

// a published table: wait (bounded) until none of its nT words is SENTINEL
__device__ __forceinline__ uint32_t read_table(const WideArgs& a, const uint32_t* tab, bool& abort) {
  const int lane = threadIdx.x & 31;
  const bool act = lane < int(a.g.nT);
  uint32_t v = act ? __ldcg(tab + lane) : 0;
  if (__all_sync(0xffffffffu, v != SENT)) return v;
  uint32_t it = 0;
  while (!abort) {
    __nanosleep(64);
    v = act ? __ldcg(tab + lane) : 0;
    if (__all_sync(0xffffffffu, v != SENT)) return v;
    if (++it > kSpinLimitW) {
      if (lane == 0) atomicCAS(&a.st->code, 0, GWCP_ERR_TIMEOUT);
      abort = true;
    }
  }
  return v == SENT ? 0u : v;
}

__device__ __forceinline__ void publish(const WideArgs& a, uint32_t* tab, uint32_t id, bool& dirty) {
  if (dirty) __threadfence();  // the tiles this warp wrote are visible before the table is
  dirty = false;
  if ((threadIdx.x & 31) < int(a.g.nT)) __stcg(tab + (threadIdx.x & 31), id);
}

__device__ __forceinline__ uint32_t entry_of(const WideArgs& a, uint32_t my, uint32_t t) {
  // entry t of the warp's table, 0 for t >= W; every lane may ask for a different t.
  // All lanes take part in the shuffle.
  const bool ok = t < a.g.W;
  const uint32_t id = __shfl_sync(0xffffffffu, my, ok ? int(t / kTileW) : 0);
  return ok ? __ldcg(a.tiles + size_t(id) * kTileW + t % kTileW) : 0u;
}

// Join of one tile over a CTA's members (lane m holds member m's id for the tile), with
// the members' own entries raised to their local times (C_m[u_m] = N_m; H_m[u_m] = N_m,
// which the walker keeps implicit). One pass over the distinct input tiles keeps the
// running maximum and which input equals it so far (an input equals the final maximum
// iff it is >= every other input); the result keeps that input's id when the own
// entries raise nothing, else it is written as a new tile.
__device__ __noinline__ uint32_t join_members(const WideArgs& a, uint32_t idm, uint32_t nm, uint32_t apb, uint32_t first,
                                 uint32_t T, bool own, bool& dirty, TileAlloc& ta) {
  const int lane = threadIdx.x & 31;
  const bool act = uint32_t(lane) < apb && idm != 0;
  const uint32_t same = __match_any_sync(0xffffffffu, act ? idm : 0xFFFFFFFFu);
  const uint32_t leaders = __ballot_sync(0xffffffffu, act && (__ffs(same) - 1) == lane);
  // members whose own entry lies in tile T
  const uint32_t lo = T * kTileW, hi = lo + kTileW;
  const bool own_here = own && uint32_t(lane) < apb && first + lane >= lo && first + lane < hi;
  const uint32_t ovm = __ballot_sync(0xffffffffu, own_here);
  if (!ovm && __popc(leaders) <= 1) return leaders ? __shfl_sync(0xffffffffu, idm, __ffs(leaders) - 1) : 0u;
  uint4 r0 = make_uint4(0, 0, 0, 0), r1 = r0;
  bool have = leaders == 0;  // no input: the zero tile (id 0) equals the maximum so far
  uint32_t cid = 0;          // id of an input equal to the maximum so far (when have)
  for (uint32_t m = leaders; m; m &= m - 1) {
    const uint32_t id = __shfl_sync(0xffffffffu, idm, __ffs(m) - 1);
    const uint4* p = tile_src(a, id);
    const uint4 x0 = __ldca(p), x1 = __ldca(p + 1);
    const bool le = __all_sync(0xffffffffu, eq4(max4(r0, x0), r0) && eq4(max4(r1, x1), r1));  // x <= r
    const bool ge = __all_sync(0xffffffffu, eq4(max4(r0, x0), x0) && eq4(max4(r1, x1), x1));  // x >= r
    r0 = max4(r0, x0);
    r1 = max4(r1, x1);
    if (!(le && have)) cid = id;
    have = (le && have) || ge;
  }
  bool raised = false;
  for (uint32_t m = ovm; m; m &= m - 1) {
    const int mm = __ffs(m) - 1;
    const uint32_t e = first + mm - lo, val = __shfl_sync(0xffffffffu, nm, mm);
    if (lane == int(e >> 3)) raised |= raise8(r0, r1, e & 7, val);
  }
  const bool keep = have && !__any_sync(0xffffffffu, raised);
  ta.count(__popc(leaders), keep ? 0u : 1u);
  if (keep) return cid;
  const uint32_t nid = alloc_tile(a, ta);
  if (!nid) return leaders ? __shfl_sync(0xffffffffu, idm, __ffs(leaders) - 1) : 0u;
  uint4* d = tile_dst(a, nid);
  d[0] = r0;
  d[1] = r1;
  dirty = true;
  return nid;
}

// One warp per agent, one CTA per block of the traced program (agents_per_block <= 32).
// MINB = CTAs of 1024 threads that must share an SM for all blocks to be co-resident.
template <int MINB>
__global__ void __launch_bounds__(1024, MINB) k_prop_wide(WideArgs a) {
  extern __shared__ uint32_t sm[];
  const Geo& g = a.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t apb = g.apb;
  const uint32_t first = blockIdx.x * apb;
  const uint32_t u = first + warp;
  uint32_t* tabs = sm;                  // [apb][3][32] member tables (P, H, JN)
  uint32_t* nbuf = sm + apb * 96;       // [apb] member epochs
  uint32_t* J = nbuf + 32;              // [3][32] joined tables
  uint32_t* tcnt = J + 96 + warp * 2;   // [apb][2] tiles this warp read and wrote (lane 0 counts)
  __shared__ int start_code;
  if (threadIdx.x == 0) start_code = *(volatile int*)&a.st->code;
  __syncthreads();
  if (start_code) return;
  const bool act = lane < int(g.nT);
  bool dirty = false, abort = false;
  TileAlloc ta;
  ta.cnt = tcnt;
  if (lane == 0) tcnt[0] = tcnt[1] = 0;
  // H_t = bottom{t := 1}: the table starts at bottom and H_t[t] = N_t is kept implicit (in
  // N), so no tile is copied when it increments; a release snapshot writes it out
  // JN_t (jid): the join of every H snapshot joined into P_t, carried along with P_t (joined
  // at acquires from the lock's published JN, at barriers over the members). H moves only by
  // whole-clock joins, so JN_t[v] >= e means P_t already holds the H snapshot of v's release
  // at epoch e: such a join (release loop, in-section access) changes nothing and is skipped.
  uint32_t pid = 0, hid = 0, jid = 0;
  uint32_t N = 1;
  unsigned long long joins = 0, visits = 0;
  if (act) a.rows[size_t(a.rowbase[u]) * kTabW + lane] = a.hb_only ? hid : 0u;
  const uint32_t k0 = a.sy_start[u], k1 = a.sy_start[u + 1];
  const uint32_t pb = k0 + a.incs_off[k0], pe = k1 + a.incs_off[k1];
  uint32_t* const cursor_row = a.cursor + size_t(u) * a.n_locks;
  uint4 na = make_uint4(0, 0, 0, 0), nb = na;
  if (pb < pe) {
    na = a.plan[2 * size_t(pb)];
    nb = a.plan[2 * size_t(pb) + 1];
  }
  for (uint32_t p = pb; p < pe; ++p) {
    const uint4 ea = na, eb = nb;
    if (p + 1 < pe) {  // the next entry's loads overlap this one
      na = a.plan[2 * size_t(p + 1)];
      nb = a.plan[2 * size_t(p + 1) + 1];
    }
    const uint32_t t = ea.x & 0xFF, row = ea.y;
    if (t == P_ACQ || t == P_INCS) {
      // acquire: P_t |= P_<l,s'>, H_t |= H_<l,s'>; in-section access: P_t |= L^w (| L^r)
      const uint32_t off = ea.z, w = ea.w;
      const uint32_t* list = t == P_ACQ ? a.pool : a.flat;
      for (uint32_t q = 0; q < w; ++q) {
        uint32_t x;
        if (w <= 4)
          x = q == 0 ? eb.x : q == 1 ? eb.y : q == 2 ? eb.z : eb.w;
        else
          x = __ldcg(list + off + q);
        if (t == P_ACQ) {
          // the three published tables are loaded together (a table still being written is
          // then waited for), and every tile the three merges read is prefetched first
          uint32_t sp = lane < int(g.nT) ? __ldcg(a.psnap + size_t(x) * kTabW + lane) : 0;
          uint32_t sh = lane < int(g.nT) ? __ldcg(a.hsnap + size_t(x) * kTabW + lane) : 0;
          uint32_t sj = lane < int(g.nT) ? __ldcg(a.jsnap + size_t(x) * kTabW + lane) : 0;
          if (!__all_sync(0xffffffffu, sp != SENT && sh != SENT && sj != SENT)) {
            sp = read_table(a, a.psnap + size_t(x) * kTabW, abort);
            sh = read_table(a, a.hsnap + size_t(x) * kTabW, abort);
            sj = read_table(a, a.jsnap + size_t(x) * kTabW, abort);
          }
          prefetch_merge(a, hid, sh);
          prefetch_merge(a, jid, sj);
          merge_table(a, pid, sp, dirty, ta);
          merge_table(a, hid, sh, dirty, ta);
          merge_table(a, jid, sj, dirty, ta);
          joins += 2;
        } else {
          // L^w / L^r: the H snapshot of section x's release, unless JN_t already covers it
          const uint4 mx = __ldg(a.recmeta + x);
          if (entry_of(a, jid, mx.x & 0xFFFF) < mx.w) {
            const uint32_t sx = read_table(a, a.hsnap + size_t(x) * kTabW, abort);
            prefetch_merge(a, jid, sx);
            merge_table(a, pid, sx, dirty, ta);
            merge_table(a, jid, sx, dirty, ta);
            joins += 1;
          }
        }
      }
    } else if (t == P_REL) {
      // release: pop other agents' records on this lock while their acquire is ordered
      // before C_t, joining the released ones whose scope overlaps; then publish
      const uint32_t c = ea.z, L = ea.w;
      const uint32_t lo = eb.x, hi = eb.y, s = eb.z, my_idx = eb.w;
      uint32_t cur = __ldcg(cursor_row + L);
      bool stop = false;
      while (!stop && lo + cur < hi) {
        const uint32_t rec = lo + cur + lane;
        const uint32_t nbr = min(32u, hi - (lo + cur));
        uint4 m = make_uint4(NONE, 0, NONE, 0);
        if (rec < hi) m = __ldg(a.recmeta + rec);
        const uint32_t mag = m.x == NONE ? NONE : (m.x & 0xFFFF);
        const uint32_t msid = m.x >> 16;
        const bool mine = mag == u;
        const bool joinable = !mine && m.z != NONE && m.z < my_idx && scopes_overlap(msid, s);
        uint32_t start = 0;
        uint32_t pv = entry_of(a, pid, mag), jv = entry_of(a, jid, mag);
        while (start < nbr) {
          const bool in = uint32_t(lane) >= start && uint32_t(lane) < nbr;
          const uint32_t fail = __ballot_sync(0xffffffffu, in && !mine && m.y > pv);
          const uint32_t f = fail ? uint32_t(__ffs(fail) - 1) : nbr;
          const uint32_t popped = __ballot_sync(0xffffffffu, in && uint32_t(lane) < f && joinable);
          // join only releases not already in P, and of one agent's popped records only the
          // latest (records of one agent are in acquire order, so its H dominates)
          const bool cand = ((popped >> lane) & 1u) && m.w > jv;
          const uint32_t same = __match_any_sync(0xffffffffu, cand ? mag : 0xFFFFFFFFu);
          const uint32_t wave = __ballot_sync(0xffffffffu, cand && (same >> lane) <= 1u);
          visits += __popc(__ballot_sync(0xffffffffu, in && uint32_t(lane) <= f && !mine));
          for (uint32_t wm = wave; wm; wm &= wm - 1) {
            const uint32_t r = lo + cur + (__ffs(wm) - 1);
            const uint32_t sx = read_table(a, a.hsnap + size_t(r) * kTabW, abort);
            prefetch_merge(a, jid, sx);
            merge_table(a, pid, sx, dirty, ta);
            merge_table(a, jid, sx, dirty, ta);
            ++joins;
          }
          if (f == nbr) {
            start = nbr;
          } else if (wave) {
            start = f;  // P grew: test the failing record again
            pv = entry_of(a, pid, mag);
            jv = entry_of(a, jid, mag);
          } else {
            stop = true;  // P unchanged: the record stays unordered
            start = f;
            break;
          }
        }
        cur += start;
      }
      if (lane == 0) __stcg(cursor_row + L, cur);
      uint32_t hp = hid;  // the snapshot of H_t carries its own entry N_t
      set_entry_w(a, hp, u, N, dirty, ta);
      publish(a, a.psnap + size_t(c) * kTabW, pid, dirty);
      publish(a, a.hsnap + size_t(c) * kTabW, hp, dirty);
      publish(a, a.jsnap + size_t(c) * kTabW, jid, dirty);
      ++N;  // H_t[t] = N_t, implicit
    } else {
      // barrier: C and H joined over the members
      const uint32_t mode = eb.x;
      if (eb.y != N) N = eb.y;  // forced compression at barriers: enter with the members' highest N
      if (mode == BAR_SINGLE) {
        set_entry_w(a, pid, u, N, dirty, ta);  // P_t = C_t
      } else {
        if (act) {
          tabs[(warp * 3) * 32 + lane] = pid;
          tabs[(warp * 3 + 1) * 32 + lane] = hid;
          tabs[(warp * 3 + 2) * 32 + lane] = jid;
        }
        if (lane == 0) nbuf[warp] = N;
        __syncthreads();
        const uint32_t nw = blockDim.x >> 5;
        bool wrote = false;
        for (uint32_t T = warp; T < g.nT; T += nw) {
          const bool mem = uint32_t(lane) < apb;
          const uint32_t cm = mem ? tabs[(lane * 3) * 32 + T] : 0, hm = mem ? tabs[(lane * 3 + 1) * 32 + T] : 0;
          const uint32_t jm = mem ? tabs[(lane * 3 + 2) * 32 + T] : 0;
          const uint32_t nm = mem ? nbuf[lane] : 0;
          if (cm) prefetch_tile(a, cm);
          if (hm) prefetch_tile(a, hm);
          if (jm) prefetch_tile(a, jm);
          const uint32_t jc = join_members(a, cm, nm, apb, first, T, true, wrote, ta);
          const uint32_t jh = join_members(a, hm, nm, apb, first, T, true, wrote, ta);
          const uint32_t jj = join_members(a, jm, nm, apb, first, T, false, wrote, ta);
          if (lane == 0) {
            J[T] = jc;
            J[32 + T] = jh;
            J[64 + T] = jj;
          }
        }
        if (wrote) __threadfence();  // members may publish the joined tiles at once
        __syncthreads();
        pid = act ? J[lane] : 0;
        hid = act ? J[32 + lane] : 0;
        jid = act ? J[64 + lane] : 0;
        joins += 2;  // this member's C_t and H_t joined into the block's
        // J is rewritten only after the next barrier's first __syncthreads, which every
        // member reaches after reading it here
      }
      ++N;  // H_t[t] = N_t, implicit
    }
    if (act) a.rows[size_t(row) * kTabW + lane] = a.hb_only ? hid : pid;
  }
  if (dirty) __threadfence();
  if (lane == 0) {
    atomicAdd(&a.st->joins, joins);
    atomicAdd(&a.st->loop_visits, visits);
    atomicAdd(&a.st->tiles_read, (unsigned long long)tcnt[0]);
    atomicAdd(&a.st->tiles_written, (unsigned long long)tcnt[1]);
  }
}

// ---- check ---------------------------------------------------------------------------

__global__ void k_wc_runflags(const uint64_t* key, uint32_t n, uint32_t* flag) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) flag[p] = (p == 0 || key[p] != key[p - 1]) ? 1u : 0u;
}

// composite key (run, class, agent) for the stable regrouping; value = key-order position
// composite keys (run, class, agent) of the key-ordered accesses; also the fields of each
// access record the check needs, copied into key order (a sequential read for the check
// instead of a gather by trace index)
__global__ void k_wc_compose(const uint32_t* run_excl, const uint32_t* flag, const uint32_t* idx,
                             const AccInfo* info, uint32_t n, uint64_t* ck, uint32_t* cv, uint32_t* s_who,
                             uint32_t* s_row, uint32_t* s_ep) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t run = run_excl[p] + flag[p] - 1;
  const AccInfo in = info[idx[p]];
  ck[p] = (uint64_t(run) << 15) | (uint64_t(who_class(in.who)) << 13) | who_agent(in.who);
  cv[p] = p;
  s_who[p] = in.who;
  s_row[p] = in.row;
  s_ep[p] = in.epoch;
}

// A location that no write-class access touches has no races (two reads never conflict):
// its accesses are left out of the regrouping, so the check finds no partner groups there.
__global__ void k_wc_runwrite(const uint64_t* ck, uint32_t n, uint32_t* run_w) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && ((ck[p] >> 13) & 3u) != C_READ) run_w[ck[p] >> 15] = 1u;
}
__global__ void k_wc_keep(const uint64_t* ck, uint32_t n, const uint32_t* run_w, uint32_t* keep) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) keep[p] = run_w[ck[p] >> 15];
}
__global__ void k_wc_compact(const uint64_t* ck, const uint32_t* cv, const uint32_t* keep, const uint32_t* kpos,
                             uint32_t n, uint64_t* ck2, uint32_t* cv2) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && keep[p]) {
    ck2[kpos[p]] = ck[p];
    cv2[kpos[p]] = cv[p];
  }
}

// group starts over the sorted composite keys (the first *n_dev of n), and per (run, class)
// group counts
__global__ void k_wc_groupflags(const uint64_t* ck, uint32_t n, const uint32_t* n_dev, uint32_t* gflag) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) gflag[i] = (i < *n_dev && (i == 0 || ck[i] != ck[i - 1])) ? 1u : 0u;
}

__global__ void k_wc_groups(const uint64_t* ck, const uint32_t* gflag, const uint32_t* gexcl, uint32_t n,
                            uint32_t* grp_lo, uint32_t* grp_agent, uint32_t* rc_cnt) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !gflag[i]) return;
  const uint32_t gi = gexcl[i];
  grp_lo[gi] = i;
  grp_agent[gi] = uint32_t(ck[i] & 0x1FFF);
  atomicAdd(rc_cnt + (ck[i] >> 13), 1u);  // (run << 2 | class)
}

struct WideCheckArgs {
  Geo g;
  uint32_t n;
  const uint32_t* n_dev;     // the count on the device (at most n), or null
  const uint32_t* idx;       // key order -> trace index
  const uint32_t* flag;      // run starts
  const uint32_t* run_excl;  // exclusive scan of flag
  const uint32_t* gs;        // grouped order -> key-order position (grouped: the trace index itself)
  uint32_t grouped;          // the primary order is the grouped order (compare trace indices)
  const uint32_t* grp_lo;    // [n_groups + 1]
  const uint32_t* grp_agent;
  const uint32_t* rc_off;    // [(run << 2 | class) + 1]
  const AccInfo* info;
  const uint32_t *s_who, *s_row, *s_ep;  // record fields in key order
  const uint32_t* rows;
  const uint32_t* tiles;
  unsigned long long tile_cap;  // ids at or above it (rows a failed walk left stale) read as zero
  uint64_t* races;
  unsigned long long race_cap;
  DevStatus* st;
  uint32_t dense_wp;             // 0: clocks are tile tables; else dense rows of this many words
  const uint32_t* cv_pool;       // non-null: compressed versions (rows holds B headers each)
  unsigned long long cv_cap;
  uint32_t row_words;            // words per entry of rows
  unsigned long long* chunk_ns;  // optional timeline: globaltimer at each block's end
  uint32_t* chunk_races;         // and the races it found
};

// position j in group gi of the latest member with gs[j] < x (gs ascends within a group:
// key-order positions, or trace indices in the grouped order), or NONE
__device__ __forceinline__ uint32_t pred_in_group(const WideCheckArgs& a, uint32_t gi, uint32_t x) {
  uint32_t lo = a.grp_lo[gi], hi = a.grp_lo[gi + 1];
  if (lo == hi || a.gs[lo] >= x) return NONE;
  while (hi - lo > 1) {  // invariant: gs[lo] < x, and gs[hi] >= x or hi is the end
    const uint32_t mid = (lo + hi) >> 1;
    if (a.gs[mid] < x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// classes a later access of class cb conflicts with and is not exempt from (bit q = class
// q), given whether the partner shares b's block
__device__ __forceinline__ uint32_t conflict_classes(uint32_t cb, bool same_block) {
  switch (cb) {
    case C_READ: return 0b1110;
    case C_WRITE: return 0b1111;
    case C_ATOM_CTA: return same_block ? 0b0011 : 0b0111;
    default: return 0b0011;
  }
}

// Races found by a warp are staged in shared memory and appended with one global atomic
// per warp; a warp that finds more than kRaceStage spills the rest with one atomic each.
// Per warp, not per block: the threads of an access at a hot location search many more
// partner groups than the rest, and a block-wide append would hold every warp of the
// block until its slowest thread is done.
constexpr uint32_t kRaceStage = 256;
constexpr uint32_t kCheckThreads = 256;

__device__ __forceinline__ void emit_race(const WideCheckArgs& a, uint64_t v, uint32_t* s_cnt, uint64_t* s_buf) {
  const uint32_t slot = atomicAdd(s_cnt, 1u);
  if (slot == 0) atomicCAS(&a.st->first_race_ns, 0ull, global_ns());  // the warp's first race: the earliest
                                                                       // stamp wins
  if (slot < kRaceStage) {
    s_buf[slot] = v;
    return;
  }
  const unsigned long long at = atomicAdd(&a.st->n_races, 1ull);
  if (at < a.race_cap) a.races[at] = v;
}

// partner tests of the access at key-order position p; returns how many were made
// REP: how the clock versions are held (one instantiation each, so that the common
// representations keep their registers and occupancy)
enum : int { REP_TILES = 0, REP_DENSE = 1, REP_COMPRESSED = 2 };

template <int REP>
__device__ uint32_t check_one(const WideCheckArgs& a, uint32_t p, uint32_t* s_cnt, uint64_t* s_buf) {
  const uint32_t b = a.idx[p];
  const uint32_t bwho = a.s_who[p];
  const uint32_t u = who_agent(bwho), cb = who_class(bwho), bu = who_block(bwho);
  const uint32_t run = a.run_excl[p] + a.flag[p] - 1;
  const uint32_t* rowtab = a.rows + size_t(a.s_row[p]) * a.row_words;
  const uint32_t any_mask = conflict_classes(cb, false) | conflict_classes(cb, true);
  const uint32_t x = a.grouped ? b : p;  // "earlier than b" in the order gs holds
  uint32_t tests = 0;
  // The location's groups of each class are sorted by agent: walk the classes' lists
  // together (a merge by agent), so that each agent is handled once, from the class
  // holding its latest conflicting access before b (ties: the lower class).
  uint32_t cur[4], end[4];
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    const bool on = (any_mask >> q) & 1u;
    cur[q] = on ? a.rc_off[(run << 2) | q] : 0u;
    end[q] = on ? a.rc_off[((run << 2) | q) + 1] : 0u;
  }
  for (;;) {
    uint32_t v = NONE;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q)
      if (cur[q] < end[q]) v = min(v, a.grp_agent[cur[q]]);
    if (v == NONE) break;
    const uint32_t cm = conflict_classes(cb, v / a.g.apb == bu);
    uint32_t j = NONE, pos = NONE;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      if (cur[q] >= end[q] || a.grp_agent[cur[q]] != v) continue;
      const uint32_t gi = cur[q]++;
      if (v == u || !((cm >> q) & 1u)) continue;
      const uint32_t jq = pred_in_group(a, gi, x);
      if (jq == NONE) continue;
      const uint32_t pq = a.gs[jq];
      if (pos == NONE || pq > pos) {
        pos = pq;
        j = jq;
      }
    }
    if (pos == NONE) continue;
    {
      ++tests;
      const uint32_t qa = a.grouped ? j : pos;  // a*'s position in the primary order
      const uint32_t ai = a.idx[qa];
      const uint32_t na = a.s_ep[qa];
      uint32_t cv;
      if constexpr (REP == REP_COMPRESSED) {
        cv = cv_entry(rowtab, a.cv_pool, a.cv_cap, v, a.g.apb, cv_group(a.g.gran));
      } else if constexpr (REP == REP_DENSE) {
        cv = __ldg(rowtab + v);
      } else {
        const uint32_t tid = __ldg(rowtab + v / kTileW);
        cv = tid < a.tile_cap ? __ldg(a.tiles + size_t(tid) * kTileW + v % kTileW) : 0u;
      }
      if (na > cv) emit_race(a, (uint64_t(b) << 32) | ai, s_cnt, s_buf);  // N(a*) > C_b[v]
    }
  }
  return tests;
}

template <int REP>
__global__ void __launch_bounds__(kCheckThreads, 8) k_wc_check(WideCheckArgs a) {
  constexpr uint32_t kWarps = kCheckThreads / 32;
  __shared__ uint32_t s_cnt[kWarps];
  __shared__ uint64_t s_buf[kWarps][kRaceStage];
  __shared__ uint32_t s_done, s_found;  // timeline: warps finished, races found by the block
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_cnt[warp] = 0;
  if (threadIdx.x == 0) s_done = s_found = 0;
  __syncthreads();
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n_eff = a.n_dev ? min(a.n, *a.n_dev) : a.n;
  uint32_t tests = 0;
  if (p < n_eff) tests = check_one<REP>(a, p, &s_cnt[warp], s_buf[warp]);
  tests = __reduce_add_sync(0xffffffffu, tests);
  __syncwarp();
  const uint32_t found = s_cnt[warp];
  const uint32_t n = min(found, kRaceStage);
  unsigned long long base = 0;
  if (lane == 0) {
    if (tests) atomicAdd(&a.st->partner_tests, (unsigned long long)tests);
    if (n) base = atomicAdd(&a.st->n_races, (unsigned long long)n);
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  for (uint32_t i = lane; i < n; i += 32)
    if (base + i < a.race_cap) a.races[base + i] = s_buf[warp][i];
  if (a.chunk_ns && lane == 0) {  // the block's last warp stamps the block's end
    atomicAdd(&s_found, found);
    __threadfence_block();
    if (atomicAdd(&s_done, 1u) == kWarps - 1) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      a.chunk_ns[blockIdx.x] = t;
      a.chunk_races[blockIdx.x] = atomicAdd(&s_found, 0u);
    }
  }
}

// ---- grouped order: the accesses sorted once by (location, class, agent, trace index) ----
// Before the sort, the accesses of locations without a write-class access are left out
// (two reads never race): the sort's first pass keeps only those whose location's bit is
// set in the hashed bitmap that the decoding pass filled from the write-class accesses. A
// bit shared with a written location keeps a few read-only locations; they have no partners.

// location runs and (class, agent) groups of the composite keys (the first *n_dev keys)
__global__ void k_gr_flags(const uint64_t* ck, uint32_t n, const uint32_t* n_dev, uint32_t* run_flag,
                           uint32_t* grp_flag) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (p >= *n_dev) {
    run_flag[p] = 0;
    grp_flag[p] = 0;
    return;
  }
  run_flag[p] = (p == 0 || (ck[p] >> 15) != (ck[p - 1] >> 15)) ? 1u : 0u;
  grp_flag[p] = (p == 0 || ck[p] != ck[p - 1]) ? 1u : 0u;
}

// The groups ascend by (run, class, agent); rc_off[(run << 2) | q] is the first group whose
// (run, class) slot is >= (run, q). The first group of a slot writes it and the empty slots
// before it; the last access writes the slots after the last group (up to 4 * runs).
__global__ void k_gr_groups(const uint64_t* ck, const uint32_t* run_flag, const uint32_t* run_excl,
                            const uint32_t* gflag, const uint32_t* gexcl, const uint32_t* n_dev, uint32_t* grp_lo,
                            uint32_t* grp_agent, uint32_t* rc_off) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = *n_dev;
  if (i >= n) return;
  const uint32_t run = run_excl[i] + run_flag[i] - 1;
  const uint32_t slot = (run << 2) | uint32_t((ck[i] >> 13) & 3u);
  if (i == n - 1) {
    const uint32_t n_groups = gexcl[i] + gflag[i];
    grp_lo[n_groups] = n;
    for (uint32_t t = slot + 1; t <= (run << 2) + 4; ++t) rc_off[t] = n_groups;
  }
  if (!gflag[i]) return;
  const uint32_t gi = gexcl[i];
  grp_lo[gi] = i;
  grp_agent[gi] = uint32_t(ck[i] & 0x1FFF);
  // slot of the previous group (-1 before the first)
  const int64_t prev = i == 0 ? -1 : int64_t(((run - run_flag[i]) << 2) | uint32_t((ck[i - 1] >> 13) & 3u));
  for (int64_t t = prev + 1; t <= int64_t(slot); ++t) rc_off[t] = gi;
}

// the fields of each access record the check needs, copied into the primary order
__global__ void k_wc_fields(const uint32_t* idx, const AccInfo* info, const uint32_t* n_dev, uint32_t* s_who,
                            uint32_t* s_row, uint32_t* s_ep) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= *n_dev) return;
  const AccInfo in = info[idx[p]];
  s_who[p] = in.who;
  s_row[p] = in.row;
  s_ep[p] = in.epoch;
}

__global__ void k_wc_grp_end(const uint32_t* n_groups, const uint32_t* n_dev, uint32_t* grp_lo) {
  grp_lo[*n_groups] = *n_dev;
}

inline uint32_t nblk(uint64_t n, uint32_t t) { return uint32_t((n + t - 1) / t); }

}  // namespace

// Launch of the wide walker (the plan stream is already built on s).
int phaseG_wide(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s) {
  WideArgs a{};
  a.g = g;
  a.st = b.st;
  a.sy_start = b.sy_start;
  a.incs_off = b.incs_cnt;
  a.rowbase = b.vcount;
  a.plan = b.plan;
  a.recmeta = b.recmeta;
  a.pool = b.dep_pool;
  a.flat = b.flat;
  a.rows = b.rows;
  a.psnap = b.psnap;
  a.hsnap = b.hsnap;
  a.cursor = b.cursor;
  a.jsnap = b.jsnap;
  a.tiles = b.tiles;
  a.tile_ctr = reinterpret_cast<unsigned long long*>(&b.st->spare[2]);
  a.tile_cap = z.tile_cap;
  a.n_locks = z.n_locks;
  a.hb_only = z.hb_only;
  const uint32_t threads = g.apb * 32;
  const size_t smem = (size_t(g.apb) * 96 + 32 + 96 + 2 * size_t(g.apb)) * 4;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the variant with the most registers whose CTAs are all co-resident; packed: two CTAs
  // per SM first, which leaves SMs to other streams' kernels
  void* kern = nullptr;
  void* order[2] = {reinterpret_cast<void*>(k_prop_wide<1>), reinterpret_cast<void*>(k_prop_wide<2>)};
  if (z.pack_walkers) std::swap(order[0], order[1]);
  for (void* k : order) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, int(threads), smem) != cudaSuccess)
      return GWCP_ERR_CUDA;
    if (uint64_t(per_sm) * sms >= g.B) {
      kern = k;
      break;
    }
  }
  if (!kern) return GWCP_ERR_UNSUPPORTED;  // walkers must be co-resident
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(kern, dim3(g.B), dim3(threads), args, smem, s) != cudaSuccess) return GWCP_ERR_CUDA;
  count_launch();
  return GWCP_OK;
}

// Regrouping of the key-sorted accesses by (location, class, agent); runs beside the
// propagation (it needs AccInfo and the key order, not the clocks).
void phaseI_wide_group(Bufs& b, const Geo& g, Sizes& z, uint32_t* tmp, cudaStream_t s, Prof& p) {
  const uint32_t n = z.n_acc;
  if (!n) return;
  p.begin("i_wide_group", double(n) * (8 + 4 + 16 + 12 * 3 * 5 + 16), s);
  k_wc_runflags<<<nblk(n, 256), 256, 0, s>>>(b.acc_key, n, b.wc_flag);
  count_launch();
  scan_exclusive(b.wc_flag, b.wc_run, n, b.wc_run + n, tmp, s);
  k_wc_compose<<<nblk(n, 256), 256, 0, s>>>(b.wc_run, b.wc_flag, b.acc_idx, b.acc_info, n, b.wc_key, b.wc_val,
                                            b.wc_who, b.wc_row, b.wc_ep);
  count_launch();
  // accesses of locations with a write-class access, compacted (count on the device, at
  // wc_gexcl[n]); wc_grp_lo, wc_gflag and wc_gexcl serve as scratch until the groups are built
  uint32_t* run_w = b.wc_grp_lo;
  uint32_t* keep = b.wc_gflag;
  uint32_t* kpos = b.wc_gexcl;
  uint32_t* n_keep = b.wc_gexcl + n;
  cudaMemsetAsync(run_w, 0, (size_t(n) + 1) * 4, s);
  k_wc_runwrite<<<nblk(n, 256), 256, 0, s>>>(b.wc_key, n, run_w);
  count_launch();
  k_wc_keep<<<nblk(n, 256), 256, 0, s>>>(b.wc_key, n, run_w, keep);
  count_launch();
  scan_exclusive(keep, kpos, n, n_keep, tmp, s);
  k_wc_compact<<<nblk(n, 256), 256, 0, s>>>(b.wc_key, b.wc_val, keep, kpos, n, b.wc_key2, b.wc_val2);
  count_launch();
  std::swap(b.wc_key, b.wc_key2);
  std::swap(b.wc_val, b.wc_val2);
  uint32_t* const n_kept = b.wc_run + n + 1;  // the count, copied out of the scratch
  cudaMemcpyAsync(n_kept, n_keep, 4, cudaMemcpyDeviceToDevice, s);
  // runs < n <= 2^30: key bits 15 .. 15 + ceil(log2 n); class bits 13-14; agent bits below
  // 13, of which only ceil(log2 W) vary
  uint32_t rb = 1, ab = 0;
  while ((1ull << rb) < n) ++rb;
  while ((1u << ab) < g.W) ++ab;
  const uint64_t mask = (((1ull << rb) - 1) << 15) | (3ull << 13) | ((1ull << ab) - 1);
  if (radix_sort_pairs(b.wc_key, b.wc_val, b.wc_key2, b.wc_val2, n, mask, tmp, s, n_kept)) {
    std::swap(b.wc_key, b.wc_key2);
    std::swap(b.wc_val, b.wc_val2);
  }
  k_wc_groupflags<<<nblk(n, 256), 256, 0, s>>>(b.wc_key, n, n_kept, b.wc_gflag);
  count_launch();
  scan_exclusive(b.wc_gflag, b.wc_gexcl, n, b.wc_gexcl + n, tmp, s);
  cudaMemsetAsync(b.wc_rc, 0, (size_t(n) * 4 + 2) * 4, s);
  k_wc_groups<<<nblk(n, 256), 256, 0, s>>>(b.wc_key, b.wc_gflag, b.wc_gexcl, n, b.wc_grp_lo, b.wc_grp_agent,
                                          b.wc_rc);
  count_launch();
  k_wc_grp_end<<<1, 1, 0, s>>>(b.wc_gexcl + n, n_kept, b.wc_grp_lo);  // grp_lo[n_groups] = kept count
  count_launch();
  scan_exclusive(b.wc_rc, b.wc_rc, size_t(n) * 4 + 1, nullptr, tmp, s);
  p.end();
}

// Groups of the grouped order (the accesses already sorted by (location, class, agent),
// trace order within): location runs, (class, agent) groups, the first group of each
// (run, class), and the record fields in that order. One sort instead of a location sort
// followed by a regrouping sort.
void phaseI_grouped(Bufs& b, const Geo& g, Sizes& z, uint32_t* tmp, cudaStream_t s, Prof& p) {
  (void)g;
  const uint32_t n = z.n_kept;  // the accesses the written-location filter kept
  if (!n) return;
  p.begin("i_wide_group", double(n) * (8 + 4 * 4 + 16 + 12 + 16), s);  // ~ per access
  k_gr_flags<<<nblk(n, 256), 256, 0, s>>>(b.acc_key, n, b.n_kept, b.wc_flag, b.wc_gflag);
  count_launch();
  scan_exclusive(b.wc_flag, b.wc_run, n, b.wc_run + n, tmp, s);
  scan_exclusive(b.wc_gflag, b.wc_gexcl, n, b.wc_gexcl + n, tmp, s);
  k_gr_groups<<<nblk(n, 256), 256, 0, s>>>(b.acc_key, b.wc_flag, b.wc_run, b.wc_gflag, b.wc_gexcl, b.n_kept,
                                          b.wc_grp_lo, b.wc_grp_agent, b.wc_rc);
  count_launch();
  k_wc_fields<<<nblk(n, 256), 256, 0, s>>>(b.acc_idx, b.acc_info, b.n_kept, b.wc_who, b.wc_row, b.wc_ep);
  count_launch();
  p.end();
}


uint32_t sparse_check_blocks(uint32_t n_acc) { return nblk(n_acc, kCheckThreads); }

void phaseI_wide_check(const Bufs& b, const Geo& g, const Sizes& z, cudaStream_t s, Prof& p) {
  const uint32_t n = z.grouped ? z.n_kept : z.n_acc;
  if (!n) return;
  WideCheckArgs a{};
  a.g = g;
  a.n = n;
  a.n_dev = z.grouped ? b.n_kept : nullptr;
  a.idx = b.acc_idx;
  a.flag = b.wc_flag;
  a.run_excl = b.wc_run;
  a.gs = z.grouped ? b.acc_idx : b.wc_val;
  a.grouped = z.grouped ? 1u : 0u;
  a.grp_lo = b.wc_grp_lo;
  a.grp_agent = b.wc_grp_agent;
  a.rc_off = b.wc_rc;
  a.info = b.acc_info;
  a.s_who = b.wc_who;
  a.s_row = b.wc_row;
  a.s_ep = b.wc_ep;
  a.rows = b.rows;
  a.tiles = b.tiles;
  a.tile_cap = z.tile_cap;
  a.races = b.races;
  a.race_cap = z.race_cap;
  a.st = b.st;
  a.dense_wp = g.nT ? 0u : g.Wp;
  a.cv_pool = z.compress ? b.cv_pool : nullptr;
  a.cv_cap = z.cv_cap;
  a.row_words = z.compress ? g.B : g.RW;
  a.chunk_ns = b.chunk_ns;
  a.chunk_races = b.chunk_races;
  p.begin("i_check", double(n) * (4 + 16 + 4 + 4 + 4 + 8));
  if (z.compress)
    k_wc_check<REP_COMPRESSED><<<nblk(n, kCheckThreads), kCheckThreads, 0, s>>>(a);
  else if (g.nT)
    k_wc_check<REP_TILES><<<nblk(n, kCheckThreads), kCheckThreads, 0, s>>>(a);
  else
    k_wc_check<REP_DENSE><<<nblk(n, kCheckThreads), kCheckThreads, 0, s>>>(a);
  count_launch();
  p.end();
}

}  // namespace gwcp
