// GWCP reference oracle: a plain, slow, single-threaded CPU implementation of the
// paper's predictive race analysis ("Predictive Data Race Detection for GPUs",
// arXiv 2111.12478).
//
// TEST INFRASTRUCTURE ONLY. This file is the oracle that the CUDA path is checked
// against. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
// load it. It shares no code, header, table or helper with the CUDA library: the two
// agree only through the trace format, which each side declares on its own.
//
// What it follows, step by step:
//   * Metadata: per-thread N_t, P_t, H_t (C_t = P_t{t := N_t}); per scoped lock
//     <l,s> the clocks P_<l,s>, H_<l,s>; per (lock, scope, location) L^r and L^w;
//     per-thread locksets; acquire/release records (section "Tracking GWCP",
//     "Metadata").
//   * sync / acquire / release: Algorithm 1 (ACM form), with the IEEE form's scope
//     encoding: scope id 0 = device, b+1 = block b.
//   * read / write: Algorithm 2.
//   * GPU adaptations (section "Tracking GWCP", four paragraphs after Algorithm 2):
//     shared memory is keyed per block; two atomics with overlapping scopes do not
//     race; scoped locks are distinct locks and device acquires join every block's
//     copy; barriers join C_t, not P_t.
//   * Race check: R_x / W_x style last-access state compared against C_t at each
//     access (section "Tracking GWCP", Metadata paragraph on R_x and W_x).
//
// Readings where the paper is silent or inconsistent (each one is listed in the
// design notes of the repository):
//   A1  initial values: N_t = 1, H_t = bottom{t := 1}, P_t = bottom.
//   A2  release loop joins a popped record when the two scopes overlap (device on
//       either side, or the same block); option release_scope_ieee switches to the
//       literal IEEE test (record scope is device, or the releasing thread's block).
//   A3  sync increments N_t and H_t[t] for every thread in the barrier's scope.
//   A4  one list of critical-section records per lock plus a per-(thread, lock)
//       cursor stands in for the per-thread Acq/Rel queues; the thread's own records
//       are skipped, and a popped record whose release has not happened yet is not
//       joined.
//   A5  race set: for each access b by thread u and each other thread v, the latest
//       earlier access a* by v to the same location that conflicts with b and is not
//       exempt; (a*, b) is reported when N(a*) > C_b[v].
//   A6  atomic exemption when both are atomics with overlapping scopes (same block,
//       or either is device-scoped); option atomic_scope_lesser switches to "both
//       device-scoped, or same block".
//   A7  ATOMIC is a write for conflicts and critical-section write sets; FENCE has no
//       effect on the order.
//   A8  a shared-memory location is keyed (1<<63) | (block << 40) | addr.
//   A10 an access inside a critical section joins first, then is checked.
//   A11 an access is added to the read/write set of every held lock.
//   A12 one BARRIER event per barrier instance; scope CTA covers the block named in
//       addr, scope WARP covers the lanes of addr's mask (thread granularity) or the
//       event's agent alone (warp granularity).
//   A13 the release loop re-derives C_t after every join and tests acqC <= C_t
//       component-wise; it also counts how often the one-entry epoch test
//       acqC[agent] <= C_t[agent] would have answered differently.
//   C1  (option forced_barrier; section "Vector Clock Compression") after a barrier's
//       join, every participant's entry in both joined clocks and every participant's
//       local time become the highest among the participants.
//   C2  (option version_words) a clock version is P_t (H_t with hb_only) at the start
//       and after each acquire, release, barrier and access made while holding a lock;
//       its compressed size is one word per block, plus, for a block whose entries
//       differ, one word per warp and 32 values per warp whose entries differ.

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

namespace {

// ---- trace format (16-byte records, trace order = array order) -------------------
struct Event {
  uint32_t agent;
  uint8_t op, scope, space, flags;
  uint64_t addr;
};
static_assert(sizeof(Event) == 16, "event record is 16 bytes");

enum Op : uint8_t { READ = 0, WRITE = 1, ATOMIC = 2, ACQ = 3, REL = 4, BARRIER = 5, FENCE = 6 };
enum Scope : uint8_t { CTA = 0, DEVICE = 1, WARP = 2 };
enum Space : uint8_t { GLOBAL = 0, SHARED = 1 };

struct Geometry {
  uint32_t num_agents, agents_per_block, granularity, reserved;
};

// access classes for the per-location last-access state
enum Cls : int { C_READ = 0, C_WRITE = 1, C_ATOM_CTA = 2, C_ATOM_DEV = 3 };

constexpr int kMaxNesting = 4;  // deepest lockset a valid trace may hold

using VC = std::vector<uint32_t>;

inline void join(VC& a, const VC& b) {
  for (size_t k = 0; k < a.size(); ++k) a[k] = std::max(a[k], b[k]);
}

// ---- error codes shared with the Python wrapper ------------------------------------
enum {
  OK = 0,
  ERR_INVALID_TRACE = -1,
  ERR_ARGS = -2,
};

}  // namespace

extern "C" {

struct OracleOptions {
  int32_t all_pairs;            // report every racing pair, not only (a*, b)
  int32_t release_scope_ieee;   // A2 alternative
  int32_t atomic_scope_lesser;  // A6 alternative
  int32_t hb_only;              // check against H_t instead of C_t
  int32_t forced_barrier;       // forced compression at barriers (section "Vector Clock
                                // Compression", second paragraph of its two ideas)
  int32_t version_words;        // size every clock version in the block/warp compressed form
};

struct OracleResult {
  std::vector<uint64_t> races;  // flattened (earlier, later) pairs
  // counters
  uint64_t joins = 0;                 // vector-clock joins performed
  uint64_t epoch_test_disagree = 0;   // A13: epoch test vs component-wise test
  uint64_t loop_visits = 0;           // release-loop record visits
  uint64_t partner_tests = 0;         // (b, v) pairs with a candidate a*
  uint64_t invariant_violations = 0;  // H_t[t] != N_t or a clock that went down
  // option version_words: the clock versions (P_t, or H_t with hb_only, at the start and
  // after each acquire, release, barrier and access made while holding a lock) and the
  // words they take in the compressed form
  uint64_t versions = 0, version_words = 0;
  // clocks captured at requested events
  std::vector<uint64_t> clock_events;
  std::vector<uint32_t> clock_c, clock_h;  // row-major [k][W]
  std::vector<uint8_t> clock_valid;
  uint32_t W = 0;
};

}  // extern "C"

namespace {

struct Geo {
  uint32_t W, apb, B, gran;
  uint32_t block(uint32_t t) const { return t / apb; }
};

// Scope ids: 0 = device, b + 1 = block b (IEEE form of Algorithm 1).
inline uint32_t scope_id(const Geo& g, uint32_t agent, uint8_t scope) {
  return scope == DEVICE ? 0u : g.block(agent) + 1u;
}

// Two scoped uses overlap iff one is device-scoped or both are from the same block
// (section "Extending WCP to GPU Programs", paragraph on scoped locks).
inline bool overlap(uint32_t s1, uint32_t s2) { return s1 == 0 || s2 == 0 || s1 == s2; }

inline uint64_t location_key(const Geo& g, const Event& e) {
  if (e.space == SHARED)
    return (uint64_t(1) << 63) | (uint64_t(g.block(e.agent)) << 40) | e.addr;
  return e.addr;
}

inline int access_class(const Event& e) {
  if (e.op == READ) return C_READ;
  if (e.op == WRITE) return C_WRITE;
  return e.scope == DEVICE ? C_ATOM_DEV : C_ATOM_CTA;
}

inline bool is_write_class(int c) { return c != C_READ; }
inline bool is_atomic_class(int c) { return c == C_ATOM_CTA || c == C_ATOM_DEV; }

// Participants of a barrier event (reading A12).
bool barrier_members(const Geo& g, const Event& e, std::vector<uint32_t>& out) {
  out.clear();
  if (e.scope == CTA) {
    if (e.addr >= g.B) return false;
    for (uint32_t t = 0; t < g.apb; ++t) out.push_back(uint32_t(e.addr) * g.apb + t);
    return true;
  }
  if (e.scope == WARP) {
    uint64_t mask = e.addr;
    if (mask == 0 || mask > 0xffffffffull) return false;
    if (g.gran == 1) {  // warp granularity: the warp is one agent
      out.push_back(e.agent);
      return true;
    }
    uint32_t blk = g.block(e.agent);
    uint32_t base = blk * g.apb + ((e.agent - blk * g.apb) / 32u) * 32u;
    for (uint32_t lane = 0; lane < 32; ++lane) {
      if (!((mask >> lane) & 1)) continue;
      uint32_t t = base + lane;
      if (t >= (blk + 1) * g.apb) return false;  // lane outside the block
      out.push_back(t);
    }
    return true;
  }
  return false;
}

// ---- well-formedness W1-W4 -----------------------------------------------------------
struct HeldV {
  uint64_t lock;
  uint32_t sid;
};

int validate(const Geo& g, const Event* ev, uint64_t n, uint64_t* bad) {
  std::vector<std::vector<HeldV>> held(g.W);
  // per lock: open critical sections per scope id
  std::unordered_map<uint64_t, std::map<uint32_t, uint32_t>> open;
  std::vector<uint32_t> members;
  for (uint64_t i = 0; i < n; ++i) {
    const Event& e = ev[i];
    auto fail = [&]() {
      *bad = i;
      return ERR_INVALID_TRACE;
    };
    // W1: agent and field ranges
    if (e.agent >= g.W || e.op > FENCE || e.scope > WARP || e.space > SHARED) return fail();
    if (e.scope == WARP && e.op != BARRIER) return fail();
    if (e.space == SHARED && e.op > ATOMIC) return fail();
    if (e.op <= ATOMIC) {
      if (e.space == SHARED && e.addr >= (uint64_t(1) << 40)) return fail();
      if (e.space == GLOBAL && e.addr >= (uint64_t(1) << 63)) return fail();
    }
    if (e.op == BARRIER) {
      if (!barrier_members(g, e, members)) return fail();
    } else if (e.op == ACQ) {
      uint32_t sid = scope_id(g, e.agent, e.scope);
      auto& o = open[e.addr];
      // W3: no open critical section on this lock with an overlapping scope
      for (auto& kv : o)
        if (kv.second > 0 && overlap(kv.first, sid)) return fail();
      if (held[e.agent].size() >= size_t(kMaxNesting)) return fail();
      o[sid] += 1;
      held[e.agent].push_back({e.addr, sid});
    } else if (e.op == REL) {
      uint32_t sid = scope_id(g, e.agent, e.scope);
      auto& h = held[e.agent];
      // W2: releases match the innermost held acquire (same lock, same scope)
      if (h.empty() || h.back().lock != e.addr || h.back().sid != sid) return fail();
      h.pop_back();
      open[e.addr][sid] -= 1;
    }
  }
  return OK;
}

// ---- the analysis --------------------------------------------------------------------
struct CSRecord {
  uint32_t agent;
  uint32_t sid;
  VC acqC;  // C_t at the acquire, after its joins
  bool released = false;
  VC relH;  // H_t at the release
};

struct LockState {
  std::unordered_map<uint32_t, VC> P, H;  // per scope id
  std::vector<CSRecord> records;          // in acquire order
};

struct Held {
  uint64_t lock;
  uint32_t sid;
  size_t rec;
  std::vector<uint64_t> R, Wr;  // locations read / written inside this section
};

struct LKey {
  uint64_t lock;
  uint32_t sid;
  uint64_t x;
  bool operator==(const LKey& o) const { return lock == o.lock && sid == o.sid && x == o.x; }
};
struct LKeyHash {
  size_t operator()(const LKey& k) const {
    uint64_t h = k.lock * 0x9E3779B97F4A7C15ull ^ (k.x + 0x632BE59BD9B4E019ull + (uint64_t(k.sid) << 32));
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    return size_t(h);
  }
};
struct LClocks {
  VC r, w;
};

struct Last {
  uint64_t idx = ~uint64_t(0);  // ~0 = none
  uint32_t epoch = 0;
};

struct HistEntry {
  uint64_t idx;
  uint32_t agent;
  int cls;
  uint32_t epoch;
};

class Analysis {
 public:
  Analysis(const Geo& g, const OracleOptions& opt, OracleResult* res)
      : g_(g), opt_(opt), res_(res), N_(g.W, 1), P_(g.W, VC(g.W, 0)), H_(g.W, VC(g.W, 0)), held_(g.W) {
    for (uint32_t t = 0; t < g.W; ++t) H_[t][t] = 1;  // A1
  }

  void run(const Event* ev, uint64_t n, const std::vector<int64_t>& want_clock) {
    for (uint32_t t = 0; t < g_.W; ++t) version(t);
    for (uint64_t i = 0; i < n; ++i) {
      const Event& e = ev[i];
      switch (e.op) {
        case READ:
        case WRITE:
        case ATOMIC:
          access(i, e);
          break;
        case ACQ:
          acquire(e.agent, e.addr, scope_id(g_, e.agent, e.scope));
          break;
        case REL:
          release(e.agent, e.addr, scope_id(g_, e.agent, e.scope));
          break;
        case BARRIER: {
          std::vector<uint32_t> m;
          barrier_members(g_, e, m);
          sync(m);
          break;
        }
        case FENCE:  // A7: no effect on the order
          break;
      }
      if (want_clock[i] >= 0) capture(size_t(want_clock[i]), e);
      if (e.op == ACQ || e.op == REL) check_invariant(e.agent);
    }
    std::sort(pairs_.begin(), pairs_.end(), [](const std::pair<uint64_t, uint64_t>& a,
                                                const std::pair<uint64_t, uint64_t>& b) {
      return a.second != b.second ? a.second < b.second : a.first < b.first;
    });
    pairs_.erase(std::unique(pairs_.begin(), pairs_.end()), pairs_.end());
    res_->races.reserve(pairs_.size() * 2);
    for (auto& p : pairs_) {
      res_->races.push_back(p.first);
      res_->races.push_back(p.second);
    }
  }

 private:
  VC C(uint32_t t) const {
    VC c = P_[t];
    c[t] = N_[t];
    return c;
  }

  void joinc(VC& a, const VC& b) {
    join(a, b);
    res_->joins++;
  }

  // Algorithm 1, procedure sync(scope): join the C and H clocks of every thread in
  // scope, give the joins to all of them, then increment (reading A3).
  // Forced compression (option forced_barrier): after the join, the entries of the
  // participants are all set to the highest of them, in both joined clocks, and so are
  // the participants' local times; every participant leaves the barrier at the same
  // logical time, so each one's clock holds one common value for the whole scope.
  void sync(const std::vector<uint32_t>& scope) {
    VC joined(g_.W, 0), joinedHB(g_.W, 0);
    for (uint32_t t : scope) {
      joinc(joined, C(t));
      joinc(joinedHB, H_[t]);
    }
    if (opt_.forced_barrier) {
      uint32_t top = 0;
      for (uint32_t t : scope) top = std::max({top, joined[t], joinedHB[t]});
      for (uint32_t t : scope) {
        joined[t] = joinedHB[t] = top;
        N_[t] = top;
      }
    }
    for (uint32_t t : scope) {
      P_[t] = joined;
      H_[t] = joinedHB;
    }
    for (uint32_t t : scope) {
      N_[t] += 1;
      H_[t][t] += 1;
      check_invariant(t);
      version(t);
    }
  }

  LockState& lock(uint64_t l) { return locks_[l]; }

  void join_lock_clock(uint32_t t, LockState& L, uint32_t sid) {
    auto p = L.P.find(sid);
    if (p != L.P.end()) joinc(P_[t], p->second);
    auto h = L.H.find(sid);
    if (h != L.H.end()) joinc(H_[t], h->second);
  }

  // Algorithm 1, procedure acquire(t, l, s).
  void acquire(uint32_t t, uint64_t l, uint32_t sid) {
    LockState& L = lock(l);
    join_lock_clock(t, L, sid);
    if (sid == 0) {  // device-level lock: also every block-level copy
      for (uint32_t b = 0; b < g_.B; ++b) join_lock_clock(t, L, b + 1);
    } else {  // block-level lock: also the device-level copy
      join_lock_clock(t, L, 0);
    }
    // "Acq_l(t').enque(<C_t, s>) for all t' != t": one shared record (reading A4)
    CSRecord rec;
    rec.agent = t;
    rec.sid = sid;
    rec.acqC = C(t);
    L.records.push_back(std::move(rec));
    held_[t].push_back(Held{l, sid, L.records.size() - 1, {}, {}});
    version(t);
  }

  bool leq(const VC& a, const VC& b) const {
    for (size_t k = 0; k < a.size(); ++k)
      if (a[k] > b[k]) return false;
    return true;
  }

  // Algorithm 1, procedure release(t, l, R, W, s).
  void release(uint32_t t, uint64_t l, uint32_t sid) {
    LockState& L = lock(l);
    size_t& cur = cursor_[std::make_pair(uint64_t(t), l)];
    while (cur < L.records.size()) {
      const CSRecord& rec = L.records[cur];
      if (rec.agent == t) {  // the thread's own acquires are never in its queue
        ++cur;
        continue;
      }
      VC c = C(t);  // re-derived after every join (A13)
      bool full = leq(rec.acqC, c);
      bool epoch = rec.acqC[rec.agent] <= c[rec.agent];
      if (full != epoch) res_->epoch_test_disagree++;
      res_->loop_visits++;
      if (!full) break;
      ++cur;
      if (!rec.released) continue;  // matching release not yet seen (A4)
      bool ok = opt_.release_scope_ieee ? (rec.sid == 0 || rec.sid == g_.block(t) + 1)
                                        : overlap(rec.sid, sid);
      if (ok) joinc(P_[t], rec.relH);
    }
    Held h = held_[t].back();
    held_[t].pop_back();
    for (uint64_t x : h.R) {
      LClocks& lc = lclk(l, sid, x);
      joinc(lc.r, H_[t]);
    }
    for (uint64_t x : h.Wr) {
      LClocks& lc = lclk(l, sid, x);
      joinc(lc.w, H_[t]);
    }
    L.H[sid] = H_[t];
    L.P[sid] = P_[t];
    CSRecord& own = L.records[h.rec];
    own.released = true;
    own.relH = H_[t];
    N_[t] += 1;
    H_[t][t] += 1;
    version(t);
  }

  LClocks& lclk(uint64_t l, uint32_t sid, uint64_t x) {
    LClocks& lc = lmap_[LKey{l, sid, x}];
    if (lc.r.empty()) {
      lc.r.assign(g_.W, 0);
      lc.w.assign(g_.W, 0);
    }
    return lc;
  }

  void join_l(uint32_t t, uint64_t l, uint32_t sid, uint64_t x, bool write) {
    auto it = lmap_.find(LKey{l, sid, x});
    if (it == lmap_.end()) return;
    joinc(P_[t], it->second.w);
    if (write) joinc(P_[t], it->second.r);
  }

  // Algorithm 2 (read / write) for an access made while holding locks, then the
  // race check against C_t (reading A10).
  void access(uint64_t i, const Event& e) {
    const uint32_t u = e.agent;
    const uint64_t x = location_key(g_, e);
    const int cls = access_class(e);
    const bool write = is_write_class(cls);  // A7
    for (Held& h : held_[u]) {
      join_l(u, h.lock, h.sid, x, write);
      if (h.sid == 0) {
        for (uint32_t b = 0; b < g_.B; ++b) join_l(u, h.lock, b + 1, x, write);
      } else {
        join_l(u, h.lock, 0, x, write);
      }
    }
    for (Held& h : held_[u]) (write ? h.Wr : h.R).push_back(x);  // A11
    if (!held_[u].empty()) version(u);

    // C_b[v] is read only for agents v != u, where C_u = P_u{u := N_u} equals P_u, so the
    // check reads P_u (H_u with hb_only) in place of forming C_u
    const VC& cb = opt_.hb_only ? H_[u] : P_[u];
    const uint32_t bu = g_.block(u);
    auto exempt = [&](int ca, uint32_t ba) {
      if (!is_atomic_class(ca) || !is_atomic_class(cls)) return false;
      if (opt_.atomic_scope_lesser) return (ca == C_ATOM_DEV && cls == C_ATOM_DEV) || ba == bu;
      return ca == C_ATOM_DEV || cls == C_ATOM_DEV || ba == bu;
    };
    if (opt_.all_pairs) {
      std::vector<HistEntry>& hist = hist_[x];
      for (const HistEntry& a : hist) {
        if (a.agent == u) continue;
        if (!is_write_class(a.cls) && !write) continue;
        if (exempt(a.cls, g_.block(a.agent))) continue;
        if (a.epoch > cb[a.agent]) pairs_.emplace_back(a.idx, i);
      }
      hist.push_back(HistEntry{i, u, cls, N_[u]});
    } else {
      // Per location and class, every agent's latest access of that class. Agents that
      // never accessed x have none and are not visited; neither is a class that b cannot
      // race with whatever the other agent's block (two reads never conflict; two atomics
      // may be exempt by scope alone), so the reads of a location nobody writes visit
      // nothing. a* of agent v is the latest of v's accesses over the remaining classes.
      std::array<std::map<uint32_t, Last>, 4>& last = last_[x];
      std::map<uint32_t, const Last*> best;  // agent v -> its a*
      for (int c = 0; c < 4; ++c) {
        if (!is_write_class(c) && !write) continue;
        // exempt(c, .) depends on the other agent's block only through "same block as u"
        if (exempt(c, bu) && exempt(c, bu + 1)) continue;
        for (const auto& [v, l] : last[c]) {
          if (v == u || exempt(c, g_.block(v))) continue;
          const Last*& b = best[v];
          if (!b || l.idx > b->idx) b = &l;
        }
      }
      for (const auto& [v, b] : best) {
        res_->partner_tests++;
        if (b->epoch > cb[v]) pairs_.emplace_back(b->idx, i);  // A5
      }
      Last& mine = last[cls][u];
      mine.idx = i;
      mine.epoch = N_[u];
    }
  }

  // Words of clock v in the compressed form of section "Vector Clock Compression": one
  // word per block (its common value when all its entries are equal); an expanded block
  // adds one word per warp (a warp is one agent at warp granularity, 32 threads at thread
  // granularity), and a warp whose entries differ adds its 32 values.
  uint64_t compressed_words(const VC& v) const {
    const uint32_t gs = g_.gran == 1 ? 1 : 32;
    const uint32_t nw = (g_.apb + gs - 1) / gs;
    uint64_t words = g_.B;
    for (uint32_t b = 0; b < g_.B; ++b) {
      const uint32_t* x = v.data() + size_t(b) * g_.apb;
      bool block_equal = true;
      uint64_t extra = nw;
      for (uint32_t w = 0; w < nw; ++w) {
        const uint32_t lo = w * gs, hi = std::min(lo + gs, g_.apb);
        bool warp_equal = true;
        for (uint32_t i = lo; i < hi; ++i) {
          if (x[i] != x[lo]) warp_equal = false;
          if (x[i] != x[0]) block_equal = false;
        }
        if (!warp_equal) extra += 32;
      }
      if (!block_equal) words += extra;
    }
    return words;
  }

  void version(uint32_t t) {
    if (!opt_.version_words) return;
    res_->versions++;
    res_->version_words += compressed_words(opt_.hb_only ? H_[t] : P_[t]);
  }

  void capture(size_t k, const Event& e) {
    uint32_t t = e.agent;
    VC c = C(t);
    std::copy(c.begin(), c.end(), res_->clock_c.begin() + k * g_.W);
    std::copy(H_[t].begin(), H_[t].end(), res_->clock_h.begin() + k * g_.W);
    res_->clock_valid[k] = 1;
    if (e.op == REL) {  // report the clocks the release published, before its increment
      res_->clock_c[k * g_.W + t] -= 1;
      res_->clock_h[k * g_.W + t] -= 1;
    }
  }

  void check_invariant(uint32_t t) {
    if (H_[t][t] != N_[t]) res_->invariant_violations++;
  }

  Geo g_;
  OracleOptions opt_;
  OracleResult* res_;
  std::vector<uint32_t> N_;
  std::vector<VC> P_, H_;
  std::vector<std::vector<Held>> held_;
  std::unordered_map<uint64_t, LockState> locks_;
  std::map<std::pair<uint64_t, uint64_t>, size_t> cursor_;
  std::unordered_map<LKey, LClocks, LKeyHash> lmap_;
  std::unordered_map<uint64_t, std::array<std::map<uint32_t, Last>, 4>> last_;  // location -> class -> agent
  std::unordered_map<uint64_t, std::vector<HistEntry>> hist_;
  std::vector<std::pair<uint64_t, uint64_t>> pairs_;
};

bool make_geo(const Geometry* gm, Geo* g) {
  if (!gm || gm->num_agents == 0 || gm->agents_per_block == 0) return false;
  if (gm->num_agents % gm->agents_per_block != 0 || gm->granularity > 1) return false;
  g->W = gm->num_agents;
  g->apb = gm->agents_per_block;
  g->B = gm->num_agents / gm->agents_per_block;
  g->gran = gm->granularity;
  return true;
}

}  // namespace

extern "C" {

int oracle_validate(const void* events, uint64_t n, const Geometry* gm, uint64_t* bad_index) {
  Geo g;
  if (!make_geo(gm, &g)) return ERR_ARGS;
  uint64_t bad = ~uint64_t(0);
  int rc = validate(g, static_cast<const Event*>(events), n, &bad);
  if (bad_index) *bad_index = bad;
  return rc;
}

// Runs the analysis over a validated trace. clock_events (may be null) lists event
// indices whose C_t and H_t are captured (for an access: after its joins; for an
// acquire: after its joins; for a release: the clocks it published, before the
// increment). Returns a result handle through *out.
int oracle_run(const void* events, uint64_t n, const Geometry* gm, const OracleOptions* opt,
               const uint64_t* clock_events, uint64_t n_clock, OracleResult** out, uint64_t* bad_index) {
  Geo g;
  if (!make_geo(gm, &g) || !out) return ERR_ARGS;
  const Event* ev = static_cast<const Event*>(events);
  uint64_t bad = ~uint64_t(0);
  int rc = validate(g, ev, n, &bad);
  if (bad_index) *bad_index = bad;
  if (rc != OK) return rc;
  OracleOptions o{};
  if (opt) o = *opt;
  auto* res = new OracleResult();
  res->W = g.W;
  std::vector<int64_t> want(n, -1);
  res->clock_events.assign(clock_events, clock_events + n_clock);
  res->clock_c.assign(size_t(n_clock) * g.W, 0);
  res->clock_h.assign(size_t(n_clock) * g.W, 0);
  res->clock_valid.assign(n_clock, 0);
  for (uint64_t k = 0; k < n_clock; ++k)
    if (clock_events[k] < n) want[clock_events[k]] = int64_t(k);
  Analysis a(g, o, res);
  a.run(ev, n, want);
  *out = res;
  return OK;
}

uint64_t oracle_num_races(const OracleResult* r) { return r->races.size() / 2; }
void oracle_copy_races(const OracleResult* r, uint64_t* out) {
  std::memcpy(out, r->races.data(), r->races.size() * sizeof(uint64_t));
}
void oracle_counters(const OracleResult* r, uint64_t* out5) {
  out5[0] = r->joins;
  out5[1] = r->epoch_test_disagree;
  out5[2] = r->loop_visits;
  out5[3] = r->partner_tests;
  out5[4] = r->invariant_violations;
}
void oracle_versions(const OracleResult* r, uint64_t* out2) {
  out2[0] = r->versions;
  out2[1] = r->version_words;
}
// Copies the captured clocks of the k-th requested event; returns 0 if captured.
int oracle_clock(const OracleResult* r, uint64_t k, uint32_t* c_out, uint32_t* h_out) {
  if (k >= r->clock_valid.size() || !r->clock_valid[k]) return -1;
  std::memcpy(c_out, r->clock_c.data() + k * r->W, r->W * sizeof(uint32_t));
  std::memcpy(h_out, r->clock_h.data() + k * r->W, r->W * sizeof(uint32_t));
  return 0;
}
void oracle_free(OracleResult* r) { delete r; }

}  // extern "C"
