// Seeded synthetic GPU-program trace generator (inputs only; no analysis).
//
// Produces well-formed traces in the 16-byte event format: every release matches the
// innermost held acquire; two critical sections on one lock with overlapping scopes
// never interleave; barriers are one event per instance. Every address class follows
// a synchronisation discipline that makes it race-free, and a small fraction of
// accesses is planted to break one (flags bit 0), so every race in a generated trace
// involves a planted access.
//
// Address classes (disjoint regions of the address space):
//   P  private: one copy per agent and rank; only the owner touches it.
//   B  block-phase: one copy per block and rank; in each barrier phase one agent of the
//      block (a hash of rank, block and phase) owns it.
//   L  lock-guarded: four addresses per lock; device locks have one copy, block-scoped
//      locks one copy per block; touched only inside a critical section on that lock.
//   A  atomic counters: device-scoped atomics on one copy per rank, block-scoped atomics
//      on one copy per block and rank.
//   R  read-only.
// Planted kinds: a write to an R address; a write to another agent's P copy; a write to
// an L address outside a critical section; a block-scoped atomic on another block's A
// copy; a read of a device atomic counter.
//
// Random numbers: xoshiro256** seeded through splitmix64; Zipf ranks by
// rejection-inversion (Hormann and Derflinger, 1996).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Event {
  uint32_t agent;
  uint8_t op, scope, space, flags;
  uint64_t addr;
};
static_assert(sizeof(Event) == 16, "event record is 16 bytes");

enum : uint8_t { READ = 0, WRITE = 1, ATOMIC = 2, ACQ = 3, REL = 4, BARRIER = 5, FENCE = 6 };
enum : uint8_t { CTA = 0, DEVICE = 1, WARPSC = 2 };

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Xoshiro {
  uint64_t s[4];
  explicit Xoshiro(uint64_t seed) {
    for (auto& v : s) v = splitmix64(seed);
  }
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return r;
  }
  double uniform() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
  uint64_t below(uint64_t n) { return n ? next() % n : 0; }
};

uint64_t mix(uint64_t a, uint64_t b = 0, uint64_t c = 0) {
  uint64_t x = a * 0x9E3779B97F4A7C15ull + b * 0xC2B2AE3D27D4EB4Full + c * 0x165667B19E3779F9ull + 1;
  return splitmix64(x);
}

// Zipf(s) over ranks 1..n by rejection-inversion.
class Zipf {
 public:
  Zipf(uint64_t n, double s) : n_(n), s_(s) {
    if (s_ <= 0) return;
    hx1_ = H(1.5) - 1.0;
    hn_ = H(double(n_) + 0.5);
    t_ = 2.0 - Hinv(H(2.5) - h(2.0));
  }
  uint64_t operator()(Xoshiro& rng) const {  // 0-based rank
    if (s_ <= 0) return rng.below(n_);
    for (;;) {
      double u = hn_ + rng.uniform() * (hx1_ - hn_);
      double x = Hinv(u);
      double kd = std::floor(x + 0.5);
      if (kd < 1) kd = 1;
      if (kd > double(n_)) kd = double(n_);
      if (kd - x <= t_ || u >= H(kd + 0.5) - h(kd)) return uint64_t(kd) - 1;
    }
  }

 private:
  static double log1p_over(double x) { return std::fabs(x) > 1e-8 ? std::log1p(x) / x : 1.0 - x / 2.0; }
  static double expm1_over(double x) { return std::fabs(x) > 1e-8 ? std::expm1(x) / x : 1.0 + x / 2.0; }
  double h(double x) const { return std::exp(-s_ * std::log(x)); }
  double H(double x) const {
    double lx = std::log(x);
    return expm1_over((1.0 - s_) * lx) * lx;
  }
  double Hinv(double x) const {
    double t = x * (1.0 - s_);
    if (t < -1.0) t = -1.0;
    return std::exp(log1p_over(t) * x);
  }
  uint64_t n_;
  double s_, hx1_ = 0, hn_ = 0, t_ = 0;
};

}  // namespace

extern "C" {

struct GenParams {
  uint64_t seed;
  uint64_t n_events;
  uint32_t num_blocks;
  uint32_t agents_per_block;
  uint32_t granularity;  // 0 thread, 1 warp
  uint32_t n_ranks;
  double zipf_s;
  uint32_t n_locks;
  double dev_lock_frac;
  double p_read, p_write, p_atomic, p_acqrel, p_fence, p_barrier;
  double atomic_dev_frac;
  double plant_frac;
  uint32_t n_plant_exact;
  double cs_len_mean;
  double nest_prob;
  double shared_frac;
  double p_syncwarp;
  uint32_t plant_min_rank;  // planted accesses use address ranks >= this (0: any rank)
};

int gwcp_tracegen_run(const GenParams* p, void* out_events, uint64_t* n_written) {
  if (!p || !out_events || p->num_blocks == 0 || p->agents_per_block == 0 || p->n_ranks == 0) return -1;
  Event* out = static_cast<Event*>(out_events);
  const uint32_t B = p->num_blocks, apb = p->agents_per_block, W = B * apb;
  const uint64_t n = p->n_events;
  Xoshiro rng(p->seed);
  Zipf zipf(p->n_ranks, p->zipf_s);

  // address regions (byte addresses, 4-byte words); shared copies live in [0, 2^40)
  const uint64_t R_BASE = 0x100000000000ull, P_BASE = 0x200000000000ull, B_BASE = 0x300000000000ull;
  const uint64_t L_BASE = 0x400000000000ull, A_BASE = 0x500000000000ull, AC_BASE = 0x600000000000ull;
  const uint64_t NR = p->n_ranks;

  struct Held {
    uint32_t lock;
    uint8_t scope;
  };
  std::vector<std::vector<Held>> held(W);
  std::vector<uint32_t> dev_holder(p->n_locks, UINT32_MAX);                   // device locks
  std::vector<uint32_t> blk_holder(size_t(p->n_locks) * B, UINT32_MAX);       // block-scoped locks
  std::vector<uint32_t> phase(B, 0);
  std::vector<uint32_t> held_in_block(B, 0);  // agents of the block currently holding a lock
  auto is_dev_lock = [&](uint32_t l) { return double(mix(l, 77) % 1000000) < p->dev_lock_frac * 1e6; };

  // planting schedule
  std::vector<uint64_t> plant_at;
  if (p->n_plant_exact) {
    for (uint32_t k = 0; k < p->n_plant_exact; ++k) plant_at.push_back((k + 1) * n / (p->n_plant_exact + 1));
  }
  size_t next_plant = 0;

  uint64_t i = 0;
  auto emit = [&](uint32_t agent, uint8_t op, uint8_t scope, uint8_t space, uint64_t addr, uint8_t flags = 0) {
    if (i < n) out[i++] = Event{agent, op, scope, space, flags, addr};
  };
  auto block_of = [&](uint32_t t) { return t / apb; };
  auto b_owner = [&](uint64_t r, uint32_t b) { return b * apb + uint32_t(mix(r, b, phase[b]) % apb); };
  const double p_acq = p->p_acqrel / 2.0;

  auto shared_pick = [&]() { return rng.uniform() < p->shared_frac; };

  // a plain (unplanted) access by t following the class disciplines
  auto access = [&](uint32_t t, double r_op) {
    const uint32_t b = block_of(t);
    uint64_t r = zipf(rng);
    double tot = p->p_read + p->p_write + p->p_atomic;
    if (r_op * tot < p->p_atomic) {
      if (rng.uniform() < p->atomic_dev_frac) {
        emit(t, ATOMIC, DEVICE, 0, A_BASE + r * 4);
      } else if (shared_pick()) {
        emit(t, ATOMIC, CTA, 1, (r % (1u << 20)) * 4 + 0x800000);  // shared per block
      } else {
        emit(t, ATOMIC, CTA, 0, AC_BASE + (r * B + b) * 4);
      }
      return;
    }
    const bool write = r_op * tot < p->p_atomic + p->p_write;
    double c = rng.uniform();
    if (!write && c < 0.5) {
      emit(t, READ, 0, 0, R_BASE + r * 4);
    } else if (c < 0.8 || b_owner(r, b) != t) {
      emit(t, write ? WRITE : READ, 0, 0, P_BASE + (r * W + t) * 4);
    } else if (shared_pick()) {
      emit(t, write ? WRITE : READ, 0, 1, (r % (1u << 20)) * 4);  // shared per block
    } else {
      emit(t, write ? WRITE : READ, 0, 0, B_BASE + (r * B + b) * 4);
    }
  };
  auto l_addr = [&](uint32_t l, uint32_t b, uint32_t j) {
    return is_dev_lock(l) ? L_BASE + (uint64_t(l) * 4 + j) * 4
                          : L_BASE + ((uint64_t(l) * B + b) * 4 + j) * 4 + 0x10000000000ull;
  };
  auto planted = [&](uint32_t t, bool exact) {
    const uint32_t b = block_of(t);
    uint64_t r = zipf(rng);
    if (r < p->plant_min_rank && p->plant_min_rank < NR) r = p->plant_min_rank + rng.below(NR - p->plant_min_rank);
    uint32_t kind = exact ? 0 : uint32_t(rng.below(5));
    if (exact) {
      // a read by another agent directly before the planted write: nothing can order
      // the two, so the planted write races for sure
      uint32_t v = (t + 1 + uint32_t(rng.below(W - 1 ? W - 1 : 1))) % W;
      if (v == t) v = (t + 1) % W;
      emit(v, READ, 0, 0, R_BASE + r * 4);
      emit(t, WRITE, 0, 0, R_BASE + r * 4, 1);
      return;
    }
    switch (kind) {
      case 0:
        emit(t, WRITE, 0, 0, R_BASE + r * 4, 1);
        break;
      case 1: {
        uint32_t v = uint32_t(rng.below(W));
        if (v == t) v = (v + 1) % W;
        emit(t, WRITE, 0, 0, P_BASE + (r * W + v) * 4, 1);
        break;
      }
      case 2: {
        uint32_t l = uint32_t(rng.below(p->n_locks));
        emit(t, WRITE, 0, 0, l_addr(l, b, uint32_t(rng.below(4))), 1);
        break;
      }
      case 3: {
        uint32_t ob = (b + 1) % B;
        emit(t, ATOMIC, CTA, 0, AC_BASE + (r * B + ob) * 4, 1);
        break;
      }
      default:
        emit(t, READ, 0, 0, A_BASE + r * 4, 1);
        break;
    }
  };
  auto try_acquire = [&](uint32_t t) -> bool {
    const uint32_t b = block_of(t);
    for (int tries = 0; tries < 4; ++tries) {
      uint32_t l = uint32_t(rng.below(p->n_locks));
      bool dup = false;
      for (auto& h : held[t]) dup |= h.lock == l;
      if (dup) continue;
      if (is_dev_lock(l)) {
        if (dev_holder[l] != UINT32_MAX) continue;
        dev_holder[l] = t;
        if (held[t].empty()) held_in_block[b]++;
        held[t].push_back({l, DEVICE});
        emit(t, ACQ, DEVICE, 0, l);
      } else {
        uint32_t& h = blk_holder[size_t(l) * B + b];
        if (h != UINT32_MAX) continue;
        h = t;
        if (held[t].empty()) held_in_block[b]++;
        held[t].push_back({l, CTA});
        emit(t, ACQ, CTA, 0, l);
      }
      return true;
    }
    return false;
  };
  auto release = [&](uint32_t t) {
    const uint32_t b = block_of(t);
    Held h = held[t].back();
    held[t].pop_back();
    if (h.scope == DEVICE)
      dev_holder[h.lock] = UINT32_MAX;
    else
      blk_holder[size_t(h.lock) * B + b] = UINT32_MAX;
    if (held[t].empty()) held_in_block[b]--;
    emit(t, REL, h.scope, 0, h.lock);
  };

  const double p_rel = p->cs_len_mean > 0 ? 1.0 / p->cs_len_mean : 1.0;
  while (i < n) {
    if (next_plant < plant_at.size() && i >= plant_at[next_plant]) {
      uint32_t t = uint32_t(rng.below(W));
      if (held[t].empty()) {
        planted(t, true);
        ++next_plant;
        continue;
      }
    }
    double u = rng.uniform();
    if (u < p->p_barrier) {
      uint32_t b = uint32_t(rng.below(B));
      if (held_in_block[b] == 0) {
        if (p->granularity == 0 && apb > 1 && rng.uniform() < p->p_syncwarp) {
          uint32_t nwarps = (apb + 31) / 32;
          uint32_t w = uint32_t(rng.below(nwarps));
          uint32_t lanes = std::min<uint32_t>(32, apb - w * 32);
          uint64_t mask = lanes == 32 ? 0xffffffffull : ((1ull << lanes) - 1);
          emit(b * apb + w * 32, BARRIER, WARPSC, 0, mask);
        } else {
          emit(b * apb, BARRIER, CTA, 0, b);
          phase[b]++;
        }
      }
      continue;
    }
    uint32_t t = uint32_t(rng.below(W));
    const uint32_t b = block_of(t);
    if (!held[t].empty()) {
      double v = rng.uniform();
      if (v < p_rel) {
        release(t);
      } else if (v < p_rel + p->nest_prob * p_rel && held[t].size() < 2) {
        if (!try_acquire(t)) access(t, rng.uniform());
      } else if (v < 0.6) {
        // an access to an address guarded by the innermost held lock
        const Held& h = held[t].back();
        uint32_t j = uint32_t(rng.below(4));
        double c = rng.uniform();
        emit(t, c < 0.5 ? READ : WRITE, 0, 0, l_addr(h.lock, b, j));
      } else {
        access(t, rng.uniform());
      }
      continue;
    }
    double tot = p->p_read + p->p_write + p->p_atomic + p_acq + p->p_fence;
    double v = rng.uniform() * tot;
    if (v < p_acq) {
      if (!try_acquire(t)) access(t, rng.uniform());
    } else if (v < p_acq + p->p_fence) {
      emit(t, FENCE, rng.uniform() < 0.5 ? DEVICE : CTA, 0, 0);
    } else if (!p->n_plant_exact && rng.uniform() < p->plant_frac) {
      planted(t, false);
    } else {
      access(t, rng.uniform());
    }
  }
  *n_written = i;
  return 0;
}

}  // extern "C"
