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
  const uint32_t *sy_start, *sy_idx, *sy_kind, *sy_N, *sy_ver, *sy_aux;
  const uint32_t *incs_off, *incs_ver, *incs_k, *exp_off, *ex_dep_off, *ex_dep_cnt;
  const uint32_t* rowbase;
  const uint32_t *cs_of_sync, *cs_agent, *cs_sid, *cs_epoch, *cs_rel_idx, *cs_lock, *lock_cs_lo;
  const uint32_t *acq_dep_off, *acq_dep_cnt, *pool;
  uint32_t* rows;
  uint32_t *psnap, *hsnap, *done, *cursor;
  uint32_t *bar_j, *bar_cnt;
  uint32_t n_locks;
  int cta_barriers;
};

template <int K>
__device__ __forceinline__ void load_row(const uint32_t* row, uint32_t (&x)[K]) {
  const int lane = threadIdx.x & 31;
  const uint32_t* p = row + lane * K;
  if constexpr (K == 1) {
    x[0] = __ldcg(p);
  } else if constexpr (K == 2) {
    uint2 a = __ldcg(reinterpret_cast<const uint2*>(p));
    x[0] = a.x;
    x[1] = a.y;
  } else {
#pragma unroll
    for (int j = 0; j < K; j += 4) {
      uint4 a = __ldcg(reinterpret_cast<const uint4*>(p + j));
      x[j] = a.x;
      x[j + 1] = a.y;
      x[j + 2] = a.z;
      x[j + 3] = a.w;
    }
  }
}

template <int K>
__device__ __forceinline__ void store_row(uint32_t* row, const uint32_t (&x)[K]) {
  const int lane = threadIdx.x & 31;
  uint32_t* p = row + lane * K;
  if constexpr (K == 1) {
    __stcg(p, x[0]);
  } else if constexpr (K == 2) {
    __stcg(reinterpret_cast<uint2*>(p), make_uint2(x[0], x[1]));
  } else {
#pragma unroll
    for (int j = 0; j < K; j += 4) __stcg(reinterpret_cast<uint4*>(p + j), make_uint4(x[j], x[j + 1], x[j + 2], x[j + 3]));
  }
}

// the same blocked layout in shared memory (plain stores: __stcg is for global memory)
template <int K>
__device__ __forceinline__ void store_row_shared(uint32_t* row, const uint32_t (&x)[K]) {
  uint32_t* p = row + (threadIdx.x & 31) * K;
#pragma unroll
  for (int j = 0; j < K; ++j) p[j] = x[j];
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

// Bounded wait for a release's completion flag (lane 0 spins; the warp then reads the
// snapshot after __syncwarp, which orders it after lane 0's acquire).
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, bool& abort, DevStatus* st) {
  if (abort) return false;
  bool ok = true;
  if ((threadIdx.x & 31) == 0) {
    uint32_t it = 0;
    while (!ld_acquire(flag)) {
      if (++it > kSpinLimit) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
    if (!ok) atomicCAS(&st->code, 0, GWCP_ERR_TIMEOUT);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  if (!ok) abort = true;
  return ok;
}

template <int K>
__global__ void __launch_bounds__(1024) k_propagate(PropArgs a) {
  extern __shared__ uint32_t xchg[];  // CTA barriers: [2 buffers][warps][C | H][Wp]
  const Geo& g = a.g;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t u = a.cta_barriers ? blockIdx.x * g.apb + warp : blockIdx.x * 32 + warp;
  // one read of the status per CTA, so all warps of a CTA agree on whether to run
  __shared__ int start_code;
  if (threadIdx.x == 0) start_code = *(volatile int*)&a.st->code;
  __syncthreads();
  if (start_code) return;
  const bool active = a.cta_barriers ? (uint32_t(warp) < g.apb) : (u < g.W);
  if (!active) return;

  uint32_t P[K], H[K];
#pragma unroll
  for (int j = 0; j < K; ++j) P[j] = H[j] = 0;
  set_entry<K>(H, u, 1u);  // H_t = bottom{t := 1}, N_t = 1
  bool abort = false;
  uint64_t joins = 0, visits = 0;
  uint32_t nbar = 0;
  const uint32_t rb = a.rowbase[u];
  store_row<K>(a.rows + size_t(rb) * g.Wp, P);

  const uint32_t k0 = a.sy_start[u], k1 = a.sy_start[u + 1];
  uint32_t r = a.incs_off[k0];
  const uint32_t r1 = a.incs_off[k1];

  // Algorithm 2 for an in-section access: join L^w (and L^r for writes) of every held
  // lock, i.e. the H snapshots of the releases found by the per-location walk.
  auto in_section = [&](uint32_t rr) {
    for (uint32_t e = a.exp_off[rr]; e < a.exp_off[rr + 1]; ++e) {
      const uint32_t off = a.ex_dep_off[e], cnt = a.ex_dep_cnt[e];
      for (uint32_t q = 0; q < cnt; ++q) {
        const uint32_t d = a.pool[off + q];
        if (!wait_flag(a.done + d, abort, a.st)) continue;
        join_row<K>(P, a.hsnap + size_t(d) * g.Wp);
        ++joins;
      }
    }
    store_row<K>(a.rows + size_t(rb + a.incs_ver[rr]) * g.Wp, P);
  };

  for (uint32_t k = k0; k < k1; ++k) {
    while (r < r1 && a.incs_k[r] < k) in_section(r++);
    const uint32_t kind = a.sy_kind[k];
    if (kind == K_ACQ) {
      // Algorithm 1, acquire: P_t |= P_<l,s'>, H_t |= H_<l,s'> over overlapping scopes
      const uint32_t c = a.cs_of_sync[k];
      const uint32_t off = a.acq_dep_off[c], cnt = a.acq_dep_cnt[c];
      for (uint32_t q = 0; q < cnt; ++q) {
        const uint32_t d = a.pool[off + q];
        if (!wait_flag(a.done + d, abort, a.st)) continue;
        join_row<K>(P, a.psnap + size_t(d) * g.Wp);
        join_row<K>(H, a.hsnap + size_t(d) * g.Wp);
        joins += 2;
      }
    } else if (kind == K_REL) {
      // Algorithm 1, release: pop records of other agents' sections on this lock while
      // their acquire is ordered before C_t; join the released ones whose scope overlaps
      const uint32_t c = a.cs_of_sync[k];
      const uint32_t L = a.cs_lock[c], s = a.cs_sid[c], my_idx = a.sy_idx[k];
      uint32_t* curp = a.cursor + size_t(u) * a.n_locks + L;
      uint32_t cur = *curp;
      const uint32_t lo = a.lock_cs_lo[L], hi = a.lock_cs_lo[L + 1];
      bool stop = false;
      while (!stop && lo + cur < hi) {
        const uint32_t rec = lo + cur + lane;
        uint32_t ag = NONE, ep = 0, rel = NONE, sd = 0;
        if (rec < hi) {
          ag = a.cs_agent[rec];
          ep = a.cs_epoch[rec];
          rel = a.cs_rel_idx[rec];
          sd = a.cs_sid[rec];
        }
        const uint32_t nb = min(32u, hi - (lo + cur));
        for (uint32_t i = 0; i < nb; ++i) {
          const uint32_t agi = __shfl_sync(0xffffffffu, ag, i);
          if (agi == u) {
            ++cur;
            continue;
          }
          ++visits;
          // acqC <= C_t, tested on the acquiring agent's entry (the acquire's epoch)
          const uint32_t epi = __shfl_sync(0xffffffffu, ep, i);
          if (epi > get_entry<K>(P, agi)) {
            stop = true;
            break;
          }
          ++cur;
          const uint32_t reli = __shfl_sync(0xffffffffu, rel, i);
          const uint32_t sdi = __shfl_sync(0xffffffffu, sd, i);
          if (reli != NONE && reli < my_idx && scopes_overlap(sdi, s)) {
            const uint32_t recid = lo + cur - 1;
            if (wait_flag(a.done + recid, abort, a.st)) {
              join_row<K>(P, a.hsnap + size_t(recid) * g.Wp);
              ++joins;
            }
          }
        }
      }
      if (lane == 0) *curp = cur;
      store_row<K>(a.psnap + size_t(c) * g.Wp, P);
      store_row<K>(a.hsnap + size_t(c) * g.Wp, H);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(a.done + c, 1u);
      set_entry<K>(H, u, get_entry<K>(H, u) + 1);  // N_t++, H_t[t]++
    } else {
      // Algorithm 1, sync: join C_t and H_t of every agent in the barrier's scope
      const uint32_t N_before = a.sy_N[k] - 1;
      uint32_t C[K];
#pragma unroll
      for (int j = 0; j < K; ++j) C[j] = P[j];
      set_entry<K>(C, u, N_before);
      const Event e = a.ev[a.sy_idx[k]];
      const BarMembers bm = barrier_members(e, g);
      if (bm.count == 1) {
#pragma unroll
        for (int j = 0; j < K; ++j) P[j] = C[j];
      } else if (a.cta_barriers && e.scope == GWCP_SCOPE_CTA) {
        uint32_t* buf = xchg + size_t(nbar & 1) * nwarps * 2 * g.Wp;
        store_row_shared<K>(buf + size_t(warp) * 2 * g.Wp, C);
        store_row_shared<K>(buf + size_t(warp) * 2 * g.Wp + g.Wp, H);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < K; ++j) P[j] = H[j] = 0;
        for (int w = 0; w < nwarps; ++w) {
          uint32_t c2[K], h2[K];
          const uint32_t* src = buf + size_t(w) * 2 * g.Wp + lane * K;
#pragma unroll
          for (int j = 0; j < K; ++j) {
            c2[j] = src[j];
            h2[j] = src[g.Wp + j];
            P[j] = max(P[j], c2[j]);
            H[j] = max(H[j], h2[j]);
          }
        }
        joins += 2 * nwarps;
        ++nbar;
      } else {
        const uint32_t bid = a.sy_aux[k];
        uint32_t* J = a.bar_j + size_t(bid) * 2 * g.Wp;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          atomicMax(J + lane * K + j, C[j]);
          atomicMax(J + g.Wp + lane * K + j, H[j]);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(a.bar_cnt + bid, 1u);
        if (!abort) {
          bool ok = true;
          if (lane == 0) {
            uint32_t it = 0;
            while (ld_acquire(a.bar_cnt + bid) < bm.count) {
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
        load_row<K>(J + g.Wp, H);
        joins += 2;
      }
      set_entry<K>(H, u, get_entry<K>(H, u) + 1);
    }
    store_row<K>(a.rows + size_t(rb + a.sy_ver[k]) * g.Wp, P);
  }
  while (r < r1) in_section(r++);
  if (lane == 0) {
    atomicAdd(&a.st->joins, (unsigned long long)joins);
    atomicAdd(&a.st->loop_visits, (unsigned long long)visits);
  }
}

template <int K>
int launch(const PropArgs& a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s) {
  auto kern = k_propagate<K>;
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

}  // namespace

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
    case 1: rc = launch<1>(a, grid, threads, smem, s); break;
    case 2: rc = launch<2>(a, grid, threads, smem, s); break;
    case 4: rc = launch<4>(a, grid, threads, smem, s); break;
    case 8: rc = launch<8>(a, grid, threads, smem, s); break;
    case 16: rc = launch<16>(a, grid, threads, smem, s); break;
    case 32: rc = launch<32>(a, grid, threads, smem, s); break;
    default: rc = GWCP_ERR_UNSUPPORTED;
  }
  p.end();
  return rc;
}

}  // namespace gwcp
