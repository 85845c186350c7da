// Device-wide primitives of libgwcp: exclusive scan of u32 and a stable LSD radix sort
// of (u64 key, u32 value) pairs restricted to the key bits that vary.
#include <atomic>

#include "gwcp_internal.cuh"

namespace gwcp {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;

__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[SC_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < SC_THREADS / 32 ? warp_tot[lane] : 0;
    uint32_t wi = warp_inclusive_scan(w);
    if (lane < SC_THREADS / 32) warp_tot[lane] = wi - w;
    if (lane == SC_THREADS / 32 - 1) *total = wi;
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + inc - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const uint32_t* in, size_t n, uint32_t* sums) {
  const size_t base = size_t(blockIdx.x) * SC_TILE + size_t(threadIdx.x) * SC_ITEMS;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j)
    if (base + j < n) s += in[base + j];
  __shared__ uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint32_t* sums, uint32_t nb, uint32_t* total) {
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nb; base += SC_THREADS) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < nb ? sums[i] : 0;
    uint32_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const uint32_t* in, uint32_t* out, size_t n, const uint32_t* sums) {
  const size_t base = size_t(blockIdx.x) * SC_TILE + size_t(threadIdx.x) * SC_ITEMS;
  uint32_t v[SC_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    s += v[j];
  }
  __shared__ uint32_t tot;
  uint32_t ex = block_exclusive_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    if (base + j < n) out[base + j] = ex;
    ex += v[j];
  }
}

constexpr int RS_THREADS = 256, RS_ITEMS = 8, RS_TILE = RS_THREADS * RS_ITEMS;

// a pair the filter of the first pass keeps
__device__ __forceinline__ bool radix_kept(uint64_t key, const RadixKeep& kp) {
  if (!kp.bits) return true;
  const uint32_t h = wl_bit(key >> kp.shift, kp.log2);
  return (__ldg(kp.bits + (h >> 5)) >> (h & 31)) & 1u;
}

__global__ void k_radix_hist(const uint64_t* keys, size_t n, const uint32_t* n_dev, int shift, uint32_t* hist,
                             uint32_t ntiles, RadixKeep kp) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  if (n_dev && *n_dev < n) n = *n_dev;  // the count may be known on the device only
  __syncthreads();
  const size_t base = size_t(blockIdx.x) * RS_TILE;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    size_t i = base + size_t(j) * RS_THREADS + threadIdx.x;
    if (i < n) {
      const uint64_t k = keys[i];
      if (radix_kept(k, kp)) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  hist[size_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of a tile owns items [w*256, w*256+256) of the tile, visited in
// rounds of 32 consecutive items; ranks within a round follow lane order. The tile is
// first put in digit order in shared memory, then written out so that consecutive threads
// write consecutive positions of one digit's run (coalesced stores instead of one sector
// per item). Five blocks per SM (48 registers; 60 allowed only four): measured 0.75 ms
// faster per 200M-event analysis; six spill.
__global__ void __launch_bounds__(RS_THREADS, 5) k_radix_scatter(const uint64_t* kin, const uint32_t* vin,
                                                              uint64_t* kout, uint32_t* vout, size_t n,
                                                              const uint32_t* n_dev, int shift,
                                                              const uint32_t* offs, uint32_t ntiles,
                                                              RadixKeep kp) {
  if (n_dev && *n_dev < n) n = *n_dev;
  __shared__ uint32_t cnt[RS_THREADS / 32][256];
  __shared__ uint32_t tile_off[256];  // first position of each digit in the tile's digit order
  __shared__ uint32_t glob[256];      // global position of the tile's first item of each digit
  __shared__ uint64_t sk[RS_TILE];
  __shared__ uint32_t sv[RS_TILE];
  __shared__ uint32_t tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) cnt[warp][d] = 0;
  __syncwarp();
  const size_t tile_base = size_t(blockIdx.x) * RS_TILE;
  const size_t base = tile_base + size_t(warp) * (RS_ITEMS * 32);
  uint64_t k[RS_ITEMS];
  uint32_t v[RS_ITEMS], dig[RS_ITEMS], rank[RS_ITEMS];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    size_t i = base + size_t(r) * 32 + lane;
    k[r] = i < n ? kin[i] : 0;
    const bool valid = i < n && radix_kept(k[r], kp);
    v[r] = (valid && vin) ? vin[i] : 0;
    uint32_t d = valid ? uint32_t((k[r] >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = __popc(peers & lt);
    uint32_t b0 = valid ? cnt[warp][d] : 0;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
    __syncwarp();
    rank[r] = b0 + before;
    dig[r] = d;
  }
  __syncthreads();
  {
    const uint32_t d = threadIdx.x;  // one digit per thread: warp prefixes, tile count
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) {
      uint32_t t = cnt[w][d];
      cnt[w][d] = run;
      run += t;
    }
    glob[d] = offs[size_t(d) * ntiles + blockIdx.x];
    tile_off[d] = block_exclusive_scan(run, &tot);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (dig[r] < 256) {
      const uint32_t lp = tile_off[dig[r]] + cnt[warp][dig[r]] + rank[r];
      sk[lp] = k[r];
      sv[lp] = v[r];
    }
  }
  __syncthreads();
  const uint32_t nvalid = tot;  // the tile's (kept) pairs, in digit order in sk / sv
  for (uint32_t i = threadIdx.x; i < nvalid; i += RS_THREADS) {
    const uint64_t key = sk[i];
    const uint32_t d = uint32_t((key >> shift) & 255u);
    const uint32_t pos = glob[d] + (i - tile_off[d]);
    kout[pos] = key;
    if (vout) vout[pos] = sv[i];
  }
}

}  // namespace

size_t scan_tmp_need(size_t n) { return (n + SC_TILE - 1) / SC_TILE + 1; }

void scan_exclusive(const uint32_t* in, uint32_t* out, size_t n, uint32_t* total_dev, uint32_t* tmp,
                    cudaStream_t s) {
  if (n == 0) {
    if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
    return;
  }
  const uint32_t nb = uint32_t((n + SC_TILE - 1) / SC_TILE);
  k_scan_reduce<<<nb, SC_THREADS, 0, s>>>(in, n, tmp);
  count_launch();
  k_scan_sums<<<1, SC_THREADS, 0, s>>>(tmp, nb, total_dev);
  count_launch();
  k_scan_apply<<<nb, SC_THREADS, 0, s>>>(in, out, n, tmp);
  count_launch();
}

std::vector<int> radix_windows(uint64_t mask) {
  std::vector<int> w;
  int b = 0;
  while (b < 64) {
    if (!((mask >> b) & 1)) {
      ++b;
      continue;
    }
    int lo = b > 56 ? 56 : b;
    w.push_back(lo);
    b = lo + 8;
  }
  return w;
}

size_t radix_tmp_need(size_t n) {
  size_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  return 256 * ntiles + scan_tmp_need(256 * ntiles) + 1;
}

bool radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, size_t n, uint64_t mask,
                      uint32_t* tmp, cudaStream_t s, const uint32_t* n_dev, RadixKeep keep) {
  if (keep.bits) {
    if (n == 0) {
      cudaMemsetAsync(keep.n_out, 0, 4, s);
      return false;
    }
    if (mask == 0) mask = 1;  // the filter needs one pass
  } else if (n <= 1) {
    return false;
  }
  const uint32_t ntiles = uint32_t((n + RS_TILE - 1) / RS_TILE);
  uint32_t* hist = tmp;
  uint32_t* stmp = tmp + size_t(256) * ntiles;
  bool in_second = false, first = true;
  for (int lo : radix_windows(mask)) {
    uint64_t* kin = in_second ? k1 : k0;
    uint32_t* vin = in_second ? v1 : v0;
    uint64_t* kout = in_second ? k0 : k1;
    uint32_t* vout = in_second ? v0 : v1;
    const RadixKeep kp = first ? keep : RadixKeep{};
    first = false;
    k_radix_hist<<<ntiles, RS_THREADS, 0, s>>>(kin, n, n_dev, lo, hist, ntiles, kp);
    count_launch();
    scan_exclusive(hist, hist, size_t(256) * ntiles, kp.bits ? kp.n_out : nullptr, stmp, s);
    k_radix_scatter<<<ntiles, RS_THREADS, 0, s>>>(kin, vin, kout, vout, n, n_dev, lo, hist, ntiles, kp);
    count_launch();
    if (kp.bits) n_dev = kp.n_out;  // later passes sort the kept pairs
    in_second = !in_second;
  }
  return in_second;
}

}  // namespace gwcp
