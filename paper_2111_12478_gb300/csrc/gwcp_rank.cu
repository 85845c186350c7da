// Address ranker: per-location features, a BF16 MLP 16 -> 64 -> 64 -> 1 (inference on
// the tensor cores, training with hand-written gradient and Adam kernels), and the ranked
// order of the per-location check. Not from the paper: the ranker only reorders the
// check's work so that locations likely to race are checked first; every location is
// still checked and the race set is unchanged.
//
// Features of a location (its accesses in trace order), 16 floats:
//   0 log1p(n)  1 log1p(reads)  2 log1p(writes)  3 log1p(atomics)
//   4 log1p(distinct agent mod 64)  5 log1p(distinct block mod 64)
//   6 block-scoped atomics / n  7 device-scoped atomics / n  8 accesses in a section / n
//   9 shared-memory location  10 (acquires, releases, barriers in [first, last]) / span
//   11 log1p(last - first)  12 share of the first access's agent
//   13 agent switches / max(n-1, 1)  14 agent switches with a write or atomic / max(n-1, 1)
//   15 writes and atomics in a section / max(writes + atomics, 1)
// Network: z1 = bf(x) bf(W1)^T + b1, h1 = bf(relu(z1)), z2 = h1 bf(W2)^T + b2,
// h2 = relu(z2), s = h2 . w3 + b3 (bf = round to bfloat16; parameters in one float
// vector: W1[64][16], b1, W2[64][64], b2, w3, b3).
#include <cuda_bf16.h>

#include <algorithm>

#include "gwcp_internal.cuh"

namespace gwcp {

namespace {

constexpr int NF = 16, NH = 64;
constexpr int P_W1 = 0, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH,
              P_B3 = P_W3 + NH, N_PARAMS = P_B3 + 1;
static_assert(N_PARAMS == kRankParams, "parameter layout");

// per-location counters
enum { A_N, A_R, A_W, A_A, A_CTA, A_DEV, A_INS, A_INSW, A_FIRST, A_SW, A_CSW, A_COUNT };

inline uint32_t nblk(uint64_t n, uint32_t t) { return uint32_t((n + t - 1) / t); }

__global__ void k_rk_incs(const uint32_t* incs_idx, uint32_t n_incs, uint32_t* bits) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_incs) atomicOr(bits + (incs_idx[r] >> 5), 1u << (incs_idx[r] & 31));
}

__global__ void k_rk_flags(const uint64_t* key, uint32_t n, uint32_t* flag) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
  if (i == n) flag[n] = 0u;  // so that the scan's total counts the locations
}

__global__ void k_rk_starts(const uint32_t* flag, const uint32_t* excl, uint32_t n, uint32_t* loc_start) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) loc_start[excl[i]] = i;
  if (i == 0) loc_start[excl[n]] = n;  // excl[n] = number of locations
}

struct AccArgs {
  const uint64_t* key;
  const uint32_t* idx;
  const AccInfo* info;
  const uint32_t *flag, *excl, *loc_start, *bits;
  uint32_t n;
  uint32_t stride;  // entries per counter array
  uint32_t* cnt;    // [A_COUNT][stride]
  unsigned long long* masks;  // [2][stride]: agents mod 64, blocks mod 64
};

// One warp per 32 sorted accesses: each lane's contribution, reduced over the runs of one
// location inside the warp; a run that the warp holds whole is stored, one that crosses
// a warp boundary is added atomically.
__global__ void k_rk_acc(AccArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
  if (base >= a.n) return;
  const uint32_t i = base + lane;
  const bool valid = i < a.n;
  const uint32_t flag = valid ? a.flag[i] : 1u;
  const uint32_t loc = valid ? a.excl[i] + flag - 1u : 0u;
  const uint32_t ix = valid ? a.idx[i] : 0u;
  const uint32_t who = valid ? a.info[ix].who : 0u;
  const uint32_t agent = who_agent(who), cls = who_class(who), blk = who_block(who);
  const bool wc = cls != C_READ;
  const bool ins = valid && ((a.bits[ix >> 5] >> (ix & 31)) & 1u);
  // the previous access of the same location
  uint32_t pagent = __shfl_up_sync(0xffffffffu, agent, 1);
  uint32_t pwc = __shfl_up_sync(0xffffffffu, uint32_t(wc), 1);
  const bool has_prev = valid && !flag;
  if (lane == 0 && has_prev) {
    const uint32_t pw = a.info[a.idx[i - 1]].who;
    pagent = who_agent(pw);
    pwc = who_class(pw) != C_READ;
  }
  // runs inside the warp: heads and ends
  const uint32_t starts = __ballot_sync(0xffffffffu, flag != 0u || lane == 0);
  const uint32_t le = lanemask_lt() | (1u << lane);
  const uint32_t head = 31u - __clz(starts & le);
  const uint32_t above = starts & ~le;
  const uint32_t end = above ? uint32_t(__ffs(above)) - 2u : 31u;
  // agent of the location's first access
  uint32_t fagent = __shfl_sync(0xffffffffu, agent, head);
  const uint32_t head_flag = __shfl_sync(0xffffffffu, flag, head);
  if (valid && !head_flag) fagent = who_agent(a.info[a.idx[a.loc_start[loc]]].who);
  uint32_t v[A_COUNT];
  v[A_N] = valid;
  v[A_R] = valid && cls == C_READ;
  v[A_W] = valid && cls == C_WRITE;
  v[A_A] = valid && cls >= C_ATOM_CTA;
  v[A_CTA] = valid && cls == C_ATOM_CTA;
  v[A_DEV] = valid && cls == C_ATOM_DEV;
  v[A_INS] = ins;
  v[A_INSW] = ins && wc;
  v[A_FIRST] = valid && agent == fagent;
  v[A_SW] = has_prev && agent != pagent;
  v[A_CSW] = has_prev && agent != pagent && (wc || pwc);
  unsigned long long am = valid ? 1ull << (agent & 63u) : 0ull, bm = valid ? 1ull << (blk & 63u) : 0ull;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const bool take = lane + o <= end;
#pragma unroll
    for (int q = 0; q < A_COUNT; ++q) {
      const uint32_t t = __shfl_down_sync(0xffffffffu, v[q], o);
      if (take) v[q] += t;
    }
    const unsigned long long ta = __shfl_down_sync(0xffffffffu, am, o);
    const unsigned long long tb = __shfl_down_sync(0xffffffffu, bm, o);
    if (take) {
      am |= ta;
      bm |= tb;
    }
  }
  if (!valid || head != lane) return;
  // the run is the location whole when it starts at the location's first access and the
  // location ends inside the warp
  const bool owned = flag && (end < 31u || base + 32u >= a.n || a.flag[base + 32u]);
  if (owned) {
#pragma unroll
    for (int q = 0; q < A_COUNT; ++q) a.cnt[size_t(q) * a.stride + loc] = v[q];
    a.masks[loc] = am;
    a.masks[size_t(a.stride) + loc] = bm;
  } else {
#pragma unroll
    for (int q = 0; q < A_COUNT; ++q)
      if (v[q]) atomicAdd(a.cnt + size_t(q) * a.stride + loc, v[q]);
    atomicOr(a.masks + loc, am);
    atomicOr(a.masks + size_t(a.stride) + loc, bm);
  }
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* p, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t m = (lo + hi) >> 1;
    if (p[m] < x) lo = m + 1; else hi = m;
  }
  return lo;
}

struct FinalArgs {
  const uint64_t* key;
  const uint32_t* idx;
  const uint32_t* loc_start;
  const uint32_t* n_loc;  // device count
  uint32_t n, stride;
  const uint32_t* cnt;
  const unsigned long long* masks;
  const uint32_t *acqrel, *bar;  // sync events in trace order
  uint32_t n_acqrel, n_bar;
  float* feat;      // [n_loc][16]
  uint64_t* loc_key;
};

__global__ void k_rk_final(FinalArgs a) {
  const uint32_t L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= *a.n_loc) return;
  const uint32_t lo = a.loc_start[L], hi = a.loc_start[L + 1];
  const uint32_t first = a.idx[lo], last = a.idx[hi - 1];
  const uint64_t k = a.key[lo];
  uint32_t c[A_COUNT];
#pragma unroll
  for (int q = 0; q < A_COUNT; ++q) c[q] = a.cnt[size_t(q) * a.stride + L];
  const uint32_t sync = (lower_bound_u32(a.acqrel, a.n_acqrel, last + 1) - lower_bound_u32(a.acqrel, a.n_acqrel, first)) +
                        (lower_bound_u32(a.bar, a.n_bar, last + 1) - lower_bound_u32(a.bar, a.n_bar, first));
  const float n = float(c[A_N]);
  const float span = float(last - first);
  const float pairs = float(max(c[A_N], 2u) - 1u);
  float f[NF];
  f[0] = log1pf(n);
  f[1] = log1pf(float(c[A_R]));
  f[2] = log1pf(float(c[A_W]));
  f[3] = log1pf(float(c[A_A]));
  f[4] = log1pf(float(__popcll(a.masks[L])));
  f[5] = log1pf(float(__popcll(a.masks[size_t(a.stride) + L])));
  f[6] = float(c[A_CTA]) / n;
  f[7] = float(c[A_DEV]) / n;
  f[8] = float(c[A_INS]) / n;
  f[9] = (k >> 63) ? 1.0f : 0.0f;
  f[10] = float(sync) / (span + 1.0f);
  f[11] = log1pf(span);
  f[12] = float(c[A_FIRST]) / n;
  f[13] = float(c[A_SW]) / pairs;
  f[14] = float(c[A_CSW]) / pairs;
  f[15] = float(c[A_INSW]) / float(max(c[A_W] + c[A_A], 1u));
  float4* o = reinterpret_cast<float4*>(a.feat + size_t(L) * NF);
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
  a.loc_key[L] = k;
}

// ---- MLP inference on the tensor cores ------------------------------------------------

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One warp scores 16 locations per step: layer 1 is one k-step of 8 n-tiles, layer 2 four
// k-steps of 8 n-tiles whose A fragments are layer 1's accumulators (same lanes, same
// rows), layer 3 a dot product over the accumulator fragments and the 4 lanes of a row.
__global__ void __launch_bounds__(256) k_mlp_fwd(const float* theta, const float* feat, const uint32_t* n_dev,
                                                 uint32_t n_host, float* score) {
  __shared__ uint32_t sW1[NH * NF / 2];  // bf16 pairs, row-major [64][16]
  __shared__ uint32_t sW2[NH * NH / 2];  // [64][64]
  __shared__ float sb1[NH], sb2[NH], sw3[NH];
  for (int p = threadIdx.x; p < NH * NF / 2; p += blockDim.x)
    sW1[p] = pack_bf16(theta[P_W1 + 2 * p], theta[P_W1 + 2 * p + 1]);
  for (int p = threadIdx.x; p < NH * NH / 2; p += blockDim.x)
    sW2[p] = pack_bf16(theta[P_W2 + 2 * p], theta[P_W2 + 2 * p + 1]);
  for (int p = threadIdx.x; p < NH; p += blockDim.x) {
    sb1[p] = theta[P_B1 + p];
    sb2[p] = theta[P_B2 + p];
    sw3[p] = theta[P_W3 + p];
  }
  __syncthreads();
  const float b3 = theta[P_B3];
  const uint32_t n = n_dev ? *n_dev : n_host;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; size_t(tile) * 16 < n; tile += warps) {
    const uint32_t r0 = tile * 16 + g, r1 = r0 + 8;
    float x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0};  // cols 2t, 2t+1, 2t+8, 2t+9
    if (r0 < n) {
      const float* p = feat + size_t(r0) * NF;
      x0[0] = p[2 * t], x0[1] = p[2 * t + 1], x0[2] = p[2 * t + 8], x0[3] = p[2 * t + 9];
    }
    if (r1 < n) {
      const float* p = feat + size_t(r1) * NF;
      x1[0] = p[2 * t], x1[1] = p[2 * t + 1], x1[2] = p[2 * t + 8], x1[3] = p[2 * t + 9];
    }
    const uint32_t a0 = pack_bf16(x0[0], x0[1]), a1 = pack_bf16(x1[0], x1[1]);
    const uint32_t a2 = pack_bf16(x0[2], x0[3]), a3 = pack_bf16(x1[2], x1[3]);
    uint32_t h[8][2];  // layer-1 output as bf16 pairs: [n-tile][row g / row g+8]
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float d[4] = {0, 0, 0, 0};
      const int row = 8 * j + g;
      mma_bf16(d, a0, a1, a2, a3, sW1[row * 8 + t], sW1[row * 8 + t + 4]);
      const float c0 = sb1[8 * j + 2 * t], c1 = sb1[8 * j + 2 * t + 1];
      h[j][0] = pack_bf16(fmaxf(d[0] + c0, 0.f), fmaxf(d[1] + c1, 0.f));
      h[j][1] = pack_bf16(fmaxf(d[2] + c0, 0.f), fmaxf(d[3] + c1, 0.f));
    }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float d[4] = {0, 0, 0, 0};
      const int row = 8 * j + g;
#pragma unroll
      for (int kb = 0; kb < 4; ++kb)
        mma_bf16(d, h[2 * kb][0], h[2 * kb][1], h[2 * kb + 1][0], h[2 * kb + 1][1], sW2[row * 32 + 8 * kb + t],
                 sW2[row * 32 + 8 * kb + t + 4]);
      const int c = 8 * j + 2 * t;
      s0 += fmaxf(d[0] + sb2[c], 0.f) * sw3[c] + fmaxf(d[1] + sb2[c + 1], 0.f) * sw3[c + 1];
      s1 += fmaxf(d[2] + sb2[c], 0.f) * sw3[c] + fmaxf(d[3] + sb2[c + 1], 0.f) * sw3[c + 1];
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    if (t == 0) {
      if (r0 < n) score[r0] = s0 + b3;
      if (r1 < n) score[r1] = s1 + b3;
    }
  }
}

// ---- training: loss gradient over a batch, Adam ---------------------------------------

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One thread per sample: forward with the inference roundings, backward with the roundings
// taken as the identity; gradients summed over the warp, then the block (shared memory),
// then added to `grad`. Scaled by inv_b (1 / batch size).
__global__ void __launch_bounds__(128) k_mlp_grad(const float* theta, const float* feat, const float* y, uint32_t lo,
                                                  uint32_t hi, float pos_weight, float inv_b, float* grad,
                                                  float* loss) {
  __shared__ float sW1[NH * NF], sW2[NH * NH], sb1[NH], sb2[NH], sw3[NH];
  __shared__ float G[N_PARAMS];
  for (int p = threadIdx.x; p < NH * NF; p += blockDim.x) sW1[p] = bf16r(theta[P_W1 + p]);
  for (int p = threadIdx.x; p < NH * NH; p += blockDim.x) sW2[p] = bf16r(theta[P_W2 + p]);
  for (int p = threadIdx.x; p < NH; p += blockDim.x) {
    sb1[p] = theta[P_B1 + p];
    sb2[p] = theta[P_B2 + p];
    sw3[p] = theta[P_W3 + p];
  }
  for (int p = threadIdx.x; p < N_PARAMS; p += blockDim.x) G[p] = 0.f;
  __syncthreads();
  const uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < hi;
  float x[NF], h1[NH], h2[NH];
  unsigned long long m1 = 0, m2 = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) x[f] = valid ? bf16r(feat[size_t(i) * NF + f]) : 0.f;
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    float z = sb1[k];
#pragma unroll
    for (int f = 0; f < NF; ++f) z = fmaf(sW1[k * NF + f], x[f], z);
    m1 |= (z > 0.f ? 1ull : 0ull) << k;
    h1[k] = bf16r(fmaxf(z, 0.f));
  }
  float s = theta[P_B3];
#pragma unroll
  for (int n = 0; n < NH; ++n) {
    float z = sb2[n];
#pragma unroll 16
    for (int k = 0; k < NH; ++k) z = fmaf(sW2[n * NH + k], h1[k], z);
    m2 |= (z > 0.f ? 1ull : 0ull) << n;
    h2[n] = fmaxf(z, 0.f);
    s = fmaf(h2[n], sw3[n], s);
  }
  const float yi = valid ? y[i] : 0.f;
  const float wt = yi > 0.f ? pos_weight : 1.f;
  const float sig = 1.f / (1.f + __expf(-s));
  const float ds = valid ? wt * (sig - yi) * inv_b : 0.f;
  const float li = valid ? wt * (fmaxf(s, 0.f) + log1pf(__expf(-fabsf(s))) - yi * s) * inv_b : 0.f;
  const int lane = threadIdx.x & 31;
  // output layer
  {
    const float t = warp_sum(ds);
    if (lane == 0) atomicAdd(&G[P_B3], t);
    const float l = warp_sum(li);
    if (lane == 0) atomicAdd(loss, l);
  }
  for (int n = 0; n < NH; ++n) {
    const float t = warp_sum(ds * h2[n]);
    if (lane == 0) atomicAdd(&G[P_W3 + n], t);
  }
  // dz2 in place of h2
#pragma unroll
  for (int n = 0; n < NH; ++n) h2[n] = ((m2 >> n) & 1ull) ? ds * sw3[n] : 0.f;
  for (int n = 0; n < NH; ++n) {
    const float dz = h2[n];
    if (__any_sync(0xffffffffu, dz != 0.f)) {
      const float t = warp_sum(dz);
      if (lane == 0) atomicAdd(&G[P_B2 + n], t);
      for (int k = 0; k < NH; ++k) {
        const float u = warp_sum(dz * h1[k]);
        if (lane == 0) atomicAdd(&G[P_W2 + n * NH + k], u);
      }
    }
  }
  // dz1 in place of h1
#pragma unroll
  for (int k = 0; k < NH; ++k) {
    float dh = 0.f;
#pragma unroll 16
    for (int n = 0; n < NH; ++n) dh = fmaf(h2[n], sW2[n * NH + k], dh);
    h1[k] = ((m1 >> k) & 1ull) ? dh : 0.f;
  }
  for (int k = 0; k < NH; ++k) {
    const float dz = h1[k];
    if (__any_sync(0xffffffffu, dz != 0.f)) {
      const float t = warp_sum(dz);
      if (lane == 0) atomicAdd(&G[P_B1 + k], t);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float u = warp_sum(dz * x[f]);
        if (lane == 0) atomicAdd(&G[P_W1 + k * NF + f], u);
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < N_PARAMS; p += blockDim.x)
    if (G[p] != 0.f) atomicAdd(grad + p, G[p]);
}

__global__ void k_adam(float* theta, float* m, float* v, float* grad, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N_PARAMS) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
  grad[p] = 0.f;
}

// Adam with the step count in device memory (one epoch of steps is a replayable graph):
// step t = *step + 1; bias corrections 1 / (1 - beta^t)
__global__ void k_adam_dev(float* theta, float* m, float* v, float* grad, float lr, const uint32_t* step) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N_PARAMS) return;
  const float t = float(*step + 1);
  const float c1 = 1.f / (1.f - powf(0.9f, t)), c2 = 1.f / (1.f - powf(0.999f, t));
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
  grad[p] = 0.f;
}

__global__ void k_step_inc(uint32_t* step) { ++*step; }

// end of an epoch: its accumulated loss into losses[epoch], then the next epoch
__global__ void k_epoch_end(float* loss_acc, float* losses, uint32_t* epoch) {
  losses[*epoch] = *loss_acc;
  *loss_acc = 0.f;
  ++*epoch;
}

// ---- ranked order of the check --------------------------------------------------------

// key = (16 bits of the score, high scores first) << 32 | location ordinal
__global__ void k_rk_compose(const uint32_t* flag, const uint32_t* excl, const float* score, uint32_t n, uint64_t* rkey,
                             uint32_t* rval) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t loc = excl[i] + flag[i] - 1u;
  uint32_t b = __float_as_uint(score[loc]);
  b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // order-preserving
  const uint32_t q = (~b) >> 16;                     // descending
  rkey[i] = (uint64_t(q) << 32) | loc;
  rval[i] = i;
}

__global__ void k_rk_gather(const uint32_t* pos, uint32_t n, const uint64_t* key, const uint32_t* idx, uint64_t* key_out,
                            uint32_t* idx_out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t p = pos[i];
  key_out[i] = key[p];
  idx_out[i] = idx[p];
}

__global__ void k_stamp(unsigned long long* at) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *at = t;
}

}  // namespace

void stamp_now(unsigned long long* at, cudaStream_t s) {
  k_stamp<<<1, 1, 0, s>>>(at);
  count_launch();
}

size_t rank_tmp_words(uint32_t n_acc) {
  // flag, excl (n + 1), loc_start (n + 1), counters, masks (u64), in-section bits
  const size_t s = size_t(n_acc) + 1;
  return 3 * s + 1 + A_COUNT * s + 4 * s + 64;
}

void rank_features(const RankIn& in, uint32_t* tmp, size_t bits_words, float* feat, uint64_t* loc_key,
                   uint32_t* n_loc_dev, uint32_t* scan_tmp, cudaStream_t s) {
  const uint32_t n = in.n_acc;
  const size_t st = size_t(n) + 1;
  uint32_t* flag = tmp;
  uint32_t* excl = flag + st;
  uint32_t* loc_start = excl + st;
  uint32_t* cnt = loc_start + st + 1;
  size_t mw = 3 * st + 1 + A_COUNT * st;
  mw += mw & 1;  // 8-byte alignment of the masks (tmp itself is 256-byte aligned)
  auto* masks = reinterpret_cast<unsigned long long*>(tmp + mw);
  uint32_t* bits = in.bits;
  cudaMemsetAsync(bits, 0, bits_words * 4, s);
  if (in.n_incs) {
    k_rk_incs<<<nblk(in.n_incs, 256), 256, 0, s>>>(in.incs_idx, in.n_incs, bits);
    count_launch();
  }
  k_rk_flags<<<nblk(uint64_t(n) + 1, 256), 256, 0, s>>>(in.key, n, flag);
  count_launch();
  scan_exclusive(flag, excl, size_t(n) + 1, n_loc_dev, scan_tmp, s);
  k_rk_starts<<<nblk(n, 256), 256, 0, s>>>(flag, excl, n, loc_start);
  count_launch();
  cudaMemsetAsync(cnt, 0, size_t(A_COUNT) * st * 4, s);
  cudaMemsetAsync(masks, 0, 2 * st * 8, s);
  AccArgs a{in.key, in.idx, in.info, flag, excl, loc_start, bits, n, uint32_t(st), cnt, masks};
  k_rk_acc<<<nblk(uint64_t(nblk(n, 32)) * 32, 256), 256, 0, s>>>(a);
  count_launch();
  FinalArgs f{in.key, in.idx, loc_start, n_loc_dev, n, uint32_t(st), cnt, masks, in.acqrel, in.bar,
              in.n_acqrel, in.n_bar, feat, loc_key};
  k_rk_final<<<nblk(n, 256), 256, 0, s>>>(f);
  count_launch();
}

void rank_scores(const float* theta, const float* feat, const uint32_t* n_dev, uint32_t n_bound, float* score,
                 cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t tiles = nblk(n_bound, 16);
  const uint32_t grid = std::max(1u, std::min<uint32_t>(nblk(tiles, 8), uint32_t(sms) * 8));
  k_mlp_fwd<<<grid, 256, 0, s>>>(theta, feat, n_dev, n_bound, score);
  count_launch();
}

void rank_order(const RankIn& in, const uint32_t* tmp, const float* score, uint64_t* rkey, uint32_t* rval,
                uint64_t* rkey2, uint32_t* rval2, uint64_t* key_out, uint32_t* idx_out, uint32_t* sort_tmp,
                cudaStream_t s) {
  const uint32_t n = in.n_acc;
  const size_t st = size_t(n) + 1;
  const uint32_t* flag = tmp;
  const uint32_t* excl = flag + st;
  k_rk_compose<<<nblk(n, 256), 256, 0, s>>>(flag, excl, score, n, rkey, rval);
  count_launch();
  uint64_t mask = 0xFFFFull << 32;
  for (uint64_t v = n; v; v >>= 1) mask |= (mask & 0xFFFFFFFFull) << 1 | 1;
  const bool second = radix_sort_pairs(rkey, rval, rkey2, rval2, n, mask, sort_tmp, s);
  k_rk_gather<<<nblk(n, 256), 256, 0, s>>>(second ? rval2 : rval, n, in.key, in.idx, key_out, idx_out);
  count_launch();
}

int rank_grad(const float* theta, const float* feat, const float* y, uint32_t lo, uint32_t hi, float pos_weight,
              float inv_b, float* grad, float* loss, cudaStream_t s) {
  if (hi <= lo) return GWCP_OK;
  k_mlp_grad<<<nblk(hi - lo, 128), 128, 0, s>>>(theta, feat, y, lo, hi, pos_weight, inv_b, grad, loss);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
}

// One epoch of training as launches on stream s: per batch the gradient, Adam and the
// step count; then the epoch's loss. Counters: ctr[0] Adam steps, ctr[1] epochs.
int rank_epoch(float* theta, const float* feat, const float* y, uint32_t n, uint32_t batch, float lr,
               float pos_weight, float* m, float* v, float* grad, float* loss_acc, float* losses, uint32_t* ctr,
               cudaStream_t s) {
  const uint32_t nb = (n + batch - 1) / batch;
  for (uint32_t q = 0; q < nb; ++q) {
    const uint32_t lo = q * batch, hi = std::min(n, lo + batch);
    int rc = rank_grad(theta, feat, y, lo, hi, pos_weight, 1.0f / float(hi - lo) / float(nb), grad, loss_acc, s);
    if (rc) return rc;
    k_adam_dev<<<nblk(N_PARAMS, 256), 256, 0, s>>>(theta, m, v, grad, lr, ctr);
    count_launch();
    k_step_inc<<<1, 1, 0, s>>>(ctr);
    count_launch();
  }
  k_epoch_end<<<1, 1, 0, s>>>(loss_acc, losses, ctr + 1);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? GWCP_OK : GWCP_ERR_CUDA;
}

void rank_adam(float* theta, float* m, float* v, float* grad, float lr, float c1, float c2, cudaStream_t s) {
  k_adam<<<nblk(N_PARAMS, 256), 256, 0, s>>>(theta, m, v, grad, lr, c1, c2);
  count_launch();
}

}  // namespace gwcp
