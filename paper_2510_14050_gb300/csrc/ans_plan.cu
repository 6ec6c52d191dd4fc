// Device-side planning of a batch whose window offsets live in device
// memory (Sec. III-C batching with the offsets produced on the GPU).
//
// The host knows only the number of windows and a capacity (an upper bound
// on the batch's packets); it sizes scratch and grids for that bound.  This
// kernel turns the offsets into the plan every other kernel reads -- each
// window's input offset, length, padded start and first tile (an exclusive
// scan of the windows' tile counts), the hash path's per-window table sizes
// and offsets, and the time sum's matrix descriptors -- so that nothing
// returns to the host.  Tiles past the plan's last one find no items and
// leave at once.  Offsets that decrease, a window of 2^31 packets or more,
// or a batch above the capacity make every window empty and set kErrPlan in
// the context's error word; the batch then reports ANS_ERR_INVALID_ARG.
#include <algorithm>

#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr int kPlanThreads = 1024;

__device__ __forceinline__ uint32_t table_lg(uint64_t len) {
  uint32_t l = 13;  // at least one tile of slots
  while ((1ull << l) < 2 * len) ++l;
  return l;
}

// Block-wide exclusive scan of one uint64 per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ uint64_t scan_excl_u64(uint64_t v, uint64_t* tmp, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  uint64_t off = 0, tot = 0;
  for (int w = 0; w < kPlanThreads / 32; ++w) {
    const uint64_t s = tmp[w];
    off += w < warp ? s : 0ull;
    tot += s;
  }
  *total = tot;
  __syncthreads();
  return off + x - v;
}

__global__ void __launch_bounds__(kPlanThreads) k_plan(const uint64_t* __restrict__ off, uint32_t nseg, uint64_t cap,
                                                       DevPlanOut o, uint32_t* err) {
  __shared__ uint64_t s_tmp[kPlanThreads / 32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // validate: nondecreasing, every window below 2^31 packets, total within the capacity
  int bad = 0;
  for (uint32_t s = threadIdx.x; s < nseg; s += kPlanThreads) {
    const uint64_t a = off[s], b = off[s + 1];
    if (b < a || b - a > kMaxWindowItems) bad = 1;
  }
  if (threadIdx.x == 0 && off[nseg] >= off[0] && off[nseg] - off[0] > cap) bad = 1;
  if (bad) s_bad = 1;
  __syncthreads();
  const bool ok = s_bad == 0;
  if (!ok && threadIdx.x == 0) atomicOr(err, (uint32_t)kErrPlan);

  uint64_t tile_carry = 0, slot_carry = 0;
  for (uint32_t c0 = 0; c0 < nseg; c0 += kPlanThreads) {
    const uint32_t s = c0 + threadIdx.x;
    const bool in = s < nseg;
    const uint64_t len = in && ok ? off[s + 1] - off[s] : 0ull;
    const uint64_t tiles = (len + kTile - 1) / kTile;
    const uint64_t slots = len ? (1ull << table_lg(len)) : 0ull;
    uint64_t ttot, stot;
    const uint64_t tex = scan_excl_u64(tiles, s_tmp, &ttot);
    const uint64_t sex = scan_excl_u64(slots, s_tmp, &stot);
    if (in) {
      const uint64_t ft = tile_carry + tex;
      const uint64_t base = ft * kTile;
      o.in_off[s] = ok ? off[s] : 0ull;
      o.len[s] = len;
      o.base[s] = base;
      o.first_tile[s] = (uint32_t)ft;
      if (o.blk_base) o.blk_base[s] = base;
      if (o.tab_lg) {
        o.tab_lg[s] = table_lg(len);
        o.tab_base[s] = slot_carry + sex;
      }
      if (o.md) {
        MatDesc d;
        d.row_ids = o.row_ids + base;
        d.row_ptr = o.row_ptr + base + s;
        d.col_ids = o.col_ids + base;
        d.vals = o.vals + base;
        d.hdr = o.hdr + 2 * (uint64_t)s;
        d.neg = 0;
        o.md[s] = d;
      }
    }
    tile_carry += ttot;
    slot_carry += stot;
  }
  if (threadIdx.x == 0) {
    o.first_tile[nseg] = (uint32_t)tile_carry;
    if (o.pk_in_off) {
      o.pk_in_off[0] = ok ? off[0] : 0ull;
      o.pk_len[0] = ok ? off[nseg] - off[0] : 0ull;
    }
  }
}

// Small arrays copied by a kernel (host plans and descriptors to the device,
// quantities out): CTA (x, i) copies bytes [x * kSmallCopyChunk, (x + 1) *
// kSmallCopyChunk) of item i; either side may be page-locked host memory,
// which the device reads and writes in place.  A kernel, not a copy-engine
// transfer, so these copies never queue behind another stream's bulk copies
// (e.g. the next batch's packets arriving meanwhile).
constexpr uint64_t kSmallCopyChunk = 1u << 16;
__global__ void __launch_bounds__(256) k_small_copy(SmallCopyBatch b) {
  if (blockIdx.y >= b.n) return;
  const SmallCopyItem it = b.it[blockIdx.y];
  const uint64_t lo = (uint64_t)blockIdx.x * kSmallCopyChunk;
  if (lo >= it.bytes) return;
  const uint64_t hi = umin64(lo + kSmallCopyChunk, it.bytes);
  uint8_t* dst = static_cast<uint8_t*>(it.dst);
  const uint8_t* src = static_cast<const uint8_t*>(it.src);
  uint64_t i = lo;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) == 0) {
    // 16-byte vectors, four loads in flight per thread
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const uint64_t v_lo = lo / 16, v_hi = hi / 16;
    uint64_t v = v_lo + threadIdx.x;
    for (; v + 3 * blockDim.x < v_hi; v += 4 * blockDim.x) {
      uint4 x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = s4[v + k * blockDim.x];
#pragma unroll
      for (int k = 0; k < 4; ++k) d4[v + k * blockDim.x] = x[k];
    }
    for (; v < v_hi; v += blockDim.x) d4[v] = s4[v];
    i = v_hi * 16;
  }
  for (i += threadIdx.x; i < hi; i += blockDim.x) dst[i] = src[i];
}

// Guard g of the list: one warp, one 64-bit word per lane (kGuardBytes = 32
// words).  Fill without `err`; with it, compare and report a mismatch.
__device__ __forceinline__ uint64_t guard_word(uint32_t i) { return 0xA5C3E1F00F1E3C5Aull ^ (0x9E3779B97F4A7C15ull * (i + 1)); }
static_assert(kGuardBytes == 32 * 8, "a guard is one word per lane of a warp");
__global__ void __launch_bounds__(32) k_guards(GuardList g, uint32_t* err) {
  if (blockIdx.x >= g.n) return;
  uint64_t* w = reinterpret_cast<uint64_t*>(g.addr[blockIdx.x]);
  const uint32_t lane = threadIdx.x;
  if (!err) {
    w[lane] = guard_word(lane);
  } else if (w[lane] != guard_word(lane)) {
    atomicOr(err, (uint32_t)kErrGuard);
  }
}

__global__ void k_guard_probe_write(uint64_t* guard) { guard[0] = ~guard[0]; }

// n 32-bit words from src to dst by one CTA: 16-byte vectors when both
// addresses have the same alignment modulo 16 (after a short head), else
// words; several loads in flight per thread either way (src may sit across
// the host link).
__device__ void copy_words(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint64_t n) {
  const uint64_t t = threadIdx.x, nt = blockDim.x;
  uint64_t done = 0;  // words below this are copied by the vector part
  if (((reinterpret_cast<uintptr_t>(dst) ^ reinterpret_cast<uintptr_t>(src)) & 15u) == 0) {
    const uint64_t head = umin64(n, ((16u - (reinterpret_cast<uintptr_t>(src) & 15u)) & 15u) / 4u);
    if (t < head) dst[t] = src[t];
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    uint4* d4 = reinterpret_cast<uint4*>(dst + head);
    const uint64_t nv = (n - head) / 4;
    uint64_t v = t;  // this thread's vectors: t, t + nt, t + 2 nt, ...
    for (; v + 3 * nt < nv; v += 4 * nt) {
      uint4 x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = s4[v + k * nt];
#pragma unroll
      for (int k = 0; k < 4; ++k) d4[v + k * nt] = x[k];
    }
    for (; v < nv; v += nt) d4[v] = s4[v];
    done = head + nv * 4;
  }
  uint64_t w = done + t;  // this thread's words: w, w + nt, ...
  for (; w + 7 * nt < n; w += 8 * nt) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = src[w + k * nt];
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[w + k * nt] = x[k];
  }
  for (; w < n; w += nt) dst[w] = src[w];
}

__global__ void __launch_bounds__(256) k_gather_windows(const GatherWin* __restrict__ wins, uint32_t nwin,
                                                        uint32_t* __restrict__ gsrc, uint32_t* __restrict__ gdst) {
  for (uint32_t w = blockIdx.x; w < nwin; w += gridDim.x) {
    const GatherWin g = wins[w];
    copy_words(gsrc + g.off, reinterpret_cast<const uint32_t*>(g.src), g.len);
    copy_words(gdst + g.off, reinterpret_cast<const uint32_t*>(g.dst), g.len);
  }
}

// One 32-bit word copied on the device (error-word snapshots).
__global__ void k_copy_word(uint32_t* dst, const uint32_t* src) { *dst = *src; }

}  // namespace

cudaError_t launch_small_copy(const SmallCopyBatch& b, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  if (b.n > kSmallCopyItems) return cudaErrorInvalidValue;
  uint64_t chunks = 1;
  for (uint32_t i = 0; i < b.n; ++i) chunks = umax64(chunks, (b.it[i].bytes + kSmallCopyChunk - 1) / kSmallCopyChunk);
  if (chunks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  k_small_copy<<<dim3((unsigned)chunks, b.n), 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_guards(const GuardList& g, uint32_t* err, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  if (g.n > kGuardsPerLaunch) return cudaErrorInvalidValue;
  k_guards<<<g.n, 32, 0, st>>>(g, err);
  return cudaGetLastError();
}

cudaError_t launch_gather_windows(const GatherWin* wins, uint32_t nwin, uint32_t* gsrc, uint32_t* gdst,
                                  cudaStream_t st) {
  if (nwin == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint32_t grid = std::min<uint32_t>(nwin, (uint32_t)std::max(sms, 1) * 8u);
  k_gather_windows<<<grid, 256, 0, st>>>(wins, nwin, gsrc, gdst);
  return cudaGetLastError();
}

cudaError_t launch_guard_probe_write(uint64_t* guard, cudaStream_t st) {
  k_guard_probe_write<<<1, 1, 0, st>>>(guard);
  return cudaGetLastError();
}

cudaError_t launch_copy_word(uint32_t* dst, const uint32_t* src, cudaStream_t st) {
  k_copy_word<<<1, 1, 0, st>>>(dst, src);
  return cudaGetLastError();
}

cudaError_t launch_plan(const uint64_t* d_offsets, uint32_t nseg, uint64_t cap, const DevPlanOut& o, uint32_t* err,
                        cudaStream_t st) {
  k_plan<<<1, kPlanThreads, 0, st>>>(d_offsets, nseg, cap, o, err);
  return cudaGetLastError();
}

}  // namespace ans
