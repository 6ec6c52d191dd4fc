// On-chip window sort: one thread-block cluster sorts one whole window.
//
// A window of up to 2^17 packets holds at most 1 MiB of 64-bit link keys
// (src << 32 | dst, the DCSR order of Sec. IV-B), which fits in the
// distributed shared memory of an 8-CTA cluster (8 x 128 KiB).  The cluster
// reads the (src, dst) pairs from HBM once, runs all eight stable 8-bit LSD
// passes inside the cluster and writes the sorted keys once, instead of
// sixteen global passes over the keys (one histogram sweep plus eight
// read-and-write digit passes).
//
// Each CTA owns a slice of sorted positions and keeps its keys in registers
// between passes.  Per pass it ranks them with warp-private digit counters
// (lanes with equal digits merged by digit_peers), writes them into its own
// shared memory grouped by digit, and publishes its digit counts and digit
// starts.  After a cluster barrier every CTA knows, for each (digit, source
// CTA) run, where the run lands in the window's order; it then *pulls* the
// keys of its own slice from the source CTAs' shared memory (neighbouring
// lanes read neighbouring addresses of one run, so remote reads coalesce),
// and a second barrier frees the buffers for the next pass.  Pulling instead
// of pushing needs one buffer per CTA and no scattered remote stores.
// Cluster barriers are hardware barriers; every CTA of a cluster executes the
// same sequence of them, including CTAs with no keys.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr int kCluster = kWindowCluster;          // CTAs per cluster
constexpr int kChunkMax = kClusterWindowMax / kCluster;  // keys per CTA (16384)

constexpr int kSegs = kRadix * kCluster;  // (digit, source CTA) runs per pass

template <int kCT>
struct CLayout {
  static constexpr int kW = kCT / 32;
  static constexpr size_t keys = 0;                                  // [kChunkMax] u64
  static constexpr size_t wc = keys + (size_t)kChunkMax * 8;         // [kW][kRadix + 1]
  static constexpr size_t cnt = wc + (size_t)kW * (kRadix + 1) * 4;  // [kRadix] this CTA's digit counts
  static constexpr size_t lstart = cnt + (size_t)kRadix * 4;         // [kRadix] this CTA's digit starts
  static constexpr size_t seg_g = lstart + (size_t)kRadix * 4;       // [kSegs + 1] run starts in the window
  static constexpr size_t seg_l = seg_g + (size_t)(kSegs + 4) * 4;   // [kSegs] run starts in the source CTA
  static constexpr size_t tmp = seg_l + (size_t)kSegs * 4;           // [8]
  static constexpr size_t bytes = tmp + 8 * 4;
};

// Launched with clusters of kCluster CTAs along x.  Cluster `cid` sorts
// segment seg_ids[cid] (or cid).  The window's items are spread over the CTAs
// in power-of-two slices of `chunk` keys (512 .. 16384): CTA r owns sorted
// positions [r * chunk, (r + 1) * chunk), thread (warp w, lane l) the
// positions w * kP * 32 + i * 32 + l of the slice, i < kP.
template <int kCT, int kRank>
__global__ void __launch_bounds__(kCT, 1)
    k_cluster_sort(SegPlan p, const uint32_t* __restrict__ seg_ids, const uint32_t* __restrict__ src,
                   const uint32_t* __restrict__ dst, uint64_t* __restrict__ keys, uint32_t* __restrict__ tickets) {
  using L = CLayout<kCT>;
  constexpr int kP = kChunkMax / kCT;  // key slots per thread
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem + L::keys);
  uint32_t* s_wc = reinterpret_cast<uint32_t*>(smem + L::wc);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + L::cnt);
  uint32_t* s_lstart = reinterpret_cast<uint32_t*>(smem + L::lstart);
  uint32_t* s_segg = reinterpret_cast<uint32_t*>(smem + L::seg_g);
  uint32_t* s_segl = reinterpret_cast<uint32_t*>(smem + L::seg_l);
  uint32_t* s_tmp = reinterpret_cast<uint32_t*>(smem + L::tmp);

  const uint32_t me = cta_rank();
  const uint32_t cid = cluster_id();
  const uint32_t seg = seg_ids ? seg_ids[cid] : cid;
  if (cid == 0 && me == 0 && threadIdx.x < 32) tickets[threadIdx.x] = 0;
  const uint64_t len = p.len[seg];
  if (len > kClusterWindowMax) return;  // the host never sends these (the whole cluster leaves)
  const uint32_t n = (uint32_t)len;
  uint32_t lg = 9;
  while ((1u << lg) * kCluster < n) ++lg;
  const uint32_t chunk = 1u << lg;
  const uint32_t lo = me * chunk;
  const uint32_t cnt = n > lo ? min(n - lo, chunk) : 0u;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * (kP * 32);
  const uint32_t keys_saddr = (uint32_t)__cvta_generic_to_shared(s_keys);
  const uint32_t cnt_saddr = (uint32_t)__cvta_generic_to_shared(s_cnt);
  const uint32_t lstart_saddr = (uint32_t)__cvta_generic_to_shared(s_lstart);
  uint32_t* wc = s_wc + warp * (kRadix + 1);

  uint64_t k[kP];
  {
    const uint32_t *ws, *wd;
    window_inputs(p, seg, src, dst, &ws, &wd);
    ws += lo;
    wd += lo;
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      k[i] = idx < cnt ? ((uint64_t)__ldg(ws + idx) << 32) | __ldg(wd + idx) : 0ull;
    }
  }

  for (int pass = 0; pass < kPasses; ++pass) {
    const int shift = pass * kRadixBits;
    for (int i = lane; i < kRadix + 1; i += 32) wc[i] = 0;
    __syncwarp();
    // Stable rank inside (warp, digit); two 16-bit ranks per register.
    uint32_t r[(kP + 1) / 2];
#pragma unroll
    for (int i = 0; i < (kP + 1) / 2; ++i) r[i] = 0;
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      const bool valid = idx < cnt;
      const uint32_t d = valid ? (uint32_t)(k[i] >> shift) & 0xffu : (uint32_t)kRadix;
      const uint32_t peers = digit_peers<kRank>(d, valid);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (valid && lane == leader) {
        old = wc[d];
        wc[d] = old + __popc(peers);
      }
      __syncwarp();
      old = __shfl_sync(0xffffffffu, old, valid ? leader : lane);
      r[i / 2] |= (old + __popc(peers & lanemask_lt())) << ((i & 1) * 16);
    }
    __syncthreads();
    // Per digit: exclusive offsets across warps, this CTA's count and start.
    const uint32_t d = threadIdx.x;
    uint32_t c = 0;
    if (d < kRadix) {
#pragma unroll 4
      for (int w = 0; w < L::kW; ++w) {
        const uint32_t x = s_wc[w * (kRadix + 1) + d];
        s_wc[w * (kRadix + 1) + d] = c;
        c += x;
      }
    }
    const uint32_t ls = scan256_excl(d < kRadix ? c : 0u, s_tmp, nullptr);
    if (d < kRadix) {
      s_cnt[d] = c;
      s_lstart[d] = ls;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      if (idx < cnt) {
        const uint32_t dg = (uint32_t)(k[i] >> shift) & 0xffu;
        s_keys[s_lstart[dg] + wc[dg] + ((r[i / 2] >> ((i & 1) * 16)) & 0xffffu)] = k[i];
      }
    }
    cluster_sync();  // every CTA's keys grouped by digit, with counts and starts, are visible
    // Runs (digit d, source CTA q) in window order: start in the window and
    // in the source's buffer.
    uint32_t tot = 0;
    if (d < kRadix) {
#pragma unroll
      for (int q = 0; q < kCluster; ++q) {
        const uint32_t x = ld_cluster(map_rank(cnt_saddr + d * 4, q));
        s_segg[d * kCluster + q] = tot;  // relative to the digit's start for now
        s_segl[d * kCluster + q] = ld_cluster(map_rank(lstart_saddr + d * 4, q));
        tot += x;
      }
    }
    const uint32_t gstart = scan256_excl(d < kRadix ? tot : 0u, s_tmp, nullptr);
    if (d < kRadix) {
#pragma unroll
      for (int q = 0; q < kCluster; ++q) s_segg[d * kCluster + q] += gstart;
    }
    if (threadIdx.x == 0) s_segg[kSegs] = 0xffffffffu;
    __syncthreads();
    // Pull this thread's sorted positions: the run holding position P is the
    // last run starting at or before P (runs of length 0 share the next run's
    // start and are passed over).
    {
      const uint32_t p0 = lo + wbase + lane;
      uint32_t a = 0, b = kSegs;  // s_segg[a] <= p0 < s_segg[b]
      while (b - a > 1) {
        const uint32_t mid = (a + b) >> 1;
        if (s_segg[mid] <= p0) a = mid; else b = mid;
      }
      uint32_t j = a;
#pragma unroll
      for (int i = 0; i < kP; ++i) {
        const uint32_t idx = wbase + i * 32 + lane;
        if (idx < cnt) {
          const uint32_t P = lo + idx;
          while (s_segg[j + 1] <= P) ++j;
          const uint32_t off = s_segl[j] + (P - s_segg[j]);
          k[i] = ld_cluster_u64(map_rank(keys_saddr + off * 8, j & (kCluster - 1)));
        }
      }
    }
    cluster_sync();  // every pull is done: buffers and counts may be rewritten
  }

  uint64_t* out = keys + p.base[seg] + lo;
#pragma unroll
  for (int i = 0; i < kP; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    if (idx < cnt) out[idx] = k[i];
  }
}

template <int kCT, int kRank>
cudaError_t run_cluster_variant(const SegPlan& p, const uint32_t* seg_ids, uint32_t nclusters, const uint32_t* src,
                                const uint32_t* dst, uint64_t* keys, uint32_t* tickets, cudaStream_t st) {
  static unsigned long long configured = 0;  // one bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_cluster_sort<kCT, kRank>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CLayout<kCT>::bytes);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured |= 1ull << dev;
  }
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.gridDim = dim3(nclusters * kCluster, 1, 1);
  lc.blockDim = dim3(kCT, 1, 1);
  lc.dynamicSmemBytes = CLayout<kCT>::bytes;
  lc.stream = st;
  return cudaLaunchKernelEx(&lc, k_cluster_sort<kCT, kRank>, p, seg_ids, src, dst, keys, tickets);
}

}  // namespace

cudaError_t launch_cluster_sort(const SegPlan& p, const uint32_t* seg_ids, uint32_t nclusters, const uint32_t* src,
                                const uint32_t* dst, uint64_t* keys, uint32_t* tickets, const SortCfg& cfg,
                                cudaStream_t st) {
  if (nclusters == 0) return cudaSuccess;
  if (cfg.threads == 512) {
    if (cfg.rank == kRankBallot) return run_cluster_variant<512, kRankBallot>(p, seg_ids, nclusters, src, dst, keys, tickets, st);
    return run_cluster_variant<512, kRankMatch>(p, seg_ids, nclusters, src, dst, keys, tickets, st);
  }
  if (cfg.rank == kRankBallot) return run_cluster_variant<1024, kRankBallot>(p, seg_ids, nclusters, src, dst, keys, tickets, st);
  return run_cluster_variant<1024, kRankMatch>(p, seg_ids, nclusters, src, dst, keys, tickets, st);
}

int cluster_sort_clusters(int device) {
  static int cached[64];
  static bool have[64];
  if (device >= 0 && device < 64 && have[device]) return cached[device];
  int best = 0;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kCluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  lc.attrs = &attr;
  lc.numAttrs = 1;
  lc.gridDim = dim3(kCluster, 1, 1);
  lc.blockDim = dim3(1024, 1, 1);
  lc.dynamicSmemBytes = CLayout<1024>::bytes;
  if (cudaFuncSetAttribute(k_cluster_sort<1024, kRankMatch>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)CLayout<1024>::bytes) == cudaSuccess) {
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster_sort<1024, kRankMatch>, &lc) == cudaSuccess) best = n;
  }
  cudaGetLastError();
  if (device >= 0 && device < 64) {
    cached[device] = best;
    have[device] = true;
  }
  return best;
}

}  // namespace ans
