// Time sum by merging: the stored links of every input matrix are already in
// DCSR order (rows ascending, columns ascending within a row, Sec. IV-B), so
// the links of k matrices, gathered back to back as (src << 32 | dst, count)
// runs, become one sorted run by ceil(log2 k) rounds of pairwise merges.
// Equal links of different matrices end up adjacent (the first matrix's
// first), and the run-length reduction that follows adds their counts: the
// sum of Table I's A_t over t.
//
// One round merges runs 2j and 2j + 1 of the previous round (run j of round
// r spans matrices [j * 2^r, (j + 1) * 2^r) of the concatenation).  Each CTA
// produces a fixed span of kMergeTile output positions: it finds, per pair
// overlapping the span, how many of the span's items come from each run (a
// merge-path co-rank search, one warp per end of the span), stages those
// slices in shared memory, and each item's output position is its index in
// its own slice plus its rank in the other slice (ties: the earlier run
// first).  Reads and writes are contiguous; one pass moves 32 bytes per link.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr int kMergeThreads = 512;

// Number of items of A among the first x items of merge(A, B), A first on
// equal keys, found by one warp: each step tests 32 evenly spaced candidates
// of the remaining range at once (the test is monotone: true below the
// answer), so a range of 2^k candidates needs about k / 5 dependent loads.
__device__ __forceinline__ uint64_t co_rank_warp(const uint64_t* A, uint64_t na, const uint64_t* B, uint64_t nb,
                                                 uint64_t x) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t lo = x > nb ? x - nb : 0, hi = x < na ? x : na;  // the answer lies in [lo, hi]
  while (lo < hi) {
    const uint64_t p = lo + ((hi - lo) * (lane + 1)) / 33;  // lo <= p < hi, nondecreasing in lane
    const bool below = A[p] <= B[x - p - 1];
    const uint32_t m = __ballot_sync(0xffffffffu, below);
    const int nt = __popc(m);  // the lanes testing true are a prefix
    const uint64_t p_last = __shfl_sync(0xffffffffu, p, nt > 0 ? nt - 1 : 0);
    const uint64_t p_first = __shfl_sync(0xffffffffu, p, nt < 32 ? nt : 31);
    if (nt > 0) lo = p_last + 1;
    if (nt < 32) hi = p_first;
  }
  return lo;
}

// kMergeTile output positions per CTA (4096, or 2048 for more resident CTAs
// per SM: the shared memory holds the two slices, keys and values).
template <int kMergeTile>
constexpr size_t merge_smem() {
  return (size_t)kMergeTile * 8 * 2;
}

// cat_off: k + 1 dense run starts of round 0 (cat_off[k] = total); run_base
// (null: cat_off) where each matrix's items sit.  Round `round` merges pairs
// of runs of 2^round matrices each; CTAs cover spans of dense output
// positions.
template <int kMergeTile>
__global__ void __launch_bounds__(kMergeThreads) k_merge(const uint64_t* __restrict__ cat_off,
                                                         const uint64_t* __restrict__ run_base, uint32_t k, int round,
                                                         const uint64_t* __restrict__ kin,
                                                         const uint64_t* __restrict__ vin, uint64_t* __restrict__ kout,
                                                         uint64_t* __restrict__ vout) {
  extern __shared__ __align__(16) uint64_t smem[];
  uint64_t* s_k = smem;  // slice of A, then slice of B
  uint64_t* s_v = smem + kMergeTile;
  __shared__ uint64_t s_cut[2];
  const uint64_t total = cat_off[k];
  const uint64_t o0 = (uint64_t)blockIdx.x * kMergeTile;
  if (o0 >= total) return;
  const uint64_t o1 = umin64(o0 + kMergeTile, total);
  const uint64_t width = 1ull << round;              // matrices per input run
  const uint64_t njobs = (k + 2 * width - 1) / (2 * width);
  auto start = [&](uint64_t m) { return cat_off[umin64(m, (uint64_t)k)]; };
  // The job (pair of runs) holding output position o0.
  uint64_t lo = 0, hi = njobs;  // start(lo * 2w) <= o0 < start(hi * 2w)
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (start(mid * 2 * width) <= o0) lo = mid; else hi = mid;
  }
  for (uint64_t j = lo; j < njobs; ++j) {
    const uint64_t a_beg = start(j * 2 * width), b_beg = start(j * 2 * width + width),
                   b_end = start(j * 2 * width + 2 * width);
    if (a_beg >= o1) break;
    if (b_end <= o0) continue;
    const uint64_t na = b_beg - a_beg, nb = b_end - b_beg;
    const uint64_t x0 = (o0 > a_beg ? o0 : a_beg) - a_beg, x1 = umin64(o1, b_end) - a_beg;
    // where the two runs and the merged run sit (a missing B run is empty)
    const uint64_t pa = run_base ? run_base[j * 2 * width] : a_beg;
    const uint64_t pb = run_base ? (nb ? run_base[j * 2 * width + width] : pa) : b_beg;
    const uint64_t* A = kin + pa;
    const uint64_t* B = kin + pb;
    if (threadIdx.x < 64) {
      const uint64_t c = co_rank_warp(A, na, B, nb, threadIdx.x < 32 ? x0 : x1);
      if ((threadIdx.x & 31) == 0) s_cut[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    const uint64_t a0 = s_cut[0], a1 = s_cut[1];
    const uint64_t b0 = x0 - a0, b1 = x1 - a1;
    const uint32_t ca = (uint32_t)(a1 - a0), cb = (uint32_t)(b1 - b0);  // ca + cb = x1 - x0 <= kMergeTile
    for (uint32_t i = threadIdx.x; i < ca; i += kMergeThreads) {
      s_k[i] = A[a0 + i];
      s_v[i] = vin[pa + a0 + i];
    }
    for (uint32_t i = threadIdx.x; i < cb; i += kMergeThreads) {
      s_k[ca + i] = B[b0 + i];
      s_v[ca + i] = vin[pb + b0 + i];
    }
    __syncthreads();
    uint64_t* ko = kout + pa + x0;
    uint64_t* vo = vout + pa + x0;
    for (uint32_t i = threadIdx.x; i < ca + cb; i += kMergeThreads) {
      const uint64_t key = s_k[i];
      uint32_t pos;
      if (i < ca) {  // B items strictly before it
        uint32_t l = 0, h = cb;
        while (l < h) {
          const uint32_t m = (l + h) >> 1;
          if (s_k[ca + m] < key) l = m + 1; else h = m;
        }
        pos = i + l;
      } else {  // A items at or before it
        uint32_t l = 0, h = ca;
        while (l < h) {
          const uint32_t m = (l + h) >> 1;
          if (s_k[m] <= key) l = m + 1; else h = m;
        }
        pos = (i - ca) + l;
      }
      ko[pos] = key;
      vo[pos] = s_v[i];
    }
    __syncthreads();
  }
}

template <int kMergeTile>
cudaError_t run_merge(const uint64_t* cat_off, const uint64_t* run_base, uint32_t k, uint64_t total_cap, int round,
                      const uint64_t* kin, const uint64_t* vin, uint64_t* kout, uint64_t* vout, cudaStream_t st) {
  const uint64_t blocks = (total_cap + kMergeTile - 1) / kMergeTile;
  if (blocks == 0) return cudaSuccess;
  static unsigned long long configured = 0;  // one bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_merge<kMergeTile>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)merge_smem<kMergeTile>());
    if (e != cudaSuccess) return e;
    if (dev < 64) configured |= 1ull << dev;
  }
  k_merge<kMergeTile><<<(unsigned)blocks, kMergeThreads, merge_smem<kMergeTile>(), st>>>(cat_off, run_base, k, round,
                                                                                       kin, vin, kout, vout);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_merge(const uint64_t* cat_off, const uint64_t* run_base, uint32_t k, uint64_t total_cap, int round,
                         const uint64_t* kin, const uint64_t* vin, uint64_t* kout, uint64_t* vout, int tile,
                         cudaStream_t st) {
  if (tile == 2048) return run_merge<2048>(cat_off, run_base, k, total_cap, round, kin, vin, kout, vout, st);
  return run_merge<4096>(cat_off, run_base, k, total_cap, round, kin, vin, kout, vout, st);
}

}  // namespace ans
