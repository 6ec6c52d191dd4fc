// Hash aggregation of a window's packets (the alternative to sorting every
// packet): A(i, j) = #{k : s_k = i, d_k = j} (Table I caption) is first
// counted in an open-addressing table keyed by the link key src << 32 | dst,
// and only the U distinct links are then sorted (with their counts) into DCSR
// order.  Worth it when windows repeat links heavily (U << P).
//
//  * k_hash_insert: lanes of a warp holding the same key are merged
//    (__match_any_sync on the 64-bit key), and the lowest such lane claims or
//    finds the key's slot by linear probing from a SplitMix64-finalizer hash
//    (atomicCAS on the key word) and adds the merged count.  Every window has
//    its own table of a power-of-two size of at least twice its packets, so
//    the load stays at or below one half and every probe sequence ends.
//    The slots a tile claims (keys new to the window) are appended to the
//    window's claim list, one atomic per tile.
//  * k_hash_compact: walks each window's claim list (U entries, not the
//    table), moves every (key, count) to the window's slice of the sort
//    buffers (claim order; the sort follows), builds the kv sort's digit
//    histograms and empties the claimed slots, so the tables are clean for
//    the next call.
// The all-ones key (src = dst = 0xFFFFFFFF) is the empty-slot marker, so its
// count is kept beside the table instead.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;

// Finalizer of SplitMix64 (Steele, Lea and Flood, 2014): a bijective 64-bit
// mix, so the low bits of the slot index depend on every key bit.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Adds c to key's slot; returns the slot if this call claimed it (the key
// was new), else ~0.
__device__ __forceinline__ uint32_t table_add(uint64_t* keys, uint32_t* cnt, uint32_t mask, uint64_t key, uint32_t c,
                                              uint32_t* err) {
  uint32_t h = (uint32_t)mix64(key) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    uint64_t cur = *(volatile uint64_t*)(keys + h);
    bool claimed = false;
    if (cur == kEmptyKey) {
      cur = atomicCAS((unsigned long long*)(keys + h), (unsigned long long)kEmptyKey, (unsigned long long)key);
      if (cur == kEmptyKey) {
        cur = key;
        claimed = true;
      }
    }
    if (cur == key) {
      atomicAdd(cnt + h, c);
      return claimed ? h : ~0u;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, (uint32_t)kErrHashFull);  // cannot happen at load <= 1/2
  return ~0u;
}

// One tile of packets per CTA.  The slots this tile claims are collected in
// shared memory and appended to the window's claim list (claims + base[s],
// count in nclaim[s]) with one atomic per tile.
__global__ void __launch_bounds__(kThreads) k_hash_insert(SegPlan p, const uint32_t* __restrict__ src,
                                                          const uint32_t* __restrict__ dst, HashTabs h,
                                                          uint32_t* err) {
  __shared__ Tile s_tile;
  __shared__ uint32_t s_claim[kTile];
  __shared__ uint32_t s_n;
  __shared__ uint64_t s_base;
  const Tile tl = block_tile(p, blockIdx.x, &s_tile);
  if (tl.count == 0) return;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const uint32_t *ws, *wd;
  window_inputs(p, tl.seg, src, dst, &ws, &wd);
  ws += tl.start;
  wd += tl.start;
  uint64_t* keys = h.keys + h.off[tl.seg];
  uint32_t* cnt = h.cnt + h.off[tl.seg];
  const uint32_t mask = (uint32_t)((1ull << h.lg[tl.seg]) - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = warp * (kPerThread * 32) + i * 32 + lane;
    const bool valid = idx < tl.count;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    if (!valid) continue;
    const uint64_t key = ((uint64_t)__ldg(ws + idx) << 32) | __ldg(wd + idx);
    const uint32_t peers = __match_any_sync(vmask, key);
    if (lane != __ffs(peers) - 1) continue;
    const uint32_t c = __popc(peers);
    if (key == kEmptyKey) {
      atomicAdd((unsigned long long*)(h.special + tl.seg), (unsigned long long)c);
    } else {
      const uint32_t slot = table_add(keys, cnt, mask, key, c, err);
      if (slot != ~0u) s_claim[atomicAdd(&s_n, 1u)] = slot;
    }
  }
  __syncthreads();
  const uint32_t n = s_n;
  if (n == 0) return;
  if (threadIdx.x == 0) s_base = atomicAdd((unsigned long long*)(h.nclaim + tl.seg), (unsigned long long)n);
  __syncthreads();
  uint32_t* out = h.claims + p.base[tl.seg] + s_base;
  for (uint32_t i = threadIdx.x; i < n; i += kThreads) out[i] = s_claim[i];
}

// `pc`: the windows with len = nclaim.  Moves window s's claimed slots to
// okeys/ovals + base[s] (the all-ones key's count, if any, after them), sets
// ulen[s], builds the kv sort's digit histograms and empties the slots; also
// zeroes the sort's first status words and tickets[0..32).
__global__ void __launch_bounds__(kThreads) k_hash_compact(SegPlan pc, HashTabs h, uint64_t* __restrict__ ulen,
                                                           uint64_t* __restrict__ okeys, uint64_t* __restrict__ ovals,
                                                           uint32_t* __restrict__ seg_hist, uint64_t* __restrict__ status0,
                                                           uint32_t* __restrict__ tickets) {
  __shared__ uint32_t hs[kPasses * kRadix];
  __shared__ Tile s_tile;
  const uint32_t t = blockIdx.x;
  const Tile tl = block_tile(pc, t, &s_tile);
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) hs[i] = 0;
  if (t == 0 && threadIdx.x < 32) tickets[threadIdx.x] = 0;
  if (threadIdx.x < kRadix) status0[(uint64_t)t * kRadix + threadIdx.x] = 0;
  __syncthreads();
  const uint32_t s = tl.seg;
  uint64_t* ok = okeys + tl.base;
  uint64_t* ov = ovals + tl.base;
  auto hist = [&](uint64_t key) {
#pragma unroll
    for (int q = 0; q < kPasses; ++q) atomicAdd(&hs[q * kRadix + ((key >> (q * kRadixBits)) & 0xffu)], 1u);
  };
  if (tl.j == 0 && threadIdx.x == 0) {
    const uint64_t c = h.special[s];
    ulen[s] = tl.len + (c ? 1 : 0);
    if (c) {
      ok[tl.len] = kEmptyKey;
      ov[tl.len] = c;
      hist(kEmptyKey);
    }
  }
  if (tl.count > 0) {
    uint64_t* keys = h.keys + h.off[s];
    uint32_t* cnt = h.cnt + h.off[s];
    const uint32_t* cl = h.claims + tl.base + tl.start;
    for (uint32_t i = threadIdx.x; i < tl.count; i += kThreads) {
      const uint32_t slot = cl[i];
      const uint64_t key = keys[slot];
      ok[tl.start + i] = key;
      ov[tl.start + i] = cnt[slot];
      keys[slot] = kEmptyKey;
      cnt[slot] = 0;
      hist(key);
    }
  }
  __syncthreads();
  uint32_t* g = seg_hist + (size_t)s * kPasses * kRadix;
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) {
    const uint32_t c = hs[i];
    if (c) atomicAdd(&g[i], c);
  }
}

}  // namespace

cudaError_t launch_hash_insert(const SegPlan& p, const uint32_t* src, const uint32_t* dst, const HashTabs& h,
                               uint32_t* err, cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
  k_hash_insert<<<p.ntiles, kThreads, 0, st>>>(p, src, dst, h, err);
  return cudaGetLastError();
}

cudaError_t launch_hash_compact(const SegPlan& pc, const HashTabs& h, uint64_t* ulen, uint64_t* okeys,
                                uint64_t* ovals, uint32_t* seg_hist, uint64_t* status0, uint32_t* tickets,
                                cudaStream_t st) {
  if (pc.ntiles == 0) return cudaSuccess;
  k_hash_compact<<<pc.ntiles, kThreads, 0, st>>>(pc, h, ulen, okeys, ovals, seg_hist, status0, tickets);
  return cudaGetLastError();
}

}  // namespace ans
