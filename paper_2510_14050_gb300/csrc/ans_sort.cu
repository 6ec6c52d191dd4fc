// Segmented onesweep LSD radix sorts.
//
// Building a traffic matrix A(i, j) = #packets i -> j (Table I caption) from
// raw packets means grouping equal (src, dst) pairs; sorting the packed key
// src << 32 | dst puts equal links next to each other in DCSR order (rows =
// sources ascending, columns ascending within a row, Sec. IV-B).  The column
// statistics (Table I: unique destinations, max fan-in; Sec. IV-C: max
// destination packets) group the stored links by destination instead: a sort
// of 32-bit destination keys carrying the link counts.
//
// Design (sm_103a):
//  * one histogram sweep builds the digit counts of every pass for every
//    segment at once (shared-memory counters; lanes holding identical keys
//    are merged with __match_any_sync first, which matters for Zipf traffic
//    where a few links dominate);
//  * each pass is one kernel: a CTA ranks its 8192-key tile with warp-private
//    digit counters (warp-aggregated via __match_any_sync), obtains the
//    tile's global digit offsets by bounded decoupled look-back over the
//    previous tiles of its segment, reorders the tile in shared memory and
//    writes runs of equal digits to contiguous addresses;
//  * loads of the raw (src, dst) stream are 128-bit when the window is
//    16-byte aligned.
#include <type_traits>

#include "ans_internal.cuh"

namespace ans {

namespace {

__device__ __forceinline__ void hist_add(uint32_t* h, uint64_t key, bool valid, uint32_t vmask) {
  if (!valid) return;
  const uint32_t peers = __match_any_sync(vmask, key);
  if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) {
    const uint32_t c = __popc(peers);
#pragma unroll
    for (int p = 0; p < kPasses; ++p) atomicAdd(&h[p * kRadix + ((key >> (p * kRadixBits)) & 0xff)], c);
  }
}

__device__ __forceinline__ void hist_flush(const uint32_t* h, uint32_t* seg_hist, uint32_t seg) {
  uint32_t* g = seg_hist + (size_t)seg * kPasses * kRadix;
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) {
    const uint32_t c = h[i];
    if (c) atomicAdd(&g[i], c);
  }
}

// Digit counts of one key (count c) into one of kHistCopies histogram copies
// (a warp's copy is warp % kHistCopies, which spreads the shared-memory
// atomics of a CTA's warps).
constexpr int kHistCopies = 4;
__device__ __forceinline__ void hist_add_plain(uint32_t* h, uint64_t key, uint32_t c) {
#pragma unroll
  for (int p = 0; p < kPasses; ++p) atomicAdd(&h[p * kRadix + ((key >> (p * kRadixBits)) & 0xff)], c);
}

__global__ void __launch_bounds__(kThreads) k_pack_hist(SegPlan p, const uint32_t* __restrict__ src,
                                                        const uint32_t* __restrict__ dst,
                                                        uint64_t* __restrict__ keys,
                                                        uint32_t* __restrict__ seg_hist,
                                                        uint64_t* __restrict__ status0,
                                                        uint32_t* __restrict__ tickets, uint32_t sub) {
  __shared__ uint32_t hc[kHistCopies][kPasses * kRadix];
  uint32_t* h = hc[0];
  __shared__ Tile s_tile;
  const uint32_t t = blockIdx.x;
  const Tile tl = block_tile(p, t, &s_tile);
  for (int i = threadIdx.x; i < kHistCopies * kPasses * kRadix; i += kThreads) (&hc[0][0])[i] = 0;
  if (t == 0 && threadIdx.x < 32) tickets[threadIdx.x] = 0;
  for (uint32_t i = threadIdx.x; i < sub * kRadix; i += kThreads) status0[(uint64_t)t * sub * kRadix + i] = 0;
  __syncthreads();
  if (tl.count == 0) return;

  const uint32_t *ws, *wd;
  window_inputs(p, tl.seg, src, dst, &ws, &wd);
  ws += tl.start;
  wd += tl.start;
  uint64_t* out = keys + tl.base + tl.start;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool aligned = ((((uintptr_t)ws) | ((uintptr_t)wd)) & 15u) == 0;

  if (aligned && tl.count == kTile) {
    // 128-bit loads: each lane reads 4 consecutive sources and destinations.
    const uint4* s4 = reinterpret_cast<const uint4*>(ws);
    const uint4* d4 = reinterpret_cast<const uint4*>(wd);
    ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out);
#pragma unroll 2
    for (int i = 0; i < kPerThread / 4; ++i) {
      const int v = warp * (kPerThread * 8) + i * 32 + lane;  // uint4 index inside the tile
      const uint4 a = __ldg(s4 + v), b = __ldg(d4 + v);
      const uint64_t k0 = ((uint64_t)a.x << 32) | b.x, k1 = ((uint64_t)a.y << 32) | b.y;
      const uint64_t k2 = ((uint64_t)a.z << 32) | b.z, k3 = ((uint64_t)a.w << 32) | b.w;
      o2[2 * v] = make_ulonglong2(k0, k1);
      o2[2 * v + 1] = make_ulonglong2(k2, k3);
      // The four keys are consecutive packets: equal neighbours (bursts of
      // one link) are counted once.
      uint32_t* hw = hc[warp % kHistCopies];
      uint32_t c = 1;
      if (k1 == k0) ++c; else { hist_add_plain(hw, k0, c); c = 1; }
      if (k2 == k1) ++c; else { hist_add_plain(hw, k1, c); c = 1; }
      if (k3 == k2) ++c; else { hist_add_plain(hw, k2, c); c = 1; }
      hist_add_plain(hw, k3, c);
    }
  } else {
    for (int i = 0; i < kPerThread; ++i) {
      const uint32_t idx = warp * (kPerThread * 32) + i * 32 + lane;
      const bool valid = idx < tl.count;
      const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
      uint64_t key = 0;
      if (valid) {
        key = ((uint64_t)ws[idx] << 32) | wd[idx];
        out[idx] = key;
      }
      hist_add(h, key, valid, vmask);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 1; k < kHistCopies; ++k) c += hc[k][i];
    h[i] += c;
  }
  __syncthreads();
  hist_flush(h, seg_hist, tl.seg);
}

struct NoVal {};

// Per-warp digit counters: kRadix + 1 uint32 counters, or (table ranking)
// kRadix uint64 entries {count << 32 | lanes holding the digit}.
template <int kRank>
constexpr size_t warp_counter_bytes() {
  return kRank == kRankTable ? (size_t)kRadix * 8 : (size_t)(kRadix + 1) * 4;
}

template <typename K, typename V, int kT, int kRank, int kSub>
constexpr size_t onesweep_smem_bytes() {
  return (size_t)(kTile / kSub) * sizeof(K) +
         (std::is_same<V, NoVal>::value ? 0 : (size_t)(kTile / kSub) * sizeof(V)) +
         (size_t)(kT / 32) * warp_counter_bytes<kRank>();
}

// One stable digit pass over keys of type K (8 passes for 64-bit keys, 4 for
// 32-bit keys, 2 for 16-bit keys; seg_hist holds sizeof(K) histograms per
// segment), optionally carrying values of type V.  Each 8192-key tile of the
// plan is split into kSub sub-tiles, one CTA each (look-back runs over
// sub-tiles: status word u * kRadix + d belongs to sub-tile u = kSub * tile +
// half); kT threads share a sub-tile (kTile / kSub / kT keys each); kRank
// selects how lanes with equal digits find each other.
//
// `pass` is the digit index, plus kPassStable when the input order of equal
// digits must survive pass 0 too (by default pass 0 ranks with plain
// shared-memory atomics: the LSD passes after it only need a partition).
// With `remap` (16-bit keys only), a key k is written to its sorted position
// plus remap[min(k, nremap - 1)]; with a null `kout` only the values are
// written.  A 16-bit key or value shares a 32-bit register with the key's
// rank inside the tile (below 2^16), which keeps the kv forms at the
// registers of the key-only form.
template <typename K, typename V, int kT, int kRank, int kMinB, int kSub>
__global__ void __launch_bounds__(kT, kMinB)
    k_onesweep(SegPlan p, int pass, const K* __restrict__ kin, K* __restrict__ kout,
               const V* __restrict__ vin, V* __restrict__ vout, const uint32_t* __restrict__ seg_hist,
               uint64_t* st_cur, uint64_t* __restrict__ st_next, uint32_t* ticket, uint32_t* err,
               const uint64_t* __restrict__ remap, uint32_t nremap) {
  constexpr bool kVals = !std::is_same<V, NoVal>::value;
  constexpr int kNumPasses = (int)sizeof(K);
  constexpr uint32_t kTT = kTile / kSub;  // keys per CTA
  constexpr int kP = kTT / kT;            // keys per thread
  constexpr int kW = kT / 32;             // warps
  // 16-bit keys live in the low half of the rank word (rank in the high
  // half); 16-bit values in its high half (rank in the low half).
  constexpr bool kPackK = sizeof(K) == 2;
  constexpr bool kPackV = kVals && !kPackK && sizeof(V) == 2;
  static_assert(kTT <= 0xFFFFu, "ranks must fit 16 bits");
  const bool atomic_rank = pass == 0;  // pass 0 without kPassStable
  pass &= kPassMask;
  extern __shared__ __align__(16) uint8_t smem[];
  K* s_keys = reinterpret_cast<K*>(smem);
  V* s_vals = reinterpret_cast<V*>(smem + (size_t)kTT * sizeof(K));
  uint8_t* s_cnt = smem + (size_t)kTT * sizeof(K) + (kVals ? (size_t)kTT * sizeof(V) : 0);
  uint32_t* s_wc = reinterpret_cast<uint32_t*>(s_cnt);   // [kW][kRadix+1] (match / ballot ranking)
  uint64_t* s_tab = reinterpret_cast<uint64_t*>(s_cnt);  // [kW][kRadix]   (table ranking)
  __shared__ uint32_t s_grel[kRadix];
  __shared__ uint32_t s_dstart[kRadix];
  __shared__ uint32_t s_hv[kRadix];
  __shared__ uint64_t s_tmp[8];
  __shared__ uint32_t s_ticket;
  __shared__ Tile s_tile;

  const uint32_t u = block_ticket(ticket, &s_ticket);  // sub-tile
  const uint32_t t = u / kSub, half = u % kSub;
  Tile tl = block_tile(p, t, &s_tile);
  if (threadIdx.x < kRadix) st_next[(uint64_t)u * kRadix + threadIdx.x] = 0;
  if constexpr (kSub > 1) {
    const uint32_t off = half * kTT;
    tl.count = tl.count > off ? (uint32_t)umin64(tl.count - off, kTT) : 0u;
    tl.start += off;
  }
  if (tl.count == 0) return;
  // the segment's count of this pass's digit: copied to shared memory
  // asynchronously now, read after ranking (no register held meanwhile)
  if (threadIdx.x < kRadix) {
    const uint32_t* src = seg_hist + ((size_t)tl.seg * kNumPasses + pass) * kRadix + threadIdx.x;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n\tcp.async.commit_group;" ::"r"(smem_addr(&s_hv[threadIdx.x])),
                 "l"(src)
                 : "memory");
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The pass's digit is one byte of the key: byte pass % 4 of its low or
  // (64-bit keys, pass >= 4) high word, extracted by one byte permute.
  const bool dig_hi = sizeof(K) == 8 && pass >= 4;
  const uint32_t dig_sel = 0x4440u | (uint32_t)(pass & 3);
  auto digit = [&](K key) -> uint32_t {
    if constexpr (sizeof(K) == 8) return __byte_perm(dig_hi ? (uint32_t)(key >> 32) : (uint32_t)key, 0u, dig_sel);
    else return __byte_perm((uint32_t)key, 0u, dig_sel);
  };
  uint32_t* wc = s_wc + warp * (kRadix + 1);
  uint64_t* tab = s_tab + warp * kRadix;
  if constexpr (kRank == kRankTable) {
    for (int i = lane; i < kRadix; i += 32) tab[i] = 0;
  } else {
    for (int i = lane; i < kRadix + 1; i += 32) wc[i] = 0;
  }
  __syncwarp();

  const uint64_t g0 = tl.base + tl.start;
  const uint32_t wbase = warp * (kP * 32);
  K k[kPackK ? 1 : kP] = {};  // (every element is written by the load loop below)
  V v[(kVals && !kPackV) ? kP : 1] = {};
  uint32_t r[kP] = {};
  // the key, value and rank of item i, wherever they are held
  auto key_of = [&](int i) -> K {
    if constexpr (kPackK) return (K)(r[i] & 0xFFFFu);
    else return k[i];
  };
  auto val_of = [&](int i) -> V {
    if constexpr (kPackV) return (V)(r[i] >> 16);
    else return v[i];
  };
  auto rank_of = [&](int i) -> uint32_t {
    if constexpr (kPackK) return r[i] >> 16;
    else if constexpr (kPackV) return r[i] & 0xFFFFu;
    else return r[i];
  };
  auto set_rank = [&](int i, uint32_t x) {
    if constexpr (kPackK) r[i] = (r[i] & 0xFFFFu) | (x << 16);
    else if constexpr (kPackV) r[i] = (r[i] & 0xFFFF0000u) | x;
    else r[i] = x;
  };

  // Everything from the loads to the write-out, compiled twice: for a full
  // sub-tile (every item valid: no bounds tests, no inactive lanes) and for
  // the last, partial one of a segment.
  auto run = [&](auto full_tag) {
    constexpr bool kFull = decltype(full_tag)::value;
    auto valid_at = [&](uint32_t idx) -> bool {
      if constexpr (kFull) return true;
      else return idx < tl.count;
    };
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      const bool valid = valid_at(idx);
      if constexpr (kPackK) {
        r[i] = valid ? (uint32_t)kin[g0 + idx] : 0u;
      } else {
        k[i] = valid ? kin[g0 + idx] : K(0);
        r[i] = 0;
      }
      if constexpr (kPackV) r[i] = valid ? (uint32_t)vin[g0 + idx] << 16 : 0u;
      else if constexpr (kVals) v[i] = valid ? vin[g0 + idx] : V(0);
    }
    // Stable rank inside (warp, digit): lanes with equal digits find each
    // other (digit_peers); every lane reads its digit's count so far, the
    // lowest lane of the digit advances it.
#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      const bool valid = valid_at(idx);
      if constexpr (kRank == kRankTable) {
        // Each lane sets its bit in its digit's entry; every lane then reads
        // the entry (the lanes sharing its digit, and the digit's count so
        // far), and the lowest of them advances the count and clears the bits.
        const uint32_t d = digit(key_of(i));
        if (valid) atomicOr(reinterpret_cast<unsigned int*>(tab + d), 1u << lane);
        __syncwarp();
        const uint64_t e = valid ? tab[d] : 0ull;
        __syncwarp();
        const uint32_t peers = (uint32_t)e, old = (uint32_t)(e >> 32);
        if (valid && lane == __ffs(peers) - 1) tab[d] = (uint64_t)(old + __popc(peers)) << 32;
        __syncwarp();
        set_rank(i, old + __popc(peers & lanemask_lt()));
      } else if (atomic_rank) {
        // The first pass needs no stability (any order of equal digits is a
        // valid start for the stable passes after it): one shared-memory
        // atomic per key gives each its slot among the warp's equal digits.
        const uint32_t d = digit(key_of(i));
        set_rank(i, valid ? atomicAdd(&wc[d], 1u) : 0u);
      } else {
        // (inactive lanes of a partial tile share the spare digit kRadix)
        const uint32_t d = valid ? digit(key_of(i)) : (uint32_t)kRadix;
        const uint32_t peers = digit_peers<kRank>(d, valid);
        const uint32_t old = wc[d];
        __syncwarp();
        if (lane == __ffs(peers) - 1) wc[d] = old + __popc(peers);
        __syncwarp();
        set_rank(i, old + __popc(peers & lanemask_lt()));
      }
    }
    __syncthreads();

    // Per digit: exclusive offsets across warps and the tile's count.
    const int d = threadIdx.x;
    uint32_t cnt = 0;
    uint64_t excl = 0;
    if (d < kRadix) {
#pragma unroll 4
      for (int w = 0; w < kW; ++w) {
        if constexpr (kRank == kRankTable) {
          const uint32_t c = (uint32_t)(s_tab[w * kRadix + d] >> 32);
          s_tab[w * kRadix + d] = (uint64_t)cnt << 32;
          cnt += c;
        } else {
          const uint32_t c = s_wc[w * (kRadix + 1) + d];
          s_wc[w * (kRadix + 1) + d] = cnt;
          cnt += c;
        }
      }
      uint64_t* my = st_cur + (uint64_t)u * kRadix + d;
      if (tl.j == 0 && half == 0) {
        st_relaxed(my, kFlagPre | cnt);
      } else {
        st_relaxed(my, kFlagAgg | cnt);
        excl = lookback(st_cur + d, kRadix, kSub * (t - tl.j), u, err);
        st_relaxed(my, kFlagPre | (excl + cnt));
      }
    }
    // one scan for both: the digit's start in this tile (low half) and in the
    // segment (high half; the segment holds fewer than 2^31 keys)
    uint32_t hv = 0;
    if (d < kRadix) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      hv = s_hv[d];  // this thread's own copy
    }
    const uint64_t both = scan256_excl64(((uint64_t)hv << 32) | (d < kRadix ? cnt : 0u), s_tmp);
    const uint32_t dstart = (uint32_t)both, bstart = (uint32_t)(both >> 32);
    if (d < kRadix) {
      s_dstart[d] = dstart;
      // sorted tile position i of a key with digit d goes to segment
      // position s_grel[d] + i (exact modulo 2^32: the sum lies below 2^31)
      s_grel[d] = bstart + (uint32_t)excl - dstart;
    }
    __syncthreads();

#pragma unroll
    for (int i = 0; i < kP; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      if (valid_at(idx)) {
        const K key = key_of(i);
        const uint32_t dg = digit(key);
        const uint32_t woff = kRank == kRankTable ? (uint32_t)(tab[dg] >> 32) : wc[dg];
        const uint32_t pos = s_dstart[dg] + woff + rank_of(i);
        s_keys[pos] = key;
        if constexpr (kVals) s_vals[pos] = val_of(i);
      }
    }
    __syncthreads();
    // write-out: runs of equal digits go to contiguous segment positions
    K* ko = kout ? kout + tl.base : nullptr;
    [[maybe_unused]] V* vo = kVals ? vout + tl.base : nullptr;
    auto put = [&](uint32_t i) {
      const K key = s_keys[i];
      const uint32_t rel = s_grel[digit(key)] + i;
      if constexpr (kPackK) {
        if (remap) {
          const uint64_t o = tl.base + rel + remap[umin64((uint64_t)key, (uint64_t)nremap - 1)];
          if (kout) kout[o] = key;
          if constexpr (kVals) vout[o] = s_vals[i];
          return;
        }
      }
      if (ko) ko[rel] = key;
      if constexpr (kVals) vo[rel] = s_vals[i];
    };
    if constexpr (kFull) {  // a fixed trip count the compiler unrolls
#pragma unroll 4
      for (uint32_t i = threadIdx.x; i < kTT; i += kT) put(i);
    } else {
      for (uint32_t i = threadIdx.x; i < tl.count; i += kT) put(i);
    }
  };
  if (tl.count == kTT) run(std::true_type{});
  else run(std::false_type{});
}

// Last row r of matrix m with row_ptr[r] <= u.
// The row holding stored link u: the last r < nrows with row_ptr[r] <= u,
// found by one warp (all 32 lanes call it; every lane gets the result).
// Each step tests 32 evenly spaced candidates of the remaining range at once
// (the test is monotone: true up to the answer), so a range of 2^k rows
// needs about k / 5 dependent loads.
__device__ __forceinline__ uint64_t row_of_warp(const MatDesc& m, uint64_t nrows, uint64_t u) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t lo = 0, hi = nrows;  // row_ptr[lo] <= u; the answer lies in [lo, hi)
  while (hi - lo > 1) {
    const uint64_t c = lo + ((hi - lo) * (lane + 1)) / 33;  // lo <= c < hi, nondecreasing in lane
    const uint32_t le = __ballot_sync(0xffffffffu, m.row_ptr[c] <= u);
    const int nt = __popc(le);  // the lanes testing true are a prefix
    const uint64_t c_last = __shfl_sync(0xffffffffu, c, nt > 0 ? nt - 1 : 0);
    const uint64_t c_first = __shfl_sync(0xffffffffu, c, nt < 32 ? nt : 31);
    if (nt > 0) lo = c_last;
    if (nt < 32) hi = c_first;
  }
  return lo;
}

constexpr size_t kGatherSmem = 2 * (size_t)(kTile + 1) * sizeof(uint32_t);

// One tile per CTA over the stored links of matrix `seg`: writes the links as
// (src << 32 | dst, count) at the matrix's offset in the concatenation and,
// unless sum_hist is null, accumulates the digit histograms of the single
// time-sum segment.  The rows
// that cover the tile (at most one per link) are staged in shared memory, so
// each link finds its row by a binary search there.  Also zeroes the tickets
// and, unless status0 is null, the sum sort's first status words (k_hist's
// other duties).
__global__ void __launch_bounds__(kThreads) k_gather(SegPlan p, const MatDesc* __restrict__ mats,
                                                     const uint64_t* __restrict__ cat_off,
                                                     uint64_t* __restrict__ keys, uint64_t* __restrict__ vals,
                                                     uint32_t* __restrict__ sum_hist,
                                                     uint64_t* __restrict__ status0,
                                                     uint32_t* __restrict__ tickets) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* s_rp = reinterpret_cast<uint32_t*>(smem);  // row starts relative to the tile, rows r0..r1+1
  uint32_t* s_ri = s_rp + kTile + 1;                    // row ids of rows r0..r1
  __shared__ uint32_t h[kPasses * kRadix];
  __shared__ Tile s_tile;
  __shared__ uint64_t s_r0;
  __shared__ uint32_t s_nr;
  const uint32_t t = blockIdx.x;
  const Tile tl = block_tile(p, t, &s_tile);
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) h[i] = 0;
  if (t == 0 && threadIdx.x < 32) tickets[threadIdx.x] = 0;
  if (status0 && threadIdx.x < kRadix) status0[(uint64_t)t * kRadix + threadIdx.x] = 0;
  if (tl.count == 0) return;
  const MatDesc m = mats[tl.seg];
  __shared__ uint64_t s_r1;
  if (threadIdx.x < 64) {  // warp 0: the tile's first row, warp 1: its last
    const uint64_t r = row_of_warp(m, m.hdr[0], threadIdx.x < 32 ? tl.start : tl.start + tl.count - 1);
    if (threadIdx.x == 0) s_r0 = r;
    if (threadIdx.x == 32) s_r1 = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) s_nr = (uint32_t)(s_r1 - s_r0 + 1);
  __syncthreads();
  const uint64_t r0 = s_r0;
  const uint32_t nr = s_nr;
  for (uint32_t i = threadIdx.x; i <= nr; i += kThreads) {
    const uint64_t rp = m.row_ptr[r0 + i];
    s_rp[i] = rp <= tl.start ? 0u : (uint32_t)umin64(rp - tl.start, tl.count);
    if (i < nr) s_ri[i] = m.row_ids[r0 + i];
  }
  __syncthreads();
  const uint64_t o = cat_off[tl.seg] + tl.start;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = 0; it < kPerThread; ++it) {
    const uint32_t i = warp * (kPerThread * 32) + it * 32 + lane;
    const bool valid = i < tl.count;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    uint64_t key = 0;
    if (valid) {
      uint32_t lo = 0, hi = nr;  // last row r with s_rp[r] <= i
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_rp[mid] <= i) lo = mid; else hi = mid;
      }
      key = ((uint64_t)s_ri[lo] << 32) | m.col_ids[tl.start + i];
      keys[o + i] = key;
      vals[o + i] = m.neg ? 0ull - m.vals[tl.start + i] : m.vals[tl.start + i];
    }
    if (sum_hist) hist_add(h, key, valid, vmask);
  }
  if (!sum_hist) return;
  __syncthreads();
  hist_flush(h, sum_hist, 0);
}

__global__ void __launch_bounds__(1024) k_count_prefix(const MatDesc* __restrict__ mats, uint32_t k,
                                                       uint64_t* __restrict__ cat_off,
                                                       uint64_t* __restrict__ lens,
                                                       uint64_t* __restrict__ total) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t c0 = 0; c0 < k; c0 += 1024) {
    const uint32_t i = c0 + threadIdx.x;
    const uint64_t v = i < k ? mats[i].hdr[1] : 0ull;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint64_t off = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      off += w < warp ? s_w[w] : 0ull;
      tot += s_w[w];
    }
    const uint64_t carry = s_carry;
    if (i < k) {
      cat_off[i] = carry + off + x - v;
      lens[i] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = s_carry;
    cat_off[k] = s_carry;
  }
}

// Dynamic shared memory is configured once per kernel instance and device.
template <typename K, typename V, int kT, int kRank, int kMinB, int kSub>
cudaError_t configure_onesweep_variant() {
  static unsigned long long done = 0;  // one bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((done >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_onesweep<K, V, kT, kRank, kMinB, kSub>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)onesweep_smem_bytes<K, V, kT, kRank, kSub>());
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

template <typename K, typename V, int kT, int kRank, int kMinB, int kSub = 1>
cudaError_t run_onesweep_variant(const SegPlan& p, int pass, const K* kin, K* kout, const V* vin, V* vout,
                                 const uint32_t* seg_hist, uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket,
                                 uint32_t* err, cudaStream_t st, const uint64_t* remap = nullptr,
                                 uint32_t nremap = 0) {
  cudaError_t e = configure_onesweep_variant<K, V, kT, kRank, kMinB, kSub>();
  if (e != cudaSuccess) return e;
  k_onesweep<K, V, kT, kRank, kMinB, kSub><<<kSub * p.ntiles, kT, onesweep_smem_bytes<K, V, kT, kRank, kSub>(), st>>>(
      p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, err, remap, nremap);
  return cudaGetLastError();
}

// The kv forms of the one packet sort of a batch (64-bit keys carrying
// 16-bit window ids, and the regrouping by window id carrying the keys):
// only the 4096-key sub-tile shape (256 threads, four CTAs per SM), with the
// key passes' ranking mode.
template <typename K, typename V>
cudaError_t run_onesweep_sub(const SegPlan& p, int pass, const K* kin, K* kout, const V* vin, V* vout,
                             const uint32_t* seg_hist, uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket,
                             uint32_t* err, const SortCfg& cfg, cudaStream_t st, const uint64_t* remap,
                             uint32_t nremap) {
  if (p.ntiles == 0) return cudaSuccess;
  if (cfg.rank == kRankBallot)
    return run_onesweep_variant<K, V, 256, kRankBallot, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                              st_next, ticket, err, st, remap, nremap);
  if (cfg.rank == kRankTable)
    return run_onesweep_variant<K, V, 256, kRankTable, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                             st_next, ticket, err, st, remap, nremap);
  return run_onesweep_variant<K, V, 256, kRankMatch, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                           st_next, ticket, err, st, remap, nremap);
}

// Window ids of a batch's packets in its one-segment packet plan `pk`: CTA w
// writes id w over window w's packets (at in_off[w] - pk_in_off[0]), the
// offset that takes window w's packets from their place in the batch sorted
// by window to the window's padded base (shift[w] = base[w] - that place),
// and adds the window's packets to the two digit histograms of the ids
// (hist[0][w & 255], hist[1][w >> 8]; zeroed by the caller).
__global__ void __launch_bounds__(256) k_wid_fill(SegPlan p, const uint64_t* __restrict__ pk_in_off,
                                                  uint16_t* __restrict__ wid, uint64_t* __restrict__ shift,
                                                  uint32_t* __restrict__ hist) {
  const uint32_t w = blockIdx.x;
  if (w >= p.nseg) return;
  const uint64_t len = p.len[w];
  const uint64_t at = p.in_off[w] - pk_in_off[0];
  if (threadIdx.x == 0) {
    shift[w] = p.base[w] - at;
    if (len) {
      atomicAdd(&hist[w & 0xffu], (uint32_t)len);
      atomicAdd(&hist[kRadix + ((w >> 8) & 0xffu)], (uint32_t)len);
    }
  }
  uint16_t* out = wid + at;
  const uint16_t id = (uint16_t)w;
  for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) out[i] = id;
}

template <typename K, typename V>
cudaError_t run_onesweep(const SegPlan& p, int pass, const K* kin, K* kout, const V* vin, V* vout,
                         const uint32_t* seg_hist, uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket,
                         uint32_t* err, const SortCfg& cfg, cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
#define ANS_OS(T, R, B)                                                                                        \
  return run_onesweep_variant<K, V, T, R, B>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, \
                                             err, st)
  if constexpr ((std::is_same<K, uint64_t>::value && std::is_same<V, NoVal>::value) ||
                (std::is_same<K, uint32_t>::value && std::is_same<V, uint32_t>::value)) {
    if (cfg.threads == 256) {  // two 4096-key sub-tiles per tile, four CTAs per SM
      if (cfg.rank == kRankBallot)
        return run_onesweep_variant<K, V, 256, kRankBallot, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                                  st_next, ticket, err, st);
      if (cfg.rank == kRankTable)
        return run_onesweep_variant<K, V, 256, kRankTable, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                                 st_next, ticket, err, st);
      return run_onesweep_variant<K, V, 256, kRankMatch, 4, 2>(p, pass, kin, kout, vin, vout, seg_hist, st_cur,
                                                               st_next, ticket, err, st);
    }
  }
  if (cfg.threads == 1024) {
    if (cfg.rank == kRankBallot) ANS_OS(1024, kRankBallot, 1);
    if (cfg.rank == kRankTable) ANS_OS(1024, kRankTable, 1);
    ANS_OS(1024, kRankMatch, 1);
  }
  if (cfg.blocks == 2) {
    if (cfg.rank == kRankBallot) ANS_OS(512, kRankBallot, 2);
    if (cfg.rank == kRankTable) ANS_OS(512, kRankTable, 2);
    ANS_OS(512, kRankMatch, 2);
  }
  if (cfg.rank == kRankBallot) ANS_OS(512, kRankBallot, 1);
  if (cfg.rank == kRankTable) ANS_OS(512, kRankTable, 1);
  ANS_OS(512, kRankMatch, 1);
#undef ANS_OS
}

}  // namespace

cudaError_t launch_pack_hist(const SegPlan& p, const uint32_t* src, const uint32_t* dst,
                             uint64_t* keys, uint32_t* seg_hist, uint64_t* status0, uint32_t* tickets,
                             cudaStream_t st, uint32_t sub) {
  if (p.ntiles == 0) return cudaSuccess;
  k_pack_hist<<<p.ntiles, kThreads, 0, st>>>(p, src, dst, keys, seg_hist, status0, tickets, sub);
  return cudaGetLastError();
}


cudaError_t launch_onesweep(const SegPlan& p, int pass, const uint64_t* kin, uint64_t* kout,
                            const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                            uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                            const SortCfg& cfg, cudaStream_t st) {
  if (vin)
    return run_onesweep<uint64_t, uint64_t>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket,
                                            err, cfg, st);
  return run_onesweep<uint64_t, NoVal>(p, pass, kin, kout, (const NoVal*)nullptr, (NoVal*)nullptr, seg_hist,
                                       st_cur, st_next, ticket, err, cfg, st);
}

cudaError_t launch_onesweep_col32(const SegPlan& p, int pass, const uint32_t* kin, uint32_t* kout,
                                  const uint32_t* vin, uint32_t* vout, const uint32_t* seg_hist,
                                  uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                  const SortCfg& cfg, cudaStream_t st) {
  return run_onesweep<uint32_t, uint32_t>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, err,
                                          cfg, st);
}

cudaError_t launch_onesweep_col(const SegPlan& p, int pass, const uint32_t* kin, uint32_t* kout,
                                const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                                uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                const SortCfg& cfg, cudaStream_t st) {
  return run_onesweep<uint32_t, uint64_t>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, err,
                                          cfg, st);
}

cudaError_t launch_onesweep_wid(const SegPlan& p, int pass, const uint64_t* kin, uint64_t* kout,
                                const uint16_t* vin, uint16_t* vout, const uint32_t* seg_hist, uint64_t* st_cur,
                                uint64_t* st_next, uint32_t* ticket, uint32_t* err, const SortCfg& cfg,
                                cudaStream_t st) {
  return run_onesweep_sub<uint64_t, uint16_t>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, err,
                                              cfg, st, nullptr, 0);
}

cudaError_t launch_onesweep_regroup(const SegPlan& p, int pass, const uint16_t* kin, uint16_t* kout,
                                    const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                                    uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                    const SortCfg& cfg, const uint64_t* remap, uint32_t nremap, cudaStream_t st) {
  if (remap && nremap == 0) return cudaErrorInvalidValue;
  return run_onesweep_sub<uint16_t, uint64_t>(p, pass, kin, kout, vin, vout, seg_hist, st_cur, st_next, ticket, err,
                                              cfg, st, remap, nremap);
}

cudaError_t launch_wid_fill(const SegPlan& p, const uint64_t* pk_in_off, uint16_t* wid, uint64_t* shift,
                            uint32_t* hist, cudaStream_t st) {
  if (p.nseg == 0) return cudaSuccess;
  if (p.nseg > kMaxRegroupWindows) return cudaErrorInvalidValue;
  k_wid_fill<<<p.nseg, 256, 0, st>>>(p, pk_in_off, wid, shift, hist);
  return cudaGetLastError();
}

cudaError_t launch_gather(const SegPlan& p, const MatDesc* mats, const uint64_t* cat_off, uint64_t* keys,
                          uint64_t* vals, uint32_t* sum_hist, uint64_t* status0, uint32_t* tickets,
                          cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
  static unsigned long long configured = 0;  // one bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGatherSmem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured |= 1ull << dev;
  }
  k_gather<<<p.ntiles, kThreads, kGatherSmem, st>>>(p, mats, cat_off, keys, vals, sum_hist, status0, tickets);
  return cudaGetLastError();
}

cudaError_t launch_count_prefix(const MatDesc* mats, uint32_t k, uint64_t* cat_off, uint64_t* lens,
                                uint64_t* total, cudaStream_t st) {
  k_count_prefix<<<1, 1024, 0, st>>>(mats, k, cat_off, lens, total);
  return cudaGetLastError();
}

}  // namespace ans
