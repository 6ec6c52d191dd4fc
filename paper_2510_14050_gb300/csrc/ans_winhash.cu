// Window quantities by on-chip hashing, without sorting (aggregation path 2;
// batches that return no per-window DCSR).
//
// The nine quantities of a window (Table I, Sec. IV-C) need three groupings
// of its packets: by link (unique links, max link packets), by source over
// the distinct links (unique sources, max source packets, max fan-out) and
// by destination over the distinct links (unique destinations, max
// destination packets, max fan-in).  None needs the links in order, so each
// grouping is done by counting in shared-memory hash tables:
//  1. one CTA per window regroups its packets by a hash of the link into
//     ceil(P / 4096) partitions (a counting pass and a scatter pass);
//  2. one CTA per (window, partition) counts the partition's links in a
//     table of 8192 link keys, adds the partition's distinct links and its
//     largest count into the window's accumulator, and appends the distinct
//     links as (source, destination, count) triples to the window's list;
//  3. the same two steps over the distinct links keyed by source (partitions
//     of 8192 links, tables of 16384 sources: links and packets per source),
//     then keyed by destination.
// A partition whose table overflows (more distinct keys than it holds at
// three quarters load), or a window of more than 2^18 packets, marks the
// window failed; the batch then sorts exactly the failed windows (their
// plan length is kept, every other window's is set to 0) and the hashed
// quantities are written over the sorted windows' results only where the
// window did not fail.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr int kHqThreads = 1024;
constexpr int kHqUnroll = 4;
constexpr uint32_t kLinkPartPackets = 4096;                  // packets per link partition (mean)
constexpr uint32_t kLinkParts = kHqMaxPackets / kLinkPartPackets;  // 64
constexpr uint32_t kLinkSlots = 8192;                        // link table: uint64 key + uint32 count
constexpr uint32_t kLinkMaxFill = kLinkSlots / 4 * 3;
constexpr size_t kLinkSmem = (size_t)kLinkSlots * 12;
constexpr uint64_t kLinkEmpty = ~0ull;                       // marks an empty slot (that link is counted apart)
constexpr uint32_t kKeyPartLinks = 4096;                     // links per source / destination partition (mean)
constexpr uint32_t kKeyParts = kHqMaxPackets / kKeyPartLinks;  // 64
constexpr uint32_t kKeySlots = 8192;                         // key, links, packets (uint32 each): 96 KB
constexpr uint32_t kKeyMaxFill = kKeySlots / 4 * 3;
constexpr size_t kKeySmem = (size_t)kKeySlots * 12;
constexpr uint32_t kKeyEmpty = 0xFFFFFFFFu;
static_assert(kLinkParts * kLinkPartPackets == kHqMaxPackets, "link partitions cover the largest window");
static_assert(kKeyParts * kKeyPartLinks == kHqMaxPackets, "key partitions cover the largest window's links");

// MurmurHash3's finalizers (Appleby): bijective 64- and 32-bit mixes.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}
__device__ __forceinline__ uint32_t fmix32h(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Partitions: the high bits of the mix, scaled to [0, parts); table slots
// use the low bits.
__device__ __forceinline__ uint32_t link_part(uint64_t key, uint32_t parts) {
  return (uint32_t)(((fmix64(key) >> 40) * parts) >> 24);
}
__device__ __forceinline__ uint32_t key_part(uint32_t key, uint32_t parts) {
  return (uint32_t)(((uint64_t)(fmix32h(key) >> 14) * parts) >> 18);
}

__device__ __forceinline__ uint32_t ceil_div(uint64_t n, uint32_t d) { return (uint32_t)((n + d - 1) / d); }

// Warp-aggregated slot in a partition: lanes with the same partition share
// one shared-memory atomic on its cursor.
__device__ __forceinline__ uint32_t claim_slot(uint32_t* cur, uint32_t pt, bool valid) {
  const int lane = threadIdx.x & 31;
  const uint32_t peers = __match_any_sync(0xffffffffu, valid ? pt : 0xFFFFFFFFu);
  const int leader = __ffs(peers) - 1;
  uint32_t pos = 0;
  if (valid && lane == leader) pos = atomicAdd(&cur[pt], __popc(peers));
  return __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & lanemask_lt());
}

// Step 1: one CTA per window regroups its packets (as link keys) by link
// partition into keys + base[s]; partition starts in lstart[s][0..parts].
// A window above kHqMaxPackets is marked failed (it will be sorted).
__global__ void __launch_bounds__(kHqThreads, 2) k_hq_split(SegPlan p, const uint32_t* __restrict__ src,
                                                            const uint32_t* __restrict__ dst,
                                                            uint64_t* __restrict__ keys, uint32_t* __restrict__ lstart,
                                                            HqWin* __restrict__ win) {
  __shared__ uint32_t s_cnt[kLinkParts], s_cur[kLinkParts];
  const uint32_t s = blockIdx.x;
  if (s >= p.nseg) return;
  const uint64_t n = p.len[s];
  if (n == 0) return;
  if (n > kHqMaxPackets) {
    if (threadIdx.x == 0) win[s].fail = 1;
    return;
  }
  const uint32_t parts = ceil_div(n, kLinkPartPackets);
  const uint32_t *ws, *wd;
  window_inputs(p, s, src, dst, &ws, &wd);
  if (threadIdx.x < kLinkParts) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t w0 = threadIdx.x & ~31u; w0 < n; w0 += kHqUnroll * kHqThreads) {
    const uint32_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint64_t k[kHqUnroll];
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const uint32_t u = u0 + j * kHqThreads;
      k[j] = u < n ? ((uint64_t)ws[u] << 32) | wd[u] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const bool valid = u0 + j * kHqThreads < n;
      const uint32_t pt = valid ? link_part(k[j], parts) : 0u;
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? pt : 0xFFFFFFFFu);
      if (valid && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_cnt[pt], __popc(peers));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t r = 0; r < parts; ++r) {
      s_cur[r] = run;
      lstart[(uint64_t)s * (kLinkParts + 1) + r] = run;
      run += s_cnt[r];
    }
    lstart[(uint64_t)s * (kLinkParts + 1) + parts] = run;
  }
  __syncthreads();
  uint64_t* out = keys + p.base[s];
  for (uint32_t w0 = threadIdx.x & ~31u; w0 < n; w0 += kHqUnroll * kHqThreads) {
    const uint32_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint64_t k[kHqUnroll];
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const uint32_t u = u0 + j * kHqThreads;
      k[j] = u < n ? ((uint64_t)ws[u] << 32) | wd[u] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const bool valid = u0 + j * kHqThreads < n;
      const uint32_t pt = valid ? link_part(k[j], parts) : 0u;
      const uint32_t pos = claim_slot(s_cur, pt, valid);
      if (valid) out[pos] = k[j];
    }
  }
}

// Block reduction of (sum, max) over all threads; thread 0 gets the result.
__device__ __forceinline__ void block_sum_max(unsigned long long& sum, unsigned long long& mx,
                                              unsigned long long (*red)[kHqThreads / 32]) {
  sum = warp_sum(sum);
  mx = warp_max(mx);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = sum;
    red[1][warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sum = 0;
    mx = 0;
    for (int w = 0; w < kHqThreads / 32; ++w) {
      sum += red[0][w];
      mx = red[1][w] > mx ? red[1][w] : mx;
    }
  }
}

// Work items of the counting steps: items[v] = the first item of virtual
// segment v (an exclusive prefix of per-segment partition counts; the last
// entry is the total), for kind 0 the windows' link partitions, for kind 1
// the source partitions of every window followed by the destination ones.
// One CTA; also zeroes the queue counter the persistent kernels draw from.
__global__ void __launch_bounds__(kHqThreads) k_hq_items(SegPlan p, const HqWin* __restrict__ win, int kind,
                                                         uint32_t* __restrict__ items, uint32_t* __restrict__ counter) {
  __shared__ uint32_t s_tmp[kHqThreads / 32];
  const uint32_t nv = kind == 0 ? p.nseg : 2 * p.nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (uint32_t c0 = 0; c0 < nv; c0 += kHqThreads) {
    const uint32_t v = c0 + threadIdx.x;
    uint32_t cnt = 0;
    if (v < nv) {
      if (kind == 0) {
        const uint64_t n = p.len[v];
        cnt = (n == 0 || n > kHqMaxPackets) ? 0u : ceil_div(n, kLinkPartPackets);
      } else {
        const HqWin& w = win[v % p.nseg];
        cnt = (w.nlinks == 0 || w.fail) ? 0u : ceil_div(w.nlinks, kKeyPartLinks);
      }
    }
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_tmp[warp] = x;
    __syncthreads();
    uint32_t off = 0, tot = 0;
    for (int w = 0; w < kHqThreads / 32; ++w) {
      off += w < warp ? s_tmp[w] : 0u;
      tot += s_tmp[w];
    }
    if (v < nv) items[v] = carry + off + x - cnt;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    items[nv] = carry;
    *counter = 0;
  }
}

// The next work item of a persistent CTA (every thread gets it), and its
// virtual segment: the last v with items[v] <= item.  Returns false when the
// queue is empty.
__device__ __forceinline__ bool next_item(uint32_t* counter, const uint32_t* items, uint32_t nv, uint32_t* s_item,
                                          uint32_t* v_out, uint32_t* r_out) {
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t it = *s_item;
  __syncthreads();  // everyone has read it before the next draw overwrites it
  if (it >= items[nv]) return false;
  uint32_t lo = 0, hi = nv;  // items[lo] <= it < items[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (items[mid] <= it) lo = mid; else hi = mid;
  }
  *v_out = lo;
  *r_out = it - items[lo];
  return true;
}

// Step 2 (persistent: each CTA draws (window, link partition) items): the
// partition's links counted in a table of kLinkSlots keys; the window's
// accumulator gets the partition's distinct links and largest link count,
// and the distinct links are appended as (source, destination, count) at
// lsrc / ldst / lcnt + base[s] + (the window's running link count).
__global__ void __launch_bounds__(kHqThreads, 2) k_hq_links(SegPlan p, const uint64_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ lstart,
                                                            uint32_t* __restrict__ lsrc, uint32_t* __restrict__ ldst,
                                                            uint32_t* __restrict__ lcnt, HqWin* __restrict__ win,
                                                            const uint32_t* __restrict__ items, uint32_t* counter) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t* t_key = reinterpret_cast<uint64_t*>(smem);
  uint32_t* t_cnt = reinterpret_cast<uint32_t*>(smem + (size_t)kLinkSlots * 8);
  __shared__ uint32_t s_fill, s_over, s_spec, s_off, s_item;
  __shared__ unsigned long long s_red[2][kHqThreads / 32];
  __shared__ uint32_t s_wcnt[kHqThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t s, r;
  while (next_item(counter, items, p.nseg, &s_item, &s, &r)) {
    const uint32_t lo = lstart[(uint64_t)s * (kLinkParts + 1) + r];
    const uint32_t hi = lstart[(uint64_t)s * (kLinkParts + 1) + r + 1];
    const uint64_t* in = keys + p.base[s];
    for (uint32_t i = threadIdx.x; i < kLinkSlots; i += kHqThreads) {
      t_key[i] = kLinkEmpty;
      t_cnt[i] = 0;
    }
    if (threadIdx.x == 0) s_fill = s_over = s_spec = 0;
    __syncthreads();
    for (uint32_t u0 = lo; u0 < hi; u0 += kHqThreads) {  // the same bound for every thread
      const uint32_t u = u0 + threadIdx.x;
      const bool valid = u < hi;
      const uint64_t k = valid ? in[u] : kLinkEmpty;
      // lanes holding the same link add it once (lanes past the partition's
      // end hold a filler equal to the all-ones link: masked out)
      const uint32_t peers = __match_any_sync(0xffffffffu, k) & __ballot_sync(0xffffffffu, valid);
      if (!valid || lane != __ffs(peers) - 1) continue;
      const uint32_t c = __popc(peers);
      if (k == kLinkEmpty) {
        atomicAdd(&s_spec, c);
        continue;
      }
      if (*(volatile uint32_t*)&s_over) continue;
      uint32_t h = (uint32_t)fmix64(k) & (kLinkSlots - 1);
      for (uint32_t probe = 0; probe < kLinkSlots; ++probe) {
        unsigned long long cur = *(volatile unsigned long long*)&t_key[h];
        if (cur == kLinkEmpty) {
          cur = atomicCAS((unsigned long long*)&t_key[h], (unsigned long long)kLinkEmpty, (unsigned long long)k);
          if (cur == kLinkEmpty) {
            cur = k;
            if (atomicAdd(&s_fill, 1u) + 1 > kLinkMaxFill) s_over = 1;
          }
        }
        if (cur == k) {
          atomicAdd(&t_cnt[h], c);
          break;
        }
        h = (h + 1) & (kLinkSlots - 1);
      }
    }
    __syncthreads();
    HqWin* w = win + s;
    if (s_over) {  // the window is sorted instead
      if (threadIdx.x == 0) atomicOr(&w->fail, 1u);
      continue;    // (uniform: s_over is shared)
    }
    // distinct links of this partition: count, largest count, then append
    // (each thread its own slots' links, at its exclusive offset in the CTA)
    unsigned long long nl = 0, mx = 0;
    for (uint32_t i = threadIdx.x; i < kLinkSlots; i += kHqThreads) {
      if (t_key[i] != kLinkEmpty) {
        ++nl;
        mx = t_cnt[i] > mx ? t_cnt[i] : mx;
      }
    }
    const uint32_t mine = (uint32_t)nl;
    uint32_t x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wcnt[warp] = x;
    unsigned long long tot = nl, m2 = mx;
    block_sum_max(tot, m2, s_red);
    if (threadIdx.x == 0) {
      const uint32_t spec = s_spec;
      tot += spec ? 1 : 0;
      m2 = spec > m2 ? spec : m2;
      s_off = atomicAdd(&w->nlinks, (uint32_t)tot);
      if (tot) atomicAdd(&w->links, tot);
      if (m2) atomicMax(&w->max_link, m2);
      s_fill = (uint32_t)tot;  // (the table is done: reuse the word for the total)
    }
    __syncthreads();
    uint32_t woff = 0;
    for (int v = 0; v < warp; ++v) woff += s_wcnt[v];
    uint32_t o = s_off + woff + x - mine;
    const uint64_t b = p.base[s];
    for (uint32_t i = threadIdx.x; i < kLinkSlots; i += kHqThreads) {
      const uint64_t k = t_key[i];
      if (k != kLinkEmpty) {
        lsrc[b + o] = (uint32_t)(k >> 32);
        ldst[b + o] = (uint32_t)k;
        lcnt[b + o] = t_cnt[i];
        ++o;
      }
    }
    if (threadIdx.x == 0 && s_spec) {  // the all-ones link, counted apart, goes last
      const uint32_t last = s_off + s_fill - 1;
      lsrc[b + last] = kKeyEmpty;
      ldst[b + last] = kKeyEmpty;
      lcnt[b + last] = s_spec;
    }
    __syncthreads();  // the table is read no more
  }
}

// Step 3a: one CTA per window regroups its distinct links' (key, count) --
// key = source (stage 0) or destination (stage 1) -- by key partition into
// pkey / pval + base[s]; partition starts in kstart[s][0..parts].
__global__ void __launch_bounds__(kHqThreads, 2) k_hq_keysplit(SegPlan p, HqBufs bufs) {
  __shared__ uint32_t s_cnt[kKeyParts], s_cur[kKeyParts];
  const uint32_t stage = blockIdx.x / p.nseg, s = blockIdx.x % p.nseg;  // both stages in one grid
  const uint32_t* kin = stage == 0 ? bufs.lsrc : bufs.ldst;
  const uint32_t* cin = bufs.lcnt;
  uint32_t* pkey = bufs.pkey[stage];
  uint32_t* pval = bufs.pval[stage];
  uint32_t* kstart = bufs.kstart + (size_t)stage * p.nseg * (kKeyParts + 1);
  const HqWin* win = bufs.win;
  const HqWin& w = win[s];
  const uint32_t n = w.nlinks;
  if (n == 0 || w.fail) return;
  const uint32_t parts = ceil_div(n, kKeyPartLinks);
  const uint64_t b = p.base[s];
  if (threadIdx.x < kKeyParts) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t w0 = threadIdx.x & ~31u; w0 < n; w0 += kHqUnroll * kHqThreads) {
    const uint32_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint32_t k[kHqUnroll];
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const uint32_t u = u0 + j * kHqThreads;
      k[j] = u < n ? kin[b + u] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const bool valid = u0 + j * kHqThreads < n;
      const uint32_t pt = valid ? key_part(k[j], parts) : 0u;
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? pt : 0xFFFFFFFFu);
      if (valid && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_cnt[pt], __popc(peers));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t r = 0; r < parts; ++r) {
      s_cur[r] = run;
      kstart[(uint64_t)s * (kKeyParts + 1) + r] = run;
      run += s_cnt[r];
    }
    kstart[(uint64_t)s * (kKeyParts + 1) + parts] = run;
  }
  __syncthreads();
  for (uint32_t w0 = threadIdx.x & ~31u; w0 < n; w0 += kHqUnroll * kHqThreads) {
    const uint32_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint32_t k[kHqUnroll], c[kHqUnroll];
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const uint32_t u = u0 + j * kHqThreads;
      k[j] = u < n ? kin[b + u] : 0u;
      c[j] = u < n ? cin[b + u] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kHqUnroll; ++j) {
      const bool valid = u0 + j * kHqThreads < n;
      const uint32_t pt = valid ? key_part(k[j], parts) : 0u;
      const uint32_t pos = claim_slot(s_cur, pt, valid);
      if (valid) {
        pkey[b + pos] = k[j];
        pval[b + pos] = c[j];
      }
    }
  }
}

// Step 3b (persistent: each CTA draws (stage, window, key partition)
// items): the partition's keys counted, per key its links (fan-out /
// fan-in) and packets; the window gets the number of distinct keys, the
// largest link count and the largest packet count of the stage.
__global__ void __launch_bounds__(kHqThreads, 2) k_hq_keyhash(SegPlan p, HqBufs bufs, const uint32_t* __restrict__ items,
                                                              uint32_t* counter) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_lnk = sm + kKeySlots;
  uint32_t* t_pkt = sm + 2 * kKeySlots;
  __shared__ uint32_t s_fill, s_over, s_spec_l, s_spec_p, s_item;
  __shared__ unsigned long long s_red[3][kHqThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t v, r;
  while (next_item(counter, items, 2 * p.nseg, &s_item, &v, &r)) {
    const uint32_t st = v / p.nseg, s = v % p.nseg;
    const uint32_t* pkey = bufs.pkey[st];
    const uint32_t* pval = bufs.pval[st];
    const uint32_t* kstart = bufs.kstart + (size_t)st * p.nseg * (kKeyParts + 1);
    HqWin* w = bufs.win + s;
    const uint64_t b = p.base[s];
    const uint32_t lo = kstart[(uint64_t)s * (kKeyParts + 1) + r], hi = kstart[(uint64_t)s * (kKeyParts + 1) + r + 1];
    for (uint32_t i = threadIdx.x; i < kKeySlots; i += kHqThreads) {
      t_key[i] = kKeyEmpty;
      t_lnk[i] = 0;
      t_pkt[i] = 0;
    }
    if (threadIdx.x == 0) s_fill = s_over = s_spec_l = s_spec_p = 0;
    __syncthreads();
    for (uint32_t u = lo + threadIdx.x; u < hi; u += kHqThreads) {
      if (*(volatile uint32_t*)&s_over) break;
      const uint32_t k = pkey[b + u];
      const uint32_t c = pval[b + u];
      if (k == kKeyEmpty) {
        atomicAdd(&s_spec_l, 1u);
        atomicAdd(&s_spec_p, c);
        continue;
      }
      uint32_t h = fmix32h(k) & (kKeySlots - 1);
      for (uint32_t probe = 0; probe < kKeySlots; ++probe) {
        uint32_t cur = *(volatile uint32_t*)&t_key[h];
        if (cur == kKeyEmpty) {
          cur = atomicCAS(&t_key[h], kKeyEmpty, k);
          if (cur == kKeyEmpty) {
            cur = k;
            if (atomicAdd(&s_fill, 1u) + 1 > kKeyMaxFill) s_over = 1;
          }
        }
        if (cur == k) {
          atomicAdd(&t_lnk[h], 1u);
          atomicAdd(&t_pkt[h], c);
          break;
        }
        h = (h + 1) & (kKeySlots - 1);
      }
    }
    __syncthreads();
    if (s_over) {  // the window is sorted instead (uniform: s_over is shared)
      if (threadIdx.x == 0) atomicOr(&w->fail, 1u);
      continue;
    }
    unsigned long long cnt = 0, ml = 0, mp = 0;
    for (uint32_t i = threadIdx.x; i < kKeySlots; i += kHqThreads) {
      if (t_key[i] != kKeyEmpty) {
        ++cnt;
        ml = t_lnk[i] > ml ? t_lnk[i] : ml;
        mp = t_pkt[i] > mp ? t_pkt[i] : mp;
      }
    }
    cnt = warp_sum(cnt);
    ml = warp_max(ml);
    mp = warp_max(mp);
    if (lane == 0) {
      s_red[0][warp] = cnt;
      s_red[1][warp] = ml;
      s_red[2][warp] = mp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cnt = ml = mp = 0;
      for (int q = 0; q < kHqThreads / 32; ++q) {
        cnt += s_red[0][q];
        ml = s_red[1][q] > ml ? s_red[1][q] : ml;
        mp = s_red[2][q] > mp ? s_red[2][q] : mp;
      }
      if (s_spec_l) {
        ++cnt;
        ml = s_spec_l > ml ? s_spec_l : ml;
        mp = s_spec_p > mp ? s_spec_p : mp;
      }
      if (cnt) atomicAdd(&w->keys[st], cnt);
      if (ml) atomicMax(&w->max_links[st], ml);
      if (mp) atomicMax(&w->max_packets[st], mp);
    }
    __syncthreads();  // the table is read no more
  }
}

// Before the sort: the windows the hash finished get sort length 0 (the
// sort, run statistics and column pass then leave them empty); the others,
// failed or too large, keep their length.
__global__ void k_hq_mask(SegPlan p, const HqWin* __restrict__ win, uint64_t* __restrict__ sort_len) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.nseg; s += gridDim.x * blockDim.x) {
    const uint64_t n = p.len[s];
    sort_len[s] = (n == 0 || win[s].fail || n > kHqMaxPackets) ? n : 0ull;
  }
}

// After the sorted windows' statistics: the hashed windows' nine quantities.
__global__ void k_hq_write(SegPlan p, const HqWin* __restrict__ win, ans_quantities* __restrict__ q) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.nseg; s += gridDim.x * blockDim.x) {
    const uint64_t n = p.len[s];
    const HqWin& w = win[s];
    if (n == 0 || w.fail || n > kHqMaxPackets) continue;
    ans_quantities r;
    r.valid_packets = n;
    r.unique_links = w.links;
    r.max_link_packets = w.max_link;
    r.unique_sources = w.keys[0];
    r.max_source_packets = w.max_packets[0];
    r.max_source_fanout = w.max_links[0];
    r.unique_destinations = w.keys[1];
    r.max_destination_packets = w.max_packets[1];
    r.max_destination_fanin = w.max_links[1];
    q[s] = r;
  }
}

// Persistent CTAs of the counting kernels: two per SM (96 KB of shared
// memory and 1024 threads each).
unsigned persistent_ctas() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 2 * 148;
  if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 2 * 148;
  }
  return 2u * (unsigned)sms[dev];
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes, unsigned long long* configured) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && ((*configured >> dev) & 1ull)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 64) *configured |= 1ull << dev;
  return e;
}

}  // namespace

cudaError_t launch_hq_stage(int stage, const SegPlan& p, const uint32_t* src, const uint32_t* dst, const HqBufs& b,
                            cudaStream_t st) {
  if (p.nseg == 0) return cudaSuccess;
  static unsigned long long cfg_links = 0, cfg_keys = 0;
  cudaError_t e;
  switch (stage) {
    case 0:
      k_hq_split<<<p.nseg, kHqThreads, 0, st>>>(p, src, dst, b.keys, b.lstart, b.win);
      break;
    case 1:
      if ((e = set_smem(k_hq_links, kLinkSmem, &cfg_links)) != cudaSuccess) return e;
      k_hq_items<<<1, kHqThreads, 0, st>>>(p, b.win, 0, b.items, b.counter);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      k_hq_links<<<persistent_ctas(), kHqThreads, kLinkSmem, st>>>(p, b.keys, b.lstart, b.lsrc, b.ldst, b.lcnt, b.win,
                                                                  b.items, b.counter);
      break;
    case 2:
      k_hq_keysplit<<<2 * p.nseg, kHqThreads, 0, st>>>(p, b);
      break;
    case 3:
      if ((e = set_smem(k_hq_keyhash, kKeySmem, &cfg_keys)) != cudaSuccess) return e;
      k_hq_items<<<1, kHqThreads, 0, st>>>(p, b.win, 1, b.items, b.counter);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      k_hq_keyhash<<<persistent_ctas(), kHqThreads, kKeySmem, st>>>(p, b, b.items, b.counter);
      break;
    default: {
      const uint32_t g = (p.nseg + 255) / 256;
      k_hq_mask<<<g < 1024 ? g : 1024, 256, 0, st>>>(p, b.win, b.sort_len);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_hq_write(const SegPlan& p, const HqWin* win, ans_quantities* q, cudaStream_t st) {
  if (p.nseg == 0) return cudaSuccess;
  const uint32_t g = (p.nseg + 255) / 256;
  k_hq_write<<<g < 1024 ? g : 1024, 256, 0, st>>>(p, win, q);
  return cudaGetLastError();
}

}  // namespace ans
