// From sorted link keys to DCSR and the nine network quantities.
//
//  * k_rle: run-length reduce-by-key.  A position starts a link run when its
//    key differs from its predecessor, and starts a row when the source half
//    differs.  Run and row counts are carried across tiles by bounded
//    decoupled look-back, so each tile writes its part of col_ids, row_ids and
//    row_ptr directly (Sec. IV-B containers: edges, degrees as row_ptr
//    differences).  Run and row start *positions* are kept so that counts and
//    row sums become differences of positions (or of a value prefix).
//  * k_scan_u64: exclusive prefix of uint64 values (time sums, imported
//    matrices), same look-back scheme.
//  * k_finish: link values A(i,j) (Table I), the link maximum, per-row
//    nonzero counts (fan-out) and packet sums (Sec. IV-C); it also builds the
//    digit histograms of the destination keys for the column sort.
//  * k_colstat / k_colstat_fin: the transpose-free column pass.  Once the
//    stored links are sorted by destination (32-bit keys carrying the link
//    counts), every run of equal destinations is one column: its length is the
//    fan-in and its value sum the destination's packets (Table I, Sec. IV-C).
//    Runs inside a tile are reduced in place; runs that cross tiles are
//    completed from per-tile boundary records.
//  * k_colhash / k_colhash_cl: the same three column quantities of a window
//    from a shared-memory hash of its destinations (one CTA per window, or a
//    thread-block cluster per window whose CTAs merge their tables over
//    distributed shared memory); windows with more distinct destinations than
//    the table takes are left to the column sort.
// Maxima are combined with 64-bit atomicMax; every value is an exact integer.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr uint64_t kLow31 = (1ull << 31) - 1;

__global__ void __launch_bounds__(kThreads, 2) k_rle(StatsArgs a) {
  __shared__ uint32_t s_ticket;
  __shared__ Tile s_tile;
  __shared__ uint32_t s_wh[kWarps], s_wr[kWarps];
  __shared__ uint64_t s_eh, s_er;

  const uint32_t t = block_ticket(a.ticket, &s_ticket);
  const Tile tl = block_tile(a.plan, t, &s_tile);
  const uint64_t bs = tl.base + tl.seg;  // start of the "+1" arrays of this segment
  if (tl.count == 0) {
    if (tl.j == 0 && threadIdx.x == 0) {  // empty segment of device-computed length
      if (a.run_start) a.run_start[bs] = 0;
      if (a.row_pos) a.row_pos[bs] = 0;
      a.row_ptr[bs] = 0;
      a.hdr[2 * tl.seg] = 0;
      a.hdr[2 * tl.seg + 1] = 0;
    }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * (kPerThread * 32);
  const uint64_t* keys = a.keys + tl.base + tl.start;

  uint64_t k[kPerThread];
  uint32_t hb[kPerThread], rb[kPerThread];
  uint64_t carry = 0;
  bool carry_valid = false;
  if (tl.start + wbase > 0 && wbase < tl.count) {
    carry = keys[(int64_t)wbase - 1];
    carry_valid = true;
  }
  uint32_t nh = 0, nr = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    const bool valid = idx < tl.count;
    k[i] = valid ? keys[idx] : 0ull;
    uint64_t prev = __shfl_up_sync(0xffffffffu, k[i], 1);
    bool has_prev = true;
    if (lane == 0) {
      prev = carry;
      has_prev = (i > 0) || carry_valid;
    }
    const bool head = valid && (!has_prev || prev != k[i]);
    const bool rhead = valid && (!has_prev || (prev >> 32) != (k[i] >> 32));
    hb[i] = __ballot_sync(0xffffffffu, head);
    rb[i] = __ballot_sync(0xffffffffu, rhead);
    nh += __popc(hb[i]);
    nr += __popc(rb[i]);
    carry = __shfl_sync(0xffffffffu, k[i], 31);
  }
  if (lane == 0) {
    s_wh[warp] = nh;
    s_wr[warp] = nr;
  }
  __syncthreads();
  if (warp == 0) {  // the tile's counts, then the look-back by the whole warp
    uint32_t th = 0, tr = 0;
    if (lane == 0) {
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t x = s_wh[w], y = s_wr[w];
        s_wh[w] = th;
        s_wr[w] = tr;
        th += x;
        tr += y;
      }
    }
    th = __shfl_sync(0xffffffffu, th, 0);
    tr = __shfl_sync(0xffffffffu, tr, 0);
    const uint64_t agg = ((uint64_t)th << 31) | tr;
    uint64_t* my = a.lookback + t;
    uint64_t excl = 0;
    if (tl.j == 0) {
      if (lane == 0) st_relaxed(my, kFlagPre | agg);
    } else {
      if (lane == 0) st_relaxed(my, kFlagAgg | agg);
      excl = warp_lookback(a.lookback, 1, t - tl.j, t, a.err);
      if (lane == 0) st_relaxed(my, kFlagPre | (excl + agg));
    }
    if (lane == 0) {
      const uint64_t eh = excl >> 31, er = excl & kLow31;
      s_eh = eh;
      s_er = er;
      if (tl.start + tl.count == tl.len) {  // last tile: terminators and header
        const uint64_t u = eh + th, r = er + tr;
        if (a.run_start) a.run_start[bs + u] = tl.len;
        if (a.row_pos) a.row_pos[bs + r] = tl.len;
        a.row_ptr[bs + r] = u;
        a.hdr[2 * tl.seg] = r;
        a.hdr[2 * tl.seg + 1] = u;
      }
    }
  }
  __syncthreads();
  uint64_t uh = s_eh + s_wh[warp], ur = s_er + s_wr[warp];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    if ((hb[i] >> lane) & 1u) {
      const uint64_t u = uh + __popc(hb[i] & lt);
      a.col_ids[tl.base + u] = (uint32_t)k[i];
      if (a.sum_keys) a.sum_keys[tl.base + u] = k[i];
      if (a.run_start) a.run_start[bs + u] = tl.start + idx;
      if ((rb[i] >> lane) & 1u) {
        const uint64_t r = ur + __popc(rb[i] & lt);
        a.row_ids[tl.base + r] = (uint32_t)(k[i] >> 32);
        a.row_ptr[bs + r] = u;
        if (a.row_pos) a.row_pos[bs + r] = tl.start + idx;
      }
    }
    uh += __popc(hb[i]);
    ur += __popc(rb[i]);
  }
}

// Prefixes are kept mod 2^62 (the width of a look-back status value), and
// every difference of two of them is reduced mod 2^62: exact for any sum of
// counts below 2^62, and for signed combinations whose results are
// nonnegative and below 2^61.
__global__ void __launch_bounds__(kThreads) k_scan_u64(SegPlan p, const uint64_t* __restrict__ in,
                                                       uint64_t* __restrict__ out, uint64_t* lookback_st,
                                                       uint32_t* ticket, uint32_t* err) {
  __shared__ uint32_t s_ticket;
  __shared__ Tile s_tile;
  __shared__ uint64_t s_w[kWarps];
  __shared__ uint64_t s_excl;
  const uint32_t t = block_ticket(ticket, &s_ticket);
  const Tile tl = block_tile(p, t, &s_tile);
  const uint64_t bs = tl.base + tl.seg;
  if (tl.count == 0) {
    if (tl.j == 0 && threadIdx.x == 0) out[bs] = 0;
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * (kPerThread * 32);
  uint64_t ex[kPerThread];
  uint64_t run = 0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    const uint64_t v = idx < tl.count ? in[tl.base + tl.start + idx] : 0ull;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    ex[i] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) s_w[warp] = run;
  __syncthreads();
  if (warp == 0) {  // the tile's total, then the look-back by the whole warp
    uint64_t tot = 0;
    if (lane == 0) {
      for (int w = 0; w < kWarps; ++w) {
        const uint64_t x = s_w[w];
        s_w[w] = tot;
        tot += x;
      }
    }
    tot = __shfl_sync(0xffffffffu, tot, 0);
    uint64_t* my = lookback_st + t;
    uint64_t excl = 0;
    if (tl.j == 0) {
      if (lane == 0) st_relaxed(my, kFlagPre | (tot & kValMask));
    } else {
      if (lane == 0) st_relaxed(my, kFlagAgg | (tot & kValMask));
      excl = warp_lookback(lookback_st, 1, t - tl.j, t, err);
      if (lane == 0) st_relaxed(my, kFlagPre | ((excl + tot) & kValMask));
    }
    if (lane == 0) {
      s_excl = excl;
      if (tl.start + tl.count == tl.len) out[bs + tl.len] = (excl + tot) & kValMask;
    }
  }
  __syncthreads();
  const uint64_t off = s_excl + s_w[warp];
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    if (idx < tl.count) out[bs + tl.start + idx] = (off + ex[i]) & kValMask;
  }
}

// Finalizer of MurmurHash3 (Appleby): a bijective 32-bit mix.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

template <int kMode, bool kHKeys>
__global__ void __launch_bounds__(kThreads, 3) k_finish(StatsArgs a) {
  __shared__ Tile s_tile;
  __shared__ uint64_t s_red[3][kWarps];
  __shared__ uint32_t s_h[kColPasses * kRadix];
  const uint32_t t = blockIdx.x;
  const Tile tl = block_tile(a.plan, t, &s_tile);
  const uint32_t s = tl.seg;
  const uint64_t nrows = a.hdr[2 * s], nnz = a.hdr[2 * s + 1];
  const uint64_t bs = tl.base + s;
  for (int i = threadIdx.x; i < kColPasses * kRadix; i += kThreads) s_h[i] = 0;
  // Prepare the column sort: its first-pass status words, its tickets and
  // the number of links per segment.
  if (t == 0 && threadIdx.x < 32) a.col_tickets[threadIdx.x] = 0;
  // (two sub-tiles' worth per tile: the column passes may run sub-tiles)
  for (uint32_t i = threadIdx.x; i < 2 * kRadix; i += kThreads) a.col_st0[(uint64_t)t * 2 * kRadix + i] = 0;
  if (tl.j == 0 && threadIdx.x == 0) a.ulen[s] = nnz;
  __syncthreads();

  auto P = [&](uint64_t x) -> uint64_t { return a.pre ? a.pre[bs + x] : x; };

  uint64_t mlink = 0, mfan = 0, mrow = 0;
  const uint64_t u_end = umin64(tl.start + kTile, nnz);
  // kU links per thread and step, their loads issued before any use (the
  // loads of one link depend on one another, the links do not).
  constexpr int kU = 4;
  for (uint64_t u0 = tl.start + threadIdx.x; u0 < u_end; u0 += (uint64_t)kU * kThreads) {
    uint64_t x0[kU], x1[kU];
    uint32_t dst[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const uint64_t u = u0 + (uint64_t)j * kThreads;
      x0[j] = x1[j] = 0;
      dst[j] = 0;
      if (u < u_end) {
        if (kMode == kModeMatrix) {
          x0[j] = a.vals[tl.base + u];
        } else {
          x0[j] = a.run_start[bs + u];
          x1[j] = a.run_start[bs + u + 1];
        }
        dst[j] = a.col_ids[tl.base + u];
      }
    }
    if (kMode != kModeMatrix && a.pre) {
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        if (u0 + (uint64_t)j * kThreads < u_end) {
          x0[j] = a.pre[bs + x0[j]];
          x1[j] = a.pre[bs + x1[j]];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const uint64_t u = u0 + (uint64_t)j * kThreads;
      if (u >= u_end) continue;
      const uint64_t v = kMode == kModeMatrix ? x0[j] : (x1[j] - x0[j]) & kValMask;
      if (kMode != kModeMatrix) {
        a.vals[tl.base + u] = v;
        if (a.vals32) a.vals32[tl.base + u] = (uint32_t)v;
      }
      mlink = v > mlink ? v : mlink;
      // the column sort's key: the destination, or its bijective mix when
      // the sum's column statistics group destinations by hash
      uint32_t ck = dst[j];
      if constexpr (kHKeys) {
        ck = fmix32(ck);
        a.col_hkeys[tl.base + u] = ck;
      }
#pragma unroll
      for (int p = 0; p < kColPasses; ++p)
        atomicAdd(&s_h[p * kRadix + ((ck >> (p * kRadixBits)) & 0xffu)], 1u);
    }
  }
  const uint64_t r_end = umin64(tl.start + kTile, nrows);
  for (uint64_t r = tl.start + threadIdx.x; r < r_end; r += kThreads) {
    const uint64_t p0 = a.row_ptr[bs + r], p1 = a.row_ptr[bs + r + 1];
    const uint64_t fan = p1 - p0;
    const uint64_t rs = (kMode == kModeMatrix ? P(p1) - P(p0) : P(a.row_pos[bs + r + 1]) - P(a.row_pos[bs + r])) &
                        kValMask;
    mfan = fan > mfan ? fan : mfan;
    mrow = rs > mrow ? rs : mrow;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mlink = warp_max(mlink);
  mfan = warp_max(mfan);
  mrow = warp_max(mrow);
  if (lane == 0) {
    s_red[0][warp] = mlink;
    s_red[1][warp] = mfan;
    s_red[2][warp] = mrow;
  }
  __syncthreads();
  uint32_t* gh = a.col_hist + (size_t)s * kColPasses * kRadix;
  for (int i = threadIdx.x; i < kColPasses * kRadix; i += kThreads) {
    const uint32_t c = s_h[i];
    if (c) atomicAdd(&gh[i], c);
  }
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) {
      mlink = umax64(mlink, s_red[0][w]);
      mfan = umax64(mfan, s_red[1][w]);
      mrow = umax64(mrow, s_red[2][w]);
    }
    ans_quantities* q = a.q + s;
    if (mlink) atomicMax((unsigned long long*)&q->max_link_packets, (unsigned long long)mlink);
    if (mfan) atomicMax((unsigned long long*)&q->max_source_fanout, (unsigned long long)mfan);
    if (mrow) atomicMax((unsigned long long*)&q->max_source_packets, (unsigned long long)mrow);
    if (tl.j == 0) {
      const uint64_t total = kMode == kModeMatrix ? P(nnz) : P(a.run_start[bs + nnz]);
      q->valid_packets = total;
      q->unique_links = nnz;
      q->unique_sources = nrows;
    }
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

// Column runs inside one tile of destination-sorted (dst, count) pairs.
// Each thread scans 16 consecutive pairs; a run that crosses thread chunks is
// completed by the thread holding its successor head, from a segmented scan
// over the chunks.  Runs that cross the tile boundary are summarised in
// bnd[t] (leading part, trailing part) for k_colstat_fin.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_colstat(SegPlan p, const uint32_t* __restrict__ keys,
                                                      const V* __restrict__ vals,
                                                      ColBnd* __restrict__ bnd, ans_quantities* q) {
  __shared__ Tile s_tile;
  __shared__ uint64_t s_ll[kThreads], s_ls[kThreads], s_tl[kThreads], s_ts[kThreads];
  __shared__ uint32_t s_wf[kWarps];
  __shared__ uint64_t s_wl[kWarps], s_ws[kWarps];
  __shared__ uint64_t s_red[kWarps];
  __shared__ int s_first, s_last;
  const uint32_t t = blockIdx.x;
  const Tile tl = block_tile(p, t, &s_tile);
  if (tl.count == 0) return;
  const uint64_t g0 = tl.base + tl.start;
  const uint32_t i0 = threadIdx.x * kPerThread;
  const uint32_t n = i0 < tl.count ? min((uint32_t)kPerThread, tl.count - i0) : 0u;
  uint64_t lead_len = 0, lead_sum = 0, cur_len = 0, cur_sum = 0, mlen = 0, msum = 0;
  uint32_t heads = 0;
  bool has_head = false;
  if (n > 0) {
    bool has_prev = (tl.start + i0) > 0;
    uint32_t prev = has_prev ? keys[g0 + i0 - 1] : 0u;
    for (uint32_t e = 0; e < n; ++e) {
      const uint32_t k = keys[g0 + i0 + e];
      const uint64_t v = vals[g0 + i0 + e];
      const bool head = !has_prev || k != prev;
      has_prev = true;
      prev = k;
      if (head) {
        if (has_head) {
          mlen = umax64(mlen, cur_len);
          msum = umax64(msum, cur_sum);
        } else {
          lead_len = cur_len;
          lead_sum = cur_sum;
        }
        has_head = true;
        ++heads;
        cur_len = 1;
        cur_sum = v;
      } else {
        ++cur_len;
        cur_sum += v;
      }
    }
    if (!has_head) {
      lead_len = cur_len;
      lead_sum = cur_sum;
      cur_len = 0;
      cur_sum = 0;
    }
  }
  s_ll[threadIdx.x] = lead_len;
  s_ls[threadIdx.x] = lead_sum;
  s_tl[threadIdx.x] = cur_len;
  s_ts[threadIdx.x] = cur_sum;
  if (threadIdx.x == 0) {
    s_first = kThreads;
    s_last = -1;
  }
  __syncthreads();
  if (has_head) {
    atomicMin(&s_first, (int)threadIdx.x);
    atomicMax(&s_last, (int)threadIdx.x);
  }
  // The run that ends just before this chunk's first head began at the last
  // head of an earlier chunk: a segmented exclusive scan over the chunks of
  // (has a head, its tail if so else the whole chunk) gives its length and
  // sum up to this chunk (operator: (f1, v1) + (f2, v2) = (f1 | f2, f2 ? v2 :
  // v1 + v2)), warp by warp with shuffles, then across warps.
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool f = has_head;
    uint64_t vl = has_head ? cur_len : lead_len, vs = has_head ? cur_sum : lead_sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const bool pf = __shfl_up_sync(0xffffffffu, f, o);
      const uint64_t pl = __shfl_up_sync(0xffffffffu, vl, o), ps = __shfl_up_sync(0xffffffffu, vs, o);
      if (lane >= o) {
        if (!f) {
          vl += pl;
          vs += ps;
        }
        f = f || pf;
      }
    }
    // exclusive within the warp
    bool xf = __shfl_up_sync(0xffffffffu, f, 1);
    uint64_t xl = __shfl_up_sync(0xffffffffu, vl, 1), xs = __shfl_up_sync(0xffffffffu, vs, 1);
    if (lane == 0) {
      xf = false;
      xl = xs = 0;
    }
    if (lane == 31) {
      s_wf[warp] = f ? 1u : 0u;
      s_wl[warp] = vl;
      s_ws[warp] = vs;
    }
    __syncthreads();
    // prefix of the earlier warps
    bool pf = false;
    uint64_t pl = 0, ps = 0;
    for (int w = 0; w < warp; ++w) {
      if (s_wf[w]) {
        pl = s_wl[w];
        ps = s_ws[w];
      } else {
        pl += s_wl[w];
        ps += s_ws[w];
      }
      pf = pf || s_wf[w];
    }
    if (xf) {
      pl = xl;
      ps = xs;
    } else {
      pl += xl;
      ps += xs;
    }
    pf = pf || xf;
    if (has_head && pf) {  // it began inside this tile; otherwise it is the tile's leading run
      mlen = umax64(mlen, pl + lead_len);
      msum = umax64(msum, ps + lead_sum);
    }
  }
  __syncthreads();
  const int hf = s_first, hl = s_last;
  const int me = (int)threadIdx.x;
  // Leading run of the tile: chunks up to (and including the lead of) the first head.
  const uint64_t pl = me <= hf ? s_ll[me] : 0ull, ps = me <= hf ? s_ls[me] : 0ull;
  // Trailing run: the last head's run plus the headless chunks after it.
  const uint64_t ql = hl < 0 ? 0ull : (me == hl ? s_tl[me] : (me > hl ? s_ll[me] : 0ull));
  const uint64_t qs = hl < 0 ? 0ull : (me == hl ? s_ts[me] : (me > hl ? s_ls[me] : 0ull));
  const uint64_t lead_l = block_sum(pl, s_red);
  const uint64_t lead_s = block_sum(ps, s_red);
  const uint64_t tail_l = block_sum(ql, s_red);
  const uint64_t tail_s = block_sum(qs, s_red);
  const uint64_t nheads = block_sum((uint64_t)heads, s_red);
  mlen = warp_max(mlen);
  msum = warp_max(msum);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s_ll[threadIdx.x >> 5] = mlen;
    s_ls[threadIdx.x >> 5] = msum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) {
      mlen = umax64(mlen, s_ll[w]);
      msum = umax64(msum, s_ls[w]);
    }
    ColBnd b;
    b.lead_len = lead_l;
    b.lead_sum = lead_s;
    b.tail_len = tail_l;
    b.tail_sum = tail_s;
    b.has_head = hl >= 0 ? 1u : 0u;
    b.pad = 0;
    bnd[t] = b;
    ans_quantities* qq = q + tl.seg;
    if (nheads) atomicAdd((unsigned long long*)&qq->unique_destinations, (unsigned long long)nheads);
    if (mlen) atomicMax((unsigned long long*)&qq->max_destination_fanin, (unsigned long long)mlen);
    if (msum) atomicMax((unsigned long long*)&qq->max_destination_packets, (unsigned long long)msum);
  }
}

// Complete the column runs that cross tile boundaries: the run ending just
// before a tile's first head, and the run ending at the segment's end.
__global__ void k_colstat_fin(SegPlan p, const ColBnd* __restrict__ bnd, ans_quantities* q) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.ntiles) return;
  const Tile tl = make_tile(p, t);
  if (tl.count == 0) return;
  const ColBnd b = bnd[t];
  const uint32_t first = t - tl.j;
  uint64_t mlen = 0, msum = 0;
  auto walk_back = [&](uint64_t L, uint64_t S) {
    for (uint32_t u = t; u > first;) {
      --u;
      const ColBnd c = bnd[u];
      if (c.has_head) {
        L += c.tail_len;
        S += c.tail_sum;
        break;
      }
      L += c.lead_len;
      S += c.lead_sum;
    }
    mlen = umax64(mlen, L);
    msum = umax64(msum, S);
  };
  if (b.has_head && tl.j > 0) walk_back(b.lead_len, b.lead_sum);
  if (tl.start + tl.count == tl.len) {
    if (b.has_head) {
      mlen = umax64(mlen, b.tail_len);
      msum = umax64(msum, b.tail_sum);
    } else {
      walk_back(b.lead_len, b.lead_sum);
    }
  }
  ans_quantities* qq = q + tl.seg;
  if (mlen) atomicMax((unsigned long long*)&qq->max_destination_fanin, (unsigned long long)mlen);
  if (msum) atomicMax((unsigned long long*)&qq->max_destination_packets, (unsigned long long)msum);
}

// Segments that own no tile (length 0 known on the host).
__global__ void k_empty_fixup(StatsArgs a) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.plan.nseg) return;
  if (a.plan.first_tile[s] != a.plan.first_tile[s + 1]) return;
  const uint64_t bs = a.plan.base[s] + s;
  a.row_ptr[bs] = 0;
  if (a.run_start) a.run_start[bs] = 0;
  if (a.row_pos) a.row_pos[bs] = 0;
  a.hdr[2 * s] = 0;
  a.hdr[2 * s + 1] = 0;
  if (a.ulen) a.ulen[s] = 0;
}

__global__ void k_tile_seg(SegPlan p, uint32_t* __restrict__ out) {
  p.tile_seg = nullptr;  // search first_tile
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < p.ntiles; t += gridDim.x * blockDim.x)
    out[t] = find_seg(p, t);
}

// Warp 0 waits with warp_lookback, thread 32 with lookback, both for tile 0
// of a chain that nobody publishes; both give up at the poll limit.
__global__ void k_wait_probe(const uint64_t* st, uint32_t* err) {
  if (threadIdx.x < 32) {
    warp_lookback(st, 1, 0, 1, err);
  } else if (threadIdx.x == 32) {
    lookback(st, 1, 0, 1, err);
  }
}

// Zero `bytes` bytes at p (4-byte aligned): a kernel instead of a memset so
// that a recorded launch sequence keeps its topology when sizes change.
__global__ void k_zero(uint32_t* __restrict__ p, size_t words, uint8_t* __restrict__ tail, uint32_t ntail) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) p[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

// Canonical-DCSR check of an imported matrix (Sec. IV-B containers; rows
// ascending, every stored row nonempty, columns ascending within a row, no
// stored zero).  Sets bits of *bad: 1 row_ptr does not run from 0 to nnz,
// 2 a row is empty or row_ptr decreases, 4 row ids not strictly ascending,
// 8 a zero value, 16 columns not strictly ascending within a row.
__global__ void k_check_dcsr(uint64_t nrows, uint64_t nnz, const uint32_t* __restrict__ row_ids,
                             const uint64_t* __restrict__ row_ptr, const uint32_t* __restrict__ col_ids,
                             const uint64_t* __restrict__ vals, uint32_t* bad) {
  const uint64_t n = nrows + 1 > nnz ? nrows + 1 : nnz;
  uint32_t f = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (i == 0 && (row_ptr[0] != 0 || row_ptr[nrows] != nnz)) f |= 1u;
    if (i < nrows) {
      if (row_ptr[i] >= row_ptr[i + 1]) f |= 2u;
      if (i + 1 < nrows && row_ids[i] >= row_ids[i + 1]) f |= 4u;
    }
    if (i < nnz) {
      if (vals[i] == 0) f |= 8u;
      if (i + 1 < nnz && col_ids[i] >= col_ids[i + 1]) {  // then i + 1 must start a row
        uint64_t lo = 0, hi = nrows + 1;                    // first r with row_ptr[r] >= i + 1
        while (lo < hi) {
          const uint64_t mid = (lo + hi) >> 1;
          if (row_ptr[mid] < i + 1) lo = mid + 1; else hi = mid;
        }
        if (lo > nrows || row_ptr[lo] != i + 1) f |= 16u;
      }
    }
  }
  if (f) atomicOr(bad, f);
}

__global__ void k_nonzero_flags(SegPlan p, const uint64_t* __restrict__ vals, uint64_t* __restrict__ flags,
                                uint32_t* err) {
  const uint64_t n = p.len[0];
  uint32_t bad = 0;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = vals[p.base[0] + u];
    flags[p.base[0] + u] = v != 0 ? 1ull : 0ull;
    if (v >> 61) bad = 1;  // prefixes run mod 2^62: a negative count lands at or above 2^61
  }
  if (bad) atomicOr(err, (uint32_t)kErrNegative);
}

__global__ void k_scatter_nonzero(SegPlan p, const uint64_t* __restrict__ kin, const uint64_t* __restrict__ vin,
                                  const uint64_t* __restrict__ pos, uint64_t* __restrict__ kout,
                                  uint64_t* __restrict__ vout, uint64_t* count) {
  const uint64_t n = p.len[0];
  const uint64_t b = p.base[0];  // pos is an exclusive prefix at base + seg (seg 0)
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[b + n];
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = vin[b + u];
    if (v != 0) {
      const uint64_t o = pos[b + u];
      kout[b + o] = kin[b + u];
      vout[b + o] = v;
    }
  }
}

// ---- window column statistics by a shared-memory hash of destinations -----
//
// One CTA per window counts, per distinct destination, its links (fan-in)
// and their packets (destination packets) in a shared-memory open-addressing
// table, then reduces the table to the three column quantities (Table I;
// Sec. IV-C).  This replaces the four column-sort passes for every window
// whose distinct destinations fit the table: once the table passes three
// quarters full the CTA gives up and leaves the window to the sort; a window
// it finished gets ulen = 0, so the column sort and its run reduction skip it.

constexpr int kColHashThreads = 1024;
constexpr uint32_t kColHashSlots = 1u << 14;                 // 16384
constexpr uint32_t kColHashMaxFill = kColHashSlots / 4 * 3;  // give up above this
constexpr size_t kColHashSmem = (size_t)kColHashSlots * 12;  // key, links, packets (uint32 each)
constexpr uint32_t kColEmpty = 0xFFFFFFFFu;                  // empty slot (that destination is counted apart)

__global__ void __launch_bounds__(kColHashThreads, 1) k_colhash(SegPlan p, uint64_t* __restrict__ ulen,
                                                                 const uint32_t* __restrict__ col_ids,
                                                                 const uint32_t* __restrict__ vals32,
                                                                 ans_quantities* __restrict__ q) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_cnt = sm + kColHashSlots;
  uint32_t* t_sum = sm + 2 * kColHashSlots;
  __shared__ uint32_t s_fill, s_over, s_spec_cnt, s_spec_sum;
  __shared__ unsigned long long s_red[3][kColHashThreads / 32];
  const uint32_t s = blockIdx.x;
  if (s >= p.nseg) return;
  const uint64_t n = ulen[s];
  const uint64_t b = p.base[s];
  for (uint32_t i = threadIdx.x; i < kColHashSlots; i += kColHashThreads) {
    t_key[i] = kColEmpty;
    t_cnt[i] = 0;
    t_sum[i] = 0;
  }
  if (threadIdx.x == 0) s_fill = s_over = s_spec_cnt = s_spec_sum = 0;
  __syncthreads();
  for (uint64_t u = threadIdx.x; u < n; u += kColHashThreads) {
    if (*(volatile uint32_t*)&s_over) break;
    const uint32_t d = col_ids[b + u];
    const uint32_t v = vals32[b + u];
    if (d == kColEmpty) {
      atomicAdd(&s_spec_cnt, 1u);
      atomicAdd(&s_spec_sum, v);
      continue;
    }
    uint32_t h = fmix32(d) & (kColHashSlots - 1);
    for (uint32_t probe = 0; probe < kColHashSlots; ++probe) {
      uint32_t cur = *(volatile uint32_t*)&t_key[h];
      if (cur == kColEmpty) {
        cur = atomicCAS(&t_key[h], kColEmpty, d);
        if (cur == kColEmpty) {
          cur = d;
          if (atomicAdd(&s_fill, 1u) + 1 > kColHashMaxFill) s_over = 1;
        }
      }
      if (cur == d) {
        atomicAdd(&t_cnt[h], 1u);
        atomicAdd(&t_sum[h], v);
        break;
      }
      h = (h + 1) & (kColHashSlots - 1);
    }
  }
  __syncthreads();
  if (s_over) return;  // the column sort takes this window
  unsigned long long c = 0, mcnt = 0, msum = 0;
  for (uint32_t i = threadIdx.x; i < kColHashSlots; i += kColHashThreads) {
    if (t_key[i] != kColEmpty) {
      ++c;
      mcnt = t_cnt[i] > mcnt ? t_cnt[i] : mcnt;
      msum = t_sum[i] > msum ? t_sum[i] : msum;
    }
  }
  c = warp_sum(c);
  mcnt = warp_max(mcnt);
  msum = warp_max(msum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_red[0][warp] = c;
    s_red[1][warp] = mcnt;
    s_red[2][warp] = msum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c = 0;
    mcnt = msum = 0;
    for (int w = 0; w < kColHashThreads / 32; ++w) {
      c += s_red[0][w];
      mcnt = s_red[1][w] > mcnt ? s_red[1][w] : mcnt;
      msum = s_red[2][w] > msum ? s_red[2][w] : msum;
    }
    if (s_spec_cnt) {
      ++c;
      mcnt = s_spec_cnt > mcnt ? s_spec_cnt : mcnt;
      msum = s_spec_sum > msum ? s_spec_sum : msum;
    }
    q[s].unique_destinations = c;
    q[s].max_destination_fanin = mcnt;
    q[s].max_destination_packets = msum;
    ulen[s] = 0;  // done: the column sort skips this window
  }
}

// The same statistics with one cluster of C CTAs per window (launched with
// clusters along x; cluster i takes window i; C a power of two): CTA r
// counts links [r, r + 1) * ceil(n / C) of the window in its own table;
// then, in log2(C) rounds, CTA r pulls the table of CTA r + 2^k (for r a
// multiple of 2^(k+1)) over distributed shared memory and adds it into its
// own, so CTA 0 ends with the window's table and reduces it.  A table that
// passes kColHashMaxFill -- its own links, or a pulled table -- marks its CTA
// overflowing, and the mark travels with the pulls: the window gives up
// (ulen kept) exactly when it has more distinct destinations than that.
// Every CTA of a cluster passes the same cluster barriers.
__global__ void __launch_bounds__(kColHashThreads, 1) k_colhash_cl(SegPlan p, uint64_t* __restrict__ ulen,
                                                                    const uint32_t* __restrict__ col_ids,
                                                                    const uint32_t* __restrict__ vals32,
                                                                    ans_quantities* __restrict__ q) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_cnt = sm + kColHashSlots;
  uint32_t* t_sum = sm + 2 * kColHashSlots;
  __shared__ uint32_t s_fill, s_over, s_spec_cnt, s_spec_sum;
  __shared__ unsigned long long s_red[3][kColHashThreads / 32];
  const uint32_t me = cta_rank(), nc = cluster_nctarank();
  const uint32_t s = cluster_id();
  // A launch whose grid is not one cluster per window (the same for every
  // CTA, so all leave before any cluster barrier) counts nothing: its
  // windows keep their ulen and the column sort takes them.
  if (gridDim.x != p.nseg * nc || gridDim.y != 1 || gridDim.z != 1) return;
  const uint64_t n = s < p.nseg ? ulen[s] : 0;
  const uint64_t b = s < p.nseg ? p.base[s] : 0;
  for (uint32_t i = threadIdx.x; i < kColHashSlots; i += kColHashThreads) {
    t_key[i] = kColEmpty;
    t_cnt[i] = 0;
    t_sum[i] = 0;
  }
  if (threadIdx.x == 0) s_fill = s_over = s_spec_cnt = s_spec_sum = 0;
  __syncthreads();
  // Adds (d, c links, v packets) to this CTA's table.
  auto insert = [&](uint32_t d, uint32_t c, uint32_t v) {
    uint32_t h = fmix32(d) & (kColHashSlots - 1);
    for (uint32_t probe = 0; probe < kColHashSlots; ++probe) {
      uint32_t cur = *(volatile uint32_t*)&t_key[h];
      if (cur == kColEmpty) {
        cur = atomicCAS(&t_key[h], kColEmpty, d);
        if (cur == kColEmpty) {
          cur = d;
          if (atomicAdd(&s_fill, 1u) + 1 > kColHashMaxFill) s_over = 1;
        }
      }
      if (cur == d) {
        atomicAdd(&t_cnt[h], c);
        atomicAdd(&t_sum[h], v);
        return;
      }
      h = (h + 1) & (kColHashSlots - 1);
    }
  };
  const uint64_t chunk = (n + nc - 1) / nc;
  const uint64_t lo = umin64((uint64_t)me * chunk, n), hi = umin64(lo + chunk, n);
  for (uint64_t u = lo + threadIdx.x; u < hi; u += kColHashThreads) {
    if (*(volatile uint32_t*)&s_over) break;
    const uint32_t d = col_ids[b + u];
    const uint32_t v = vals32[b + u];
    if (d == kColEmpty) {
      atomicAdd(&s_spec_cnt, 1u);
      atomicAdd(&s_spec_sum, v);
      continue;
    }
    insert(d, 1u, v);
  }
  cluster_sync();  // every local table is complete
  for (uint32_t step = 1; step < nc; step <<= 1) {
    if ((me & (2 * step - 1)) == 0 && me + step < nc) {
      const uint32_t r = me + step;
      const uint32_t key_r = map_rank(smem_addr(t_key), r), cnt_r = map_rank(smem_addr(t_cnt), r),
                     sum_r = map_rank(smem_addr(t_sum), r);
      if (ld_cluster(map_rank(smem_addr(&s_over), r)) != 0) {
        if (threadIdx.x == 0) s_over = 1;
      } else {
        constexpr int kU = 4;  // slots read per round trip
        for (uint32_t i0 = threadIdx.x; i0 < kColHashSlots; i0 += kU * kColHashThreads) {
          if (*(volatile uint32_t*)&s_over) break;
          uint32_t d[kU];
#pragma unroll
          for (int j = 0; j < kU; ++j) d[j] = ld_cluster(key_r + 4 * (i0 + j * kColHashThreads));
#pragma unroll
          for (int j = 0; j < kU; ++j) {
            if (d[j] == kColEmpty) continue;
            const uint32_t i = i0 + j * kColHashThreads;
            insert(d[j], ld_cluster(cnt_r + 4 * i), ld_cluster(sum_r + 4 * i));
          }
        }
        if (threadIdx.x == 0) {
          s_spec_cnt += ld_cluster(map_rank(smem_addr(&s_spec_cnt), r));
          s_spec_sum += ld_cluster(map_rank(smem_addr(&s_spec_sum), r));
        }
      }
    }
    cluster_sync();  // this round's pulls are done: their sources are read no more
  }
  if (me != 0 || s_over || s >= p.nseg) return;  // an overflowing window is left to the column sort
  unsigned long long c = 0, mcnt = 0, msum = 0;
  for (uint32_t i = threadIdx.x; i < kColHashSlots; i += kColHashThreads) {
    if (t_key[i] != kColEmpty) {
      ++c;
      mcnt = t_cnt[i] > mcnt ? t_cnt[i] : mcnt;
      msum = t_sum[i] > msum ? t_sum[i] : msum;
    }
  }
  c = warp_sum(c);
  mcnt = warp_max(mcnt);
  msum = warp_max(msum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_red[0][warp] = c;
    s_red[1][warp] = mcnt;
    s_red[2][warp] = msum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c = 0;
    mcnt = msum = 0;
    for (int w = 0; w < kColHashThreads / 32; ++w) {
      c += s_red[0][w];
      mcnt = s_red[1][w] > mcnt ? s_red[1][w] : mcnt;
      msum = s_red[2][w] > msum ? s_red[2][w] : msum;
    }
    if (s_spec_cnt) {
      ++c;
      mcnt = s_spec_cnt > mcnt ? s_spec_cnt : mcnt;
      msum = s_spec_sum > msum ? s_spec_sum : msum;
    }
    q[s].unique_destinations = c;
    q[s].max_destination_fanin = mcnt;
    q[s].max_destination_packets = msum;
    ulen[s] = 0;  // done: the column sort skips this window
  }
}

// Windows with more destinations than one table holds: the destinations
// are split between up to kColParts partitions by a hash, and each
// partition's links are counted by its own CTA in its own shared-memory
// table.  A window of n links gets ceil(n / kColPartLinks) partitions (n
// bounds its distinct destinations).  First one CTA per window groups the
// window's links by partition (a counting pass and a scatter pass, both
// warp-aggregated); then CTA r of the window counts partition r's links.
// Partial results meet in a per-window accumulator; the last CTA of a
// window to finish writes the window's three quantities and marks it done
// (ulen = 0) -- unless some partition overflowed its table, in which case
// the window is left, untouched, to the column sort.
constexpr uint32_t kColParts = 32;
constexpr uint32_t kColPartLinks = 8192;
constexpr int kSplitThreads = 1024;
constexpr int kSplitUnroll = 4;

// Finalizer-derived partition of a destination: the high bits of its mix
// (the table slot uses the low bits), scaled to [0, parts).
__device__ __forceinline__ uint32_t col_part(uint32_t d, uint32_t parts) {
  return (uint32_t)(((uint64_t)(fmix32(d) >> 14) * parts) >> 18);
}

// Partitions of window s of n links, or 0 if the partitioned hash does not
// take it (empty, finished, within one table, too large, or an index past
// the 2^27 windows whose (window, partition) items fit 32 bits).
__device__ __forceinline__ uint32_t col_parts_of(uint64_t n, uint32_t s) {
  const uint64_t parts = (n + kColPartLinks - 1) / kColPartLinks;
  return parts >= 2 && parts <= kColParts && s < (1u << 27) ? (uint32_t)parts : 0u;
}

// One CTA per window: the window's (destination, count) links regrouped by
// partition into okeys/ovals at the window's base; the partition starts in
// bstart[s][0..parts]; the window's (window, partition) items s * 32 + r
// appended to `items` (their count in work->count).
__global__ void __launch_bounds__(kSplitThreads, 2) k_colpart_split(SegPlan p, const uint64_t* __restrict__ ulen,
                                                                    const uint32_t* __restrict__ col_ids,
                                                                    const uint32_t* __restrict__ vals32,
                                                                    uint32_t* __restrict__ okeys,
                                                                    uint32_t* __restrict__ ovals,
                                                                    uint32_t* __restrict__ bstart,
                                                                    ColPartAcc* __restrict__ work,
                                                                    uint32_t* __restrict__ items) {
  __shared__ uint32_t s_cnt[kColParts], s_cur[kColParts];
  const uint32_t s = blockIdx.x;
  if (s >= p.nseg) return;
  const uint64_t n = ulen[s];
  const uint32_t parts = col_parts_of(n, s);
  if (!parts) return;
  const uint64_t b = p.base[s];
  const uint32_t* ci = col_ids + b;
  const uint32_t* vi = vals32 + b;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kColParts) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  // pass 1: links per partition
  for (uint64_t w0 = threadIdx.x & ~31u; w0 < n; w0 += (uint64_t)kSplitUnroll * kSplitThreads) {
    const uint64_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint32_t d[kSplitUnroll];
#pragma unroll
    for (int k = 0; k < kSplitUnroll; ++k) {
      const uint64_t u = u0 + (uint64_t)k * kSplitThreads;
      d[k] = u < n ? ci[u] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kSplitUnroll; ++k) {
      const bool valid = u0 + (uint64_t)k * kSplitThreads < n;
      const uint32_t pt = valid ? col_part(d[k], parts) : kColParts;
      const uint32_t peers = __match_any_sync(0xffffffffu, pt);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[pt], __popc(peers));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t r = 0; r < parts; ++r) {
      s_cur[r] = run;
      bstart[(uint64_t)s * (kColParts + 1) + r] = run;
      run += s_cnt[r];
    }
    bstart[(uint64_t)s * (kColParts + 1) + parts] = run;
    const uint32_t first = (uint32_t)atomicAdd(&work->count, (unsigned long long)parts);
    for (uint32_t r = 0; r < parts; ++r) items[first + r] = s * kColParts + r;
  }
  __syncthreads();
  // pass 2: scatter each link to its partition (order within a partition is free)
  uint32_t* ko = okeys + b;
  uint32_t* vo = ovals + b;
  for (uint64_t w0 = threadIdx.x & ~31u; w0 < n; w0 += (uint64_t)kSplitUnroll * kSplitThreads) {
    const uint64_t u0 = w0 + (threadIdx.x & 31);  // the loop bound is the same for the whole warp
    uint32_t d[kSplitUnroll], v[kSplitUnroll];
#pragma unroll
    for (int k = 0; k < kSplitUnroll; ++k) {
      const uint64_t u = u0 + (uint64_t)k * kSplitThreads;
      d[k] = u < n ? ci[u] : 0u;
      v[k] = u < n ? vi[u] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kSplitUnroll; ++k) {
      const bool valid = u0 + (uint64_t)k * kSplitThreads < n;
      const uint32_t pt = valid ? col_part(d[k], parts) : kColParts;
      const uint32_t peers = __match_any_sync(0xffffffffu, pt);
      const int leader = __ffs(peers) - 1;
      uint32_t pos = 0;
      if (valid && lane == leader) pos = atomicAdd(&s_cur[pt], __popc(peers));
      pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & lanemask_lt());
      if (valid) {
        ko[pos] = d[k];
        vo[pos] = v[k];
      }
    }
  }
}

// Partitions counted by persistent CTAs (one per SM: the table takes the
// SM's shared memory), each taking the next (window s, partition r) item
// that k_colpart_split listed and counting partition r's links.  The links
// are read in chunks of kColPartChunk per thread, the first chunk's loads
// issued before the table is cleared; the table's fill is counted once per
// warp.
constexpr int kColPartChunk = 8;
__global__ void __launch_bounds__(kColHashThreads, 1) k_colhash_part(SegPlan p, uint64_t* __restrict__ ulen,
                                                                      const uint32_t* __restrict__ pkeys,
                                                                      const uint32_t* __restrict__ pvals,
                                                                      const uint32_t* __restrict__ bstart,
                                                                      ColPartAcc* __restrict__ acc,
                                                                      const uint32_t* __restrict__ items,
                                                                      ans_quantities* __restrict__ q) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_cnt = sm + kColHashSlots;
  uint32_t* t_sum = sm + 2 * kColHashSlots;
  __shared__ uint32_t s_fill, s_over, s_spec_cnt, s_spec_sum, s_last, s_item;
  __shared__ unsigned long long s_red[3][kColHashThreads / 32];
  ColPartAcc* work = acc + p.nseg;
  const uint32_t nitems = (uint32_t)work->count;  // written by k_colpart_split
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t i = atomicAdd(&work->done, 1u);
      s_item = i < nitems ? items[i] : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item == 0xFFFFFFFFu) break;
    const uint32_t s = item / kColParts, r = item % kColParts;
    const uint32_t parts = col_parts_of(ulen[s], s);
    const uint64_t b = p.base[s];
    const uint32_t lo = bstart[(uint64_t)s * (kColParts + 1) + r], hi = bstart[(uint64_t)s * (kColParts + 1) + r + 1];
    const uint32_t* pk = pkeys + b;
    const uint32_t* pv = pvals + b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t d[kColPartChunk], v[kColPartChunk];
    auto load = [&](uint32_t u0) {
#pragma unroll
      for (int j = 0; j < kColPartChunk; ++j) {
        const uint32_t u = u0 + (uint32_t)j * kColHashThreads + threadIdx.x;
        d[j] = u < hi ? __ldg(pk + u) : 0u;
        v[j] = u < hi ? __ldg(pv + u) : 0u;
      }
    };
    load(lo);
    {
      uint4* k4 = reinterpret_cast<uint4*>(t_key);
      uint4* c4 = reinterpret_cast<uint4*>(t_cnt);  // t_cnt and t_sum, back to back
      const uint4 empty = make_uint4(kColEmpty, kColEmpty, kColEmpty, kColEmpty), zero = make_uint4(0, 0, 0, 0);
      for (uint32_t i = threadIdx.x; i < kColHashSlots / 4; i += kColHashThreads) k4[i] = empty;
      for (uint32_t i = threadIdx.x; i < kColHashSlots / 2; i += kColHashThreads) c4[i] = zero;
    }
    if (threadIdx.x == 0) s_fill = s_over = s_spec_cnt = s_spec_sum = 0;
    __syncthreads();
    constexpr uint32_t kStep = (uint32_t)kColPartChunk * kColHashThreads;
    for (uint32_t u0 = lo; u0 < hi; u0 += kStep) {  // the same trip count for every thread
      if (u0 != lo) load(u0);
      if (__any_sync(0xffffffffu, *(volatile uint32_t*)&s_over != 0)) break;  // warp-uniform
#pragma unroll
      for (int j = 0; j < kColPartChunk; ++j) {
        const uint32_t u = u0 + (uint32_t)j * kColHashThreads + threadIdx.x;
        bool claimed = false;
        if (u < hi) {
          if (d[j] == kColEmpty) {
            atomicAdd(&s_spec_cnt, 1u);
            atomicAdd(&s_spec_sum, v[j]);
          } else {
            uint32_t h = fmix32(d[j]) & (kColHashSlots - 1);
            for (uint32_t probe = 0; probe < kColHashSlots; ++probe) {
              uint32_t cur = *(volatile uint32_t*)&t_key[h];
              if (cur == kColEmpty) {
                cur = atomicCAS(&t_key[h], kColEmpty, d[j]);
                if (cur == kColEmpty) {
                  cur = d[j];
                  claimed = true;
                }
              }
              if (cur == d[j]) {
                atomicAdd(&t_cnt[h], 1u);
                atomicAdd(&t_sum[h], v[j]);
                break;
              }
              h = (h + 1) & (kColHashSlots - 1);
            }
          }
        }
        // new slots counted once per warp; past three quarters the table gives
        // up (at most one slot per thread more can still be claimed meanwhile)
        const uint32_t nc = __popc(__ballot_sync(0xffffffffu, claimed));
        if (lane == 0 && nc && atomicAdd(&s_fill, nc) + nc > kColHashMaxFill) s_over = 1;
      }
    }
    __syncthreads();
    ColPartAcc* a = acc + s;
    if (!s_over) {
      unsigned long long c = 0, mcnt = 0, msum = 0;
      for (uint32_t i = threadIdx.x; i < kColHashSlots; i += kColHashThreads) {
        if (t_key[i] != kColEmpty) {
          ++c;
          mcnt = t_cnt[i] > mcnt ? t_cnt[i] : mcnt;
          msum = t_sum[i] > msum ? t_sum[i] : msum;
        }
      }
      c = warp_sum(c);
      mcnt = warp_max(mcnt);
      msum = warp_max(msum);
      if (lane == 0) {
        s_red[0][warp] = c;
        s_red[1][warp] = mcnt;
        s_red[2][warp] = msum;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        c = 0;
        mcnt = msum = 0;
        for (int w = 0; w < kColHashThreads / 32; ++w) {
          c += s_red[0][w];
          mcnt = s_red[1][w] > mcnt ? s_red[1][w] : mcnt;
          msum = s_red[2][w] > msum ? s_red[2][w] : msum;
        }
        if (s_spec_cnt) {
          ++c;
          mcnt = s_spec_cnt > mcnt ? s_spec_cnt : mcnt;
          msum = s_spec_sum > msum ? s_spec_sum : msum;
        }
        if (c) atomicAdd(&a->count, c);
        if (mcnt) atomicMax(&a->max_fanin, mcnt);
        if (msum) atomicMax(&a->max_packets, msum);
      }
    } else if (threadIdx.x == 0) {
      atomicOr(&a->fail, 1u);
    }
    // The last partition of the window to arrive publishes the result.
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&a->done, 1u) == parts - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_last) {
      __threadfence();
      const volatile ColPartAcc* va = a;
      if (va->fail == 0) {
        q[s].unique_destinations = va->count;
        q[s].max_destination_fanin = va->max_fanin;
        q[s].max_destination_packets = va->max_packets;
        ulen[s] = 0;  // done: the column sort skips this window
      }
    }
    __syncthreads();  // the table and the shared words are reused by the next item
  }
}

// ---- column statistics of one large segment (a time sum) by hash groups ---
//
// The column statistics only need equal destinations grouped, in any order,
// and h = fmix32(dst) is a bijection: after the first two column passes over
// h (its low 16 bits), the links form 2^16 groups of equal h & 0xffff, each
// holding every link of its destinations.  Each group's distinct h (= its
// destinations) are counted in a shared-memory table by persistent CTAs and
// the three column quantities reduced into an accumulator.  A group of more
// than kHGroupPartLinks links (a heavily linked destination lands all its
// links in one group) is cut into parts counted by different CTAs, whose
// tables are written out and merged per group afterwards.  If every table
// fits, the last CTA publishes the quantities and sets the segment's length
// to 0, so the two remaining column passes and the run reduction find
// nothing to do; otherwise they complete the sort by h and count the runs.
constexpr int kHGroupThreads = 512;
constexpr uint32_t kHGroupSlots = 1u << 13;                   // 8192
constexpr uint32_t kHGroupMaxFill = kHGroupSlots / 4 * 3;     // give up above this
constexpr size_t kHGroupSmem = (size_t)kHGroupSlots * 12;     // key, links, packets
constexpr int kHGroupChunk = 8;
constexpr uint32_t kHNone = 0xFFFFFFFFu;
static_assert(kHGroupPartWords == 3 * (kHGroupMaxFill + 1), "a part's entries: its table's fill and the key apart");

// bnd[g] = first position of group g (g in [0, 2^16]; bnd[2^16] = n) in the
// n = *len keys sorted by their low 16 bits.
__global__ void __launch_bounds__(256) k_hgroup_bounds(const uint32_t* __restrict__ keys, const uint64_t* len,
                                                       uint32_t* __restrict__ bnd) {
  const uint64_t n = *len;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t prev = i == 0 ? -1 : (int64_t)(keys[i - 1] & 0xFFFFu);
    const int64_t cur = i == n ? (int64_t)kHGroups : (int64_t)(keys[i] & 0xFFFFu);
    for (int64_t g = prev + 1; g <= cur; ++g) bnd[g] = (uint32_t)i;
  }
}

// One CTA: the work items (one per group, ceil(links / kHGroupPartLinks) per
// group above that), their exclusive prefix item_start, the parts of the
// groups cut in parts (prefix hpart, list heavy) and the counts in meta
// {items, heavy groups, heavy parts}; too many heavy parts for the buffer
// fail the hash (the column sort then finishes the job).
__global__ void __launch_bounds__(1024) k_hgroup_plan(HGroupBufs b, uint32_t max_hparts) {
  constexpr uint32_t kPer = kHGroups / 1024;
  __shared__ uint32_t s_a[1024], s_b[1024], s_c[1024];
  const uint32_t g0 = threadIdx.x * kPer;
  uint32_t items = 0, hparts = 0, heavy = 0;
  for (uint32_t k = 0; k < kPer; ++k) {
    const uint32_t n = b.bnd[g0 + k + 1] - b.bnd[g0 + k];
    const uint32_t parts = n > kHGroupPartLinks ? (n + kHGroupPartLinks - 1) / kHGroupPartLinks : 1u;
    items += parts;
    if (parts > 1) {
      hparts += parts;
      ++heavy;
    }
  }
  s_a[threadIdx.x] = items;
  s_b[threadIdx.x] = hparts;
  s_c[threadIdx.x] = heavy;
  __syncthreads();
  for (uint32_t off = 1; off < 1024; off <<= 1) {  // inclusive scans (Hillis-Steele)
    const uint32_t a = threadIdx.x >= off ? s_a[threadIdx.x - off] : 0u;
    const uint32_t bb = threadIdx.x >= off ? s_b[threadIdx.x - off] : 0u;
    const uint32_t c = threadIdx.x >= off ? s_c[threadIdx.x - off] : 0u;
    __syncthreads();
    s_a[threadIdx.x] += a;
    s_b[threadIdx.x] += bb;
    s_c[threadIdx.x] += c;
    __syncthreads();
  }
  uint32_t ia = s_a[threadIdx.x] - items, ib = s_b[threadIdx.x] - hparts, ic = s_c[threadIdx.x] - heavy;
  for (uint32_t k = 0; k < kPer; ++k) {
    const uint32_t g = g0 + k;
    const uint32_t n = b.bnd[g + 1] - b.bnd[g];
    const uint32_t parts = n > kHGroupPartLinks ? (n + kHGroupPartLinks - 1) / kHGroupPartLinks : 1u;
    b.item_start[g] = ia;
    b.hpart[g] = ib;
    ia += parts;
    if (parts > 1) {
      b.heavy[ic++] = g;
      ib += parts;
    }
  }
  if (threadIdx.x == 1023) {
    b.item_start[kHGroups] = ia;
    b.hpart[kHGroups] = ib;
    b.meta[0] = ia;
    b.meta[1] = ic;
    b.meta[2] = ib;
    if (ib > max_hparts) atomicOr(&b.acc[0].fail, 1u);
  }
}

// Count (key, links, packets) into the group's table; true if this call took
// a new slot.  The fill stays below the table size (the callers give up at
// three quarters, and each thread takes at most one slot meanwhile), so a
// slot is always found.
__device__ __forceinline__ bool hg_insert(uint32_t* t_key, uint32_t* t_cnt, uint32_t* t_sum, uint32_t key,
                                          uint32_t cnt, uint32_t sum) {
  uint32_t h = (key >> 16) & (kHGroupSlots - 1);  // the group fixes the low 16 bits
  for (uint32_t probe = 0; probe < kHGroupSlots; ++probe) {
    uint32_t cur = *(volatile uint32_t*)&t_key[h];
    bool claimed = false;
    if (cur == kColEmpty) {
      cur = atomicCAS(&t_key[h], kColEmpty, key);
      if (cur == kColEmpty) {
        cur = key;
        claimed = true;
      }
    }
    if (cur == key) {
      atomicAdd(&t_cnt[h], cnt);
      atomicAdd(&t_sum[h], sum);
      return claimed;
    }
    h = (h + 1) & (kHGroupSlots - 1);
  }
  return false;
}

struct HGroupShared {
  uint32_t fill, over, spec_cnt, spec_sum, item, nflush;
  unsigned long long red[3][kHGroupThreads / 32];
};

__device__ __forceinline__ void hg_clear(uint32_t* t_key, HGroupShared& sh) {
  uint4* k4 = reinterpret_cast<uint4*>(t_key);
  uint4* c4 = reinterpret_cast<uint4*>(t_key + kHGroupSlots);  // t_cnt and t_sum, back to back
  const uint4 empty = make_uint4(kColEmpty, kColEmpty, kColEmpty, kColEmpty), zero = make_uint4(0, 0, 0, 0);
  for (uint32_t i = threadIdx.x; i < kHGroupSlots / 4; i += kHGroupThreads) k4[i] = empty;
  for (uint32_t i = threadIdx.x; i < kHGroupSlots / 2; i += kHGroupThreads) c4[i] = zero;
  if (threadIdx.x == 0) sh.fill = sh.over = sh.spec_cnt = sh.spec_sum = sh.nflush = 0;
}

// After an insert step of every thread of the warp: new slots counted once
// per warp; past three quarters the table gives up.
__device__ __forceinline__ void hg_count_fill(bool claimed, HGroupShared& sh) {
  const uint32_t nc = __popc(__ballot_sync(0xffffffffu, claimed));
  if ((threadIdx.x & 31) == 0 && nc && atomicAdd(&sh.fill, nc) + nc > kHGroupMaxFill) sh.over = 1;
}

// The table's (distinct keys, most links, most packets), the key counted
// apart included, added into acc (call with the whole CTA).
__device__ void hg_reduce(const uint32_t* t_key, const uint32_t* t_cnt, const uint32_t* t_sum, HGroupShared& sh,
                          ColPartAcc* acc) {
  unsigned long long c = 0, mcnt = 0, msum = 0;
  for (uint32_t i = threadIdx.x; i < kHGroupSlots; i += kHGroupThreads) {
    if (t_key[i] != kColEmpty) {
      ++c;
      mcnt = t_cnt[i] > mcnt ? t_cnt[i] : mcnt;
      msum = t_sum[i] > msum ? t_sum[i] : msum;
    }
  }
  c = warp_sum(c);
  mcnt = warp_max(mcnt);
  msum = warp_max(msum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh.red[0][warp] = c;
    sh.red[1][warp] = mcnt;
    sh.red[2][warp] = msum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    c = 0;
    mcnt = msum = 0;
    for (int w = 0; w < kHGroupThreads / 32; ++w) {
      c += sh.red[0][w];
      mcnt = sh.red[1][w] > mcnt ? sh.red[1][w] : mcnt;
      msum = sh.red[2][w] > msum ? sh.red[2][w] : msum;
    }
    if (sh.spec_cnt) {
      ++c;
      mcnt = sh.spec_cnt > mcnt ? sh.spec_cnt : mcnt;
      msum = sh.spec_sum > msum ? sh.spec_sum : msum;
    }
    if (c) atomicAdd(&acc->count, c);
    if (mcnt) atomicMax(&acc->max_fanin, mcnt);
    if (msum) atomicMax(&acc->max_packets, msum);
  }
}

// Persistent CTAs over the work items: item i is part k of group g.  A
// group in one part is reduced into acc[0] at once; a part of a cut group
// writes its table's entries (key, links, packets; the key counted apart as
// kColEmpty) to its region of hbuf and their number to hcnt.
__global__ void __launch_bounds__(kHGroupThreads, 2) k_hgroup_hash(const uint32_t* __restrict__ keys,
                                                                   const uint32_t* __restrict__ vals,
                                                                   HGroupBufs b) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_cnt = sm + kHGroupSlots;
  uint32_t* t_sum = sm + 2 * kHGroupSlots;
  __shared__ HGroupShared sh;
  const uint32_t nitems = b.meta[0];
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t i = atomicAdd(&b.acc[1].done, 1u);
      sh.item = i < nitems && *(volatile uint32_t*)&b.acc[0].fail == 0 ? i : kHNone;
    }
    __syncthreads();
    const uint32_t i = sh.item;
    if (i == kHNone) break;
    uint32_t lo_g = 0, hi_g = kHGroups;  // the group: the last g with item_start[g] <= i
    while (hi_g - lo_g > 1) {
      const uint32_t mid = (lo_g + hi_g) >> 1;
      if (b.item_start[mid] <= i) lo_g = mid; else hi_g = mid;
    }
    const uint32_t g = lo_g;
    const uint32_t parts = b.item_start[g + 1] - b.item_start[g], k = i - b.item_start[g];
    const uint32_t lo = b.bnd[g] + k * kHGroupPartLinks;
    const uint32_t hi = min(lo + kHGroupPartLinks, b.bnd[g + 1]);
    if (lo == hi) {  // an empty group (never cut in parts): nothing to count
      __syncthreads();
      continue;
    }
    uint32_t d[kHGroupChunk], v[kHGroupChunk];
    auto load = [&](uint32_t u0) {
#pragma unroll
      for (int j = 0; j < kHGroupChunk; ++j) {
        const uint32_t u = u0 + (uint32_t)j * kHGroupThreads + threadIdx.x;
        d[j] = u < hi ? __ldg(keys + u) : 0u;
        v[j] = u < hi ? __ldg(vals + u) : 0u;
      }
    };
    load(lo);
    hg_clear(t_key, sh);
    __syncthreads();
    constexpr uint32_t kStep = (uint32_t)kHGroupChunk * kHGroupThreads;
    for (uint32_t u0 = lo; u0 < hi; u0 += kStep) {  // the same trip count for every thread
      if (u0 != lo) load(u0);
      if (__any_sync(0xffffffffu, *(volatile uint32_t*)&sh.over != 0)) break;  // warp-uniform
#pragma unroll
      for (int j = 0; j < kHGroupChunk; ++j) {
        const uint32_t u = u0 + (uint32_t)j * kHGroupThreads + threadIdx.x;
        bool claimed = false;
        if (u < hi) {
          if (d[j] == kColEmpty) {  // the one destination whose mix is the empty marker
            atomicAdd(&sh.spec_cnt, 1u);
            atomicAdd(&sh.spec_sum, v[j]);
          } else {
            claimed = hg_insert(t_key, t_cnt, t_sum, d[j], 1u, v[j]);
          }
        }
        hg_count_fill(claimed, sh);
      }
    }
    __syncthreads();
    if (sh.over) {
      if (threadIdx.x == 0) atomicOr(&b.acc[0].fail, 1u);
    } else if (parts == 1) {
      hg_reduce(t_key, t_cnt, t_sum, sh, &b.acc[0]);
    } else {  // a part of a cut group: its entries out
      const uint64_t pidx = (uint64_t)b.hpart[g] + k;
      uint32_t* out = b.hbuf + pidx * kHGroupPartWords;
      for (uint32_t e = threadIdx.x; e < kHGroupSlots; e += kHGroupThreads) {
        if (t_key[e] != kColEmpty) {
          const uint32_t at = atomicAdd(&sh.nflush, 1u);
          out[3 * at] = t_key[e];
          out[3 * at + 1] = t_cnt[e];
          out[3 * at + 2] = t_sum[e];
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t n = sh.nflush;
        if (sh.spec_cnt) {
          out[3 * n] = kColEmpty;
          out[3 * n + 1] = sh.spec_cnt;
          out[3 * n + 2] = sh.spec_sum;
          ++n;
        }
        b.hcnt[pidx] = n;
      }
    }
    __syncthreads();  // the table and the shared words are reused by the next item
  }
}

// Persistent CTAs over the cut groups: each group's parts' entries merged in
// one table and reduced into acc[0].  The last CTA to finish publishes the
// segment's quantities unless a table overflowed.
__global__ void __launch_bounds__(kHGroupThreads, 2) k_hgroup_merge(HGroupBufs b, uint64_t* len,
                                                                    ans_quantities* __restrict__ q) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* t_key = sm;
  uint32_t* t_cnt = sm + kHGroupSlots;
  uint32_t* t_sum = sm + 2 * kHGroupSlots;
  __shared__ HGroupShared sh;
  const uint32_t nheavy = b.meta[1];
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t j = atomicAdd(&b.acc[2].done, 1u);
      sh.item = j < nheavy && *(volatile uint32_t*)&b.acc[0].fail == 0 ? b.heavy[j] : kHNone;
    }
    __syncthreads();
    const uint32_t g = sh.item;
    if (g == kHNone) break;
    const uint32_t parts = b.item_start[g + 1] - b.item_start[g];
    hg_clear(t_key, sh);
    __syncthreads();
    for (uint32_t k = 0; k < parts; ++k) {
      const uint64_t pidx = (uint64_t)b.hpart[g] + k;
      const uint32_t* in = b.hbuf + pidx * kHGroupPartWords;
      const uint32_t n = b.hcnt[pidx];
      for (uint32_t e0 = 0; e0 < n; e0 += kHGroupThreads) {  // the same trip count for every thread
        if (__any_sync(0xffffffffu, *(volatile uint32_t*)&sh.over != 0)) break;
        const uint32_t e = e0 + threadIdx.x;
        bool claimed = false;
        if (e < n) {
          const uint32_t key = in[3 * e], cnt = in[3 * e + 1], sum = in[3 * e + 2];
          if (key == kColEmpty) {
            atomicAdd(&sh.spec_cnt, cnt);
            atomicAdd(&sh.spec_sum, sum);
          } else {
            claimed = hg_insert(t_key, t_cnt, t_sum, key, cnt, sum);
          }
        }
        hg_count_fill(claimed, sh);
      }
    }
    __syncthreads();
    if (sh.over) {
      if (threadIdx.x == 0) atomicOr(&b.acc[0].fail, 1u);
    } else {
      hg_reduce(t_key, t_cnt, t_sum, sh, &b.acc[0]);
    }
    __syncthreads();  // the table and the shared words are reused by the next group
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&b.acc[0].done, 1u) == gridDim.x - 1) {
      __threadfence();
      const volatile ColPartAcc* va = b.acc;
      if (va->fail == 0) {
        q->unique_destinations = va->count;
        q->max_destination_fanin = va->max_fanin;
        q->max_destination_packets = va->max_packets;
        *len = 0;  // done: the remaining column passes and their run reduction skip the segment
      }
    }
  }
}

// CTAs per window for the cluster form (1 = the one-CTA kernel): enough to
// cover the SMs with the batch's windows, if the device hosts such clusters.
uint32_t colhash_cluster_size(uint32_t nseg) {
  static int ok[4][64];  // per size index and device: 0 unknown, 1 yes, 2 no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 1;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  for (uint32_t c = 8, k = 3; c >= 2; c >>= 1, --k) {
    if ((uint64_t)nseg * c > (uint64_t)sms) continue;
    if (ok[k][dev] == 0) {
      cudaLaunchConfig_t lc = {};
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = c;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      lc.attrs = &attr;
      lc.numAttrs = 1;
      lc.gridDim = dim3(c, 1, 1);
      lc.blockDim = dim3(kColHashThreads, 1, 1);
      lc.dynamicSmemBytes = kColHashSmem;
      int n = 0;
      ok[k][dev] = cudaFuncSetAttribute(k_colhash_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kColHashSmem) == cudaSuccess &&
                           cudaOccupancyMaxActiveClusters(&n, k_colhash_cl, &lc) == cudaSuccess && n > 0
                       ? 1
                       : 2;
      cudaGetLastError();
    }
    if (ok[k][dev] == 1) return c;
  }
  return 1;
}

}  // namespace

uint32_t colhash_ctas(uint32_t nseg) { return nseg ? colhash_cluster_size(nseg) : 1u; }

cudaError_t launch_colhash(const SegPlan& p, uint64_t* ulen, const uint32_t* col_ids, const uint32_t* vals32,
                           ans_quantities* q, cudaStream_t st) {
  if (p.nseg == 0) return cudaSuccess;
  static unsigned long long configured = 0;  // one bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_colhash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColHashSmem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured |= 1ull << dev;
  }
  const uint32_t c = colhash_cluster_size(p.nseg);
  if (c > 1) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    lc.gridDim = dim3(p.nseg * c, 1, 1);
    lc.blockDim = dim3(kColHashThreads, 1, 1);
    lc.dynamicSmemBytes = kColHashSmem;
    lc.stream = st;
    return cudaLaunchKernelEx(&lc, k_colhash_cl, p, ulen, col_ids, vals32, q);
  }
  k_colhash<<<p.nseg, kColHashThreads, kColHashSmem, st>>>(p, ulen, col_ids, vals32, q);
  return cudaGetLastError();
}

cudaError_t launch_colhash_part(const SegPlan& p, uint64_t* ulen, const uint32_t* col_ids, const uint32_t* vals32,
                                uint32_t* pkeys, uint32_t* pvals, uint32_t* bstart, ColPartAcc* acc, uint32_t* items,
                                ans_quantities* q, cudaStream_t st) {
  if (p.nseg == 0) return cudaSuccess;
  static unsigned long long configured = 0;  // one bit per device ordinal
  static int sms[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_colhash_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColHashSmem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (dev < 64) {
      sms[dev] = n;
      configured |= 1ull << dev;
    }
  }
  const unsigned ctas = dev < 64 && sms[dev] > 0 ? (unsigned)sms[dev] : 1u;
  k_colpart_split<<<p.nseg, kSplitThreads, 0, st>>>(p, ulen, col_ids, vals32, pkeys, pvals, bstart, acc + p.nseg,
                                                    items);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_colhash_part<<<ctas, kColHashThreads, kColHashSmem, st>>>(p, ulen, pkeys, pvals, bstart, acc, items, q);
  return cudaGetLastError();
}

cudaError_t launch_hgroup_stats(const uint32_t* keys, const uint32_t* vals32, uint64_t* len, const HGroupBufs& b,
                                uint32_t max_hparts, ans_quantities* q, cudaStream_t st) {
  static unsigned long long configured = 0;  // one bit per device ordinal
  static int sms[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_hgroup_hash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHGroupSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_hgroup_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHGroupSmem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (dev < 64) {
      sms[dev] = n;
      configured |= 1ull << dev;
    }
  }
  const unsigned ctas = 2u * (dev < 64 && sms[dev] > 0 ? (unsigned)sms[dev] : 1u);
  k_hgroup_bounds<<<ctas * 4, 256, 0, st>>>(keys, len, b.bnd);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_hgroup_plan<<<1, 1024, 0, st>>>(b, max_hparts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_hgroup_hash<<<ctas, kHGroupThreads, kHGroupSmem, st>>>(keys, vals32, b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_hgroup_merge<<<ctas, kHGroupThreads, kHGroupSmem, st>>>(b, len, q);
  return cudaGetLastError();
}

cudaError_t launch_nonzero_flags(const SegPlan& p, const uint64_t* vals, uint64_t* flags, uint32_t* err,
                                 cudaStream_t st) {
  const unsigned blocks = p.ntiles ? (p.ntiles * 16u > 4096u ? 4096u : p.ntiles * 16u) : 1u;
  k_nonzero_flags<<<blocks, 512, 0, st>>>(p, vals, flags, err);
  return cudaGetLastError();
}

cudaError_t launch_scatter_nonzero(const SegPlan& p, const uint64_t* kin, const uint64_t* vin, const uint64_t* pos,
                                   uint64_t* kout, uint64_t* vout, uint64_t* count, cudaStream_t st) {
  const unsigned blocks = p.ntiles ? (p.ntiles * 16u > 4096u ? 4096u : p.ntiles * 16u) : 1u;
  k_scatter_nonzero<<<blocks, 512, 0, st>>>(p, kin, vin, pos, kout, vout, count);
  return cudaGetLastError();
}

cudaError_t launch_check_dcsr(uint64_t nrows, uint64_t nnz, const uint32_t* row_ids, const uint64_t* row_ptr,
                              const uint32_t* col_ids, const uint64_t* vals, uint32_t* bad, cudaStream_t st) {
  const uint64_t n = nrows + 1 > nnz ? nrows + 1 : nnz;
  const uint64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want > 4096 ? 4096 : want);
  k_check_dcsr<<<blocks, 256, 0, st>>>(nrows, nnz, row_ids, row_ptr, col_ids, vals, bad);
  return cudaGetLastError();
}

cudaError_t launch_tile_seg(const SegPlan& p, uint32_t* tile_seg, cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
  const uint32_t want = (p.ntiles + 255) / 256;
  k_tile_seg<<<want < 4096 ? want : 4096, 256, 0, st>>>(p, tile_seg);
  return cudaGetLastError();
}

cudaError_t launch_wait_probe(const uint64_t* st, uint32_t* err, cudaStream_t stream) {
  k_wait_probe<<<1, 64, 0, stream>>>(st, err);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) {
  const size_t words = bytes / 4;
  const uint32_t ntail = (uint32_t)(bytes % 4);
  const size_t want = (words + 1023) / 1024;
  const unsigned blocks = (unsigned)(want < 1 ? 1 : (want > 2048 ? 2048 : want));
  k_zero<<<blocks, 256, 0, st>>>((uint32_t*)p, words, (uint8_t*)p + words * 4, ntail);
  return cudaGetLastError();
}

cudaError_t launch_rle(const StatsArgs& a, cudaStream_t st) {
  if (a.plan.ntiles == 0) return cudaSuccess;
  k_rle<<<a.plan.ntiles, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scan_u64(const SegPlan& p, const uint64_t* in, uint64_t* out, uint64_t* lookback_st,
                            uint32_t* ticket, uint32_t* err, cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
  k_scan_u64<<<p.ntiles, kThreads, 0, st>>>(p, in, out, lookback_st, ticket, err);
  return cudaGetLastError();
}

cudaError_t launch_finish(const StatsArgs& a, cudaStream_t st) {
  if (a.plan.ntiles == 0) return cudaSuccess;
  const bool h = a.col_hkeys != nullptr;
  switch (a.mode) {
    case kModeWindow:
      if (h) k_finish<kModeWindow, true><<<a.plan.ntiles, kThreads, 0, st>>>(a);
      else k_finish<kModeWindow, false><<<a.plan.ntiles, kThreads, 0, st>>>(a);
      break;
    case kModeSum:
      if (h) k_finish<kModeSum, true><<<a.plan.ntiles, kThreads, 0, st>>>(a);
      else k_finish<kModeSum, false><<<a.plan.ntiles, kThreads, 0, st>>>(a);
      break;
    default: k_finish<kModeMatrix, false><<<a.plan.ntiles, kThreads, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <typename V>
cudaError_t run_colstat(const SegPlan& p, const uint32_t* keys, const V* vals, ColBnd* bnd, ans_quantities* q,
                        cudaStream_t st) {
  if (p.ntiles == 0) return cudaSuccess;
  k_colstat<V><<<p.ntiles, kThreads, 0, st>>>(p, keys, vals, bnd, q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_colstat_fin<<<(p.ntiles + 255) / 256, 256, 0, st>>>(p, bnd, q);
  return cudaGetLastError();
}

cudaError_t launch_colstat(const SegPlan& p, const uint32_t* keys, const uint64_t* vals, ColBnd* bnd,
                           ans_quantities* q, cudaStream_t st) {
  return run_colstat(p, keys, vals, bnd, q, st);
}

cudaError_t launch_colstat32(const SegPlan& p, const uint32_t* keys, const uint32_t* vals, ColBnd* bnd,
                             ans_quantities* q, cudaStream_t st) {
  return run_colstat(p, keys, vals, bnd, q, st);
}

cudaError_t launch_empty_fixup(const StatsArgs& a, cudaStream_t st) {
  if (a.plan.nseg == 0) return cudaSuccess;
  k_empty_fixup<<<(a.plan.nseg + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ans
