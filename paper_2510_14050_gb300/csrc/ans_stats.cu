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
//    nonzero counts (fan-out) and packet sums (Sec. IV-C), and the
//    transpose-free column pass: every stored link adds (1, A(i,j)) to its
//    destination's slot in an open-addressing table keyed on dst.
//  * k_col_scan: unique destinations, max fan-in and max destination packets
//    from the table; each slot is cleared as it is read, so the table is all
//    zero again for the next call without a memset.
// Maxima are combined with 64-bit atomicMax; every value is an exact integer.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr uint64_t kLow31 = (1ull << 31) - 1;

__global__ void __launch_bounds__(kThreads) k_rle(StatsArgs a) {
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
  if (threadIdx.x == 0) {
    uint32_t th = 0, tr = 0;
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t x = s_wh[w], y = s_wr[w];
      s_wh[w] = th;
      s_wr[w] = tr;
      th += x;
      tr += y;
    }
    const uint64_t agg = ((uint64_t)th << 31) | tr;
    uint64_t* my = a.lookback + t;
    uint64_t excl = 0;
    if (tl.j == 0) {
      st_relaxed(my, kFlagPre | agg);
    } else {
      st_relaxed(my, kFlagAgg | agg);
      excl = lookback(a.lookback, 1, t - tl.j, t, a.err);
      st_relaxed(my, kFlagPre | (excl + agg));
    }
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
  __syncthreads();
  uint64_t uh = s_eh + s_wh[warp], ur = s_er + s_wr[warp];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    if ((hb[i] >> lane) & 1u) {
      const uint64_t u = uh + __popc(hb[i] & lt);
      a.col_ids[tl.base + u] = (uint32_t)k[i];
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
  if (threadIdx.x == 0) {
    uint64_t tot = 0;
    for (int w = 0; w < kWarps; ++w) {
      const uint64_t x = s_w[w];
      s_w[w] = tot;
      tot += x;
    }
    uint64_t* my = lookback_st + t;
    uint64_t excl = 0;
    if (tl.j == 0) {
      st_relaxed(my, kFlagPre | (tot & kValMask));
    } else {
      st_relaxed(my, kFlagAgg | (tot & kValMask));
      excl = lookback(lookback_st, 1, t - tl.j, t, err);
      st_relaxed(my, kFlagPre | ((excl + tot) & kValMask));
    }
    s_excl = excl;
    if (tl.start + tl.count == tl.len) out[bs + tl.len] = excl + tot;
  }
  __syncthreads();
  const uint64_t off = s_excl + s_w[warp];
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const uint32_t idx = wbase + i * 32 + lane;
    if (idx < tl.count) out[bs + tl.start + idx] = off + ex[i];
  }
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Capacity of a segment's column table: load factor <= 1/2.
__device__ __forceinline__ uint64_t table_cap(uint64_t nnz, uint32_t seg_tiles) {
  return umin64(2 * nnz + 64, 2ull * seg_tiles * kTile);
}

// Slot word = dst << 32 | (number of links into dst); 0 = empty (every
// occupied slot has at least one link, so the low half is never 0).
__device__ __forceinline__ void col_insert(unsigned long long* table, unsigned long long* sums,
                                           uint64_t cap, uint32_t dst, uint64_t v, uint32_t* err) {
  uint64_t i = ((uint64_t)fmix32(dst) * cap) >> 32;
  const unsigned long long want = ((unsigned long long)dst << 32) | 1ull;
  for (uint64_t probe = 0; probe < cap; ++probe) {
    unsigned long long w = ld_relaxed(reinterpret_cast<const uint64_t*>(table + i));
    if (w == 0ull) {
      w = atomicCAS(table + i, 0ull, want);
      if (w == 0ull) {
        atomicAdd(sums + i, (unsigned long long)v);
        return;
      }
    }
    if ((uint32_t)(w >> 32) == dst) {
      atomicAdd(table + i, 1ull);
      atomicAdd(sums + i, (unsigned long long)v);
      return;
    }
    if (++i == cap) i = 0;
  }
  atomicOr(err, (uint32_t)kErrHashFull);
}

template <int kMode>
__global__ void __launch_bounds__(kThreads) k_finish(StatsArgs a) {
  __shared__ Tile s_tile;
  __shared__ uint64_t s_red[3][kWarps];
  const Tile tl = block_tile(a.plan, blockIdx.x, &s_tile);
  const uint32_t s = tl.seg;
  const uint64_t nrows = a.hdr[2 * s], nnz = a.hdr[2 * s + 1];
  const uint64_t bs = tl.base + s;
  const uint64_t cap = table_cap(nnz, tl.seg_tiles);
  unsigned long long* table = a.table + 2 * tl.base;
  unsigned long long* tsum = a.table_sum + 2 * tl.base;

  auto P = [&](uint64_t x) -> uint64_t { return a.pre ? a.pre[bs + x] : x; };

  uint64_t mlink = 0, mfan = 0, mrow = 0;
  const uint64_t u_end = umin64(tl.start + kTile, nnz);
  for (uint64_t u = tl.start + threadIdx.x; u < u_end; u += kThreads) {
    uint64_t v;
    if (kMode == kModeMatrix) {
      v = a.vals[tl.base + u];
    } else {
      v = P(a.run_start[bs + u + 1]) - P(a.run_start[bs + u]);
      a.vals[tl.base + u] = v;
    }
    mlink = v > mlink ? v : mlink;
    col_insert(table, tsum, cap, a.col_ids[tl.base + u], v, a.err);
  }
  const uint64_t r_end = umin64(tl.start + kTile, nrows);
  for (uint64_t r = tl.start + threadIdx.x; r < r_end; r += kThreads) {
    const uint64_t p0 = a.row_ptr[bs + r], p1 = a.row_ptr[bs + r + 1];
    const uint64_t fan = p1 - p0;
    const uint64_t rs = kMode == kModeMatrix ? P(p1) - P(p0) : P(a.row_pos[bs + r + 1]) - P(a.row_pos[bs + r]);
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

__global__ void __launch_bounds__(kThreads) k_col_scan(StatsArgs a) {
  __shared__ Tile s_tile;
  __shared__ uint64_t s_red[3][kWarps];
  const Tile tl = block_tile(a.plan, blockIdx.x, &s_tile);
  const uint32_t s = tl.seg;
  const uint64_t nnz = a.hdr[2 * s + 1];
  const uint64_t cap = table_cap(nnz, tl.seg_tiles);
  unsigned long long* table = a.table + 2 * tl.base;
  unsigned long long* tsum = a.table_sum + 2 * tl.base;
  uint64_t c = 0, mfan = 0, mpk = 0;
  if (nnz > 0) {
    const uint64_t s0 = 2 * tl.start, s1 = umin64(s0 + 2 * kTile, cap);
    for (uint64_t i = s0 + threadIdx.x; i < s1; i += kThreads) {
      const unsigned long long w = table[i];
      if (w) {
        const uint64_t pk = tsum[i];
        ++c;
        mfan = umax64(mfan, w & 0xffffffffull);
        mpk = umax64(mpk, pk);
        table[i] = 0ull;
        tsum[i] = 0ull;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c = warp_sum(c);
  mfan = warp_max(mfan);
  mpk = warp_max(mpk);
  if (lane == 0) {
    s_red[0][warp] = c;
    s_red[1][warp] = mfan;
    s_red[2][warp] = mpk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) {
      c += s_red[0][w];
      mfan = umax64(mfan, s_red[1][w]);
      mpk = umax64(mpk, s_red[2][w]);
    }
    ans_quantities* q = a.q + s;
    if (c) atomicAdd((unsigned long long*)&q->unique_destinations, (unsigned long long)c);
    if (mfan) atomicMax((unsigned long long*)&q->max_destination_fanin, (unsigned long long)mfan);
    if (mpk) atomicMax((unsigned long long*)&q->max_destination_packets, (unsigned long long)mpk);
  }
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
}

}  // namespace

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
  switch (a.mode) {
    case kModeWindow: k_finish<kModeWindow><<<a.plan.ntiles, kThreads, 0, st>>>(a); break;
    case kModeSum: k_finish<kModeSum><<<a.plan.ntiles, kThreads, 0, st>>>(a); break;
    default: k_finish<kModeMatrix><<<a.plan.ntiles, kThreads, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_col_scan(const StatsArgs& a, cudaStream_t st) {
  if (a.plan.ntiles == 0) return cudaSuccess;
  k_col_scan<<<a.plan.ntiles, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_empty_fixup(const StatsArgs& a, cudaStream_t st) {
  if (a.plan.nseg == 0) return cudaSuccess;
  k_empty_fixup<<<(a.plan.nseg + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ans
