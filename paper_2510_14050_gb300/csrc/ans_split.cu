// Row partition of a matrix across ranks: the exchange step of a time sum
// computed on several devices (Sec. III-A, Fig. 4: data split evenly over
// devices; the global A summed over t is owned in row partitions).
//
// Rank o owns the rows whose source address hashes to o: the owner of row i
// is ((i * 0x9E3779B1 mod 2^32) * nparts) >> 32, a multiplicative hash, so
// clustered sources spread over the ranks.  The matrix's rows are split,
// stably, into one DCSR per owner:
//  1. k_split_count: per tile of 8192 rows, the rows and links of each owner;
//  2. k_split_scan: per owner, exclusive offsets of those counts over the
//     tiles, and each owner's totals;
//  3. k_split_rows: per tile, each row's position among its owner's rows
//     (warps count per owner, a scan over warps, then rows in order) --
//     written to the owner's row_ids / row_ptr -- and its owner and first
//     link position kept per row;
//  4. k_split_links: per link (tiles of 8192 links; each link finds its row
//     among the rows covering the tile, staged in shared memory), its column
//     and count copied to the owner's arrays.
// Rows keep their order within an owner, and a row's links stay together, so
// every piece is canonical DCSR.
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr int kSplitRowThreads = 512;
constexpr uint32_t kSplitRowTile = 8192;
constexpr int kSplitWarps = kSplitRowThreads / 32;
constexpr uint32_t kRowsPerWarp = kSplitRowTile / kSplitWarps;  // 512

__device__ __forceinline__ uint32_t row_owner_of(uint32_t row, uint32_t nparts) {
  const uint64_t h = (uint64_t)(uint32_t)(row * 0x9E3779B1u);
  return (uint32_t)((h * nparts) >> 32);
}

// tcnt: [tiles][nparts] rows (uint32) and links (uint64) of each owner.
__global__ void __launch_bounds__(kSplitRowThreads) k_split_count(uint64_t nrows, const uint32_t* __restrict__ row_ids,
                                                                  const uint64_t* __restrict__ row_ptr, uint32_t nparts,
                                                                  uint32_t* __restrict__ trows,
                                                                  uint64_t* __restrict__ tlinks) {
  __shared__ uint32_t s_r[kMaxSplitParts];
  __shared__ unsigned long long s_l[kMaxSplitParts];
  if (threadIdx.x < kMaxSplitParts) {
    s_r[threadIdx.x] = 0;
    s_l[threadIdx.x] = 0;
  }
  __syncthreads();
  const uint64_t r0 = (uint64_t)blockIdx.x * kSplitRowTile;
  const uint64_t r1 = umin64(r0 + kSplitRowTile, nrows);
  for (uint64_t r = r0 + threadIdx.x; r < r1; r += kSplitRowThreads) {
    const uint32_t o = row_owner_of(row_ids[r], nparts);
    atomicAdd(&s_r[o], 1u);
    atomicAdd(&s_l[o], (unsigned long long)(row_ptr[r + 1] - row_ptr[r]));
  }
  __syncthreads();
  if (threadIdx.x < nparts) {
    trows[(uint64_t)blockIdx.x * nparts + threadIdx.x] = s_r[threadIdx.x];
    tlinks[(uint64_t)blockIdx.x * nparts + threadIdx.x] = s_l[threadIdx.x];
  }
}

// One CTA: thread o scans owner o's counts over the tiles (exclusive, in
// place) and writes the totals to totals[o] = {rows, links}.
__global__ void k_split_scan(uint32_t ntiles, uint32_t nparts, uint32_t* __restrict__ trows,
                             uint64_t* __restrict__ tlinks, uint64_t* __restrict__ totals) {
  const uint32_t o = threadIdx.x;
  if (o >= nparts) return;
  uint64_t rr = 0, ll = 0;
  for (uint32_t t = 0; t < ntiles; ++t) {
    const uint64_t i = (uint64_t)t * nparts + o;
    const uint32_t a = trows[i];
    const uint64_t b = tlinks[i];
    trows[i] = (uint32_t)rr;
    tlinks[i] = ll;
    rr += a;
    ll += b;
  }
  totals[2 * o] = rr;
  totals[2 * o + 1] = ll;
}

// Per tile: every row's owner, its index among the owner's rows and its
// first link there; the owner's row_ids / row_ptr written.
__global__ void __launch_bounds__(kSplitRowThreads) k_split_rows(uint64_t nrows, const uint32_t* __restrict__ row_ids,
                                                                 const uint64_t* __restrict__ row_ptr, uint32_t nparts,
                                                                 const uint32_t* __restrict__ trows,
                                                                 const uint64_t* __restrict__ tlinks,
                                                                 SplitOut out, uint32_t* __restrict__ rown,
                                                                 uint64_t* __restrict__ rlink) {
  __shared__ uint32_t s_wr[kSplitWarps][kMaxSplitParts];
  __shared__ unsigned long long s_wl[kSplitWarps][kMaxSplitParts];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < kSplitWarps * kMaxSplitParts; i += kSplitRowThreads) {
    (&s_wr[0][0])[i] = 0;
    (&s_wl[0][0])[i] = 0;
  }
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * kSplitRowTile;
  const uint64_t w0 = t0 + (uint64_t)warp * kRowsPerWarp;
  const uint64_t w1 = umin64(w0 + kRowsPerWarp, nrows);
  // pass 1: rows and links of each owner in this warp's rows
  for (uint64_t c = w0; c < w1; c += 32) {  // the same bound for the whole warp
    const uint64_t r = c + lane;
    const bool valid = r < w1;
    const uint32_t o = valid ? row_owner_of(row_ids[r], nparts) : 0xFFFFFFFFu;
    const uint64_t len = valid ? row_ptr[r + 1] - row_ptr[r] : 0ull;
    if (valid) {
      atomicAdd(&s_wr[warp][o], 1u);
      atomicAdd(&s_wl[warp][o], (unsigned long long)len);
    }
  }
  __syncthreads();
  // exclusive offsets of each warp per owner, plus the tile's offset
  if (threadIdx.x < nparts) {
    const uint32_t o = threadIdx.x;
    uint32_t rr = trows[(uint64_t)blockIdx.x * nparts + o];
    unsigned long long ll = tlinks[(uint64_t)blockIdx.x * nparts + o];
    for (int w = 0; w < kSplitWarps; ++w) {
      const uint32_t a = s_wr[w][o];
      const unsigned long long b = s_wl[w][o];
      s_wr[w][o] = rr;
      s_wl[w][o] = ll;
      rr += a;
      ll += b;
    }
  }
  __syncthreads();
  // pass 2: rows in order; lanes with the same owner take consecutive places
  for (uint64_t c = w0; c < w1; c += 32) {
    const uint64_t r = c + lane;
    const bool valid = r < w1;
    const uint32_t id = valid ? row_ids[r] : 0u;
    const uint32_t o = valid ? row_owner_of(id, nparts) : 0xFFFFFFFFu;
    const uint64_t len = valid ? row_ptr[r + 1] - row_ptr[r] : 0ull;
    const uint32_t peers = __match_any_sync(0xffffffffu, o);
    const uint32_t below = peers & lanemask_lt();
    // links of the same-owner lanes before this one: every lane of the group
    // walks the whole group (the same shuffles in the same order) and adds the
    // lengths of the lanes below it
    unsigned long long before = 0;
    for (uint32_t m = peers; m; m &= m - 1) {
      const int l = __ffs(m) - 1;
      const unsigned long long v = __shfl_sync(peers, (unsigned long long)len, l);
      if (l < lane) before += v;
    }
    if (valid) {
      const uint32_t ri = s_wr[warp][o] + __popc(below);
      const unsigned long long li = s_wl[warp][o] + before;
      out.row_ids[o][ri] = id;
      out.row_ptr[o][ri] = li;
      rown[r] = o;
      rlink[r] = li;
    }
    __syncwarp();
    // advance this warp's per-owner cursors by the chunk (the highest lane of each owner)
    if (valid && (peers >> lane) == 1u) {
      s_wr[warp][o] += __popc(peers);
      s_wl[warp][o] += before + len;
    }
    __syncwarp();
  }
}

// Per tile of 8192 links: each link's column and count copied to its row's
// owner at the row's first link there plus the link's place in the row.  The
// rows covering the tile are found by two warps (binary searches of row_ptr)
// and staged in shared memory.
constexpr size_t kSplitLinkSmem = (size_t)(kTile + 1) * sizeof(uint32_t);

__global__ void __launch_bounds__(kSplitRowThreads) k_split_links(uint64_t nrows, uint64_t nnz,
                                                                  const uint64_t* __restrict__ row_ptr,
                                                                  const uint32_t* __restrict__ col_ids,
                                                                  const uint64_t* __restrict__ vals,
                                                                  const uint32_t* __restrict__ rown,
                                                                  const uint64_t* __restrict__ rlink, SplitOut out) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* s_rp = reinterpret_cast<uint32_t*>(smem);  // row starts relative to the tile
  __shared__ uint64_t s_r0, s_r1;
  const uint64_t u0 = (uint64_t)blockIdx.x * kTile;
  if (u0 >= nnz) return;
  const uint32_t cnt = (uint32_t)umin64(kTile, nnz - u0);
  if (threadIdx.x < 64) {  // warp 0: the row of the tile's first link, warp 1: of its last
    const uint64_t u = threadIdx.x < 32 ? u0 : u0 + cnt - 1;
    const uint32_t lane = threadIdx.x & 31;
    uint64_t lo = 0, hi = nrows;  // row_ptr[lo] <= u < row_ptr[hi]
    while (hi - lo > 1) {
      const uint64_t c = lo + ((hi - lo) * (lane + 1)) / 33;
      const uint32_t le = __ballot_sync(0xffffffffu, row_ptr[c] <= u);
      const int nt = __popc(le);
      const uint64_t c_last = __shfl_sync(0xffffffffu, c, nt > 0 ? nt - 1 : 0);
      const uint64_t c_first = __shfl_sync(0xffffffffu, c, nt < 32 ? nt : 31);
      if (nt > 0) lo = c_last;
      if (nt < 32) hi = c_first;
    }
    if (lane == 0) {
      if (threadIdx.x < 32) s_r0 = lo;
      else s_r1 = lo;
    }
  }
  __syncthreads();
  const uint64_t r0 = s_r0;
  const uint32_t nr = (uint32_t)(s_r1 - r0 + 1);
  for (uint32_t i = threadIdx.x; i <= nr; i += kSplitRowThreads) {
    const uint64_t rp = row_ptr[r0 + i];
    s_rp[i] = rp <= u0 ? 0u : (uint32_t)umin64(rp - u0, cnt);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += kSplitRowThreads) {
    uint32_t lo = 0, hi = nr;  // last row with s_rp <= i
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_rp[mid] <= i) lo = mid; else hi = mid;
    }
    const uint64_t r = r0 + lo;
    const uint64_t u = u0 + i;
    const uint32_t o = rown[r];
    const uint64_t pos = rlink[r] + (u - row_ptr[r]);
    out.col_ids[o][pos] = col_ids[u];
    out.vals[o][pos] = vals[u];
  }
}

// Closing row pointers and headers of the owners' pieces.
__global__ void k_split_close(uint32_t nparts, const uint64_t* __restrict__ totals, SplitOut out) {
  const uint32_t o = threadIdx.x;
  if (o >= nparts) return;
  out.row_ptr[o][totals[2 * o]] = totals[2 * o + 1];
  out.hdr[o][0] = totals[2 * o];
  out.hdr[o][1] = totals[2 * o + 1];
}

}  // namespace

uint32_t split_row_tiles(uint64_t nrows) { return (uint32_t)((nrows + kSplitRowTile - 1) / kSplitRowTile); }

cudaError_t launch_split_count(uint64_t nrows, const uint32_t* row_ids, const uint64_t* row_ptr, uint32_t nparts,
                               uint32_t* trows, uint64_t* tlinks, uint64_t* totals, cudaStream_t st) {
  const uint32_t nt = split_row_tiles(nrows);
  if (nt) {
    k_split_count<<<nt, kSplitRowThreads, 0, st>>>(nrows, row_ids, row_ptr, nparts, trows, tlinks);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_split_scan<<<1, kMaxSplitParts, 0, st>>>(nt, nparts, trows, tlinks, totals);
  return cudaGetLastError();
}

cudaError_t launch_split_fill(uint64_t nrows, uint64_t nnz, const uint32_t* row_ids, const uint64_t* row_ptr,
                              const uint32_t* col_ids, const uint64_t* vals, uint32_t nparts, const uint32_t* trows,
                              const uint64_t* tlinks, const uint64_t* totals, uint32_t* rown, uint64_t* rlink,
                              const SplitOut& out, cudaStream_t st) {
  cudaError_t e;
  const uint32_t nt = split_row_tiles(nrows);
  if (nt) {
    k_split_rows<<<nt, kSplitRowThreads, 0, st>>>(nrows, row_ids, row_ptr, nparts, trows, tlinks, out, rown, rlink);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const uint64_t lt = (nnz + kTile - 1) / kTile;
  if (lt) {
    static unsigned long long configured = 0;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev >= 64 || !((configured >> dev) & 1ull)) {
      e = cudaFuncSetAttribute(k_split_links, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSplitLinkSmem);
      if (e != cudaSuccess) return e;
      if (dev < 64) configured |= 1ull << dev;
    }
    k_split_links<<<(unsigned)lt, kSplitRowThreads, kSplitLinkSmem, st>>>(nrows, nnz, row_ptr, col_ids, vals, rown,
                                                                        rlink, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_split_close<<<1, kMaxSplitParts, 0, st>>>(nparts, totals, out);
  return cudaGetLastError();
}

}  // namespace ans
