// Allocation-free quantities of one window: ans_window_quantities_noalloc.
//
// Some callers cannot allocate device memory once they are running: a
// capture appliance whose device memory is owned up front by another
// framework's caching allocator (a cudaMalloc would fail or fragment it), or a
// latency-critical ingest loop that cannot afford cudaMalloc/cudaFree's
// implicit synchronisation and unpredictable latency.  For them this entry
// point runs the same sort / run-length / statistics kernels as
// ans_build_window, but every intermediate buffer lives in one file-scope
// device array of fixed size, so the call allocates nothing (no cudaMalloc,
// no cudaFree, no pinned host buffer, no torch allocation).
//
// Limits and sharing:
//  * at most kNoAllocMaxPackets (65,536) packets per call; larger windows are
//    rejected with ANS_ERR_INVALID_ARG;
//  * the array (kNoAllocBytes, about 5 MiB) exists on every GPU that loads
//    the library and is held until the process exits;
//  * every call uses the same array, and the array keeps the previous call's
//    contents: the call clears what must start at zero itself, and calls
//    whose work overlaps on the GPU (different streams, or different host
//    threads without ordering) race and give wrong results;
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress with that device current); make that first call
//    before any stream capture begins.  The address is kept for the life of
//    the process, so the entry point must not be used after a
//    cudaDeviceReset() of that device (the array's old address would be
//    stale).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ans.h"
#include "ans_internal.cuh"

namespace ans {

namespace {

constexpr uint64_t kNoAllocMaxPackets = 1ull << 16;
constexpr uint32_t kNoAllocTiles = (uint32_t)(kNoAllocMaxPackets / kTile);
// The buffers below are sized for kNoAllocMaxPackets items, which must cover
// the padded index space (whole tiles) of the largest window.
static_assert(kNoAllocMaxPackets % kTile == 0, "the packet limit must be a whole number of tiles");
// The key passes run with the default launch shape; its sub-tiles' status
// words must fit the two per tile reserved at oSt0 / oSt1.
constexpr SortCfg kNoAllocSort{};
static_assert(key_subtiles(kNoAllocSort) <= 2, "status words hold at most two sub-tiles per tile");
constexpr size_t kAl = 256;
constexpr size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// Byte offsets inside the scratch array.
constexpr size_t oPlan = 0;                                        // in_off, len, base, first_tile[2]
constexpr size_t oKeysA = al(oPlan + 64);
constexpr size_t oKeysB = al(oKeysA + kNoAllocMaxPackets * 8);
constexpr size_t oHist = al(oKeysB + kNoAllocMaxPackets * 8);
// look-back status words: two sub-tiles' worth per tile (k_finish clears
// that many for the column passes)
constexpr size_t oSt0 = al(oHist + (size_t)kPasses * kRadix * 4);
constexpr size_t oSt1 = al(oSt0 + (size_t)kNoAllocTiles * 2 * kRadix * 8);
constexpr size_t oLb = al(oSt1 + (size_t)kNoAllocTiles * 2 * kRadix * 8);
constexpr size_t oTickets = al(oLb + (size_t)kNoAllocTiles * 8);
constexpr size_t oRunStart = al(oTickets + 128 * 4);
constexpr size_t oRowPos = al(oRunStart + (kNoAllocMaxPackets + 1) * 8);
constexpr size_t oColIds = al(oRowPos + (kNoAllocMaxPackets + 1) * 8);
constexpr size_t oVals = al(oColIds + kNoAllocMaxPackets * 4);
constexpr size_t oRowIds = al(oVals + kNoAllocMaxPackets * 8);
constexpr size_t oRowPtr = al(oRowIds + kNoAllocMaxPackets * 4);
constexpr size_t oHdr = al(oRowPtr + (kNoAllocMaxPackets + 1) * 8);
constexpr size_t oQ = al(oHdr + 16);
constexpr size_t oErr = al(oQ + sizeof(ans_quantities));
constexpr size_t oColHist = al(oErr + 8);                          // destination digit counts
constexpr size_t oUlen = al(oColHist + (size_t)kColPasses * kRadix * 4);
constexpr size_t oCkA = al(oUlen + 8);                             // destination-sort ping-pong
constexpr size_t oCkB = al(oCkA + kNoAllocMaxPackets * 4);
constexpr size_t oCvA = al(oCkB + kNoAllocMaxPackets * 4);
constexpr size_t oCvB = al(oCvA + kNoAllocMaxPackets * 8);
constexpr size_t oBnd = al(oCvB + kNoAllocMaxPackets * 8);
constexpr size_t kNoAllocBytes = al(oBnd + (size_t)kNoAllocTiles * sizeof(ColBnd));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// One-segment plan for a window of n packets, written on the device.
__global__ void k_noalloc_plan(uint64_t n, uint32_t ntiles) {
  if (threadIdx.x != 0) return;
  uint64_t* p = reinterpret_cast<uint64_t*>(g_noalloc_scratch + oPlan);
  p[0] = 0;  // in_off
  p[1] = n;  // len
  p[2] = 0;  // base
  uint32_t* ft = reinterpret_cast<uint32_t*>(p + 3);
  ft[0] = 0;
  ft[1] = ntiles;
}

std::mutex g_mu;
void* g_addr[64] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = ptr;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ans

using namespace ans;

extern "C" int ans_window_quantities_noalloc(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                                             ans_quantities* d_out, uint32_t* d_status, void* stream) {
  if (!d_out) return set_last_error(ANS_ERR_INVALID_ARG, "d_out is NULL");
  if (n > kNoAllocMaxPackets)
    return set_last_error(ANS_ERR_INVALID_ARG, "ans_window_quantities_noalloc takes at most 65536 packets, got " +
                                                   std::to_string(n));
  if (n && (!d_src || !d_dst)) return set_last_error(ANS_ERR_INVALID_ARG, "NULL packet arrays");
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess)
    return set_last_error(ANS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  char* m = static_cast<char*>(base);
  uint32_t* err = reinterpret_cast<uint32_t*>(m + oErr);
  ans_quantities* q = reinterpret_cast<ans_quantities*>(m + oQ);
  auto cu = [&](cudaError_t x, const char* what) -> int {
    if (x == cudaSuccess) return ANS_OK;
    return set_last_error(ANS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(x));
  };
  int rc;
  if ((rc = cu(cudaMemsetAsync(q, 0, sizeof(ans_quantities), st), "memset"))) return rc;
  if ((rc = cu(cudaMemsetAsync(err, 0, 8, st), "memset"))) return rc;  // error bits; default poll limit
  const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
  if (ntiles) {
    if ((rc = cu(cudaMemsetAsync(m + oHist, 0, (size_t)kPasses * kRadix * 4, st), "memset"))) return rc;
    if ((rc = cu(cudaMemsetAsync(m + oLb, 0, (size_t)ntiles * 8, st), "memset"))) return rc;
    if ((rc = cu(cudaMemsetAsync(m + oColHist, 0, (size_t)kColPasses * kRadix * 4, st), "memset"))) return rc;
    k_noalloc_plan<<<1, 32, 0, st>>>(n, ntiles);
    if ((rc = cu(cudaGetLastError(), "plan"))) return rc;
    SegPlan p;
    uint64_t* pl = reinterpret_cast<uint64_t*>(m + oPlan);
    p.in_off = pl;
    p.len = pl + 1;
    p.base = pl + 2;
    p.first_tile = reinterpret_cast<const uint32_t*>(pl + 3);
    p.nseg = 1;
    p.ntiles = ntiles;
    uint64_t* ka = reinterpret_cast<uint64_t*>(m + oKeysA);
    uint64_t* kb = reinterpret_cast<uint64_t*>(m + oKeysB);
    uint64_t* st0 = reinterpret_cast<uint64_t*>(m + oSt0);
    uint64_t* st1 = reinterpret_cast<uint64_t*>(m + oSt1);
    uint32_t* hist = reinterpret_cast<uint32_t*>(m + oHist);
    uint32_t* tickets = reinterpret_cast<uint32_t*>(m + oTickets);
    if ((rc = cu(launch_pack_hist(p, d_src, d_dst, ka, hist, st0, tickets, st, key_subtiles(kNoAllocSort)), "pack"))) return rc;
    for (int pass = 0; pass < kPasses; ++pass) {
      const bool even = (pass % 2) == 0;
      if ((rc = cu(launch_onesweep(p, pass, even ? ka : kb, even ? kb : ka, nullptr, nullptr, hist,
                                   even ? st0 : st1, even ? st1 : st0, tickets + pass, err, kNoAllocSort, st),
                   "onesweep")))
        return rc;
    }
    StatsArgs a;
    a.plan = p;
    a.hdr = reinterpret_cast<uint64_t*>(m + oHdr);
    a.q = q;
    a.keys = ka;
    a.col_ids = reinterpret_cast<uint32_t*>(m + oColIds);
    a.vals = reinterpret_cast<uint64_t*>(m + oVals);
    a.row_ids = reinterpret_cast<uint32_t*>(m + oRowIds);
    a.row_ptr = reinterpret_cast<uint64_t*>(m + oRowPtr);
    a.run_start = reinterpret_cast<uint64_t*>(m + oRunStart);
    a.row_pos = reinterpret_cast<uint64_t*>(m + oRowPos);
    a.pre = nullptr;
    a.lookback = reinterpret_cast<uint64_t*>(m + oLb);
    a.ticket = tickets + kPasses;
    a.col_hist = reinterpret_cast<uint32_t*>(m + oColHist);
    a.ulen = reinterpret_cast<uint64_t*>(m + oUlen);
    a.col_st0 = st0;
    a.col_tickets = tickets + 32;
    a.err = err;
    a.mode = kModeWindow;
    if ((rc = cu(launch_rle(a, st), "rle"))) return rc;
    if ((rc = cu(launch_finish(a, st), "finish"))) return rc;
    // Column statistics: sort the stored links by destination, reduce the runs.
    SegPlan cp = p;
    cp.len = a.ulen;
    uint32_t* cka = reinterpret_cast<uint32_t*>(m + oCkA);
    uint32_t* ckb = reinterpret_cast<uint32_t*>(m + oCkB);
    uint64_t* cva = reinterpret_cast<uint64_t*>(m + oCvA);
    uint64_t* cvb = reinterpret_cast<uint64_t*>(m + oCvB);
    for (int pass = 0; pass < kColPasses; ++pass) {
      const uint32_t* kin = pass == 0 ? a.col_ids : (pass % 2 ? cka : ckb);
      const uint64_t* vin = pass == 0 ? a.vals : (pass % 2 ? cva : cvb);
      if ((rc = cu(launch_onesweep_col(cp, pass, kin, pass % 2 ? ckb : cka, vin, pass % 2 ? cvb : cva, a.col_hist,
                                       pass % 2 ? st1 : st0, pass % 2 ? st0 : st1, a.col_tickets + pass, err,
                                       kNoAllocSort, st),
                   "onesweep_col")))
        return rc;
    }
    if ((rc = cu(launch_colstat(cp, ckb, cvb, reinterpret_cast<ColBnd*>(m + oBnd), q, st), "colstat"))) return rc;
  }
  if ((rc = cu(cudaMemcpyAsync(d_out, q, sizeof(ans_quantities), cudaMemcpyDefault, st), "copy out"))) return rc;
  if (d_status && (rc = cu(cudaMemcpyAsync(d_status, err, 4, cudaMemcpyDefault, st), "copy status"))) return rc;
  return ANS_OK;
}
