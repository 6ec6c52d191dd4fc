// Internal declarations shared by the CUDA translation units of libans.so.
//
// Work is organised in *segments* (one per window, one per time sum, one per
// matrix) that are cut into fixed tiles of kTile items.  Every segment starts
// at a multiple of kTile in a padded index space, so tiles never straddle
// segments and 16-byte vector accesses of scratch are always aligned.  Kernels
// that carry a running prefix from tile to tile (radix digit offsets, run and
// row counts, value prefixes) use single-pass decoupled look-back over tile
// status words; tiles take tickets in launch order so a tile only ever waits
// for tiles that are already running, and every wait is bounded.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ans.h"

namespace ans {

constexpr int kThreads = 512;                  // threads per tile CTA
constexpr int kPerThread = 16;                 // items per thread
constexpr int kTile = kThreads * kPerThread;   // 8192 items per tile
constexpr int kWarps = kThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPasses = 64 / kRadixBits;       // LSD passes over a 64-bit key
constexpr int kColPasses = 32 / kRadixBits;    // LSD passes over a 32-bit destination key
constexpr int kWindowCluster = 8;              // CTAs of the on-chip window sort's cluster
constexpr uint32_t kClusterWindowMax = 1u << 17;  // largest window sorted on chip (1 MiB of keys)

// Look-back status word: 2 flag bits over a 62-bit value.
constexpr uint64_t kFlagAgg = 1ull << 62;      // tile aggregate available
constexpr uint64_t kFlagPre = 2ull << 62;      // inclusive prefix available
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 20;      // default polls (about 1 s) before a wait gives up
constexpr uint32_t kSpinLimitMax = 1u << 24;   // largest settable poll limit (about 16 s)

// Every kernel that waits receives `err`, the device error word of its
// context: err[0] collects ErrBits, err[1] holds the context's poll limit for
// bounded waits (0 = kSpinLimit).
enum ErrBits : uint32_t {
  kErrLookback = 1u,   // a look-back wait hit its poll limit
  kErrHashFull = 2u,   // a hash probe sequence found no free slot
  kErrNegative = 4u,   // a signed combination left a negative count
  kErrPlan = 8u,       // device-resident batch offsets were invalid or above the capacity
  kErrGuard = 16u,     // a scratch guard (debug mode) was overwritten
};
constexpr uint64_t kMaxWindowItems = (1ull << 31) - 1;  // packets of one window, links of one time sum
constexpr int kPassStable = 0x100;  // digit-pass flag: pass 0 keeps the input order of equal digits
constexpr int kPassMask = 0xFF;
constexpr uint32_t kMaxRegroupWindows = 1u << 16;  // window ids carried as 16-bit values

// How a onesweep pass is launched (chosen per context by the autotuner):
// threads per 8192-key tile (512 or 1024; for the 64-bit key passes and the
// column passes with 32-bit counts also 256, which splits every tile into
// two 4096-key sub-tiles with one CTA each and four resident CTAs per SM), how lanes with equal digits are found (one
// __match_any_sync; eight ballots; or a per-warp shared-memory table where
// each lane ORs its bit into its digit's entry, which also holds the digit's
// running count), and whether a 512-thread tile is compiled to leave room for
// two resident CTAs per SM (64 registers).
enum RankMode : int { kRankMatch = 0, kRankBallot = 1, kRankTable = 2 };
struct SortCfg {
  int threads = 512;
  int rank = kRankMatch;
  int blocks = 1;
};

// One entry per segment; device pointers.
struct SegPlan {
  const uint64_t* in_off = nullptr;     // first item in the input stream (window path)
  const uint64_t* src_at = nullptr;     // or: per-segment addresses of the src / dst arrays
  const uint64_t* dst_at = nullptr;     //     (device-accessible; then in_off is unused)
  const uint64_t* len = nullptr;        // items in the segment (may be computed on the device)
  const uint64_t* base = nullptr;       // padded start, a multiple of kTile
  const uint32_t* first_tile = nullptr; // nseg + 1 entries
  // Optional: the segment of every tile (ntiles entries, launch_tile_seg),
  // which saves each tile a binary search over first_tile.
  const uint32_t* tile_seg = nullptr;
  uint32_t nseg = 0;
  uint32_t ntiles = 0;
};

// Where each phase reads and writes (all device pointers; see the launchers).
struct StatsArgs {
  SegPlan plan;
  uint64_t* hdr = nullptr;        // [nseg][2] = {nrows, nnz}
  ans_quantities* q = nullptr;    // [nseg]
  const uint64_t* keys = nullptr; // sorted keys (padded space)
  uint32_t* col_ids = nullptr;    // at base[s]
  uint64_t* vals = nullptr;       // at base[s]
  uint32_t* vals32 = nullptr;     // optional uint32 copy of vals (column pass input), at base[s]
  uint32_t* row_ids = nullptr;    // at base[s]
  uint64_t* row_ptr = nullptr;    // at base[s] + s  (nrows + 1 entries)
  uint64_t* run_start = nullptr;  // at base[s] + s  (nnz + 1 entries); null = identity
  uint64_t* row_pos = nullptr;    // at base[s] + s  (nrows + 1 entries); null = row_ptr
  const uint64_t* pre = nullptr;  // exclusive value prefix at base[s] + s; null = identity
  uint64_t* lookback = nullptr;   // [ntiles] status words (zeroed)
  uint32_t* ticket = nullptr;     // zeroed counter
  uint32_t* col_hist = nullptr;   // [nseg][kColPasses][kRadix] destination digit counts, zero on entry
  uint64_t* ulen = nullptr;       // [nseg] links per segment (written for the column sort)
  uint64_t* col_st0 = nullptr;    // first column pass's status words (zeroed here)
  uint32_t* col_tickets = nullptr;  // the column passes' tickets (zeroed here)
  uint32_t* err = nullptr;
  // Optional (window mode): each link's key (src << 32 | dst) also written
  // at base[s] + u, beside its column id -- with the link values this is the
  // time sum's input run of the window, read in place by the merge.
  uint64_t* sum_keys = nullptr;
  // Optional: each link's mixed destination fmix32(dst) written at base[s] +
  // u (the column sort's keys when a time sum's column statistics group
  // destinations by hash); the column histograms then count its bytes.
  uint32_t* col_hkeys = nullptr;
  int mode = 0;
};

enum StatsMode : int {
  kModeWindow = 0,  // vals = run lengths; row sums = packets per row
  kModeSum = 1,     // vals = sums of sorted input values; pre = their prefix
  kModeMatrix = 2,  // vals given; run_start identity; row_pos = row_ptr
};

// Per-tile summary of the column runs that touch the tile's boundaries.
struct ColBnd {
  uint64_t lead_len, lead_sum;  // items before the tile's first head (all items if it has none)
  uint64_t tail_len, tail_sum;  // from the tile's last head to its end
  uint32_t has_head, pad;
};

// Per-window hash tables of the hash aggregation path (device pointers):
// window s owns slots [off[s], off[s] + 2^lg[s]) of keys/cnt; special[s]
// counts the all-ones key, which marks empty slots; the slots window s
// claimed are listed at claims + base[s] (its padded start), nclaim[s] of
// them.
struct HashTabs {
  uint64_t* keys = nullptr;
  uint32_t* cnt = nullptr;
  const uint64_t* off = nullptr;
  const uint32_t* lg = nullptr;
  uint64_t* special = nullptr;
  uint32_t* claims = nullptr;
  uint64_t* nclaim = nullptr;
};

// Matrix descriptor for the time-sum gather.
struct MatDesc {
  const uint32_t* row_ids;
  const uint64_t* row_ptr;
  const uint32_t* col_ids;
  const uint64_t* vals;
  const uint64_t* hdr;  // {nrows, nnz}
  uint64_t neg = 0;     // 1: the matrix enters a combination with sign -1 (values negated mod 2^64)
};

// Outputs of the device-side batch planner (launch_plan): the window plan
// (in_off, len, base: nseg entries; first_tile: nseg + 1), optionally the
// hash path's table plan (tab_lg, tab_base), a copy of the padded starts in
// the per-window matrix block (blk_base), the offset and length of all the
// batch's packets as one segment (pk_in_off, pk_len), and the time sum's matrix
// descriptors (md) over the statistics arrays row_ids / row_ptr / col_ids /
// vals / hdr.  Null pointers are skipped.
struct DevPlanOut {
  uint64_t* in_off = nullptr;
  uint64_t* len = nullptr;
  uint64_t* base = nullptr;
  uint32_t* first_tile = nullptr;
  uint32_t* tab_lg = nullptr;
  uint64_t* tab_base = nullptr;
  uint64_t* blk_base = nullptr;
  uint64_t* pk_in_off = nullptr;  // the batch's packets as one segment: its offset and length
  uint64_t* pk_len = nullptr;
  MatDesc* md = nullptr;
  const uint32_t* row_ids = nullptr;
  const uint64_t* row_ptr = nullptr;
  const uint32_t* col_ids = nullptr;
  const uint64_t* vals = nullptr;
  const uint64_t* hdr = nullptr;
};

// ---- window quantities by on-chip hashing (ans_winhash.cu) -----------------
constexpr uint32_t kHqMaxPackets = 1u << 18;  // larger windows are sorted
// Per-window accumulator of the hashed statistics (zeroed before the batch):
// the link stage's distinct links and largest count, then per stage (0 =
// sources, 1 = destinations) the distinct keys, the largest number of links
// of a key (fan-out / fan-in) and the largest packet count of a key; fail =
// some table overflowed (the window is sorted instead); nlinks = the
// window's distinct links appended so far.
struct HqWin {
  unsigned long long links, max_link;
  unsigned long long keys[2], max_links[2], max_packets[2];
  uint32_t fail, nlinks;
};
// Device buffers of the hashed statistics (keys: packets regrouped by link
// partition, at each window's padded base; lsrc / ldst / lcnt: the windows'
// distinct links; pkey[st] / pval[st]: links regrouped by source (st = 0) or
// destination (1) partition; lstart: 65 link-partition starts per window;
// kstart: 65 key-partition starts per window and stage, stage 0 first;
// sort_len: the plan lengths the sort path then uses).
struct HqBufs {
  uint64_t* keys = nullptr;
  uint32_t* lsrc = nullptr;
  uint32_t* ldst = nullptr;
  uint32_t* lcnt = nullptr;
  uint32_t* pkey[2] = {nullptr, nullptr};
  uint32_t* pval[2] = {nullptr, nullptr};
  uint32_t* lstart = nullptr;
  uint32_t* kstart = nullptr;
  HqWin* win = nullptr;
  uint64_t* sort_len = nullptr;
  uint32_t* items = nullptr;    // work-item prefix of the counting steps (2 * nseg + 1)
  uint32_t* counter = nullptr;  // their queue counter
};
// The hashed statistics of every window of p (win zeroed by the caller), in
// five launches, stage 0 .. 4: regroup packets by link partition, count
// links, regroup the distinct links by source and destination partition,
// count sources and destinations, set sort_len.  The quantities are written
// by launch_hq_write once the sort path has run over sort_len.
cudaError_t launch_hq_stage(int stage, const SegPlan& p, const uint32_t* src, const uint32_t* dst, const HqBufs& b,
                            cudaStream_t st);
cudaError_t launch_hq_write(const SegPlan& p, const HqWin* win, ans_quantities* q, cudaStream_t st);

// ---- row partition across ranks (ans_split.cu) ----------------------------
constexpr uint32_t kMaxSplitParts = 64;
// The owners' pieces (device pointers per owner; hdr = {nrows, nnz}).
struct SplitOut {
  uint32_t* row_ids[kMaxSplitParts];
  uint64_t* row_ptr[kMaxSplitParts];
  uint32_t* col_ids[kMaxSplitParts];
  uint64_t* vals[kMaxSplitParts];
  uint64_t* hdr[kMaxSplitParts];
};
// Row tiles of a matrix of nrows rows (8192 rows each).
uint32_t split_row_tiles(uint64_t nrows);
// Per tile and owner the rows (trows) and links (tlinks) of a DCSR, turned
// into exclusive offsets over the tiles; totals[2 o] / [2 o + 1] = owner o's
// rows / links.  trows and tlinks hold split_row_tiles(nrows) * nparts entries.
cudaError_t launch_split_count(uint64_t nrows, const uint32_t* row_ids, const uint64_t* row_ptr, uint32_t nparts,
                               uint32_t* trows, uint64_t* tlinks, uint64_t* totals, cudaStream_t st);
// The owners' pieces written (rows in order, each row's links after its
// first one); rown / rlink: nrows words of scratch each.
cudaError_t launch_split_fill(uint64_t nrows, uint64_t nnz, const uint32_t* row_ids, const uint64_t* row_ptr,
                              const uint32_t* col_ids, const uint64_t* vals, uint32_t nparts, const uint32_t* trows,
                              const uint64_t* tlinks, const uint64_t* totals, uint32_t* rown, uint64_t* rlink,
                              const SplitOut& out, cudaStream_t st);

// ---- launcher (ans_plan.cu) ------------------------------------------------
// Plan the nseg windows [d_offsets[s], d_offsets[s+1]) on the device (one
// CTA; nseg > 0).  Invalid offsets, or more than `cap` packets in all, give
// every window length 0 and set kErrPlan in err[0].
cudaError_t launch_plan(const uint64_t* d_offsets, uint32_t nseg, uint64_t cap, const DevPlanOut& o, uint32_t* err,
                        cudaStream_t st);

// Record `msg` as the calling thread's ans_last_error() text; returns code.
int set_last_error(int code, const std::string& msg);

// ---- launchers (ans_sort.cu) ---------------------------------------------
// Pack (src, dst) into keys src << 32 | dst, build per-segment digit
// histograms of all passes, zero the pass-0 status words (sub * kRadix per
// tile, for key passes over `sub` sub-tiles per tile) and the tickets.
cudaError_t launch_pack_hist(const SegPlan& p, const uint32_t* src, const uint32_t* dst,
                             uint64_t* keys, uint32_t* seg_hist, uint64_t* status0,
                             uint32_t* tickets, cudaStream_t st, uint32_t sub = 1);
// Sub-tiles per tile of a key-pass configuration.
constexpr uint32_t key_subtiles(const SortCfg& cfg) { return cfg.threads == 256 ? 2u : 1u; }
// One onesweep digit pass (stable), optionally carrying uint64 values.
cudaError_t launch_onesweep(const SegPlan& p, int pass, const uint64_t* kin, uint64_t* kout,
                            const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                            uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket,
                            uint32_t* err, const SortCfg& cfg, cudaStream_t st);
// The one packet sort of a batch that also yields its windows' order
// (agg_path 3): a digit pass over the 64-bit keys carrying each packet's
// 16-bit window id, and a stable digit pass over the window ids carrying the
// keys (pass | kPassStable for its first pass; with `remap`, a key whose
// window is w lands at its sorted place + remap[w]; a null kout drops the
// ids).  Both in the 4096-key sub-tile shape with cfg's ranking mode.
cudaError_t launch_onesweep_wid(const SegPlan& p, int pass, const uint64_t* kin, uint64_t* kout,
                                const uint16_t* vin, uint16_t* vout, const uint32_t* seg_hist, uint64_t* st_cur,
                                uint64_t* st_next, uint32_t* ticket, uint32_t* err, const SortCfg& cfg,
                                cudaStream_t st);
cudaError_t launch_onesweep_regroup(const SegPlan& p, int pass, const uint16_t* kin, uint16_t* kout,
                                    const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                                    uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                    const SortCfg& cfg, const uint64_t* remap, uint32_t nremap, cudaStream_t st);
// Window ids of the windows of `p` over their packets in the batch's
// one-segment packet order, each window's offset from that order (sorted by
// window) to its padded base, and the ids' two digit histograms.
cudaError_t launch_wid_fill(const SegPlan& p, const uint64_t* pk_in_off, uint16_t* wid, uint64_t* shift,
                            uint32_t* hist, cudaStream_t st);
// One digit pass over 32-bit destination keys carrying uint64 counts.
cudaError_t launch_onesweep_col(const SegPlan& p, int pass, const uint32_t* kin, uint32_t* kout,
                                const uint64_t* vin, uint64_t* vout, const uint32_t* seg_hist,
                                uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                const SortCfg& cfg, cudaStream_t st);
// The same with uint32 counts (window matrices: every count fits 31 bits).
cudaError_t launch_onesweep_col32(const SegPlan& p, int pass, const uint32_t* kin, uint32_t* kout,
                                  const uint32_t* vin, uint32_t* vout, const uint32_t* seg_hist,
                                  uint64_t* st_cur, uint64_t* st_next, uint32_t* ticket, uint32_t* err,
                                  const SortCfg& cfg, cudaStream_t st);
// Gather the stored links of k matrices into (key, value) pairs at their
// concatenation offsets, accumulating the time-sum segment's digit histograms
// (sum_hist, zeroed by the caller; null: none) and zeroing the sum sort's
// first status words and tickets.  status0 needs p.ntiles * kRadix words.
cudaError_t launch_gather(const SegPlan& p, const MatDesc* mats, const uint64_t* cat_off, uint64_t* keys,
                          uint64_t* vals, uint32_t* sum_hist, uint64_t* status0, uint32_t* tickets,
                          cudaStream_t st);
// Exclusive prefix of the matrices' nnz (hdr[1]) -> cat_off[0..k), nnz ->
// lens, their sum -> *total and cat_off[k].
cudaError_t launch_count_prefix(const MatDesc* mats, uint32_t k, uint64_t* cat_off, uint64_t* lens,
                                uint64_t* total, cudaStream_t st);

// ---- launchers (ans_cluster.cu) ------------------------------------------
// Sort the keys src << 32 | dst of every segment seg_ids[0..nclusters) (or
// 0..nclusters if seg_ids is null; each at most kClusterWindowMax items) on
// chip, one 8-CTA cluster per segment, writing them to keys at base[s]; also
// zeroes tickets[0..32).  cfg.threads is 512 or 1024, cfg.rank as for onesweep.
cudaError_t launch_cluster_sort(const SegPlan& p, const uint32_t* seg_ids, uint32_t nclusters, const uint32_t* src,
                                const uint32_t* dst, uint64_t* keys, uint32_t* tickets, const SortCfg& cfg,
                                cudaStream_t st);
// Clusters of the window sort that fit on `device` at once (0: unavailable).
int cluster_sort_clusters(int device);

// ---- launchers (ans_hash.cu) ---------------------------------------------
// Count the packets of every window of `p` into its hash table (tables clean
// on entry; special and nclaim zeroed), listing the claimed slots.
cudaError_t launch_hash_insert(const SegPlan& p, const uint32_t* src, const uint32_t* dst, const HashTabs& h,
                               uint32_t* err, cudaStream_t st);
// pc: the window plan with len = h.nclaim.  Move every window's (key, count)
// pairs out of its table to okeys/ovals at base[s], their number to ulen[s],
// their digit histograms to seg_hist (zeroed); empties the claimed slots;
// zeroes the first status words of pc's tiles and tickets[0..32).
cudaError_t launch_hash_compact(const SegPlan& pc, const HashTabs& h, uint64_t* ulen, uint64_t* okeys,
                                uint64_t* ovals, uint32_t* seg_hist, uint64_t* status0, uint32_t* tickets,
                                cudaStream_t st);

// ---- launchers (ans_merge.cu) --------------------------------------------
// One round of pairwise merges of sorted (key, value) runs: runs of 2^round
// matrices of the concatenation described by cat_off (k + 1 dense starts on
// the device) are merged pairwise from kin/vin into kout/vout.  Matrix m's
// items sit at run_base[m] (device, k entries, nondecreasing, with room for
// each matrix's items before the next one's base; null: at cat_off[m]); a
// merged run is written from the base of its first matrix, so the last
// round leaves all items dense from run_base[0] = 0.  total_cap bounds
// cat_off[k] (it sizes the grid).
// `tile`: output positions per CTA, 4096 or 2048.
cudaError_t launch_merge(const uint64_t* cat_off, const uint64_t* run_base, uint32_t k, uint64_t total_cap, int round,
                         const uint64_t* kin, const uint64_t* vin, uint64_t* kout, uint64_t* vout, int tile,
                         cudaStream_t st);

// ---- launchers (ans_stats.cu) --------------------------------------------
// Signed combinations: flags[u] = (vals[u] != 0) over the single segment of
// p (a value of 2^61 or more, a negative count, sets kErrNegative), then the
// nonzero (key, value) pairs moved to kout/vout at their exclusive flag
// prefix pos[u], their number to *count.
cudaError_t launch_nonzero_flags(const SegPlan& p, const uint64_t* vals, uint64_t* flags, uint32_t* err,
                                 cudaStream_t st);
cudaError_t launch_scatter_nonzero(const SegPlan& p, const uint64_t* kin, const uint64_t* vin, const uint64_t* pos,
                                   uint64_t* kout, uint64_t* vout, uint64_t* count, cudaStream_t st);
// Run-length reduce sorted keys into DCSR structure (col_ids, row_ids,
// row_ptr) plus run/row start positions; writes hdr.
cudaError_t launch_rle(const StatsArgs& a, cudaStream_t st);
// Exclusive prefix of uint64 values per segment (len + 1 entries at base+s),
// mod 2^62.
cudaError_t launch_scan_u64(const SegPlan& p, const uint64_t* in, uint64_t* out,
                            uint64_t* lookback, uint32_t* ticket, uint32_t* err, cudaStream_t st);
// Values, row statistics, link maximum, and the destination digit histograms
// for the column pass.
cudaError_t launch_finish(const StatsArgs& a, cudaStream_t st);
// Column statistics from destination-sorted (dst, count) pairs of the
// segments of `p` (p.len = links per segment): unique destinations, max
// fan-in, max destination packets.  bnd holds one record per tile.
cudaError_t launch_colstat(const SegPlan& p, const uint32_t* keys, const uint64_t* vals, ColBnd* bnd,
                           ans_quantities* q, cudaStream_t st);
cudaError_t launch_colstat32(const SegPlan& p, const uint32_t* keys, const uint32_t* vals, ColBnd* bnd,
                             ans_quantities* q, cudaStream_t st);
// Canonical-DCSR check of an imported matrix; ORs failure bits into *bad.
cudaError_t launch_check_dcsr(uint64_t nrows, uint64_t nnz, const uint32_t* row_ids, const uint64_t* row_ptr,
                              const uint32_t* col_ids, const uint64_t* vals, uint32_t* bad, cudaStream_t st);
// CTAs per window launch_colhash uses for a batch of nseg windows (its
// launch shape: part of the key of a cached batch graph).
uint32_t colhash_ctas(uint32_t nseg);
// Window column statistics from a shared-memory hash of destinations, one
// CTA per window of p (links: col_ids / vals32 at base[s], ulen[s] of them);
// a window whose distinct destinations fit gets its three column quantities
// in q and ulen[s] = 0 (the column sort then skips it).
cudaError_t launch_colhash(const SegPlan& p, uint64_t* ulen, const uint32_t* col_ids, const uint32_t* vals32,
                           ans_quantities* q, cudaStream_t st);
// One bounded look-back wait (both forms: the single-thread walk of the
// radix passes and the warp walk of the run reductions and scans) for the
// predecessor of tile 1 of a chain whose tile 0 never publishes (st: two
// words, zero on entry).  Each wait gives up after the context's poll limit
// and sets kErrLookback in err[0].
cudaError_t launch_wait_probe(const uint64_t* st, uint32_t* err, cudaStream_t stream);
// Per-window accumulator of the partitioned column hash (zeroed before it).
struct ColPartAcc {
  unsigned long long count, max_fanin, max_packets;
  uint32_t fail, done;
};
// Window column statistics of the windows launch_colhash left (ulen[s] > 0)
// with more than 8192 and at most 32 x 8192 links (window index below 2^27):
// their destinations split by a hash into partitions (the links regrouped
// by partition into pkeys/pvals at the window's base, partition starts in
// bstart[s][0..33), the (window, partition) items listed in items[nseg *
// 32]), one shared-memory table per partition, counted by one persistent
// CTA per SM; windows whose partitions all fit get their three column
// quantities and ulen[s] = 0.  acc: nseg + 1 zeroed accumulators (the last
// one counts and hands out the items).
cudaError_t launch_colhash_part(const SegPlan& p, uint64_t* ulen, const uint32_t* col_ids, const uint32_t* vals32,
                                uint32_t* pkeys, uint32_t* pvals, uint32_t* bstart, ColPartAcc* acc, uint32_t* items,
                                ans_quantities* q, cudaStream_t st);
// Column statistics of one segment of *len links (a time sum) whose mixed
// destinations `keys` (fmix32 of each destination, with uint32 counts
// `vals32`) have been sorted by their low 16 bits (two column passes): the
// 2^16 groups counted in shared-memory tables by persistent CTAs (groups of
// more than kHGroupPartLinks links in parts, merged afterwards).  If every
// table fits, the segment's three column quantities go to *q and *len
// becomes 0; otherwise nothing is published and the column sort goes on.
// The buffers (HGroupBufs, acc zeroed) hold up to max_hparts parts of cut
// groups; more fail the hash the same way.
constexpr uint32_t kHGroups = 1u << 16;
constexpr uint32_t kHGroupBounds = kHGroups + 1;
constexpr uint32_t kHGroupPartLinks = 1u << 16;
constexpr uint64_t kHGroupMinLinks = 1ull << 24;  // smaller sums take the column sort
constexpr uint32_t kHGroupPartWords = 3 * ((1u << 13) / 4 * 3 + 1);  // a part's entries: its table's fill + 1
struct HGroupBufs {
  uint32_t* bnd = nullptr;         // [kHGroupBounds] group starts
  uint32_t* item_start = nullptr;  // [kHGroupBounds] first work item of each group
  uint32_t* hpart = nullptr;       // [kHGroupBounds] first part (of cut groups) of each group
  uint32_t* heavy = nullptr;       // [kHGroups] the cut groups
  uint32_t* meta = nullptr;        // [4] items, cut groups, their parts
  uint32_t* hcnt = nullptr;        // [max_hparts] entries of each part
  uint32_t* hbuf = nullptr;        // [max_hparts][kHGroupPartWords] (key, links, packets) entries
  ColPartAcc* acc = nullptr;       // [3] zeroed: quantities + fail + CTAs done; item and group counters
};
cudaError_t launch_hgroup_stats(const uint32_t* keys, const uint32_t* vals32, uint64_t* len, const HGroupBufs& b,
                                uint32_t max_hparts, ans_quantities* q, cudaStream_t st);
// tile_seg[t] = the segment of tile t of `p` (its first_tile searched once
// per tile), for SegPlan::tile_seg.
cudaError_t launch_tile_seg(const SegPlan& p, uint32_t* tile_seg, cudaStream_t st);
// Zero `bytes` bytes at p (4-byte aligned pointer); a kernel, unlike a memset.
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
// Copies of small arrays by a kernel instead of the copy engines (so they
// never queue behind other streams' bulk transfers): item i copies bytes from
// src to dst, either of which may be page-locked host memory (read or written
// in place) or device memory.  At most kSmallCopyItems items per launch.
constexpr int kSmallCopyItems = 16;
struct SmallCopyItem {
  void* dst;
  const void* src;
  uint64_t bytes;
};
struct SmallCopyBatch {
  uint32_t n = 0;
  SmallCopyItem it[kSmallCopyItems];
};
cudaError_t launch_small_copy(const SmallCopyBatch& b, cudaStream_t st);
// Windows in their own arrays gathered into one contiguous pair of device
// arrays: window w's len packets from (src, dst) -- device or page-locked
// host memory, read in place -- to gsrc/gdst + off.
struct GatherWin {
  uint64_t src, dst, off, len;
};
cudaError_t launch_gather_windows(const GatherWin* wins, uint32_t nwin, uint32_t* gsrc, uint32_t* gdst,
                                  cudaStream_t st);
// Scratch guards (debug mode): kGuardBytes after every region of a guarded
// layout hold a fixed pattern, written before a batch's kernels and compared
// after them; launch_guards fills (err == NULL) or checks the guards at the
// given device addresses (a mismatch sets kErrGuard in err[0]).
constexpr size_t kGuardBytes = 256;
constexpr int kGuardsPerLaunch = 64;
struct GuardList {
  uint32_t n = 0;
  uint64_t addr[kGuardsPerLaunch];
};
cudaError_t launch_guards(const GuardList& g, uint32_t* err, cudaStream_t st);
// Overwrites the first word of the guard at `guard`, as a write one word past
// the end of the region before it would: a later check must report it.
cudaError_t launch_guard_probe_write(uint64_t* guard, cudaStream_t st);
// *dst = *src for one device word, by a kernel.
cudaError_t launch_copy_word(uint32_t* dst, const uint32_t* src, cudaStream_t st);
// Zero-length segments: row_ptr[0] = 0 and hdr = {0, 0}.
cudaError_t launch_empty_fixup(const StatsArgs& a, cudaStream_t st);

// ---- device helpers --------------------------------------------------------
#ifdef __CUDACC__

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Segment of a tile: the last s with first_tile[s] <= t (empty segments are
// skipped because their first_tile equals the next one's).
__device__ __forceinline__ uint32_t find_seg(const SegPlan& p, uint32_t t) {
  if (p.tile_seg) return p.tile_seg[t];
  uint32_t lo = 0, hi = p.nseg;  // first_tile[lo] <= t < first_tile[hi]
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (p.first_tile[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Window `seg`'s packet arrays: its own addresses when the plan has them,
// else its offset into the one input stream (src, dst).
__device__ __forceinline__ void window_inputs(const SegPlan& p, uint32_t seg, const uint32_t* src,
                                              const uint32_t* dst, const uint32_t** ws, const uint32_t** wd) {
  if (p.src_at) {
    *ws = reinterpret_cast<const uint32_t*>(p.src_at[seg]);
    *wd = reinterpret_cast<const uint32_t*>(p.dst_at[seg]);
  } else {
    *ws = src + p.in_off[seg];
    *wd = dst + p.in_off[seg];
  }
}

struct Tile {
  uint32_t seg, j;     // segment and tile index within it
  uint64_t len;        // segment length
  uint64_t base;       // padded segment start
  uint64_t start;      // first item of the tile within the segment
  uint32_t count;      // items in this tile (0 if the segment ended before it)
  uint32_t seg_tiles;  // tiles reserved for the segment
};

__device__ __forceinline__ Tile make_tile(const SegPlan& p, uint32_t t) {
  Tile r;
  r.seg = find_seg(p, t);
  r.j = t - p.first_tile[r.seg];
  r.seg_tiles = p.first_tile[r.seg + 1] - p.first_tile[r.seg];
  r.len = p.len[r.seg];
  r.base = p.base[r.seg];
  r.start = (uint64_t)r.j * kTile;
  r.count = r.len > r.start ? (uint32_t)umin64(kTile, r.len - r.start) : 0u;
  return r;
}

// Broadcast a Tile computed by thread 0 through shared memory.
__device__ __forceinline__ Tile block_tile(const SegPlan& p, uint32_t t, Tile* sm) {
  if (threadIdx.x == 0) *sm = make_tile(p, t);
  __syncthreads();
  return *sm;
}

// Take a ticket (tiles are processed in ticket order so that look-back only
// waits on tiles that have started).
__device__ __forceinline__ uint32_t block_ticket(uint32_t* counter, uint32_t* sm) {
  if (threadIdx.x == 0) *sm = atomicAdd(counter, 1u);
  __syncthreads();
  return *sm;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xffffffffu, v, o);
    v = y > v ? y : v;
  }
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Bounded decoupled look-back for one value chain.  `st` points at tile 0 of
// the chain's status array with `stride` words between consecutive tiles;
// `first` is the first tile of the segment, `t` this tile (t > first).
// Returns the exclusive prefix; on timeout flags kErrLookback and returns the
// partial sum (never larger than the true prefix, so indexes stay in range).
// Poll limit of the bounded waits of the context whose error word is `err`.
__device__ __forceinline__ uint32_t wait_limit(const uint32_t* err) {
  const uint32_t l = err[1];
  return l ? l : kSpinLimit;
}

__device__ __forceinline__ uint64_t lookback(const uint64_t* st, uint32_t stride, uint32_t first,
                                             uint32_t t, uint32_t* err) {
  uint64_t excl = 0;
  uint32_t q = t - 1;
  uint32_t spins = 0;
  uint32_t limit = 0;  // read at the first wait only
  while (true) {
    uint64_t v = ld_relaxed(st + (uint64_t)q * stride);
    uint64_t f = v & ~kValMask;
    if (f == 0) {
      if (spins == 0) limit = wait_limit(err);
      if (++spins > limit) {
        atomicOr(err, (uint32_t)kErrLookback);
        break;
      }
      if (spins > 64) __nanosleep(spins > 4096 ? 1000 : 64);
      continue;
    }
    excl += v & kValMask;
    if (f == kFlagPre || q == first) break;
    --q;
  }
  return excl;
}

// The same for a whole warp (all 32 lanes call it; every lane gets the
// result): lane i reads the status of tile q - i, so one round trip covers 32
// predecessors.  The nearest tile with its inclusive prefix ends the walk
// (tiles before `first` count as such a tile with value 0); if a nearer tile
// has not published yet, the window is read again.
__device__ __forceinline__ uint64_t warp_lookback(const uint64_t* st, uint32_t stride, uint32_t first, uint32_t t,
                                                  uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t excl = 0;
  uint32_t q = t - 1;  // newest tile not yet added; q >= first
  uint32_t spins = 0;
  uint32_t limit = 0;  // read at the first wait only
  while (true) {
    const uint64_t v = lane <= q - first ? ld_relaxed(st + (uint64_t)(q - lane) * stride) : kFlagPre;
    const uint64_t f = v & ~kValMask;
    const uint32_t pre = __ballot_sync(0xffffffffu, f == kFlagPre);
    const uint32_t none = __ballot_sync(0xffffffffu, f == 0);
    const int p = pre ? __ffs(pre) - 1 : 32;              // nearest tile with its prefix
    const uint32_t upto = p == 32 ? 0xffffffffu : (2u << p) - 1u;  // lanes 0..p
    if (none & upto) {                                     // a nearer tile is not ready
      if (spins == 0) limit = wait_limit(err);
      if (++spins > limit) {
        if (lane == 0) atomicOr(err, (uint32_t)kErrLookback);
        return excl;
      }
      if (spins > 64) __nanosleep(spins > 4096 ? 1000 : 64);
      continue;
    }
    excl += warp_sum((uint64_t)(lane <= (uint32_t)p ? (v & kValMask) : 0ull));
    if (p < 32) return excl;
    q -= 32;  // 32 aggregates added; look further back
  }
}

// ---- thread-block cluster helpers (shared::cluster addresses are 32-bit)
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// Shared-memory address of the same location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ uint64_t ld_cluster_u64(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_cluster(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
// All threads of all CTAs of the cluster; orders shared-memory writes before
// the barrier (local and remote) with reads after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Block-wide exclusive scan of one uint32 per thread for the first 256
// threads (others pass 0 and ignore the result).  `tmp` needs 8 words.
__device__ __forceinline__ uint32_t scan256_excl(uint32_t v, uint32_t* tmp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (warp < 8 && lane == 31) tmp[warp] = x;
  __syncthreads();
  uint32_t off = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    uint32_t s = tmp[w];
    off += (w < warp) ? s : 0u;
    tot += s;
  }
  if (total) *total = tot;
  __syncthreads();
  return off + x - v;
}

// The same over uint64 (two 32-bit counts packed in one word are scanned
// together as long as neither half's total overflows).  `tmp` needs 8 words.
__device__ __forceinline__ uint64_t scan256_excl64(uint64_t v, uint64_t* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (warp < 8 && lane == 31) tmp[warp] = x;
  __syncthreads();
  uint64_t off = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) off += (w < warp) ? tmp[w] : 0ull;
  __syncthreads();
  return off + x - v;
}

// Peer mask of lanes holding the same 8-bit digit: one __match_any_sync, or
// eight ballots (one per digit bit) intersected.  `valid` lanes only.
template <int kRank>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid) {
  if constexpr (kRank == kRankMatch) {
    return __match_any_sync(0xffffffffu, valid ? d : (uint32_t)kRadix);
  } else {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      const uint32_t ones = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? ones : ~ones;
    }
    return peers;
  }
}

#endif  // __CUDACC__

}  // namespace ans
