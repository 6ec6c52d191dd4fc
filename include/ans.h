/*
 * ans.h -- C ABI of the GB300 anonymized-network-sensing library (libans.so).
 *
 * The library turns windows of anonymized (src, dst) uint32 packet pairs into
 * hypersparse 2^32 x 2^32 traffic matrices stored as DCSR, sums windows over
 * time, and reduces matrices to the Graph Challenge network quantities.  Every
 * result is an exact integer.
 *
 * Definitions (paper: Table I, Sec. IV-B, Sec. IV-C):
 *   A(i, j)  = number of packets from source i to destination j in a window
 *              (Table I caption; rows are sources, columns destinations).
 *   DCSR     = nonempty rows ascending (row_ids), row_ptr = exclusive prefix of
 *              per-row nonzero counts (the paper's "degrees", Sec. IV-B), column
 *              ids ascending within a row ("edges"), uint64 values ("weights").
 *   time sum = (sum_t A_t)(i, j) = sum_t A_t(i, j)  (Table I: A_t at time t).
 *
 * Conventions shared by every entry point:
 *   - Return value: ANS_OK (0) or a negative ANS_ERR_* code.  ans_last_error()
 *     gives a human-readable detail for the calling thread.
 *   - Pointers prefixed d_ are device pointers on the context's device;
 *     h_ are host pointers.  Inputs are borrowed: they must stay valid and
 *     unmodified until the work of the call has completed on its stream.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are stream-ordered and asynchronous unless a comment says otherwise.
 *     Calls that share one context must be ordered (one stream, or the caller
 *     orders them): the context's scratch memory is reused from call to call.
 *     A batch may run part of its work on a second stream of the context
 *     (the time sum's merge rounds beside the window column pass); that work
 *     is forked from and joined back into `stream`, so completion on
 *     `stream` covers it.
 *   - Matrices are owned by the caller once returned and released with
 *     ans_matrix_free().  A matrix keeps its memory alive independently of
 *     the context's scratch.
 *   - Every packet is valid (the paper does not say what makes a packet
 *     invalid), so a window's valid-packet count is its length.  Addresses 0
 *     and 0xFFFFFFFF are ordinary.  Self-links (src == dst) are ordinary
 *     diagonal entries.  Quantities of an empty matrix are all 0.
 *   - Limits: a window holds at most 2^31 - 1 packets; a time sum combines at
 *     most 2^31 - 1 stored links per call.
 */
#ifndef ANS_H
#define ANS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define ANS_OK               0
#define ANS_ERR_INVALID_ARG (-1)  /* bad pointer, size or flag */
#define ANS_ERR_BUDGET      (-2)  /* the call would exceed the context's memory budget */
#define ANS_ERR_OOM         (-3)  /* the allocator failed */
#define ANS_ERR_CUDA        (-4)  /* a CUDA runtime call failed */
#define ANS_ERR_TIMEOUT     (-5)  /* ans_wait ran out of time, or a bounded device wait gave up */
#define ANS_ERR_INTERNAL    (-6)  /* a device-side consistency check failed */

/* Flags of ans_batch_submit. */
#define ANS_BATCH_MATRICES   0x1u /* return one DCSR matrix per window in per_window[] */
#define ANS_BATCH_SUM        0x2u /* return the time sum of all windows in *sum */
#define ANS_BATCH_SYNC       0x4u /* block until the batch has completed */

typedef struct ans_ctx ans_ctx;       /* opaque: device, allocator, budget, scratch */
typedef struct ans_matrix ans_matrix; /* opaque: one DCSR matrix in device memory */
typedef uint64_t ans_ticket;          /* completion handle of an asynchronous batch */

/* The nine network quantities of one matrix, in this order (Table I rows and
 * the maxima of Sec. IV-C).  Fan-out/fan-in are the largest per-row/per-column
 * nonzero counts (Table I's C++ column: max of the per-row degrees). */
typedef struct {
    uint64_t valid_packets;           /* sum_ij A(i,j) */
    uint64_t unique_links;            /* #{(i,j) : A(i,j) > 0} */
    uint64_t max_link_packets;        /* max_ij A(i,j) */
    uint64_t unique_sources;          /* #{i : row i nonempty} */
    uint64_t max_source_packets;      /* max_i sum_j A(i,j) */
    uint64_t max_source_fanout;       /* max_i #{j : A(i,j) > 0} */
    uint64_t unique_destinations;     /* #{j : column j nonempty} */
    uint64_t max_destination_packets; /* max_j sum_i A(i,j) */
    uint64_t max_destination_fanin;   /* max_j #{i : A(i,j) > 0} */
} ans_quantities;

/* Device allocator hooks.  alloc returns NULL on failure; both receive the
 * stream the memory is used on and the `user` pointer given at creation. */
typedef void* (*ans_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*ans_free_fn)(void* ptr, void* stream, void* user);

/* Create a context on CUDA device `device`.
 * mem_budget_bytes: ceiling on the device memory the context holds at once
 *   (scratch plus live matrices); 0 = no ceiling.  A call that would exceed it
 *   fails with ANS_ERR_BUDGET and leaves no work queued.
 * alloc/free: both NULL selects cudaMallocAsync/cudaFreeAsync; otherwise both
 *   must be given.  Errors: ANS_ERR_INVALID_ARG, ANS_ERR_CUDA. */
int ans_ctx_create(ans_ctx** out, int device, size_t mem_budget_bytes,
                   ans_alloc_fn alloc, ans_free_fn free_fn, void* user);

/* Wait for the context's outstanding work and release its scratch and
 * tickets; the handle is invalid afterwards.  Matrices created from the
 * context stay valid: the context's remaining state (its free hook and user
 * pointer included, which must stay usable) is released with the last of
 * them.  Destroying a context twice is ANS_ERR_INVALID_ARG (while matrices
 * keep it alive) or undefined. */
int ans_ctx_destroy(ans_ctx* ctx);

/* Traffic matrix of one window (Table I caption): A(i,j) = #{k : d_src[k] == i,
 * d_dst[k] == j} for k < n, as DCSR with uint64 counts.  d_src/d_dst: device
 * arrays of n uint32 (any alignment).  n == 0 gives an empty matrix.  The
 * matrix's quantities are computed in the same pass and are returned by
 * ans_matrix_quantities() without further device work.
 * Errors: ANS_ERR_INVALID_ARG (NULL pointers with n > 0, n >= 2^31),
 * ANS_ERR_BUDGET, ANS_ERR_OOM, ANS_ERR_CUDA. */
int ans_build_window(ans_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                     ans_matrix** out, void* stream);

/* Time sum of k matrices (Table I: A_t indexed by t): (sum_t A_t)(i,j) =
 * sum_t A_t(i,j), as a new DCSR matrix.  The inputs are only read; they may
 * come from different calls on the same device.  k == 0 gives an empty matrix.
 * Errors: ANS_ERR_INVALID_ARG, ANS_ERR_BUDGET, ANS_ERR_OOM, ANS_ERR_CUDA. */
int ans_sum_windows(ans_ctx* ctx, const ans_matrix* const* mats, size_t k, ans_matrix** out,
                    void* stream);

/* Signed time sum: out = sum_i signs[i] * A_i with signs[i] = +1 or -1 --
 * the exact update of a sliding time sum (Table I's A_t summed over t) when
 * windows leave it.  Links whose counts cancel are dropped, so the result is
 * canonical DCSR again.  Every combined count must be >= 0 (and every
 * count and partial sum below 2^61): a negative one makes ans_matrix_view /
 * ans_matrix_quantities of the result return ANS_ERR_INVALID_ARG.  With a -1 sign the call waits for the combination
 * (the cancelled links are compacted out in a second pass).  Arguments,
 * ownership and other errors as ans_sum_windows. */
int ans_combine(ans_ctx* ctx, const ans_matrix* const* mats, const int* signs, size_t k, ans_matrix** out,
                void* stream);

/* The nine quantities of a matrix (Table I, Sec. IV-C), recomputed on the
 * device from its DCSR arrays: row statistics by segmented reductions over
 * rows, column statistics by a transpose-free pass that sorts the stored links
 * by destination and reduces the destination runs.
 * out: host or device pointer to one ans_quantities.  With a device pointer
 * (or pinned host memory) the call is asynchronous; with pageable host memory
 * it returns once the result has been written. */
int ans_network_quantities(ans_ctx* ctx, const ans_matrix* m, ans_quantities* out, void* stream);

/* Batched analysis of nwin windows stored back to back (Sec. III-C batching,
 * taken to its limit: every window of the batch in one fixed launch sequence).
 *   d_src, d_dst : device arrays; window w is packets [d_offsets[w],
 *                  d_offsets[w+1]) of them.  They may also be page-locked
 *                  host memory that the device addresses (cudaHostAlloc or
 *                  cudaHostRegister): the kernels then read the pairs in
 *                  place over the host link, so the host-to-device transfer
 *                  happens inside the batch, without a staging copy.  With
 *                  agg_path 3 the pairs are read exactly once (by the packet
 *                  pack); the other paths read them once or twice.
 *   d_offsets    : DEVICE array of nwin + 1 nondecreasing uint64 offsets
 *                  (d_offsets[0] may be nonzero).  The batch is planned on the
 *                  device (window lengths, tile table, padded starts: one
 *                  scan kernel at the head of the launch sequence), so the
 *                  offsets may be written by earlier work on `stream`.
 *                  With a capacity set (ans_set_batch_capacity) the call
 *                  never reads the offsets on the host and sizes scratch and
 *                  grids for that many packets; without one it first copies
 *                  d_offsets[0] and d_offsets[nwin] to the host (waiting for
 *                  `stream`).  Offsets that decrease, a window of 2^31 packets
 *                  or more, or a batch above the capacity are found on the
 *                  device: every window then comes out empty and ans_wait,
 *                  ans_matrix_view and ans_matrix_quantities report
 *                  ANS_ERR_INVALID_ARG.  Per-window matrices of such a batch
 *                  learn their layout when the batch completes: summing or
 *                  re-analysing them waits for it.  Every window is sorted by
 *                  the radix passes (win_path is not consulted).
 *   flags        : ANS_BATCH_* bits.
 *   out          : nwin ans_quantities (host or device memory; pageable host
 *                  memory makes the call blocking).  May be NULL.
 *   per_window   : with ANS_BATCH_MATRICES, receives nwin matrices.
 *   sum          : with ANS_BATCH_SUM, receives the time sum of all windows.
 *   ticket       : optional; ans_wait(ctx, *ticket, ...) waits for the batch.
 * Results equal those of one ans_build_window per window followed by
 * ans_sum_windows.  Errors: ANS_ERR_INVALID_ARG, ANS_ERR_BUDGET, ANS_ERR_OOM,
 * ANS_ERR_CUDA. */
int ans_batch_submit(ans_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst,
                     const uint64_t* d_offsets, size_t nwin, uint32_t flags, ans_quantities* out,
                     ans_matrix** per_window, ans_matrix** sum, ans_ticket* ticket, void* stream);

/* The same with the offsets in HOST memory (h_offsets, nwin + 1 entries,
 * read during the call): the host plans the tiles, sizes everything
 * exactly, and validates the offsets before any work is queued (bad offsets
 * fail the call with ANS_ERR_INVALID_ARG). */
int ans_batch_submit_host(ans_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst,
                          const uint64_t* h_offsets, size_t nwin, uint32_t flags, ans_quantities* out,
                          ans_matrix** per_window, ans_matrix** sum, ans_ticket* ticket, void* stream);

/* Capacity, in packets, of batches submitted with device-resident offsets
 * (ans_batch_submit): scratch, output blocks and grids are sized for it, so
 * a larger capacity costs memory (about 100 bytes per packet of scratch,
 * and the per-window and time-sum blocks at 24 bytes per packet each) and
 * some empty tiles.  0 (the default) sizes each batch by reading its first
 * and last offset back.  Errors: ANS_ERR_INVALID_ARG. */
int ans_set_batch_capacity(ans_ctx* ctx, uint64_t max_packets);

/* The same analysis with every window in its own arrays: window w is
 * srcs[w][0..lens[w]) and dsts[w][0..lens[w]), in device memory, in
 * page-locked host memory (read by the kernels directly over the host link,
 * no staging copy: the serving path for windows that arrive in pinned
 * buffers), or in any host memory if the device reads pageable memory
 * (cudaDevAttrPageableMemoryAccess).  srcs, dsts and lens are host arrays of
 * nwin entries, read during the call; the windows' arrays must stay valid
 * until the batch completes.  On the paths that sort a batch's packets as one
 * segment (agg_path 2 or 3, sum_path 2) a kernel first gathers every window's
 * pairs, read in place, into one context-owned device buffer (8 bytes per
 * packet, kept for later calls and counted against the budget) and the batch
 * is analysed from there; if that buffer cannot be allocated the windows are
 * analysed in place on the other paths.  Every other argument, result and
 * error as ans_batch_submit_host; ANS_ERR_INVALID_ARG also for a window the
 * device cannot read. */
int ans_batch_submit_windows(ans_ctx* ctx, const uint32_t* const* srcs, const uint32_t* const* dsts,
                             const uint64_t* lens, size_t nwin, uint32_t flags, ans_quantities* out,
                             ans_matrix** per_window, ans_matrix** sum, ans_ticket* ticket, void* stream);

/* Wait (bounded) for a batch.  timeout_ns == 0 polls once.  Returns ANS_OK,
 * ANS_ERR_TIMEOUT (still running), ANS_ERR_INTERNAL (a bounded device wait or
 * a device consistency check failed inside the batch: its results are not
 * valid) or
 * ANS_ERR_INVALID_ARG (unknown ticket). */
int ans_wait(ans_ctx* ctx, ans_ticket ticket, uint64_t timeout_ns);

/* Poll limit of the context's bounded device waits (the decoupled look-back
 * of the radix passes, run reductions and scans waits for the tile before it
 * to publish; after `polls` polls with back-off the wait gives up, sets the
 * context's error word and returns, and the batch reports ANS_ERR_INTERNAL).
 * polls == 0 restores the default of 2^20 polls (about one second); at most
 * 2^24.  Waits for the device before it changes the limit, which applies to
 * work queued afterwards.  Not in the paper: failure detection of this
 * implementation.  Errors: ANS_ERR_INVALID_ARG, ANS_ERR_CUDA. */
int ans_set_wait_limit(ans_ctx* ctx, uint32_t polls);

/* Health check of the bounded waits (not in the paper): runs, on `stream`,
 * one look-back wait of each form for a predecessor tile that never
 * publishes, so each can only end by giving up at the context's poll limit.
 * The expiry is reported exactly as inside a batch: ans_wait(*ticket) and
 * ans_matrix_view / ans_matrix_quantities of *out (an empty matrix, optional)
 * return ANS_ERR_INTERNAL, and the context stays usable for later calls.
 * ticket and out may be NULL.  Errors: ANS_ERR_INVALID_ARG, ANS_ERR_OOM,
 * ANS_ERR_BUDGET, ANS_ERR_CUDA. */
int ans_probe_wait_expiry(ans_ctx* ctx, ans_matrix** out, ans_ticket* ticket, void* stream);

/* Scratch guards, a debug mode standing in for a memory checker (not in the
 * paper): a context created while the environment variable
 * ANS_SCRATCH_GUARDS is set (and not "0") places 256 bytes of a fixed pattern
 * after every region of a batch's scratch layout and of its output blocks,
 * writes them before the batch's kernels and compares them after; an
 * overwritten guard is reported like a failed device check (ans_wait and the
 * batch's matrices give ANS_ERR_INTERNAL).  ans_probe_guards checks that the
 * mechanism reports: it fills one guard, overwrites its first word as a write
 * one word past its region's end would, and checks it, so ans_wait(*ticket)
 * must return ANS_ERR_INTERNAL; the context stays usable.  It works whether
 * or not the context has the debug mode.  Errors: ANS_ERR_INVALID_ARG,
 * ANS_ERR_OOM, ANS_ERR_BUDGET, ANS_ERR_CUDA. */
int ans_probe_guards(ans_ctx* ctx, ans_ticket* ticket, void* stream);

/* Host-side view of a matrix: counts and device pointers to its arrays
 * (row_ids[nrows], row_ptr[nrows + 1], col_ids[nnz], vals[nnz]).  Blocks
 * until the matrix has been computed.  Any output pointer may be NULL. */
int ans_matrix_view(const ans_matrix* m, uint64_t* nrows, uint64_t* nnz, const uint32_t** row_ids,
                    const uint64_t** row_ptr, const uint32_t** col_ids, const uint64_t** vals);

/* Quantities computed while the matrix was built (host copy; blocks until
 * the matrix is complete). */
int ans_matrix_quantities(const ans_matrix* m, ans_quantities* out);

/* Release a matrix.  Waits for the work that produces it and for every
 * library call that reads it (ans_sum_windows, ans_network_quantities) to
 * finish, so a matrix may be freed right after enqueueing such a call, on any
 * stream.  Work of the caller's own that reads the matrix must be complete.
 * NULL is a no-op. */
int ans_matrix_free(ans_matrix* m);

/* A second handle to the same matrix (no copy): the memory is released when
 * every handle has been freed.  Serves data structures that hold one matrix
 * in several places, e.g. a batch sum that belongs to a one-minute and a
 * one-hour running sum. */
int ans_matrix_retain(const ans_matrix* m, ans_matrix** out);

/* Quantities of one window without allocating anything.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they run -- for example a capture process whose device memory is all
 * owned up front by another framework's caching allocator, or a
 * latency-critical ingest loop that cannot absorb cudaMalloc/cudaFree's
 * implicit synchronisation.  It runs the same kernels as ans_build_window and
 * writes the nine quantities of the window d_src/d_dst[0..n) to *d_out; it
 * needs no context and performs no allocation of any kind.
 *   n        : at most 65536 packets; larger n fails with ANS_ERR_INVALID_ARG.
 *   d_out    : device memory (or pinned host memory) for one ans_quantities.
 *   d_status : optional device word receiving 0, or nonzero if a bounded
 *              device wait gave up (the result is then invalid).
 * All intermediate data lives in one fixed device array of about 5 MiB,
 * present on every GPU that loads the library until the process exits.
 * Every call shares that array and it keeps the previous call's contents (the
 * call clears what must start at zero); calls whose work overlaps on the GPU
 * -- on different streams, or from threads that do not order their calls --
 * race and produce wrong results.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * Asynchronous on `stream`. */
int ans_window_quantities_noalloc(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n,
                                  ans_quantities* d_out, uint32_t* d_status, void* stream);

/* Memory accounting for admission control.  ans_ctx_memory reports the
 * device bytes the context holds now (scratch plus live matrices) and its
 * budget (0 = none).  ans_batch_bytes gives the additional device bytes that
 * ans_batch_submit_host with these offsets and flags would allocate if called now
 * (scratch growth plus output matrices); nothing is allocated. */
int ans_ctx_memory(ans_ctx* ctx, size_t* live_bytes, size_t* budget_bytes);
int ans_batch_bytes(ans_ctx* ctx, const uint64_t* h_offsets, size_t nwin, uint32_t flags, size_t* bytes);

/* Launch configuration of the three families of radix passes: the 64-bit link
 * keys of window sorts (key_*), the 64-bit keys with counts of time sums
 * (kv_*), and the 32-bit destination keys of the column pass (col_*).
 * *_threads: threads per 8192-key tile, 512 or 1024.  *_rank: how lanes
 * holding equal digits find each other, 0 = one __match_any_sync per key,
 * 1 = eight ballots per key, 2 = a per-warp shared-memory table (each lane
 * ORs its bit into its digit's entry, which also carries the digit's count).  *_blocks: CTAs per SM the kernel is compiled
 * for, 1, or 2 (512 threads only: registers capped at 64).  The key passes
 * and the column passes also take 256 threads with blocks 4: every 8192-key
 * tile is split into two 4096-key sub-tiles, one CTA each, four CTAs
 * resident per SM (column passes carrying 64-bit counts then run the
 * 512-thread shape).
 * win_path: how window keys are sorted, 0 = on chip, one 8-CTA thread-block
 * cluster per window of at most 2^17 packets sorting it in distributed shared
 * memory (larger windows, and every window when the device cannot host such
 * a cluster, take the key_* passes), 1 = the key_* passes for every window.
 * win_threads (512 or 1024) and win_rank (0 or 1, as *_rank) configure the
 * cluster kernel.  sum_path: how time sums order the links of their input matrices,
 * 0 = ceil(log2 k) rounds of pairwise merges of the matrices' already sorted
 * links, 1 = the kv_* radix passes over all gathered links, 2 = (a batch's
 * own time sum, windows stored back to back) every packet of the batch
 * sorted again as one segment by the key_* passes and reduced like a window
 * -- the sum of Table I's A_t is the matrix of the concatenated packets;
 * batches of windows in their own arrays then take the kv_* passes, and sums
 * of k given matrices merge them (k <= 256) or take the kv_* passes.  agg_path: how
 * a window's equal packets are grouped, 0 = sorting every packet's link key,
 * 1 = counting links in a per-window hash table (2^k >= 2 x packets slots of
 * 12 bytes, kept by the context between calls) and sorting only the distinct
 * links with their counts (kv_* passes); worth it when windows repeat links
 * heavily; 2 = for batches that return no per-window matrix (and whose time
 * sum, if any, takes sum_path 2): every quantity of a window by counting in
 * shared-memory hash tables -- its packets grouped by link hash into
 * partitions of ~4096, one table of 8192 links per partition, then its
 * distinct links grouped by source and by destination, one table of 16384
 * keys per partition -- with no sort; a window whose table overflows, or of
 * more than 2^18 packets, is sorted instead (other batches sort as agg_path 0);
 * 3 = for batches with a time sum, 2 to 2^16 windows and the packets in one
 * stream: no window sort -- the time sum always comes from the batch's
 * packets sorted as one segment (sum_path 2's sort), each packet carrying
 * its 16-bit window id through the key_* passes, and a stable sort of the
 * sorted packets by window id (two digit passes, the second writing each
 * window at its padded base) leaves every window's packets in key order,
 * as the window sort would (other batches sort as agg_path 0).  Setting
 * agg_path 0 waits for the device and releases the tables.  graph: 1 = a batch's launch sequence is recorded into a CUDA
 * graph and replayed through a cached executable graph of the same shape
 * (updated in place with the call's pointers), 0 = launched directly; per-
 * kernel profiling always launches directly.  col_hash: 1 = each window's
 * column statistics are first counted in a shared-memory hash of its
 * destinations (one CTA, or a cluster, per window; up to 12288 distinct
 * destinations), then windows with more destinations and at most 2^18 links
 * in shared-memory hashes of destination partitions (up to 32 CTAs per
 * window, one partition each), and only windows neither fits take the
 * column sort; 0 = the column sort for every window.  merge_tile: output positions per CTA of the time sum's merge
 * rounds, 4096 or 2048 (more resident CTAs per SM, twice the merge-path
 * searches).  Results never depend on the configuration. */
typedef struct {
    uint32_t key_threads, key_rank, key_blocks;
    uint32_t kv_threads, kv_rank, kv_blocks;
    uint32_t col_threads, col_rank, col_blocks;
    uint32_t win_path, win_threads, win_rank;
    uint32_t sum_path;
    uint32_t agg_path;
    uint32_t graph;
    uint32_t col_hash;
    uint32_t merge_tile;
} ans_tuning;

/* Read / set a context's configuration (default: 512 threads, rank 0, one
 * block; win_path 1, win_threads 1024, win_rank 0; sum_path 0; agg_path 0;
 * graph 1; col_hash 1; merge_tile 4096).
 * ans_set_tuning fails with ANS_ERR_INVALID_ARG on values other than the
 * ones listed above. */
int ans_get_tuning(ans_ctx* ctx, ans_tuning* out);
int ans_set_tuning(ans_ctx* ctx, const ans_tuning* tuning);

/* Autotuner: runs the caller's representative batch once per candidate
 * configuration, three times each, times every radix pass with CUDA events on
 * `stream` (these runs return per-window matrices and the time sum, so that
 * every pass family runs), and keeps, per family, the configuration with the
 * least total pass time; it then times the on-chip window sort (win_path 0,
 * three cluster configurations) and keeps it if the batch's windows sort
 * faster that way than by the best key passes plus their histogram sweep, and
 * finally picks sum_path, merge_tile (with merge rounds), then agg_path (2
 * only without ANS_BATCH_MATRICES in `flags`, together with sum_path 2 when
 * the batch has a time sum; 3 only with ANS_BATCH_SUM and 2 to 2^16
 * windows, together with sum_path 2) by the batch's device time as submitted with
 * `flags` (ANS_BATCH_* bits of the batches the context will run; one CUDA
 * graph with its concurrent branches, between CUDA events on `stream`, the
 * host's planning included).  With those paths fixed, it last retries the
 * column passes' shape (when the chosen paths run column passes) and, with
 * agg_path 3, the key passes' ranking mode, by the same device time.  An
 * optional path whose trial cannot get its
 * device memory (ANS_ERR_OOM / ANS_ERR_BUDGET) is skipped; the call fails
 * with ANS_ERR_OOM only if the default paths do not fit.  The choice is
 * applied to the context and returned in *chosen (optional).  The call
 * blocks until the runs have finished; it leaves per-kernel profiling
 * disabled and its data cleared.  With the environment variable
 * ANS_AUTOTUNE_LOG set (and not "0"), every trial writes one line to stderr:
 * its paths and shapes, the batch's device time and the per-kernel times. */
int ans_autotune(ans_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, const uint64_t* h_offsets,
                 size_t nwin, uint32_t flags, ans_tuning* chosen, void* stream);

/* Diagnostics: per-kernel timing.  While enabled, every kernel launch of the
 * context is bracketed by CUDA events on its launching stream (the paper
 * reports wall-clock analysis time, Sec. V-A; this splits it by kernel).
 * ans_profile_enable clears the accumulated data.  ans_profile_read waits for
 * the recorded launches, then writes one line per kernel name,
 * "<name> <launches> <total milliseconds>\n", NUL-terminated and truncated to
 * buflen; *needed (optional) receives the full length including the NUL. */
int ans_profile_enable(ans_ctx* ctx, int enable);
int ans_profile_read(ans_ctx* ctx, char* buf, size_t buflen, size_t* needed);

/* Import a traffic matrix given as DCSR -- the paper's own input form, the
 * flat containers of Sec. IV-B (row ids; row pointers, the prefix of the
 * per-row degrees; column ids, the edges; uint64 values, the weights) -- as
 * a matrix of the context, so that ans_network_quantities, ans_sum_windows
 * and the views work on it.  nrows rows, nnz links; row_ids[nrows],
 * row_ptr[nrows + 1], col_ids[nnz], vals[nnz], in device or host memory
 * (copied; the caller keeps ownership).  The input must be canonical: row
 * ids strictly ascending, row_ptr from 0 to nnz and strictly increasing (no
 * empty stored row), column ids strictly ascending within a row, no zero
 * value.  The call checks this on the device and waits for the check; the
 * quantities are then computed asynchronously on `stream`.  Errors:
 * ANS_ERR_INVALID_ARG (NULL arrays, nnz > 2^31 - 1, not canonical),
 * ANS_ERR_BUDGET, ANS_ERR_OOM, ANS_ERR_CUDA. */
int ans_matrix_import(ans_ctx* ctx, uint64_t nrows, uint64_t nnz, const uint32_t* row_ids,
                      const uint64_t* row_ptr, const uint32_t* col_ids, const uint64_t* vals,
                      ans_matrix** out, void* stream);

/* Row partition of a matrix for the exchange step of a time sum computed on
 * several devices (Sec. III-A, Fig. 4: each device's windows summed there,
 * the global sum owned in row partitions).  Rank o of nparts owns the rows
 * whose source address i has ((i * 0x9E3779B1 mod 2^32) * nparts) >> 32 == o;
 * out[o] receives those rows of m with all their links, as a new canonical
 * DCSR matrix with its quantities (so sum_o out[o] == m, row by row).  Each
 * piece can then be sent to its owner (its arrays through ans_matrix_view)
 * and added there to the pieces of the other ranks (ans_matrix_import +
 * ans_sum_windows).  nparts: 1 .. 64.  Waits for m and for the pieces'
 * sizes.  Errors: ANS_ERR_INVALID_ARG, ANS_ERR_BUDGET, ANS_ERR_OOM,
 * ANS_ERR_CUDA; a failed m's status. */
int ans_matrix_split_rows(ans_ctx* ctx, const ans_matrix* m, uint32_t nparts, ans_matrix** out, void* stream);

/* Static description of a status code. */
const char* ans_status_string(int status);

/* Detail of the last failure on the calling thread ("" if none). */
const char* ans_last_error(ans_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ANS_H */
