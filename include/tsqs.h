/*
 * tsqs.h -- C-ABI of the GB300-native three-way partition sort (Triple State
 * QuickSort, Muqaddas, arXiv 1505.00558).
 *
 * The library replaces qsort() for fixed key kinds (the paper's stated goal, abstract
 * and Section VII): a comparator pointer becomes a key kind, the element size must
 * match that kind, and the sort runs on one CUDA device (sm_103a) as
 *   presortedness     a root segment whose sample is in order is checked in full and,
 *                     if it is non-decreasing (non-increasing), finished as it stands
 *                     (by one reversal)                          (Section III.I)
 *   pivot kernel      a sampled median per segment        (Section III.H, V.C)
 *   partition kernel  <p | =p | >p split of every segment (Section III.A-F)
 *   work queue        device-built segment frontier that replaces recursion (Fig. 1)
 *   leaf kernel       on-chip sort of segments of <= small_threshold elements and
 *                     the fill of every =p run                  (Section IV, III.F)
 *
 * Conventions for every entry point:
 *   - Pointers named d_* / base are DEVICE pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The library owns its scratch (see
 *     tsqs_free_storage) and never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).  Calls
 *     are asynchronous on that stream unless stated otherwise.
 *   - Sorting is ascending under a total order on whole elements (integers numeric,
 *     floats IEEE 754 totalOrder, records (key, payload)).  Equal elements are
 *     bitwise identical, so the sorted output is unique and deterministic.
 *   - Return value: TSQS_OK or a tsqs_status code.  Nothing is thrown across the ABI.
 *     Argument errors are reported before any work is queued.  Errors raised on the
 *     device (a bounded wait that expired, an internal inconsistency) are sticky in the
 *     context and reported by tsqs_last_device_status(); after such an error the
 *     contents of the array are unspecified.
 *   - Limits: nmemb < 2^31 per segment (partition counters are 31-bit fields); base must
 *     be aligned to elem_size (16 bytes for records).
 */
#ifndef TSQS_H
#define TSQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key kinds (replace the paper's cmp callback, Section III / VII). */
typedef enum {
    TSQS_I32 = 1,          /* int32,  elem_size 4                                   */
    TSQS_U32 = 2,          /* uint32, elem_size 4                                   */
    TSQS_F32 = 3,          /* float32 under IEEE totalOrder, elem_size 4            */
    TSQS_I64 = 4,          /* int64,  elem_size 8                                   */
    TSQS_U64 = 5,          /* uint64, elem_size 8                                   */
    TSQS_F64 = 6,          /* float64 under IEEE totalOrder, elem_size 8            */
    TSQS_U64_U64_REC = 7   /* {uint64 key; uint64 payload}, ordered by (key, payload),
                              elem_size 16                                          */
} tsqs_key_kind;

typedef enum {
    TSQS_OK = 0,
    TSQS_EINVAL = 1,       /* bad argument (null pointer, size mismatch, alignment)  */
    TSQS_ENOMEM = 2,       /* device scratch could not be allocated / over budget    */
    TSQS_ECUDA = 3,        /* a CUDA runtime call failed                             */
    TSQS_ETIMEOUT = 4,     /* a bounded device-side wait expired                     */
    TSQS_EINTERNAL = 5     /* device-side consistency check failed                   */
} tsqs_status;

/* Tunables of one sort (the plan the autotuner picks).  Zero fields take defaults. */
typedef struct {
    int32_t  tile_items;       /* partition kernel shape, 0..3 (0 = default), given as
                                  consumer threads x keys per thread x staged tiles:
                                  4-byte keys 192x24x3, 192x32x3, 256x24x3, 256x16x3;
                                  8-byte keys 192x12x3, 192x16x3, 256x12x3, 256x8x3;
                                  records     192x6x3,  192x8x3,  256x6x3,  256x4x3      */
    int32_t  small_threshold;  /* segments of <= this many elements finish on chip,
                                  512..4096 (default 4096) for every key kind          */
    int32_t  ctas_per_sm;      /* resident CTAs per SM for the persistent kernels     */
    int32_t  sample_count;     /* pivot sample size (odd, at most 63; default 31)       */
    int32_t  offset_mode;      /* where a tile writes its <p and >p runs:
                                  0 = reserved with one 64-bit atomic on a per-segment
                                      cursor (default; tiles never wait on each other),
                                  1 = decoupled look-back over (#<p, #>p) in tile order
                                      (deterministic intermediate layout)              */
    int32_t  schedule;         /* order of the partition steps:
                                  0 = by size (default): inputs of at most 2^24
                                      elements run task-parallel, larger ones level by
                                      level,
                                  1 = level by level: one launch of each step per level
                                      of the recursion, every segment of a level at once,
                                  2 = task-parallel at any size: one persistent launch
                                      in which each segment is partitioned as soon as
                                      its parent is done, with no level barrier.
                                  Look-back offsets (offset_mode 1) always run level by
                                  level.                                                */
    uint64_t seed;             /* seed of the jittered sample positions (Section V.C)   */
} tsqs_plan;

/* Per-context statistics of the last completed sort (filled by tsqs_ctx_stats). */
typedef struct {
    uint32_t levels;           /* partition levels run (task-parallel schedule: depths
                                  of the recursion reached)                             */
    uint32_t max_frontier;     /* most segments in one level (0 task-parallel)          */
    uint64_t partition_keys;   /* keys read by all partition levels                     */
    uint64_t leaf_sorted_keys; /* keys finished by the on-chip sorter                   */
    uint64_t leaf_filled_keys; /* keys written by =p fills                              */
    uint64_t leaf_items;       /* leaf work items processed                             */
    uint64_t presorted_keys;   /* keys of root segments found already in order or in
                                  reverse order (finished without a partition level)   */
    uint64_t deep_sorted_keys; /* keys sorted by the depth guard's bitonic fallback      */
    uint32_t level_keys_count; /* entries used in level_keys                            */
    uint32_t pad;
    uint64_t level_keys[64];   /* keys partitioned at level (or depth) i (first 64)     */
} tsqs_stats;

typedef struct tsqs_ctx tsqs_ctx;   /* scratch + captured graphs of one independent sorter */

/* ---------------------------------------------------------------------------------
 * Core sort (Section III-IV: the qsort replacement, one segment).
 *   base       device array of nmemb elements of elem_size bytes, sorted in place.
 *   key_kind   tsqs_key_kind; elem_size must equal its size.
 *   nmemb <= 1 returns TSQS_OK with no launch.
 * Uses the library's default context; calls from several streams are serialised on
 * its scratch by events.
 * ------------------------------------------------------------------------------- */
int tsqs_sort(void *base, size_t nmemb, size_t elem_size, int key_kind, void *stream);

/* Segmented sort: sorts every segment [d_seg_offsets[s], d_seg_offsets[s+1]) of base
 * independently, all in one launch sequence.  d_seg_offsets is a DEVICE array of
 * nseg+1 non-decreasing uint64 offsets with d_seg_offsets[nseg] <= total capacity of
 * base; nmemb_total must equal d_seg_offsets[nseg] (used to size scratch). */
int tsqs_sort_segmented(void *base, size_t nmemb_total, const uint64_t *d_seg_offsets,
                        size_t nseg, size_t elem_size, int key_kind, void *stream);

/* Host-memory convenience (the paper's qsort(): array in host memory).  Copies h_base
 * to library-owned device memory and sorts it there.  If h_base is page-locked and
 * mapped (cudaHostAlloc / cudaHostRegister / a pinned torch tensor), the kernels write
 * the sorted result straight into h_base, so the last on-chip pass overlaps the
 * transfer back; any other host array is copied back after the sort.  Synchronises
 * `stream` before returning.  For a sequence of host arrays, tsqs_ctx_sort_host_stream
 * overlaps the copies of neighbouring arrays with the sorts. */
int tsqs_sort_host(void *h_base, size_t nmemb, size_t elem_size, int key_kind, void *stream);

/* Large elements (Section VIII.G-H, "late swapping"; the qsort of an array of wide
 * structures).  base (device) holds nmemb elements of elem_size bytes; element i is
 * ordered by the key of kind key_kind (TSQS_I32 .. TSQS_F64, not records) stored at byte
 * offset key_offset inside it, under that kind's total order, and elements with equal
 * keys keep their original order (the sort is stable, so the result is unique).
 * elem_size must be a multiple of 4 and of the key size, key_offset a multiple of the
 * key size with the key inside the element, base aligned to 4 and to the key size, and
 * nmemb < 2^31; otherwise TSQS_EINVAL.  (key, index) records are sorted by the record
 * path, then every element is moved once by a gather into library scratch
 * (16 + elem_size bytes per element, kept until tsqs_free_storage) and copied back.
 * Asynchronous on `stream`; TSQS_ENOMEM if the scratch cannot be allocated.  The paper
 * switches to this scheme above 320-byte elements; here the caller chooses it. */
int tsqs_sort_wide(void *base, size_t nmemb, size_t elem_size, size_t key_offset,
                   int key_kind, void *stream);

/* Frees the default context's device scratch (Section III.G:
 * FreeTripleStateQuickSortStorage).  Synchronises the device first. */
void tsqs_free_storage(void);

/* Synchronises `stream` and returns the default context's sticky device status
 * (TSQS_OK, TSQS_ETIMEOUT or TSQS_EINTERNAL), then clears it. */
int tsqs_last_device_status(void *stream);

/* ---------------------------------------------------------------------------------
 * Allocation-free sort (the paper has no counterpart).
 * For callers that cannot allocate device memory when they need a sort: programs whose
 * device memory is owned entirely by another allocator (a framework's caching pool or a
 * fixed arena, where a raw cudaMalloc fails or fragments it), services that account for
 * every device byte up front, and latency-critical paths that cannot afford a cudaMalloc
 * that may synchronise the device.  The result is the same as tsqs_sort's; all scratch
 * lives in a static device array that is part of this library's device code
 * (TSQS_NOALLOC_MAX_BYTES for the second buffer plus 4 MiB for the queues).  Every GPU
 * on which that code is loaded keeps the array until the process exits.
 *   - Sizes: nmemb * elem_size <= TSQS_NOALLOC_MAX_BYTES, else TSQS_EINVAL and nothing
 *     is queued.  Other arguments as tsqs_sort.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device does the set-up: it looks up the array's device
 *     address with cudaGetSymbolAddress and sets kernel attributes.  Make that first
 *     call before any stream capture begins.
 *   - The call runs the level loop from the host: it synchronises `stream` after every
 *     partition level and returns only after the sort has finished.  If `stream` is
 *     being captured it returns TSQS_EINVAL and queues nothing.
 *   - Every call shares the one array, which keeps the previous call's contents (each
 *     call clears what must start at zero).  Calls whose GPU work overlapped would race
 *     on it; this entry point prevents that within a process by holding a lock for the
 *     whole call and returning only after its sort has finished on `stream`.
 *   - Returns the sort's device status (TSQS_OK, TSQS_ETIMEOUT, TSQS_EINTERNAL).
 * ------------------------------------------------------------------------------- */
#define TSQS_NOALLOC_MAX_BYTES (16u << 20)
int tsqs_sort_noalloc(void *base, size_t nmemb, size_t elem_size, int key_kind, void *stream);

/* ---------------------------------------------------------------------------------
 * Explicit contexts: independent scratch and graphs, e.g. one per stream.
 * ------------------------------------------------------------------------------- */
tsqs_ctx *tsqs_ctx_create(const tsqs_plan *plan);          /* NULL plan = defaults */
void tsqs_ctx_destroy(tsqs_ctx *ctx);                      /* synchronises first  */
int tsqs_ctx_sort(tsqs_ctx *ctx, void *base, size_t nmemb, size_t elem_size, int key_kind,
                  void *stream);
int tsqs_ctx_sort_segmented(tsqs_ctx *ctx, void *base, size_t nmemb_total,
                            const uint64_t *d_seg_offsets, size_t nseg, size_t elem_size,
                            int key_kind, void *stream);
/* Caller-held graph of a whole sort (batching, pattern 2: capture once, replay; the
 * paper's qsort-replacement call of the abstract and Section VII, issued as one CUDA
 * graph).  graph_exec points to a cudaGraphExec_t passed as void*:
 *   *graph_exec == NULL  the call builds the whole segmented sort of these arguments as
 *                        one graph (the per-call setup kernel, then the sort's nodes),
 *                        instantiates it into *graph_exec and launches it on `stream`;
 *   otherwise            *graph_exec must come from an earlier call with the same ctx and
 *                        key_kind (else TSQS_EINVAL): its setup node is updated to these
 *                        arguments and it is launched.  A call whose size takes the other
 *                        schedule of the ctx's plan (tsqs_plan.schedule: task-parallel up
 *                        to 2^24 elements by default, level by level above) releases that
 *                        graph, builds the other one and stores its new handle in
 *                        *graph_exec; within one schedule the handle stays.
 * The graph holds the same nodes as the ctx's own sort for that size: presortedness, then
 * the task kernel or the conditional level loop, the leaf pass and the depth guard.
 * d_seg_offsets == NULL sorts base[0, nmemb_total) as one segment; otherwise as
 * tsqs_ctx_sort_segmented.  Nothing to sort (no segment, or one segment of <= 1
 * element) returns TSQS_OK with no graph made.  The caller may also replay the graph
 * itself with cudaGraphLaunch(*graph_exec, s) to sort the same arrays again (after
 * refilling them) for as long as ctx lives and its scratch is not regrown: reserve it
 * first with tsqs_ctx_reserve for the largest shape.  Replays and other sorts of the
 * same ctx must not overlap on the device (they share its scratch): the calls order
 * themselves on the ctx's completion event, direct replays are ordered by the caller.
 * The graph belongs to ctx: release it with tsqs_graph_exec_destroy (tsqs_ctx_destroy
 * releases any that remain).  Argument errors as tsqs_ctx_sort_segmented;
 * TSQS_ENOMEM if scratch cannot be allocated, TSQS_ECUDA if a graph call fails. */
int tsqs_graph_sort_segmented(tsqs_ctx *ctx, void *base, size_t nmemb_total,
                              const uint64_t *d_seg_offsets, size_t nseg, size_t elem_size,
                              int key_kind, void *stream, void **graph_exec);
/* Waits for ctx's sorts, then destroys a graph made by tsqs_graph_sort_segmented on ctx
 * (no-op for any other pointer). */
void tsqs_graph_exec_destroy(tsqs_ctx *ctx, void *graph_exec);

/* Reserves scratch for sorts up to (nmemb_total, nseg) of elem_size so that later calls
 * allocate nothing (and may run under stream capture). */
int tsqs_ctx_reserve(tsqs_ctx *ctx, size_t nmemb_total, size_t nseg, size_t elem_size);
size_t tsqs_ctx_scratch_bytes(const tsqs_ctx *ctx);
int tsqs_ctx_device_status(tsqs_ctx *ctx, void *stream);   /* sync + read + clear */
int tsqs_ctx_stats(tsqs_ctx *ctx, void *stream, tsqs_stats *out);   /* sync + read */
int tsqs_ctx_set_plan(tsqs_ctx *ctx, const tsqs_plan *plan);
int tsqs_ctx_get_plan(const tsqs_ctx *ctx, tsqs_plan *out);

/* ---------------------------------------------------------------------------------
 * Streaming host arrays through the GPU (the paper's qsort() on host memory, applied
 * to a sequence of independent arrays).
 *   h_in[i]    host array of nmemb[i] elements of elem_size bytes (read only).
 *   h_out[i]   host array that receives item i sorted ascending; it may be h_in[i]
 *              (in place).  h_out == NULL sorts every item in place.
 *   h_status   NULL, or a host array of count ints that receives each item's device
 *              status (TSQS_OK, TSQS_ETIMEOUT, TSQS_EINTERNAL).
 * Each item is copied to one of three device staging slots owned by the context, sorted
 * there on `stream` (the items' sorts run one after another), and copied back.  The
 * copies in and out run on two streams of the context's own, so while item i is sorted
 * item i+1 is uploaded and item i-1 downloaded; with page-locked host arrays all three
 * overlap, with pageable ones the copies are staged by the driver and overlap less.
 * The staging slots (3 x the largest item's bytes) are kept until tsqs_ctx_destroy.
 * Work queued on `stream` before the call is ordered before the first copy.  Returns
 * after every item is in h_out: TSQS_OK, the first nonzero item status, TSQS_EINVAL
 * (kind/size mismatch, an item of 2^31 or more elements, a NULL array for a non-empty
 * item; nothing is queued), TSQS_ENOMEM (staging or scratch could not be allocated;
 * nothing is queued) or TSQS_ECUDA.  Arrays of 0 or 1 element are copied unchanged.
 * ------------------------------------------------------------------------------- */
int tsqs_ctx_sort_host_stream(tsqs_ctx *ctx, const void *const *h_in, void *const *h_out,
                              const size_t *nmemb, size_t count, size_t elem_size,
                              int key_kind, void *stream, int *h_status);

/* Bytes of device scratch a context needs for a sort of this shape. */
size_t tsqs_scratch_bytes_for(size_t nmemb_total, size_t nseg, size_t elem_size,
                              const tsqs_plan *plan);

/* Default plan for a key kind and size (autotuned values when a tuning table was
 * loaded with tsqs_plan_load, built-in defaults otherwise). */
int tsqs_plan_default(int key_kind, size_t n_hint, tsqs_plan *out);

/* ---------------------------------------------------------------------------------
 * Instrumented run (for measurement): the same kernels as the context's graph for this
 * size, launched one at a time from the host.  Synchronises `stream`.
 * Level-by-level schedule: a CUDA event pair around every partition launch; writes up
 * to max_levels partition-kernel durations (ms) to h_ms, the keys each of those
 * launches read to h_keys and each level's leaf-launch duration to h_leaf_ms; returns
 * the number of levels through *levels.
 * Task-parallel schedule (plan.schedule, size): one entry: the task kernel's duration,
 * the keys it partitioned over all depths, and the leaf pass's duration; *levels = 1.
 * ------------------------------------------------------------------------------- */
int tsqs_ctx_sort_timed(tsqs_ctx *ctx, void *base, size_t nmemb, size_t elem_size,
                        int key_kind, void *stream, float *h_ms, uint64_t *h_keys,
                        int max_levels, int *levels, float *h_leaf_ms);

/* ---------------------------------------------------------------------------------
 * Step-level entry points (used to test each kernel alone against the oracle).
 * ------------------------------------------------------------------------------- */

/* Pivot kernel on one segment [seg_begin, seg_end) of base with exactly sample_count
 * samples (at most 63; clamped to the segment length and made odd): writes the
 * sample positions it used (h_positions holds sample_count uint64, host) and the pivot
 * element (elem_size bytes, host, original representation).  Synchronises `stream`. */
int tsqs_debug_pivot(const void *base, size_t nmemb, size_t elem_size, int key_kind,
                     uint64_t seg_begin, uint64_t seg_end, int sample_count, uint64_t seed,
                     uint64_t *h_positions, void *h_pivot, void *stream);

/* One partition level: for every segment s of d_seg_offsets (device, nseg+1) with pivot
 * d_pivots[s] (device, original representation, elem_size bytes each), reads src and
 * writes dst over the same range: the elements < p packed from the left, the elements
 * > p packed from the right; the =p run in between is not written.  Writes
 * d_counts[2*s] = #<p and d_counts[2*s+1] = #>p (device uint64).  src and dst must
 * not overlap.  Synchronises `stream`. */
int tsqs_debug_partition(const void *src, void *dst, size_t nmemb, size_t elem_size,
                         int key_kind, const uint64_t *d_seg_offsets, size_t nseg,
                         const void *d_pivots, uint64_t *d_counts, void *stream);

/* Leaf kernel alone: sorts every segment of d_seg_offsets (each must hold at most
 * small_threshold elements of the default plan) in place.  Synchronises `stream`. */
int tsqs_debug_small_sort(void *base, size_t nmemb, size_t elem_size, int key_kind,
                          const uint64_t *d_seg_offsets, size_t nseg, void *stream);

/* Forces the bounded look-back wait of the next partition level of the default
 * context to give up after `polls` polls (0 restores the default).  Used by tests
 * to check that an expired wait surfaces as TSQS_ETIMEOUT. */
void tsqs_debug_set_spin_limit(uint32_t polls);

/* Sets the depth guard's level for sorts that start afterwards (every context): a
 * segment that would be partitioned at this level or deeper is sorted by the bitonic
 * fallback instead (Section V.B-C's worst-case mitigation).  0 restores the default,
 * 2 ceil(log2 n) + 8, which sampled pivots never reach in practice; tests set a small
 * value to run the fallback on ordinary inputs. */
void tsqs_debug_set_deep_level(uint32_t level);

/* Caps, for sorts that start afterwards (every context), how many leaf items may wait
 * in the queue before the level loop pauses for a leaf pass.  By default the queue holds
 * two levels' worth of items and the loop pauses once more than one level's worth is
 * waiting, which ordinary inputs never reach, so all leaves are sorted in one pass after
 * the last level.  Tests set a small value to run the pause-and-resume path of the level
 * loop on ordinary inputs.  0 restores the default. */
void tsqs_debug_set_leaf_defer(uint32_t items);

/* When on == 1, partition tile 1 of every later level-by-level sort never publishes
 * its look-back word, so the waits of its successors must run into the spin limit and
 * the sort must end with TSQS_ETIMEOUT.  When on == 2, the first segment of every later
 * task-parallel sort never publishes its tile rows, so every block that claimed one of
 * its tiles must run into the spin limit, with the same result.  Both are host-side
 * fault injections that neither fault nor hang the device.  0 restores normal
 * operation. */
void tsqs_debug_withhold_publish(int on);

/* ---------------------------------------------------------------------------------
 * Batching: one captured CUDA graph per (context, key kind) replayed for every call;
 * tsqs_plan_autotune times candidate plans on a synthetic batch and returns the best.
 * ------------------------------------------------------------------------------- */
int tsqs_plan_autotune(int key_kind, size_t n_hint, size_t nseg_hint, void *stream,
                       tsqs_plan *out);
/* Writes / reads the autotuned plans of this process as text (one plan per line). */
int tsqs_plan_cache_save(const char *path);
int tsqs_plan_cache_load(const char *path);

/* ---------------------------------------------------------------------------------
 * Serving: continuous batching of sort requests that arrive over time.
 * ------------------------------------------------------------------------------- */
typedef struct tsqs_server tsqs_server;

typedef struct {
    int32_t  status;        /* tsqs_status of the request (TSQS_OK when sorted)        */
    int32_t  done;          /* 1 once the result is complete on the device             */
    double   t_submit;      /* host seconds (monotonic) when tsqs_server_submit ran   */
    double   t_start;       /* host seconds when the request was launched              */
    double   t_done;        /* host seconds when its completion was observed           */
    uint32_t batch_id;      /* launch that carried it                                  */
    uint32_t batch_size;    /* requests in that launch                                 */
} tsqs_result;

/* mem_budget_bytes bounds the device scratch plus in-flight request bytes;
 * n_streams launches may be in flight at once; max_batch bounds requests per launch.
 * Every lane sorts with the level-by-level schedule (tsqs_plan.schedule 1): its launches
 * interleave with the other lanes' on the GPU. */
tsqs_server *tsqs_server_create(size_t mem_budget_bytes, int n_streams, int max_batch);
/* Queues a request on d_base (device, caller-owned, must stay valid until done).
 * Returns TSQS_ENOMEM if the request alone can never fit the budget. */
int tsqs_server_submit(tsqs_server *s, void *d_base, size_t nmemb, size_t elem_size,
                       int key_kind, uint64_t *ticket);
/* Admits queued requests that fit, launches batches, retires finished ones.  Call it
 * from the host loop; returns the number of requests still pending or in flight. */
int tsqs_server_progress(tsqs_server *s);
int tsqs_server_poll(tsqs_server *s, uint64_t ticket, tsqs_result *out);
int tsqs_server_drain(tsqs_server *s);          /* progress until nothing is pending */
void tsqs_server_destroy(tsqs_server *s);

#ifdef __cplusplus
}
#endif
#endif /* TSQS_H */
