// tsqs_internal.h -- structures shared by the host runtime and the kernels.
//
// One sort is a level-synchronous walk over a device-built work queue:
//   frontier[par]  segments larger than the small threshold waiting for a partition
//                  level (the recursion of Fig. 1 turned into a breadth-first queue);
//   leaves         work for the on-chip pass: segments of <= small threshold elements
//                  to sort (Section IV's role) and runs of =p to fill with p
//                  (Section III.F: the equals are placed once and never compared again).
//                  Items of every level queue up (each remembers the buffer holding its
//                  keys; no later level touches its range) and run in one pass after
//                  the level loop, or earlier only if the queue would overflow.
// Level L reads buffer L%2 (0 = caller's array, 1 = scratch) and writes buffer
// (L+1)%2; every element reaches its final place in the caller's array exactly once,
// through a leaf sort or an =p fill.
#pragma once
#include <stdint.h>

namespace tsqs {

constexpr int kMaxSamples = 63;
constexpr uint32_t kFillChunk = 16384;      // =p fills are split into items of this size
constexpr uint32_t kInlineFill = 16;        // =p runs up to this long are written by the level-end kernel
constexpr int kMaxSmall = 4096;             // largest on-chip segment
constexpr int kStatLevels = 64;
constexpr uint32_t kTaskGridMax = 4096;     // end-of-work rows reserved past the last tile


enum LeafKind : uint32_t { LEAF_SORT = 0, LEAF_FILL = 1 };
// LeafItem::kind flag: the item's keys are in buffer 1 (alt) rather than buffer 0
constexpr uint32_t kLeafInAlt = 0x100u;

// A segment [begin, end) waiting for a partition level.
struct SegDesc {
    uint64_t begin, end;
    int64_t  s0;              // element index where tile 0 starts (16-byte aligned, <= begin)
    uint32_t tile_begin;      // first global tile id of this segment in its level
    uint32_t ntiles;
    uint64_t piv_lo, piv_hi;  // canonical pivot (hi used by 16-byte records only)
};

// A segment of the task-parallel schedule (inputs up to a size bound, see k_task):
// partitioned as soon as it is pushed, with its own finished-tile count and cursor.
struct alignas(16) TaskSeg {
    uint64_t begin, end;
    int64_t  s0;              // element index where tile 0 starts (16-byte aligned, <= begin)
    uint64_t piv_lo, piv_hi;  // canonical pivot
    uint32_t tile_begin;      // first global tile id (tile ids run over the whole sort)
    uint32_t ntiles_depth;    // tiles | recursion depth << 24 (keys in buffer depth % 2)
    unsigned long long done;  // finished tiles << 42 | their #<p << 21 | their #>p (the
                              // counts only for segments below 2^21 elements)
    unsigned long long cursor;   // reserved (#<p | #>p << 32)
};
static_assert(sizeof(TaskSeg) == 64, "TaskSeg is four 16-byte words");

struct LeafItem {
    uint64_t begin;
    uint32_t len;
    uint32_t kind;            // LeafKind, | kLeafInAlt for a sort whose keys are in alt
    uint64_t v_lo, v_hi;      // canonical fill value for LEAF_FILL
};

// Mutable device state of one sort; zeroed by the setup kernel of every call.
struct Ctl {
    uint32_t level;           // current level (iteration of the level loop)
    uint32_t status;          // sticky tsqs_status of the device side
    uint32_t tile_claim;      // partition tiles claimed in this level
    uint32_t leaf_claim;      // leaf items claimed by the running leaf pass
    uint32_t seg_claim;       // frontier segments claimed by the pivot kernel
    uint32_t cont;            // the level loop runs another level now (graph: inner loop)
    uint32_t nfront[2];
    uint32_t ntiles[2];
    uint32_t nleaf;           // leaf items queued (across levels, until a leaf pass)
    uint32_t leaf_blocks;     // leaf-pass blocks finished (last one empties the queue)
    uint32_t presort_any;     // some root segment's sample is in order (presortedness pass)
    uint32_t ndeep;           // segments handed to the depth-guard sorter
    uint32_t deep_kk, deep_jj;  // its next stage: merge width 2^kk, stride 2^jj (11: on-chip)
    uint32_t deep_maxlog;     // log2 of the largest padded deep segment
    uint32_t deep_blocks;     // stage-kernel blocks finished (the last one advances the stage)
    uint32_t deep_cont;       // more stages (host-driven mode reads it)
    uint32_t max_front;
    uint32_t levels_done;
    uint32_t blocks_done;     // level-end blocks finished (last one runs level control)
    uint32_t more;            // levels remain (after a leaf pass if cont is 0); host-driven
                              // mode reads it
    uint32_t tclaim;          // task schedule: tile ids claimed
    uint32_t talloc;          // task schedule: tile ids given to pushed segments
    uint32_t tsegs;           // task schedule: segments pushed
    uint32_t live;            // task schedule: pushed segments not yet finished
    uint32_t coop_count, coop_gen, coop_go;   // grid barrier of the cooperative deep kernel
    uint64_t front_keys[2];
    uint64_t partition_keys;
    uint64_t leaf_sorted, leaf_filled, leaf_items;
    uint64_t presorted;       // keys of root segments found already in order (or reversed)
    uint64_t deep_keys;       // keys sorted by the depth-guard sorter
    uint64_t level_keys[kStatLevels];
};

// Per-call description, written by the setup kernel and read by every kernel.
struct Job {
    void *base;               // buffer 0: the caller's array
    void *alt;                // buffer 1: scratch with the same 16-byte phase as base
    void *out;                // where leaf sorts and =p fills write the result: base, or a
                              // device-mapped host array with base's 16-byte phase
    uint64_t n;               // elements addressable in base (and alt)
    const uint64_t *seg_offsets;   // nullptr: one segment [0, n)
    uint64_t nseg;
    SegDesc *front[2];
    LeafItem *leaves;         // leaf items of every level since the last leaf pass
    uint32_t *tile_seg;       // tile id -> frontier index, current level
    unsigned long long *tile_status;   // decoupled look-back words, current level
    uint32_t *seg_done;       // finished tiles per frontier segment
    unsigned long long *seg_cursor;    // reserved (#<p | #>p << 32) per frontier segment
    uint32_t *presort;        // per root segment: 0, or 1 / 2 while it may be / is known to be
                              // non-decreasing / non-increasing
    LeafItem *deep;           // segments that reached deep_level (kind flag: buffer 1)
    uint32_t *deep_tiles;     // prefix over deep segments of their 4096-element tiles
    uint32_t *deep_chunks;    // prefix over deep segments of their pair chunks
    uint32_t cap_front, cap_tiles, cap_leaves;
    uint32_t leaf_defer;      // a level's leaf pass runs only above this many queued items
    uint32_t cap_deep;        // capacity of deep (segments above small_T are disjoint)
    uint32_t deep_level;      // a child that would be partitioned at this level or later goes
                              // to the depth-guard sorter instead
    uint32_t small_T;         // on-chip threshold
    uint32_t samples;         // pivot sample count (odd, <= kMaxSamples)
    uint32_t vec_off;         // (address of base / elem_size) mod (16 / elem_size)
    uint32_t spin_limit;      // polls before a look-back wait gives up
    uint32_t pad;             // bit 1: tile id 1 withholds its look-back status (test of
                              // the bounded wait)
    uint32_t max_levels;      // level cap; exceeding it stops the loop with an error
    uint32_t offset_mode;     // 0: per-segment atomic cursor, 1: decoupled look-back
    uint32_t tile;            // keys per partition tile of the partition kernel in use
                              // (of the task kernel in the task schedule)
    uint32_t pad3;
    uint64_t seed;            // sample jitter seed
    // task schedule (k_task); null / zero when the call runs level by level
    TaskSeg *tseg;            // pushed segments
    unsigned long long *trow; // tile id -> (tile origin, buffer, segment), 0 while the
                              // segment is not pushed (k_orient zeroes the rows of a call)
    uint32_t cap_tseg, cap_trow;
    uint32_t task_grid;       // blocks of k_task that take part (the rest return at once;
                              // one end-of-work row each)
    uint32_t pad4;
    // step-level test hooks
    const void *dbg_pivots;   // debug partition: pivots of the given segments
    uint64_t *dbg_counts;     // debug partition: (#<p, #>p) per segment
    uint64_t *dbg_positions;  // debug pivot: sample positions
    void *dbg_pivot_out;      // debug pivot: chosen pivot (original representation)
};

// One compiled shape of the partition kernel.
struct PartVariant {
    const void *k_partition;
    int tile;                 // keys per tile
    int threads;              // consumer warps + one producer warp
    int smem;                 // dynamic shared memory
    int nbuf;                 // depth of the shared-memory ring
};
constexpr int kPartVariants = 4;

// Kernel entry points of one key kind (filled by the per-kind translation units).
struct KindOps {
    int kind;
    int elem_size;
    int leaf_block, pivot_block;
    int leaf_smem;            // dynamic shared memory of the leaf kernel
    int leaf_max;             // largest segment the leaf kernel sorts (32 x keys per lane)
    PartVariant part[kPartVariants];   // [0] is the default shape
    const void *k_init, *k_leaf, *k_pivot, *k_finish;
    const void *k_orient, *k_orient_if, *k_check, *k_presort;
    const void *k_deep_prep, *k_deep_tiles, *k_deep_stage, *k_deep_finish, *k_deep_all;
    int deep_smem;            // dynamic shared memory of the on-chip deep stages
    const void *k_dbg_setup_partition, *k_dbg_counts, *k_dbg_pivot;
    const void *k_task_init, *k_task;   // task schedule
    // leaf pass of the task graph for small inputs (items in one wave: more threads per
    // item); the same kernel as k_leaf where no such variant exists
    const void *k_leaf_small;
    int leaf_small_block, leaf_small_smem;
    int task_block, task_tile;
};

// Large elements (tsqs_wide.cu): (key, index) records of every element, and the gather
// of the elements in record order.  `stream` is a cudaStream_t.
int wide_keys(int kind, const void *base, uint64_t n, uint64_t es, uint64_t key_off, void *rec,
              int sms, void *stream);
int wide_gather(const void *src, uint64_t n, uint64_t es, const void *rec, void *dst, int sms,
                void *stream);

const KindOps *ops_k4(int kind);
const KindOps *ops_k8(int kind);
const KindOps *ops_k16(int kind);

}  // namespace tsqs
