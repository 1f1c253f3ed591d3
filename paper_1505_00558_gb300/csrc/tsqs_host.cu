// tsqs_host.cu -- host runtime and C-ABI of the three-way partition sort.
//
// A context owns one block of device scratch (the second buffer of the ping-pong,
// the work queues and the look-back words; the analogue of the persistent temporary
// storage of Section III.G) and two CUDA graphs per key kind.  The level-by-level one is
//     orient -> if (a root is a candidate) { check -> presort } -> init
//       -> while (levels remain) { while (frontier not empty) { pivot ; partition ; level end } ;
//                                  leaf pass ; control }
//       -> if (a segment reached the depth bound) { deep prep -> deep tiles -> while (stages)
//                                                   { deep stage } -> deep finish }
// and the task-parallel one (inputs up to a size bound)
//     orient -> check -> presort -> task init -> task kernel -> leaf pass
//       -> depth guard (one cooperative kernel; returns at once with no deep segment)
// with the loop conditions set on the device (by the level-end and deep-stage kernels),
// so a whole sort is one graph launch with no host round trip between levels.  Every kernel reads the
// per-call description (Job) from device memory, written by a one-thread setup kernel
// launched just before the graph, so the same graph serves every array of its kind.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "tsqs.h"
#include "tsqs_internal.h"

using namespace tsqs;

namespace tsqs {
__global__ void k_setup(Job *job, Ctl *ctl, Job j);
__global__ void k_keep_status(const Ctl *ctl, uint32_t *dst, int ran);
__global__ void k_outer_control(const Ctl *ctl, cudaGraphConditionalHandle h_levels,
                                cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_deep);
}
bool tsqs_cached_plan(int kind, size_t n, size_t nseg, tsqs_plan *out);

namespace {

constexpr uint32_t kDefaultSpin = 1u << 22;     // look-back polls before giving up

const KindOps *get_ops(int kind) {
    if (kind >= TSQS_I32 && kind <= TSQS_F32) return ops_k4(kind);
    if (kind >= TSQS_I64 && kind <= TSQS_F64) return ops_k8(kind);
    if (kind == TSQS_U64_U64_REC) return ops_k16(kind);
    return nullptr;
}

// Partition shape chosen by the plan (tile_items selects one of the compiled shapes).
const PartVariant &part_of(const KindOps *o, const tsqs_plan &p) {
    int v = p.tile_items;
    if (v < 0 || v >= kPartVariants) v = 0;
    return o->part[v];
}

size_t kind_size(int kind) {
    const KindOps *o = get_ops(kind);
    return o ? (size_t)o->elem_size : 0;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t g_debug_spin = 0;        // 0 = default
uint32_t g_debug_deep = 0;        // depth-guard level; 0 = default (2 log2 n + 8)
uint32_t g_debug_defer = 0;       // leaf-queue pause threshold; 0 = default (one level's worth)
int g_debug_withhold = 0;         // 1: a look-back word withheld; 2: a task segment's rows

// Inputs of at most this many elements run the task-parallel schedule (k_task): every
// segment is partitioned as soon as its parent is done, with no level barrier.
constexpr size_t kTaskMaxN = size_t(1) << 24;

// Whether a sort of n elements under plan p runs the task-parallel schedule: schedule 0
// below the size bound, 2 at any size, never with look-back offsets (their deterministic
// layout is a level-by-level one) or schedule 1.
bool task_schedule(const tsqs_plan &p, size_t n) {
    if (p.offset_mode == 1 || g_debug_withhold == 1 || p.schedule == 1) return false;
    return p.schedule == 2 || n <= kTaskMaxN;
}

// Up to this many elements the task graph's leaf pass takes the small-input leaf kernel:
// its items fit in one wave, and more threads per item shorten the pass (1e6 int32:
// 7.5 us); above it the default leaf's throughput wins.
constexpr size_t kSmallLeafN = size_t(1) << 20;

struct Layout {
    size_t alt_off, front_off[2], leaves_off, tseg_off, tstat_off, done_off, cursor_off, presort_off,
        deep_off, dtiles_off, dchunks_off, misc_off, ttask_off, trow_off, total;
    uint32_t cap_front, cap_tiles, cap_leaves, leaf_defer, cap_tseg, cap_trow;
};

// Scratch needed for nmemb elements in nseg segments (bounds, not estimates):
//   frontier  segments above small_T in one level are disjoint: <= n/(T+1) (+ nseg for
//             the step-level partition test, which seeds every given segment)
//   tiles     <= n/TILE + 2 per segment (partial first and last tiles)
//   leaves    one level adds <= 2 children per partitioned segment, n/kFillChunk + 1
//             fill items per segment, plus the small root segments: cl.  Items queue up
//             across levels; a level's leaf pass runs once more than cl are queued, so
//             the queue never holds more than 2 cl
//   task schedule (task_tile > 0): segments above small_T of one depth are disjoint, and
//             depths stop at the depth guard's level D, so <= D (n/(T+1) + 1) task
//             segments and <= D (n/TILE + 2 (n/(T+1) + 1)) tile ids (+ the end-of-work
//             rows); all leaves of the sort queue up for one pass: <= 3 per task segment
//             (two children and a fill item beyond whole chunks), n/kFillChunk whole
//             fill chunks and the small roots
// Effective on-chip threshold: the plan's, capped by what the kind's leaf kernel holds.
size_t eff_threshold(const tsqs_plan &plan, int leaf_max) {
    return std::min<size_t>((size_t)plan.small_threshold, (size_t)leaf_max);
}

// Depth-guard level of a sort of n elements: 2 ceil(log2(n + 1)) + 8.
uint32_t deep_level_for(size_t n) {
    unsigned lg = 1;
    while ((1ull << lg) < (unsigned long long)n + 1 && lg < 63) lg++;
    return 2u * lg + 8u;
}

Layout make_layout(size_t n, size_t nseg, size_t es, const tsqs_plan &plan, int tile, int leaf_max,
                   int task_tile = 0) {
    Layout L{};
    const size_t T = eff_threshold(plan, leaf_max);
    const size_t cf = n / (T + 1) + nseg + 4;
    const size_t ct = n / (size_t)tile + 2 * cf + 4;
    const size_t cl = 3 * cf + n / kFillChunk + nseg + 4;
    size_t cts = 0, ctr = 0, clt = 0;
    if (task_tile > 0) {
        const size_t D = std::max<size_t>(deep_level_for(n), g_debug_deep);
        const size_t per = n / (T + 1) + 1;
        cts = D * per + 4;
        ctr = D * (n / (size_t)task_tile + 2 * per) + kTaskGridMax + 4;
        clt = 3 * cts + n / kFillChunk + nseg + 4;
    }
    L.cap_front = (uint32_t)std::min<size_t>(cf, 0xFFFFFFF0u);
    L.cap_tiles = (uint32_t)std::min<size_t>(ct, 0xFFFFFFF0u);
    L.cap_leaves = (uint32_t)std::min<size_t>(std::max(2 * cl, clt), 0xFFFFFFF0u);
    L.leaf_defer = (uint32_t)std::min<size_t>(cl, 0x7FFFFFF0u);
    L.cap_tseg = (uint32_t)std::min<size_t>(cts, 0xFFFFFFF0u);
    L.cap_trow = (uint32_t)std::min<size_t>(ctr, 0xFFFFFFF0u);
    size_t off = 0;
    L.alt_off = off;            off = align_up(off + n * es + 16, 256);
    L.front_off[0] = off;       off = align_up(off + cf * sizeof(SegDesc), 256);
    L.front_off[1] = off;       off = align_up(off + cf * sizeof(SegDesc), 256);
    L.leaves_off = off;         off = align_up(off + std::max(2 * cl, clt) * sizeof(LeafItem), 256);
    L.tseg_off = off;           off = align_up(off + ct * sizeof(uint32_t), 256);
    L.tstat_off = off;          off = align_up(off + ct * sizeof(unsigned long long), 256);
    L.done_off = off;           off = align_up(off + cf * sizeof(uint32_t), 256);
    L.cursor_off = off;         off = align_up(off + cf * sizeof(unsigned long long), 256);
    L.presort_off = off;        off = align_up(off + (nseg ? nseg : 1) * sizeof(uint32_t), 256);
    L.deep_off = off;           off = align_up(off + cf * sizeof(LeafItem), 256);
    L.dtiles_off = off;         off = align_up(off + (cf + 1) * sizeof(uint32_t), 256);
    L.dchunks_off = off;        off = align_up(off + (cf + 1) * sizeof(uint32_t), 256);
    L.misc_off = off;           off = align_up(off + 4096, 256);   // debug buffers
    L.ttask_off = off;          off = align_up(off + cts * sizeof(TaskSeg), 256);
    L.trow_off = off;           off = align_up(off + ctr * sizeof(unsigned long long), 256);
    L.total = off;
    return L;
}

void fill_default_plan(int key_kind, size_t, tsqs_plan *p) {
    (void)key_kind;
    p->tile_items = 0;            // partition shape 0 (see KindOps::part)
    p->small_threshold = kMaxSmall;
    p->ctas_per_sm = 0;           // occupancy-derived
    p->sample_count = 31;
    p->offset_mode = 0;
    p->schedule = 0;
    p->seed = 0x5EED5EED12345678ull;
}

void normalise_plan(tsqs_plan *p) {
    tsqs_plan d;
    fill_default_plan(TSQS_I32, 0, &d);
    if (p->small_threshold <= 0) p->small_threshold = d.small_threshold;
    if (p->small_threshold > kMaxSmall) p->small_threshold = kMaxSmall;
    if (p->small_threshold < 512) p->small_threshold = 512;
    if (p->sample_count <= 0) p->sample_count = d.sample_count;
    if (p->sample_count > kMaxSamples) p->sample_count = kMaxSamples;
    if ((p->sample_count & 1) == 0) p->sample_count -= 1;
    if (p->seed == 0) p->seed = d.seed;
    if (p->ctas_per_sm < 0) p->ctas_per_sm = 0;
    if (p->offset_mode != 1) p->offset_mode = 0;
    if (p->schedule < 0 || p->schedule > 2) p->schedule = 0;
    if (p->tile_items < 0 || p->tile_items >= kPartVariants) p->tile_items = 0;
}

}  // namespace

struct tsqs_ctx {
    tsqs_plan plan{};
    int device = -1;
    int sms = 0;
    Job *d_job = nullptr;
    Ctl *d_ctl = nullptr;
    char *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaGraph_t graph[8] = {};
    cudaGraphExec_t exec[8] = {};
    // the task-parallel schedule's graphs per kind: [0] with the leaf pass of k_leaf,
    // [1] with k_leaf_small (small inputs)
    cudaGraph_t graph_task[8][2] = {};
    cudaGraphExec_t exec_task[8][2] = {};
    int part_grid[8] = {}, leaf_grid[8] = {}, leaf_small_grid[8] = {}, task_grid[8] = {}, deep_grid[8] = {};
    bool attrs_set[8] = {};
    cudaEvent_t done_ev = nullptr;
    bool ev_valid = false;
    unsigned int *h_cont = nullptr;    // pinned word for the host-driven loop
    char *wide_rec = nullptr;          // large elements: (key, index) records
    size_t wide_rec_bytes = 0;
    char *wide_tmp = nullptr;          // large elements: the gathered copy
    size_t wide_tmp_bytes = 0;
    // host-array streaming: device staging slots, the two copy streams, their events
    char *stage[3] = {};
    size_t stage_bytes = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_entry = nullptr, ev_in[3] = {}, ev_sorted[3] = {}, ev_out[3] = {};
    uint32_t *d_item_status = nullptr;
    size_t item_status_cap = 0;
    // caller-held graphs (tsqs_graph_sort_segmented): each exec with its graph, the
    // setup node whose Job argument a later call updates, and its key kind
    // variant: 0 level by level, 1 task-parallel, 2 task-parallel with the small-input leaf
    struct Held { cudaGraphExec_t exec; cudaGraph_t graph; cudaGraphNode_t setup; int kind; int variant; };
    std::vector<Held> held;
    std::recursive_mutex mu;
};

namespace {

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            if (getenv("TSQS_VERBOSE"))                                                  \
                fprintf(stderr, "tsqs: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
            return TSQS_ECUDA;                                                           \
        }                                                                                \
    } while (0)

int ctx_init_device(tsqs_ctx *c) {
    if (c->device >= 0) return TSQS_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaMalloc((void **)&c->d_job, sizeof(Job)));
    CK(cudaMalloc((void **)&c->d_ctl, sizeof(Ctl)));
    CK(cudaMemset(c->d_ctl, 0, sizeof(Ctl)));
    CK(cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming));
    CK(cudaHostAlloc((void **)&c->h_cont, sizeof(unsigned int), cudaHostAllocDefault));
    c->device = dev;
    return TSQS_OK;
}

int ctx_kind_setup(tsqs_ctx *c, const KindOps *o) {
    const int k = o->kind;
    if (c->attrs_set[k]) return TSQS_OK;
    CK(cudaFuncSetAttribute(o->k_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, o->leaf_smem));
    CK(cudaFuncSetAttribute(o->k_leaf_small, cudaFuncAttributeMaxDynamicSharedMemorySize, o->leaf_small_smem));
    CK(cudaFuncSetAttribute(o->k_deep_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, o->deep_smem));
    CK(cudaFuncSetAttribute(o->k_deep_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, o->deep_smem));
    CK(cudaFuncSetAttribute(o->k_deep_all, cudaFuncAttributeMaxDynamicSharedMemorySize, o->deep_smem));
    for (int v = 0; v < kPartVariants; v++)
        CK(cudaFuncSetAttribute(o->part[v].k_partition, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                o->part[v].smem));
    const PartVariant &pv = part_of(o, c->plan);
    int occ_p = 0, occ_l = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, pv.k_partition, pv.threads, pv.smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, o->k_leaf, o->leaf_block, o->leaf_smem));
    int occ_ls = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ls, o->k_leaf_small, o->leaf_small_block,
                                                     o->leaf_small_smem));
    c->leaf_small_grid[k] = std::max(1, occ_ls) * c->sms;
    int occ_t = 0, occ_d = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, o->k_task, o->task_block, 0));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, o->k_deep_all, 512, o->deep_smem));
    // the cooperative depth-guard kernel: every block resident
    c->deep_grid[k] = std::max(1, occ_d) * c->sms;
    if (c->plan.ctas_per_sm > 0) occ_p = std::min(occ_p, c->plan.ctas_per_sm);
    c->part_grid[k] = std::max(1, occ_p) * c->sms;
    c->leaf_grid[k] = std::max(1, occ_l) * c->sms;
    // every block of the task kernel resident at once (the end-of-work rows cover one
    // claim per block)
    c->task_grid[k] = std::min<int>(std::max(1, occ_t) * c->sms, (int)kTaskGridMax);
    c->attrs_set[k] = true;
    return TSQS_OK;
}

// Waits for all work that may still use the scratch (every stream that sorted with it).
int ctx_quiesce(tsqs_ctx *c) {
    if (c->ev_valid) CK(cudaEventSynchronize(c->done_ev));
    return TSQS_OK;
}

// Tile size of the task kernel when a sort of n elements under plan p runs the task
// schedule, else 0 (no task tables in the layout).
int task_tile_for(const KindOps *o, const tsqs_plan &p, size_t n) {
    return task_schedule(p, n) ? o->task_tile : 0;
}

int ctx_ensure_scratch(tsqs_ctx *c, const KindOps *o, size_t n, size_t nseg) {
    const size_t es = (size_t)o->elem_size;
    const Layout L = make_layout(n, nseg, es, c->plan, part_of(o, c->plan).tile, o->leaf_max,
                                 task_tile_for(o, c->plan, n));
    if (c->scratch && L.total <= c->scratch_bytes) return TSQS_OK;
    int rc = ctx_quiesce(c);
    if (rc) return rc;
    if (c->scratch) { cudaFree(c->scratch); c->scratch = nullptr; c->scratch_bytes = 0; }
    const size_t want = L.total + L.total / 8;          // headroom against regrowth
    if (cudaMalloc((void **)&c->scratch, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc((void **)&c->scratch, L.total) != cudaSuccess) {
            cudaGetLastError();
            c->scratch = nullptr;
            return TSQS_ENOMEM;
        }
        c->scratch_bytes = L.total;
    } else {
        c->scratch_bytes = want;
    }
    return TSQS_OK;
}

// Fills the per-call description.  The scratch buffer gets the same 16-byte phase as
// base so that both buffers use the same tile geometry.
// task: the call runs the task schedule (its tables are filled in, and `tile` is the
// task kernel's).
int make_job(tsqs_ctx *c, const KindOps *o, void *base, size_t n, const uint64_t *offs,
             size_t nseg, Job *j, bool task = false) {
    const size_t es = (size_t)o->elem_size;
    const int task_tile = task ? o->task_tile : 0;
    const Layout L = make_layout(n, nseg, es, c->plan, part_of(o, c->plan).tile, o->leaf_max, task_tile);
    if (L.total > c->scratch_bytes) return TSQS_EINTERNAL;
    memset(j, 0, sizeof(*j));
    const uintptr_t b = (uintptr_t)base;
    j->base = base;
    j->out = base;
    j->alt = c->scratch + L.alt_off + (b & 15u);
    j->n = n;
    j->seg_offsets = offs;
    j->nseg = offs ? nseg : 1;
    j->front[0] = (SegDesc *)(c->scratch + L.front_off[0]);
    j->front[1] = (SegDesc *)(c->scratch + L.front_off[1]);
    j->leaves = (LeafItem *)(c->scratch + L.leaves_off);
    j->tile_seg = (uint32_t *)(c->scratch + L.tseg_off);
    j->tile_status = (unsigned long long *)(c->scratch + L.tstat_off);
    j->seg_done = (uint32_t *)(c->scratch + L.done_off);
    j->seg_cursor = (unsigned long long *)(c->scratch + L.cursor_off);
    j->presort = (uint32_t *)(c->scratch + L.presort_off);
    j->deep = (LeafItem *)(c->scratch + L.deep_off);
    j->deep_tiles = (uint32_t *)(c->scratch + L.dtiles_off);
    j->deep_chunks = (uint32_t *)(c->scratch + L.dchunks_off);
    j->cap_deep = L.cap_front;
    j->cap_front = L.cap_front;
    j->cap_tiles = L.cap_tiles;
    j->cap_leaves = L.cap_leaves;
    j->leaf_defer = g_debug_defer ? std::min(g_debug_defer, L.leaf_defer) : L.leaf_defer;
    j->small_T = (uint32_t)eff_threshold(c->plan, o->leaf_max);
    j->samples = (uint32_t)c->plan.sample_count;
    j->vec_off = (uint32_t)((b / es) % (16 / es));
    j->spin_limit = g_debug_spin ? g_debug_spin : kDefaultSpin;
    j->pad = g_debug_withhold == 1 ? 2u : g_debug_withhold == 2 ? 4u : 0u;
    // depth cap: far above what sampled medians need (about log2(n / T) + a few)
    unsigned lg = 1;
    while ((1ull << lg) < (unsigned long long)n + 1 && lg < 63) lg++;
    j->max_levels = 256u + 8u * lg;
    j->deep_level = g_debug_deep ? g_debug_deep : 2u * lg + 8u;
    j->offset_mode = (c->plan.offset_mode == 1 || g_debug_withhold == 1) ? 1u : 0u;
    j->tile = (uint32_t)part_of(o, c->plan).tile;
    j->seed = c->plan.seed;
    if (task_tile) {
        j->tile = (uint32_t)task_tile;
        j->tseg = (TaskSeg *)(c->scratch + L.ttask_off);
        j->trow = (unsigned long long *)(c->scratch + L.trow_off);
        j->cap_tseg = L.cap_tseg;
        j->cap_trow = L.cap_trow;
        // blocks that take part: as many as the tiles one depth can hold at once (the keys'
        // tiles plus two partial tiles per segment), at most the launched grid; the others
        // return at once and leave their SMs to other streams' work
        const size_t T = eff_threshold(c->plan, o->leaf_max);
        const size_t want = n / (size_t)task_tile + 2 * (n / (T + 1)) + 8;
        j->task_grid = (uint32_t)std::min<size_t>(want, (size_t)c->task_grid[o->kind]);
    }
    return TSQS_OK;
}

int add_deep_branch(tsqs_ctx *c, const KindOps *o, cudaGraph_t g, cudaGraphNode_t after,
                    cudaGraphConditionalHandle h_if);

// Adds the presortedness nodes to graph g after `dep` (nullptr: none): the orientation
// kernel, then IF (it flagged a candidate) { full check ; finishing pass }.  *last is the
// node the sort's next node depends on.
int add_presort_nodes(tsqs_ctx *c, const KindOps *o, cudaGraph_t g, const cudaGraphNode_t *dep,
                      cudaGraphNode_t *last) {
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    cudaGraphConditionalHandle h_pre;
    CK(cudaGraphConditionalHandleCreate(&h_pre, g, 0, cudaGraphCondAssignDefault));
    void *argso[] = {&pj, &pc, &h_pre};
    cudaKernelNodeParams kp{};
    kp.func = (void *)o->k_orient_if;
    kp.gridDim = dim3(c->sms * 4);
    kp.blockDim = dim3(256);
    kp.kernelParams = argso;
    cudaGraphNode_t n_ori, n_if, n_chk, n_pre;
    CK(cudaGraphAddKernelNode(&n_ori, g, dep, dep ? 1 : 0, &kp));
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_pre;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    CK(cudaGraphAddNode(&n_if, g, &n_ori, nullptr, 1, &ip));
    cudaGraph_t body = ip.conditional.phGraph_out[0];
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_check;
    kp.gridDim = dim3(c->sms * 4);
    kp.blockDim = dim3(256);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_chk, body, nullptr, 0, &kp));
    kp.func = (void *)o->k_presort;
    CK(cudaGraphAddKernelNode(&n_pre, body, &n_chk, 1, &kp));
    *last = n_if;
    return TSQS_OK;
}

// Adds the nodes of one whole sort of kind o to graph g, the first of them depending on
// `dep` (nullptr: none).  Every kernel reads the per-call Job from c->d_job.
int build_sort_nodes(tsqs_ctx *c, const KindOps *o, cudaGraph_t g, const cudaGraphNode_t *dep) {
    const int k = o->kind;
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};

    // presortedness: sample orientation; full check and finish only for candidates
    cudaGraphNode_t n_pre, n_init;
    int rc = add_presort_nodes(c, o, g, dep, &n_pre);
    if (rc) return rc;
    cudaKernelNodeParams kp{};
    kp.func = (void *)o->k_init;
    kp.gridDim = dim3(c->sms * 2);
    kp.blockDim = dim3(256);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_init, g, &n_pre, 1, &kp));

    // outer loop: { level loop ; leaf pass ; control }.  The level loop pauses only when
    // the leaf queue could not take another level's items; normally the outer body runs
    // once and its leaf pass is the single one after all levels.
    cudaGraphConditionalHandle h_out;
    CK(cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cpo{};
    cpo.type = cudaGraphNodeTypeConditional;
    cpo.conditional.handle = h_out;
    cpo.conditional.type = cudaGraphCondTypeWhile;
    cpo.conditional.size = 1;
    cudaGraphNode_t n_outer;
    CK(cudaGraphAddNode(&n_outer, g, &n_init, nullptr, 1, &cpo));
    cudaGraph_t outer = cpo.conditional.phGraph_out[0];

    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_loop;
    CK(cudaGraphAddNode(&n_loop, outer, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    cudaGraphNode_t n_piv, n_part, n_fin, n_last, n_octl;
    int leaf_last = 1;
    void *argsl_last[] = {&pj, &pc, &leaf_last};
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_pivot;
    kp.gridDim = dim3(c->sms * 4);
    kp.blockDim = dim3(o->pivot_block);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_piv, body, nullptr, 0, &kp));
    kp = cudaKernelNodeParams{};
    const PartVariant &pv = part_of(o, c->plan);
    kp.func = (void *)pv.k_partition;
    kp.gridDim = dim3(c->part_grid[k]);
    kp.blockDim = dim3(pv.threads);
    kp.sharedMemBytes = (unsigned)pv.smem;
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_part, body, &n_piv, 1, &kp));
    int use_h = 1;
    unsigned int unused = 0;
    void *argsf[] = {&pj, &pc, &h, &use_h, &unused};
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_finish;
    kp.gridDim = dim3(c->sms);
    kp.blockDim = dim3(128);
    kp.kernelParams = argsf;
    CK(cudaGraphAddKernelNode(&n_fin, body, &n_part, 1, &kp));
    // the leaf pass after the level loop: every queued item, then the queue is empty
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_leaf;
    kp.gridDim = dim3(c->leaf_grid[k]);
    kp.blockDim = dim3(o->leaf_block);
    kp.sharedMemBytes = (unsigned)o->leaf_smem;
    kp.kernelParams = argsl_last;
    CK(cudaGraphAddKernelNode(&n_last, outer, &n_loop, 1, &kp));
    // the depth guard's branch after the loops, under an IF node set by the control
    cudaGraphConditionalHandle h_if;
    CK(cudaGraphConditionalHandleCreate(&h_if, g, 0, cudaGraphCondAssignDefault));
    const Ctl *pcc = pc;
    void *argso[] = {&pcc, &h, &h_out, &h_if};
    kp = cudaKernelNodeParams{};
    kp.func = (void *)k_outer_control;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = argso;
    CK(cudaGraphAddKernelNode(&n_octl, outer, &n_last, 1, &kp));
    return add_deep_branch(c, o, g, n_outer, h_if);
}

// Adds the depth guard's branch to graph g after node `after`: IF (h_if) some segment
// reached the bound, prep, tile sorts, a WHILE over the stages, finish.
int add_deep_branch(tsqs_ctx *c, const KindOps *o, cudaGraph_t g, cudaGraphNode_t after,
                    cudaGraphConditionalHandle h_if) {
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    cudaKernelNodeParams kp{};
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_if;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t n_if;
    CK(cudaGraphAddNode(&n_if, g, &after, nullptr, 1, &ip));
    cudaGraph_t dg = ip.conditional.phGraph_out[0];
    cudaGraphConditionalHandle hd;
    CK(cudaGraphConditionalHandleCreate(&hd, dg, 0, cudaGraphCondAssignDefault));
    int use_hd = 1;
    void *argsd[] = {&pj, &pc, &hd, &use_hd};
    cudaGraphNode_t n_dprep, n_dtiles, n_dloop, n_dstage, n_dfin;
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_deep_prep;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(512);
    kp.kernelParams = argsd;
    CK(cudaGraphAddKernelNode(&n_dprep, dg, nullptr, 0, &kp));
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_deep_tiles;
    kp.gridDim = dim3(c->sms * 2);
    kp.blockDim = dim3(512);
    kp.sharedMemBytes = (unsigned)o->deep_smem;
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_dtiles, dg, &n_dprep, 1, &kp));
    cudaGraphNodeParams dp{};
    dp.type = cudaGraphNodeTypeConditional;
    dp.conditional.handle = hd;
    dp.conditional.type = cudaGraphCondTypeWhile;
    dp.conditional.size = 1;
    CK(cudaGraphAddNode(&n_dloop, dg, &n_dtiles, nullptr, 1, &dp));
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_deep_stage;
    kp.gridDim = dim3(c->sms * 2);
    kp.blockDim = dim3(512);
    kp.sharedMemBytes = (unsigned)o->deep_smem;
    kp.kernelParams = argsd;
    CK(cudaGraphAddKernelNode(&n_dstage, dp.conditional.phGraph_out[0], nullptr, 0, &kp));
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_deep_finish;
    kp.gridDim = dim3(c->sms * 2);
    kp.blockDim = dim3(512);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_dfin, dg, &n_dloop, 1, &kp));
    return TSQS_OK;
}

int ctx_build_graph(tsqs_ctx *c, const KindOps *o) {
    const int k = o->kind;
    if (c->exec[k]) return TSQS_OK;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    int rc = build_sort_nodes(c, o, g, nullptr);
    cudaGraphExec_t ex = nullptr;
    if (rc == TSQS_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) rc = TSQS_ECUDA;
    if (rc) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return rc;
    }
    c->graph[k] = g;
    c->exec[k] = ex;
    return TSQS_OK;
}

// The task schedule's graph for kind o:
//     orient -> check -> presort -> task init -> task kernel -> leaf pass -> depth guard
// with the depth guard as one cooperative kernel (no conditional node).
int build_task_nodes(tsqs_ctx *c, const KindOps *o, cudaGraph_t g, const cudaGraphNode_t *dep,
                     bool small_leaf) {
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    // presortedness as a plain chain: at the sizes this graph serves, an IF node around the
    // check and finishing passes costs more than their two launches that return at once
    cudaKernelNodeParams kp{};
    cudaGraphNode_t n_ori, n_chk, n_pre, n_init, n_task, n_leaf;
    kp.func = (void *)o->k_orient;
    kp.gridDim = dim3(c->sms * 4);
    kp.blockDim = dim3(256);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_ori, g, dep, dep ? 1 : 0, &kp));
    kp.func = (void *)o->k_check;
    CK(cudaGraphAddKernelNode(&n_chk, g, &n_ori, 1, &kp));
    kp.func = (void *)o->k_presort;
    CK(cudaGraphAddKernelNode(&n_pre, g, &n_chk, 1, &kp));
    kp.func = (void *)o->k_task_init;
    kp.gridDim = dim3(c->sms * 2);
    CK(cudaGraphAddKernelNode(&n_init, g, &n_pre, 1, &kp));
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_task;
    kp.gridDim = dim3(c->task_grid[o->kind]);
    kp.blockDim = dim3(o->task_block);
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_task, g, &n_init, 1, &kp));
    int leaf_last = 1;
    void *argsl[] = {&pj, &pc, &leaf_last};
    kp = cudaKernelNodeParams{};
    kp.func = small_leaf ? (void *)o->k_leaf_small : (void *)o->k_leaf;
    kp.gridDim = dim3(small_leaf ? c->leaf_small_grid[o->kind] : c->leaf_grid[o->kind]);
    kp.blockDim = dim3(small_leaf ? o->leaf_small_block : o->leaf_block);
    kp.sharedMemBytes = (unsigned)(small_leaf ? o->leaf_small_smem : o->leaf_smem);
    kp.kernelParams = argsl;
    CK(cudaGraphAddKernelNode(&n_leaf, g, &n_task, 1, &kp));
    // the depth guard as one cooperative kernel, which returns at once when no segment
    // reached the bound: a graph without conditional nodes launches 7-8 us faster at the
    // sizes this schedule serves
    cudaGraphNode_t n_deep;
    kp = cudaKernelNodeParams{};
    kp.func = (void *)o->k_deep_all;
    kp.gridDim = dim3(c->deep_grid[o->kind]);
    kp.blockDim = dim3(512);
    kp.sharedMemBytes = (unsigned)o->deep_smem;
    kp.kernelParams = args2;
    CK(cudaGraphAddKernelNode(&n_deep, g, &n_leaf, 1, &kp));
    cudaKernelNodeAttrValue coop{};
    coop.cooperative = 1;
    CK(cudaGraphKernelNodeSetAttribute(n_deep, cudaKernelNodeAttributeCooperative, &coop));
    return TSQS_OK;
}

int ctx_build_task_graph(tsqs_ctx *c, const KindOps *o, int v) {
    const int k = o->kind;
    if (c->exec_task[k][v]) return TSQS_OK;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    int rc = build_task_nodes(c, o, g, nullptr, v == 1);
    cudaGraphExec_t ex = nullptr;
    if (rc == TSQS_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) rc = TSQS_ECUDA;
    if (rc) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return rc;
    }
    c->graph_task[k][v] = g;
    c->exec_task[k][v] = ex;
    return TSQS_OK;
}

// Depth guard, host-driven (the graph runs the same kernels under a WHILE node).
cudaError_t run_deep_host(tsqs_ctx *c, const KindOps *o, cudaStream_t s, Job *pj, Ctl *pc) {
    cudaGraphConditionalHandle hd = 0;
    int use_hd = 0;
    void *argsd[] = {&pj, &pc, &hd, &use_hd};
    void *args2[] = {&pj, &pc};
    cudaError_t e;
    if ((e = cudaLaunchKernel(o->k_deep_prep, dim3(1), dim3(512), argsd, 0, s)) != cudaSuccess) return e;
    if ((e = cudaLaunchKernel(o->k_deep_tiles, dim3(c->sms * 2), dim3(512), args2, (size_t)o->deep_smem, s)) != cudaSuccess) return e;
    for (int it = 0; it < 4096; it++) {
        if ((e = cudaMemcpyAsync(c->h_cont, &pc->deep_cont, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (!*c->h_cont) break;
        if ((e = cudaLaunchKernel(o->k_deep_stage, dim3(c->sms * 2), dim3(512), argsd, (size_t)o->deep_smem, s)) != cudaSuccess) return e;
    }
    return cudaLaunchKernel(o->k_deep_finish, dim3(c->sms * 2), dim3(512), args2, 0, s);
}

int validate(void *base, size_t nmemb, size_t elem_size, int key_kind) {
    const size_t es = kind_size(key_kind);
    if (!es || es != elem_size) return TSQS_EINVAL;
    if (nmemb > 1 && !base) return TSQS_EINVAL;
    const size_t align = es == 16 ? 16 : es;
    if ((uintptr_t)base % align) return TSQS_EINVAL;
    return TSQS_OK;
}

// Queues one sort (single segment when offs == nullptr).
int ctx_launch(tsqs_ctx *c, void *base, size_t n, const uint64_t *offs, size_t nseg,
               size_t elem_size, int key_kind, cudaStream_t stream, void *out = nullptr) {
    int rc = validate(base, n, elem_size, key_kind);
    if (rc) return rc;
    if (!offs && n >= (1ull << 31)) return TSQS_EINVAL;
    if (offs && nseg == 0) return TSQS_OK;
    if (!offs && n <= 1) return TSQS_OK;
    if (offs && n == 0) return TSQS_OK;
    const KindOps *o = get_ops(key_kind);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if ((rc = ctx_init_device(c))) return rc;
    if ((rc = ctx_kind_setup(c, o))) return rc;
    if ((rc = ctx_ensure_scratch(c, o, n, offs ? nseg : 1))) return rc;
    const bool task = task_schedule(c->plan, n);
    const int tv = (task && n <= kSmallLeafN) ? 1 : 0;       // task graph variant
    if ((rc = task ? ctx_build_task_graph(c, o, tv) : ctx_build_graph(c, o))) return rc;
    Job j;
    if ((rc = make_job(c, o, base, n, offs, nseg, &j, task))) return rc;
    if (out) j.out = out;
    if (c->ev_valid) CK(cudaStreamWaitEvent(stream, c->done_ev, 0));
    k_setup<<<1, 256, 0, stream>>>(c->d_job, c->d_ctl, j);
    CK(cudaGetLastError());
    CK(cudaGraphLaunch(task ? c->exec_task[key_kind][tv] : c->exec[key_kind], stream));
    CK(cudaEventRecord(c->done_ev, stream));
    c->ev_valid = true;
    return TSQS_OK;
}

std::mutex g_default_mu;
tsqs_ctx *g_default = nullptr;

tsqs_ctx *default_ctx() {
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (!g_default) g_default = tsqs_ctx_create(nullptr);
    return g_default;
}

int read_status(tsqs_ctx *c, cudaStream_t stream, bool clear) {
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (c->device < 0) return TSQS_OK;
    CK(cudaStreamSynchronize(stream));
    if (c->ev_valid) CK(cudaEventSynchronize(c->done_ev));
    uint32_t st = 0;
    CK(cudaMemcpy(&st, &c->d_ctl->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (clear && st) CK(cudaMemset(&c->d_ctl->status, 0, sizeof(uint32_t)));
    return (int)st;
}

int ctx_stream_setup(tsqs_ctx *c, size_t slot_bytes, size_t count) {
    if (!c->s_in) {
        CK(cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->ev_entry, cudaEventDisableTiming));
        for (int k = 0; k < 3; k++) {
            CK(cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->ev_sorted[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming));
        }
    }
    // every call ends with its streams drained, so the slots are idle here
    if (slot_bytes > c->stage_bytes) {
        for (int k = 0; k < 3; k++) {
            if (c->stage[k]) cudaFree(c->stage[k]);
            c->stage[k] = nullptr;
        }
        c->stage_bytes = 0;
        for (int k = 0; k < 3; k++) {
            if (cudaMalloc((void **)&c->stage[k], slot_bytes) != cudaSuccess) {
                cudaGetLastError();
                for (int q = 0; q <= k; q++) {
                    if (c->stage[q]) cudaFree(c->stage[q]);
                    c->stage[q] = nullptr;
                }
                return TSQS_ENOMEM;
            }
        }
        c->stage_bytes = slot_bytes;
    }
    if (count > c->item_status_cap) {
        if (c->d_item_status) cudaFree(c->d_item_status);
        c->d_item_status = nullptr;
        c->item_status_cap = 0;
        if (cudaMalloc((void **)&c->d_item_status, count * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return TSQS_ENOMEM;
        }
        c->item_status_cap = count;
    }
    return TSQS_OK;
}

}  // namespace

// =================================================================================
// C-ABI
// =================================================================================

extern "C" {

tsqs_ctx *tsqs_ctx_create(const tsqs_plan *plan) {
    tsqs_ctx *c = new (std::nothrow) tsqs_ctx();
    if (!c) return nullptr;
    if (plan) c->plan = *plan;
    else fill_default_plan(TSQS_I32, 0, &c->plan);
    normalise_plan(&c->plan);
    return c;
}

void tsqs_ctx_destroy(tsqs_ctx *c) {
    if (!c) return;
    {
        std::lock_guard<std::recursive_mutex> lk(c->mu);
        ctx_quiesce(c);
        for (int k = 0; k < 8; k++) {
            if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
            if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
            for (int v = 0; v < 2; v++) {
                if (c->exec_task[k][v]) cudaGraphExecDestroy(c->exec_task[k][v]);
                if (c->graph_task[k][v]) cudaGraphDestroy(c->graph_task[k][v]);
            }
        }
        for (auto &h : c->held) {
            cudaGraphExecDestroy(h.exec);
            cudaGraphDestroy(h.graph);
        }
        c->held.clear();
        if (c->scratch) cudaFree(c->scratch);
        if (c->wide_rec) cudaFree(c->wide_rec);
        if (c->wide_tmp) cudaFree(c->wide_tmp);
        for (int k = 0; k < 3; k++) {
            if (c->stage[k]) cudaFree(c->stage[k]);
            if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
            if (c->ev_sorted[k]) cudaEventDestroy(c->ev_sorted[k]);
            if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
        }
        if (c->ev_entry) cudaEventDestroy(c->ev_entry);
        if (c->s_in) cudaStreamDestroy(c->s_in);
        if (c->s_out) cudaStreamDestroy(c->s_out);
        if (c->d_item_status) cudaFree(c->d_item_status);
        if (c->d_job) cudaFree(c->d_job);
        if (c->d_ctl) cudaFree(c->d_ctl);
        if (c->done_ev) cudaEventDestroy(c->done_ev);
        if (c->h_cont) cudaFreeHost(c->h_cont);
    }
    delete c;
}

int tsqs_ctx_set_plan(tsqs_ctx *c, const tsqs_plan *plan) {
    if (!c || !plan) return TSQS_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int rc = ctx_quiesce(c);
    if (rc) return rc;
    c->plan = *plan;
    normalise_plan(&c->plan);
    for (int k = 0; k < 8; k++) {            // grids depend on the plan
        if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
        if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
        for (int v = 0; v < 2; v++) {
            if (c->exec_task[k][v]) cudaGraphExecDestroy(c->exec_task[k][v]);
            if (c->graph_task[k][v]) cudaGraphDestroy(c->graph_task[k][v]);
            c->exec_task[k][v] = nullptr;
            c->graph_task[k][v] = nullptr;
        }
        c->exec[k] = nullptr;
        c->graph[k] = nullptr;
        c->attrs_set[k] = false;
    }
    return TSQS_OK;
}

int tsqs_ctx_get_plan(const tsqs_ctx *c, tsqs_plan *out) {
    if (!c || !out) return TSQS_EINVAL;
    *out = c->plan;
    return TSQS_OK;
}

int tsqs_ctx_sort(tsqs_ctx *c, void *base, size_t nmemb, size_t elem_size, int key_kind,
                  void *stream) {
    if (!c) return TSQS_EINVAL;
    return ctx_launch(c, base, nmemb, nullptr, 0, elem_size, key_kind, (cudaStream_t)stream);
}

int tsqs_ctx_sort_segmented(tsqs_ctx *c, void *base, size_t nmemb_total,
                            const uint64_t *d_seg_offsets, size_t nseg, size_t elem_size,
                            int key_kind, void *stream) {
    if (!c || (nseg && !d_seg_offsets)) return TSQS_EINVAL;
    return ctx_launch(c, base, nmemb_total, d_seg_offsets, nseg, elem_size, key_kind,
                      (cudaStream_t)stream);
}

int tsqs_graph_sort_segmented(tsqs_ctx *c, void *base, size_t nmemb_total,
                              const uint64_t *d_seg_offsets, size_t nseg, size_t elem_size,
                              int key_kind, void *stream, void **graph_exec) {
    if (!c || !graph_exec || (nseg && !d_seg_offsets)) return TSQS_EINVAL;
    int rc = validate(base, nmemb_total, elem_size, key_kind);
    if (rc) return rc;
    const uint64_t *offs = d_seg_offsets;
    if (!offs && nmemb_total >= (1ull << 31)) return TSQS_EINVAL;
    if ((offs && (nseg == 0 || nmemb_total == 0)) || (!offs && nmemb_total <= 1))
        return TSQS_OK;                                   // nothing to sort, no graph made
    const KindOps *o = get_ops(key_kind);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    tsqs_ctx::Held *h = nullptr;
    if (*graph_exec) {
        for (auto &x : c->held)
            if ((void *)x.exec == *graph_exec) h = &x;
        if (!h || h->kind != key_kind) return TSQS_EINVAL;     // not this ctx's, or another kind
    }
    if ((rc = ctx_init_device(c))) return rc;
    if ((rc = ctx_kind_setup(c, o))) return rc;
    if ((rc = ctx_ensure_scratch(c, o, nmemb_total, offs ? nseg : 1))) return rc;
    const bool task = task_schedule(c->plan, nmemb_total);
    const int variant = task ? (nmemb_total <= kSmallLeafN ? 2 : 1) : 0;
    Job j;
    if ((rc = make_job(c, o, base, nmemb_total, offs, offs ? nseg : 1, &j, task))) return rc;
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args[] = {&pj, &pc, &j};
    cudaKernelNodeParams kp{};
    kp.func = (void *)k_setup;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    if (h && (h->variant == 0) != (variant == 0)) {
        // this size takes the other schedule: the graph is rebuilt under a new handle (a
        // task graph keeps the leaf kernel it was built with: either sorts every item)
        ctx_quiesce(c);
        cudaGraphExecDestroy(h->exec);
        cudaGraphDestroy(h->graph);
        c->held.erase(c->held.begin() + (h - c->held.data()));
        h = nullptr;
        *graph_exec = nullptr;
    }
    if (!h) {
        tsqs_ctx::Held nh{};
        nh.kind = key_kind;
        nh.variant = variant;
        CK(cudaGraphCreate(&nh.graph, 0));
        rc = cudaGraphAddKernelNode(&nh.setup, nh.graph, nullptr, 0, &kp) == cudaSuccess
                 ? (task ? build_task_nodes(c, o, nh.graph, &nh.setup, variant == 2)
                         : build_sort_nodes(c, o, nh.graph, &nh.setup))
                 : TSQS_ECUDA;
        if (rc == TSQS_OK && cudaGraphInstantiate(&nh.exec, nh.graph, 0) != cudaSuccess) rc = TSQS_ECUDA;
        if (rc) {
            cudaGetLastError();
            cudaGraphDestroy(nh.graph);
            return rc;
        }
        c->held.push_back(nh);
        h = &c->held.back();
        *graph_exec = (void *)nh.exec;
    } else {
        CK(cudaGraphExecKernelNodeSetParams(h->exec, h->setup, &kp));
    }
    if (c->ev_valid) CK(cudaStreamWaitEvent(s, c->done_ev, 0));
    CK(cudaGraphLaunch(h->exec, s));
    CK(cudaEventRecord(c->done_ev, s));
    c->ev_valid = true;
    return TSQS_OK;
}

void tsqs_graph_exec_destroy(tsqs_ctx *c, void *graph_exec) {
    if (!c || !graph_exec) return;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    for (size_t i = 0; i < c->held.size(); i++) {
        if ((void *)c->held[i].exec != graph_exec) continue;
        ctx_quiesce(c);
        cudaGraphExecDestroy(c->held[i].exec);
        cudaGraphDestroy(c->held[i].graph);
        c->held.erase(c->held.begin() + (long)i);
        return;
    }
}

int tsqs_ctx_reserve(tsqs_ctx *c, size_t nmemb_total, size_t nseg, size_t elem_size) {
    if (!c) return TSQS_EINVAL;
    int kind = elem_size == 4 ? TSQS_U32 : elem_size == 8 ? TSQS_U64 : elem_size == 16 ? TSQS_U64_U64_REC : 0;
    const KindOps *o = get_ops(kind);
    if (!o) return TSQS_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int rc = ctx_init_device(c);
    if (rc) return rc;
    return ctx_ensure_scratch(c, o, nmemb_total, nseg ? nseg : 1);
}

size_t tsqs_ctx_scratch_bytes(const tsqs_ctx *c) { return c ? c->scratch_bytes : 0; }

size_t tsqs_scratch_bytes_for(size_t nmemb_total, size_t nseg, size_t elem_size,
                              const tsqs_plan *plan) {
    int kind = elem_size == 4 ? TSQS_U32 : elem_size == 8 ? TSQS_U64 : elem_size == 16 ? TSQS_U64_U64_REC : 0;
    const KindOps *o = get_ops(kind);
    if (!o) return 0;
    tsqs_plan p;
    if (plan) p = *plan; else fill_default_plan(kind, nmemb_total, &p);
    normalise_plan(&p);
    return make_layout(nmemb_total, nseg ? nseg : 1, elem_size, p, part_of(o, p).tile, o->leaf_max,
                       task_tile_for(o, p, nmemb_total)).total;
}

int tsqs_ctx_device_status(tsqs_ctx *c, void *stream) {
    if (!c) return TSQS_EINVAL;
    return read_status(c, (cudaStream_t)stream, true);
}

int tsqs_ctx_stats(tsqs_ctx *c, void *stream, tsqs_stats *out) {
    if (!c || !out) return TSQS_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    memset(out, 0, sizeof(*out));
    if (c->device < 0) return TSQS_OK;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (c->ev_valid) CK(cudaEventSynchronize(c->done_ev));
    Ctl h;
    CK(cudaMemcpy(&h, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    out->levels = h.levels_done;
    out->max_frontier = h.max_front;
    out->partition_keys = h.partition_keys;
    out->leaf_sorted_keys = h.leaf_sorted;
    out->leaf_filled_keys = h.leaf_filled;
    out->leaf_items = h.leaf_items;
    out->presorted_keys = h.presorted;
    out->deep_sorted_keys = h.deep_keys;
    // levels run (level-by-level schedule) or depths reached (task schedule)
    const uint32_t nl = std::min<uint32_t>(std::max(h.level, h.levels_done), (uint32_t)kStatLevels);
    out->level_keys_count = nl;
    for (uint32_t i = 0; i < nl; i++) out->level_keys[i] = h.level_keys[i];
    return TSQS_OK;
}

int tsqs_plan_default(int key_kind, size_t n_hint, tsqs_plan *out) {
    if (!out || !get_ops(key_kind)) return TSQS_EINVAL;
    if (n_hint && tsqs_cached_plan(key_kind, n_hint, 1, out)) {
        normalise_plan(out);
        return TSQS_OK;
    }
    fill_default_plan(key_kind, n_hint, out);
    normalise_plan(out);
    return TSQS_OK;
}

int tsqs_sort(void *base, size_t nmemb, size_t elem_size, int key_kind, void *stream) {
    tsqs_ctx *c = default_ctx();
    if (!c) return TSQS_ENOMEM;
    return tsqs_ctx_sort(c, base, nmemb, elem_size, key_kind, stream);
}

int tsqs_sort_segmented(void *base, size_t nmemb_total, const uint64_t *d_seg_offsets,
                        size_t nseg, size_t elem_size, int key_kind, void *stream) {
    tsqs_ctx *c = default_ctx();
    if (!c) return TSQS_ENOMEM;
    return tsqs_ctx_sort_segmented(c, base, nmemb_total, d_seg_offsets, nseg, elem_size,
                                   key_kind, stream);
}

void tsqs_free_storage(void) {
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (g_default) {
        tsqs_ctx_destroy(g_default);
        g_default = nullptr;
    }
}

int tsqs_last_device_status(void *stream) {
    tsqs_ctx *c = default_ctx();
    if (!c) return TSQS_ENOMEM;
    return read_status(c, (cudaStream_t)stream, true);
}

int tsqs_sort_wide(void *base, size_t nmemb, size_t elem_size, size_t key_offset, int key_kind,
                   void *stream) {
    if (key_kind < TSQS_I32 || key_kind > TSQS_F64) return TSQS_EINVAL;
    const size_t ks = kind_size(key_kind);
    if (elem_size == 0 || elem_size % 4 || elem_size % ks || key_offset % ks ||
        key_offset + ks > elem_size)
        return TSQS_EINVAL;
    if (nmemb > 1 && (!base || (uintptr_t)base % ks || (uintptr_t)base % 4)) return TSQS_EINVAL;
    if (nmemb >= (1ull << 31)) return TSQS_EINVAL;
    if (nmemb <= 1) return TSQS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    tsqs_ctx *c = default_ctx();
    if (!c) return TSQS_ENOMEM;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int rc = ctx_init_device(c);
    if (rc) return rc;
    const size_t rec_bytes = nmemb * 16, tmp_bytes = nmemb * elem_size;
    if (rec_bytes > c->wide_rec_bytes || tmp_bytes > c->wide_tmp_bytes) {
        ctx_quiesce(c);
        CK(cudaStreamSynchronize(s));
        if (rec_bytes > c->wide_rec_bytes) {
            if (c->wide_rec) cudaFree(c->wide_rec);
            c->wide_rec = nullptr;
            c->wide_rec_bytes = 0;
            if (cudaMalloc((void **)&c->wide_rec, rec_bytes) != cudaSuccess) { cudaGetLastError(); return TSQS_ENOMEM; }
            c->wide_rec_bytes = rec_bytes;
        }
        if (tmp_bytes > c->wide_tmp_bytes) {
            if (c->wide_tmp) cudaFree(c->wide_tmp);
            c->wide_tmp = nullptr;
            c->wide_tmp_bytes = 0;
            if (cudaMalloc((void **)&c->wide_tmp, tmp_bytes) != cudaSuccess) { cudaGetLastError(); return TSQS_ENOMEM; }
            c->wide_tmp_bytes = tmp_bytes;
        }
    }
    if (c->ev_valid) CK(cudaStreamWaitEvent(s, c->done_ev, 0));
    if ((rc = wide_keys(key_kind, base, nmemb, elem_size, key_offset, c->wide_rec, c->sms, s))) return rc;
    if ((rc = ctx_launch(c, c->wide_rec, nmemb, nullptr, 0, 16, TSQS_U64_U64_REC, s))) return rc;
    if ((rc = wide_gather(base, nmemb, elem_size, c->wide_rec, c->wide_tmp, c->sms, s))) return rc;
    CK(cudaMemcpyAsync(base, c->wide_tmp, tmp_bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(c->done_ev, s));
    c->ev_valid = true;
    return TSQS_OK;
}

void tsqs_debug_set_spin_limit(uint32_t polls) { g_debug_spin = polls; }
void tsqs_debug_set_deep_level(uint32_t level) { g_debug_deep = level; }
void tsqs_debug_set_leaf_defer(uint32_t items) { g_debug_defer = items; }
void tsqs_debug_withhold_publish(int on) { g_debug_withhold = on == 2 ? 2 : on ? 1 : 0; }

// ---------------------------------------------------------------------------------
// host-memory sort: device staging buffer owned by the default context's side store
// ---------------------------------------------------------------------------------

static std::mutex g_host_mu;
static void *g_host_dev = nullptr;
static size_t g_host_dev_bytes = 0;

int tsqs_sort_host(void *h_base, size_t nmemb, size_t elem_size, int key_kind, void *stream) {
    int rc = validate(h_base, nmemb, elem_size, key_kind);
    if (rc) return rc;
    if (nmemb <= 1) return TSQS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_host_mu);
    const size_t bytes = nmemb * elem_size;
    // device copy of the input, allocated with 16 bytes of slack so that it can take the
    // host array's 16-byte phase (the vector stores of the output then line up on both)
    if (bytes + 16 > g_host_dev_bytes) {
        if (g_host_dev) { CK(cudaStreamSynchronize(s)); cudaFree(g_host_dev); g_host_dev = nullptr; g_host_dev_bytes = 0; }
        if (cudaMalloc(&g_host_dev, bytes + 16) != cudaSuccess) { cudaGetLastError(); return TSQS_ENOMEM; }
        g_host_dev_bytes = bytes + 16;
    }
    char *dev = (char *)g_host_dev + ((uintptr_t)h_base & 15u);
    // a pinned (page-locked, device-mapped) host array receives the result straight from
    // the kernels over the host link, so the final leaf pass overlaps the transfer back;
    // any other host array gets a copy after the sort
    void *h_mapped = nullptr;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, h_base) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer && (((uintptr_t)pa.devicePointer ^ (uintptr_t)h_base) & 15u) == 0)
        h_mapped = pa.devicePointer;
    cudaGetLastError();
    CK(cudaMemcpyAsync(dev, h_base, bytes, cudaMemcpyHostToDevice, s));
    if (h_mapped) {
        tsqs_ctx *c = default_ctx();
        if (!c) return TSQS_ENOMEM;
        rc = ctx_launch(c, dev, nmemb, nullptr, 0, elem_size, key_kind, s, h_mapped);
        if (rc) return rc;
    } else {
        rc = tsqs_sort(dev, nmemb, elem_size, key_kind, stream);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h_base, dev, bytes, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return TSQS_OK;
}

// ---------------------------------------------------------------------------------
// Host arrays streamed through three device staging slots: item i's upload runs on
// s_in, its sort on the caller's stream, its download on s_out.  Slot i % 3 is reused
// by item i + 3 once item i's download has finished (ev_out), so the upload of item
// i + 1 and the download of item i - 1 overlap the sort of item i.
// ---------------------------------------------------------------------------------

int tsqs_ctx_sort_host_stream(tsqs_ctx *c, const void *const *h_in, void *const *h_out,
                              const size_t *nmemb, size_t count, size_t elem_size,
                              int key_kind, void *stream, int *h_status) {
    if (!c) return TSQS_EINVAL;
    const size_t es = kind_size(key_kind);
    if (!es || es != elem_size) return TSQS_EINVAL;
    if (count == 0) return TSQS_OK;
    if (!h_in || !nmemb) return TSQS_EINVAL;
    size_t max_n = 0;
    for (size_t i = 0; i < count; i++) {
        if (nmemb[i] >= (1ull << 31)) return TSQS_EINVAL;
        const void *out = h_out ? h_out[i] : h_in[i];
        if (nmemb[i] > 0 && (!h_in[i] || !out)) return TSQS_EINVAL;
        max_n = std::max(max_n, nmemb[i]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const KindOps *o = get_ops(key_kind);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int rc = ctx_init_device(c);
    if (rc) return rc;
    if ((rc = ctx_kind_setup(c, o))) return rc;
    // everything that can fail to allocate is allocated before anything is queued
    const size_t slot_bytes = std::max<size_t>(max_n * es, 16);
    if ((rc = ctx_stream_setup(c, slot_bytes, count))) return rc;
    if (max_n > 1) {
        if ((rc = ctx_ensure_scratch(c, o, max_n, 1))) return rc;
        if ((rc = ctx_build_graph(c, o))) return rc;
    }
    int first = TSQS_OK;
    CK(cudaEventRecord(c->ev_entry, s));
    CK(cudaStreamWaitEvent(c->s_in, c->ev_entry, 0));
    CK(cudaStreamWaitEvent(c->s_out, c->ev_entry, 0));
    for (size_t i = 0; i < count && first == TSQS_OK; i++) {
        const int k = (int)(i % 3);
        const size_t n = nmemb[i], bytes = n * es;
        void *out = h_out ? h_out[i] : const_cast<void *>(h_in[i]);
        if (i >= 3 && cudaStreamWaitEvent(c->s_in, c->ev_out[k], 0) != cudaSuccess) { first = TSQS_ECUDA; break; }
        if (bytes && cudaMemcpyAsync(c->stage[k], h_in[i], bytes, cudaMemcpyHostToDevice, c->s_in) != cudaSuccess) { first = TSQS_ECUDA; break; }
        if (cudaEventRecord(c->ev_in[k], c->s_in) != cudaSuccess ||
            cudaStreamWaitEvent(s, c->ev_in[k], 0) != cudaSuccess) { first = TSQS_ECUDA; break; }
        if (n > 1 && (first = ctx_launch(c, c->stage[k], n, nullptr, 0, es, key_kind, s)) != TSQS_OK) break;
        k_keep_status<<<1, 32, 0, s>>>(c->d_ctl, c->d_item_status + i, n > 1 ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess ||
            cudaEventRecord(c->ev_sorted[k], s) != cudaSuccess ||
            cudaStreamWaitEvent(c->s_out, c->ev_sorted[k], 0) != cudaSuccess) { first = TSQS_ECUDA; break; }
        if (bytes && cudaMemcpyAsync(out, c->stage[k], bytes, cudaMemcpyDeviceToHost, c->s_out) != cudaSuccess) { first = TSQS_ECUDA; break; }
        if (cudaEventRecord(c->ev_out[k], c->s_out) != cudaSuccess) { first = TSQS_ECUDA; break; }
    }
    // drain all three streams whatever happened, so the slots are idle for the next call
    const cudaError_t e_in = cudaStreamSynchronize(c->s_in);
    const cudaError_t e_s = cudaStreamSynchronize(s);
    const cudaError_t e_out = cudaStreamSynchronize(c->s_out);
    if (first != TSQS_OK) return first;
    if (e_in != cudaSuccess || e_s != cudaSuccess || e_out != cudaSuccess) return TSQS_ECUDA;
    uint32_t *st = (uint32_t *)malloc(count * sizeof(uint32_t));
    if (!st) return TSQS_ENOMEM;
    if (cudaMemcpy(st, c->d_item_status, count * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        free(st);
        return TSQS_ECUDA;
    }
    for (size_t i = 0; i < count; i++) {
        if (h_status) h_status[i] = (int)st[i];
        if (first == TSQS_OK && st[i]) first = (int)st[i];
    }
    free(st);
    return first;
}

// ---------------------------------------------------------------------------------
// Instrumented host-driven run (same kernels as the graph, one launch each).
// ---------------------------------------------------------------------------------

int tsqs_ctx_sort_timed(tsqs_ctx *c, void *base, size_t nmemb, size_t elem_size,
                        int key_kind, void *stream, float *h_ms, uint64_t *h_keys,
                        int max_levels, int *levels, float *h_leaf_ms) {
    if (!c) return TSQS_EINVAL;
    int rc = validate(base, nmemb, elem_size, key_kind);
    if (rc) return rc;
    if (levels) *levels = 0;
    if (nmemb <= 1) return TSQS_OK;
    if (nmemb >= (1ull << 31)) return TSQS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const KindOps *o = get_ops(key_kind);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if ((rc = ctx_init_device(c))) return rc;
    if ((rc = ctx_kind_setup(c, o))) return rc;
    if ((rc = ctx_ensure_scratch(c, o, nmemb, 1))) return rc;
    Job j;
    if ((rc = make_job(c, o, base, nmemb, nullptr, 0, &j))) return rc;
    if (c->ev_valid) CK(cudaStreamWaitEvent(s, c->done_ev, 0));
    const int k = key_kind;
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    cudaGraphConditionalHandle h = 0;
    int use_h = 0;
    unsigned int unused = 0;
    void *argsf[] = {&pj, &pc, &h, &use_h, &unused};
    int leaf_final = 0, leaf_last = 1;
    void *argsl[] = {&pj, &pc, &leaf_final};
    void *argsl_last[] = {&pj, &pc, &leaf_last};
    const bool task = task_schedule(c->plan, nmemb);
    if (task) {
        if ((rc = make_job(c, o, base, nmemb, nullptr, 0, &j, true))) return rc;
    }
    cudaEvent_t ev[4];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    k_setup<<<1, 256, 0, s>>>(c->d_job, c->d_ctl, j);
    CK(cudaLaunchKernel(o->k_orient, dim3(c->sms * 4), dim3(256), args2, 0, s));
    CK(cudaLaunchKernel(o->k_check, dim3(c->sms * 4), dim3(256), args2, 0, s));
    CK(cudaLaunchKernel(o->k_presort, dim3(c->sms * 4), dim3(256), args2, 0, s));
    if (task) {
        // task schedule: init, the task kernel, the leaf pass, the depth guard if needed
        CK(cudaLaunchKernel(o->k_task_init, dim3(c->sms * 2), dim3(256), args2, 0, s));
        CK(cudaEventRecord(ev[0], s));
        CK(cudaLaunchKernel(o->k_task, dim3(c->task_grid[k]), dim3(o->task_block), args2, 0, s));
        CK(cudaEventRecord(ev[1], s));
        if (nmemb <= kSmallLeafN)
            CK(cudaLaunchKernel(o->k_leaf_small, dim3(c->leaf_small_grid[k]), dim3(o->leaf_small_block),
                                argsl_last, (size_t)o->leaf_small_smem, s));
        else
            CK(cudaLaunchKernel(o->k_leaf, dim3(c->leaf_grid[k]), dim3(o->leaf_block), argsl_last,
                                (size_t)o->leaf_smem, s));
        CK(cudaEventRecord(ev[2], s));
        Ctl hc;
        CK(cudaMemcpyAsync(&hc, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float ms = 0.f, lms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        CK(cudaEventElapsedTime(&lms, ev[1], ev[2]));
        if (hc.status == 0u && hc.ndeep != 0u) CK(run_deep_host(c, o, s, c->d_job, c->d_ctl));
        for (auto &e : ev) cudaEventDestroy(e);
        if (max_levels >= 1) {
            if (h_ms) h_ms[0] = ms;
            if (h_leaf_ms) h_leaf_ms[0] = lms;
            if (h_keys) h_keys[0] = hc.partition_keys;
        }
        if (levels) *levels = 1;
        CK(cudaEventRecord(c->done_ev, s));
        c->ev_valid = true;
        return TSQS_OK;
    }
    CK(cudaLaunchKernel(o->k_init, dim3(c->sms * 2), dim3(256), args2, 0, s));
    int L = 0;
    for (;;) {
        CK(cudaEventRecord(ev[2], s));
        CK(cudaLaunchKernel(o->k_leaf, dim3(c->leaf_grid[k]), dim3(o->leaf_block), argsl,
                            (size_t)o->leaf_smem, s));
        CK(cudaEventRecord(ev[3], s));
        CK(cudaLaunchKernel(o->k_pivot, dim3(c->sms * 4), dim3(o->pivot_block), args2, 0, s));
        CK(cudaEventRecord(ev[0], s));
        const PartVariant &pv = part_of(o, c->plan);
        CK(cudaLaunchKernel(pv.k_partition, dim3(c->part_grid[k]), dim3(pv.threads), args2,
                            (size_t)pv.smem, s));
        CK(cudaEventRecord(ev[1], s));
        CK(cudaLaunchKernel(o->k_finish, dim3(c->sms), dim3(128), argsf, 0, s));
        CK(cudaMemcpyAsync(c->h_cont, &c->d_ctl->more, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (L < max_levels) {
            float ms = 0.f, lms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            CK(cudaEventElapsedTime(&lms, ev[2], ev[3]));
            if (h_ms) h_ms[L] = ms;
            if (h_leaf_ms) h_leaf_ms[L] = lms;
        }
        L++;
        if (!*c->h_cont) break;
        if (L > 100000) break;
    }
    // final leaf pass; its time is added to the last level's leaf entry
    CK(cudaEventRecord(ev[2], s));
    CK(cudaLaunchKernel(o->k_leaf, dim3(c->leaf_grid[k]), dim3(o->leaf_block), argsl_last,
                        (size_t)o->leaf_smem, s));
    CK(cudaEventRecord(ev[3], s));
    CK(cudaStreamSynchronize(s));
    if (L >= 1 && L - 1 < max_levels && h_leaf_ms) {
        float lms = 0.f;
        CK(cudaEventElapsedTime(&lms, ev[2], ev[3]));
        h_leaf_ms[L - 1] += lms;
    }
    CK(run_deep_host(c, o, s, c->d_job, c->d_ctl));
    for (auto &e : ev) cudaEventDestroy(e);
    if (h_keys) {
        Ctl hc;
        CK(cudaMemcpy(&hc, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        for (int i = 0; i < std::min(L, max_levels); i++)
            h_keys[i] = i < kStatLevels ? hc.level_keys[i] : 0;
    }
    if (levels) *levels = L;
    CK(cudaEventRecord(c->done_ev, s));
    c->ev_valid = true;
    return TSQS_OK;
}

// ---------------------------------------------------------------------------------
// Step-level entry points
// ---------------------------------------------------------------------------------

int tsqs_debug_pivot(const void *base, size_t nmemb, size_t elem_size, int key_kind,
                     uint64_t seg_begin, uint64_t seg_end, int sample_count, uint64_t seed,
                     uint64_t *h_positions, void *h_pivot, void *stream) {
    int rc = validate((void *)base, nmemb, elem_size, key_kind);
    if (rc) return rc;
    if (seg_end <= seg_begin || seg_end > nmemb || !h_positions || !h_pivot) return TSQS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    tsqs_ctx *c = default_ctx();
    const KindOps *o = get_ops(key_kind);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if ((rc = ctx_init_device(c))) return rc;
    if ((rc = ctx_ensure_scratch(c, o, nmemb, 1))) return rc;
    Job j;
    if ((rc = make_job(c, o, (void *)base, nmemb, nullptr, 0, &j))) return rc;
    const Layout L = make_layout(nmemb, 1, elem_size, c->plan, part_of(o, c->plan).tile, o->leaf_max);
    char *misc = c->scratch + L.misc_off;
    uint64_t *d_offs = (uint64_t *)misc;
    uint64_t *d_pos = (uint64_t *)(misc + 64);
    void *d_piv = misc + 1024;                       // 16-byte aligned (records)
    const uint64_t offs[2] = {seg_begin, seg_end};
    if (c->ev_valid) CK(cudaStreamWaitEvent(s, c->done_ev, 0));
    CK(cudaMemcpyAsync(d_offs, offs, sizeof(offs), cudaMemcpyHostToDevice, s));
    j.seg_offsets = d_offs;
    j.nseg = 1;
    j.samples = (uint32_t)(sample_count > 0 ? sample_count : c->plan.sample_count);
    j.seed = seed;
    j.dbg_positions = d_pos;
    j.dbg_pivot_out = d_piv;
    CK(cudaMemsetAsync(d_pos, 0xFF, 8 * kMaxSamples, s));
    k_setup<<<1, 256, 0, s>>>(c->d_job, c->d_ctl, j);
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    CK(cudaLaunchKernel(o->k_dbg_pivot, dim3(1), dim3(32), args2, 0, s));
    uint64_t pos[kMaxSamples];
    CK(cudaMemcpyAsync(pos, d_pos, sizeof(pos), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h_pivot, d_piv, elem_size, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the kernel draws min(sample_count, segment length) samples, made odd; the caller's
    // array holds sample_count entries, and unused ones read as all ones
    const uint32_t S = j.samples > (uint32_t)kMaxSamples ? (uint32_t)kMaxSamples : j.samples;
    for (uint32_t i = 0; i < S; i++) h_positions[i] = pos[i];
    CK(cudaEventRecord(c->done_ev, s));
    c->ev_valid = true;
    return TSQS_OK;
}

int tsqs_debug_partition(const void *src, void *dst, size_t nmemb, size_t elem_size,
                         int key_kind, const uint64_t *d_seg_offsets, size_t nseg,
                         const void *d_pivots, uint64_t *d_counts, void *stream) {
    int rc = validate((void *)src, nmemb, elem_size, key_kind);
    if (rc) return rc;
    if (!dst || !d_seg_offsets || !d_pivots || !d_counts || nseg == 0) return TSQS_EINVAL;
    if (((uintptr_t)src & 15u) != ((uintptr_t)dst & 15u)) return TSQS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    tsqs_ctx *c = default_ctx();
    const KindOps *o = get_ops(key_kind);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if ((rc = ctx_init_device(c))) return rc;
    if ((rc = ctx_kind_setup(c, o))) return rc;
    if ((rc = ctx_ensure_scratch(c, o, nmemb, nseg))) return rc;
    Job j;
    if ((rc = make_job(c, o, (void *)src, nmemb, d_seg_offsets, nseg, &j))) return rc;
    j.alt = dst;
    j.dbg_pivots = d_pivots;
    j.dbg_counts = d_counts;
    if (c->ev_valid) CK(cudaStreamWaitEvent(s, c->done_ev, 0));
    k_setup<<<1, 256, 0, s>>>(c->d_job, c->d_ctl, j);
    Job *pj = c->d_job;
    Ctl *pc = c->d_ctl;
    void *args2[] = {&pj, &pc};
    const unsigned gs = (unsigned)std::min<size_t>(nseg, (size_t)c->sms * 8);
    CK(cudaLaunchKernel(o->k_dbg_setup_partition, dim3(gs), dim3(256), args2, 0, s));
    const PartVariant &pv = part_of(o, c->plan);
    CK(cudaLaunchKernel(pv.k_partition, dim3(c->part_grid[key_kind]), dim3(pv.threads), args2,
                        (size_t)pv.smem, s));
    CK(cudaLaunchKernel(o->k_dbg_counts, dim3(c->sms), dim3(256), args2, 0, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaEventRecord(c->done_ev, s));
    c->ev_valid = true;
    return TSQS_OK;
}

int tsqs_debug_small_sort(void *base, size_t nmemb, size_t elem_size, int key_kind,
                          const uint64_t *d_seg_offsets, size_t nseg, void *stream) {
    tsqs_ctx *c = default_ctx();
    int rc = tsqs_ctx_sort_segmented(c, base, nmemb, d_seg_offsets, nseg, elem_size, key_kind, stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return TSQS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Helpers for sorts whose scratch is not owned by a context (used by the
// allocation-free entry point in tsqs_noalloc.cu).
// ---------------------------------------------------------------------------------
namespace tsqs {

const KindOps *host_ops(int key_kind) { return get_ops(key_kind); }

// Default plan, normalised, for key_kind.
void host_default_plan(int key_kind, tsqs_plan *p) {
    fill_default_plan(key_kind, 0, p);
    normalise_plan(p);
}

// Scratch bytes a single-segment sort of n elements needs under plan p.
size_t host_scratch_bytes(const KindOps *o, const tsqs_plan &p, size_t n) {
    return make_layout(n, 1, (size_t)o->elem_size, p, part_of(o, p).tile, o->leaf_max).total;
}

// Partition kernel shape the plan selects.
const PartVariant &host_part(const KindOps *o, const tsqs_plan &p) { return part_of(o, p); }

// Describes a single-segment sort of base[0, n) whose scratch is the caller-provided
// block [scratch, scratch + bytes).  TSQS_ENOMEM if the block is too small.
int host_make_job_at(const KindOps *o, const tsqs_plan &plan, void *base, size_t n, char *scratch,
                     size_t bytes, Job *j) {
    const size_t es = (size_t)o->elem_size;
    const Layout L = make_layout(n, 1, es, plan, part_of(o, plan).tile, o->leaf_max);
    if (L.total > bytes) return TSQS_ENOMEM;
    memset(j, 0, sizeof(*j));
    const uintptr_t b = (uintptr_t)base;
    j->base = base;
    j->out = base;
    j->alt = scratch + L.alt_off + (b & 15u);
    j->n = n;
    j->seg_offsets = nullptr;
    j->nseg = 1;
    j->front[0] = (SegDesc *)(scratch + L.front_off[0]);
    j->front[1] = (SegDesc *)(scratch + L.front_off[1]);
    j->leaves = (LeafItem *)(scratch + L.leaves_off);
    j->tile_seg = (uint32_t *)(scratch + L.tseg_off);
    j->tile_status = (unsigned long long *)(scratch + L.tstat_off);
    j->seg_done = (uint32_t *)(scratch + L.done_off);
    j->seg_cursor = (unsigned long long *)(scratch + L.cursor_off);
    j->presort = (uint32_t *)(scratch + L.presort_off);
    j->deep = (LeafItem *)(scratch + L.deep_off);
    j->deep_tiles = (uint32_t *)(scratch + L.dtiles_off);
    j->deep_chunks = (uint32_t *)(scratch + L.dchunks_off);
    j->cap_deep = L.cap_front;
    j->cap_front = L.cap_front;
    j->cap_tiles = L.cap_tiles;
    j->cap_leaves = L.cap_leaves;
    j->leaf_defer = g_debug_defer ? std::min(g_debug_defer, L.leaf_defer) : L.leaf_defer;
    j->small_T = (uint32_t)eff_threshold(plan, o->leaf_max);
    j->samples = (uint32_t)plan.sample_count;
    j->vec_off = (uint32_t)((b / es) % (16 / es));
    j->spin_limit = kDefaultSpin;
    j->pad = 0u;
    unsigned lg = 1;
    while ((1ull << lg) < (unsigned long long)n + 1 && lg < 63) lg++;
    j->max_levels = 256u + 8u * lg;
    j->deep_level = g_debug_deep ? g_debug_deep : 2u * lg + 8u;
    j->offset_mode = plan.offset_mode == 1 ? 1u : 0u;
    j->tile = (uint32_t)part_of(o, plan).tile;
    j->seed = plan.seed;
    return TSQS_OK;
}

}  // namespace tsqs
