// tsqs_task.cuh -- the task-parallel schedule of the three-way partition sort (sm_103a).
//
// Below a size bound the level-synchronous loop is latency-bound: every level waits for
// its slowest segment and pays three dependent launches (pivot, partition, level end)
// whose work is a handful of tiles.  Here the recursion of Section III.F runs without
// level barriers, in one persistent launch:
//   - tile ids run over the whole sort and are claimed in one global order; a segment
//     gets a range of ids when it is pushed, and each id's row (the tile's first element,
//     the buffer holding its keys and the segment index; the rows are zeroed by the
//     first kernel of the call) is written once the segment's descriptor and sampled
//     median (Section III.H, V.C) are in memory;
//   - a block that claimed an id whose row is not written yet polls it (bounded); the
//     row alone lets it start loading the tile while the descriptor is read;
//   - a tile is classified against p once, its <p and >p elements are packed at the two
//     ends of the segment through one 64-bit atomic on the segment's cursor (the roles of
//     the paper's l and r), and the =p elements are never written or compared again;
//   - the block that finishes a segment's last tile reads the final (#<p, #>p), writes
//     the =p run (or queues fill items for a long one) and pushes both children: to the
//     leaf queue (<= small_T, Section IV's role), to the depth guard's queue, or as new
//     segments partitioned as soon as their blocks pick them up;
//   - a count of live segments falling to zero ends the launch: the block that sees it
//     writes end-of-work rows for every block still polling (a launch that starts with
//     none ends at once).
// Keys of depth d are in buffer d % 2, as level d's are in the level-synchronous loop,
// and every step hands on work of the same form (leaf items, fills, deep items), so the
// leaf pass and the depth guard serve both schedules.
#pragma once
#include "tsqs_kernels.cuh"

namespace tsqs {

constexpr uint32_t kTaskInlineFill = 1u << 16;   // =p runs up to this long are written by the
                                                 // block that finishes their segment

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Tile row: [63:32] first element of the tile + kRowBias (tile origins start at most
// 15 elements below 0, so a written row is never 0), [31] buffer of the keys, [30:0]
// segment index.  kTaskEndRow: no more work.
constexpr int64_t kRowBias = 16;
constexpr unsigned long long kTaskEndRow = ~0ull;
__device__ __forceinline__ unsigned long long task_row(int64_t t0, uint32_t par, uint32_t si) {
    return ((unsigned long long)(uint32_t)(t0 + kRowBias) << 32) | ((unsigned long long)par << 31) | si;
}

// Descriptor of segment si from L2 (it may have been written in this launch after this
// block cached a neighbouring one).
__device__ __forceinline__ TaskSeg load_task_seg(const TaskSeg *p) {
    const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(p);
    const ulonglong2 w0 = __ldcg(q), w1 = __ldcg(q + 1), w2 = __ldcg(q + 2), w3 = __ldcg(q + 3);
    TaskSeg t;
    t.begin = w0.x;
    t.end = w0.y;
    t.s0 = (int64_t)w1.x;
    t.piv_lo = w1.y;
    t.piv_hi = w2.x;
    t.tile_begin = (uint32_t)w2.y;
    t.ntiles_depth = (uint32_t)(w2.y >> 32);
    t.done = w3.x;
    t.cursor = w3.y;
    return t;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// Finished-tile word: the tile count above bit 42 (2^22 tiles cover a segment of 2^31
// records in tiles of 1024); below 2^21 elements a segment's tiles also add their
// (#<p, #>p) in two 21-bit fields, so the last one reads the totals from its own atomic.
constexpr int kDoneTiles = 42, kDoneCount = 21;
constexpr uint64_t kDoneSmall = 1ull << kDoneCount;
constexpr unsigned long long kDoneMask = (1ull << kDoneCount) - 1ull;

// 16-byte L2 load of V storage elements (address 16-byte aligned).
template <class S, int V>
__device__ __forceinline__ void ldcg_vec(const S *p, S *out) {
    union { uint4 q; S s[V]; } u;
    u.q = __ldcg(reinterpret_cast<const uint4 *>(p));
#pragma unroll
    for (int j = 0; j < V; j++) out[j] = u.s[j];
}

// Threads t (of nt) write val to out[b, e): scalar up to the first 16-byte boundary,
// 16-byte stores for the body, scalar tail.
template <class S, int V>
__device__ __forceinline__ void fill_span(S *out, uint64_t b, uint64_t e, S val, uint32_t vec_off,
                                          uint32_t t, uint32_t nt) {
    if (e <= b) return;
    const uint64_t cnt = e - b;
    uint64_t head = (V - ((b + vec_off) % V)) % V;
    if (head > cnt) head = cnt;
    const uint64_t nvec = (cnt - head) / V;
    if (t < head) out[b + t] = val;
    S w[V];
#pragma unroll
    for (int j = 0; j < V; j++) w[j] = val;
    for (uint64_t q = t; q < nvec; q += nt) stg_vec<S, V>(out + b + head + q * V, w);
    const uint64_t body_end = head + nvec * V;
    if (t < cnt - body_end) out[b + body_end + t] = val;
}

// One warp: pushes [b, e) (keys in buffer d % 2) as a task segment of depth d: samples
// its median, takes a descriptor and a range of tile ids, writes the descriptor, then
// the tile rows.  Returns false (status set) when a table is full.  `withhold`: the
// rows of segment 0 are not written (test of the bounded wait).
template <class K>
__device__ bool push_task(const Job *job, Ctl *ctl, uint64_t b, uint64_t e, uint32_t d,
                          bool withhold) {
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t s0 = tile_origin<K::V>(b, job->vec_off);
    const int TILE = (int)job->tile;
    const uint32_t nt = tiles_for(e, s0, TILE);
    // the table slots first: their round trip overlaps the sample loads
    uint32_t fi = 0, tb = 0, ok = 0;
    if (lane == 0) {
        fi = atomicAdd(&ctl->tsegs, 1u);
        tb = atomicAdd(&ctl->talloc, nt);
    }
    const typename K::C p = sample_pivot<K, true>(buffer<K>(job, (int)(d & 1u)), b, e,
                                                  job->samples, job->seed, nullptr);
    if (lane == 0) {
        ok = (fi < job->cap_tseg && fi < 0x80000000u && nt < (1u << 22) && d < 256u &&
              (uint64_t)tb + nt + kTaskGridMax <= job->cap_trow) ? 1u : 0u;
        if (ok) {
            TaskSeg ts;
            ts.begin = b;
            ts.end = e;
            ts.s0 = s0;
            c_words(p, ts.piv_lo, ts.piv_hi);
            ts.tile_begin = tb;
            ts.ntiles_depth = nt | (d << 24);
            ts.done = 0ull;
            ts.cursor = 0ull;
            job->tseg[fi] = ts;
        } else {
            set_status(ctl, TSQS_EINTERNAL);
        }
    }
    fi = __shfl_sync(0xffffffffu, fi, 0);
    tb = __shfl_sync(0xffffffffu, tb, 0);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    // descriptor before rows: lane 0's stores, the warp barrier, then every lane's fence
    // ahead of its row stores (a release that covers lane 0's stores)
    __syncwarp();
    __threadfence();
    if (!(withhold && fi == 0u))
        for (uint32_t k = lane; k < nt; k += 32u)
            st_relaxed(job->trow + tb + k, task_row(s0 + (int64_t)k * TILE, d & 1u, fi));
    if (lane == 0) {                   // statistics, after the rows are out
        const unsigned long long m = e - b;
        if (d < (uint32_t)kStatLevels) atomicAdd((unsigned long long *)&ctl->level_keys[d], m);
        atomicAdd((unsigned long long *)&ctl->partition_keys, m);
        atomicMax(&ctl->levels_done, d + 1u);
    }
    return true;
}

// One thread: queues [b, e) (keys in buffer par) for the leaf pass.
__device__ __forceinline__ void push_leaf(const Job *job, Ctl *ctl, uint64_t b, uint64_t e, int par) {
    const uint32_t li = atomicAdd(&ctl->nleaf, 1u);
    if (li >= job->cap_leaves) { set_status(ctl, TSQS_EINTERNAL); return; }
    LeafItem it;
    it.begin = b;
    it.len = (uint32_t)(e - b);
    it.kind = LEAF_SORT | (par ? kLeafInAlt : 0u);
    it.v_lo = 0;
    it.v_hi = 0;
    job->leaves[li] = it;
}

// Seeds the task schedule: one warp per root segment (grid-stride).  Roots above the
// on-chip threshold become task segments of depth 0, smaller ones leaf items.
template <int KIND>
__global__ void k_task_init(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const bool withhold = (job->pad & 4u) != 0u;
    uint32_t pushed = 0;
    for (uint64_t s = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += warps) {
        uint64_t b, e;
        root_bounds(job, s, b, e);
        if (e < b || e > job->n || e - b >= (1ull << 31)) {
            if (lane == 0) set_status(ctl, TSQS_EINVAL);
            continue;
        }
        if (e - b <= 1) continue;
        if (job->presort[s] != 0u) continue;             // already in order (presortedness pass)
        if (e - b > job->small_T) {
            if (push_task<K>(job, ctl, b, e, 0u, withhold)) pushed++;
        } else if (lane == 0) {
            push_leaf(job, ctl, b, e, 0);
        }
    }
    if (lane == 0 && pushed) atomicAdd(&ctl->live, pushed);
}

// The task kernel (persistent; BLOCK threads, tiles of BLOCK x ITEMS keys).  Segments
// handed to the depth guard wait in its queue for the cooperative kernel that follows.
template <int KIND, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_task(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    using S = typename K::S;
    using C = typename K::C;
    constexpr int TILE = BLOCK * ITEMS, V = K::V, NV = ITEMS / V, NW = BLOCK / 32;
    static_assert(ITEMS % V == 0 && ITEMS <= 32 && TILE < 65536 && NW >= 4, "tile shape");
    __shared__ __align__(16) S buf[TILE + V];      // staged runs + one dummy 16-byte slot
    __shared__ uint32_t wsum[NW];
    __shared__ TaskSeg s_seg;
    __shared__ unsigned long long s_row;
    __shared__ uint32_t s_cmd, s_last, s_push[2], s_end, s_ta;
    __shared__ unsigned long long s_resv;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = (int64_t)job->n;
    const uint32_t vec_off = job->vec_off;
    // element range of the buffers that 16-byte loads may touch
    const int64_t e_lo = (int64_t)((V - (int64_t)vec_off % V) % V);
    const int64_t e_hi = n - ((n + (int64_t)vec_off) % V);
    const uint64_t T = job->small_T;
    const uint32_t spin_limit = job->spin_limit;
    // no task segment (every root was small, in order or empty): nothing to wait for
    if (*(volatile const uint32_t *)&ctl->live == 0u) return;
    // blocks past the ones this input can use leave at once (their SMs go to other work)
    const uint32_t active = min(gridDim.x, job->task_grid);
    if (blockIdx.x >= active) return;

    for (;;) {
        // ---- claim the next tile id and wait for its row
        TaskSeg seg;
        if (tid == 0) {
            uint32_t cmd = 1u;
            const uint32_t t = atomicAdd(&ctl->tclaim, 1u);
            if (t >= job->cap_trow) {
                set_status(ctl, TSQS_EINTERNAL);
            } else {
                uint32_t polls = 0;
                for (;;) {
                    const unsigned long long r = ld_acquire(job->trow + t);
                    if (r != 0ull) {
                        if (r != kTaskEndRow) {
                            s_row = r;
                            seg = load_task_seg(job->tseg + (uint32_t)(r & 0x7FFFFFFFull));
                            cmd = 0u;
                        }
                        break;
                    }
                    if (*(volatile const uint32_t *)&ctl->status != 0u) break;
                    if (++polls >= spin_limit) { set_status(ctl, TSQS_ETIMEOUT); break; }
                    __nanosleep(polls < 256 ? 32 : 128);
                }
            }
            s_cmd = cmd;
        }
        __syncthreads();
        if (s_cmd) break;

        // ---- load the tile from the row alone (the descriptor's read is in flight):
        // thread t holds the 16-byte vectors k * BLOCK + t; every element of the buffer
        // that the tile covers is read, those outside the segment are masked below
        const unsigned long long row = s_row;
        const uint32_t si = (uint32_t)(row & 0x7FFFFFFFull);
        const int par = (int)((row >> 31) & 1ull);
        const int64_t t0 = (int64_t)(uint32_t)(row >> 32) - kRowBias;
        const S *__restrict__ src = buffer<K>(job, par);
        S *__restrict__ dst = buffer<K>(job, par ^ 1);
        S v[ITEMS];
        if (t0 >= e_lo && t0 + TILE <= e_hi) {
#pragma unroll
            for (int k = 0; k < NV; k++) ldcg_vec<S, V>(src + t0 + (k * BLOCK + tid) * V, &v[k * V]);
        } else {
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const int64_t vs = t0 + (int64_t)(k * BLOCK + tid) * V;
                if (vs >= e_lo && vs + V <= e_hi) {
                    ldcg_vec<S, V>(src + vs, &v[k * V]);
                } else {
#pragma unroll
                    for (int j = 0; j < V; j++)
                        if (vs + j >= 0 && vs + j < n) v[k * V + j] = ldcg_key(src + vs + j);
                }
            }
        }
        if (tid == 0) s_seg = seg;
        __syncthreads();

        // ---- classify against the segment's pivot, inside the segment's bounds
        const int64_t sb = (int64_t)s_seg.begin, se = (int64_t)s_seg.end;
        const uint32_t depth = s_seg.ntiles_depth >> 24, ntiles = s_seg.ntiles_depth & 0xFFFFFFu;
        // a segment of one tile needs no reservation and no finished-tile count: this
        // block places its runs at the segment's ends and finishes it
        const bool single = ntiles == 1u;
        const C pc = c_from<C>(s_seg.piv_lo, s_seg.piv_hi);
        uint32_t ltm = 0, gtm = 0;
        auto classify = [&](auto dom, auto pd) {
        if (t0 >= sb && t0 + TILE <= se) {
#pragma unroll
            for (int i = 0; i < ITEMS; i++) {
                const auto d = dom(v[i]);
                if (c_lt(d, pd)) ltm |= 1u << i;
                if (c_lt(pd, d)) gtm |= 1u << i;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const int64_t vs = t0 + (int64_t)(k * BLOCK + tid) * V;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const bool in = vs + j >= sb && vs + j < se;
                    const auto d = dom(v[k * V + j]);
                    ltm |= (uint32_t)(in && c_lt(d, pd)) << (k * V + j);
                    gtm |= (uint32_t)(in && c_lt(pd, d)) << (k * V + j);
                }
            }
        }
        };
        if constexpr (kFloatKind<KIND>) {
            // raw words against the pivot's sign (see RawDom): signed compare, or unsigned
            // compare with the masks swapped
            using SI = typename std::make_signed<S>::type;
            const S praw = K::uncanon(pc);
            if ((SI)praw >= 0) {
                classify(RawDom<SI>{}, (SI)praw);
            } else {
                classify(RawDom<S>{}, praw);
                const uint32_t t = ltm;
                ltm = gtm;
                gtm = t;
            }
        } else {
            classify(CanonDom<K>{}, K::pdom(pc));
        }

        // ---- block offsets, reservation on the segment's cursor, staging
        const uint32_t cnt = (uint32_t)__popc(ltm) | ((uint32_t)__popc(gtm) << 16);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        const uint32_t ws = lane < NW ? wsum[lane] : 0u;
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, wi, NW - 1);
        const uint32_t wex = __shfl_sync(0xffffffffu, wi - ws, warp);
        const uint32_t texcl = wex + inc - cnt;
        const uint32_t tlt = total & 0xFFFFu, tgt = total >> 16;
        if (tid == 0 && !single)
            s_resv = atomicAdd(&job->tseg[si].cursor, ((unsigned long long)tgt << 32) | tlt);
        {
            const uint32_t b0 = smem_addr(buf), es = (uint32_t)sizeof(S);
            uint32_t la = b0 + (texcl & 0xFFFFu) * es;
            uint32_t ga = b0 + ((TILE - 1) - (texcl >> 16)) * es;
            const uint32_t da = b0 + (uint32_t)TILE * es;
#pragma unroll
            for (int k = 0; k < ITEMS; k++) {
                const bool l = (ltm >> k) & 1u, g = (gtm >> k) & 1u;
                sts_raw(l ? la : (g ? ga : da), v[k]);
                la += l ? es : 0u;
                ga -= g ? es : 0u;
            }
        }
        __syncthreads();               // staged; s_resv ready
        // ---- write both runs: <p at sb + ex_lt, >p ending at se - ex_gt
        {
            const unsigned long long resv = single ? 0ull : s_resv;
            const uint64_t ex_lt = resv & 0xFFFFFFFFull, ex_gt = resv >> 32;
            copy_run<S, V, BLOCK>(dst, (uint64_t)sb + ex_lt, buf, tlt, vec_off);
            copy_run<S, V, BLOCK>(dst, (uint64_t)se - ex_gt - tgt, buf + (TILE - tgt), tgt, vec_off);
        }
        __syncthreads();               // every run written (and buf read) by the block
        if (single) {
            if (tid == 0) {
                s_last = 1u;
                s_resv = ((unsigned long long)tgt << 32) | tlt;
                s_push[0] = s_push[1] = 0u;
            }
        } else if (tid == 0) {
            // release this tile's runs with its count; the last count acquires every
            // other tile's runs and reservation
            const bool small = (uint64_t)(se - sb) < kDoneSmall;
            const unsigned long long add = (1ull << kDoneTiles) |
                (small ? (((unsigned long long)tlt << kDoneCount) | tgt) : 0ull);
            const unsigned long long old = atom_add_acq_rel(&job->tseg[si].done, add);
            s_last = (uint32_t)(old >> kDoneTiles) + 1u == ntiles ? 1u : 0u;
            if (s_last) {
                const unsigned long long fin = old + add;
                s_resv = small ? ((((fin >> kDoneCount) & kDoneMask)) | ((fin & kDoneMask) << 32))
                               : ld_relaxed(&job->tseg[si].cursor);
                s_push[0] = s_push[1] = 0u;
            }
        }
        __syncthreads();
        if (!s_last) continue;

        // ---- the segment is done: =p run and children (block-uniform from here)
        const unsigned long long fin = s_resv;
        const uint64_t nlt = fin & 0xFFFFFFFFull, ngt = fin >> 32;
        const uint64_t m = (uint64_t)(se - sb);
        if (nlt + ngt >= m) {
            // p is an element of the segment, so the =p run is never empty; a violation
            // means corrupted state: stop instead of looping forever
            if (tid == 0) set_status(ctl, TSQS_EINTERNAL);
            continue;
        }
        const uint32_t cd = depth + 1u;
        const int cpar = (int)(cd & 1u);
        if (warp < 2) {
            // warp c pushes child c: [sb, sb + #<p) or [se - #>p, se)
            const uint64_t cb = warp == 0 ? (uint64_t)sb : (uint64_t)se - ngt;
            const uint64_t ce = warp == 0 ? (uint64_t)sb + nlt : (uint64_t)se;
            const uint64_t len = ce - cb;
            if (len > T && cd < job->deep_level) {
                if (push_task<K>(job, ctl, cb, ce, cd, false) && lane == 0) s_push[warp] = 1u;
            } else if (len > T) {
                if (lane == 0) {
                    // depth guard: the bitonic sorter takes it after this launch
                    const uint32_t bd = atomicAdd(&ctl->ndeep, 1u);
                    if (bd >= job->cap_deep) {
                        set_status(ctl, TSQS_EINTERNAL);
                    } else {
                        LeafItem it;
                        it.begin = cb;
                        it.len = (uint32_t)len;
                        it.kind = cpar ? kLeafInAlt : 0u;
                        it.v_lo = 0;
                        it.v_hi = 0;
                        job->deep[bd] = it;
                    }
                }
            } else if (len >= 1 && lane == 0) {
                push_leaf(job, ctl, cb, ce, cpar);
            }
        } else {
            // the other warps place the =p run: written here up to kTaskInlineFill
            // elements, else queued as fill items for the leaf pass
            const uint64_t eqb = (uint64_t)sb + nlt, eqe = (uint64_t)se - ngt;
            const uint32_t t = (uint32_t)tid - 64u;
            if (eqe - eqb <= kTaskInlineFill) {
                fill_span<S, V>(reinterpret_cast<S *>(job->out), eqb, eqe, K::uncanon(pc), vec_off,
                                t, (uint32_t)BLOCK - 64u);
                if (t == 0) atomicAdd((unsigned long long *)&ctl->leaf_filled, (unsigned long long)(eqe - eqb));
            } else if (t == 0) {
                const uint32_t nch = (uint32_t)((eqe - eqb + kFillChunk - 1) / kFillChunk);
                const uint32_t bl = atomicAdd(&ctl->nleaf, nch);
                for (uint32_t c = 0; c < nch; c++) {
                    if (bl + c >= job->cap_leaves) { set_status(ctl, TSQS_EINTERNAL); break; }
                    LeafItem li;
                    li.begin = eqb + (uint64_t)c * kFillChunk;
                    const uint64_t rest = eqe - li.begin;
                    li.len = (uint32_t)(rest < kFillChunk ? rest : kFillChunk);
                    li.kind = LEAF_FILL;
                    li.v_lo = s_seg.piv_lo;
                    li.v_hi = s_seg.piv_hi;
                    job->leaves[bl + c] = li;
                }
            }
        }
        __syncthreads();
        // children are published before this segment leaves the live count, so the count
        // reaches zero only when no segment is pushed or in progress
        if (tid == 0) {
            const uint32_t np = s_push[0] + s_push[1];
            const uint32_t old = atomicAdd(&ctl->live, np - 1u);
            s_end = old + np - 1u == 0u ? 1u : 0u;
            if (s_end) {
                __threadfence();
                s_ta = *(volatile const uint32_t *)&ctl->talloc;
            }
        }
        __syncthreads();
        if (s_end) {
            // every taking-part block holds at most one claim past the last tile id
            const uint32_t ta = s_ta;
            for (uint32_t g = (uint32_t)tid; g < active && (uint64_t)ta + g < job->cap_trow; g += BLOCK)
                st_relaxed(job->trow + ta + g, kTaskEndRow);
        }
    }
}

}  // namespace tsqs
