// tsqs_kernels.cuh -- device code of the three-way partition sort (sm_103a).
//
// Kernels of one level of the level loop (see tsqs_internal.h for the queue layout):
//   k_leaf       on-chip pass over the leaf items produced by the previous level:
//                sorts segments of <= small_T elements in shared memory (the role of
//                the insertion sort of Section IV) and fills =p runs (Section III.F)
//   k_pivot      sampled median of every frontier segment (Section III.H, V.C) and
//                the per-level tile tables
//   k_partition  the three-way split of Section III: every element is classified
//                against p once, <p elements are packed from the segment's left end
//                and >p elements from its right end (the roles of the paper's l and r
//                cursors), the =p run in the middle is never written or compared
//                again; offsets come from a decoupled look-back over (#<p, #>p), and
//                the last tile of a segment pushes its children (the recursion on
//                [a, l] and [r, b] of Section III.F) to the next level's queues
//   k_finish     advances the level and decides whether the loop continues
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tsqs_internal.h"
#include "tsqs.h"

namespace tsqs {

// ---------------------------------------------------------------------------------
// Key traits: storage type S, canonical unsigned type C with an order-preserving
// bijection S -> C, so that the whole method compares unsigned integers.
//   signed ints : flip the sign bit
//   floats      : flip all bits of negatives, only the sign bit of non-negatives
//                 (this maps IEEE totalOrder onto unsigned order)
//   records     : (key, payload) compared as one 128-bit unsigned number
// ---------------------------------------------------------------------------------

struct U128 { unsigned long long lo, hi; };
struct __align__(16) Rec16 { unsigned long long key, pay; };

template <int KIND> struct Key;

template <> struct Key<TSQS_I32> {
    using S = unsigned int; using C = unsigned int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) { return x ^ 0x80000000u; }
    static __device__ __forceinline__ S uncanon(C c) { return c ^ 0x80000000u; }
};
template <> struct Key<TSQS_U32> {
    using S = unsigned int; using C = unsigned int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) { return x; }
    static __device__ __forceinline__ S uncanon(C c) { return c; }
};
template <> struct Key<TSQS_F32> {
    using S = unsigned int; using C = unsigned int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) {
        return x ^ ((unsigned int)((int)x >> 31) | 0x80000000u);
    }
    static __device__ __forceinline__ S uncanon(C c) {
        return c ^ (~(unsigned int)((int)c >> 31) | 0x80000000u);
    }
};
template <> struct Key<TSQS_I64> {
    using S = unsigned long long; using C = unsigned long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) { return x ^ 0x8000000000000000ull; }
    static __device__ __forceinline__ S uncanon(C c) { return c ^ 0x8000000000000000ull; }
};
template <> struct Key<TSQS_U64> {
    using S = unsigned long long; using C = unsigned long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) { return x; }
    static __device__ __forceinline__ S uncanon(C c) { return c; }
};
template <> struct Key<TSQS_F64> {
    using S = unsigned long long; using C = unsigned long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) {
        return x ^ ((unsigned long long)((long long)x >> 63) | 0x8000000000000000ull);
    }
    static __device__ __forceinline__ S uncanon(C c) {
        return c ^ (~(unsigned long long)((long long)c >> 63) | 0x8000000000000000ull);
    }
};
template <> struct Key<TSQS_U64_U64_REC> {
    using S = Rec16; using C = U128; static constexpr int V = 1;
    static __device__ __forceinline__ C canon(S x) { return U128{x.pay, x.key}; }
    static __device__ __forceinline__ S uncanon(C c) { Rec16 r; r.key = c.hi; r.pay = c.lo; return r; }
};

// canonical-order helpers, overloaded on C
__device__ __forceinline__ bool c_lt(unsigned int a, unsigned int b) { return a < b; }
__device__ __forceinline__ bool c_lt(unsigned long long a, unsigned long long b) { return a < b; }
__device__ __forceinline__ bool c_lt(U128 a, U128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool c_eq(unsigned int a, unsigned int b) { return a == b; }
__device__ __forceinline__ bool c_eq(unsigned long long a, unsigned long long b) { return a == b; }
__device__ __forceinline__ bool c_eq(U128 a, U128 b) { return a.hi == b.hi && a.lo == b.lo; }

template <class C> __device__ __forceinline__ C c_max();
template <> __device__ __forceinline__ unsigned int c_max<unsigned int>() { return 0xFFFFFFFFu; }
template <> __device__ __forceinline__ unsigned long long c_max<unsigned long long>() { return ~0ull; }
template <> __device__ __forceinline__ U128 c_max<U128>() { return U128{~0ull, ~0ull}; }

__device__ __forceinline__ void c_words(unsigned int c, uint64_t &lo, uint64_t &hi) { lo = c; hi = 0; }
__device__ __forceinline__ void c_words(unsigned long long c, uint64_t &lo, uint64_t &hi) { lo = c; hi = 0; }
__device__ __forceinline__ void c_words(U128 c, uint64_t &lo, uint64_t &hi) { lo = c.lo; hi = c.hi; }
template <class C> __device__ __forceinline__ C c_from(uint64_t lo, uint64_t hi);
template <> __device__ __forceinline__ unsigned int c_from<unsigned int>(uint64_t lo, uint64_t) { return (unsigned int)lo; }
template <> __device__ __forceinline__ unsigned long long c_from<unsigned long long>(uint64_t lo, uint64_t) { return lo; }
template <> __device__ __forceinline__ U128 c_from<U128>(uint64_t lo, uint64_t hi) { return U128{lo, hi}; }

__device__ __forceinline__ unsigned int c_shfl(unsigned int v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ unsigned long long c_shfl(unsigned long long v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ U128 c_shfl(U128 v, int l) {
    return U128{__shfl_sync(0xffffffffu, v.lo, l), __shfl_sync(0xffffffffu, v.hi, l)};
}

// 16-byte vector load of V consecutive storage elements (address 16-byte aligned).
template <class S, int V>
__device__ __forceinline__ void load_vec(const S *p, S *out) {
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
    union { uint4 q; S s[V]; } u;
    u.q = q;
#pragma unroll
    for (int j = 0; j < V; j++) out[j] = u.s[j];
}

// ---------------------------------------------------------------------------------
// small device utilities
// ---------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void set_status(Ctl *ctl, uint32_t code) {
    atomicCAS(&ctl->status, 0u, code);
}
// SplitMix64 finaliser, used to jitter sample positions.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class K>
__device__ __forceinline__ typename K::S *buffer(const Job *job, int which) {
    return reinterpret_cast<typename K::S *>(which ? job->alt : job->base);
}

// Tile geometry: tiles of a segment start at the 16-byte boundary at or below begin.
template <int V>
__device__ __forceinline__ int64_t tile_origin(uint64_t begin, uint32_t vec_off) {
    return (int64_t)begin - (int64_t)((begin + vec_off) & (uint64_t)(V - 1));
}
__device__ __forceinline__ uint32_t tiles_for(uint64_t end, int64_t s0, int tile) {
    return (uint32_t)(((int64_t)end - s0 + tile - 1) / tile);
}

// Look-back status word: [63:62] flag (0 empty, 1 aggregate, 2 inclusive prefix),
// [61:31] count of <p, [30:0] count of >p.
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62;
__device__ __forceinline__ unsigned long long lb_pack(unsigned long long flag, uint64_t lt, uint64_t gt) {
    return flag | ((lt & 0x7FFFFFFFull) << 31) | (gt & 0x7FFFFFFFull);
}

// Pushes [b, e) to the next level: frontier if larger than small_T, leaf otherwise.
template <int V, int TILE>
__device__ void push_segment(const Job *job, Ctl *ctl, int np, uint64_t b, uint64_t e) {
    if (e <= b) return;
    const uint64_t m = e - b;
    if (m > job->small_T) {
        const uint32_t fi = atomicAdd(&ctl->nfront[np], 1u);
        const int64_t s0 = tile_origin<V>(b, job->vec_off);
        const uint32_t nt = tiles_for(e, s0, TILE);
        const uint32_t tb = atomicAdd(&ctl->ntiles[np], nt);
        if (fi >= job->cap_front || (uint64_t)tb + nt > job->cap_tiles) {
            set_status(ctl, TSQS_EINTERNAL);
            return;
        }
        SegDesc d;
        d.begin = b; d.end = e; d.s0 = s0; d.tile_begin = tb; d.ntiles = nt;
        d.piv_lo = 0; d.piv_hi = 0;
        job->front[np][fi] = d;
        atomicAdd((unsigned long long *)&ctl->front_keys[np], (unsigned long long)m);
    } else {
        const uint32_t li = atomicAdd(&ctl->nleaf[np], 1u);
        if (li >= job->cap_leaves) { set_status(ctl, TSQS_EINTERNAL); return; }
        LeafItem it;
        it.begin = b; it.len = (uint32_t)m; it.kind = LEAF_SORT; it.v_lo = 0; it.v_hi = 0;
        job->leaves[np][li] = it;
    }
}

// ---------------------------------------------------------------------------------
// Setup and init
// ---------------------------------------------------------------------------------

// One thread: stores the job description and zeroes the control block.
__global__ void k_setup(Job *job, Ctl *ctl, Job j);

// Seeds level 0: one segment [0, n) or every segment of seg_offsets.  Segments of 0 or
// 1 element are already in place; small ones go straight to the leaf queue.
template <int KIND, int TILE>
__global__ void k_init(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = job->seg_offsets ? job->seg_offsets[s] : 0;
        const uint64_t e = job->seg_offsets ? job->seg_offsets[s + 1] : job->n;
        if (e < b || e > job->n || e - b >= (1ull << 31)) { set_status(ctl, TSQS_EINVAL); continue; }
        if (e - b <= 1) continue;
        push_segment<K::V, TILE>(job, ctl, 0, b, e);
    }
}

// ---------------------------------------------------------------------------------
// Pivot: exact lower median of a jittered, stratified sample (one warp).
// Sample k of a segment of m elements is drawn uniformly from stratum
// [b + m k / S, b + m (k+1) / S): equally spaced like the paper's ninther and
// fifteenther, with every position shifted by a seeded random amount (Section V.C).
// ---------------------------------------------------------------------------------

template <class K>
__device__ typename K::C sample_pivot(const typename K::S *src, uint64_t b, uint64_t e,
                                      uint32_t S_req, uint64_t seed, uint64_t *positions) {
    using C = typename K::C;
    const int lane = threadIdx.x & 31;
    const uint64_t m = e - b;
    uint32_t S = S_req > (uint32_t)kMaxSamples ? (uint32_t)kMaxSamples : S_req;
    if ((uint64_t)S > m) S = (uint32_t)m;
    if ((S & 1u) == 0) S -= 1;                       // odd: one true median
    if (S == 0) S = 1;
    C v[2];
    bool ok[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const uint32_t k = (uint32_t)lane + 32u * h;
        ok[h] = k < S;
        v[h] = c_max<C>();
        if (ok[h]) {
            const uint64_t lo = b + (m * k) / S, hi = b + (m * (k + 1)) / S;
            const uint64_t z = mix64(seed ^ (b * 0x9E3779B97F4A7C15ull) ^ (e * 0xC2B2AE3D27D4EB4Full)
                                     ^ ((uint64_t)(k + 1) * 0x165667B19E3779F9ull));
            const uint64_t pos = lo + (hi > lo ? z % (hi - lo) : 0);
            if (positions) positions[k] = pos;
            v[h] = K::canon(src[pos]);
        }
    }
    // rank of each sample: #smaller + #equal with a lower index (ties broken by index)
    uint32_t rank[2] = {0, 0};
    for (int sl = 0; sl < 32; sl++) {
#pragma unroll
        for (int g = 0; g < 2; g++) {
            const C y = c_shfl(v[g], sl);
            const uint32_t ky = (uint32_t)sl + 32u * g;
            if (ky < S) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t k = (uint32_t)lane + 32u * h;
                    rank[h] += (c_lt(y, v[h]) || (c_eq(y, v[h]) && ky < k)) ? 1u : 0u;
                }
            }
        }
    }
    const uint32_t want = (S - 1) / 2;
    C piv = v[0];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const unsigned hit = __ballot_sync(0xffffffffu, ok[h] && rank[h] == want);
        if (hit) piv = c_shfl(v[h], __ffs(hit) - 1);
    }
    return piv;
}

// One block per frontier segment (grid-stride): pivot by warp 0, tile tables by all.
template <int KIND, int TILE>
__global__ void k_pivot(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const int par = ctl->level & 1;
    if (*(volatile uint32_t *)&ctl->status) return;        // queues may be inconsistent
    const uint32_t nf = min(ctl->nfront[par], job->cap_front);
    const typename K::S *src = buffer<K>(job, par);
    for (uint32_t si = blockIdx.x; si < nf; si += gridDim.x) {
        SegDesc *d = &job->front[par][si];
        const uint64_t b = d->begin, e = d->end;
        const uint32_t tb = d->tile_begin, nt = d->ntiles;
        if (threadIdx.x < 32) {
            const typename K::C p = sample_pivot<K>(src, b, e, job->samples, job->seed, nullptr);
            if (threadIdx.x == 0) c_words(p, d->piv_lo, d->piv_hi);
        }
        for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
            job->tile_seg[tb + t] = si;
            job->tile_status[tb + t] = 0ull;
        }
        if (threadIdx.x == 0) job->seg_done[si] = 0u;
    }
}

// ---------------------------------------------------------------------------------
// Decoupled look-back (one warp): exclusive prefix (#<p, #>p) of tile `tile`, whose
// segment's tile 0 has global id `first`.  A window of 32 predecessors is read at
// once; the nearest inclusive prefix ends the walk.  Every wait is bounded: after
// spin_limit polls the status becomes TSQS_ETIMEOUT and the walk stops.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ void lookback(const unsigned long long *status, uint32_t tile,
                                         uint32_t first, uint32_t spin_limit, Ctl *ctl,
                                         uint64_t &ex_lt, uint64_t &ex_gt) {
    const int lane = threadIdx.x & 31;
    uint64_t acc_lt = 0, acc_gt = 0;
    int64_t top = (int64_t)tile - 1;
    for (;;) {
        const int64_t i = top - lane;
        const bool inr = i >= (int64_t)first;
        unsigned long long w = 0;
        bool to = false;
        if (inr) {
            uint32_t polls = 0;
            for (;;) {
                w = ld_relaxed(status + i);
                if (w >> 62) break;
                if (++polls >= spin_limit) { to = true; break; }
                __nanosleep(polls < 64 ? 32 : 256);
            }
        }
        if (__any_sync(0xffffffffu, to)) {
            if (lane == 0) set_status(ctl, TSQS_ETIMEOUT);
            break;
        }
        const unsigned inc = __ballot_sync(0xffffffffu, inr && (w >> 62) == 2ull);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        uint64_t c_lt = (inr && lane <= stop) ? ((w >> 31) & 0x7FFFFFFFull) : 0;
        uint64_t c_gt = (inr && lane <= stop) ? (w & 0x7FFFFFFFull) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_lt += __shfl_xor_sync(0xffffffffu, c_lt, o);
            c_gt += __shfl_xor_sync(0xffffffffu, c_gt, o);
        }
        acc_lt += c_lt;
        acc_gt += c_gt;
        if (inc) break;
        top -= 32;
        if (top < (int64_t)first) {          // cannot happen: tile 0 publishes inclusive
            if (lane == 0) set_status(ctl, TSQS_EINTERNAL);
            break;
        }
    }
    ex_lt = acc_lt;
    ex_gt = acc_gt;
}

// ---------------------------------------------------------------------------------
// Partition (persistent): tiles of TILE = BLOCK * ITEMS keys claimed in order.
// ---------------------------------------------------------------------------------

template <int KIND, int BLOCK, int ITEMS>
struct PartSmem {
    using S = typename Key<KIND>::S;
    S stage[BLOCK * ITEMS];
    uint32_t wsum[BLOCK / 32];
    uint32_t tile, tot, last, nch;
    unsigned long long ex_lt, ex_gt;
    uint64_t eqb, eqe, fb;
};

template <int KIND, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) k_partition(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    using S = typename K::S;
    using C = typename K::C;
    constexpr int TILE = BLOCK * ITEMS, V = K::V, NV = ITEMS / V, NW = BLOCK / 32;
    static_assert(ITEMS % V == 0 && ITEMS <= 32 && TILE < 65536, "tile shape");
    __shared__ __align__(16) PartSmem<KIND, BLOCK, ITEMS> sm;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int par = ctl->level & 1;
    if (*(volatile uint32_t *)&ctl->status) return;        // queues may be inconsistent
    const uint32_t ntiles = min(ctl->ntiles[par], job->cap_tiles);
    const uint32_t nfront = min(ctl->nfront[par], job->cap_front);
    const S *__restrict__ src = buffer<K>(job, par);
    S *__restrict__ dst = buffer<K>(job, par ^ 1);
    const bool epilogue = (job->pad & 1u) == 0;      // debug runs skip the epilogue

    for (;;) {
        if (tid == 0) sm.tile = atomicAdd(&ctl->tile_claim, 1u);
        __syncthreads();
        const uint32_t tile = sm.tile;
        if (tile >= ntiles) break;
        const uint32_t si = job->tile_seg[tile];
        if (si >= nfront) {                              // cannot happen with a sane queue
            if (tid == 0) set_status(ctl, TSQS_EINTERNAL);
            __syncthreads();
            continue;
        }
        const SegDesc sd = job->front[par][si];
        const C piv = c_from<C>(sd.piv_lo, sd.piv_hi);
        const uint32_t tl = tile - sd.tile_begin;
        const int64_t t0 = sd.s0 + (int64_t)tl * TILE;
        const int64_t sb = (int64_t)sd.begin, se = (int64_t)sd.end;

        // ---- load and classify: 16-byte loads inside the segment, scalar at its ends
        S v[ITEMS];
        uint32_t ltm = 0, gtm = 0;
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const int64_t e0 = t0 + (int64_t)(k * BLOCK + tid) * V;
            if (e0 >= sb && e0 + V <= se) {
                load_vec<S, V>(src + e0, &v[k * V]);
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const C c = K::canon(v[k * V + j]);
                    ltm |= (uint32_t)c_lt(c, piv) << (k * V + j);
                    gtm |= (uint32_t)c_lt(piv, c) << (k * V + j);
                }
            } else {
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const int64_t e = e0 + j;
                    if (e >= sb && e < se) {
                        v[k * V + j] = src[e];
                        const C c = K::canon(v[k * V + j]);
                        ltm |= (uint32_t)c_lt(c, piv) << (k * V + j);
                        gtm |= (uint32_t)c_lt(piv, c) << (k * V + j);
                    }
                }
            }
        }

        // ---- tile scan of packed counts (#<p in bits 0-15, #>p in bits 16-31)
        const uint32_t cnt = (uint32_t)__popc(ltm) | ((uint32_t)__popc(gtm) << 16);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) sm.wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t ws = lane < NW ? sm.wsum[lane] : 0u;
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < NW) sm.wsum[lane] = wi - ws;
            const uint32_t total = __shfl_sync(0xffffffffu, wi, NW - 1);
            const uint64_t agg_lt = total & 0xFFFFu, agg_gt = total >> 16;
            uint64_t ex_lt = 0, ex_gt = 0;
            unsigned long long *stw = job->tile_status + tile;
            // test hook: tile 1 never publishes, so its successors' waits must expire
            const bool publish = !((job->pad & 2u) && tile == 1u);
            if (tl == 0) {
                if (lane == 0 && publish) st_relaxed(stw, lb_pack(kFlagInc, agg_lt, agg_gt));
            } else {
                if (lane == 0 && publish) st_relaxed(stw, lb_pack(kFlagAgg, agg_lt, agg_gt));
                lookback(job->tile_status, tile, sd.tile_begin, job->spin_limit, ctl, ex_lt, ex_gt);
                if (lane == 0 && publish)
                    st_relaxed(stw, lb_pack(kFlagInc, ex_lt + agg_lt, ex_gt + agg_gt));
            }
            if (lane == 0) { sm.ex_lt = ex_lt; sm.ex_gt = ex_gt; sm.tot = total; }
        }
        __syncthreads();

        // ---- stage: <p from the front of the tile buffer, >p from its back
        const uint32_t texcl = sm.wsum[warp] + inc - cnt;
        uint32_t lp = texcl & 0xFFFFu, gp = texcl >> 16;
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            if ((ltm >> i) & 1u) sm.stage[lp++] = v[i];
            else if ((gtm >> i) & 1u) sm.stage[TILE - 1 - gp++] = v[i];
        }
        __syncthreads();

        // ---- coalesced write-out: <p ascending from begin, >p descending from end
        const uint32_t tlt = sm.tot & 0xFFFFu, tgt = sm.tot >> 16;
        S *dl = dst + (sd.begin + sm.ex_lt);
        for (uint32_t i = tid; i < tlt; i += BLOCK) dl[i] = sm.stage[i];
        S *dr = dst + (sd.end - 1 - sm.ex_gt);
        for (uint32_t i = tid; i < tgt; i += BLOCK) *(dr - i) = sm.stage[TILE - 1 - i];

        // ---- last tile of the segment: push the children and the =p fill
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const uint32_t d = atomicAdd(&job->seg_done[si], 1u);
            sm.last = (d + 1 == sd.ntiles) ? 1u : 0u;
        }
        __syncthreads();
        if (sm.last && epilogue) {
            if (tid == 0) {
                __threadfence();
                const unsigned long long w = ld_relaxed(job->tile_status + sd.tile_begin + sd.ntiles - 1);
                const uint64_t nlt = (w >> 31) & 0x7FFFFFFFull, ngt = w & 0x7FFFFFFFull;
                const uint64_t m = sd.end - sd.begin;
                const int np = par ^ 1;
                sm.nch = 0;
                if ((w >> 62) != 2ull || nlt + ngt >= m) {
                    // p is an element of the segment, so the =p run is never empty; a
                    // violation means corrupted state: stop instead of looping forever
                    set_status(ctl, TSQS_EINTERNAL);
                } else {
                    push_segment<V, TILE>(job, ctl, np, sd.begin, sd.begin + nlt);
                    push_segment<V, TILE>(job, ctl, np, sd.end - ngt, sd.end);
                    sm.eqb = sd.begin + nlt;
                    sm.eqe = sd.end - ngt;
                    const uint32_t nch = (uint32_t)((sm.eqe - sm.eqb + kFillChunk - 1) / kFillChunk);
                    const uint32_t fb = atomicAdd(&ctl->nleaf[np], nch);
                    if ((uint64_t)fb + nch > job->cap_leaves) set_status(ctl, TSQS_EINTERNAL);
                    else { sm.nch = nch; sm.fb = fb; }
                }
            }
            __syncthreads();
            const uint32_t nch = sm.nch;
            for (uint32_t c = tid; c < nch; c += BLOCK) {
                LeafItem it;
                it.begin = sm.eqb + (uint64_t)c * kFillChunk;
                const uint64_t rest = sm.eqe - it.begin;
                it.len = (uint32_t)(rest < kFillChunk ? rest : kFillChunk);
                it.kind = LEAF_FILL;
                it.v_lo = sd.piv_lo;
                it.v_hi = sd.piv_hi;
                job->leaves[par ^ 1][sm.fb + c] = it;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// Leaf pass (persistent): on-chip bitonic sort of small segments and =p fills.
// ---------------------------------------------------------------------------------

template <class C>
__device__ __forceinline__ void bitonic_smem(C *s, uint32_t P, int nthreads) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < (P >> 1); i += nthreads) {
                const uint32_t a = 2 * i - (i & (j - 1));
                const uint32_t b = a + j;
                const bool up = (a & k) == 0;
                const C x = s[a], y = s[b];
                if (up ? c_lt(y, x) : c_lt(x, y)) { s[a] = y; s[b] = x; }
            }
            __syncthreads();
        }
    }
}

template <int KIND, int LB>
__global__ void __launch_bounds__(LB) k_leaf(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    using S = typename K::S;
    using C = typename K::C;
    extern __shared__ __align__(16) unsigned char leaf_raw[];
    C *s = reinterpret_cast<C *>(leaf_raw);
    __shared__ uint32_t s_item;
    const int par = ctl->level & 1;
    if (*(volatile uint32_t *)&ctl->status) return;        // queues may be inconsistent
    const uint32_t nl = min(ctl->nleaf[par], job->cap_leaves);
    const S *src = buffer<K>(job, par);          // may be the same buffer as out
    S *out = reinterpret_cast<S *>(job->base);
    uint64_t sorted = 0, filled = 0, items = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctl->leaf_claim, 1u);
        __syncthreads();
        const uint32_t ii = s_item;
        if (ii >= nl) break;
        const LeafItem it = job->leaves[par][ii];
        items++;
        if (it.kind == LEAF_FILL) {
            const S val = K::uncanon(c_from<C>(it.v_lo, it.v_hi));
            for (uint32_t i = threadIdx.x; i < it.len; i += LB) out[it.begin + i] = val;
            filled += it.len;
        } else if (it.len > (uint32_t)kMaxSmall) {
            if (threadIdx.x == 0) set_status(ctl, TSQS_EINTERNAL);
        } else {
            const uint32_t len = it.len;
            uint32_t P = 1;
            while (P < len) P <<= 1;
            for (uint32_t i = threadIdx.x; i < P; i += LB)
                s[i] = i < len ? K::canon(src[it.begin + i]) : c_max<C>();
            __syncthreads();
            bitonic_smem<C>(s, P, LB);
            for (uint32_t i = threadIdx.x; i < len; i += LB) out[it.begin + i] = K::uncanon(s[i]);
            sorted += len;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && items) {
        atomicAdd((unsigned long long *)&ctl->leaf_sorted, (unsigned long long)sorted);
        atomicAdd((unsigned long long *)&ctl->leaf_filled, (unsigned long long)filled);
        atomicAdd((unsigned long long *)&ctl->leaf_items, (unsigned long long)items);
    }
}

// ---------------------------------------------------------------------------------
// Step-level test hooks
// ---------------------------------------------------------------------------------

// Frontier[0] <- the given segments with the given pivots (original representation).
template <int KIND, int TILE>
__global__ void k_dbg_setup_partition(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const typename K::S *piv = reinterpret_cast<const typename K::S *>(job->dbg_pivots);
    for (uint64_t s = blockIdx.x; s < job->nseg; s += gridDim.x) {
        __shared__ uint32_t s_tb, s_nt;
        const uint64_t b = job->seg_offsets[s], e = job->seg_offsets[s + 1];
        const int64_t s0 = tile_origin<K::V>(b, job->vec_off);
        if (threadIdx.x == 0) {
            s_nt = e > b ? tiles_for(e, s0, TILE) : 0u;
            s_tb = atomicAdd(&ctl->ntiles[0], s_nt);
            SegDesc d;
            d.begin = b; d.end = e; d.s0 = s0; d.tile_begin = s_tb; d.ntiles = s_nt;
            c_words(K::canon(piv[s]), d.piv_lo, d.piv_hi);
            job->front[0][s] = d;
            job->seg_done[s] = 0u;
        }
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < s_nt; t += blockDim.x) {
            job->tile_seg[s_tb + t] = (uint32_t)s;
            job->tile_status[s_tb + t] = 0ull;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nfront[0] = (uint32_t)job->nseg;
}

__global__ void k_dbg_counts(const Job *__restrict__ job, Ctl *ctl);

template <int KIND>
__global__ void k_dbg_pivot(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const uint64_t b = job->seg_offsets[0], e = job->seg_offsets[1];
    const typename K::C p = sample_pivot<K>(buffer<K>(job, 0), b, e, job->samples, job->seed,
                                            job->dbg_positions);
    if (threadIdx.x == 0)
        *reinterpret_cast<typename K::S *>(job->dbg_pivot_out) = K::uncanon(p);
}

// Level control (one thread).  Records the level's statistics, resets the consumed
// queues, advances the level and sets the loop condition.
__global__ void k_finish(const Job *job, Ctl *ctl, cudaGraphConditionalHandle handle,
                         int use_handle, uint32_t max_levels);

}  // namespace tsqs
