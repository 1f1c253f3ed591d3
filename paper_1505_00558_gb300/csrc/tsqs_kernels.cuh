// tsqs_kernels.cuh -- device code of the three-way partition sort (sm_103a).
//
// Kernels of one level of the level loop (see tsqs_internal.h for the queue layout):
//   k_leaf       on-chip pass over the queued leaf items of the levels so far:
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
//   k_level_end  pushes every segment's children and =p fill, then advances the
//                level and decides whether the loop continues
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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

// D is the domain the partition compares in: the native signed/unsigned integer
// where the hardware orders it directly, the canonical form otherwise.
template <> struct Key<TSQS_I32> {
    using S = unsigned int; using C = unsigned int; using D = int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) { return x ^ 0x80000000u; }
    static __device__ __forceinline__ S uncanon(C c) { return c ^ 0x80000000u; }
    static __device__ __forceinline__ D dom(S x) { return (int)x; }
    static __device__ __forceinline__ D pdom(C c) { return (int)(c ^ 0x80000000u); }
};
template <> struct Key<TSQS_U32> {
    using S = unsigned int; using C = unsigned int; using D = unsigned int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) { return x; }
    static __device__ __forceinline__ S uncanon(C c) { return c; }
    static __device__ __forceinline__ D dom(S x) { return x; }
    static __device__ __forceinline__ D pdom(C c) { return c; }
};
template <> struct Key<TSQS_F32> {
    using S = unsigned int; using C = unsigned int; static constexpr int V = 4;
    static __device__ __forceinline__ C canon(S x) {
        return x ^ ((unsigned int)((int)x >> 31) | 0x80000000u);
    }
    static __device__ __forceinline__ S uncanon(C c) {
        return c ^ (~(unsigned int)((int)c >> 31) | 0x80000000u);
    }
    using D = unsigned int;
    static __device__ __forceinline__ D dom(S x) { return canon(x); }
    static __device__ __forceinline__ D pdom(C c) { return c; }
};
template <> struct Key<TSQS_I64> {
    using S = unsigned long long; using C = unsigned long long; using D = long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) { return x ^ 0x8000000000000000ull; }
    static __device__ __forceinline__ S uncanon(C c) { return c ^ 0x8000000000000000ull; }
    static __device__ __forceinline__ D dom(S x) { return (long long)x; }
    static __device__ __forceinline__ D pdom(C c) { return (long long)(c ^ 0x8000000000000000ull); }
};
template <> struct Key<TSQS_U64> {
    using S = unsigned long long; using C = unsigned long long; using D = unsigned long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) { return x; }
    static __device__ __forceinline__ S uncanon(C c) { return c; }
    static __device__ __forceinline__ D dom(S x) { return x; }
    static __device__ __forceinline__ D pdom(C c) { return c; }
};
template <> struct Key<TSQS_F64> {
    using S = unsigned long long; using C = unsigned long long; static constexpr int V = 2;
    static __device__ __forceinline__ C canon(S x) {
        return x ^ ((unsigned long long)((long long)x >> 63) | 0x8000000000000000ull);
    }
    static __device__ __forceinline__ S uncanon(C c) {
        return c ^ (~(unsigned long long)((long long)c >> 63) | 0x8000000000000000ull);
    }
    using D = unsigned long long;
    static __device__ __forceinline__ D dom(S x) { return canon(x); }
    static __device__ __forceinline__ D pdom(C c) { return c; }
};
template <> struct Key<TSQS_U64_U64_REC> {
    using S = Rec16; using C = U128; static constexpr int V = 1;
    static __device__ __forceinline__ C canon(S x) { return U128{x.pay, x.key}; }
    static __device__ __forceinline__ S uncanon(C c) { Rec16 r; r.key = c.hi; r.pay = c.lo; return r; }
    using D = U128;
    static __device__ __forceinline__ D dom(S x) { return canon(x); }
    static __device__ __forceinline__ D pdom(C c) { return c; }
};

// Comparison against a pivot fixed for a whole tile.  RawDom compares the storage words
// as integers of type T; CanonDom through the key kind's own domain.  Float keys use
// raw words (float_raw_classify): with a pivot whose sign bit is clear, a signed compare
// of the raw words is IEEE totalOrder; with it set, an unsigned compare is the reverse
// order, so the <p and >p masks swap.  That saves the per-key canonical transform.
template <class T> struct RawDom {
    template <class S> __device__ __forceinline__ T operator()(S x) const { return (T)x; }
};
template <class K> struct CanonDom {
    __device__ __forceinline__ typename K::D operator()(typename K::S x) const { return K::dom(x); }
};
template <int KIND> constexpr bool kFloatKind = KIND == TSQS_F32 || KIND == TSQS_F64;

// canonical-order helpers, overloaded on C (and on the comparison domains D)
__device__ __forceinline__ bool c_lt(int a, int b) { return a < b; }
__device__ __forceinline__ bool c_lt(long long a, long long b) { return a < b; }
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

// 16-byte shared-memory load of V storage elements (address 16-byte aligned).
template <class S, int V>
__device__ __forceinline__ void lds_vec(const S *p, S *out) {
    union { uint4 q; S s[V]; } u;
    u.q = *reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int j = 0; j < V; j++) out[j] = u.s[j];
}
// 16-byte global store of V storage elements (address 16-byte aligned).
template <class S, int V>
__device__ __forceinline__ void stg_vec(S *p, const S *in) {
    union { uint4 q; S s[V]; } u;
#pragma unroll
    for (int j = 0; j < V; j++) u.s[j] = in[j];
    *reinterpret_cast<uint4 *>(p) = u.q;
}

// Body of copy_run: nvec 16-byte destination vectors.  Destination vector q takes the
// staged elements SH + q V .. SH + q V + V - 1 counted from the 16-byte-aligned shared
// address sa, so it is assembled from one (SH = 0) or two aligned 16-byte shared loads
// and no scalar shared access is needed.
__device__ __forceinline__ uint32_t smem_addr_of(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <class S, int V, int NT, int SH>
__device__ __forceinline__ void copy_body(S *__restrict__ d, const S *sa, uint32_t nvec) {
    for (uint32_t q = threadIdx.x; q < nvec; q += NT) {
        S a[V], b[V], o[V];
        lds_vec<S, V>(sa + q * V, a);
        if (SH != 0) lds_vec<S, V>(sa + q * V + V, b);
#pragma unroll
        for (int j = 0; j < V; j++) o[j] = (j + SH < V) ? a[j + SH] : b[j + SH - V];
        stg_vec<S, V>(d + q * V, o);
    }
}

// Copies cnt staged elements st[0, cnt) to dst[x, x + cnt): scalar up to the first
// 16-byte boundary of the destination, 16-byte stores for the body, scalar tail.
// (element x of dst is 16-byte aligned iff (x + vec_off) % V == 0; st lies in a
// 16-byte-aligned shared buffer, so the vectors it reads never leave that buffer)
template <class S, int V, int NT>
__device__ __forceinline__ void copy_run(S *__restrict__ dst, uint64_t x, const S *st,
                                         uint32_t cnt, uint32_t vec_off) {
    if (cnt == 0) return;
    uint32_t head = (uint32_t)((V - ((x + vec_off) % V)) % V);
    if (head > cnt) head = cnt;
    const uint32_t nvec = (cnt - head) / V;
    const uint32_t body_end = head + nvec * V;
    const int t = threadIdx.x;
    if ((uint32_t)t < head) dst[x + t] = st[t];
    if (nvec != 0) {
        // misalignment (in elements) of the body's first staged element
        const uint32_t sh = (uint32_t)((smem_addr_of(st + head) / sizeof(S)) % V);
        const S *sa = st + head - sh;
        S *d = dst + x + head;
        if (sh == 0) copy_body<S, V, NT, 0>(d, sa, nvec);
        else if (V > 1 && sh == 1) copy_body<S, V, NT, (V > 1 ? 1 : 0)>(d, sa, nvec);
        else if (V > 2 && sh == 2) copy_body<S, V, NT, (V > 2 ? 2 : 0)>(d, sa, nvec);
        else if (V > 3) copy_body<S, V, NT, (V > 3 ? 3 : 0)>(d, sa, nvec);
    }
    const uint32_t tail = cnt - body_end;
    if ((uint32_t)t < tail) dst[x + body_end + t] = st[body_end + t];
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
// Block-uniform read of the sticky status: every thread of the block gets the same
// answer, so an early return never splits a warp or a barrier.
__device__ __forceinline__ bool block_aborted(const Ctl *ctl) {
    __shared__ uint32_t s_abort;
    if (threadIdx.x == 0) s_abort = *(volatile const uint32_t *)&ctl->status;
    __syncthreads();
    const bool a = s_abort != 0u;
    __syncthreads();
    return a;
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

// Final (#<p, #>p) of a segment once all its tiles are counted: the cursor in atomic
// mode, the last tile's inclusive prefix in look-back mode.  False if not available.
__device__ __forceinline__ bool seg_totals(const Job *job, uint32_t si, uint32_t tile_begin,
                                           uint32_t ntiles, uint64_t &nlt, uint64_t &ngt) {
    if (job->offset_mode == 0u) {
        const unsigned long long c = ld_relaxed(job->seg_cursor + si);
        nlt = c & 0xFFFFFFFFull;
        ngt = c >> 32;
        return true;
    }
    if (ntiles == 0) { nlt = ngt = 0; return true; }
    const unsigned long long w = ld_relaxed(job->tile_status + tile_begin + ntiles - 1);
    nlt = (w >> 31) & 0x7FFFFFFFull;
    ngt = w & 0x7FFFFFFFull;
    return (w >> 62) == 2ull;
}

// Pushes [b, e) to the next level: frontier if larger than small_T, leaf otherwise.
template <int V>
__device__ void push_segment(const Job *job, Ctl *ctl, int np, uint64_t b, uint64_t e) {
    const int TILE = (int)job->tile;
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
        const uint32_t li = atomicAdd(&ctl->nleaf, 1u);
        if (li >= job->cap_leaves) { set_status(ctl, TSQS_EINTERNAL); return; }
        LeafItem it;
        it.begin = b; it.len = (uint32_t)m; it.kind = LEAF_SORT | (np ? kLeafInAlt : 0u);
        it.v_lo = 0; it.v_hi = 0;
        job->leaves[li] = it;
    }
}

// ---------------------------------------------------------------------------------
// Setup and init
// ---------------------------------------------------------------------------------

// One thread: stores the job description and zeroes the control block.
__global__ void k_setup(Job *job, Ctl *ctl, Job j);

// Seeds level 0: one segment [0, n) or every segment of seg_offsets.  Segments of 0 or
// 1 element are already in place; small ones go straight to the leaf queue.
template <int KIND>
__global__ void k_init(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = job->seg_offsets ? job->seg_offsets[s] : 0;
        const uint64_t e = job->seg_offsets ? job->seg_offsets[s + 1] : job->n;
        if (e < b || e > job->n || e - b >= (1ull << 31)) { set_status(ctl, TSQS_EINVAL); continue; }
        if (e - b <= 1) continue;
        if (job->presort[s] != 0u) continue;             // already in order (presortedness pass)
        push_segment<K::V>(job, ctl, 0, b, e);
    }
}

// ---------------------------------------------------------------------------------
// Presortedness (the GPU counterpart of Section III.I's possibly-sorted and possibly-
// reversed handlers).  The paper reads the orientation of its median-of-3 sample and,
// when the sample is in order, checks the segment while partitioning.  Here every root
// segment above the on-chip threshold draws 31 evenly spaced samples (one warp); a
// segment whose samples are non-decreasing (or non-increasing) is checked in full by a
// chunked pass that stops early once an adjacent pair is out of order.  A segment that
// passes is final as it stands (non-decreasing) or after one reversal (non-increasing),
// and k_init leaves it out of the level loop.  Random input pays one warp of samples
// per root segment and two launches that return at once.
// ---------------------------------------------------------------------------------

constexpr int kPresortChunk = 8192;

__device__ __forceinline__ void root_bounds(const Job *job, uint64_t s, uint64_t &b, uint64_t &e) {
    b = job->seg_offsets ? job->seg_offsets[s] : 0;
    e = job->seg_offsets ? job->seg_offsets[s + 1] : job->n;
}

// Root segment containing element x (the last s with offsets[s] <= x), by binary search.
__device__ __forceinline__ uint64_t root_of(const Job *job, uint64_t x) {
    if (!job->seg_offsets) return 0;
    uint64_t lo = 0, hi = job->nseg;                  // offsets[lo] <= x < offsets[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (job->seg_offsets[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Orientation samples of every root segment (and the task schedule's row reset).  In a
// graph (use_handle) a flagged segment also sets the IF node that runs the full check
// and the finishing pass; with no candidate both are skipped.
template <int KIND>
__device__ __forceinline__ void orient_body(const Job *__restrict__ job, Ctl *ctl,
                                            cudaGraphConditionalHandle handle, bool use_handle) {
    using K = Key<KIND>;
    using C = typename K::C;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const typename K::S *src = buffer<K>(job, 0);
    if (job->trow) {                   // task schedule: this call's tile rows start empty
        const uint32_t stride = gridDim.x * blockDim.x;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < job->cap_trow; i += stride)
            job->trow[i] = 0ull;
    }
    for (uint64_t s = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += warps) {
        uint64_t b, e;
        root_bounds(job, s, b, e);
        uint32_t flag = 0;
        if (e > b && e <= job->n && e - b > (uint64_t)job->small_T) {
            const uint64_t m = e - b;
            const uint32_t k = min(lane, 30u);          // 31 samples, first and last included
            const C x = K::canon(src[b + ((m - 1) * k) / 30u]);
            const C y = c_shfl(x, (int)((lane + 1u) & 31u));   // lanes 30, 31 compare nothing
            const bool up_ok = lane >= 30u || !c_lt(y, x);
            const bool down_ok = lane >= 30u || !c_lt(x, y);
            if (__all_sync(0xffffffffu, up_ok)) flag = 1;
            else if (__all_sync(0xffffffffu, down_ok)) flag = 2;
        }
        if (lane == 0) {
            job->presort[s] = flag;
            if (flag) atomicOr(&ctl->presort_any, 1u);
            if (flag && use_handle) cudaGraphSetConditional(handle, 1u);
        }
    }
}

template <int KIND>
__global__ void k_orient(const Job *__restrict__ job, Ctl *ctl) {
    orient_body<KIND>(job, ctl, 0, false);
}

template <int KIND>
__global__ void k_orient_if(const Job *__restrict__ job, Ctl *ctl, cudaGraphConditionalHandle handle) {
    orient_body<KIND>(job, ctl, handle, true);
}

// Clears the flag of every candidate segment that has an adjacent pair out of order.
template <int KIND>
__global__ void k_check(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    if (*(volatile const uint32_t *)&ctl->presort_any == 0u) return;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    const uint64_t n = job->n;
    const typename K::S *src = buffer<K>(job, 0);
    __shared__ uint64_t s_first;
    __shared__ uint32_t s_flag;
    for (uint64_t c0 = (uint64_t)blockIdx.x * kPresortChunk; c0 < n; c0 += (uint64_t)gridDim.x * kPresortChunk) {
        const uint64_t c1 = min(c0 + (uint64_t)kPresortChunk, n);
        if (threadIdx.x == 0) s_first = root_of(job, c0);
        __syncthreads();
        for (uint64_t s = s_first; s < nseg; s++) {
            uint64_t b, e;
            root_bounds(job, s, b, e);
            if (b >= c1) break;
            // another block may clear the flag at any moment: one thread reads it and the
            // block acts on that one value, so every thread reaches the same barriers
            if (threadIdx.x == 0) s_flag = *(volatile const uint32_t *)&job->presort[s];
            __syncthreads();
            const uint32_t flag = s_flag;
            if (flag == 0u || e <= c0 || e <= b) {
                __syncthreads();                         // s_flag read by all before reuse
                continue;
            }
            // pairs (i, i + 1) with i in [max(c0, b), min(c1, e - 1))
            const uint64_t i0 = max(c0, b), i1 = min(c1, e - 1);
            bool bad = false;
            for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const typename K::C x = K::canon(src[i]), y = K::canon(src[i + 1]);
                bad |= flag == 1u ? c_lt(y, x) : c_lt(x, y);
            }
            if (__syncthreads_or(bad) && threadIdx.x == 0) job->presort[s] = 0u;
        }
        __syncthreads();
    }
}

// Finishes every segment that passed: reverses a non-increasing one, and writes either
// kind to the output array when that is not the input array.
template <int KIND>
__global__ void k_presort(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    using S = typename K::S;
    if (*(volatile const uint32_t *)&ctl->presort_any == 0u) return;
    const uint64_t nseg = job->seg_offsets ? job->nseg : 1;
    const uint64_t n = job->n;
    S *src = buffer<K>(job, 0);
    S *out = reinterpret_cast<S *>(job->out);
    const bool in_place = job->out == job->base;
    __shared__ uint64_t s_first;
    for (uint64_t c0 = (uint64_t)blockIdx.x * kPresortChunk; c0 < n; c0 += (uint64_t)gridDim.x * kPresortChunk) {
        const uint64_t c1 = min(c0 + (uint64_t)kPresortChunk, n);
        if (threadIdx.x == 0) s_first = root_of(job, c0);
        __syncthreads();
        for (uint64_t s = s_first; s < nseg; s++) {
            uint64_t b, e;
            root_bounds(job, s, b, e);
            if (b >= c1) break;
            const uint32_t flag = job->presort[s];
            if (flag == 0u || e <= b) continue;
            if (threadIdx.x == 0 && c0 <= b && b < c1)
                atomicAdd((unsigned long long *)&ctl->presorted, (unsigned long long)(e - b));
            if (flag == 1u) {
                if (!in_place)
                    for (uint64_t i = max(c0, b) + threadIdx.x; i < min(c1, e); i += blockDim.x) out[i] = src[i];
            } else if (in_place) {
                // swap i with its mirror for every i of the first half that lies in the chunk
                const uint64_t h = b + (e - b) / 2;
                for (uint64_t i = max(c0, b) + threadIdx.x; i < min(c1, h); i += blockDim.x) {
                    const uint64_t j = e - 1 - (i - b);
                    const S t = src[i];
                    src[i] = src[j];
                    src[j] = t;
                }
            } else {
                for (uint64_t i = max(c0, b) + threadIdx.x; i < min(c1, e); i += blockDim.x)
                    out[e - 1 - (i - b)] = src[i];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// Pivot: exact lower median of a jittered, stratified sample (one warp).
// Sample k of a segment of m elements is drawn uniformly from stratum
// [b + m k / S, b + m (k+1) / S): equally spaced like the paper's ninther and
// fifteenther, with every position shifted by a seeded random amount (Section V.C).
// ---------------------------------------------------------------------------------

// L2 loads (no L1 allocation) of one storage element: for data other blocks of the same
// launch have written since this block last read that memory.
__device__ __forceinline__ unsigned int ldcg_key(const unsigned int *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ldcg_key(const unsigned long long *p) { return __ldcg(p); }
__device__ __forceinline__ Rec16 ldcg_key(const Rec16 *p) {
    const ulonglong2 q = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    Rec16 r;
    r.key = q.x;
    r.pay = q.y;
    return r;
}

// kL2: read the samples from L2 (the task schedule samples keys written in the same launch)
template <class K, bool kL2 = false>
__device__ typename K::C sample_pivot(const typename K::S *src, uint64_t b, uint64_t e,
                                      uint32_t S_req, uint64_t seed, uint64_t *positions) {
    using C = typename K::C;
    const int lane = threadIdx.x & 31;
    const uint64_t m = e - b;
    uint32_t S = S_req > (uint32_t)kMaxSamples ? (uint32_t)kMaxSamples : S_req;
    if ((uint64_t)S > m) S = (uint32_t)m;
    if ((S & 1u) == 0) S -= 1;                       // odd: one true median
    if (S == 0) S = 1;
    // stratum k is [b + floor(m k / S), b + floor(m (k+1) / S)); with m = q S + r,
    // floor(m k / S) = q k + floor(r k / S), and r k < 63 * 64, so below 2^32 elements
    // every division is a 32-bit one
    const bool narrow = m < (1ull << 32);
    const uint32_t q = narrow ? (uint32_t)m / S : 0u, r = narrow ? (uint32_t)m % S : 0u;
    C v[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const uint32_t k = (uint32_t)lane + 32u * h;
        v[h] = c_max<C>();
        if (k < S) {
            uint64_t lo, w;
            if (narrow) {
                const uint32_t a0 = q * k + (r * k) / S, a1 = q * (k + 1) + (r * (k + 1)) / S;
                lo = b + a0;
                w = a1 - a0;
            } else {
                lo = b + (m * k) / S;
                w = b + (m * (k + 1)) / S - lo;
            }
            const uint64_t z = mix64(seed ^ (b * 0x9E3779B97F4A7C15ull) ^ (e * 0xC2B2AE3D27D4EB4Full)
                                     ^ ((uint64_t)(k + 1) * 0x165667B19E3779F9ull));
            // offset in [0, w): below 2^32 elements the high word of z times w, shifted
            // down (Lemire's multiply-shift range reduction), else z mod w
            const uint64_t pos = lo + (narrow ? (((z >> 32) * w) >> 32) : z % w);
            if (positions) positions[k] = pos;
            v[h] = K::canon(kL2 ? ldcg_key(src + pos) : src[pos]);
        }
    }
    // the median is the sample of rank (S - 1) / 2: sort the samples across the warp
    // with a bitonic network (unused entries hold the largest key, so they sort last)
    const uint32_t want = (S - 1) / 2;
    if (S <= 32u) {
        // one sample per lane, element index = lane
        C x = v[0];
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const C y = c_shfl(x, lane ^ (int)j);
                const bool keep_min = (((uint32_t)lane & k) == 0u) == (((uint32_t)lane & j) == 0u);
                if (keep_min ? c_lt(y, x) : c_lt(x, y)) x = y;
            }
        }
        return c_shfl(x, (int)want);
    }
    // two samples per lane: element 2 lane + h holds the sample drawn as lane + 32 h
    // (the assignment of samples to elements does not change their order statistics)
    C x0 = v[0], x1 = v[1];
#pragma unroll
    for (uint32_t k = 2; k <= 64; k <<= 1) {
        const bool asc = ((2u * (uint32_t)lane) & k) == 0u;
#pragma unroll
        for (uint32_t j = k >> 1; j > 1; j >>= 1) {
            const C y0 = c_shfl(x0, lane ^ (int)(j >> 1));
            const C y1 = c_shfl(x1, lane ^ (int)(j >> 1));
            const bool keep_min = asc == (((2u * (uint32_t)lane) & j) == 0u);
            if (keep_min ? c_lt(y0, x0) : c_lt(x0, y0)) x0 = y0;
            if (keep_min ? c_lt(y1, x1) : c_lt(x1, y1)) x1 = y1;
        }
        // stride 1: the lane's own pair
        const bool sw = asc ? c_lt(x1, x0) : c_lt(x0, x1);
        const C t = x0;
        x0 = sw ? x1 : x0;
        x1 = sw ? t : x1;
    }
    const C m0 = c_shfl(x0, (int)(want >> 1)), m1 = c_shfl(x1, (int)(want >> 1));
    return (want & 1u) ? m1 : m0;
}

// One warp per frontier segment (grid-stride over warps): the sampled median, then the
// segment's rows of the tile table.
template <int KIND>
__global__ void k_pivot(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const int par = ctl->level & 1;
    if (block_aborted(ctl)) return;                         // queues may be inconsistent
    const uint32_t nf = min(ctl->nfront[par], job->cap_front);
    const typename K::S *src = buffer<K>(job, par);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    const bool lb = job->offset_mode != 0u;
    for (uint32_t si = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); si < nf; si += warps) {
        SegDesc *d = &job->front[par][si];
        const uint64_t b = d->begin, e = d->end;
        const uint32_t tb = d->tile_begin, nt = d->ntiles;
        const typename K::C p = sample_pivot<K>(src, b, e, job->samples, job->seed, nullptr);
        if (lane == 0) {
            c_words(p, d->piv_lo, d->piv_hi);
            job->seg_done[si] = 0u;
            job->seg_cursor[si] = 0ull;
        }
        for (uint32_t t = lane; t < nt; t += 32u) {
            job->tile_seg[tb + t] = si;
            if (lb) job->tile_status[tb + t] = 0ull;
        }
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
// Async-proxy helpers: 1-D bulk copies (TMA) completing on shared-memory mbarriers.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }"
                 ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_addr(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` try_wait rounds (each blocks for a short,
// hardware-defined time); returns false then.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; i++)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Barrier among the consumer warps only (the producer warp never joins it).
template <int N>
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}
// Shared-memory store through a 32-bit shared-window address.
__device__ __forceinline__ void sts_raw(uint32_t a, unsigned int v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v));
}
__device__ __forceinline__ void sts_raw(uint32_t a, unsigned long long v) {
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v));
}
__device__ __forceinline__ void sts_raw(uint32_t a, Rec16 v) {
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(v.key), "l"(v.pay));
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// ---------------------------------------------------------------------------------
// Partition (persistent, warp-specialised).
//   producer warp   claims tiles in order, reads each tile's segment, and stages the
//                   tile's 16-byte-aligned interior into a ring of NBUF shared-memory
//                   buffers with one bulk copy (TMA), NBUF-1 tiles ahead
//   consumer warps  classify the tile against p, scan the packed counts, stage the
//                   <p / >p elements back into the same buffer while warp 0 runs the
//                   decoupled look-back, then write both runs out coalesced
// Tiles are claimed in increasing order and every CTA processes its tiles in claim
// order, so the lowest unpublished tile is always one a consumer is working on: the
// look-back always makes progress.
// ---------------------------------------------------------------------------------

struct TileMeta {
    int64_t t0, cs, ce;            // tile origin, bulk-copied element range [cs, ce)
    uint64_t sb, se;               // segment bounds
    uint64_t piv_lo, piv_hi;
    uint32_t tile, si, tl, ntiles_seg, tile_begin, valid;
};

// Producer: claims tile `it` of this CTA (two tiles per atomic in atomic mode, one in
// look-back mode) and fills its TileMeta from the tile table and the segment descriptor.
template <int TILE, int V>
__device__ __forceinline__ void producer_meta(const Job *job, Ctl *ctl, int par, uint32_t it,
                                              uint32_t &claim, uint32_t ntiles, uint32_t nfront,
                                              int64_t e_lo, int64_t e_hi, TileMeta &m) {
    if (job->offset_mode != 0u) {
        m.tile = atomicAdd(&ctl->tile_claim, 1u);
    } else {
        if ((it & 1u) == 0u) claim = atomicAdd(&ctl->tile_claim, 2u);
        m.tile = claim + (it & 1u);
    }
    m.valid = 0;
    m.cs = m.ce = 0;
    if (m.tile < ntiles) {
        m.si = job->tile_seg[m.tile];
        if (m.si < nfront) {
            const SegDesc sd = job->front[par][m.si];
            m.valid = 1;
            m.sb = sd.begin; m.se = sd.end;
            m.piv_lo = sd.piv_lo; m.piv_hi = sd.piv_hi;
            m.tile_begin = sd.tile_begin; m.ntiles_seg = sd.ntiles;
            m.tl = m.tile - sd.tile_begin;
            m.t0 = sd.s0 + (int64_t)m.tl * TILE;
            // aligned hull of the segment inside the tile, clipped to the buffer
            const int64_t a_sb = (int64_t)sd.begin - (((int64_t)sd.begin + job->vec_off) % V);
            const int64_t a_se = (int64_t)sd.end + ((V - (((int64_t)sd.end + job->vec_off) % V)) % V);
            m.cs = max(max(m.t0, a_sb), e_lo);
            m.ce = min(min(m.t0 + TILE, a_se), e_hi);
            if (m.ce < m.cs) m.ce = m.cs;
        } else {
            set_status(ctl, TSQS_EINTERNAL);
        }
    } else {
        m.tile = 0xFFFFFFFFu;                      // end of work
    }
}

template <int KIND, int BLOCK, int ITEMS, int NBUF>
struct PartLayout {
    using S = typename Key<KIND>::S;
    static constexpr int TILE = BLOCK * ITEMS;
    static constexpr int NW = BLOCK / 32;
    // one ring slot: the tile plus one 16-byte dummy slot that absorbs =p elements
    static constexpr int SLOT = TILE + Key<KIND>::V;
    static constexpr size_t buf_bytes = (size_t)SLOT * sizeof(S);
    static constexpr size_t off_bar = NBUF * buf_bytes;
    static constexpr size_t off_meta = off_bar + 2 * NBUF * sizeof(unsigned long long);
    static constexpr size_t off_misc = off_meta + NBUF * sizeof(TileMeta);
    static constexpr size_t bytes = off_misc + 128 + NW * sizeof(uint32_t);
    static_assert(2 * 24 <= 128, "misc area");
};

// Resident CTAs per SM the register budget of a partition shape aims at; `words` is
// the 32-bit registers one thread's keys take (keys per thread x key size / 4).
constexpr int part_min_blocks(int block, int words) {
    return words >= 32 ? (block >= 256 ? 2 : (block >= 192 ? 3 : 4))
         : words >= 24 ? (block <= 192 ? 4 : 3)
         : (block >= 512 ? 2 : (block >= 256 ? 4 : 6));
}

struct PartMisc {
    unsigned long long ex_lt, ex_gt;
    uint32_t total, pad;
};

template <int KIND, int BLOCK, int ITEMS, int NBUF>
__global__ void __launch_bounds__(BLOCK + 32, part_min_blocks(BLOCK, ITEMS * (int)sizeof(typename Key<KIND>::S) / 4)) k_partition(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    using S = typename K::S;
    using C = typename K::C;
    using LY = PartLayout<KIND, BLOCK, ITEMS, NBUF>;
    using D = typename K::D;
    constexpr int TILE = LY::TILE, V = K::V, NW = LY::NW, SLOT = LY::SLOT, NV = ITEMS / V;
    static_assert(ITEMS % V == 0, "whole 16-byte vectors per thread");
    static_assert(ITEMS <= 32 && TILE < 65536 && (TILE % V) == 0, "tile shape");
    extern __shared__ __align__(128) unsigned char psm[];
    S *bufs = reinterpret_cast<S *>(psm);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(psm + LY::off_bar);
    unsigned long long *empty = full + NBUF;
    TileMeta *meta = reinterpret_cast<TileMeta *>(psm + LY::off_meta);
    PartMisc *misc = reinterpret_cast<PartMisc *>(psm + LY::off_misc);
    uint32_t *wsum = reinterpret_cast<uint32_t *>(psm + LY::off_misc + 128);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int par = ctl->level & 1;
    if (block_aborted(ctl)) return;                         // queues may be inconsistent
    const uint32_t ntiles = min(ctl->ntiles[par], job->cap_tiles);
    const uint32_t nfront = min(ctl->nfront[par], job->cap_front);
    const S *__restrict__ src = buffer<K>(job, par);
    S *__restrict__ dst = buffer<K>(job, par ^ 1);
    const uint32_t wait_limit = 1u << 20;

    if (tid == 0) {
        for (int s = 0; s < NBUF; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NW) {
        // ================================ producer ================================
        if (lane != 0) return;
        // element range of the buffer that 16-byte copies may touch
        const int64_t n = (int64_t)job->n;
        const int64_t e_lo = (int64_t)((V - (int64_t)job->vec_off % V) % V);
        const int64_t e_hi = n - ((n + (int64_t)job->vec_off) % V);
        uint32_t claim = 0;
        const bool lookback_mode = job->offset_mode != 0u;
        TileMeta m;
        for (uint32_t it = 0;; it++) {
            const int s = (int)(it % NBUF);
            // atomic mode: tile it's claim and descriptor were read before the wait below
            // (at the end of the previous iteration), so their latency overlaps the wait
            // for the slot.  Look-back mode: a claimed tile must start at once (its
            // successors wait for its aggregate), so it is claimed after the wait.
            if (it == 0u && !lookback_mode) producer_meta<TILE, V>(job, ctl, par, it, claim, ntiles, nfront, e_lo, e_hi, m);
            if (it >= (uint32_t)NBUF && !mbar_wait(&empty[s], ((it / NBUF) - 1) & 1u, wait_limit)) {
                set_status(ctl, TSQS_ETIMEOUT);
            }
            if (lookback_mode) producer_meta<TILE, V>(job, ctl, par, it, claim, ntiles, nfront, e_lo, e_hi, m);
            meta[s] = m;
            if (m.valid && m.ce > m.cs) {
                const uint32_t bytes = (uint32_t)((m.ce - m.cs) * (int64_t)sizeof(S));
                mbar_arrive_tx(&full[s], bytes);
                tma_load_1d(bufs + (size_t)s * SLOT + (m.cs - m.t0), src + m.cs, bytes, &full[s]);
            } else {
                mbar_arrive(&full[s]);
            }
            if (m.tile == 0xFFFFFFFFu) break;
            if (!lookback_mode) producer_meta<TILE, V>(job, ctl, par, it + 1, claim, ntiles, nfront, e_lo, e_hi, m);
        }
        return;
    }

    // ================================ consumers ================================
    // job fields read once: the asm memory clobbers below would otherwise reload them
    const uint32_t c_offset_mode = job->offset_mode, c_vec_off = job->vec_off;
    unsigned long long *const c_cursor = job->seg_cursor;
    // Two-stage software pipeline over this CTA's tiles: phase A of tile i (classify,
    // scan, stage in place, reserve the output runs) runs before phase B of tile i-1
    // (write-out), so the reservation's round trip overlaps with the next tile's work.
    bool have_prev = false;
    int prev_slot = 0;
    uint64_t prev_sb = 0, prev_se = 0;
    unsigned long long prev_resv = 0ull;   // packed (ex_gt << 32 | ex_lt), thread 0
    uint32_t prev_total = 0;               // packed (tgt << 16 | tlt), thread 0
    for (uint32_t it = 0;; it++) {
        const int s = (int)(it % NBUF);
        if (!mbar_wait(&full[s], (it / NBUF) & 1u, wait_limit)) {
            if (tid == 0) set_status(ctl, TSQS_ETIMEOUT);
            mbar_wait(&full[s], (it / NBUF) & 1u, wait_limit);   // let any copy land
        }
        const TileMeta m = meta[s];
        const bool end = m.tile == 0xFFFFFFFFu;
        const bool work = !end && m.valid;
        S *buf = bufs + (size_t)s * SLOT;

        // ---- phase A, part 1: classify.  Thread t holds the 16-byte vectors
        // k * BLOCK + t of the tile (k < NV), i.e. elements (k * BLOCK + t) * V + j.
        S v[ITEMS];
        uint32_t ltm = 0, gtm = 0;
        if (work) {
            const int64_t sb = (int64_t)m.sb, se = (int64_t)m.se;
            const bool full_tile = m.t0 >= sb && m.t0 + TILE <= se && m.cs == m.t0 && m.ce == m.t0 + TILE;
            // tile-local bounds of the segment and of the bulk-copied range
            const int lo = (int)max((int64_t)0, sb - m.t0), hi = (int)min((int64_t)TILE, se - m.t0);
            const bool covered = m.cs - m.t0 <= lo && m.ce - m.t0 >= hi;
            auto classify = [&](auto dom, auto pd) {
            if (full_tile) {                             // interior tile: no bounds checks
#pragma unroll
                for (int k = 0; k < NV; k++) lds_vec<S, V>(buf + (k * BLOCK + tid) * V, &v[k * V]);
#pragma unroll
                for (int i = 0; i < ITEMS; i++) {
                    const auto d = dom(v[i]);
                    if (c_lt(d, pd)) ltm |= 1u << i;
                    if (c_lt(pd, d)) gtm |= 1u << i;
                }
            } else if (covered) {                        // segment ends inside the tile
                // range tests per 16-byte vector: a vector wholly outside [lo, hi) is
                // neither loaded nor classified (no bits; staging sends it to the dummy
                // slot), one wholly inside takes the unchecked compares, and only the
                // vectors holding lo or hi test every element
#pragma unroll
                for (int k = 0; k < NV; k++) {
                    const int vs = (k * BLOCK + tid) * V;
                    if (vs + V <= lo || vs >= hi) continue;
                    lds_vec<S, V>(buf + vs, &v[k * V]);
                    if (vs >= lo && vs + V <= hi) {
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            const auto d = dom(v[k * V + j]);
                            if (c_lt(d, pd)) ltm |= 1u << (k * V + j);
                            if (c_lt(pd, d)) gtm |= 1u << (k * V + j);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            const bool in = vs + j >= lo && vs + j < hi;
                            const auto d = dom(v[k * V + j]);
                            ltm |= (uint32_t)(in && c_lt(d, pd)) << (k * V + j);
                            gtm |= (uint32_t)(in && c_lt(pd, d)) << (k * V + j);
                        }
                    }
                }
            } else {                                     // the buffer's own ends
#pragma unroll
                for (int k = 0; k < NV; k++) {
#pragma unroll
                    for (int j = 0; j < V; j++) {
                        const int idx = (k * BLOCK + tid) * V + j;
                        const int64_t e = m.t0 + idx;
                        if (e >= sb && e < se) {
                            v[k * V + j] = (e >= m.cs && e < m.ce) ? buf[idx] : src[e];
                            const auto d = dom(v[k * V + j]);
                            ltm |= (uint32_t)c_lt(d, pd) << (k * V + j);
                            gtm |= (uint32_t)c_lt(pd, d) << (k * V + j);
                        }
                    }
                }
            }
            };
            if constexpr (kFloatKind<KIND>) {
                using SI = typename std::make_signed<S>::type;
                const S praw = K::uncanon(c_from<C>(m.piv_lo, m.piv_hi));
                if ((SI)praw >= 0) {
                    classify(RawDom<SI>{}, (SI)praw);
                } else {
                    classify(RawDom<S>{}, praw);
                    const uint32_t t = ltm;
                    ltm = gtm;
                    gtm = t;
                }
            } else {
                classify(CanonDom<K>{}, K::pdom(c_from<C>(m.piv_lo, m.piv_hi)));
            }
        }
        const uint32_t cnt = (uint32_t)__popc(ltm) | ((uint32_t)__popc(gtm) << 16);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        if (tid == 0 && have_prev) {                     // the previous tile's offsets
            misc[(it - 1) & 1u].ex_lt = prev_resv & 0xFFFFFFFFull;
            misc[(it - 1) & 1u].ex_gt = prev_resv >> 32;
            misc[(it - 1) & 1u].total = prev_total;
        }
        consumer_sync<BLOCK>();        // reads of buf done; wsum and misc[it-1] ready

        // ---- phase A, part 2: block offsets, reservation, staging
        unsigned long long resv = 0ull;
        uint32_t total = 0;
        if (work) {
            const uint32_t ws = lane < NW ? wsum[lane] : 0u;
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            total = __shfl_sync(0xffffffffu, wi, NW - 1);
            const uint32_t wex = __shfl_sync(0xffffffffu, wi - ws, warp);
            const uint32_t texcl = wex + inc - cnt;
            const uint64_t agg_lt = total & 0xFFFFu, agg_gt = total >> 16;
            // atomic mode: one 64-bit atomic on the segment's cursor reserves both runs
            // (#<p in the low word, #>p in the high word); its result is used one tile
            // later
            if (tid == 0 && c_offset_mode == 0u)
                resv = atomicAdd(c_cursor + m.si, (unsigned long long)((agg_gt << 32) | agg_lt));
            // stage without branches: <p from the front, >p from the back, =p (and
            // elements outside the segment) into the dummy slot at TILE
            // (32-bit shared-window addresses keep the address arithmetic to one add)
            const uint32_t b0 = smem_addr(buf), es = (uint32_t)sizeof(S);
            uint32_t la = b0 + (texcl & 0xFFFFu) * es;
            uint32_t ga = b0 + ((TILE - 1) - (texcl >> 16)) * es;
            const uint32_t da = b0 + (uint32_t)TILE * es;
            constexpr uint32_t kAll = ITEMS == 32 ? 0xFFFFFFFFu : ((1u << ITEMS) - 1u);
            if (ltm == kAll || gtm == kAll) {
                // all of this thread's keys go to one run (ordered input): write them
                // permuted by the lane inside the thread's own stretch of the run, so
                // that a warp's store covers 32 banks instead of one
                constexpr uint32_t kRot = (uint32_t)(ITEMS & -ITEMS) - 1u;   // keeps k ^ rot < ITEMS
                const uint32_t rot = (lane & kRot) * es;
                const uint32_t base = ltm == kAll ? la : ga;
                const int sgn = ltm == kAll ? 1 : -1;
#pragma unroll
                for (int k = 0; k < ITEMS; k++)
                    sts_raw(base + sgn * (int)(((uint32_t)k * es) ^ rot), v[k]);
            } else {
#pragma unroll
                for (int k = 0; k < ITEMS; k++) {
                    const bool l = (ltm >> k) & 1u, g = (gtm >> k) & 1u;
                    sts_raw(l ? la : (g ? ga : da), v[k]);
                    la += l ? es : 0u;
                    ga -= g ? es : 0u;
                }
            }
            if (warp == 0 && c_offset_mode != 0u) {
                // look-back mode: publish the aggregate, walk back, publish the inclusive
                uint64_t ex_lt = 0, ex_gt = 0;
                unsigned long long *stw = job->tile_status + m.tile;
                const bool publish = !((job->pad & 2u) && m.tile == 1u);   // test hook
                if (m.tl == 0) {
                    if (lane == 0 && publish) st_relaxed(stw, lb_pack(kFlagInc, agg_lt, agg_gt));
                } else {
                    if (lane == 0 && publish) st_relaxed(stw, lb_pack(kFlagAgg, agg_lt, agg_gt));
                    lookback(job->tile_status, m.tile, m.tile_begin, job->spin_limit, ctl, ex_lt, ex_gt);
                    if (lane == 0 && publish)
                        st_relaxed(stw, lb_pack(kFlagInc, ex_lt + agg_lt, ex_gt + agg_gt));
                }
                resv = (unsigned long long)((ex_gt << 32) | ex_lt);
            }
        }

        // ---- phase B of the previous tile: coalesced write-out of both runs
        if (have_prev) {
            const PartMisc &pm = misc[(it - 1) & 1u];
            const S *pbuf = bufs + (size_t)prev_slot * SLOT;
            const uint32_t tlt = pm.total & 0xFFFFu, tgt = pm.total >> 16;
            // <p run: staged [0, tlt) -> dst[sb + ex_lt, +tlt); >p run: staged
            // [TILE - tgt, TILE) -> dst[se - ex_gt - tgt, se - ex_gt), both ascending
            copy_run<S, V, BLOCK>(dst, prev_sb + pm.ex_lt, pbuf, tlt, c_vec_off);
            copy_run<S, V, BLOCK>(dst, prev_se - pm.ex_gt - tgt, pbuf + (TILE - tgt), tgt, c_vec_off);
        }
        fence_proxy_async();
        consumer_sync<BLOCK>();        // previous buffer fully read, this tile staged
        if (tid == 0) {
            if (have_prev) mbar_arrive(&empty[prev_slot]);
            if (!work && !end) mbar_arrive(&empty[s]);   // a skipped tile frees its slot now
        }
        if (end) break;
        have_prev = work;
        prev_slot = s;
        prev_sb = m.sb;
        prev_se = m.se;
        prev_resv = resv;
        prev_total = total;
    }
}

// ---------------------------------------------------------------------------------
// Leaf pass (persistent): on-chip sort of small segments and =p fills.
// One block (LB threads) per leaf item.  A segment of len <= 4096 elements is padded
// with the largest canonical key to P = max(32, 2^ceil(log2 len)); thread t owns the
// E consecutive elements [t E, t E + E), E = min(32, P / 32), so P / E threads work.
// The network is the bitonic sort in its "mirror" form: each merge of width k first
// compares element i with i ^ (k - 1), then runs half-cleaners i vs i ^ j
// (j = k/4 .. 1), and every comparator puts the minimum at the lower index, so all
// in-thread comparators have compile-time directions.  Strides below E stay inside a
// thread, strides below 32 E cross lanes through __shfl_xor_sync (with E = 32, a run of
// three to five such strides runs in registers between two warp-local transposes),
// larger strides go through shared memory (one pad word per 32 keeps the accesses
// conflict-free).  Items queue up across levels and run in as few passes as the queue
// capacity allows: normally one, after the level loop.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ unsigned int c_min(unsigned int a, unsigned int b) { return min(a, b); }
__device__ __forceinline__ unsigned int c_maxv(unsigned int a, unsigned int b) { return max(a, b); }
__device__ __forceinline__ unsigned long long c_min(unsigned long long a, unsigned long long b) { return min(a, b); }
__device__ __forceinline__ unsigned long long c_maxv(unsigned long long a, unsigned long long b) { return max(a, b); }
__device__ __forceinline__ U128 c_min(U128 a, U128 b) { return c_lt(b, a) ? b : a; }
__device__ __forceinline__ U128 c_maxv(U128 a, U128 b) { return c_lt(b, a) ? a : b; }
__device__ __forceinline__ unsigned int c_shfl_xor(unsigned int v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ unsigned long long c_shfl_xor(unsigned long long v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ U128 c_shfl_xor(U128 v, int m) {
    return U128{__shfl_xor_sync(0xffffffffu, v.lo, m), __shfl_xor_sync(0xffffffffu, v.hi, m)};
}

// One side of a comparator whose partner value w lives in another thread or in shared
// memory: the lower side keeps the minimum, the upper side the maximum.
template <class C>
__device__ __forceinline__ C cx_side(C v, C w, bool lower) {
    return (c_lt(w, v) == lower) ? w : v;
}

// min to the lower index, max to the upper
template <class C>
__device__ __forceinline__ void cx(C &lo, C &hi) {
    const C a = lo, b = hi;
    lo = c_min(a, b);
    hi = c_maxv(a, b);
}

// Padded shared-memory index of element i of a sort buffer of C: one pad element after
// every 128 bytes of elements (32 four-byte, 16 eight-byte or 8 sixteen-byte ones).  Shared
// memory serves a warp's 4-, 8- and 16-byte accesses in phases of 32, 16 and 8 lanes; lane
// t of a network stage touches element E t + r, so with one pad per 128 bytes the lanes of a
// phase fall in distinct bank groups.
template <class C> constexpr uint32_t kPadGroup = 128u / (uint32_t)sizeof(C);
template <class C>
__device__ __forceinline__ uint32_t padc(uint32_t i) { return i + i / kPadGroup<C>; }

// Sorts s[0, P) ascending; P a power of two with 32 E <= P <= E * blockDim.x, and
// s[len, P) holding the largest key.  Every thread of the block must call it (it
// contains block barriers).  In the mirror form the padding never moves: every
// comparator that touches it leaves both elements in place.  So a warp whose
// elements are all padding does no work, and its shared-memory slots keep the
// padding its partners read.
template <class C, int E>
__device__ __forceinline__ void bitonic_mirror(C *s, uint32_t P, uint32_t len) {
    const uint32_t t = threadIdx.x, lane = t & 31u;
    const uint32_t NT = P / E;
    const bool act = t < NT && (t & ~31u) * (uint32_t)E < len;
    C v[E];
    if (act) {
#pragma unroll
        for (int r = 0; r < E; r++) v[r] = s[padc<C>(t * E + r)];
        // merges of width k <= E: inside the thread
#pragma unroll
        for (int k = 2; k <= E; k <<= 1) {
#pragma unroll
            for (int r = 0; r < E; r++) {
                const int q = r ^ (k - 1);
                if (q > r) cx(v[r], v[q]);
            }
#pragma unroll
            for (int j = k >> 2; j >= 1; j >>= 1) {
#pragma unroll
                for (int r = 0; r < E; r++)
                    if ((r & j) == 0) cx(v[r], v[r | j]);
            }
        }
    }
    for (uint32_t k = 2 * E; k <= P; k <<= 1) {
        // ---- mirror stage: element i vs i ^ (k - 1)
        if (k <= 32u * E) {
            if (act) {                                   // partner lane t ^ (k/E - 1), register E-1-r
                const int lm = (int)(k / E - 1);
                const bool lower = (t & (k / (2 * E))) == 0u;
#pragma unroll
                for (int r = 0; r < (E + 1) / 2; r++) {
                    const C wa = c_shfl_xor(v[E - 1 - r], lm);
                    if (r != E - 1 - r) {
                        const C wb = c_shfl_xor(v[r], lm);
                        v[E - 1 - r] = cx_side(v[E - 1 - r], wb, lower);
                    }
                    v[r] = cx_side(v[r], wa, lower);
                }
            }
        } else {                                         // across warps: shared memory
            __syncthreads();
            if (act) {
#pragma unroll
                for (int r = 0; r < E; r++) s[padc<C>(t * E + r)] = v[r];
            }
            __syncthreads();
            if (act) {
                const bool lower = ((t * E) & (k >> 1)) == 0u;
#pragma unroll
                for (int r = 0; r < E; r++) {
                    const C w = s[padc<C>((t * E + r) ^ (k - 1))];
                    v[r] = cx_side(v[r], w, lower);
                }
            }
        }
        // ---- half-cleaners across warps
        for (uint32_t j = k >> 2; j >= 32u * E; j >>= 1) {
            __syncthreads();
            if (act) {
#pragma unroll
                for (int r = 0; r < E; r++) s[padc<C>(t * E + r)] = v[r];
            }
            __syncthreads();
            if (act) {
                const bool lower = ((t * E) & j) == 0u;
#pragma unroll
                for (int r = 0; r < E; r++) {
                    const C w = s[padc<C>((t * E + r) ^ j)];
                    v[r] = cx_side(v[r], w, lower);
                }
            }
        }
        // the transposed lane stages below reuse this warp's stretch of the buffer,
        // which other warps read in a shared-memory stage just above
        if constexpr (E == 32) if (k > 32u * E) __syncthreads();
        if (act) {
            // ---- half-cleaners across lanes
            uint32_t jl = min(k >> 2, 16u * E);
            if constexpr (E == 32) if (jl >= 4u * E) {
                // Three to five lane strides in a row: transpose the warp's 32 x 32 block
                // (lane <-> register) through its own stretch of the padded buffer, run the
                // strides as in-register comparators, transpose back.  In the padded
                // layout element (lane l, register r) of warp w sits at w*1056 + l*33 + r,
                // so both directions are free of bank conflicts.  Lane l writes and later
                // reads row l, and in between reads and writes column l, so the two
                // __syncwarp calls order every cross-lane access.
                C *wb = s + (t >> 5) * (32u * 33u);
#pragma unroll
                for (int r = 0; r < E; r++) wb[lane * 33u + r] = v[r];
                __syncwarp();
#pragma unroll
                for (int r = 0; r < E; r++) v[r] = wb[r * 33u + lane];
#pragma unroll
                for (int rs = 16; rs >= 1; rs >>= 1) {
                    if ((uint32_t)rs * (uint32_t)E <= jl) {
#pragma unroll
                        for (int r = 0; r < E; r++)
                            if ((r & rs) == 0) cx(v[r], v[r | rs]);
                    }
                }
#pragma unroll
                for (int r = 0; r < E; r++) wb[r * 33u + lane] = v[r];
                __syncwarp();
#pragma unroll
                for (int r = 0; r < E; r++) v[r] = wb[lane * 33u + r];
                jl = 0;                                  // lane strides done
            }
            for (uint32_t j = jl; j >= (uint32_t)E; j >>= 1) {
                const int lm = (int)(j / E);
                const bool lower = (lane & (uint32_t)lm) == 0u;
#pragma unroll
                for (int r = 0; r < E; r++) {
                    const C w = c_shfl_xor(v[r], lm);
                    v[r] = cx_side(v[r], w, lower);
                }
            }
            // ---- half-cleaners inside the thread
#pragma unroll
            for (int j = E >> 1; j >= 1; j >>= 1) {
#pragma unroll
                for (int r = 0; r < E; r++)
                    if ((r & j) == 0) cx(v[r], v[r | j]);
            }
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int r = 0; r < E; r++) s[padc<C>(t * E + r)] = v[r];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// Items of 513 .. 4096 elements: 32 keys per thread, P = 1024, 2048 or 4096.  Lane l of
// warp w holds v[r] = element w*1024 + l*32 + r ("rows").  The network is bitonic: each
// merge of width k = 2^K takes two sorted halves and compares i with i ^ (k - 1), then
// runs the half-cleaners k/4 .. 1, with the minimum to the lower index (the mirror form,
// as in bitonic_mirror).  Every compare-exchange is between two registers of one thread:
//   - strides 16 .. 1 in rows;
//   - for k <= 1024, the mirror stage and strides k/4 .. 32 in "columns" (lane l' holds
//     in register q element q*32 + l'), reached by a warp-local transpose through the
//     warp's 32 x 33 region of the block buffer (element (a, b) at w*1056 + a*33 + b:
//     both directions touch 32 distinct banks) that writes the upper half of each k-block
//     reversed (its lanes store row l ^ (k/64 - 1), column 31 - r): the mirror stage is
//     then the half-cleaner of stride k/2, a register pair as well;
//   - for k = 2048 and 4096 the mirror stage (and the stride 1024) cross warps: each
//     thread reads its element and the partner's from the block buffer and keeps its
//     side, then strides 512 .. 32 run in columns.
// One copy of the code serves every merge width (a loop over K), so the kernel's
// instructions stay in the instruction cache.  Warps holding only padding (the largest
// key) skip the network: the padding sits at the top and never moves, and reads of their
// regions take the largest key instead.
// ---------------------------------------------------------------------------------

template <class C>
__device__ __forceinline__ void rows_cleaners(C (&v)[32]) {
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
#pragma unroll
        for (int r = 0; r < 32; r++)
            if ((r & j) == 0) cx(v[r], v[r | j]);
    }
}

// Sorts the item held in rows by warps 0 .. P/1024 - 1 (warps nact and above hold only
// padding); s is the block buffer (32 x 33 elements per warp).  Every thread of the
// block calls it (block barriers when P > 1024).  Leaves the sorted item in rows.
template <class C>
__device__ __forceinline__ void sort_item32(C (&v)[32], C *s, uint32_t P, uint32_t nact) {
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const bool act = w < nact;
    C *wb = s + w * 1056u;
    if (act) {                                   // merges of width 2 .. 32 in registers
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int r = 0; r < 32; r++) {
                const int q = r ^ (k - 1);
                if (q > r) cx(v[r], v[q]);
            }
#pragma unroll
            for (int j = k >> 2; j >= 1; j >>= 1) {
#pragma unroll
                for (int r = 0; r < 32; r++)
                    if ((r & j) == 0) cx(v[r], v[r | j]);
            }
        }
    }
#pragma unroll 1
    for (uint32_t K = 6; (1u << K) <= P; K++) {
        uint32_t lim;                            // largest column stride left, in rows
        if (K <= 10u) {
            lim = 1u << (K - 6);
            if (act) {
                __syncwarp();                    // every lane has read its row
                if (lane & lim) {                // upper half: reversed
                    C *b = wb + (lane ^ (lim - 1u)) * 33u + 31u;
#pragma unroll
                    for (int r = 0; r < 32; r++) b[-r] = v[r];
                } else {
                    C *b = wb + lane * 33u;
#pragma unroll
                    for (int r = 0; r < 32; r++) b[r] = v[r];
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 32; q++) v[q] = wb[q * 33u + lane];
            }
        } else {
            // k = 2048 or 4096: the mirror stage i vs i ^ (k - 1) reads the partner from
            // warp w ^ (k/1024 - 1) with row and column reversed (no data moves, so the
            // regions of padding warps keep meaning the largest key); this thread keeps
            // the side of its element in columns
            lim = 16u;
            __syncthreads();                                 // all reads of the buffer done
            if (act) {
#pragma unroll
                for (int r = 0; r < 32; r++) wb[lane * 33u + r] = v[r];
            }
            __syncthreads();
            if (act) {
                const uint32_t half = 1u << (K - 11);        // warp bit of the upper half
                const uint32_t pw = w ^ (2u * half - 1u);
                const bool lower = (w & half) == 0u, pact = pw < nact;
                const C *pb = s + pw * 1056u + (31u - lane);
#pragma unroll
                for (int q = 0; q < 32; q++) {
                    const C part = pact ? pb[(31 - q) * 33] : c_max<C>();
                    v[q] = cx_side(wb[q * 33u + lane], part, lower);
                    if ((q & 7) == 7) asm volatile("" ::: "memory");   // loads in groups of 8
                }
            }
            if (K == 12u) {                                  // stride 1024: warp w ^ 1
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int q = 0; q < 32; q++) wb[q * 33u + lane] = v[q];
                }
                __syncthreads();
                if (act) {
                    const uint32_t pw = w ^ 1u;
                    const bool lower = (w & 1u) == 0u, pact = pw < nact;
                    const C *pb = s + pw * 1056u + lane;
#pragma unroll
                    for (int q = 0; q < 32; q++) {
                        const C part = pact ? pb[q * 33] : c_max<C>();
                        v[q] = cx_side(v[q], part, lower);
                        if ((q & 7) == 7) asm volatile("" ::: "memory");
                    }
                }
            }
            __syncthreads();                                 // partner reads done
        }
        if (act) {
            // column strides lim*32 .. 32 in registers
#pragma unroll
            for (int js = 16; js >= 1; js >>= 1) {
                if ((uint32_t)js <= lim) {
#pragma unroll
                    for (int q = 0; q < 32; q++)
                        if ((q & js) == 0) cx(v[q], v[q | js]);
                }
            }
            // columns -> rows (each lane rewrites the words it read), strides 16 .. 1
#pragma unroll
            for (int q = 0; q < 32; q++) wb[q * 33u + lane] = v[q];
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 32; r++) v[r] = wb[lane * 33u + r];
            rows_cleaners(v);
        }
    }
}

// ---------------------------------------------------------------------------------
// Records (16-byte {key, payload}, ordered by (key, payload)) in the leaf pass.  A
// 128-bit compare-exchange costs about three times a 64-bit one, so an item is sorted by
// 64-bit packed keys: ((key - min key) >> sh) << 12 | index in the item, sh the bits the
// item's key range has beyond 52.  The packed order is the record order except among
// records whose shifted keys are equal (equal keys, or keys that differ only in the sh
// dropped bits): such runs are then put in (key, payload) order from the records
// themselves.  Runs are short on ordinary inputs; an item with a run longer than 32
// is sorted once more by an indirect network that compares whole records.
// ---------------------------------------------------------------------------------

constexpr unsigned long long kPackNone = ~0ull;            // padding: above every packed key

__device__ __forceinline__ U128 rec_canon(const Rec16 &r) { return U128{r.pay, r.key}; }

// Indirect bitonic sort of the packed entries s[0, P) (padded layout) by the records they
// index, src[base + (x & 0xFFF)]; padding entries (index >= len) sort last.  Every thread
// of the block calls it.
template <int LB>
__device__ void rec_sort_indirect(unsigned long long *s, uint32_t P, uint32_t len, const Rec16 *src,
                                  uint64_t base) {
    using C64 = unsigned long long;
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j >= 1; j >>= 1) {
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < P; i += LB) {
                const uint32_t q = i ^ j;
                if (q <= i) continue;
                const C64 a = s[padc<C64>(i)], b = s[padc<C64>(q)];
                const uint32_t ia = (uint32_t)(a & 0xFFFu), ib = (uint32_t)(b & 0xFFFu);
                bool gt;                                     // record(a) > record(b)
                if (ia >= len || ib >= len) gt = ia >= len && ib < len;
                else gt = c_lt(rec_canon(src[base + ib]), rec_canon(src[base + ia]));
                const bool up = (i & k) == 0u;
                if (gt == up) {
                    s[padc<C64>(i)] = b;
                    s[padc<C64>(q)] = a;
                }
            }
        }
    }
    __syncthreads();
}

// Shared-memory layout of the leaf kernel: the padded sort buffer, then the raw
// prefetch slot (the next item's 16-byte-aligned hull) and its mbarrier.
template <int KIND>
struct LeafLayout {
    using S = typename Key<KIND>::S;
    // the sort buffer holds the canonical keys, for records the packed 64-bit sort keys
    using C = typename std::conditional<KIND == TSQS_U64_U64_REC, unsigned long long,
                                        typename Key<KIND>::C>::type;
    static constexpr int PRE = kMaxSmall + 2 * Key<KIND>::V;          // elements per slot
    static constexpr size_t sort_bytes = ((kMaxSmall + kMaxSmall / kPadGroup<C>) * sizeof(C) + 127) / 128 * 128;
    static constexpr size_t off_pre = sort_bytes;
    // one prefetch slot: an item's keys leave it for the sort buffer before the next
    // item's bulk copy is issued into it, so a second slot would only cost occupancy
    static constexpr int NSLOT = 1;
    static constexpr size_t off_bar = off_pre + NSLOT * (size_t)PRE * sizeof(S);
    static constexpr size_t bytes = off_bar + NSLOT * sizeof(unsigned long long);
};

template <int KIND, int LB, int MAXE, int MINB>
__global__ void __launch_bounds__(LB, MINB) k_leaf(const Job *__restrict__ job, Ctl *ctl, int final_pass) {
    using K = Key<KIND>;
    using S = typename K::S;
    using C = typename K::C;
    using LY = LeafLayout<KIND>;
    constexpr int V = K::V;
    static_assert(LB * MAXE >= kMaxSmall, "block too small for the largest leaf");
    extern __shared__ __align__(128) unsigned char leaf_raw[];
    C *s = reinterpret_cast<C *>(leaf_raw);
    unsigned long long *sp64 = reinterpret_cast<unsigned long long *>(leaf_raw);   // records
    __shared__ unsigned long long s_kmin[LB / 32], s_kmax[LB / 32];
    __shared__ uint32_t s_sh;
    S *pre = reinterpret_cast<S *>(leaf_raw + LY::off_pre);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(leaf_raw + LY::off_bar);
    if (block_aborted(ctl)) return;                         // queues may be inconsistent
    // Leaf items queue up across levels (their ranges are never touched by a later
    // partition); a level's pass runs only when the queue would otherwise outgrow its
    // capacity, and one final pass after the level loop runs the rest.  nleaf does not
    // change while this kernel runs, so every block takes the same decision.
    const uint32_t nl = min(ctl->nleaf, job->cap_leaves);
    if (!final_pass && nl <= job->leaf_defer) return;
    S *out = reinterpret_cast<S *>(job->out);
    const uint32_t wait_limit = 1u << 20;
    // per-block totals, kept by thread 0 in shared memory (registers stay free for keys)
    __shared__ unsigned long long s_sorted, s_filled, s_items;
    // Claimed items, two deep: the item being sorted and the next one, whose hull is
    // copied into the prefetch slot as soon as the current keys have left it.  Claiming
    // (the queue read and the hull arithmetic) happens after an item is written out, when
    // no keys are held in registers; issuing the copy takes a few words from here.
    struct Meta { LeafItem it; int64_t cs, ce; const S *from; uint32_t bytes, ok; };
    __shared__ Meta s_meta[2];

    // thread 0: claim the next item into s_meta[m] (no copy yet)
    auto prepare = [&](int m) {
        Meta &d = s_meta[m];
        const uint32_t ii = atomicAdd(&ctl->leaf_claim, 1u);
        d.ok = ii < nl ? 1u : 0u;
        d.cs = d.ce = 0;
        d.bytes = 0;
        if (!d.ok) return;
        const LeafItem it = job->leaves[ii];
        d.it = it;
        if ((it.kind & 0xFFu) == LEAF_SORT && it.len <= (uint32_t)kMaxSmall) {
            const int64_t n = (int64_t)job->n;
            const int64_t e_lo = (int64_t)((V - (int64_t)job->vec_off % V) % V);
            const int64_t e_hi = n - ((n + (int64_t)job->vec_off) % V);
            const S *src = buffer<K>(job, (it.kind & kLeafInAlt) ? 1 : 0);
            const int64_t b = (int64_t)it.begin, e = b + it.len;
            const int64_t cs = max(b - ((b + (int64_t)job->vec_off) % V), e_lo);
            const int64_t ce = min(e + ((V - ((e + (int64_t)job->vec_off) % V)) % V), e_hi);
            if (ce > cs) {
                d.cs = cs;
                d.ce = ce;
                d.from = src + cs;
                d.bytes = (uint32_t)((ce - cs) * (int64_t)sizeof(S));
            }
        }
    };
    // thread 0: start the bulk copy of s_meta[m]'s hull into the prefetch slot
    auto issue = [&](int m) {
        const uint32_t bytes = s_meta[m].bytes;
        if (s_meta[m].ok && bytes) {
            mbar_arrive_tx(&bar[0], bytes);
            tma_load_1d(pre, s_meta[m].from, bytes, &bar[0]);
        }
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        fence_mbar_init();
        s_sorted = s_filled = s_items = 0ull;
        prepare(0);
        issue(0);
        prepare(1);
    }
    __syncthreads();
    uint32_t phase = 0;
    for (uint32_t iter = 0;; iter++) {
        const int cur = (int)(iter & 1u);
        if (!s_meta[cur].ok) break;
        const LeafItem it = s_meta[cur].it;
        const int64_t cs = s_meta[cur].cs, ce = s_meta[cur].ce;
        if (threadIdx.x == 0) s_items++;
        const bool is_fill = (it.kind & 0xFFu) == LEAF_FILL;
        const bool is_sort = !is_fill && it.len <= (uint32_t)kMaxSmall;
        const S *src = buffer<K>(job, (it.kind & kLeafInAlt) ? 1 : 0);   // may equal out
        uint32_t P = 32;
        // items above 512 elements: 32 keys per thread in registers (sort_item32)
        const bool wide = MAXE == 32 && is_sort && it.len > 512u;
        const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
        C v[32];
        if (is_sort) {
            if (ce > cs) {
                if (!mbar_wait(&bar[0], phase, wait_limit)) {
                    if (threadIdx.x == 0) set_status(ctl, TSQS_ETIMEOUT);
                    mbar_wait(&bar[0], phase, wait_limit);        // let the copy land
                }
                phase ^= 1u;
            }
            const S *slot = pre;
            while (P < it.len) P <<= 1;
            if constexpr (KIND == TSQS_U64_U64_REC) {
                // packed keys: the item's key range first (block min / max), then
                // ((key - min) >> sh) << 12 | index, padding above every packed key
                constexpr int RQ = (kMaxSmall + LB - 1) / LB;
                unsigned long long kv[RQ];
                unsigned long long lo = ~0ull, hi = 0ull;
                const int64_t b = (int64_t)it.begin;
#pragma unroll
                for (int q = 0; q < RQ; q++) {
                    const uint32_t i = threadIdx.x + (uint32_t)(q * LB);
                    kv[q] = 0ull;
                    if (i < it.len) {
                        const int64_t e = b + i;
                        kv[q] = ((e >= cs && e < ce) ? slot[e - cs] : src[e]).key;
                        lo = min(lo, kv[q]);
                        hi = max(hi, kv[q]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, (unsigned long long)__shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, (unsigned long long)__shfl_xor_sync(0xffffffffu, hi, o));
                }
                if ((threadIdx.x & 31u) == 0u) { s_kmin[threadIdx.x >> 5] = lo; s_kmax[threadIdx.x >> 5] = hi; }
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int q = 1; q < LB / 32; q++) { lo = min(lo, s_kmin[q]); hi = max(hi, s_kmax[q]); }
                    const unsigned long long range = hi - lo;
                    const uint32_t bits = range ? 64u - (uint32_t)__clzll((long long)range) : 0u;
                    s_sh = bits > 52u ? bits - 52u : 0u;
                    s_kmin[0] = lo;
                }
                __syncthreads();
                const unsigned long long kmin = s_kmin[0];
                const uint32_t sh = s_sh;
#pragma unroll
                for (int q = 0; q < RQ; q++) {
                    const uint32_t i = threadIdx.x + (uint32_t)(q * LB);
                    if (i < P)
                        sp64[padc<unsigned long long>(i)] =
                            i < it.len ? (((kv[q] - kmin) >> sh) << 12) | i : kPackNone;
                }
            } else if (wide) {
                // straight from the prefetch slot into registers: lane l of warp w takes
                // elements w*1024 + q*32 + l (the input order does not matter to the
                // network, so they serve as its rows); padding is the largest key
                if (w * 1024u < it.len) {
                    const int64_t b = (int64_t)it.begin;
                    const uint32_t i0 = w * 1024u + lane;
                    if (cs <= b && b + (int64_t)it.len <= ce && (w + 1u) * 1024u <= it.len) {
                        const S *sp = slot + (b - cs) + i0;
#pragma unroll
                        for (int q = 0; q < 32; q++) v[q] = K::canon(sp[q * 32]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; q++) {
                            const uint32_t i = i0 + 32u * q;
                            C c = c_max<C>();
                            if (i < it.len) {
                                const int64_t e = b + i;
                                c = K::canon((e >= cs && e < ce) ? slot[e - cs] : src[e]);
                            }
                            v[q] = c;
                        }
                    }
                }
            } else if constexpr (KIND != TSQS_U64_U64_REC) {
#pragma unroll 4
                for (uint32_t i = threadIdx.x; i < P; i += LB) {
                    C c = c_max<C>();
                    if (i < it.len) {
                        const int64_t e = (int64_t)it.begin + i;
                        c = K::canon((e >= cs && e < ce) ? slot[e - cs] : src[e]);
                    }
                    s[padc<C>(i)] = c;
                }
            }
        }
        // records keep the slot until they are written out (the output is gathered from
        // it); every other item has left it
        const bool hold_slot = KIND == TSQS_U64_U64_REC && is_sort;
        fence_proxy_async();                // this slot's reads precede its next bulk copy
        __syncthreads();                    // keys loaded, slot free, s_meta[cur] read
        if (threadIdx.x == 0 && !hold_slot) issue(cur ^ 1);   // prefetch the next item meanwhile
        if (is_fill) {
            const S val = K::uncanon(c_from<C>(it.v_lo, it.v_hi));
            S rep[V];
#pragma unroll
            for (int j = 0; j < V; j++) rep[j] = val;
            const uint64_t x = it.begin;
            uint32_t head = (uint32_t)((V - ((x + job->vec_off) % V)) % V);
            if (head > it.len) head = it.len;
            const uint32_t nvec = (it.len - head) / V, body_end = head + nvec * V;
            if (threadIdx.x < head) out[x + threadIdx.x] = val;
            for (uint32_t q = threadIdx.x; q < nvec; q += LB) stg_vec<S, V>(out + x + head + q * V, rep);
            for (uint32_t i = body_end + threadIdx.x; i < it.len; i += LB) out[x + i] = val;
            if (threadIdx.x == 0) s_filled += it.len;
        } else if (!is_sort) {
            if (threadIdx.x == 0) set_status(ctl, TSQS_EINTERNAL);
        } else if constexpr (KIND == TSQS_U64_U64_REC) {
            using C64 = unsigned long long;
            // the item's records, in the prefetch slot (16-byte elements: the hull is the
            // item itself)
            const Rec16 *rsrc = reinterpret_cast<const Rec16 *>(pre) - cs;
            const uint32_t E = min((uint32_t)MAXE, P / 32u);
            if (E == 1) bitonic_mirror<C64, 1>(sp64, P, it.len);
            else if (E == 2) bitonic_mirror<C64, 2>(sp64, P, it.len);
            else if (E == 4) bitonic_mirror<C64, 4>(sp64, P, it.len);
            else if (E == 8) bitonic_mirror<C64, (MAXE >= 8 ? 8 : 1)>(sp64, P, it.len);
            else bitonic_mirror<C64, (MAXE >= 16 ? 16 : 1)>(sp64, P, it.len);
            // runs of equal shifted keys: a run longer than 32 sends the item to the
            // indirect network; shorter ones are put in record order by their first thread
            bool longrun = false;
            for (uint32_t j = threadIdx.x; j + 32u < it.len; j += LB)
                longrun |= (sp64[padc<C64>(j)] >> 12) == (sp64[padc<C64>(j + 32u)] >> 12);
            if (__syncthreads_or(longrun)) {
                rec_sort_indirect<LB>(sp64, P, it.len, rsrc, it.begin);
            } else {
                for (uint32_t j = threadIdx.x; j + 1u < it.len; j += LB) {
                    const C64 h = sp64[padc<C64>(j)] >> 12;
                    if ((j > 0u && (sp64[padc<C64>(j - 1u)] >> 12) == h) ||
                        (sp64[padc<C64>(j + 1u)] >> 12) != h) continue;
                    uint32_t e = j + 1u;                         // run [j, e)
                    while (e < it.len && (sp64[padc<C64>(e)] >> 12) == h) e++;
                    for (uint32_t a = j + 1u; a < e; a++) {      // insertion by (key, payload)
                        const C64 x = sp64[padc<C64>(a)];
                        const U128 xv = rec_canon(rsrc[it.begin + (x & 0xFFFu)]);
                        uint32_t c = a;
                        while (c > j) {
                            const C64 y = sp64[padc<C64>(c - 1u)];
                            if (!c_lt(xv, rec_canon(rsrc[it.begin + (y & 0xFFFu)]))) break;
                            sp64[padc<C64>(c)] = y;
                            c--;
                        }
                        sp64[padc<C64>(c)] = x;
                    }
                }
                __syncthreads();
            }
            // write out in order, gathered from the slot (a copy: the output may be the
            // records' own buffer), then release the slot to the next item's copy
            Rec16 *rout = reinterpret_cast<Rec16 *>(out);
            for (uint32_t j = threadIdx.x; j < it.len; j += LB)
                rout[it.begin + j] = rsrc[it.begin + (sp64[padc<C64>(j)] & 0xFFFu)];
            if (threadIdx.x == 0) s_sorted += it.len;
            fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) issue(cur ^ 1);
        } else if (wide) {
            const uint32_t nact = (it.len + 1023u) / 1024u;
            sort_item32<C>(v, s, P, nact);
            // rows -> columns through the warp's region, then stores of 32 consecutive
            // elements per warp instruction
            if (w < nact) {
                C *wb = s + w * 1056u;
#pragma unroll
                for (int r = 0; r < 32; r++) wb[lane * 33u + r] = v[r];
                __syncwarp();
                S *op = out + it.begin + w * 1024u + lane;
                if ((w + 1u) * 1024u <= it.len) {
#pragma unroll
                    for (int q = 0; q < 32; q++) op[q * 32] = K::uncanon(wb[q * 33u + lane]);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; q++)
                        if (w * 1024u + 32u * q + lane < it.len) op[q * 32] = K::uncanon(wb[q * 33u + lane]);
                }
            }
            if (threadIdx.x == 0) s_sorted += it.len;
        } else {
            // E = min(MAXE, P / 32) keys per thread; with the 32-key path for items
            // above 512, at most 8 here (two warps for P = 512)
            constexpr uint32_t EMAX = MAXE == 32 ? 8u : (uint32_t)MAXE;
            const uint32_t E = min(EMAX, P / 32u);
            if (E == 1) bitonic_mirror<C, 1>(s, P, it.len);
            else if (E == 2) bitonic_mirror<C, 2>(s, P, it.len);
            else if (E == 4) bitonic_mirror<C, 4>(s, P, it.len);
            else if (E == 8) bitonic_mirror<C, (EMAX >= 8 ? 8 : 1)>(s, P, it.len);
            else if (E == 16) bitonic_mirror<C, (EMAX >= 16 ? 16 : 1)>(s, P, it.len);
            else bitonic_mirror<C, (EMAX >= 32 ? 32 : 1)>(s, P, it.len);
            for (uint32_t i = threadIdx.x; i < it.len; i += LB) out[it.begin + i] = K::uncanon(s[padc<C>(i)]);
            if (threadIdx.x == 0) s_sorted += it.len;
        }
        if (threadIdx.x == 0) prepare(cur);              // the item after the next one
        __syncthreads();                    // sort buffer free, next item's meta visible
    }
    if (threadIdx.x == 0 && s_items) {
        atomicAdd((unsigned long long *)&ctl->leaf_sorted, s_sorted);
        atomicAdd((unsigned long long *)&ctl->leaf_filled, s_filled);
        atomicAdd((unsigned long long *)&ctl->leaf_items, s_items);
    }
    // the last block to finish empties the queue (every block has read nleaf and made
    // its last claim by then)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->leaf_blocks, 1u) + 1u == gridDim.x) {
            ctl->nleaf = 0u;
            ctl->leaf_claim = 0u;
            ctl->leaf_blocks = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------
// Step-level test hooks
// ---------------------------------------------------------------------------------

// Frontier[0] <- the given segments with the given pivots (original representation).
template <int KIND>
__global__ void k_dbg_setup_partition(const Job *__restrict__ job, Ctl *ctl) {
    using K = Key<KIND>;
    const typename K::S *piv = reinterpret_cast<const typename K::S *>(job->dbg_pivots);
    for (uint64_t s = blockIdx.x; s < job->nseg; s += gridDim.x) {
        __shared__ uint32_t s_tb, s_nt;
        const uint64_t b = job->seg_offsets[s], e = job->seg_offsets[s + 1];
        const int64_t s0 = tile_origin<K::V>(b, job->vec_off);
        if (threadIdx.x == 0) {
            s_nt = e > b ? tiles_for(e, s0, (int)job->tile) : 0u;
            s_tb = atomicAdd(&ctl->ntiles[0], s_nt);
            SegDesc d;
            d.begin = b; d.end = e; d.s0 = s0; d.tile_begin = s_tb; d.ntiles = s_nt;
            c_words(K::canon(piv[s]), d.piv_lo, d.piv_hi);
            job->front[0][s] = d;
            job->seg_done[s] = 0u;
            job->seg_cursor[s] = 0ull;
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

// ---------------------------------------------------------------------------------
// Depth guard (the worst-case mitigation of Section V.B-C: seeded sample jitter plus a
// bounded depth, after which the segment goes to a sorter whose cost does not depend on
// the pivots -- the introsort idea the paper cites).  A segment that would be
// partitioned at deep_level or later is sorted in place, in the buffer that holds it,
// by a bitonic network in mirror form over its length padded to a power of two; the
// padding is virtual (+infinity, which never moves in mirror form), so only the real
// elements are stored.  Every 4096-element tile is first sorted on chip; each larger
// merge then takes one global pass per stride >= 4096 and one on-chip pass for the
// strides below 4096.  O(n log^2 n) whatever the input.
// ---------------------------------------------------------------------------------

constexpr int kDeepTile = 4096;
constexpr uint32_t kDeepChunk = 2048;    // pairs per block step of a global stage
constexpr int kDeepThreads = 512;

__device__ __forceinline__ uint32_t deep_log2(uint64_t m) {
    uint32_t l = 0;
    while ((1ull << l) < m) l++;
    return l;
}

// Deep segment holding prefix entry x of `pre` (pre has nd + 1 entries), by binary search.
__device__ __forceinline__ uint32_t deep_find(const uint32_t *pre, uint32_t nd, uint32_t x) {
    uint32_t lo = 0, hi = nd;                 // pre[lo] <= x < pre[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// One block: prefix sums of the deep segments' tiles and global-stage pair chunks, and
// the first stage.  Returns (thread 0) whether any global stage follows.
__device__ __forceinline__ uint32_t deep_prep_body(const Job *__restrict__ job, Ctl *ctl) {
    __shared__ uint32_t s_t[kDeepThreads], s_c[kDeepThreads], s_l[kDeepThreads];
    uint32_t cont = 0;
    const uint32_t nd = min(ctl->ndeep, job->cap_deep);
    const uint32_t t = threadIdx.x, per = (nd + blockDim.x - 1) / blockDim.x;
    const uint32_t a = min(nd, t * per), b = min(nd, a + per);
    uint32_t st = 0, sc = 0, ml = 0;
    for (uint32_t s = a; s < b; s++) {
        const uint64_t len = job->deep[s].len;
        const uint32_t lg = deep_log2(len);
        st += (uint32_t)((len + kDeepTile - 1) / kDeepTile);
        sc += (uint32_t)(((1ull << lg) / 2 + kDeepChunk - 1) / kDeepChunk);
        ml = max(ml, lg);
    }
    s_t[t] = st; s_c[t] = sc; s_l[t] = ml;
    __syncthreads();
    if (t == 0) {                                          // exclusive scan over threads
        uint32_t at = 0, ac = 0, al = 0;
        for (uint32_t k = 0; k < blockDim.x; k++) {
            const uint32_t x = s_t[k], y = s_c[k];
            s_t[k] = at; s_c[k] = ac;
            at += x; ac += y; al = max(al, s_l[k]);
        }
        job->deep_tiles[nd] = at;
        job->deep_chunks[nd] = ac;
        ctl->deep_maxlog = al;
        ctl->deep_kk = 13u;                                // first merge above one tile
        ctl->deep_jj = 12u;                                // its mirror stage (stride 2^12)
        ctl->deep_blocks = 0u;
        cont = (nd > 0u && al >= 13u && ctl->status == 0u) ? 1u : 0u;
        ctl->deep_cont = cont;
    }
    __syncthreads();
    uint32_t at = s_t[t], ac = s_c[t];
    for (uint32_t s = a; s < b; s++) {
        const uint64_t len = job->deep[s].len;
        job->deep_tiles[s] = at;
        job->deep_chunks[s] = ac;
        at += (uint32_t)((len + kDeepTile - 1) / kDeepTile);
        ac += (uint32_t)(((1ull << deep_log2(len)) / 2 + kDeepChunk - 1) / kDeepChunk);
    }
    return cont;
}

template <int KIND>
__global__ void k_deep_prep(const Job *__restrict__ job, Ctl *ctl, cudaGraphConditionalHandle h,
                            int use_handle) {
    const uint32_t cont = deep_prep_body(job, ctl);
    if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(h, cont);
}

// Shared-memory bitonic steps on one 4096-element tile (padded layout, +inf beyond cnt):
// merges of width 2 .. kk_hi in full (kk_hi = 4096) or only the half-cleaners of
// strides 2048 .. 1 (full = false).
template <class C>
__device__ __forceinline__ void deep_tile_network(C *sm, bool full) {
    const uint32_t t = threadIdx.x;
    for (uint32_t k = full ? 2u : (uint32_t)kDeepTile * 2u; k <= (uint32_t)kDeepTile * 2u; k <<= 1) {
        if (full && k <= (uint32_t)kDeepTile) {
            for (uint32_t q = t; q < (uint32_t)kDeepTile / 2; q += blockDim.x) {    // mirror
                const uint32_t half = k >> 1, i = (q / half) * k + (q % half), p = i ^ (k - 1u);
                cx(sm[padc<C>(i)], sm[padc<C>(p)]);
            }
            __syncthreads();
        }
        const uint32_t jtop = (full && k <= (uint32_t)kDeepTile) ? k >> 2 : (uint32_t)kDeepTile / 2;
        for (uint32_t j = jtop; j >= 1u; j >>= 1) {
            for (uint32_t q = t; q < (uint32_t)kDeepTile / 2; q += blockDim.x) {
                const uint32_t i = (q / j) * 2u * j + (q % j);
                cx(sm[padc<C>(i)], sm[padc<C>(i + j)]);
            }
            __syncthreads();
        }
        if (!full || k == (uint32_t)kDeepTile) break;
    }
}

// Loads tile ti of deep segment `it` into sm (canonical keys, +inf padding), runs the
// network, stores the real elements back.
template <int KIND>
__device__ __forceinline__ void deep_tile(const Job *job, const LeafItem &it, uint32_t ti,
                                          typename Key<KIND>::C *sm, bool full) {
    using K = Key<KIND>;
    typename K::S *buf = buffer<K>(job, (it.kind & kLeafInAlt) ? 1 : 0) + it.begin;
    const uint64_t base = (uint64_t)ti * kDeepTile;
    const uint32_t cnt = (uint32_t)min((uint64_t)kDeepTile, (uint64_t)it.len - base);
    for (uint32_t i = threadIdx.x; i < (uint32_t)kDeepTile; i += blockDim.x)
        sm[padc<typename K::C>(i)] = i < cnt ? K::canon(buf[base + i]) : c_max<typename K::C>();
    __syncthreads();
    deep_tile_network(sm, full);
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) buf[base + i] = K::uncanon(sm[padc<typename K::C>(i)]);
    __syncthreads();
}

template <int KIND>
__device__ __forceinline__ void deep_tiles_body(const Job *__restrict__ job, uint32_t nd,
                                                typename Key<KIND>::C *sm, uint32_t &s_seg) {
    const uint32_t total = job->deep_tiles[nd];
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) s_seg = deep_find(job->deep_tiles, nd, t);
        __syncthreads();
        const uint32_t s = s_seg;
        const LeafItem it = job->deep[s];
        deep_tile<KIND>(job, it, t - job->deep_tiles[s], sm, true);
    }
}

template <int KIND>
__global__ void __launch_bounds__(kDeepThreads) k_deep_tiles(const Job *__restrict__ job, Ctl *ctl) {
    using C = typename Key<KIND>::C;
    extern __shared__ __align__(16) unsigned char deep_raw[];
    __shared__ uint32_t s_seg;
    const uint32_t nd = min(ctl->ndeep, job->cap_deep);
    if (nd == 0u) return;
    deep_tiles_body<KIND>(job, nd, reinterpret_cast<C *>(deep_raw), s_seg);
}

// The stage after (merge width 2^kk, stride 2^jj): the global half-cleaners down to
// stride 2^12, then the on-chip strides, then the next merge's mirror stage.
__device__ __forceinline__ void deep_next(uint32_t &kk, uint32_t &jj) {
    if (jj > 12u) jj--;
    else if (jj == 12u) jj = 11u;
    else { kk++; jj = kk - 1u; }
}

// One stage for every deep segment whose padded length reaches the merge width 2^kk.
template <int KIND>
__device__ __forceinline__ void deep_stage_body(const Job *__restrict__ job, uint32_t nd, uint32_t kk,
                                                uint32_t jj, typename Key<KIND>::C *sm, uint32_t &s_seg) {
    using K = Key<KIND>;
    using S = typename K::S;
    if (jj >= 12u) {                                      // a global stride
        const uint32_t total = job->deep_chunks[nd];
        const bool mirror = jj == kk - 1u;
        for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
            if (threadIdx.x == 0) s_seg = deep_find(job->deep_chunks, nd, c);
            __syncthreads();
            const uint32_t s = s_seg;
            __syncthreads();
            const LeafItem it = job->deep[s];
            const uint64_t len = it.len, P = 1ull << deep_log2(len);
            if (P < (1ull << kk)) continue;
            S *buf = buffer<K>(job, (it.kind & kLeafInAlt) ? 1 : 0) + it.begin;
            const uint64_t q0 = (uint64_t)(c - job->deep_chunks[s]) * kDeepChunk;
            const uint64_t q1 = min(q0 + kDeepChunk, P / 2);
            for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                uint64_t i, p;
                if (mirror) {
                    i = ((q >> (kk - 1u)) << kk) | (q & ((1ull << (kk - 1u)) - 1u));
                    p = i ^ ((1ull << kk) - 1u);
                } else {
                    i = ((q >> jj) << (jj + 1u)) | (q & ((1ull << jj) - 1u));
                    p = i + (1ull << jj);
                }
                if (p < len) {                            // p beyond the end is +infinity
                    const S x = buf[i], y = buf[p];
                    if (c_lt(K::canon(y), K::canon(x))) { buf[i] = y; buf[p] = x; }
                }
            }
        }
    } else {                                              // strides 2048 .. 1, on chip
        const uint32_t total = job->deep_tiles[nd];
        for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
            if (threadIdx.x == 0) s_seg = deep_find(job->deep_tiles, nd, t);
            __syncthreads();
            const uint32_t s = s_seg;
            const LeafItem it = job->deep[s];
            if ((1ull << deep_log2(it.len)) < (1ull << kk)) { __syncthreads(); continue; }
            deep_tile<KIND>(job, it, t - job->deep_tiles[s], sm, false);
        }
    }
}

// One stage per launch; the last block to finish advances the stage and sets the loop
// condition.
template <int KIND>
__global__ void __launch_bounds__(kDeepThreads) k_deep_stage(const Job *__restrict__ job, Ctl *ctl,
                                                             cudaGraphConditionalHandle h, int use_handle) {
    using C = typename Key<KIND>::C;
    extern __shared__ __align__(16) unsigned char deep_raw[];
    __shared__ uint32_t s_seg;
    const uint32_t nd = min(ctl->ndeep, job->cap_deep);
    const uint32_t kk = ctl->deep_kk, jj = ctl->deep_jj;
    deep_stage_body<KIND>(job, nd, kk, jj, reinterpret_cast<C *>(deep_raw), s_seg);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->deep_blocks, 1u) + 1u == gridDim.x) {
            uint32_t nk = kk, nj = jj;
            deep_next(nk, nj);
            const uint32_t cont = (nk <= ctl->deep_maxlog && ctl->status == 0u) ? 1u : 0u;
            ctl->deep_kk = nk;
            ctl->deep_jj = nj;
            ctl->deep_blocks = 0u;
            ctl->deep_cont = cont;
            if (use_handle) cudaGraphSetConditional(h, cont);
        }
    }
}

// Moves every deep segment to the output array when its buffer is not the output.
template <int KIND>
__device__ __forceinline__ void deep_finish_body(const Job *__restrict__ job, Ctl *ctl, uint32_t nd,
                                                 uint32_t &s_seg) {
    using K = Key<KIND>;
    using S = typename K::S;
    const uint32_t total = job->deep_tiles[nd];
    S *out = reinterpret_cast<S *>(job->out);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) s_seg = deep_find(job->deep_tiles, nd, t);
        __syncthreads();
        const uint32_t s = s_seg;
        __syncthreads();
        const LeafItem it = job->deep[s];
        const uint32_t ti = t - job->deep_tiles[s];
        if (threadIdx.x == 0 && ti == 0)
            atomicAdd((unsigned long long *)&ctl->deep_keys, (unsigned long long)it.len);
        const S *buf = buffer<K>(job, (it.kind & kLeafInAlt) ? 1 : 0);
        if ((const void *)buf == job->out) continue;
        const uint64_t base = it.begin + (uint64_t)ti * kDeepTile;
        const uint64_t end = min(base + (uint64_t)kDeepTile, (uint64_t)it.begin + it.len);
        for (uint64_t i = base + threadIdx.x; i < end; i += blockDim.x) out[i] = buf[i];
    }
}

template <int KIND>
__global__ void k_deep_finish(const Job *__restrict__ job, Ctl *ctl) {
    __shared__ uint32_t s_seg;
    const uint32_t nd = min(ctl->ndeep, job->cap_deep);
    if (nd == 0u) return;
    deep_finish_body<KIND>(job, ctl, nd, s_seg);
}

// Barrier over the whole grid of a cooperative launch (every block resident).  The last
// block to arrive publishes, with the next generation, whether the status is still clean,
// so every block takes the same decision; a wait that runs past `limit` polls sets
// TSQS_ETIMEOUT.  False: stop (the status is set).
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, uint32_t &gen, uint32_t limit) {
    __shared__ uint32_t s_go;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        uint32_t go = 0u;
        if (atomicAdd(&ctl->coop_count, 1u) + 1u == gridDim.x) {
            ctl->coop_count = 0u;
            ctl->coop_go = *(volatile const uint32_t *)&ctl->status == 0u ? 1u : 0u;
            __threadfence();
            atomicExch(&ctl->coop_gen, gen + 1u);
        } else {
            uint32_t polls = 0;
            while (*(volatile const uint32_t *)&ctl->coop_gen == gen) {
                if (++polls >= limit) { set_status(ctl, TSQS_ETIMEOUT); break; }
                __nanosleep(polls < 64 ? 32 : 256);
            }
            __threadfence();
        }
        go = *(volatile const uint32_t *)&ctl->coop_gen == gen + 1u ? *(volatile const uint32_t *)&ctl->coop_go : 0u;
        s_go = go;
    }
    __syncthreads();
    gen++;
    return s_go != 0u;
}

// The depth guard's whole branch in one cooperative launch (the task schedule's graph
// holds no conditional node): prep, tile sorts, every stage, finish, with a grid barrier
// between steps.  With no deep segment every block returns at once.
template <int KIND>
__global__ void __launch_bounds__(kDeepThreads) k_deep_all(const Job *__restrict__ job, Ctl *ctl) {
    using C = typename Key<KIND>::C;
    extern __shared__ __align__(16) unsigned char deep_raw[];
    C *sm = reinterpret_cast<C *>(deep_raw);
    __shared__ uint32_t s_seg;
    const uint32_t nd = min(*(volatile const uint32_t *)&ctl->ndeep, job->cap_deep);
    if (nd == 0u || *(volatile const uint32_t *)&ctl->status != 0u) return;
    const uint32_t limit = job->spin_limit;
    // the barrier's generation goes on from any earlier cooperative launch of this call
    uint32_t gen = *(volatile const uint32_t *)&ctl->coop_gen;
    if (blockIdx.x == 0) deep_prep_body(job, ctl);
    if (!grid_barrier(ctl, gen, limit)) return;
    deep_tiles_body<KIND>(job, nd, sm, s_seg);
    if (!grid_barrier(ctl, gen, limit)) return;
    const uint32_t maxlog = *(volatile const uint32_t *)&ctl->deep_maxlog;
    for (uint32_t kk = 13u, jj = 12u; kk <= maxlog;) {
        deep_stage_body<KIND>(job, nd, kk, jj, sm, s_seg);
        if (!grid_barrier(ctl, gen, limit)) return;
        deep_next(kk, jj);
    }
    deep_finish_body<KIND>(job, ctl, nd, s_seg);
}

// Level control (one thread).  Records the level's statistics, resets the consumed
// queues, advances the level and sets the loop condition: `more` when the next level's
// frontier is not empty, `cont` (the graph's level loop) only while the leaf queue also
// has room for another level's items; otherwise the loop pauses for a leaf pass.
__device__ __forceinline__ void level_control(const Job *job, Ctl *ctl, cudaGraphConditionalHandle handle,
                              int use_handle) {
    const uint32_t L = ctl->level;
    const int par = L & 1;
    if (L < (uint32_t)kStatLevels) ctl->level_keys[L] = ctl->front_keys[par];
    ctl->partition_keys += ctl->front_keys[par];
    if (ctl->nfront[par] > ctl->max_front) ctl->max_front = ctl->nfront[par];
    if (ctl->nfront[par]) ctl->levels_done++;
    ctl->nfront[par] = 0u;
    ctl->ntiles[par] = 0u;
    ctl->front_keys[par] = 0ull;
    ctl->tile_claim = 0u;
    ctl->seg_claim = 0u;
    ctl->level = L + 1;
    const bool more = ctl->nfront[par ^ 1] != 0u;    // queued leaves wait for a leaf pass
    if (more && L + 1 >= job->max_levels) set_status(ctl, TSQS_EINTERNAL);
    const uint32_t go = (ctl->status == 0u && more) ? 1u : 0u;
    const uint32_t cont = (go && ctl->nleaf <= job->leaf_defer) ? 1u : 0u;
    ctl->more = go;
    ctl->cont = cont;
    if (use_handle) cudaGraphSetConditional(handle, cont);
}


// End of a level: for every segment of the level, read its final (#<p, #>p) and push
// its children [a, a + #<p) and [b - #>p, b) and the fill of its =p run (the exit and
// recursion of Section III.F); the last block to finish then runs the level control.
template <int KIND>
__global__ void k_level_end(const Job *__restrict__ job, Ctl *ctl,
                            cudaGraphConditionalHandle handle, int use_handle, uint32_t) {
    using K = Key<KIND>;
    __shared__ uint32_t s_last, s_ok;
    const int par = ctl->level & 1;
    // block-uniform: the loop below holds warp-wide shuffles and a block barrier follows
    if (threadIdx.x == 0) s_ok = *(volatile uint32_t *)&ctl->status == 0u ? 1u : 0u;
    __syncthreads();
    const bool ok_state = s_ok != 0u;
    const uint32_t nf = min(ctl->nfront[par], job->cap_front);
    const int np = par ^ 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t T = job->small_T;
    const int TILE = (int)job->tile;
    // depth guard: a child that would be partitioned at deep_level or later goes to the
    // bitonic sorter after the loop (this level is ctl->level, its children's is + 1)
    const bool to_deep = ctl->level + 1u >= job->deep_level;
    // every lane takes one segment; a warp makes one atomic per counter for all its
    // pushes (frontier entries, tiles, leaf items, keys) and hands out the offsets
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t base0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint32_t wb = base0; ok_state && wb < nf; wb += stride) {
        const uint32_t si = wb + lane;
        const bool have = si < nf;
        uint64_t cb[2] = {0, 0}, ce[2] = {0, 0}, eqb = 0, eqe = 0;
        uint64_t piv_lo = 0, piv_hi = 0;
        bool bad = false;
        if (have) {
            const SegDesc sd = job->front[par][si];
            uint64_t nlt, ngt;
            const bool ok = seg_totals(job, si, sd.tile_begin, sd.ntiles, nlt, ngt);
            const uint64_t m = sd.end - sd.begin;
            if (!ok || nlt + ngt >= m) {
                // p is an element of the segment, so the =p run is never empty; a
                // violation means corrupted state: stop instead of looping forever
                bad = true;
            } else {
                cb[0] = sd.begin; ce[0] = sd.begin + nlt;
                cb[1] = sd.end - ngt; ce[1] = sd.end;
                eqb = sd.begin + nlt; eqe = sd.end - ngt;
                piv_lo = sd.piv_lo; piv_hi = sd.piv_hi;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(ctl, TSQS_EINTERNAL);
        // per lane: up to two frontier pushes, two leaf pushes, and nch fill items
        uint32_t nfr = 0, ntl = 0, nlf = 0, ndp = 0;
        uint64_t keys = 0;
        int64_t s0[2] = {0, 0};
        uint32_t ntc[2] = {0, 0};
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const uint64_t msz = ce[c] - cb[c];
            if (msz > T && to_deep) {
                ndp++;
            } else if (msz > T) {
                s0[c] = tile_origin<K::V>(cb[c], job->vec_off);
                ntc[c] = tiles_for(ce[c], s0[c], TILE);
                nfr++; ntl += ntc[c]; keys += msz;
            } else if (msz >= 1) {
                nlf++;
            }
        }
        // a short =p run is written right here (no later kernel reads or writes it), so
        // the leaf pass does not spend a claim round trip on a one-element fill
        const bool inline_fill = eqe - eqb <= kInlineFill;
        const uint32_t nch = inline_fill ? 0u : (uint32_t)((eqe - eqb + kFillChunk - 1) / kFillChunk);
        uint64_t ifill = 0;
        if (inline_fill && eqe > eqb) {
            typename K::S *outp = reinterpret_cast<typename K::S *>(job->out);
            const typename K::S val = K::uncanon(c_from<typename K::C>(piv_lo, piv_hi));
            for (uint64_t x = eqb; x < eqe; x++) outp[x] = val;
            ifill = eqe - eqb;
        }
        nlf += nch;
        // warp-exclusive offsets and one atomic per counter
        uint32_t xf = nfr, xt = ntl, xl = nlf, xd = ndp;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a = __shfl_up_sync(0xffffffffu, xf, o);
            const uint32_t b2 = __shfl_up_sync(0xffffffffu, xt, o);
            const uint32_t c2 = __shfl_up_sync(0xffffffffu, xl, o);
            const uint32_t d2 = __shfl_up_sync(0xffffffffu, xd, o);
            if (lane >= (uint32_t)o) { xf += a; xt += b2; xl += c2; xd += d2; }
        }
        uint64_t ksum = keys, fsum = ifill;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ksum += __shfl_xor_sync(0xffffffffu, ksum, o);
            fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
        }
        uint32_t bf = 0, bt = 0, bl = 0, bd = 0;
        if (lane == 31) {
            bf = atomicAdd(&ctl->nfront[np], xf);
            bt = atomicAdd(&ctl->ntiles[np], xt);
            bl = atomicAdd(&ctl->nleaf, xl);
            if (xd) bd = atomicAdd(&ctl->ndeep, xd);
            if (ksum) atomicAdd((unsigned long long *)&ctl->front_keys[np], (unsigned long long)ksum);
            if (fsum) atomicAdd((unsigned long long *)&ctl->leaf_filled, (unsigned long long)fsum);
        }
        bf = __shfl_sync(0xffffffffu, bf, 31) + xf - nfr;
        bt = __shfl_sync(0xffffffffu, bt, 31) + xt - ntl;
        bl = __shfl_sync(0xffffffffu, bl, 31) + xl - nlf;
        bd = __shfl_sync(0xffffffffu, bd, 31) + xd - ndp;
        // write this lane's pushes
        bool overflow = false;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const uint64_t msz = ce[c] - cb[c];
            if (msz > T && to_deep) {
                if (bd >= job->cap_deep) overflow = true;
                else {
                    LeafItem it;
                    it.begin = cb[c]; it.len = (uint32_t)msz;
                    it.kind = np ? kLeafInAlt : 0u;      // keys in the buffer this level wrote
                    it.v_lo = 0; it.v_hi = 0;
                    job->deep[bd] = it;
                }
                bd++;
            } else if (msz > T) {
                if (bf >= job->cap_front || (uint64_t)bt + ntc[c] > job->cap_tiles) {
                    overflow = true;
                } else {
                    SegDesc d;
                    d.begin = cb[c]; d.end = ce[c]; d.s0 = s0[c]; d.tile_begin = bt; d.ntiles = ntc[c];
                    d.piv_lo = 0; d.piv_hi = 0;
                    job->front[np][bf] = d;
                }
                bf++; bt += ntc[c];
            } else if (msz >= 1) {
                if (bl >= job->cap_leaves) overflow = true;
                else {
                    LeafItem it;
                    it.begin = cb[c]; it.len = (uint32_t)msz;
                    it.kind = LEAF_SORT | (np ? kLeafInAlt : 0u);     // written by this level
                    it.v_lo = 0; it.v_hi = 0;
                    job->leaves[bl] = it;
                }
                bl++;
            }
        }
        for (uint32_t c = 0; c < nch; c++) {
            if (bl + c >= job->cap_leaves) { overflow = true; break; }
            LeafItem li;
            li.begin = eqb + (uint64_t)c * kFillChunk;
            const uint64_t rest = eqe - li.begin;
            li.len = (uint32_t)(rest < kFillChunk ? rest : kFillChunk);
            li.kind = LEAF_FILL;
            li.v_lo = piv_lo;
            li.v_hi = piv_hi;
            job->leaves[bl + c] = li;
        }
        if (overflow) set_status(ctl, TSQS_EINTERNAL);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&ctl->blocks_done, 1u);
        s_last = (d + 1 == gridDim.x) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        ctl->blocks_done = 0u;
        level_control(job, ctl, handle, use_handle);
    }
}

}  // namespace tsqs
