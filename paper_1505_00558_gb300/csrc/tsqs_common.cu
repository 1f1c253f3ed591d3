// tsqs_common.cu -- kernels that do not depend on the key kind.
#include "tsqs_kernels.cuh"

namespace tsqs {

__global__ void k_setup(Job *job, Ctl *ctl, Job j) {
    if (threadIdx.x == 0) *job = j;
    uint32_t *c = reinterpret_cast<uint32_t *>(ctl);
    for (uint32_t i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) c[i] = 0u;
}

__global__ void k_finish(const Job *job, Ctl *ctl, cudaGraphConditionalHandle handle,
                         int use_handle, uint32_t) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t L = ctl->level;
    const int par = L & 1;
    if (L < (uint32_t)kStatLevels) ctl->level_keys[L] = ctl->front_keys[par];
    ctl->partition_keys += ctl->front_keys[par];
    if (ctl->nfront[par] > ctl->max_front) ctl->max_front = ctl->nfront[par];
    if (ctl->nfront[par]) ctl->levels_done++;
    ctl->nfront[par] = 0u;
    ctl->ntiles[par] = 0u;
    ctl->nleaf[par] = 0u;
    ctl->front_keys[par] = 0ull;
    ctl->tile_claim = 0u;
    ctl->leaf_claim = 0u;
    ctl->seg_claim = 0u;
    ctl->level = L + 1;
    const bool more = (ctl->nfront[par ^ 1] | ctl->nleaf[par ^ 1]) != 0u;
    if (more && L + 1 >= job->max_levels) set_status(ctl, TSQS_EINTERNAL);
    const uint32_t cont = (ctl->status == 0u && more) ? 1u : 0u;
    ctl->cont = cont;
    if (use_handle) cudaGraphSetConditional(handle, cont);
}

__global__ void k_dbg_counts(const Job *__restrict__ job, Ctl *) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < job->nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const SegDesc d = job->front[0][s];
        uint64_t lt = 0, gt = 0;
        if (d.ntiles) {
            const unsigned long long w = job->tile_status[d.tile_begin + d.ntiles - 1];
            lt = (w >> 31) & 0x7FFFFFFFull;
            gt = w & 0x7FFFFFFFull;
        }
        job->dbg_counts[2 * s] = lt;
        job->dbg_counts[2 * s + 1] = gt;
    }
}

}  // namespace tsqs
