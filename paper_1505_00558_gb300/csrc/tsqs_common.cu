// tsqs_common.cu -- kernels that do not depend on the key kind.
#include "tsqs_kernels.cuh"

namespace tsqs {

__global__ void k_setup(Job *job, Ctl *ctl, Job j) {
    if (threadIdx.x == 0) *job = j;
    uint32_t *c = reinterpret_cast<uint32_t *>(ctl);
    for (uint32_t i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) c[i] = 0u;
}

// Keeps one sort's device status (0 when no sort ran for the item) in a per-item word.
__global__ void k_keep_status(const Ctl *ctl, uint32_t *dst, int ran) {
    if (threadIdx.x == 0) *dst = ran ? ctl->status : 0u;
}

__global__ void k_dbg_counts(const Job *__restrict__ job, Ctl *) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < job->nseg;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const SegDesc d = job->front[0][s];
        uint64_t lt = 0, gt = 0;
        seg_totals(job, (uint32_t)s, d.tile_begin, d.ntiles, lt, gt);
        job->dbg_counts[2 * s] = lt;
        job->dbg_counts[2 * s + 1] = gt;
    }
}

}  // namespace tsqs
