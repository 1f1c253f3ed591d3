// tsqs_common.cu -- kernels that do not depend on the key kind.
#include "tsqs_kernels.cuh"

namespace tsqs {

__global__ void k_setup(Job *job, Ctl *ctl, Job j) {
    if (threadIdx.x == 0) *job = j;
    uint32_t *c = reinterpret_cast<uint32_t *>(ctl);
    for (uint32_t i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) c[i] = 0u;
}

// After a leaf pass in the graph: run more levels (the level loop and the loop around
// it continue) while levels remain and the status is clean; once they are done, the
// depth guard's branch runs only if some segment reached its level.
__global__ void k_outer_control(const Ctl *ctl, cudaGraphConditionalHandle h_levels,
                                cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_deep) {
    if (threadIdx.x == 0) {
        const bool ok = ctl->status == 0u;
        const unsigned int go = (ctl->more != 0u && ok) ? 1u : 0u;
        cudaGraphSetConditional(h_levels, go);
        cudaGraphSetConditional(h_outer, go);
        cudaGraphSetConditional(h_deep, (!go && ok && ctl->ndeep != 0u) ? 1u : 0u);
    }
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
