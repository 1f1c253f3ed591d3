// tsqs_noalloc.cu -- a sort entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a sort: code whose
// device memory is entirely owned by another allocator (a framework's caching pool,
// a fixed arena, where a raw cudaMalloc fails or fragments it), services that account
// for every device byte up front, and latency-critical paths that cannot pay for an
// allocation that may synchronise the device.  tsqs_sort_noalloc serves them: it runs
// the same kernels as tsqs_sort, but every piece of scratch -- the second buffer of
// the ping-pong, the segment and leaf queues, the tile table, the per-call description
// and the control block -- lives in the static device arrays below, which are part of
// this library's device code.  Each GPU on which this code is loaded holds the arrays
// until the process exits.
//
// The call drives the level loop from the host: it reads the loop flag back and
// synchronises `stream` after every level, and it returns only once its sort has
// finished.  A stream that is being captured cannot be synchronised, so the call
// refuses one (TSQS_EINVAL, nothing queued).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "tsqs.h"
#include "tsqs_internal.h"

namespace tsqs {
__global__ void k_setup(Job *job, Ctl *ctl, Job j);
const KindOps *host_ops(int key_kind);
void host_default_plan(int key_kind, tsqs_plan *p);
size_t host_scratch_bytes(const KindOps *o, const tsqs_plan &p, size_t n);
const PartVariant &host_part(const KindOps *o, const tsqs_plan &p);
int host_make_job_at(const KindOps *o, const tsqs_plan &plan, void *base, size_t n, char *scratch,
                     size_t bytes, Job *j);
}  // namespace tsqs

using namespace tsqs;

namespace {

// The largest array the entry point sorts is TSQS_NOALLOC_MAX_BYTES (16 MiB); the
// scratch adds a second buffer of the same size plus the queues, which stay below
// 4 MiB for that size and every key kind (checked at set-up).
constexpr size_t kNoAllocScratch = TSQS_NOALLOC_MAX_BYTES + (4u << 20);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratch];
static __device__ Job g_noalloc_job;
static __device__ Ctl g_noalloc_ctl;

struct DevState {
    bool ready = false;
    char *scratch = nullptr;   // device address of g_noalloc_scratch on this device
    Job *job = nullptr;
    Ctl *ctl = nullptr;
    int sms = 0;
    int part_grid[8] = {};
    int leaf_grid[8] = {};
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DevState g_dev[kMaxDevices];
unsigned int g_cont[kMaxDevices];       // host copy of the loop flag, per device

// Once per device, with that device current: resolve the arrays' device addresses
// (the names are host-side stand-ins in host code) and size the persistent grids.
int setup_device(int dev, DevState &d) {
    if (d.ready) return TSQS_OK;
    if (cudaGetSymbolAddress((void **)&d.scratch, g_noalloc_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void **)&d.job, g_noalloc_job) != cudaSuccess ||
        cudaGetSymbolAddress((void **)&d.ctl, g_noalloc_ctl) != cudaSuccess) {
        cudaGetLastError();
        return TSQS_ECUDA;
    }
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TSQS_ECUDA;
    for (int kind = TSQS_I32; kind <= TSQS_U64_U64_REC; kind++) {
        const KindOps *o = host_ops(kind);
        tsqs_plan p;
        host_default_plan(kind, &p);
        const PartVariant &pv = host_part(o, p);
        // the largest accepted array must fit the static scratch
        if (host_scratch_bytes(o, p, TSQS_NOALLOC_MAX_BYTES / (size_t)o->elem_size) > kNoAllocScratch)
            return TSQS_EINTERNAL;
        int occ_p = 0, occ_l = 0;
        if (cudaFuncSetAttribute(o->k_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, o->leaf_smem) != cudaSuccess ||
            cudaFuncSetAttribute(o->k_deep_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, o->deep_smem) != cudaSuccess ||
            cudaFuncSetAttribute(o->k_deep_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, o->deep_smem) != cudaSuccess ||
            cudaFuncSetAttribute(pv.k_partition, cudaFuncAttributeMaxDynamicSharedMemorySize, pv.smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, pv.k_partition, pv.threads, pv.smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, o->k_leaf, o->leaf_block, o->leaf_smem) != cudaSuccess) {
            cudaGetLastError();
            return TSQS_ECUDA;
        }
        d.part_grid[kind] = (occ_p > 0 ? occ_p : 1) * d.sms;
        d.leaf_grid[kind] = (occ_l > 0 ? occ_l : 1) * d.sms;
    }
    d.ready = true;
    return TSQS_OK;
}

}  // namespace

extern "C" int tsqs_sort_noalloc(void *base, size_t nmemb, size_t elem_size, int key_kind,
                                 void *stream) {
    const KindOps *o = host_ops(key_kind);
    if (!o || (size_t)o->elem_size != elem_size) return TSQS_EINVAL;
    if (nmemb > 1 && !base) return TSQS_EINVAL;
    if ((uintptr_t)base % (elem_size == 16 ? 16 : elem_size)) return TSQS_EINVAL;
    if (nmemb > TSQS_NOALLOC_MAX_BYTES / elem_size) return TSQS_EINVAL;   // over the limit
    if (nmemb <= 1) return TSQS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TSQS_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) { cudaGetLastError(); return TSQS_EINVAL; }
    if (cap != cudaStreamCaptureStatusNone) return TSQS_EINVAL;          // would break the capture
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[dev];
    int rc = setup_device(dev, d);
    if (rc) return rc;
    tsqs_plan plan;
    host_default_plan(key_kind, &plan);
    Job j;
    if ((rc = host_make_job_at(o, plan, base, nmemb, d.scratch, kNoAllocScratch, &j))) return rc;
    const PartVariant &pv = host_part(o, plan);
    Job *pj = d.job;
    Ctl *pc = d.ctl;
    void *args2[] = {&pj, &pc};
    cudaGraphConditionalHandle h = 0;
    int use_h = 0;
    unsigned int unused = 0;
    void *argsf[] = {&pj, &pc, &h, &use_h, &unused};
    int leaf_final = 0, leaf_last = 1;
    void *argsl[] = {&pj, &pc, &leaf_final};
    void *argsl_last[] = {&pj, &pc, &leaf_last};
    int use_hd = 0;
    void *argsd[] = {&pj, &pc, &h, &use_hd};
    uint32_t status = 0;
    // setup zeroes the control block, so nothing a previous call left in the shared
    // arrays is read before it is rewritten
    k_setup<<<1, 256, 0, s>>>(d.job, d.ctl, j);
    if (cudaGetLastError() != cudaSuccess) goto failed;
    // from here on every failure goes through `failed`, which waits for the kernels
    // already queued before the lock is released, so a later call never rewrites the
    // shared arrays under them
    if (cudaLaunchKernel(o->k_orient, dim3(d.sms * 4), dim3(256), args2, 0, s) != cudaSuccess ||
        cudaLaunchKernel(o->k_check, dim3(d.sms * 4), dim3(256), args2, 0, s) != cudaSuccess ||
        cudaLaunchKernel(o->k_presort, dim3(d.sms * 4), dim3(256), args2, 0, s) != cudaSuccess ||
        cudaLaunchKernel(o->k_init, dim3(d.sms * 2), dim3(256), args2, 0, s) != cudaSuccess)
        goto failed;
    for (uint32_t level = 0; level <= j.max_levels; level++) {
        if (cudaLaunchKernel(o->k_leaf, dim3(d.leaf_grid[key_kind]), dim3(o->leaf_block), argsl,
                             (size_t)o->leaf_smem, s) != cudaSuccess ||
            cudaLaunchKernel(o->k_pivot, dim3(d.sms * 4), dim3(o->pivot_block), args2, 0, s) != cudaSuccess ||
            cudaLaunchKernel(pv.k_partition, dim3(d.part_grid[key_kind]), dim3(pv.threads), args2,
                             (size_t)pv.smem, s) != cudaSuccess ||
            cudaLaunchKernel(o->k_finish, dim3(d.sms), dim3(128), argsf, 0, s) != cudaSuccess)
            goto failed;
        // the loop flag comes back into ordinary host memory: the copy returns once the
        // level is done
        if (cudaMemcpyAsync(&g_cont[dev], &d.ctl->more, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            goto failed;
        if (!g_cont[dev]) break;
    }
    // the final leaf pass over every queued item
    if (cudaLaunchKernel(o->k_leaf, dim3(d.leaf_grid[key_kind]), dim3(o->leaf_block), argsl_last,
                         (size_t)o->leaf_smem, s) != cudaSuccess)
        goto failed;
    // depth guard: segments that reached the level bound are sorted by the bitonic stages
    if (cudaLaunchKernel(o->k_deep_prep, dim3(1), dim3(512), argsd, 0, s) != cudaSuccess ||
        cudaLaunchKernel(o->k_deep_tiles, dim3(d.sms * 2), dim3(512), args2, (size_t)o->deep_smem, s) != cudaSuccess)
        goto failed;
    for (int it = 0; it < 4096; it++) {
        if (cudaMemcpyAsync(&g_cont[dev], &d.ctl->deep_cont, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            goto failed;
        if (!g_cont[dev]) break;
        if (cudaLaunchKernel(o->k_deep_stage, dim3(d.sms * 2), dim3(512), argsd, (size_t)o->deep_smem, s) != cudaSuccess)
            goto failed;
    }
    if (cudaLaunchKernel(o->k_deep_finish, dim3(d.sms * 2), dim3(512), args2, 0, s) != cudaSuccess)
        goto failed;
    if (cudaMemcpyAsync(&status, &d.ctl->status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        goto failed;
    return (int)status;
failed:
    cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return TSQS_ECUDA;
}
