// One persistent launch for a batch of unequal grids.
//
// The work list is every tile of every pass of every instance, pass-major:
// segment s = pass·B + instance holds the tiles of one pass (zfwd, yfwd,
// xdiv, yinv, zinv) of one instance.  Blocks take items in order from an
// atomic counter.  Before the first write of segment (pass, i) a block waits
// until every tile of segment (pass-1, i) has completed: the tiles it waits
// for have lower item numbers, so they are held by blocks that are already
// running and never wait on later items; the wait therefore ends unless
// something is broken, and it is bounded in time all the same (the block
// then records PSOLVE_ERR_TIMEOUT in the status word and leaves).
// Data written by other blocks of the same launch are read with L2-only
// loads (ld.global.cg).  Lines are planned with at most 16 points per
// thread (12 for lengths 3·2^a); lines needing 2, 3 or 6 are not covered
// (the planner then launches per pass).  Lines of 12…256 points in radix
// order 0 run compile-time plans (batched_ct_supported), the others run-time
// plans; each (points per thread, length) variant is a separate device
// function, so the one kernel does not carry the registers of the largest.
#include "psolve.h"
#include "launch.h"
#include "tma.cuh"

#ifndef PSOLVE_BATCH_MINB
#define PSOLVE_BATCH_MINB 4
#endif

namespace psolve {

namespace {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *counter >= need, at most limit_ns; false on timeout.
__device__ bool wait_count(const int *counter, long long need, unsigned long long limit_ns)
{
    if (ld_acquire(counter) >= need) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        __nanosleep(256);
        if (ld_acquire(counter) >= need) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// One tile of one pass; LC > 0: the line length, with its compile-time plan.
// Not inlined: each variant gets its own register allocation (a tile is
// thousands of instructions, so the call costs nothing measurable).
template <typename T, int E, int LC> __device__ __noinline__ void run_item(const BatchSeg<T> *__restrict__ sgp,
                                                                          long long tile, const T *f, T *u,
                                                                          unsigned char *smem)
{
    const BatchSeg<T> &sg = *sgp;
    T *ui = u + sg.off;
    switch (sg.kind) {
    case 0: zfwd_tile<T, E, LC, true>(sg.z, f + sg.off, ui, tile, smem); break;
    case 1: ypass_tile<T, E, false, LC, true>(sg.y, ui, tile, smem); break;
    case 2: xfused_tile<T, E, LC, true>(sg.x, ui, tile, smem); break;
    case 3: ypass_tile<T, E, true, LC, true>(sg.y, ui, tile, smem); break;
    default: zinv_tile<T, E, LC, true>(sg.z, ui, ui, tile, smem); break;
    }
}

// Compile-time plans: 2^a-point lines with 16 points per thread, 3·2^a-point
// lines with 12 (the run-time planner's choices for batches).
template <typename T> __device__ __forceinline__ void run_item_any(const BatchSeg<T> &sg, long long tile,
                                                                   const T *f, T *u, unsigned char *smem)
{
    switch (sg.E) {
    case 4: run_item<T, 4, 0>(&sg, tile, f, u, smem); break;
    case 8: run_item<T, 8, 0>(&sg, tile, f, u, smem); break;
    case 12:
        switch (sg.lc) {
        case 12: run_item<T, 12, 12>(&sg, tile, f, u, smem); break;
        case 24: run_item<T, 12, 24>(&sg, tile, f, u, smem); break;
        case 48: run_item<T, 12, 48>(&sg, tile, f, u, smem); break;
        case 96: run_item<T, 12, 96>(&sg, tile, f, u, smem); break;
        case 192: run_item<T, 12, 192>(&sg, tile, f, u, smem); break;
        default: run_item<T, 12, 0>(&sg, tile, f, u, smem); break;
        }
        break;
    case 16:
        switch (sg.lc) {
        case 16: run_item<T, 16, 16>(&sg, tile, f, u, smem); break;
        case 32: run_item<T, 16, 32>(&sg, tile, f, u, smem); break;
        case 64: run_item<T, 16, 64>(&sg, tile, f, u, smem); break;
        case 128: run_item<T, 16, 128>(&sg, tile, f, u, smem); break;
        case 256: run_item<T, 16, 256>(&sg, tile, f, u, smem); break;
        default: run_item<T, 16, 0>(&sg, tile, f, u, smem); break;
        }
        break;
    default: break;
    }
}

template <typename T>
__global__ void __launch_bounds__(kBatchThreads, PSOLVE_BATCH_MINB) k_batched(const BatchSeg<T> *segs, int nseg,
                                                              long long total, const T *f, T *u,
                                                              unsigned long long *work, int *done, int *status,
                                                              unsigned long long wait_ns)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ long long s_item, s_next;
    __shared__ int s_seg, s_abort;
    if (threadIdx.x == 0) {
        s_next = (long long)atomicAdd(work, 1ull);
        s_seg = 0;
    }
    while (true) {
        __syncthreads(); // the previous item's shared-memory reads are finished
        if (threadIdx.x == 0) {
            s_item = s_next;
            s_abort = 0;
            if (s_item < total) {
                // Items grow per block: walk forward from the last segment.
                int sgi = s_seg;
                while (sgi + 1 < nseg && segs[sgi + 1].first <= s_item) ++sgi;
                s_seg = sgi;
                const int dep = segs[sgi].dep;
                if (dep >= 0 && !wait_count(&done[dep], segs[sgi].need, wait_ns)) {
                    s_abort = 1;
                    atomicExch(status, (int)PSOLVE_ERR_TIMEOUT);
                }
                // Take the next item now; it is only claimed, not started.
                s_next = (long long)atomicAdd(work, 1ull);
            }
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= total || s_abort) return;
        const BatchSeg<T> &sg = segs[s_seg];
        const long long tile = item - sg.first;
        run_item_any<T>(sg, tile, f, u, smraw);
        // Publish this tile: the barrier orders every thread's stores before
        // thread 0's fence (cumulative at GPU scope), then one count.
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[s_seg], 1);
        }
    }
}

} // namespace

// FP32 only; FP64 plans of unequal grids use one launch per pass and instance.
template <typename T> const void *batched_kernel() { return reinterpret_cast<const void *>(&k_batched<T>); }
template const void *batched_kernel<float>();

template <typename T> cudaError_t batched_prepare(size_t smem)
{
    return cudaFuncSetAttribute(k_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template cudaError_t batched_prepare<float>(size_t);

bool batched_supports_E(int E) { return E == 4 || E == 8 || E == 12 || E == 16; }

bool batched_ct_supported(int L, int E)
{
    if (E == 12) return L == 12 || L == 24 || L == 48 || L == 96 || L == 192;
    if (E == 16) return L == 16 || L == 32 || L == 64 || L == 128 || L == 256;
    return false;
}

} // namespace psolve
