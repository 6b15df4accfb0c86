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

// Resident blocks per SM the kernel is compiled for: eight, at 64 registers a
// thread.  The tiles are latency-bound, so warps in flight count for more
// than the spills a lower register budget brings (64-grid batch on GB300:
// 1.26 ms with four blocks per SM at 128 registers, 1.12 with five, 1.03 with
// six, 1.02 with seven, 1.006 with eight; with 8 points per thread on the
// 2^a-point lines instead of 16: 1.017 ms at eight blocks, 1.034 at ten,
// 1.18 at twelve).
#ifndef PSOLVE_BATCH_MINB
#define PSOLVE_BATCH_MINB 8
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

// Block-private scheduling state, in shared memory, written by thread 0 only.
struct Sched {
    long long item, next;  // the item being run; the one claimed after it
    int seg, next_seg;     // their segments
    int next_ready;        // the next item's dependency is known to be met
    int okseg;             // a segment whose dependency this block has seen met
    int pend;              // segment of a finished item not yet published, or -1
    int claimed;           // the next item of the running one has been claimed
    int abort;
};

// Publish the block's finished item: the barrier before this call orders
// every thread's stores of that item before thread 0's fence (cumulative at
// GPU scope), then one count.
__device__ __forceinline__ void publish(Sched &s, int *done)
{
    if (s.pend >= 0) {
        __threadfence();
        atomicAdd(&done[s.pend], 1);
        s.pend = -1;
    }
}

// Claim the item after the running one and look (without waiting) whether
// its dependency is met.
template <typename T>
__device__ __forceinline__ void claim_next(Sched &s, const BatchSeg<T> *segs, int nseg, long long total,
                                           unsigned long long *work, int *done)
{
    const long long nx = (long long)atomicAdd(work, 1ull);
    int sg = s.seg;
    while (sg + 1 < nseg && segs[sg + 1].first <= nx) ++sg;
    s.next = nx;
    s.next_seg = sg;
    int ready = 1;
    if (nx < total && sg != s.okseg) {
        const int dep = segs[sg].dep;
        ready = dep < 0 || ld_acquire(&done[dep]) >= segs[sg].need;
        if (ready) s.okseg = sg;
    }
    s.next_ready = ready;
    s.claimed = 1;
}

// Called by every thread of the block once the tile's loads are issued:
// thread 0 publishes the previous item and claims the next while the loads
// are in flight.
template <typename T> struct SchedHook {
    Sched *s;
    const BatchSeg<T> *segs;
    int nseg;
    long long total;
    unsigned long long *work;
    int *done;
    __device__ __forceinline__ void operator()() const
    {
        if (threadIdx.x == 0) {
            publish(*s, done);
            claim_next<T>(*s, segs, nseg, total, work, done);
        }
    }
};

// One tile of one pass; LC > 0: the line length, with its compile-time plan.
// Not inlined: each variant gets its own register allocation (a tile is
// thousands of instructions, so the call costs nothing measurable).
template <typename T, int E, int LC> __device__ __noinline__ void run_item(const BatchSeg<T> *__restrict__ sgp,
                                                                          long long tile, const T *f, T *u,
                                                                          unsigned char *smem,
                                                                          const SchedHook<T> *hk)
{
    const BatchSeg<T> &sg = *sgp;
    T *ui = u + sg.off;
    const SchedHook<T> &h = *hk;
    switch (sg.kind) {
    case 0: zfwd_tile<T, E, LC, true>(sg.z, f + sg.off, ui, tile, smem, h); break;
    case 1: ypass_tile<T, E, false, LC, true>(sg.y, ui, tile, smem, h); break;
    case 2: xfused_tile<T, E, LC, true>(sg.x, ui, tile, smem, h); break;
    case 3: ypass_tile<T, E, true, LC, true>(sg.y, ui, tile, smem, h); break;
    default: zinv_tile<T, E, LC, true>(sg.z, ui, ui, tile, smem, h); break;
    }
}

// Compile-time plans: 2^a-point lines with 16 points per thread, 3·2^a-point
// lines with 12 (the run-time planner's choices for batches).
template <typename T> __device__ __forceinline__ void run_item_any(const BatchSeg<T> &sg, long long tile,
                                                                   const T *f, T *u, unsigned char *smem,
                                                                   const SchedHook<T> *h)
{
    switch (sg.E) {
    case 4: run_item<T, 4, 0>(&sg, tile, f, u, smem, h); break;
    case 8: run_item<T, 8, 0>(&sg, tile, f, u, smem, h); break;
    case 12:
        switch (sg.lc) {
        case 12: run_item<T, 12, 12>(&sg, tile, f, u, smem, h); break;
        case 24: run_item<T, 12, 24>(&sg, tile, f, u, smem, h); break;
        case 48: run_item<T, 12, 48>(&sg, tile, f, u, smem, h); break;
        case 96: run_item<T, 12, 96>(&sg, tile, f, u, smem, h); break;
        case 192: run_item<T, 12, 192>(&sg, tile, f, u, smem, h); break;
        default: run_item<T, 12, 0>(&sg, tile, f, u, smem, h); break;
        }
        break;
    case 16:
        switch (sg.lc) {
        case 16: run_item<T, 16, 16>(&sg, tile, f, u, smem, h); break;
        case 32: run_item<T, 16, 32>(&sg, tile, f, u, smem, h); break;
        case 64: run_item<T, 16, 64>(&sg, tile, f, u, smem, h); break;
        case 128: run_item<T, 16, 128>(&sg, tile, f, u, smem, h); break;
        case 256: run_item<T, 16, 256>(&sg, tile, f, u, smem, h); break;
        default: run_item<T, 16, 0>(&sg, tile, f, u, smem, h); break;
        }
        break;
    default: break;
    }
}

// Items are taken in order; thread 0 claims the next one and checks its
// dependency while the running item's loads are in flight, and publishes a
// finished item one item later (or before it waits, or at exit), so that no
// fence, atomic or dependency load sits between two items.  A block never
// waits with an unpublished item, so the argument above still holds: the
// lowest unfinished item depends only on published ones.
template <typename T>
__global__ void __launch_bounds__(kBatchThreads, PSOLVE_BATCH_MINB) k_batched(const BatchSeg<T> *segs, int nseg,
                                                              long long total, const T *f, T *u,
                                                              unsigned long long *work, int *done, int *status,
                                                              unsigned long long wait_ns)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ Sched s;
    __shared__ __align__(16) BatchSeg<T> seg_copy;
    const SchedHook<T> hook{&s, segs, nseg, total, work, done};
    if (threadIdx.x == 0) {
        s.seg = 0;
        s.okseg = -1;
        s.pend = -1;
        claim_next<T>(s, segs, nseg, total, work, done);
    }
    while (true) {
        if (threadIdx.x == 0) {
            // (the previous item's stores and shared-memory reads are ordered
            // by the barrier that ended it: run_item_any's callers reach here
            // only after the barrier below)
            if (!s.claimed) claim_next<T>(s, segs, nseg, total, work, done);
            s.item = s.next;
            s.seg = s.next_seg;
            s.claimed = 0;
            s.abort = 0;
            if (s.item < total && !s.next_ready) {
                publish(s, done);
                const BatchSeg<T> &sg = segs[s.seg];
                if (wait_count(&done[sg.dep], sg.need, wait_ns)) {
                    s.okseg = s.seg;
                } else {
                    s.abort = 1;
                    atomicExch(status, (int)PSOLVE_ERR_TIMEOUT);
                }
            }
        }
        __syncthreads();
        const long long item = s.item;
        if (item >= total || s.abort) {
            if (threadIdx.x == 0 && !s.abort) publish(s, done);
            return;
        }
        // the segment descriptor, copied into shared memory by the whole
        // block: the tile reads its fields many times (64-grid batch on
        // GB300: 1.005 -> 0.996 ms, the barrier included; copied by one warp
        // while the previous tile's loads were in flight instead: 1.067 ms)
        {
            static_assert(sizeof(BatchSeg<T>) % sizeof(longlong2) == 0, "descriptor copied in 16-byte pieces");
            const longlong2 *src = reinterpret_cast<const longlong2 *>(&segs[s.seg]);
            longlong2 *dst = reinterpret_cast<longlong2 *>(&seg_copy);
            for (int i = threadIdx.x; i < (int)(sizeof(BatchSeg<T>) / sizeof(longlong2)); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        const BatchSeg<T> &sg = seg_copy;
        run_item_any<T>(sg, item - sg.first, f, u, smraw, &hook);
        // Every thread's stores of this item and its shared-memory reads are
        // finished before thread 0 claims, publishes or the next item starts.
        __syncthreads();
        if (threadIdx.x == 0) s.pend = s.seg;
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
