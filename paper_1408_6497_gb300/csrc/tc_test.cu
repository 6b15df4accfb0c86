// Stand-alone check of the tensor-core radix-16 stage: 16-point DFTs of
// independent butterflies through tc_dft16, exposed as
// psolve_debug_tc_dft16 so the tests can compare it with a reference DFT.
#include "psolve.h"
#include "tc.cuh"

namespace psolve {
namespace {

constexpr int kTestThreads = 256;                 // 2 MMA groups of 128 rows
constexpr int kTestCols = 32 * (kTestThreads / 128);

__device__ int g_tc_test_status;

__global__ void __launch_bounds__(kTestThreads) k_tc_dft16_test(const float2 *in, float2 *out, int nb, int inverse)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *a_hi = sm;
    unsigned char *a_lo = a_hi + kTestThreads * kTcRowBytes;
    unsigned char *f = a_lo + kTestThreads * kTcRowBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(f + 4 * kTcFBytes);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    uint32_t *phase = slot + 1;
    int *abort_flag = reinterpret_cast<int *>(phase + 1);

    tc_build_dft16(f, f + kTcFBytes, f + 2 * kTcFBytes, f + 3 * kTcFBytes);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *phase = 0;
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 32) tmem_alloc(slot, kTestCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcCtx ctx;
    ctx.a_hi = a_hi;
    ctx.a_lo = a_lo;
    ctx.f_hi[0] = f;
    ctx.f_lo[0] = f + kTcFBytes;
    ctx.f_hi[1] = f + 2 * kTcFBytes;
    ctx.f_lo[1] = f + 3 * kTcFBytes;
    ctx.tmem = *slot;
    ctx.bar = bar;
    ctx.phase = phase;
    ctx.abort = abort_flag;
    ctx.status = &g_tc_test_status;

    const long long id = (long long)blockIdx.x * kTestThreads + threadIdx.x;
    float2 a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = id < nb ? in[id * 16 + k] : make_float2(0.f, 0.f);
    if (inverse) tc_dft16<true>(a, ctx);
    else tc_dft16<false>(a, ctx);
    if (!*abort_flag && id < nb) {
#pragma unroll
        for (int k = 0; k < 16; ++k) out[id * 16 + k] = a[k];
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(ctx.tmem, kTestCols);
    }
}

} // namespace
} // namespace psolve

extern "C" psolve_status psolve_debug_tc_dft16(const void *in, void *out, int nbutterflies, int inverse,
                                               void *stream)
{
    using namespace psolve;
    if (!in || !out || nbutterflies <= 0) return PSOLVE_ERR_INVALID_ARG;
    const size_t smem = 2 * (size_t)kTestThreads * kTcRowBytes + 4 * kTcFBytes + 64;
    cudaError_t e = cudaFuncSetAttribute(k_tc_dft16_test, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return PSOLVE_ERR_CUDA;
    int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_test_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return PSOLVE_ERR_CUDA;
    const unsigned grid = (unsigned)((nbutterflies + kTestThreads - 1) / kTestThreads);
    k_tc_dft16_test<<<grid, kTestThreads, smem, (cudaStream_t)stream>>>((const float2 *)in, (float2 *)out,
                                                                       nbutterflies, inverse);
    e = cudaGetLastError();
    if (e != cudaSuccess) return PSOLVE_ERR_CUDA;
    int st = 0;
    e = cudaMemcpyFromSymbolAsync(&st, g_tc_test_status, sizeof(int), 0, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return PSOLVE_ERR_CUDA;
    return st == 0 ? PSOLVE_OK : (psolve_status)st;
}
