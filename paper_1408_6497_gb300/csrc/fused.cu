// z and y transforms of a plane in one launch (forward: z then y; inverse:
// y then z), so the spectrum of a plane makes its z→y hand-off through L2
// instead of a round trip to HBM.
//
// A thread-block cluster of C blocks owns one x-plane (ny rows of nz reals ⇔
// ny × M complex).  Phase 1: each block transforms every C-th row tile
// (forward) or column tile (inverse) of the plane and writes it back; a
// cluster barrier with release/acquire semantics then makes those writes
// visible to the whole cluster; phase 2: each block transforms every C-th
// tile of the other direction, reading the phase-1 results with L2-only
// loads.  With two blocks per SM and C = 4, about 76 planes (76 MiB at
// 512³) are in flight, which L2 holds, so the hand-off costs no HBM traffic
// beyond one read of the input and one write of the output.
#include "launch.h"

namespace psolve {

namespace {

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int EZ, int LZ, int EY, int LY, bool INV>
__global__ void __launch_bounds__(kFusedThreads, 2) k_zy(ZArgs<float> az, SArgs<float> ay, FusedArgs fa)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const unsigned r = cluster_rank();
    const long long plane = blockIdx.x / fa.cluster;
    if (!INV) {
        for (int i = (int)r; i < fa.ztiles; i += fa.cluster) {
            zfwd_tile<float, EZ, LZ, false>(az, az.in, az.out, plane * fa.ztiles + i, smraw);
            __syncthreads();
        }
        cluster_sync();
        for (int i = (int)r; i < fa.ytiles; i += fa.cluster) {
            ypass_tile<float, EY, false, LY, true>(ay, ay.data, plane * fa.ytiles + i, smraw);
            __syncthreads();
        }
    } else {
        for (int i = (int)r; i < fa.ytiles; i += fa.cluster) {
            ypass_tile<float, EY, true, LY, false>(ay, ay.data, plane * fa.ytiles + i, smraw);
            __syncthreads();
        }
        cluster_sync();
        for (int i = (int)r; i < fa.ztiles; i += fa.cluster) {
            zinv_tile<float, EZ, LZ, true>(az, az.in, az.out, plane * fa.ztiles + i, smraw);
            __syncthreads();
        }
    }
}

template <int EZ, int LZ, int EY, int LY>
cudaError_t run(const ZArgs<float> &az, const SArgs<float> &ay, const FusedArgs &fa, bool inverse, size_t smem,
                cudaStream_t s)
{
    auto kern = inverse ? k_zy<EZ, LZ, EY, LY, true> : k_zy<EZ, LZ, EY, LY, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(fa.planes * fa.cluster));
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)fa.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, az, ay, fa);
}

} // namespace

bool fused_supported(int M, int ny) { return (M == 256 || M == 512) && (ny == 256 || ny == 512 || ny == 1024); }

cudaError_t launch_fused_zy(const ZArgs<float> &az, const SArgs<float> &ay, const FusedArgs &fa, bool inverse,
                            size_t smem, cudaStream_t s)
{
#define PSOLVE_FUSED_Y(MM)                                                                   \
    switch (ay.pl.L) {                                                                       \
    case 256: return run<16, MM, 16, 256>(az, ay, fa, inverse, smem, s);                     \
    case 512: return run<16, MM, 16, 512>(az, ay, fa, inverse, smem, s);                     \
    case 1024: return run<16, MM, 16, 1024>(az, ay, fa, inverse, smem, s);                   \
    default: return cudaErrorInvalidValue;                                                   \
    }
    if (az.pl.E != 16 || ay.pl.E != 16) return cudaErrorInvalidValue;
    switch (az.M) {
    case 256: PSOLVE_FUSED_Y(256)
    case 512: PSOLVE_FUSED_Y(512)
    default: return cudaErrorInvalidValue;
    }
#undef PSOLVE_FUSED_Y
}

} // namespace psolve
