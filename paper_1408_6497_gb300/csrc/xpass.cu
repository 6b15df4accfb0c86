// x-direction pass with the spectral division fused between the transforms.
#include "launch.h"

namespace psolve {

template <typename T, typename K>
static cudaError_t run(K kernel, const XArgs<T> &a, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xfused(const XArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s)
{
    // Compile-time plans for the hot FP32 line lengths.
    if constexpr (sizeof(T) == 4) if (a.pl.E == 16 && !a.force_runtime) {
        switch (a.pl.L) {
        case 256: return run(k_xfused<T, 16, 256>, a, grid, block, smem, s);
        case 512: return run(k_xfused<T, 16, 512>, a, grid, block, smem, s);
        case 1024: return run(k_xfused<T, 16, 1024>, a, grid, block, smem, s);
        default: break;
        }
    }
    switch (a.pl.E) {
    case 2: return run(k_xfused<T, 2, 0>, a, grid, block, smem, s);
    case 3: return run(k_xfused<T, 3, 0>, a, grid, block, smem, s);
    case 4: return run(k_xfused<T, 4, 0>, a, grid, block, smem, s);
    case 6: return run(k_xfused<T, 6, 0>, a, grid, block, smem, s);
    case 8: return run(k_xfused<T, 8, 0>, a, grid, block, smem, s);
    case 12: return run(k_xfused<T, 12, 0>, a, grid, block, smem, s);
    case 16: return run(k_xfused<T, 16, 0>, a, grid, block, smem, s);
    case 24: return run(k_xfused<T, 24, 0>, a, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_xfused<float>(const XArgs<float> &, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_xfused<double>(const XArgs<double> &, unsigned, unsigned, size_t, cudaStream_t);

} // namespace psolve
