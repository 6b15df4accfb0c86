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
    switch (a.pl.E) {
    case 2: return run(k_xfused<T, 2>, a, grid, block, smem, s);
    case 3: return run(k_xfused<T, 3>, a, grid, block, smem, s);
    case 4: return run(k_xfused<T, 4>, a, grid, block, smem, s);
    case 6: return run(k_xfused<T, 6>, a, grid, block, smem, s);
    case 8: return run(k_xfused<T, 8>, a, grid, block, smem, s);
    case 12: return run(k_xfused<T, 12>, a, grid, block, smem, s);
    case 16: return run(k_xfused<T, 16>, a, grid, block, smem, s);
    case 24: return run(k_xfused<T, 24>, a, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_xfused<float>(const XArgs<float> &, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_xfused<double>(const XArgs<double> &, unsigned, unsigned, size_t, cudaStream_t);

} // namespace psolve
