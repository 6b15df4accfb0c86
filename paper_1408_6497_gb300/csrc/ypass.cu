// y-direction c2c passes over tiles of W adjacent kz-columns.
#include "launch.h"

namespace psolve {

template <typename T, typename K>
static cudaError_t run(K kernel, const SArgs<T> &a, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, bool INV>
static cudaError_t dispatch(const SArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s)
{
    // Compile-time plans for the hot FP32 line lengths.
    if constexpr (sizeof(T) == 4) if (a.pl.E == 16 && !a.force_runtime) {
        switch (a.pl.L) {
        case 256: return run(k_ypass<T, 16, INV, 256>, a, grid, block, smem, s);
        case 512: return run(k_ypass<T, 16, INV, 512>, a, grid, block, smem, s);
        case 1024: return run(k_ypass<T, 16, INV, 1024>, a, grid, block, smem, s);
        default: break;
        }
    }
    switch (a.pl.E) {
    case 2: return run(k_ypass<T, 2, INV, 0>, a, grid, block, smem, s);
    case 3: return run(k_ypass<T, 3, INV, 0>, a, grid, block, smem, s);
    case 4: return run(k_ypass<T, 4, INV, 0>, a, grid, block, smem, s);
    case 6: return run(k_ypass<T, 6, INV, 0>, a, grid, block, smem, s);
    case 8: return run(k_ypass<T, 8, INV, 0>, a, grid, block, smem, s);
    case 12: return run(k_ypass<T, 12, INV, 0>, a, grid, block, smem, s);
    case 16: return run(k_ypass<T, 16, INV, 0>, a, grid, block, smem, s);
    case 24: return run(k_ypass<T, 24, INV, 0>, a, grid, block, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_ypass(const SArgs<T> &a, bool inverse, unsigned grid, unsigned block, size_t smem,
                         cudaStream_t s)
{
    return inverse ? dispatch<T, true>(a, grid, block, smem, s) : dispatch<T, false>(a, grid, block, smem, s);
}

template cudaError_t launch_ypass<float>(const SArgs<float> &, bool, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_ypass<double>(const SArgs<double> &, bool, unsigned, unsigned, size_t, cudaStream_t);

} // namespace psolve
