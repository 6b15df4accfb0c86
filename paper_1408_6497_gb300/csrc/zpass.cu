// z-direction passes: real rows <-> packed half-spectrum rows.
#include "launch.h"

namespace psolve {

template <typename T, int E, typename K>
static cudaError_t run(K kernel, const ZArgs<T> &a, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// Compile-time plans for the hot FP32 row lengths, the run-time plan otherwise.
#define PSOLVE_Z_DISPATCH(KERNEL)                                                   \
    if constexpr (sizeof(T) == 4) if (a.pl.E == 16 && !a.force_runtime) {                               \
        switch (a.pl.L) {                                                           \
        case 256: return run<T, 16>(KERNEL<T, 16, 256>, a, grid, block, smem, s);   \
        case 512: return run<T, 16>(KERNEL<T, 16, 512>, a, grid, block, smem, s);   \
        case 1024: return run<T, 16>(KERNEL<T, 16, 1024>, a, grid, block, smem, s); \
        default: break;                                                             \
        }                                                                           \
    }                                                                               \
    switch (a.pl.E) {                                                               \
    case 2: return run<T, 2>(KERNEL<T, 2, 0>, a, grid, block, smem, s);             \
    case 3: return run<T, 3>(KERNEL<T, 3, 0>, a, grid, block, smem, s);             \
    case 4: return run<T, 4>(KERNEL<T, 4, 0>, a, grid, block, smem, s);             \
    case 6: return run<T, 6>(KERNEL<T, 6, 0>, a, grid, block, smem, s);             \
    case 8: return run<T, 8>(KERNEL<T, 8, 0>, a, grid, block, smem, s);             \
    case 12: return run<T, 12>(KERNEL<T, 12, 0>, a, grid, block, smem, s);          \
    case 16: return run<T, 16>(KERNEL<T, 16, 0>, a, grid, block, smem, s);          \
    case 24: return run<T, 24>(KERNEL<T, 24, 0>, a, grid, block, smem, s);          \
    default: return cudaErrorInvalidValue;                                          \
    }

template <typename T>
cudaError_t launch_zfwd(const ZArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s)
{
    PSOLVE_Z_DISPATCH(k_zfwd)
}

template <typename T>
cudaError_t launch_zinv(const ZArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s)
{
    PSOLVE_Z_DISPATCH(k_zinv)
}

template cudaError_t launch_zfwd<float>(const ZArgs<float> &, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_zfwd<double>(const ZArgs<double> &, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_zinv<float>(const ZArgs<float> &, unsigned, unsigned, size_t, cudaStream_t);
template cudaError_t launch_zinv<double>(const ZArgs<double> &, unsigned, unsigned, size_t, cudaStream_t);

} // namespace psolve
