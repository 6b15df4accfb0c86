// Host-side launchers of the pass kernels (one translation unit per pass kind,
// compiled in parallel).  Each picks the instantiation for E at run time.
#pragma once

#include "passes.cuh"

namespace psolve {

// Largest block the instantiation for (T, E) accepts (mirrors Bound<T, E>).
inline int max_threads(bool fp64, int E) { return (fp64 || E > 16) ? 256 : 512; }

// Points per thread the engine is instantiated for.
inline bool supported_E(int E)
{
    return E == 2 || E == 3 || E == 4 || E == 6 || E == 8 || E == 12 || E == 16 || E == 24;
}

template <typename T>
cudaError_t launch_zfwd(const ZArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_zinv(const ZArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_ypass(const SArgs<T> &a, bool inverse, unsigned grid, unsigned block, size_t smem,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_xfused(const XArgs<T> &a, unsigned grid, unsigned block, size_t smem, cudaStream_t s);

// Twiddles e^{-2πi j/denom}, j < count, computed in FP64 and rounded to T.
template <typename T>
cudaError_t launch_roots(void *dst, int count, int denom, cudaStream_t s);

// Signed wavenumbers of the half spectrum (nx, ny, nz/2+1) as int3 triples.
cudaError_t launch_kvec(int *dst, int nx, int ny, int nz, cudaStream_t s);

// FP64 sums and maxima of (a - ref) and ref into out[4] (device, zeroed by caller).
template <typename T>
cudaError_t launch_norms(const T *a, const T *ref, size_t n, double *out, cudaStream_t s);

} // namespace psolve
