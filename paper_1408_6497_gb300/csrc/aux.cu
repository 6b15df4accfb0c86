// Set-up and diagnostic kernels: FP64 twiddle generation, the wavenumber
// export used by the bit-exact indexing test, and FP64 error norms.
#include "launch.h"

namespace psolve {

// dst[j] = e^{-2πi j/denom}: sincospi in FP64 (exact at multiples of 1/4
// turn), rounded once to T.
template <typename T>
__global__ void k_roots(typename cplx_of<T>::type *dst, int count, int denom)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)denom, &s, &c);
        dst[j] = {(T)c, (T)s};
    }
}

template <typename T> cudaError_t launch_roots(void *dst, int count, int denom, cudaStream_t s)
{
    using C = typename cplx_of<T>::type;
    if (count <= 0) return cudaSuccess;
    k_roots<T><<<(count + 255) / 256, 256, 0, s>>>(reinterpret_cast<C *>(dst), count, denom);
    return cudaGetLastError();
}
template cudaError_t launch_roots<float>(void *, int, int, cudaStream_t);
template cudaError_t launch_roots<double>(void *, int, int, cudaStream_t);

// The wavenumber triple of every half-spectrum index, with the same device
// function the division kernel uses.
__global__ void k_kvec(int *dst, int nx, int ny, int nz)
{
    const int H = nz / 2 + 1;
    const long long n = (long long)nx * ny * H;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int jz = (int)(i % H);
        const long long r = i / H;
        const int jy = (int)(r % ny);
        const int jx = (int)(r / ny);
        dst[3 * i + 0] = kvec_dev(jx, nx);
        dst[3 * i + 1] = kvec_dev(jy, ny);
        dst[3 * i + 2] = kvec_dev(jz, nz);
    }
}

cudaError_t launch_kvec(int *dst, int nx, int ny, int nz, cudaStream_t s)
{
    k_kvec<<<256, 256, 0, s>>>(dst, nx, ny, nz);
    return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    // Non-negative doubles order like their bit patterns.
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void k_norms(const T *__restrict__ a, const T *__restrict__ r, size_t n, double *out)
{
    double sd = 0.0, sr = 0.0, md = 0.0, mr = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)r[i];
        const double rv = (double)r[i];
        sd += d * d;
        sr += rv * rv;
        md = fmax(md, fabs(d));
        mr = fmax(mr, fabs(rv));
    }
    for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = sd;
        red[1][wid] = sr;
        red[2][wid] = md;
        red[3][wid] = mr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 1; k < nw; ++k) {
            sd += red[0][k];
            sr += red[1][k];
            md = fmax(md, red[2][k]);
            mr = fmax(mr, red[3][k]);
        }
        atomicAdd(out + 0, sd);
        atomicAdd(out + 1, sr);
        atomic_max_nonneg(out + 2, md);
        atomic_max_nonneg(out + 3, mr);
    }
}

template <typename T> cudaError_t launch_norms(const T *a, const T *ref, size_t n, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_norms<T><<<(unsigned)blocks, 256, 0, s>>>(a, ref, n, out);
    return cudaGetLastError();
}
template cudaError_t launch_norms<float>(const float *, const float *, size_t, double *, cudaStream_t);
template cudaError_t launch_norms<double>(const double *, const double *, size_t, double *, cudaStream_t);

} // namespace psolve
