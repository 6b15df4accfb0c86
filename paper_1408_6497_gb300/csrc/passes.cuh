// The five pass kernels of one solve (§2.1, §3: forward 3D FFT, diagonal
// scaling by the inverse Laplacian symbol, inverse 3D FFT), as templates over
// the precision T and the points-per-thread E.
//
// Data layout.  f and u are real (nx, ny, nz), z contiguous.  The half
// spectrum is formed inside u's own bytes as complex S[x][y][kz],
// 0 <= kz < M = nz/2: a row of nz reals and a row of M complex values have
// the same size, so every pass works in place and no workspace of the grid's
// size exists.  The z-Nyquist coefficient X[M] of a real z-line is real, as
// is X[0]; the pair is packed into slot 0 as X[0] + i·X[M].  The y and x
// transforms act linearly on that packed column, and the x-pass separates
// the two real-signal spectra with the mirror row (-ky) before scaling them.
//
//   zfwd   : real rows -> packed complex rows (M-point FFT + split post-twiddle)
//   ypass  : c2c along y, tiles of W adjacent kz-columns at fixed x
//   xfused : c2c along x, scale by 1/(4π²|k|²N), inverse c2c along x; extra
//            blocks handle the packed kz = 0 / kz = M column pairs
//   zinv   : packed complex rows -> real rows (pre-twiddle + M-point FFT)
#pragma once

#include "fft_core.cuh"

#ifndef PSOLVE_CT_MINB
#define PSOLVE_CT_MINB 2
#endif

namespace psolve {

template <typename T> struct ZArgs {
    using C = typename cplx_of<T>::type;
    const T *in;      // zfwd: f;  zinv: packed spectrum
    T *out;           // zfwd: packed spectrum;  zinv: u
    long long rows;   // lines of nz reals
    int nz, M, W;     // W rows per block
    LinePlan pl;      // L = M
    const C *tw;      // e^{-2πi j/M}, j < M
    const C *post;    // e^{-2πi k/nz}, k < M
    int force_runtime; // host dispatch: 1 = run-time stage plan even for hot lengths
};

template <typename T> struct SArgs {
    using C = typename cplx_of<T>::type;
    T *data;          // packed spectrum
    long long nplanes;
    long long sPlane; // complex elements between planes
    long long sL;     // complex elements between points of a line
    int M, W, ncb;    // columns per row, columns per tile, tiles per plane
    LinePlan pl;
    const C *tw;
    int force_runtime;
};

// The solve's spectral multiplier (the step between the forward and inverse
// transforms): û(k) = coef · F[f](k) / den(k), coef = 1/(4π²N), with
//   op 0, Poisson −Δu = f (§2.1):      den = |k|²          (0 at k = 0: mean dropped)
//   op 1, Helmholtz −Δu + c·u = f:     den = |k|² + c/(4π²), c > 0
//   op 2, the second-order 7-point finite-difference Laplacian, whose
//         eigenvalues diagonalise the same way (the stencil variant of §1):
//         den = Λx(jx) + Λy(jy) + Λz(jz), Λ(j) = (n/π)² sin²(π j/n)
// (den = 0 gives 0).  lx, ly, lz: device tables of Λ per index (z: kz ≤ M),
// in FP64 and rounded to FP32 (each kernel reads its own precision: the FP32
// passes do no FP64 arithmetic).
struct OpArgs {
    int op;
    double c4;                        // op 1: c/(4π²)
    const double *lx, *ly, *lz;       // op 2
    const float *lx32, *ly32, *lz32;
};

template <typename T> __device__ __forceinline__ const T *op_table(const double *d, const float *f);
template <> __device__ __forceinline__ const double *op_table<double>(const double *d, const float *) { return d; }
template <> __device__ __forceinline__ const float *op_table<float>(const double *, const float *f) { return f; }

template <typename T>
__device__ __forceinline__ T op_den(const OpArgs &o, int kx, int ky, int kz, int jx, int jy, int jz)
{
    if (o.op == 1) return (T)(kx * kx + ky * ky + kz * kz) + (T)o.c4;
    if (o.op == 2)
        return op_table<T>(o.lx, o.lx32)[jx] + op_table<T>(o.ly, o.ly32)[jy] + op_table<T>(o.lz, o.lz32)[jz];
    return (T)(kx * kx + ky * ky + kz * kz);
}

template <typename T> struct XArgs {
    using C = typename cplx_of<T>::type;
    T *data;
    int batch, nx, ny, M;
    long long sInst;     // complex elements between instances
    int W, ncb;
    long long main_tiles;
    long long npairs;    // batch · (ny/2 + 1)
    LinePlan pl;         // L = nx
    const C *tw;
    T coef;              // 1 / (4π² N), N = nx·ny·nz
    OpArgs op;           // spectral multiplier (op 0: Poisson)
    int force_runtime;
};

// Launch bound per instantiation: the host mirrors this in max_threads().
// Compile-time-plan (LC > 0) FP32 kernels ask for two resident blocks.
template <typename T, int E, int LC> struct Bound {
    static constexpr int value = (sizeof(T) == 8 || E > 16) ? 256 : 512;
    static constexpr int minb = (LC > 0 && sizeof(T) == 4) ? PSOLVE_CT_MINB : 1;
};

// Global loads of the pass data.  CG = true bypasses L1 (ld.global.cg): the
// batched persistent kernel reads data that other blocks wrote earlier in
// the same launch, which a stale L1 line could otherwise hide.
template <bool CG, typename C> __device__ __forceinline__ C ld_data(const C *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Every tile function below is called by all threads of a block (it
// synchronises); threads beyond the tile's W·TL lanes are idle.  `smem` is
// the block's dynamic shared memory: the line's twiddle table, then the
// exchange buffer.  `hook` is called once by every thread as soon as the
// tile's global loads are issued, before the first barrier: the persistent
// batched kernel schedules its next item there, while the loads are in
// flight; the one-pass kernels pass the no-op.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// --------------------------------------------------------------- z forward
template <typename T, int E, int LC, bool CG = false, class Hook = NoHook>
__device__ __forceinline__ void zfwd_tile(const ZArgs<T> &a, const T *in, T *out, long long tile,
                                          unsigned char *smem, const Hook &hook = Hook())
{
    using C = typename cplx_of<T>::type;
    C *stw = reinterpret_cast<C *>(smem);
    const int M = LC > 0 ? LC : a.M;
    C *sx = stw + M;
    const int TL = LC > 0 ? LC / E : a.pl.TL;
    const int tid = threadIdx.x;
    const int w = tid / TL, t = tid - w * TL;
    const long long row = tile * a.W + w;
    const bool active = (w < a.W) && (row < a.rows);
    for (int i = tid; i < M; i += blockDim.x) stw[i] = a.tw[i];
    C v[E];
    if (active) {
        const C *src = reinterpret_cast<const C *>(in + row * (2 * M)) + t;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld_data<CG>(src + m * TL);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = C{0, 0};
    }
    hook();
    __syncthreads();
    const int LP = M + (M >> 4) + 1;
    const MapRow<> map{w * LP};
    line_fft_any<false, LC>(v, t, a.pl, stw, sx, map, active);
    // Z[k] -> X[k] needs Z[M-k]: exchange through shared memory.
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) sx[map(t + m * TL)] = v[m];
    }
    __syncthreads();
    if (active) {
        C *dst = reinterpret_cast<C *>(out) + row * M;
        const T half = (T)0.5;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + m * TL;
            const C z = v[m];
            if (k == 0) {
                dst[0] = C{z.x + z.y, z.x - z.y}; // X[0] + i X[M]
            } else {
                const C zp = sx[map(M - k)];
                const C e = {(z.x + zp.x) * half, (z.y - zp.y) * half};   // (Z + conj Zp)/2
                const C o = {(z.y + zp.y) * half, (zp.x - z.x) * half};   // (Z - conj Zp)/(2i)
                dst[k] = cadd(e, cmul(o, a.post[k]));
            }
        }
    }
}

// --------------------------------------------------------------- z inverse
template <typename T, int E, int LC, bool CG = false, class Hook = NoHook>
__device__ __forceinline__ void zinv_tile(const ZArgs<T> &a, const T *in, T *out, long long tile,
                                          unsigned char *smem, const Hook &hook = Hook())
{
    using C = typename cplx_of<T>::type;
    C *stw = reinterpret_cast<C *>(smem);
    const int M = LC > 0 ? LC : a.M;
    C *sx = stw + M;
    const int TL = LC > 0 ? LC / E : a.pl.TL;
    const int tid = threadIdx.x;
    const int w = tid / TL, t = tid - w * TL;
    const long long row = tile * a.W + w;
    const bool active = (w < a.W) && (row < a.rows);
    for (int i = tid; i < M; i += blockDim.x) stw[i] = a.tw[i];
    C v[E];
    const int LP = M + (M >> 4) + 1;
    const MapRow<> map{w * LP};
    if (active) {
        const C *src = reinterpret_cast<const C *>(in) + row * M + t;
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld_data<CG>(src + m * TL);
    }
    hook();
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) sx[map(t + m * TL)] = v[m];
    }
    __syncthreads(); // the whole row is in registers and shared memory (in place)
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = t + m * TL;
            const C x = v[m];
            if (k == 0) {
                v[m] = C{x.x + x.y, x.x - x.y};
            } else {
                const C xp = sx[map(M - k)];
                const C e = {x.x + xp.x, x.y - xp.y};                  // X + conj Xp
                const C o = cmulc(C{x.x - xp.x, x.y + xp.y}, a.post[k]); // (X - conj Xp) e^{+2πik/nz}
                v[m] = C{e.x - o.y, e.y + o.x};                        // E + i O
            }
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = C{0, 0};
    }
    __syncthreads(); // partner reads done before the transform reuses the buffer
    line_fft_any<true, LC>(v, t, a.pl, stw, sx, map, active);
    if (active) {
        C *dst = reinterpret_cast<C *>(out + row * (2 * M)) + t;
#pragma unroll
        for (int m = 0; m < E; ++m) dst[m * TL] = v[m];
    }
}

// ------------------------------------------------------- strided c2c (y)
template <typename T, int E, bool INV, int LC, bool CG = false, class Hook = NoHook>
__device__ __forceinline__ void ypass_tile(const SArgs<T> &a, T *data, long long tile, unsigned char *smem,
                                           const Hook &hook = Hook())
{
    using C = typename cplx_of<T>::type;
    C *stw = reinterpret_cast<C *>(smem);
    const int L = LC > 0 ? LC : a.pl.L;
    C *sx = stw + L;
    const int W = a.W, TL = LC > 0 ? LC / E : a.pl.TL;
    const int tid = threadIdx.x;
    const int w = tid % W, t = tid / W;
    const int cb = (int)(tile % a.ncb);
    const long long plane = tile / a.ncb;
    const int col = cb * W + w;
    const bool active = (col < a.M) && (t < TL);
    for (int i = tid; i < L; i += blockDim.x) stw[i] = a.tw[i];
    C *base = reinterpret_cast<C *>(data) + plane * a.sPlane + col + (long long)t * a.sL;
    const long long step = (long long)TL * a.sL;
    C v[E];
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld_data<CG>(base + m * step);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = C{0, 0};
    }
    hook();
    __syncthreads();
    const MapStrided map{W, w};
    line_fft_any<INV, LC>(v, t, a.pl, stw, sx, map, active);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[m * step] = v[m];
    }
}

// Packed column kz = 0 holds X0 + i·XM for every (x, y) line.  After the
// 2D (y, x) transform H = G0 + i·G1 with G0, G1 the spectra of two real
// planes, so G0(k) = (H(k) + conj H(-k))/2, G1(k) = (H(k) - conj H(-k))/(2i).
// Each is scaled by its own symbol (kz = 0 and kz = M) and recombined:
//   H'(k) = ((D0 + D1)/2) H(k) + ((D0 - D1)/2) conj H(-k).
// Lines 2q and 2q+1 of the block hold rows ky and (ny - ky) mod ny; block
// `pidx` takes pairs pidx·(W/2) .. pidx·(W/2) + W/2 - 1.  All threads of the
// block must call it (it synchronises).
// G: x-split factor of the spectrum layout (1: natural; else TL % G == 0).
// OPS = false: the Poisson multiplier only (op is not read).
template <typename T, int E, int LC, bool CG = false, bool OPS = true, class Hook = NoHook>
__device__ __forceinline__ void xpair_block(T *data, int nx_rt, int ny, int M, long long sInst, long long npairs,
                                            T coef, const OpArgs &op, const LinePlan &pl, int W, int TL,
                                            long long pidx, int t,
                                            int w, const typename cplx_of<T>::type *stw,
                                            typename cplx_of<T>::type *sx, int G = 1, const Hook &hook = Hook())
{
    using C = typename cplx_of<T>::type;
    const int nx = LC > 0 ? LC : nx_rt;
    const long long sL = (long long)ny * M;
    const long long step = (long long)TL * sL;
    const MapStrided map{W, w};
    C v[E];
    const int half = W >> 1;
    const int q = w >> 1, side = w & 1;
    const long long pair = pidx * half + q;
    const bool active = (w < 2 * half) && (pair < npairs) && (t < TL);
    const int per = ny / 2 + 1;
    const long long b = active ? pair / per : 0;
    const int ky = active ? (int)(pair % per) : 0;
    const int row = side ? (ny - ky) % ny : ky;
    // point x = t + m·TL of row `row`: spec_row(x, row) with x / G = t / G + m·TL / G
    C *base = reinterpret_cast<C *>(data) + b * sInst + (long long)row * G * M +
              ((long long)(t / G) * ny * G + t % G) * M;
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld_data<CG>(base + m * step);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = C{0, 0};
    }
    hook();
    __syncthreads();
    line_fft_any<false, LC>(v, t, pl, stw, sx, map, active);
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) sx[map(t + m * TL)] = v[m];
    }
    __syncthreads();
    if (active) {
        const int kys = kvec_dev(row, ny);
        const int partner = w ^ 1;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int jx = t + m * TL;
            const int jm = (jx == 0) ? 0 : nx - jx;
            const C h1 = v[m];
            const C h2 = sx[jm * W + partner];
            const int kx = kvec_dev(jx, nx);
            // symbols of the two real planes kz = 0 and kz = M
            T den0, den1;
            if constexpr (OPS) {
                den0 = op_den<T>(op, kx, kys, 0, jx, row, 0);
                den1 = op_den<T>(op, kx, kys, M, jx, row, M);
            } else {
                den0 = (T)(kx * kx + kys * kys);
                den1 = (T)(kx * kx + kys * kys + M * M);
            }
            const T d0 = (den0 == (T)0) ? (T)0 : coef / den0;
            const T d1 = coef / den1;
            const T sp = (d0 + d1) * (T)0.5, sm = (d0 - d1) * (T)0.5;
            v[m] = C{sp * h1.x + sm * h2.x, sp * h1.y - sm * h2.y};
        }
    }
    __syncthreads();
    line_fft_any<true, LC>(v, t, pl, stw, sx, map, active);
    if (active && !(side == 1 && row == ky)) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[m * step] = v[m];
    }
}

// ----------------------------------- x forward, spectral division, x inverse
// Tiles [0, main_tiles) are (instance, y, column block); the following ones
// are groups of packed-column pairs.
template <typename T, int E, int LC, bool CG = false, class Hook = NoHook>
__device__ __forceinline__ void xfused_tile(const XArgs<T> &a, T *data, long long tile, unsigned char *smem,
                                            const Hook &hook = Hook())
{
    using C = typename cplx_of<T>::type;
    C *stw = reinterpret_cast<C *>(smem);
    const int nx = LC > 0 ? LC : a.nx;
    C *sx = stw + nx;
    const int W = a.W, TL = LC > 0 ? LC / E : a.pl.TL, ny = a.ny, M = a.M;
    const int tid = threadIdx.x;
    const int w = tid % W, t = tid / W;
    const long long sL = (long long)ny * M;
    const long long step = (long long)TL * sL;
    for (int i = tid; i < nx; i += blockDim.x) stw[i] = a.tw[i];
    const MapStrided map{W, w};

    if (tile >= a.main_tiles) {
        xpair_block<T, E, LC, CG, true, Hook>(data, nx, ny, M, a.sInst, a.npairs, a.coef, a.op, a.pl, W, TL,
                                              tile - a.main_tiles, t, w, stw, sx, 1, hook);
        return;
    }
    C v[E];
    const int cb = (int)(tile % a.ncb);
    const long long rest = tile / a.ncb;
    const int y = (int)(rest % ny);
    const long long b = rest / ny;
    const int col = cb * W + w;
    const bool active = (col < M) && (t < TL);
    C *base = reinterpret_cast<C *>(data) + b * a.sInst + (long long)y * M + col + (long long)t * sL;
    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = ld_data<CG>(base + m * step);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = C{0, 0};
    }
    hook();
    __syncthreads();
    line_fft_any<false, LC>(v, t, a.pl, stw, sx, map, active);
    const int ky = kvec_dev(y, ny);
    if (a.op.op == 0) {
        const int kyz = ky * ky + col * col;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int kx = kvec_dev(t + m * TL, nx);
            const int k2 = kx * kx + kyz;
            const T d = (k2 == 0) ? (T)0 : a.coef / (T)k2;
            v[m] = cscale(v[m], d);
        }
    } else if (a.op.op == 1) {
        const T c4 = (T)a.op.c4;
        const int kyz = ky * ky + col * col;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int kx = kvec_dev(t + m * TL, nx);
            v[m] = cscale(v[m], a.coef / ((T)(kx * kx + kyz) + c4));
        }
    } else if (active) {
        const T *lx = op_table<T>(a.op.lx, a.op.lx32);
        const T lyz = op_table<T>(a.op.ly, a.op.ly32)[y] + op_table<T>(a.op.lz, a.op.lz32)[col];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const T den = lx[t + m * TL] + lyz;
            v[m] = cscale(v[m], (den == (T)0) ? (T)0 : a.coef / den);
        }
    }
    line_fft_any<true, LC>(v, t, a.pl, stw, sx, map, active);
    if (active && col != 0) {
#pragma unroll
        for (int m = 0; m < E; ++m) base[m * step] = v[m];
    }
}

// ------------------------------------------------------- one-pass kernels
template <typename T, int E, int LC>
__global__ void __launch_bounds__(Bound<T, E, LC>::value, Bound<T, E, LC>::minb) k_zfwd(ZArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    zfwd_tile<T, E, LC>(a, a.in, a.out, blockIdx.x, smraw);
}

template <typename T, int E, int LC>
__global__ void __launch_bounds__(Bound<T, E, LC>::value, Bound<T, E, LC>::minb) k_zinv(ZArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    zinv_tile<T, E, LC>(a, a.in, a.out, blockIdx.x, smraw);
}

template <typename T, int E, bool INV, int LC>
__global__ void __launch_bounds__(Bound<T, E, LC>::value, Bound<T, E, LC>::minb) k_ypass(SArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    ypass_tile<T, E, INV, LC>(a, a.data, blockIdx.x, smraw);
}

template <typename T, int E, int LC>
__global__ void __launch_bounds__(Bound<T, E, LC>::value, Bound<T, E, LC>::minb) k_xfused(XArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    xfused_tile<T, E, LC>(a, a.data, blockIdx.x, smraw);
}

} // namespace psolve
