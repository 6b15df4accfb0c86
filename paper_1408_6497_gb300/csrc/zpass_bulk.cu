// Persistent z passes fed by 1D bulk copies, FP32 rows of M = 64, 128, 256
// or 512 complex points (nz = 128 … 1024).
//
// A tile is W consecutive rows (W·nz reals, contiguous in HBM), 32 KiB; one
// cp.async.bulk brings tile i+1 into shared memory while tile i is being
// transformed (two buffers, two mbarriers, time-bounded waits).  Threads read
// their strided class of a row from the tile (conflict-free: a row is
// contiguous), exchange through a padded buffer (a spare slot every 16
// points), and store the result row straight from registers.
//   forward: real row -> M-point FFT -> split post-twiddle -> packed row
//   inverse: packed row -> pre-twiddle merge -> inverse FFT -> real row
#include "psolve.h"
#include "launch.h"
#include "tma.cuh"

namespace psolve {

namespace {

constexpr uint64_t kZWaitNs = 2000000000ull;

// M = 64, 128, 256: 16 points per thread (radix 16 × 4, 16 × 8, 16 × 16);
// M = 512: 32 points per thread (radix 32 × 16: one exchange instead of two).
// Threads per block (measured on GB300 at 512³): the forward pass runs best
// as 128-thread blocks four per SM (16 KiB tiles), the inverse as 256-thread
// blocks two per SM (32 KiB tiles); M = 512 uses 128 threads two per SM.
constexpr int zb_threads(int M, bool inv) { return M >= 512 ? 128 : (inv ? 256 : 128); }
constexpr int zb_blocks(int M, bool inv) { return M >= 512 ? 2 : 512 / zb_threads(M, inv); }
template <int M, bool INV> struct ZShape {
    static constexpr int E = M >= 512 ? 32 : 16;
    static constexpr int TL = M / E;
    static constexpr int NT = zb_threads(M, INV);
    static constexpr int MINB = zb_blocks(M, INV);
    static constexpr int SH = E >= 32 ? 5 : 4;              // exchange padding period
    static constexpr int W = NT / TL;                       // rows per tile
    static constexpr int LP = M + (M >> 4) + 1;             // padded row pitch (complex)
    static constexpr uint32_t TILE_BYTES = (uint32_t)(W * M * 8);
};

template <int M, bool INV>
__global__ void __launch_bounds__(ZShape<M, INV>::NT, ZShape<M, INV>::MINB) k_z_bulk(ZBulkArgs a)
{
    using S = ZShape<M, INV>;
    constexpr int E = S::E, TL = S::TL, W = S::W;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *buf0 = reinterpret_cast<float2 *>(smraw);
    float2 *buf1 = buf0 + W * M;
    float2 *xb = buf1 + W * M;                 // W padded rows
    float2 *stw = xb + W * S::LP;              // e^{-2πij/M}
    float2 *spost = stw + M;                   // e^{-2πik/nz}, k < M
    uint64_t *bar = reinterpret_cast<uint64_t *>(spost + M);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const int w = tid / TL, t = tid - w * TL;
    const long long ntiles = a.rows / W;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < M; i += blockDim.x) {
        stw[i] = a.tw[i];
        spost[i] = a.post[i];
    }
    __syncthreads();
    const float *src = INV ? reinterpret_cast<const float *>(a.spec) : a.real_in;
    auto issue = [&](long long tile, float2 *dst, uint64_t *b) {
        mbar_expect_tx(b, S::TILE_BYTES);
        bulk_load(dst, src + tile * (long long)W * (2 * M), S::TILE_BYTES, b);
    };
    long long tile = blockIdx.x;
    // Set-up above may overlap the previous pass's last blocks; its output is
    // read only from here on.
    grid_dependency_wait();
    if (tid == 0 && tile < ntiles) issue(tile, buf0, &bar[0]);
    const MapRow<S::SH> xm{w * S::LP};

    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        float2 *cur = (k & 1) ? buf1 : buf0;
        const long long next = tile + gridDim.x;
        if (tid == 0) {
            if (next < ntiles) {
                fence_proxy_async_smem();
                issue(next, (k & 1) ? buf0 : buf1, &bar[(k + 1) & 1]);
            }
            if (!mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), kZWaitNs)) {
                *abort_flag = 1;
                atomicExch(a.status, (int)PSOLVE_ERR_TIMEOUT);
                if (next < ntiles) mbar_wait_bounded(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), kZWaitNs);
            }
        }
        __syncthreads();
        if (*abort_flag) break;

        // forward: tile rows are rows of f (natural order); inverse: rows of
        // the spectrum (x-split order), written back to their natural row
        const long long row = tile * W + w;
        const float2 *rowp = cur + w * M;
        float2 v[E];
        if (!INV) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = rowp[t + m * TL];
            line_fft_ct_from<false, M, 0>(v, t, stw, xb, xm, true);
            // Z[k] -> X[k] needs Z[M-k]
#pragma unroll
            for (int m = 0; m < E; ++m) xb[xm(t + m * TL)] = v[m];
            __syncthreads();
            const long long srow = a.G > 1 ? spec_row(row / a.ny, row % a.ny, a.ny, a.G) : row;
            float2 *dst = reinterpret_cast<float2 *>(a.spec) + srow * M;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kk = t + m * TL;
                const float2 z = v[m];
                if (kk == 0) {
                    dst[0] = make_float2(z.x + z.y, z.x - z.y);
                } else {
                    const float2 zp = xb[xm(M - kk)];
                    const float2 e = make_float2((z.x + zp.x) * 0.5f, (z.y - zp.y) * 0.5f);
                    const float2 o = make_float2((z.y + zp.y) * 0.5f, (zp.x - z.x) * 0.5f);
                    dst[kk] = cadd(e, cmul(o, spost[kk]));
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kk = t + m * TL;
                const float2 x = rowp[kk];
                if (kk == 0) {
                    v[m] = make_float2(x.x + x.y, x.x - x.y);
                } else {
                    const float2 xp = rowp[M - kk];
                    const float2 e = make_float2(x.x + xp.x, x.y - xp.y);
                    const float2 o = cmulc(make_float2(x.x - xp.x, x.y + xp.y), spost[kk]);
                    v[m] = make_float2(e.x - o.y, e.y + o.x);
                }
            }
            line_fft_ct_from<true, M, 0>(v, t, stw, xb, xm, true);
            long long nrow = row;
            if (a.G > 1) {
                const long long q = row / a.G;
                nrow = ((q / a.ny) * a.G + row % a.G) * a.ny + q % a.ny;
            }
            float2 *dst = reinterpret_cast<float2 *>(a.real_out + nrow * (2 * M)) + t;
#pragma unroll
            for (int m = 0; m < E; ++m) dst[m * TL] = v[m];
        }
        __syncthreads(); // `cur` and `xb` are free for the next tile
    }
}

template <int M, bool INV> cudaError_t run(const ZBulkArgs &a, unsigned grid, cudaStream_t s, bool pdl)
{
    using S = ZShape<M, INV>;
    const size_t smem = z_bulk_smem(M, INV);
    auto kern = k_z_bulk<M, INV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(S::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {programmatic_serialization()};
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

} // namespace

bool z_bulk_supported(int M) { return M == 64 || M == 128 || M == 256 || M == 512; }

int z_bulk_rows(int M, bool inverse) { return zb_threads(M, inverse) / (M / (M >= 512 ? 32 : 16)); }

int z_bulk_blocks_per_sm(int M, bool inverse) { return zb_blocks(M, inverse); }

size_t z_bulk_smem(int M, bool inverse)
{
    const int W = z_bulk_rows(M, inverse);
    const int LP = M + (M >> 4) + 1;
    return (size_t)(2 * W * M + W * LP + 2 * M) * 8 + 2 * 8 + 16;
}

cudaError_t launch_z_bulk(const ZBulkArgs &a, int M, bool inverse, unsigned grid, cudaStream_t s, bool pdl)
{
    if (M == 64) return inverse ? run<64, true>(a, grid, s, pdl) : run<64, false>(a, grid, s, pdl);
    if (M == 128) return inverse ? run<128, true>(a, grid, s, pdl) : run<128, false>(a, grid, s, pdl);
    if (M == 256) return inverse ? run<256, true>(a, grid, s, pdl) : run<256, false>(a, grid, s, pdl);
    if (M == 512) return inverse ? run<512, true>(a, grid, s, pdl) : run<512, false>(a, grid, s, pdl);
    return cudaErrorInvalidValue;
}

} // namespace psolve
