// Persistent, TMA-fed y and x passes for FP32 lines of 256, 512 or 1024 points.
//
// One block per SM walks the tile list.  A tile is L points × W adjacent
// kz-columns (64 KiB: W = 8192 / L), fetched by the Tensor Memory
// Accelerator straight into shared memory while the previous tile is being
// transformed, so HBM reads overlap the butterflies (double buffering with
// two mbarriers).  The transform runs in place in the tile's buffer with the
// same register/shared-memory Stockham engine as the other passes; results go
// back to HBM from registers.  The x kind adds the spectral division between
// its forward and inverse transforms (§2.1: Hadamard product with the inverse
// Laplacian symbol) and, after its main tiles, the packed kz = 0 / kz = M
// column pairs.
#include "psolve.h"
#include "launch.h"
#include "tma.cuh"

namespace psolve {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull; // 2 s per copy, then PSOLVE_ERR_TIMEOUT

// NARROW = 0: 64 KiB tiles (W = 8192/L columns, 512 threads, one block per
// SM); NARROW = 1: 32 KiB tiles (half the columns, 256 threads, two blocks per
// SM, so one block's barriers overlap the other's butterflies).
// CFG 2: as NARROW but 8 points per thread (twice the threads, about half
// the registers each), so 32 warps per SM hide the barrier and shared-memory
// latencies of the butterflies.
template <int L, int CFG> struct TmaShape {
    static constexpr int NARROW = CFG > 0 ? 1 : 0;
    static constexpr int E = CFG == 2 ? 8 : 16;
    static constexpr int TL = L / E;
    static constexpr int W = (8192 / L) >> NARROW;  // columns per tile
    static constexpr int NT = W * TL;               // threads per block
    static constexpr int MINB = NARROW ? 2 : 1;
    static constexpr int BOXR = L < 256 ? L : 256;  // rows per TMA box
    static constexpr int NLOAD = L / BOXR;
    static constexpr uint32_t TILE_BYTES = (uint32_t)(L * W * 8);
};

// KIND: 0 = y forward, 1 = y inverse, 2 = x forward + division + x inverse.
template <int L, int KIND, int CFG>
__global__ void __launch_bounds__(TmaShape<L, CFG>::NT, TmaShape<L, CFG>::MINB)
    k_strided_tma(const __grid_constant__ CUtensorMap tmap, TmaArgs a)
{
    using S = TmaShape<L, CFG>;
    constexpr int E = S::E, TL = S::TL, W = S::W;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *buf0 = reinterpret_cast<float2 *>(smraw);
    float2 *buf1 = buf0 + L * W;
    float2 *xbuf = buf1 + L * W; // exchange buffer alternating with the tile's own
    float2 *stw = xbuf + L * W;
    uint64_t *bar = reinterpret_cast<uint64_t *>(stw + L);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const int w = tid % W, t = tid / W;
    const long long ntiles = a.main_tiles;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmap);
    }
    for (int i = tid; i < L; i += blockDim.x) stw[i] = a.tw[i];
    __syncthreads();

    // Tile -> TMA coordinates (c0 = first column, c1, c2 of the first row).
    auto issue = [&](long long tile, float2 *dst, uint64_t *b) {
        const int cb = (int)(tile % a.ncb);
        const long long rest = tile / a.ncb;
        mbar_expect_tx(b, S::TILE_BYTES);
#pragma unroll
        for (int r = 0; r < S::NLOAD; ++r) {
            if (KIND == 2) {
                const int y = (int)(rest % a.ny);
                const long long inst = rest / a.ny;
                tma_load_3d(dst + r * S::BOXR * W, &tmap, b, cb * W, y, (int)(inst * L + r * S::BOXR));
            } else {
                tma_load_3d(dst + r * S::BOXR * W, &tmap, b, cb * W, r * S::BOXR, (int)rest);
            }
        }
    };

    long long tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) issue(tile, buf0, &bar[0]);

    const MapStrided map{W, w};
    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        float2 *cur = (k & 1) ? buf1 : buf0;
        const long long next = tile + gridDim.x;
        if (tid == 0) {
            if (next < ntiles) {
                // The other buffer was released by the barrier that ended the
                // previous iteration; order those generic accesses before TMA.
                fence_proxy_async_smem();
                issue(next, (k & 1) ? buf0 : buf1, &bar[(k + 1) & 1]);
            }
            if (!mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), kWaitLimitNs)) {
                *abort_flag = 1;
                atomicExch(a.status, (int)PSOLVE_ERR_TIMEOUT);
                // Let the copy already issued for `next` land before leaving.
                if (next < ntiles) mbar_wait_bounded(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), kWaitLimitNs);
            }
        }
        __syncthreads();
        if (*abort_flag) return;

        const int cb = (int)(tile % a.ncb);
        const long long rest = tile / a.ncb;
        const int col = cb * W + w;
        const bool active = col < a.M;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cur[(t + m * TL) * W + w];
        // Exchanges alternate xbuf, cur, xbuf, ...: the first writes go to
        // xbuf, so the tile reads above need no barrier of their own.
        line_fft_ct_db<KIND == 1, L, 0, 0>(v, t, stw, xbuf, cur, map);

        float2 *base;
        long long step;
        if (KIND == 2) {
            const int y = (int)(rest % a.ny);
            const long long inst = rest / a.ny;
            const int ky = kvec_dev(y, a.ny);
            const int kyz = ky * ky + col * col;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kx = kvec_dev(t + m * TL, L);
                const int k2 = kx * kx + kyz;
                // coef·(1/k²) with the hardware reciprocal: about 2 ulp in FP32
                const float d = (k2 == 0) ? 0.f : __fdividef(a.coef, (float)k2);
                v[m] = cscale(v[m], d);
            }
            // Continue the alternation where the forward transform left it.
            constexpr int PAR = ct_exchanges(L, E) & 1;
            line_fft_ct_db<true, L, 0, PAR>(v, t, stw, xbuf, cur, map);
            step = (long long)TL * a.ny * a.M;
            base = a.data + inst * a.sInst + (long long)y * a.M + col + (long long)t * a.ny * a.M;
        } else {
            step = (long long)TL * a.M;
            base = a.data + rest * (long long)a.ny * a.M + col + (long long)t * a.M;
        }
        if (active && !(KIND == 2 && col == 0)) {
#pragma unroll
            for (int m = 0; m < E; ++m) base[m * step] = v[m];
        }
        __syncthreads(); // `cur` is free for the copy issued next iteration
    }

    if (KIND == 2) {
        // Packed column pairs, one group of W/2 pairs per block-iteration.
        const long long npt = (a.npairs + W / 2 - 1) / (W / 2);
        for (long long p = blockIdx.x; p < npt; p += gridDim.x) {
            xpair_block<float, E, (E == 16 ? L : 0)>(reinterpret_cast<float *>(a.data), L, a.ny, a.M, a.sInst,
                                                     a.npairs, a.coef, a.pl_x, W, TL, p, t, w, stw, buf0);
            __syncthreads();
        }
    }
}

template <int L, int KIND, int CFG>
cudaError_t run(const CUtensorMap &map, const TmaArgs &a, unsigned grid, cudaStream_t s)
{
    using S = TmaShape<L, CFG>;
    const size_t smem = tma_smem_bytes(L, S::NARROW);
    auto kern = k_strided_tma<L, KIND, CFG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, S::NT, smem, s>>>(map, a);
    return cudaGetLastError();
}

} // namespace

size_t tma_smem_bytes(int L, int narrow) { return (size_t)3 * (8192 >> (narrow > 0 ? 1 : 0)) * 8 + (size_t)L * 8 + 2 * 8 + 16; }

int tma_columns(int L, int cfg) { return (8192 / L) >> (cfg > 0 ? 1 : 0); }

int tma_threads(int L, int cfg) { return tma_columns(L, cfg) * L / (cfg == 2 ? 8 : 16); }

bool tma_supported(int L) { return L == 256 || L == 512 || L == 1024; }

cudaError_t launch_strided_tma(const CUtensorMap &map, const TmaArgs &a, int L, int kind, int cfg,
                               unsigned grid, cudaStream_t s)
{
#define PSOLVE_TMA_KIND(LL, CF)                                                         \
    if (kind == 0) return run<LL, 0, CF>(map, a, grid, s);                              \
    if (kind == 1) return run<LL, 1, CF>(map, a, grid, s);                              \
    return run<LL, 2, CF>(map, a, grid, s);
#define PSOLVE_TMA_CASE(LL)                                                             \
    case LL:                                                                            \
        if (cfg == 2) { PSOLVE_TMA_KIND(LL, 2) }                                        \
        if (cfg == 1) { PSOLVE_TMA_KIND(LL, 1) }                                        \
        PSOLVE_TMA_KIND(LL, 0)
    switch (L) {
        PSOLVE_TMA_CASE(256)
        PSOLVE_TMA_CASE(512)
        PSOLVE_TMA_CASE(1024)
    default: return cudaErrorInvalidValue;
    }
#undef PSOLVE_TMA_CASE
#undef PSOLVE_TMA_KIND
}

} // namespace psolve
