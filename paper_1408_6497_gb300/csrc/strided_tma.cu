// Persistent, TMA-fed y and x passes for FP32 lines of 256, 512 or 1024 points.
//
// One block per SM walks the tile list.  A tile is L points × W adjacent
// kz-columns (64 KiB: W = 8192 / L), fetched by the Tensor Memory
// Accelerator straight into shared memory while the previous tile is being
// transformed, so HBM reads overlap the butterflies (double buffering with
// two mbarriers).  The transform runs in place in the tile's buffer with the
// same register/shared-memory Stockham engine as the other passes; results go
// back to HBM from registers.  The x kind adds the spectral division between
// its forward and inverse transforms (§2.1: each coefficient times 1/(4π²|k|²))
// and, after its main tiles, the packed kz = 0 / kz = M
// column pairs.
#include "psolve.h"
#include "launch.h"
#include "tma.cuh"
#include "tc.cuh"

namespace psolve {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull; // 2 s per copy, then PSOLVE_ERR_TIMEOUT

// NARROW = 0: 64 KiB tiles (W = 8192/L columns, 512 threads, one block per
// SM); NARROW = 1: 32 KiB tiles (half the columns, 256 threads, two blocks per
// SM, so one block's barriers overlap the other's butterflies).
// CFG 2: as NARROW but 8 points per thread (twice the threads, about half
// the registers each), so 32 warps per SM hide the barrier and shared-memory
// latencies of the butterflies.
// CFG 3: as NARROW but 32 points per thread (radix-32 register butterflies:
// one exchange per transform of 512 points instead of two).
// CFG 4: 64 KiB tiles with 32 points per thread (wide radix-32; for lines of
// 1024 points, whose narrow tiles would have 32-byte rows).
template <int L, int CFG> struct TmaShape {
    static constexpr int NARROW = (CFG > 0 && CFG < 4) ? 1 : 0;
    static constexpr int E = CFG == 2 ? 8 : (CFG >= 3 ? 32 : 16);
    static constexpr int TL = L / E;
    static constexpr int W = (8192 / L) >> NARROW;  // columns per tile
    static constexpr int NT = W * TL;               // threads per block
    static constexpr int MINB = NARROW ? 2 : 1;
    static constexpr int BOXR = L < 256 ? L : 256;  // rows per TMA box
    static constexpr int NLOAD = L / BOXR;
    static constexpr uint32_t TILE_BYTES = (uint32_t)(L * W * 8);
};

// KIND: 0 = y forward, 1 = y inverse, 2 = x forward + division + x inverse.
// TC: radix-16 stages on the tensor cores (FP16 hi/lo with a power-of-two
// scale per row, FP32 accumulation in TMEM).  With 16 points per thread
// (plans 16·16·…) every radix-16 stage runs there, the exchange buffer
// holding the FP16 operand rows (it has
// exactly their size: one 128-byte row per thread).  With 32 points per
// thread (512 = 32 × 16) the radix-32 stage stays in FP32 and the radix-16
// stage, the last, runs on the tensor cores per warpgroup (tc32_last_stage),
// its operand rows in the tile buffer once the tile has been read.
template <int L, int KIND, int CFG, bool TC, bool OPS = false>
__global__ void __launch_bounds__(TmaShape<L, CFG>::NT, TmaShape<L, CFG>::MINB)
    k_strided_tma(const __grid_constant__ CUtensorMap tmap, TmaArgs a)
{
    using S = TmaShape<L, CFG>;
    constexpr int E = S::E, TL = S::TL, W = S::W;
    constexpr bool TC32 = TC && E == 32;
    static_assert(!TC || ((E == 16 || (E == 32 && L == 512)) && S::NT % 128 == 0),
                  "tensor-core stages: 16 points per thread, or 32 for 512-point lines");
    constexpr int NWG = S::NT / 128; // warpgroups per block
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *buf0 = reinterpret_cast<float2 *>(smraw);
    float2 *buf1 = buf0 + L * W;
    float2 *xbuf = buf1 + L * W; // exchange buffer alternating with the tile's own (padded)
    float2 *stw = xbuf + (L + L / 16) * W;
    uint64_t *bar = reinterpret_cast<uint64_t *>(stw + L);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);
    // tensor-core state after the FP32 layout: MMA barrier(s) (one per
    // warpgroup with 32 points per thread), counters, DFT matrices
    uint64_t *mbar = bar + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(TC32 ? bar + 6 : mbar + 1);
    uint32_t *tphase = tslot + 1;
    unsigned char *fmat = reinterpret_cast<unsigned char *>(bar + 8);
    constexpr uint32_t kCols = (TC32 ? 64 : 32) * NWG;

    const int tid = threadIdx.x;
    const int w = tid % W, t = tid / W;
    const long long ntiles = a.main_tiles;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        if constexpr (TC) {
            for (int g = 0; g < (TC32 ? NWG : 1); ++g) mbar_init(mbar + g, 1);
            *tphase = 0;
        }
        fence_mbar_init();
        tma_prefetch_desc(&tmap);
    }
    for (int i = tid; i < L; i += blockDim.x) stw[i] = a.tw[i];
    TcCtx tc{};
    Tc32Ctx tc32{};
    uint32_t nphase = 0; // this warpgroup's completed MMA batches (32 points per thread)
    if constexpr (TC) {
        tc_build_dft16(fmat, fmat + kTcFBytes, fmat + 2 * kTcFBytes, fmat + 3 * kTcFBytes);
        if (tid < 32) tmem_alloc(tslot, kCols);
        tc_fence_before();
    }
    __syncthreads();
    if constexpr (TC) {
        tc_fence_after();
        tc.a_hi = reinterpret_cast<unsigned char *>(xbuf);
        tc.a_lo = tc.a_hi + S::NT * kTcRowBytes;
        tc.f_hi[0] = fmat;
        tc.f_lo[0] = fmat + kTcFBytes;
        tc.f_hi[1] = fmat + 2 * kTcFBytes;
        tc.f_lo[1] = fmat + 3 * kTcFBytes;
        tc.tmem = *tslot;
        tc.bar = mbar;
        tc.phase = tphase;
        tc.abort = abort_flag;
        tc.status = a.status;
        tc32.f_hi[0] = tc.f_hi[0];
        tc32.f_lo[0] = tc.f_lo[0];
        tc32.f_hi[1] = tc.f_hi[1];
        tc32.f_lo[1] = tc.f_lo[1];
        tc32.tmem = tc.tmem;
        tc32.bar = mbar;
        tc32.abort = abort_flag;
        tc32.status = a.status;
    }

    // Tile -> TMA coordinates (c0 = first column, c1, c2 of the first row).
    auto issue = [&](long long tile, float2 *dst, uint64_t *b) {
        const int cb = (int)(tile % a.ncb);
        const long long rest = tile / a.ncb;
        mbar_expect_tx(b, S::TILE_BYTES);
#pragma unroll
        for (int r = 0; r < S::NLOAD; ++r) {
            // x-split layout (G > 1): x lines through a 4D map (M, G, ny,
            // planes / G) whose box (W, G, 1, BOXR / G) lands in shared
            // memory in plain x order, exactly like the 3D box
            if (KIND == 2) {
                const int y = (int)(rest % a.ny);
                const long long inst = rest / a.ny;
                const int x0 = (int)(inst * L + r * S::BOXR);
                if (a.G > 1) tma_load_4d(dst + r * S::BOXR * W, &tmap, b, cb * W, 0, y, x0 / a.G);
                else tma_load_3d(dst + r * S::BOXR * W, &tmap, b, cb * W, y, x0);
            } else {
                // y lines: 3D either way; in the x-split layout the map's rows
                // are G·M wide and the plane's x mod G selects the column block
                const int c0 = a.G > 1 ? (int)(rest % a.G) * a.M + cb * W : cb * W;
                tma_load_3d(dst + r * S::BOXR * W, &tmap, b, c0, r * S::BOXR, (int)(rest / a.G));
            }
        }
    };

    long long tile = blockIdx.x;
    // Set-up above may overlap the previous pass's last blocks; its output is
    // read only from here on.
    grid_dependency_wait();
    if (tid == 0 && tile < ntiles) issue(tile, buf0, &bar[0]);

    // exchanges in the tile buffer: rows swizzled, no spare space there
    const MapStridedSwz<(ct_radix(L, 0, E) >= 32 ? 5 : (ct_radix(L, 0, E) >= 16 ? 4 : 3))> map{W, w};
    // spare row every R0 rows, R0 = the radix of the first stage
    constexpr int PADSH = ct_radix(L, 0, E) >= 32 ? 5 : 4;
    const MapStridedPad<PADSH> xmap{W, w};
    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        float2 *cur = (k & 1) ? buf1 : buf0;
        const long long next = tile + gridDim.x;
        if (tid == 0) {
            if (next < ntiles && !*abort_flag) {
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
        if (*abort_flag) break;

        const int cb = (int)(tile % a.ncb);
        const long long rest = tile / a.ncb;
        const int col = cb * W + w;
        const bool active = col < a.M;
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = cur[(t + m * TL) * W + w];
        if constexpr (TC32) {
            // radix 32 in FP32, exchange through xbuf, radix 16 on the tensor
            // cores with operand rows in `cur` (read out above, before the
            // exchange barrier)
            tc32.op = reinterpret_cast<unsigned char *>(cur);
            fft_stage_ct<32, KIND == 1, false, TL, 1, L / 32>(v, t, stw, xbuf, xmap, true);
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = xbuf[xmap(t + m * TL)];
            tc32_last_stage<KIND == 1>(v, t, stw, tc32, nphase);
        } else if constexpr (TC) {
            __syncthreads(); // single-buffer exchanges in `cur`
            line_fft_tc_from<KIND == 1, L, 0>(v, t, stw, cur, map, tc);
            if (*abort_flag) break;
        } else {
            // Exchanges alternate xbuf, cur, xbuf, ...: the first writes go to
            // xbuf, so the tile reads above need no barrier of their own.
            line_fft_ct_db<KIND == 1, L, 0, 0>(v, t, stw, xbuf, cur, xmap, map);
        }

        float2 *base;
        long long step;
        if (KIND == 2) {
            const int y = (int)(rest % a.ny);
            const long long inst = rest / a.ny;
            const int ky = kvec_dev(y, a.ny);
            if constexpr (!OPS) {
                // the Poisson multiplier (the instantiation for other
                // operators is separate, so this one keeps its registers)
                // Point x = t + m·TL has kx = t + c with c = m·TL for m < E/2
                // and c = (m - E)·TL beyond (at m = E/2, t = 0 that is -L/2,
                // whose square is the Nyquist mode's (+L/2)²), so |k|² =
                // (t² + ky² + kz²) + c·2t + c² with c compile-time: two FP32
                // operations per point, exact (integers below 2^24), and only
                // m = 0 can hold k = 0.
                const float base = (float)(t * t + ky * ky + col * col), t2 = (float)(2 * t);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int c = (2 * m < E ? m : m - E) * TL;
                    const float k2 = fmaf((float)c, t2, base + (float)(c * c));
                    // coef·(1/k²) with the hardware reciprocal: about 2 ulp in FP32
                    const float d = (m == 0 && k2 == 0.f) ? 0.f : __fdividef(a.coef, k2);
                    v[m] = cscale(v[m], d);
                }
            } else if (a.op.op == 1) {
                const float c4 = (float)a.op.c4;
                const int kyz = ky * ky + col * col;
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int kx = kvec_dev(t + m * TL, L);
                    v[m] = cscale(v[m], __fdividef(a.coef, (float)(kx * kx + kyz) + c4));
                }
            } else if (active) {
                // finite-difference Laplacian: Λx per point, Λy + Λz per line
                const float lyz = a.op.ly32[y] + a.op.lz32[col];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const float den = __ldg(&a.op.lx32[t + m * TL]) + lyz;
                    v[m] = cscale(v[m], den == 0.f ? 0.f : __fdividef(a.coef, den));
                }
            }
            if constexpr (TC32) {
                // Every warpgroup is past its forward stages (xbuf reads,
                // MMAs on `cur`) before xbuf and `cur` are reused.
                __syncthreads();
                fft_stage_ct<32, true, false, TL, 1, L / 32>(v, t, stw, xbuf, xmap, true);
                __syncthreads();
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = xbuf[xmap(t + m * TL)];
                tc32_last_stage<true>(v, t, stw, tc32, nphase);
            } else if constexpr (TC) {
                line_fft_tc_from<true, L, 0>(v, t, stw, cur, map, tc);
                if (*abort_flag) break;
            } else {
                // Continue the alternation where the forward transform left it.
                constexpr int PAR = ct_exchanges(L, E) & 1;
                line_fft_ct_db<true, L, 0, PAR>(v, t, stw, xbuf, cur, xmap, map);
            }
            // point x = t + m·TL of line (y, col): row spec_row(x, y) (TL % G == 0)
            step = (long long)TL * a.ny * a.M;
            base = a.data + inst * a.sInst + (long long)y * a.G * a.M + col +
                   ((long long)(t / a.G) * a.ny * a.G + t % a.G) * a.M;
        } else {
            // point y = t + m·TL of plane `rest`: row spec_row(rest, y)
            step = (long long)TL * a.G * a.M;
            base = a.data + ((rest / a.G) * a.ny * a.G + (long long)t * a.G + rest % a.G) * a.M + col;
        }
        if (active && !(KIND == 2 && col == 0)) {
#pragma unroll
            for (int m = 0; m < E; ++m) base[m * step] = v[m];
        }
        __syncthreads(); // `cur` is free for the copy issued next iteration
    }

    if (KIND == 2 && !*abort_flag) {
        // Packed column pairs, one group of W/2 pairs per block-iteration.
        const long long npt = (a.npairs + W / 2 - 1) / (W / 2);
        for (long long p = blockIdx.x; p < npt; p += gridDim.x) {
            xpair_block<float, E, (E == 16 || E == 32 ? L : 0), false, OPS>(
                reinterpret_cast<float *>(a.data), L, a.ny, a.M, a.sInst, a.npairs, a.coef, a.op, a.pl_x, W,
                TL, p, t, w, stw, buf0, a.G);
            __syncthreads();
        }
    }
    if constexpr (TC) {
        tc_fence_before();
        __syncthreads();
        if constexpr (TC32) {
            // After a timed-out wait, let issued MMAs drain before TMEM is freed.
            if (*abort_flag && (tid & 127) == 0)
                mbar_wait_bounded(mbar + (tid >> 7), (nphase - 1) & 1u, 2000000000ull);
            __syncthreads();
        }
        if (tid < 32) {
            tc_fence_after();
            tmem_dealloc(tc.tmem, kCols);
        }
    }
}

template <int L, int KIND, int CFG, bool TC, bool OPS = false>
cudaError_t run(const CUtensorMap &map, const TmaArgs &a, unsigned grid, cudaStream_t s, bool pdl)
{
    using S = TmaShape<L, CFG>;
    const size_t smem = tma_smem_bytes(L, S::NARROW) + (TC ? 64 + 4 * kTcFBytes : 0);
    auto kern = k_strided_tma<L, KIND, CFG, TC, OPS>;
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
    return cudaLaunchKernelEx(&cfg, kern, map, a);
}

} // namespace

size_t tma_smem_bytes(int L, int narrow)
{
    const size_t tile = (size_t)(8192 >> (narrow > 0 ? 1 : 0)) * 8;
    return 3 * tile + tile / 16 + (size_t)L * 8 + 2 * 8 + 16;
}

int tma_columns(int L, int cfg) { return (8192 / L) >> ((cfg > 0 && cfg < 4) ? 1 : 0); }

int tma_threads(int L, int cfg) { return tma_columns(L, cfg) * L / (cfg == 2 ? 8 : (cfg >= 3 ? 32 : 16)); }

bool tma_supported(int L) { return L == 256 || L == 512 || L == 1024; }

// TMA x-pass configurations instantiated for every operator.
bool tma_ops_supported(int L, int cfg) { return (L == 512 && cfg == 3) || (L == 1024 && cfg == 4) || (L == 256 && cfg == 1); }

cudaError_t launch_strided_tma(const CUtensorMap &map, const TmaArgs &a, int L, int kind, int cfg,
                               unsigned grid, cudaStream_t s, bool pdl)
{
    if (kind == 2 && a.op.op != 0) {
        // other operators: the default FP32 configurations only (y passes
        // carry no multiplier and ignore a.op)
        if (a.tc) return cudaErrorInvalidValue;
        if (L == 512 && cfg == 3) return run<512, 2, 3, false, true>(map, a, grid, s, pdl);
        if (L == 1024 && cfg == 4) return run<1024, 2, 4, false, true>(map, a, grid, s, pdl);
        if (L == 256 && cfg == 1) return run<256, 2, 1, false, true>(map, a, grid, s, pdl);
        return cudaErrorInvalidValue;
    }
    if (a.tc) {
        if (cfg == 2) return cudaErrorInvalidValue;
        if (cfg >= 3) { // 32 points per thread: 512-point lines only
            if (L != 512) return cudaErrorInvalidValue;
            if (cfg == 3) {
                if (kind == 0) return run<512, 0, 3, true>(map, a, grid, s, pdl);
                if (kind == 1) return run<512, 1, 3, true>(map, a, grid, s, pdl);
                return run<512, 2, 3, true>(map, a, grid, s, pdl);
            }
            if (kind == 0) return run<512, 0, 4, true>(map, a, grid, s, pdl);
            if (kind == 1) return run<512, 1, 4, true>(map, a, grid, s, pdl);
            return run<512, 2, 4, true>(map, a, grid, s, pdl);
        }
#define PSOLVE_TMA_TC(LL)                                                               \
        if (L == LL) {                                                                  \
            if (cfg == 1) {                                                             \
                if (kind == 0) return run<LL, 0, 1, true>(map, a, grid, s, pdl);             \
                if (kind == 1) return run<LL, 1, 1, true>(map, a, grid, s, pdl);             \
                return run<LL, 2, 1, true>(map, a, grid, s, pdl);                            \
            }                                                                           \
            if (kind == 0) return run<LL, 0, 0, true>(map, a, grid, s, pdl);                 \
            if (kind == 1) return run<LL, 1, 0, true>(map, a, grid, s, pdl);                 \
            return run<LL, 2, 0, true>(map, a, grid, s, pdl);                                \
        }
        PSOLVE_TMA_TC(256)
        PSOLVE_TMA_TC(512)
        PSOLVE_TMA_TC(1024)
#undef PSOLVE_TMA_TC
        return cudaErrorInvalidValue;
    }
#define PSOLVE_TMA_KIND(LL, CF)                                                         \
    if (kind == 0) return run<LL, 0, CF, false>(map, a, grid, s, pdl);                       \
    if (kind == 1) return run<LL, 1, CF, false>(map, a, grid, s, pdl);                       \
    return run<LL, 2, CF, false>(map, a, grid, s, pdl);
#define PSOLVE_TMA_CASE(LL)                                                             \
    case LL:                                                                            \
        if (cfg == 4) { PSOLVE_TMA_KIND(LL, 4) }                                        \
        if (cfg == 3) { PSOLVE_TMA_KIND(LL, 3) }                                        \
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
