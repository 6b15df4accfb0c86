// z and y transforms of a plane held in a thread-block cluster's distributed
// shared memory: the forward pass reads f and writes the y-transformed
// spectrum, the inverse pass reads that spectrum (after the x pass) and
// writes u, so a solve makes three trips through HBM instead of five (§2.1:
// the axis-by-axis transform with its transposes, Fig. 1; here the
// transpose between the z and y transforms is a read of the neighbouring
// blocks' shared memory instead of a pass through HBM).
//
// A cluster of C = 16 blocks owns one x-plane at a time: NY rows of NZ =
// 2M reals, i.e. NY × M packed complex values (the r2c layout of the other
// passes: X[0] + i·X[M] in slot 0).  Block c holds rows [c·R, (c+1)·R)
// (R = NY/16) in phase Z and columns [c·Q, (c+1)·Q) (Q = M/16) in phase Y;
// its share of a plane (R·M = NY·Q values) is one 1/16 of it.
//
// Forward, per plane:
//   Z: one 1D bulk copy brings the block's R rows of f (contiguous) into
//      zbuf; the rows are transformed (M-point FFT of the real pairs, split
//      post-twiddle) and the packed rows written back into zbuf;
//   cluster barrier (every block's zbuf holds its rows of the plane, and
//      every block has finished reading the previous plane);
//   Y: each thread reads its column's points from the 16 blocks' zbuf
//      (ld.shared::cluster), the y transform runs with exchanges in the
//      block's own buffer, and the results go to HBM from registers.
// Inverse, per plane: a TMA box brings the block's Q columns of all NY rows
// of the spectrum into zbuf, the inverse y transform runs and writes them
// back into zbuf; cluster barrier; each block merges X[k] and X[M-k] of its
// R rows from the 16 blocks' zbuf (pre-twiddle), runs the inverse z
// transform and writes the real rows of u.
//
// Two zbuf per block: the copy for the next plane lands in the other one
// while the current plane is transformed, and a zbuf is refilled only after
// the cluster barrier that follows every block's last read of it.  All
// blocks of a cluster run the same number of planes, so every block meets
// every barrier; a copy that does not complete in time is recorded as
// PSOLVE_ERR_TIMEOUT, the block stops waiting for its copies, still meets
// the barriers, and lets its copies in flight land before it exits.  A final
// barrier keeps every block's shared memory alive until the others have
// read it.
#include "psolve.h"
#include "launch.h"
#include "tma.cuh"

namespace psolve {

namespace {

constexpr int kZyC = 16;                         // blocks per cluster (one plane)
constexpr uint64_t kZyWaitNs = 2000000000ull;    // 2 s per copy, then PSOLVE_ERR_TIMEOUT

__device__ __forceinline__ unsigned zy_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned zy_cluster_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned zy_num_clusters()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void zy_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory address of the same variable in block `rank` of the cluster.
__device__ __forceinline__ uint32_t zy_mapa(uint32_t addr, unsigned rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// (volatile keeps it after the cluster barrier, itself a volatile asm with
// a memory clobber; no clobber here, so the loads of a phase issue together)
__device__ __forceinline__ float2 zy_ld_remote(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

template <int NY, int M> struct ZyShape {
    static constexpr int E = 16;                 // points per thread, both phases
    static constexpr int R = NY / kZyC;          // rows per block (phase Z)
    static constexpr int Q = M / kZyC;           // columns per block (phase Y)
    static constexpr int TLZ = M / E;            // threads per z row
    static constexpr int TLY = NY / E;           // threads per y line
    static constexpr int NT = R * TLZ;           // threads per block (= Q · TLY)
    static constexpr int LPZ = M + (M >> 4) + 1; // padded z-row pitch of the exchange buffer
    static constexpr int ZBUF = R * M;           // complex values of one zbuf (= NY · Q)
    static constexpr int XZ = R * LPZ;
    static constexpr int XY = (NY + NY / 16) * Q;
    static constexpr int XBUF = XZ > XY ? XZ : XY;
    static_assert(NT == Q * TLY, "both phases use every thread");
    static_assert(TLY == R && TLZ == Q, "a thread's points come one from each block");
};

template <int NY, int M> constexpr size_t zy_smem()
{
    using S = ZyShape<NY, M>;
    return (size_t)(2 * S::ZBUF + S::XBUF + NY + 2 * M) * 8 + 2 * 8 + 16;
}

// planes: x-planes of all instances; spec: packed spectrum (natural layout);
// the forward pass reads real rows from `real`, the inverse writes them.
template <int NY, int M, bool INV>
__global__ void __launch_bounds__(ZyShape<NY, M>::NT, 1)
    k_zy_cluster(const __grid_constant__ CUtensorMap tmap, ZyArgs a)
{
    using S = ZyShape<NY, M>;
    constexpr int E = S::E, R = S::R, Q = S::Q, TLZ = S::TLZ, TLY = S::TLY;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *zbuf0 = reinterpret_cast<float2 *>(smraw);
    float2 *zbuf1 = zbuf0 + S::ZBUF;
    float2 *xb = zbuf1 + S::ZBUF;
    float2 *stw_y = xb + S::XBUF;   // e^{-2πij/NY}
    float2 *stw_z = stw_y + NY;     // e^{-2πij/M}
    float2 *spost = stw_z + M;      // e^{-2πik/NZ}, k < M
    uint64_t *bar = reinterpret_cast<uint64_t *>(spost + M);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const unsigned c = zy_rank();
    const long long nplanes = a.planes;
    const long long p0 = zy_cluster_id(), pstep = zy_num_clusters();
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_mbar_init();
        if (INV) tma_prefetch_desc(&tmap);
    }
    for (int i = tid; i < NY; i += blockDim.x) stw_y[i] = a.tw_y[i];
    for (int i = tid; i < M; i += blockDim.x) {
        stw_z[i] = a.tw_z[i];
        spost[i] = a.post[i];
    }
    __syncthreads();

    // The block's share of plane p: forward, R real rows of f (contiguous);
    // inverse, Q spectrum columns of all NY rows (a TMA box per 256 rows).
    auto issue = [&](long long p, float2 *dst, uint64_t *b) {
        mbar_expect_tx(b, (uint32_t)(S::ZBUF * 8));
        if (!INV) {
            bulk_load(dst, a.real_in + (p * NY + (long long)c * R) * (2 * M), (uint32_t)(S::ZBUF * 8), b);
        } else {
            constexpr int BOXR = NY < 256 ? NY : 256;
#pragma unroll
            for (int r = 0; r < NY / BOXR; ++r)
                tma_load_3d(dst + r * BOXR * Q, &tmap, b, (int)c * Q, r * BOXR, (int)p);
        }
    };
    // Copies in flight per buffer and the barrier phase each completes
    // (thread 0's bookkeeping; the block leaves only after they land).
    bool pending[2] = {false, false};
    uint32_t pend_par[2] = {0u, 0u};

    grid_dependency_wait();
    if (tid == 0 && p0 < nplanes) {
        issue(p0, zbuf0, &bar[0]);
        pending[0] = true;
    }
    const uint32_t zb_addr[2] = {smem_u32(zbuf0), smem_u32(zbuf1)};

    for (long long p = p0, k = 0; p < nplanes; p += pstep, ++k) {
        const int cur = (int)(k & 1);
        float2 *zb = cur ? zbuf1 : zbuf0;
        if (tid == 0 && pending[cur]) {
            if (!*abort_flag && !mbar_wait_bounded(&bar[cur], (uint32_t)((k >> 1) & 1), kZyWaitNs)) {
                *abort_flag = 1;
                atomicExch(a.status, (int)PSOLVE_ERR_TIMEOUT);
            }
            if (!*abort_flag) pending[cur] = false;
        }
        __syncthreads();
        const bool live = !*abort_flag;

        if (!INV) {
            // ---- Z: rows c·R + w of the plane, M-point FFT + split post-twiddle
            if (live) {
                const int w = tid / TLZ, t = tid - w * TLZ;
                const MapRow<4> xm{w * S::LPZ};
                float2 v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = zb[w * M + t + m * TLZ];
                line_fft_ct_from<false, M, 0>(v, t, stw_z, xb, xm, true);
                // Z[k] -> X[k] needs Z[M-k]
#pragma unroll
                for (int m = 0; m < E; ++m) xb[xm(t + m * TLZ)] = v[m];
                __syncthreads();
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int kk = t + m * TLZ;
                    const float2 z = v[m];
                    float2 X;
                    if (kk == 0) {
                        X = make_float2(z.x + z.y, z.x - z.y);
                    } else {
                        const float2 zp = xb[xm(M - kk)];
                        const float2 e = make_float2((z.x + zp.x) * 0.5f, (z.y - zp.y) * 0.5f);
                        const float2 o = make_float2((z.y + zp.y) * 0.5f, (zp.x - z.x) * 0.5f);
                        X = cadd(e, cmul(o, spost[kk]));
                    }
                    zb[w * M + kk] = X; // every thread read its row points before the exchanges
                }
            }
            zy_cluster_sync();
            if (tid == 0) {
                const long long pn = p + pstep;
                if (pn < nplanes && !*abort_flag) {
                    // The other zbuf was last read remotely before the barrier above.
                    fence_proxy_async_smem();
                    issue(pn, cur ? zbuf0 : zbuf1, &bar[cur ^ 1]);
                    pending[cur ^ 1] = true;
                    pend_par[cur ^ 1] = (uint32_t)(((k + 1) >> 1) & 1);
                }
            }
            // ---- Y: columns c·Q + w, point y = t + m·TLY lives in block m, row t
            if (live) {
                const int w = tid % Q, t = tid / Q;
                float2 v[E];
                const uint32_t off = zb_addr[cur] + (uint32_t)((t * M + (int)c * Q + w) * 8);
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = zy_ld_remote(zy_mapa(off, (unsigned)m));
                const MapStridedPad<4> ym{Q, w};
                line_fft_ct_from<false, NY, 0>(v, t, stw_y, xb, ym, true);
                float2 *dst = a.spec + (p * NY + t) * M + (long long)c * Q + w;
#pragma unroll
                for (int m = 0; m < E; ++m) dst[(long long)m * TLY * M] = v[m];
            }
        } else {
            // ---- Y inverse: columns c·Q + w of all NY rows, in place in zbuf
            if (live) {
                const int w = tid % Q, t = tid / Q;
                float2 v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = zb[(t + m * TLY) * Q + w];
                const MapStridedPad<4> ym{Q, w};
                line_fft_ct_from<true, NY, 0>(v, t, stw_y, xb, ym, true);
#pragma unroll
                for (int m = 0; m < E; ++m) zb[(t + m * TLY) * Q + w] = v[m];
            }
            zy_cluster_sync();
            if (tid == 0) {
                const long long pn = p + pstep;
                if (pn < nplanes && !*abort_flag) {
                    fence_proxy_async_smem();
                    issue(pn, cur ? zbuf0 : zbuf1, &bar[cur ^ 1]);
                    pending[cur ^ 1] = true;
                    pend_par[cur ^ 1] = (uint32_t)(((k + 1) >> 1) & 1);
                }
            }
            // ---- Z inverse: row y = c·R + w; X[kk] lives in block kk / Q at
            // column kk % Q (kk = t + m·TLZ: block m, column t)
            if (live) {
                const int w = tid / TLZ, t = tid - w * TLZ;
                const int y = (int)c * R + w;
                const uint32_t row = zb_addr[cur] + (uint32_t)(y * Q * 8);
                float2 v[E];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int kk = t + m * TLZ;
                    const float2 x = zy_ld_remote(zy_mapa(row + (uint32_t)(t * 8), (unsigned)m));
                    if (kk == 0) {
                        v[m] = make_float2(x.x + x.y, x.x - x.y);
                    } else {
                        const int kp = M - kk; // block kp / Q, column kp % Q
                        const float2 xp =
                            zy_ld_remote(zy_mapa(row + (uint32_t)((kp % Q) * 8), (unsigned)(kp / Q)));
                        const float2 e = make_float2(x.x + xp.x, x.y - xp.y);
                        const float2 o = cmulc(make_float2(x.x - xp.x, x.y + xp.y), spost[kk]);
                        v[m] = make_float2(e.x - o.y, e.y + o.x);
                    }
                }
                const MapRow<4> xm{w * S::LPZ};
                line_fft_ct_from<true, M, 0>(v, t, stw_z, xb, xm, true);
                float2 *dst = reinterpret_cast<float2 *>(a.real_out + (p * NY + y) * (2 * M)) + t;
#pragma unroll
                for (int m = 0; m < E; ++m) dst[m * TLZ] = v[m];
            }
        }
        __syncthreads(); // xb is free for the next plane
    }
    // Let copies in flight land, then keep this block's shared memory alive
    // until every block of the cluster has finished reading it.
    if (tid == 0) {
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait_bounded(&bar[b], pend_par[b], kZyWaitNs);
    }
    zy_cluster_sync();
}

template <int NY, int M, bool INV>
cudaError_t run(const CUtensorMap &map, const ZyArgs &a, int clusters, cudaStream_t s, bool pdl)
{
    auto kern = k_zy_cluster<NY, M, INV>;
    const size_t smem = zy_smem<NY, M>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(clusters * kZyC));
    cfg.blockDim = dim3(ZyShape<NY, M>::NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kZyC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1] = programmatic_serialization();
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, map, a);
}

template <int NY, int M, bool INV> cudaError_t max_clusters(int *out)
{
    auto kern = k_zy_cluster<NY, M, INV>;
    const size_t smem = zy_smem<NY, M>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)kZyC);
    cfg.blockDim = dim3(ZyShape<NY, M>::NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kZyC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

} // namespace

bool zy_cluster_supported(int M, int ny)
{
    return (ny == 256 || ny == 512) && (M == 128 || M == 256);
}

int zy_cluster_size() { return kZyC; }

cudaError_t zy_cluster_max_active(int M, int ny, bool inverse, int *clusters)
{
    *clusters = 0;
#define PSOLVE_ZY_MAX(NY_, M_) (inverse ? max_clusters<NY_, M_, true>(clusters) : max_clusters<NY_, M_, false>(clusters))
    if (ny == 256 && M == 128) return PSOLVE_ZY_MAX(256, 128);
    if (ny == 256 && M == 256) return PSOLVE_ZY_MAX(256, 256);
    if (ny == 512 && M == 128) return PSOLVE_ZY_MAX(512, 128);
    if (ny == 512 && M == 256) return PSOLVE_ZY_MAX(512, 256);
#undef PSOLVE_ZY_MAX
    return cudaErrorInvalidValue;
}

cudaError_t launch_zy_cluster(const CUtensorMap &map, const ZyArgs &a, int M, int ny, bool inverse, int clusters,
                              cudaStream_t s, bool pdl)
{
#define PSOLVE_ZY_RUN(NY_, M_) (inverse ? run<NY_, M_, true>(map, a, clusters, s, pdl) : run<NY_, M_, false>(map, a, clusters, s, pdl))
    if (ny == 256 && M == 128) return PSOLVE_ZY_RUN(256, 128);
    if (ny == 256 && M == 256) return PSOLVE_ZY_RUN(256, 256);
    if (ny == 512 && M == 128) return PSOLVE_ZY_RUN(512, 128);
    if (ny == 512 && M == 256) return PSOLVE_ZY_RUN(512, 256);
#undef PSOLVE_ZY_RUN
    return cudaErrorInvalidValue;
}

} // namespace psolve
