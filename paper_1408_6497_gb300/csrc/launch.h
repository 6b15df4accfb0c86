// Host-side launchers of the pass kernels (one translation unit per pass kind,
// compiled in parallel).  Each picks the instantiation for E at run time.
#pragma once

#include <cuda.h>

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

// Persistent TMA-fed FP32 y/x passes for lines of 256, 512 or 1024 points.
struct TmaArgs {
    float2 *data;          // packed spectrum
    int M, ny, ncb;        // columns per row, rows per plane, column tiles per row
    long long main_tiles;  // y: planes·ncb; x: instances·ny·ncb
    long long sInst;       // complex elements per instance
    long long npairs;      // x: instances·(ny/2 + 1)
    const float2 *tw;      // e^{-2πi j/L}
    float coef;            // 1 / (4π² N)
    OpArgs op;             // spectral multiplier (op 0: Poisson; others: tma_ops_supported configurations)
    int *status;           // device status word
    LinePlan pl_x;         // run-time plan of the x line (packed-column pairs)
    int tc;                // radix-16 stages on the tensor cores (cfg 0 and 1 only)
    int G;                 // x-split factor of the spectrum layout (1: natural; see
                           // spec_row); x lines then use a 4D map (M, G, ny, planes/G),
                           // y lines a 3D one (G·M, ny, planes/G)
};

// Row (x, y) of the packed spectrum, x counted over all instances of a group
// (x = instance·nx + x_local), in the x-split layout with factor G: rows are
// ordered (x / G, y, x mod G), so the G rows of an x-group at one y are
// adjacent.  A line along x then touches L/G separate places in memory
// instead of L (fewer address translations per tile); G = 1 is the natural
// (x, y) order.
__host__ __device__ inline long long spec_row(long long x, long long y, int ny, int G)
{
    return ((x / G) * ny + y) * G + (x % G);
}
bool tma_supported(int L);
bool tma_ops_supported(int L, int cfg);
// cfg 0: 64 KiB tiles, 16 points per thread, one 512-thread block per SM;
// cfg 1: 32 KiB tiles, 16 points per thread, 256-thread blocks, two per SM;
// cfg 2: 32 KiB tiles, 8 points per thread, 512-thread blocks, two per SM;
// cfg 3: 32 KiB tiles, 32 points per thread (radix-32), 128-thread blocks;
// cfg 4: 64 KiB tiles, 32 points per thread, one block per SM.
int tma_columns(int L, int cfg);
int tma_threads(int L, int cfg);
size_t tma_smem_bytes(int L, int cfg);
// kind: 0 = y forward, 1 = y inverse, 2 = x with the spectral division.
// pdl: launch with programmatic stream serialisation (the kernel's set-up
// may overlap the previous kernel's last blocks).
cudaError_t launch_strided_tma(const CUtensorMap &map, const TmaArgs &a, int L, int kind, int cfg,
                               unsigned grid, cudaStream_t s, bool pdl = true);

// Persistent z passes fed by 1D bulk copies (FP32, M = 256 or 512).
struct ZBulkArgs {
    const float *real_in; // forward: f rows
    float *real_out;      // inverse: u rows
    float2 *spec;         // packed spectrum rows (forward output, inverse input)
    long long rows;       // multiple of z_bulk_rows(M, direction)
    const float2 *tw;     // e^{-2πi j/M}
    const float2 *post;   // e^{-2πi k/nz}, k < M
    int *status;
    int ny, G;            // spectrum rows in the x-split layout (spec_row; G = 1: natural)
};
bool z_bulk_supported(int M);
int z_bulk_rows(int M, bool inverse);
size_t z_bulk_smem(int M, bool inverse);
int z_bulk_blocks_per_sm(int M, bool inverse);
cudaError_t launch_z_bulk(const ZBulkArgs &a, int M, bool inverse, unsigned grid, cudaStream_t s, bool pdl = true);

// z and y passes of a plane fused through L2 in one cluster launch.
constexpr int kFusedThreads = 256;
struct FusedArgs {
    long long planes; // x-planes (instances · nx)
    int cluster;      // blocks per plane (cluster size)
    int ztiles;       // row tiles per plane
    int ytiles;       // column tiles per plane
};
bool fused_supported(int M, int ny);
cudaError_t launch_fused_zy(const ZArgs<float> &az, const SArgs<float> &ay, const FusedArgs &fa, bool inverse,
                            size_t smem, cudaStream_t s);

// z and y passes of a plane in one launch, the plane held in the distributed
// shared memory of a 16-block cluster (FP32; ny = 256 or 512 rows of
// M = 128 or 256 packed complex values).
struct ZyArgs {
    const float *real_in; // forward: f rows
    float *real_out;      // inverse: u rows
    float2 *spec;         // packed spectrum, natural layout (forward output; the inverse reads it by TMA)
    long long planes;     // x-planes of all instances
    const float2 *tw_y;   // e^{-2πi j/ny}
    const float2 *tw_z;   // e^{-2πi j/M}
    const float2 *post;   // e^{-2πi k/nz}, k < M
    int *status;
};
bool zy_cluster_supported(int M, int ny);
int zy_cluster_size();
// Clusters of the kernel that fit on the device at once (0: none).
cudaError_t zy_cluster_max_active(int M, int ny, bool inverse, int *clusters);
// map: the spectrum as a 3D tensor (M, ny, planes) of 8-byte elements with
// box (M / 16, min(ny, 256), 1), read by the inverse pass.
cudaError_t launch_zy_cluster(const CUtensorMap &map, const ZyArgs &a, int M, int ny, bool inverse, int clusters,
                              cudaStream_t s, bool pdl = true);

// Persistent batched kernel: one segment per (pass, instance), pass-major.
// Threads of a batched-launch block: 128 (the barriers of a tile hold four
// warps; 256-thread blocks measured slower on GB300), eight blocks per SM
// (PSOLVE_BATCH_MINB in batched.cu).
#ifndef PSOLVE_BATCH_THREADS
#define PSOLVE_BATCH_THREADS 128
#endif
constexpr int kBatchThreads = PSOLVE_BATCH_THREADS;
template <typename T> struct BatchSeg {
    int kind;           // 0 zfwd, 1 yfwd, 2 xdiv, 3 yinv, 4 zinv
    int E;              // points per thread of the pass's line
    int lc;             // line length of a compile-time plan (batched_ct_supported), else 0
    int dep;            // segment that must complete first, or -1
    int need;           // completed tiles of `dep` to wait for (its tile count)
    long long first;    // first item number of this segment
    long long ntiles;
    long long off;      // element offset of the instance in f and u
    ZArgs<T> z;         // the member for this segment's pass is used;
    SArgs<T> y;         // pointers to f/u are filled in by the kernel
    XArgs<T> x;
};
template <typename T> const void *batched_kernel();
template <typename T> cudaError_t batched_prepare(size_t smem);
bool batched_supports_E(int E);
// (line length, points per thread) pairs the batched kernel holds compile-time
// plans for (radix-3 stages first, then the largest power-of-two radices).
bool batched_ct_supported(int L, int E);

// Twiddles e^{-2πi j/denom}, j < count, computed in FP64 and rounded to T.
template <typename T>
cudaError_t launch_roots(void *dst, int count, int denom, cudaStream_t s);

// Signed wavenumbers of the half spectrum (nx, ny, nz/2+1) as int3 triples.
cudaError_t launch_kvec(int *dst, int nx, int ny, int nz, cudaStream_t s);

// FP64 sums and maxima of (a - ref) and ref into out[4] (device, zeroed by caller).
template <typename T>
cudaError_t launch_norms(const T *a, const T *ref, size_t n, double *out, cudaStream_t s);

} // namespace psolve
