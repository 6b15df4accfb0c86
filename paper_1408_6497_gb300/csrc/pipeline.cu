// The pass pipeline: tensor maps of the TMA passes, the launch of each pass
// with the kernels and tile shapes its plan chose, the persistent batched
// launch replayed from a CUDA graph, and solves from device or host buffers.
#include "plan.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <mutex>

namespace psolve {

// Events for one solve, or an empty set when profiling is off.
std::vector<cudaEvent_t> *take_events(psolve_plan *p)
{
    if (!p->profiling) return nullptr;
    if (p->prof_every > 1 && (p->prof_count++ % (unsigned)p->prof_every) != 0) return nullptr;
    std::vector<cudaEvent_t> set;
    if (!p->ev_free.empty()) {
        set = std::move(p->ev_free.back());
        p->ev_free.pop_back();
    } else {
        set.resize(kPasses + 1);
        for (auto &e : set)
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    }
    p->ev_used.push_back(std::move(set));
    return &p->ev_used.back();
}

namespace {

unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3D map over complex FP32 values seen as 8-byte elements, dims innermost first.
bool encode_map(CUtensorMap *m, void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
                uint32_t b2)
{
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {d0 * 8, d0 * d1 * 8};
    cuuint32_t box[3] = {b0, b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


bool encode_map4(CUtensorMap *m, void *base, const uint64_t (&d)[4], const uint32_t (&b)[4])
{
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[4] = {d[0], d[1], d[2], d[3]};
    cuuint64_t strides[3] = {d[0] * 8, d[0] * d[1] * 8, d[0] * d[1] * d[2] * 8};
    cuuint32_t box[4] = {b[0], b[1], b[2], b[3]};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// x-split factor a solve of group g uses: every pass must be one that knows
// the layout (bulk z passes, TMA y/x passes), the spectrum stays on the
// device, and G divides nx and the x line's threads.
int xs_factor(const psolve_plan *p, const Group &g, bool host_io)
{
    if (!p->xsbuf || g.xs <= 1 || host_io || g.fused > 0 || !g.zbulk || g.cfg_y < 0 || g.cfg_x < 0 ||
        p->op != PSOLVE_OP_POISSON)
        return 1;
    if (g.nx % g.xs != 0 || tma_threads(g.nx, g.cfg_x) / tma_columns(g.nx, g.cfg_x) % g.xs != 0) return 1;
    if ((g.nx < 256 ? g.nx : 256) % g.xs != 0) return 1;
    return g.xs;
}

template <typename T>
psolve_status run_tma_pass(const psolve_plan *p, const Group &g, T *ui, int kind, cudaStream_t s, int G = 1)
{
    if constexpr (sizeof(T) != 4) {
        return fail(PSOLVE_ERR_INTERNAL, "TMA pass is FP32 only");
    } else {
        const int L = kind == 2 ? g.nx : g.ny;
        const int narrow = kind == 2 ? g.cfg_x : g.cfg_y;
        const int W = tma_columns(L, narrow);
        const int boxr = L < 256 ? L : 256;
        CUtensorMap map;
        bool ok;
        if (G > 1 && kind == 2) {
            // x-split layout, x lines: 4D (M, G, ny, planes / G)
            const uint64_t d[4] = {(uint64_t)g.M, (uint64_t)G, (uint64_t)g.ny, (uint64_t)g.nx * g.count / G};
            const uint32_t bx[4] = {(uint32_t)W, (uint32_t)G, 1u, (uint32_t)(boxr / G)};
            ok = encode_map4(&map, ui, d, bx);
        } else if (G > 1) {
            // x-split layout, y lines: 3D (G·M, ny, planes / G), the inner
            // coordinate (x mod G)·M + column (a 4D map with unit box
            // dimensions measured 11% slower for the y passes)
            ok = encode_map(&map, ui, (uint64_t)G * g.M, (uint64_t)g.ny, (uint64_t)g.nx * g.count / G,
                            (uint32_t)W, (uint32_t)boxr, 1u);
        } else {
            ok = kind == 2 ? encode_map(&map, ui, (uint64_t)g.M, (uint64_t)g.ny, (uint64_t)g.nx * g.count,
                                        (uint32_t)W, 1u, (uint32_t)boxr)
                           : encode_map(&map, ui, (uint64_t)g.M, (uint64_t)g.ny, (uint64_t)g.nx * g.count,
                                        (uint32_t)W, (uint32_t)boxr, 1u);
        }
        if (!ok) return fail(PSOLVE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        TmaArgs a{};
        a.data = reinterpret_cast<float2 *>(ui);
        a.M = g.M;
        a.ny = g.ny;
        a.ncb = (g.M + W - 1) / W;
        a.main_tiles = kind == 2 ? (long long)g.count * g.ny * a.ncb : (long long)g.count * g.nx * a.ncb;
        a.sInst = (long long)g.nx * g.ny * g.M;
        a.npairs = (long long)g.count * (g.ny / 2 + 1);
        a.tw = reinterpret_cast<const float2 *>(p->tables) + (kind == 2 ? g.tw_x : g.tw_y);
        a.coef = (float)(1.0 / (4.0 * M_PI * M_PI * ((double)g.nx * g.ny * g.nz)));
        a.op = op_args(p, g);
        a.status = p->status;
        a.tc = p->dtype == PSOLVE_F32_TC ? 1 : 0;
        a.G = G;
        if (narrow == 2 && kind == 2 && !make_line_plan_E(g.nx, 8, a.pl_x))
            return fail(PSOLVE_ERR_INTERNAL, "no 8-point plan for the x line");
        long long work = a.main_tiles;
        if (kind == 2) work = std::max(work, (a.npairs + W / 2 - 1) / (W / 2));
        const int per_sm = (narrow >= 1 && narrow <= 3) ? 2 : 1;
        const unsigned grid = (unsigned)std::min<long long>(work, (long long)p->num_sms * per_sm);
        cudaError_t e = launch_strided_tma(map, a, L, kind, narrow, grid, s, !p->serial);
        if (e != cudaSuccess) return cuda_fail(e, "TMA pass");
        return PSOLVE_OK;
    }
}

// Enqueue pass `kind` (0 zfwd, 1 yfwd, 2 x with division, 3 yinv, 4 zinv)
// of a group with its current tile choices.
} // namespace

template <typename T>
psolve_status launch_pass(const psolve_plan *p, const Group &g, int kind, const T *fi, T *ui, cudaStream_t s,
                          bool force_runtime, T *zout, bool host_io, int G)
{
    using C = typename cplx_of<T>::type;
    const C *tab = reinterpret_cast<const C *>(p->tables);
    const int dtype = p->dtype;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        // Bulk-copy z passes read/write device memory only (host_io: f or u
        // is pinned host memory, handled by the per-tile kernels' loads).
        if ((kind == 0 || kind == 4) && g.zbulk && !force_runtime && !host_io) {
            ZBulkArgs zb{};
            zb.real_in = fi;
            zb.real_out = (kind == 4 && zout) ? zout : ui;
            zb.spec = reinterpret_cast<float2 *>(ui);
            zb.rows = (long long)g.count * g.nx * g.ny;
            zb.tw = tab + g.tw_z;
            zb.post = tab + g.post;
            zb.status = p->status;
            zb.ny = g.ny;
            zb.G = G;
            const long long ntiles = zb.rows / z_bulk_rows(g.M, kind == 4);
            const unsigned grid =
                (unsigned)std::min<long long>(ntiles, (long long)z_bulk_blocks_per_sm(g.M, kind == 4) * p->num_sms);
            e = launch_z_bulk(zb, g.M, kind == 4, grid, s, !p->serial);
            if (e != cudaSuccess) return cuda_fail(e, kind == 0 ? "z forward pass" : "z inverse pass");
            return PSOLVE_OK;
        }
    }
    if (kind == 0 || kind == 4) {
        ZArgs<T> z{};
        z.in = kind == 0 ? fi : ui;
        z.out = (kind == 4 && zout) ? zout : ui;
        z.rows = (long long)g.count * g.nx * g.ny;
        z.nz = g.nz;
        z.M = g.M;
        z.W = g.Wz;
        z.pl = g.pz;
        z.tw = tab + g.tw_z;
        z.post = tab + g.post;
        z.force_runtime = force_runtime;
        const unsigned grid = ceil_div(z.rows, g.Wz);
        const unsigned block = (unsigned)(g.Wz * g.pz.TL);
        e = kind == 0 ? launch_zfwd<T>(z, grid, block, z_smem(g, dtype), s)
                      : launch_zinv<T>(z, grid, block, z_smem(g, dtype), s);
        if (e != cudaSuccess) return cuda_fail(e, kind == 0 ? "z forward pass" : "z inverse pass");
        return PSOLVE_OK;
    }
    if (kind == 1 || kind == 3) {
        if (g.cfg_y >= 0) return run_tma_pass<T>(p, g, ui, kind == 1 ? 0 : 1, s, G);
        SArgs<T> y{};
        y.data = ui;
        y.nplanes = (long long)g.count * g.nx;
        y.sPlane = (long long)g.ny * g.M;
        y.sL = g.M;
        y.M = g.M;
        y.W = g.Wy;
        y.ncb = (g.M + g.Wy - 1) / g.Wy;
        y.pl = g.py;
        y.tw = tab + g.tw_y;
        y.force_runtime = force_runtime;
        const unsigned grid = (unsigned)(y.nplanes * y.ncb);
        const unsigned block = (unsigned)(g.Wy * g.py.TL);
        e = launch_ypass<T>(y, kind == 3, grid, block, s_smem(g.ny, g.Wy, dtype), s);
        if (e != cudaSuccess) return cuda_fail(e, kind == 1 ? "y forward pass" : "y inverse pass");
        return PSOLVE_OK;
    }
    // Other operators than Poisson have TMA x-pass instantiations for the
    // default FP32 configurations only; otherwise they take the per-tile pass.
    if (g.cfg_x >= 0 && (p->op == PSOLVE_OP_POISSON ||
                         (p->dtype == PSOLVE_F32 && tma_ops_supported(g.nx, g.cfg_x))))
        return run_tma_pass<T>(p, g, ui, 2, s, G);
    XArgs<T> x{};
    x.data = ui;
    x.batch = g.count;
    x.nx = g.nx;
    x.ny = g.ny;
    x.M = g.M;
    x.sInst = (long long)g.nx * g.ny * g.M;
    x.W = g.Wx;
    x.ncb = (g.M + g.Wx - 1) / g.Wx;
    x.main_tiles = (long long)g.count * g.ny * x.ncb;
    x.npairs = (long long)g.count * (g.ny / 2 + 1);
    x.pl = g.px;
    x.tw = tab + g.tw_x;
    x.coef = (T)(1.0 / (4.0 * M_PI * M_PI * ((double)g.nx * g.ny * g.nz)));
    x.op = op_args(p, g);
    x.force_runtime = force_runtime;
    const unsigned grid = (unsigned)(x.main_tiles + (x.npairs + g.Wx / 2 - 1) / (g.Wx / 2));
    const unsigned block = (unsigned)(g.Wx * g.px.TL);
    e = launch_xfused<T>(x, grid, block, s_smem(g.nx, g.Wx, dtype), s);
    if (e != cudaSuccess) return cuda_fail(e, "x pass with spectral division");
    return PSOLVE_OK;
}

namespace {

// z+y (forward) or y+z (inverse) of every plane in one cluster launch.
template <typename T>
psolve_status launch_fused(const psolve_plan *p, const Group &g, bool inverse, const T *fi, T *ui, cudaStream_t s,
                           T *zout = nullptr)
{
    if constexpr (sizeof(T) != 4) {
        return fail(PSOLVE_ERR_INTERNAL, "fused z/y passes are FP32 only");
    } else {
        using C = float2;
        const C *tab = reinterpret_cast<const C *>(p->tables);
        if (g.fused == zy_cluster_size()) {
            // the plane in a 16-block cluster's distributed shared memory
            const long long planes = (long long)g.count * g.nx;
            ZyArgs za{};
            za.real_in = fi;
            za.real_out = (inverse && zout) ? zout : ui;
            za.spec = reinterpret_cast<float2 *>(ui);
            za.planes = planes;
            za.tw_y = tab + g.tw_y;
            za.tw_z = tab + g.tw_z;
            za.post = tab + g.post;
            za.status = p->status;
            CUtensorMap map{};
            if (inverse && !encode_map(&map, ui, (uint64_t)g.M, (uint64_t)g.ny, (uint64_t)planes,
                                       (uint32_t)(g.M / zy_cluster_size()), (uint32_t)std::min(g.ny, 256), 1u))
                return fail(PSOLVE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
            const int clusters = (int)std::min<long long>(planes, g.zy_clusters);
            cudaError_t e = launch_zy_cluster(map, za, g.M, g.ny, inverse, clusters, s, !p->serial);
            if (e != cudaSuccess)
                return cuda_fail(e, inverse ? "fused y/z inverse pass (cluster)" : "fused z/y forward pass (cluster)");
            return PSOLVE_OK;
        }
        const int NT = kFusedThreads;
        ZArgs<float> z{};
        z.in = inverse ? ui : fi;
        z.out = (inverse && zout) ? zout : ui;
        z.rows = (long long)g.count * g.nx * g.ny;
        z.nz = g.nz;
        z.M = g.M;
        z.W = NT / g.pz.TL;
        z.pl = g.pz;
        z.tw = tab + g.tw_z;
        z.post = tab + g.post;
        SArgs<float> y{};
        y.data = ui;
        y.nplanes = (long long)g.count * g.nx;
        y.sPlane = (long long)g.ny * g.M;
        y.sL = g.M;
        y.M = g.M;
        y.W = std::min(g.M, NT / g.py.TL);
        y.ncb = (g.M + y.W - 1) / y.W;
        y.pl = g.py;
        y.tw = tab + g.tw_y;
        FusedArgs fa{};
        fa.planes = (long long)g.count * g.nx;
        fa.cluster = g.fused;
        fa.ztiles = g.ny / z.W;
        fa.ytiles = y.ncb;
        const size_t smem = std::max((size_t)(g.M + (size_t)z.W * zpitch(g.M)) * sizeof(C),
                                     s_smem(g.ny, y.W, p->dtype));
        cudaError_t e = launch_fused_zy(z, y, fa, inverse, smem, s);
        if (e != cudaSuccess) return cuda_fail(e, inverse ? "fused y/z inverse pass" : "fused z/y forward pass");
        return PSOLVE_OK;
    }
}

} // namespace

// `uout`, if given, receives u from the last pass (the spectrum stays in u).
template <typename T>
psolve_status run_group(const psolve_plan *p, const Group &g, const T *f, T *u, cudaStream_t s,
                        const std::vector<cudaEvent_t> *ev, T *uout, bool host_io)
{
    const T *fi = f + g.off0;
    T *ui = u + g.off0;
    T *uo = uout ? uout + g.off0 : nullptr;
    if (ev) cudaEventRecord((*ev)[0], s);
    // (the cluster kernels copy f in with bulk copies: device memory only)
    if (g.fused > 0 && !(host_io && g.fused == zy_cluster_size())) {
        psolve_status st = launch_fused<T>(p, g, false, fi, ui, s);
        if (st != PSOLVE_OK) return st;
        if (ev) cudaEventRecord((*ev)[1], s);
        st = launch_pass<T>(p, g, 2, fi, ui, s);
        if (st != PSOLVE_OK) return st;
        if (ev) cudaEventRecord((*ev)[2], s);
        st = launch_fused<T>(p, g, true, fi, ui, s, uo);
        if (st != PSOLVE_OK) return st;
        if (ev) {
            cudaEventRecord((*ev)[3], s);
            cudaEventRecord((*ev)[4], s);
            cudaEventRecord((*ev)[5], s);
        }
        return PSOLVE_OK;
    }
    // one layout for the five passes of this solve
    const int G = sizeof(T) == 4 ? xs_factor(p, g, host_io) : 1;
    // x-split solves keep their spectrum in the plan's own buffer: the layout
    // change cannot be made in place
    T *work = G > 1 ? reinterpret_cast<T *>(p->xsbuf) + g.off0 : ui;
    for (int kind = 0; kind < kPasses; ++kind) {
        T *zo = kind == 4 ? (uo ? uo : (G > 1 ? ui : nullptr)) : nullptr;
        psolve_status st = launch_pass<T>(p, g, kind, fi, work, s, false, zo, host_io, G);
        if (st != PSOLVE_OK) return st;
        if (ev) cudaEventRecord((*ev)[kind + 1], s);
    }
    return PSOLVE_OK;
}

template psolve_status launch_pass<float>(const psolve_plan *, const Group &, int, const float *, float *,
                                          cudaStream_t, bool, float *, bool, int);
template psolve_status launch_pass<double>(const psolve_plan *, const Group &, int, const double *, double *,
                                           cudaStream_t, bool, double *, bool, int);
template psolve_status run_group<float>(const psolve_plan *, const Group &, const float *, float *, cudaStream_t,
                                        const std::vector<cudaEvent_t> *, float *, bool);
template psolve_status run_group<double>(const psolve_plan *, const Group &, const double *, double *,
                                         cudaStream_t, const std::vector<cudaEvent_t> *, double *, bool);

namespace {

psolve_status check_buffers(const psolve_plan *p, const void *f, const void *u)
{
    if (!f || !u) return fail(PSOLVE_ERR_INVALID_ARG, "null array pointer");
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15))
        return fail(PSOLVE_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    if (f != u) {
        const uintptr_t a0 = (uintptr_t)f, b0 = (uintptr_t)u;
        const uintptr_t len = (uintptr_t)(p->total * rsize(p->dtype));
        if (a0 < b0 + len && b0 < a0 + len) return fail(PSOLVE_ERR_INVALID_ARG, "f and u partially overlap");
    }
    return PSOLVE_OK;
}

} // namespace

// One graph: zero the counters, then the persistent kernel.  Built on first
// use; later solves only rewrite the kernel node's f/u pointers.
psolve_status run_batched(psolve_plan *p, const void *f, void *u, cudaStream_t s)
{
    int *status = p->status;
    unsigned long long *work = reinterpret_cast<unsigned long long *>(p->counters);
    int *done = reinterpret_cast<int *>(reinterpret_cast<char *>(p->counters) + 8);
    const void *segs = p->segs_dev;
    int nseg = p->nseg;
    long long total = p->total_items;
    const void *fa = f;
    void *ua = u;
    unsigned long long wait = p->wait_ns;
    void *args[] = {(void *)&segs, (void *)&nseg, (void *)&total, (void *)&fa, (void *)&ua,
                    (void *)&work, (void *)&done, (void *)&status, (void *)&wait};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(batched_kernel<float>());
    kp.gridDim = dim3(p->grid_batched);
    kp.blockDim = dim3(kBatchThreads);
    kp.sharedMemBytes = (unsigned)p->batch_smem;
    kp.kernelParams = args;
    cudaError_t e;
    if (!p->gexec) {
        e = cudaGraphCreate(&p->graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
        cudaMemsetParams mp{};
        mp.dst = p->counters;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = (8 + 4 * (size_t)p->nseg) / 4;
        mp.height = 1;
        mp.pitch = 0;
        cudaGraphNode_t mnode;
        e = cudaGraphAddMemsetNode(&mnode, p->graph, nullptr, 0, &mp);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&p->knode, p->graph, &mnode, 1, &kp);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, p->graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "build batched graph");
        p->g_f = f;
        p->g_u = u;
        p->g_wait = wait;
    } else if (p->g_f != f || p->g_u != u || p->g_wait != wait) {
        e = cudaGraphExecKernelNodeSetParams(p->gexec, p->knode, &kp);
        if (e != cudaSuccess) return cuda_fail(e, "update batched graph");
        p->g_f = f;
        p->g_u = u;
        p->g_wait = wait;
    }
    const std::vector<cudaEvent_t> *ev = take_events(p);
    if (ev) cudaEventRecord((*ev)[0], s);
    e = cudaGraphLaunch(p->gexec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if (ev)
        for (int i = 1; i <= kPasses; ++i) cudaEventRecord((*ev)[i], s);
    return PSOLVE_OK;
}

psolve_status solve(psolve_plan *p, const void *f, void *u, void *stream)
{
    if (!plan_ok(p)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    psolve_status st = check_buffers(p, f, u);
    if (st != PSOLVE_OK) return st;
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "select device");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->batched) return run_batched(p, f, u, s);
    for (const auto &g : p->groups) {
        const std::vector<cudaEvent_t> *ev = take_events(p);
        st = p->dtype == PSOLVE_F64
                 ? run_group<double>(p, g, (const double *)f, (double *)u, s, ev)
                 : run_group<float>(p, g, (const float *)f, (float *)u, s, ev);
        if (st != PSOLVE_OK) return st;
    }
    return PSOLVE_OK;
}


namespace {

// Device address of a pinned host buffer, or nullptr for pageable memory.
const void *device_view(const void *host)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (attr.type != cudaMemoryTypeHost || attr.devicePointer == nullptr) return nullptr;
    return attr.devicePointer;
}

} // namespace

// One host-buffer solve on `s` through the device buffer `stage` (no sync).
// zero_copy: pinned buffers are read and written by the first and last
// passes across the host link (fastest for one solve at a time); otherwise
// the copy engines move f in and u out (they overlap with other streams'
// copies and kernels, so pipelined solves go faster this way: measured on
// GB300 at 512^3, 3.8 ms per pipelined solve against 5.9 ms zero-copy).
psolve_status host_solve(psolve_plan *plan, const void *f_host, void *u_host, void *stage, cudaStream_t s,
                         bool zero_copy)
{
    const size_t bytes = plan->total * rsize(plan->dtype);
    const void *fdev = zero_copy ? device_view(f_host) : nullptr;
    void *udev = zero_copy ? const_cast<void *>(device_view(u_host)) : nullptr;
    const char *zc = std::getenv("PSOLVE_ZERO_COPY");
    if (fdev && udev && !plan->batched && !(zc && zc[0] == '0')) {
        for (const auto &g : plan->groups) {
            psolve_status st = plan->dtype == PSOLVE_F64
                                   ? run_group<double>(plan, g, (const double *)fdev, (double *)stage, s,
                                                       take_events(plan), (double *)udev, true)
                                   : run_group<float>(plan, g, (const float *)fdev, (float *)stage, s,
                                                      take_events(plan), (float *)udev, true);
            if (st != PSOLVE_OK) return st;
        }
        return PSOLVE_OK;
    }
    cudaError_t e = cudaMemcpyAsync(stage, f_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy f to device");
    // Passes of host-buffer solves run strictly in order: with early set-up
    // their waiting blocks would hold SMs that another stream's solve of the
    // pipeline needs (measured: 3.4 -> 6.6 ms per pipelined solve).
    plan->serial = true;
    psolve_status st = solve(plan, stage, stage, s);
    plan->serial = false;
    if (st != PSOLVE_OK) return st;
    e = cudaMemcpyAsync(u_host, stage, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy u to host");
    return PSOLVE_OK;
}

} // namespace psolve
