// The planner: stage plans of the lines, tile shapes of the per-tile
// kernels, the choice of pass kernels per axis, the persistent batched
// schedule, and plan creation and release.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>

namespace psolve {

const char *const kPassNames[kPasses] = {"zfwd", "yfwd", "xdiv", "yinv", "zinv"};

bool factor23(int n, int &a, int &b)
{
    a = b = 0;
    if (n <= 0) return false;
    while (n % 2 == 0) { n /= 2; ++a; }
    while (n % 3 == 0) { n /= 3; ++b; }
    return n == 1;
}

bool size_ok(int n)
{
    int a, b;
    return n >= 4 && n <= 2048 && (n % 2) == 0 && factor23(n, a, b);
}

namespace {

// Plan of an L-point line from its radices rad[0..n) (a fixed array:
// planning allocates nothing, so the plan-free solve uses it too); false if
// there are more than kMaxStages.
bool fill_plan(int L, int E, const int *rad, int n, LinePlan &p)
{
    if (n > kMaxStages) return false;
    std::memset(&p, 0, sizeof(p));
    p.L = L;
    p.E = E;
    p.TL = L / E;
    p.nst = n;
    int ns = 1;
    for (int s = 0; s < n; ++s) {
        p.radix[s] = rad[s];
        p.ns[s] = ns;
        p.twstep[s] = L / (ns * rad[s]);
        ns *= rad[s];
    }
    line_plan_finish(p);
    return true;
}

} // namespace

// Any radix order is a valid Stockham factorisation; the autotuner times them.
bool make_line_plan(int L, LinePlan &p, int order, int e3cap)
{
    int a, b;
    if (!factor23(L, a, b) || L < 2) return false;
    const int E = b > 0 ? 3 * (1 << std::min(a, e3cap)) : (1 << std::min(a, 4));
    if (!supported_E(E)) return false;
    int p2 = 1;
    while (E % (p2 * 2) == 0 && p2 * 2 <= 16) p2 *= 2;
    int rad[64];
    int n = 0;
    for (int i = 0; i < b; ++i) rad[n++] = 3;
    for (int rem = 1 << a; rem > 1;) {
        const int r = std::min(p2, rem);
        rad[n++] = r;
        rem /= r;
    }
    if (order == 1) std::reverse(rad, rad + n);
    if (order == 2) std::rotate(rad, rad + b, rad + n);
    return fill_plan(L, E, rad, n, p);
}

size_t csize(int dtype) { return dtype == PSOLVE_F64 ? 16 : 8; }

// Stage plan with a given number of points per thread E (a power of two
// dividing L): the largest power-of-two radices (<= 16) dividing E.
bool make_line_plan_E(int L, int E, LinePlan &p)
{
    int a, b;
    if (!factor23(L, a, b) || b != 0 || L % E != 0 || !supported_E(E)) return false;
    int p2 = 1;
    while (E % (p2 * 2) == 0 && p2 * 2 <= 16) p2 *= 2;
    int rad[64];
    int n = 0;
    for (int rem = L; rem > 1;) {
        const int r = std::min(p2, rem);
        rad[n++] = r;
        rem /= r;
    }
    return fill_plan(L, E, rad, n, p);
}

size_t rsize(int dtype) { return dtype == PSOLVE_F64 ? 8 : 4; }

int zpitch(int M) { return M + (M >> 4) + 1; }
size_t z_smem(const Group &g, int dtype) { return (size_t)(g.M + (size_t)g.Wz * zpitch(g.M)) * csize(dtype); }
size_t s_smem(int L, int W, int dtype) { return (size_t)L * (1 + W) * csize(dtype); }

bool tiles_fit(const Group &g, int dtype)
{
    const bool fp64 = dtype == PSOLVE_F64;
    return g.Wz * g.pz.TL <= max_threads(fp64, g.pz.E) && g.Wy * g.py.TL <= max_threads(fp64, g.py.E) &&
           g.Wx * g.px.TL <= max_threads(fp64, g.px.E);
}

bool fused_ok(const Group &g, int dtype, bool uniform, int fused)
{
    if (!uniform || dtype != PSOLVE_F32) return false;
    if (fused == zy_cluster_size()) return zy_cluster_supported(g.M, g.ny) && g.zy_clusters > 0;
    return (fused == 2 || fused == 4 || fused == 8) && fused_supported(g.M, g.ny) && g.pz.E == 16 &&
           g.py.E == 16;
}

namespace {

// Optional override "Wz,Wy,Wx" from PSOLVE_TILE_W (tuning runs); a value
// that breaks a launch limit is ignored.
void override_tiles(Group &g, int dtype)
{
    const char *env = std::getenv("PSOLVE_TILE_W");
    if (!env) return;
    int wz = 0, wy = 0, wx = 0;
    if (std::sscanf(env, "%d,%d,%d", &wz, &wy, &wx) != 3) return;
    const bool fp64 = dtype == PSOLVE_F64;
    if (wz >= 1 && wz * g.pz.TL <= max_threads(fp64, g.pz.E)) {
        const int keep = g.Wz;
        g.Wz = wz;
        if (z_smem(g, dtype) > kSmemCap) g.Wz = keep;
    }
    if (wy >= 1 && wy <= g.M && wy * g.py.TL <= max_threads(fp64, g.py.E) &&
        s_smem(g.ny, wy, dtype) <= kSmemCap)
        g.Wy = wy;
    if (wx >= 2 && wx * g.px.TL <= max_threads(fp64, g.px.E) && s_smem(g.nx, wx, dtype) <= kSmemCap)
        g.Wx = wx;
}

} // namespace

void choose_tiles(Group &g, int dtype, bool env_override)
{
    const bool fp64 = dtype == PSOLVE_F64;
    // z: about 128 threads, W rows each of TL threads (8 rows of 256 points).
    {
        const int mt = max_threads(fp64, g.pz.E);
        g.Wz = std::max(1, std::min(128, mt) / g.pz.TL);
        while (g.Wz > 1 && z_smem(g, dtype) > kSmemCap) g.Wz /= 2;
    }
    // y and x: W adjacent columns (16 columns = 128 B runs in FP32).
    {
        const int mt = max_threads(fp64, g.py.E);
        int W = std::min(16, std::max(1, mt / g.py.TL));
        W = std::min(W, g.M);
        while (W > 1 && s_smem(g.ny, W, dtype) > kSmemCap) W /= 2;
        g.Wy = std::max(1, W);
    }
    {
        const int mt = max_threads(fp64, g.px.E);
        int W = std::min(16, std::max(2, mt / g.px.TL));
        W = std::max(2, std::min(W, std::max(2, g.M)));
        while (W > 2 && s_smem(g.nx, W, dtype) > kSmemCap) W /= 2;
        g.Wx = W;
    }
    if (env_override) override_tiles(g, dtype);
}

void destroy_events(psolve_plan *p)
{
    for (auto *pool : {&p->ev_used, &p->ev_free})
        for (auto &set : *pool)
            for (auto e : set) cudaEventDestroy(e);
    p->ev_used.clear();
    p->ev_free.clear();
}

void release(psolve_plan *p)
{
    if (!p) return;
    destroy_events(p);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->segs_dev) cudaFree(p->segs_dev);
    if (p->counters) cudaFree(p->counters);
    if (p->tables) cudaFree(p->tables);
    if (p->status) cudaFree(p->status);
    if (p->stage) cudaFree(p->stage);
    if (p->xsbuf) cudaFree(p->xsbuf);
    if (p->optab) cudaFree(p->optab);
    for (int i = 0; i < kAsyncRing; ++i) {
        if (p->astage[i]) cudaFree(p->astage[i]);
        if (p->aev[i]) cudaEventDestroy(p->aev[i]);
    }
    p->magic = 0;
    delete p;
}

// Whether the persistent TMA pass applies to lines of length L over M columns.
int tma_variant(int setting, int L) { return setting >= 0 ? setting : (tma_columns(L, 1) >= 8 ? 1 : 0); }

// Untuned FP32 choice per axis (measured on GB300): radix-32 tiles for the
// long lines, 64 KiB ones for y and 1024-point x lines, 32 KiB ones for the
// 512-point x lines (two blocks per SM hide the double transform's latency).
// TMA configurations with tensor-core variants: 16 points per thread (0, 1)
// for every line length, 32 points per thread (3, 4) for 512-point lines.
bool tc_cfg_ok(int cfg, int L) { return cfg == 0 || cfg == 1 || (L == 512 && (cfg == 3 || cfg == 4)); }

int tma_default(int L, bool x_axis)
{
    if (L >= 1024) return 4;
    if (L == 512) return x_axis ? 3 : 4;
    return 1;
}

bool tma_fits(const psolve_plan *p, int L, int M, int narrow)
{
    return p->use_tma && p->dtype != PSOLVE_F64 && tma_supported(L) && (M % 2) == 0 &&
           M >= tma_columns(L, narrow);
}

// Segments of the persistent batched launch: pass-major, one per (pass,
// instance), each with a tile width that fits kBatchThreads threads.
// The group's spectral multiplier as the kernels read it.
OpArgs op_args(const psolve_plan *p, const Group &g)
{
    OpArgs o{};
    o.op = p->op;
    o.c4 = p->op == 1 ? p->op_c / (4.0 * M_PI * M_PI) : 0.0;
    if (p->op == 2 && p->optab) {
        o.lx = p->optab + g.op_lx;
        o.ly = p->optab + g.op_ly;
        o.lz = p->optab + g.op_lz;
        const float *t32 = reinterpret_cast<const float *>(p->optab + p->optab_n);
        o.lx32 = t32 + g.op_lx;
        o.ly32 = t32 + g.op_ly;
        o.lz32 = t32 + g.op_lz;
    }
    return o;
}

template <typename T> psolve_status setup_batched(psolve_plan *p)
{
    using C = typename cplx_of<T>::type;
    const C *tab = reinterpret_cast<const C *>(p->tables);
    const int B = (int)p->groups.size();
    const size_t cs = sizeof(C);
    const int NT = kBatchThreads;
    std::vector<BatchSeg<T>> segs(5 * (size_t)B);
    long long first = 0;
    size_t smem = 0;
    // Line plans in the radix order the knobs select (the tables are per
    // length), on a copy: the plan's groups change only once the whole
    // schedule is known to fit.
    std::vector<Group> gs = p->groups;
    for (auto &g : gs) {
        make_line_plan(g.M, g.pz, p->bknob[3], 2);
        make_line_plan(g.ny, g.py, p->bknob[4], 2);
        make_line_plan(g.nx, g.px, p->bknob[5], 2);
    }
    // Radix order 0 with a compile-time plan for the line: the kernel's
    // instantiation for that length (same stages, constants folded).
    const char *cte = std::getenv("PSOLVE_BATCH_CT");
    const bool use_ct = !(cte && cte[0] == '0');
    auto lc_of = [&](const LinePlan &pl, int order) {
        return (use_ct && order == 0 && batched_ct_supported(pl.L, pl.E)) ? pl.L : 0;
    };
    // segments by (pass, instance) first; ordered below
    std::vector<BatchSeg<T>> raw(5 * (size_t)B);
    for (int pass = 0; pass < 5; ++pass) {
        for (int i = 0; i < B; ++i) {
            const Group &g = gs[i];
            BatchSeg<T> sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.kind = pass;
            sg.dep = -1;
            sg.off = (long long)g.off0;
            const int M = g.M;
            if (pass == 0 || pass == 4) {
                int W = std::max(1, NT / g.pz.TL / p->bknob[0]);
                const int LP = M + (M >> 4) + 1;
                while (W > 1 && (size_t)(M + (size_t)W * LP) * cs > kSmemCap) W /= 2;
                sg.E = g.pz.E;
                sg.lc = lc_of(g.pz, p->bknob[3]);
                sg.z.rows = (long long)g.nx * g.ny;
                sg.z.nz = g.nz;
                sg.z.M = M;
                sg.z.W = W;
                sg.z.pl = g.pz;
                sg.z.tw = tab + g.tw_z;
                sg.z.post = tab + g.post;
                sg.ntiles = (sg.z.rows + W - 1) / W;
                smem = std::max(smem, (size_t)(M + (size_t)W * LP) * cs);
            } else if (pass == 1 || pass == 3) {
                int W = std::min(M, std::max(1, NT / g.py.TL / p->bknob[1]));
                while (W > 1 && s_smem(g.ny, W, p->dtype) > kSmemCap) W /= 2;
                sg.E = g.py.E;
                sg.lc = lc_of(g.py, p->bknob[4]);
                sg.y.nplanes = g.nx;
                sg.y.sPlane = (long long)g.ny * M;
                sg.y.sL = M;
                sg.y.M = M;
                sg.y.W = W;
                sg.y.ncb = (M + W - 1) / W;
                sg.y.pl = g.py;
                sg.y.tw = tab + g.tw_y;
                sg.ntiles = (long long)g.nx * sg.y.ncb;
                smem = std::max(smem, s_smem(g.ny, W, p->dtype));
            } else {
                int W = std::max(2, std::min(std::max(2, M), NT / g.px.TL / p->bknob[2]));
                while (W > 2 && s_smem(g.nx, W, p->dtype) > kSmemCap) W /= 2;
                // (the caller then launches per pass and instance)
                if (W * g.px.TL > NT) return fail(PSOLVE_ERR_UNSUPPORTED_SIZE, "x line too long for a batch tile");
                sg.E = g.px.E;
                sg.lc = lc_of(g.px, p->bknob[5]);
                sg.x.batch = 1;
                sg.x.nx = g.nx;
                sg.x.ny = g.ny;
                sg.x.M = M;
                sg.x.sInst = (long long)g.nx * g.ny * M;
                sg.x.W = W;
                sg.x.ncb = (M + W - 1) / W;
                sg.x.main_tiles = (long long)g.ny * sg.x.ncb;
                sg.x.npairs = g.ny / 2 + 1;
                sg.x.pl = g.px;
                sg.x.tw = tab + g.tw_x;
                sg.x.coef = (T)(1.0 / (4.0 * M_PI * M_PI * ((double)g.nx * g.ny * g.nz)));
                sg.x.op = op_args(p, g);
                sg.ntiles = sg.x.main_tiles + (sg.x.npairs + W / 2 - 1) / (W / 2);
                smem = std::max(smem, s_smem(g.nx, W, p->dtype));
            }
            raw[(size_t)pass * B + i] = sg;
        }
    }
    // Within a pass the instances are ordered by tile variant (points per
    // thread, compile-time line length), so that the blocks, which take items
    // in order, run one variant's code at a time; passes stay in order, so
    // every segment's dependency (the same instance's previous pass) lies on
    // earlier items.  PSOLVE_BATCH_SORT = 0 keeps the instance order.
    const char *se = std::getenv("PSOLVE_BATCH_SORT");
    const bool by_variant = !(se && se[0] == '0');
    std::vector<int> pos(5 * (size_t)B);
    std::vector<int> order(B);
    for (int pass = 0; pass < 5; ++pass) {
        for (int i = 0; i < B; ++i) order[i] = i;
        if (by_variant)
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                const BatchSeg<T> &a = raw[(size_t)pass * B + x], &b = raw[(size_t)pass * B + y];
                return a.E != b.E ? a.E < b.E : a.lc < b.lc;
            });
        for (int k = 0; k < B; ++k) {
            const size_t idx = (size_t)pass * B + k;
            segs[idx] = raw[(size_t)pass * B + order[k]];
            segs[idx].first = first;
            first += segs[idx].ntiles;
            pos[(size_t)pass * B + order[k]] = (int)idx;
        }
    }
    for (int pass = 1; pass < 5; ++pass)
        for (int i = 0; i < B; ++i) {
            BatchSeg<T> &sg = segs[pos[(size_t)pass * B + i]];
            sg.dep = pos[(size_t)(pass - 1) * B + i];
            sg.need = (int)segs[sg.dep].ntiles;
        }
    p->groups = gs;
    p->nseg = (int)segs.size();
    p->total_items = first;
    p->batch_smem = smem;
    const size_t bytes = segs.size() * sizeof(BatchSeg<T>);
    p->segs_host.assign(reinterpret_cast<unsigned char *>(segs.data()),
                        reinterpret_cast<unsigned char *>(segs.data()) + bytes);
    if (cudaMalloc(&p->segs_dev, bytes) != cudaSuccess) {
        p->segs_dev = nullptr;
        return fail(PSOLVE_ERR_OOM, "batch segment table");
    }
    if (cudaMalloc(&p->counters, 8 + 4 * (size_t)p->nseg) != cudaSuccess) {
        p->counters = nullptr;
        return fail(PSOLVE_ERR_OOM, "batch counters");
    }
    cudaError_t e = cudaMemcpy(p->segs_dev, segs.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload batch segments");
    e = batched_prepare<T>(smem);
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel attributes");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T>(), kBatchThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "batched kernel occupancy");
    p->grid_batched = (unsigned)std::min<long long>(first, (long long)p->num_sms * per_sm);
    p->batched = true;
    return PSOLVE_OK;
}

template psolve_status setup_batched<float>(psolve_plan *p);

psolve_status build_plan(const std::vector<int> &nx, const std::vector<int> &ny, const std::vector<int> &nz,
                         int dtype, bool uniform, psolve_plan **out)
{
    const int batch = (int)nx.size();
    const size_t align = 32;
    std::unique_ptr<psolve_plan> p(new psolve_plan());
    p->magic = kMagic;
    p->uniform = uniform;
    p->dtype = dtype;
    p->batch = batch;
    p->tables = nullptr;
    p->status = nullptr;
    p->stage = nullptr;
    p->xsbuf = nullptr;
    p->op = 0;
    p->op_c = 0.0;
    p->optab = nullptr;
    p->optab_n = 0;
    p->stage_bytes = 0;
    for (int i = 0; i < kAsyncRing; ++i) {
        p->astage[i] = nullptr;
        p->aev[i] = nullptr;
        p->aev_used[i] = false;
    }
    p->aring = 0;
    p->profiling = false;
    p->serial = false;
    p->prof_every = 0;
    p->prof_count = 0;
    p->batched = false;
    p->segs_dev = nullptr;
    p->counters = nullptr;
    p->graph = nullptr;
    p->gexec = nullptr;
    p->knode = nullptr;
    p->g_f = nullptr;
    p->g_u = nullptr;
    p->nseg = 0;
    p->total_items = 0;
    p->batch_smem = 0;
    p->grid_batched = 0;
    p->wait_ns = 2000000000ull;
    p->g_wait = 0;
    for (int k = 0; k < 6; ++k) p->bknob[k] = k < 3 ? 1 : 0;
    size_t off = 0;
    for (int b = 0; b < batch; ++b) {
        const size_t N = (size_t)nx[b] * ny[b] * nz[b];
        if (uniform) {
            if (b == 0) {
                Group g{};
                g.nx = nx[0]; g.ny = ny[0]; g.nz = nz[0]; g.M = nz[0] / 2;
                g.count = batch; g.off0 = 0; g.stride = N;
                p->groups.push_back(g);
            }
            p->inst_off.push_back((size_t)b * N);
            off = (size_t)(b + 1) * N;
        } else {
            Group g{};
            g.nx = nx[b]; g.ny = ny[b]; g.nz = nz[b]; g.M = nz[b] / 2;
            g.count = 1; g.off0 = off; g.stride = N;
            p->groups.push_back(g);
            p->inst_off.push_back(off);
            off += (N + align - 1) / align * align;
        }
    }
    p->total = uniform ? off : (p->inst_off.back() + (size_t)nx.back() * ny.back() * nz.back());

    // Stage plans, tile shapes and the table layout.
    std::map<int, size_t> roots_at; // L -> offset
    std::map<int, size_t> post_at;  // nz -> offset
    size_t tcount = 0;
    for (auto &g : p->groups) {
        // Unequal grids share the persistent batched kernel, which holds at
        // most 16 points per thread (12 for lengths 3·2^a).
        const int e3cap = uniform ? 3 : 2;
        if (!make_line_plan(g.M, g.pz, 0, e3cap) || !make_line_plan(g.ny, g.py, 0, e3cap) ||
            !make_line_plan(g.nx, g.px, 0, e3cap))
            return fail(PSOLVE_ERR_UNSUPPORTED_SIZE, "no stage plan for this size");
        choose_tiles(g, dtype);
        if (!tiles_fit(g, dtype))
            return fail(PSOLVE_ERR_UNSUPPORTED_SIZE,
                        "no tile of this grid fits a block (FP64 x lines of 1458 = 2·3^6 points: 486 threads for "
                        "the two columns the x pass needs, 256 allowed)");
        for (int L : {g.M, g.ny, g.nx})
            if (!roots_at.count(L)) { roots_at[L] = tcount; tcount += L; }
        if (!post_at.count(g.nz)) { post_at[g.nz] = tcount; tcount += g.M; }
        g.tw_z = roots_at[g.M];
        g.tw_y = roots_at[g.ny];
        g.tw_x = roots_at[g.nx];
        g.post = post_at[g.nz];
    }

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    {
        const char *env = std::getenv("PSOLVE_TMA");
        p->use_tma = !(env && env[0] == '0');
        // "y,x" tile variants of the TMA passes (0 wide, 1 narrow); narrow
        // tiles only while their rows stay >= 64 bytes (W >= 8 columns).
        p->tma_narrow_y = -1;
        p->tma_narrow_x = -1;
        const char *nv = std::getenv("PSOLVE_TMA_NARROW");
        int ny_ = 0, nx_ = 0;
        if (nv && std::sscanf(nv, "%d,%d", &ny_, &nx_) == 2) {
            p->tma_narrow_y = ny_ < 0 || ny_ > 4 ? 0 : ny_;
            p->tma_narrow_x = nx_ < 0 || nx_ > 4 ? 0 : nx_;
        }
    }
    for (auto &g : p->groups) {
        {
            const char *zb = std::getenv("PSOLVE_ZBULK");
            const long long rows = (long long)g.count * g.nx * g.ny;
            g.zbulk = (dtype != PSOLVE_F64 && z_bulk_supported(g.M) && g.pz.E == 16 &&
                       rows % z_bulk_rows(g.M, false) == 0 && rows % z_bulk_rows(g.M, true) == 0 &&
                       !(zb && zb[0] == '0'))
                          ? 1
                          : 0;
        }
        {
            // x-split spectrum layout (spec_row), used by solves whose passes
            // all support it; PSOLVE_XSPLIT = 1 keeps the natural layout, 2..16
            // asks for that factor
            const char *xe = std::getenv("PSOLVE_XSPLIT");
            const double xstride = (double)g.ny * g.M * csize(dtype);
            const int G = xe ? std::atoi(xe) : (xstride >= kXSplitStride ? kXSplit : 1);
            g.xs = (G == 2 || G == 4 || G == 8 || G == 16) ? G : 1;
        }
        g.fused = 0;
        g.zy_clusters = 0;
        if (uniform && dtype == PSOLVE_F32 && zy_cluster_supported(g.M, g.ny)) {
            int cf = 0, ci = 0;
            if (zy_cluster_max_active(g.M, g.ny, false, &cf) == cudaSuccess &&
                zy_cluster_max_active(g.M, g.ny, true, &ci) == cudaSuccess)
                g.zy_clusters = std::min(cf, ci);
            cudaGetLastError();
        }
        {
            // Off by default (the L2 hand-off measured slower than the
            // separate TMA passes on GB300 at 512^3 and 1024^3); the
            // autotuner times every fusion that applies.
            const char *fe = std::getenv("PSOLVE_FUSED");
            const int want = fe ? std::atoi(fe) : 0;
            if (fused_ok(g, dtype, uniform, want)) g.fused = want;
        }
        auto pick = [&](int setting, int L, bool x_axis) {
            if (dtype == PSOLVE_F32_TC) {
                // 32 points per thread and 32 KiB tiles (one tensor-core stage
                // per 512-point line; measured fastest on both axes) unless a
                // configuration is asked for
                int c = tma_variant(setting, L);
                if (setting < 0 && L == 512 && tma_fits(p.get(), L, g.M, 3)) c = 3;
                return tma_fits(p.get(), L, g.M, c) && tc_cfg_ok(c, L) ? c : -1;
            }
            if (setting >= 0) {
                const int c = tma_variant(setting, L);
                return tma_fits(p.get(), L, g.M, c) ? c : -1;
            }
            // preferred configuration, else the narrower tiles that fit
            for (int c : {tma_default(L, x_axis), 3, 1})
                if (tma_fits(p.get(), L, g.M, c)) return c;
            return -1;
        };
        g.cfg_y = pick(p->tma_narrow_y, g.ny, false);
        g.cfg_x = pick(p->tma_narrow_x, g.nx, true);
    }
    apply_tuning_cache(p.get());
    {
        bool want_xs = false;
        for (const auto &g : p->groups) want_xs = want_xs || (g.xs > 1 && g.zbulk);
        if (want_xs && dtype != PSOLVE_F64 && cudaMalloc(&p->xsbuf, p->total * rsize(dtype)) != cudaSuccess) {
            p->xsbuf = nullptr; // natural layout in u instead
            cudaGetLastError();
        }
    }
    e = cudaMalloc(&p->tables, tcount * csize(dtype));
    if (e != cudaSuccess) {
        p->tables = nullptr;
        release(p.release());
        return fail(PSOLVE_ERR_OOM, "twiddle tables: cudaMalloc failed");
    }
    e = cudaMalloc((void **)&p->status, sizeof(int));
    if (e != cudaSuccess) {
        p->status = nullptr;
        release(p.release());
        return fail(PSOLVE_ERR_OOM, "status word: cudaMalloc failed");
    }
    cudaMemset(p->status, 0, sizeof(int));
    char *tb = (char *)p->tables;
    const size_t cs = csize(dtype);
    for (auto &kv : roots_at) {
        e = dtype == PSOLVE_F64 ? launch_roots<double>(tb + kv.second * cs, kv.first, kv.first, 0)
                                : launch_roots<float>(tb + kv.second * cs, kv.first, kv.first, 0);
        if (e != cudaSuccess) { release(p.release()); return cuda_fail(e, "twiddle generation"); }
    }
    for (auto &kv : post_at) {
        e = dtype == PSOLVE_F64 ? launch_roots<double>(tb + kv.second * cs, kv.first / 2, kv.first, 0)
                                : launch_roots<float>(tb + kv.second * cs, kv.first / 2, kv.first, 0);
        if (e != cudaSuccess) { release(p.release()); return cuda_fail(e, "twiddle generation"); }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { release(p.release()); return cuda_fail(e, "plan set-up"); }
    if (!uniform) {
        const char *env = std::getenv("PSOLVE_BATCHED");
        if (!(env && env[0] == '0')) {
            bool ok = dtype != PSOLVE_F64;
            for (const auto &g : p->groups)
                ok = ok && batched_supports_E(g.pz.E) && batched_supports_E(g.py.E) && batched_supports_E(g.px.E);
            if (ok) {
                // a grid whose x lines do not fit a batch tile keeps the
                // launches per pass and instance
                psolve_status st = setup_batched<float>(p.get());
                if (st == PSOLVE_ERR_UNSUPPORTED_SIZE) {
                    drop_batched(p.get());
                } else if (st != PSOLVE_OK) {
                    release(p.release());
                    return st;
                }
            }
        }
    }
    *out = p.release();
    return PSOLVE_OK;
}

} // namespace psolve
