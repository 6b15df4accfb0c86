// C-ABI of the solver: plan creation (size checks, 1D stage plans, tile
// shapes, FP64 twiddle generation on the device) and the five-pass solve.
// See include/psolve.h for the contract of every entry point.
#include "psolve.h"
#include "launch.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>
#include <unistd.h>

using namespace psolve;

namespace {

thread_local std::string g_last_error;

psolve_status fail(psolve_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

psolve_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(PSOLVE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr unsigned kMagic = 0x50534F4Cu; // "PSOL"
constexpr size_t kSmemCap = 200 * 1024;

// Device staging buffers of psolve_execute_host_async, used in turn: three
// let a pipeline of solves keep both directions of the host link busy while
// a third solve computes.
constexpr int kAsyncRing = 3;

// x-split factor of the spectrum layout (spec_row) for grids whose x lines
// are at least kXSplitStride bytes apart in the natural layout (measured on
// GB300: at 1024³, 4 MiB apart, the x pass drops from 3.47 to 2.36 ms while
// the y and z passes lose 0.5 ms; at 512³, 1 MiB apart, it is a loss).
constexpr int kXSplit = 4;
constexpr double kXSplitStride = 4.0 * 1048576.0;

// Instances of equal dimensions laid out back to back at `stride` elements.
struct Group {
    int nx, ny, nz, M;
    int count;
    size_t off0, stride;
    LinePlan pz, py, px;
    size_t tw_z, tw_y, tw_x, post; // complex-element offsets into the table buffer
    size_t op_lx, op_ly, op_lz;    // offsets of the group's finite-difference symbol tables (op 2)
    int Wz, Wy, Wx;
    int cfg_y, cfg_x;    // TMA configuration of the y / x pass (-1: per-tile kernel)
    int fused;           // z and y passes fused per plane through L2: cluster size, 0 = off
    int zbulk;           // z passes by the persistent bulk-copy kernel (1) or per-tile blocks (0)
    int xs;              // x-split factor of the spectrum layout when every pass can use it (1: natural)
};

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

// Stage plan of an L-point line: radix-3 stages for the factors of 3, then
// the largest power-of-two radices (<= 16) that divide E (order 0).  Order 1
// runs the same radices in reverse, order 2 puts the radix-3 stages last;
// any order is a valid Stockham factorisation, and the autotuner times them.
bool make_line_plan(int L, LinePlan &p, int order = 0, int e3cap = 3)
{
    int a, b;
    if (!factor23(L, a, b) || L < 2) return false;
    const int E = b > 0 ? 3 * (1 << std::min(a, e3cap)) : (1 << std::min(a, 4));
    if (!supported_E(E)) return false;
    std::memset(&p, 0, sizeof(p));
    p.L = L;
    p.E = E;
    p.TL = L / E;
    int p2 = 1;
    while (E % (p2 * 2) == 0 && p2 * 2 <= 16) p2 *= 2;
    std::vector<int> rad(b, 3);
    int rem = 1 << a;
    while (rem > 1) {
        const int r = std::min(p2, rem);
        rad.push_back(r);
        rem /= r;
    }
    if ((int)rad.size() > kMaxStages) return false;
    if (order == 1) std::reverse(rad.begin(), rad.end());
    if (order == 2) std::rotate(rad.begin(), rad.begin() + b, rad.end());
    p.nst = (int)rad.size();
    int ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        p.radix[s] = rad[s];
        p.ns[s] = ns;
        p.twstep[s] = L / (ns * rad[s]);
        ns *= rad[s];
    }
    line_plan_finish(p);
    return true;
}

size_t csize(int dtype) { return dtype == PSOLVE_F64 ? 16 : 8; }

} // namespace

// Stage plan with a given number of points per thread E (a power of two
// dividing L): the largest power-of-two radices (<= 16) dividing E.
bool make_line_plan_E(int L, int E, LinePlan &p)
{
    int a, b;
    if (!factor23(L, a, b) || b != 0 || L % E != 0 || !supported_E(E)) return false;
    std::memset(&p, 0, sizeof(p));
    p.L = L;
    p.E = E;
    p.TL = L / E;
    int p2 = 1;
    while (E % (p2 * 2) == 0 && p2 * 2 <= 16) p2 *= 2;
    std::vector<int> rad;
    int rem = L;
    while (rem > 1) {
        const int r = std::min(p2, rem);
        rad.push_back(r);
        rem /= r;
    }
    if ((int)rad.size() > kMaxStages) return false;
    p.nst = (int)rad.size();
    int ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        p.radix[s] = rad[s];
        p.ns[s] = ns;
        p.twstep[s] = L / (ns * rad[s]);
        ns *= rad[s];
    }
    line_plan_finish(p);
    return true;
}

namespace {
size_t rsize(int dtype) { return dtype == PSOLVE_F64 ? 8 : 4; }

int zpitch(int M) { return M + (M >> 4) + 1; }
size_t z_smem(const Group &g, int dtype) { return (size_t)(g.M + (size_t)g.Wz * zpitch(g.M)) * csize(dtype); }
size_t s_smem(int L, int W, int dtype) { return (size_t)L * (1 + W) * csize(dtype); }

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

void choose_tiles(Group &g, int dtype)
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
    override_tiles(g, dtype);
}

} // namespace

struct psolve_plan {
    unsigned magic;
    bool uniform; // psolve_plan_create (equal grids back to back)
    int dtype;
    int device;
    int num_sms;
    bool use_tma;
    int tma_narrow_y, tma_narrow_x; // tile variant per pass (see launch.h)
    int batch;
    std::vector<Group> groups;
    std::vector<size_t> inst_off;
    size_t total;
    void *tables;
    void *xsbuf; // spectrum in the x-split layout (plans that use it): the z passes go f -> xsbuf -> u
    int op;          // spectral multiplier (OpArgs): 0 Poisson, 1 Helmholtz, 2 finite-difference Laplacian
    double op_c;     // Helmholtz c
    double *optab;   // finite-difference symbol tables of all groups (op 2): optab_n FP64, then FP32
    size_t optab_n;
    int *status;
    void *stage;
    size_t stage_bytes;
    // asynchronous host-buffer solves: two staging buffers used in turn, each
    // guarded by an event recorded after its last use
    void *astage[kAsyncRing];
    cudaEvent_t aev[kAsyncRing];
    bool aev_used[kAsyncRing];
    unsigned aring;
    // persistent batched path (plans of unequal grids)
    bool batched;
    void *segs_dev;                 // BatchSeg<T>[nseg]
    std::vector<unsigned char> segs_host;
    int nseg;
    long long total_items;
    size_t batch_smem;
    unsigned grid_batched;
    void *counters;                 // work counter (8 B) + done[nseg]
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    cudaGraphNode_t knode;
    const void *g_f;
    void *g_u;
    unsigned long long wait_ns;
    unsigned long long g_wait;
    int bknob[6]; // batched launch: tile-width divisor (z, y, x) and radix order (z, y, x)
    // per-pass profiling: one set of kPasses+1 events per recorded solve,
    // every prof_every-th solve
    bool profiling;
    bool serial; // launch the passes strictly in order (host-buffer solves: no early set-up)
    int prof_every;
    unsigned prof_count;
    std::vector<std::vector<cudaEvent_t>> ev_used;
    std::vector<std::vector<cudaEvent_t>> ev_free;
};

namespace {

bool plan_ok(const psolve_plan *p) { return p != nullptr && p->magic == kMagic; }

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            changed = err == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

constexpr int kPasses = 5;
const char *kPassNames[kPasses] = {"zfwd", "yfwd", "xdiv", "yinv", "zinv"};

void destroy_events(psolve_plan *p)
{
    for (auto *pool : {&p->ev_used, &p->ev_free})
        for (auto &set : *pool)
            for (auto e : set) cudaEventDestroy(e);
    p->ev_used.clear();
    p->ev_free.clear();
}

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

// ------------------------------------------------------------ tuning cache
// One line per tuned choice:
//   <gpu>|<dtype>|<path>|<axis>|<L>|<M> <W> <cfg> <order>
// path "pass" = the one-pass-per-launch solve, "batch" = the persistent
// batched launch; axis z (rows of M), y or x (lines of L over M columns).
std::string tune_cache_path()
{
    if (const char *e = std::getenv("PSOLVE_TUNE_CACHE")) return e;
    if (const char *h = std::getenv("HOME")) return std::string(h) + "/.cache/psolve/tune-v1.txt";
    return "";
}

std::string gpu_key(int device)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (auto &c : n)
        if (c == ' ' || c == '|') c = '_';
    return n;
}

std::string tune_key(const psolve_plan *p, const char *path, char axis, int L, int M)
{
    return gpu_key(p->device) + "|" + std::to_string(p->dtype) + "|" + path + "|" + axis + "|" +
           std::to_string(L) + "|" + std::to_string(M);
}

struct TuneChoice {
    int W, cfg, order;
};

std::map<std::string, TuneChoice> read_tune_cache()
{
    std::map<std::string, TuneChoice> m;
    const std::string path = tune_cache_path();
    if (path.empty()) return m;
    FILE *fh = std::fopen(path.c_str(), "r");
    if (!fh) return m;
    char key[512];
    int W, cfg, order;
    while (std::fscanf(fh, "%511s %d %d %d", key, &W, &cfg, &order) == 4) m[key] = TuneChoice{W, cfg, order};
    std::fclose(fh);
    return m;
}

void write_tune_cache(const std::map<std::string, TuneChoice> &m)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *fh = std::fopen(tmp.c_str(), "w");
    if (!fh) return;
    for (const auto &kv : m) std::fprintf(fh, "%s %d %d %d\n", kv.first.c_str(), kv.second.W, kv.second.cfg, kv.second.order);
    std::fclose(fh);
    std::rename(tmp.c_str(), path.c_str());
}

// Key of a batched plan: FNV-1a over its instance shapes.
std::string batch_key(const psolve_plan *p)
{
    unsigned long long h = 1469598103934665603ull;
    for (const auto &g : p->groups)
        for (int v : {g.nx, g.ny, g.nz}) {
            h ^= (unsigned long long)v;
            h *= 1099511628211ull;
        }
    char buf[32];
    std::snprintf(buf, sizeof(buf), "%016llx", h);
    return gpu_key(p->device) + "|" + std::to_string(p->dtype) + "|batch|" + buf;
}

// Apply cached choices that are still valid for this plan.
void apply_tuning_cache(psolve_plan *p)
{
    const auto m = read_tune_cache();
    if (m.empty()) return;
    if (!p->uniform) {
        // knobs are stored as three entries: divisors, orders (W, cfg, order per axis)
        for (int axis = 0; axis < 3; ++axis) {
            auto it = m.find(batch_key(p) + "|" + "zyx"[axis]);
            if (it == m.end()) continue;
            if (it->second.W >= 1 && it->second.W <= 8) p->bknob[axis] = it->second.W;
            if (it->second.order >= 0 && it->second.order <= 2) p->bknob[3 + axis] = it->second.order;
        }
        return;
    }
    const bool fp64 = p->dtype == PSOLVE_F64;
    for (auto &g : p->groups) {
        const char *path = "pass";
        auto it = m.find(tune_key(p, path, 'z', g.M, g.M));
        if (it != m.end() && it->second.W >= 1) {
            const int keep = g.Wz;
            g.Wz = it->second.W;
            if (g.Wz * g.pz.TL > max_threads(fp64, g.pz.E) || z_smem(g, p->dtype) > kSmemCap) g.Wz = keep;
            if (it->second.cfg < 0) g.zbulk = 0; // the tuner found the per-tile kernels faster
        }
        it = m.find(tune_key(p, path, 'f', g.ny, g.M));
        if (it != m.end() && p->dtype == PSOLVE_F32 && fused_supported(g.M, g.ny) && g.pz.E == 16 &&
            g.py.E == 16 && (it->second.W == 0 || it->second.W == 2 || it->second.W == 4 || it->second.W == 8))
            g.fused = it->second.W;
        it = m.find(tune_key(p, path, 'y', g.ny, g.M));
        if (it != m.end()) {
            const TuneChoice c = it->second;
            if (c.cfg >= 0 && c.cfg <= 4 && tma_fits(p, g.ny, g.M, c.cfg) && !(p->dtype == PSOLVE_F32_TC && !tc_cfg_ok(c.cfg, g.ny))) g.cfg_y = c.cfg;
            else if (c.cfg < 0 && !(p->dtype == PSOLVE_F32_TC && g.cfg_y >= 0) && c.W >= 1 && c.W <= g.M && c.W * g.py.TL <= max_threads(fp64, g.py.E) &&
                     s_smem(g.ny, c.W, p->dtype) <= kSmemCap) {
                g.cfg_y = -1;
                g.Wy = c.W;
            }
        }
        it = m.find(tune_key(p, path, 'x', g.nx, g.M));
        if (it != m.end()) {
            const TuneChoice c = it->second;
            if (c.cfg >= 0 && c.cfg <= 4 && tma_fits(p, g.nx, g.M, c.cfg) && !(p->dtype == PSOLVE_F32_TC && !tc_cfg_ok(c.cfg, g.nx))) g.cfg_x = c.cfg;
            else if (c.cfg < 0 && !(p->dtype == PSOLVE_F32_TC && g.cfg_x >= 0) && c.W >= 2 && c.W * g.px.TL <= max_threads(fp64, g.px.E) &&
                     s_smem(g.nx, c.W, p->dtype) <= kSmemCap) {
                g.cfg_x = -1;
                g.Wx = c.W;
            }
        }
    }
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
    // Line plans in the radix order the knobs select (the tables are per length).
    for (auto &g : p->groups) {
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
    for (int pass = 0; pass < 5; ++pass) {
        for (int i = 0; i < B; ++i) {
            const Group &g = p->groups[i];
            BatchSeg<T> sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.kind = pass;
            sg.dep = pass == 0 ? -1 : (pass - 1) * B + i;
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
            sg.first = first;
            first += sg.ntiles;
            segs[(size_t)pass * B + i] = sg;
        }
    }
    for (auto &sg : segs)
        if (sg.dep >= 0) sg.need = (int)segs[sg.dep].ntiles;
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
        if (uniform && dtype == PSOLVE_F32 && fused_supported(g.M, g.ny) && g.pz.E == 16 && g.py.E == 16) {
            // Off by default (measured slower than the separate TMA passes on
            // GB300 at 512^3 and 1024^3); the autotuner times it.
            const char *fe = std::getenv("PSOLVE_FUSED");
            g.fused = 0;
            if (fe && fe[0] >= '1' && fe[0] <= '8') g.fused = fe[0] - '0';
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
                psolve_status st = setup_batched<float>(p.get());
                if (st != PSOLVE_OK) {
                    release(p.release());
                    return st;
                }
            }
        }
    }
    *out = p.release();
    return PSOLVE_OK;
}

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
template <typename T>
psolve_status launch_pass(const psolve_plan *p, const Group &g, int kind, const T *fi, T *ui, cudaStream_t s,
                          bool force_runtime = false, T *zout = nullptr, bool host_io = false, int G = 1)
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

// `uout`, if given, receives u from the last pass (the spectrum stays in u).
template <typename T>
psolve_status run_group(const psolve_plan *p, const Group &g, const T *f, T *u, cudaStream_t s,
                        const std::vector<cudaEvent_t> *ev, T *uout = nullptr, bool host_io = false)
{
    const T *fi = f + g.off0;
    T *ui = u + g.off0;
    T *uo = uout ? uout + g.off0 : nullptr;
    if (ev) cudaEventRecord((*ev)[0], s);
    if (g.fused > 0) {
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


// ------------------------------------------------------------- autotuner
psolve_status run_batched(psolve_plan *p, const void *f, void *u, cudaStream_t s);

void drop_batched(psolve_plan *p)
{
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->segs_dev) cudaFree(p->segs_dev);
    if (p->counters) cudaFree(p->counters);
    p->gexec = nullptr;
    p->graph = nullptr;
    p->segs_dev = nullptr;
    p->counters = nullptr;
    p->batched = false;
}

// The persistent batched launch is tuned as a whole: coordinate descent over
// its plan-wide knobs (tile-width divisor and radix order per axis), each
// candidate timed as complete batched solves on scratch buffers.
psolve_status autotune_batched(psolve_plan *p, cudaStream_t s, std::map<std::string, TuneChoice> &cache)
{
    const size_t bytes = p->total * rsize(p->dtype);
    void *f = nullptr, *u = nullptr;
    if (cudaMalloc(&f, bytes) != cudaSuccess) return fail(PSOLVE_ERR_OOM, "autotune scratch");
    if (cudaMalloc(&u, bytes) != cudaSuccess) {
        cudaFree(f);
        return fail(PSOLVE_ERR_OOM, "autotune scratch");
    }
    cudaMemsetAsync(f, 0x3c, bytes, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = p->profiling;
    p->profiling = false;
    auto measure = [&]() -> float {
        drop_batched(p);
        if (setup_batched<float>(p) != PSOLVE_OK) return 1e30f;
        if (run_batched(p, f, u, s) != PSOLVE_OK) return 1e30f;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) run_batched(p, f, u, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3;
    };
    float best = measure();
    const int choices[6][3] = {{1, 2, 4}, {1, 2, 4}, {1, 2, 4}, {0, 1, 2}, {0, 1, 2}, {0, 1, 2}};
    for (int round = 0; round < 2; ++round)
        for (int k = 0; k < 6; ++k) {
            const int keep = p->bknob[k];
            int bv = keep;
            for (int c : choices[k]) {
                if (c == keep) continue;
                p->bknob[k] = c;
                const float t = measure();
                if (t < best) { best = t; bv = c; }
            }
            p->bknob[k] = bv;
        }
    drop_batched(p);
    psolve_status st = setup_batched<float>(p);
    p->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(f);
    cudaFree(u);
    for (int axis = 0; axis < 3; ++axis)
        cache[batch_key(p) + "|" + "zyx"[axis]] = TuneChoice{p->bknob[axis], -1, p->bknob[3 + axis]};
    return st;
}
// Times candidate tile widths, TMA configurations and radix orders of each
// pass on a scratch instance and keeps the fastest (the analogue of the FFT
// library "MEASURE" planning the paper's setup phase pays once, §3 Table 1).
template <typename T> psolve_status autotune_impl(psolve_plan *p, cudaStream_t s)
{
    const bool fp64 = p->dtype == PSOLVE_F64;
    size_t maxN = 0;
    for (const auto &g : p->groups) maxN = std::max(maxN, (size_t)g.nx * g.ny * g.nz);
    T *buf = nullptr;
    if (cudaMalloc(&buf, maxN * sizeof(T)) != cudaSuccess) return fail(PSOLVE_ERR_OOM, "autotune scratch");
    cudaMemsetAsync(buf, 0x3c, maxN * sizeof(T), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const float inf = 1e30f;
    auto timed = [&](const Group &gt, int kind, bool rt) -> float {
        if (launch_pass<T>(p, gt, kind, buf, buf, s, rt) != PSOLVE_OK) return inf;
        const int reps = 3;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r)
            if (launch_pass<T>(p, gt, kind, buf, buf, s, rt) != PSOLVE_OK) return inf;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return inf;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / reps;
    };
    auto cache = read_tune_cache();
    const int wlist[] = {1, 2, 4, 8, 16, 32, 64};
    for (auto &g : p->groups) {
        Group gt = g;
        gt.count = 1;
        gt.off0 = 0;
        if (!p->batched && p->uniform) {
            // z rows per block of the per-tile kernels, then the bulk-copy kernel
            float best = inf;
            int bw = g.Wz;
            const int zb0 = g.zbulk;
            gt.zbulk = 0;
            for (int W : wlist) {
                gt.Wz = W;
                if (W * gt.pz.TL > max_threads(fp64, gt.pz.E) || z_smem(gt, p->dtype) > kSmemCap) continue;
                const float t = timed(gt, 0, false) + timed(gt, 4, false);
                if (t < best) { best = t; bw = W; }
            }
            g.Wz = gt.Wz = bw;
            int zbest = 0;
            if (zb0) {
                gt.zbulk = 1;
                const float t = timed(gt, 0, false) + timed(gt, 4, false);
                if (t < best) zbest = 1;
            }
            g.zbulk = gt.zbulk = zbest;
            cache[tune_key(p, "pass", 'z', g.M, g.M)] = TuneChoice{bw, zbest ? 1 : -1, 0};
            // y and x: TMA configurations and per-tile widths
            for (int axis = 0; axis < 2; ++axis) {
                const int L = axis == 0 ? g.ny : g.nx;
                const int kind = axis == 0 ? 1 : 2;
                const LinePlan &pl = axis == 0 ? g.py : g.px;
                float bt = inf;
                int bcfg = -1, bW = axis == 0 ? g.Wy : g.Wx;
                // A tensor-core plan keeps its passes on the tensor cores: only
                // the TMA configurations with tensor-core variants compete.
                const bool tc = p->dtype == PSOLVE_F32_TC;
                for (int cfg = 0; cfg < 5 && !fp64; ++cfg) {
                    if (!tma_fits(p, L, g.M, cfg) || (tc && !tc_cfg_ok(cfg, L))) continue;
                    if (axis == 0) gt.cfg_y = cfg; else gt.cfg_x = cfg;
                    const float t = timed(gt, kind, false);
                    if (t < bt) { bt = t; bcfg = cfg; }
                }
                if (axis == 0) gt.cfg_y = -1; else gt.cfg_x = -1;
                for (int W : wlist) {
                    if (tc && bcfg >= 0) break;
                    if (W < (axis == 0 ? 1 : 2) || (axis == 0 && W > g.M) || W * pl.TL > max_threads(fp64, pl.E) ||
                        s_smem(L, W, p->dtype) > kSmemCap)
                        continue;
                    if (axis == 0) gt.Wy = W; else gt.Wx = W;
                    const float t = timed(gt, kind, false);
                    if (t < bt) { bt = t; bcfg = -1; bW = W; }
                }
                if (axis == 0) { g.cfg_y = gt.cfg_y = bcfg; g.Wy = gt.Wy = bW; }
                else { g.cfg_x = gt.cfg_x = bcfg; g.Wx = gt.Wx = bW; }
                cache[tune_key(p, "pass", axis == 0 ? 'y' : 'x', L, g.M)] = TuneChoice{bW, bcfg, 0};
            }
            // z/y fused through L2 against separate passes, timed as whole solves.
            if (p->dtype == PSOLVE_F32 && fused_supported(g.M, g.ny) && g.pz.E == 16 && g.py.E == 16) {
                float bt = inf;
                int bf = 0;
                for (int fz : {0, 4, 8}) {
                    gt.fused = fz;
                    if (run_group<T>(p, gt, buf, buf, s, nullptr) != PSOLVE_OK) continue;
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < 3; ++r) run_group<T>(p, gt, buf, buf, s, nullptr);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms / 3 < bt) { bt = ms / 3; bf = fz; }
                }
                g.fused = gt.fused = bf;
                cache[tune_key(p, "pass", 'f', g.ny, g.M)] = TuneChoice{bf, -1, 0};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (p->batched) {
        psolve_status st = autotune_batched(p, s, cache);
        if (st != PSOLVE_OK) return st;
    }
    write_tune_cache(cache);
    return PSOLVE_OK;
}

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

std::mutex g_norm_mu;
double *g_norm_buf[64] = {nullptr};

} // namespace

extern "C" {

psolve_status psolve_plan_create(int nx, int ny, int nz, int dtype, int batch, psolve_plan **out)
{
    if (!out) return fail(PSOLVE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (dtype != PSOLVE_F64 && dtype != PSOLVE_F32 && dtype != PSOLVE_F32_TC)
        return fail(PSOLVE_ERR_INVALID_ARG, "unknown dtype");
    if (batch < 1) return fail(PSOLVE_ERR_INVALID_ARG, "batch must be >= 1");
    if (!size_ok(nx) || !size_ok(ny) || !size_ok(nz))
        return fail(PSOLVE_ERR_UNSUPPORTED_SIZE, "each n must be 2^a 3^b, even, 4 <= n <= 2048");
    std::vector<int> X(batch, nx), Y(batch, ny), Z(batch, nz);
    return build_plan(X, Y, Z, dtype, true, out);
}

psolve_status psolve_plan_create_many(const int *nx, const int *ny, const int *nz, int batch, int dtype,
                                      psolve_plan **out)
{
    if (!out) return fail(PSOLVE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!nx || !ny || !nz) return fail(PSOLVE_ERR_INVALID_ARG, "null size array");
    if (dtype != PSOLVE_F64 && dtype != PSOLVE_F32 && dtype != PSOLVE_F32_TC)
        return fail(PSOLVE_ERR_INVALID_ARG, "unknown dtype");
    if (dtype == PSOLVE_F32_TC)
        return fail(PSOLVE_ERR_INVALID_ARG, "tensor-core precision applies to plans of equal grids");
    if (batch < 1) return fail(PSOLVE_ERR_INVALID_ARG, "batch must be >= 1");
    std::vector<int> X(nx, nx + batch), Y(ny, ny + batch), Z(nz, nz + batch);
    for (int b = 0; b < batch; ++b)
        if (!size_ok(X[b]) || !size_ok(Y[b]) || !size_ok(Z[b]))
            return fail(PSOLVE_ERR_UNSUPPORTED_SIZE, "instance " + std::to_string(b) +
                                                         ": each n must be 2^a 3^b, even, 4 <= n <= 2048");
    return build_plan(X, Y, Z, dtype, false, out);
}

psolve_status psolve_execute(psolve_plan *plan, const void *f, void *u, void *stream)
{
    return solve(plan, f, u, stream);
}

psolve_status psolve_adjoint(psolve_plan *plan, const void *g, void *grad_f, void *stream)
{
    // A = F^{-1} D F with D real and even in k is symmetric: A^T = A.
    return solve(plan, g, grad_f, stream);
}

psolve_status psolve_execute_host(psolve_plan *plan, const void *f_host, void *u_host, void *stream)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (!f_host || !u_host) return fail(PSOLVE_ERR_INVALID_ARG, "null host pointer");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "select device");
    const size_t bytes = plan->total * rsize(plan->dtype);
    if (plan->stage_bytes < bytes) {
        if (plan->stage) cudaFree(plan->stage);
        plan->stage = nullptr;
        plan->stage_bytes = 0;
        if (cudaMalloc(&plan->stage, bytes) != cudaSuccess) {
            plan->stage = nullptr;
            return fail(PSOLVE_ERR_OOM, "device staging buffer: cudaMalloc failed");
        }
        plan->stage_bytes = bytes;
    }
    cudaStream_t s = (cudaStream_t)stream;
    psolve_status st = host_solve(plan, f_host, u_host, plan->stage, s, true);
    if (st != PSOLVE_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise stream");
    return PSOLVE_OK;
}

psolve_status psolve_execute_host_async(psolve_plan *plan, const void *f_host, void *u_host, void *stream)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (!f_host || !u_host) return fail(PSOLVE_ERR_INVALID_ARG, "null host pointer");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "select device");
    const size_t bytes = plan->total * rsize(plan->dtype);
    const unsigned i = plan->aring++ % kAsyncRing;
    if (!plan->astage[i]) {
        if (cudaMalloc(&plan->astage[i], bytes) != cudaSuccess) {
            plan->astage[i] = nullptr;
            return fail(PSOLVE_ERR_OOM, "device staging buffer: cudaMalloc failed");
        }
        if (cudaEventCreateWithFlags(&plan->aev[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(PSOLVE_ERR_CUDA, "staging event");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // The previous solve that used this staging buffer must be done with it.
    if (plan->aev_used[i]) {
        cudaError_t e = cudaStreamWaitEvent(s, plan->aev[i], 0);
        if (e != cudaSuccess) return cuda_fail(e, "wait for staging buffer");
    }
    psolve_status st = host_solve(plan, f_host, u_host, plan->astage[i], s, false);
    if (st != PSOLVE_OK) return st;
    cudaError_t e = cudaEventRecord(plan->aev[i], s);
    if (e != cudaSuccess) return cuda_fail(e, "record staging event");
    plan->aev_used[i] = true;
    return PSOLVE_OK;
}

psolve_status psolve_destroy(psolve_plan *plan)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    DeviceGuard dg(plan->device);
    release(plan);
    return PSOLVE_OK;
}

size_t psolve_instance_offset(const psolve_plan *plan, int b)
{
    if (!plan_ok(plan) || b < 0 || b >= plan->batch) return (size_t)-1;
    return plan->inst_off[b];
}

size_t psolve_total_elements(const psolve_plan *plan)
{
    if (!plan_ok(plan)) return 0;
    return plan->total;
}

psolve_status psolve_get_status(psolve_plan *plan, void *stream)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    DeviceGuard dg(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise stream");
    int word = 0;
    e = cudaMemcpy(&word, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read status word");
    cudaMemset(plan->status, 0, sizeof(int));
    if (word == 0) return PSOLVE_OK;
    if (word == PSOLVE_ERR_TIMEOUT) return fail(PSOLVE_ERR_TIMEOUT, "a device-side wait gave up");
    return fail(PSOLVE_ERR_INTERNAL, "device status word " + std::to_string(word));
}

psolve_status psolve_debug_kvec(const psolve_plan *plan, int b, int *kxyz_out)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (b < 0 || b >= plan->batch || !kxyz_out) return fail(PSOLVE_ERR_INVALID_ARG, "bad instance or buffer");
    const Group &g = plan->groups[plan->groups.size() == 1 ? 0 : b];
    DeviceGuard dg(plan->device);
    const size_t n = (size_t)g.nx * g.ny * (g.nz / 2 + 1) * 3;
    int *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(int)) != cudaSuccess) return fail(PSOLVE_ERR_OOM, "kvec buffer");
    cudaError_t e = launch_kvec(d, g.nx, g.ny, g.nz, 0);
    if (e == cudaSuccess) e = cudaMemcpy(kxyz_out, d, n * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "kvec export");
    return PSOLVE_OK;
}

psolve_status psolve_error_norms(const void *a, const void *ref, size_t n, int dtype, double *out4, void *stream)
{
    if (!a || !ref || !out4) return fail(PSOLVE_ERR_INVALID_ARG, "null pointer");
    if (dtype != PSOLVE_F64 && dtype != PSOLVE_F32 && dtype != PSOLVE_F32_TC)
        return fail(PSOLVE_ERR_INVALID_ARG, "unknown dtype");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(PSOLVE_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_norm_mu);
    if (!g_norm_buf[dev]) {
        if (cudaMalloc((void **)&g_norm_buf[dev], 4 * sizeof(double)) != cudaSuccess) {
            g_norm_buf[dev] = nullptr;
            return fail(PSOLVE_ERR_OOM, "norm buffer");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *buf = g_norm_buf[dev];
    e = cudaMemsetAsync(buf, 0, 4 * sizeof(double), s);
    if (e == cudaSuccess)
        e = dtype == PSOLVE_F64 ? launch_norms<double>((const double *)a, (const double *)ref, n, buf, s)
                                : launch_norms<float>((const float *)a, (const float *)ref, n, buf, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out4, buf, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "error norms");
    return PSOLVE_OK;
}

psolve_status psolve_autotune(psolve_plan *plan, void *stream)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "select device");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise stream");
    return plan->dtype == PSOLVE_F64 ? autotune_impl<double>(plan, s) : autotune_impl<float>(plan, s);
}

psolve_status psolve_set_operator(psolve_plan *plan, int op, double c)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (op < PSOLVE_OP_POISSON || op > PSOLVE_OP_FD_LAPLACIAN) return fail(PSOLVE_ERR_INVALID_ARG, "unknown operator");
    if (op == PSOLVE_OP_HELMHOLTZ && !(c > 0.0 && c < 1e300))
        return fail(PSOLVE_ERR_INVALID_ARG, "Helmholtz c must be positive and finite");
    DeviceGuard dg(plan->device);
    if (dg.err != cudaSuccess) return cuda_fail(dg.err, "select device");
    if (op == PSOLVE_OP_FD_LAPLACIAN && !plan->optab) {
        // Λ(j) = (n/π)² sin²(π j/n) per axis and group, z indices kz = 0..M
        std::vector<double> tab;
        for (auto &g : plan->groups) {
            auto add = [&](int n, int count) {
                const size_t off = tab.size();
                for (int j = 0; j < count; ++j) {
                    const double s = std::sin(M_PI * (double)j / (double)n);
                    tab.push_back((double)n * (double)n / (M_PI * M_PI) * s * s);
                }
                return off;
            };
            g.op_lx = add(g.nx, g.nx);
            g.op_ly = add(g.ny, g.ny);
            g.op_lz = add(g.nz, g.M + 1);
        }
        // FP64 tables, then the same rounded to FP32
        const size_t n = tab.size();
        std::vector<unsigned char> bytes(n * sizeof(double) + n * sizeof(float));
        std::memcpy(bytes.data(), tab.data(), n * sizeof(double));
        float *t32 = reinterpret_cast<float *>(bytes.data() + n * sizeof(double));
        for (size_t i = 0; i < n; ++i) t32[i] = (float)tab[i];
        double *d = nullptr;
        if (cudaMalloc(&d, bytes.size()) != cudaSuccess)
            return fail(PSOLVE_ERR_OOM, "finite-difference symbol tables: cudaMalloc failed");
        cudaError_t e = cudaMemcpy(d, bytes.data(), bytes.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "upload finite-difference symbol tables");
        }
        plan->optab = d;
        plan->optab_n = n;
    }
    plan->op = op;
    plan->op_c = op == PSOLVE_OP_HELMHOLTZ ? c : 0.0;
    if (plan->batched) {
        // the persistent launch's segment table holds the multiplier
        drop_batched(plan);
        psolve_status st = setup_batched<float>(plan);
        if (st != PSOLVE_OK) return st;
    }
    return PSOLVE_OK;
}

psolve_status psolve_set_profiling(psolve_plan *plan, int enable)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (enable < 0) return fail(PSOLVE_ERR_INVALID_ARG, "profiling interval must be >= 0");
    plan->profiling = enable != 0;
    plan->prof_every = enable;
    plan->prof_count = 0;
    return PSOLVE_OK;
}

int plan_passes(const psolve_plan *p)
{
    if (p->batched) return 1;
    return (p->groups.size() == 1 && p->groups[0].fused > 0) ? 3 : kPasses;
}

psolve_status psolve_pass_times(psolve_plan *plan, double *ms, int cap, int *n_passes, int *n_solves)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (!ms || cap < 0) return fail(PSOLVE_ERR_INVALID_ARG, "null output");
    DeviceGuard dg(plan->device);
    for (int i = 0; i < cap; ++i) ms[i] = 0.0;
    int solves = 0;
    for (auto &set : plan->ev_used) {
        cudaError_t e = cudaEventSynchronize(set[kPasses]);
        if (e != cudaSuccess) return cuda_fail(e, "profiling events");
        for (int i = 0; i < kPasses && i < cap; ++i) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, set[i], set[i + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "profiling events");
            ms[i] += t;
        }
        ++solves;
    }
    for (auto &set : plan->ev_used) plan->ev_free.push_back(std::move(set));
    plan->ev_used.clear();
    if (n_passes) *n_passes = plan_passes(plan);
    if (n_solves) *n_solves = solves;
    return PSOLVE_OK;
}

const char *psolve_pass_name(const psolve_plan *plan, int i)
{
    if (!plan_ok(plan) || i < 0 || i >= kPasses) return nullptr;
    if (plan->batched) return i == 0 ? "batched" : "none";
    if (plan_passes(plan) == 3) {
        static const char *fused_names[3] = {"zyfwd", "xdiv", "yzinv"};
        return i < 3 ? fused_names[i] : "none";
    }
    if (plan->dtype == PSOLVE_F32_TC) {
        const Group &g = plan->groups[0];
        if ((i == 1 || i == 3) && g.cfg_y >= 0) return i == 1 ? "yfwd_tc" : "yinv_tc";
        if (i == 2 && g.cfg_x >= 0 && plan->op == PSOLVE_OP_POISSON) return "xdiv_tc";
    }
    return kPassNames[i];
}

int psolve_launches_per_solve(const psolve_plan *plan)
{
    if (!plan_ok(plan)) return 0;
    if (plan->batched) return 1;
    return plan_passes(plan) * (int)plan->groups.size();
}

psolve_status psolve_debug_set_wait(psolve_plan *plan, unsigned long long wait_ns, int unsatisfiable)
{
    if (!plan_ok(plan)) return fail(PSOLVE_ERR_INVALID_ARG, "invalid or destroyed plan");
    if (!plan->batched) return fail(PSOLVE_ERR_INVALID_ARG, "plan has no persistent batched launch");
    DeviceGuard dg(plan->device);
    plan->wait_ns = wait_ns;
    // Segment nseg/5 (pass 1 of instance 0) waits on segment 0.
    const size_t seg_bytes = plan->segs_host.size() / (size_t)plan->nseg;
    const int target = plan->nseg / 5;
    unsigned char entry[4096];
    if (seg_bytes > sizeof(entry)) return fail(PSOLVE_ERR_INTERNAL, "segment too large");
    std::memcpy(entry, plan->segs_host.data() + (size_t)target * seg_bytes, seg_bytes);
    // the leading int fields have the same offsets in BatchSeg<float> and <double>
    const size_t off_need = offsetof(BatchSeg<float>, need);
    static_assert(offsetof(BatchSeg<float>, need) == offsetof(BatchSeg<double>, need), "segment layout");
    int need = 0;
    std::memcpy(&need, entry + off_need, sizeof(int));
    if (unsatisfiable) ++need;
    std::memcpy(entry + off_need, &need, sizeof(int));
    cudaError_t e = cudaMemcpy((char *)plan->segs_dev + (size_t)target * seg_bytes, entry, seg_bytes,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "update segment");
    return PSOLVE_OK;
}

const char *psolve_status_string(psolve_status s)
{
    switch (s) {
    case PSOLVE_OK: return "ok";
    case PSOLVE_ERR_INVALID_ARG: return "invalid argument";
    case PSOLVE_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case PSOLVE_ERR_OOM: return "out of device memory";
    case PSOLVE_ERR_CUDA: return "CUDA error";
    case PSOLVE_ERR_TIMEOUT: return "device-side wait timed out";
    case PSOLVE_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *psolve_last_error(void) { return g_last_error.c_str(); }

int psolve_version(void) { return 100; }

} // extern "C"
