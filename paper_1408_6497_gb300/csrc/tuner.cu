// The autotuner and its per-GPU cache: candidate tile widths, TMA
// configurations, radix orders and z/y fusion of each pass, timed on scratch
// buffers (the analogue of the planning the paper's FFT libraries do once
// in their setup phase, §3 Table 1), and the choices kept in a text file.
#include "plan.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <sys/stat.h>
#include <unistd.h>

namespace psolve {

namespace {

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

} // namespace

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
        if (it != m.end() && (it->second.W == 0 || fused_ok(g, p->dtype, p->uniform, it->second.W)))
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

namespace {

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
            // z/y fused per plane (through L2, or in a cluster's distributed
            // shared memory) against separate passes, timed as whole solves.
            if (fused_ok(g, p->dtype, p->uniform, 4) || fused_ok(g, p->dtype, p->uniform, zy_cluster_size())) {
                float bt = inf;
                int bf = 0;
                for (int fz : {0, 4, 8, zy_cluster_size()}) {
                    if (fz != 0 && !fused_ok(g, p->dtype, p->uniform, fz)) continue;
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

} // namespace

} // namespace psolve

using namespace psolve;

extern "C" {

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

} // extern "C"
