// The C ABI (include/psolve.h): plan creation and destruction, solves from
// device and host buffers, status and last-error reporting, operators,
// profiling, and the test hooks.  The work behind each call lives in
// planner.cu, tuner.cu and pipeline.cu.
#include "plan.h"

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace psolve {

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

} // namespace psolve

using namespace psolve;

namespace {

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
    // Segment nseg/5 (the first of pass 1) waits on one segment of pass 0.
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
