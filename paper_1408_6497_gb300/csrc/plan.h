// Host side of the library, shared by its translation units: the plan
// object, the planner (stage plans, tile shapes, the persistent batched
// schedule), the autotuner and its cache, and the pass pipeline that
// enqueues a solve.  Files: planner.cu (plans, tiles, set-up), tuner.cu
// (tuning cache, autotuner), pipeline.cu (tensor maps, pass launches, solves,
// host-buffer solves), api.cu (the C ABI), noalloc.cu (the plan-free solve).
#pragma once

#include "psolve.h"
#include "launch.h"

#include <map>
#include <string>
#include <vector>

namespace psolve {

// Record `msg` as the calling thread's last error (psolve_last_error) and
// return `s`.
psolve_status fail(psolve_status s, const std::string &msg);
psolve_status cuda_fail(cudaError_t e, const char *where);

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
    int fused;           // z and y passes fused per plane: cluster size 2, 4 or 8 (hand-off through
                         // L2), 16 (the plane in the cluster's distributed shared memory), 0 = off
    int zy_clusters;     // 16-block clusters the distributed-shared-memory z/y kernels run at once
    int zbulk;           // z passes by the persistent bulk-copy kernel (1) or per-tile blocks (0)
    int xs;              // x-split factor of the spectrum layout when every pass can use it (1: natural)
};

// ------------------------------------------------------------ planner
bool factor23(int n, int &a, int &b);
// Each n must be 2^a 3^b, even, 4 <= n <= 2048.
bool size_ok(int n);
// Stage plan of an L-point line: radix-3 stages for the factors of 3, then
// the largest power-of-two radices (<= 16) that divide E (order 0).  Order 1
// runs the same radices in reverse, order 2 puts the radix-3 stages last.
// e3cap bounds the power of two in E for lengths 3·2^a (points per thread).
bool make_line_plan(int L, LinePlan &p, int order = 0, int e3cap = 3);
// Stage plan with a given number of points per thread E (a power of two dividing L).
bool make_line_plan_E(int L, int E, LinePlan &p);
size_t csize(int dtype);
size_t rsize(int dtype);
int zpitch(int M);
size_t z_smem(const Group &g, int dtype);
size_t s_smem(int L, int W, int dtype);
// Whether every per-tile pass of group g fits a block with its chosen tile
// widths (the x pass needs two columns: FP64 x lines of 1458 points do not).
bool tiles_fit(const Group &g, int dtype);
// Whether the z/y fusion with cluster size `fused` can run for group g.
bool fused_ok(const Group &g, int dtype, bool uniform, int fused);
// Tile widths of the per-tile kernels; with `env_override` the widths asked
// for in PSOLVE_TILE_W replace them where they fit.
void choose_tiles(Group &g, int dtype, bool env_override = true);

} // namespace psolve

struct psolve_plan {
    unsigned magic;
    bool uniform; // psolve_plan_create (equal grids back to back)
    int dtype;
    int device;
    int num_sms;
    bool use_tma;
    int tma_narrow_y, tma_narrow_x; // tile variant per pass (see launch.h)
    int batch;
    std::vector<psolve::Group> groups;
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
    void *astage[psolve::kAsyncRing];
    cudaEvent_t aev[psolve::kAsyncRing];
    bool aev_used[psolve::kAsyncRing];
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

namespace psolve {

inline bool plan_ok(const psolve_plan *p) { return p != nullptr && p->magic == kMagic; }

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
extern const char *const kPassNames[kPasses];

void destroy_events(psolve_plan *p);
std::vector<cudaEvent_t> *take_events(psolve_plan *p);
void release(psolve_plan *p);
int tma_variant(int setting, int L);
bool tc_cfg_ok(int cfg, int L);
int tma_default(int L, bool x_axis);
bool tma_fits(const psolve_plan *p, int L, int M, int narrow);
OpArgs op_args(const psolve_plan *p, const Group &g);
template <typename T> psolve_status setup_batched(psolve_plan *p);
psolve_status build_plan(const std::vector<int> &nx, const std::vector<int> &ny, const std::vector<int> &nz,
                         int dtype, bool uniform, psolve_plan **out);

// ------------------------------------------------------------ tuner
struct TuneChoice {
    int W, cfg, order;
};
void apply_tuning_cache(psolve_plan *p);
void drop_batched(psolve_plan *p);

// ------------------------------------------------------------ pipeline
template <typename T>
psolve_status launch_pass(const psolve_plan *p, const Group &g, int kind, const T *fi, T *ui, cudaStream_t s,
                          bool force_runtime = false, T *zout = nullptr, bool host_io = false, int G = 1);
template <typename T>
psolve_status run_group(const psolve_plan *p, const Group &g, const T *f, T *u, cudaStream_t s,
                        const std::vector<cudaEvent_t> *ev, T *uout = nullptr, bool host_io = false);
psolve_status run_batched(psolve_plan *p, const void *f, void *u, cudaStream_t s);
psolve_status solve(psolve_plan *p, const void *f, void *u, void *stream);
psolve_status host_solve(psolve_plan *plan, const void *f_host, void *u_host, void *stage, cudaStream_t s,
                         bool zero_copy);

} // namespace psolve
