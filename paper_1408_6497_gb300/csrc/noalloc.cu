// Allocation-free solve: psolve_execute_noalloc.
//
// Some callers cannot call cudaMalloc: code running inside a custom device
// allocator or memory-pool callback, code under a framework that forbids
// allocation during a step (a capture or a fixed-memory budget), or embedded
// hosts that pre-reserve all device memory.  For them this entry point runs
// the per-tile pass kernels of psolve_execute without a plan, with the same
// stage plans and tile shapes the planner gives those kernels: the only
// memory beyond the caller's f and u is the twiddle tables, and those live in
// a fixed file-scope device array instead of plan-owned allocations.  Nothing
// here calls cudaMalloc, cudaFree or any other allocating routine, on the
// device or on the host (the planner's line plans and tile choice use fixed
// arrays on the stack).
#include "plan.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

using namespace psolve;

namespace {

// Capacity of the shared table array: 64 KiB.  A grid needs
// (2·(nz/2) + ny + nx) complex twiddles (8 B each in FP32, 16 B in FP64), so
// every valid FP32 grid fits (at most 48 KiB) and FP64 grids fit while
// nx + ny + nz <= 4096.
constexpr size_t kNoAllocBytes = 64 * 1024;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_tables[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_table_addr[kMaxDevices] = {nullptr};

// The reason is stated where each status is returned; psolve_last_error()
// is not updated by this entry point.
psolve_status err(psolve_status s, const char *reason)
{
    (void)reason;
    return s;
}

// Device address of the table array on the current device, looked up once
// per device (with that device current, on the first call there) and cached;
// a reset of that device after the first call is not supported.
psolve_status table_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PSOLVE_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return err(PSOLVE_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_table_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_tables);
        if (e != cudaSuccess || ptr == nullptr)
            return err(PSOLVE_ERR_CUDA, "cudaGetSymbolAddress of the table array failed");
        g_table_addr[dev] = ptr;
    }
    *out = g_table_addr[dev];
    return PSOLVE_OK;
}

template <typename T>
psolve_status run(int nx, int ny, int nz, const T *f, T *u, unsigned char *tables, cudaStream_t s)
{
    using C = typename cplx_of<T>::type;
    const int dtype = sizeof(T) == 8 ? PSOLVE_F64 : PSOLVE_F32;
    const int M = nz / 2;
    // The planner's stage plans and tile widths (without the PSOLVE_TILE_W
    // override), as psolve_execute's per-tile passes of this grid would use.
    Group g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.M = M;
    if (!make_line_plan(M, g.pz) || !make_line_plan(ny, g.py) || !make_line_plan(nx, g.px))
        return err(PSOLVE_ERR_UNSUPPORTED_SIZE, "no stage plan for this size");
    choose_tiles(g, dtype, false);
    if (!tiles_fit(g, dtype)) return err(PSOLVE_ERR_UNSUPPORTED_SIZE, "no tile of this grid fits a block");
    const LinePlan &pz = g.pz, &py = g.py, &px = g.px;
    const int Wz = g.Wz, Wy = g.Wy, Wx = g.Wx;

    // Table layout: [e^{-2πij/M}][e^{-2πij/ny}][e^{-2πij/nx}][e^{-2πik/nz}, k < M]
    const size_t o_z = 0, o_y = o_z + M, o_x = o_y + ny, o_p = o_x + nx;
    C *tab = reinterpret_cast<C *>(tables);
    cudaError_t e = launch_roots<T>(tab + o_z, M, M, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_y, ny, ny, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_x, nx, nx, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_p, M, nz, s);
    if (e != cudaSuccess) return err(PSOLVE_ERR_CUDA, "twiddle generation launch failed");

    ZArgs<T> z{};
    z.in = f;
    z.out = u;
    z.rows = (long long)nx * ny;
    z.nz = nz;
    z.M = M;
    z.W = Wz;
    z.pl = pz;
    z.tw = tab + o_z;
    z.post = tab + o_p;
    const unsigned zgrid = (unsigned)((z.rows + Wz - 1) / Wz);
    const unsigned zblock = (unsigned)(Wz * pz.TL);
    const size_t zsm = z_smem(g, dtype);
    if (launch_zfwd<T>(z, zgrid, zblock, zsm, s) != cudaSuccess) return err(PSOLVE_ERR_CUDA, "z forward pass");

    SArgs<T> y{};
    y.data = u;
    y.nplanes = nx;
    y.sPlane = (long long)ny * M;
    y.sL = M;
    y.M = M;
    y.W = Wy;
    y.ncb = (M + Wy - 1) / Wy;
    y.pl = py;
    y.tw = tab + o_y;
    const unsigned ygrid = (unsigned)(y.nplanes * y.ncb);
    const unsigned yblock = (unsigned)(Wy * py.TL);
    const size_t ysm = s_smem(ny, Wy, dtype);
    if (launch_ypass<T>(y, false, ygrid, yblock, ysm, s) != cudaSuccess)
        return err(PSOLVE_ERR_CUDA, "y forward pass");

    XArgs<T> x{};
    x.data = u;
    x.batch = 1;
    x.nx = nx;
    x.ny = ny;
    x.M = M;
    x.sInst = (long long)nx * ny * M;
    x.W = Wx;
    x.ncb = (M + Wx - 1) / Wx;
    x.main_tiles = (long long)ny * x.ncb;
    x.npairs = ny / 2 + 1;
    x.pl = px;
    x.tw = tab + o_x;
    x.coef = (T)(1.0 / (4.0 * M_PI * M_PI * ((double)nx * ny * nz)));
    const unsigned xgrid = (unsigned)(x.main_tiles + (x.npairs + Wx / 2 - 1) / (Wx / 2));
    const unsigned xblock = (unsigned)(Wx * px.TL);
    if (launch_xfused<T>(x, xgrid, xblock, s_smem(nx, Wx, dtype), s) != cudaSuccess)
        return err(PSOLVE_ERR_CUDA, "x pass with spectral division");

    if (launch_ypass<T>(y, true, ygrid, yblock, ysm, s) != cudaSuccess)
        return err(PSOLVE_ERR_CUDA, "y inverse pass");

    ZArgs<T> zi = z;
    zi.in = u;
    zi.out = u;
    if (launch_zinv<T>(zi, zgrid, zblock, zsm, s) != cudaSuccess) return err(PSOLVE_ERR_CUDA, "z inverse pass");
    return PSOLVE_OK;
}

} // namespace

extern "C" {

psolve_status psolve_execute_noalloc(int nx, int ny, int nz, int dtype, const void *f, void *u, void *stream)
{
    if (dtype != PSOLVE_F64 && dtype != PSOLVE_F32)
        return err(PSOLVE_ERR_INVALID_ARG, "psolve_execute_noalloc supports PSOLVE_F64 and PSOLVE_F32");
    if (!size_ok(nx) || !size_ok(ny) || !size_ok(nz))
        return err(PSOLVE_ERR_UNSUPPORTED_SIZE, "each n must be 2^a 3^b, even, 4 <= n <= 2048");
    const size_t cs = dtype == PSOLVE_F64 ? 16 : 8;
    const size_t need = ((size_t)nz + ny + nx) * cs;
    if (need > kNoAllocBytes)
        return err(PSOLVE_ERR_UNSUPPORTED_SIZE,
                   "psolve_execute_noalloc: the twiddle tables of this grid exceed the fixed 64 KiB "
                   "table array ((nx + ny + nz) complex values must fit)");
    if (!f || !u) return err(PSOLVE_ERR_INVALID_ARG, "null array pointer");
    if (((uintptr_t)f & 15) || ((uintptr_t)u & 15))
        return err(PSOLVE_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    if (f != u) {
        const uintptr_t a0 = (uintptr_t)f, b0 = (uintptr_t)u;
        const uintptr_t len = (uintptr_t)((size_t)nx * ny * nz * (cs / 2));
        if (a0 < b0 + len && b0 < a0 + len) return err(PSOLVE_ERR_INVALID_ARG, "f and u partially overlap");
    }
    void *tables = nullptr;
    psolve_status st = table_address(&tables);
    if (st != PSOLVE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return dtype == PSOLVE_F64
               ? run<double>(nx, ny, nz, (const double *)f, (double *)u, (unsigned char *)tables, s)
               : run<float>(nx, ny, nz, (const float *)f, (float *)u, (unsigned char *)tables, s);
}

} // extern "C"
