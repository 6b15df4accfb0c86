// Allocation-free solve: psolve_execute_noalloc.
//
// Some callers cannot call cudaMalloc: code running inside a custom device
// allocator or memory-pool callback, code under a framework that forbids
// allocation during a step (a capture or a fixed-memory budget), or embedded
// hosts that pre-reserve all device memory.  For them this entry point runs
// the same five pass kernels as psolve_execute without a plan: the only
// memory beyond the caller's f and u is the twiddle tables, and those live in
// a fixed file-scope device array instead of plan-owned allocations.  Nothing
// here calls cudaMalloc, cudaFree or any other allocating routine, on the
// device or on the host (the planning below uses the stack only).
#include "psolve.h"
#include "launch.h"

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

bool f23(int n, int &a, int &b)
{
    a = b = 0;
    if (n <= 0) return false;
    while (n % 2 == 0) { n /= 2; ++a; }
    while (n % 3 == 0) { n /= 3; ++b; }
    return n == 1;
}

bool valid_n(int n)
{
    int a, b;
    return n >= 4 && n <= 2048 && (n % 2) == 0 && f23(n, a, b);
}

// Same stage plan as the planned path: radix-3 stages, then the largest
// power-of-two radices (<= 16) dividing the points-per-thread E.
bool line_plan(int L, LinePlan &p)
{
    int a, b;
    if (!f23(L, a, b) || L < 2) return false;
    const int E = b > 0 ? 3 * (1 << (a < 3 ? a : 3)) : (1 << (a < 4 ? a : 4));
    if (!supported_E(E)) return false;
    std::memset(&p, 0, sizeof(p));
    p.L = L;
    p.E = E;
    p.TL = L / E;
    int p2 = 1;
    while (E % (p2 * 2) == 0 && p2 * 2 <= 16) p2 *= 2;
    int rad[kMaxStages];
    int n = 0;
    for (int i = 0; i < b; ++i) rad[n++] = 3;
    int rem = 1 << a;
    while (rem > 1) {
        if (n >= kMaxStages) return false;
        const int r = p2 < rem ? p2 : rem;
        rad[n++] = r;
        rem /= r;
    }
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

constexpr size_t kSmemCap = 200 * 1024;

// Device address of the table array on the current device, looked up once
// per device (with that device current) and cached.
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
    const bool fp64 = sizeof(T) == 8;
    const size_t cs = sizeof(C);
    const int M = nz / 2;
    LinePlan pz, py, px;
    if (!line_plan(M, pz) || !line_plan(ny, py) || !line_plan(nx, px))
        return err(PSOLVE_ERR_UNSUPPORTED_SIZE, "no stage plan for this size");

    // Table layout: [e^{-2πij/M}][e^{-2πij/ny}][e^{-2πij/nx}][e^{-2πik/nz}, k < M]
    const size_t o_z = 0, o_y = o_z + M, o_x = o_y + ny, o_p = o_x + nx;
    C *tab = reinterpret_cast<C *>(tables);
    cudaError_t e = launch_roots<T>(tab + o_z, M, M, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_y, ny, ny, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_x, nx, nx, s);
    if (e == cudaSuccess) e = launch_roots<T>(tab + o_p, M, nz, s);
    if (e != cudaSuccess) return err(PSOLVE_ERR_CUDA, "twiddle generation launch failed");

    // Tile shapes (as in the planned path).
    int Wz = 1, Wy = 1, Wx = 2;
    {
        const int mt = max_threads(fp64, pz.E);
        Wz = (mt < 256 ? mt : 256) / pz.TL;
        if (Wz < 1) Wz = 1;
        const int LP = M + (M >> 4) + 1;
        while (Wz > 1 && (size_t)(M + (size_t)Wz * LP) * cs > kSmemCap) Wz /= 2;
    }
    {
        const int mt = max_threads(fp64, py.E);
        int W = mt / py.TL;
        if (W < 1) W = 1;
        if (W > 16) W = 16;
        if (W > M) W = M;
        while (W > 1 && (size_t)ny * (1 + W) * cs > kSmemCap) W /= 2;
        Wy = W < 1 ? 1 : W;
    }
    {
        const int mt = max_threads(fp64, px.E);
        int W = mt / px.TL;
        if (W < 2) W = 2;
        if (W > 16) W = 16;
        const int cap = M < 2 ? 2 : M;
        if (W > cap) W = cap;
        while (W > 2 && (size_t)nx * (1 + W) * cs > kSmemCap) W /= 2;
        Wx = W;
    }

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
    const size_t zsm = (size_t)(M + (size_t)Wz * (M + (M >> 4) + 1)) * cs;
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
    const size_t ysm = (size_t)ny * (1 + Wy) * cs;
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
    if (launch_xfused<T>(x, xgrid, xblock, (size_t)nx * (1 + Wx) * cs, s) != cudaSuccess)
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
    if (!valid_n(nx) || !valid_n(ny) || !valid_n(nz))
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
