// Radix-16 DFT stages on the 5th-generation tensor cores (tcgen05, sm_100+).
//
// A block of 128·G threads holds 128·G butterflies, thread tid the 16
// complex inputs of butterfly (row) tid.  The stage computes, per row,
//     b = F a,   F[k][r] = e^{∓2πi kr/16},
// as the real product of the row [Re a | Im a] (32 values) with the 32×32
// real form of F, [[Re F, -Im F], [Im F, Re F]], on the tensor cores.
//
// Operand format: FP16 hi + lo with a power-of-two scale per row.  Each
// thread scales its own row so that its largest |value| lies in
// [2^14, 2^15) (exact: a power of two), splits every value as
// x = hi + lo (hi = fp16(x), lo = fp16(x - hi): 22 significant bits, the
// residual at most 2^-22 |x|), and the DFT matrix is split the same way from
// its FP64 values.  The tensor cores accumulate hi·Fhi + hi·Flo + lo·Fhi in
// FP32 in tensor memory (TMEM); the dropped lo·Flo term is about 2^-22
// relative.  Each thread reads its own accumulator row back (tcgen05.ld
// 32x32b: warp w sees TMEM lanes 32·(w mod 4) ..) and undoes the scale, so
// the outputs land where the FP32 butterfly would have left them.  The scale
// keeps FP16's range (largest finite 65504, smallest normal 2^-14) around
// every row whatever the magnitudes the transform has reached.  A CPU
// emulation of one stage on unit-variance rows gives a relative L2 error of
// 7.6e-8 for this format (FP32 arithmetic: 6.3e-8), against 3.1e-6 for BF16
// hi/lo with the same three products, whose 2^-18 residual of x dominates.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows × 16 bytes (8 FP16), 128 bytes each, K-adjacent core
// matrices 128 B apart (leading byte offset) and 8-row groups 512 B apart
// (stride byte offset) for K = 32.
#pragma once

#include <cuda_fp16.h>

#include "fft_core.cuh"
#include "tma.cuh"

namespace psolve {

constexpr int kTcK = 32;             // real K (16 complex inputs)
constexpr int kTcN = 32;             // real N (16 complex outputs)
constexpr int kTcRowBytes = kTcK * 2; // one FP16 row of A
constexpr int kTcFBytes = kTcN * kTcRowBytes; // one 32×32 FP16 matrix (2 KiB)

// Byte offset of element (row, k) of a K-major no-swizzle 16-bit operand with K = 32.
__host__ __device__ constexpr int tc_offset(int row, int k)
{
    return ((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start >> 4, leading byte offset
// >> 4, stride byte offset >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(p) & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B FP16
// (type fields at bits 7-9 and 10-12 = 0; A and B always share one type),
// both K-major, N = 32, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one full warp; the base address is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                 "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32])
{
    uint32_t u[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                   "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                   "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]),
                   "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]),
                   "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

// Power-of-two scale s of a row of 16 complex values that brings its largest
// |component| m into [2^14, 2^15), and 1/s in *inv (both exact).  The
// exponent of m is clamped to [-112, 113] so that s and 1/s stay normal
// FP32 numbers: rows with m below 2^-112 keep fewer bits (a zero row is
// harmless), rows with m at or above 2^114 would overflow FP16 and are
// outside the supported range.
__device__ __forceinline__ float tc_row_scale(const float2 (&a)[16], float &inv)
{
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) m = fmaxf(m, fmaxf(fabsf(a[k].x), fabsf(a[k].y)));
    int e = (int)((__float_as_uint(m) >> 23) & 0xFFu) - 127; // floor(log2 m) for normal m
    e = max(-112, min(113, e));
    inv = __uint_as_float((uint32_t)(127 - 14 + e) << 23);
    return __uint_as_float((uint32_t)(127 + 14 - e) << 23);
}

// Split s·x into FP16 hi + lo, packed two values per 32-bit word (x0 in the
// low half): the scaling is exact, hi is one paired conversion, the residual
// s·x - hi is exact in FP32, and lo is one more paired conversion.
__device__ __forceinline__ void f16_split2(float x0, float x1, float s, uint32_t &hi, uint32_t &lo)
{
    const float2 xs = cscale(make_float2(x0, x1), s);
    const __half2 h = __floats2half2_rn(xs.x, xs.y);
    const float2 r = csub(xs, __half22float2(h));
    const __half2 l = __floats2half2_rn(r.x, r.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// One operand row [Re a | Im a] as FP16 hi/lo words (hi[0..7]: Re, hi[8..15]:
// Im), scaled by s.
__device__ __forceinline__ void tc_split_row(const float2 (&a)[16], float s, uint32_t (&hi)[16], uint32_t (&lo)[16])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        f16_split2(a[2 * i].x, a[2 * i + 1].x, s, hi[i], lo[i]);         // Re a
        f16_split2(a[2 * i].y, a[2 * i + 1].y, s, hi[8 + i], lo[8 + i]); // Im a
    }
}

// Shared state of a block's tensor-core stages.
struct TcCtx {
    unsigned char *a_hi, *a_lo;   // 128·G rows × 64 B each
    const unsigned char *f_hi[2]; // [forward, inverse] 32×32 FP16, hi part
    const unsigned char *f_lo[2];
    uint32_t tmem;                // TMEM base (32·G columns)
    uint64_t *bar;                // MMA completion barrier
    uint32_t *phase;              // completed MMA batches (shared counter)
    int *abort;                   // shared flag set on a timed-out wait
    int *status;                  // device status word
};

// Build the four 32×32 FP16 DFT matrices (hi/lo × forward/inverse) in shared
// memory, from FP64 sincospi: hi = fp16(F), lo = fp16(F - hi) with the
// residual taken in FP64; called by the whole block.
__device__ __forceinline__ void tc_build_dft16(unsigned char *f_hi_fwd, unsigned char *f_lo_fwd,
                                               unsigned char *f_hi_inv, unsigned char *f_lo_inv)
{
    for (int i = threadIdx.x; i < kTcN * kTcK; i += blockDim.x) {
        const int n = i / kTcK, k = i % kTcK;
        const int kn = n & 15, kr = k & 15;
        double s, c;
        sincospi(2.0 * (double)((kn * kr) & 15) / 16.0, &s, &c); // angle 2π kn kr / 16
        for (int inv = 0; inv < 2; ++inv) {
            const double fi = inv ? s : -s; // Im F = ∓ sin
            double v;
            if (n < 16 && k < 16) v = c;
            else if (n < 16) v = -fi;
            else if (k < 16) v = fi;
            else v = c;
            const __half h = __float2half_rn((float)v);
            const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
            unsigned char *hp = inv ? f_hi_inv : f_hi_fwd;
            unsigned char *lp = inv ? f_lo_inv : f_lo_fwd;
            *reinterpret_cast<__half *>(hp + tc_offset(n, k)) = h;
            *reinterpret_cast<__half *>(lp + tc_offset(n, k)) = l;
        }
    }
}

// a[16] (this thread's butterfly) <- F a on the tensor cores.  All threads
// of the block call it; blockDim.x must be a multiple of 128.
template <bool INV>
__device__ __forceinline__ void tc_dft16(float2 (&a)[16], const TcCtx &ctx)
{
    const int tid = threadIdx.x;
    // 1. this row of A, scaled and split into FP16 hi/lo, four 16-byte chunks each
    float inv_s;
    {
        uint32_t hi[16], lo[16];
        tc_split_row(a, tc_row_scale(a, inv_s), hi, lo);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int off = tc_offset(tid, 8 * c);
            *reinterpret_cast<uint4 *>(ctx.a_hi + off) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
            *reinterpret_cast<uint4 *>(ctx.a_lo + off) = make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
        }
    }
    fence_proxy_async_smem(); // generic-proxy writes of A before the tensor core reads them
    tc_fence_before();
    __syncthreads();
    const uint32_t ph = *ctx.phase;
    if (tid == 0) {
        tc_fence_after();
        const int groups = blockDim.x >> 7;
        const unsigned char *fh = ctx.f_hi[INV ? 1 : 0];
        const unsigned char *fl = ctx.f_lo[INV ? 1 : 0];
        for (int g = 0; g < groups; ++g) {
            const uint32_t d = ctx.tmem + (uint32_t)(kTcN * g);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int kofs = ks * 256; // two core matrices of K per step
                const uint64_t ah = tc_smem_desc(ctx.a_hi + g * 128 * kTcRowBytes + kofs, 128, 512);
                const uint64_t al = tc_smem_desc(ctx.a_lo + g * 128 * kTcRowBytes + kofs, 128, 512);
                const uint64_t bh = tc_smem_desc(fh + kofs, 128, 512);
                const uint64_t bl = tc_smem_desc(fl + kofs, 128, 512);
                tc_mma(d, ah, bh, ks > 0 ? 1u : 0u);
                tc_mma(d, ah, bl, 1u);
                tc_mma(d, al, bh, 1u);
            }
        }
        tc_commit(ctx.bar);
        if (!mbar_wait_bounded(ctx.bar, ph & 1u, 2000000000ull)) {
            *ctx.abort = 1;
            atomicExch(ctx.status, 5 /* PSOLVE_ERR_TIMEOUT */);
            mbar_wait_bounded(ctx.bar, ph & 1u, 2000000000ull); // let issued MMAs drain before TMEM is freed
        }
        *ctx.phase = ph + 1;
    }
    __syncthreads();
    tc_fence_after();
    if (*ctx.abort) return; // the caller checks ctx.abort too
    // 2. this thread's accumulator row: columns 0..15 real, 16..31 imaginary
    const int w = tid >> 5;
    const uint32_t taddr = ctx.tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(kTcN * (w >> 2));
    float r[32];
    tmem_ld32(taddr, r);
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = cscale(make_float2(r[k], r[16 + k]), inv_s);
    tc_fence_before(); // these reads precede the next batch of MMAs
}

// ---------------------------------------------------------------------------
// Radix-16 stage on the tensor cores for lines of 512 points held 32 per
// thread (plan 32 × 16: radix-32 butterflies in FP32, then the radix-16 stage
// here, which is the last one).  Each thread owns two butterflies (rows), so
// a warpgroup of 128 threads forms two 128-row A operands.  Warpgroups work
// independently: each writes its operand rows, meets only its own 128
// threads at a named barrier, has one elected thread issue its MMAs and
// commit them to its own mbarrier, and then every thread waits on that
// mbarrier and reads its two accumulator rows back.  TMEM columns
// [64·g, 64·g + 64) belong to warpgroup g.

// Named barrier over the 128 threads of warpgroup g (id 0 is __syncthreads).
__device__ __forceinline__ void wg_barrier(int g)
{
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

// 64 consecutive FP32 columns of this thread's TMEM lane (one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&r)[64])
{
    uint32_t u[64];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
                 "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
                 "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                   "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                   "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]),
                   "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]),
                   "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31]),
                   "=r"(u[32]), "=r"(u[33]), "=r"(u[34]), "=r"(u[35]), "=r"(u[36]), "=r"(u[37]),
                   "=r"(u[38]), "=r"(u[39]), "=r"(u[40]), "=r"(u[41]), "=r"(u[42]), "=r"(u[43]),
                   "=r"(u[44]), "=r"(u[45]), "=r"(u[46]), "=r"(u[47]), "=r"(u[48]), "=r"(u[49]),
                   "=r"(u[50]), "=r"(u[51]), "=r"(u[52]), "=r"(u[53]), "=r"(u[54]), "=r"(u[55]),
                   "=r"(u[56]), "=r"(u[57]), "=r"(u[58]), "=r"(u[59]), "=r"(u[60]), "=r"(u[61]),
                   "=r"(u[62]), "=r"(u[63])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) r[i] = __uint_as_float(u[i]);
}

struct Tc32Ctx {
    unsigned char *op;            // operand rows: [warpgroup][butterfly b][hi, lo] × 8 KiB
    const unsigned char *f_hi[2]; // [forward, inverse] 32×32 FP16 DFT matrices
    const unsigned char *f_lo[2];
    uint32_t tmem;                // TMEM base (64 columns per warpgroup)
    uint64_t *bar;                // one MMA completion barrier per warpgroup
    int *abort;                   // shared flag set on a timed-out wait
    int *status;                  // device status word
};

constexpr int kTcOpBytes = 128 * kTcRowBytes; // one 128-row FP16 operand (8 KiB)

// Last stage (radix 16, Ns = 32) of a 512-point line, v[m] = x[t + 16·m]
// on entry (the exchanged radix-32 outputs) and out[t + 16·m] on exit, with
// the stage's twiddles w_512^{r·j} applied in FP32 first.  `nphase` counts
// this warpgroup's completed MMA batches (identical in all its threads).
template <bool INV>
__device__ __forceinline__ void tc32_last_stage(float2 (&v)[32], int t, const float2 *__restrict__ tw,
                                                const Tc32Ctx &c, uint32_t &nphase)
{
    constexpr int TL = 16, NB = 2;
    const int tid = threadIdx.x, g = tid >> 7, rl = tid & 127;
    const unsigned char *fh = c.f_hi[INV ? 1 : 0];
    const unsigned char *fl = c.f_lo[INV ? 1 : 0];
    float inv_s[NB]; // each butterfly row's scale, undone on the way back
    // Butterfly 0's MMAs run while butterfly 1's operand rows are formed.
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * TL; // butterfly j < Ns = 32: twiddle exponent r·j
        float2 a[16];
        a[0] = v[b];
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            const float2 w = tw[r * j];
            a[r] = INV ? cmulc(v[b + r * NB], w) : cmul(v[b + r * NB], w);
        }
        uint32_t hi[16], lo[16];
        tc_split_row(a, tc_row_scale(a, inv_s[b]), hi, lo);
        unsigned char *oh = c.op + ((g * NB + b) * 2) * kTcOpBytes;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int off = tc_offset(rl, 8 * q);
            *reinterpret_cast<uint4 *>(oh + off) = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
            *reinterpret_cast<uint4 *>(oh + kTcOpBytes + off) =
                make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
        }
        fence_proxy_async_smem(); // operand rows before the tensor core reads them
        tc_fence_before();
        wg_barrier(g);
        if (rl == 0) {
            tc_fence_after();
            const uint32_t d = c.tmem + (uint32_t)(64 * g + 32 * b);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int kofs = ks * 256; // two core matrices of K per step
                const uint64_t ah = tc_smem_desc(oh + kofs, 128, 512);
                const uint64_t al = tc_smem_desc(oh + kTcOpBytes + kofs, 128, 512);
                const uint64_t bh = tc_smem_desc(fh + kofs, 128, 512);
                const uint64_t bl = tc_smem_desc(fl + kofs, 128, 512);
                tc_mma(d, ah, bh, ks > 0 ? 1u : 0u);
                tc_mma(d, ah, bl, 1u);
                tc_mma(d, al, bh, 1u);
            }
            if (b == NB - 1) tc_commit(&c.bar[g]); // completion of both butterflies' MMAs
        }
    }
    const bool done = mbar_wait_bounded(&c.bar[g], nphase & 1u, 2000000000ull);
    if (!done) {
        *c.abort = 1;
        atomicExch(c.status, 5 /* PSOLVE_ERR_TIMEOUT */);
    }
    ++nphase;
    // After a timed-out wait the accumulator is not read: the MMAs may still
    // be running (the kernel lets them drain before it frees TMEM).  The read
    // is warp-collective, so a warp skips it as a whole.
    if (!__all_sync(0xFFFFFFFFu, done)) return;
    tc_fence_after();
    const int wq = (tid >> 5) & 3; // TMEM lanes 32·wq .. 32·wq + 31 for this warp
    float r[64];
    tmem_ld64(c.tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(64 * g), r);
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < 16; ++k) v[b + k * NB] = cscale(make_float2(r[32 * b + k], r[32 * b + 16 + k]), inv_s[b]);
    tc_fence_before(); // these reads precede the warpgroup's next MMAs
}

// Compile-time-plan line transform in which every radix-16 stage runs on the
// tensor cores (E = 16: one butterfly per thread and stage).  Twiddles and
// other radices stay in FP32.  Single-buffer exchanges in `sm`.  All threads
// of the block call it; on a timed-out tensor-core wait it returns early
// with *ctx.abort set (uniformly across the block).
template <bool INV, int L, int S, typename Map>
__device__ __forceinline__ void line_fft_tc_from(float2 (&v)[16], int t, const float2 *__restrict__ tw,
                                                 float2 *sm, const Map &map, const TcCtx &ctx)
{
    constexpr int E = 16;
    constexpr int NST = ct_nst(L, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(L, S, E);
        constexpr int NS = ct_ns(L, S, E);
        constexpr int TL = L / E;
        constexpr bool LAST = (S + 1 == NST);
        if constexpr (R == 16) {
            const int jm = t % NS;
            if constexpr (NS > 1) {
                const int q = jm * (L / (NS * 16));
#pragma unroll
                for (int r = 1; r < 16; ++r) {
                    const float2 w = tw[r * q];
                    v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
                }
            }
            tc_dft16<INV>(v, ctx);
            if (*ctx.abort) return;
            if constexpr (!LAST) {
                const int base = (t - jm) * 16 + jm;
#pragma unroll
                for (int k = 0; k < 16; ++k) sm[map(base + k * NS)] = v[k];
            }
        } else {
            fft_stage_ct<R, INV, LAST, TL, NS, L / (NS * R)>(v, t, tw, sm, map, true);
        }
        if constexpr (!LAST) {
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = sm[map(t + m * TL)];
            __syncthreads();
            line_fft_tc_from<INV, L, S + 1>(v, t, tw, sm, map, ctx);
        }
    }
}

} // namespace psolve
