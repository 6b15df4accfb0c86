// Register/shared-memory FFT engine shared by every pass kernel.
//
// A line of L complex points is processed by TL = L/E threads, each holding
// E points in registers.  Thread t starts and ends holding the "strided
// class" of the line: v[m] = x[t + m·TL], m = 0..E-1.  The transform is a
// mixed-radix Stockham (self-sorting) FFT: stage s with radix R and
// Ns = R_1·…·R_{s-1} takes butterfly j (0 <= j < L/R) over the inputs
// x[j + r·L/R], multiplies input r by w_{Ns·R}^{r·(j mod Ns)}, applies the
// R-point DFT and writes output k to y[(j / Ns)·Ns·R + (j mod Ns) + k·Ns].
// Thread t owns butterflies j = t + b·TL (b < E/R), whose inputs are exactly
// v[b + r·E/R], so only the outputs go through shared memory; the last stage
// (Ns·R = L) writes back into the strided class, i.e. stays in registers.
// This is the 1D building block of the 3D transform in §2.1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace psolve {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a · conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return {a.x * s, a.y * s}; }

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(PSOLVE_NO_F32X2)
// Blackwell packed FP32x2 arithmetic: one instruction per complex add, sub
// (a - b as the fused b·(-1) + a, exact) or real scale.  Products and ±i
// rotations stay scalar: on pairs they need the swapped pair (a.y, a.x),
// whose moves cost more than the packing saves (measured).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
#endif

// a · (c + i s) for a real pair (c, s).
template <typename C, typename T> __device__ __forceinline__ C cmul_cs(C a, T c, T s)
{
    return C{a.x * c - a.y * s, a.x * s + a.y * c};
}
// a - i·b (DN = true) or a + i·b, the odd outputs of the radix-4 butterfly.
template <bool DN, typename C> __device__ __forceinline__ C cadd_rot(C a, C b)
{
    return DN ? C{a.x + b.y, a.y - b.x} : C{a.x - b.y, a.y + b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }

// Multiply by -i (forward direction) or +i (inverse direction).
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a)
{
    return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

// Exact values of cos(πm/8), sin(πm/8), m = 0..8, for the radix-8/16 kernels.
struct Oct {
    static constexpr double c[9] = {1.0,
                                    0.923879532511286756128183189396788933,
                                    0.707106781186547524400844362104849039,
                                    0.382683432365089771728459984030398866,
                                    0.0,
                                    -0.382683432365089771728459984030398866,
                                    -0.707106781186547524400844362104849039,
                                    -0.923879532511286756128183189396788933,
                                    -1.0};
    static constexpr double s[9] = {0.0,
                                    0.382683432365089771728459984030398866,
                                    0.707106781186547524400844362104849039,
                                    0.923879532511286756128183189396788933,
                                    1.0,
                                    0.923879532511286756128183189396788933,
                                    0.707106781186547524400844362104849039,
                                    0.382683432365089771728459984030398866,
                                    0.0};
};

// a · w_16^m with w_16 = e^{∓2πi/16} (forward/inverse), 0 <= m <= 8.
template <bool INV, int M, typename C> __device__ __forceinline__ C mul_w16(C a)
{
    using T = decltype(a.x);
    if constexpr (M == 0) {
        return a;
    } else if constexpr (M == 4) {
        return rot90<INV>(a);
    } else if constexpr (M == 8) {
        return C{-a.x, -a.y};
    } else {
        const T c = (T)Oct::c[M];
        const T s = INV ? (T)Oct::s[M] : -(T)Oct::s[M];
        return cmul_cs(a, c, s);
    }
}

// ---------------------------------------------------------------- butterflies
// In-place R-point DFT  a[k] <- Σ_r a[r] e^{∓2πi rk/R}.

template <bool INV, typename C> __device__ __forceinline__ void dft2(C *a)
{
    C t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C *a)
{
    using T = decltype(a[0].x);
    const T h = (T)0.866025403784438646763723170752936183; // √3/2
    C t1 = cadd(a[1], a[2]);
    C t2 = csub(a[1], a[2]);
    C m = {a[0].x - (T)0.5 * t1.x, a[0].y - (T)0.5 * t1.y};
    a[0] = cadd(a[0], t1);
    // forward: out1 = m - i h t2, out2 = m + i h t2
    C r = {h * t2.y, -h * t2.x}; // -i h t2
    if (INV) r = C{-r.x, -r.y};
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C *a)
{
    C a0 = cadd(a[0], a[2]), a1 = csub(a[0], a[2]);
    C a2 = cadd(a[1], a[3]), d = csub(a[1], a[3]);
    a[0] = cadd(a0, a2);
    a[2] = csub(a0, a2);
    // a1 ∓ i·d (forward: out1 = a1 - i d, out3 = a1 + i d)
    a[1] = cadd_rot<!INV>(a1, d);
    a[3] = cadd_rot<INV>(a1, d);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C *a)
{
    C e[4] = {a[0], a[2], a[4], a[6]};
    C o[4] = {a[1], a[3], a[5], a[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    o[1] = mul_w16<INV, 2>(o[1]);
    o[2] = mul_w16<INV, 4>(o[2]);
    o[3] = mul_w16<INV, 6>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = cadd(e[k], o[k]);
        a[k + 4] = csub(e[k], o[k]);
    }
}

// 16 = 4 × 4:  n = 4 n1 + n2,  k = k1 + 4 k2.
template <bool INV, typename C> __device__ __forceinline__ void dft16(C *a)
{
    C y[4][4]; // y[n2][k1]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C col[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
        dft4<INV>(col);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = col[k1];
    }
    // twiddles w16^{n2·k1}
    y[1][1] = mul_w16<INV, 1>(y[1][1]);
    y[1][2] = mul_w16<INV, 2>(y[1][2]);
    y[1][3] = mul_w16<INV, 3>(y[1][3]);
    y[2][1] = mul_w16<INV, 2>(y[2][1]);
    y[2][2] = mul_w16<INV, 4>(y[2][2]);
    y[2][3] = mul_w16<INV, 6>(y[2][3]);
    y[3][1] = mul_w16<INV, 3>(y[3][1]);
    y[3][2] = mul_w16<INV, 6>(y[3][2]);
    {
        // w16^9 = -w16^1
        C t = mul_w16<INV, 1>(y[3][3]);
        y[3][3] = C{-t.x, -t.y};
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C row[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
        dft4<INV>(row);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = row[k2];
    }
}

// Exact values of cos(πk/16), sin(πk/16) for odd k = 1, 3, 5, 7.
struct Hex {
    static constexpr double c[4] = {0.980785280403230449126182236134239037, 0.831469612302545237078788377617905757,
                                    0.555570233019602224742830813948532874, 0.195090322016128267848284868477022241};
};

// a · w_32^k with w_32 = e^{∓2πi/32}, 0 <= k < 16.
template <bool INV, int K, typename C> __device__ __forceinline__ C mul_w32(C a)
{
    using T = decltype(a.x);
    if constexpr (K % 2 == 0) {
        return mul_w16<INV, K / 2>(a);
    } else {
        // cos(πK/16), sin(πK/16) from the first octant: K = 1,3,5,7 direct,
        // K = 9..15 via cos(π - x) = -cos x, sin(π - x) = sin x.
        constexpr int k = K < 8 ? K : 16 - K;
        const T c0 = (T)Hex::c[(k - 1) / 2];
        const T s0 = (T)Hex::c[3 - (k - 1) / 2]; // sin(πk/16) = cos(π(8-k)/16)
        const T c = K < 8 ? c0 : -c0;
        const T s = INV ? s0 : -s0;
        return cmul_cs(a, c, s);
    }
}

// 32 = 2 × 16 (decimation in time).
template <bool INV, typename C> __device__ __forceinline__ void dft32(C *a)
{
    C e[16], o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        e[k] = a[2 * k];
        o[k] = a[2 * k + 1];
    }
    dft16<INV>(e);
    dft16<INV>(o);
#define PSOLVE_R32(K)                                                                              \
    {                                                                                              \
        const C t = mul_w32<INV, K>(o[K]);                                                         \
        a[K] = cadd(e[K], t);                                                                      \
        a[K + 16] = csub(e[K], t);                                                                 \
    }
    PSOLVE_R32(0) PSOLVE_R32(1) PSOLVE_R32(2) PSOLVE_R32(3) PSOLVE_R32(4) PSOLVE_R32(5) PSOLVE_R32(6)
    PSOLVE_R32(7) PSOLVE_R32(8) PSOLVE_R32(9) PSOLVE_R32(10) PSOLVE_R32(11) PSOLVE_R32(12) PSOLVE_R32(13)
    PSOLVE_R32(14) PSOLVE_R32(15)
#undef PSOLVE_R32
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C *a)
{
    if constexpr (R == 2) dft2<INV>(a);
    else if constexpr (R == 3) dft3<INV>(a);
    else if constexpr (R == 4) dft4<INV>(a);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 16) dft16<INV>(a);
    else if constexpr (R == 32) dft32<INV>(a);
}

// ------------------------------------------------------------------ plans

constexpr int kMaxStages = 16;

// One 1D transform of length L split into stages; computed on the host.
struct LinePlan {
    int L;                      // line length (complex points)
    int E;                      // points per thread
    int TL;                     // threads per line = L / E
    int nst;                    // number of stages
    int radix[kMaxStages];      // R_s
    int ns[kMaxStages];         // Ns before stage s
    int twstep[kMaxStages];     // L / (Ns·R): twiddle index step
    unsigned nsmag[kMaxStages]; // ceil(2^32 / Ns) for Ns >= 2: j / Ns = umulhi(j, nsmag), exact while j·Ns < 2^32
};

// Fill the division multipliers of a plan whose ns[] are set.
inline void line_plan_finish(LinePlan &p)
{
    for (int s = 0; s < p.nst; ++s)
        p.nsmag[s] = p.ns[s] >= 2 ? (unsigned)(((1ull << 32) + (unsigned long long)p.ns[s] - 1) /
                                               (unsigned long long)p.ns[s])
                                  : 0u;
}

// Index map of a line's point p into the shared exchange buffer.
struct MapStrided { // [p][w], pitch P: lines side by side (y and x passes)
    int P, w;
    __device__ __forceinline__ int operator()(int p) const { return p * P + w; }
};
// [p][w] with a spare row after every 2^SH rows.  The first Stockham stage
// (radix R = 2^SH) writes rows R apart from neighbouring threads; the spare
// row makes that distance R + 1, so with rows of 8 columns (half the banks)
// neighbouring threads land in opposite bank halves instead of the same one.
template <int SH = 4> struct MapStridedPad {
    int P, w;
    __device__ __forceinline__ int operator()(int p) const { return (p + (p >> SH)) * P + w; }
};
// [p][w] in exactly L·P slots (the tile buffer itself): row p trades places
// with row p ^ 1 when bit SH of p is set.  With rows of 8 columns (half the
// banks), the first stage's writes from neighbouring threads, 2^SH rows
// apart, then land in opposite bank halves, and rows read together stay
// adjacent pairs.
template <int SH> struct MapStridedSwz {
    int P, w;
    __device__ __forceinline__ int operator()(int p) const { return (p ^ ((p >> SH) & 1)) * P + w; }
};
template <int SH = 4> struct MapRow { // [w][p], one row per line with a spare slot every 2^SH (z passes)
    int base;
    __device__ __forceinline__ int operator()(int p) const { return base + p + (p >> SH); }
};

template <int R, bool INV, bool LAST, int E, typename C, typename Map>
__device__ __forceinline__ void fft_stage(C (&v)[E], int t, int TL, int Ns, unsigned nsmag, int twstep,
                                          const C *__restrict__ tw, C *sm, const Map &map,
                                          bool active)
{
    constexpr int NB = E / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * TL;
        // j mod Ns by a multiply-high (lines are far shorter than 2^16 points)
        const int jm = Ns > 1 ? j - (int)__umulhi((unsigned)j, nsmag) * Ns : 0;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[b + r * NB];
        if (Ns > 1) {
            const int q = jm * twstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = tw[r * q];
                a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
            }
        }
        dft<R, INV>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = a[r];
        } else {
            if (active) {
                const int base = (j - jm) * R + jm;
#pragma unroll
                for (int r = 0; r < R; ++r) sm[map(base + r * Ns)] = a[r];
            }
        }
    }
}

template <int R, int E> struct RadixOk { static constexpr bool value = (E % R) == 0; };

template <bool INV, bool LAST, int E, typename C, typename Map>
__device__ __forceinline__ void fft_stage_dispatch(int R, C (&v)[E], int t, int TL, int Ns, unsigned nsmag, int twstep,
                                                   const C *__restrict__ tw, C *sm, const Map &map,
                                                   bool active)
{
    switch (R) {
    case 16:
        if constexpr (RadixOk<16, E>::value) fft_stage<16, INV, LAST>(v, t, TL, Ns, nsmag, twstep, tw, sm, map, active);
        break;
    case 8:
        if constexpr (RadixOk<8, E>::value) fft_stage<8, INV, LAST>(v, t, TL, Ns, nsmag, twstep, tw, sm, map, active);
        break;
    case 4:
        if constexpr (RadixOk<4, E>::value) fft_stage<4, INV, LAST>(v, t, TL, Ns, nsmag, twstep, tw, sm, map, active);
        break;
    case 3:
        if constexpr (RadixOk<3, E>::value) fft_stage<3, INV, LAST>(v, t, TL, Ns, nsmag, twstep, tw, sm, map, active);
        break;
    case 2:
        if constexpr (RadixOk<2, E>::value) fft_stage<2, INV, LAST>(v, t, TL, Ns, nsmag, twstep, tw, sm, map, active);
        break;
    default:
        break;
    }
}

// Full line transform.  All threads of the block must call it (it contains
// __syncthreads); `active` masks the shared-memory writes of idle threads.
template <bool INV, int E, typename C, typename Map>
__device__ __forceinline__ void line_fft(C (&v)[E], int t, const LinePlan &pl,
                                         const C *__restrict__ tw, C *sm, const Map &map, bool active)
{
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s];
        if (s + 1 == pl.nst) {
            fft_stage_dispatch<INV, true>(R, v, t, pl.TL, pl.ns[s], pl.nsmag[s], pl.twstep[s], tw, sm, map, active);
        } else {
            fft_stage_dispatch<INV, false>(R, v, t, pl.TL, pl.ns[s], pl.nsmag[s], pl.twstep[s], tw, sm, map, active);
            __syncthreads();
            if (active) {
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = sm[map(t + m * pl.TL)];
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------- compile-time line plans
// The same stage plan as the host's make_line_plan, evaluated at compile time
// for hot line lengths: radix-3 stages first, then the largest power-of-two
// radices (<= 16) dividing E.  With every stage constant, the j mod Ns and
// twiddle-index arithmetic folds to shifts and masks.
constexpr int ct_pow2(int L) { int a = 0; while (L % 2 == 0) { L /= 2; ++a; } return a; }
constexpr int ct_pow3(int L)
{
    while (L % 2 == 0) L /= 2;
    int b = 0;
    while (L % 3 == 0) { L /= 3; ++b; }
    return b;
}
constexpr int ct_min(int a, int b) { return a < b ? a : b; }
constexpr int ct_E(int L)
{
    return ct_pow3(L) > 0 ? 3 * (1 << ct_min(ct_pow2(L), 3)) : (1 << ct_min(ct_pow2(L), 4));
}
constexpr int ct_p2(int E) { int p = 1; while (E % (p * 2) == 0 && p * 2 <= 32) p *= 2; return p; }
constexpr int ct_radix(int L, int s, int E = 0)
{
    const int b = ct_pow3(L);
    if (s < b) return 3;
    int rem = 1 << ct_pow2(L);
    const int p2 = ct_p2(E > 0 ? E : ct_E(L));
    for (int i = b;; ++i) {
        const int r = p2 < rem ? p2 : rem;
        if (i == s) return rem > 1 ? r : 1;
        rem /= r;
    }
}
constexpr int ct_nst(int L, int E = 0)
{
    int n = 0;
    while (ct_radix(L, n, E) > 1) ++n;
    return n;
}
constexpr int ct_ns(int L, int s, int E = 0)
{
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= ct_radix(L, i, E);
    return ns;
}

template <int R, bool INV, bool LAST, int TL, int NS, int TWS, int E, typename C, typename Map>
__device__ __forceinline__ void fft_stage_ct(C (&v)[E], int t, const C *__restrict__ tw, C *sm,
                                             const Map &map, bool active)
{
    constexpr int NB = E / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + b * TL;
        const int jm = j % NS;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[b + r * NB];
        if constexpr (NS > 1) {
            const int q = jm * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const C w = tw[r * q];
                a[r] = INV ? cmulc(a[r], w) : cmul(a[r], w);
            }
        }
        dft<R, INV>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * NB] = a[r];
        } else {
            if (active) {
                const int base = (j - jm) * R + jm;
#pragma unroll
                for (int r = 0; r < R; ++r) sm[map(base + r * NS)] = a[r];
            }
        }
    }
}

template <bool INV, int L, int S, int E, typename C, typename Map>
__device__ __forceinline__ void line_fft_ct_from(C (&v)[E], int t, const C *__restrict__ tw, C *sm,
                                                 const Map &map, bool active)
{
    constexpr int NST = ct_nst(L, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(L, S, E);
        constexpr int NS = ct_ns(L, S, E);
        constexpr int TL = L / E;
        constexpr bool LAST = (S + 1 == NST);
        static_assert(E % R == 0, "radix must divide the points per thread");
        fft_stage_ct<R, INV, LAST, TL, NS, L / (NS * R)>(v, t, tw, sm, map, active);
        if constexpr (!LAST) {
            __syncthreads();
            if (active) {
#pragma unroll
                for (int m = 0; m < E; ++m) v[m] = sm[map(t + m * TL)];
            }
            __syncthreads();
            line_fft_ct_from<INV, L, S + 1>(v, t, tw, sm, map, active);
        }
    }
}

// As line_fft_ct_from, but stage s writes its outputs to bufs[(PAR + s) & 1]
// (each buffer with its own index map) and needs a single barrier per exchange: a buffer is written again only two
// exchanges later, after every thread has passed the barrier that follows its
// last read of it.  The caller must not read either buffer concurrently with
// the first exchange's writes to bufs[PAR].
template <bool INV, int L, int S, int PAR, int E, typename C, typename Map0, typename Map1>
__device__ __forceinline__ void line_fft_ct_db(C (&v)[E], int t, const C *__restrict__ tw, C *buf0, C *buf1,
                                               const Map0 &map0, const Map1 &map1)
{
    constexpr int NST = ct_nst(L, E);
    if constexpr (S < NST) {
        constexpr int R = ct_radix(L, S, E);
        constexpr int NS = ct_ns(L, S, E);
        constexpr int TL = L / E;
        constexpr bool LAST = (S + 1 == NST);
        constexpr bool ONE = ((PAR + S) & 1) != 0;
        if constexpr (ONE) {
            fft_stage_ct<R, INV, LAST, TL, NS, L / (NS * R)>(v, t, tw, buf1, map1, true);
        } else {
            fft_stage_ct<R, INV, LAST, TL, NS, L / (NS * R)>(v, t, tw, buf0, map0, true);
        }
        if constexpr (!LAST) {
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = ONE ? buf1[map1(t + m * TL)] : buf0[map0(t + m * TL)];
            line_fft_ct_db<INV, L, S + 1, PAR>(v, t, tw, buf0, buf1, map0, map1);
        }
    }
}

// Number of exchanges (shared-memory round trips) of an L-point line.
constexpr int ct_exchanges(int L, int E) { return ct_nst(L, E) - 1; }

// Line transform with a compile-time plan when LC > 0, else the run-time plan.
template <bool INV, int LC, int E, typename C, typename Map>
__device__ __forceinline__ void line_fft_any(C (&v)[E], int t, const LinePlan &pl, const C *__restrict__ tw,
                                             C *sm, const Map &map, bool active)
{
    if constexpr (LC > 0) {
        static_assert(LC % E == 0 && (ct_pow3(LC) == 0 || E % 3 == 0),
                      "compile-time plan: E divides the line, and holds the radix-3 factor if there is one");
        line_fft_ct_from<INV, LC, 0>(v, t, tw, sm, map, active);
    } else {
        line_fft<INV>(v, t, pl, tw, sm, map, active);
    }
}

// Signed wavenumber of index j on an axis of n points: j for j <= n/2,
// j - n otherwise (the Nyquist index counts as +n/2).
__device__ __forceinline__ int kvec_dev(int j, int n) { return (2 * j <= n) ? j : j - n; }

} // namespace psolve
