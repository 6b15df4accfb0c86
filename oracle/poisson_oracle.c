/*
 * FP64 CPU oracle for the periodic Poisson solve -Δu = f on the unit cube.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which is
 * loaded by the test-suite, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg.  The CUDA library never links, includes or calls it, and it
 * shares no code, header or table with the CUDA kernels.
 *
 * What it computes (the plain definition, no blocking, no fusion):
 *   §1, Eq. 1.1:  -Δu = f, f smooth and periodic on [0,1)^3.
 *   §2.1:         transform f, multiply each coefficient by the reciprocal of
 *                 the Laplacian's spectral symbol, transform back.
 *   §3:           the solve as timed there: a forward 3D FFT, a pointwise
 *                 scaling, an inverse 3D FFT.
 * On the grid x_j = j/n the discrete Fourier coefficients are
 *     F[k] = sum_x f[x] e^{-2πi k·x/n}   (per axis, no scaling),
 * the spectral symbol of -Δ is 4π²|k|² with the signed wavenumber
 *     k(j) = j for j <= n/2, j - n otherwise,
 * û = F / (4π²|k|²) with û(0) = 0 (the mean of f is projected out), and
 *     u[x] = (1/N) sum_k û[k] e^{+2πi k·x/n}.
 *
 * The same transforms invert two further operators (oracle_op_inverse):
 * Helmholtz −Δu + c·u = f, multiplier 1/(4π²|k|² + c), and the 7-point
 * finite-difference Laplacian of the grid, multiplier 1/Σ(2n²)(1 − cos 2πk/n).
 *
 * The 1D transforms are computed either by the direct O(n^2) sum of that
 * definition, or by a plain recursive Cooley–Tukey split by the smallest factor
 * (2, then 3; anything else falls back to the direct sum) applied to full
 * complex lines.  Twiddles are cos/sin of 2π·(m mod n)/n with the integer m
 * reduced exactly before the conversion to double.
 */
#include <complex.h>
#include <math.h>
/* ORACLE_MUTANT selects a deliberately wrong variant, compiled only by the
 * mutation test to show that the pins catch each plausible slip; 0 (the
 * default, and the only value any build of liboracle.so uses) is the oracle. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static const double ORACLE_PI = 3.14159265358979323846264338327950288;
static const double ORACLE_TWO_PI = 6.28318530717958647692528676655900577;
static const double ORACLE_FOUR_PI_SQ = 39.4784176043574344753379639995046046;

/* e^{sign·2πi·m/n}, m reduced exactly mod n first. */
static cplx unit_root(long long m, long long n, int sign)
{
    m %= n;
    if (m < 0) m += n;
    double ang = ORACLE_TWO_PI * (double)m / (double)n;
    return cos(ang) + (double)sign * sin(ang) * I;
}

/* Signed wavenumber of index j on an axis of n points (§2.1 reading: the
 * Nyquist index j = n/2 is taken as +n/2; only k² enters the multiplier). */
int oracle_kvec(int j, int n)
{
#if ORACLE_MUTANT == 3
    return j; /* planted: wrap-around forgotten */
#endif
    return (2 * j <= n) ? j : j - n;
}

/* Direct DFT of one line: out[k] = sum_j in[j·is] e^{sign 2πi jk/n}. */
static void dft_direct_line(const cplx *in, ptrdiff_t is, cplx *out, int n, int sign)
{
    for (int k = 0; k < n; ++k) {
        cplx acc = 0.0;
        for (int j = 0; j < n; ++j)
            acc += in[(ptrdiff_t)j * is] * unit_root((long long)j * k, n, sign);
        out[k] = acc;
    }
}

/* Recursive Cooley–Tukey: out[0..n) = DFT_n(in[0], in[is], in[2 is], ...).
 * Split n = p·m with p the smallest of {2, 3} dividing n:
 *   Y_s = DFT_m of the subsequence in[(p j + s)·is], j = 0..m-1,
 *   X[k + q m] = sum_s e^{sign 2πi s (k + q m)/n} Y_s[k].
 * w is the table e^{sign 2πi e/ntop}, e = 0..ntop-1, with n | ntop. */
static void fft_rec(const cplx *in, ptrdiff_t is, cplx *out, int n, int sign,
                    const cplx *w, int ntop)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = (n % 2 == 0) ? 2 : ((n % 3 == 0) ? 3 : n);
    if (p == n && n > 3) {
        dft_direct_line(in, is, out, n, sign);
        return;
    }
    int m = n / p;
    for (int s = 0; s < p; ++s)
        fft_rec(in + (ptrdiff_t)s * is, is * p, out + (ptrdiff_t)s * m, m, sign, w, ntop);
    int scale = ntop / n;
    cplx y[3], r[3];
    for (int k = 0; k < m; ++k) {
        for (int s = 0; s < p; ++s) y[s] = out[s * m + k];
        for (int q = 0; q < p; ++q) {
            cplx acc = 0.0;
            for (int s = 0; s < p; ++s) {
                long long e = ((long long)s * (k + q * m)) % n;
#if ORACLE_MUTANT == 2
                acc += y[s] * conj(w[e * scale]); /* planted: twiddle sign */
#elif ORACLE_MUTANT == 7
                acc += y[s] * w[(((long long)s * (k + q)) % n) * scale]; /* planted: index */
#else
                acc += y[s] * w[e * scale];
#endif
            }
            r[q] = acc;
        }
        for (int q = 0; q < p; ++q) out[k + q * m] = r[q];
    }
}

static int oracle_threads = 0;

void oracle_set_threads(int n) { oracle_threads = n; }

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return oracle_threads > 0 ? oracle_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* 1D transform along one axis of the C-order complex array a (nx, ny, nz),
 * in place, for every line of that axis. */
static void transform_axis(cplx *a, int nx, int ny, int nz, int axis, int sign, int direct)
{
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    ptrdiff_t stride = axis == 0 ? (ptrdiff_t)ny * nz : (axis == 1 ? nz : 1);
    long long lines = (long long)nx * ny * nz / n;
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) w[e] = unit_root(e, n, sign);
    int nthr = oracle_get_threads();
    (void)nthr;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthr)
#endif
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (long long l = 0; l < lines; ++l) {
            /* base offset of line l: enumerate the two other axes */
            ptrdiff_t base;
            if (axis == 2) {
                base = (ptrdiff_t)l * nz;
            } else if (axis == 1) {
                long long x = l / nz, z = l % nz;
                base = (ptrdiff_t)x * ny * nz + z;
            } else {
                base = (ptrdiff_t)l; /* l = y*nz + z */
            }
            for (int j = 0; j < n; ++j) line[j] = a[base + (ptrdiff_t)j * stride];
            if (direct)
                dft_direct_line(line, 1, res, n, sign);
            else
                fft_rec(line, 1, res, n, sign, w, n);
            for (int j = 0; j < n; ++j) a[base + (ptrdiff_t)j * stride] = res[j];
        }
        free(line);
        free(res);
    }
    free(w);
}

/* 3D DFT of the interleaved (re, im) array in place (the transform of §2.1
 * written out: one 1D DFT per line along each axis).  sign = -1 forward,
 * +1 inverse; never scaled. */
void oracle_dft3d(double *re_im, int nx, int ny, int nz, int sign, int direct)
{
    cplx *a = (cplx *)re_im;
    transform_axis(a, nx, ny, nz, 2, sign, direct);
    transform_axis(a, nx, ny, nz, 1, sign, direct);
    transform_axis(a, nx, ny, nz, 0, sign, direct);
}

/* The spectral multiplier of the solve, 1/(4π²|k|²), 0 at k = 0 (§2.1). */
double oracle_symbol_inverse(int jx, int jy, int jz, int nx, int ny, int nz)
{
    long long kx = oracle_kvec(jx, nx), ky = oracle_kvec(jy, ny), kz = oracle_kvec(jz, nz);
#if ORACLE_MUTANT == 4
    kx = oracle_kvec(jx, ny); ky = oracle_kvec(jy, nx); /* planted: axes swapped */
#endif
    long long k2 = kx * kx + ky * ky + kz * kz;
    if (k2 == 0) return 0.0;
#if ORACLE_MUTANT == 1
    return 1.0 / (double)k2; /* planted: 4π² dropped */
#elif ORACLE_MUTANT == 5
    if (2 * jx == nx || 2 * jy == ny || 2 * jz == nz) return 0.0; /* planted: Nyquist dropped */
#endif
    return 1.0 / (ORACLE_FOUR_PI_SQ * (double)k2);
}

/* Multiplier of the other operators the same transforms invert:
 *   op 1, Helmholtz −Δu + c·u = f: 1/(4π²|k|² + c), c > 0, every mode kept;
 *   op 2, the 7-point finite-difference Laplacian on the grid (h = 1/n per
 *         axis), whose Fourier modes are eigenvectors with eigenvalue
 *         Σ_axes (2/h²)(1 − cos(2πk/n)): 1/eigenvalue, 0 at k = 0 (the stencil
 *         variant the paper's footnote to §1 mentions).  Each term is
 *         evaluated as (4/h²) sin²(πk/n), the same number by the half-angle
 *         identity 1 − cos 2x = 2 sin² x: the cosine form cancels for the
 *         lowest modes of fine grids (at n = 2048, k = 1 it keeps only about
 *         11 of its 16 digits), and those modes dominate u;
 *   op 0, anything else: the Poisson multiplier above. */
double oracle_op_inverse(int op, double c, int jx, int jy, int jz, int nx, int ny, int nz)
{
    long long kx = oracle_kvec(jx, nx), ky = oracle_kvec(jy, ny), kz = oracle_kvec(jz, nz);
#if ORACLE_MUTANT == 9
    c = 0.0 * c + 1.0; /* planted: the Helmholtz shift replaced by 1 */
#endif
    if (op == 1) return 1.0 / (ORACLE_FOUR_PI_SQ * (double)(kx * kx + ky * ky + kz * kz) + c);
    if (op == 2) {
        if (kx == 0 && ky == 0 && kz == 0) return 0.0;
        double lam = 0.0;
        const long long k[3] = {kx, ky, kz};
        const int n[3] = {nx, ny, nz};
        for (int a = 0; a < 3; ++a) {
#if ORACLE_MUTANT == 8
            const double s = sin(ORACLE_PI * (double)(2 * k[a]) / (double)n[a]); /* planted: 2k */
#else
            const double s = sin(ORACLE_PI * (double)k[a] / (double)n[a]);
#endif
            lam += 4.0 * (double)n[a] * (double)n[a] * s * s;
        }
        return 1.0 / lam;
    }
    return oracle_symbol_inverse(jx, jy, jz, nx, ny, nz);
}

/* u = F^{-1}[ F[f] · multiplier(op) ]; op 0 gives the Poisson solve of
 * §2.1 (the three steps §3 times) u = F^{-1}[ F[f] / (4π²|k|²) ], û(0) = 0.  Returns 0 on success, -1 on
 * allocation failure.  *max_imag receives max |Im u| before it is dropped. */
int oracle_solve_op(const double *f, double *u, int nx, int ny, int nz, int direct, int op, double c,
                    double *max_imag)
{
    size_t N = (size_t)nx * ny * nz;
    cplx *a = (cplx *)malloc(sizeof(cplx) * N);
    if (!a) return -1;
    for (size_t i = 0; i < N; ++i) a[i] = f[i];
    oracle_dft3d((double *)a, nx, ny, nz, -1, direct);
    for (int jx = 0; jx < nx; ++jx)
        for (int jy = 0; jy < ny; ++jy)
            for (int jz = 0; jz < nz; ++jz) {
                size_t i = ((size_t)jx * ny + jy) * nz + jz;
                a[i] *= op == 0 ? oracle_symbol_inverse(jx, jy, jz, nx, ny, nz)
                                : oracle_op_inverse(op, c, jx, jy, jz, nx, ny, nz);
            }
    oracle_dft3d((double *)a, nx, ny, nz, +1, direct);
    double mi = 0.0, inv_n = 1.0 / (double)N;
#if ORACLE_MUTANT == 6
    inv_n = 2.0 / (double)N; /* planted: wrong normalisation */
#endif
    for (size_t i = 0; i < N; ++i) {
        u[i] = creal(a[i]) * inv_n;
        double im = fabs(cimag(a[i])) * inv_n;
        if (im > mi) mi = im;
    }
    if (max_imag) *max_imag = mi;
    free(a);
    return 0;
}

int oracle_solve(const double *f, double *u, int nx, int ny, int nz, int direct, double *max_imag)
{
    return oracle_solve_op(f, u, nx, ny, nz, direct, 0, 0.0, max_imag);
}
