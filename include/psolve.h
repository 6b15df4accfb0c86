/*
 * psolve — spectral Poisson solver for -Δu = f, periodic on the unit cube,
 * as hand-written CUDA kernels for one GB300 (sm_103a).  C ABI.
 *
 * The operation (§1, Eq. 1.1; §2.1; §3 of Gholami, Malhotra, Sundar, Biros,
 * "FFT, FMM, or Multigrid?"): forward 3D FFT of f, each coefficient divided
 * by the Laplacian's spectral symbol, inverse 3D FFT:
 *
 *     u = A f,   A = F^{-1} D F,   D(k) = 1 / (4π² |k|²),   D(0) = 0,
 *
 * on the grid x_j = j/n_i (j = 0..n_i-1) per axis, with signed wavenumbers
 * k(j) = j for j <= n/2, j - n otherwise (the Nyquist index counts as +n/2;
 * only k² enters D).  The mean of f is projected out (û(0) = 0), so u has
 * zero mean and the caller need not subtract the mean of f.
 *
 * Arrays.  f and u are real, C-order (nx, ny, nz) with z contiguous, in the
 * plan's precision (double for PSOLVE_F64, float otherwise).  A plan with
 * batch B > 1 takes B instances back to back: instance b starts at element
 * psolve_instance_offset(plan, b).  Pointers passed to psolve_execute and
 * psolve_adjoint are DEVICE pointers on the plan's device, 16-byte aligned.
 *
 * Streams.  Every `stream` argument is a cudaStream_t passed as void*
 * (NULL = the legacy default stream).  Execution is asynchronous on that
 * stream; the library never synchronises it except where stated.
 *
 * Errors.  Every call returns a psolve_status.  Host-detectable problems
 * (bad sizes, null or misaligned pointers, partial aliasing, a destroyed
 * plan) are returned before anything is enqueued.  A CUDA launch or copy
 * failure returns PSOLVE_ERR_CUDA.  Asynchronous device-side errors are
 * recorded in the plan's device status word and read by psolve_get_status.
 * psolve_last_error() gives a human-readable message for the calling thread.
 */
#ifndef PSOLVE_H
#define PSOLVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSOLVE_F64 = 0,     /* double in, double out, FP64 butterflies          */
    PSOLVE_F32 = 1,     /* float in, float out, FP32 butterflies            */
    PSOLVE_F32_TC = 2   /* float in/out; radix-16 stages of the y and x passes on the tensor
                           cores (tcgen05; FP16 hi/lo operands with a power-of-two scale
                           per butterfly row, FP32 accumulation in TMEM)
                           where those passes use the TMA kernels (lines of 256, 512 or 1024
                           points); every other stage in FP32.  Lines of 512 points use the
                           plan 32 × 16 by default (radix-32 stage in FP32, the radix-16
                           stage on the tensor cores); the others, and 512 when asked, plans
                           of radix-16 stages (16 × 16 × …), each on the tensor cores.
                           psolve_pass_name reports "yfwd_tc", "xdiv_tc", "yinv_tc" for the
                           passes that do.  Equal-grid plans only. */
} psolve_dtype;

typedef enum {
    PSOLVE_OK = 0,
    PSOLVE_ERR_INVALID_ARG = 1,      /* null/misaligned pointer, bad batch, bad dtype, partial overlap */
    PSOLVE_ERR_UNSUPPORTED_SIZE = 2, /* an n is not 2^a 3^b, is odd, < 4 or > 2048 (FP64: nx = 1458) */
    PSOLVE_ERR_OOM = 3,              /* device allocation failed                                       */
    PSOLVE_ERR_CUDA = 4,             /* a CUDA call failed (no device, launch error, ...)              */
    PSOLVE_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up                             */
    PSOLVE_ERR_INTERNAL = 6          /* a device-side consistency check failed                         */
} psolve_status;

/* The operator a plan inverts: the step between the forward and inverse
 * transforms multiplies the spectrum by 1/den(k) (with the transforms' 1/N).
 *   PSOLVE_OP_POISSON       −Δu = f (§1, Eq. 1.1; §2.1): den = 4π²|k|², 0 at
 *                           k = 0 (the mean of f is dropped, u has mean 0).
 *   PSOLVE_OP_HELMHOLTZ     −Δu + c·u = f, c > 0: den = 4π²|k|² + c (every
 *                           mode kept; a constant f gives u = f/c).
 *   PSOLVE_OP_FD_LAPLACIAN  the second-order 7-point finite-difference
 *                           Laplacian of the grid, which the same transforms
 *                           diagonalise (footnote to §1): den = Σ_axes
 *                           4 n² sin²(π k/n), 0 at k = 0; u solves the
 *                           discrete equation up to rounding. */
typedef enum {
    PSOLVE_OP_POISSON = 0,
    PSOLVE_OP_HELMHOLTZ = 1,
    PSOLVE_OP_FD_LAPLACIAN = 2
} psolve_operator;

typedef struct psolve_plan psolve_plan;

/* Create a plan for `batch` equal grids nx × ny × nz (§3: the setup is paid
 * once and amortised over solves with new right-hand sides).  Each n must
 * be 2^a·3^b, even, 4 <= n <= 2048; FP64 plans also reject nx = 1458
 * (2·3^6: the x pass's tile of two such lines needs 486 threads, more than
 * an FP64 block holds), with PSOLVE_ERR_UNSUPPORTED_SIZE.  Allocates the plan's twiddle tables
 * (computed on the device in FP64) and status word on the current device.
 * The spectrum is formed inside u itself, so no workspace of the grid's
 * size is allocated, except for FP32 grids whose x lines lie 4 MiB or more
 * apart (ny·(nz/2)·8 bytes, e.g. 1024³): their plans also own a spectrum
 * buffer of the grid's size (nx·ny·nz floats per grid), in which the
 * spectrum is kept in an x-split order that serves the x transform better;
 * if that allocation fails the plan keeps the in-place layout.  On success
 * *out owns the plan; release it with psolve_destroy.  On failure *out is
 * set to NULL. */
psolve_status psolve_plan_create(int nx, int ny, int nz, int dtype, int batch,
                                 psolve_plan **out);

/* Create a plan for `batch` grids of unequal sizes (nx[b], ny[b], nz[b]),
 * solved together.  Instance b starts at element psolve_instance_offset(b)
 * of the packed f/u arrays; offsets are aligned up to 32 elements.  FP32
 * plans whose every line fits a 128-thread tile (at most 16 points a
 * thread, 12 for lengths 3·2^a; x lines of at most 64 threads) solve every
 * pass of every instance in one persistent kernel launched from a CUDA
 * graph; other plans (FP64, or lines such as 2048 points or 2·3^b points)
 * launch each pass of each instance in turn, with the same results to
 * rounding.  psolve_launches_per_solve tells which.  Size rules and errors
 * as psolve_plan_create. */
psolve_status psolve_plan_create_many(const int *nx, const int *ny, const int *nz, int batch,
                                      int dtype, psolve_plan **out);

/* u = A f for every instance (§2.1).  f, u: device pointers holding
 * psolve_total_elements(plan) values.  u == f (in place) is allowed; any
 * other overlap is PSOLVE_ERR_INVALID_ARG.  f is not modified unless u == f.
 * Enqueued on `stream` without synchronising.  Solves of one plan must not
 * overlap on the device: the plan's spectrum buffer (x-split plans), the
 * persistent batched launch's work counters and the status word are shared
 * by its solves, so solves on several streams need one plan per stream or
 * streams ordered by events. */
psolve_status psolve_execute(psolve_plan *plan, const void *f, void *u, void *stream);

/* grad_f = A^T g.  A is real symmetric (D is real and even in k), so this is
 * the same operator; it is the backward of psolve_execute. */
psolve_status psolve_adjoint(psolve_plan *plan, const void *g, void *grad_f, void *stream);

/* psolve_execute on HOST buffers, synchronous on `stream`.  Uses a device
 * buffer owned by the plan (allocated on first use) for the spectrum.  When
 * both buffers are pinned (page-locked, e.g. cudaHostAlloc) and the plan is
 * of equal grids, the first pass reads f and the last pass writes u directly
 * across the host link; otherwise f is copied in and u copied out.  Either
 * way f_host and u_host may not overlap. */
psolve_status psolve_execute_host(psolve_plan *plan, const void *f_host, void *u_host,
                                  void *stream);

/* Asynchronous psolve_execute_host for pipelines: enqueue on `stream` and
 * return at once.  f is copied in and u copied out by the copy engines
 * (pinned buffers make these asynchronous).  The plan keeps three device
 * staging buffers of the grid's size, allocated on first use and used in
 * turn, each guarded by an event, so consecutive calls issued on different
 * streams (three or more) overlap one solve's output copy with the next
 * one's input copy and a third one's kernels.  f_host and u_host must stay valid and unchanged
 * until the work on `stream` completes; synchronise the streams to collect
 * u.  Calls for one plan must come from one host thread. */
psolve_status psolve_execute_host_async(psolve_plan *plan, const void *f_host, void *u_host, void *stream);

/* Choose the operator the plan's later solves (and adjoints: the operator
 * is self-adjoint) invert; plans start with PSOLVE_OP_POISSON.  c is used by
 * PSOLVE_OP_HELMHOLTZ only and must be positive and finite.  The first
 * switch to PSOLVE_OP_FD_LAPLACIAN allocates the symbol tables (a few KiB,
 * FP64).  Synchronous (blocking) and not to be called while a solve of the
 * plan is in flight.  Returns PSOLVE_ERR_INVALID_ARG for an unknown operator
 * or a bad c.  With an operator other than Poisson, FP32 grids whose x
 * lines have 256, 512 or 1024 points keep the TMA-fed x pass (forward x
 * transform, multiplier, inverse x transform) at its default configuration;
 * every other case runs it in the per-tile kernels, in FP32 also for
 * PSOLVE_F32_TC plans (psolve_pass_name then reports "xdiv").  Grids keep
 * the natural spectrum layout.
 * psolve_execute_noalloc always solves the Poisson equation. */
psolve_status psolve_set_operator(psolve_plan *plan, int op, double c);

/* Free everything the plan owns.  The plan pointer is invalid afterwards. */
psolve_status psolve_destroy(psolve_plan *plan);

/* Element offset of instance b in the packed f/u arrays; (size_t)-1 on error. */
size_t psolve_instance_offset(const psolve_plan *plan, int b);

/* Number of elements the packed f/u arrays hold; 0 on error. */
size_t psolve_total_elements(const psolve_plan *plan);

/* Synchronise `stream`, read and clear the plan's device status word. */
psolve_status psolve_get_status(psolve_plan *plan, void *stream);

/* Write the signed wavenumbers the division kernel uses for instance b, as
 * computed on the device: for every spectrum index (jx, jy, jz),
 * 0 <= jz <= nz/2, three int32 (kx, ky, kz) at
 * kxyz_out[3 * ((jx * ny + jy) * (nz/2 + 1) + jz)].  kxyz_out is a HOST
 * buffer of 3·nx·ny·(nz/2+1) ints.  Synchronous. */
psolve_status psolve_debug_kvec(const psolve_plan *plan, int b, int *kxyz_out);

/* FP64 reductions over n elements of two device arrays a, ref of `dtype`:
 * out4[0] = Σ (a - ref)², out4[1] = Σ ref², out4[2] = max |a - ref|,
 * out4[3] = max |ref|.  out4 is a HOST array of 4 doubles.  Synchronous on
 * `stream`. */
psolve_status psolve_error_norms(const void *a, const void *ref, size_t n, int dtype,
                                 double *out4, void *stream);

/* Autotune the plan in place: time candidate tile widths, TMA tile
 * configurations and (for the persistent batched launch) radix orders of
 * each pass on a scratch copy of one instance, keep the fastest, and store
 * the choices in a per-GPU cache file ($PSOLVE_TUNE_CACHE, else
 * $HOME/.cache/psolve/tune-v1.txt) that later psolve_plan_create /
 * psolve_plan_create_many calls read.  This is the setup-time tuning that
 * §3 and Table 1 amortise over many solves.  Synchronises `stream`,
 * allocates and frees one instance of scratch, and must not run while a
 * solve of this plan is in flight.  Results are unchanged up to rounding. */
psolve_status psolve_autotune(psolve_plan *plan, void *stream);

/* Per-pass timing with CUDA events recorded on the solve's own stream.
 * After psolve_set_profiling(plan, k), k >= 1, every k-th
 * psolve_execute/psolve_adjoint (the first, then every k-th after it)
 * records an event before the first pass and after each pass; the kernels
 * and their order are unchanged.  A recorded solve runs its passes strictly
 * one after the other (an event between two passes stops the next one from
 * starting its set-up while the previous one drains), so k > 1 leaves most
 * solves as fast as unprofiled ones.  psolve_pass_times synchronises the
 * events, writes into ms[i] the summed milliseconds of pass i over all
 * recorded solves (at most cap passes), sets *n_passes and *n_solves, and
 * clears the record.  psolve_set_profiling(plan, 0) stops recording; a
 * negative k is PSOLVE_ERR_INVALID_ARG. */
psolve_status psolve_set_profiling(psolve_plan *plan, int enable);
psolve_status psolve_pass_times(psolve_plan *plan, double *ms, int cap, int *n_passes, int *n_solves);

/* Name of pass i of the plan's solve ("zfwd", "yfwd", "xdiv", "yinv",
 * "zinv"), or NULL. */
const char *psolve_pass_name(const psolve_plan *plan, int i);

/* Number of kernel launches one psolve_execute enqueues; 0 on error.  A plan
 * of unequal grids (psolve_plan_create_many) runs every pass of every
 * instance in ONE persistent kernel launched from a CUDA graph (a memset
 * node zeroes its work counters first), and its profile has a single pass
 * named "batched". */
int psolve_launches_per_solve(const psolve_plan *plan);

/* Test hook for the persistent batched launch: its blocks wait for the
 * tiles of an instance's previous pass with a time limit of wait_ns
 * nanoseconds (default 2 s), after which they record PSOLVE_ERR_TIMEOUT in
 * the status word (read by psolve_get_status) and exit; the GPU context stays
 * usable.  unsatisfiable = 1 makes pass 1 of instance 0 wait for one more
 * tile than pass 0 has, so that wait must run out; 0 restores it.
 * PSOLVE_ERR_INVALID_ARG for a plan without the batched launch. */
psolve_status psolve_debug_set_wait(psolve_plan *plan, unsigned long long wait_ns, int unsatisfiable);

/* Allocation-free solve, for callers that cannot allocate device memory:
 * code inside a custom allocator or memory-pool callback, frameworks that
 * forbid allocation during a step, hosts that reserve all device memory up
 * front.  The paper has no counterpart.  It solves one grid nx × ny × nz
 * without a plan, with the same argument checks as psolve_execute and the
 * per-tile pass kernels psolve_execute uses where its TMA and bulk-copy
 * passes do not apply (those are not used here), with the planner's stage
 * plans and tile shapes; results agree with psolve_execute's within the
 * dtype's tolerance, not bit for bit.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The only
 * memory besides f and u is the twiddle tables, held in one fixed 64 KiB
 * device array inside the library (every GPU that loads the library keeps
 * it until the process exits); a grid needs (nx + ny + nz) complex values
 * there (8 B each in FP32, 16 B in FP64), so every valid FP32 grid fits and
 * an FP64 grid fits while nx + ny + nz <= 4096; larger grids (and the
 * sizes psolve_plan_create rejects, FP64 nx = 1458 included) return
 * PSOLVE_ERR_UNSUPPORTED_SIZE before anything is enqueued.
 * dtype: PSOLVE_F32 or PSOLVE_F64 (else PSOLVE_ERR_INVALID_ARG).  f, u:
 * device pointers as for psolve_execute (u == f allowed).
 * The first call on each device looks up the array's device address with
 * that device current (cudaGetSymbolAddress) and keeps it; make that call
 * before any stream capture.  Resetting the device (cudaDeviceReset) after
 * that first call is not supported.  Every call rewrites the whole array on `stream` before its
 * kernels read it, so nothing carries over from the previous call, but calls
 * whose work overlaps on the GPU (different streams, no ordering) race on
 * the shared array and give wrong results: order them.
 * psolve_last_error() is not updated by this call. */
psolve_status psolve_execute_noalloc(int nx, int ny, int nz, int dtype, const void *f, void *u,
                                     void *stream);

/* Test hook for the tensor-core radix-16 stage used by PSOLVE_F32_TC: for
 * each of `nbutterflies` rows of 16 complex FP32 values (in, device,
 * interleaved re/im, row-major), out = F·in with F[k][r] = e^{-2πi kr/16}
 * (inverse = 1: e^{+2πi kr/16}), computed as FP16 hi/lo products (each
 * row scaled by a power of two first) accumulated in FP32 in tensor memory.  Synchronises `stream`.  Returns
 * PSOLVE_ERR_TIMEOUT if the tensor-core completion wait ran out. */
psolve_status psolve_debug_tc_dft16(const void *in, void *out, int nbutterflies, int inverse, void *stream);

/* Static description of a status code. */
const char *psolve_status_string(psolve_status s);

/* Message for the last error reported on the calling thread ("" if none). */
const char *psolve_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int psolve_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PSOLVE_H */
