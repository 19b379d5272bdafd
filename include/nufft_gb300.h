/*
 * nufft_gb300.h -- C ABI of a GB300 (sm_103a) implementation of the type-1 and
 * type-2 non-uniform FFT with the "exponential of semicircle" (ES) kernel of
 * Barnett, Magland & af Klinteberg, arXiv:1808.06736.
 *
 * Transforms (Sec. 1, Eq. (1) and Eq. (2)), with the sign flag isign = +1 or -1:
 *   type 1 (non-uniform to uniform):  f_k = sum_{j=1..M} c_j exp(i isign k.x_j),  k in I_N
 *   type 2 (uniform to non-uniform):  c_j = sum_{k in I_N} f_k exp(i isign k.x_j), j = 1..M
 * computed to relative tolerance eps by spreading / interpolation with the ES
 * kernel on a 2x upsampled grid, an FFT and a diagonal correction (Sec. 3).
 * I_N = I_{N_1} x ... x I_{N_d}, I_{N_i} = {-floor(N_i/2), ..., N_i - 1 - floor(N_i/2)}.
 * The type-2 transform with sign -isign is the adjoint of the type-1 transform
 * with sign isign.
 *
 * Conventions shared by every entry point:
 *  - Points x_j, y_j, z_j are given in radians; the transforms are 2 pi
 *    periodic, so any finite value is accepted (opts.chkbnds = 1 restricts
 *    them to [-3 pi, 3 pi], as Sec. 2 describes).
 *  - Complex arrays are interleaved (re, im): float pairs for NUFFT_C64,
 *    double pairs for NUFFT_C128.  Point arrays are float resp. double.
 *  - Mode arrays f hold N_1 * ... * N_d values, dimension 1 fastest, each
 *    dimension in increasing k (opts.modeord = 0) or in FFT order
 *    0, 1, ..., -1 (opts.modeord = 1).
 *  - Every pointer handed to nufft_setpts / nufft_execute is DEVICE memory on
 *    the plan's device; the caller keeps ownership.  All device work is
 *    enqueued on the plan's CUDA stream and is asynchronous with respect to
 *    the host; nufft_get_status / nufft_get_timings synchronise that stream.
 *  - Return values: 0 success, > 0 warning (the call still did its work),
 *    < 0 error (the call did nothing further).  nufft_strerror names them.
 *  - A plan is not thread-safe; use one plan per host thread.
 */
#ifndef NUFFT_GB300_H
#define NUFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* precision selector for nufft_makeplan */
#define NUFFT_C64 1  /* complex64 data, float points, float arithmetic   */
#define NUFFT_C128 2 /* complex128 data, double points, double arithmetic */

/* status codes */
#define NUFFT_OK 0
#define NUFFT_WARN_EPS_TOO_SMALL 1   /* eps below what the precision (or w <= 16) can deliver */
#define NUFFT_ERR_BAD_ARG (-1)       /* invalid type, dim, N_i, isign, ntransf, eps, M, prec or NULL pointer */
#define NUFFT_ERR_OUT_OF_RANGE (-2)  /* opts.chkbnds = 1 and a point lies outside [-3 pi, 3 pi] (or is not finite) */
#define NUFFT_ERR_ALLOC (-3)         /* device allocation failed */
#define NUFFT_ERR_CUDA (-4)          /* a CUDA runtime call or kernel launch failed */
#define NUFFT_ERR_CUFFT (-5)         /* cuFFT planning or execution failed */
#define NUFFT_ERR_NOT_SET (-6)       /* nufft_execute before nufft_setpts */
#define NUFFT_ERR_TOO_BIG (-7)       /* M >= 2^31, or a grid the index types cannot address */
#define NUFFT_ERR_TIMEOUT (-8)       /* serving: a request was not done within the server's time limit */
#define NUFFT_ERR_REJECTED (-9)      /* serving: a request needs more device memory than the whole budget */
#define NUFFT_ERR_SHUTDOWN (-10)     /* serving: the server was destroyed before the request ran */

typedef struct nufft_plan_s* nufft_plan;

/*
 * Options (Sec. 2 describes debug and chkbnds; the rest are GPU tunables).
 * nufft_default_opts fills every field; 0 in a tunable means "choose".
 */
typedef struct {
  int debug;          /* 1: record CUDA-event timings of every step (nufft_get_timings) */
  int chkbnds;        /* 1: points outside [-3 pi, 3 pi] make nufft_get_status return NUFFT_ERR_OUT_OF_RANGE */
  int modeord;        /* 0: increasing k per dimension; 1: FFT order (0..N/2-1 then -N/2..-1) */
  int bin_size[3];    /* bin extent in fine-grid cells per dimension (0: choose from d, w, precision) */
  int max_subprob;    /* most points one thread block handles at a time (0: choose) */
  int threads;        /* threads per block of the spread / interp kernels (0: choose) */
  int sparse_max;     /* subproblems of at most this many points (<= 32) run one per warp straight
                         on the fine grid instead of through a shared-memory tile (0: 32, -1: never) */
  int kerevalmeth;    /* kernel evaluation in the spread / interp kernels: 0 the ES formula (one exp and one
                         sqrt per node), 1 the piecewise polynomial of Sec. 5.3 (w intervals of degree
                         w + 3, Horner's scheme; see nufft_horner_coeffs; the autotuner tries both).
                         The complex128 interpolation (double-float) and the gradient kernels always
                         use the formula. */
  int kernel;         /* 0: the ES kernel, Eq. (ES); 1: its smooth variant 2 e^-beta cosh(beta sqrt(1 - z^2))
                         (Remark in Sec. 7: within e^-beta of ES, bounded derivatives; same w and beta, its
                         own correction factors), for point gradients (nufft_execute_grad).  The spread
                         and interp kernels evaluate it through its piecewise polynomial (Sec. 5.3),
                         the gradient and complex128 interpolation kernels through its formula */
  int reserved[5];    /* set to zero */
  double upsampfac;   /* fine grid / modes per dimension, sigma: 2 (0 means 2) or 1.25 (smaller FFTs and
                         grids, wider kernel: w from the slope of Eq. (ESerr), beta from Eq. (gam); more
                         rounding amplification, see nufft_choose_params_sigma) */
} nufft_opts;

/* Fill *o with defaults.  Returns NUFFT_OK, or NUFFT_ERR_BAD_ARG for o == NULL. */
int nufft_default_opts(nufft_opts* o);

/*
 * Create a plan for ntransf transforms of one type that share the points.
 *   type      1 or 2.
 *   dim       1, 2 or 3.
 *   nmodes    host array of dim mode counts N_i >= 1.
 *   isign     +1 or -1: the sign of i in the exponent (Sec. 2).
 *   ntransf   >= 1 vectors per nufft_execute (strided by M resp. N_1...N_d).
 *   eps       requested relative tolerance > 0.  Sets the kernel width
 *             w = ceil(log10(1/eps)) + 1 and beta = 2.30 w (Eq. (params)),
 *             and the fine grid n_i = smallest 2^a 3^b 5^c >= max(2 N_i, 2 w)
 *             (Sec. 3.1.1).  w is clamped to [2, 16].  eps below 1e-6
 *             (C64) or 1e-15 (C128) returns NUFFT_WARN_EPS_TOO_SMALL with
 *             a valid plan: the precision cannot deliver that accuracy.
 *   prec      NUFFT_C64 or NUFFT_C128.
 *   stream    a cudaStream_t (NULL = the legacy default stream); the plan uses
 *             the current CUDA device.
 *   opts      NULL for defaults.
 *   out       receives the plan (NULL on error).
 * Work: computes the correction factors of Eq. (pk) (host, double precision,
 * Gauss-Legendre rule of Eq. (quad)), allocates the fine grid and plans cuFFT.
 * Synchronous.  Errors: BAD_ARG, ALLOC, CUDA, CUFFT, TOO_BIG.
 */
int nufft_makeplan(int type, int dim, const int64_t* nmodes, int isign, int ntransf, double eps,
                   int prec, void* stream, const nufft_opts* opts, nufft_plan* out);

/*
 * Set the M points (device arrays; y NULL when dim < 2, z NULL when dim < 3).
 * Folds each coordinate onto the fine grid, bins the points by a counting sort
 * over fine-grid bins (cf. Sec. 5.1) and builds the subproblem list (cf. Sec.
 * 5.2).  The plan keeps the sorted, folded coordinates, so the caller may
 * free or overwrite x, y, z after the call has completed on the stream.
 * M = 0 is allowed.  Errors: BAD_ARG (M < 0, NULL with M > 0), TOO_BIG
 * (M >= 2^31), ALLOC, CUDA.  Out-of-range points are reported later by
 * nufft_get_status when opts.chkbnds = 1.
 */
int nufft_setpts(nufft_plan plan, int64_t M, const void* x, const void* y, const void* z);

/*
 * nufft_setpts_from -- give plan dst the points src has binned, without binning
 * them again.  The bin sort of Sec. 5.1 depends on the points, the fine grid
 * and the bins only, so a type-1 and a type-2 plan on the same points (or two
 * plans of one type) can share it; typical use: setpts on a type-1 plan, then
 * nufft_setpts_from(type-2 plan, type-1 plan).
 *
 * The two plans must have the same device, precision, dimension, fine grid
 * n_i, bin extents (opts.bin_size), largest subproblem (opts.max_subprob) and
 * per-warp threshold (opts.sparse_max); isign, type, ntransf, eps with the
 * same grid and kernel options may differ.  The binned points are shared, not
 * copied: neither plan may be destroyed from under the other (both keep them
 * alive), and a later nufft_setpts on either plan gives that plan a new set,
 * leaving the other's unchanged.  No device work is enqueued; dst's executes
 * must be ordered after src's setpts (same stream, or an event) by the caller.
 * Points outside [-3 pi, 3 pi] (opts.chkbnds) are reported by src's
 * nufft_get_status only.
 *
 * Returns NUFFT_OK; NUFFT_ERR_BAD_ARG (NULL plan, or the plans differ in any
 * of the above); NUFFT_ERR_NOT_SET (src has no points).
 */
int nufft_setpts_from(nufft_plan dst, nufft_plan src);

/*
 * Run the ntransf transforms on device arrays c (ntransf * M complex) and f
 * (ntransf * N_1 ... N_d complex).  Type 1 reads c and writes f (spread,
 * Eq. (bl); FFT, Eq. (dft1); truncate and correct, Eq. (pb1)).  Type 2 reads
 * f and writes c (pre-correct and pad, Sec. 3.2 step 1; FFT, Eq. (dft);
 * interpolate, Eq. (interp)).  With M = 0 a type-1 plan writes f = 0 and a
 * type-2 plan does nothing.  Errors: BAD_ARG, NOT_SET, CUDA, CUFFT.
 */
int nufft_execute(nufft_plan plan, void* c, void* f);

/*
 * Type-2 plans only: nufft_execute plus the gradient of each value in its
 * point.  Writes c as nufft_execute does and dc, dim * M complex values per
 * transform (row d at dc + d * M holds dc_j / dx_{j,d}), obtained by
 * differentiating the interpolation (Eq. (interp)) with the derivative of the
 * ES kernel, phi'(z) = -beta z / sqrt(1 - z^2) phi(z) (the paper's remark on
 * kernel derivatives, Sec. 7, notes that phi' is unbounded at z = +-1; the
 * factor 1 / sqrt(1 - z^2) is capped at 1e3).  The exact gradient is
 * sum_k f_k (i isign k_d) exp(i isign k.x_j); this one approximates it with a
 * relative error a few times eps (aliased frequencies near the fine-grid size
 * are weighted by their own size).  Transform t reads f + t N, writes
 * c + t M and dc + t dim M.  Errors: BAD_ARG (type-1 plan, NULL pointer),
 * NOT_SET, CUDA, CUFFT.
 */
int nufft_execute_grad(nufft_plan plan, void* c, void* dc, const void* f);

/* Free every resource of the plan (synchronises its stream).  NULL is accepted. */
int nufft_destroy(nufft_plan plan);

/*
 * Synchronise the plan's stream and return the first asynchronous error the
 * device recorded since the last call (NUFFT_ERR_OUT_OF_RANGE, or
 * NUFFT_ERR_CUDA for a failed launch), then clear it.  NUFFT_OK otherwise.
 */
int nufft_get_status(nufft_plan plan);

/*
 * With opts.debug = 1: synchronise and copy up to n step timings in
 * milliseconds of the most recent setpts / execute into ms:
 *   [0] setpts: fold + bin count   [1] setpts: scans + subproblem list
 *   [2] setpts: scatter            [3] execute: spread or pre-correct/pad
 *   [4] execute: FFT               [5] execute: deconvolve or interpolate
 * (for type 2, [3] is pre-correct and [5] interpolation).  Returns the number
 * of entries written, or a negative error code.
 */
int nufft_get_timings(nufft_plan plan, double* ms, int n);

/*
 * Plan facts, for callers and tests.  Any output pointer may be NULL.
 * w, beta: kernel width and ES parameter; n: dim fine-grid sizes;
 * bins: dim bin extents; nsub: number of subproblems of the last setpts
 * (synchronises the stream).
 */
int nufft_plan_info(nufft_plan plan, int* w, double* beta, int64_t* n, int* bins, int64_t* nsub);

/* Static text for a status code. */
const char* nufft_strerror(int code);

/* ------------------------------------------------------------------ host-only
 * The following run on the host only (no device call), so they work without
 * a GPU.  They expose the plan's parameter rules and correction factors.
 */

/*
 * Parameters of Eq. (params) and Sec. 3.1.1 for tolerance eps:
 * *w, *beta, and n[0..dim-1] from nmodes[0..dim-1].  Returns NUFFT_OK,
 * NUFFT_WARN_EPS_TOO_SMALL, or NUFFT_ERR_BAD_ARG.
 */
int nufft_choose_params(int dim, const int64_t* nmodes, double eps, int prec, int* w, double* beta,
                        int64_t* n);
/* The same for upsampling factor sigma = 2 or 1.25 (NUFFT_ERR_BAD_ARG otherwise).
 * At 1.25 NUFFT_WARN_EPS_TOO_SMALL also flags eps that needs w > 16 (about
 * eps < 1e-9), and eps below unit roundoff times rmax^dim, rmax =
 * exp((1 - sqrt(1 - (2 sigma - 1)^-2)) beta) (Eq. (rmax)): the correction
 * amplifies rounding by up to that factor, e^{0.25 beta} per dimension at 1.25
 * (complex64: fine for 1D down to eps 1e-5, 2D 1e-3, 3D 1e-3; complex128 to 1e-9
 * in 1D and 2D, about 1e-6 in 3D). */
int nufft_choose_params_sigma(int dim, const int64_t* nmodes, double eps, int prec, double sigma, int* w,
                              double* beta, int64_t* n);

/*
 * Correction factors of Eq. (pk1) for one dimension: out[m] = 2 / (w phi^(alpha k)),
 * k = m - floor(N/2), m = 0..N-1, alpha = pi w / n (Eq. (al)), with phi^ from
 * the 2p-node Gauss-Legendre rule of Eq. (quad), p = ceil(1.5 w + 2), and the
 * cosines generated by phase winding (Sec. 3.1.1).  Double precision.
 * Returns NUFFT_OK or NUFFT_ERR_BAD_ARG.
 */
int nufft_correction_factors(int64_t N, int64_t n, int w, double beta, double* out);

/* Smallest 2^a 3^b 5^c >= m (m >= 1); returns -1 on overflow or m < 1. */
int64_t nufft_next235(int64_t m);

/* Host-only: the piecewise polynomial of Sec. 5.3 used with opts.kerevalmeth = 1.  The kernel
 * psi(tau) = phi(2 tau / w) on its support tau in [-w/2, w/2] (fine-grid cells) is split into
 * w unit intervals; on interval t (tau in [t - w/2, t - w/2 + 1]) it is the polynomial
 * sum_m out[t (w + 4) + m] s^m of degree w + 3 in s = 2 (tau - t + w/2) - 1 in [-1, 1].
 * Coefficients by interpolation at the w + 4 Chebyshev points of the first kind, converted to
 * monomials.  out: w (w + 4) doubles.  Returns NUFFT_OK or NUFFT_ERR_BAD_ARG (w outside
 * [2, 16], beta <= 0, out NULL). */
int nufft_horner_coeffs(int w, double beta, double* out);

/* ------------------------------------------------------------------ batches
 * Many independent transforms in one plan: B transforms of one type,
 * dimension, precision, sign and eps, each with its own mode counts (the
 * many-vector / plan interfaces Remark r:small of the paper asks for, for
 * repeated small problems).  Every step runs as one launch over all
 * transforms and the execute sequence is captured in a CUDA graph (when the
 * plan has a non-NULL stream) and replayed while c, f and the point set stay
 * the same.
 */
typedef struct nufft_batch_s* nufft_batch;

/* nmodes: host array of B * dim mode counts (transform-major).  Errors as in
 * nufft_makeplan; returns NUFFT_WARN_EPS_TOO_SMALL like it. */
int nufft_batch_makeplan(int type, int dim, int B, const int64_t* nmodes, int isign, double eps, int prec,
                         void* stream, const nufft_opts* opts, nufft_batch* out);

/* Points of all transforms, concatenated: transform t owns points
 * offsets[t] .. offsets[t+1]-1 (offsets: host array of B + 1 values,
 * offsets[0] = 0, non-decreasing, offsets[B] < 2^31).  x, y, z: device arrays
 * of offsets[B] coordinates.  Errors: BAD_ARG, TOO_BIG, ALLOC, CUDA. */
int nufft_batch_setpts(nufft_batch plan, const int64_t* offsets, const void* x, const void* y, const void* z);

/* c: all strengths / results, concatenated like the points; f: all mode
 * arrays concatenated in transform order (each N_1 ... N_d, dimension 1
 * fastest).  Type 1 reads c and writes f, type 2 reads f and writes c. */
int nufft_batch_execute(nufft_batch plan, void* c, void* f);

/* Synchronise and return the first recorded device error (see nufft_get_status). */
int nufft_batch_get_status(nufft_batch plan);

/* Free everything; NULL is accepted. */
int nufft_batch_destroy(nufft_batch plan);

/* ---------------------------------------------------------------- autotuning
 * Time launch configurations on the caller's own points and data and return
 * the fastest as options for nufft_makeplan / nufft_batch_makeplan: the bin
 * extents (hence the shared-memory tile, bin + w per dimension; 1D 256..4096,
 * 2D {8,16,32,64}^2, 3D B1 >= B2 >= B3 in {4,8,16,32}, those whose tile fits
 * in shared memory), the largest subproblem (max_subprob 256..4096), the
 * per-warp threshold (sparse_max -1, 8, 16, default 32), the threads per
 * block (128, default 256) and the upsampling factor (1.25 when eps needs no
 * more than w = 16 there, default 2).  Staged search: bins first, then each further
 * tunable from the best so far; the default options are timed first, so
 * *best_ms <= *default_ms.  A configuration is timed as one untimed setpts +
 * execute, then reps timed ones (CUDA events on stream; the minimum counts);
 * each trial makes and destroys its own plan.  in / out are the transform's
 * input and a scratch output (type 1: c and f; type 2: f and c), device
 * memory; for the batch variant offsets, x, y, z, in and out are as for
 * nufft_batch_setpts / nufft_batch_execute.  best_ms / default_ms may be
 * NULL.  Returns NUFFT_OK, BAD_ARG, or CUDA when even the default fails.
 */
int nufft_tune(int type, int dim, const int64_t* nmodes, int isign, double eps, int prec, int64_t M, const void* x,
               const void* y, const void* z, const void* in, void* out, void* stream, int reps, nufft_opts* best,
               double* best_ms, double* default_ms);
int nufft_batch_tune(int type, int dim, int B, const int64_t* nmodes, int isign, double eps, int prec,
                     const int64_t* offsets, const void* x, const void* y, const void* z, const void* in, void* out,
                     void* stream, int reps, nufft_opts* best, double* best_ms, double* default_ms);

/* Host-only: the bin shapes the tuner tries for this dimension, precision and
 * kernel width, written to bins (3 ints each, at most max shapes); returns
 * how many there are, or NUFFT_ERR_BAD_ARG. */
int nufft_tune_candidates(int dim, int prec, int w, int* bins, int max);

/* ------------------------------------------------------------------ type 3
 * Type 3 (non-uniform to non-uniform, Sec. 1, Eq. (3)):
 *   f_k = sum_{j=1..M} c_j exp(i isign s_k.x_j),  k = 1..N,
 * with M source points x_j and N target frequencies s_k in R^d, both
 * arbitrary finite reals (no periodicity, no range limit), computed by the
 * algorithm of Sec. 3.3: translate both sets to their centres (Eq. (trans)),
 * dilate the sources by gamma_i and spread them onto a fine grid of
 * n_i = next235(max(2 sigma X_i S_i / pi + w, 2 w)) cells (Eq. (ng); X_i, S_i
 * the half-widths of the two bounding boxes), evaluate that grid as a
 * Fourier series at the rescaled targets with an inner type-2 plan (Eq.
 * (bkt3)), and divide by the kernel's Fourier transform at the targets.
 * The error is governed by eps as for types 1 and 2; the work grows with the
 * space-bandwidth product X_i S_i, which fixes n_i.
 *
 * Same conventions as above: device pointers on the plan's device, caller
 * keeps ownership, work enqueued on the plan's stream.  nufft3_setpts reads
 * both bounding boxes back to the host (it synchronises the stream) and
 * (re)allocates the grid, which may grow between calls.
 */
typedef struct nufft_plan3_s* nufft_plan3;

/* dim 1..3; isign +1 / -1; eps and prec as for nufft_makeplan; opts may be
 * NULL (defaults; bin_size, max_subprob, sparse_max, threads and upsampfac
 * apply to the spreading step and to the inner type-2 plan).  Returns NUFFT_OK,
 * NUFFT_WARN_EPS_TOO_SMALL, or an error (*out = NULL). */
int nufft3_makeplan(int dim, int isign, double eps, int prec, void* stream, const nufft_opts* opts,
                    nufft_plan3* out);
/* Sources x, y, z (M reals each; y NULL if dim < 2, z NULL if dim < 3) and
 * targets s, t, u (N reals each, likewise).  M = 0 or N = 0 is allowed.
 * Returns NUFFT_OK; NUFFT_ERR_BAD_ARG (M < 0, N < 0, NULL pointer);
 * NUFFT_ERR_OUT_OF_RANGE (a coordinate not finite); NUFFT_ERR_TOO_BIG (M or
 * N >= 2^31, or a space-bandwidth product whose grid is too large);
 * NUFFT_ERR_ALLOC / _CUDA / _CUFFT. */
int nufft3_setpts(nufft_plan3 plan, int64_t M, const void* x, const void* y, const void* z, int64_t N,
                  const void* s, const void* t, const void* u);
/* c: M input strengths, f: N outputs (complex, device).  NUFFT_ERR_NOT_SET
 * before nufft3_setpts. */
int nufft3_execute(nufft_plan3 plan, const void* c, void* f);
/* Kernel width, ES beta, and per dimension the fine grid n_i and dilation
 * gamma_i chosen by the last nufft3_setpts (any pointer may be NULL). */
int nufft3_plan_info(nufft_plan3 plan, int* w, double* beta, int64_t* n, double* gamma);
/* Synchronise the plan's stream; return any error recorded on the device. */
int nufft3_get_status(nufft_plan3 plan);
/* Free the plan (NULL is allowed).  Synchronises its stream first. */
int nufft3_destroy(nufft_plan3 plan);

/* ------------------------------------------------------------ unit peaks
 * Microbenchmarks of the units that bound the spread and interp kernels, for
 * their rooflines, run on the current device and enqueued on stream (a
 * cudaStream_t; the call synchronises it): out[0] FP32 FMA throughput in
 * TFLOP/s, out[1] FP64 FMA in TFLOP/s, out[2] special-function operations
 * (exp2 and reciprocal square root) in G ops/s, out[3] 32-bit shared-memory
 * atomic adds per second with conflict-free addresses.  Each figure is the
 * second of two launches of 8 blocks of 256 threads per SM running 8
 * independent chains per thread; about 3 ms in all.  n >= 4.  Returns
 * NUFFT_OK, NUFFT_ERR_BAD_ARG, NUFFT_ERR_ALLOC or NUFFT_ERR_CUDA. */
int nufft_measure_peaks(void* stream, double* out, int n);

/* ------------------------------------------------------------ no allocation
 * nufft_spread_noalloc -- the spreading step of a complex64 type-1 transform
 * onto the fine grid, for callers that cannot allocate device
 * memory: code running under another owner's memory pool or arena, latency-
 * critical paths that cannot take an allocation's implicit synchronisation,
 * and plugin hosts that forbid allocation.  The paper has no counterpart; it
 * is a deployment variant of the plan path above.
 *
 * Computes b = spread(x, y, z, c) on the fine grid n[0..dim-1] with kernel
 * width w and ES parameter beta (take them from nufft_choose_params), and
 * OVERWRITES grid (n_1 ... n_d complex64, dimension 1 fastest, device
 * memory) with it.  x, y, z: M float device arrays (y NULL if dim < 2, z NULL
 * if dim < 3); c: M complex64 device strengths.  Enqueued on stream (a
 * cudaStream_t, NULL = legacy default); asynchronous.
 *
 * It calls no cudaMalloc / cudaFree and no allocating library routine: its
 * binning arrays live in one static device array of 32 MiB that every GPU
 * loading the library holds until exit.  All calls share that array and it
 * keeps the previous call's contents (each call clears what must start at
 * zero), so calls whose device work overlaps race: serialise them.  The
 * array's device address is looked up (cudaGetSymbolAddress) during the
 * first call on each device; make that first call before any stream capture.
 *
 * Returns NUFFT_OK; NUFFT_ERR_BAD_ARG (dim, w outside [2, 16], n_i < 2w or
 * > 2^30, beta <= 0, M < 0, NULL pointer); NUFFT_ERR_TOO_BIG when M >= 2^31 - 1,
 * when the grid has 2^31 or more cells, or when M points and the bins of this
 * grid need more than the 32 MiB array (16 bytes per point plus about 16
 * bytes per bin: roughly two million points); NUFFT_ERR_CUDA when a launch
 * fails.
 */
int nufft_spread_noalloc(int dim, const int64_t* n, int w, double beta, int64_t M, const float* x,
                         const float* y, const float* z, const void* c, void* grid, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT_GB300_H */
