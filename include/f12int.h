/*
 * f12int.h -- C ABI of the GB300 library for the two-electron integrals that
 * explicitly correlated (F12) methods need with the range-separated
 * correlation factor of Silkowski, Lesiuk and Moszynski (arXiv:1412.5070).
 *
 * Conventions shared by every entry point
 *   - Every call returns an f12int_status; nothing throws across the ABI.
 *   - Host arrays passed in are borrowed for the duration of the call and
 *     copied; the caller keeps ownership.
 *   - Device pointers (suffix _dev) are owned by the caller, must be
 *     allocated on the context's device and must stay valid until the work
 *     queued on the given stream has finished.
 *   - Streams are raw cudaStream_t values passed as void*; NULL means the
 *     context's own stream.
 *   - Units are bohr.  Primitives are the unnormalised Cartesian Gaussians
 *     x_A^i y_A^k z_A^m exp(-a r_A^2) of Sec. 2.1 (Eq. basis); contraction
 *     coefficients multiply them as given.
 *   - Cartesian components of a shell of angular momentum l are ordered
 *     lexicographically: for l = 2 xx, xy, xz, yy, yz, zz; for l = 3 xxx,
 *     xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz.
 *   - A block of a shell quartet (ab|cd) is dense FP64, row-major
 *     [a][b][c][d] over those components.
 */
#ifndef F12INT_H
#define F12INT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct f12int_ctx f12int_ctx;

typedef enum {
  F12INT_OK = 0,
  F12INT_EINVAL = -1,    /* an argument is out of range or inconsistent        */
  F12INT_ENOMEM = -2,    /* device memory beyond the context's HBM budget       */
  F12INT_EDOMAIN = -3,   /* correlation-factor parameters outside the domain    */
  F12INT_ENOTREADY = -4, /* a basis or factor was not set before use            */
  F12INT_ETIMEOUT = -5,  /* a bounded wait ran out                              */
  F12INT_ECUDA = -6,     /* a CUDA runtime call failed                          */
  F12INT_EDEVICE = -7    /* a device-side check failed (status word)            */
} f12int_status;

/* Integral classes of Sec. 2.1: I1 (ab|1/r12|cd), Eq. I1; I2 (ab|f/r12|cd),
 * Eq. I2; I3 (ab|f|cd), Eq. I3; I4 (ab|f f'|cd), Eq. I4; I5 (ab|[f,T1]|cd),
 * Eq. I5, evaluated as 1/2 (lap_A - lap_B) I3 (Eq. I5_); I6 (ab|[[f,T1],f']|cd)
 * = (ab|f_r f'_r|cd), Eq. I6_. */
typedef enum { F12INT_I1 = 1, F12INT_I2, F12INT_I3, F12INT_I4, F12INT_I5, F12INT_I6 } f12int_class;

/* Range-separated correlation factor, Sec. 3.1, Eq. rs12 with the
 * Tang-Toennies damping of Eq. ttdamp:
 *   f(r) = (1 + r/2) exp(-mu r^2) + S_n(mu r^2) c0 r^rho exp(B r). */
typedef struct {
  double c0, rho, B, mu;
  int n;
} f12int_factor;

/* One term c r^a exp(b r - g r^2) of a correlation factor given as a sum of
 * terms: the general form the kernels of Eqs. k1-k6 are built from (the
 * factor of Eq. rs12 expands into five or more such terms).  It covers the
 * Ten-no factor exp(-w r) (one term, b = -w) and Gaussian-type geminals
 * sum_i c_i exp(-g_i r^2) (Sec. 1 and the factors cited there). */
typedef struct {
  double c, a, b, g;
} f12int_term;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context allocates (0 = no cap).  cuda_stream is the
 * default stream for the context (NULL = the legacy default stream).
 * On success *ctx receives a new context the caller must f12int_destroy. */
int f12int_create(f12int_ctx **ctx, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Release every device and host resource of the context. */
int f12int_destroy(f12int_ctx *ctx);

/* Upload a basis and build its shell-pair data on the device (Sec. 2.2,
 * Eqs. AB, Lambda, Erec0-Erect and the F = dE/dAB recursions).
 *   nshell        number of shells
 *   centers[3n]   shell centres (bohr)
 *   l[n]          angular momentum, 0..3
 *   nprim[n]      primitives per shell, >= 1
 *   exps[], coefs[]  primitive exponents (> 0) and contraction coefficients,
 *                 shell after shell (sum nprim entries each)
 * The pair data stays resident in device memory until the context is
 * destroyed.  *basis_id receives the handle used by the other calls.
 * Errors: F12INT_EINVAL for out-of-range input, F12INT_ENOMEM when the pair
 * data would exceed the budget. */
int f12int_set_basis(f12int_ctx *ctx, int nshell, const double *centers, const int *l,
                     const int *nprim, const double *exps, const double *coefs, int *basis_id);

/* Set the correlation factors f and f' (Eq. rs12; fprime = NULL means
 * f' = f).  Builds, on the host, the term lists of the kernels k1..k6
 * (Eqs. k1-k6) as sums of c x^a exp(b x - g x^2) and their radial
 * derivatives, and copies them to the device.
 * B may have either sign: B > 0 grows at long range, B < 0 decays (a
 * Ten-no-like tail; its term families, b < 0, are integrated by a
 * Gauss-Legendre quadrature in a second evaluation launch).
 * Errors: F12INT_EDOMAIN when mu <= 0, c0 < 0, n < 0 or n > 20, a value is
 * not finite, or rho + 2n + 2 <= 0 (the damped long-range term must be
 * integrable at r = 0, Sec. 3.1).
 * Classes: the auxiliary stage evaluates the term families x^a e^{bx - gx^2}
 * of x^2 k(x) through S(alpha, beta, gamma) (Eq. sila).  Families with a < -1
 * (a factor r^rho with rho <= -1, made integrable by its damping) are
 * evaluated together with the families of the same b, their singular terms
 * cancelled between them; a = -1 on its own is a finite part (Sec. 3.3.2).
 * A class is left out of an accepted factor, and every call for it (compute,
 * aux, submit) returns F12INT_EDOMAIN, when x^2 k(x) is not integrable at
 * r = 0, when a power below -1 is neither an integer nor a half-integer, or
 * when a family with b < 0 has such a power.  For f' = f and c0 > 0 the
 * lowest powers are rho + 2 (I3, I5), rho + 1 (I2), 2 rho + 2 (I4) and
 * 2 rho (I6): every class is served for rho > -1 (B >= 0) and, for smaller
 * rho, when 2 rho is an integer; with B < 0, 2 rho must be an integer.
 * Accuracy of hat g_n for the singular groups: 1e-10 relative for xi <= 2,
 * 1e-8 up to xi = 50. */
int f12int_set_factor(f12int_ctx *ctx, const f12int_factor *f, const f12int_factor *fprime);

/* Host-only view of the term lists that f12int_set_factor uploads: writes
 * x^{2l+2} (D_r^l k_cls)(x), D_r = x^-1 d/dx, for the kernel of class cls
 * (Eqs. k1-k6; class 5 uses k3) built from f and f' (fprime = NULL means
 * f' = f), evaluated from the generated families at x > 0.  Needs no GPU.
 * Errors: F12INT_EINVAL for cls, l (0..14) or x out of range,
 * F12INT_EDOMAIN as for f12int_set_factor. */
int f12int_kernel_radial(int cls, const f12int_factor *f, const f12int_factor *fprime, int l, double x,
                         double *value);

/* Set the correlation factors as sums of terms: f(r) = sum_{i<nf} f[i].c
 * r^{f[i].a} exp(f[i].b r - f[i].g r^2), and f' likewise from fprime/nfp
 * (fprime = NULL means f' = f).  Everything after the kernels' term lists is
 * as for f12int_set_factor, which this call replaces.
 * Arguments: host arrays, read during the call only; 1 <= nf, nfp <= 64.
 * Errors: F12INT_EINVAL for a NULL f or a count out of range; F12INT_EDOMAIN
 * when a value is not finite or some g < 0.
 * Classes: the rules of f12int_set_factor, and one more that the damping of
 * Eq. rs12 guarantees there: a class whose x^2 k(x) has a net x^-1 term at
 * r -> 0 (a kernel like r^-3, whose integrals diverge) is left out.  A
 * kernel holds at most 24 term families (distinct (b, g) and power
 * lattice): a Gaussian geminal of six terms fits every class (I4 and I6 have
 * one family per pair g_i + g_j), one of seven only I1-I3 and I5.  A family
 * polynomial longer than 48 terms makes the call return F12INT_EDOMAIN. */
int f12int_set_factor_terms(f12int_ctx *ctx, const f12int_term *f, int nf, const f12int_term *fprime, int nfp);

/* Host-only: which classes a factor pair serves, without a GPU or context.
 * flags[c] for c = 1..6 (flags[0] unused) receives 0 when class c would be
 * left out (its calls return F12INT_EDOMAIN), 1 when it is served by the
 * series and peak quadrature alone, 3 when some of its families also need
 * the quadrature launch (b < 0, or singular families).  fprime = NULL means
 * f' = f.  Errors as for f12int_set_factor / f12int_set_factor_terms. */
int f12int_factor_classes(const f12int_factor *f, const f12int_factor *fprime, int *flags);
int f12int_factor_classes_terms(const f12int_term *f, int nf, const f12int_term *fprime, int nfp, int *flags);

/* Host-only view of f12int_kernel_radial for factors given as terms (the
 * arguments of f12int_set_factor_terms).  Needs no GPU. */
int f12int_kernel_radial_terms(int cls, const f12int_term *f, int nf, const f12int_term *fprime, int nfp, int l,
                               double x, double *value);

/* Schwarz-type screening for class cls: bound(ab) = sqrt(max |(ab|k|ab)|)
 * over the diagonal block (the I3 diagonal for I5), times a growth factor
 * for kernels that grow with r12 (Eq. rs12 with B > 0; the diagonal samples
 * the kernel at short range only): estimate(ab|cd) = bound(ab) bound(cd)
 * max_w G(R + w) exp(-xi w^2) over w = 0, 0.5, .., 3 / sqrt(xi), with
 * G(x) = max(1, max_{1<=s<=x} |k(s)| / max_{1/2<=s<=3/2} |k(s)|), R the
 * distance between the centres of the two pairs' most diffuse primitive
 * pairs and xi = pq/(p+q) of those (G = 1 for I1); for I5 and I6 the
 * estimate carries a further factor 8.  Writes the canonical shell quartets whose estimate is >= thresh into
 * quartets_out[4*i]
 * (host memory, room for cap quartets) and their count into *n_out.
 * Canonical means a >= b, c >= d and (ab) >= (cd) for I1-I4 and I6; for I5
 * (no bra-ket symmetry, antisymmetric in a <-> b) it means a >= b, c >= d
 * with every (ab), (cd) combination.  If more than cap quartets survive,
 * *n_out holds the full count and nothing beyond cap is written.
 * The bound is rigorous for I1 (positive-definite kernel); for the F12
 * kernels the estimate is a heuristic. */
int f12int_screen(f12int_ctx *ctx, int basis_id, int cls, double thresh, int32_t *quartets_out,
                  int64_t cap, int64_t *n_out);

/* The screening estimate of f12int_screen for n given quartets (host
 * [n][4] shell indices) into est_out[n] (host).  The first call of a (basis,
 * class) computes its shell-pair bounds. */
int f12int_quartet_estimates(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets, int64_t n,
                             double *est_out);

/* The shell-pair bounds that f12int_screen multiplies: bounds_out[a*nshell
 * + b] = sqrt(max |(ab|k|ab)|) over the diagonal block of class cls (the I3
 * kernel for I5); host memory of nshell*nshell doubles.  Computed on the
 * device on first use for a (basis, class) and cached. */
int f12int_pair_bounds(f12int_ctx *ctx, int basis_id, int cls, double *bounds_out);

/* Compute the contracted blocks of class cls (Eq. ii for I1-I4 and I6,
 * Eq. I5byI3_ for I5) for n shell quartets.
 *   quartets_dev[4n]  shell indices (a, b, c, d), device memory
 *   offsets_dev[n]    element offset of each block in out_dev, device memory
 *   out_dev           output, device memory, FP64
 * The work runs on cuda_stream.  The call reads the quartet list back to
 * plan its launches (which waits for earlier work on that stream) and
 * returns when the blocks are written (it synchronises the stream); many
 * small requests are better served by f12int_submit.
 * Scratch memory is allocated by the context (bounded by its budget).
 * Errors: F12INT_ENOTREADY without basis or factor, F12INT_EINVAL for bad
 * arguments, F12INT_ENOMEM when scratch would exceed the budget. */
int f12int_compute_class(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev,
                         int64_t n, double *out_dev, const int64_t *offsets_dev, void *cuda_stream);

/* Mixed-precision variant of f12int_compute_class: quartets whose shell-pair
 * bound product (as in f12int_screen) is below fp32_below run the Hermite
 * recursion and the contraction in FP32 with FP32 accumulation; the
 * auxiliary functions g_n, the shell-pair data and every other quartet stay
 * FP64, and so do the quartets of total angular momentum <= 3 (<= 2 for I5),
 * whose one-lane-per-primitive-quartet FP64 contraction is faster than the
 * FP32 form of the general one.  fp32_below = 0 is f12int_compute_class.  Meant for quartets whose
 * blocks are small in absolute terms: the error is bounded by about 1e-7
 * times the magnitude of the terms an element sums, not relative to the
 * element.  The first call of a (basis, class) computes its shell-pair
 * bounds.  Errors as for f12int_compute_class; F12INT_EINVAL for a negative
 * or NaN fp32_below. */
int f12int_compute_class_mixed(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev,
                               int64_t n, double *out_dev, const int64_t *offsets_dev, double fp32_below,
                               void *cuda_stream);

/* Radial derivatives g_n = (Q^-1 d/dQ)^n B_i of the basic integral of
 * class cls at given xi = pq/(p+q) and D = |P - Q| (Sec. 2.3, Eq. bfinal;
 * Sec. 2.5), without the prefactor sqrt(pi^5/(p+q))/(pq):
 *   out_dev[i*(nmax+1) + n] = int_0^inf k(r) r (Q^-1 d/dQ)^n
 *                              [(e^{-xi (r-D)^2} - e^{-xi (r+D)^2}) / D] dr
 * for i < npts, n <= nmax (nmax <= 14).  xi_dev, D_dev, out_dev are
 * device arrays.  This is the auxiliary-function stage of compute_class,
 * exposed for testing. */
int f12int_aux(f12int_ctx *ctx, int cls, int64_t npts, const double *xi_dev, const double *D_dev,
               int nmax, double *out_dev, void *cuda_stream);

/* The blocks of f12int_compute_class, from a call that allocates no device
 * memory: every scratch buffer comes from one file-scope device array of
 * F12INT_STATIC_SCRATCH_BYTES (64 MiB) that each GPU which loads the library
 * holds until the process exits.  It is meant for callers that cannot call
 * cudaMalloc while they run, such as applications that reserve all device
 * memory up front for their own pool, or services in which the device-wide
 * synchronisation of an allocation would stall work on other streams.  The
 * paper has no counterpart: this is a deployment interface, not part of the
 * method.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (the call clears what must start at zero).  Calls whose
 *     work overlaps on the GPU (other streams, other contexts of the same
 *     device) race on it and must be serialised by the caller.
 *   - Primitive screening: the call uses the primitive-quartet screen of
 *     f12int_compute_class when that table exists for the (basis, class),
 *     i.e. after one allocating call of the class on the basis (or a
 *     f12int_submit of it); the blocks are then bitwise those of
 *     f12int_compute_class.  Without the table (building it allocates) every
 *     primitive quartet is evaluated: more work, and blocks that differ from
 *     f12int_compute_class's by the screened contributions only (below the
 *     absolute accuracy the FP64 tolerance asks of elements near 1e-12).
 *   - Limits: the list itself takes 40 bytes per quartet plus 8 bytes per
 *     contraction task, one task per range of ket components (quartets of
 *     high angular momentum, or with many primitive quartets, are split into
 *     several ranges, up to 100): about 1.4M quartets of one range each, far
 *     fewer when most are split.  Per shell quartet, its primitive quartets
 *     times the kernel's term families must fit in the rest (about 500k work
 *     items).  Every size check is made before any work is queued.
 *   - Errors: F12INT_EINVAL when the list or one shell quartet's primitive
 *     work does not fit in the array (nothing is then queued or written);
 *     the other errors as for f12int_compute_class. */
int f12int_compute_class_static(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev,
                                int64_t n, double *out_dev, const int64_t *offsets_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batched requests.  A request asks for the blocks of one or more classes over
 * one list of shell quartets of a basis (the integrals of
 * f12int_compute_class).  f12int_submit copies the request and queues it; a
 * worker thread of the context merges the pending requests of any bases into
 * batches and runs each batch as one replay of a captured CUDA graph on the
 * context's own batch stream.  The paper has no counterpart: this is the
 * scheduling layer for many small requests.
 */
typedef struct {
  int64_t n_quartets;          /* number of shell quartets (>= 0)                        */
  const int32_t *quartets;     /* host [n_quartets][4] shell indices; copied by submit   */
  uint32_t class_mask;         /* bit c-1 set: compute class c (1..6); at least one bit  */
  int precision;               /* 0: FP64; 1: mixed, as f12int_compute_class_mixed with
                                  the bound set by f12int_set_fp32_below                  */
  double schwarz_thresh;       /* > 0: quartets whose screening estimate (as in
                                  f12int_screen) is below it get zero blocks; 0: none     */
  double *out_dev;             /* device output, FP64, caller-owned; must stay valid and
                                  untouched until the request is done                    */
  const int64_t *offsets;      /* host [nclass][n_quartets] element offsets into out_dev,
                                  one row per requested class in increasing class order;
                                  copied by submit                                       */
} f12int_request;

/* Queue a request; *ticket identifies it in f12int_poll.  The first request
 * of a (basis, class) computes that class's primitive and shell-pair bounds
 * synchronously; the first request of the context allocates the batch
 * buffers (see f12int_batch_limits) and starts the worker.
 * Errors: F12INT_EINVAL for bad arguments (shell index out of range, empty or
 * unknown class mask, precision not 0 or 1), F12INT_ENOTREADY without basis or
 * factor, F12INT_ENOMEM when the request alone exceeds one batch (split it)
 * or when the first request of a (basis, class) would need more device
 * memory for that class's bounds than is free on the device at submit (or
 * than the context's budget leaves): admission by free device memory. */
int f12int_submit(f12int_ctx *ctx, int basis_id, const f12int_request *req, uint64_t *ticket);

/* Wait at most timeout_us microseconds (0: do not wait) for a request.
 * *done = 1 once it has finished; the call then returns the request's status
 * (F12INT_OK, or F12INT_EDEVICE if a device-side check of its batch failed)
 * and forgets the ticket.  While it is queued or running, *done = 0 and the
 * call returns F12INT_OK for timeout_us = 0 (a query) and F12INT_ETIMEOUT when
 * a wait of timeout_us > 0 ran out (the ticket stays valid).  F12INT_EINVAL
 * for an unknown or already reported ticket. */
int f12int_poll(f12int_ctx *ctx, uint64_t ticket, int64_t timeout_us, int *done);

/* Capacity of one batch, per class: max_quartets shell quartets and
 * max_items auxiliary work items (primitive quartets times the kernel's term
 * families); each class has its own item buffers (136 bytes per item).
 * Default 2^19 quartets; the default item capacity is set from free device
 * memory when the engine starts (the six classes' item buffers take at most
 * a quarter of it, 2^26 items per class at most).  Only before the first
 * f12int_submit. */
int f12int_batch_limits(f12int_ctx *ctx, int64_t max_quartets, int64_t max_items);

/* Pick each class's batch schedule by measurement: for every class in
 * class_mask, run the n sample quartets (host [n][4] shell indices of the
 * basis) alone through the batch path under each candidate -- the work
 * target of one contraction task (6.25e6, 1.5e7, 5e7, 2e8 flops) times the
 * grid of the persistent auxiliary-stage launch (full or half residency) --
 * and keep the fastest.  report (may be NULL) receives, per class c,
 * report[3(c-1)] the chosen target, [3(c-1)+1] the grid divisor and
 * [3(c-1)+2] the best time in seconds.  Needs an idle engine (no request
 * queued or running); allocates a temporary output. */
int f12int_batch_autotune(f12int_ctx *ctx, int basis_id, const int32_t *quartets, int64_t n,
                          uint32_t class_mask, double *report);

/* Screening estimate below which mixed requests (precision 1) run the
 * Hermite recursion and contraction in FP32 (default 1e-5, where the FP32
 * difference stayed below 4.1e-11 on a 40-atom f-shell sample; at 1e-4 it
 * reached 1.5e-10).  Applies to batches built after the call. */
int f12int_set_fp32_below(f12int_ctx *ctx, double bound);

/* stats[0] batches launched, stats[1] requests finished, stats[2] requests
 * waiting for a batch. */
int f12int_batch_stats(f12int_ctx *ctx, int64_t *stats);

/* Number of kernel launches the context has issued so far (monotonic). */
int64_t f12int_launch_count(const f12int_ctx *ctx);

/* Switch per-kernel timing on (on != 0) or off.  While on, the library
 * records CUDA events on the launching stream around every launch of the
 * auxiliary-function evaluation and of the contraction, and counts the
 * auxiliary stage's core multiply-adds (one per series term and polynomial
 * coefficient, one per quadrature node and coefficient).  Measurement aid;
 * the paper has no counterpart. */
int f12int_set_timing(f12int_ctx *ctx, int on);

/* Totals since the last reset, written to stats[0..5]:
 *   [0] milliseconds in auxiliary-evaluation launches, [1] their number,
 *   [2] milliseconds in contraction launches, [3] their number,
 *   [4] FP64 flops of the auxiliary stage's core multiply-adds (2 per FMA),
 *   [5] algorithmic FP64 flops of the Hermite recursion and contraction of
 *       the primitive quartets processed (2 C(L+4,4) + 2 nh(lab) nh(lcd) Ncd
 *       + 2 Nab nh(lab) Ncd per primitive quartet; bra step x4 and L+2 for I5).
 * reset != 0 clears them.  Synchronises the context's stream. */
int f12int_kernel_stats(f12int_ctx *ctx, int reset, double *stats);

/* Host-side planning time of f12int_compute_class calls since the last reset:
 * stats[0] milliseconds (wall clock, from the call's entry to its first
 * launch: reading the list, ordering the quartets, uploading the plan),
 * stats[1] the number of calls.  reset != 0 clears them.  Measurement aid;
 * the paper has no counterpart. */
int f12int_host_stats(f12int_ctx *ctx, int reset, double *stats);

/* Measured arithmetic peak of CUDA device `device`, in TFLOP/s, written to
 * *tflops: the denominators of the library's roofline figures.  kind 0: FP64
 * fused multiply-add (the DFMA pipe); 1, 2, 3: FP64 matrix multiply-accumulate
 * (mma.sync, shapes m8n8k4, m16n8k4, m16n8k16); 4: FP32 fused multiply-add.
 * Independent instruction chains on SMs x 8 blocks of 256 threads, one
 * warm-up launch, CUDA events around one launch of a few hundred ms; 2 flops
 * per FMA and 2 m n k per matrix instruction.  Allocates and frees a small
 * device buffer; needs no context.  Measurement aid; the paper has no
 * counterpart.  Errors: F12INT_EINVAL for a bad kind or device. */
int f12int_measure_peak(int device, int kind, double *tflops);

/* Cap on the length of the auxiliary stage's series (default and maximum 400
 * terms; the longest series of the supported range needs about 200).  An
 * item whose series has not converged at the cap sets bit 1 of the device
 * status word, which f12int_device_status and f12int_poll report as
 * F12INT_EDEVICE; no kernel faults or waits.  Lowering the cap is a way to
 * exercise that path in tests; 0 restores the default.  Takes effect for
 * later launches (the batch graph is captured again).  Errors: F12INT_EINVAL
 * for a negative cap.  Test aid; the paper has no counterpart. */
int f12int_set_series_cap(f12int_ctx *ctx, int kmax);

/* Read and clear the device status word (a device-side check failing sets
 * it).  Synchronises the context's stream.  Returns F12INT_OK or
 * F12INT_EDEVICE. */
int f12int_device_status(f12int_ctx *ctx);

/* Human-readable message for a status code (static storage). */
const char *f12int_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* F12INT_H */
