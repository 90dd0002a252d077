/*
 * epr.h -- C ABI of the GB300 fast eikonal phase retrieval library (libepr).
 *
 * The library implements the iterative solver of arXiv 2601.22793 ("Fast
 * Eikonal Phase Retrieval for High-Throughput Beamlines"): per projection and
 * per spectral line, the eikonal ray shift from the thickness map (Eq. 2 with
 * the single-material phase of Eqs. 6-7), the mass-conserving bilinear
 * redistribution of the object intensity onto the detector (Eq. 3 and its
 * "Discrete implementation" paragraph), the polychromatic sum (Eq. 5), the
 * exact adjoint by bilinear interpolation (Eq. 4), the FFT-diagonal
 * Paganin-type preconditioner, and the single-thickness update (Eq. 7 and the
 * "Iterative inversion" subsection).  The local O(L^2) closure (Eq. 1) is the
 * same loop with the transport replaced by its finite-difference stencil.
 *
 * Conventions shared by every entry point:
 *  - Maps are float32, row-major [ny][nx] (y = row), contiguous; a batch of B
 *    projections is [B][ny][nx]; per-line maps are [B][n_lines][ny][nx].
 *  - Thickness T is in metres; intensities are flat-field normalised (I_in = 1).
 *  - Array arguments may be device pointers or host pointers (pageable or
 *    pinned); the kind is detected with cudaPointerGetAttributes.  Host
 *    buffers are staged through plan-owned device memory with copies on the
 *    given stream; pinned host memory makes those copies asynchronous.
 *    The caller owns every array; the library never frees them.  Maps
 *    start on a 16-byte boundary (cudaMalloc and torch allocations do);
 *    an unaligned map is rejected with EPR_ERR_INVALID_ARG.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    asynchronous on it, except where an entry point says it synchronises.
 *  - Sizes: nx and ny of the form 2^a 3^b with a >= 3, 16 <= n <= 4096.
 *  - No exception, abort or device trap crosses the ABI.  Device-side
 *    failures (a full overflow list, a non-finite input) are reported through
 *    a status word read back by the solve calls.
 *  - A plan is not thread safe: calls on one plan must not overlap in time
 *    from several host threads.  Different plans are independent.
 */
#ifndef EPR_H
#define EPR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epr_plan_s* epr_plan_t;

typedef enum {
    EPR_OK = 0,
    EPR_ERR_INVALID_ARG = 1,      /* a NULL pointer, bad count or option */
    EPR_ERR_UNSUPPORTED_SIZE = 2, /* nx or ny not 2^a 3^b in [16, 4096]  */
    EPR_ERR_OOM = 3,              /* device allocation failed           */
    EPR_ERR_CUDA = 4,             /* a CUDA runtime or launch error     */
    EPR_ERR_NONFINITE = 5,        /* NaN or Inf in the data D of a solve */
    EPR_ERR_TIMEOUT = 6,          /* a bounded device wait on a bulk copy ran out */
    EPR_ERR_NOT_CONVERGED = 7,    /* reserved                           */
    EPR_ERR_SHIFT_OVERFLOW = 8    /* more large-shift sources than the overflow list holds */
} epr_status;

/* Forward models (Eq. 5: F_s is M_s for the non-local model, P_{m,s} for the
 * local closure of order m).  EPR_MODEL_NONLOCAL_WKB1 is the non-local model
 * to second order (the caption of the paper's non-local grid figure calls the
 * non-local model second order; the Methods define M_s as WKB0 transport):
 * P_s = M_s[I_s] - eps_s^2/(4 p^4) D_i(I_s D_i Q_s), the diffraction-pressure
 * term of Eq. 1 evaluated on the detector grid with the object intensity, as
 * the local closure of order 2 evaluates it. */
typedef enum {
    EPR_MODEL_NONLOCAL = 0,
    EPR_MODEL_LOCAL1 = 1,
    EPR_MODEL_LOCAL2 = 2,
    EPR_MODEL_NONLOCAL_WKB1 = 3
} epr_model;

/* Plan options (NULL = defaults). */
typedef struct {
    int max_shift_px;      /* fast-path reach of the splat, in pixels (default 4,
                              range 1..32).  Sources whose shift exceeds it in
                              either axis are not lost: they go through an
                              overflow list and are added with global atomics. */
    int deterministic;     /* 1 = accumulate the splat in int64 fixed point
                              (value * 2^40, round to nearest even): results are
                              bit-identical across runs.  0 (default) = the
                              tile accumulators hold round(value * 2^S) in
                              uint32, S = 32 - ceil(log2(2 (2 max_shift_px + 3)^2))
                              (24 at the default reach), and the long-shift
                              sources are added with float atomics. */
    int overflow_capacity; /* overflow entries per projection (default
                              max(4096, nx*ny/16)); a fuller list sets
                              EPR_ERR_SHIFT_OVERFLOW. */
    int use_graphs;        /* 1 = capture solver iterations in a CUDA graph
                              and replay it (default 1). */
    int autotune;          /* 1 = after the first solve, time the splat's tile
                              shapes, reach and blocks per SM, the column
                              pass's radix plan, column-tile width and blocks
                              per SM (float mode, no oversampling, uniform
                              spectrum) and
                              the one-line row passes' blocks per SM, on
                              that solve's result, and keep the fastest for
                              later solves (default 0).  The choices change
                              only the rounding of the float path
                              (fixed-point splat sums are unchanged).  The
                              tuning allocates a scratch map: the first solve
                              of a tuned plan must not be stream-captured. */
    int serial_launches;   /* 1 = launch every kernel only after its predecessor
                              has finished.  0 (default) = the solver kernels use
                              programmatic dependent launch: a kernel starts
                              its independent loads while its predecessor
                              drains, and waits on the device for the
                              predecessor's results.  Results are identical. */
    int oversample;        /* o >= 1 (0 = 1): solve on an internal grid of
                              (o ny) x (o nx) pixels of size pixel_m / o
                              ("Results": the paper's solves run on such grids).
                              nx, ny and pixel_m of the plan are the detector's;
                              o nx and o ny must be supported sizes.  With
                              o > 1 the data D of the solvers and the output P of
                              epr_forward are detector images (P is the mean of
                              each o x o block of the fine model), the thickness
                              T of the solvers and of epr_forward is the fine
                              map, epr_adjoint and epr_precondition act on fine
                              maps, and epr_vjp and the batch API are not
                              available (EPR_ERR_INVALID_ARG). */
    int fft_radix;         /* largest radix of the column transforms: 0 = the
                              default (8; with autotune the tuner may pick 16),
                              8, or 16 (radix-16 stages where the 2048-row
                              bulk-copy column pass has them).  Changes only
                              the rounding of the preconditioner. */
    int reserved[4];       /* must be zero */
} epr_options;

/* Solver options. */
typedef struct {
    int n_iter;       /* maximum iterations (>= 0) */
    double omega;     /* relaxation of the update (the paper uses 0.4 in its
                         multi-pixel stress test); > 0 */
    double tol;       /* stop a projection once kappa <= tol; 0 = run n_iter */
    double eps_I;     /* positivity floor of the updated line intensity,
                         relative to its spectral weight (default 1e-8) */
    int init;         /* 0 = start from the flat field (T := 0), 1 = start
                         from the caller's T */
} epr_solve_opts;

/* Per-projection results of a solve, filled after the call synchronises
 * its stream.  Each pointer is a HOST array of `batch` entries (or
 * batch * n_iter for the histories), or NULL to skip it. */
typedef struct {
    int* iters;          /* iterations run per projection */
    double* rho;         /* last |D - P| / |D| (residual before the last update) */
    double* kappa;       /* last |T' - T| / |T'| */
    double* rho_hist;    /* [batch][n_iter] */
    double* kappa_hist;  /* [batch][n_iter] */
    long long overflow_sources; /* out: sources that took the overflow path,
                                   summed over projections and iterations */
} epr_solve_info;

/* Create a plan for nx x ny projections with pixel size pixel_m and
 * propagation distance L_m, and n_lines spectral lines (1..16) with energies
 * (keV), refractive index decrements delta_s, absorption indices beta_s and
 * non-negative spectral weights (normalised to sum 1 by the library).
 * Derived per line: lambda = hc/E, k = 2 pi/lambda, mu = 2 k beta, shift
 * coefficient -L delta / p^2 (pixels per thickness step), Paganin symbol
 * mu / (mu + L delta |q|^2).  Host arrays.  *out is NULL on failure. */
epr_status epr_plan_create(epr_plan_t* out, int nx, int ny, double pixel_m, double L_m,
                           int n_lines, const double* energy_keV, const double* delta,
                           const double* beta, const double* weights, const epr_options* opt);

/* x-dependent effective spectrum (the paper's "Remark on spatially varying
 * spectra", with db_s(x) of Eq. 6 and f_s(x), gamma_s(x) of Eq. 7; the
 * paper's table format is in a supplement that is not available, so this
 * one is the library's own).  x is the detector column.  A table gives K
 * knot columns (pixel units, strictly ascending) and, per line s and knot k,
 * row-major [n_lines][K] host arrays of the spectral weight (> 0), delta and
 * beta (>= 0).  Each is interpolated linearly in x between knots and held
 * constant beyond the end knots; per column the weights are normalised to
 * sum 1 (f_s(x)), mu_s(x) = 2 k_s beta_s(x) with the plan's line energies,
 * and the shift is u_s = -(L delta_s(x) / p^2) G[T] (the table is held
 * constant under the derivative: slow variation).  The residual split falls
 * back to f_s(x), the update floors at eps_I f_s(x) and the projection weighs
 * each column by f_s(x) mu_s(x).  The preconditioner, which must be
 * FFT-diagonal, uses each line's column means of mu_s(x) and L delta_s(x).
 * K = 1 is a uniform spectrum. */
typedef struct {
    int n_knots;            /* K >= 1 */
    const double* x_knots;  /* [K] */
    const double* weights;  /* [n_lines][K] */
    const double* delta;    /* [n_lines][K] */
    const double* beta;     /* [n_lines][K] */
} epr_xspec;

/* Give the plan an x-dependent spectrum (table != NULL; host arrays, copied)
 * or return it to the uniform spectrum it was created with (NULL).  While a
 * table is set, epr_forward (model EPR_MODEL_NONLOCAL), epr_adjoint,
 * epr_precondition and epr_solve_nonlocal use it; the local solves, the
 * second-order model, epr_vjp and oversampled plans return
 * EPR_ERR_INVALID_ARG.  Synchronises the device.  EPR_ERR_INVALID_ARG for a
 * malformed table or a column without an absorbing line. */
epr_status epr_plan_set_xspec(epr_plan_t plan, const epr_xspec* table);

/* New L, delta_s and beta_s for an existing plan (host arrays of n_lines),
 * keeping its grid, energies, weights, options and workspace: the per-line
 * constants are derived again and nothing is allocated, so a calibration
 * loop can change them every step.  Cached solve graphs are dropped (work
 * already queued keeps the old constants).  EPR_ERR_INVALID_ARG for invalid
 * values, for values that leave no line both weighted and absorbing, or
 * while an x-dependent spectrum is set. */
epr_status epr_plan_set_params(epr_plan_t plan, double L_m, const double* delta, const double* beta);

/* Release the plan and its device workspace (synchronises the device). */
void epr_plan_destroy(epr_plan_t plan);

/* Forward model: P = sum_s F_s[f_s exp(-mu_s T)] for `batch` projections
 * (Eq. 5).  Ps (may be NULL) receives the per-line predictions
 * [batch][n_lines][ny][nx].  model is an epr_model (0..3).  Splat targets
 * outside the grid are dropped. */
epr_status epr_forward(epr_plan_t plan, const float* T, float* P, float* Ps, int batch,
                       int model, void* stream);

/* Adjoint of the non-local forward of line `line` at fixed T (Eq. 4):
 * g = M_line^T r, the bilinear interpolation of the detector map r at the
 * mapped coordinates; corners outside the grid read 0. */
epr_status epr_adjoint(epr_plan_t plan, const float* T, const float* r, float* g, int line,
                       int batch, void* stream);

/* Vector-Jacobian product of the non-local forward model (not in the paper:
 * the analytic transpose of Eq. 3 with the shift of Eq. 2 and the intensity
 * of Eq. 7, for calibration by gradient descent).  With gbar = dF/dP for
 * `batch` projections, writes Tbar = dF/dT and, when the host arrays are not
 * NULL, delta_bar[batch][n_lines] = dF/ddelta_s, beta_bar[batch][n_lines] =
 * dF/dbeta_s and L_bar[batch] = dF/dL.  Where a mapped point sits exactly on
 * a pixel boundary the transport is not differentiable; the right
 * derivative is returned.  Synchronises the stream when scalars or host
 * buffers are requested. */
epr_status epr_vjp(epr_plan_t plan, const float* T, const float* gbar, float* Tbar,
                   double* delta_bar, double* beta_bar, double* L_bar, int batch, void* stream);

/* Reverse mode through the unrolled non-local solve (not in the paper: the
 * calibration of L, delta_s and beta_s by gradient descent through a fixed
 * number of iterations of "Iteration structure").  Runs n_iter iterations of
 * epr_solve_nonlocal from T0 (NULL = the flat field, T := 0) on the data D,
 * without early stop, with relaxation omega and floor eps_I, and for
 * F = <Tbar, tau_N> returns dF/dT0, dF/dD and, per projection and line,
 * dF/ddelta_s, dF/dbeta_s and dF/dL.  Each iteration is recomputed from its
 * iterate and undone step by step: the projection and the floor of the
 * update (no gradient at the floor), the preconditioner (self-adjoint, and
 * its symbol's dependence on mu_s and L delta_s), the adjoint transport, the
 * residual split, the transport and the intensity and shift of each line.
 * The iterates are kept every checkpoint_every iterations (0 or 1 = every
 * one; m > 1 keeps n_iter / m + 1 of them and recomputes the others one
 * segment at a time, for less memory).  Where a mapped point sits exactly on
 * a pixel boundary the right derivative is taken.
 * D, T0, Tbar [batch][ny][nx] and the outputs T_out (tau_N), T0_bar, D_bar
 * (each may be NULL) are device memory; delta_bar, beta_bar [batch][n_lines]
 * and L_bar [batch] are host arrays (may be NULL; when any is given the call
 * synchronises the stream).  Needs mu_s > 0 and L delta_s > 0 for every line,
 * and a plan without oversampling or x-dependent spectrum
 * (EPR_ERR_INVALID_ARG otherwise).  The plan holds the iterates and about
 * 6 n_lines + 8 maps per projection of workspace, allocated on first use. */
epr_status epr_solve_vjp(epr_plan_t plan, const float* D, const float* T0, int batch, int n_iter,
                         double omega, double eps_I, int checkpoint_every, const float* Tbar,
                         float* T_out, float* T0_bar, float* D_bar, double* delta_bar,
                         double* beta_bar, double* L_bar, void* stream);

/* Paganin-type preconditioner of line `line`, in place: g <- Re F^-1[H_s F[g]],
 * periodic, no padding. */
epr_status epr_precondition(epr_plan_t plan, float* g, int line, int batch, void* stream);

/* Non-local solve ("Iterative inversion"): per iteration, forward splat of all
 * lines, residual D - P split across lines by P_s / P, adjoint gather,
 * preconditioner, relaxed update floored at eps_I f_s and least-squares
 * projection onto one thickness (Eq. 7).  T is the initial thickness when
 * opts->init = 1 and receives the result.  info may be NULL; when it is not,
 * the call synchronises the stream and fills it, and returns
 * EPR_ERR_NONFINITE when D holds a NaN or an infinity (the result is then
 * meaningless) and EPR_ERR_SHIFT_OVERFLOW when an overflow list overfilled.
 * Without info the same conditions are read by epr_check_device_status. */
epr_status epr_solve_nonlocal(epr_plan_t plan, const float* D, float* T, int batch,
                              const epr_solve_opts* opts, epr_solve_info* info, void* stream);

/* Non-local solve with the second-order model EPR_MODEL_NONLOCAL_WKB1 as
 * forward model: the iteration of epr_solve_nonlocal (same back-transport,
 * the transport's adjoint of Eq. 4), with the diffraction-pressure term of
 * Eq. 1 added to every line's prediction before the residual is formed.
 * Arguments, synchronisation and status codes as epr_solve_nonlocal. */
epr_status epr_solve_nonlocal_wkb1(epr_plan_t plan, const float* D, float* T, int batch,
                                   const epr_solve_opts* opts, epr_solve_info* info, void* stream);

/* Local solve: the same iteration with the local closure of order 1 or 2
 * (Eq. 1) as forward model and the identity as back-transport. */
epr_status epr_solve_local(epr_plan_t plan, const float* D, float* T, int batch, int order,
                           const epr_solve_opts* opts, epr_solve_info* info, void* stream);

/* The plan's kernel choices (not in the paper), as 9 host ints: splat tile
 * rows and columns, splat reach (px), column tile width (0 = the default
 * pass), largest radix of the column transforms (8 or 16), row-pass blocks
 * per SM (5 or 6), blocks per SM of the radix-16 column pass (4 or 5),
 * blocks per SM of the one-line residual splat (5 or 6; 6 exists for tiles
 * below 64 x 64 at reach 3 and 4) and whether the autotuner has run (1) or
 * the defaults hold (0). */
epr_status epr_plan_get_tuning(epr_plan_t plan, int* out);

/* Set those choices (the first 8 ints of the same layout), e.g. to reproduce
 * a tuned plan in another process.  The splat tile must fit the plan's
 * lines in shared memory; 5 column-pass blocks per SM need radix 16, 6 splat
 * blocks per SM a tile and reach that have the variant.  The
 * autotuner does not run over them.  EPR_ERR_INVALID_ARG for a value outside
 * the supported set. */
epr_status epr_plan_set_tuning(epr_plan_t plan, const int* in);

/* Synchronise `stream`, read and clear the plan's device error word:
 * EPR_ERR_NONFINITE if the data of a solve since the last check held a NaN or
 * an infinity, EPR_ERR_TIMEOUT if a bounded device wait on a bulk copy ran
 * out, EPR_ERR_SHIFT_OVERFLOW if a splat overfilled its overflow list (its
 * prediction then lacks those sources), else EPR_OK (first match wins). */
epr_status epr_check_device_status(epr_plan_t plan, void* stream);

/* Paganin-type preconditioner of one line without a plan and without any
 * device allocation: g <- Re F^-1[H F[g]] in place for `batch` maps of
 * nx x ny (the operation of epr_precondition, for a single line with the
 * given energy, delta and beta; L_m and pixel_m as for a plan).  The paper
 * has no counterpart: this serves callers that cannot let a library call
 * cudaMalloc (their device memory is owned by their own pool allocator or
 * fixed at start-up, or an allocation's possible device synchronisation is
 * not acceptable).  Scratch lives in a static device array of 16 MiB + 64 KiB
 * that every GPU loading the library holds until the process exits; it
 * bounds batch * nx * ny to 4 Mi pixels (e.g. one 2048 x 2048 map), and a
 * larger request returns EPR_ERR_UNSUPPORTED_SIZE.  Every call looks up the
 * array's device address with the current device (cudaGetSymbolAddress,
 * which allocates nothing); the first call on each device also sets the
 * kernels' shared-memory attributes once, so make that first call before any
 * stream capture (and, as for plans, not across a cudaDeviceReset, which
 * drops those attributes).  All calls share the array and nothing in it has
 * to start at zero (each call writes what it reads); calls whose work
 * overlaps on the GPU race.  g is device memory, 16-byte aligned. */
epr_status epr_precondition_noalloc(float* g, int nx, int ny, double pixel_m, double L_m,
                                    double energy_keV, double delta, double beta, int batch,
                                    void* stream);

/* Kernel kinds reported by epr_profile_read. */
typedef enum {
    EPR_KERNEL_SPLAT = 0,    /* forward transport (bilinear redistribution)   */
    EPR_KERNEL_ROW_FWD = 1,  /* split + adjoint gather + R2C row FFT          */
    EPR_KERNEL_COL = 2,      /* column FFT + Paganin filter + inverse         */
    EPR_KERNEL_ROW_INV = 3,  /* C2R row FFT + update + projection             */
    EPR_KERNEL_LOCAL = 4,    /* local closure stencil                         */
    EPR_KERNEL_OTHER = 5,    /* standalone gather, conversions                */
    EPR_KERNEL_KINDS = 6
} epr_kernel_kind;

/* Kernel timing for benchmarks.  While enabled, every kernel the plan
 * launches is bracketed by CUDA events recorded on the kernel's own stream;
 * a solve is then captured afresh into a CUDA graph that contains those
 * event records, so its kernels run back to back exactly as in an untimed
 * solve.  epr_profile_read synchronises the events and returns, per kind,
 * the number of launches and their summed duration in milliseconds since
 * the last read (the counters are then cleared).  Disabling drops pending
 * records. */
epr_status epr_profile_enable(epr_plan_t plan, int enable);
epr_status epr_profile_read(epr_plan_t plan, int* launches, double* total_ms);

/* Batched solve of projections of uneven sizes (not in the paper: serving
 * many projections of a scan at once).  A batch object holds the geometry
 * and spectrum shared by all projections and one plan per projection size,
 * created on first use.  Each size group is gathered into plan-owned device
 * memory and solved as one batched, graph-replayed solve on its own stream;
 * the groups run concurrently and join the caller's stream.  Every
 * projection stops on its own convergence test (opts->tol).  info, when
 * not NULL, is filled per projection in the order of `descs` (histories are
 * [n][opts->n_iter]); the call then synchronises. */
typedef struct epr_batch_s* epr_batch_t;

typedef struct {
    int nx, ny;        /* size of this projection (2^a 3^b, a >= 3, 16..4096) */
    const float* D;    /* measured data [ny][nx], device or host */
    float* T;          /* thickness [ny][nx]: initial value when opts->init = 1,
                          result on return; device or host */
} epr_batch_desc;

epr_status epr_batch_create(epr_batch_t* out, double pixel_m, double L_m, int n_lines,
                            const double* energy_keV, const double* delta, const double* beta,
                            const double* weights, const epr_options* opt);
void epr_batch_destroy(epr_batch_t batch);
epr_status epr_solve_nonlocal_batched(epr_batch_t batch, const epr_batch_desc* descs, int n,
                                      const epr_solve_opts* opts, epr_solve_info* info,
                                      void* stream);

/* Human-readable name of a status code (static string). */
const char* epr_status_string(epr_status s);

/* Number of kernels this library has launched in the process so far (graph
 * replays count every kernel node).  For launch accounting in benchmarks. */
long long epr_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* EPR_H */
