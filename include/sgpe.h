/*
 * sgpe.h -- C ABI of libsgpe: GB300 (sm_103a) kernels for the split-step
 * Crank-Nicolson time step of the three-component spin-1 Gross-Pitaevskii
 * equation with spin-orbit (SO) and Rabi coupling, in 1D and 2D, imaginary and
 * real time (arXiv:2009.13507, Eqs. (1)-(2), Sec. 3 and Appendix A).
 *
 * Conventions shared by every entry point
 *  - The wave function psi is a contiguous array [3][ny][nx] of interleaved
 *    complex numbers (re, im), x fastest; component index 0, 1, 2 holds the
 *    spin components +1, 0, -1 (the paper's CP(L,I,J), L = 1, 2, 3, Sec. 3).
 *    Element type: double (SGPE_C128, 16 bytes per complex), float
 *    (SGPE_C64, 8 bytes), or for SGPE_CDF four floats (re_hi, re_lo, im_hi,
 *    im_lo; 16 bytes) holding each real part as the unevaluated sum hi + lo.
 *    ny = 1 in 1D.
 *  - Grid: x_i = (i - nx/2) dx, y_k = (k - ny/2) dy (integer division), with
 *    homogeneous Dirichlet boundaries (psi = 0 outside the grid).
 *  - Memory: the caller owns every device buffer (state, workspace, Omega(t)
 *    tables) and keeps it alive while the context uses it; the library never
 *    allocates or frees device memory for the caller's data. The context itself
 *    (a small host object) is allocated by sgpe_init_grid and released by
 *    sgpe_destroy; sgpe_set_params also uploads a few small coefficient tables
 *    into the caller's workspace.
 *  - Streams: work is enqueued on the stream given to sgpe_init_grid and is
 *    asynchronous unless a function says it synchronises.
 *  - Errors: every function returns an sgpe_status; invalid arguments are
 *    rejected before anything is launched, and a textual reason is available
 *    from sgpe_last_error. Nothing traps or aborts.
 *  - Thread safety: one context must not be used from two host threads at once.
 */
#ifndef SGPE_H
#define SGPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgpe_ctx sgpe_ctx; /* opaque, library-owned host object */

typedef enum {
    SGPE_OK = 0,
    SGPE_EINVAL = 1,      /* bad argument (null pointer, size, parameter, alignment) */
    SGPE_ENOMEM = 2,      /* host allocation of the context failed */
    SGPE_ECUDA = 3,       /* a CUDA runtime call failed; see sgpe_last_error */
    SGPE_ENONFINITE = 4,  /* the norm of the state is not finite (NaN/Inf in psi) */
    SGPE_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    SGPE_ESTATE = 6,      /* call out of order (no buffers bound, no parameters set) */
    SGPE_EUNSUPPORTED = 7 /* size or option outside what the kernels support */
} sgpe_status;

/*
 * Arithmetic of the step:
 *  SGPE_C128  complex128 state, FP64 arithmetic (the plain FP64 form).
 *  SGPE_C64   complex64 state and sweeps, FP64 reductions (the precision form).
 *  SGPE_CDF   "double-float": every real number is a pair of FP32 numbers
 *             (about 48 significant bits), all step arithmetic on the FP32
 *             pipe, reductions and the renormalisation in FP64. Results agree
 *             with the complex128 form to ~1e-13; on GB300, whose FP64 rate is
 *             ~1/60 of its FP32 rate, it is the fast FP64-accurate form.
 *             sgpe_set_state / sgpe_get_state / sgpe_load_state take and
 *             return complex128; the bound psi buffer holds the pair layout.
 *             Not available for the batched and adjoint entry points
 *             (SGPE_EUNSUPPORTED).
 */
typedef enum { SGPE_C128 = 0, SGPE_C64 = 1, SGPE_CDF = 2 } sgpe_precision;

/*
 * Physical parameters (the inputs of the paper's Table 2 and Sec. 2).
 *  c0, c2   density-density and spin-exchange nonlinearities of Eqs. (1)-(2).
 *  so_type  OPT_SO (Sec. 3). 1D: 0 none, 1 gamma p_x Sigma_x, 2 gamma p_x Sigma_y,
 *           3 gamma p_x Sigma_z. 2D: 0 none, 1 Rashba (eta = 1), 2 Dresselhaus
 *           (eta = -1), 3 equal Rashba-Dresselhaus mixture (eta = 0), for the 2D
 *           coupling gamma (eta p_y Sigma_x - p_x Sigma_y) of Sec. 2.
 *  gamma    SO strength; omega: Rabi strength Omega (the coupling is Omega/sqrt2).
 *  wx, wy   trap V = (wx^2 x^2 + wy^2 y^2)/2 (the paper: wx = wy = 1); wy unused in 1D.
 *  dt       time step Delta (> 0).
 *  renorm   imaginary time only: 0 none, 1 Eq. (DJ2) (unit norm), 2 Eq. (DJ) (unit
 *           norm and magnetisation mag, |mag| < 1). Real time never renormalises.
 *  split    0: Lie splitting, the substeps treated successively with one full dt
 *           each (Sec. 3). 1: Strang splitting: SO, CALCNU and HERM with dt/2,
 *           Crank-Nicolson along x and y with dt, then HERM, CALCNU and SO with
 *           dt/2 (second order in dt where every substep is symmetric).
 *  so_mode  0: the SO substep by explicit Euler, Appendix A Eqs. (p1)-(p2) (in real
 *           time the norm grows by dt^2 |H_SO psi|^2 per step). 1: the SO operator
 *           treated by Crank-Nicolson like the kinetic term, (I + z/2 H_SO) psi' =
 *           (I - z/2 H_SO) psi along lines (2D: the part -gamma Sigma_y p_x along x
 *           lines, then gamma eta Sigma_x p_y along y lines; the reverse order in the
 *           second half of a Strang step): unitary in real time. Needs lines of at
 *           most 1024 points (SGPE_EUNSUPPORTED from sgpe_set_params otherwise).
 *           split or so_mode other than 0: unfused kernels (more launches per step);
 *           not available for the batched and adjoint entry points.
 */
typedef struct {
    double c0, c2;
    int so_type;
    double gamma, omega;
    double wx, wy;
    double dt;
    int renorm;
    double mag;
    int split;
    int so_mode;
} sgpe_params;

/* Indices of the observables written by sgpe_energy (SGPE_NOBS doubles). */
enum {
    SGPE_OBS_NP = 0,     /* N_{+1} = integral of rho_{+1} */
    SGPE_OBS_N0 = 1,     /* N_0 */
    SGPE_OBS_NM = 2,     /* N_{-1} */
    SGPE_OBS_N = 3,      /* N = N_{+1} + N_0 + N_{-1}, Eq. (noma) */
    SGPE_OBS_MAG = 4,    /* m = N_{+1} - N_{-1}, Eq. (noma) */
    SGPE_OBS_E = 5,      /* energy functional, Eq. (energy) */
    SGPE_OBS_MU = 6,     /* (E_kin + E_trap + E_SO + E_Rabi + 2 E_int) / N */
    SGPE_OBS_RMSP = 7,   /* sqrt(<r^2>) of rho_{+1} (LENGTH / RADIUS, Sec. 3) */
    SGPE_OBS_RMS0 = 8,
    SGPE_OBS_RMSM = 9,
    SGPE_OBS_RMS = 10,   /* of the total density */
    SGPE_OBS_EKIN = 11,  /* parts of E: kinetic, trap, c0/c2 interaction, Rabi, SO */
    SGPE_OBS_ETRAP = 12,
    SGPE_OBS_EINT = 13,
    SGPE_OBS_ERABI = 14,
    SGPE_OBS_ESO = 15,
    SGPE_NOBS = 16
};

/*
 * Create a context for one grid. dim = 1 or 2; nx >= 3 (and ny >= 3 in 2D, ny
 * ignored and taken as 1 in 1D); dx, dy > 0. nx, ny <= 4096 for SGPE_C128 and
 * SGPE_CDF and <= 8192 for SGPE_C64 (a whole grid line is staged in shared
 * memory).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream). The context
 * uses the CUDA device current at this call for all later calls.
 * Returns SGPE_EINVAL / SGPE_EUNSUPPORTED / SGPE_ENOMEM / SGPE_ECUDA.
 */
sgpe_status sgpe_init_grid(sgpe_ctx** out, int dim, int nx, int ny, double dx, double dy,
                           sgpe_precision prec, void* cuda_stream);

/* Bytes of device workspace the context needs (256-byte aligned start required). */
sgpe_status sgpe_workspace_bytes(const sgpe_ctx* ctx, size_t* bytes);

/*
 * Bind caller-owned device buffers: psi_dev ([3][ny][nx] complex, 16-byte
 * aligned, the state the step functions advance in place) and workspace_dev
 * (sgpe_workspace_bytes bytes, 256-byte aligned). Binding resets the pending
 * renormalisation scale to 1. Rebinding is allowed at any time between calls.
 */
sgpe_status sgpe_bind(sgpe_ctx* ctx, void* psi_dev, void* workspace_dev);

/*
 * Set the physical parameters and build the Crank-Nicolson coefficient tables
 * (the paper's COEF module) in the workspace with a small kernel. Requires
 * bound buffers. Returns SGPE_EINVAL for dt <= 0, a bad so_type, a bad renorm
 * mode or |mag| >= 1 with renorm = 2.
 */
sgpe_status sgpe_set_params(sgpe_ctx* ctx, const sgpe_params* p);

/*
 * Advance the bound state by nsteps imaginary-time steps (z = dt): per step
 * SO (Appendix A Eqs. (p1)-(p2)) -> CALCNU (diagonal trap and c0/c2 terms) ->
 * HERM (Appendix A Eqs. (nu), (11)) -> Crank-Nicolson along x -> along y (2D)
 * -> renormalisation by params.renorm (Eqs. (DJ2)/(DJ)). The renormalisation
 * scale of the last step is kept pending and folded into the next step's first
 * kernel; sgpe_normalize, sgpe_energy and sgpe_get_state apply it.
 * Asynchronous. nsteps >= 0.
 */
sgpe_status sgpe_step_imag(sgpe_ctx* ctx, int nsteps);

/*
 * Advance by nsteps real-time steps (z = i dt), same substeps, no
 * renormalisation. omega_dev (nullable) is a device array of at least nsteps
 * doubles giving Omega for each step; NULL uses params.omega. Asynchronous;
 * omega_dev must stay valid until the work completes.
 */
sgpe_status sgpe_step_real(sgpe_ctx* ctx, int nsteps, const double* omega_dev);

/*
 * Apply the pending renormalisation scale to the state, then write the norms
 * N_{+1}, N_0, N_{-1} of the state (grid sums times dx, or dx dy) to norms_out
 * (host, 3 doubles; nullable). Synchronises the stream. Returns
 * SGPE_ENONFINITE if a norm is NaN or infinite.
 */
sgpe_status sgpe_normalize(sgpe_ctx* ctx, double* norms_out);

/*
 * Apply the pending scale, then compute the SGPE_NOBS observables (indices
 * above; energy of Eq. (energy) with params.omega as the Rabi strength) into
 * out (host, SGPE_NOBS doubles). Synchronises the stream. SGPE_ENONFINITE if
 * the norm is not finite.
 */
sgpe_status sgpe_energy(sgpe_ctx* ctx, double* out);

/*
 * Copy a host state ([3][ny][nx] complex of the context's precision) into the
 * bound state (resets the pending scale), or copy the bound state (after
 * applying the pending scale) to host memory. Both synchronise the stream;
 * pinned host memory makes the copies faster but is not required.
 */
sgpe_status sgpe_set_state(sgpe_ctx* ctx, const void* host_psi);
sgpe_status sgpe_get_state(sgpe_ctx* ctx, void* host_psi);

/*
 * Copy a device state (caller-owned, must not overlap the bound state) into the
 * bound state and reset the pending scale. Layout [3][ny][nx] complex of the
 * context's precision: complex128 for SGPE_C128 and SGPE_CDF (split into the
 * pair layout by a kernel), complex64 for SGPE_C64. Asynchronous on the
 * context's stream.
 */
sgpe_status sgpe_load_state(sgpe_ctx* ctx, const void* psi_dev);

/*
 * Apply ONE substep to the bound state, for per-substep checks: which = 0 SO,
 * 1 CALCNU, 2 HERM, 3 Crank-Nicolson along x, 4 along y (2D only), 5
 * renormalisation by params.renorm, 6 the SO substep by Crank-Nicolson (x lines
 * then y lines; with the step's SO time step: dt, or dt/2 when params.split =
 * 1), 7 the same in the reverse order; imag selects z = dt (1) or z = i dt (0);
 * omega is the Rabi strength used by HERM. The pending scale is applied first.
 * Asynchronous.
 */
sgpe_status sgpe_substep(sgpe_ctx* ctx, int which, int imag, double omega);

/*
 * Measurement aid: run nsteps steps (imag = 1 imaginary, 0 real time, constant
 * Omega) with launches enqueued one by one and CUDA events recorded on the
 * context's stream around every kernel; writes the summed device time in ms of
 * each kernel kind to ms_out[0..3] (0 pointwise SO/CALCNU/HERM, 1 Crank-Nicolson
 * along x, 2 along y, 3 end-of-step norm reduction and renormalisation scale;
 * unused kinds 0) and the launch counts to launches_out[0..3]. On 2D grids
 * with lines of at most 1024 points (except double-float grids of 320..1024
 * points an axis, which launch all four kinds) kind 0 is a fused kernel (pending
 * scale, pointwise substeps and the x sweep), kind 1 has no launches, and the end
 * of step runs inside kinds 0 and 2 (kind 3 has no launches; one untimed
 * end-of-steps launch follows the last step). On complex64 2D grids with even
 * rows of 1025..2048 points kind 0 is the fused pointwise + x-sweep kernel too
 * and kind 1 has no launches (kind 3 only in imaginary time).
 * Advances the state exactly like the step functions. Synchronises the stream.
 */
sgpe_status sgpe_profile_steps(sgpe_ctx* ctx, int nsteps, int imag, double* ms_out, int* launches_out);

/*
 * Measurement aid (no counterpart in the paper): the FP64 fused multiply-add
 * rate of the current device in TFLOP/s (FMA = 2 flops), from a kernel of
 * independent FMA chains, 8 blocks of 256 threads per SM, timed with CUDA events
 * on cuda_stream (best of three timed launches after one warm-up, ~0.1 s).
 * It is the measured roof of the FP64 step kernels. Synchronises the stream.
 * Returns SGPE_EINVAL for a null output, SGPE_ECUDA if a CUDA call fails
 * (sgpe_last_error(NULL) then says which).
 */
sgpe_status sgpe_measure_fp64_rate(void* cuda_stream, double* tflops_out);

/*
 * Check aid (no counterpart in the paper): y[i] = exp(x[i]) - 1 by the FP32
 * routine of the complex64 CALCNU substep (Sec. 3's exp(-z mu) factor, applied
 * as u + (exp(-dt mu) - 1) u in imaginary time), for comparison with other
 * implementations. x_dev, y_dev: device arrays of n floats (caller-owned; they
 * may be the same array). Asynchronous on cuda_stream. Returns SGPE_EINVAL for
 * n < 0 or a null array with n > 0, SGPE_ECUDA if the launch fails.
 */
sgpe_status sgpe_eval_expm1f(void* cuda_stream, const float* x_dev, float* y_dev, int n);

/*
 * sgpe_observables_noalloc -- the SGPE_NOBS observables of sgpe_energy for a
 * state given by pointer, without a context and without any device memory from
 * the caller beyond its input and output. The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory (a host framework
 * that owns every allocation through its own pool, a plug-in that only sees the
 * buffers it is handed, a latency-critical loop that must not allocate).
 *  psi_dev  device state [3][ny][nx] complex of precision prec (16-byte aligned;
 *           for SGPE_CDF the pair layout of the bound state);
 *           it is read as it is (no pending renormalisation scale exists here).
 *  obs_dev  device output, SGPE_NOBS doubles (8-byte aligned), same indices as
 *           sgpe_energy; written asynchronously on cuda_stream.
 *  p        physics (c0, c2, so_type, gamma, omega, wx, wy used; dt ignored).
 * Scratch: a static 1 MiB device array inside the library, present on every
 * GPU that loads the library until the process exits. Grids needing more
 * reduction blocks than it holds (ceil(nx/32)*ceil(ny/4) > 11912, roughly more
 * than 1.5 million points) are rejected with SGPE_EUNSUPPORTED before anything
 * is launched; sgpe_last_error(NULL) then says why. No call allocates or frees
 * device memory. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the one array, so calls whose work overlaps on the
 * GPU (other streams, other host threads) race: order them on one stream.
 * The address is kept for the life of the process: after cudaDeviceReset the
 * library's module and its array are gone, so do not call this entry point on
 * that device again in the same process.
 * Returns SGPE_EINVAL for null or misaligned pointers or bad parameters,
 * SGPE_ECUDA if a CUDA call fails. Asynchronous: a state holding NaN or Inf is
 * not reported through the return code (that would need a synchronisation); it
 * shows up as a non-finite obs_dev[SGPE_OBS_N].
 */
sgpe_status sgpe_observables_noalloc(const void* psi_dev, int dim, int nx, int ny, double dx, double dy,
                                     sgpe_precision prec, const sgpe_params* p, double* obs_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Differentiation form: gradient of the final-density loss
 *     L = dx dy sum_r (rho_N(r) - rho_tgt(r))^2,  rho = sum_j |psi_j|^2,
 * after nsteps real-time steps (Sec. 3, z = i dt) from the bound state, with
 * respect to the per-step Rabi strengths Omega_n and the trap frequencies
 * (wx, wy) of V = (wx^2 x^2 + wy^2 y^2)/2, by a hand-written adjoint of the
 * discrete propagator (the exact reverse of every substep) with a state
 * checkpoint every checkpoint_every steps and recomputation in between.
 * ------------------------------------------------------------------------ */

/* Bytes of the caller-owned adjoint workspace for nsteps and checkpoint_every. */
sgpe_status sgpe_adjoint_workspace_bytes(const sgpe_ctx* ctx, int nsteps, int checkpoint_every, size_t* bytes);

/*
 * Run nsteps real-time steps from the bound state (which ends as psi_N; a
 * pending renormalisation scale is applied first), with Omega_n from
 * omega_dev (device, nsteps doubles) and the other parameters from
 * sgpe_set_params; then compute L and its gradient.
 *  rho_target_dev  device [ny][nx] doubles (the target density).
 *  adj_workspace   device, sgpe_adjoint_workspace_bytes bytes, 256-byte aligned.
 *  loss_out        host, 1 double (nullable); dw_out host, 2 doubles dL/dwx,
 *                  dL/dwy (nullable; dL/dwy = 0 in 1D).
 *  domega_dev      device, nsteps doubles: dL/dOmega_n.
 * Reductions are FP64 in both precisions. Synchronises the stream. This is
 * sgpe_adjoint_forward, the loss and its cotangent at psi_N, and
 * sgpe_adjoint_step, in one call.
 * SGPE_ESTATE without bound buffers or parameters; SGPE_EINVAL for bad sizes,
 * null or misaligned pointers.
 */
sgpe_status sgpe_adjoint_loss_grad(sgpe_ctx* ctx, int nsteps, const double* omega_dev, const double* rho_target_dev,
                                   int checkpoint_every, void* adj_workspace, double* loss_out, double* domega_dev,
                                   double* dw_out);

/*
 * The adjoint of nsteps real-time steps for any final-state cotangent, in two
 * calls. With the convention g = dL/dRe(psi) + i dL/dIm(psi) (PyTorch's), a
 * loss L(psi_N, Omega, wx, wy) defined by the caller is differentiated through
 * the discrete propagator psi_N = S_{N-1} ... S_0 psi_0, S_n the real-time split
 * step of Sec. 3 (SO -> CALCNU -> HERM with Omega_n -> CN along x -> along y),
 * by reversing every substep (Appendix A's substeps, transposed).
 *
 * sgpe_adjoint_forward: run nsteps real-time steps from the bound state psi_0
 * (which ends as psi_N; a pending renormalisation scale is applied first), with
 * Omega_n from omega_dev (device, nsteps doubles) and the other parameters from
 * sgpe_set_params, storing psi_n every checkpoint_every steps in adj_workspace
 * (device, sgpe_adjoint_workspace_bytes(nsteps, checkpoint_every) bytes, 256-byte
 * aligned). Synchronises the stream (it reads the Omega table).
 *
 * sgpe_adjoint_step: reverse the nsteps steps whose checkpoints adj_workspace
 * holds (same nsteps, checkpoint_every and Omega table as the forward call; the
 * parameters must not change in between). lambda_dev (device, [3][ny][nx]
 * complex of the context's precision, aligned to its element size) holds
 * dL/dpsi_N on entry and dL/dpsi_0 on exit. domega_dev (device, nsteps doubles)
 * receives the part of dL/dOmega_n that flows through the propagator, dw_out
 * (host, 2 doubles, nullable) that of (dL/dwx, dL/dwy) (dL/dwy = 0 in 1D). The
 * bound state is not touched; the reverse recomputes the steps between
 * checkpoints in the workspace. Reductions are FP64 in both precisions.
 * Synchronises the stream. SGPE_ESTATE when the workspace holds no forward pass
 * of these nsteps and checkpoint_every, or without bound buffers / parameters;
 * SGPE_EINVAL for bad sizes, null or misaligned pointers; SGPE_EUNSUPPORTED
 * for SGPE_CDF.
 */
sgpe_status sgpe_adjoint_forward(sgpe_ctx* ctx, int nsteps, const double* omega_dev, int checkpoint_every,
                                 void* adj_workspace);
sgpe_status sgpe_adjoint_step(sgpe_ctx* ctx, int nsteps, const double* omega_dev, int checkpoint_every,
                              void* adj_workspace, void* lambda_dev, double* domega_dev, double* dw_out);

/* ------------------------------------------------------------------------
 * Batched form: many independent grids advanced together by the split step of
 * Sec. 3 (same substeps and readings as a single grid), each with its own size
 * and physical parameters, in grouped launches (one per kernel kind and chunk
 * length, covering every instance) replayed from CUDA graphs.
 * ------------------------------------------------------------------------ */
typedef struct sgpe_batch sgpe_batch; /* opaque, library-owned host object */

/* One instance: dim 1 or 2, nx (and ny in 2D) in [3, 1024], dx (dy) > 0, params. */
typedef struct {
    int dim, nx, ny;
    double dx, dy;
    sgpe_params params;
} sgpe_instance;

/*
 * Create a batch of n instances (copied). All states share one precision.
 * Errors: SGPE_EINVAL (bad grid or parameters; sgpe_last_error(NULL) names the
 * instance), SGPE_EUNSUPPORTED (a line longer than 1024 points), SGPE_ENOMEM.
 */
sgpe_status sgpe_batch_create(sgpe_batch** out, int n, const sgpe_instance* inst, sgpe_precision prec,
                              void* cuda_stream);

/* Total complex elements of the batch state and bytes of its workspace. */
sgpe_status sgpe_batch_sizes(const sgpe_batch* b, size_t* state_elems, size_t* workspace_bytes);

/* Element offset of each instance's [3][ny][nx] state in the batch state (n entries). */
sgpe_status sgpe_batch_offsets(const sgpe_batch* b, size_t* offsets);

/*
 * Bind the caller-owned batch state (state_elems complex elements, 16-byte
 * aligned) and workspace (256-byte aligned); uploads the work lists and builds
 * every instance's Crank-Nicolson tables. Synchronises the stream.
 */
sgpe_status sgpe_batch_bind(sgpe_batch* b, void* psi_dev, void* workspace_dev);

/* Copy a device batch state (same layout) into the bound state; resets the pending scales. Async. */
sgpe_status sgpe_batch_load_state(sgpe_batch* b, const void* psi_dev);

/* nsteps imaginary-time (with each instance's renorm) or real-time steps of every instance. Async. */
sgpe_status sgpe_batch_step_imag(sgpe_batch* b, int nsteps);
sgpe_status sgpe_batch_step_real(sgpe_batch* b, int nsteps);

/*
 * Apply the pending scales, then write each instance's SGPE_NOBS observables
 * to out[i * SGPE_NOBS ...] (host, n * SGPE_NOBS doubles). Synchronises.
 * SGPE_ENONFINITE if an instance's norm is not finite.
 */
sgpe_status sgpe_batch_energy(sgpe_batch* b, double* out);

/*
 * Choose the launch shape by timing nsteps imaginary-time steps per candidate
 * with CUDA events: the x part (0: pointwise substeps and x sweep fused, one
 * 256-thread block per row, the default; 1, 2 or 4: warps per block of a
 * separate x sweep after a pointwise kernel) and the warps per block of the y
 * sweep (1, 2 or 4). Writes the choice to choice[0..1] (nullable). Advances the
 * bound state by 12 * (nsteps + 1) steps: tune before loading the state to be
 * advanced. Synchronises.
 */
sgpe_status sgpe_batch_autotune(sgpe_batch* b, int nsteps, int* choice);

/* Set the launch shape directly (x in {0, 1, 2, 4}, y in {1, 2, 4}, as chosen by
 * sgpe_batch_autotune); SGPE_EINVAL otherwise. Results do not depend on it
 * beyond rounding. */
sgpe_status sgpe_batch_set_tiles(sgpe_batch* b, int x, int y);

/* Kernel launches per batched step; last error of a batch; release (not the buffers). */
int sgpe_batch_launches_per_step(const sgpe_batch* b);
const char* sgpe_batch_last_error(const sgpe_batch* b);
sgpe_status sgpe_batch_destroy(sgpe_batch* b);

/*
 * Number of kernel launches one imaginary-time step enqueues (for launch
 * accounting): 2 on 2D grids with lines of at most 1024 points whose step needs
 * no finalize launch (the register path; the tiled complex64 path of grids of
 * 129..1024 points an axis), plus one end-of-steps launch per sgpe_step_imag /
 * sgpe_step_real call; 3 on complex64 grids with even rows of 1025..2048 points
 * (fused pointwise + x sweep, row-tiled y sweep, finalize) and 4 on other 2D
 * paths (double-float tiled grids, longer lines); 0 on 1D grids whose whole step
 * loop is one launch per call (lines of at most 1024 points in SGPE_C64 and
 * SGPE_CDF, at most 256 in SGPE_C128), 3 on other 1D grids.
 */
int sgpe_launches_per_step(const sgpe_ctx* ctx);

/* Last error message of this context (never NULL; "" when there is none). With
 * ctx = NULL: the message of the last failed sgpe_init_grid on this host thread. */
const char* sgpe_last_error(const sgpe_ctx* ctx);

/* Release the context (not the caller's buffers). NULL is accepted. */
sgpe_status sgpe_destroy(sgpe_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SGPE_H */
