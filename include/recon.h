/*
 * recon.h -- C ABI of librecon: one-step iterative estimation of effective
 * atomic number (Z) and relative electron density (rho_e) maps from
 * dual-energy CT with multi-domain gradient-L0 regularisation
 * (Wang et al., "One-step Iterative Estimation of Effective Atomic Number
 * and Electron Density for Dual Energy CT", arXiv 2308.01290).
 *
 * The library runs Algorithm 1 of Sec. II-D on the GPU: per iteration the
 * hard threshold of the auxiliary gradients of f1, f2, rho_e and Z^m
 * (eq. sol_hv), the FFT-diagonalised updates of f1, f2 and rho_e, and the
 * Z^m quadratic update (a preconditioned CG solve), followed by the beta
 * continuation.  Inputs are either reconstructed mu images at the low and
 * high energy (the paper's input, Sec. III) or -log sinograms of a fan-beam
 * scan, which the library reconstructs by FBP first.
 *
 * Conventions, for every function below:
 *  - return 0 (RECON_OK) on success, a negative RECON_E* code otherwise; no
 *    C++ exception crosses this boundary; recon_last_error() gives a message;
 *  - images are row-major float32, ny rows of nx values, concatenated slice
 *    after slice (no padding); sinograms are n_views rows of n_bins values;
 *  - pointers marked "device" are CUDA device pointers on the current
 *    device, "host" are host pointers; the caller owns every buffer passed
 *    in and the library only borrows it for the duration of the call (for
 *    device buffers: until the work queued on the handle's stream finishes);
 *  - attenuation images are in 1/mm; energies in keV;
 *  - a handle is not thread-safe; distinct handles may be used from
 *    different threads; all work of a handle is queued on its CUDA stream.
 */
#ifndef RECON_H
#define RECON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RECON_OK 0
#define RECON_EINVAL (-1)   /* bad argument (sizes, geometry, parameters) */
#define RECON_ENOMEM (-2)   /* device or host allocation failed */
#define RECON_ECUDA (-3)    /* a CUDA call failed */
#define RECON_ETIMEOUT (-4) /* a bounded device wait expired */
#define RECON_ENAN (-5)     /* non-finite values in inputs or results */
#define RECON_EBUDGET (-6)  /* request exceeds the configured memory budget */
#define RECON_ESTATE (-7)   /* call out of order (e.g. step before set_data) */

#define RECON_MAX_FILTERS 4
#define RECON_MAX_SIDE 2048

/* Scan and image geometry.  Image: nx x ny pixels of pixel_mm centred on the
 * isocentre (row j at y = (j - (ny-1)/2) pixel_mm).  Fan beam: source at
 * sid_mm (cos t, sin t), t = start_rad + arc_rad k / n_views; flat detector
 * at sdd_mm from the source, bin b centred at (b - (n_bins-1)/2) bin_mm.
 * n_views = 0 means the inputs are images, not sinograms. */
typedef struct recon_geometry {
    int32_t nx, ny;
    double pixel_mm;
    int32_t n_views, n_bins;
    double sid_mm, sdd_mm, bin_mm;
    double start_rad, arc_rad;
} recon_geometry;

typedef struct recon_filter {
    double Z, rhoe, thickness_mm;
} recon_filter;

/* One energy arm.  kind 0: monoenergetic at kev.  kind 1: Kramers spectrum
 * (kvp - E)/E on 1 keV bins E = 10 .. kvp-1 keV, filtered by the listed
 * filters through the attenuation model, photon-counting detection. */
typedef struct recon_spectrum {
    int32_t kind;
    int32_t n_filters;
    double kev;
    double kvp;
    recon_filter filters[RECON_MAX_FILTERS];
} recon_spectrum;

/* Parameters of Algorithm 1.  The paper prints none of lambda, beta0,
 * beta_max, tau, kappa ("experimentally optimized", Sec. IV);
 * recon_default_params() fills the values this library was validated with. */
typedef struct recon_params {
    recon_spectrum low, high;        /* acquisition arms E_L, E_H */
    double e1_kev, e2_kev;           /* synthesis energies (50, 200 keV, Sec. II-A) */
    double basis_z[2], basis_rhoe[2];/* basis materials 1, 2 (Z, rho_e) */
    double lambda;                   /* L0 weight (normalised units) */
    double beta0, beta_max, tau;     /* beta schedule, beta~ = tau beta */
    double kappa;                    /* <= 0: (beta_max/beta0)^(1/iters) */
    int32_t iters;                   /* iterations of Algorithm 1 */
    int32_t precision;               /* 1: FP32 maps + FP64 reductions/Newton; 0: FP64 */
    int32_t order;                   /* 0: f1,f2 Jacobi as printed; 1: Gauss-Seidel */
    int32_t cg_max_iters;            /* cap of the Z^m PCG per iteration */
    double cg_tol;                   /* relative residual of the Z^m PCG */
    double z_clip_max;               /* initial Z^m clipped to Z <= z_clip_max */
    double rho_air;                  /* initial Z^m set to water where rho_e < rho_air */
    int32_t pcg_kernel;              /* Z^m solve.  0: multigrid-preconditioned PCG on slices whose sides
                                        halve down to a small grid (below), FFT-preconditioned elsewhere;
                                        2: FFT-preconditioned PCG on every slice; 3: as 0, with every
                                        FP32 strip level on the ghost-column strip kernels, which the
                                        band kernels match bit for bit (a check; slower; 1 is refused) */
    int32_t domain;                  /* data terms of the arms: 0 on the image pair (Sec. II-B, as printed);
                                        1 on the sinograms through the projector, linear model (below);
                                        2 on the sinograms, polyenergetic model by Gauss-Newton (below) */
} recon_params;

/* Preconditioners of the Z^m PCG (Alg. 1, Z^m step: [diag(a^2) + beta~ L] z =
 * rhs, L = dx'dx + dy'dy periodic).  Both stop at the relative residual
 * cg_tol.  FFT: D^-1/2 (mean(a^2) + beta~ L)^-1 D^-1/2 with D = diag((a^2 +
 * 4 beta~) / (mean(a^2) + 4 beta~)), applied by real FFTs.  Multigrid: one
 * V-cycle, two damped Jacobi steps (weight 0.8) before and after the coarse
 * correction on every level, grids of half the sides (residual and a^2 restricted as
 * 2x2 means, corrections prolonged piecewise constant, beta~/4 per level),
 * an exact solve on the coarsest grid (its operator inverted once per Z^m
 * solve).  A slice takes the multigrid cycle
 * (pcg_kernel 0) when it has more than 4096 pixels and both sides stay
 * even while it halves down to at most 4096 pixels and on to at most 64; the
 * choice is per slice, so a slice gives the same result alone and in a
 * batch. */

/* domain = 1 (sinogram-domain data terms).  The paper fits the reconstructed
 * image pair; with sinograms s_L, s_H as data, the basis-fidelity terms of
 * eq. obj_unconstraint become, per arm i,
 *     (1/gamma) || A (f1 mu1(E_i) + f2 mu2(E_i)) - s_i / S ||^2,
 * A the Joseph projector of recon_project, S the water electron density
 * (mu in 1/mm = S mu_hat), gamma = ||A 1||^2 / (nx ny).  The model-
 * consistency terms, the L0 relaxation and the rho_e and Z^m steps are
 * unchanged; each f update solves its normal equations by conjugate
 * gradients (warm start, cap cg_max_iters, relative residual cg_tol) with
 * the FFT preconditioner (sum_i mu_k(E_i)^2 + sum_j b_kj^2 + beta K)^-1.
 * Requires sinogram inputs (n_views > 0), the same geometry for every slice
 * of a batch, precision 1 and order 0.  A^T adds with atomics, so results
 * may differ in the last bits between runs.  The solve starts from the FBP
 * image pair; recon_stats.fid_low/fid_high are 0 in this mode.
 *
 * domain = 2 (polyenergetic sinogram fidelity, linearised by Gauss-Newton).
 * With polyenergetic arms the -log sinogram of a ray is the nonlinear
 *     h_i(l1, l2) = -ln sum_b w_ib exp(-S (mu1(E_b) l1 + mu2(E_b) l2)) / S
 * of the basis line integrals l_k = A f_k (w_ib the arm's normalised
 * detected spectrum; two basis materials span the photoelectric / Compton
 * model at every energy, Sec. II-B).  Each iteration linearises the data term
 * (1/gamma) sum_i ||h_i(A f1, A f2) - s_i / S||^2 at the iterate: with
 * J_ik = dh_i/dl_k (the spectrum reweighted by the ray's attenuation),
 * W_kl = sum_i J_ik J_il and d_i = s_i / S - h_i + J_i1 l1 + J_i2 l2, the f_k
 * normal equations are those of domain 1 with A^T diag(W_kk) A / gamma in
 * place of sum_i mu_k(E_i)^2 A^T A / gamma and A^T (sum_i J_ik d_i - W_ko l_o)
 * / gamma as the data image.  With monoenergetic arms this is domain 1.  Same
 * requirements as domain 1, and the same spectra and basis materials for every
 * slice of a batch. */

/* Per-slice statistics of the last iteration run by recon_step.  The
 * objective terms are those of eq. obj_unconstraint at the iterate the
 * iteration started from, with its own thresholded gradients. */
typedef struct recon_stats {
    int32_t k;                 /* iterations done */
    int32_t cg_iters;          /* PCG steps of the last Z^m solve */
    double beta;               /* beta of the last iteration */
    double fid_low, fid_high;  /* ||f1 mu1 + f2 mu2 - mu||^2 at E_L, E_H */
    double model_e1, model_e2; /* model-consistency terms at E1, E2 */
    double relax;              /* beta sum_g ||d g - (h_g, v_g)||^2 */
    double l0;                 /* lambda sum_g C(h_g, v_g) */
    int64_t nnz[4];            /* C(h_g, v_g) for f1, f2, rho_e, Z^m */
    double cg_rel_residual;    /* final relative residual of the Z^m PCG */
} recon_stats;

typedef struct recon_ctx recon_ctx;

/* Fill p with the library defaults: mono 60/90 keV arms, E1/E2 = 50/200 keV,
 * bone-like (13, 1.7) and water (7.45, 1.0) bases, lambda 1e-2,
 * beta0 = 2 lambda, beta_max 1e5, tau 1, iters 50, precision 1, order 0,
 * cg_max_iters 64, cg_tol 1e-6, z_clip_max 30, rho_air 0.1, pcg_kernel 0, domain 0. */
int recon_default_params(recon_params* p);

/* Create a handle for one slice (recon_init) or a batch of n slices of
 * possibly different sizes and parameters (recon_init_batch; geoms and
 * params are host arrays of n entries; every entry must have the same
 * precision).  stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates all device memory of the solve up front.  Errors: EINVAL for
 * sizes outside [1, RECON_MAX_SIDE] or sizes whose prime factors are not all
 * in {2, 3, 5, 7}, ENOMEM, ECUDA. */
int recon_init(const recon_geometry* geom, const recon_params* params, void* stream, recon_ctx** out);
int recon_init_batch(int32_t n, const recon_geometry* geoms, const recon_params* params, void* stream,
                     recon_ctx** out);

/* Load the inputs of every slice and run the initialisation of Algorithm 1
 * (Cramer decomposition, synthesis, closed-form rho_e and Z^m).  low/high:
 * mu images (1/mm) when the geometry has n_views = 0, else -log sinograms
 * which are reconstructed by FBP; host or device (on_device = 1) buffers.
 * Host sinograms are copied one FBP group (up to 8 slices of one geometry)
 * at a time on a copy stream of the handle, beside the FBP of the groups
 * before.  Reads of host buffers are asynchronous for pinned memory (keep it
 * unchanged until recon_step or recon_sync returns) and finish before the
 * call returns for pageable memory.  Resets the iteration counter and
 * beta. */
int recon_set_data(recon_ctx* ctx, const float* low, const float* high, int on_device);

/* Run n_iters iterations of Algorithm 1 on every slice that has not yet done
 * its params.iters iterations (slices that finish stop early).  stats: NULL
 * or a host array of one recon_stats per slice (computing them adds
 * reductions).  Resumable: successive calls continue the same solve. */
int recon_step(recon_ctx* ctx, int32_t n_iters, recon_stats* stats);

/* Copy results out: Z = Z_w (Z^m/Z_w^m)^(1/m) by FP64 Newton (1 where
 * Z^m <= 0), rho_e, f1, f2; any pointer may be NULL; host or device. */
int recon_get(recon_ctx* ctx, float* Z, float* rhoe, float* f1, float* f2, int on_device);

/* recon_get into host buffers without waiting for the copies: the maps are
 * extracted on the handle's stream into output staging of the handle's own
 * (two unpadded float maps, allocated on the first call) and copied to the
 * host, one group of up to 8 slices at a time, on a device-to-host stream of
 * the handle.  The next recon_set_data and recon_step may run while the
 * copies proceed, so a stream of volumes overlaps each volume's maps going
 * out with the next one's work.  The host buffers (pinned memory, for the
 * copies to overlap) must stay valid, and are not complete, until
 * recon_sync returns; a later recon_get_async into the same buffers is
 * ordered after the earlier copies.  Errors: RECON_EINVAL (null handle),
 * RECON_ESTATE (before recon_set_data), RECON_ENOMEM / RECON_ECUDA. */
int recon_get_async(recon_ctx* ctx, float* Z, float* rhoe, float* f1, float* f2);

/* Blocks until the handle's queued work is done, including host copies
 * started by recon_set_data and recon_get_async. */
int recon_sync(recon_ctx* ctx);

/* Outputs of the comparison the paper's Sec. III makes (they do not change
 * the solve's state):
 * recon_direct: Z and rho_e of the two-step image-based method -- the
 *   decomposition of the loaded image pair (eq. lac_EL/EH), the synthesis at
 *   E1, E2 (eq. mac_E1/E2) and the closed forms eq. rho_e, eq. Z_m with no
 *   regularisation, i.e. the maps of iteration 0 of Algorithm 1.  With the
 *   sinogram-domain data terms (domain 1 or 2) the pair is the FBP of the
 *   staged sinograms, formed again by this call.  Z, rho_e:
 *   caller-owned buffers of the total pixel count (slices unpadded, in order),
 *   host or device as on_device says.  RECON_ESTATE before recon_set_data.
 * recon_mono: monoenergetic images at n_e energies kev[0..n_e-1] (keV > 0,
 *   1 <= n_e <= 16), mu(E) = S (f1 mu_1(E) + f2 mu_2(E)) in
 *   1/mm from the current basis fractions (eq. mac_E1/E2 at E).  out holds
 *   n_e blocks of the total pixel count, energy-major.  The slices must share
 *   their basis materials (RECON_EINVAL otherwise). */
int recon_direct(recon_ctx* ctx, float* Z, float* rhoe, int on_device);
int recon_mono(recon_ctx* ctx, int32_t n_e, const double* kev, float* out, int on_device);

/* Image-quality metrics of Sec. III for n slices of nx x ny pixels (both at
 * least 11): out[3 s + 0..2] = PSNR, NMAD and SSIM of slice s of x against
 * slice s of ref.  x, ref: device, n * nx * ny floats, slice-major; mask:
 * device, n * nx * ny bytes (nonzero: pixel counted by PSNR and NMAD) or NULL
 * for every pixel; out: host, 3 n doubles.  The paper prints no definitions;
 * the library takes PSNR = 10 log10(max|ref|^2 / MSE), NMAD = sum|x - ref| /
 * sum|ref|, both over the mask, and SSIM (Wang et al. 2004) as the mean over
 * the pixels whose 11 x 11 Gaussian window (sigma 1.5) fits in the slice,
 * with C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max(ref) - min(ref).  Scratch
 * is allocated on the stream (stream-ordered); the call returns once out is
 * written. */
int recon_iqa(int32_t n, int32_t nx, int32_t ny, const float* x, const float* ref, const uint8_t* mask,
              double* out, void* stream);

void recon_destroy(recon_ctx* ctx);

/* One-shot solve of one slice with default parameters (lambda, beta0 = beta,
 * iters overridden): init + set_data + step + get + destroy.  lowE/highE are
 * host images or sinograms (see recon_set_data); Z_out and rhoe_out host. */
int recon_solve(const float* lowE, const float* highE, const recon_geometry* geom, double lambda, double beta,
                int32_t iters, float* Z_out, float* rhoe_out);

const char* recon_strerror(int code);
const char* recon_last_error(void);

/* ---- serving: continuous batching of independent slice solves ----
 *
 * A server holds max_slots solve slots on the device, each sized for images
 * up to max_nx x max_ny (and sinograms up to max_views x max_bins).
 * recon_submit queues a request (its host inputs are copied, so the caller's
 * buffers are free on return).  recon_server_step admits queued requests into
 * free slots while the summed device footprint of the in-flight solves stays
 * within hbm_budget_bytes, loads them (FBP for sinogram requests), runs
 * n_iters iterations of Algorithm 1 on every active slot in the same kernel
 * launches (each slot at its own iteration count and parameters), and
 * retires slots that have done their params.iters iterations, copying Z and
 * rho_e to host memory.  recon_poll hands a finished result over.  A slot's
 * result is bit-identical to the same request solved alone.  Not
 * thread-safe: one thread drives a server. */
typedef struct recon_server recon_server;

typedef struct recon_server_config {
    int32_t max_slots;          /* concurrent solves */
    int32_t max_nx, max_ny;     /* largest image a slot holds */
    int32_t max_views, max_bins;/* largest sinogram a slot holds (0: image requests only) */
    int32_t precision;          /* as recon_params.precision; every request must match */
    double hbm_budget_bytes;    /* admission budget of the in-flight solves; <= 0: slots only */
} recon_server_config;

typedef struct recon_request {
    recon_geometry geom;        /* n_views = 0: images; else -log sinograms */
    recon_params params;
    const float* low;           /* host, copied by recon_submit */
    const float* high;
} recon_request;

typedef struct recon_result {
    int32_t status;             /* RECON_OK or the error of the solve */
    int32_t iters;              /* iterations run */
    double queue_ms;            /* submit -> admitted to a slot */
    double latency_ms;          /* submit -> result on the host */
} recon_result;

int recon_server_create(const recon_server_config* cfg, void* stream, recon_server** out);
/* Errors: EINVAL (size above the slot capacity, precision mismatch,
 * size not 7-smooth), EBUDGET (footprint alone above the budget). */
int recon_submit(recon_server* srv, const recon_request* req, uint64_t* ticket);
/* *n_active (may be NULL): active slots after the step. */
int recon_server_step(recon_server* srv, int32_t n_iters, int32_t* n_active);
/* 1 and the result (Z, rho_e host buffers of ny*nx floats, may be NULL) when
 * done, 0 while queued or running; EINVAL for an unknown ticket. */
int recon_poll(recon_server* srv, uint64_t ticket, float* Z, float* rhoe, recon_result* res);
/* out4: queued, active, finished-not-polled, in-flight footprint bytes. */
int recon_server_stats(recon_server* srv, int64_t* out4);
void recon_server_destroy(recon_server* srv);

/* ---- fan-beam input stage (n slices of the same geometry, device buffers,
 * queued on stream) ---- */

/* sino = A img: Joseph ray-driven line integrals (mm * 1/mm). */
int recon_project(const recon_geometry* geom, int32_t n, const float* img, float* sino, void* stream);
/* img = A^T sino: the exact transpose of recon_project (scatter; img is
 * overwritten). */
int recon_backproject(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream);
/* Flat-detector fan-beam FBP of a full scan (cosine weight, Ram-Lak ramp,
 * 1/U^2 weighted pixel-driven backprojection). */
int recon_fbp(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream);
/* recon_fbp without any device allocation, for callers that cannot allocate
 * device memory when they call: for example a real-time reconstruction loop
 * that forbids allocation once it has started, or a service that reserves all
 * of its device memory up front and hands the library only its own buffers.
 * (The paper has no counterpart: this is an interface of the library.)
 * Same arguments, kernels and result as recon_fbp.  The filtered sinograms
 * go to a fixed scratch array inside the library of RECON_FBP_NOALLOC_MAX
 * floats (8 MiB), which every GPU that loads the library holds until the
 * process exits; calls with n * n_views * n_bins above that return
 * RECON_EINVAL.  The first call on a device looks up the array's device
 * address (with that device current) and keeps it for the life of the
 * process, so make that first call before any stream capture; a device reset
 * (cudaDeviceReset, or the primary context destroyed and created again)
 * invalidates the kept address, so do not call this function after one.  Every call shares the one array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Each call overwrites every scratch value it
 * reads, so nothing has to be cleared between calls. */
#define RECON_FBP_NOALLOC_MAX (2 * 1024 * 1024)
int recon_fbp_noalloc(const recon_geometry* geom, int32_t n, const float* sino, float* img, void* stream);

/* Synthetic scan: -log sinograms of both arms of params for truth maps Z and
 * rho_e (images, device).  noise: NULL (noiseless) or 2 * n * n_views *
 * n_bins standard normal deviates (low arm first) used as the Gaussian
 * approximation of Poisson counting noise at i0 photons per bin; counts are
 * floored at 0.5 before the log. */
int recon_simulate(const recon_geometry* geom, const recon_params* params, int32_t n, const float* Z,
                   const float* rhoe, const float* noise, double i0, float* sino_low, float* sino_high,
                   void* stream);

/* ---- introspection for tests (operators of one iteration) ---- */

/* Scalar tables the solve uses (host FP64): out[0..3] basis at (E_L, E_H)
 * a11 a12 a21 a22 (a_ki = mu_k(E_i) / S), out[4..7] at (E1, E2) b11 b12 b21
 * b22, out[8..9] P1 P2, out[10..11] psi1 psi2, out[12] r = (E1/E2)^n,
 * out[13..14] c_f1 c_f2, out[15] c_rho, out[16] a_w, out[17] S (1/mm per
 * barn).  Returns the number of values written (18). */
int recon_model_tables(const recon_params* params, double* out);

/* Field identifiers for recon_debug_field. */
#define RECON_F_F1 0
#define RECON_F_F2 1
#define RECON_F_RHO 2
#define RECON_F_Z 3
#define RECON_F_MUL 4
#define RECON_F_MUH 5
#define RECON_F_RHS_F1 6
#define RECON_F_RHS_F2 7
#define RECON_F_DIV_RHO 8
#define RECON_F_DIV_Z 9
#define RECON_F_RHS_RHO 10
#define RECON_F_A2 11
#define RECON_F_RHS_Z 12
#define RECON_F_CG_R 13
#define RECON_F_CG_P0 14
#define RECON_F_CG_P1 15
#define RECON_F_CG_Q 16
#define RECON_F_CG_Y 17
#define RECON_F_CG_R2 18   /* second residual buffer of the multigrid PCG */
#define RECON_F_COUNT 19

/* Device pointer of field f of slice s (storage: float, or double when
 * precision = 0; row pitch in elements in *pitch). */
int recon_debug_field(recon_ctx* ctx, int32_t field, int32_t slice, void** dev_ptr, int32_t* pitch,
                      int32_t* elem_bytes);

/* Copy field f of slice s to (to_device = 0) or from (to_device = 1) a host
 * FP64 array of ny * nx values (row-major, no padding); synchronous. */
int recon_debug_io(recon_ctx* ctx, int32_t field, int32_t slice, double* host, int32_t to_device);

/* Operator identifiers for recon_debug_op: each runs one stage of an
 * iteration on every active slice at the handle's current beta. */
#define RECON_OP_INIT 0        /* mu images -> f1, f2, rho_e, z */
#define RECON_OP_THRESH_RHS 1  /* eq. sol_hv + right-hand sides of f1, f2; beta~ div(h,v) of rho_e, z */
#define RECON_OP_SOLVE_F 2     /* FFT solves of f1, f2 */
#define RECON_OP_SYNTH 3       /* mu(E_j) from new f; rhs of rho_e; a^2, rhs of Z^m */
#define RECON_OP_SOLVE_RHO 4   /* FFT solve of rho_e */
#define RECON_OP_SOLVE_Z 5     /* PCG of Z^m */
#define RECON_OP_NEXT_BETA 6   /* beta <- kappa beta, k <- k + 1 */
#define RECON_OP_Z_MATVEC 7    /* q = [diag(a^2) + beta~ L] p (Alg. 1, Z^m line): p from CG_P0, q into CG_Q
                                  (and p into CG_P1), by the kernel that forms q inside each slice's PCG.
                                  FP32 multigrid slices also run their update pass, which forms q again:
                                  with alpha = 1 it leaves -q in CG_R and p in Z (CG_R2 cleared).  Leaves
                                  the PCG state mid-solve */
int recon_debug_op(recon_ctx* ctx, int32_t op);

/* Per-slice scalars: out[0] beta, [1] beta~, [2] k, [3] mean a^2, [4] PCG
 * steps of the last solve, [5] final relative residual. */
int recon_debug_scalars(recon_ctx* ctx, int32_t slice, double* out);

/* Autotuner of the launch shapes.  mode 0: off (default; grid 32 x SMs and
 * the built-in item sizes).  1: the next recon_set_data also times one
 * stencil kernel and one FFT solve on scratch fields with grids of
 * {16, 32, 64} x SMs and keeps the fastest; the arithmetic, and so every
 * result, is unchanged.  2: as 1, and row items of {2048, 3072, 4096}
 * complex slots (FP32), which regroups the per-item partial sums of the
 * PCG reductions and so changes results in the last bits.  The choice holds
 * for the handle. */
int recon_set_autotune(recon_ctx* ctx, int32_t mode);

/* The launch shape in use: out2[0] grid multiplier (grid = out2[0] x SMs),
 * out2[1] complex slots of a row item (0: built-in). */
int recon_tuning(recon_ctx* ctx, int32_t* out2);

/* Run each following iteration of recon_step as one CUDA graph launch
 * (on = 1) or as separate launches (0, the default).  The graph is captured
 * on first use: the steps of Algorithm 1 up to the first PCG step of the
 * Z^m solve, a conditional WHILE node whose body runs two PCG steps and then
 * sets the loop condition on the device (continue while a slice has not
 * converged and fewer than ceil(cg_max_iters / 2) bodies have run), and the
 * beta update.  Results are bitwise those of the separate launches (PCG
 * steps past a slice's convergence skip that slice).  The graph runs on a
 * stream of the handle, ordered after earlier and before later work of the
 * handle's stream; the iteration that fills recon_stats, and iterations
 * while recon_profile is on, still run as separate launches.  Needs domain 0
 * (RECON_EINVAL otherwise). */
int recon_set_graph(recon_ctx* ctx, int32_t on);

/* Number of kernels this handle has launched since creation (counting
 * each launch of each of the library's kernels). */
int64_t recon_kernel_launches(recon_ctx* ctx);

/* Kernel families of the solver, for recon_profile*: 0 threshold + rhs,
 * 1 FFT rows forward, 2 FFT columns (spectral divide), 3 FFT rows inverse,
 * 4 synthesis, 5 PCG start (r = b - M z), and the three passes of a PCG
 * step: 6 update of z and r, convergence test and forward row transforms of
 * D^-1/2 r; 7 column transforms with the preconditioner's divide and r.y;
 * 8 inverse row transforms, new search direction p and q = M p.  9 the CG of
 * the sinogram-domain f updates (its pointwise, stencil and preconditioner
 * column passes), 10 projector and backprojector inside the solve (domain
 * 1); the multigrid-preconditioned PCG: 11 update of z and r, convergence
 * test and the first restriction, 12 fine-level correction and smoothing
 * with r.y, 13 new search direction p, q = M p and p.q, 14 the coarse tile
 * levels (restriction and correction passes), 15 the in-block levels of
 * each slice and its coarsest solve, 16 a^2 of the levels and the coarsest
 * inverse (once per Z^m solve); 17 other. */
#define RECON_KF_COUNT 18

/* Time the launches of the kernel families whose bit is set in mask with
 * CUDA events on the handle's stream (0 = off).  Algorithmic bytes and launch
 * counts are always accounted. */
int recon_profile(recon_ctx* ctx, uint32_t mask);

/* Since the previous read (or creation): per family the summed event time in
 * ms (families not timed: 0), launches, and algorithmic bytes (the bytes each
 * launch must read and write in HBM: interior elements of its inputs and
 * outputs, counted per processed tile / row group / column group).  Arrays of
 * RECON_KF_COUNT entries, each may be NULL.  Synchronises the stream. */
int recon_profile_read(recon_ctx* ctx, double* ms, int64_t* launches, uint64_t* bytes);

/* Name of kernel family f. */
const char* recon_profile_name(int32_t family);

/* sizeof of recon_geometry, recon_spectrum, recon_params, recon_stats as
 * compiled into the library (for bindings to check their layouts). */
int recon_abi_sizes(int64_t* out4);

#ifdef __cplusplus
}
#endif
#endif /* RECON_H */
