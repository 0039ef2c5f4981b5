/*
 * vfmm — periodic FMM evaluation of the Gaussian-regularised Biot-Savart velocity and
 * vortex-stretching term of a vortex-particle system, for NVIDIA GB300 (sm_103a).
 *
 * The operation (Yokota & Barba, "FMM-based vortex method for simulation of isotropic
 * turbulence on GPUs, compared with a spectral method"):
 *
 *   u_i  = sum_n sum_j' K(r) gamma_j x r                                    Eq. (biotsavart)
 *   S_i  = sum_n sum_j' [ K(r) gamma_j x gamma_i + F(r)(gamma_i . r)(gamma_j x r) ]
 *        = (gamma_i . grad) u at x_i                                          Eq. (stretching)
 *   r = x_i - x_j - n L,  rho = |r|/sigma,
 *   q(rho) = erf(rho/sqrt2) - sqrt(2/pi) rho exp(-rho^2/2)                    Eq. (cutoff)
 *   K = q/(4 pi |r|^3),  F = K'(|r|)/|r|
 *
 * over the image boxes n of a cube of 3^(S+1) boxes per side around the primary box
 * [0, L)^3 (S = periodic_levels; S = 2 is the 27^3 images of Section 4.1), skipping the
 * self pair.  The FMM (Section 3.1, Eqs. fmm3dm, fmm3dl, biotsavartfmm1-2,
 * stretchingfmm1-2) evaluates the far field from expansions of the vector potential
 * psi = sum_j gamma_j G with g_sigma = 1, and the near field exactly; the images beyond
 * the central 3^3 boxes come from the root multipole through a precomputed lattice
 * operator (Section 3.1, last paragraph; Section 5.6).
 *
 * Conventions
 *  - Every function returns an int status: VFMM_OK (0) or a negative VFMM_ERR_* code.
 *    vfmm_strerror() names a code; vfmm_last_error() gives the detail of the last
 *    failure on a handle.
 *  - Pointer arguments of vfmm_build_tree / vfmm_eval_* are DEVICE pointers owned by the
 *    caller, contiguous row-major n x 3 arrays of float (cfg.dtype = VFMM_F32) or
 *    double (VFMM_F64).  Outputs are in the caller's particle order.
 *    vfmm_eval_host takes HOST pointers and does the copies itself.
 *  - The handle owns all workspace (tree, expansions, operators); it allocates device
 *    memory in vfmm_create / vfmm_build_tree / the first evaluation of a size.
 *  - Work is enqueued on cfg.stream (a cudaStream_t; NULL = legacy default stream).
 *    vfmm_eval_* is asynchronous: device-side errors (e.g. a leaf overflow) are
 *    reported by the next vfmm_sync().  vfmm_build_tree synchronises the stream once, after
 *    the key and scatter kernels (the largest leaf sizes the per-leaf sort; non-finite
 *    positions are reported there); the per-leaf sort runs on after it returns.  With
 *    concurrent_far the FP32 evaluation forks its far field onto a handle-owned
 *    high-priority stream and joins it back before its last kernel, so on cfg.stream the
 *    call still follows earlier work and precedes later work.
 *  - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef VFMM_H
#define VFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VFMM_OK 0
#define VFMM_ERR_ARG (-1)         /* invalid argument (n <= 0, p < 2, non-finite sigma ...) */
#define VFMM_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define VFMM_ERR_OOM (-3)         /* device allocation failed */
#define VFMM_ERR_NOT_BUILT (-4)   /* evaluation before vfmm_build_tree */
#define VFMM_ERR_BOUNDS (-5)      /* a device-side bounds check fired */
#define VFMM_ERR_TIMEOUT (-6)     /* a bounded device-side wait gave up */
#define VFMM_ERR_UNSUPPORTED (-7) /* configuration outside what is implemented */

/* element type of the caller's arrays, and the arithmetic of P2P and the expansions */
#define VFMM_F32 0
#define VFMM_F64 1

/* arithmetic of the M2L translations (FP32 / FP64 on CUDA cores; TF32 or BF16 inputs on
 * the tensor cores with FP32 accumulation and a three-product hi/lo split) */
#define VFMM_M2L_FP32 0
#define VFMM_M2L_FP64 1
#define VFMM_M2L_TF32X3 2
#define VFMM_M2L_BF16X3 3

/* evaluation method */
#define VFMM_METHOD_FMM 0    /* tree + expansions + near field */
#define VFMM_METHOD_DIRECT 1 /* all pairs over the (2K+1)^3 image cube, K = direct_images */

typedef struct vfmm_config {
    int p;               /* expansion order: degrees 0..p, (p+1)^2 coefficients (Eq. fmm3dm); 2 <= p <= 10 */
    int depth;           /* leaf depth D of the uniform octree; 0 = choose from ncrit */
    int ncrit;           /* target mean particles per leaf when depth == 0 */
    int near_rings;      /* R: near field = (2R+1)^3 leaves with the smoothed kernel; 0 = automatic: 1 for the
                          * FP32 velocity / stretching evaluation, else the smallest R with R w >= rho_cut sigma.
                          * Where R w < rho_cut sigma <= 2 w in FP32 (not the gradient), ring 2 is left to the
                          * M2L and the source octants of ring 2 closer than rho_cut sigma get the smoothed-
                          * minus-singular correction pair by pair, so every pair closer than rho_cut sigma
                          * still takes the smoothed kernel.  R <= 2; rho_cut sigma > 2 w is an error. */
    double rho_cut;      /* pairs farther apart than rho_cut sigma may take the singular kernel (default 5:
                          * 1 - q(5) = 1.5e-5) */
    int periodic_levels; /* S: image cube of 3^(S+1) boxes per side; 0 = the 27 central boxes only */
    double box;          /* L, the period (default 2 pi) */
    int dtype;           /* VFMM_F32 | VFMM_F64 */
    int m2l_prec;        /* VFMM_M2L_*; with dtype F64 only VFMM_M2L_FP64 is accepted */
    int method;          /* VFMM_METHOD_FMM | VFMM_METHOD_DIRECT */
    int direct_images;   /* K for VFMM_METHOD_DIRECT */
    void *stream;        /* cudaStream_t */
    int concurrent_far;  /* 1 (default): in the FP32 velocity / stretching evaluation the far field runs on an
                          * internal high-priority stream while the near-field P2P runs on `stream`, joined
                          * before the far field is added; 0: every phase in line on `stream` */
} vfmm_config;

typedef struct vfmm_ctx *vfmm_handle;

/* Fill *cfg with defaults: p=10, depth=0, ncrit=64, near_rings=0, rho_cut=5, S=2, L=2 pi,
 * F32, M2L BF16X3, FMM, K=1, stream NULL, concurrent_far 1. */
int vfmm_config_default(vfmm_config *cfg);

/* Create a handle; precomputes the FP64 translation and lattice operators on the host and
 * uploads them.  *out receives the handle (NULL on failure). */
int vfmm_create(const vfmm_config *cfg, vfmm_handle *out);

/* Release the handle and all its device memory (synchronises its stream). */
int vfmm_destroy(vfmm_handle h);

/* Change the stream later calls enqueue on. */
int vfmm_set_stream(vfmm_handle h, void *stream);

/* Tries of each bounded wait in the tensor-core M2L pipeline before a CTA gives up (0 = the
 * default, 2^26).  A CTA that gives up stops its pipeline, waits for its own copies and MMAs to
 * complete, frees its tensor memory and sets the timeout bit: the evaluation then reports
 * VFMM_ERR_TIMEOUT at vfmm_sync and its outputs are not valid; the handle stays usable.  A
 * small limit makes the waits give up on purpose, which is how that path is tested (failure
 * injection; the paper has no counterpart).  Errors: tries < 0 -> VFMM_ERR_ARG. */
int vfmm_set_wait_limit(vfmm_handle h, int64_t tries);

/* Sort n particles into the uniform octree (Section 3.2; tree construction ran on the CPU in
 * the paper, Section 2.2).  x: device n x 3 positions; positions are wrapped into [0, L)^3
 * by x - L floor(x/L) (any finite value is accepted).  Keys are leaf indices, the sort is a
 * counting sort with a per-leaf index sort, so the order is deterministic.
 * Errors: n <= 0 -> VFMM_ERR_ARG; a NaN or infinite coordinate -> VFMM_ERR_ARG (detected on the
 * device, reported by this call, which synchronises; the handle then has no tree); a leaf with
 * more than 4096 particles -> VFMM_ERR_UNSUPPORTED. */
int vfmm_build_tree(vfmm_handle h, int64_t n, const void *x);

/* u and S at every particle for strengths gamma (device n x 3, caller order) and core
 * size sigma (Eqs. biotsavart, stretching).  u_out: device n x 3; s_out: device n x 3 or
 * NULL to skip the stretching term.  Errors: sigma not finite or <= 0 -> VFMM_ERR_ARG;
 * before vfmm_build_tree -> VFMM_ERR_NOT_BUILT; a near field that would need R > 2 ->
 * VFMM_ERR_UNSUPPORTED (use a shallower tree). */
int vfmm_eval_velocity_stretching(vfmm_handle h, const void *gamma, double sigma, void *u_out,
                                  void *s_out);

/* Velocity and its gradient at every particle: u_out n x 3 and g_out n x 9 with
 * g_out[9 i + 3 a + k] = du_a/dx_k at x_i (device, caller order).  Same sum as
 * vfmm_eval_velocity_stretching (S_i = G_i gamma_i); the self pair is excluded.  Used by the
 * adjoint and by callers that need the full tensor (e.g. the transpose stretching scheme).
 * Errors as vfmm_eval_velocity_stretching. */
int vfmm_eval_velocity_gradient(vfmm_handle h, const void *gamma, double sigma, void *u_out, void *g_out);

/* Adjoint of u = A(x) gamma for a loss L(u) with w = dL/du (device n x 3, caller order), on the
 * tree of the last vfmm_build_tree (positions frozen to their leaves):
 *   dgamma = A^T w,   dx_m = dL/dx_m,
 * the exact gradient (to rounding) of u as vfmm_eval_velocity_gradient evaluates it.  With
 * VFMM_METHOD_DIRECT, A^T w = A w (the Biot-Savart matrix is symmetric: A_ji = A_ij^T) and
 * dx_m = (grad u^gamma(x_m))^T w_m + (grad u^w(x_m))^T gamma_m, u^w the velocity of strengths w.
 * With the FMM, A^T is the transpose of the evaluated operator: the near field (all near rings
 * with the smoothed kernel, a symmetric pair set) as for the direct sum, and the far field run
 * backwards through the transposed chain (transposed L2P as a P2M of the curl of the local basis,
 * L2L^T, M2L^T with the transposed translation matrices, lattice and root M2M transposed in
 * FP64, M2M^T, P2M^T as an evaluation of the dual multipole); dx_m adds to the target term the
 * source term gamma_m . grad of that dual potential.  The transposed operators are built on the
 * first FMM call (host FP64, then uploaded: 2 x 343 matrices of 128 x 128 and their tensor-core
 * tiles).  In FP32 the velocity-gradient path (all near rings smoothed) is the operator; it agrees
 * with vfmm_eval_velocity_stretching's one ring + Gaussian-tail correction to the FMM tolerance.
 * v (dL/dS) must be NULL (VFMM_ERR_UNSUPPORTED otherwise).  dgamma, dx: device n x 3.  Uses
 * handle-owned temporaries of 21 n values. */
int vfmm_eval_adjoint(vfmm_handle h, const void *gamma, double sigma, const void *w, const void *v, void *dgamma,
                      void *dx);

/* One time step of the vortex method (Section 2.2: Eqs. convection, stretching, csm) by the
 * explicit trapezoid (Heun) rule: (u1, S1) at (x, gamma, sigma); (u2, S2) at
 * (x + dt u1, gamma + dt S1, sqrt(sigma^2 + 2 nu dt)); then x += dt (u1 + u2)/2 wrapped into
 * [0, L), gamma += dt (S1 + S2)/2, sigma^2 += 2 nu dt (core spreading, exact).  x, gamma: device
 * n x 3 (caller order), updated in place; sigma: host, updated.  Builds the tree twice; with
 * depth 0 and near_rings 0 in the configuration each build takes the ncrit depth made
 * shallower where the stage's core needs it (2 w >= rho_cut sigma), so growing cores stay
 * within the two-ring near field.  The handle's tree is stale afterwards (call
 * vfmm_build_tree before the next evaluation).
 * Errors: n <= 0, NULL pointers, non-finite dt or nu, nu < 0, sigma <= 0 -> VFMM_ERR_ARG. */
int vfmm_rk_step(vfmm_handle h, int64_t n, void *x, void *gamma, double *sigma, double dt, double nu);

/* Reinitialise n particles (x, gamma, core sigma; device n x 3, caller order) onto the m^3
 * cell-centre lattice of [0, L)^3 with core sigma_new (<= 0: the lattice spacing h = L/m)
 * (Section 2.2, RBF interpolation): omega(x_g) = sum_j gamma_j zeta_sigma(x_g - x_j) with the
 * Gaussian basis of Eq. (gaussian), then iters steepest-descent steps with exact line search
 * on 0.5 |Z gamma' - omega|^2, Z_gk = zeta_sigma_new(x_g - x_k), from gamma' = omega h^3
 * (Section 5.3).  x_new, gamma_new: device m^3 x 3 outputs, lattice order (ix m + iy) m + iz.
 * residual (host, may be NULL): |omega - Z gamma'| / |omega|.  Gaussians are cut at 6 sigma.
 * Synchronises the stream; the handle's tree is stale afterwards.
 * Errors: bad sizes or non-finite sigma -> VFMM_ERR_ARG; a lattice finer than 64 points per
 * leaf side or more than 32 stencil taps -> VFMM_ERR_UNSUPPORTED. */
int vfmm_reinit(vfmm_handle h, int64_t n, const void *x, const void *gamma, double sigma, int m, double sigma_new,
                int iters, void *x_new, void *gamma_new, double *residual);

/* FP64 sums over n particles (device arrays; u may be NULL): out[0..2] = sum gamma (total
 * vorticity), out[3..5] = sum x cross gamma (twice the linear impulse), out[6] = sum |u|^2,
 * out[7] = sum |gamma|^2.  Synchronises the stream. */
int vfmm_diagnostics(vfmm_handle h, int64_t n, const void *x, const void *gamma, const void *u, double *out);

/* Energy spectrum of a velocity field sampled on the n^3 lattice (Section 5.2 evaluates the
 * velocity on a lattice with the Biot-Savart law and takes a 3-D FFT):
 *   E(k) = sum over integer wave vectors with k - 1/2 <= |k| < k + 1/2 of 0.5 |u_hat(k)|^2,
 *   u_hat(k) = n^-3 sum_x u(x) exp(-i k.x),  k = 0..kmax,
 * so that sum_k E(k) = 0.5 <|u|^2> once kmax >= sqrt(3) n / 2.  u_lattice: device n^3 x 3 of the
 * configured dtype in lattice order (ix n + iy) n + iz (the order of a lattice particle set);
 * n a power of two in [4, 1024]; 0 <= kmax <= 4096.  E_out: host, kmax + 1 doubles.  FP64
 * throughout; the handle keeps a 48 n^3-byte workspace after the first call.  Synchronises
 * the stream.  Errors: bad pointers or kmax -> VFMM_ERR_ARG; other n -> VFMM_ERR_UNSUPPORTED. */
int vfmm_energy_spectrum(vfmm_handle h, int n, const void *u_lattice, int kmax, double *E_out);

/* Velocity-derivative moments (Section 5.2: F_n = mean(u_x^n) / mean(u_x^2)^(n/2), F_3 the
 * skewness, F_4 the flatness).  The samples are the three longitudinal derivatives
 * du_a/dx_a of each particle (isotropy), read from a gradient g (device n x 9, g[9 i + 3 a + k]
 * = du_a/dx_k, as vfmm_eval_velocity_gradient writes it).  out (host, 5 doubles): mean d^2,
 * mean d^3, mean d^4, F_3, F_4, accumulated in FP64.  Synchronises the stream. */
int vfmm_derivative_moments(vfmm_handle h, int64_t n, const void *grad, double *out);

/* End to end from HOST memory: copies x and gamma to the device, builds the tree,
 * evaluates, copies u and S back, and synchronises.  Pointers are host n x 3 arrays of the
 * configured dtype; s_out may be NULL. */
int vfmm_eval_host(vfmm_handle h, int64_t n, const void *x, const void *gamma, double sigma,
                   void *u_out, void *s_out);

/* Wait for the handle's stream; returns the first device-side error since the last call. */
int vfmm_sync(vfmm_handle h);

/* Milliseconds per phase of the last evaluation (CUDA events; valid after vfmm_sync):
 * [0] tree build, [1] P2M, [2] M2M, [3] M2L, [4] periodic lattice operator, [5] L2L,
 * [6] L2P, [7] P2P + output.  Writes min(nphase, 8) values. */
int vfmm_get_timings(vfmm_handle h, double *ms_per_phase, int nphase);

/* Tree facts: out[0] = depth D, out[1] = near rings R used by the last evaluation,
 * out[2] = leaves per side, out[3] = maximum particles in one leaf, out[4] = particles,
 * out[5] = CUDA kernels launched by the last vfmm_build_tree plus the evaluations since,
 * out[6] = outer ring of the Gaussian-tail correction in the last evaluation (0 = none),
 * out[7] = source-target pairs of real targets computed by the last FP32 near-field launch, as
 * counted on the device by a library built with -DVFMM_CHECK=1 (waits for the handle's stream;
 * 0 in the default build).  Writes min(nout, 8) values. */
int vfmm_get_tree_info(vfmm_handle h, int64_t *out, int nout);

/* Peak-rate probes, the measured denominators of the roofline fractions (measurement only;
 * the paper has no counterpart).  Launches one kernel on stream (a cudaStream_t) on the
 * current device that performs *ops operations of one kind, for the caller to time with CUDA
 * events on that stream:
 *   VFMM_PROBE_FFMA   FP32 fmaf, 8 independent chains per thread, 64 warps per SM; 2 flops each
 *   VFMM_PROBE_EX2    MUFU ex2.approx.ftz.f32; 1 op per lane
 *   VFMM_PROBE_RSQRT  MUFU rsqrt.approx.ftz.f32; 1 op per lane
 *   VFMM_PROBE_DFMA   FP64 fma; 2 flops each
 *   VFMM_PROBE_MMA_TF32 / _BF16  one CTA per SM issuing tcgen05.mma (M 128, N 256, K 8 TF32 /
 *                     16 BF16, shared-memory operands, TMEM accumulator); 2 M N K flops each
 * reps scales the work (the ALU probes run 128 reps of each chain step per unit; the MMA
 * probes reps instructions per SM).  err_dev: device int that the MMA probes OR with 4
 * (timeout of their bounded completion wait); may be NULL for the ALU probes.  Nothing is
 * allocated.  Errors: unknown kind, reps <= 0, ops NULL, or err_dev NULL for an MMA probe ->
 * VFMM_ERR_ARG; a failed launch -> VFMM_ERR_CUDA. */
#define VFMM_PROBE_FFMA 0
#define VFMM_PROBE_EX2 1
#define VFMM_PROBE_RSQRT 2
#define VFMM_PROBE_DFMA 3
#define VFMM_PROBE_MMA_TF32 4
#define VFMM_PROBE_MMA_BF16 5
int vfmm_probe_peak(int kind, int64_t reps, void *stream, int *err_dev, double *ops);

/* Largest n accepted by vfmm_direct_eval_noalloc. */
#define VFMM_NOALLOC_MAX_N 65536

/* Direct sum of u and S (VFMM_METHOD_DIRECT, FP32) that allocates nothing.
 *
 * For callers that cannot allocate device memory when they call in: a host program that
 * gives all device memory to its own pool up front, or a latency-critical loop that must not
 * pay cudaMalloc's implicit device synchronisation.  This call makes no cudaMalloc, cudaFree
 * or other allocating call.  The paper has no counterpart; it evaluates the same sum as a
 * handle created with method VFMM_METHOD_DIRECT and direct_images = images.
 *
 * x, gamma: device n x 3 float positions (wrapped into [0, box)^3) and strengths; u_out:
 * device n x 3 float; s_out: device n x 3 float or NULL.  Outputs are in input order.  Work is
 * enqueued on stream (a cudaStream_t); the call does not synchronise.
 * Scratch: one file-scope device array of 2 x VFMM_NOALLOC_MAX_N float4 (2 MiB), present on
 * every device that loads the library until the process exits.  Every call on a device uses
 * the same array and overwrites the part it needs, so calls whose work overlaps on the GPU
 * (other streams, other host threads) race: order them on one stream or synchronise between.
 * Each call outside stream capture looks up the array's device address (cudaGetSymbolAddress,
 * with the device current; a host-side lookup that allocates nothing), so the address stays
 * right after cudaDeviceReset reloads the module; a call during stream capture reuses the
 * address of the last call outside capture on that device, so make a first call before any
 * capture (a capture with no earlier call does the lookup itself).
 * Errors: n <= 0, a NULL x/gamma/u_out, sigma or box not finite and > 0, or images outside
 * [0, 20] -> VFMM_ERR_ARG; n > VFMM_NOALLOC_MAX_N -> VFMM_ERR_UNSUPPORTED (nothing is
 * launched); a failed address look-up or launch -> VFMM_ERR_CUDA. */
int vfmm_direct_eval_noalloc(int64_t n, const float *x, const float *gamma, double sigma, double box, int images,
                             float *u_out, float *s_out, void *stream);

/* Name of a status code (static string). */
const char *vfmm_strerror(int status);

/* Detail message of the last failure on h (valid until the next call on h). */
const char *vfmm_last_error(vfmm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* VFMM_H */
