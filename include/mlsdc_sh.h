/*
 * mlsdc_sh.h -- C ABI of the GB300 (sm_103a) MLSDC-SH library.
 *
 * The library integrates the rotating shallow-water equations in
 * vorticity-divergence-geopotential form (Hamon, Schreiber, Minion, Sec. 2,
 * Eqs. geopotential_equation, vorticity_equation, divergence_equation) with
 * a global spherical-harmonic (SH) discretisation (Sec. 3) and IMEX
 * spectral deferred corrections, single-level (Sec. 4.2) or two-level MLSDC
 * (Sec. 4.3, Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Spectral field at triangular truncation R (Sec. 3, Eq. spectral_space with
 * r = m the zonal wavenumber and s = n the total degree, m >= 0 only):
 *   N_c = (R+1)(R+2)/2 complex coefficients xi^m_n, 0 <= m <= n <= R, stored
 *   m-major (for m = 0..R: n = m..R, index m(R+1) - m(m-1)/2 + (n-m)), each
 *   complex as two consecutive doubles (re, im).  Im xi^0_n is zero.
 *   Legendre functions are orthonormal on [-1, 1] without Condon-Shortley
 *   phase, so a field is f = sum_n xi^0_n P^0_n + 2 Re sum_{m>=1} xi^m_n P^m_n e^{i m lambda}.
 * State: [3][N_c] complex in the order (Phi', zeta, delta), Phi' = Phi - Phibar.
 * Grid field: [J][I] doubles, latitude-major from north (mu_0 > 0) to south,
 *   longitude lambda_i = 2 pi i / I contiguous.
 * Node arrays ("space-time vectors", Sec. 4.2): [M+1][3][N_c] complex.
 *
 * Memory: every data pointer is a DEVICE pointer owned by the caller, 16-byte
 * aligned, contiguous.  The entry points that take complex arrays refuse a
 * pointer that is not 16-byte aligned with MLSDC_ERR_INVALID (the argument
 * named in mlsdc_last_error()) before any launch.  Plans, levels and MLSDC objects own their tables and
 * scratch (allocated at creation, freed at destroy).  Calls are asynchronous
 * on the given CUDA stream (NULL = legacy default stream); calls that share a
 * plan, level or MLSDC object must be ordered on one stream, since they share
 * that object's scratch.  No exception crosses the ABI; each call returns a
 * status.  Argument errors are detected before any launch; a CUDA error is
 * reported as MLSDC_ERR_CUDA with its text in mlsdc_last_error().
 */
#ifndef MLSDC_SH_H
#define MLSDC_SH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mlsdc_status;
#define MLSDC_OK 0
#define MLSDC_ERR_INVALID (-1)     /* bad size, null pointer, unsupported configuration */
#define MLSDC_ERR_CUDA (-2)        /* a CUDA runtime call or launch failed */
#define MLSDC_ERR_NONFINITE (-3)   /* a state check found NaN or Inf */
#define MLSDC_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define MLSDC_ERR_ALLOC (-5)       /* device memory allocation failed */

/* Arithmetic of the Legendre stage (Sec. 3, Eq. legendre_transform and its
 * inverse).  MLSDC_FP64: everything in float64.  MLSDC_TF32 / MLSDC_BF16X3:
 * the Legendre contractions run on tcgen05 tensor cores (TF32 operands, or
 * bf16 hi+lo splits with the three products hi*hi + hi*lo + lo*hi), with
 * float32 accumulation; the longitude FFTs and grid products run in float32;
 * the Legendre recurrence, quadrature, SDC matrices, implicit solve and all
 * state accumulation stay float64.  MLSDC_FP32: as the tensor-core modes but
 * with float32 FMA contractions on the CUDA cores. */
typedef enum {
    MLSDC_FP64 = 0,
    MLSDC_TF32 = 1,
    MLSDC_BF16X3 = 2,
    MLSDC_FP32 = 3
} mlsdc_precision;

/* Physical constants in SI units (Sec. 2): Earth radius a, rotation rate
 * Omega (f = 2 Omega mu), gravity g, mean geopotential Phibar, diffusion nu. */
typedef struct {
    double a, omega, g, phibar, nu;
} swe_params;

typedef struct sh_plan_s* sh_plan_t;
typedef struct sdc_level_s* sdc_level_t;
typedef struct mlsdc_s* mlsdc_t;
typedef struct mlsdc_ensemble_s* mlsdc_ensemble_t;
typedef struct mlsdc_adjoint_s* mlsdc_adjoint_t;
typedef struct mlsdc_levels_s* mlsdc_levels_t;
typedef struct pfasst_s* pfasst_t;

/* Text of a status code, and the last CUDA error message seen by this thread. */
const char* mlsdc_status_string(mlsdc_status s);
const char* mlsdc_last_error(void);

/* ---------------------------------------------------------------------------
 * sh_plan: Gaussian grid and Legendre tables of one truncation (Sec. 3:
 * Eq. legendre_transform's Gaussian latitudes and weights; the normalised
 * associated Legendre functions of Eq. spectral_to_physical_space and
 * H = (1 - mu^2) dP/dmu for the velocity and divergence/curl transforms).
 * R >= 1; nlon a power of two in [16, 1024] with nlon >= 3R+1 (alias-free
 * quadratic products); nlat even with nlat >= (3R+1)/2 and nlat/2 <= 1024.
 * Tables are computed on the host in float64 and copied to the device of the
 * current CUDA context.  Returns MLSDC_ERR_INVALID for other sizes.
 */
mlsdc_status sh_plan(int R, int nlon, int nlat, int precision, sh_plan_t* out);
/* sh_plan_batched: the same plan with scratch for up to max_members
 * ensemble members per F_E launch (1 <= max_members <= 4096).  For the
 * tensor-core precisions the number of members per CTA (1, 2, 4, 8 or 16)
 * is chosen at creation by timing each feasible choice on a full batch. */
mlsdc_status sh_plan_batched(int R, int nlon, int nlat, int precision, int max_members, sh_plan_t* out);
mlsdc_status sh_plan_destroy(sh_plan_t plan);
/* Copies of the host-side grid: mu[nlat], w[nlat] (north to south). */
mlsdc_status sh_plan_grid(sh_plan_t plan, double* mu_host, double* w_host);
/* Bytes of device memory the plan holds (tables plus scratch). */
mlsdc_status sh_plan_device_bytes(sh_plan_t plan, int64_t* bytes);
/* Device-side error code recorded by the plan's tensor-core kernels (0 = none;
 * 1 = a TMA wait gave up, 2 = an MMA completion wait gave up).  Every such
 * wait is bounded (2 s of the global timer): on timeout the kernel records
 * the code, releases its tensor memory and returns without writing results.
 * Synchronises the device.  Always 0 for MLSDC_FP64 / MLSDC_FP32 plans. */
mlsdc_status sh_plan_device_error(sh_plan_t plan, int* code);
/* Check of the bounded device-side wait used by the tensor-core kernels:
 * one CTA waits on an mbarrier that nothing completes, with the same wait
 * loop (polls bounded by the global timer) and a limit of timeout_ms
 * (1..2000); the wait must give up and the kernel records 2 (the code of a
 * gave-up MMA wait) and returns, leaving the context usable.  *code is the
 * recorded value (0 would mean the barrier completed).  Synchronises the
 * device.  MLSDC_ERR_INVALID for a null pointer or a limit out of range. */
mlsdc_status mlsdc_selftest_wait_timeout(int timeout_ms, int* code);
/* How the float32 CUDA-core synthesis (MLSDC_FP32, and the synthesis of
 * tensor-core plans where it runs on CUDA cores) reads its Legendre tables:
 * 0 = by size (TMA into shared memory for up to two 32-row boxes per work
 * item, R <= 63, or three boxes with at most 4 members; plain loads
 * otherwise), 1 = TMA whenever the plan allows it (nlat/2 a multiple of 4),
 * 2 = plain loads.  Results are identical either way (the same sums in the
 * same order).  MLSDC_ERR_INVALID for float64 plans or other modes. */
mlsdc_status sh_plan_set_synth_tma(sh_plan_t plan, int mode);
/* Check of the float32 -> float64 conversion the analysis kernels use for
 * F_E (bit rearrangement on the integer pipes instead of the conversion
 * instruction, which uses the slow float64 pipe): for n device values f_in
 * writes the library's conversion to d_ours and the hardware's to d_hw
 * (asynchronous on `stream`).  Not a paper operation. */
mlsdc_status mlsdc_selftest_convert(const float* f_in, int n, double* d_ours, double* d_hw, void* stream);
/* Which kernel each Legendre stage of a tensor-core plan (MLSDC_TF32 /
 * MLSDC_BF16X3) runs: the tcgen05 kernel or the float32 CUDA-core kernel of
 * MLSDC_FP32.  By default the choice follows a fixed rule per launch (measured
 * on GB300): the analysis on tensor cores for R >= 64, the synthesis on
 * tensor cores for R >= 128 with at least 8 members in the launch, the
 * CUDA-core kernels otherwise.  The CUDA-core kernels use float32 operands,
 * at least as accurate as split-BF16 or TF32; the rule depends on sizes only,
 * so results are reproducible.  sh_plan_stage_kernels reports the kernels a
 * launch of `members` states uses (1 = tcgen05; 0, 0 for other precisions).
 * sh_plan_set_stage_kernels sets each stage's mode: 0 = the rule, 1 = always
 * tcgen05, 2 = always the CUDA-core kernel (MLSDC_ERR_INVALID for other
 * precisions or modes). */
mlsdc_status sh_plan_stage_kernels(sh_plan_t plan, int members, int* synth_tc, int* anal_tc);
mlsdc_status sh_plan_set_stage_kernels(sh_plan_t plan, int synth_mode, int anal_mode);
/* The launch configuration of each tensor-core Legendre stage (stage 0: the
 * synthesis, 2: the analysis), chosen at plan creation by timing each
 * feasible choice of that stage alone on a full batch of the plan's
 * max_members: members per CTA (1, 2, 4, 8 or 16; the members form the
 * MMA's N dimension, 16 columns each), the depth of the shared-memory
 * pipeline over K (1 or 2 stages) and, for the analysis of launches of 3 or
 * more members, whether it runs the warp-specialised kernel (1: persistent
 * CTAs of two warpgroups, one staging operands and issuing the MMAs, one
 * running the epilogue of the previous tile from a second accumulator buffer
 * in tensor memory; up to 8 members per CTA).  sh_plan_tc_config reports it
 * (zeros for MLSDC_FP64 / MLSDC_FP32 plans; pointers may be NULL);
 * sh_plan_set_tc_config replaces it (results are the same to rounding;
 * MLSDC_ERR_INVALID for other precisions or stages, a member count that is
 * not a power of two up to min(16, max_members), a depth other than 1 or 2,
 * warp specialisation for the synthesis or with more than 8 members per CTA,
 * or a choice whose shared memory does not fit a CTA). */
mlsdc_status sh_plan_tc_config(sh_plan_t plan, int stage, int* members_per_cta, int* stages, int* warp_specialised);
mlsdc_status sh_plan_set_tc_config(sh_plan_t plan, int stage, int members_per_cta, int stages,
                                   int warp_specialised);

/* sh_inverse: spectral -> grid for nf independent scalar fields,
 * Eq. spectral_to_physical_space (Legendre sum per m, then the inverse
 * longitude DFT).  spec: [nf][N_c] complex; grid: [nf][J][I]; 1 <= nf <= 16. */
mlsdc_status sh_inverse(sh_plan_t plan, const double* spec, double* grid, int nf, void* stream);

/* sh_inverse_static: the same synthesis as sh_inverse, for callers that must
 * not allocate device memory at all -- for example a host framework that has
 * already handed every byte of the GPU to its own memory pool, or a long-running
 * service whose device-memory footprint is fixed when it starts and may not
 * grow afterwards.  Such callers cannot create an sh_plan (it allocates its
 * tables and scratch), so this entry point takes the sizes directly, computes
 * the Gaussian latitudes, Legendre functions and FFT twiddles on the device,
 * and keeps its intermediate values in one static 4 MiB device array that
 * every GPU loading this library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  The paper has no
 * counterpart: this is an interface variant, not a step of the method.
 * Sizes: as sh_plan (R >= 1; nlon a power of two in [16, 1024], nlon >= 3R+1;
 * nlat even, nlat >= (3R+1)/2, nlat <= 2048), 1 <= nf <= 16, and
 * nf * nlat * (R+1) <= 261120 (e.g. nf <= 5 at T170 on 512 x 256); larger
 * requests return MLSDC_ERR_INVALID with the limit in mlsdc_last_error().
 * spec: [nf][N_c] complex, grid: [nf][nlat][nlon] (caller-owned device memory,
 * both 16-byte aligned: a pointer at an odd double offset is refused with
 * MLSDC_ERR_INVALID before any launch).  Every invalid argument sets a
 * message in mlsdc_last_error().
 * Every call made outside stream capture looks up the static array's device
 * address (cudaGetSymbolAddress) with the current device, so the address stays
 * right after a cudaDeviceReset reloads the module; a call under capture
 * reuses the address found by the last uncaptured call on that device, so
 * make a first call on each device before any stream capture (and again after
 * a device reset, before capturing).  All calls share the one array and it keeps the last
 * call's contents; every value a call reads from it is written earlier in
 * the same call, so nothing needs clearing, but calls that overlap on the GPU
 * (different streams, or different host threads, at the same time) race on
 * it and must be ordered by the caller. */
mlsdc_status sh_inverse_static(int R, int nlon, int nlat, const double* spec, double* grid, int nf,
                               void* stream);

/* sh_forward: grid -> spectral, Eq. fourier_transform (with its 1/I) then
 * Eq. legendre_transform (Gaussian weights); Im of m = 0 set to zero.
 * grid: [nf][J][I]; spec: [nf][N_c] complex; 1 <= nf <= 16. */
mlsdc_status sh_forward(sh_plan_t plan, const double* grid, double* spec, int nf, void* stream);

/* swe_explicit_rhs: F_E = L_F + N (Sec. 4.1, Eq. system_of_odes_explicit_part)
 * of a state, by the transform method:
 *   F_E = [ -div(Phi' V), -div((zeta+f) V), curl((zeta+f) V) - lap(V.V/2) ].
 * state, FE: [3][N_c] complex (must not alias).  Uses the plan's precision. */
/* swe_explicit_rhs_batched: F_E of `members` states in one launch per stage
 * (states: [members][3][N_c], FE: the same layout; members <= the plan's
 * max_members).  Each member's result equals swe_explicit_rhs on it. */
mlsdc_status swe_explicit_rhs_batched(sh_plan_t plan, const swe_params* prm, const double* states, double* FE,
                                      int members, void* stream);
mlsdc_status swe_explicit_rhs(sh_plan_t plan, const swe_params* prm, const double* state,
                              double* FE, void* stream);

/* swe_implicit_rhs: F_I = L_G (Sec. 2, Eq.
 * linear_wave_motion_induced_by_gravitational_forces; Sec. 4.1):
 *   F_I = [ -Phibar delta + nu lap Phi', nu lap zeta, -lap Phi' + nu lap delta ].
 * Always float64.  state, FI: [3][N_c]; FI may alias state. */
mlsdc_status swe_implicit_rhs(sh_plan_t plan, const swe_params* prm, const double* state,
                              double* FI, void* stream);

/* swe_implicit_solve: x - alpha F_I(x) = b (Sec. 4.4, Eq. implicit_systems),
 * diagonal per coefficient: zeta = b_zeta / c, then the 2x2 (Phi', delta)
 * elimination, c = 1 + alpha nu n(n+1)/a^2.  alpha = dt * q~I_{m+1,m+1} >= 0.
 * b, x: [3][N_c]; x may alias b.  Always float64. */
mlsdc_status swe_implicit_solve(sh_plan_t plan, const swe_params* prm, double alpha,
                                const double* b, double* x, void* stream);

/* Options of the splitting F = F_I + F_E (Sec. 4.1).  0: the paper's split,
 * F_I = L_G, F_E = L_F + N.  MLSDC_CORIOLIS_IMPLICIT: the alternative with
 * the Coriolis terms implicit, F_I = L_G + L_F, F_E = N; L_F is the exact
 * spectral Coriolis operator (tridiagonal in n for each m, from the mu and
 * (1 - mu^2) d/dmu recurrences of the Legendre functions), and F_E is then
 * swe_explicit_rhs with Omega = 0. */
#define MLSDC_CORIOLIS_IMPLICIT 1

/* swe_implicit_rhs_ex: F_I of the splitting `options` (0: swe_implicit_rhs;
 * MLSDC_CORIOLIS_IMPLICIT: L_G + L_F).  state, FI: [3][N_c] float64; FI must
 * not alias state with MLSDC_CORIOLIS_IMPLICIT (L_F reads the neighbouring
 * degrees).  Unknown option bits: MLSDC_ERR_INVALID. */
mlsdc_status swe_implicit_rhs_ex(sh_plan_t plan, const swe_params* prm, const double* state,
                                 double* FI, int options, void* stream);

/* swe_implicit_solve_ex: x - alpha F_I(x) = b for the splitting `options`.
 * With MLSDC_CORIOLIS_IMPLICIT the system couples degrees n - 1, n, n + 1 of
 * each zonal wavenumber m: Phi' is eliminated per coefficient, and the rest
 * is two complex tridiagonal systems per m, (zeta_m, delta_{m+1}, zeta_{m+2}, ...)
 * and (delta_m, zeta_{m+1}, ...), factored by the Thomas algorithm (no
 * pivoting: the systems are diagonally dominant while 2 Omega alpha stays
 * well below 1, i.e. alpha below about 3000 s) and substituted by warp-wide
 * scans.  alpha >= 0; b, x: [3][N_c]; x may alias b.  Always float64; the
 * factor table is a stream-ordered allocation freed before return. */
mlsdc_status swe_implicit_solve_ex(sh_plan_t plan, const swe_params* prm, double alpha,
                                   const double* b, double* x, int options, void* stream);

/* ---------------------------------------------------------------------------
 * sdc_level: one space-time level: a plan, the physics, and n_nodes
 * Gauss-Lobatto nodes on [0, 1] with the collocation matrix Q (Sec. 4.2,
 * Eq. weights), the forward-Euler weights q~E and the LU-trick weights q~I
 * (q~I[1:,1:] = U^T where Q[1:,1:]^T = L U, Doolittle).  2 <= n_nodes <= 9.
 * The level keeps a pointer to the plan, which must outlive it.
 */
mlsdc_status sdc_level_create(sh_plan_t plan, const swe_params* prm, int n_nodes, sdc_level_t* out);
/* sdc_level_create_batched: a level advancing `members` ensemble members in
 * lockstep (members <= the plan's max_members).  Every state argument of
 * sdc_step / mlsdc_step on such a level is [members][3][N_c], and the node
 * arrays of sdc_sweep are [members][M+1][3][N_c]. */
mlsdc_status sdc_level_create_batched(sh_plan_t plan, const swe_params* prm, int n_nodes, int members,
                                      sdc_level_t* out);
/* sdc_level_create_ex: sdc_level_create_batched with a splitting `options`
 * (0 or MLSDC_CORIOLIS_IMPLICIT, see swe_implicit_solve_ex).  An
 * implicit-Coriolis level evaluates F_E with Omega = 0 and F_I = L_G + L_F;
 * its node updates solve the coupled system per wavenumber, with the chains
 * factored once per step size and node.  Both levels of an mlsdc_t must use
 * the same options; the adjoint (mlsdc_adjoint_create) accepts only 0. */
mlsdc_status sdc_level_create_ex(sh_plan_t plan, const swe_params* prm, int n_nodes, int members, int options,
                                 sdc_level_t* out);
mlsdc_status sdc_level_destroy(sdc_level_t lev);
/* Host copies of the node times t[n_nodes] and row-major Q, QE, QI [n_nodes^2]
 * (any pointer may be NULL). */
mlsdc_status sdc_level_matrices(sdc_level_t lev, double* t, double* Q, double* QE, double* QI);

/* sdc_sweep: one IMEX SDC sweep (Sec. 4.2, Eq.
 * update_equation_sdcq_discrete_form; with tau != NULL the coarse-level form
 * Eq. modified_update_equation_sdcq_discrete_form).  For m = 0..M-1 in order:
 * b = Theta[0] + dt sum_{j<=m} q~E_{m+1,j}(FE_new[j] - FE_old[j])
 *   + dt sum_{j<=m} q~I_{m+1,j}(FI_new[j] - FI_old[j]) - dt q~I_{m+1,m+1} FI_old[m+1]
 *   + dt sum_j q_{m+1,j}(FI_old[j] + FE_old[j]) + tau[m+1];
 * Theta[m+1] = implicit solve of b with alpha = dt q~I_{m+1,m+1};
 * FI_new[m+1] = F_I(Theta[m+1]); FE_new[m+1] = F_E(Theta[m+1]).
 * Theta: [M+1][3][N_c] in/out (node 0 is read only); FI_old, FE_old: inputs;
 * FI_new, FE_new: outputs (node 0 copied from the old arrays); tau:
 * [M+1][3][N_c] or NULL.  The old and new F arrays must not alias. */
mlsdc_status sdc_sweep(sdc_level_t lev, double dt, double* Theta, const double* FI_old,
                       const double* FE_old, double* FI_new, double* FE_new, const double* tau,
                       void* stream);

/* sdc_step: one step of single-level SDC(M+1, n_sweeps): Theta^n copied to
 * every node and F evaluated once (Sec. 4.3.2 initialisation), n_sweeps
 * sweeps, result = last node.  state: [3][N_c] in/out. */
mlsdc_status sdc_step(sdc_level_t lev, double* state, double dt, int n_sweeps, void* stream);

/* ---------------------------------------------------------------------------
 * mlsdc: two space-time levels (Sec. 4.3).  The coarse level must have
 * R_c <= R_f and nodes whose Lagrange transfer matrices Pi^c_f, Pi^f_c
 * (Sec. 4.3.3) are computed from the two node sets.  Both levels must
 * outlive the object.
 */
mlsdc_status mlsdc_create(sdc_level_t fine, sdc_level_t coarse, mlsdc_t* out);
mlsdc_status mlsdc_destroy(mlsdc_t ml);

/* mlsdc_step: one time step of two-level MLSDC: initialisation, then n_iter
 * iterations of Algorithm 1 -- A) fine sweep; B) restriction (time
 * interpolation Pi^c_f, then spectral truncation, Eqs. two_step_restriction,
 * time_restriction, space_restriction) and coarse F evaluation, saved;
 * C) FAS correction tau_c = A_c(R Theta_f) - R A_f(Theta_f) (Eq.
 * tau_term_level_l+1) and n_coarse_sweeps coarse sweeps; D) zero-pad and
 * Pi^f_c interpolation of the coarse corrections of Theta, F_I and F_E added
 * to fine nodes 1..M_f.  Result: the last fine node.
 * state: [3][N_c,fine] in/out.  With use_graph != 0 the launch sequence is
 * captured once into a CUDA graph per (state, dt, n_iter, n_coarse_sweeps)
 * and replayed on `stream` afterwards. */
mlsdc_status mlsdc_step(mlsdc_t ml, double* state, double dt, int n_iter, int n_coarse_sweeps,
                        int use_graph, void* stream);

/* Kernel launches issued by the last mlsdc_step / sdc_step call made without
 * a graph replay (a count of this library's kernels, for reporting). */
mlsdc_status mlsdc_launch_count(mlsdc_t ml, int64_t* launches);

/* ---------------------------------------------------------------------------
 * MLSDC on 2 <= L <= 8 space-time levels (levels[0] the finest; truncations
 * non-increasing, equal member counts and splitting options, no level twice).
 * The paper treats two levels (Algorithm 1) and leaves more for future work;
 * it describes the iteration as a V-cycle and writes the FAS term for any
 * pair of levels (Eq. tau_term_level_l+1, tau_{l+1} = A_{l+1}(R Theta_l)
 * - R A_l(Theta_l) + R tau_l).  One iteration here: a sweep on level 0; down,
 * for each pair, Algorithm 1's steps B and C (restrict nodes 1..M, evaluate,
 * save; FAS term with the restricted tau of the finer level; n_coarse_sweeps
 * sweeps); up, step D for each pair (interpolated corrections of Theta, F_I,
 * F_E), followed by one sweep on every intermediate level.  With two levels
 * this is exactly mlsdc_step.  The object keeps a level pair (the
 * mlsdc_create data) per consecutive levels; the levels must outlive it.
 * state: [members][3][N_c] of levels[0], in place; use_graph as mlsdc_step. */
mlsdc_status mlsdc_levels_create(const sdc_level_t* levels, int n_levels, mlsdc_levels_t* out);
mlsdc_status mlsdc_levels_destroy(mlsdc_levels_t h);
mlsdc_status mlsdc_levels_step(mlsdc_levels_t h, double* state, double dt, int n_iter, int n_coarse_sweeps,
                               int use_graph, void* stream);
mlsdc_status mlsdc_levels_launch_count(mlsdc_levels_t h, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Two-level PFASST, time-parallel MLSDC, on one GPU.  The paper names the
 * parallel full approximation scheme in space and time as the time-parallel
 * extension of MLSDC (Sec. 1, conclusions) without printing it; this is the
 * published two-level iteration built on Algorithm 1's steps.  P time slices
 * of length dt, slice p covering [t0 + p dt, t0 + (p+1) dt], are the P
 * members of the two batched levels (created with members = P; the coarse
 * plan with max_members >= P * coarse nodes evaluates every slice's coarse
 * nodes in one launch per stage, a smaller one node by node).  One call:
 *   predictor: every slice's fine nodes = u0; the coarse level runs serially
 *     over the slices (slice 0 from R u0, slice p from slice p-1's coarse end
 *     value; spread, n_predictor_sweeps sweeps); slices p >= 1 then start
 *     from u0 + zero-pad(their coarse initial value - R u0), spread;
 *   n_iter iterations of: fine initial value of slice p = slice p-1's fine
 *     end value from the previous iteration (F re-evaluated); one fine sweep
 *     of every slice (batched); restriction of fine nodes 0..M_c, coarse F,
 *     FAS term (batched); the coarse pipeline: slice after slice, coarse node
 *     0 = the previous slice's coarse end value of this iteration (F
 *     re-evaluated), n_coarse_sweeps sweeps with tau; interpolation of the
 *     coarse corrections to fine nodes 1..M_f (batched).
 * With P = 1 (and for slice 0 always) the result is mlsdc_step's; with
 * enough iterations every slice reaches the serial sequence of fine
 * collocation steps.  Only the paper's splitting; levels must outlive the
 * object.  u0: [3][N_c,fine] (device, read only); ends: [P][3][N_c,fine]
 * receives every slice's end value (ends[P-1] = the state at t0 + P dt).
 * n_predictor_sweeps < 0 means n_coarse_sweeps.  use_graph as mlsdc_step
 * (one graph per u0, ends, dt and iteration counts). */
mlsdc_status pfasst_create(sdc_level_t fine, sdc_level_t coarse, pfasst_t* out);
mlsdc_status pfasst_destroy(pfasst_t pf);
mlsdc_status pfasst_step(pfasst_t pf, const double* u0, double* ends, double dt, int n_iter, int n_coarse_sweeps,
                         int n_predictor_sweeps, int use_graph, void* stream);
mlsdc_status pfasst_launch_count(pfasst_t pf, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Ensembles of uneven truncation: one MLSDC object per truncation group
 * (each built on batched levels holding that group's members), stepped
 * together.  The groups' steps run on separate streams forked from `stream`
 * and joined back; with use_graph != 0 the whole fork/join is captured once
 * per (states, dt, n_iter, n_coarse_sweeps) into one CUDA graph with one
 * branch per group and replayed with a single graph launch.  The groups
 * must outlive the ensemble.  states: host array of ngroups device pointers,
 * group g's [members_g][3][N_c,g]. */
mlsdc_status mlsdc_ensemble_create(const mlsdc_t* groups, int ngroups, mlsdc_ensemble_t* out);
mlsdc_status mlsdc_ensemble_destroy(mlsdc_ensemble_t ens);
mlsdc_status mlsdc_ensemble_step(mlsdc_ensemble_t ens, double* const* states, double dt, int n_iter,
                                 int n_coarse_sweeps, int use_graph, void* stream);
mlsdc_status mlsdc_ensemble_launch_count(mlsdc_ensemble_t ens, int64_t* launches);

/* The same ensemble step as ONE persistent kernel launch (with two 4-byte
 * memsets) captured in a CUDA graph: the groups' launches of the step are
 * recorded once per (states, dt, n_iter, n_coarse_sweeps) and laid out as
 * phases (phase i = the i-th launch of every group's step; Algorithm 1,
 * Sec. 4.3.2, for all members), which one cooperative launch of one CTA per
 * SM runs with device-side synchronisation between phases (the schedule:
 * mlsdc_ensemble_persistent_schedule).  Every device wait is bounded (4 s of
 * the global timer): a wait that gives up ends the launch and leaves code 3
 * in mlsdc_ensemble_device_error.  Results: the same device code over the
 * same blocks as mlsdc_ensemble_step, so the same values up to the
 * compiler's own choices in the two compilations (measured: split-BF16
 * ensembles identical bit for bit, float64 ensembles within 6e-16, some
 * float64 products contracted into FMAs differently).  MLSDC_ERR_INVALID, with the reason in mlsdc_last_error(), for
 * implicit-Coriolis levels or a launch the kernel cannot host; a stream that
 * cannot capture the cooperative launch gets it launched directly. */
mlsdc_status mlsdc_ensemble_step_persistent(mlsdc_ensemble_t ens, double* const* states, double dt, int n_iter,
                                            int n_coarse_sweeps, void* stream);
/* Which schedule later persistent steps use (one graph per schedule):
 * 0 (the default) lockstep: every CTA meets every other at a grid barrier
 * after each phase; 1 dataflow: one ticket counter hands out the work items
 * of all recorded launches in phase order, and an item first waits (bounded,
 * code 3 on giving up) until the previous launch of its own group has
 * completed, so the groups advance through their phases independently, as
 * per-group streams do.  MLSDC_ERR_INVALID for other values. */
mlsdc_status mlsdc_ensemble_persistent_schedule(mlsdc_ensemble_t ens, int schedule);
/* Shape of the last persistent step: phases, recorded launches, CTAs of the
 * launch, and whether it runs from a graph.  MLSDC_ERR_INVALID before the
 * first persistent step.  Null outputs are skipped. */
mlsdc_status mlsdc_ensemble_persistent_info(mlsdc_ensemble_t ens, int* phases, int* records, int* ctas,
                                            int* in_graph);
/* Measurement utility: one more run of the last persistent step on `stream`
 * (synchronous), with CTA 0 reading the global timer at every phase
 * boundary: phase_us[p] = duration of phase p (microseconds), phase_body[p]
 * = the body (enum Body of the library's sources) of the phase's largest
 * recorded launch.  cap: room in both arrays (at least the phase count).
 * The step's states advance by one step.  Lockstep schedule only
 * (MLSDC_ERR_INVALID otherwise). */
mlsdc_status mlsdc_ensemble_persistent_phase_times(mlsdc_ensemble_t ens, float* phase_us, int* phase_body, int cap,
                                                   void* stream);
/* The persistent kernel's error word (sticky): 0, or 3 when a grid-barrier
 * wait gave up (synchronous read). */
mlsdc_status mlsdc_ensemble_device_error(mlsdc_ensemble_t ens, int* code);
/* Check of the grid barrier's bound: two CTAs wait at a barrier that
 * expects one arrival more than the grid makes, with a limit of timeout_ms
 * (1..2000); *code = 3 when the waits gave up and returned (synchronous).
 * Not a paper operation. */
mlsdc_status mlsdc_selftest_grid_barrier_timeout(int timeout_ms, int* code);

/* Stage timing of swe_explicit_rhs for roofline reporting: captures `reps`
 * back-to-back launches of each of the plan's F_E stage kernels into a CUDA
 * graph (as the step runs them), replays it once to warm up and once timed
 * with CUDA events on `stream`, and writes the mean milliseconds per launch of
 * [0] the Legendre synthesis, [1] the longitude FFT / grid-product kernel,
 * [2] the Legendre analysis to ms_host[3] (synchronises the stream).  Not a
 * paper operation: a measurement utility over the same kernels. */
mlsdc_status mlsdc_profile_rhs(sh_plan_t plan, const swe_params* prm, const double* state, double* FE,
                               int reps, float* ms_host, void* stream);
/* The same for a batch of `members` states ([members][3][N_c]) per launch. */
mlsdc_status mlsdc_profile_rhs_batched(sh_plan_t plan, const swe_params* prm, const double* states, double* FE,
                                       int members, int reps, float* ms_host, void* stream);
/* mlsdc_profile_node: device time of each node update of a level (the
 * update, implicit solve and F_I of node m + 1, Sec. 4.2 and Sec. 4.4; with
 * MLSDC_CORIOLIS_IMPLICIT the coupled per-wavenumber solve), on the level's
 * own node arrays as the last sweep left them: ms_out[m], m = 0..n_nodes-2,
 * is the mean of `reps` back-to-back launches timed with CUDA events on
 * `stream`.  Overwrites nodes 1..M of the level's current arrays (no step's
 * result lives there).  Synchronises the stream. */
mlsdc_status mlsdc_profile_node(sdc_level_t lev, double dt, int reps, float* ms_out, void* stream);

/* ---------------------------------------------------------------------------
 * Adjoint (reverse mode) of the MLSDC time step with respect to its initial
 * state, float64, single member.  Inner product: a state is the real vector
 * of the (Re, Im) parts of its stored coefficients, <x, y> = sum Re(conj(x) y);
 * Im of m = 0 is not a degree of freedom (the fields are real, Sec. 3), so
 * every adjoint returned has it zero and every adjoint passed in is
 * projected (that part dropped).  This is the convention of PyTorch's
 * complex gradients (dL/dRe + i dL/dIm for a real L).
 *
 * Only F_E is nonlinear; every other operation of a step (Sec. 4.2 node
 * update, Sec. 4.4 implicit solve and F_I, Sec. 4.3.3 transfers, the FAS
 * correction of Algorithm 1 step C) is linear with constant coefficients.
 * The step is a fixed list of operations; its adjoint applies their
 * transposes in reverse order, with F_E replaced by the transpose of its
 * Jacobian at the input the forward step recorded.
 *
 * swe_explicit_rhs_adjoint: state_bar += F_E'(state)^t lambda, and lambda
 * is set to zero (its value consumed).  state, lambda, state_bar: [3][N_c],
 * pairwise distinct.  Needs an MLSDC_FP64 plan (one member).
 */
mlsdc_status swe_explicit_rhs_adjoint(sh_plan_t plan, const swe_params* prm, const double* state,
                                      double* lambda, double* state_bar, void* stream);

/* mlsdc_phi_misfit: J = 1/2 ||Phi'(state) - phi_target||^2 in the Parseval
 * norm of Sec. 3 (sum |.|^2 over m = 0 plus twice over m >= 1, which equals
 * 1/2 (1/I) sum_{i,j} w_j (Phi - Phi_t)^2 on the grid), written to the
 * device double *J, and its gradient lambda = dJ/dstate ([3][N_c]: the
 * weighted residual in the Phi' field, zeta and delta zero).  phi_target:
 * [N_c] complex. */
mlsdc_status mlsdc_phi_misfit(sh_plan_t plan, const double* state, const double* phi_target, double* J,
                              double* lambda, void* stream);

/* mlsdc_adjoint_create: a reverse-mode driver for n_steps steps of
 * mlsdc_step(ml, ., dt, n_iter, n_coarse_sweeps) that stores the state every
 * checkpoint_every steps (>= 1; n_steps/checkpoint_every states) and, during
 * the backward pass, recomputes one segment of checkpoint_every steps at a
 * time, recording that segment's F_E inputs, then walks it backwards.  Device
 * memory: the checkpoints, checkpoint_every steps of F_E inputs, and one
 * adjoint copy of every buffer a step uses.  The MLSDC object (float64 plans,
 * one member) must outlive the adjoint object and shares its buffers: order calls
 * on one stream. */
mlsdc_status mlsdc_adjoint_create(mlsdc_t ml, int n_steps, int checkpoint_every, double dt, int n_iter,
                                  int n_coarse_sweeps, mlsdc_adjoint_t* out);
mlsdc_status mlsdc_adjoint_destroy(mlsdc_adjoint_t adj);
/* mlsdc_adjoint_forward: state_T = n_steps MLSDC steps from state0 ([3][N_c]
 * each; may alias), storing the checkpoints.  The same arithmetic as
 * mlsdc_step. */
mlsdc_status mlsdc_adjoint_forward(mlsdc_adjoint_t adj, const double* state0, double* state_T, int use_graph,
                                   void* stream);
/* mlsdc_adjoint_backward: lambda_0 = (d state_T / d state0)^t lambda_T for
 * the trajectory of the last mlsdc_adjoint_forward call (MLSDC_ERR_INVALID
 * if there was none).  lambda_T, lambda_0: [3][N_c] (may alias).  With
 * use_graph != 0 each recomputed step and each reverse step is one CUDA graph
 * launch (captured on first use). */
mlsdc_status mlsdc_adjoint_backward(mlsdc_adjoint_t adj, const double* lambda_T, double* lambda_0, int use_graph,
                                    void* stream);
/* Stage timing of swe_explicit_rhs_adjoint (as mlsdc_profile_rhs): mean ms
 * per launch of [0] the Legendre sums of state and adjoint, [1] the FFT /
 * grid-point transpose kernel, [2] the unweighted Gaussian sums.  lambda is
 * consumed (zeroed) by the first evaluation; a measurement utility. */
mlsdc_status mlsdc_profile_rhs_adjoint(sh_plan_t plan, const swe_params* prm, const double* state, double* lambda,
                                       double* state_bar, int reps, float* ms_host, void* stream);
/* Kernel launches of one forward step and of one reverse step (reporting). */
mlsdc_status mlsdc_adjoint_launch_count(mlsdc_adjoint_t adj, int64_t* forward_step, int64_t* reverse_step);

/* Device check that a state (n doubles) is finite: writes 1 to *ok_host if
 * every value is finite, else 0 (synchronises the stream). */
mlsdc_status mlsdc_check_finite(const double* state, int64_t n, int* ok_host, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLSDC_SH_H */
