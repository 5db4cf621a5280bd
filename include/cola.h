/*
 * cola.h -- C ABI of the GB300 (sm_103a) COLA hot path.
 *
 * COLA (COmoving Lagrangian Acceleration; Tassev, Zaldarriaga & Eisenstein 2013,
 * arXiv:1301.0322) evolves particles of a periodic box in the frame comoving with their
 * second-order Lagrangian perturbation theory (2LPT) trajectories:
 *     x = q + s,  s_res = s - D1 s1 - D2 s2                                   (App. A.3)
 *     T^2[s_res] = -(3/2) Om a d_x d_x^-2 delta - T^2[D1] s1 - T^2[D2] s2      (eq. eomALC)
 * with the modified Kick/Drift operators of eq. KDKALC (u(a) = a^nLPT) applied in the order
 * of eq. ALCtimestep and the frame changes L-/L+ of eq. Lops.  The force is a particle-mesh
 * (PM) force on a periodic mesh (Sec. 2).
 *
 * Conventions shared by every call
 *  - Particles live on an np^3 Lagrangian lattice, q = L (ix, iy, iz) / np, particle index
 *    p = (iz np + iy) np + ix.  Per-particle vectors are structure-of-arrays float32 [3][np^3]
 *    (all x components, then y, then z).  Meshes are float32 or int64 [iz][iy][ix], ng^3.
 *  - "s" is the displacement of eq. eom (x = q + s, positions taken modulo L); "v" is the
 *    velocity T[s] (the residual velocity v_res between L- and L+, App. A.3).
 *  - All array pointers are DEVICE pointers owned by the caller; the library never allocates
 *    device memory.  It needs one caller-allocated workspace (cola_workspace_bytes,
 *    cola_set_workspace) that holds its meshes, tables and sort buffers.
 *  - Calls are asynchronous on the given CUDA stream (cola_stream = cudaStream_t; NULL = the
 *    legacy default stream).  Host-side argument errors return immediately; errors found by a
 *    kernel are latched in the workspace and reported by cola_status.
 *  - Return codes: COLA_OK or one of the COLA_E* values below; cola_last_error() gives a
 *    message for the calling thread.  No C++ exception crosses this boundary.
 *  - A plan is not thread-safe: calls on one plan must be serialised by the caller (calls on
 *    different plans with different workspaces are independent).
 */
#ifndef COLA_GB300_H
#define COLA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COLA_OK 0
#define COLA_EINVAL 1          /* bad argument (size, pointer, range)                      */
#define COLA_ECUDA 2           /* a CUDA runtime call failed                               */
#define COLA_EOVERFLOW 3       /* a device check failed (fixed-point overflow, non-finite) */
#define COLA_EUNSUPPORTED 4    /* mesh or lattice size without an FFT kernel               */
#define COLA_ENOWORKSPACE 5    /* cola_set_workspace has not been called                   */
#define COLA_ETIMEOUT 6        /* a kernel's bounded wait on its asynchronous copies ran out */

#define COLA_NCOEF 16 /* columns of the cola_coeffs table */

typedef void* cola_stream; /* cudaStream_t */
typedef struct cola_plan cola_plan;

/* Background cosmology (flat or curved LCDM without radiation) and the linear spectrum. */
typedef struct {
  double omega_m;  /* matter density today (eq. eom: Om)                               */
  double omega_l;  /* cosmological constant; curvature 1 - Om - OL enters H(a)         */
  double h;        /* H0 / (100 km/s/Mpc), enters the BBKS shape Gamma = Om h          */
  double sigma8;   /* rms linear density in 8 Mpc/h top hats at a = 1                  */
  double n_s;      /* primordial spectral index                                        */
} cola_cosmo;

/* One simulation: lattice, mesh, box, cosmology and the time stepping of App. A.3. */
typedef struct {
  int64_t np;         /* particles per side; np^3 particles                                 */
  int64_t ng;         /* PM mesh cells per side (Sec. 2 uses ng = 3 np)                       */
  double box;         /* periodic box side L in Mpc/h                                         */
  cola_cosmo cosmo;
  double n_lpt;       /* u(a) = a^nLPT of eq. KDKALC; the paper uses -2.5 (App. A.3.2)        */
  int32_t nsteps;     /* number of time steps, uniform in a (App. A.3.2)                      */
  double a_init;      /* initial scale factor (z = 9 -> 0.1 in Sec. 2)                        */
  double a_final;     /* final scale factor (1.0)                                            */
  int32_t deconv;     /* CIC deconvolution power p in 1/W(k)^p of the force: 0, 1 (default), 2 */
  int32_t fixed_bits; /* F: CIC positions are quantised to 2^-F cell (default 16, 8..20)      */
  int32_t adjoint;    /* 1: also reserve the workspace of cola_step_adjoint (3 more meshes)      */
  int32_t scheme;     /* Kick/Drift operators, one of COLA_SCHEME_* below (default COLA)         */
  int32_t log_a;      /* 0: steps uniform in a (default, App. A.3.2); 1: uniform in ln a (App. A.2) */
} cola_config;

/* Time integrators (cola_config.scheme).  All use the merged Kicks of eq. ALCtimestep.
 *  COLA_SCHEME_COLA     eq. KDKALC, u = a^nLPT in Kick and Drift (the paper's optimal variant)
 *  COLA_SCHEME_COLA_STD eq. KDKALCstd: the LPT frame with the standard coefficients
 *                       int (a/a_c)/Q da (Kick) and int da/Q (Drift)
 *  COLA_SCHEME_PM       eq. KDKStd: standard PM leapfrog, no LPT frame (s1, s2 only set the
 *                       2LPT initial conditions; v starts at T[D1] s1 + T[D2] s2, no L+-)
 *  COLA_SCHEME_COLA_U1  eq. KDKALC with u = 1 in the Drift, u = a^nLPT in the Kick (the
 *                       footnote on u = A + B a^nLPT, App. A.3.2)
 * The mid-point scale factor is a_{i+1/2} = (a_i + a_{i+1}) / 2 on either grid (App. A.2). */
#define COLA_SCHEME_COLA 0
#define COLA_SCHEME_COLA_STD 1
#define COLA_SCHEME_PM 2
#define COLA_SCHEME_COLA_U1 3

/* Fill *cfg with the 32^3-particle / 64^3-mesh defaults (L = 100 Mpc/h, Om = 0.27, OL = 0.73,
 * h = 0.7, sigma8 = 0.8, ns = 0.96, nLPT = -2.5, 10 steps uniform in a from a = 0.1 to 1,
 * deconv 1, F 16, scheme COLA). */
int cola_config_default(cola_config* cfg);

/* Validate cfg and build a plan: float64 growth factors and step coefficients on the host
 * (App. A.3), FFT twiddle tables.  np and ng must be in {32, 48, 64, 96, 128, 192, 256, 384,
 * 512, 768, 1024, 1536, 2048} (COLA_EUNSUPPORTED otherwise), ng a multiple of 4.  Host memory
 * only.  *out receives the plan; destroy it with cola_plan_destroy. */
int cola_plan_create(const cola_config* cfg, cola_plan** out);
int cola_plan_destroy(cola_plan* plan);

/* Device workspace the plan needs, in bytes (meshes, sort bins, tables). */
int cola_workspace_bytes(const cola_plan* plan, size_t* bytes);

/* Hand the plan a device buffer of at least cola_workspace_bytes bytes, 256-byte aligned.
 * The caller keeps ownership and must keep it alive while the plan is used.  The twiddle
 * and coefficient tables are copied into it on `stream`. */
int cola_set_workspace(cola_plan* plan, void* dev_ptr, size_t bytes, cola_stream stream);

/* Host float64 table of the per-force-evaluation coefficients, (nsteps+1) rows x COLA_NCOEF:
 *  0 a_i (force time)           1 (3/2) Om a_i             2 c_K = (u(kb)-u(ka))/T[u](a_i)
 *  3 T^2[D1](a_i)               4 T^2[D2](a_i)             5 c_D = int_{a_i}^{a_i+1} u/Q da / u(a_i+1/2)
 *  6 D1(a_i+1)-D1(a_i)          7 D2(a_i+1)-D2(a_i)        8 T[D1](a_i)
 *  9 T[D2](a_i)                10 D1(a_i)                 11 D2(a_i)
 * 12 ka (kick start)           13 kb (kick end)           14 a_i+1 (0 on the last row)
 * 15 D2u(1), the 2LPT normalisation s2 = D2u(1) psi2.
 * Row i merges K(a_i-1/2, a_i; a_i) K(a_i, a_i+1/2; a_i) of eq. ALCtimestep (ka = a_0 on the
 * first row, kb = a_n on the last); rows i < nsteps also carry D(a_i, a_i+1; a_i+1/2).
 * table must hold (nsteps+1)*COLA_NCOEF doubles. */
int cola_coeffs(const cola_plan* plan, double* table);

/* Unit-variance Gaussian white noise on the np^3 lattice: Philox4x32-10 (Salmon et al. 2011)
 * with key = seed, counter block = cell / 4, Box-Muller on ((r >> 8) + 1) 2^-24 uniforms.
 * noise: device float32 [np^3].  (The paper's initial conditions are Gaussian, Sec. 2.) */
int cola_noise(cola_plan* plan, uint64_t seed, float* noise, cola_stream stream);

/* 2LPT initial conditions at a_init (Sec. 2; App. A.3):
 *   delta_k = w_k sqrt(P(k) np^3 / L^3) (BBKS P normalised to sigma8, k = 0 removed),
 *   s1 = i k delta_k / k^2, s2 = D2u(1) * (-i k mu2_k / k^2) with
 *   mu2 = sum_{i<j} (s1_i,i s1_j,j - s1_i,j^2), derivatives zero on their Nyquist plane;
 *   s = D1(a_init) s1 + D2(a_init) s2 and v = 0 (the 2LPT velocity after L-(a_init), eq. Lops).
 * noise: device float32 [np^3] (read only).  s, v, s1, s2: device float32 [3][np^3] outputs. */
int cola_ic_2lpt(cola_plan* plan, const float* noise, float* s, float* v, float* s1, float* s2,
                 cola_stream stream);

/* Force evaluation `step` (0..nsteps) of eq. ALCtimestep at a_step, in place on (s, v):
 * PM force at the current positions, Kick from ka to kb with a_c = a_step, then (step < nsteps)
 * Drift from a_step to a_step+1 with a_c = a_step+1/2 (eq. KDKALC), or (step == nsteps) L+.
 * s, v: device float32 [3][np^3], read and written; s1, s2: device float32 [3][np^3]. */
int cola_step(cola_plan* plan, int32_t step, float* s, float* v, const float* s1, const float* s2,
              cola_stream stream);

/* The unit PM force g = -d_x d_x^-2 delta at the particles (eq. eom without (3/2) Om a),
 * CIC deposit -> FFT -> i k_j / (k^2 W^p) -> inverse FFT -> CIC gather.
 * s: device float32 [3][np^3]; g: device float32 [3][np^3] output. */
int cola_force(cola_plan* plan, const float* s, float* g, cola_stream stream);

/* Reverse-mode derivatives (the paper has none; these are the exact transposes of the
 * forward calls, with the CIC weights differentiated almost everywhere at the forward path's
 * quantised positions).  They propagate adjoints lam_* = dLoss/d(*) backwards:
 *
 * cola_step_adjoint: transpose of cola_step(step).  s_ckpt: the displacements cola_step(step)
 * started from (device float32 [3][np^3], read only).  On entry lam_s, lam_v hold the adjoints
 * of the step's outputs (s, v); on exit, of its inputs.  lam_s1, lam_s2 accumulate (+=) the
 * adjoints of s1, s2.  Needs a plan created with cola_config.adjoint = 1 (COLA_EINVAL
 * otherwise).  Run it for step = nsteps .. 0 with the matching checkpoints.
 *
 * cola_density_adjoint: lam_s = (d delta / d s)^T delta_bar for the float density of
 * cola_density (delta_bar: device float32 [ng^3]; lam_s: device float32 [3][np^3], written).
 *
 * cola_ic_2lpt_adjoint: transpose of cola_ic_2lpt.  lam_s: adjoint of the initial s (read);
 * lam_s1, lam_s2: the accumulated adjoints of s1, s2 (read and overwritten: they get
 * lam_s's D1(a_init), D2(a_init) share added); grad_noise: device float32 [np^3], the
 * derivative with respect to the white noise (written). */
int cola_step_adjoint(cola_plan* plan, int32_t step, const float* s_ckpt, float* lam_s, float* lam_v, float* lam_s1,
                      float* lam_s2, cola_stream stream);
int cola_density_adjoint(cola_plan* plan, const float* s, const float* delta_bar, float* lam_s, cola_stream stream);
int cola_ic_2lpt_adjoint(cola_plan* plan, const float* noise, const float* lam_s, float* lam_s1, float* lam_s2,
                         float* grad_noise, cola_stream stream);

/* CIC density of the particles at displacements s (Sec. 3.1 analysis; the deposit of the
 * force).  rho_fix (may be NULL): device int64 [ng^3], sum of integer CIC weights with
 * positions quantised to 2^-F cell (sum = np^3 2^3F exactly); delta (may be NULL): device
 * float32 [ng^3], rho_fix ng^3 / (np^3 2^3F) - 1. */
int cola_density(cola_plan* plan, const float* s, int64_t* rho_fix, float* delta, cola_stream stream);

/* Shell-averaged power spectrum of a density mesh (Sec. 3.1): P = (L^3/ng^6) |delta_k|^2 /
 * W(k)^2 averaged over shells (b - 1/2) k_F <= |k| < (b + 1/2) k_F, b = 1..nbins.
 * delta: device float32 [ng^3] (read only); k, pk: device float64 [nbins]; nmodes: device
 * int64 [nbins].  nbins <= ng. */
int cola_power(cola_plan* plan, const float* delta, int32_t nbins, double* k, double* pk,
               int64_t* nmodes, cola_stream stream);

/* The power spectrum of cola_power of the CIC density of cola_density at displacements s (Sec.
 * 3.1), without a caller-owned mesh: the transform of the density goes to the plan's force
 * meshes, which hold nothing between calls that write them (the next force evaluation rebuilds
 * them), through the force evaluation's fused deposit and real-to-complex pass.  The same
 * arithmetic as cola_density + cola_power, so the same k, pk, nmodes bit for bit.
 * s: device float32 [3][np^3] (read only); k, pk: device float64 [nbins]; nmodes: device int64
 * [nbins]; nbins <= ng. */
int cola_density_power(cola_plan* plan, const float* s, int32_t nbins, double* k, double* pk, int64_t* nmodes,
                       cola_stream stream);

/* Cross-correlation of two density meshes (Sec. 3.1) and n_max (eq. nmax, App. B), for
 * comparing a run with a reference run of the same initial conditions.  Per shell
 * b = 1..nbins (the shells and weights of cola_power): k, P_a and P_b as cola_power,
 * P_ab = (L^3/ng^6) Re(delta_a,k delta_b,k^*) / W(k)^2 averaged over the shell,
 * rho = P_ab / sqrt(P_a P_b) (read with the square root, as App. B uses it) and
 * nmax = (2/3) rho / sqrt(1 - rho^2) (+inf where rho = 1).  delta_a, delta_b: device float32
 * [ng^3] (read only); k, pk_a, pk_b, pk_ab, rho, nmax: device float64 [nbins]; nmodes: device
 * int64 [nbins].  nbins <= ng.  Deterministic (fixed reduction order). */
int cola_cross_power(cola_plan* plan, const float* delta_a, const float* delta_b, int32_t nbins, double* k,
                     double* pk_a, double* pk_b, double* pk_ab, double* rho, double* nmax, int64_t* nmodes,
                     cola_stream stream);

/* Friends-of-friends halo groups (Sec. 3.2: linking length 0.2, at least 25 particles) of the
 * particles at displacements s (device float32 [3][np^3], read only).  Positions are the
 * fixed-point CIC coordinates of the force (2^-F cell); two particles are friends iff their
 * periodic minimum-image distance d satisfies d < b s_mean, s_mean = (ng/np) 2^F, b =
 * b_num / b_den (1 <= b_num <= b_den <= 50; the paper's b = 1/5), tested exactly in integers
 * (b_den^2 d^2 < b_num^2 s_mean^2), so the groups are unique.  Outputs (device, may be NULL
 * but not both): group [np^3] int32 = the smallest particle index of the particle's group if
 * the group has at least nmin particles, else -1; size [np^3] int32 = the size of its group.
 * Mass function: n_ge (device int64 [nthr]) = the number of halos (groups >= nmin) with at
 * least thresholds[k] (host int32 [nthr], nthr <= 32) particles.  Needs ng a multiple of np;
 * uses the plan's mesh buffers as scratch (their contents are lost).  A union-find that runs
 * out of retries latches COLA_ETIMEOUT for cola_status. */
int cola_fof(cola_plan* plan, const float* s, int32_t b_num, int32_t b_den, int32_t nmin, int32_t* group,
             int32_t* size, int32_t nthr, const int32_t* thresholds, int64_t* n_ge, cola_stream stream);

/* Retry limit of the friends-of-friends union-find (this library's bounded loop; the paper has
 * no counterpart): each union of two roots is attempted at most `tries` times (compare-and-swap
 * rounds against concurrent unions) before cola_fof gives up on it and latches COLA_ETIMEOUT.
 * Default 2^20.  tries = 0 makes every union give up at once, so that the failure path can be
 * exercised without a fault: a run either reports COLA_ETIMEOUT through cola_status or its
 * groups are exact.  0 <= tries <= 2^30 (COLA_EINVAL otherwise).  Host only; takes effect at the
 * next cola_fof call on this plan. */
int cola_set_fof_union_tries(cola_plan* plan, int32_t tries);

/* Forward 3-D real-to-complex DFT (exp(-i k.x), unscaled) of a real mesh of side n, where
 * n is the plan's ng (which = 0) or np (which = 1).  in: device float32 [n^3]; out: device
 * complex64 [n][n][n/2+1] (interleaved re, im). */
int cola_fft_r2c(cola_plan* plan, int32_t which, const float* in, float* out, cola_stream stream);

/* Synchronise `stream` and report errors latched by kernels since the last call
 * (COLA_EOVERFLOW for a fixed-point overflow or a non-finite position, COLA_ETIMEOUT if a
 * kernel stopped waiting for its bulk copies), then clear them. */
int cola_status(cola_plan* plan, cola_stream stream);

/* cola_power without a plan, a workspace or any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate device memory
 * themselves -- code hosted inside an application whose own pool allocator owns all device
 * memory (where cudaMalloc/cudaFree are off limits and would synchronise the device), or a
 * monitor attached to a running simulation that must not change its memory footprint.
 * Same result as cola_power on a plan with this ng and box: P(k) of the float32 density
 * delta [ng^3] in shells b = 1..nbins, written to the caller's device arrays k, pk (float64)
 * and nmodes (int64).  Its scratch is one static device array sized for ng <= 128 (about
 * 10.7 MiB held on every GPU that loads the library until the process exits); ng > 128 is
 * rejected with COLA_EINVAL, sizes other than 32, 48, 64, 96 and 128 with COLA_EUNSUPPORTED.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress), and the first call for each
 * mesh size on a device uploads that size's twiddle table into the array (a synchronous copy);
 * make those first calls before any stream capture on the device.  Every call shares the one
 * array and leaves its contents behind (each call overwrites every partial sum it reads), so
 * calls that overlap on the GPU -- on different streams or from different threads -- race and
 * must be serialised by the caller. */
#define COLA_NOALLOC_MAX_NG 128
int cola_power_noalloc(const float* delta, int32_t ng, double box, int32_t nbins, double* k, double* pk,
                       int64_t* nmodes, cola_stream stream);

/* ---- Ensembles of independent boxes -------------------------------------------------------
 * An ensemble evolves nbox independent realisations -- boxes of different np, ng and L, the
 * mock catalogues that motivate COLA's speed (Sec. 1, Sec. 4) -- with one launch per kernel
 * class per force evaluation for all boxes together: persistent kernels walk a work list of
 * (box, tile) items, so small boxes do not leave the GPU idle and there is no per-box launch
 * cost.  Each step (cola_ensemble_step) is recorded once as a CUDA graph and replayed.
 *
 * Every box follows eq. ALCtimestep exactly as a single-box plan with the same cola_config
 * does: the per-box results are those of cola_step on that box alone.
 *
 * Layout: the per-box particle arrays are concatenated.  Box b owns particles
 * [poff[b], poff[b+1]) of the ensemble (poff from cola_ensemble_offsets, poff[b+1] - poff[b]
 * = np_b^3); a [3][np^3] SoA array of box b starts at element 3 poff[b] of the ensemble array
 * (s, v, s1, s2), a scalar per-particle array (noise) at element poff[b], and a density mesh
 * at element moff[b] (moff[b+1] - moff[b] = ng_b^3).
 *
 * Requirements: 1 <= nbox <= 4096; every box has the same nsteps; ng in {64, 96, 128, 192,
 * 256}; the total particle count below 2^31.  Other fields are free per box. */
typedef struct cola_ensemble cola_ensemble;

/* Tunable launch shape of the ensemble step (chosen by cola_ensemble_tune):
 *  threads       block size of every persistent kernel, 128 or 256; it fixes the FFT
 *                columns per block (threads / (n / E)) and the deposit tile rows
 *  tile_shape    deposit tile (y x z rows) for a given row count: 0 = 4x2, 4x4, 8x4, 8x8,
 *                16x8 for 8, 16, 32, 64, 128 rows; 1 = 2x4, 8x2, 4x8, 16x4, 8x16.  Tiles are
 *                also the particle bins.
 *  blocks_per_sm persistent grid = blocks_per_sm x SM count, capped by occupancy; 0 = the
 *                occupancy limit
 *  radix         FFT factorisation of every transform length: 0 = the single-box one
 *                (e.g. 256 = 16 x 16, 16 elements per thread), 1 = a second one with another
 *                number of elements per thread (256 = 8 x 8 x 4, 8 per thread).  Variant 0
 *                reproduces the single-box results bit for bit; variant 1 rounds differently
 *                (same transforms, another order of operations).
 *  launch        0 = the multi-box persistent kernels above (one launch per kernel class and
 *                force evaluation for all boxes); 1, 2 or 4 = every box's own single-box
 *                launches, the boxes dealt round-robin over that many streams forked inside
 *                the step graph, one box after another on each (threads, tile_shape,
 *                blocks_per_sm and radix are then unused; the results equal the single-box
 *                ones bit for bit).  Either way each step is replayed from a CUDA graph.
 *  mesh_streams  launch 0 only: 0 = the mesh passes as multi-box kernels too; 1, 2 or 4 =
 *                hybrid: the binning (keys, scan, scatter), the gather and the kick/drift stay
 *                multi-box launches for all boxes, and each box runs its own single-box mesh
 *                passes (deposit + x r2c .. inverse x) from the ensemble's records, the boxes
 *                dealt round-robin over that many streams forked inside the step graph (the
 *                bins then follow each box's plan; the results equal the single-box ones bit
 *                for bit). */
typedef struct {
  int32_t threads;
  int32_t tile_shape;
  int32_t blocks_per_sm;
  int32_t radix;
  int32_t launch;
  int32_t mesh_streams;
} cola_ensemble_tuning;

#define COLA_ENSEMBLE_TUNE_CANDIDATES 25

/* Create / destroy.  boxes: host array of nbox configurations (see the requirements above). */
int cola_ensemble_create(const cola_config* boxes, int32_t nbox, cola_ensemble** out);
int cola_ensemble_destroy(cola_ensemble* ens);
/* Bytes of device workspace (all boxes' meshes and tables, the shared sort buffers). */
int cola_ensemble_workspace_bytes(const cola_ensemble* ens, size_t* bytes);
/* Attach a caller-owned device workspace (256-byte aligned, >= the size above) and upload the
 * tables on `stream`.  Also creates the library's private capture stream. */
int cola_ensemble_set_workspace(cola_ensemble* ens, void* dev_ptr, size_t bytes, cola_stream stream);
/* Host arrays of nbox + 1 entries: poff (particle offsets) and moff (mesh-cell offsets). */
int cola_ensemble_offsets(const cola_ensemble* ens, int64_t* poff, int64_t* moff);
/* The four calls below and cola_ensemble_step run as CUDA graphs: recorded on the library's
 * capture stream the first time they see a set of pointers (and seeds, nbins), replayed on
 * `stream` afterwards (cola_ensemble_use_graphs(ens, 0) or profiling issues the launches
 * directly). */
/* Philox white noise of every box (cola_noise with seeds[b] into noise + poff[b]). */
int cola_ensemble_noise(cola_ensemble* ens, const uint64_t* seeds, float* noise, cola_stream stream);
/* 2LPT initial conditions of every box (cola_ic_2lpt on each box's slices). */
int cola_ensemble_ic_2lpt(cola_ensemble* ens, const float* noise, float* s, float* v, float* s1, float* s2,
                          cola_stream stream);
/* One step of eq. ALCtimestep (cola_step semantics, step = 0..nsteps) for every box: 11
 * kernel launches in total (binning 5, fused mesh passes 5, gather + kick + drift 1), replayed
 * from a CUDA graph recorded on the first call with these pointers and this tuning. */
int cola_ensemble_step(cola_ensemble* ens, int32_t step, float* s, float* v, const float* s1, const float* s2,
                       cola_stream stream);
/* CIC overdensity of every box: delta + moff[b] receives box b's mesh (cola_density). */
int cola_ensemble_density(cola_ensemble* ens, const float* s, float* delta, cola_stream stream);
/* P(k) of every box (cola_power); box b writes rows [b nbins, (b+1) nbins) of k, pk, nmodes.
 * nbins <= the smallest ng of the ensemble. */
int cola_ensemble_power(cola_ensemble* ens, const float* delta, int32_t nbins, double* k, double* pk,
                        int64_t* nmodes, cola_stream stream);
/* Autotuner: times one force evaluation without the particle update (binning, mesh passes and
 * the gather into scratch) of all boxes at displacements s (read only), replayed from a CUDA
 * graph as the steps are (launched directly if cola_ensemble_use_graphs(ens, 0)), for each of
 * the COLA_ENSEMBLE_TUNE_CANDIDATES launch shapes (reps timed
 * repetitions after one warm-up, CUDA events on `stream`; synchronises), keeps the fastest
 * and writes it to *best (may be NULL).  ms (may be NULL): host array receiving the mean
 * milliseconds of each candidate: first the 16 multi-box shapes (launch 0) in the order
 * threads in {128, 256} x tile_shape in {0, 1} x blocks_per_sm in {0, 2} x radix in {0, 1}
 * (radix fastest), then launch 1, 2 and 4, then the hybrid mode with mesh_streams in {1, 2, 4}
 * x threads in {128, 256} (threads fastest).  Candidates with radix 0, the per-box and the
 * hybrid ones give results bit-identical to the single-box runs. */
int cola_ensemble_tune(cola_ensemble* ens, const float* s, int32_t reps, cola_ensemble_tuning* best, double* ms,
                       cola_stream stream);
int cola_ensemble_get_tuning(const cola_ensemble* ens, cola_ensemble_tuning* tuning);
int cola_ensemble_set_tuning(cola_ensemble* ens, const cola_ensemble_tuning* tuning, cola_stream stream);
/* Graph replay on (1, default) or off (0: every launch issued directly; used while profiling). */
int cola_ensemble_use_graphs(cola_ensemble* ens, int32_t enable);
/* cola_status over all boxes: the first box with a latched error decides the code. */
int cola_ensemble_status(cola_ensemble* ens, cola_stream stream);
/* Measurement hooks as cola_profile / cola_profile_read, for the ensemble's own kernels (the
 * step runs without graphs while profiling is on). */
int cola_ensemble_profile(cola_ensemble* ens, int32_t enable);
int cola_ensemble_profile_read(cola_ensemble* ens, int32_t max_entries, char* names, int64_t* launches, double* ms,
                               int32_t* count);

/* Measurement hooks (not part of the method).  cola_profile(plan, 1) makes every kernel the
 * plan's calls launch record a CUDA event pair on the launching stream; cola_profile_read
 * synchronises those events and returns, per kernel name (NUL-terminated, 64 bytes each in
 * `names`), the launch count and total milliseconds, then clears the records.  At most
 * max_entries kernels are returned; *count receives how many. */
int cola_profile(cola_plan* plan, int32_t enable);
int cola_profile_read(cola_plan* plan, int32_t max_entries, char* names, int64_t* launches, double* ms,
                      int32_t* count);

/* Process-wide number of kernels this library has launched (all plans, all threads). */
int cola_launch_count(uint64_t* count);

/* Message of the last failing call on this thread ("" if none). */
const char* cola_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* COLA_GB300_H */
