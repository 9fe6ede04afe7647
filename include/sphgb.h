/*
 * sphgb.h -- C ABI of the GB300 (sm_103a) self-gravitating SPH right-hand
 * side of Khrapov & Khoperskov, "Smoothed-Particle Hydrodynamics Models:
 * Implementation Features on GPUs" (arXiv:1807.08116).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* or documented as "device" are CUDA device pointers
 *    owned by the caller; the library never frees or reallocates them and
 *    never calls cudaMalloc.  Host pointers are named h_* or documented.
 *  - Particle arrays are in the caller's ("original") order, gas particles
 *    first: indices [0, n_gas) are gas (SPH), [n_gas, n) are collisionless.
 *  - float4 arrays are passed as float* with 4 floats per particle (16-byte
 *    aligned); FP64 vectors are structure-of-arrays: r[3*n] holds x[0..n),
 *    y[0..n), z[0..n).
 *  - Every call that takes a stream is asynchronous with respect to the host
 *    unless stated otherwise and returns an int status (SPH_OK or an error
 *    code below).  Argument errors are detected on the host before anything
 *    is launched.  Errors found by a kernel (a too-wide search, an exhausted
 *    list capacity, a wait that ran out of time) are recorded in a device
 *    status word and read with sph_ctx_device_status / pp_gravity_status.
 *  - Counts are int32: n < 2^31, and the total neighbour-list length < 2^31.
 *  - No C++ exception crosses this boundary.
 */
#ifndef SPHGB_H
#define SPHGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *sph_stream_t;

/* Status codes. */
#define SPH_OK               0
#define SPH_ERR_INVALID_ARG  1  /* a pointer, size or parameter is out of range */
#define SPH_ERR_CUDA         2  /* a CUDA runtime call failed */
#define SPH_ERR_NB_OVERFLOW  3  /* neighbour lists exceed the context capacity */
#define SPH_ERR_BUDGET       4  /* serving: request exceeds the memory budget */
#define SPH_ERR_TIMEOUT      5  /* a bounded device wait ran out */
#define SPH_ERR_NOT_FOUND    6  /* serving: unknown job id */
#define SPH_ERR_DEVICE       7  /* a kernel recorded an error in the status word */

/* Device status-word bits (sph_ctx_device_status, pp_gravity_status). */
#define SPH_FLAG_NB_OVERFLOW   1   /* neighbour entries beyond capacity were dropped */
#define SPH_FLAG_SEARCH_WIDE   2   /* a search box exceeded 2^24 cells and was skipped */
#define SPH_FLAG_TIMEOUT       4   /* a bounded mbarrier wait gave up */
#define SPH_FLAG_ROW_UNSORTED  8   /* reserved: never set (segments of any length are canonicalised) */
#define SPH_FLAG_GRAV_RANGE   16   /* pp_gravity_pairs: masses / eps put its fixed-point scale out of range */

/* Model constants (Sect. 2): gravitational constant G and softening length
 * eps of Eq. 4 (Plummer form, |dr|^2 + eps^2); adiabatic index gamma of
 * Eq. 5; artificial-viscosity alpha, beta, eta (after Eq. 11); smoothing-
 * length factor sigma of h = sigma (m / rho)^(1/3) (after Eq. 8). */
typedef struct SphParams {
    float G, eps, gamma, alpha, beta, eta, sigma;
} SphParams;

/* Multi-level hashed grid of the sorting stage (Sect. 3, "hierarchical grid
 * sorting").  A gas particle with smoothing length h is on level l, the
 * smallest l >= 0 with h <= L0 * 2^l (L0 = 2^log2_L0), clamped to
 * n_levels - 1.  Its cell on that level is floor((x - x0) / (L0 * 2^l)) per
 * axis in FP32, clamped to [0, 2^21 - 1]; its bucket (the paper's cell index
 * k of CellSPH) is (bit-interleave(cx, cy, cz) + l * 0x9E3779B97F4A7C15)
 * mod 2^log2_M. */
typedef struct SphGrid {
    float x0, y0, z0;
    int32_t log2_L0;   /* in [-100, 100] */
    int32_t n_levels;  /* in [1, 32] */
    int32_t log2_M;    /* in [4, 30]; must equal the context's */
} SphGrid;

/* ------------------------------------------------------------------------ */
/* Context: the scratch of the sorting, neighbour and SPH stages.           */
/* ------------------------------------------------------------------------ */

typedef struct sph_ctx sph_ctx;

/* Bytes of device workspace a context for up to n_gas_max gas particles,
 * 2^log2_M buckets and nb_capacity neighbour entries needs.  Returns 0 on
 * invalid arguments. */
size_t sph_ctx_workspace_bytes(int32_t n_gas_max, int32_t log2_M, int64_t nb_capacity);

/* Create a context over caller-allocated device workspace d_workspace of
 * workspace_bytes (>= sph_ctx_workspace_bytes(...), 256-byte aligned).  The
 * context carves all its arrays out of that buffer; the caller keeps
 * ownership and must keep it alive until sph_ctx_destroy.  Zero-fills the
 * workspace on `stream`.  *out receives a host-side handle. */
int sph_ctx_create(const SphParams *params, int32_t n_gas_max, int32_t log2_M,
                   int64_t nb_capacity, void *d_workspace, size_t workspace_bytes,
                   sph_stream_t stream, sph_ctx **out);

/* Release the host-side handle (not the workspace). */
int sph_ctx_destroy(sph_ctx *ctx);

/* Lanes that share one neighbour row in the density and force kernels
 * (1, 2, 4 or 8; default 4): a tuning knob, results differ only in the
 * order of the per-lane partial sums. */
int sph_ctx_set_lanes(sph_ctx *ctx, int32_t lanes);

/* Octaves added to the finest cell size of the grid sph_bin_and_sort
 * derives (h_grid == NULL): L0 = 2^(ceil(log2 min h) + shift), and as many
 * levels as max h then needs; shift in [-4, 4], default 0.  A tuning knob of
 * the neighbour search: any shift gives the same neighbour sets. */
int sph_ctx_set_grid_shift(sph_ctx *ctx, int32_t shift);

/* How sph_bin_and_sort runs the sorting stage: 1 (default) as one
 * cooperative launch whose phases are separated by grid-wide barriers, 0 as
 * a sequence of kernels (the form it also takes while `stream` is being
 * captured into a CUDA graph).  Both give bitwise the same results. */
int sph_ctx_set_sort_fused(sph_ctx *ctx, int32_t fused);

/* Replace the model constants used by later calls. */
int sph_ctx_set_params(sph_ctx *ctx, const SphParams *params);

/* Synchronise `stream`, then read and clear the context's device status word
 * (SPH_FLAG_* bits) into *h_flags.  Returns SPH_ERR_DEVICE if any bit was
 * set, SPH_OK otherwise. */
int sph_ctx_device_status(sph_ctx *ctx, sph_stream_t stream, int32_t *h_flags);

/* Synchronise `stream` and read the grid the last sph_bin_and_sort used. */
int sph_ctx_get_grid(sph_ctx *ctx, sph_stream_t stream, SphGrid *h_grid);

/* Synchronise `stream` and read the total neighbour-list length of the last
 * sph_build_neighbors (its "needed" capacity). */
int sph_ctx_nb_total(sph_ctx *ctx, sph_stream_t stream, int64_t *h_total);

/* ------------------------------------------------------------------------ */
/* Stage SP: grid sorting of the gas particles (Sect. 3, SP0..SP4).          */
/* ------------------------------------------------------------------------ */

/* Bin the n_gas gas particles d_pos_h ([n_gas][4]: x, y, z, h) into buckets
 * and counting-sort them: bucket counts with atomics (SP1), an exclusive
 * prefix sum over the 2^log2_M buckets with a warp-shuffle / shared-memory
 * cascade (SP2, SP3), and a scatter into bucket order (SP4), canonicalised so
 * that particles inside one bucket are in ascending original index (a stable
 * counting sort).  h_grid != NULL fixes the grid; h_grid == NULL derives it
 * on the device from the particles (x0 = floor(min x) - 1 per axis,
 * L0 = 2^ceil(log2 min h), enough levels for max h).  The context keeps the
 * sorted working set for the following stages.  Optional copies of the
 * results (NULL to skip): d_key_out[n_gas] bucket of each particle,
 * d_cell_start_out[M + 1] exclusive bucket starts (the paper's inclusive
 * CellSPH[k].y is cell_start[k + 1]), d_perm_out[n_gas] original index of
 * each sorted slot. */
int sph_bin_and_sort(sph_ctx *ctx, const float *d_pos_h, int32_t n_gas,
                     const SphGrid *h_grid, int32_t *d_key_out,
                     int32_t *d_cell_start_out, int32_t *d_perm_out,
                     sph_stream_t stream);

/* Allocation-free variant of sph_bin_and_sort.  The paper has no counterpart:
 * it is for callers that cannot allocate device memory -- a host framework
 * that owns all device memory through its own fixed arena, a plugin handed
 * only its input and output buffers, a loop that must never call cudaMalloc
 * because it can synchronise the device.  It needs no context: its scratch is
 * one file-scope device array of SPH_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits.  The caller passes the
 * input d_pos_h[n_gas][4] and the results d_key[n_gas], d_cell_start[2^log2_M
 * + 1], d_perm[n_gas] (same meaning and values as sph_bin_and_sort; no sorted
 * copy is kept).  Limits: n_gas <= SPH_NOALLOC_MAX_GAS and log2_M <=
 * SPH_NOALLOC_MAX_LOG2_M, else SPH_ERR_INVALID_ARG before anything runs.
 * h_grid == NULL derives the grid on the device as sph_bin_and_sort does.
 * Every call looks up the array's device address with the caller's device
 * current (cudaGetSymbolAddress, a host call that allocates nothing), so a
 * device reset or another context never leaves it a stale address; the
 * first call on a device may load the library's device code, so make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents (the call clears what must start at zero):
 * calls whose work may overlap on the GPU race on it, so order them (one
 * stream). */
#define SPH_NOALLOC_MAX_GAS 65536
#define SPH_NOALLOC_MAX_LOG2_M 17
#define SPH_NOALLOC_SCRATCH_BYTES 2097152
int sph_bin_and_sort_noalloc(const float *d_pos_h, int32_t n_gas, int32_t log2_M,
                             const SphGrid *h_grid, int32_t *d_key, int32_t *d_cell_start,
                             int32_t *d_perm, sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Neighbour lists (used by DC and HFC, Sect. 3).                            */
/* ------------------------------------------------------------------------ */

/* Build the neighbour list of every gas particle of the last sort: all gas
 * j != i with (in FP32) ((dx*dx + dy*dy) + dz*dz) < (h_i + h_j)^2, i.e.
 * |r_ij| < 2 h_ij, the support of W and W_p (Eqs. 8-9).  Lists are CSR in
 * sorted space: row s (sorted slot) spans [nb_start[s], nb_start[s+1]) and
 * holds sorted slots; perm maps slots to original indices.  The order inside
 * a row is deterministic.
 * If h_needed != NULL the call synchronises `stream`, writes the total list
 * length to *h_needed and returns SPH_ERR_NB_OVERFLOW (lists not built) when
 * it exceeds the context capacity.  If h_needed == NULL the call stays
 * asynchronous and an overflow sets SPH_FLAG_NB_OVERFLOW instead.
 * Optional copies (NULL to skip): d_nb_start_out[n_gas + 1] and
 * d_nb_idx_out[out_capacity] (copied only if the total fits). */
int sph_build_neighbors(sph_ctx *ctx, int32_t n_gas, int32_t *d_nb_start_out,
                        int32_t *d_nb_idx_out, int64_t out_capacity,
                        int64_t *h_needed, sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Stage DC: density (Eq. 7) and the next smoothing length.                 */
/* ------------------------------------------------------------------------ */

/* rho_i = m_i W(0, h_i) + sum_{j in list(i)} m_j W(|r_ij|, h_ij), the cubic
 * spline W of Eq. 8, h_ij = (h_i + h_j)/2; then h_next_i = sigma
 * (m_i / rho_i)^(1/3).  d_mass[n_gas] is in original order; d_rho[n_gas] and
 * d_h_next[n_gas] are written in original order.  FP32 with compensated
 * summation. */
int sph_density(sph_ctx *ctx, int32_t n_gas, const float *d_mass, float *d_rho,
                float *d_h_next, sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Stage HFC: hydrodynamic accelerations and heating (Eqs. 10-11).           */
/* ------------------------------------------------------------------------ */

/* a_i = -sum_j m_j Pi_ij grad W_p(|r_ij|, h_ij) and de_i/dt = 1/2 sum_j m_j
 * Pi_ij dv_ij . grad W_p over the neighbour list, with Pi_ij = p_i/rho_i^2
 * + p_j/rho_j^2 + nu_ij (Monaghan viscosity, Sect. 2.2), p = (gamma - 1)
 * rho e (Eq. 5), c = sqrt(gamma p / rho) (0 if p < 0), grad W_p = 0 at
 * |r_ij| = 0.  Inputs in original order: d_vel_e[n_gas][4] (vx, vy, vz, e),
 * d_rho[n_gas], d_mass[n_gas]; output d_acc_dedt[n_gas][4] (ax, ay, az,
 * de/dt) in original order.  Positions and h are those of the last sort.
 * FP32 with compensated (Kahan) summation. */
int sph_forces(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
               const float *d_mass, float *d_acc_dedt, sph_stream_t stream);

/* Time step of the modified CFL condition, Eq. 17, for the gas particles of
 * the last sort and lists: dt_i = C s_min / (c_max (1 + 1.2 alpha) +
 * 1.2 beta mu_max + sqrt(s_min (|Q_i| + |E_i|))) with s_min the smallest
 * |r_ij|, c_max the largest c_ij and mu_max the largest |mu_ij| over the
 * neighbours (mu_ij <= 0 as defined, so its magnitude is meant), Q_i =
 * |a_hyd + g|, E_i = |de/dt|; a particle without neighbours sets no bound.
 * Inputs in original order: d_vel_e, d_rho, d_mass as for sph_forces,
 * d_acc_hyd[n_gas][4] and d_grav (at least n_gas float4; the gas part of a
 * state's grav).  Writes min_i dt_i to the device float *d_dt_min (+inf if
 * no particle is bounded) and, if d_dt_particle != NULL, every dt_i
 * (original order).  FP32. */
int sph_cfl_dt(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
               const float *d_mass, const float *d_acc_hyd, const float *d_grav, float C_cfl,
               float *d_dt_particle, float *d_dt_min, sph_stream_t stream);

/* sph_forces with the time step of Eq. 17 taken in the same pass over the
 * neighbour lists: writes d_acc_dedt as sph_forces does, and min(dt_max,
 * min_i dt_i) to *d_dt_min (dt_i as for sph_cfl_dt, from the acceleration
 * this pass computes plus d_grav at the same positions; bitwise the value
 * sph_cfl_dt gives for that acceleration).  d_dt_particle optional.
 * C_cfl > 0, dt_max > 0. */
int sph_forces_cfl(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
                   const float *d_mass, float *d_acc_dedt, const float *d_grav, float C_cfl,
                   float dt_max, float *d_dt_particle, float *d_dt_min, sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Stage GFC: direct particle-particle gravity (Eq. 4).                      */
/* ------------------------------------------------------------------------ */

#define SPH_GRAV_POTENTIAL 1  /* also write phi_i = -G sum_{j!=i} m_j / sqrt(r^2+eps^2) */
#define SPH_GRAV_NO_KAHAN  2  /* plain FP32 running sums instead of per-tile compensation */

/* g_i = -G sum_{j != i} m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2) over
 * all n particles (gas and dark), the Plummer-softened reading of Eq. 4.
 * d_pos_m[n][4] = (x, y, z, m); d_acc_pot[n][4] = (gx, gy, gz, phi) with
 * phi = 0 unless SPH_GRAV_POTENTIAL.  eps >= 0; with eps = 0 coincident
 * pairs contribute nothing.  No context: the j-range is split across the
 * CTAs of a thread-block cluster and reduced through distributed shared
 * memory, so the call needs no scratch.  n = 0 is a no-op. */
int pp_gravity(const float *d_pos_m, int32_t n, float G, float eps, float *d_acc_pot,
               int32_t flags, sph_stream_t stream);

/* The rows [i0, i1) of pp_gravity: g_i (and phi_i) of the targets i0 <= i <
 * i1 over all n sources of d_pos_m[n][4], written to d_acc_pot[(i1 - i0)][4]
 * (row i at d_acc_pot[i - i0]).  This is the per-GPU share of the paper's
 * particle partition (Sect. 3: each of k GPUs computes the dynamics of N/k
 * particles): a GPU that owns the rows [i0, i1) and has gathered every
 * particle's (x, y, z, m) computes the gravity of its own particles.  The
 * same one-sided kernel and summation order as pp_gravity: with the plan
 * fixed by sph_gravity_tune(R, 1) the rows are bitwise those of pp_gravity.
 * 0 <= i0 <= i1 <= n; i0 == i1 is a no-op. */
int pp_gravity_rows(const float *d_pos_m, int32_t n, int32_t i0, int32_t i1, float G,
                    float eps, float *d_acc_pot, int32_t flags, sph_stream_t stream);

/* Launch plan pp_gravity uses for n particles and `flags`: *h_R targets per
 * thread (256 R per CTA, R in {2, 4, 8}; pairs of targets share packed FP32x2
 * instructions) and the cluster split *h_S of the source range. */
int sph_gravity_plan(int32_t n, int32_t flags, int32_t *h_R, int32_t *h_S);

/* Fix the plan of later pp_gravity calls (process-wide, for autotuning):
 * R in {2, 4, 8}, S in {1, 2, 4, 8, 16} (clamped to the number of source
 * tiles); R = 0 returns to the built-in cost model. */
int sph_gravity_tune(int32_t R, int32_t S);

/* The same g_i (and phi_i) as pp_gravity with every unordered pair evaluated
 * once (Newton's third law: one inverse cube serves both bodies, 16 instead
 * of 2 x 12 FP32 operations per pair; 14 in a tile whose bodies all have the
 * same mass, which leaves the mass out of the pair sums and applies it once
 * per tile sum).  Bodies are cut into blocks of 1024;
 * each tile of block pairs (I <= J) is one CTA, and the per-tile partial
 * sums are accumulated exactly as 64-bit fixed-point integers whose scale is
 * set per launch from sum |m_j| and eps, so the result is bitwise
 * reproducible whatever the order the tiles run in.
 * d_work (256-byte aligned, >= pp_gravity_pairs_workspace_bytes(n) bytes) is
 * caller-owned scratch, overwritten.  Runs pp_gravity instead when the call
 * is not eligible (pp_gravity_pairs_eligible), the scratch is missing or too
 * small, or n is above ~1.3e8 (more tiles than one grid can launch).  SPH_FLAG_GRAV_RANGE in the status word: the masses or eps put
 * the fixed-point scale outside 2^-250..2^250. */
int pp_gravity_pairs(const float *d_pos_m, int32_t n, float G, float eps, float *d_acc_pot,
                     int32_t flags, void *d_work, size_t work_bytes, sph_stream_t stream);

/* Launch plan of pp_gravity_pairs on one simulation (process-wide, for
 * autotuning): `threads` per CTA and R targets per thread -- (128, 6),
 * (128, 8), (128, 10) or (256, 8), i.e. blocks of 768, 1024, 1280 or 2048
 * bodies -- and tiles visited in super-tiles of 2^super_log2_side blocks on a
 * side (0..8; -1: chosen by size).  threads = 0 restores the default (128, 8,
 * -1).  Results of different plans agree to force rounding (other block
 * boundaries, so another summation order); one plan is bitwise reproducible.
 * Batches (pp_gravity_pairs_batched) take the plan's block shape too (the
 * super-tile side does not apply to them). */
int pp_gravity_pairs_plan(int32_t threads, int32_t R, int32_t super_log2_side);

/* The plan pp_gravity_pairs uses for n bodies: threads per CTA, targets per
 * thread and the super-tile side (log2). */
int pp_gravity_pairs_get_plan(int32_t n, int32_t *h_threads, int32_t *h_R, int32_t *h_super_log2);

/* Scratch bytes of pp_gravity_pairs for n bodies (4096 + 32 n). */
size_t pp_gravity_pairs_workspace_bytes(int32_t n);

/* 1 if pp_gravity_pairs would use the pair-once kernel for n bodies: eps^2 > 0
 * in FP32, no SPH_GRAV_NO_KAHAN, no plan fixed by sph_gravity_tune, and
 * n >= the threshold of pp_gravity_pairs_min_n (default 16384, where the
 * pair-once kernel overtakes the one-sided one on GB300). */
int pp_gravity_pairs_eligible(int32_t n, float eps, int32_t flags);

/* Set the smallest n for which pp_gravity_pairs uses the pair-once kernel
 * (process-wide; 0 restores the default 16384). */
int pp_gravity_pairs_min_n(int32_t n_min);

/* Synchronise `stream`, read and clear the gravity kernel's device status
 * word (SPH_FLAG_TIMEOUT).  Returns SPH_ERR_DEVICE if a bit was set. */
int pp_gravity_status(sph_stream_t stream, int32_t *h_flags);

/* Failure detection (no counterpart in the paper).  Every mbarrier wait of
 * the TMA-fed gravity kernels is bounded in time: a wait that runs out sets
 * SPH_FLAG_TIMEOUT in the gravity status word, the block waits (within the
 * same limit) for the copies it still has in flight and returns, so the
 * CUDA context stays usable and the host reads the failure through
 * pp_gravity_status.  sph_set_wait_limit_ns sets that limit for every later
 * launch on the current device (process-wide; 1 us .. 60 s; 0 restores the
 * default of 2 s; a synchronous host call). */
int sph_set_wait_limit_ns(int64_t limit_ns);

/* Probe of the timeout path: one block runs the bounded wait on an mbarrier
 * that expects 16 bytes no copy will bring, so the wait runs out after the
 * limit, SPH_FLAG_TIMEOUT is recorded and the kernel returns.  Nothing is
 * read or written but the status word; no copy is issued. */
int sph_wait_probe(sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Stage SU: leapfrog predictor-corrector (Eqs. 12-16).                      */
/* ------------------------------------------------------------------------ */

#define SPH_PREDICT 0  /* Eqs. 12-14 */
#define SPH_CORRECT 1  /* Eqs. 15-16 */
#define SPH_EMIT    2  /* no update: only write the FP32 working copies */

/* FP64 state (device, SoA): d_r[3n], d_v[3n], d_e[n_gas], and the saved
 * d_v_save[3n], d_e_save[n_gas] (written by PREDICT, read by CORRECT).
 * Accelerations Q_i = a_hyd_i + g_i for gas, g_i for dark, E_i = de_i/dt:
 * d_acc_hyd[n_gas][4] (ax, ay, az, de/dt), d_grav[n][4].
 * PREDICT: v_save = v, e_save = e, v <- v + dt Q, e <- e + dt E,
 *          r <- r + dt/2 (v_new + v_save).
 * CORRECT: v <- (v_save + v)/2 + dt/2 Q, e <- (e_save + e)/2 + dt/2 E.
 * Then (all phases) writes the FP32 working copies, each optional (NULL to
 * skip): d_pos_m[n][4] = (x, y, z, m), d_pos_h[n_gas][4] = (x, y, z, h),
 * d_vel_e[n_gas][4] = (vx, vy, vz, e), from d_mass[n] and d_h[n_gas]. */
int integrate_step(int32_t phase, double dt, int32_t n, int32_t n_gas, double *d_r,
                   double *d_v, double *d_e, double *d_v_save, double *d_e_save,
                   const float *d_acc_hyd, const float *d_grav, const float *d_mass,
                   const float *d_h, float *d_pos_m, float *d_pos_h, float *d_vel_e,
                   sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Whole steps.                                                              */
/* ------------------------------------------------------------------------ */

/* Device arrays of one simulation (caller-owned, original order). */
typedef struct SphState {
    int32_t n, n_gas;
    double *r, *v, *e;            /* FP64 state: [3n], [3n], [n_gas] */
    double *v_save, *e_save;      /* predictor saves: [3n], [n_gas] */
    float *mass;                  /* [n] */
    float *h;                     /* [n_gas] smoothing length for the next evaluation */
    float *pos_m;                 /* [n][4] FP32 working copy (x, y, z, m) */
    float *pos_h;                 /* [n_gas][4] FP32 working copy (x, y, z, h) */
    float *vel_e;                 /* [n_gas][4] FP32 working copy (vx, vy, vz, e) */
    float *rho;                   /* [n_gas] density of the current evaluation */
    float *acc_hyd;               /* [n_gas][4] (ax, ay, az, de/dt) */
    float *grav;                  /* [n][4] (gx, gy, gz, phi) */
    int32_t fresh;                /* 1 after sph_rhs_initial: the next step reuses its RHS */
    int32_t grav_flags;           /* flags passed to pp_gravity */
    void **events;                /* NULL, or 2 * SPH_NUM_STAGES cudaEvent_t (see sph_step) */
    void *grav_work;              /* NULL, or scratch of pp_gravity_pairs for n bodies ... */
    size_t grav_work_bytes;       /* ... of this many bytes (then gravity uses it) */
} SphState;

/* Stages of one sph_step, in launch order. */
#define SPH_STAGE_HFC_PRED 0  /* HFC at (r_n, v_n, e_n) */
#define SPH_STAGE_SU_PRED  1  /* predictor, Eqs. 12-14 */
#define SPH_STAGE_SP       2  /* grid sort */
#define SPH_STAGE_NB       3  /* neighbour lists */
#define SPH_STAGE_DC       4  /* density, Eq. 7 */
#define SPH_STAGE_GFC      5  /* gravity, Eq. 4 */
#define SPH_STAGE_HFC_CORR 6  /* HFC at (r_{n+1}, v~, e~) */
#define SPH_STAGE_SU_CORR  7  /* corrector, Eqs. 15-16 */
#define SPH_NUM_STAGES     8

/* First right-hand-side evaluation at the current state: FP32 working
 * copies, SP, neighbour lists, DC (rho, next h), GFC and HFC.  Sets fresh. */
int sph_rhs_initial(sph_ctx *ctx, SphState *st, sph_stream_t stream);

/* One predictor-corrector step of size dt (Sect. 2.2): HFC at (r, v, e)
 * unless fresh; PREDICT; SP; neighbour lists; DC; GFC once per step at the
 * new positions; HFC at (r', v~, e~); CORRECT.  SP, DC and HFC are skipped
 * when n_gas == 0 (collisionless run).  Asynchronous: a neighbour-list
 * overflow shows as SPH_FLAG_NB_OVERFLOW in the device status word.
 * If st->events != NULL, events[2 s] and events[2 s + 1] are recorded on
 * `stream` before and after stage s (SPH_STAGE_*; a skipped stage records
 * both back to back). */
int sph_step(sph_ctx *ctx, SphState *st, double dt, sph_stream_t stream);

/* One step of sph_step with an adaptive size chosen on the device: the first
 * HFC (at r, v, e, with the gravity of the previous step) also evaluates
 * Eq. 17 and writes dt = min(dt_max, min_i dt_i) to the device float *d_dt,
 * which both leapfrog phases read; no host round trip, so the step can be
 * captured in a CUDA graph.  Right after sph_rhs_initial only the time step
 * is evaluated (the forces are current).  Needs gas (n_gas >= 1); with a
 * batch attached the step is the smallest over all its simulations.  On
 * return *d_dt holds the step just taken. */
int sph_step_cfl(sph_ctx *ctx, SphState *st, float C_cfl, float dt_max, float *d_dt,
                 sph_stream_t stream);

/* FP64 reductions of one state in a fixed order (deterministic) by one
 * thread block: d_out[8] (device) = {kinetic sum m v^2 / 2, thermal
 * sum_gas m e, potential sum m phi / 2 (phi read from grav.w), px, py, pz,
 * total mass, 0}. */
int sph_diagnostics(const SphState *st, double *d_out, sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent simulations advanced by the same launches.     */
/* ------------------------------------------------------------------------ */

/* A batch lays K simulations out in one SphState: all gas first, simulation
 * by simulation (gas of s = [gas_off[s], gas_off[s+1])), then all dark
 * (dark of s = n_gas + [dark_off[s], dark_off[s+1])), n_gas = gas_off[K].
 * Simulations never interact: gravity sums only over a simulation's own
 * particles, and the grid sort hashes the simulation index with the level so
 * neighbour lists never cross simulations.  The per-simulation gravity of a
 * batch is computed with the same tile boundaries and summation order as
 * pp_gravity on that simulation alone with no cluster split (R and S = 1
 * fixed by sph_gravity_tune), so it is bitwise identical to it. */
typedef struct sph_batch sph_batch;

/* Device workspace bytes of a batch (0 on invalid offsets).  h_gas_off and
 * h_dark_off are host arrays of n_sims + 1 non-decreasing offsets from 0. */
size_t sph_batch_workspace_bytes(int32_t n_sims, const int32_t *h_gas_off,
                                 const int32_t *h_dark_off);

/* Create a batch over caller-allocated workspace (256-byte aligned).
 * d_sim_of_gas[n_gas] (device, caller-owned, kept by reference) gives the
 * simulation index of every gas particle.  Uploads the per-simulation table
 * and the gravity work list (blocks of 256 R targets, largest simulations
 * first; R = 4) and synchronises `stream`. */
int sph_batch_create(int32_t n_sims, const int32_t *h_gas_off, const int32_t *h_dark_off,
                     const int32_t *d_sim_of_gas, void *d_workspace, size_t workspace_bytes,
                     sph_stream_t stream, sph_batch **out);
int sph_batch_destroy(sph_batch *b);

/* Re-cut the gravity work list for R targets per thread (2, 4 or 8);
 * synchronises `stream`. */
int sph_batch_set_plan(sph_batch *b, int32_t R, sph_stream_t stream);

/* Eq. 4 for every simulation of the batch in one persistent launch (work
 * queue over the blocks of all simulations).  d_pos_m / d_acc_pot as in
 * pp_gravity over the batch's n particles. */
int pp_gravity_batched(const sph_batch *b, const float *d_pos_m, float G, float eps,
                       float *d_acc_pot, int32_t flags, sph_stream_t stream);

/* pp_gravity_pairs for every simulation of the batch in one launch: the
 * tiles of all simulations' triangles, one CTA each, fixed-point sums over
 * the batch's n particles, each simulation with the scale of its own sum |m|
 * (kept in the batch's workspace).  d_work as
 * for pp_gravity_pairs(b's n); runs pp_gravity_batched when not eligible
 * (pp_gravity_pairs_eligible on the batch's n) or d_work is missing / too
 * small. */
int pp_gravity_pairs_batched(const sph_batch *b, const float *d_pos_m, float G, float eps,
                             float *d_acc_pot, int32_t flags, void *d_work, size_t work_bytes,
                             sph_stream_t stream);

/* Attach a batch to a context (NULL detaches): later sorts use the batch's
 * simulation map, and sph_rhs_initial / sph_step use pp_gravity_pairs_batched
 * (state with grav_work) or pp_gravity_batched. */
int sph_ctx_set_batch(sph_ctx *ctx, const sph_batch *b);

/* ------------------------------------------------------------------------ */
/* Serving: simulations as requests (continuous batching).                   */
/* ------------------------------------------------------------------------ */

/* One simulation request: host arrays (copied by sim_submit, so the caller
 * may free them on return): r[3n], v[3n] FP64 SoA, m[n] FP32, and for the
 * gas particles [0, n_gas): e[n_gas] FP64 and the initial h[n_gas] FP32;
 * n_steps predictor-corrector steps of size dt after one initial RHS. */
typedef struct SimRequest {
    int32_t n, n_gas, n_steps;
    double dt;
    const double *h_r, *h_v, *h_e;
    const float *h_m, *h_h;
} SimRequest;

#define SIM_QUEUED  0
#define SIM_RUNNING 1
#define SIM_DONE    2
#define SIM_FAILED  3

/* Status of one request.  Times are seconds of a monotonic host clock.  The
 * step latency percentiles are over the job's own steps (CUDA events on its
 * stream).
 * When state == SIM_DONE, h_r / h_v / h_e point to the final state (owned by
 * the server, valid until sim_release). */
typedef struct SimStatus {
    int32_t state, error, n, n_gas, n_steps, steps_done;
    double submit_s, admit_s, done_s;
    double step_ms_p50, step_ms_p99;
    const double *h_r, *h_v, *h_e;
} SimStatus;

typedef struct SphServerInfo {
    int32_t queued, resident;
    size_t arena_bytes, arena_free_bytes;
} SphServerInfo;

typedef struct sph_server sph_server;

/* A server over a caller-allocated device arena of arena_bytes (256-byte
 * aligned): the memory budget.  Each admitted simulation takes its state
 * and context workspace from the arena (first fit) and gives them back when
 * it finishes.  At most max_resident simulations are resident together, each
 * on a CUDA stream of its own out of max(n_streams, max_resident) streams the
 * server creates; half of them have the device's higher stream priority and
 * take the jobs below 131,072 particles, so the GPU schedules a small job's
 * thread blocks ahead of a large job's as SMs free up. */
int sph_server_create(const SphParams *params, void *d_arena, size_t arena_bytes,
                      int32_t max_resident, int32_t n_streams, sph_server **out);
int sph_server_destroy(sph_server *s);

/* Queue a request (thread-safe).  SPH_ERR_BUDGET if it can never fit the
 * arena; otherwise *job_id identifies it. */
int sim_submit(sph_server *s, const SimRequest *req, uint64_t *job_id);

/* One serving step (continuous batching, no lockstep): admit queued
 * requests (first fit, in the policy's order) while memory and slots allow; collect
 * every resident simulation's step that has finished (its CUDA event),
 * retire the simulations that are done (final state to host, memory back to
 * the arena) and launch the next step (the initial RHS on the first) of
 * every simulation with nothing in flight.  If no step had finished, waits
 * for the first that does.  So a small simulation takes many steps while a
 * large one takes one.  Returns the number still resident and the wall time
 * of the call in milliseconds (either may be NULL); SPH_ERR_TIMEOUT if no
 * step finished within an hour. */
int sph_server_step(sph_server *s, int32_t *h_resident, double *h_step_ms);

/* Order in which queued requests are admitted: SPH_SERVE_FIFO (default,
 * arrival order) or SPH_SERVE_SHORTEST_FIRST (least estimated GPU work left
 * first: steps x (N^2 gravity + N SPH + per-step launches); under overload it
 * completes the most requests and starves the largest). */
#define SPH_SERVE_FIFO           0
#define SPH_SERVE_SHORTEST_FIRST 1
int sph_server_set_policy(sph_server *s, int32_t policy);

/* Latencies (ms) of every simulation step the server has completed, in
 * completion order: each from CUDA events on the simulation's stream around
 * its own step (so they include time spent queued behind other jobs' work).
 * Writes min(count, cap) of them to h_ms and the count to *h_count. */
int sph_server_step_times(sph_server *s, float *h_ms, int32_t cap, int32_t *h_count);

/* Status of a request (thread-safe); SPH_ERR_NOT_FOUND for an unknown id. */
int sim_poll(sph_server *s, uint64_t job_id, SimStatus *out);

/* Checkpoint of a resident request (thread-safe): waits for its step in
 * flight (counting it), then copies its state to caller-owned host arrays:
 * h_r[3n], h_v[3n] FP64 SoA, h_e[n_gas] FP64, and h_h[n_gas] the smoothing
 * lengths its last evaluation used; *h_steps_done the steps taken.  The job
 * keeps running.  Submitting the checkpoint as a new request (same masses,
 * dt, and n_steps minus the steps taken) resumes it: the first evaluation
 * of the new request recomputes exactly the right-hand side the job would
 * have used next, so the resumed run is bitwise the uninterrupted one.
 * SPH_ERR_INVALID_ARG if the job is not resident or has not started. */
int sim_checkpoint(sph_server *s, uint64_t job_id, double *h_r, double *h_v, double *h_e,
                   float *h_h, int32_t *h_steps_done);

/* Forget a finished, failed or still-queued request and its results. */
int sim_release(sph_server *s, uint64_t job_id);

int sph_server_info(sph_server *s, SphServerInfo *out);

/* Timing helpers over the CUDA runtime (for callers without their own):
 * create / destroy `count` timing-enabled events into h_events[count], and
 * the elapsed milliseconds between two recorded events (synchronises on b). */
int sph_events_create(int32_t count, void **h_events);
int sph_events_destroy(int32_t count, void **h_events);
int sph_event_elapsed_ms(void *a, void *b, float *h_ms);

/* Number of kernels this library has launched in this process so far. */
int64_t sph_launch_count(void);

int sph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPHGB_H */
