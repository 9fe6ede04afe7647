// kernels.cuh -- host-side launchers shared between translation units.
#pragma once

#include "common.cuh"

namespace sphgb {

// sort.cu
int launch_scan_exclusive(const int *in, int n, int *out, int *block_sums, cudaStream_t st);
int scan_block_count(long long n);
// canonical order inside the buckets: unordered is the scatter's output
// (left scrambled), perm receives each bucket's members in ascending order
int launch_sort_buckets(const int *key, int n, const int *start, int *unordered, int *perm,
                        int *long_list, int *long_count, cudaStream_t st);
int launch_segsort_rows(const int *nb_start, const int *own, int n, int cap, int *data, int *tmp,
                        int *long_list, int *long_count, cudaStream_t st);
// shift: octaves added to the derived finest cell size (0: L0 = 2^ceil(log2 min h))
int launch_grid_auto(const float4 *pos_h, int n, unsigned *red, int log2_M, GridDev *grid,
                     cudaStream_t st, int shift = 0);
int launch_grid_set(const SphGrid &h, GridDev *grid, cudaStream_t st);
int launch_bin(const float4 *pos_h, const int *sim_of, int n, const GridDev *grid, int *key,
               int *count, cudaStream_t st);
// sorted copies (pos_h_s, and sim_s when sim_of is given) and the bucket,
// super-cell and level statistics, taken over the sorted order
int launch_gather_bin(const float4 *pos_h, const int *sim_of, const int *perm, int n,
                      const GridDev *grid, float4 *pos_h_s, int *sim_s, unsigned *tag_s, unsigned *occ,
                      int log2_B, unsigned *hmax_cell, int *lvl_count, unsigned *lvl_hmax,
                      cudaStream_t st);
int launch_scatter(const int *key, int n, const int *start, int *count, int *perm, cudaStream_t st);
// the whole sorting stage (grid, bin, scan, scatter, rank, long buckets,
// sorted copies and statistics) as one cooperative launch; bitwise the
// results of the launches above in sequence
struct SortArgs {
    const float4 *pos_h;
    const int *sim_of;      // simulation of each particle, or NULL
    int n;
    int log2_M;
    int auto_grid;          // 1: derive the grid; 0: use `given`
    int grid_shift;         // octaves added to the derived finest cell size
    GridDev given;
    unsigned *red;          // [5] extremes, 0 between calls
    GridDev *grid;          // out
    int *key, *count, *start, *block_sums, *tmp, *perm, *long_list, *long_count;
    int block_sums_cap;     // entries of block_sums (bounds the grid)
    float4 *pos_h_s;
    int *sim_s;             // or NULL
    unsigned *tag_s;        // cell tag of each sorted particle, or NULL
    unsigned *occ;
    int log2_B;
    unsigned *hmax_cell;
    int *lvl_count;
    unsigned *lvl_hmax;
};
int launch_sort_fused(const SortArgs &a, cudaStream_t st);
void grid_reset_red(unsigned *red, const unsigned *v, cudaStream_t st);

// gravity.cu: the batched kernel's work description (host side)
int launch_gravity_batched(const float4 *pos, const int4 *sims, const int2 *units, int n_units,
                           int *counter, int R, float G, float eps, float4 *out, int flags,
                           cudaStream_t st);
int gravity_num_sms();
// gravity_pairs.cu: tiles of one simulation with ns bodies, and the pair-once
// evaluation of a batch (sims (g0, ng, d0, nd), tile_off[n_sims + 1])
// in blocks of B bodies; the block shapes of the pair-once plans, their
// block sizes and the shape the current plan names
constexpr int kPairsNumShapes = 4;
long long pairs_tiles(long long ns, int B);
int pairs_shape_block(int shape);
int pairs_current_shape();
size_t pairs_scale_bytes();   // bytes of one simulation's fixed-point scale
int launch_gravity_pairs_batched(const float4 *pos, int n, int n_gas, const int4 *d_sims,
                                 const long long *d_tile_off, int n_sims, long long n_tiles,
                                 int shape, void *d_scales, float G, float eps, float4 *out,
                                 int flags, void *d_work, cudaStream_t st);
// device address of the gravity kernels' status word (SPH_FLAG_*)
int *gravity_flags_device();
// true while sph_gravity_tune has fixed a one-sided launch plan
bool gravity_plan_forced();

// neighbors.cu
struct NbArgs {
    const float4 *pos_h_s;   // sorted (x, y, z, h)
    const int *cell_start;   // [M + 1]
    const unsigned *hmax_cell;
    const int *lvl_count;    // [kMaxLevels]
    const unsigned *lvl_hmax;
    const GridDev *grid;
    const int *sim_s;        // [n] simulation of each sorted particle, or NULL (one simulation)
    const unsigned *tag_s;   // [n] cell tag of each sorted particle (cell_tag), or NULL
    const unsigned *occ;     // super-cell occupancy bits, or NULL
    int log2_B;
    int n;
    int *own;                // [n] own-search count
    int *rev;                // [n] reverse count / cursor
    const int *nb_start;     // [n + 1]
    int *nb_idx;
    long long capacity;
    int *flags;
    int *stage;              // [n * stage_k] own entries of the single-search build, or NULL
    int stage_k;
    int *list;               // rows whose own part exceeds stage_k
    int *list_count;
};
int launch_nb_count(const NbArgs &a, cudaStream_t st);
int launch_nb_fill(const NbArgs &a, cudaStream_t st);
int launch_row_len(const int *own, const int *rev, int n, int *row_len, cudaStream_t st);

// hydro.cu
struct HydroParams {
    float gamma, alpha, beta, eta, sigma;
};
int launch_density(const float4 *pos_h_s, const float *mass, const int *perm, const int *nb_start,
                   const int *nb_idx, int cap, int n, float sigma, int lanes, float *rho_s,
                   float *rho_out, float *h_next_out, float *mass_s, int *mixed, cudaStream_t st);
int launch_hydro_prep(const float4 *vel_e, const float *rho, const float *mass, const int *perm,
                      int n, HydroParams hp, float4 *vel_s, float4 *aux_s, cudaStream_t st);
// integrate.cu: integrate_step with the step size optionally read from
// device memory (d_dt != NULL)
int integrate_launch(int phase, double dt, const float *d_dt, int n, int n_gas, double *d_r,
                     double *d_v, double *d_e, double *d_v_save, double *d_e_save,
                     const float *d_acc_hyd, const float *d_grav, const float *d_mass,
                     const float *d_h, float *d_pos_m, float *d_pos_h, float *d_vel_e,
                     sph_stream_t stream);
int launch_cfl(const float4 *pos_h_s, const float4 *vel_s, const float4 *aux_s, const int *perm,
               const int *nb_start, const int *nb_idx, int cap, int n, HydroParams hp, float C,
               const float4 *acc_hyd, const float4 *grav, float *dt_out, float *dt_min,
               float dt_cap, cudaStream_t st);
// dt_min != NULL: also the CFL time step of Eq. 17 in the same pass (grav at
// the same positions; *dt_min = min(dt_cap, smallest particle step))
int launch_forces(const float4 *pos_h_s, const float4 *vel_s, const float4 *aux_s,
                  const int *perm, const int *nb_start, const int *nb_idx, int cap, int n,
                  HydroParams hp, int lanes, float4 *acc_out, cudaStream_t st,
                  const float4 *grav = nullptr, float C = 0.0f, float *dt_out = nullptr,
                  float *dt_min = nullptr, float dt_cap = 0.0f);

}  // namespace sphgb
