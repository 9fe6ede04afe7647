// api.cu -- the C ABI of include/sphgb.h: context over caller-owned
// workspace, the stage entry points SP / neighbour lists / DC / HFC, and the
// whole-step driver that sequences them as the paper's predictor-corrector
// flow (Sect. 2.2 and the kernel list of Sect. 3).
#include <algorithm>
#include <limits>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

using namespace sphgb;

namespace sphgb {
static std::atomic<long long> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int device_num_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    return sms;
}
}  // namespace sphgb

extern "C" int64_t sph_launch_count(void) { return g_launches.load(); }

extern "C" int sph_events_create(int32_t count, void **h_events) {
    if (count < 0 || (count > 0 && !h_events)) return SPH_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy((cudaEvent_t)h_events[j]);
            return SPH_ERR_CUDA;
        }
        h_events[i] = (void *)e;
    }
    return SPH_OK;
}

extern "C" int sph_events_destroy(int32_t count, void **h_events) {
    if (count < 0 || (count > 0 && !h_events)) return SPH_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (h_events[i]) cudaEventDestroy((cudaEvent_t)h_events[i]);
    return SPH_OK;
}

extern "C" int sph_event_elapsed_ms(void *a, void *b, float *h_ms) {
    if (!a || !b || !h_ms) return SPH_ERR_INVALID_ARG;
    SPH_CUDA_TRY(cudaEventSynchronize((cudaEvent_t)b));
    SPH_CUDA_TRY(cudaEventElapsedTime(h_ms, (cudaEvent_t)a, (cudaEvent_t)b));
    return SPH_OK;
}

struct sph_ctx {
    SphParams params;
    int n_max;
    int log2_M;
    long long M;
    long long capacity;
    void *ws;
    size_t ws_bytes;
    // carved arrays
    int *key, *count, *start, *perm, *tmp, *long_list, *long_count;
    unsigned *hmax_cell;
    unsigned *occ;   // super-cell occupancy bits, 2^(log2_M + 1) bits
    int *lvl_count;
    unsigned *lvl_hmax;
    GridDev *grid;
    unsigned *red;
    unsigned *red_fused;   // extremes of the one-launch sort (0 between calls)
    int block_sums_cap;
    int *flags;
    int *block_sums;
    float4 *pos_h_s, *vel_s, *aux_s;
    float *rho_s, *mass_s;
    int *own, *rev, *row_len, *nb_start, *nb_idx;
    int *sim_s;      // simulation of each sorted particle (batched runs)
    unsigned *tag_s; // cell tag of each sorted particle (level, low cell bits)
    int n_sorted;    // n_gas of the last sort
    int nb_built;    // 1 once lists match the last sort
    int sorted_batched;        // the last sort used the batch's simulation map
    int hydro_lanes;           // lanes per row in DC / HFC (1, 2, 4 or 8)
    int sort_fused;            // 1: the sorting stage as one cooperative launch
    int grid_shift;            // octaves added to the derived finest cell size
    const sph_batch *batch;    // NULL: one simulation
};

// Many independent simulations in one state (see sph_batch_create).
struct sph_batch {
    int n_sims, n_gas, n;
    int R;                       // targets per thread the work units were cut for
    std::vector<int4> h_sims;    // (g0, ng, d0, nd) per simulation
    std::vector<int2> h_units;   // (simulation, first virtual target), largest first
    std::vector<int> h_gas_off, h_dark_off;
    int4 *d_sims;
    int2 *d_units;
    int *d_counter;
    size_t units_cap;
    const int *d_sim_of_gas;
    // pair-once gravity: first tile of each simulation [n_sims + 1] and the
    // tile count, for each block shape a plan may name
    long long *d_tile_off[kPairsNumShapes];
    long long n_pair_tiles[kPairsNumShapes];
    void *d_pair_scales;         // pair-once gravity: fixed-point scale of each simulation
};

namespace {

struct Carver {
    char *base;
    size_t off;
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void carve(sph_ctx *c, char *base, size_t *total) {
    Carver cv{base, 0};
    const size_t n = (size_t)c->n_max, M = (size_t)c->M;
    const size_t seg_list = n > M ? n : M;
    c->key = cv.take<int>(n);
    c->count = cv.take<int>(M);
    c->start = cv.take<int>(M + 1);
    c->hmax_cell = cv.take<unsigned>(M);
    c->occ = cv.take<unsigned>(M / 16 + 1);
    c->perm = cv.take<int>(n);
    c->tmp = cv.take<int>(c->capacity > (long long)n ? (size_t)c->capacity : n);
    c->long_list = cv.take<int>(seg_list);
    c->long_count = cv.take<int>(4);
    c->lvl_count = cv.take<int>(kMaxLevels);
    c->lvl_hmax = cv.take<unsigned>(kMaxLevels);
    c->grid = cv.take<GridDev>(1);
    c->red = cv.take<unsigned>(8);
    c->red_fused = cv.take<unsigned>(8);
    // [0] status bits; [1] set when the masses of the last density pass were
    // not all equal (its equal-mass loop reads no mass array)
    c->flags = cv.take<int>(4);
    // the scan's block totals, also the chunk totals of the one-launch sort,
    // whose grid they cap: room for a full resident grid (a few blocks per SM)
    size_t nb_scan = (size_t)scan_block_count((long long)(M > n ? M : n));
    const size_t n_sums = std::max<size_t>(nb_scan + 32, 4096);
    c->block_sums = cv.take<int>(n_sums);
    c->block_sums_cap = (int)n_sums;
    c->pos_h_s = cv.take<float4>(n);
    c->vel_s = cv.take<float4>(n);
    c->aux_s = cv.take<float4>(n);
    c->rho_s = cv.take<float>(n);
    c->mass_s = cv.take<float>(n);
    c->own = cv.take<int>(n);
    c->rev = cv.take<int>(n);
    c->row_len = cv.take<int>(n);
    c->nb_start = cv.take<int>(n + 1);
    c->nb_idx = cv.take<int>((size_t)c->capacity);
    c->sim_s = cv.take<int>(n);
    c->tag_s = cv.take<unsigned>(n);
    *total = (cv.off + 255) & ~size_t(255);
}

bool params_ok(const SphParams *p) {
    return p && p->G == p->G && p->eps >= 0.0f && p->gamma > 1.0f && p->alpha >= 0.0f &&
           p->beta >= 0.0f && p->eta >= 0.0f && p->sigma > 0.0f;
}

HydroParams hydro_params(const sph_ctx *c) {
    return HydroParams{c->params.gamma, c->params.alpha, c->params.beta, c->params.eta,
                       c->params.sigma};
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int sph_version(void) { return 1; }

extern "C" size_t sph_ctx_workspace_bytes(int32_t n_gas_max, int32_t log2_M, int64_t nb_capacity) {
    if (n_gas_max < 0 || log2_M < 4 || log2_M > 30 || nb_capacity < 0 ||
        nb_capacity > 0x7fffffffLL)
        return 0;
    sph_ctx c;
    std::memset(&c, 0, sizeof(c));
    c.n_max = n_gas_max;
    c.log2_M = log2_M;
    c.M = 1ll << log2_M;
    c.capacity = nb_capacity;
    size_t total = 0;
    carve(&c, nullptr, &total);
    return total;
}

extern "C" int sph_ctx_create(const SphParams *params, int32_t n_gas_max, int32_t log2_M,
                              int64_t nb_capacity, void *d_workspace, size_t workspace_bytes,
                              sph_stream_t stream, sph_ctx **out) {
    if (!out || !params_ok(params) || !d_workspace) return SPH_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255u) != 0) return SPH_ERR_INVALID_ARG;
    size_t need = sph_ctx_workspace_bytes(n_gas_max, log2_M, nb_capacity);
    if (need == 0 || workspace_bytes < need) return SPH_ERR_INVALID_ARG;
    sph_ctx *c = new (std::nothrow) sph_ctx;
    if (!c) return SPH_ERR_INVALID_ARG;
    std::memset(c, 0, sizeof(*c));
    c->params = *params;
    c->n_max = n_gas_max;
    c->log2_M = log2_M;
    c->M = 1ll << log2_M;
    c->capacity = nb_capacity;
    c->ws = d_workspace;
    c->ws_bytes = workspace_bytes;
    c->hydro_lanes = 4;
    c->sort_fused = 1;
    size_t total = 0;
    carve(c, static_cast<char *>(d_workspace), &total);
    if (cudaMemsetAsync(d_workspace, 0, total, (cudaStream_t)stream) != cudaSuccess) {
        delete c;
        return SPH_ERR_CUDA;
    }
    *out = c;
    return SPH_OK;
}

extern "C" int sph_ctx_destroy(sph_ctx *ctx) {
    delete ctx;
    return SPH_OK;
}

extern "C" int sph_ctx_set_lanes(sph_ctx *ctx, int32_t lanes) {
    if (!ctx || (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)) return SPH_ERR_INVALID_ARG;
    ctx->hydro_lanes = lanes;
    return SPH_OK;
}

extern "C" int sph_ctx_set_grid_shift(sph_ctx *ctx, int32_t shift) {
    if (!ctx || shift < -4 || shift > 4) return SPH_ERR_INVALID_ARG;
    ctx->grid_shift = shift;
    return SPH_OK;
}

extern "C" int sph_ctx_set_sort_fused(sph_ctx *ctx, int32_t fused) {
    if (!ctx || (fused != 0 && fused != 1)) return SPH_ERR_INVALID_ARG;
    ctx->sort_fused = fused;
    return SPH_OK;
}

extern "C" int sph_ctx_set_params(sph_ctx *ctx, const SphParams *params) {
    if (!ctx || !params_ok(params)) return SPH_ERR_INVALID_ARG;
    ctx->params = *params;
    return SPH_OK;
}

extern "C" int sph_ctx_device_status(sph_ctx *ctx, sph_stream_t stream, int32_t *h_flags) {
    if (!ctx || !h_flags) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    SPH_CUDA_TRY(cudaMemcpyAsync(&v, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPH_CUDA_TRY(cudaMemsetAsync(ctx->flags, 0, sizeof(int), st));
    SPH_CUDA_TRY(cudaStreamSynchronize(st));
    *h_flags = v;
    return v ? SPH_ERR_DEVICE : SPH_OK;
}

extern "C" int sph_ctx_get_grid(sph_ctx *ctx, sph_stream_t stream, SphGrid *h_grid) {
    if (!ctx || !h_grid) return SPH_ERR_INVALID_ARG;
    GridDev g;
    cudaStream_t st = (cudaStream_t)stream;
    SPH_CUDA_TRY(cudaMemcpyAsync(&g, ctx->grid, sizeof(g), cudaMemcpyDeviceToHost, st));
    SPH_CUDA_TRY(cudaStreamSynchronize(st));
    h_grid->x0 = g.x0;
    h_grid->y0 = g.y0;
    h_grid->z0 = g.z0;
    h_grid->log2_L0 = g.log2_L0;
    h_grid->n_levels = g.n_levels;
    h_grid->log2_M = g.log2_M;
    return SPH_OK;
}

extern "C" int sph_ctx_nb_total(sph_ctx *ctx, sph_stream_t stream, int64_t *h_total) {
    if (!ctx || !h_total) return SPH_ERR_INVALID_ARG;
    int t = 0;
    cudaStream_t st = (cudaStream_t)stream;
    SPH_CUDA_TRY(cudaMemcpyAsync(&t, ctx->nb_start + ctx->n_sorted, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    SPH_CUDA_TRY(cudaStreamSynchronize(st));
    *h_total = t;
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// SP
// ---------------------------------------------------------------------------

extern "C" int sph_bin_and_sort(sph_ctx *ctx, const float *d_pos_h, int32_t n_gas,
                                const SphGrid *h_grid, int32_t *d_key_out,
                                int32_t *d_cell_start_out, int32_t *d_perm_out,
                                sph_stream_t stream) {
    if (!ctx || n_gas < 0 || n_gas > ctx->n_max) return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && (!d_pos_h || !aligned16(d_pos_h))) return SPH_ERR_INVALID_ARG;
    if (h_grid) {
        if (h_grid->log2_M != ctx->log2_M || h_grid->n_levels < 1 || h_grid->n_levels > kMaxLevels ||
            h_grid->log2_L0 < -100 || h_grid->log2_L0 > 100 ||
            !(h_grid->x0 == h_grid->x0) || !(h_grid->y0 == h_grid->y0) || !(h_grid->z0 == h_grid->z0))
            return SPH_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const float4 *pos = reinterpret_cast<const float4 *>(d_pos_h);
    const int M = (int)ctx->M;
    const int *sim_of = ctx->batch ? ctx->batch->d_sim_of_gas : nullptr;
    if (sim_of && n_gas != ctx->batch->n_gas) return SPH_ERR_INVALID_ARG;
    int rc;
    // The whole stage as one cooperative launch; while the stream is being
    // captured into a graph (or if the launch is refused) the same stage runs
    // as the sequence of kernels below, with bitwise the same results.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SPH_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    bool fused = false;
    if (cap == cudaStreamCaptureStatusNone && ctx->sort_fused) {
        SortArgs fa{};
        fa.pos_h = pos;
        fa.sim_of = sim_of;
        fa.n = n_gas;
        fa.log2_M = ctx->log2_M;
        fa.auto_grid = h_grid ? 0 : 1;
        fa.grid_shift = ctx->grid_shift;
        if (h_grid)
            fa.given = GridDev{h_grid->x0, h_grid->y0, h_grid->z0, h_grid->log2_L0, h_grid->n_levels,
                               h_grid->log2_M};
        fa.red = ctx->red_fused;
        fa.grid = ctx->grid;
        fa.key = ctx->key;
        fa.count = ctx->count;
        fa.start = ctx->start;
        fa.block_sums = ctx->block_sums;
        fa.block_sums_cap = ctx->block_sums_cap;
        fa.tmp = ctx->tmp;
        fa.perm = ctx->perm;
        fa.long_list = ctx->long_list;
        fa.long_count = ctx->long_count;
        fa.pos_h_s = ctx->pos_h_s;
        fa.sim_s = sim_of ? ctx->sim_s : nullptr;
        fa.tag_s = ctx->tag_s;
        fa.occ = ctx->occ;
        fa.log2_B = ctx->log2_M + 1;
        fa.hmax_cell = ctx->hmax_cell;
        fa.lvl_count = ctx->lvl_count;
        fa.lvl_hmax = ctx->lvl_hmax;
        if (launch_sort_fused(fa, st) == SPH_OK) fused = true;
        else cudaGetLastError();   // a refused launch leaves no sticky error
    }
    if (!fused) {
        if (h_grid) rc = launch_grid_set(*h_grid, ctx->grid, st);
        else rc = launch_grid_auto(pos, n_gas, ctx->red, ctx->log2_M, ctx->grid, st, ctx->grid_shift);
        if (rc) return rc;
        // SP0: zero the per-bucket and per-level arrays
        SPH_CUDA_TRY(cudaMemsetAsync(ctx->count, 0, sizeof(int) * (size_t)M, st));
        SPH_CUDA_TRY(cudaMemsetAsync(ctx->hmax_cell, 0, sizeof(unsigned) * (size_t)M, st));
        SPH_CUDA_TRY(cudaMemsetAsync(ctx->occ, 0, sizeof(unsigned) * ((size_t)M / 16 + 1), st));
        SPH_CUDA_TRY(cudaMemsetAsync(ctx->lvl_count, 0, sizeof(int) * kMaxLevels, st));
        SPH_CUDA_TRY(cudaMemsetAsync(ctx->lvl_hmax, 0, sizeof(unsigned) * kMaxLevels, st));
        // SP1
        if ((rc = launch_bin(pos, sim_of, n_gas, ctx->grid, ctx->key, ctx->count, st))) return rc;
        // SP2 + SP3
        if ((rc = launch_scan_exclusive(ctx->count, M, ctx->start, ctx->block_sums, st))) return rc;
        // SP4 + canonical order inside buckets
        if ((rc = launch_scatter(ctx->key, n_gas, ctx->start, ctx->count, ctx->tmp, st))) return rc;
        if ((rc = launch_sort_buckets(ctx->key, n_gas, ctx->start, ctx->tmp, ctx->perm, ctx->long_list,
                                      ctx->long_count, st)))
            return rc;
        // sorted copies and the bucket / super-cell / level statistics
        if ((rc = launch_gather_bin(pos, sim_of, ctx->perm, n_gas, ctx->grid, ctx->pos_h_s,
                                    sim_of ? ctx->sim_s : nullptr, ctx->tag_s, ctx->occ, ctx->log2_M + 1,
                                    ctx->hmax_cell, ctx->lvl_count, ctx->lvl_hmax, st)))
            return rc;
    }
    ctx->sorted_batched = sim_of != nullptr;
    ctx->n_sorted = n_gas;
    ctx->nb_built = 0;
    if (d_key_out && n_gas)
        SPH_CUDA_TRY(cudaMemcpyAsync(d_key_out, ctx->key, sizeof(int) * (size_t)n_gas,
                                     cudaMemcpyDeviceToDevice, st));
    if (d_cell_start_out)
        SPH_CUDA_TRY(cudaMemcpyAsync(d_cell_start_out, ctx->start, sizeof(int) * ((size_t)M + 1),
                                     cudaMemcpyDeviceToDevice, st));
    if (d_perm_out && n_gas)
        SPH_CUDA_TRY(cudaMemcpyAsync(d_perm_out, ctx->perm, sizeof(int) * (size_t)n_gas,
                                     cudaMemcpyDeviceToDevice, st));
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// Neighbour lists
// ---------------------------------------------------------------------------

extern "C" int sph_build_neighbors(sph_ctx *ctx, int32_t n_gas, int32_t *d_nb_start_out,
                                   int32_t *d_nb_idx_out, int64_t out_capacity,
                                   int64_t *h_needed, sph_stream_t stream) {
    if (!ctx || n_gas != ctx->n_sorted || out_capacity < 0) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = n_gas;
    NbArgs a;
    a.pos_h_s = ctx->pos_h_s;
    a.cell_start = ctx->start;
    a.hmax_cell = ctx->hmax_cell;
    a.lvl_count = ctx->lvl_count;
    a.lvl_hmax = ctx->lvl_hmax;
    a.grid = ctx->grid;
    a.sim_s = ctx->sorted_batched ? ctx->sim_s : nullptr;
    a.tag_s = ctx->tag_s;
    a.occ = ctx->occ;
    a.log2_B = ctx->log2_M + 1;
    a.n = n;
    a.own = ctx->own;
    a.rev = ctx->rev;
    a.nb_start = ctx->nb_start;
    a.nb_idx = ctx->nb_idx;
    a.capacity = ctx->capacity;
    a.flags = ctx->flags;
    // single search pass when the scratch array can stage >= 48 own entries
    // per row; otherwise count and fill with two searches
    const long long room = n > 0 ? std::max<long long>(ctx->capacity, n) / n : 0;
    a.stage_k = (int)std::min<long long>(128, room & ~15ll);
    a.stage = a.stage_k >= 48 ? ctx->tmp : nullptr;
    a.list = ctx->long_list;
    a.list_count = ctx->long_count;
    int rc;
    if (n > 0) SPH_CUDA_TRY(cudaMemsetAsync(ctx->rev, 0, sizeof(int) * (size_t)n, st));
    if (a.stage) SPH_CUDA_TRY(cudaMemsetAsync(ctx->long_count, 0, sizeof(int), st));
    if ((rc = launch_nb_count(a, st))) return rc;
    if ((rc = launch_row_len(ctx->own, ctx->rev, n, ctx->row_len, st))) return rc;
    if ((rc = launch_scan_exclusive(ctx->row_len, n, ctx->nb_start, ctx->block_sums, st))) return rc;
    long long total = -1;
    if (h_needed) {
        int t = 0;
        SPH_CUDA_TRY(cudaMemcpyAsync(&t, ctx->nb_start + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        SPH_CUDA_TRY(cudaStreamSynchronize(st));
        total = t;
        *h_needed = total;
        if (total > ctx->capacity) return SPH_ERR_NB_OVERFLOW;
    }
    if (n > 0) SPH_CUDA_TRY(cudaMemsetAsync(ctx->rev, 0, sizeof(int) * (size_t)n, st));
    if ((rc = launch_nb_fill(a, st))) return rc;
    if ((rc = launch_segsort_rows(ctx->nb_start, ctx->own, n, (int)ctx->capacity, ctx->nb_idx,
                                  ctx->tmp, ctx->long_list, ctx->long_count, st)))
        return rc;
    ctx->nb_built = 1;
    if (d_nb_start_out)
        SPH_CUDA_TRY(cudaMemcpyAsync(d_nb_start_out, ctx->nb_start, sizeof(int) * ((size_t)n + 1),
                                     cudaMemcpyDeviceToDevice, st));
    if (d_nb_idx_out) {
        if (total < 0) {
            int t = 0;
            SPH_CUDA_TRY(cudaMemcpyAsync(&t, ctx->nb_start + n, sizeof(int), cudaMemcpyDeviceToHost, st));
            SPH_CUDA_TRY(cudaStreamSynchronize(st));
            total = t;
        }
        if (total <= out_capacity && total <= ctx->capacity && total > 0)
            SPH_CUDA_TRY(cudaMemcpyAsync(d_nb_idx_out, ctx->nb_idx, sizeof(int) * (size_t)total,
                                         cudaMemcpyDeviceToDevice, st));
        else if (total > out_capacity)
            return SPH_ERR_NB_OVERFLOW;
    }
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// DC, HFC
// ---------------------------------------------------------------------------

extern "C" int sph_density(sph_ctx *ctx, int32_t n_gas, const float *d_mass, float *d_rho,
                           float *d_h_next, sph_stream_t stream) {
    if (!ctx || n_gas != ctx->n_sorted || !ctx->nb_built) return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && (!d_mass || !d_rho || !d_h_next)) return SPH_ERR_INVALID_ARG;
    return launch_density(ctx->pos_h_s, d_mass, ctx->perm, ctx->nb_start, ctx->nb_idx,
                          (int)ctx->capacity, n_gas, ctx->params.sigma, ctx->hydro_lanes,
                          ctx->rho_s, d_rho, d_h_next, ctx->mass_s, ctx->flags + 1, (cudaStream_t)stream);
}

extern "C" int sph_forces(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
                          const float *d_mass, float *d_acc_dedt, sph_stream_t stream) {
    if (!ctx || n_gas != ctx->n_sorted || !ctx->nb_built) return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && (!d_vel_e || !d_rho || !d_mass || !d_acc_dedt || !aligned16(d_vel_e) ||
                      !aligned16(d_acc_dedt)))
        return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HydroParams hp = hydro_params(ctx);
    int rc;
    if ((rc = launch_hydro_prep(reinterpret_cast<const float4 *>(d_vel_e), d_rho, d_mass, ctx->perm,
                                n_gas, hp, ctx->vel_s, ctx->aux_s, st)))
        return rc;
    return launch_forces(ctx->pos_h_s, ctx->vel_s, ctx->aux_s, ctx->perm, ctx->nb_start,
                         ctx->nb_idx, (int)ctx->capacity, n_gas, hp, ctx->hydro_lanes,
                         reinterpret_cast<float4 *>(d_acc_dedt), st);
}

extern "C" int sph_cfl_dt(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
                          const float *d_mass, const float *d_acc_hyd, const float *d_grav,
                          float C_cfl, float *d_dt_particle, float *d_dt_min, sph_stream_t stream) {
    if (!ctx || n_gas != ctx->n_sorted || !ctx->nb_built || !d_dt_min || !(C_cfl > 0.0f))
        return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && (!d_vel_e || !d_rho || !d_mass || !d_acc_hyd || !d_grav || !aligned16(d_vel_e) ||
                      !aligned16(d_acc_hyd) || !aligned16(d_grav)))
        return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HydroParams hp = hydro_params(ctx);
    int rc;
    if ((rc = launch_hydro_prep(reinterpret_cast<const float4 *>(d_vel_e), d_rho, d_mass, ctx->perm,
                                n_gas, hp, ctx->vel_s, ctx->aux_s, st)))
        return rc;
    return launch_cfl(ctx->pos_h_s, ctx->vel_s, ctx->aux_s, ctx->perm, ctx->nb_start, ctx->nb_idx,
                      (int)ctx->capacity, n_gas, hp, C_cfl,
                      reinterpret_cast<const float4 *>(d_acc_hyd),
                      reinterpret_cast<const float4 *>(d_grav), d_dt_particle, d_dt_min,
                      std::numeric_limits<float>::infinity(), st);
}

extern "C" int sph_forces_cfl(sph_ctx *ctx, int32_t n_gas, const float *d_vel_e, const float *d_rho,
                              const float *d_mass, float *d_acc_dedt, const float *d_grav,
                              float C_cfl, float dt_max, float *d_dt_particle, float *d_dt_min,
                              sph_stream_t stream) {
    if (!ctx || n_gas != ctx->n_sorted || !ctx->nb_built || !d_dt_min || !(C_cfl > 0.0f) ||
        !(dt_max > 0.0f))
        return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && (!d_vel_e || !d_rho || !d_mass || !d_acc_dedt || !d_grav ||
                      !aligned16(d_vel_e) || !aligned16(d_acc_dedt) || !aligned16(d_grav)))
        return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    HydroParams hp = hydro_params(ctx);
    int rc;
    if ((rc = launch_hydro_prep(reinterpret_cast<const float4 *>(d_vel_e), d_rho, d_mass, ctx->perm,
                                n_gas, hp, ctx->vel_s, ctx->aux_s, st)))
        return rc;
    return launch_forces(ctx->pos_h_s, ctx->vel_s, ctx->aux_s, ctx->perm, ctx->nb_start,
                         ctx->nb_idx, (int)ctx->capacity, n_gas, hp, ctx->hydro_lanes,
                         reinterpret_cast<float4 *>(d_acc_dedt), st,
                         reinterpret_cast<const float4 *>(d_grav), C_cfl, d_dt_particle, d_dt_min,
                         dt_max);
}

// ---------------------------------------------------------------------------
// Whole steps
// ---------------------------------------------------------------------------

namespace {

bool state_ok(const sph_ctx *ctx, const SphState *s) {
    if (!s || s->n < 0 || s->n_gas < 0 || s->n_gas > s->n) return false;
    if (s->n_gas > 0 && (!ctx || s->n_gas > ctx->n_max)) return false;
    if (s->n > 0 && (!s->r || !s->v || !s->v_save || !s->mass || !s->pos_m || !s->grav))
        return false;
    if (s->n_gas > 0 && (!s->e || !s->e_save || !s->h || !s->pos_h || !s->vel_e || !s->rho ||
                         !s->acc_hyd))
        return false;
    return true;
}

int gravity_of(sph_ctx *ctx, SphState *s, sph_stream_t stream) {
    const float G = ctx ? ctx->params.G : 1.0f, eps = ctx ? ctx->params.eps : 0.0f;
    if (ctx && ctx->batch) {
        if (ctx->batch->n != s->n || ctx->batch->n_gas != s->n_gas) return SPH_ERR_INVALID_ARG;
        if (s->grav_work)
            return pp_gravity_pairs_batched(ctx->batch, s->pos_m, G, eps, s->grav, s->grav_flags,
                                            s->grav_work, s->grav_work_bytes, stream);
        return pp_gravity_batched(ctx->batch, s->pos_m, G, eps, s->grav, s->grav_flags, stream);
    }
    if (s->grav_work)
        return pp_gravity_pairs(s->pos_m, s->n, G, eps, s->grav, s->grav_flags, s->grav_work,
                                s->grav_work_bytes, stream);
    return pp_gravity(s->pos_m, s->n, G, eps, s->grav, s->grav_flags, stream);
}

int rhs_gas(sph_ctx *ctx, SphState *s, cudaStream_t st) {
    int rc;
    if ((rc = sph_bin_and_sort(ctx, s->pos_h, s->n_gas, nullptr, nullptr, nullptr, nullptr,
                               (sph_stream_t)st)))
        return rc;
    if ((rc = sph_build_neighbors(ctx, s->n_gas, nullptr, nullptr, 0, nullptr, (sph_stream_t)st)))
        return rc;
    return sph_density(ctx, s->n_gas, s->mass, s->rho, s->h, (sph_stream_t)st);
}

}  // namespace

extern "C" int sph_rhs_initial(sph_ctx *ctx, SphState *s, sph_stream_t stream) {
    if (!state_ok(ctx, s)) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = integrate_step(SPH_EMIT, 0.0, s->n, s->n_gas, s->r, s->v, s->e, s->v_save, s->e_save,
                             s->acc_hyd, s->grav, s->mass, s->h, s->pos_m, s->pos_h, s->vel_e,
                             stream)))
        return rc;
    if (s->n_gas > 0 && (rc = rhs_gas(ctx, s, st))) return rc;
    if ((rc = gravity_of(ctx, s, stream))) return rc;
    if (s->n_gas > 0 &&
        (rc = sph_forces(ctx, s->n_gas, s->vel_e, s->rho, s->mass, s->acc_hyd, stream)))
        return rc;
    s->fresh = 1;
    return SPH_OK;
}

namespace {

struct StageMark {
    void **ev;
    cudaStream_t st;
    int begin(int k) const {
        if (ev) SPH_CUDA_TRY(cudaEventRecord((cudaEvent_t)ev[2 * k], st));
        return SPH_OK;
    }
    int end(int k) const {
        if (ev) SPH_CUDA_TRY(cudaEventRecord((cudaEvent_t)ev[2 * k + 1], st));
        return SPH_OK;
    }
};

}  // namespace

#define SPH_STAGE(k, expr)                  \
    do {                                    \
        if ((rc = mark.begin(k))) return rc; \
        if ((rc = (expr))) return rc;        \
        if ((rc = mark.end(k))) return rc;   \
    } while (0)

extern "C" int sph_step(sph_ctx *ctx, SphState *s, double dt, sph_stream_t stream) {
    if (!state_ok(ctx, s) || !(dt == dt) || !ctx) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const StageMark mark{s->events, st};
    const bool gas = s->n_gas > 0;
    int rc;
    // HFC at (r_n, v_n, e_n) on the lists and density of r_n
    SPH_STAGE(SPH_STAGE_HFC_PRED,
              (!s->fresh && gas) ? sph_forces(ctx, s->n_gas, s->vel_e, s->rho, s->mass, s->acc_hyd,
                                              stream)
                                 : SPH_OK);
    // SU predictor: v~, e~, r_{n+1}; FP32 copies with the next h
    SPH_STAGE(SPH_STAGE_SU_PRED,
              integrate_step(SPH_PREDICT, dt, s->n, s->n_gas, s->r, s->v, s->e, s->v_save,
                             s->e_save, s->acc_hyd, s->grav, s->mass, s->h, s->pos_m, s->pos_h,
                             s->vel_e, stream));
    // SP, lists, DC at r_{n+1}
    SPH_STAGE(SPH_STAGE_SP, gas ? sph_bin_and_sort(ctx, s->pos_h, s->n_gas, nullptr, nullptr,
                                                   nullptr, nullptr, stream)
                                : SPH_OK);
    SPH_STAGE(SPH_STAGE_NB,
              gas ? sph_build_neighbors(ctx, s->n_gas, nullptr, nullptr, 0, nullptr, stream) : SPH_OK);
    SPH_STAGE(SPH_STAGE_DC, gas ? sph_density(ctx, s->n_gas, s->mass, s->rho, s->h, stream) : SPH_OK);
    // GFC once per step at r_{n+1}
    SPH_STAGE(SPH_STAGE_GFC, gravity_of(ctx, s, stream));
    // HFC at (r_{n+1}, v~, e~)
    SPH_STAGE(SPH_STAGE_HFC_CORR,
              gas ? sph_forces(ctx, s->n_gas, s->vel_e, s->rho, s->mass, s->acc_hyd, stream) : SPH_OK);
    // SU corrector
    SPH_STAGE(SPH_STAGE_SU_CORR,
              integrate_step(SPH_CORRECT, dt, s->n, s->n_gas, s->r, s->v, s->e, s->v_save,
                             s->e_save, s->acc_hyd, s->grav, s->mass, s->h, nullptr, nullptr,
                             s->vel_e, stream));
    s->fresh = 0;
    return SPH_OK;
}

extern "C" int sph_step_cfl(sph_ctx *ctx, SphState *s, float C_cfl, float dt_max, float *d_dt,
                            sph_stream_t stream) {
    if (!state_ok(ctx, s) || !ctx || s->n_gas < 1 || !d_dt || !(C_cfl > 0.0f) || !(dt_max > 0.0f))
        return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const StageMark mark{s->events, st};
    int rc;
    // HFC at (r_n, v_n, e_n) with the time step of Eq. 17 in the same pass
    // (right after sph_rhs_initial the forces are current: only the step)
    if (s->fresh) {
        HydroParams hp = hydro_params(ctx);
        SPH_STAGE(SPH_STAGE_HFC_PRED,
                  launch_cfl(ctx->pos_h_s, ctx->vel_s, ctx->aux_s, ctx->perm, ctx->nb_start,
                             ctx->nb_idx, (int)ctx->capacity, s->n_gas, hp, C_cfl,
                             reinterpret_cast<const float4 *>(s->acc_hyd),
                             reinterpret_cast<const float4 *>(s->grav), nullptr, d_dt, dt_max, st));
    } else {
        SPH_STAGE(SPH_STAGE_HFC_PRED,
                  sph_forces_cfl(ctx, s->n_gas, s->vel_e, s->rho, s->mass, s->acc_hyd, s->grav,
                                 C_cfl, dt_max, nullptr, d_dt, stream));
    }
    // the rest of the step as in sph_step, with the step size read on the device
    SPH_STAGE(SPH_STAGE_SU_PRED,
              integrate_launch(SPH_PREDICT, 0.0, d_dt, s->n, s->n_gas, s->r, s->v, s->e, s->v_save,
                               s->e_save, s->acc_hyd, s->grav, s->mass, s->h, s->pos_m, s->pos_h,
                               s->vel_e, stream));
    SPH_STAGE(SPH_STAGE_SP, sph_bin_and_sort(ctx, s->pos_h, s->n_gas, nullptr, nullptr, nullptr,
                                             nullptr, stream));
    SPH_STAGE(SPH_STAGE_NB, sph_build_neighbors(ctx, s->n_gas, nullptr, nullptr, 0, nullptr, stream));
    SPH_STAGE(SPH_STAGE_DC, sph_density(ctx, s->n_gas, s->mass, s->rho, s->h, stream));
    SPH_STAGE(SPH_STAGE_GFC, gravity_of(ctx, s, stream));
    SPH_STAGE(SPH_STAGE_HFC_CORR,
              sph_forces(ctx, s->n_gas, s->vel_e, s->rho, s->mass, s->acc_hyd, stream));
    SPH_STAGE(SPH_STAGE_SU_CORR,
              integrate_launch(SPH_CORRECT, 0.0, d_dt, s->n, s->n_gas, s->r, s->v, s->e, s->v_save,
                               s->e_save, s->acc_hyd, s->grav, s->mass, s->h, nullptr, nullptr,
                               s->vel_e, stream));
    s->fresh = 0;
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent simulations
// ---------------------------------------------------------------------------

namespace {

bool offsets_ok(int n_sims, const int32_t *off) {
    if (!off || off[0] != 0) return false;
    for (int s = 0; s < n_sims; ++s)
        if (off[s + 1] < off[s]) return false;
    return true;
}

size_t batch_units_cap(int n_sims, const int32_t *g, const int32_t *d) {
    size_t u = 0;
    for (int s = 0; s < n_sims; ++s) {
        long long ns = (long long)(g[s + 1] - g[s]) + (d[s + 1] - d[s]);
        u += (size_t)((ns + 511) / 512);   // R = 2 gives the most units
    }
    return u + 1;
}

struct BatchCarve {
    size_t sims, units, counter, tile_off, scales, total;
};

BatchCarve batch_carve(int n_sims, size_t units_cap) {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    BatchCarve c;
    c.sims = 0;
    c.units = up(sizeof(int4) * (size_t)n_sims);
    c.counter = c.units + up(sizeof(int2) * units_cap);
    c.tile_off = c.counter + 256;
    c.scales = c.tile_off + kPairsNumShapes * up(sizeof(long long) * ((size_t)n_sims + 1));
    c.total = c.scales + up(pairs_scale_bytes() * (size_t)n_sims);
    return c;
}

int batch_build_units(sph_batch *b, int R, cudaStream_t st) {
    const int per = 256 * R;
    std::vector<int> order(b->n_sims);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return b->h_sims[x].y + b->h_sims[x].w > b->h_sims[y].y + b->h_sims[y].w;
    });
    b->h_units.clear();
    for (int s : order) {
        const int ns = b->h_sims[s].y + b->h_sims[s].w;
        for (int v = 0; v < ns; v += per) b->h_units.push_back(make_int2(s, v));
    }
    if (b->h_units.size() > b->units_cap) return SPH_ERR_INVALID_ARG;
    b->R = R;
    if (!b->h_units.empty())
        SPH_CUDA_TRY(cudaMemcpyAsync(b->d_units, b->h_units.data(), sizeof(int2) * b->h_units.size(),
                                     cudaMemcpyHostToDevice, st));
    return SPH_OK;
}

}  // namespace

extern "C" size_t sph_batch_workspace_bytes(int32_t n_sims, const int32_t *h_gas_off,
                                           const int32_t *h_dark_off) {
    if (n_sims < 1 || !offsets_ok(n_sims, h_gas_off) || !offsets_ok(n_sims, h_dark_off)) return 0;
    return batch_carve(n_sims, batch_units_cap(n_sims, h_gas_off, h_dark_off)).total;
}

extern "C" int sph_batch_create(int32_t n_sims, const int32_t *h_gas_off, const int32_t *h_dark_off,
                                const int32_t *d_sim_of_gas, void *d_workspace,
                                size_t workspace_bytes, sph_stream_t stream, sph_batch **out) {
    if (!out || n_sims < 1 || !offsets_ok(n_sims, h_gas_off) || !offsets_ok(n_sims, h_dark_off))
        return SPH_ERR_INVALID_ARG;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return SPH_ERR_INVALID_ARG;
    const long long n_gas = h_gas_off[n_sims], n = n_gas + h_dark_off[n_sims];
    if (n > 0x7fffffffLL || (n_gas > 0 && !d_sim_of_gas)) return SPH_ERR_INVALID_ARG;
    const size_t cap = batch_units_cap(n_sims, h_gas_off, h_dark_off);
    const BatchCarve c = batch_carve(n_sims, cap);
    if (workspace_bytes < c.total) return SPH_ERR_INVALID_ARG;
    sph_batch *b = new (std::nothrow) sph_batch;
    if (!b) return SPH_ERR_INVALID_ARG;
    b->n_sims = n_sims;
    b->n_gas = (int)n_gas;
    b->n = (int)n;
    b->h_gas_off.assign(h_gas_off, h_gas_off + n_sims + 1);
    b->h_dark_off.assign(h_dark_off, h_dark_off + n_sims + 1);
    b->h_sims.resize(n_sims);
    for (int s = 0; s < n_sims; ++s)
        b->h_sims[s] = make_int4(h_gas_off[s], h_gas_off[s + 1] - h_gas_off[s],
                                 (int)n_gas + h_dark_off[s], h_dark_off[s + 1] - h_dark_off[s]);
    char *base = static_cast<char *>(d_workspace);
    b->d_sims = reinterpret_cast<int4 *>(base + c.sims);
    b->d_units = reinterpret_cast<int2 *>(base + c.units);
    b->d_counter = reinterpret_cast<int *>(base + c.counter);
    b->units_cap = cap;
    b->d_sim_of_gas = d_sim_of_gas;
    const size_t off_stride = (sizeof(long long) * ((size_t)n_sims + 1) + 255) & ~size_t(255);
    for (int k = 0; k < kPairsNumShapes; ++k)
        b->d_tile_off[k] = reinterpret_cast<long long *>(base + c.tile_off + k * off_stride);
    b->d_pair_scales = base + c.scales;
    std::vector<long long> tile_off[kPairsNumShapes];
    for (int k = 0; k < kPairsNumShapes; ++k) {
        tile_off[k].assign(n_sims + 1, 0);
        for (int s = 0; s < n_sims; ++s)
            tile_off[k][s + 1] = tile_off[k][s] + pairs_tiles((long long)b->h_sims[s].y + b->h_sims[s].w,
                                                              pairs_shape_block(k));
        b->n_pair_tiles[k] = tile_off[k][n_sims];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = SPH_OK;
    if (cudaMemcpyAsync(b->d_sims, b->h_sims.data(), sizeof(int4) * n_sims, cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        rc = SPH_ERR_CUDA;
    for (int k = 0; k < kPairsNumShapes && rc == SPH_OK; ++k)
        if (cudaMemcpyAsync(b->d_tile_off[k], tile_off[k].data(), sizeof(long long) * (n_sims + 1),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = SPH_ERR_CUDA;
    if (rc == SPH_OK) rc = batch_build_units(b, 4, st);
    if (rc == SPH_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SPH_ERR_CUDA;
    if (rc != SPH_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return SPH_OK;
}

extern "C" int sph_batch_destroy(sph_batch *b) {
    delete b;
    return SPH_OK;
}

extern "C" int sph_batch_set_plan(sph_batch *b, int32_t R, sph_stream_t stream) {
    if (!b || (R != 2 && R != 4 && R != 8)) return SPH_ERR_INVALID_ARG;
    int rc = batch_build_units(b, R, (cudaStream_t)stream);
    if (rc) return rc;
    SPH_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return SPH_OK;
}

extern "C" int pp_gravity_batched(const sph_batch *b, const float *d_pos_m, float G, float eps,
                                  float *d_acc_pot, int32_t flags, sph_stream_t stream) {
    if (!b || !(eps >= 0.0f) || !(G == G)) return SPH_ERR_INVALID_ARG;
    if (b->n == 0) return SPH_OK;
    if (!d_pos_m || !d_acc_pot || !aligned16(d_pos_m) || !aligned16(d_acc_pot))
        return SPH_ERR_INVALID_ARG;
    return launch_gravity_batched(reinterpret_cast<const float4 *>(d_pos_m), b->d_sims, b->d_units,
                                  (int)b->h_units.size(), b->d_counter, b->R, G, eps,
                                  reinterpret_cast<float4 *>(d_acc_pot), flags, (cudaStream_t)stream);
}

extern "C" int pp_gravity_pairs_batched(const sph_batch *b, const float *d_pos_m, float G,
                                        float eps, float *d_acc_pot, int32_t flags, void *d_work,
                                        size_t work_bytes, sph_stream_t stream) {
    if (!b || !(eps >= 0.0f) || !(G == G)) return SPH_ERR_INVALID_ARG;
    if (b->n == 0) return SPH_OK;
    const int shape = pairs_current_shape();
    if (!pp_gravity_pairs_eligible(b->n, eps, flags) || !d_work ||
        work_bytes < pp_gravity_pairs_workspace_bytes(b->n) || b->n_pair_tiles[shape] > 0x7fffffffll)
        return pp_gravity_batched(b, d_pos_m, G, eps, d_acc_pot, flags, stream);
    if (!d_pos_m || !d_acc_pot || !aligned16(d_pos_m) || !aligned16(d_acc_pot) ||
        (reinterpret_cast<uintptr_t>(d_work) & 255u))
        return SPH_ERR_INVALID_ARG;
    return launch_gravity_pairs_batched(reinterpret_cast<const float4 *>(d_pos_m), b->n, b->n_gas,
                                        b->d_sims, b->d_tile_off[shape], b->n_sims,
                                        b->n_pair_tiles[shape], shape, b->d_pair_scales, G, eps,
                                        reinterpret_cast<float4 *>(d_acc_pot), flags, d_work,
                                        (cudaStream_t)stream);
}

extern "C" int sph_ctx_set_batch(sph_ctx *ctx, const sph_batch *b) {
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (b && b->n_gas > ctx->n_max) return SPH_ERR_INVALID_ARG;
    ctx->batch = b;
    return SPH_OK;
}
