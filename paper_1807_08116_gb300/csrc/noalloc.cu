// noalloc.cu -- a variant of the grid sort (sph_bin_and_sort) for callers
// that cannot allocate device memory.
//
// sph_bin_and_sort needs a context whose workspace the caller allocates.
// Some callers cannot do that: a host framework that owns every device
// allocation through its own fixed arena, a plugin that is given only its
// input and output buffers, or a latency-critical loop that must never call
// cudaMalloc (it can synchronise the whole device).  This entry point uses
// instead one file-scope device array of fixed size as its scratch, so it
// allocates nothing; the caller still passes the particle input and the three
// result arrays.
//
// The array is created when the library is loaded and every GPU that loads
// the library holds it (SPH_NOALLOC_SCRATCH_BYTES) until the process exits.
// All calls on a device share it and it keeps the last call's contents, so
// two calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on it; order them, e.g. issue them on one stream.
#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

// Scratch layout, each part 256-byte aligned (limits in include/sphgb.h):
//   count[M], long_list[max(n, M)], tmp[n], block_sums[..], grid, red[8],
//   long_count[4]
constexpr long long kNaM = 1ll << SPH_NOALLOC_MAX_LOG2_M;
constexpr long long kNaN = SPH_NOALLOC_MAX_GAS;
constexpr long long kNaSeg = kNaM > kNaN ? kNaM : kNaN;
constexpr long long kNaBlocks = (kNaSeg + 1 + 4095) / 4096 + 32;

constexpr size_t na_up(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCount = 0;
constexpr size_t kOffLong = kOffCount + na_up(sizeof(int) * kNaM);
constexpr size_t kOffTmp = kOffLong + na_up(sizeof(int) * kNaSeg);
constexpr size_t kOffBlocks = kOffTmp + na_up(sizeof(int) * kNaN);
constexpr size_t kOffGrid = kOffBlocks + na_up(sizeof(int) * kNaBlocks);
constexpr size_t kOffRed = kOffGrid + na_up(sizeof(GridDev));
constexpr size_t kOffLongCount = kOffRed + na_up(sizeof(unsigned) * 8);
constexpr size_t kNaBytes = kOffLongCount + na_up(sizeof(int) * 4);
static_assert(kNaBytes <= SPH_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPH_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array.  The host-side name of the array is
// not a device address, so it is looked up with the caller's device current.
// The lookup is repeated on every call (a cheap host call): an address kept
// from an earlier call would belong to the context it was taken in, and is
// stale after cudaDeviceReset or under another context on the same device.
static int noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    SPH_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) return SPH_ERR_CUDA;
    *out = static_cast<unsigned char *>(p);
    return SPH_OK;
}

}  // namespace sphgb

using namespace sphgb;

extern "C" int sph_bin_and_sort_noalloc(const float *d_pos_h, int32_t n_gas, int32_t log2_M,
                                        const SphGrid *h_grid, int32_t *d_key,
                                        int32_t *d_cell_start, int32_t *d_perm,
                                        sph_stream_t stream) {
    if (n_gas < 0 || n_gas > SPH_NOALLOC_MAX_GAS) return SPH_ERR_INVALID_ARG;
    if (log2_M < 4 || log2_M > SPH_NOALLOC_MAX_LOG2_M) return SPH_ERR_INVALID_ARG;
    if (!d_cell_start || (n_gas > 0 && (!d_pos_h || !d_key || !d_perm))) return SPH_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_pos_h) & 15u) return SPH_ERR_INVALID_ARG;
    if (h_grid && (h_grid->log2_M != log2_M || h_grid->n_levels < 1 ||
                   h_grid->n_levels > kMaxLevels || h_grid->log2_L0 < -100 ||
                   h_grid->log2_L0 > 100 || !(h_grid->x0 == h_grid->x0) ||
                   !(h_grid->y0 == h_grid->y0) || !(h_grid->z0 == h_grid->z0)))
        return SPH_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    int *count = reinterpret_cast<int *>(base + kOffCount);
    int *long_list = reinterpret_cast<int *>(base + kOffLong);
    int *tmp = reinterpret_cast<int *>(base + kOffTmp);
    int *block_sums = reinterpret_cast<int *>(base + kOffBlocks);
    GridDev *grid = reinterpret_cast<GridDev *>(base + kOffGrid);
    unsigned *red = reinterpret_cast<unsigned *>(base + kOffRed);
    int *long_count = reinterpret_cast<int *>(base + kOffLongCount);

    cudaStream_t st = (cudaStream_t)stream;
    const float4 *pos = reinterpret_cast<const float4 *>(d_pos_h);
    const int M = 1 << log2_M;
    if (h_grid) rc = launch_grid_set(*h_grid, grid, st);
    else rc = launch_grid_auto(pos, n_gas, red, log2_M, grid, st);
    if (rc) return rc;
    // the shared array keeps the previous call's contents: clear the counters
    SPH_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)M, st));
    if ((rc = launch_bin(pos, nullptr, n_gas, grid, d_key, count, st))) return rc;
    if ((rc = launch_scan_exclusive(count, M, d_cell_start, block_sums, st))) return rc;
    if ((rc = launch_scatter(d_key, n_gas, d_cell_start, count, tmp, st))) return rc;
    return launch_sort_buckets(d_key, n_gas, d_cell_start, tmp, d_perm, long_list, long_count, st);
}
