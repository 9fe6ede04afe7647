// sort.cu -- the sorting stage SP of the paper (Sect. 3): binning of the gas
// particles into buckets of a multi-level hashed grid, bucket counts, a
// block-cascaded exclusive prefix sum, the counting-sort scatter, and the
// canonicalisation that makes the scatter stable (ascending original index
// inside a bucket) and so deterministic.
//
// The paper's SP1 counts with global atomics, SP2 scans inside a CUDA block
// in shared memory and adds each block total into every later block with
// atomics (O(G^2) adds), SP3 adds the block offsets, SP4 scatters with an
// atomic cursor.  Here SP2/SP3 become a reduce-then-scan cascade (warp
// shuffles, then shared memory, then one pass over block totals) with no
// spin-waits, and SP4's arbitrary within-bucket order is repaired by a rank
// pass (a particle's place is the number of its bucket's members with a
// smaller index).  The same file holds the segmented sort that orders the
// reverse part of each neighbour row.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

// ---------------------------------------------------------------------------
// Automatic grid: origin floor(min x) - 1 per axis, L0 = 2^ceil(log2 min h),
// n_levels = 1 + ceil(log2(max h / L0)) (at most 24).
// red[0..2] ordered-min of x, y, z; red[3] ordered-min of h; red[4] ordered-max of h.
// ---------------------------------------------------------------------------

__global__ void grid_reduce_kernel(const float4 *__restrict__ pos_h, int n, unsigned *red) {
    __shared__ unsigned s[5];
    if (threadIdx.x < 5) s[threadIdx.x] = threadIdx.x == 4 ? 0u : 0xffffffffu;
    __syncthreads();
    unsigned mx = 0xffffffffu, my = 0xffffffffu, mz = 0xffffffffu, mh = 0xffffffffu, Mh = 0u;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 p = pos_h[i];
        if (p.x == p.x && fabsf(p.x) < 3.0e38f) mx = min(mx, float_to_ordered(p.x));
        if (p.y == p.y && fabsf(p.y) < 3.0e38f) my = min(my, float_to_ordered(p.y));
        if (p.z == p.z && fabsf(p.z) < 3.0e38f) mz = min(mz, float_to_ordered(p.z));
        if (p.w > 0.0f && p.w < 3.0e38f) {
            mh = min(mh, float_to_ordered(p.w));
            Mh = max(Mh, float_to_ordered(p.w));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = min(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = min(my, __shfl_xor_sync(0xffffffffu, my, o));
        mz = min(mz, __shfl_xor_sync(0xffffffffu, mz, o));
        mh = min(mh, __shfl_xor_sync(0xffffffffu, mh, o));
        Mh = max(Mh, __shfl_xor_sync(0xffffffffu, Mh, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&s[0], mx); atomicMin(&s[1], my); atomicMin(&s[2], mz);
        atomicMin(&s[3], mh); atomicMax(&s[4], Mh);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMin(&red[0], s[0]); atomicMin(&red[1], s[1]); atomicMin(&red[2], s[2]);
        atomicMin(&red[3], s[3]); atomicMax(&red[4], s[4]);
    }
}

__device__ __forceinline__ int ceil_log2_pos(float v) {
    // ceil(log2(v)) for finite v > 0, exact from the FP32 bits
    unsigned b = __float_as_uint(v);
    int e = (int)((b >> 23) & 0xffu);
    unsigned mant = b & 0x7fffffu;
    if (e == 0) {   // subnormal: v = mant * 2^-149
        int lz = __clz(mant) - 8;   // leading zeros within 23 bits
        int top = 22 - lz;          // index of highest set bit
        int fl = top - 149;
        return (mant & ((1u << top) - 1u)) ? fl + 1 : fl;
    }
    int fl = e - 127;
    return mant ? fl + 1 : fl;
}

// The grid from the reduced extremes: red[0..3] ordered-min of x, y, z, h
// (0xffffffff: none), red[4] ordered-max of h (0: none).
__device__ __forceinline__ GridDev grid_from_red(const unsigned red[5], int log2_M, int shift) {
    float mins[3];
    for (int d = 0; d < 3; ++d) {
        float v = red[d] == 0xffffffffu ? 0.0f : ordered_to_float(red[d]);
        mins[d] = floorf(v) - 1.0f;
    }
    float hmin = red[3] == 0xffffffffu ? 1.0f : ordered_to_float(red[3]);
    float hmax = red[4] == 0u ? hmin : ordered_to_float(red[4]);
    // shift moves the finest cell size by whole octaves (a tuning knob)
    int l0 = ceil_log2_pos(hmin) + shift;
    l0 = max(-100, min(100, l0));
    int top = ceil_log2_pos(hmax) - l0;   // levels above L0 needed for hmax
    int nl = 1 + max(0, top);
    nl = min(nl, 24);
    GridDev g;
    g.x0 = mins[0];
    g.y0 = mins[1];
    g.z0 = mins[2];
    g.log2_L0 = l0;
    g.n_levels = nl;
    g.log2_M = log2_M;
    return g;
}

__global__ void grid_finalize_kernel(const unsigned *red, int log2_M, int shift, GridDev *grid) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned r[5] = {red[0], red[1], red[2], red[3], red[4]};
    *grid = grid_from_red(r, log2_M, shift);
}

__global__ void grid_set_kernel(GridDev g, GridDev *grid) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *grid = g;
}

// ---------------------------------------------------------------------------
// SP1: bucket of each particle and the bucket counts.  The statistics the
// neighbour search needs (per-bucket and per-level max h, per-level counts,
// super-cell occupancy) are taken after the sort, in gather_bin_kernel, where
// the particles of a bucket are adjacent and a warp needs one atomic per run
// of equal values instead of one per particle on scattered addresses.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int bucket_of_particle(const float4 &p, int sim, const GridDev &g, int &l,
                                                  int &cx, int &cy, int &cz) {
    l = level_of(p.w, g.log2_L0, g.n_levels);
    const float inv_c = pow2f(-g.log2_L0 - l);
    cx = cell_of(p.x, g.x0, inv_c);
    cy = cell_of(p.y, g.y0, inv_c);
    cz = cell_of(p.z, g.z0, inv_c);
    // simulations of a batch share the grid; the simulation index enters the
    // bucket hash next to the level (0 for a single simulation)
    return bucket_of(cx, cy, cz, l + kMaxLevels * sim, g.log2_M);
}

__global__ void bin_kernel(const float4 *__restrict__ pos_h, const int *__restrict__ sim_of, int n,
                           const GridDev *__restrict__ gridp, int *__restrict__ key,
                           int *__restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GridDev g = *gridp;
    int l, cx, cy, cz;
    const int k = bucket_of_particle(pos_h[i], sim_of ? sim_of[i] : 0, g, l, cx, cy, cz);
    key[i] = k;
    atomicAdd(&count[k], 1);
}

// Sorted copies of (x, y, z, h) and of the simulation index, plus the
// statistics: hmax_cell[k] (max h of bucket k; NaN or h <= 0 count as 0),
// the occupancy bit of every occupied super-cell (occ may be NULL), and the
// count and max h of every level.
__global__ void gather_bin_kernel(const float4 *__restrict__ pos_h, const int *__restrict__ sim_of,
                                  const int *__restrict__ perm, int n,
                                  const GridDev *__restrict__ gridp, float4 *__restrict__ pos_h_s,
                                  int *__restrict__ sim_s, unsigned *__restrict__ tag_s,
                                  unsigned *__restrict__ occ, int log2_B,
                                  unsigned *__restrict__ hmax_cell, int *__restrict__ lvl_count,
                                  unsigned *__restrict__ lvl_hmax) {
    __shared__ int s_cnt[kMaxLevels];
    __shared__ unsigned s_hmax[kMaxLevels];
    if (threadIdx.x < kMaxLevels) {
        s_cnt[threadIdx.x] = 0;
        s_hmax[threadIdx.x] = 0u;
    }
    __syncthreads();
    const GridDev g = *gridp;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int l = -1, k = -1;
    unsigned hb = 0u, sbit = 0xffffffffu;   // no super-cell bit reaches 2^31
    if (j < n) {
        const int i = perm[j];
        const float4 p = pos_h[i];
        pos_h_s[j] = p;
        const int sim = sim_of ? sim_of[i] : 0;
        if (sim_s) sim_s[j] = sim;
        int cx, cy, cz;
        k = bucket_of_particle(p, sim, g, l, cx, cy, cz);
        if (tag_s) tag_s[j] = cell_tag(l, cx, cy, cz);
        hb = (p.w > 0.0f) ? __float_as_uint(p.w) : 0u;   // NaN / <= 0 -> 0
        if (occ)
            sbit = super_bit(cx >> kSuperShift, cy >> kSuperShift, cz >> kSuperShift,
                             l + kMaxLevels * sim, log2_B);
    }
    {
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const unsigned m = __reduce_max_sync(peers, hb);
        if (k >= 0 && lane == __ffs(peers) - 1 && m > 0u) atomicMax(&hmax_cell[k], m);
    }
    if (occ) {
        const unsigned peers = __match_any_sync(0xffffffffu, sbit);
        if (k >= 0 && lane == __ffs(peers) - 1) atomicOr(&occ[sbit >> 5], 1u << (sbit & 31));
    }
    // per-level totals: one shared atomic per (warp, level)
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const unsigned hpeer = __reduce_max_sync(peers, hb);
    if (l >= 0 && lane == __ffs(peers) - 1) {
        atomicAdd(&s_cnt[l], __popc(peers));
        atomicMax(&s_hmax[l], hpeer);
    }
    __syncthreads();
    if (threadIdx.x < kMaxLevels && s_cnt[threadIdx.x]) {
        atomicAdd(&lvl_count[threadIdx.x], s_cnt[threadIdx.x]);
        atomicMax(&lvl_hmax[threadIdx.x], s_hmax[threadIdx.x]);
    }
}

// ---------------------------------------------------------------------------
// SP2/SP3: exclusive prefix sum, reduce-then-scan cascade.
// out[0..n] with out[n] = total.  Each block covers SCAN_TILE inputs.
// ---------------------------------------------------------------------------

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total.
__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < nw) s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == nw - 1) s_warp[32] = wi;
    }
    __syncthreads();
    int res = inc - v + s_warp[warp];
    *total = s_warp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const int *__restrict__ in, int n,
                                                                    int *__restrict__ block_sums) {
    __shared__ int s_warp[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) v += in[base + q];
    int total;
    block_excl_scan(v, s_warp, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block totals, in place (any count).
__global__ void __launch_bounds__(SCAN_THREADS) scan_blocks_kernel(int *block_sums, int nb) {
    __shared__ int s_warp[33];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        int idx = b0 + threadIdx.x;
        int v = idx < nb ? block_sums[idx] : 0;
        int total;
        int ex = block_excl_scan(v, s_warp, &total);
        if (idx < nb) block_sums[idx] = ex + carry;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_down_kernel(const int *__restrict__ in, int n,
                                                                  const int *__restrict__ block_sums,
                                                                  int *__restrict__ out) {
    __shared__ int s_warp[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int vals[SCAN_ITEMS];
    int v = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        vals[q] = base + q < n ? in[base + q] : 0;
        v += vals[q];
    }
    int total;
    int ex = block_excl_scan(v, s_warp, &total) + block_sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = ex;
        ex += vals[q];
    }
    if (base <= n && n < base + SCAN_ITEMS) out[n] = block_sums[blockIdx.x] + total;
}

// ---------------------------------------------------------------------------
// SP4: scatter with an atomic cursor (count is driven back to zero), then the
// canonical (ascending) order inside every bucket: a particle's place is the
// number of members of its bucket with a smaller index; buckets too long for
// that count are sorted one block per bucket.
// ---------------------------------------------------------------------------

__global__ void scatter_kernel(const int *__restrict__ key, int n, const int *__restrict__ start,
                               int *__restrict__ count, int *__restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = key[i];
    int pos = atomicSub(&count[k], 1) - 1;
    perm[start[k] + pos] = i;
}

constexpr int RANK_MAX = 64;

// unordered: the scatter's output, each bucket's members in arbitrary order.
// Writes perm[start[k] + rank] = i for buckets of up to RANK_MAX members and
// queues the longer ones (once, by the member found first) for the
// block-per-segment sort.
__global__ void bucket_rank_kernel(const int *__restrict__ key, int n, const int *__restrict__ start,
                                   const int *__restrict__ unordered, int *__restrict__ perm,
                                   int *__restrict__ long_list, int *__restrict__ long_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    const int s = start[k], e = start[k + 1];
    if (e - s > RANK_MAX) {
        if (unordered[s] == i) long_list[atomicAdd(long_count, 1)] = k;
        return;
    }
    int r = 0;
    for (int q = s; q < e; ++q) r += unordered[q] < i;
    perm[s + r] = i;
}

constexpr int WARP_RANK_MAX = 64;
constexpr int LANE_RANK_MAX = 8;

// One warp per 32 consecutive segments [begin(s), end(s)) of distinct
// values; each lane reads the bounds of one segment.  Segments of 2 to
// LANE_RANK_MAX values (nearly all of them) are sorted by their own lane in
// registers: every value's place is the number of smaller values, and the
// loads of the 32 segments are in flight together.  The warp then ranks the
// segments of LANE_RANK_MAX + 1 to WARP_RANK_MAX values one after another
// (counted over the values held in registers, up to two per lane), written
// back in place.  Longer segments are queued for the block-per-segment pass.
template <class Seg>
__global__ void __launch_bounds__(256) seg_rank_kernel(Seg seg, int nseg, int *data,
                                                       int *__restrict__ long_list,
                                                       int *__restrict__ long_count) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w * 32 >= nseg) return;   // the whole warp
    const long long sl = w * 32 + lane;
    int bl = 0, ll = 0;
    if (sl < nseg) {
        bl = seg.begin((int)sl);
        ll = seg.end((int)sl) - bl;
        if (ll > WARP_RANK_MAX) long_list[atomicAdd(long_count, 1)] = (int)sl;
    }
    if (ll >= 2 && ll <= LANE_RANK_MAX) {
        int v[LANE_RANK_MAX];
#pragma unroll
        for (int u = 0; u < LANE_RANK_MAX; ++u) v[u] = u < ll ? data[bl + u] : INT_MAX;
#pragma unroll
        for (int u = 0; u < LANE_RANK_MAX; ++u) {
            int r = 0;
#pragma unroll
            for (int t = 0; t < LANE_RANK_MAX; ++t) r += v[t] < v[u];
            if (u < ll) data[bl + r] = v[u];
        }
    }
    for (unsigned todo = __ballot_sync(0xffffffffu, ll > LANE_RANK_MAX && ll <= WARP_RANK_MAX); todo;
         todo &= todo - 1u) {
        const int src = __ffs(todo) - 1;
        const int b = __shfl_sync(0xffffffffu, bl, src), len = __shfl_sync(0xffffffffu, ll, src);
        const int v0 = lane < len ? data[b + lane] : INT_MAX;
        const int v1 = lane + 32 < len ? data[b + 32 + lane] : INT_MAX;
        int r0 = 0, r1 = 0;
        const int n0 = len < 32 ? len : 32;
        for (int t = 0; t < n0; ++t) {
            const int x = __shfl_sync(0xffffffffu, v0, t);
            r0 += x < v0;
            r1 += x < v1;
        }
        for (int t = 32; t < len; ++t) {
            const int x = __shfl_sync(0xffffffffu, v1, t - 32);
            r0 += x < v0;
            r1 += x < v1;
        }
        __syncwarp();
        if (lane < len) data[b + r0] = v0;
        if (lane + 32 < len) data[b + r1] = v1;
        __syncwarp();
    }
}

// One block per long segment.  Segments of up to SEG_CHUNK values are
// bitonic-sorted in shared memory; longer ones are sorted chunk by chunk and
// the sorted runs are merged pairwise, ping-ponging between the segment and
// the same range of the scratch array, each thread producing one slice of
// every merged run (merge path: the slice's split between the two inputs is
// found by binary search).  Values are distinct (particle indices).
constexpr int SEG_CHUNK = 4096;

__device__ __forceinline__ void block_bitonic(int *s, int n2) {
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const int a = s[i], b = s[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
}

__device__ __forceinline__ int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Sort data[b, b + len) (len <= SEG_CHUNK) in shared memory.
__device__ void chunk_sort(int *__restrict__ data, int b, int len, int *sm) {
    const int n2 = pow2_ceil(len);
    for (int q = threadIdx.x; q < n2; q += blockDim.x) sm[q] = q < len ? data[b + q] : 0x7fffffff;
    __syncthreads();
    block_bitonic(sm, n2);
    for (int q = threadIdx.x; q < len; q += blockDim.x) data[b + q] = sm[q];
    __syncthreads();
}

// Number of elements taken from A among the first k of merge(A, B).
__device__ __forceinline__ int co_rank(int k, const int *A, int na, const int *B, int nb) {
    int lo = max(0, k - nb), hi = min(k, na);
    while (lo < hi) {
        const int i = (lo + hi) >> 1;
        if (A[i] < B[k - i - 1]) lo = i + 1;
        else hi = i;
    }
    return lo;
}

// Sort segment [b, e) of data with the whole block (sm: SEG_CHUNK ints of
// shared memory).  The sorted segment is left in out, which may be data
// itself or the scratch array tmp (the three may alias, hence no
// __restrict__).
__device__ void segsort_one(int b, int e, int *data, int *tmp, int *out, int *sm) {
    const int len = e - b;
    if (len <= SEG_CHUNK) {
        chunk_sort(data, b, len, sm);
        if (out != data) {
            for (int q = threadIdx.x; q < len; q += blockDim.x) out[b + q] = data[b + q];
            __syncthreads();
        }
        return;
    }
    for (int c0 = 0; c0 < len; c0 += SEG_CHUNK) chunk_sort(data, b + c0, min(SEG_CHUNK, len - c0), sm);
    int *src = data, *dst = tmp;
    for (int width = SEG_CHUNK; width < len; width *= 2) {
        for (int p0 = 0; p0 < len; p0 += 2 * width) {
            const int na = min(width, len - p0);
            const int nb = max(0, min(width, len - p0 - width));
            const int *A = src + b + p0, *B = A + na;
            int *o = dst + b + p0;
            const int L = na + nb;
            const int per = (L + blockDim.x - 1) / blockDim.x;
            const int k0 = min(L, (int)threadIdx.x * per), k1 = min(L, k0 + per);
            int i = co_rank(k0, A, na, B, nb), j = k0 - i;
            for (int k = k0; k < k1; ++k) {
                if (j >= nb || (i < na && A[i] < B[j])) o[k] = A[i++];
                else o[k] = B[j++];
            }
        }
        __syncthreads();
        int *t = src;
        src = dst;
        dst = t;
    }
    if (src != out) {
        for (int q = threadIdx.x; q < len; q += blockDim.x) out[b + q] = src[b + q];
    }
    __syncthreads();
}

template <class Seg>
__global__ void segsort_long_kernel(Seg seg, int *data, int *tmp, int *out,
                                    const int *__restrict__ long_list,
                                    const int *__restrict__ long_count) {
    __shared__ int sm[SEG_CHUNK];
    const int nl = *long_count;
    for (int w = blockIdx.x; w < nl; w += gridDim.x) {
        const int s = long_list[w];
        segsort_one(seg.begin(s), seg.end(s), data, tmp, out, sm);
    }
}

struct BucketSeg {
    const int *start;
    __device__ int begin(int s) const { return start[s]; }
    __device__ int end(int s) const { return start[s + 1]; }
};

struct RevSeg {   // reverse part of neighbour row s, clipped to the list capacity
    const int *nb_start;
    const int *own;
    int cap;
    __device__ int end(int s) const { return min(nb_start[s + 1], cap); }
    __device__ int begin(int s) const { return min(nb_start[s] + own[s], end(s)); }
};


// ---------------------------------------------------------------------------
// The whole sorting stage as one cooperative launch.  Its phases are the
// kernels above, in the same order and with the same arithmetic (so keys,
// bucket starts, permutation and statistics are bitwise those of the
// multi-kernel path), separated by grid-wide barriers; a cooperative launch
// keeps every block resident, so the barriers cannot wait on a block that
// has not started.  Every phase is a grid-stride loop.
//   A  zero the bucket and level statistics and the bucket counts; reduce
//      the extremes of x, y, z, h (derived grid)
//   B  every block derives the same grid from the extremes; bin (SP1)
//   C  scan of the bucket counts (SP2, SP3): chunk totals, then each block
//      scans its chunk from the total of the chunks before it
//   D  scatter with the atomic cursor (SP4), which drives the counts back
//      to zero
//   E  rank inside the buckets, in the order of the scatter's slots, with
//      each particle's sorted copy and statistics written at its final slot
//   F  block sort of the buckets over 64 members, then theirs
// The extremes are reduced as atomicMax of ~ordered(min) and ordered(max),
// so 0 is the neutral value: the workspace starts zeroed, and block 0 puts
// them back to 0 once every block has read them (phase C).
// ---------------------------------------------------------------------------

namespace cgf = cooperative_groups;

constexpr int FS_THREADS = 256;

__device__ __forceinline__ void block_max_to(unsigned v, unsigned *shared5, int slot, unsigned *global) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&shared5[slot], v);
    __syncthreads();
    if (threadIdx.x == 0 && shared5[slot]) atomicMax(global, shared5[slot]);
}

// A particle's data and its bin: level, cell and bucket.
struct Binned {
    float4 p;
    int sim, k, l, cx, cy, cz;
};

__device__ __forceinline__ Binned bin_of(const SortArgs &a, const GridDev &g, int i) {
    Binned b;
    b.p = a.pos_h[i];
    b.sim = a.sim_of ? a.sim_of[i] : 0;
    b.k = bucket_of_particle(b.p, b.sim, g, b.l, b.cx, b.cy, b.cz);
    return b;
}

// A binned particle placed at sorted slot f (have = false: this lane has
// none): its sorted copies, and the bucket / super-cell / level statistics,
// aggregated over the lanes that share a value (one atomic per run).  Called
// by all 32 lanes of a warp together.
__device__ __forceinline__ void place_binned(const SortArgs &a, int f, bool have, const Binned &b,
                                             int *s_cnt, unsigned *s_hmax) {
    const int lane = threadIdx.x & 31;
    int l = -1, k = -1;
    unsigned hb = 0u, sbit = 0xffffffffu;   // no super-cell bit reaches 2^31
    if (have) {
        a.pos_h_s[f] = b.p;
        if (a.sim_s) a.sim_s[f] = b.sim;
        if (a.tag_s) a.tag_s[f] = cell_tag(b.l, b.cx, b.cy, b.cz);
        k = b.k;
        l = b.l;
        hb = (b.p.w > 0.0f) ? __float_as_uint(b.p.w) : 0u;
        if (a.occ)
            sbit = super_bit(b.cx >> kSuperShift, b.cy >> kSuperShift, b.cz >> kSuperShift,
                             b.l + kMaxLevels * b.sim, a.log2_B);
    }
    {
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const unsigned m = __reduce_max_sync(peers, hb);
        if (k >= 0 && lane == __ffs(peers) - 1 && m > 0u) atomicMax(&a.hmax_cell[k], m);
    }
    if (a.occ) {
        const unsigned peers = __match_any_sync(0xffffffffu, sbit);
        if (k >= 0 && lane == __ffs(peers) - 1) atomicOr(&a.occ[sbit >> 5], 1u << (sbit & 31));
    }
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    const unsigned hpeer = __reduce_max_sync(peers, hb);
    if (l >= 0 && lane == __ffs(peers) - 1) {
        atomicAdd(&s_cnt[l], __popc(peers));
        atomicMax(&s_hmax[l], hpeer);
    }
}

// Particle i (i < 0: none) placed at sorted slot f.
__device__ __forceinline__ void place_sorted(const SortArgs &a, const GridDev &g, int i, int f,
                                             int *s_cnt, unsigned *s_hmax) {
    Binned b{};
    if (i >= 0) b = bin_of(a, g, i);
    place_binned(a, f, i >= 0, b, s_cnt, s_hmax);
}

__global__ void __launch_bounds__(FS_THREADS) sort_fused_kernel(SortArgs a) {
    cgf::grid_group grid = cgf::this_grid();
    __shared__ unsigned s_red[5];
    __shared__ int s_warp[33];
    __shared__ int s_cnt[kMaxLevels];
    __shared__ unsigned s_hmax[kMaxLevels];
    __shared__ int s_seg[SEG_CHUNK];
    const int tid = threadIdx.x;
    const long long gtid = (long long)blockIdx.x * FS_THREADS + tid;
    const long long gstride = (long long)gridDim.x * FS_THREADS;
    const int n = a.n, M = 1 << a.log2_M;
    if (tid < 5) s_red[tid] = 0u;
    if (tid < kMaxLevels) {
        s_cnt[tid] = 0;
        s_hmax[tid] = 0u;
    }
    __syncthreads();

    // A: zero the statistics and counts; reduce the extremes
    for (long long q = gtid; q < M; q += gstride) {
        a.count[q] = 0;
        a.hmax_cell[q] = 0u;
    }
    for (long long q = gtid; q < (long long)(M / 16 + 1); q += gstride) a.occ[q] = 0u;
    if (blockIdx.x == 0 && tid < kMaxLevels) {
        a.lvl_count[tid] = 0;
        a.lvl_hmax[tid] = 0u;
    }
    if (blockIdx.x == 0 && tid == 0) *a.long_count = 0;
    if (a.auto_grid) {
        unsigned mx = 0u, my = 0u, mz = 0u, mh = 0u, Mh = 0u;
        for (long long i = gtid; i < n; i += gstride) {
            const float4 p = a.pos_h[i];
            if (p.x == p.x && fabsf(p.x) < 3.0e38f) mx = max(mx, ~float_to_ordered(p.x));
            if (p.y == p.y && fabsf(p.y) < 3.0e38f) my = max(my, ~float_to_ordered(p.y));
            if (p.z == p.z && fabsf(p.z) < 3.0e38f) mz = max(mz, ~float_to_ordered(p.z));
            if (p.w > 0.0f && p.w < 3.0e38f) {
                mh = max(mh, ~float_to_ordered(p.w));
                Mh = max(Mh, float_to_ordered(p.w));
            }
        }
        block_max_to(mx, s_red, 0, &a.red[0]);
        block_max_to(my, s_red, 1, &a.red[1]);
        block_max_to(mz, s_red, 2, &a.red[2]);
        block_max_to(mh, s_red, 3, &a.red[3]);
        block_max_to(Mh, s_red, 4, &a.red[4]);
    }
    grid.sync();

    // B: the grid, then the bucket of every particle and the counts
    GridDev g = a.given;
    if (a.auto_grid) {
        const unsigned r[5] = {~a.red[0], ~a.red[1], ~a.red[2], ~a.red[3], a.red[4]};
        g = grid_from_red(r, a.log2_M, a.grid_shift);
    }
    if (blockIdx.x == 0 && tid == 0) *a.grid = g;
    for (long long i = gtid; i < n; i += gstride) {
        int l, cx, cy, cz;
        const int k = bucket_of_particle(a.pos_h[i], a.sim_of ? a.sim_of[i] : 0, g, l, cx, cy, cz);
        a.key[i] = k;
        atomicAdd(&a.count[k], 1);
    }
    grid.sync();

    // C: chunk totals of the counts, then each chunk's exclusive scan
    const long long chunk = ((long long)M + gridDim.x - 1) / gridDim.x;
    const long long c0 = (long long)blockIdx.x * chunk, c1 = min((long long)M, c0 + chunk);
    {
        int v = 0;
        for (long long q = c0 + tid; q < c1; q += FS_THREADS) v += a.count[q];
        int total;
        block_excl_scan(v, s_warp, &total);
        if (tid == 0) a.block_sums[blockIdx.x] = total;
        if (blockIdx.x == 0 && tid < 5) a.red[tid] = 0u;   // every block has read the extremes
    }
    grid.sync();
    {
        int v = 0;
        for (int b = tid; b < (int)blockIdx.x; b += FS_THREADS) v += a.block_sums[b];
        int before;
        block_excl_scan(v, s_warp, &before);
        int carry = before;
        for (long long t0 = c0; t0 < c1; t0 += FS_THREADS) {
            const long long q = t0 + tid;
            const int x = q < c1 ? a.count[q] : 0;
            int tot;
            const int ex = block_excl_scan(x, s_warp, &tot);
            if (q < c1) a.start[q] = carry + ex;
            carry += tot;
        }
        if (blockIdx.x == gridDim.x - 1 && tid == 0) a.start[M] = carry;
    }
    grid.sync();

    // D: counting-sort scatter (the cursor drives the counts back to zero)
    for (long long i = gtid; i < n; i += gstride) {
        const int k = a.key[i];
        const int pos = atomicSub(&a.count[k], 1) - 1;
        a.tmp[a.start[k] + pos] = (int)i;
    }
    grid.sync();

    // E: rank inside the buckets (ascending original index), taken in the
    // order of the scatter's slots: the thread of slot j ranks the particle
    // that landed there among its bucket's members (adjacent slots, so the
    // bucket reads are shared by a warp) and puts it, its sorted copy and its
    // statistics in its final slot; only the particle's own data is a random
    // read (its bucket is binned again from it rather than read from key).
    // Buckets of more than RANK_MAX members are queued for phase F.  The trip
    // count is warp-uniform so that the warp-wide matches see every lane.
    const int lane = tid & 31;
    for (long long w0 = gtid - lane; w0 < n; w0 += gstride) {
        const long long j = w0 + lane;
        int i = -1, k = -1, s = 0, e = 0;
        Binned bn{};
        if (j < n) {
            i = a.tmp[j];
            bn = bin_of(a, g, i);
            k = bn.k;
            s = a.start[k];
            e = a.start[k + 1];
            if (e - s > RANK_MAX) {
                if (j == s) a.long_list[atomicAdd(a.long_count, 1)] = k;
                i = -1;   // placed and counted in phase F
            }
        }
        int f = -1;
        if (i >= 0) {
            int r = 0;
            for (int q = s; q < e; ++q) r += a.tmp[q] < i;
            f = s + r;
            a.perm[f] = i;
        }
        place_binned(a, f, i >= 0, bn, s_cnt, s_hmax);
    }
    grid.sync();

    // F: the long buckets, one block each, then their sorted copies and
    // statistics
    {
        const int nl = *a.long_count;
        for (int w = blockIdx.x; w < nl; w += gridDim.x) {
            const int k = a.long_list[w];
            const int s = a.start[k], e = a.start[k + 1];
            segsort_one(s, e, a.tmp, a.perm, a.perm, s_seg);
            for (int f0 = s; f0 < e; f0 += FS_THREADS) {
                const int f = f0 + tid;
                place_sorted(a, g, f < e ? a.perm[f] : -1, f, s_cnt, s_hmax);
            }
        }
    }
    __syncthreads();
    if (tid < kMaxLevels && s_cnt[tid]) {
        atomicAdd(&a.lvl_count[tid], s_cnt[tid]);
        atomicMax(&a.lvl_hmax[tid], s_hmax[tid]);
    }
}

int launch_sort_fused(const SortArgs &a, cudaStream_t st) {
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sort_fused_kernel, FS_THREADS, 0) !=
            cudaSuccess)
            return SPH_ERR_CUDA;
        blocks_per_sm = occ;
    }
    if (blocks_per_sm < 1) return SPH_ERR_CUDA;
    const long long want = std::max<long long>(1, ((long long)std::max(a.n, 1 << a.log2_M) + FS_THREADS - 1) /
                                                      FS_THREADS);
    const int grid = (int)std::min<long long>({want, (long long)blocks_per_sm * device_num_sms(),
                                               (long long)a.block_sums_cap});
    SortArgs args = a;
    void *params[] = {&args};
    SPH_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)sort_fused_kernel, dim3(grid), dim3(FS_THREADS),
                                             params, 0, st));
    note_launch();
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int launch_scan_exclusive(const int *in, int n, int *out, int *block_sums, cudaStream_t st) {
    int nb = (int)blocks_for((long long)n + 1, SCAN_TILE);
    scan_reduce_kernel<<<nb, SCAN_THREADS, 0, st>>>(in, n, block_sums);
    scan_blocks_kernel<<<1, SCAN_THREADS, 0, st>>>(block_sums, nb);
    scan_down_kernel<<<nb, SCAN_THREADS, 0, st>>>(in, n, block_sums, out);
    note_launch(3);
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int scan_block_count(long long n) { return (int)blocks_for(n + 1, SCAN_TILE); }

int launch_sort_buckets(const int *key, int n, const int *start, int *unordered, int *perm,
                        int *long_list, int *long_count, cudaStream_t st) {
    SPH_CUDA_TRY(cudaMemsetAsync(long_count, 0, sizeof(int), st));
    if (n > 0) {
        bucket_rank_kernel<<<blocks_for(n, 256), 256, 0, st>>>(key, n, start, unordered, perm,
                                                               long_list, long_count);
        BucketSeg seg{start};
        segsort_long_kernel<<<1024, 256, 0, st>>>(seg, unordered, perm, perm, long_list, long_count);
        note_launch(2);
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_segsort_rows(const int *nb_start, const int *own, int n, int cap, int *data, int *tmp,
                        int *long_list, int *long_count, cudaStream_t st) {
    SPH_CUDA_TRY(cudaMemsetAsync(long_count, 0, sizeof(int), st));
    RevSeg seg{nb_start, own, cap};
    if (n == 0) return SPH_OK;
    seg_rank_kernel<<<blocks_for(n, 256), 256, 0, st>>>(seg, n, data, long_list, long_count);
    segsort_long_kernel<<<1024, 256, 0, st>>>(seg, data, tmp, data, long_list, long_count);
    note_launch(2);
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_grid_auto(const float4 *pos_h, int n, unsigned *red, int log2_M, GridDev *grid,
                     cudaStream_t st, int shift) {
    const unsigned init[5] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu, 0u};
    // red is reset by a tiny kernel so the sequence stays capturable
    grid_reset_red(red, init, st);
    // a few resident blocks per SM of this device, each striding over the input
    unsigned nb = std::min<unsigned>(blocks_for(n, 256), 4u * (unsigned)device_num_sms());
    if (n > 0) grid_reduce_kernel<<<nb, 256, 0, st>>>(pos_h, n, red);
    grid_finalize_kernel<<<1, 32, 0, st>>>(red, log2_M, shift, grid);
    note_launch(n > 0 ? 3 : 2);
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_grid_set(const SphGrid &h, GridDev *grid, cudaStream_t st) {
    GridDev g{h.x0, h.y0, h.z0, h.log2_L0, h.n_levels, h.log2_M};
    grid_set_kernel<<<1, 32, 0, st>>>(g, grid);
    note_launch();
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_bin(const float4 *pos_h, const int *sim_of, int n, const GridDev *grid, int *key,
               int *count, cudaStream_t st) {
    if (n > 0) {
        bin_kernel<<<blocks_for(n, 256), 256, 0, st>>>(pos_h, sim_of, n, grid, key, count);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_gather_bin(const float4 *pos_h, const int *sim_of, const int *perm, int n,
                      const GridDev *grid, float4 *pos_h_s, int *sim_s, unsigned *tag_s, unsigned *occ,
                      int log2_B, unsigned *hmax_cell, int *lvl_count, unsigned *lvl_hmax,
                      cudaStream_t st) {
    if (n > 0) {
        gather_bin_kernel<<<blocks_for(n, 256), 256, 0, st>>>(pos_h, sim_of, perm, n, grid, pos_h_s,
                                                              sim_s, tag_s, occ, log2_B, hmax_cell,
                                                              lvl_count, lvl_hmax);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_scatter(const int *key, int n, const int *start, int *count, int *perm, cudaStream_t st) {
    if (n > 0) {
        scatter_kernel<<<blocks_for(n, 256), 256, 0, st>>>(key, n, start, count, perm);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

__global__ void reset_red_kernel(unsigned *red, unsigned a, unsigned b, unsigned c, unsigned d,
                                 unsigned e) {
    if (threadIdx.x == 0) {
        red[0] = a; red[1] = b; red[2] = c; red[3] = d; red[4] = e;
    }
}

void grid_reset_red(unsigned *red, const unsigned *v, cudaStream_t st) {
    reset_red_kernel<<<1, 32, 0, st>>>(red, v[0], v[1], v[2], v[3], v[4]);
}

}  // namespace sphgb
