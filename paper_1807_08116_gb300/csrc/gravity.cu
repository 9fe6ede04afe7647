// gravity.cu -- direct particle-particle gravity (GFC, Eq. 4 of the paper,
// Plummer-softened reading) on the FP32 pipe of sm_103a.
//
// g_i = -G sum_{j != i} m_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2)
//
// Design (the paper stages j-tiles through shared memory on Kepler; this is
// the GB300 form of the same idea):
//  * each CTA owns 256 * R target particles i (R per thread, kept in
//    registers) and streams source tiles of TJ float4 (x, y, z, m) into
//    shared memory with 1-D TMA bulk copies (cp.async.bulk), double-buffered
//    and completed through mbarriers (waits bounded in time);
//  * the inner loop is 3 FADD + 3 FFMA + 1 MUFU.RSQ + 3 FMUL + 3 FFMA per
//    interaction on one broadcast shared-memory load per source and thread;
//  * per-tile partial sums are folded into Kahan-compensated running sums;
//  * when there are too few target blocks to fill 152 SMs, the source range
//    is split over the S CTAs of a thread-block cluster and the S partial
//    sums are combined in a fixed order through distributed shared memory, so
//    the kernel needs no global scratch and stays deterministic.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "async.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace sphgb {

// Launch shape (the defaults are the tuned values; the macros exist so that
// variants can be built and timed against each other).
#ifndef SPHGB_GR_THREADS
#define SPHGB_GR_THREADS 256
#endif
#ifndef SPHGB_GR_TJ
#define SPHGB_GR_TJ 1024
#endif
#ifndef SPHGB_GR_UNROLL
#define SPHGB_GR_UNROLL 4
#endif
#ifndef SPHGB_GR_MINB
#define SPHGB_GR_MINB 2
#endif
#ifndef SPHGB_GR_NBUF
#define SPHGB_GR_NBUF 2
#endif

constexpr int GR_THREADS = SPHGB_GR_THREADS;
constexpr int GR_UNROLL = SPHGB_GR_UNROLL;
constexpr int GR_TJ = SPHGB_GR_TJ;                 // sources per tile
constexpr int GR_NBUF = SPHGB_GR_NBUF;             // raw tiles in flight (TMA ring)
// raw ring + expanded tile + mbarriers; the cluster reduction reuses the same
// space for 4 x (256 x 8) floats at most
constexpr int GR_SMEM_TILES = (GR_NBUF + 2) * GR_TJ * 16;
constexpr int GR_SMEM_RED = 4 * GR_THREADS * 8 * 4;
constexpr int GR_SMEM = (GR_SMEM_TILES > GR_SMEM_RED ? GR_SMEM_TILES : GR_SMEM_RED) + 64;

__device__ int g_grav_flags;
// time limit of every bounded mbarrier wait (sph_set_wait_limit_ns)
constexpr unsigned long long kWaitLimitDefaultNs = 2000000000ull;
__device__ unsigned long long g_wait_limit_ns = kWaitLimitDefaultNs;

// After a wait gave up: the tiles [t, t_end) were issued and not consumed, so
// their copies may still be landing in this block's shared memory; thread 0
// waits for each of them, again within the limit, before the block exits.
__device__ __forceinline__ void drain_tiles(unsigned bar0, unsigned t, unsigned t_end, int nbuf) {
    if (threadIdx.x == 0)
        for (unsigned u = t; u < t_end; ++u)
            mbar_wait_bounded(bar0 + 8 * (u % nbuf), (u / nbuf) & 1u, &g_wait_limit_ns);
    __syncthreads();
}

// Expand a landed tile (x, y, z, m) into duplicated pairs ((x, x, y, y),
// (z, z, m, m)), one per source.
__device__ __forceinline__ void expand_tile(const float4 *__restrict__ tb, float4 *__restrict__ dup,
                                            int cnt) {
    for (int q = threadIdx.x; q < cnt; q += GR_THREADS) {
        const float4 v = tb[q];
        dup[2 * q] = make_float4(v.x, v.x, v.y, v.y);
        dup[2 * q + 1] = make_float4(v.z, v.z, v.w, v.w);
    }
}

// Sums of one tile for RP target pairs: 3 FADD2, 3 FFMA2, 2 MUFU.RSQ,
// 3 FMUL2, 3 FFMA2 (+1 FADD2 for the potential) per source and pair.
// SELF: the tile holds some of this CTA's own targets; source j of the tile
// is target k of this thread when j == self_off + tid + k 256, and that term
// is left out of the potential (its acceleration term is 0: dr = 0).
template <int RP, bool POT, bool GUARD, bool SELF>
__device__ __forceinline__ void tile_sums(const float4 *__restrict__ dup, int cnt,
                                          const float2 (&nx)[RP], const float2 (&ny)[RP],
                                          const float2 (&nz)[RP], float2 e2, float2 (&sx)[RP],
                                          float2 (&sy)[RP], float2 (&sz)[RP], float2 (&sp)[RP],
                                          int self_off) {
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        sx[p] = make_float2(0.f, 0.f); sy[p] = sx[p]; sz[p] = sx[p]; sp[p] = sx[p];
    }
#pragma unroll GR_UNROLL
    for (int j = 0; j < cnt; ++j) {
        const float4 a = dup[2 * j];
        const float4 b = dup[2 * j + 1];
        const float2 qx = make_float2(a.x, a.y), qy = make_float2(a.z, a.w);
        const float2 qz = make_float2(b.x, b.y), qm = make_float2(b.z, b.w);
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            const float2 dx = __fadd2_rn(qx, nx[p]);
            const float2 dy = __fadd2_rn(qy, ny[p]);
            const float2 dz = __fadd2_rn(qz, nz[p]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            if (GUARD) {
                inv.x = r2.x > 0.f ? inv.x : 0.f;
                inv.y = r2.y > 0.f ? inv.y : 0.f;
            }
            if (SELF) {
                const int k0 = self_off + (int)threadIdx.x + (2 * p) * GR_THREADS;
                if (j == k0) inv.x = 0.f;
                if (j == k0 + GR_THREADS) inv.y = 0.f;
            }
            const float2 s = __fmul2_rn(qm, inv);
            // m / r^3 with two more FMUL2: a second MUFU op (1 / r^2) instead
            // was measured slower -- MUFU issues at a quarter of the FP32 rate
            const float2 s3 = __fmul2_rn(__fmul2_rn(s, inv), inv);
            sx[p] = __ffma2_rn(s3, dx, sx[p]);
            sy[p] = __ffma2_rn(s3, dy, sy[p]);
            sz[p] = __ffma2_rn(s3, dz, sz[p]);
            if (POT) sp[p] = __fadd2_rn(sp[p], s);
        }
    }
}

// Fold one tile's partial sums into the running (compensated) sums.
template <int RP, bool POT, bool KAHAN>
__device__ __forceinline__ void fold_tile(Kahan (&ax)[2 * RP], Kahan (&ay)[2 * RP],
                                          Kahan (&az)[2 * RP], Kahan (&ph)[2 * RP],
                                          const float2 (&sx)[RP], const float2 (&sy)[RP],
                                          const float2 (&sz)[RP], const float2 (&sp)[RP]) {
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        if (KAHAN) {
            ax[2 * p].add(sx[p].x); ax[2 * p + 1].add(sx[p].y);
            ay[2 * p].add(sy[p].x); ay[2 * p + 1].add(sy[p].y);
            az[2 * p].add(sz[p].x); az[2 * p + 1].add(sz[p].y);
            if (POT) { ph[2 * p].add(sp[p].x); ph[2 * p + 1].add(sp[p].y); }
        } else {
            ax[2 * p].s += sx[p].x; ax[2 * p + 1].s += sx[p].y;
            ay[2 * p].s += sy[p].x; ay[2 * p + 1].s += sy[p].y;
            az[2 * p].s += sz[p].x; az[2 * p + 1].s += sz[p].y;
            if (POT) { ph[2 * p].s += sp[p].x; ph[2 * p + 1].s += sp[p].y; }
        }
    }
}

// Kernel: RP pairs of targets per thread (R = 2 RP).  The two targets of a
// pair share one packed FP32x2 instruction (FADD2 / FFMA2 / FMUL2), which
// halves the issue slots of the 12 FP32 operations of an interaction, so the
// FP32 pipe, not instruction issue, bounds the loop.  The source tile that
// TMA lands as (x, y, z, m) float4 is expanded once per tile into duplicated
// pairs ((x, x, y, y), (z, z, m, m)) so each source feeds the packed operands
// straight from two broadcast 16-byte shared loads.
template <int RP, bool POT, bool GUARD, bool KAHAN>
__global__ void __launch_bounds__(GR_THREADS, RP >= 4 ? 1 : SPHGB_GR_MINB)
pp_gravity_kernel(const float4 *__restrict__ pos, int n, int row0, int row_end, int n_tiles, int S,
                  float G, float eps2, float4 *__restrict__ out) {
    constexpr int R = 2 * RP;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);            // [GR_NBUF][GR_TJ] raw
    float4 *dup = tiles + GR_NBUF * GR_TJ;                        // [GR_TJ][2] expanded
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + GR_SMEM - 64);
    const int tid = threadIdx.x;
    const int rank = blockIdx.x % S;   // cluster dims (S, 1, 1): rank == ctarank
    // targets [row0, row_end) of the n sources; target i is written to out[i - row0]
    const int i0 = row0 + (blockIdx.x / S) * (GR_THREADS * R);
    const int t_begin = (int)((long long)n_tiles * rank / S);
    const int t_end = (int)((long long)n_tiles * (rank + 1) / S);
    const int my_tiles = t_end - t_begin;

    // target k of this thread is i0 + tid + k * GR_THREADS; pair p = targets (2p, 2p + 1)
    float2 nx[RP], ny[RP], nz[RP];
    Kahan ax[R], ay[R], az[R], ph[R];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        int ia = i0 + tid + (2 * p) * GR_THREADS, ib = ia + GR_THREADS;
        float4 a = ia < row_end ? pos[ia] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 b = ib < row_end ? pos[ib] : make_float4(0.f, 0.f, 0.f, 0.f);
        nx[p] = make_float2(-a.x, -b.x);
        ny[p] = make_float2(-a.y, -b.y);
        nz[p] = make_float2(-a.z, -b.z);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) { ax[k].init(); ay[k].init(); az[k].init(); ph[k].init(); }

    const unsigned bar0 = smem_u32(&bars[0]);
    const unsigned tiles0 = smem_u32(tiles);
    if (tid == 0) {
        for (int b = 0; b < GR_NBUF; ++b) mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int b = 0; b < GR_NBUF && b < my_tiles; ++b) {
            int j0 = (t_begin + b) * GR_TJ;
            unsigned bytes = (unsigned)min(GR_TJ, n - j0) * 16u;
            mbar_expect_tx(bar0 + 8 * b, bytes);
            bulk_g2s(tiles0 + b * GR_TJ * 16, pos + j0, bytes, bar0 + 8 * b);
        }
    }

    const float2 e2 = make_float2(eps2, eps2);
    bool failed = false;
    for (int t = 0; t < my_tiles; ++t) {
        const int buf = t % GR_NBUF;
        bool ok = mbar_wait_bounded(bar0 + 8 * buf, (unsigned)((t / GR_NBUF) & 1), &g_wait_limit_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            drain_tiles(bar0, t, min(my_tiles, t + GR_NBUF), GR_NBUF);
            break;
        }
        const int cnt = min(GR_TJ, n - (t_begin + t) * GR_TJ);
        const float4 *tb = tiles + buf * GR_TJ;
        expand_tile(tb, dup, cnt);
        __syncthreads();   // raw buffer consumed, expanded tile visible
        if (tid == 0 && t + GR_NBUF < my_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            int j0 = (t_begin + t + GR_NBUF) * GR_TJ;
            unsigned bytes = (unsigned)min(GR_TJ, n - j0) * 16u;
            mbar_expect_tx(bar0 + 8 * buf, bytes);
            bulk_g2s(tiles0 + buf * GR_TJ * 16, pos + j0, bytes, bar0 + 8 * buf);
        }
        float2 sx[RP], sy[RP], sz[RP], sp[RP];
        const int j0 = (t_begin + t) * GR_TJ;
        if (POT && !GUARD && j0 < i0 + GR_THREADS * R && i0 < j0 + cnt)
            tile_sums<RP, POT, GUARD, true>(dup, cnt, nx, ny, nz, e2, sx, sy, sz, sp, i0 - j0);
        else
            tile_sums<RP, POT, GUARD, false>(dup, cnt, nx, ny, nz, e2, sx, sy, sz, sp, 0);
        fold_tile<RP, POT, KAHAN>(ax, ay, az, ph, sx, sy, sz, sp);
        __syncthreads();   // expanded tile fully read before the next expansion
    }
    if (failed && tid == 0) atomicOr(&g_grav_flags, SPH_FLAG_TIMEOUT);

    if (S == 1) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            int i = i0 + tid + k * GR_THREADS;
            if (i < row_end) {
                float pot = POT ? -G * (ph[k].s - ph[k].c) : 0.f;
                out[i - row0] = make_float4(G * (ax[k].s - ax[k].c), G * (ay[k].s - ay[k].c),
                                          G * (az[k].s - az[k].c), pot);
            }
        }
        return;
    }

    // Cluster combine: partial sums of the S source ranges meet in shared
    // memory; rank r sums a 1/S slice of the targets over ranks 0..S-1.
    cg::cluster_group cluster = cg::this_cluster();
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem);   // [4][GR_THREADS * R]
    constexpr int NB = GR_THREADS * R;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        int q = tid + k * GR_THREADS;
        red[0 * NB + q] = ax[k].s - ax[k].c;
        red[1 * NB + q] = ay[k].s - ay[k].c;
        red[2 * NB + q] = az[k].s - az[k].c;
        red[3 * NB + q] = POT ? ph[k].s - ph[k].c : 0.f;
    }
    cluster.sync();
    const int q_end = NB * (rank + 1) / S;
    for (int q = NB * rank / S + tid; q < q_end; q += GR_THREADS) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int r = 0; r < S; ++r) {
            const float *peer = cluster.map_shared_rank(red, r);
            a0 += peer[0 * NB + q];
            a1 += peer[1 * NB + q];
            a2 += peer[2 * NB + q];
            a3 += peer[3 * NB + q];
        }
        int i = i0 + q;
        if (i < row_end) out[i - row0] = make_float4(G * a0, G * a1, G * a2, POT ? -G * a3 : 0.f);
    }
    cluster.sync();
}

// Batched form: many independent simulations in one persistent launch.
// Simulation s owns gas particles [g0, g0 + ng) and dark particles
// [d0, d0 + nd) of the shared arrays; its particles are numbered "virtually"
// v = 0..ng+nd-1 (gas first), exactly the order a single-simulation launch
// of that simulation sees, so its sums (tile boundaries, summation order) are
// the same as pp_gravity's with no cluster split.  A work unit is (s, first
// virtual target of a block of 256 R); units are taken from a queue
// (atomic counter) in decreasing order of simulation size, so the largest
// blocks start first.  A tile that straddles the gas/dark boundary is landed
// with two bulk copies on one mbarrier.
template <int RP, bool POT, bool GUARD, bool KAHAN>
__global__ void __launch_bounds__(GR_THREADS, RP >= 4 ? 1 : SPHGB_GR_MINB)
pp_gravity_batched_kernel(const float4 *__restrict__ pos, const int4 *__restrict__ sims,
                          const int2 *__restrict__ units, int n_units, int *__restrict__ counter,
                          float G, float eps2, float4 *__restrict__ out) {
    constexpr int R = 2 * RP;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_unit;
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    float4 *dup = tiles + GR_NBUF * GR_TJ;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + GR_SMEM - 64);
    const int tid = threadIdx.x;
    const unsigned bar0 = smem_u32(&bars[0]);
    const unsigned tiles0 = smem_u32(tiles);
    if (tid == 0) {
        for (int b = 0; b < GR_NBUF; ++b) mbar_init(bar0 + 8 * b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    const float2 e2 = make_float2(eps2, eps2);
    unsigned seq = 0;   // tiles this CTA has landed so far (mbarrier phases)
    bool failed = false;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= n_units || failed) break;
        const int2 un = units[u];
        const int4 sr = sims[un.x];   // (g0, ng, d0, nd)
        const int ng = sr.y, ns = sr.y + sr.w;
        const int vt0 = un.y;
        const int nt = (ns + GR_TJ - 1) / GR_TJ;

        float2 nx[RP], ny[RP], nz[RP];
        Kahan ax[R], ay[R], az[R], ph[R];
#pragma unroll
        for (int p = 0; p < RP; ++p) {
            const int va = vt0 + tid + (2 * p) * GR_THREADS, vb = va + GR_THREADS;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (va < ns) a = pos[va < ng ? sr.x + va : sr.z + (va - ng)];
            if (vb < ns) b = pos[vb < ng ? sr.x + vb : sr.z + (vb - ng)];
            nx[p] = make_float2(-a.x, -b.x);
            ny[p] = make_float2(-a.y, -b.y);
            nz[p] = make_float2(-a.z, -b.z);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) { ax[k].init(); ay[k].init(); az[k].init(); ph[k].init(); }

        // land virtual source tile t into buffer (seq + t) % GR_NBUF
        auto issue = [&](int t) {
            const int v0 = t * GR_TJ, v1 = min(ns, v0 + GR_TJ);
            const int gcnt = max(0, min(v1, ng) - v0);
            const int dcnt = (v1 - v0) - gcnt;
            const unsigned buf = (seq + t) % GR_NBUF;
            const unsigned bar = bar0 + 8 * buf, dst = tiles0 + buf * GR_TJ * 16;
            mbar_expect_tx(bar, (unsigned)(v1 - v0) * 16u);
            if (gcnt) bulk_g2s(dst, pos + sr.x + v0, (unsigned)gcnt * 16u, bar);
            if (dcnt) bulk_g2s(dst + gcnt * 16, pos + sr.z + max(0, v0 - ng), (unsigned)dcnt * 16u, bar);
        };
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int b = 0; b < GR_NBUF && b < nt; ++b) issue(b);
        }
        for (int t = 0; t < nt; ++t) {
            const unsigned q = seq + t;
            const int buf = q % GR_NBUF;
            bool ok = mbar_wait_bounded(bar0 + 8 * buf, (q / GR_NBUF) & 1u, &g_wait_limit_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                drain_tiles(bar0, q, seq + min(nt, t + GR_NBUF), GR_NBUF);
                break;
            }
            const int cnt = min(GR_TJ, ns - t * GR_TJ);
            expand_tile(tiles + buf * GR_TJ, dup, cnt);
            __syncthreads();
            if (tid == 0 && t + GR_NBUF < nt) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(t + GR_NBUF);
            }
            float2 sx[RP], sy[RP], sz[RP], sp[RP];
            const int v0 = t * GR_TJ;   // virtual index of the tile's first source
            if (POT && !GUARD && v0 < vt0 + GR_THREADS * R && vt0 < v0 + cnt)
                tile_sums<RP, POT, GUARD, true>(dup, cnt, nx, ny, nz, e2, sx, sy, sz, sp, vt0 - v0);
            else
                tile_sums<RP, POT, GUARD, false>(dup, cnt, nx, ny, nz, e2, sx, sy, sz, sp, 0);
            fold_tile<RP, POT, KAHAN>(ax, ay, az, ph, sx, sy, sz, sp);
            __syncthreads();
        }
        seq += nt;
        if (failed) break;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int v = vt0 + tid + k * GR_THREADS;
            if (v < ns) {
                const int i = v < ng ? sr.x + v : sr.z + (v - ng);
                const float pot = POT ? -G * (ph[k].s - ph[k].c) : 0.f;
                out[i] = make_float4(G * (ax[k].s - ax[k].c), G * (ay[k].s - ay[k].c),
                                     G * (az[k].s - az[k].c), pot);
            }
        }
    }
    if (failed && tid == 0) atomicOr(&g_grav_flags, SPH_FLAG_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Host side: pick R (targets per thread) and S (cluster split of the sources)
// by a wave-quantisation cost model over the measured occupancy.
// ---------------------------------------------------------------------------

using GravKernel = void (*)(const float4 *, int, int, int, int, int, float, float, float4 *);

template <int RP>
static GravKernel pick_kernel(bool pot, bool guard, bool kahan) {
    if (pot) {
        if (guard) return kahan ? pp_gravity_kernel<RP, true, true, true> : pp_gravity_kernel<RP, true, true, false>;
        return kahan ? pp_gravity_kernel<RP, true, false, true> : pp_gravity_kernel<RP, true, false, false>;
    }
    if (guard) return kahan ? pp_gravity_kernel<RP, false, true, true> : pp_gravity_kernel<RP, false, true, false>;
    return kahan ? pp_gravity_kernel<RP, false, false, true> : pp_gravity_kernel<RP, false, false, false>;
}

// R targets per thread (2, 4 or 8) -> R / 2 packed pairs
static GravKernel kernel_for(int R, bool pot, bool guard, bool kahan) {
    switch (R) {
        case 2: return pick_kernel<1>(pot, guard, kahan);
        case 8: return pick_kernel<4>(pot, guard, kahan);
        default: return pick_kernel<2>(pot, guard, kahan);
    }
}

struct GravPlan {
    int R, S;
};

static int g_num_sms = 0;

static int slots_for(GravKernel k, int S) {
    if (S == 1) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, GR_THREADS, GR_SMEM) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return occ * g_num_sms;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S * 64, 1, 1);
    cfg.blockDim = dim3(GR_THREADS, 1, 1);
    cfg.dynamicSmemBytes = GR_SMEM;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = S;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters * S;
}

// Cost of a launch in "target-source pairs on the busiest SM": the grid runs
// in waves of `slots` resident CTAs; in a wave the busiest SM holds
// ceil(resident / SMs) CTAs, each doing 256 R x n / S interactions.
static double plan_cost(long long units, int slots, int R, int n, int S) {
    const double per_int = 6.0 + 1.0 + 2.0 / R;   // issue slots per interaction, packed pairs
    const double per_cta = (double)GR_THREADS * R * ((double)n / S) * per_int;
    long long full = units / slots, rem = units % slots;
    double busiest = (double)full * ((slots + g_num_sms - 1) / g_num_sms) +
                     (double)((rem + g_num_sms - 1) / g_num_sms);
    return busiest * per_cta;
}

static std::atomic<int> g_force_R{0}, g_force_S{0};

static GravPlan plan_gravity_uncached(int m, int n, bool pot, bool guard, bool kahan);

// Plans are cached per (targets m, sources n, variant) so that repeated
// launches (and launches recorded into a CUDA graph) make no occupancy queries.
static std::mutex g_plan_mutex;
static std::map<std::tuple<int, int, int>, GravPlan> g_plan_cache;

static GravPlan plan_gravity(int m, int n, bool pot, bool guard, bool kahan) {
    const int fR = g_force_R.load(), fS = g_force_S.load();
    if (fR) {
        const int n_tiles = (n + GR_TJ - 1) / GR_TJ;
        return GravPlan{fR, std::max(1, std::min(fS, std::max(1, n_tiles)))};
    }
    const auto key = std::make_tuple(m, n, (pot ? 1 : 0) | (guard ? 2 : 0) | (kahan ? 4 : 0));
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    auto it = g_plan_cache.find(key);
    if (it != g_plan_cache.end()) return it->second;
    GravPlan p = plan_gravity_uncached(m, n, pot, guard, kahan);
    g_plan_cache[key] = p;
    return p;
}

static GravPlan plan_gravity_uncached(int m, int n, bool pot, bool guard, bool kahan) {
    const int n_tiles = (n + GR_TJ - 1) / GR_TJ;
    GravPlan best{4, 1};
    double best_cost = 1e300;
    const int Rs[3] = {4, 8, 2};
    const int Ss[5] = {1, 2, 4, 8, 16};
    for (int R : Rs) {
        GravKernel k = kernel_for(R, pot, guard, kahan);
        const long long nib = (m + GR_THREADS * R - 1) / (GR_THREADS * R);
        for (int S : Ss) {
            if (S > 1 && S > n_tiles) break;
            int slots = slots_for(k, S);
            if (slots <= 0) continue;
            double cost = plan_cost(nib * S, slots, R, n, S) * (1.0 + 0.01 * (S > 1) + 0.005 * S);
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = GravPlan{R, S};
            }
        }
    }
    return best;
}

static std::once_flag g_grav_once;
static int g_grav_init_status = SPH_OK;

static void grav_init() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        g_grav_init_status = SPH_ERR_CUDA;
        return;
    }
    const int Rs[3] = {2, 4, 8};
    for (int R : Rs)
        for (int f = 0; f < 8; ++f) {
            GravKernel k = kernel_for(R, f & 1, f & 2, f & 4);
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, GR_SMEM) !=
                cudaSuccess) {
                g_grav_init_status = SPH_ERR_CUDA;
                return;
            }
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
                cudaGetLastError();
        }
}

using GravBatchedKernel = void (*)(const float4 *, const int4 *, const int2 *, int, int *, float,
                                   float, float4 *);

template <int RP>
static GravBatchedKernel pick_batched(bool pot, bool guard, bool kahan) {
    if (pot) {
        if (guard) return kahan ? pp_gravity_batched_kernel<RP, true, true, true> : pp_gravity_batched_kernel<RP, true, true, false>;
        return kahan ? pp_gravity_batched_kernel<RP, true, false, true> : pp_gravity_batched_kernel<RP, true, false, false>;
    }
    if (guard) return kahan ? pp_gravity_batched_kernel<RP, false, true, true> : pp_gravity_batched_kernel<RP, false, true, false>;
    return kahan ? pp_gravity_batched_kernel<RP, false, false, true> : pp_gravity_batched_kernel<RP, false, false, false>;
}

static GravBatchedKernel batched_for(int R, bool pot, bool guard, bool kahan) {
    switch (R) {
        case 2: return pick_batched<1>(pot, guard, kahan);
        case 8: return pick_batched<4>(pot, guard, kahan);
        default: return pick_batched<2>(pot, guard, kahan);
    }
}

static std::once_flag g_grav_batched_once;
static int g_grav_batched_status = SPH_OK;

static void grav_batched_init() {
    const int Rs[3] = {2, 4, 8};
    for (int R : Rs)
        for (int f = 0; f < 8; ++f)
            if (cudaFuncSetAttribute(batched_for(R, f & 1, f & 2, f & 4),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     GR_SMEM) != cudaSuccess) {
                g_grav_batched_status = SPH_ERR_CUDA;
                return;
            }
}

int gravity_num_sms() {
    std::call_once(g_grav_once, grav_init);
    return g_num_sms;
}

// Looked up on every call: an address kept from an earlier call would belong
// to the context it was taken in (stale after a device reset).
int *gravity_flags_device() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_grav_flags) != cudaSuccess) return nullptr;
    return static_cast<int *>(p);
}

bool gravity_plan_forced() { return g_force_R.load() != 0; }

int launch_gravity_batched(const float4 *pos, const int4 *sims, const int2 *units, int n_units,
                           int *counter, int R, float G, float eps, float4 *out, int flags,
                           cudaStream_t st) {
    std::call_once(g_grav_once, grav_init);
    if (g_grav_init_status != SPH_OK) return g_grav_init_status;
    std::call_once(g_grav_batched_once, grav_batched_init);
    if (g_grav_batched_status != SPH_OK) return g_grav_batched_status;
    if (n_units <= 0) return SPH_OK;
    const bool pot = flags & SPH_GRAV_POTENTIAL;
    const bool kahan = !(flags & SPH_GRAV_NO_KAHAN);
    const float eps2 = eps * eps;
    const bool guard = !(eps2 > 0.0f);
    GravBatchedKernel k = batched_for(R, pot, guard, kahan);
    static std::mutex occ_mutex;
    static std::map<GravBatchedKernel, int> occ_cache;
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(occ_mutex);
        auto it = occ_cache.find(k);
        if (it != occ_cache.end()) {
            occ = it->second;
        } else {
            SPH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, GR_THREADS, GR_SMEM));
            occ_cache[k] = occ;
        }
    }
    const int grid = std::max(1, std::min(n_units, occ * g_num_sms));
    SPH_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    k<<<grid, GR_THREADS, GR_SMEM, st>>>(pos, sims, units, n_units, counter, G, eps2, out);
    note_launch();
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

}  // namespace sphgb

using namespace sphgb;

namespace {

// One launch of the one-sided kernel over the targets [i0, i1) of n sources.
int gravity_rows(const float *d_pos_m, int n, int i0, int i1, float G, float eps, float *d_acc_pot,
                 int flags, sph_stream_t stream) {
    std::call_once(g_grav_once, grav_init);
    if (g_grav_init_status != SPH_OK) return g_grav_init_status;
    const int m = i1 - i0;
    const bool pot = flags & SPH_GRAV_POTENTIAL;
    const bool kahan = !(flags & SPH_GRAV_NO_KAHAN);
    const float eps2 = eps * eps;
    const bool guard = !(eps2 > 0.0f);
    GravPlan p = plan_gravity(m, n, pot, guard, kahan);
    GravKernel k = kernel_for(p.R, pot, guard, kahan);
    const int n_tiles = (n + GR_TJ - 1) / GR_TJ;
    const int nib = (m + GR_THREADS * p.R - 1) / (GR_THREADS * p.R);

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nib * p.S), 1, 1);
    cfg.blockDim = dim3(GR_THREADS, 1, 1);
    cfg.dynamicSmemBytes = GR_SMEM;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = p.S;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = p.S > 1 ? 1 : 0;
    SPH_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, reinterpret_cast<const float4 *>(d_pos_m), (int)n, i0,
                                    i1, n_tiles, p.S, G, eps2, reinterpret_cast<float4 *>(d_acc_pot)));
    note_launch();
    return SPH_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int pp_gravity(const float *d_pos_m, int32_t n, float G, float eps, float *d_acc_pot,
                          int32_t flags, sph_stream_t stream) {
    if (n < 0 || !(eps >= 0.0f) || !(G == G)) return SPH_ERR_INVALID_ARG;
    if (n == 0) return SPH_OK;
    if (!d_pos_m || !d_acc_pot || !aligned16(d_pos_m) || !aligned16(d_acc_pot))
        return SPH_ERR_INVALID_ARG;
    return gravity_rows(d_pos_m, n, 0, n, G, eps, d_acc_pot, flags, stream);
}

extern "C" int pp_gravity_rows(const float *d_pos_m, int32_t n, int32_t i0, int32_t i1, float G,
                               float eps, float *d_acc_pot, int32_t flags, sph_stream_t stream) {
    if (n < 0 || i0 < 0 || i1 < i0 || i1 > n || !(eps >= 0.0f) || !(G == G))
        return SPH_ERR_INVALID_ARG;
    if (i1 == i0) return SPH_OK;
    if (!d_pos_m || !d_acc_pot || !aligned16(d_pos_m) || !aligned16(d_acc_pot))
        return SPH_ERR_INVALID_ARG;
    return gravity_rows(d_pos_m, n, i0, i1, G, eps, d_acc_pot, flags, stream);
}

extern "C" int pp_gravity_status(sph_stream_t stream, int32_t *h_flags) {
    if (!h_flags) return SPH_ERR_INVALID_ARG;
    SPH_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0, zero = 0;
    SPH_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_grav_flags, sizeof(int)));
    SPH_CUDA_TRY(cudaMemcpyToSymbol(g_grav_flags, &zero, sizeof(int)));
    *h_flags = v;
    return v ? SPH_ERR_DEVICE : SPH_OK;
}

// ---------------------------------------------------------------------------
// Failure detection: the time limit of the bounded waits, and a probe that
// makes one such wait run out.
// ---------------------------------------------------------------------------

// One arrival with 16 bytes of expected transaction that no copy will bring:
// the phase cannot complete, the bounded wait gives up after the limit, the
// status word records it and the block returns.  No copy is ever issued, so
// nothing is in flight when it exits.
__global__ void wait_probe_kernel() {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const unsigned b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(b, 16u);
    if (!mbar_wait_bounded(b, 0u, &g_wait_limit_ns)) atomicOr(&g_grav_flags, SPH_FLAG_TIMEOUT);
}

extern "C" int sph_set_wait_limit_ns(int64_t limit_ns) {
    if (limit_ns != 0 && (limit_ns < 1000 || limit_ns > 60000000000ll)) return SPH_ERR_INVALID_ARG;
    const unsigned long long v = limit_ns ? (unsigned long long)limit_ns : kWaitLimitDefaultNs;
    SPH_CUDA_TRY(cudaMemcpyToSymbol(g_wait_limit_ns, &v, sizeof(v)));
    return SPH_OK;
}

extern "C" int sph_wait_probe(sph_stream_t stream) {
    wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>();
    note_launch();
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

// Launch plan exposed for tests and the bench's roofline accounting.
extern "C" int sph_gravity_plan(int32_t n, int32_t flags, int32_t *h_R, int32_t *h_S) {
    if (n <= 0 || !h_R || !h_S) return SPH_ERR_INVALID_ARG;
    std::call_once(g_grav_once, grav_init);
    if (g_grav_init_status != SPH_OK) return g_grav_init_status;
    GravPlan p = plan_gravity(n, n, flags & SPH_GRAV_POTENTIAL, false, !(flags & SPH_GRAV_NO_KAHAN));
    *h_R = p.R;
    *h_S = p.S;
    return SPH_OK;
}

// Fix the launch plan of later pp_gravity calls (autotuning): R in {2, 4, 8}
// targets per thread, S in {1, 2, 4, 8, 16} CTAs per cluster; R = 0 restores
// the cost-model plan.
extern "C" int sph_gravity_tune(int32_t R, int32_t S) {
    if (R != 0 && R != 2 && R != 4 && R != 8) return SPH_ERR_INVALID_ARG;
    if (R != 0 && S != 1 && S != 2 && S != 4 && S != 8 && S != 16) return SPH_ERR_INVALID_ARG;
    g_force_R.store(R);
    g_force_S.store(R ? S : 0);
    return SPH_OK;
}
