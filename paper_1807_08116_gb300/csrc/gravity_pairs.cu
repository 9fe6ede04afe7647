// gravity_pairs.cu -- direct particle-particle gravity (GFC, Eq. 4, Plummer-
// softened reading) with every unordered pair evaluated once.
//
// The force of a pair is equal and opposite (Newton's third law), and the
// softened kernel is symmetric, so one evaluation of
//     inv = (|r_j - r_i|^2 + eps^2)^(-1/2),  w = inv^3
// serves both bodies: g_i += m_j w (r_j - r_i) and g_j -= m_i w (r_j - r_i).
// Per pair that is 16 FP32-pipe operations instead of 2 x 12 for the two
// one-sided interactions.  When every body of a tile has the same mass m0
// (equal-mass particles, as in the paper's models), the sums leave the mass
// out and take m0 once per tile sum: 14 operations per pair.
//
// Layout of the work:
//  * bodies are cut into blocks of B = 1024 (128 threads x 8 targets); the
//    block pairs (I <= J) of the triangle are the tiles, one CTA each (four
//    resident per SM), visited in super-tiles of up to 256 x 256 for L2
//    locality.  (Blocks of 2048 with 256 threads were 0.4-14% slower, most
//    at 16-64 K bodies where they gave too few tiles to fill the GPU.)  A
//    diagonal tile (I, I) is evaluated one-sided (every target against every
//    source of the block, j = i left out of the potential); an off-diagonal
//    tile evaluates each of its B x B pairs once.
//  * a CTA keeps its 1024 targets (block I) in registers, two per packed
//    FP32x2 operation, and its 1024 sources (block J) in shared memory,
//    expanded to (x, x, y, y), (z, z, m, m) so that each operand of a packed
//    operation comes from one 16-byte load.
//  * inside a warp, the 32 lanes hold different targets; in step t lane l
//    takes source (l + t) mod 32 of a 32-source chunk, and the partial sum
//    of source s moves one lane down per step (one shuffle), so after 32
//    steps lane s holds the warp's sum for source s.  The warps' sums of a
//    256-source slab are then added in a fixed order through shared memory.
//  * each tile's partial sums (FP32, for its targets and for its sources)
//    are converted to 64-bit fixed-point integers and added with integer
//    atomics.  Integer addition is exact and associative, so the result does
//    not depend on the order in which the CTAs run: it is bitwise
//    reproducible.  The scale is fixed per launch (per simulation in a batch)
//    from a bound on |g|: sum_j |m_j| max_r r / (r^2 + eps^2)^(3/2) =
//    sum_j |m_j| 2 / (3 sqrt(3) eps^2), computed on the device in FP64 by a
//    fixed-order reduction, and placed 2^61 below the int64 limit.  Values below 2^-61 of that bound are
//    rounded away (an absolute error far below the FP32 rounding of any
//    acceleration that is not ~10^10 times smaller than the largest possible
//    one).
//  * keeping the CTA this simple matters: a persistent form (work units of
//    several tiles, TMA-staged source blocks, target sums kept across tiles)
//    was measured 30% slower -- its loop nest made the compiler add register
//    moves in the innermost loop (+21 ALU and +11 FMA-pipe instructions per
//    32-pair step).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "async.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

constexpr int GP_SLAB = 256;                  // sources per cross-warp reduction
constexpr int GP_MASS_BLOCKS = 256;

// Shape of a tile: THREADS threads, RP target pairs (2 RP targets) per
// thread, blocks of B = THREADS x 2 RP bodies; shared memory holds the source
// block expanded to (x, x, y, y), (z, z, m, m), the warp sums of one slab and
// the global indices of the tile's bodies.
template <int THREADS, int RP>
struct PairsShape {
    static constexpr int kB = THREADS * 2 * RP;
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kSmemDup = 2 * kB * 16;
    static constexpr int kSmemPart = kWarps * GP_SLAB * 4 * 4;
    static constexpr int kSmemIdx = 2 * kB * 4;
    static constexpr int kSmem = kSmemDup + kSmemPart + kSmemIdx;
    static_assert(kSmem <= 227 * 1024, "shared memory of the pair kernel");
    static_assert(kB % GP_SLAB == 0 && GP_SLAB % 32 == 0, "slab shape");
};

// The default shape (128 threads, 8 targets each, blocks of 1024); both a
// single simulation and a batch take the shape of pp_gravity_pairs_plan.
constexpr int GP_THREADS = 128;
constexpr int GP_RP = 4;
constexpr int GP_B = PairsShape<GP_THREADS, GP_RP>::kB;

// Fixed-point scale of one simulation: sums of g are integers times 2^e_acc,
// sums of phi integers times 2^e_pot.
struct PairsScale {
    float s_acc1, s_acc2;   // 2^-e_acc as two float factors
    float s_pot1, s_pot2;   // 2^-e_pot
    double lsb_acc, lsb_pot;
};

// Start of the workspace; the fixed-point sums follow at kPairsAccOffset.
// (A batch keeps one PairsScale per simulation in its own workspace.)
struct PairsHeader {
    PairsScale scale;
    double mass_part[GP_MASS_BLOCKS];
};
constexpr size_t kPairsAccOffset = 4096;
static_assert(sizeof(PairsHeader) <= kPairsAccOffset, "pairs header");

// Entry b of a triangle -> (I, J), I <= J, numbered by J, then I
// (b = J (J + 1) / 2 + I).
__device__ __forceinline__ void tri_of(long long b, int &I, int &J) {
    int j = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((long long)j * (j + 1) / 2 > b) --j;
    while ((long long)(j + 1) * (j + 2) / 2 <= b) ++j;
    J = j;
    I = (int)(b - (long long)j * (j + 1) / 2);
}

// CTA b -> tile (I, J).  Tiles are visited in super-tiles of S x S, S =
// 2^lg (the super-tiles themselves in triangle order, the tiles inside row by
// row), so the CTAs resident at one time touch a few target and source
// blocks: their sources and the fixed-point sums they add to stay in L2, and
// DRAM sees each block's sums about once per super-tile (a few GB per launch
// at 4,194,304 bodies, against 239 GB in plain triangle order).
// Returns false for the cells of a super-tile below the diagonal or past the
// last block (those CTAs exit at once).
__device__ __forceinline__ bool tile_of(long long b, int nb, int lg, int &I, int &J) {
    int P, Q;
    tri_of(b >> (2 * lg), P, Q);
    const int local = (int)(b & ((1ll << (2 * lg)) - 1));
    I = (P << lg) + (local >> lg);
    J = (Q << lg) + (local & ((1 << lg) - 1));
    return I <= J && J < nb;
}

// log2 of the super-tile side for nb blocks: large enough to keep DRAM
// traffic low, small enough that few CTAs fall on empty cells.
inline int super_log2(long long nb) { return nb >= 4096 ? 8 : nb >= 1024 ? 7 : nb >= 256 ? 6 : 4; }

// ---------------------------------------------------------------------------
// Scale of the fixed-point sums.
// ---------------------------------------------------------------------------
__global__ void pairs_mass_kernel(const float4 *__restrict__ pos, int n, PairsHeader *__restrict__ h) {
    __shared__ double s[256];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int lo = (int)((long long)n * b / GP_MASS_BLOCKS);
    const int hi = (int)((long long)n * (b + 1) / GP_MASS_BLOCKS);
    double v = 0.0;
    for (int i = lo + tid; i < hi; i += 256) v += fabs((double)pos[i].w);
    s[tid] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) s[tid] += s[tid + w];
        __syncthreads();
    }
    if (tid == 0) h->mass_part[b] = s[0];
}

// Power-of-two scale 2^-e with the bound below 2^(e + 61), as two float
// factors (each within the normal range for |e| <= 250) and as a double.
// Returns false if the bound is not finite or e falls outside that range.
__device__ bool place_scale(double bound, float &s1, float &s2, double &lsb) {
    bool ok = true;
    int e = 0;
    if (bound > 0.0 && bound <= 1.0e300) {
        int k;
        frexp(bound, &k);   // bound < 2^k
        e = k - 61;
    } else if (!(bound == 0.0)) {
        ok = false;
    }
    if (e < -250 || e > 250) {
        ok = false;
        e = 0;
    }
    const int e1 = -e / 2, e2 = -e - e1;
    s1 = ldexpf(1.0f, e1);
    s2 = ldexpf(1.0f, e2);
    lsb = ldexp(1.0, e);
    return ok;
}

// Both scales from the sum M of |m| over the bodies that act on each other.
// max over r of r / (r^2 + eps^2)^(3/2) is 2 / (3 sqrt 3 eps^2) < 0.385 / eps^2.
__device__ void place_scales(double M, float eps, PairsScale &sc, int *flags) {
    const double e = (double)eps;
    const bool ok_a = place_scale(0.385 * M / (e * e), sc.s_acc1, sc.s_acc2, sc.lsb_acc);
    const bool ok_p = place_scale(M / e, sc.s_pot1, sc.s_pot2, sc.lsb_pot);
    if (!(ok_a && ok_p)) atomicOr(flags, SPH_FLAG_GRAV_RANGE);
}

__global__ void pairs_scale_kernel(float eps, PairsHeader *__restrict__ h, int *__restrict__ flags) {
    __shared__ double s[GP_MASS_BLOCKS];
    const int tid = threadIdx.x;
    s[tid] = h->mass_part[tid];
    __syncthreads();
    for (int w = GP_MASS_BLOCKS / 2; w > 0; w >>= 1) {
        if (tid < w) s[tid] += s[tid + w];
        __syncthreads();
    }
    if (tid == 0) place_scales(s[0], eps, h->scale, flags);
}

// A batch: block s sums |m| over simulation s (gas range, then dark range,
// fixed order) and places that simulation's scale, so each simulation keeps
// the resolution of its own mass and unit scale.
__global__ void pairs_batch_scale_kernel(const float4 *__restrict__ pos, const int4 *__restrict__ sims,
                                         float eps, PairsScale *__restrict__ scales,
                                         int *__restrict__ flags) {
    __shared__ double s[256];
    const int tid = threadIdx.x;
    const int4 sd = sims[blockIdx.x];   // (g0, ng, d0, nd)
    double v = 0.0;
    for (int q = tid; q < sd.y; q += 256) v += fabs((double)pos[sd.x + q].w);
    for (int q = tid; q < sd.w; q += 256) v += fabs((double)pos[sd.z + q].w);
    s[tid] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) s[tid] += s[tid + w];
        __syncthreads();
    }
    if (tid == 0) place_scales(s[0], eps, scales[blockIdx.x], flags);
}

__device__ __forceinline__ unsigned long long to_fixed(float v, float s1, float s2) {
    return (unsigned long long)__float2ll_rn(__fmul_rn(__fmul_rn(v, s1), s2));
}

// ---------------------------------------------------------------------------
// One slab (GP_SLAB sources starting at s0) of a tile.  SYM: also collect
// the sums of the sources (off-diagonal tiles) into wpart[GP_SLAB][NC].
// ---------------------------------------------------------------------------
template <bool SYM, bool POT, int THREADS, int RP, bool EQ>
__device__ __forceinline__ void ring_slab(const float4 *__restrict__ dA, const float4 *__restrict__ dB,
                                          int s0, int lane, const float2 (&nx)[RP],
                                          const float2 (&ny)[RP], const float2 (&nz)[RP],
                                          const float2 (&mi)[RP], float2 e2, float2 (&ax)[RP],
                                          float2 (&ay)[RP], float2 (&az)[RP],
                                          float2 (&ap)[RP], float *__restrict__ wpart, int tid) {
    constexpr int NC = POT ? 4 : 3;
    for (int c = 0; c < GP_SLAB / 32; ++c) {
        float cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;   // sums of the source this lane holds
        const int cb = s0 + c * 32;
#pragma unroll 1
        for (int t = 0; t < 32; ++t) {
            const int s = cb + ((lane + t) & 31);
            const float4 a = dA[s];
            const float4 b = dB[s];
            const float2 qx = make_float2(a.x, a.y), qy = make_float2(a.z, a.w);
            const float2 qz = make_float2(b.x, b.y), qm = make_float2(b.z, b.w);
            float2 tx = make_float2(cx, 0.f), ty = make_float2(cy, 0.f), tz = make_float2(cz, 0.f);
            float2 tp = make_float2(cp, 0.f);
#pragma unroll
            for (int p = 0; p < RP; ++p) {
                const float2 dx = __fadd2_rn(qx, nx[p]);
                const float2 dy = __fadd2_rn(qy, ny[p]);
                const float2 dz = __fadd2_rn(qz, nz[p]);
                float2 r2 = __ffma2_rn(dx, dx, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                if (!SYM && POT) {
                    // diagonal tile: leave j = i out of the potential (targets
                    // 2p and 2p + 1 of this thread are block entries
                    // tid + 2p 256 and tid + (2p + 1) 256)
                    if (s == tid + (2 * p) * THREADS) inv.x = 0.f;
                    if (s == tid + (2 * p + 1) * THREADS) inv.y = 0.f;
                }
                const float2 w = __fmul2_rn(__fmul2_rn(inv, inv), inv);
                if (EQ) {
                    // every body of the tile has the same mass: the sums
                    // leave it out and take it once, when the tile's sums
                    // are converted (one product per pair fewer on each side)
                    ax[p] = __ffma2_rn(w, dx, ax[p]);
                    ay[p] = __ffma2_rn(w, dy, ay[p]);
                    az[p] = __ffma2_rn(w, dz, az[p]);
                    if (POT) ap[p] = __fadd2_rn(inv, ap[p]);
                    if (SYM) {
                        tx = __ffma2_rn(w, dx, tx);
                        ty = __ffma2_rn(w, dy, ty);
                        tz = __ffma2_rn(w, dz, tz);
                        if (POT) tp = __fadd2_rn(inv, tp);
                    }
                } else {
                    const float2 si = __fmul2_rn(w, qm);
                    ax[p] = __ffma2_rn(si, dx, ax[p]);
                    ay[p] = __ffma2_rn(si, dy, ay[p]);
                    az[p] = __ffma2_rn(si, dz, az[p]);
                    if (POT) ap[p] = __ffma2_rn(qm, inv, ap[p]);
                    if (SYM) {
                        const float2 sj = __fmul2_rn(w, mi[p]);
                        tx = __ffma2_rn(sj, dx, tx);
                        ty = __ffma2_rn(sj, dy, ty);
                        tz = __ffma2_rn(sj, dz, tz);
                        if (POT) tp = __ffma2_rn(mi[p], inv, tp);
                    }
                }
            }
            if (SYM) {
                const int from = (lane + 1) & 31;
                cx = __shfl_sync(0xffffffffu, __fadd_rn(tx.x, tx.y), from);
                cy = __shfl_sync(0xffffffffu, __fadd_rn(ty.x, ty.y), from);
                cz = __shfl_sync(0xffffffffu, __fadd_rn(tz.x, tz.y), from);
                if (POT) cp = __shfl_sync(0xffffffffu, __fadd_rn(tp.x, tp.y), from);
            }
        }
        if (SYM) {
            float *o = wpart + (c * 32 + lane) * NC;
            o[0] = cx;
            o[1] = cy;
            o[2] = cz;
            if (POT) o[3] = cp;
        }
    }
}

// One tile per CTA.  BATCH: many independent simulations; simulation s owns
// the tiles [tile_off[s], tile_off[s + 1]) of its own triangle, over its
// virtual bodies 0..ns-1 (virtual v < ng is global g0 + v, else d0 + v - ng).
// In a batch, the global index of every target and source of the tile (-1
// for padding) is kept in shared memory for the atomics; one simulation
// computes them (the shared-memory form cost 1.5% there).
template <bool POT, bool BATCH, int THREADS, int RP>
__global__ void __launch_bounds__(THREADS, 1)
pp_gravity_pairs_kernel(const float4 *__restrict__ pos, int n, int nb, int lg,
                        const int4 *__restrict__ sims, const long long *__restrict__ tile_off,
                        int n_sims, float eps2, const PairsScale *__restrict__ scales,
                        unsigned long long *__restrict__ acc) {
    constexpr int NC = POT ? 4 : 3;
    using Sh = PairsShape<THREADS, RP>;
    constexpr int B = Sh::kB;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *dA = reinterpret_cast<float4 *>(smem);
    float4 *dB = dA + B;
    float *part = reinterpret_cast<float *>(dB + B);                   // [warp][slab][NC]
    int *sidx = reinterpret_cast<int *>(smem + Sh::kSmemDup + Sh::kSmemPart);  // [B] sources
    int *tidx = sidx + B;                                               // [B] targets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int I, J, g0 = 0, ng = n, d0 = 0, ns = n, sim = 0;
    if (BATCH) {
        const long long b = blockIdx.x;
        int lo = 0, hi = n_sims - 1;   // last simulation whose first tile is <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        sim = lo;
        const int4 sd = sims[lo];
        g0 = sd.x;
        ng = sd.y;
        d0 = sd.z;
        ns = sd.y + sd.w;
        tri_of(b - tile_off[lo], I, J);
    } else if (!tile_of(blockIdx.x, nb, lg, I, J)) {
        return;
    }
    auto global_of = [&](int v) { return v < ng ? g0 + v : d0 + (v - ng); };
    const int cnt = min(B, ns - J * B);
    for (int q = tid; q < B; q += THREADS) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        int gi = -1;
        if (q < cnt) {
            gi = global_of(J * B + q);
            v = pos[gi];
        }
        if (BATCH) sidx[q] = gi;
        dA[q] = make_float4(v.x, v.x, v.y, v.y);
        dB[q] = make_float4(v.z, v.z, v.w, v.w);
    }
    // targets k of this thread: block entries tid + k 256; pair p = (2p, 2p + 1)
    float2 nx[RP], ny[RP], nz[RP], mi[RP], ax[RP], ay[RP], az[RP], ap[RP];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        const int ka = tid + (2 * p) * THREADS, kb = ka + THREADS;
        const int va = I * B + ka, vb = I * B + kb;
        const int ia = va < ns ? global_of(va) : -1, ib = vb < ns ? global_of(vb) : -1;
        if (BATCH) {
            tidx[ka] = ia;
            tidx[kb] = ib;
        }
        const float4 a = ia >= 0 ? pos[ia] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = ib >= 0 ? pos[ib] : make_float4(0.f, 0.f, 0.f, 0.f);
        nx[p] = make_float2(-a.x, -b.x);
        ny[p] = make_float2(-a.y, -b.y);
        nz[p] = make_float2(-a.z, -b.z);
        mi[p] = make_float2(a.w, b.w);
        ax[p] = ay[p] = az[p] = ap[p] = make_float2(0.f, 0.f);
    }
    const PairsScale sc = scales[sim];
    const float sa1 = sc.s_acc1, sa2 = sc.s_acc2, sp1 = sc.s_pot1, sp2 = sc.s_pot2;
    // A tile whose bodies all have the same mass m0 (and no padding) takes
    // the sums without the mass factors, and m0 once per sum at the end.
    // Without the mass a sum is bounded by B x 0.385 / eps^2, so eps must
    // keep that far inside FP32 (any eps above 1e-15 does).
    const float m0 = pos[global_of(I * B)].w;
    bool same = cnt == B && (I + 1) * B <= ns && eps2 > 1e-30f;
    for (int q = tid; q < B; q += THREADS) same = same && dB[q].z == m0;
#pragma unroll
    for (int p = 0; p < RP; ++p) same = same && mi[p].x == m0 && mi[p].y == m0;
    const bool eq = __syncthreads_and(same) != 0;
    const float2 e2 = make_float2(eps2, eps2);
    float *wpart = part + warp * GP_SLAB * NC;
    if (I != J) {
        for (int s0 = 0; s0 < cnt; s0 += GP_SLAB) {   // sources past cnt are massless padding
            if (eq)
                ring_slab<true, POT, THREADS, RP, true>(dA, dB, s0, lane, nx, ny, nz, mi, e2, ax, ay, az, ap,
                                                        wpart, tid);
            else
                ring_slab<true, POT, THREADS, RP, false>(dA, dB, s0, lane, nx, ny, nz, mi, e2, ax, ay, az, ap,
                                                         wpart, tid);
            __syncthreads();
            for (int q = tid; q < GP_SLAB * NC; q += THREADS) {
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < Sh::kWarps; ++w) v = __fadd_rn(v, part[w * GP_SLAB * NC + q]);
                if (eq) v = __fmul_rn(v, m0);
                const int comp = q % NC;
                int j;
                if (BATCH) j = sidx[s0 + q / NC];
                else j = (J * B + s0 + q / NC < n) ? J * B + s0 + q / NC : -1;
                if (j >= 0)
                    atomicAdd(&acc[(size_t)j * 4 + comp],
                              comp < 3 ? to_fixed(-v, sa1, sa2) : to_fixed(v, sp1, sp2));
            }
            __syncthreads();   // warp sums consumed before the next slab
        }
    } else {
        for (int s0 = 0; s0 < cnt; s0 += GP_SLAB) {
            if (eq)
                ring_slab<false, POT, THREADS, RP, true>(dA, dB, s0, lane, nx, ny, nz, mi, e2, ax, ay, az, ap,
                                                         wpart, tid);
            else
                ring_slab<false, POT, THREADS, RP, false>(dA, dB, s0, lane, nx, ny, nz, mi, e2, ax, ay, az, ap,
                                                          wpart, tid);
        }
    }
    // the tile's sums of its targets
#pragma unroll
    for (int p = 0; p < RP; ++p) {
        if (eq) {
            const float2 m2 = make_float2(m0, m0);
            ax[p] = __fmul2_rn(ax[p], m2);
            ay[p] = __fmul2_rn(ay[p], m2);
            az[p] = __fmul2_rn(az[p], m2);
            if (POT) ap[p] = __fmul2_rn(ap[p], m2);
        }
        int ia, ib;
        if (BATCH) {
            ia = tidx[tid + (2 * p) * THREADS];
            ib = tidx[tid + (2 * p + 1) * THREADS];
        } else {
            ia = I * B + tid + (2 * p) * THREADS;
            ib = ia + THREADS;
            if (ia >= n) ia = -1;
            if (ib >= n) ib = -1;
        }
        if (ia >= 0) {
            atomicAdd(&acc[(size_t)ia * 4 + 0], to_fixed(ax[p].x, sa1, sa2));
            atomicAdd(&acc[(size_t)ia * 4 + 1], to_fixed(ay[p].x, sa1, sa2));
            atomicAdd(&acc[(size_t)ia * 4 + 2], to_fixed(az[p].x, sa1, sa2));
            if (POT) atomicAdd(&acc[(size_t)ia * 4 + 3], to_fixed(ap[p].x, sp1, sp2));
        }
        if (ib >= 0) {
            atomicAdd(&acc[(size_t)ib * 4 + 0], to_fixed(ax[p].y, sa1, sa2));
            atomicAdd(&acc[(size_t)ib * 4 + 1], to_fixed(ay[p].y, sa1, sa2));
            atomicAdd(&acc[(size_t)ib * 4 + 2], to_fixed(az[p].y, sa1, sa2));
            if (POT) atomicAdd(&acc[(size_t)ib * 4 + 3], to_fixed(ap[p].y, sp1, sp2));
        }
    }
}

// Fixed-point totals -> float4 (gx, gy, gz, phi).  BATCH: body i takes the
// scale of its simulation (the last one whose gas / dark range starts at or
// before i).
template <bool POT, bool BATCH>
__global__ void pairs_final_kernel(int n, int n_gas, float G, const PairsScale *__restrict__ scales,
                                   const int4 *__restrict__ sims, int n_sims,
                                   const long long *__restrict__ acc, float4 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int sim = 0;
    if (BATCH) {
        const bool gas = i < n_gas;
        int lo = 0, hi = n_sims - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((gas ? sims[mid].x : sims[mid].z) <= i) lo = mid;
            else hi = mid - 1;
        }
        sim = lo;
    }
    const PairsScale sc = scales[sim];
    const double la = sc.lsb_acc * (double)G;
    const long long *a = acc + (size_t)i * 4;
    const float phi = POT ? (float)(-(double)G * (double)a[3] * sc.lsb_pot) : 0.f;
    out[i] = make_float4((float)((double)a[0] * la), (float)((double)a[1] * la),
                         (float)((double)a[2] * la), phi);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static std::once_flag g_pairs_once;
static int g_pairs_status = SPH_OK;
static int g_pairs_min_n = 16384;   // measured crossover with the one-sided kernel
static std::mutex g_pairs_mutex;

// Launch plan of a single simulation's tiles: threads per CTA, target pairs
// per thread, super-tile side 2^lg blocks (lg < 0: by size, super_log2).
struct PairsPlan {
    int threads, rp, lg;
};
static PairsPlan g_pairs_plan{GP_THREADS, GP_RP, -1};

using PairsKernel = void (*)(const float4 *, int, int, int, const int4 *, const long long *, int,
                             float, const PairsScale *, unsigned long long *);

struct PairsVariant {
    PairsKernel k;
    int smem;
};

template <int THREADS, int RP>
static PairsVariant pairs_variant(bool pot, bool batch) {
    const int smem = PairsShape<THREADS, RP>::kSmem;
    if (pot) return {batch ? pp_gravity_pairs_kernel<true, true, THREADS, RP>
                           : pp_gravity_pairs_kernel<true, false, THREADS, RP>, smem};
    return {batch ? pp_gravity_pairs_kernel<false, true, THREADS, RP>
                  : pp_gravity_pairs_kernel<false, false, THREADS, RP>, smem};
}

// The shapes the plan may name: (128, 3), (128, 4), (128, 5) and (256, 4),
// i.e. blocks of 768, 1024, 1280 and 2048 bodies.
static bool pairs_shape_ok(int threads, int rp) {
    return (threads == 128 && rp >= 3 && rp <= 5) || (threads == 256 && rp == 4);
}

static PairsVariant pairs_pick(int threads, int rp, bool pot, bool batch) {
    if (threads == 256) return pairs_variant<256, 4>(pot, batch);
    if (rp == 3) return pairs_variant<128, 3>(pot, batch);
    if (rp == 5) return pairs_variant<128, 5>(pot, batch);
    return pairs_variant<128, 4>(pot, batch);
}

static void pairs_init() {
    const int shapes[kPairsNumShapes][2] = {{128, 3}, {128, 4}, {128, 5}, {256, 4}};
    for (auto &sh : shapes)
        for (int f = 0; f < 4; ++f) {
            const PairsVariant v = pairs_pick(sh[0], sh[1], f & 1, f & 2);
            if (cudaFuncSetAttribute((const void *)v.k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     v.smem) != cudaSuccess)
                g_pairs_status = SPH_ERR_CUDA;
        }
}

static PairsPlan pairs_plan() {
    std::lock_guard<std::mutex> lock(g_pairs_mutex);
    return g_pairs_plan;
}

// The launches of one evaluation over n bodies: zero the scratch, the scale,
// the tiles (one simulation: nb blocks of the plan's shape in super-tiles of
// 2^lg; a batch: n_ctas tiles of the default shape described by sims /
// tile_off), then the fixed-point totals -> out.
static int pairs_launch(const float4 *pos, int n, int n_gas, float G, float eps, float4 *out,
                        int flags, void *d_work, int nb, int lg, PairsPlan plan, const int4 *sims,
                        const long long *tile_off, int n_sims, long long n_ctas,
                        PairsScale *batch_scales, cudaStream_t st) {
    std::call_once(g_pairs_once, pairs_init);
    if (g_pairs_status != SPH_OK) return g_pairs_status;
    int *flags_dev = gravity_flags_device();
    if (!flags_dev) return SPH_ERR_CUDA;
    if (n_ctas > 0x7fffffffll) return SPH_ERR_INVALID_ARG;
    const bool pot = flags & SPH_GRAV_POTENTIAL;
    const bool batch = sims != nullptr;
    PairsHeader *hdr = static_cast<PairsHeader *>(d_work);
    unsigned long long *acc =
        reinterpret_cast<unsigned long long *>(static_cast<unsigned char *>(d_work) + kPairsAccOffset);
    const float eps2 = eps * eps;
    SPH_CUDA_TRY(cudaMemsetAsync(d_work, 0, pp_gravity_pairs_workspace_bytes(n), st));
    const PairsScale *scales;
    if (batch) {
        pairs_batch_scale_kernel<<<n_sims, 256, 0, st>>>(pos, sims, eps, batch_scales, flags_dev);
        scales = batch_scales;
    } else {
        pairs_mass_kernel<<<GP_MASS_BLOCKS, 256, 0, st>>>(pos, n, hdr);
        pairs_scale_kernel<<<1, GP_MASS_BLOCKS, 0, st>>>(eps, hdr, flags_dev);
        scales = &hdr->scale;
    }
    const PairsVariant v = pairs_pick(plan.threads, plan.rp, pot, batch);
    if (n_ctas > 0)
        v.k<<<(unsigned)n_ctas, plan.threads, v.smem, st>>>(pos, n, nb, lg, sims, tile_off, n_sims, eps2,
                                                            scales, acc);
    const long long *acc_s = reinterpret_cast<const long long *>(acc);
    auto f = pot ? (batch ? pairs_final_kernel<true, true> : pairs_final_kernel<true, false>)
                 : (batch ? pairs_final_kernel<false, true> : pairs_final_kernel<false, false>);
    f<<<(n + 255) / 256, 256, 0, st>>>(n, n_gas, G, scales, sims, n_sims, acc_s, out);
    note_launch((n_ctas > 0 ? 3 : 2) + (batch ? 0 : 1));
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

size_t pairs_scale_bytes() { return sizeof(PairsScale); }

// The block shapes a plan may name, in a fixed order (index 0..3).
static const int kPairsShapes[kPairsNumShapes][2] = {{128, 3}, {128, 4}, {128, 5}, {256, 4}};

int pairs_shape_block(int shape) { return kPairsShapes[shape][0] * 2 * kPairsShapes[shape][1]; }

int pairs_current_shape() {
    const PairsPlan p = pairs_plan();
    for (int k = 0; k < kPairsNumShapes; ++k)
        if (kPairsShapes[k][0] == p.threads && kPairsShapes[k][1] == p.rp) return k;
    return 1;
}

// Tiles of simulation s with ns bodies in blocks of B: nb_s (nb_s + 1) / 2,
// nb_s = ceil(ns / B).
long long pairs_tiles(long long ns, int B) {
    const long long nb = (ns + B - 1) / B;
    return nb * (nb + 1) / 2;
}

int launch_gravity_pairs_batched(const float4 *pos, int n, int n_gas, const int4 *d_sims,
                                 const long long *d_tile_off, int n_sims, long long n_tiles,
                                 int shape, void *d_scales, float G, float eps, float4 *out,
                                 int flags, void *d_work, cudaStream_t st) {
    if (shape < 0 || shape >= kPairsNumShapes) return SPH_ERR_INVALID_ARG;
    const PairsPlan plan{kPairsShapes[shape][0], kPairsShapes[shape][1], -1};
    return pairs_launch(pos, n, n_gas, G, eps, out, flags, d_work, 0, 0, plan, d_sims, d_tile_off,
                        n_sims, n_tiles, static_cast<PairsScale *>(d_scales), st);
}

}  // namespace sphgb

using namespace sphgb;

extern "C" size_t pp_gravity_pairs_workspace_bytes(int32_t n) {
    if (n < 0) return 0;
    return kPairsAccOffset + (size_t)n * 4 * sizeof(long long);
}

extern "C" int pp_gravity_pairs_min_n(int32_t n_min) {
    if (n_min < 0) return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_pairs_mutex);
    g_pairs_min_n = n_min ? n_min : 16384;
    return SPH_OK;
}

extern "C" int pp_gravity_pairs_eligible(int32_t n, float eps, int32_t flags) {
    int min_n;
    {
        std::lock_guard<std::mutex> lock(g_pairs_mutex);
        min_n = g_pairs_min_n;
    }
    const float eps2 = eps * eps;
    return (n >= min_n && n > 0 && eps2 > 0.0f && eps2 <= 3.0e38f &&
            !(flags & SPH_GRAV_NO_KAHAN) && !gravity_plan_forced())
               ? 1
               : 0;
}

extern "C" int pp_gravity_pairs(const float *d_pos_m, int32_t n, float G, float eps,
                                float *d_acc_pot, int32_t flags, void *d_work, size_t work_bytes,
                                sph_stream_t stream) {
    if (n < 0 || !(eps >= 0.0f) || !(G == G)) return SPH_ERR_INVALID_ARG;
    if (n == 0) return SPH_OK;
    if (!pp_gravity_pairs_eligible(n, eps, flags) || !d_work ||
        work_bytes < pp_gravity_pairs_workspace_bytes(n))
        return pp_gravity(d_pos_m, n, G, eps, d_acc_pot, flags, stream);
    if (!d_pos_m || !d_acc_pot) return SPH_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_pos_m) & 15u) ||
        (reinterpret_cast<uintptr_t>(d_acc_pot) & 15u) ||
        (reinterpret_cast<uintptr_t>(d_work) & 255u))
        return SPH_ERR_INVALID_ARG;
    const PairsPlan plan = pairs_plan();
    const int B = plan.threads * 2 * plan.rp;
    const long long nb = (n + B - 1) / B;
    const int lg = plan.lg >= 0 ? plan.lg : super_log2(nb);
    const long long nsb = (nb + (1ll << lg) - 1) >> lg;
    const long long n_ctas = (nsb * (nsb + 1) / 2) << (2 * lg);
    if (n_ctas > 0x7fffffffll)   // more than ~1.3e8 bodies: one CTA per tile no longer fits a grid
        return pp_gravity(d_pos_m, n, G, eps, d_acc_pot, flags, stream);
    return pairs_launch(reinterpret_cast<const float4 *>(d_pos_m), n, n, G, eps,
                        reinterpret_cast<float4 *>(d_acc_pot), flags, d_work, (int)nb, lg, plan,
                        nullptr, nullptr, 1, n_ctas, nullptr, (cudaStream_t)stream);
}

extern "C" int pp_gravity_pairs_plan(int32_t threads, int32_t R, int32_t super_log2_side) {
    if (threads == 0) {
        std::lock_guard<std::mutex> lock(g_pairs_mutex);
        g_pairs_plan = PairsPlan{GP_THREADS, GP_RP, -1};
        return SPH_OK;
    }
    if ((R & 1) || !pairs_shape_ok(threads, R / 2) || super_log2_side < -1 || super_log2_side > 8)
        return SPH_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_pairs_mutex);
    g_pairs_plan = PairsPlan{threads, R / 2, super_log2_side};
    return SPH_OK;
}

extern "C" int pp_gravity_pairs_get_plan(int32_t n, int32_t *h_threads, int32_t *h_R,
                                         int32_t *h_super_log2) {
    if (n < 0 || !h_threads || !h_R || !h_super_log2) return SPH_ERR_INVALID_ARG;
    const PairsPlan plan = pairs_plan();
    const long long nb = ((long long)n + plan.threads * 2 * plan.rp - 1) / (plan.threads * 2 * plan.rp);
    *h_threads = plan.threads;
    *h_R = 2 * plan.rp;
    *h_super_log2 = plan.lg >= 0 ? plan.lg : super_log2(nb);
    return SPH_OK;
}
