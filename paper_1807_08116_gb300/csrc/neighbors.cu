// neighbors.cu -- per-particle neighbour lists over the multi-level hashed
// grid built by the sorting stage.  The paper's DC and HFC kernels walk the
// cells around each particle with indexPC, CellSPH and hmaxCell (Sect. 3);
// here the walk is done once per step and its result is stored as CSR lists,
// which density and both force evaluations then stream.
//
// j is a neighbour of i (j != i) iff, in FP32, ((dx*dx + dy*dy) + dz*dz) <
// (h_i + h_j)^2, i.e. |r_ij| < 2 h_ij, the support of W and W_p (Eqs. 8-9).
//
// Search: particle i (level l_i) visits only levels l >= l_i.  On level l
// every particle has h <= hmax_l, so all its possible neighbours lie in the
// cells covering [x_i - R, x_i + R] with R = h_i + hmax_l (widened by a few
// ulps so that FP32 rounding of the predicate can never reach outside).
// Because h_i <= L0 2^l_i <= L0 2^l and hmax_l <= L0 2^l, this box spans at
// most 5 cells per axis.  A pair on the same level is found from both ends;
// a pair with l_j > l_i is found only by i, which appends j to its own row
// and i to j's row ("reverse" part, atomic cursor).  Buckets are shared by
// distinct cells through the hash; each candidate is accepted only if its own
// level and cell equal the probed ones, so no pair is counted twice.
// Rows are [own part in search order | reverse part sorted ascending].
//
// The walk is warp-cooperative.  A warp takes 32 consecutive sorted rows
// (neighbours in space, since the sort is by cell) and splits them into
// groups: a leader row and every other pending row of the same simulation
// and level whose cell lies within kNbGroupReach cells of the leader's on
// that level.  A group walks the union of its members' search boxes with
// warp-uniform loops, 32 cells at a time: lane t reads the bucket of cell
// c0 + t, so one round trip covers 32 probes, and a cell is kept when it
// lies within reach of the group's box (the members' extent, largest h and
// largest rounding margins: one test per probed cell, by the lane that
// probed it).  The candidates of the kept
// cells are numbered in cell order and loaded 32 at a time (one per lane),
// their level, cell and simulation are checked once by the lane that loaded
// them, and the survivors are broadcast from shared memory to every member,
// which applies the FP32 predicate to its own row.  The box and the cut are
// conservative (no neighbour of a row lies outside them), so each member
// accepts exactly its neighbours on the level, in the order (level, z, y, x,
// sorted index) of a row-by-row walk: the lists equal the ones a per-row
// search produces.

#include <climits>

#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

__device__ __forceinline__ void search_box(float x, float R, float x0, float inv_c, int &lo,
                                           int &hi) {
    // R' >= R (1 + 16 ulp) + |x| 4 ulp: covers every FP32 rounding path of the
    // predicate and of x +- R'
    float m = fmaf(R, 1.0f + 3.814697265625e-06f, fmaf(fabsf(x), 9.5367431640625e-07f, 1e-30f));
    lo = cell_of(__fsub_rn(x, m), x0, inv_c);
    hi = cell_of(__fadd_rn(x, m), x0, inv_c);
}

constexpr unsigned kFull = 0xffffffffu;

// FP32 <-> int maps that keep the order of non-NaN values, so that the
// warp's integer min / max reductions give float extremes
__device__ __forceinline__ int ord_of(float f) {
    const int i = __float_as_int(f);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float float_of_ord(int i) {
    return __int_as_float(i ^ ((i >> 31) & 0x7fffffff));
}
__device__ __forceinline__ float warp_minf(float f) {
    return float_of_ord(__reduce_min_sync(kFull, ord_of(f)));
}
__device__ __forceinline__ float warp_maxf(float f) {
    return float_of_ord(__reduce_max_sync(kFull, ord_of(f)));
}

constexpr int kNbWarps = 4;   // warps (row groups of 32) per block
// rows whose cell lies within this many cells of the leader's join its group
// (2, 3 and 4 measured; 3 and 4 within 1% of each other, 2 is 10% slower)
constexpr int kNbGroupReach = 3;
// The first own entries of each row are staged in shared memory, column by
// column (entry c of the warp's lane r at c * 33 + r: conflict-free when the
// lanes append their c-th entries together, and when one row is read back by
// the whole warp), and written to the global staging rows with coalesced
// stores once the warp is done; later entries go to global memory directly.
constexpr int kStageSmem = 44;
constexpr int kStageStride = 33;

// MODE: NB_COUNT counts own entries (and reverse entries of the coarser
// partners); NB_FILL writes own and reverse entries into their CSR places;
// NB_STAGE counts like NB_COUNT and also writes the first stage_k own
// entries of the row to stage[i * stage_k + c], coarser partners with the top
// bit set (rows with more are queued on the overflow list); NB_FILL_LISTED
// runs NB_FILL for the queued rows only.
enum { NB_COUNT = 0, NB_FILL = 1, NB_STAGE = 2, NB_FILL_LISTED = 3 };

// Append j to the own part of row i, and count or place the reverse entry
// (i in the row of j) when j sits on a coarser level.
template <int MODE>
__device__ __forceinline__ void nb_accept(const NbArgs &a, int i, int j, bool coarser,
                                          long long base, int &cnt, int *sstage, int lane) {
    constexpr bool FILL = MODE == NB_FILL || MODE == NB_FILL_LISTED;
    if (FILL) {
        const long long w = base + cnt;
        if (w < a.capacity) a.nb_idx[w] = j;
        else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
        if (coarser) {
            const int pos = atomicAdd(&a.rev[j], 1);
            const long long wr = (long long)a.nb_start[j] + a.own[j] + pos;
            if (wr < a.capacity) a.nb_idx[wr] = i;
            else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
        }
    } else {
        if (MODE == NB_STAGE) {
            // the top bit marks a coarser partner for the copy pass
            const int v = coarser ? (int)((unsigned)j | 0x80000000u) : j;
            if (cnt < kStageSmem) sstage[cnt * kStageStride + lane] = v;
            else if (cnt < a.stage_k) a.stage[(long long)i * a.stage_k + cnt] = v;
        }
        if (coarser) atomicAdd(&a.rev[j], 1);
    }
    ++cnt;
}

template <int MODE>
__global__ void __launch_bounds__(kNbWarps * 32, 8) nb_kernel(NbArgs a) {
    constexpr bool FILL = MODE == NB_FILL || MODE == NB_FILL_LISTED;
    // candidates of a batch in pairs, (x, x', y, y') and (z, z', h, h') per
    // pair of slots, so a pair feeds packed FP32x2 operations from two
    // 16-byte loads (33 slots with the padding one)
    __shared__ __align__(16) float s_cq[kNbWarps][8 * 17];
    __shared__ int s_j[kNbWarps][32];
    __shared__ int s_stage[MODE == NB_STAGE ? kNbWarps : 1][MODE == NB_STAGE ? kStageSmem * kStageStride : 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *sq = s_cq[wib];
    int *sj = s_j[wib];
    int *sstage = s_stage[MODE == NB_STAGE ? wib : 0];
    const long long r = ((long long)blockIdx.x * kNbWarps + wib) * 32 + lane;
    const int rows = MODE == NB_FILL_LISTED ? *a.list_count : a.n;
    const bool act = r < rows;
    unsigned todo = __ballot_sync(kFull, act);
    if (todo == 0u) return;   // the whole warp lies past the last row
    const int i = act ? (MODE == NB_FILL_LISTED ? a.list[r] : (int)r) : 0;
    const GridDev g = *a.grid;
    const float4 p = act ? a.pos_h_s[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int li = level_of(p.w, g.log2_L0, g.n_levels);
    const int si = (act && a.sim_s) ? a.sim_s[i] : 0;
    int cnt = 0;
    long long base = 0;
    if (FILL && act) base = a.nb_start[i];
    const float2 px2 = make_float2(p.x, p.x), py2 = make_float2(p.y, p.y),
                 pz2 = make_float2(p.z, p.z);
    while (todo) {
        // the next group: the lowest pending row and the pending rows of its
        // simulation and level whose cells are near the leader's
        const int ld = __ffs(todo) - 1;
        const int lg = __shfl_sync(kFull, li, ld);
        const int sg = __shfl_sync(kFull, si, ld);
        bool mem;
        {
            const float inv_g = pow2f(-g.log2_L0 - lg);
            const int cx = cell_of(p.x, g.x0, inv_g), cy = cell_of(p.y, g.y0, inv_g),
                      cz = cell_of(p.z, g.z0, inv_g);
            const int gx = __shfl_sync(kFull, cx, ld), gy = __shfl_sync(kFull, cy, ld),
                      gz = __shfl_sync(kFull, cz, ld);
            mem = ((todo >> lane) & 1u) && li == lg && si == sg && abs(cx - gx) <= kNbGroupReach &&
                  abs(cy - gy) <= kNbGroupReach && abs(cz - gz) <= kNbGroupReach;
        }
        todo &= ~__ballot_sync(kFull, mem);
        const unsigned salt_sim = (unsigned)(kMaxLevels * sg);
        for (int l = lg; l < g.n_levels; ++l) {
            if (a.lvl_count[l] == 0) continue;
            const float R = __fadd_rn(p.w, __uint_as_float(a.lvl_hmax[l]));
            const float inv_c = pow2f(-g.log2_L0 - l);
            int lx = 0, hx = -1, ly = 0, hy = -1, lz = 0, hz = -1;
            bool on = mem && R >= 0.0f;
            if (on) {
                search_box(p.x, R, g.x0, inv_c, lx, hx);
                search_box(p.y, R, g.y0, inv_c, ly, hy);
                search_box(p.z, R, g.z0, inv_c, lz, hz);
                const long long ncell = (long long)(hx - lx + 1) * (hy - ly + 1) * (hz - lz + 1);
                if (ncell > (1ll << 24)) {
                    set_flag(a.flags, SPH_FLAG_SEARCH_WIDE);
                    on = false;
                }
            }
            unsigned pend = __ballot_sync(kFull, on);
            if (pend == 0u) continue;
            // a union box above the one-row cap is walked row by row (only
            // top-level rows, whose h may exceed the level's cells, get here)
            bool solo;
            {
                const int ux = __reduce_max_sync(kFull, on ? hx : INT_MIN) -
                               __reduce_min_sync(kFull, on ? lx : INT_MAX);
                const int uy = __reduce_max_sync(kFull, on ? hy : INT_MIN) -
                               __reduce_min_sync(kFull, on ? ly : INT_MAX);
                const int uz = __reduce_max_sync(kFull, on ? hz : INT_MIN) -
                               __reduce_min_sync(kFull, on ? lz : INT_MAX);
                solo = (long long)(ux + 1) * (uy + 1) * (uz + 1) > (1ll << 24);
            }
            const float csz = pow2f(g.log2_L0 + l);
            // the row in cell units of this level, less half a cell, and its
            // rounding margins (|coordinate| of anything in the row's box is
            // at most |x0| + (hi + 1) csz; 2^-20 of that covers the rounding of
            // the predicate, of the cell binning and of the distance below)
            const float uhx = __fmul_rn(__fsub_rn(p.x, g.x0), inv_c) - 0.5f;
            const float uhy = __fmul_rn(__fsub_rn(p.y, g.y0), inv_c) - 0.5f;
            const float uhz = __fmul_rn(__fsub_rn(p.z, g.z0), inv_c) - 0.5f;
            const float mhx = 0.5f + (9.5367431640625e-07f * (fabsf(p.x) + 2.0f * fabsf(g.x0) + (float)(hx + 2) * csz) + 1e-30f) * inv_c;
            const float mhy = 0.5f + (9.5367431640625e-07f * (fabsf(p.y) + 2.0f * fabsf(g.y0) + (float)(hy + 2) * csz) + 1e-30f) * inv_c;
            const float mhz = 0.5f + (9.5367431640625e-07f * (fabsf(p.z) + 2.0f * fabsf(g.z0) + (float)(hz + 2) * csz) + 1e-30f) * inv_c;
            const unsigned salt = ((unsigned)l + salt_sim) * (unsigned)kLevelSalt;
            const unsigned kmask = (1u << g.log2_M) - 1u;
            while (pend) {
                const unsigned part = solo ? (pend & (0u - pend)) : pend;
                pend &= ~part;
                const bool in = (part >> lane) & 1u;
                const int LX = __reduce_min_sync(kFull, in ? lx : INT_MAX);
                const int HX = __reduce_max_sync(kFull, in ? hx : INT_MIN);
                const int LY = __reduce_min_sync(kFull, in ? ly : INT_MAX);
                const int HY = __reduce_max_sync(kFull, in ? hy : INT_MIN);
                const int LZ = __reduce_min_sync(kFull, in ? lz : INT_MAX);
                const int HZ = __reduce_max_sync(kFull, in ? hz : INT_MIN);
                if (a.occ && l > lg) {
                    // skip the level when none of the super-cells the box
                    // touches holds a particle of it (the rows' own level is
                    // always occupied); one super-cell per lane, 32 per round
                    // trip
                    const int SX = LX >> kSuperShift, SY = LY >> kSuperShift, SZ = LZ >> kSuperShift;
                    const int nsx = (HX >> kSuperShift) - SX + 1, nsy = (HY >> kSuperShift) - SY + 1;
                    const int ns = nsx * nsy * ((HZ >> kSuperShift) - SZ + 1);
                    bool any = false;
                    for (int b0 = 0; b0 < ns && !any; b0 += 32) {
                        const int t = b0 + lane;
                        bool hit = false;
                        if (t < ns) {
                            const int qx = t / nsx, qy = qx / nsy;
                            const unsigned bit = super_bit(SX + (t - qx * nsx), SY + (qx - qy * nsy), SZ + qy,
                                                           l + kMaxLevels * sg, a.log2_B);
                            hit = (a.occ[bit >> 5] >> (bit & 31)) & 1u;
                        }
                        any = __any_sync(kFull, hit);
                    }
                    if (!any) continue;
                }
                // the end cells are open on their outer side: only boxes that
                // touch them take the slower distance
                const bool edge = LX == 0 || LY == 0 || LZ == 0 || HX == kCellMax || HY == kCellMax ||
                                  HZ == kCellMax;
                // The union box is walked 32 cells at a time in z, y, x order:
                // lane t probes cell c0 + t, so the bucket reads of 32 cells
                // are one round trip.  A row's predicate sees only its own
                // level's candidates (its h is replaced by NaN, which fails
                // every test, when it takes no part in this level).
                const float2 ph2 = in ? make_float2(p.w, p.w) : make_float2(__uint_as_float(0x7fc00000u),
                                                                           __uint_as_float(0x7fc00000u));
                const float ihw = in ? __fmul_rn(p.w, inv_c) : 0.0f;
                // the group's extent in cell units (extremes of its members'
                // u - 1/2), its largest rounding margins and its largest h
                const float inf = __int_as_float(0x7f800000);
                const float AX = warp_minf(in ? uhx : inf), BX = warp_maxf(in ? uhx : -inf);
                const float AY = warp_minf(in ? uhy : inf), BY = warp_maxf(in ? uhy : -inf);
                const float AZ = warp_minf(in ? uhz : inf), BZ = warp_maxf(in ? uhz : -inf);
                const float MX = warp_maxf(in ? mhx : 0.0f), MY = warp_maxf(in ? mhy : 0.0f),
                            MZ = warp_maxf(in ? mhz : 0.0f), IH = warp_maxf(ihw);
                const int NX = HX - LX + 1, NY = HY - LY + 1;
                const int ncell = NX * NY * (HZ - LZ + 1);
                // a probe lane's cell from its index by FP32 reciprocals: below
                // 2^22 the estimate of each quotient is off by at most one, and
                // one correction makes it exact (cheaper than integer division)
                const float rNX = 1.0f / (float)NX, rNY = 1.0f / (float)NY;
                const bool fdiv = ncell < (1 << 22);
                // candidates identified by the sort's cell tags (a box under
                // 512 cells on every axis), else by their level and cell
                const bool tagged = a.tag_s && NX < 512 && NY < 512 && HZ - LZ < 511;
                for (int c0 = 0; c0 < ncell; c0 += 32) {
                    const int ct = c0 + lane;
                    int qx, ty;
                    if (fdiv) {
                        qx = (int)__fmul_rn((float)ct, rNX);
                        {
                            const int rr = ct - qx * NX;
                            if (rr < 0) --qx;
                            else if (rr >= NX) ++qx;
                        }
                        ty = (int)__fmul_rn((float)qx, rNY);
                        {
                            const int rr = qx - ty * NY;
                            if (rr < 0) --ty;
                            else if (rr >= NY) ++ty;
                        }
                    } else {
                        qx = ct / NX;
                        ty = qx / NY;
                    }
                    const int tx = LX + (ct - qx * NX), tyy = LY + (qx - ty * NY), tz = LZ + ty;
                    int s = 0, e = 0;
                    unsigned hm = 0u;
                    if (ct < ncell) {
                        const unsigned m = spread3_lo((unsigned)tx) | (spread3_lo((unsigned)tyy) << 1) |
                                           (spread3_lo((unsigned)tz) << 2);
                        const int k = (int)((m + salt) & kmask);
                        s = a.cell_start[k];
                        e = a.cell_start[k + 1];
                        hm = a.hmax_cell[k];
                    }
                    const unsigned live = __ballot_sync(kFull, s < e);
                    const unsigned ptag = cell_tag(l, tx, tyy, tz);
                    if (live == 0u) continue;
                    const float ftx = (float)tx, fty = (float)tyy, ftz = (float)tz;
                    // the bucket's max h in cell units, by the lane that read it
                    const float hmc = __fmul_rn(__uint_as_float(hm), inv_c);
                    // keep the cells within reach of the group's box: the
                    // distance from the box to the cell against the largest
                    // h of the group plus the bucket's max h, widened by the
                    // largest rounding margins.  Each of these bounds the
                    // member's own value from the right side and rounding is
                    // monotone, so every cell within a member's own reach
                    // (and hence every cell its predicate can accept from) is
                    // kept; the predicate alone decides the lists.
                    float gx = fmaxf(fmaxf(AX - ftx, ftx - BX) - MX, 0.0f);
                    float gy = fmaxf(fmaxf(AY - fty, fty - BY) - MY, 0.0f);
                    float gz = fmaxf(fmaxf(AZ - ftz, ftz - BZ) - MZ, 0.0f);
                    if (edge) {
                        // the end cells also hold everything clamped into them
                        if ((tx == 0 && AX < 0.0f) || (tx == kCellMax && BX > (float)kCellMax)) gx = 0.0f;
                        if ((tyy == 0 && AY < 0.0f) || (tyy == kCellMax && BY > (float)kCellMax)) gy = 0.0f;
                        if ((tz == 0 && AZ < 0.0f) || (tz == kCellMax && BZ > (float)kCellMax)) gz = 0.0f;
                    }
                    const float gd2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
                    const float greach = IH + hmc;
                    const bool keep = !(gd2 > greach * greach * (1.0f + 3.0517578125e-05f));
                    const unsigned want = __ballot_sync(kFull, s < e && keep);
                    // the candidates of the kept cells, numbered in cell order
                    const int len = ((want >> lane) & 1u) ? e - s : 0;
                    int incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int total = __shfl_sync(kFull, incl, 31);
                    for (int b0 = 0; b0 < total; b0 += 32) {
                        // candidate b0 + lane: its cell t is the number of
                        // cells whose running end does not pass it
                        const int gi = b0 + lane;
                        int t = 0;
#pragma unroll
                        for (int st = 16; st >= 1; st >>= 1)
                            if (__shfl_sync(kFull, incl, t + st - 1) <= gi) t += st;
                        t = min(t, 31);
                        const int jl = __shfl_sync(kFull, s, t) + gi -
                                       (__shfl_sync(kFull, incl, t) - __shfl_sync(kFull, len, t));
                        bool ok = gi < total && (unsigned)jl < (unsigned)a.n;
                        float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        // the identity checks (same simulation, level and cell
                        // as the probed one), once per candidate
                        if (tagged) {
                            // the sort's cell tag: equal tags on one level mean
                            // the same cell or one 512 cells away on some axis,
                            // which lies outside a box under 512 cells wide and
                            // so beyond every member's reach: the predicate
                            // rejects it, and no candidate is taken twice
                            const unsigned pt = __shfl_sync(kFull, ptag, t);
                            if (ok) {
                                q = a.pos_h_s[jl];
                                ok = (!a.sim_s || a.sim_s[jl] == sg) && a.tag_s[jl] == pt;
                            }
                        } else {
                            const int cx = __shfl_sync(kFull, tx, t), cy = __shfl_sync(kFull, tyy, t),
                                      cz = __shfl_sync(kFull, tz, t);
                            if (ok) {
                                q = a.pos_h_s[jl];
                                ok = (!a.sim_s || a.sim_s[jl] == sg) &&
                                     level_of(q.w, g.log2_L0, g.n_levels) == l &&
                                     cell_of(q.x, g.x0, inv_c) == cx && cell_of(q.y, g.y0, inv_c) == cy &&
                                     cell_of(q.z, g.z0, inv_c) == cz;
                            }
                        }
                        const unsigned okm = __ballot_sync(kFull, ok);
                        const int nok = __popc(okm);
                        __syncwarp();   // the previous batch has been read
                        if (ok) {
                            // coordinates negated: p + (-q) rounds as p - q
                            const int slot = __popc(okm & ((1u << lane) - 1u));
                            float *d = sq + 8 * (slot >> 1) + (slot & 1);
                            d[0] = -q.x;
                            d[2] = -q.y;
                            d[4] = -q.z;
                            d[6] = q.w;
                            sj[slot] = jl;
                        }
                        if ((nok & 1) && lane == 0) {
                            // an odd batch gets a padding column that fails
                            // every test (h = NaN)
                            float *d = sq + 8 * (nok >> 1) + 1;
                            d[0] = 0.0f;
                            d[2] = 0.0f;
                            d[4] = 0.0f;
                            d[6] = __uint_as_float(0x7fc00000u);
                        }
                        __syncwarp();
                        // the predicate over the batch first, two candidates
                        // per packed FP32x2 operation (each element rounded
                        // as the scalar form is), collecting a bit per
                        // accepted candidate; then the appends, in candidate
                        // order, with no branch per candidate
                        unsigned acc = 0u;
                        for (int u = 0; u < nok; u += 2) {
                            const float4 A = *reinterpret_cast<const float4 *>(sq + 4 * u);
                            const float4 B = *reinterpret_cast<const float4 *>(sq + 4 * u + 4);
                            const float2 qx2 = make_float2(A.x, A.y), qy2 = make_float2(A.z, A.w);
                            const float2 qz2 = make_float2(B.x, B.y), qh2 = make_float2(B.z, B.w);
                            const float2 dx = __fadd2_rn(px2, qx2);
                            const float2 dy = __fadd2_rn(py2, qy2);
                            const float2 dz = __fadd2_rn(pz2, qz2);
                            const float2 r2 = __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)),
                                                         __fmul2_rn(dz, dz));
                            const float2 sh = __fadd2_rn(ph2, qh2);
                            const float2 s2 = __fmul2_rn(sh, sh);
                            if (r2.x < s2.x) acc |= 1u << u;
                            if (r2.y < s2.y) acc |= 2u << u;
                        }
                        while (acc) {
                            const int u = __ffs(acc) - 1;
                            acc &= acc - 1u;
                            const int jt = sj[u];
                            if (jt != i) nb_accept<MODE>(a, i, jt, l > lg, base, cnt, sstage, lane);
                        }
                    }
                }
            }
        }
    }
    if (MODE == NB_STAGE) {
        // the staged entries of the warp's rows, row by row, as coalesced
        // stores into the global staging rows
        __syncwarp();
        const int mine = act ? min(cnt, kStageSmem) : 0;
        for (int rr = 0; rr < 32; ++rr) {
            const int cr = __shfl_sync(kFull, mine, rr);
            const int ir = __shfl_sync(kFull, i, rr);
            if (lane < cr) a.stage[(long long)ir * a.stage_k + lane] = sstage[lane * kStageStride + rr];
            if (lane + 32 < cr)
                a.stage[(long long)ir * a.stage_k + lane + 32] = sstage[(lane + 32) * kStageStride + rr];
        }
    }
    if (act) {
        if (!FILL) a.own[i] = cnt;
        if (MODE == NB_STAGE && cnt > a.stage_k) a.list[atomicAdd(a.list_count, 1)] = i;
    }
}

// Second half of the single-search build: copy each staged row into its CSR
// place and append the row to the reverse part of every coarser partner
// (rows on the overflow list are filled by NB_FILL_LISTED instead).
// kCopyLanes lanes per row take its entries in turn, so a warp moves several
// rows at once with coalesced reads and writes; the search marked the
// coarser partners with the top bit of the staged index.
constexpr int kCopyThreads = 256;
constexpr int kCopyLanes = 8;
// entries a lane takes per round: their loads, the partners' row starts and
// the cursor atomics of the reverse entries are issued together, so that
// their round trips overlap instead of following one another
constexpr int kCopyUnroll = 4;   // 1 and 8 measured slower
__global__ void __launch_bounds__(kCopyThreads) nb_copy_kernel(NbArgs a) {
    const long long i = ((long long)blockIdx.x * kCopyThreads + threadIdx.x) / kCopyLanes;
    const int sl = threadIdx.x % kCopyLanes;
    if (i >= a.n) return;
    const int cnt = a.own[i];
    if (cnt > a.stage_k) return;
    const long long base = a.nb_start[i];
    const int *row = a.stage + i * a.stage_k;
    for (int c0 = sl; c0 < cnt; c0 += kCopyLanes * kCopyUnroll) {
        int v[kCopyUnroll];
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u) {
            const int c = c0 + u * kCopyLanes;
            v[u] = c < cnt ? row[c] : 0;
        }
        long long at[kCopyUnroll];
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u) {
            const int c = c0 + u * kCopyLanes;
            const int j = v[u] & 0x7fffffff;
            if (c < cnt) {
                const long long w = base + c;
                if (w < a.capacity) a.nb_idx[w] = j;
                else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
            }
            // a coarser partner: i goes to the reverse part of row j
            at[u] = (c < cnt && v[u] < 0) ? (long long)a.nb_start[j] + a.own[j] : -1;
        }
        int pos[kCopyUnroll];
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u)
            pos[u] = at[u] >= 0 ? atomicAdd(&a.rev[v[u] & 0x7fffffff], 1) : 0;
#pragma unroll
        for (int u = 0; u < kCopyUnroll; ++u) {
            if (at[u] < 0) continue;
            const long long wr = at[u] + pos[u];
            if (wr < a.capacity) a.nb_idx[wr] = (int)i;
            else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
        }
    }
}

__global__ void row_len_kernel(const int *__restrict__ own, const int *__restrict__ rev, int n,
                               int *__restrict__ len) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) len[i] = own[i] + rev[i];
}

int launch_nb_count(const NbArgs &a, cudaStream_t st) {
    if (a.n > 0) {
        if (a.stage) nb_kernel<NB_STAGE><<<(a.n + 127) / 128, 128, 0, st>>>(a);
        else nb_kernel<NB_COUNT><<<(a.n + 127) / 128, 128, 0, st>>>(a);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_nb_fill(const NbArgs &a, cudaStream_t st) {
    if (a.n > 0) {
        if (a.stage) {
            nb_copy_kernel<<<(unsigned)(((long long)a.n * kCopyLanes + kCopyThreads - 1) / kCopyThreads),
                             kCopyThreads, 0, st>>>(a);
            nb_kernel<NB_FILL_LISTED><<<(a.n + 127) / 128, 128, 0, st>>>(a);
            note_launch(2);
        } else {
            nb_kernel<NB_FILL><<<(a.n + 127) / 128, 128, 0, st>>>(a);
            note_launch();
        }
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_row_len(const int *own, const int *rev, int n, int *row_len, cudaStream_t st) {
    if (n > 0) {
        row_len_kernel<<<(n + 255) / 256, 256, 0, st>>>(own, rev, n, row_len);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

}  // namespace sphgb

