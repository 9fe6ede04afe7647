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

// Distance from coordinate x to cell c of size csz (origin x0), less a
// rounding margin m; the end cells also hold everything clamped into them,
// so they are open on their outer side.
__device__ __forceinline__ float cell_gap(float x, int c, float csz, float x0, float m) {
    const float lo = fmaf((float)c, csz, x0);
    const float below = c > 0 ? lo - x : -1.0f;
    const float above = c < kCellMax ? x - (lo + csz) : -1.0f;
    return fmaxf(0.0f, fmaxf(below, above) - m);
}

// MODE: NB_COUNT counts own entries (and reverse entries of the coarser
// partners); NB_FILL writes own and reverse entries into their CSR places;
// NB_STAGE counts like NB_COUNT and also writes the first stage_k own
// entries of the row to stage[i * stage_k + c] (rows with more are queued on
// the overflow list); NB_FILL_LISTED runs NB_FILL for the queued rows only.
enum { NB_COUNT = 0, NB_FILL = 1, NB_STAGE = 2, NB_FILL_LISTED = 3 };

template <int MODE>
__global__ void __launch_bounds__(128, 8) nb_kernel(NbArgs a) {
    constexpr bool FILL = MODE == NB_FILL || MODE == NB_FILL_LISTED;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (MODE == NB_FILL_LISTED) {
        if (i >= *a.list_count) return;
        i = a.list[i];
    }
    if (i >= a.n) return;
    const GridDev g = *a.grid;
    const float4 p = a.pos_h_s[i];
    const int li = level_of(p.w, g.log2_L0, g.n_levels);
    const int si = a.sim_s ? a.sim_s[i] : 0;
    int cnt = 0;
    long long base = 0;
    if (FILL) base = a.nb_start[i];
    for (int l = li; l < g.n_levels; ++l) {
        if (a.lvl_count[l] == 0) continue;
        const float R = __fadd_rn(p.w, __uint_as_float(a.lvl_hmax[l]));
        if (!(R >= 0.0f)) continue;
        const float inv_c = pow2f(-g.log2_L0 - l);
        int lx, hx, ly, hy, lz, hz;
        search_box(p.x, R, g.x0, inv_c, lx, hx);
        search_box(p.y, R, g.y0, inv_c, ly, hy);
        search_box(p.z, R, g.z0, inv_c, lz, hz);
        long long ncell = (long long)(hx - lx + 1) * (hy - ly + 1) * (hz - lz + 1);
        if (ncell > (1ll << 24)) {
            set_flag(a.flags, SPH_FLAG_SEARCH_WIDE);
            continue;
        }
        if (a.occ && l > li) {
            // skip the level when none of the super-cells the box touches holds
            // a particle of it (the particle's own level is always occupied)
            bool any = false;
            for (int sz = lz >> kSuperShift; sz <= (hz >> kSuperShift) && !any; ++sz)
                for (int sy = ly >> kSuperShift; sy <= (hy >> kSuperShift) && !any; ++sy)
                    for (int sx = lx >> kSuperShift; sx <= (hx >> kSuperShift) && !any; ++sx) {
                        const unsigned bit = super_bit(sx, sy, sz, l + kMaxLevels * si, a.log2_B);
                        any = (a.occ[bit >> 5] >> (bit & 31)) & 1u;
                    }
            if (!any) continue;
        }
        // per-axis distance from the particle to each probed cell, widened by a
        // margin that covers the rounding of the binning (a skipped cell cannot
        // hold a particle within h_i + hmax of the cell's bucket)
        const float csz = pow2f(g.log2_L0 + l);
        // |coordinate| of anything in the box is at most |x0| + (hi + 1) csz
        const float mx = 9.5367431640625e-07f * (fabsf(p.x) + 2.0f * fabsf(g.x0) + (float)(hx + 2) * csz) + 1e-30f;
        const float my = 9.5367431640625e-07f * (fabsf(p.y) + 2.0f * fabsf(g.y0) + (float)(hy + 2) * csz) + 1e-30f;
        const float mz = 9.5367431640625e-07f * (fabsf(p.z) + 2.0f * fabsf(g.z0) + (float)(hz + 2) * csz) + 1e-30f;
        // bucket_of(cx, cy, cz, ...) with the interleave built per axis: z
        // once per plane, y once per row, x stepped by a dilated increment
        const unsigned salt = (unsigned)(l + kMaxLevels * si) * (unsigned)kLevelSalt;
        const unsigned kmask = (1u << g.log2_M) - 1u;
        const unsigned dlx = spread3_lo((unsigned)lx);
        for (int cz = lz; cz <= hz; ++cz) {
            const float dz = cell_gap(p.z, cz, csz, g.z0, mz);
            const unsigned iz = spread3_lo((unsigned)cz) << 2;
            for (int cy = ly; cy <= hy; ++cy) {
                const float dy = cell_gap(p.y, cy, csz, g.y0, my);
                const unsigned iyz = iz | (spread3_lo((unsigned)cy) << 1);
                unsigned ix = dlx;
                for (int cx = lx; cx <= hx; ++cx, ix = spread3_next(ix)) {
                    const float dx = cell_gap(p.x, cx, csz, g.x0, mx);
                    const int k = (int)(((ix | iyz) + salt) & kmask);
                    const int s = a.cell_start[k], e = a.cell_start[k + 1];
                    if (s == e) continue;
                    {
                        const float reach = p.w + __uint_as_float(a.hmax_cell[k]);
                        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (d2 > reach * reach * (1.0f + 3.0517578125e-05f)) continue;
                    }
                    // candidates four at a time: their loads are issued together
                    for (int j0 = s; j0 < e; j0 += 4) {
                    float4 qb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        qb[u] = j0 + u < e ? a.pos_h_s[j0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = j0 + u;
                        if (j >= e || j == i) continue;
                        const float4 q = qb[u];
                        // the distance test first: most candidates fail it, and
                        // the identity checks (same simulation, level and cell
                        // as the probed one) are only needed for those that pass
                        if (!nb_pred(p, q)) continue;
                        if (a.sim_s && a.sim_s[j] != si) continue;
                        if (level_of(q.w, g.log2_L0, g.n_levels) != l) continue;
                        if (cell_of(q.x, g.x0, inv_c) != cx || cell_of(q.y, g.y0, inv_c) != cy ||
                            cell_of(q.z, g.z0, inv_c) != cz)
                            continue;
                        if (FILL) {
                            long long w = base + cnt;
                            if (w < a.capacity) a.nb_idx[w] = j;
                            else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
                            if (l > li) {
                                int pos = atomicAdd(&a.rev[j], 1);
                                long long wr = (long long)a.nb_start[j] + a.own[j] + pos;
                                if (wr < a.capacity) a.nb_idx[wr] = i;
                                else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
                            }
                        } else {
                            if (MODE == NB_STAGE && cnt < a.stage_k)
                                a.stage[(long long)i * a.stage_k + cnt] = j;
                            if (l > li) atomicAdd(&a.rev[j], 1);
                        }
                        ++cnt;
                    }
                    }
                }
            }
        }
    }
    if (!FILL) a.own[i] = cnt;
    if (MODE == NB_STAGE && cnt > a.stage_k) a.list[atomicAdd(a.list_count, 1)] = i;
}

// Second half of the single-search build: copy each staged row into its CSR
// place and append the row to the reverse part of every coarser partner
// (rows on the overflow list are filled by NB_FILL_LISTED instead).
__global__ void __launch_bounds__(128) nb_copy_kernel(NbArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int cnt = a.own[i];
    if (cnt > a.stage_k) return;
    const GridDev g = *a.grid;
    const int li = level_of(a.pos_h_s[i].w, g.log2_L0, g.n_levels);
    const long long base = a.nb_start[i];
    const int *row = a.stage + (long long)i * a.stage_k;
    for (int c = 0; c < cnt; ++c) {
        const int j = row[c];
        const long long w = base + c;
        if (w < a.capacity) a.nb_idx[w] = j;
        else set_flag(a.flags, SPH_FLAG_NB_OVERFLOW);
        if (level_of(a.pos_h_s[j].w, g.log2_L0, g.n_levels) > li) {
            const int pos = atomicAdd(&a.rev[j], 1);
            const long long wr = (long long)a.nb_start[j] + a.own[j] + pos;
            if (wr < a.capacity) a.nb_idx[wr] = i;
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
            nb_copy_kernel<<<(a.n + 127) / 128, 128, 0, st>>>(a);
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
