// hydro.cu -- the SPH sums of the paper: density DC (Eq. 7 with the cubic
// spline of Eq. 8) and the hydrodynamic force HFC (Eqs. 10-11 with the
// pressure kernel of Eq. 9 and Monaghan's viscosity, Sect. 2.2).
//
// Both run in sorted (bucket) order over the CSR neighbour lists: G lanes
// per row, FP32 arithmetic (the pair terms use the hardware reciprocal square
// root and the fast 2-ulp division; the sums are Kahan-compensated), results
// scattered back to the caller's order through perm.  The working set of a row's
// neighbours (16-48 bytes each) is read through L1/L2; the lists themselves
// stream from HBM.
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

constexpr float kInvPi = 0.318309886183790671538f;

// Cubic spline of Eq. 8 without its 1/(pi h^3) factor.
__device__ __forceinline__ float spline_shape(float xi) {
    if (xi <= 1.0f) return fmaf(xi * xi, fmaf(0.75f, xi, -1.5f), 1.0f);
    float t = 2.0f - xi;
    return xi < 2.0f ? 0.25f * t * t * t : 0.0f;
}

// |dr| from |dr|^2 with the hardware reciprocal square root (2 ulp); 0 at 0.
__device__ __forceinline__ float pair_dist(float r2) {
    return r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f;
}

// mu_ij of Monaghan's viscosity (after Eq. 11), h_ij dr.dv / (|dr|^2 + eta h_ij^2),
// with the fast division (2 ulp); the force pass and the Eq. 17 pass share it.
__device__ __forceinline__ float visc_mu(float hij, float rv, float r2, float eta) {
    return __fdividef(hij * rv, fmaf(eta * hij, hij, r2));
}

// Lanes of one row's group: G consecutive lanes of a warp (G divides 32).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if (G == 32) return 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
}

// Fixed-shape tree sum over the G lanes of a group (same order every run).
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ float group_min(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(mask, v, o));
    return v;
}

template <int G>
__device__ __forceinline__ float group_max(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o));
    return v;
}

// Time step of Eq. 17 for one gas particle from its neighbour extrema
// (s^min the smallest |r_ij|, c^max the largest c_ij, mu^max the largest
// |mu_ij|) and its total acceleration Q = a_hyd + g and heating E.
__device__ __forceinline__ float cfl_bound(float C, const HydroParams &hp, float s_min, float c_max,
                                           float mu_max, float4 a, float4 g) {
    const float qx = a.x + g.x, qy = a.y + g.y, qz = a.z + g.z;
    const float qn = sqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    const float den = c_max * (1.0f + 1.2f * hp.alpha) + 1.2f * hp.beta * mu_max +
                      sqrtf(s_min * (qn + fabsf(a.w)));
    return C * s_min / den;
}

// Minimum over the warp of a non-negative time step, one atomic per warp
// (non-negative floats order like their bit patterns).
__device__ __forceinline__ void warp_dt_min(float dt, unsigned *dt_min_bits) {
    float m = dt;
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m >= 0.0f) atomicMin(dt_min_bits, __float_as_uint(m));
}

// Density of Eq. 7: G lanes share one sorted row; lane q takes neighbours
// q, q + G, ... with its own compensated sum; the group adds the partials.
template <int G>
__global__ void __launch_bounds__(128)
density_kernel(const float4 *__restrict__ pos_h_s, const float *__restrict__ mass_s,
               const int *__restrict__ perm, const int *__restrict__ nb_start,
               const int *__restrict__ nb_idx, int cap, int n, float sigma,
               float *__restrict__ rho_s, float *__restrict__ rho_out,
               float *__restrict__ h_next_out, const int *__restrict__ mixed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / G, q = t % G;
    if (i >= n) return;   // whole groups leave together (G divides the block)
    const unsigned mask = group_mask<G>();
    const float4 p = pos_h_s[i];
    const float mi = mass_s[i];
    const float hi = p.w;
    Kahan acc;
    acc.init();
    if (q == 0) {
        float ih = 1.0f / hi;
        acc.add(mi * (ih * ih * ih) * kInvPi);   // self term m_i W(0, h_i)
    }
    // rows are clipped to the list capacity (an overflowed build is flagged)
    const int e = min(nb_start[i + 1], cap), b = min(nb_start[i], e);
    // all gas masses equal (*mixed == 0): m_j = m_i, one gather per pair
    // fewer; the arithmetic is the same, so are the results
    auto row = [&](auto same) {
#pragma unroll 4
        for (int k = b + q; k < e; k += G) {
            const int j = nb_idx[k];
            if ((unsigned)j >= (unsigned)n) continue;   // only after a flagged overflow
            const float4 o = pos_h_s[j];
            const float mj = decltype(same)::value ? mi : mass_s[j];
            const float dx = p.x - o.x, dy = p.y - o.y, dz = p.z - o.z;
            const float r = pair_dist(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            const float ih = __fdividef(1.0f, 0.5f * (hi + o.w));
            acc.add(mj * (ih * ih * ih) * kInvPi * spline_shape(r * ih));
        }
    };
    if (*mixed == 0) row(std::true_type{});
    else row(std::false_type{});
    const float rho = group_sum<G>(acc.s - acc.c, mask);
    if (q == 0) {
        const int oi = perm[i];
        rho_s[i] = rho;
        rho_out[oi] = rho;
        h_next_out[oi] = sigma * cbrtf(mi / rho);
    }
}

// Flag *mixed (zeroed before the launch) when some mass differs from
// mass[0] (bitwise; a NaN mass counts as different): one atomic per warp.
__device__ __forceinline__ void flag_mixed_mass(bool differs, int *mixed) {
    if (__ballot_sync(0xffffffffu, differs) && (threadIdx.x & 31) == 0) atomicOr(mixed, 1);
}

__global__ void gather_mass_kernel(const float *__restrict__ mass, const int *__restrict__ perm,
                                   int n, float *__restrict__ mass_s, int *__restrict__ mixed) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool differs = false;
    if (j < n) {
        const float m = mass[perm[j]];
        mass_s[j] = m;
        differs = !(m == mass[0]);
    }
    flag_mixed_mass(differs, mixed);
}

// Sorted working copies for HFC: vel_s = (vx, vy, vz, e); aux_s = (m, rho,
// P = p / rho^2 = (gamma - 1) e / rho, c = sqrt(gamma (gamma - 1) e), 0 if e < 0).
__global__ void hydro_prep_kernel(const float4 *__restrict__ vel_e, const float *__restrict__ rho,
                                  const float *__restrict__ mass, const int *__restrict__ perm,
                                  int n, HydroParams hp, float4 *__restrict__ vel_s,
                                  float4 *__restrict__ aux_s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int o = perm[j];
    const float4 v = vel_e[o];
    const float r = rho[o];
    const float gm1 = hp.gamma - 1.0f;
    const float P = gm1 * v.w / r;
    const float c = v.w >= 0.0f ? sqrtf(hp.gamma * gm1 * v.w) : 0.0f;
    vel_s[j] = v;
    aux_s[j] = make_float4(mass[o], r, P, c);
}

// Hydrodynamic acceleration and heating of Eqs. 10-11, G lanes per row.
// CFL: the same pass also takes the neighbour extrema of Eq. 17 and, once the
// row's acceleration is summed, writes the particle's time step (dt_out,
// optional) and lowers *dt_min_bits to the smallest one; grav is the gravity
// at the same positions.
template <int G, bool CFL>
__global__ void __launch_bounds__(128)
forces_kernel(const float4 *__restrict__ pos_h_s, const float4 *__restrict__ vel_s,
              const float4 *__restrict__ aux_s, const int *__restrict__ perm,
              const int *__restrict__ nb_start, const int *__restrict__ nb_idx, int cap, int n,
              HydroParams hp, float4 *__restrict__ acc_out, const float4 *__restrict__ grav,
              float C, float *__restrict__ dt_out, unsigned *__restrict__ dt_min_bits) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / G, q = t % G;
    const bool valid = i < n;
    if (!CFL && !valid) return;   // with CFL every lane takes part in the warp minimum
    const unsigned mask = group_mask<G>();
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p, ai = p;
    int b = 0, e = 0;
    if (valid) {
        p = pos_h_s[i];
        v = vel_s[i];
        ai = aux_s[i];
        // rows are clipped to the list capacity (an overflowed build is flagged)
        e = min(nb_start[i + 1], cap);
        b = min(nb_start[i], e);
    }
    // dW_p/dxi = -(45 / (64 pi)) h^-3 (2 - xi)^2  (derivative of Eq. 9)
    const float kdw = -45.0f / 64.0f * kInvPi;
    Kahan ax, ay, az, de;
    ax.init(); ay.init(); az.init(); de.init();
    float s2_min = __int_as_float(0x7f800000), c_max = 0.0f, mu_max = 0.0f;
#pragma unroll 4
    for (int k = b + q; k < e; k += G) {
        const int j = nb_idx[k];
        if ((unsigned)j >= (unsigned)n) continue;   // only after a flagged overflow
        const float4 o = pos_h_s[j];
        const float4 w = vel_s[j];
        const float4 aj = aux_s[j];
        const float dx = p.x - o.x, dy = p.y - o.y, dz = p.z - o.z;
        const float dvx = v.x - w.x, dvy = v.y - w.y, dvz = v.z - w.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
        const float r = r2 * rinv;
        const float hij = 0.5f * (p.w + o.w);
        const float ih = __fdividef(1.0f, hij);
        const float tt = fmaxf(2.0f - r * ih, 0.0f);
        // grad W_p = (dW_p/dxi) (dr / r) / h_ij = f * dr; zero at r = 0
        const float f = kdw * (ih * ih * ih) * tt * tt * ih * rinv;
        const float rv = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
        const float c_ij = 0.5f * (ai.w + aj.w);
        float nu = 0.0f;
        if (rv < 0.0f) {
            const float mu = visc_mu(hij, rv, r2, hp.eta);
            const float rho_ij = 0.5f * (ai.y + aj.y);
            nu = __fdividef(mu * fmaf(hp.beta, mu, -hp.alpha * c_ij), rho_ij);
            if (CFL) mu_max = fmaxf(mu_max, -mu);
        }
        if (CFL) {
            s2_min = fminf(s2_min, r2);
            c_max = fmaxf(c_max, c_ij);
        }
        const float Pi = ai.z + aj.z + nu;
        const float g = aj.x * Pi * f;   // m_j Pi_ij f
        ax.add(-g * dx);
        ay.add(-g * dy);
        az.add(-g * dz);
        de.add(0.5f * g * fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz)));
    }
    const float sx = group_sum<G>(ax.s - ax.c, mask);
    const float sy = group_sum<G>(ay.s - ay.c, mask);
    const float sz = group_sum<G>(az.s - az.c, mask);
    const float se = group_sum<G>(de.s - de.c, mask);
    if (!CFL) {
        if (q == 0) acc_out[perm[i]] = make_float4(sx, sy, sz, se);
        return;
    }
    s2_min = group_min<G>(s2_min, mask);
    c_max = group_max<G>(c_max, mask);
    mu_max = group_max<G>(mu_max, mask);
    float dt = __int_as_float(0x7f800000);   // +inf: no bound
    if (valid && q == 0) {
        const int oi = perm[i];
        const float4 a = make_float4(sx, sy, sz, se);
        acc_out[oi] = a;
        if (e > b) dt = cfl_bound(C, hp, sqrtf(s2_min), c_max, mu_max, a, grav[oi]);
        if (dt_out) dt_out[oi] = dt;
    }
    warp_dt_min(dt, dt_min_bits);
}

// Time step of Eq. 17 per gas particle, and its minimum.  mu^max is the
// largest |mu_ij| over the neighbours (mu_ij <= 0 as defined), c^max the
// largest c_ij, s^min the smallest |r_ij|; Q_i = |a_hyd + g|, E_i = |de/dt|.
__global__ void __launch_bounds__(128)
cfl_kernel(const float4 *__restrict__ pos_h_s, const float4 *__restrict__ vel_s,
           const float4 *__restrict__ aux_s, const int *__restrict__ perm,
           const int *__restrict__ nb_start, const int *__restrict__ nb_idx, int cap, int n,
           HydroParams hp, float C, const float4 *__restrict__ acc_hyd,
           const float4 *__restrict__ grav, float *__restrict__ dt_out,
           unsigned *__restrict__ dt_min_bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float dt = __int_as_float(0x7f800000);   // +inf: no bound
    if (i < n) {
        const float4 p = pos_h_s[i];
        const float4 v = vel_s[i];
        const float ci = aux_s[i].w;
        float s_min = dt, c_max = 0.0f, mu_max = 0.0f;
        const int e = min(nb_start[i + 1], cap), b = min(nb_start[i], e);
    #pragma unroll 4
    for (int k = b; k < e; ++k) {
            const int j = nb_idx[k];
            if ((unsigned)j >= (unsigned)n) continue;
            const float4 q = pos_h_s[j];
            const float4 w = vel_s[j];
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            s_min = fminf(s_min, sqrtf(r2));
            c_max = fmaxf(c_max, 0.5f * (ci + aux_s[j].w));
            const float rv = fmaf(dx, v.x - w.x, fmaf(dy, v.y - w.y, dz * (v.z - w.z)));
            if (rv < 0.0f)
                mu_max = fmaxf(mu_max, -visc_mu(0.5f * (p.w + q.w), rv, r2, hp.eta));
        }
        const int oi = perm[i];
        if (e > b) dt = cfl_bound(C, hp, s_min, c_max, mu_max, acc_hyd[oi], grav[oi]);
        if (dt_out) dt_out[oi] = dt;
    }
    // block minimum, then one atomic per block (dt >= 0: the bits order like the values)
    __shared__ float s_min_dt[4];
    float m = dt;
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_min_dt[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fminf(m, s_min_dt[w]);
        if (m >= 0.0f) atomicMin(dt_min_bits, __float_as_uint(m));
    }
}

static unsigned host_float_bits(float x) {
    unsigned u;
    std::memcpy(&u, &x, sizeof(u));
    return u;
}

__global__ void fill_u32_kernel(unsigned *p, unsigned v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

int launch_cfl(const float4 *pos_h_s, const float4 *vel_s, const float4 *aux_s, const int *perm,
               const int *nb_start, const int *nb_idx, int cap, int n, HydroParams hp, float C,
               const float4 *acc_hyd, const float4 *grav, float *dt_out, float *dt_min,
               float dt_cap, cudaStream_t st) {
    fill_u32_kernel<<<1, 32, 0, st>>>(reinterpret_cast<unsigned *>(dt_min), host_float_bits(dt_cap));
    note_launch();
    if (n > 0) {
        cfl_kernel<<<(n + 127) / 128, 128, 0, st>>>(pos_h_s, vel_s, aux_s, perm, nb_start, nb_idx,
                                                    cap, n, hp, C, acc_hyd, grav, dt_out,
                                                    reinterpret_cast<unsigned *>(dt_min));
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

static unsigned grid_for(long long threads) { return (unsigned)((threads + 127) / 128); }

int launch_density(const float4 *pos_h_s, const float *mass, const int *perm, const int *nb_start,
                   const int *nb_idx, int cap, int n, float sigma, int lanes, float *rho_s,
                   float *rho_out, float *h_next_out, float *mass_s, int *mixed, cudaStream_t st) {
    if (n > 0) {
        SPH_CUDA_TRY(cudaMemsetAsync(mixed, 0, sizeof(int), st));
        gather_mass_kernel<<<(n + 255) / 256, 256, 0, st>>>(mass, perm, n, mass_s, mixed);
        const long long T = (long long)n * lanes;
        switch (lanes) {
            case 1: density_kernel<1><<<grid_for(T), 128, 0, st>>>(pos_h_s, mass_s, perm, nb_start, nb_idx, cap, n, sigma, rho_s, rho_out, h_next_out, mixed); break;
            case 2: density_kernel<2><<<grid_for(T), 128, 0, st>>>(pos_h_s, mass_s, perm, nb_start, nb_idx, cap, n, sigma, rho_s, rho_out, h_next_out, mixed); break;
            case 8: density_kernel<8><<<grid_for(T), 128, 0, st>>>(pos_h_s, mass_s, perm, nb_start, nb_idx, cap, n, sigma, rho_s, rho_out, h_next_out, mixed); break;
            default: density_kernel<4><<<grid_for(T), 128, 0, st>>>(pos_h_s, mass_s, perm, nb_start, nb_idx, cap, n, sigma, rho_s, rho_out, h_next_out, mixed); break;
        }
        note_launch(2);
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_hydro_prep(const float4 *vel_e, const float *rho, const float *mass, const int *perm,
                      int n, HydroParams hp, float4 *vel_s, float4 *aux_s, cudaStream_t st) {
    if (n > 0) {
        hydro_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(vel_e, rho, mass, perm, n, hp, vel_s,
                                                           aux_s);
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

int launch_forces(const float4 *pos_h_s, const float4 *vel_s, const float4 *aux_s,
                  const int *perm, const int *nb_start, const int *nb_idx, int cap, int n,
                  HydroParams hp, int lanes, float4 *acc_out, cudaStream_t st,
                  const float4 *grav, float C, float *dt_out, float *dt_min, float dt_cap) {
    const bool cfl = dt_min != nullptr;
    unsigned *bits = reinterpret_cast<unsigned *>(dt_min);
    if (cfl) {
        fill_u32_kernel<<<1, 32, 0, st>>>(bits, host_float_bits(dt_cap));
        note_launch();
    }
    if (n > 0) {
        const long long T = (long long)n * lanes;
#define SPHGB_FORCES(G)                                                                         \
    if (cfl)                                                                                    \
        forces_kernel<G, true><<<grid_for(T), 128, 0, st>>>(pos_h_s, vel_s, aux_s, perm, nb_start, \
                                                            nb_idx, cap, n, hp, acc_out, grav, C, \
                                                            dt_out, bits);                      \
    else                                                                                        \
        forces_kernel<G, false><<<grid_for(T), 128, 0, st>>>(pos_h_s, vel_s, aux_s, perm, nb_start, \
                                                             nb_idx, cap, n, hp, acc_out, nullptr, \
                                                             0.0f, nullptr, nullptr)
        switch (lanes) {
            case 1: SPHGB_FORCES(1); break;
            case 2: SPHGB_FORCES(2); break;
            case 8: SPHGB_FORCES(8); break;
            default: SPHGB_FORCES(4); break;
        }
#undef SPHGB_FORCES
        note_launch();
    }
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

}  // namespace sphgb
