// integrate.cu -- the system update SU of the paper: the leapfrog
// predictor-corrector of Eqs. 12-16 on FP64 state, fed by FP32 forces, and
// the FP32 working copies the force stages read.  Also the FP64 energy and
// momentum reductions.
//
// FP64 operations are written one rounded operation at a time (no
// contraction into FMA) so the update is the textbook expression evaluated
// left to right.
#include "common.cuh"
#include "kernels.cuh"

namespace sphgb {

__global__ void integrate_kernel(int phase, double dt_arg, const float *__restrict__ d_dt, int n,
                                 int n_gas, double *__restrict__ r,
                                 double *__restrict__ v, double *__restrict__ e,
                                 double *__restrict__ v_save, double *__restrict__ e_save,
                                 const float4 *__restrict__ acc_hyd,
                                 const float4 *__restrict__ grav, const float *__restrict__ mass,
                                 const float *__restrict__ h, float4 *__restrict__ pos_m,
                                 float4 *__restrict__ pos_h, float4 *__restrict__ vel_e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool gas = i < n_gas;
    // the step size comes from the host, or from device memory (a time step
    // chosen on the device by the CFL condition, Eq. 17)
    const double dt = d_dt ? (double)*d_dt : dt_arg;
    const double half_dt = __dmul_rn(0.5, dt);
    if (phase != SPH_EMIT) {
        const float4 g = grav[i];
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gas) a = acc_hyd[i];
        const double qv[3] = {(double)g.x, (double)g.y, (double)g.z};
        const double av[3] = {(double)a.x, (double)a.y, (double)a.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const size_t k = (size_t)d * n + i;
            const double q = gas ? __dadd_rn(qv[d], av[d]) : qv[d];
            if (phase == SPH_PREDICT) {
                const double v0 = v[k];
                const double vt = __dadd_rn(v0, __dmul_rn(dt, q));
                v_save[k] = v0;
                v[k] = vt;
                r[k] = __dadd_rn(r[k], __dmul_rn(half_dt, __dadd_rn(vt, v0)));
            } else {
                v[k] = __dadd_rn(__dmul_rn(0.5, __dadd_rn(v_save[k], v[k])), __dmul_rn(half_dt, q));
            }
        }
        if (gas) {
            const double E = (double)a.w;
            if (phase == SPH_PREDICT) {
                const double e0 = e[i];
                e_save[i] = e0;
                e[i] = __dadd_rn(e0, __dmul_rn(dt, E));
            } else {
                e[i] = __dadd_rn(__dmul_rn(0.5, __dadd_rn(e_save[i], e[i])), __dmul_rn(half_dt, E));
            }
        }
    }
    const float x = (float)r[i], y = (float)r[(size_t)n + i], z = (float)r[2 * (size_t)n + i];
    if (pos_m) pos_m[i] = make_float4(x, y, z, mass[i]);
    if (gas) {
        if (pos_h) pos_h[i] = make_float4(x, y, z, h[i]);
        if (vel_e)
            vel_e[i] = make_float4((float)v[i], (float)v[(size_t)n + i], (float)v[2 * (size_t)n + i],
                                   (float)e[i]);
    }
}

// One block, fixed order: thread t accumulates particles t, t + T, ...; then
// a fixed-shape tree in shared memory.
constexpr int DIAG_THREADS = 512;

__global__ void __launch_bounds__(DIAG_THREADS)
diagnostics_kernel(int n, int n_gas, const double *__restrict__ v, const double *__restrict__ e,
                   const float *__restrict__ mass, const float4 *__restrict__ grav,
                   double *__restrict__ out) {
    __shared__ double s[7][DIAG_THREADS];
    double kin = 0, th = 0, pot = 0, px = 0, py = 0, pz = 0, mt = 0;
    for (int i = threadIdx.x; i < n; i += DIAG_THREADS) {
        const double m = mass[i];
        const double vx = v[i], vy = v[(size_t)n + i], vz = v[2 * (size_t)n + i];
        kin += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (i < n_gas) th += m * e[i];
        if (grav) pot += 0.5 * m * (double)grav[i].w;
        px += m * vx;
        py += m * vy;
        pz += m * vz;
        mt += m;
    }
    const double vals[7] = {kin, th, pot, px, py, pz, mt};
    for (int q = 0; q < 7; ++q) s[q][threadIdx.x] = vals[q];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 7; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 7) out[threadIdx.x] = s[threadIdx.x][0];
    if (threadIdx.x == 7) out[7] = 0.0;
}

// integrate_step with the step size optionally read from device memory
// (d_dt != NULL: one float, e.g. written by the CFL epilogue of the forces).
int integrate_launch(int phase, double dt, const float *d_dt, int n, int n_gas, double *d_r,
                     double *d_v, double *d_e, double *d_v_save, double *d_e_save,
                     const float *d_acc_hyd, const float *d_grav, const float *d_mass,
                     const float *d_h, float *d_pos_m, float *d_pos_h, float *d_vel_e,
                     sph_stream_t stream) {
    if (phase < SPH_PREDICT || phase > SPH_EMIT || n < 0 || n_gas < 0 || n_gas > n)
        return SPH_ERR_INVALID_ARG;
    if (n == 0) return SPH_OK;
    if (!d_r || !d_v) return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && !d_e) return SPH_ERR_INVALID_ARG;
    if (phase != SPH_EMIT) {
        if (!d_v_save || !d_grav || !(dt == dt)) return SPH_ERR_INVALID_ARG;
        if (n_gas > 0 && (!d_e_save || !d_acc_hyd)) return SPH_ERR_INVALID_ARG;
    }
    if (d_pos_m && !d_mass) return SPH_ERR_INVALID_ARG;
    if (n_gas > 0 && d_pos_h && !d_h) return SPH_ERR_INVALID_ARG;
    integrate_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        phase, dt, d_dt, n, n_gas, d_r, d_v, d_e, d_v_save, d_e_save,
        reinterpret_cast<const float4 *>(d_acc_hyd), reinterpret_cast<const float4 *>(d_grav),
        d_mass, d_h, reinterpret_cast<float4 *>(d_pos_m), reinterpret_cast<float4 *>(d_pos_h),
        reinterpret_cast<float4 *>(d_vel_e));
    note_launch();
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}

}  // namespace sphgb

using namespace sphgb;

extern "C" int integrate_step(int32_t phase, double dt, int32_t n, int32_t n_gas, double *d_r,
                              double *d_v, double *d_e, double *d_v_save, double *d_e_save,
                              const float *d_acc_hyd, const float *d_grav, const float *d_mass,
                              const float *d_h, float *d_pos_m, float *d_pos_h, float *d_vel_e,
                              sph_stream_t stream) {
    return integrate_launch(phase, dt, nullptr, n, n_gas, d_r, d_v, d_e, d_v_save, d_e_save,
                            d_acc_hyd, d_grav, d_mass, d_h, d_pos_m, d_pos_h, d_vel_e, stream);
}

extern "C" int sph_diagnostics(const SphState *st, double *d_out, sph_stream_t stream) {
    if (!st || !d_out || st->n < 0 || st->n_gas < 0 || st->n_gas > st->n) return SPH_ERR_INVALID_ARG;
    if (st->n > 0 && (!st->v || !st->mass || (st->n_gas > 0 && !st->e))) return SPH_ERR_INVALID_ARG;
    diagnostics_kernel<<<1, DIAG_THREADS, 0, (cudaStream_t)stream>>>(
        st->n, st->n_gas, st->v, st->e, st->mass, reinterpret_cast<const float4 *>(st->grav), d_out);
    note_launch();
    SPH_LAUNCH_CHECK();
    return SPH_OK;
}
