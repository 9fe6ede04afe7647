/*
 * sph_oracle.c -- plain, slow FP64 CPU oracle for the self-gravitating SPH
 * right-hand side of Khrapov & Khoperskov, "Smoothed-Particle Hydrodynamics
 * Models: Implementation Features on GPUs" (arXiv:1807.08116).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code, header, table or constant with the CUDA library; neither includes the
 * other.
 *
 * Every function is a direct, brute-force statement of the paper's formulas:
 * O(N^2) loops, no cells, no blocking, no reordering beyond what the
 * definition states.  Arithmetic is FP64 on inputs that are given in FP32 (the
 * working-copy precision), promoted exactly to double.  The only FP32
 * arithmetic is where the result is an integer decision that both sides must
 * take identically: the neighbour-membership predicate and the cell binning.
 * This file must be compiled with -ffp-contract=off so that those FP32
 * expressions are evaluated one rounded operation at a time.
 *
 * Readings of the paper taken here (ambiguities, garbles and silences):
 *  R1 gravity softening: Eq. 4 prints |r_i - r_j + delta|^3, which adds a
 *     scalar to a vector; read as Plummer softening (|dr|^2 + eps^2)^(3/2).
 *  R2 neighbour predicate: j is a neighbour of i (j != i) iff
 *     |r_ij| < h_i + h_j = 2 h_ij, the support of W and W_p (Eqs. 8-9),
 *     evaluated in FP32 as ((dx*dx + dy*dy) + dz*dz) < (h_i + h_j)^2.
 *  R3 dW_p/dxi is the derivative of Eq. 9 as printed; the limit value printed
 *     after Eq. 9 drops the factor (2 - xi)^2 = 4 and is not used.
 *  R4 grad W_p at |dr| = 0 is taken as the zero vector (direction undefined).
 *  R5 sound speed c = sqrt(gamma p / rho) for p >= 0 and 0 for p < 0.
 *  R6 viscosity denominator is |dr|^2 + eta h_ij^2 with eta used as printed.
 *  R7 within one RHS evaluation every stage uses the smoothing length stored
 *     from the previous density evaluation; the density stage returns
 *     h_next = sigma (m / rho)^(1/3) (Sect. 2.2).
 *  R8 gravity is evaluated once per step at r(t + dt) and reused by the next
 *     predictor (Sect. 2.2, after Eq. 16).
 *  R9 order of particles inside one cell after the counting sort: ascending
 *     original index (a stable counting sort).
 *  R10 in the time-step condition of Eq. 17, mu^max is the largest |mu_ij|
 *     over the neighbours (mu_ij <= 0 as defined, so its plain maximum would
 *     always be 0), c^max the largest c_ij and s^min the smallest |r_ij|; a
 *     particle without neighbours sets no bound.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Threads the parallel loops below use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the thread count of the parallel loops (n >= 1; no effect without
 * OpenMP).  Returns the count now in effect. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return oracle_threads();
}

/* ------------------------------------------------------------------------ */
/* Smoothing kernels, Eqs. 8 and 9.                                         */
/* ------------------------------------------------------------------------ */

/* Cubic spline W(xi, h) of Eq. 8, xi = |r_i - r_j| / h. */
double oracle_W(double xi, double h)
{
    double norm = 1.0 / (ORACLE_PI * h * h * h);
    if (xi < 0.0) xi = -xi;
    if (xi <= 1.0) return norm * (1.0 - 1.5 * xi * xi + 0.75 * xi * xi * xi);
    if (xi <= 2.0) { double t = 2.0 - xi; return norm * 0.25 * t * t * t; }
    return 0.0;
}

/* Pressure kernel W_p(xi, h) of Eq. 9. */
double oracle_Wp(double xi, double h)
{
    if (xi < 0.0) xi = -xi;
    if (xi >= 2.0) return 0.0;
    double t = 2.0 - xi;
    return 15.0 / (64.0 * ORACLE_PI * h * h * h) * t * t * t;
}

/* dW_p/dxi: derivative of Eq. 9 with respect to xi (reading R3). */
double oracle_dWp_dxi(double xi, double h)
{
    if (xi < 0.0) xi = -xi;
    if (xi >= 2.0) return 0.0;
    double t = 2.0 - xi;
    return -45.0 / (64.0 * ORACLE_PI * h * h * h) * t * t;
}

/* ------------------------------------------------------------------------ */
/* Neighbour predicate (reading R2), evaluated in FP32.                     */
/* ------------------------------------------------------------------------ */

static int nb_pred(const float *a, const float *b)
{
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    float dx2 = dx * dx;
    float dy2 = dy * dy;
    float dz2 = dz * dz;
    float r2 = dx2 + dy2;
    r2 = r2 + dz2;
    float s = a[3] + b[3];
    float s2 = s * s;
    return r2 < s2;
}

/* Number of neighbours of each listed row (pos_h is [n][4]: x, y, z, h). */
void oracle_neighbor_counts(int n, const float *pos_h, const int *rows,
                            int n_rows, int *counts)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        int c = 0;
        for (int j = 0; j < n; ++j)
            if (j != i && nb_pred(pos_h + 4 * (size_t)i, pos_h + 4 * (size_t)j)) ++c;
        counts[r] = c;
    }
}

/* Neighbour lists of each listed row in ascending j; starts has n_rows + 1
 * entries and must be the exclusive prefix sum of oracle_neighbor_counts. */
void oracle_neighbor_lists(int n, const float *pos_h, const int *rows,
                           int n_rows, const int64_t *starts, int *idx)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        int64_t w = starts[r];
        for (int j = 0; j < n; ++j)
            if (j != i && nb_pred(pos_h + 4 * (size_t)i, pos_h + 4 * (size_t)j)) idx[w++] = j;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid binning of the sorting stage (Sect. 3, kernels SP0..SP4).           */
/* A particle with smoothing length h lives on level l, the smallest l >= 0 */
/* with h <= L0 * 2^l (clamped to n_levels - 1); its integer cell at that  */
/* level is floor((x - x0) / (L0 * 2^l)) per axis, clamped to [0, 2^21-1]; */
/* the bucket ("cell" k of CellSPH) is the 63-bit bit-interleave of the    */
/* three cell coordinates plus l times a 64-bit odd constant, mod M.       */
/* ------------------------------------------------------------------------ */

#define ORACLE_CELL_MAX 2097151

static float pow2f_exact(int e)
{
    /* 2^e as an FP32 value, e in [-126, 127] (normal range). */
    uint32_t bits = (uint32_t)(e + 127) << 23;
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

static int level_of(float h, int log2_L0, int n_levels)
{
    float q = h * pow2f_exact(-log2_L0);
    int l;
    if (!(q > 1.0f)) {
        l = 0;
    } else {
        uint32_t bits;
        memcpy(&bits, &q, 4);
        int e = (int)((bits >> 23) & 0xffu) - 127;
        uint32_t mant = bits & 0x7fffffu;
        l = (mant == 0u) ? e : e + 1;
    }
    if (l > n_levels - 1) l = n_levels - 1;
    return l;
}

static int cell_of(float x, float x0, float inv_c)
{
    float t = x - x0;
    float u = t * inv_c;
    if (!(u > 0.0f)) return 0;
    if (u >= (float)ORACLE_CELL_MAX) return ORACLE_CELL_MAX;
    return (int)u;
}

static uint64_t interleave3(uint32_t cx, uint32_t cy, uint32_t cz)
{
    uint64_t m = 0;
    for (int b = 0; b < 21; ++b) {
        m |= (uint64_t)((cx >> b) & 1u) << (3 * b);
        m |= (uint64_t)((cy >> b) & 1u) << (3 * b + 1);
        m |= (uint64_t)((cz >> b) & 1u) << (3 * b + 2);
    }
    return m;
}

/* grid = {x0, y0, z0} as floats; igrid = {log2_L0, n_levels, log2_M}.
 * Outputs per particle: level, cell coords (3 ints), bucket key. */
void oracle_bin(int n, const float *pos_h, const float *grid, const int *igrid,
                int *level, int *cell, int *key)
{
    int log2_L0 = igrid[0], n_levels = igrid[1], log2_M = igrid[2];
    uint64_t mask = ((uint64_t)1 << log2_M) - 1;
    for (int i = 0; i < n; ++i) {
        const float *p = pos_h + 4 * (size_t)i;
        int l = level_of(p[3], log2_L0, n_levels);
        float inv_c = pow2f_exact(-log2_L0 - l);
        int cx = cell_of(p[0], grid[0], inv_c);
        int cy = cell_of(p[1], grid[1], inv_c);
        int cz = cell_of(p[2], grid[2], inv_c);
        uint64_t m = interleave3((uint32_t)cx, (uint32_t)cy, (uint32_t)cz);
        uint64_t k = (m + (uint64_t)l * 0x9E3779B97F4A7C15ull) & mask;
        level[i] = l;
        cell[3 * (size_t)i + 0] = cx;
        cell[3 * (size_t)i + 1] = cy;
        cell[3 * (size_t)i + 2] = cz;
        key[i] = (int)k;
    }
}

/* Sequential counting sort (the serial analogue that SP2/SP3 parallelise):
 * count[k] = particles in bucket k; cell_start[k] = sum_{k' < k} count[k']
 * (exclusive, M + 1 entries, so the paper's inclusive CellSPH[k].y is
 * cell_start[k + 1]); perm[slot] = original index, stable (reading R9). */
void oracle_counting_sort(int n, const int *key, int M, int *count,
                          int *cell_start, int *perm)
{
    for (int k = 0; k < M; ++k) count[k] = 0;
    for (int i = 0; i < n; ++i) count[key[i]] += 1;
    cell_start[0] = 0;
    for (int k = 0; k < M; ++k) cell_start[k + 1] = cell_start[k] + count[k];
    for (int k = 0; k < M; ++k) count[k] = 0;          /* reuse as cursor */
    for (int i = 0; i < n; ++i) {
        int k = key[i];
        perm[cell_start[k] + count[k]] = i;
        count[k] += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* SPH density, Eq. 7, with h_ij = (h_i + h_j)/2 and the smoothing-length   */
/* rule h = sigma (m / rho)^(1/3) (Sect. 2.2).                              */
/* ------------------------------------------------------------------------ */

void oracle_density(int n, const float *pos_h, const float *mass, double sigma,
                    const int *rows, int n_rows, double *rho, double *h_next)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        const float *pi = pos_h + 4 * (size_t)i;
        double hi = pi[3];
        double s = (double)mass[i] * oracle_W(0.0, hi);   /* j = i term */
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const float *pj = pos_h + 4 * (size_t)j;
            if (!nb_pred(pi, pj)) continue;
            double dx = (double)pi[0] - (double)pj[0];
            double dy = (double)pi[1] - (double)pj[1];
            double dz = (double)pi[2] - (double)pj[2];
            double rr = sqrt(dx * dx + dy * dy + dz * dz);
            double hij = 0.5 * (hi + (double)pj[3]);
            s += (double)mass[j] * oracle_W(rr / hij, hij);
        }
        rho[r] = s;
        h_next[r] = sigma * cbrt((double)mass[i] / s);
    }
}

/* ------------------------------------------------------------------------ */
/* SPH momentum and energy right-hand sides, Eqs. 10 and 11, with the       */
/* symmetric Pi_ij, Monaghan viscosity nu_ij and mu_ij of Sect. 2.2 and the */
/* ideal-gas closure p = (gamma - 1) rho e of Eq. 5.                        */
/* vel_e is [n][4]: vx, vy, vz, e.  par = {gamma, alpha, beta, eta}.        */
/* ------------------------------------------------------------------------ */

void oracle_hydro(int n, const float *pos_h, const float *vel_e,
                  const float *mass, const float *rho, const double *par,
                  const int *rows, int n_rows, double *acc, double *dedt)
{
    double gam = par[0], alpha = par[1], beta = par[2], eta = par[3];
    #pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        const float *pi = pos_h + 4 * (size_t)i;
        const float *vi = vel_e + 4 * (size_t)i;
        double rho_i = rho[i];
        double p_i = (gam - 1.0) * rho_i * (double)vi[3];
        double c_i = p_i >= 0.0 ? sqrt(gam * p_i / rho_i) : 0.0;
        double ax = 0.0, ay = 0.0, az = 0.0, de = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const float *pj = pos_h + 4 * (size_t)j;
            if (!nb_pred(pi, pj)) continue;
            const float *vj = vel_e + 4 * (size_t)j;
            double rho_j = rho[j];
            double p_j = (gam - 1.0) * rho_j * (double)vj[3];
            double c_j = p_j >= 0.0 ? sqrt(gam * p_j / rho_j) : 0.0;

            double dx = (double)pi[0] - (double)pj[0];
            double dy = (double)pi[1] - (double)pj[1];
            double dz = (double)pi[2] - (double)pj[2];
            double dvx = (double)vi[0] - (double)vj[0];
            double dvy = (double)vi[1] - (double)vj[1];
            double dvz = (double)vi[2] - (double)vj[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rr = sqrt(r2);
            double hij = 0.5 * ((double)pi[3] + (double)pj[3]);

            /* grad W_p = dW_p/dxi * (dr / |dr|) * (1 / h_ij); zero at |dr| = 0 */
            double gx = 0.0, gy = 0.0, gz = 0.0;
            if (rr > 0.0) {
                double f = oracle_dWp_dxi(rr / hij, hij) / (rr * hij);
                gx = f * dx; gy = f * dy; gz = f * dz;
            }

            /* artificial viscosity nu_ij (Monaghan form of Sect. 2.2) */
            double rv = dx * dvx + dy * dvy + dz * dvz;
            double nu = 0.0;
            if (rv < 0.0) {
                double mu = hij * rv / (r2 + eta * hij * hij);
                double rho_ij = 0.5 * (rho_i + rho_j);
                double c_ij = 0.5 * (c_i + c_j);
                nu = mu * (beta * mu - alpha * c_ij) / rho_ij;
            }
            double Pi = p_i / (rho_i * rho_i) + p_j / (rho_j * rho_j) + nu;
            double mj = mass[j];
            ax -= mj * Pi * gx;
            ay -= mj * Pi * gy;
            az -= mj * Pi * gz;
            de += 0.5 * mj * Pi * (dvx * gx + dvy * gy + dvz * gz);
        }
        acc[3 * (size_t)r + 0] = ax;
        acc[3 * (size_t)r + 1] = ay;
        acc[3 * (size_t)r + 2] = az;
        dedt[r] = de;
    }
}

/* ------------------------------------------------------------------------ */
/* Direct particle-particle gravity, Eq. 4 with reading R1, summed over     */
/* all N particles (gas and dark), and the softened potential.             */
/* pos_m is [n][4]: x, y, z, m.                                             */
/* ------------------------------------------------------------------------ */

void oracle_gravity(int n, const float *pos_m, double G, double eps,
                    const int *rows, int n_rows, double *acc, double *pot)
{
    double eps2 = eps * eps;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        const float *pi = pos_m + 4 * (size_t)i;
        double ax = 0.0, ay = 0.0, az = 0.0, ph = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const float *pj = pos_m + 4 * (size_t)j;
            double dx = (double)pi[0] - (double)pj[0];
            double dy = (double)pi[1] - (double)pj[1];
            double dz = (double)pi[2] - (double)pj[2];
            double d2 = dx * dx + dy * dy + dz * dz + eps2;
            double inv = 1.0 / sqrt(d2);
            double mj = pj[3];
            double s = G * mj * inv * inv * inv;
            ax -= s * dx;
            ay -= s * dy;
            az -= s * dz;
            ph -= G * mj * inv;
        }
        acc[3 * (size_t)r + 0] = ax;
        acc[3 * (size_t)r + 1] = ay;
        acc[3 * (size_t)r + 2] = az;
        pot[r] = ph;
    }
}

/* ------------------------------------------------------------------------ */
/* Leapfrog predictor-corrector, Eqs. 12-16.                                 */
/* State is SoA FP64: r[3][n], v[3][n], e[n_gas]; gas particles come first. */
/* Q_i = a_hyd_i + g_i for gas, g_i for dark; E_i = de_i/dt.                 */
/* ------------------------------------------------------------------------ */

/* Predictor (Eqs. 12-14): saves v, e; v <- v + dt Q; e <- e + dt E;
 * r <- r + dt/2 (v_pred + v_saved). */
void oracle_predict(int n, int n_gas, double dt, double *r, double *v, double *e,
                    double *v_save, double *e_save, const double *a_hyd,
                    const double *dedt, const double *grav)
{
    for (int i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            size_t k = (size_t)d * n + i;
            double q = grav[3 * (size_t)i + d];
            if (i < n_gas) q += a_hyd[3 * (size_t)i + d];
            double v0 = v[k];
            double vt = v0 + dt * q;
            v_save[k] = v0;
            v[k] = vt;
            r[k] = r[k] + 0.5 * dt * (vt + v0);
        }
        if (i < n_gas) {
            double e0 = e[i];
            e_save[i] = e0;
            e[i] = e0 + dt * dedt[i];
        }
    }
}

/* Corrector (Eqs. 15-16): v <- (v_saved + v_pred)/2 + dt/2 Q(r', v_pred, e_pred);
 * e likewise. */
void oracle_correct(int n, int n_gas, double dt, double *v, double *e,
                    const double *v_save, const double *e_save,
                    const double *a_hyd, const double *dedt, const double *grav)
{
    for (int i = 0; i < n; ++i) {
        for (int d = 0; d < 3; ++d) {
            size_t k = (size_t)d * n + i;
            double q = grav[3 * (size_t)i + d];
            if (i < n_gas) q += a_hyd[3 * (size_t)i + d];
            v[k] = 0.5 * (v_save[k] + v[k]) + 0.5 * dt * q;
        }
        if (i < n_gas) e[i] = 0.5 * (e_save[i] + e[i]) + 0.5 * dt * dedt[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Modified CFL time step, Eq. 17 (reading R10), per listed gas particle:   */
/* dt_i = C s_min / (c_max (1 + 1.2 alpha) + 1.2 beta mu_max               */
/*                   + sqrt(s_min (|Q_i| + |E_i|)))                          */
/* Q_i = total acceleration (hydro + gravity) [n][3], E_i = de_i/dt [n].    */
/* par = {gamma, alpha, beta, eta, C}.  Returns min over the rows.          */
/* ------------------------------------------------------------------------ */

double oracle_cfl(int n, const float *pos_h, const float *vel_e, const float *rho,
                  const double *Q, const double *E, const double *par, const int *rows,
                  int n_rows, double *dt_row)
{
    double gam = par[0], alpha = par[1], beta = par[2], eta = par[3], C = par[4];
    double dt_min = INFINITY;
    #pragma omp parallel for schedule(dynamic, 16) reduction(min:dt_min)
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        const float *pi = pos_h + 4 * (size_t)i;
        const float *vi = vel_e + 4 * (size_t)i;
        double p_i = (gam - 1.0) * (double)rho[i] * (double)vi[3];
        double c_i = p_i >= 0.0 ? sqrt(gam * p_i / (double)rho[i]) : 0.0;
        double s_min = INFINITY, c_max = 0.0, mu_max = 0.0;
        int found = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const float *pj = pos_h + 4 * (size_t)j;
            if (!nb_pred(pi, pj)) continue;
            const float *vj = vel_e + 4 * (size_t)j;
            found = 1;
            double dx = (double)pi[0] - (double)pj[0];
            double dy = (double)pi[1] - (double)pj[1];
            double dz = (double)pi[2] - (double)pj[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rr = sqrt(r2);
            if (rr < s_min) s_min = rr;
            double p_j = (gam - 1.0) * (double)rho[j] * (double)vj[3];
            double c_j = p_j >= 0.0 ? sqrt(gam * p_j / (double)rho[j]) : 0.0;
            double c_ij = 0.5 * (c_i + c_j);
            if (c_ij > c_max) c_max = c_ij;
            double rv = dx * ((double)vi[0] - (double)vj[0]) + dy * ((double)vi[1] - (double)vj[1]) +
                        dz * ((double)vi[2] - (double)vj[2]);
            if (rv < 0.0) {
                double hij = 0.5 * ((double)pi[3] + (double)pj[3]);
                double mu = hij * rv / (r2 + eta * hij * hij);
                if (-mu > mu_max) mu_max = -mu;
            }
        }
        double dt = INFINITY;
        if (found) {
            const double *q = Q + 3 * (size_t)i;
            double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
            double denom = c_max * (1.0 + 1.2 * alpha) + 1.2 * beta * mu_max +
                           sqrt(s_min * (qn + fabs(E[i])));
            dt = C * s_min / denom;
        }
        dt_row[r] = dt;
        if (dt < dt_min) dt_min = dt;
    }
    return dt_min;
}
