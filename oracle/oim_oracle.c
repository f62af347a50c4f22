/*
 * oim_oracle.c -- plain FP64 CPU oracle for the simulated oscillator Ising/Potts
 * machine of "GPU-Accelerated Simulated Oscillator Ising/Potts Machine Solving
 * Combinatorial Optimization Problems" (arXiv 2505.22631).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
 * of what the GPU path computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only in the seeded inputs
 * and in the published definition of the Philox4x32-10 generator, which each
 * side implements on its own.
 *
 * Everything is double precision except the phase-to-spin decision of
 * orc_readout_f32, which is taken in FP32 because the GPU path takes it in FP32
 * (the paper computes in float32, Sec. III-C).
 *
 * Layout used throughout: phases theta[r*n + i] (replica-major), symmetric CSR
 * (row_ptr[n+1], col[nnz], w[nnz]) without diagonal entries.
 *
 * Readings of the paper taken here (each one is also listed in the design notes):
 *  - coupling term +K * sum_j w_ij sin(2*pi*(theta_i - theta_j)) with J_ij := w_ij,
 *    the graph weight (Eq. 5 together with Eq. 6, whose energy it descends);
 *  - injection-locking term -Ks * sin(2*pi*q*theta_i), which puts the stable
 *    phases at k/q (Sec. II-D/II-E state N stable points; the printed sign puts
 *    them at (2k+1)/(2q), an equivalent system under a global rotation);
 *  - noise kick Kn * sqrt(dt) * xi with xi ~ N(0,1) (Algorithm 1's noise line);
 *  - synchronous (Jacobi) forward-Euler update, all derivatives from the old
 *    phases (Algorithm 1; Sec. III-A and the separate phase arrays of Sec. III-B);
 *  - wrap to [0,1) by theta - floor(theta) (Algorithm 1, "NormalizeToRange");
 *  - readout to the nearest stable phase k/q, spin = floor(q*theta + 1/2) mod q
 *    (the phase threshold kernel of Sec. III-B); it is never fed back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2.          */
/* One round maps (c0,c1,c2,c3) with key (k0,k1) to                          */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))          */
/* with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl      */
/* constants (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Map a 32-bit word to the open interval (0,1): ((x >> 9) + 1/2) * 2^-23.
 * The result is an odd multiple of 2^-24, exact in FP32 and FP64. */
double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Counter layout of the random stream (a design choice of this library, shared
 * with the GPU path by specification only):
 *   counter = (node i, step t, replica quad r>>2, (graph << 1) | stream),
 *   key     = (low 32 bits of seed, high 32 bits of seed),
 *   lane    = r & 3.
 * stream 0 draws the initial phases, stream 1 the per-step noise. */
enum { ORC_STREAM_INIT = 0, ORC_STREAM_NOISE = 1 };

static void orc_block(uint64_t seed, uint32_t graph, uint32_t stream,
                      int64_t i, int64_t t, int64_t r, uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)i, (uint32_t)t, (uint32_t)(r >> 2),
                        (graph << 1) | stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Initial phase theta0_{i,r}: uniform in (0,1), Algorithm 1 first line. */
double orc_init_phase(uint64_t seed, uint32_t graph, int64_t i, int64_t r)
{
    uint32_t x[4];
    orc_block(seed, graph, ORC_STREAM_INIT, i, 0, r, x);
    return orc_u01(x[r & 3]);
}

/* Standard normal xi_{i,r,t} by the Box-Muller transform of the block's lane
 * pairs (0,1) and (2,3): with rho = sqrt(-2 ln u_a), lane a gets
 * rho*cos(2 pi u_b) and lane b gets rho*sin(2 pi u_b). */
double orc_noise(uint64_t seed, uint32_t graph, int64_t i, int64_t t, int64_t r)
{
    uint32_t x[4];
    orc_block(seed, graph, ORC_STREAM_NOISE, i, t, r, x);
    int lane = (int)(r & 3);
    int a = lane & 2;           /* first lane of the pair */
    double ua = orc_u01(x[a]);
    double ub = orc_u01(x[a + 1]);
    double rho = sqrt(-2.0 * log(ua));
    return (lane & 1) ? rho * sin(ORC_TWO_PI * ub) : rho * cos(ORC_TWO_PI * ub);
}

void orc_init_phases(int32_t n, int32_t R, uint64_t seed, uint32_t graph, double* theta)
{
    for (int32_t r = 0; r < R; ++r)
        for (int32_t i = 0; i < n; ++i)
            theta[(int64_t)r * n + i] = orc_init_phase(seed, graph, i, r);
}

void orc_noise_block(int32_t n, int32_t R, uint64_t seed, uint32_t graph, int64_t t, double* xi)
{
    for (int32_t r = 0; r < R; ++r)
        for (int32_t i = 0; i < n; ++i)
            xi[(int64_t)r * n + i] = orc_noise(seed, graph, i, t, r);
}

/* ------------------------------------------------------------------------ */
/* Dynamics, Eq. 5 and Algorithm 1.                                          */
/* ------------------------------------------------------------------------ */

/* D_i = sum_{j in row i} w_ij * sin(2 pi (theta_i - theta_j)): the inner loop of
 * Algorithm 1, written as the direct phase difference (no trig identity). */
void orc_coupling(int32_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                  const double* theta, double* D)
{
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            acc += w[e] * sin(ORC_TWO_PI * (theta[i] - theta[col[e]]));
        D[i] = acc;
    }
}

/* f_i = K * D_i - Ks * sin(2 pi q theta_i)   (Eq. 5 without the noise term) */
void orc_derivative(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col,
                    const double* w, const double* theta, double K, double Ks, double* f)
{
    orc_coupling(n, row_ptr, col, w, theta, f);
    for (int32_t i = 0; i < n; ++i)
        f[i] = K * f[i] - Ks * sin(ORC_TWO_PI * (double)q * theta[i]);
}

static double orc_wrap(double x)
{
    double y = x - floor(x);
    return (y >= 1.0) ? 0.0 : y;
}

/* One forward-Euler / Euler-Maruyama step of one replica, Algorithm 1 loop body:
 * all derivatives from the old phases, then
 *   theta_i <- wrap(theta_i + dt*f_i + Kn*sqrt(dt)*xi_i). */
static void orc_step_one(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col,
                         const double* w, double K, double Ks, double Kn, double dt,
                         uint64_t seed, uint32_t graph, int64_t t, int64_t r,
                         double* theta, double* scratch)
{
    orc_derivative(n, q, row_ptr, col, w, theta, K, Ks, scratch);
    double sdt = sqrt(dt);
    for (int32_t i = 0; i < n; ++i) {
        double kick = Kn * sdt * orc_noise(seed, graph, i, t, r);
        theta[i] = orc_wrap(theta[i] + dt * scratch[i] + kick);
    }
}

/* Nearest stable phase k/q: spin = floor(q*theta + 1/2) mod q, in FP64. */
static int orc_spin_f64(double th, int32_t q)
{
    int k = (int)floor((double)q * th + 0.5);
    return k % q;
}

/* Same decision taken in FP32 (multiply, add, floor, each rounded to nearest,
 * no fused multiply-add), as the GPU takes it. */
static int orc_spin_f32(float th, int32_t q)
{
    float a = (float)q * th;
    float b = a + 0.5f;
    int k = (int)floorf(b);
    return k % q;
}

void orc_readout_f32(int32_t n, int32_t q, int32_t R, const float* theta, int8_t* spins)
{
    for (int64_t x = 0; x < (int64_t)n * R; ++x)
        spins[x] = (int8_t)orc_spin_f32(theta[x], q);
}

void orc_readout_f64(int32_t n, int32_t q, int32_t R, const double* theta, int8_t* spins)
{
    for (int64_t x = 0; x < (int64_t)n * R; ++x)
        spins[x] = (int8_t)orc_spin_f64(theta[x], q);
}

/* Score of one spin assignment (Eq. 1-2 read as max-cut / colouring):
 *   q == 2: cut       = sum_{i<j} w_ij [s_i != s_j]
 *   q >= 3: conflicts = sum_{i<j} w_ij [s_i == s_j]
 * Summed in CSR order over the upper triangle. */
static double orc_score_one(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col,
                            const double* w, const int8_t* s)
{
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j <= i) continue;
            int differ = s[i] != s[j];
            if (q == 2 ? differ : !differ) acc += w[e];
        }
    return acc;
}

void orc_scores(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col, const double* w,
                int32_t R, const int8_t* spins, double* score)
{
    for (int32_t r = 0; r < R; ++r)
        score[r] = orc_score_one(n, q, row_ptr, col, w, spins + (int64_t)r * n);
}

/* Eq. 6: E = sum_{i<j} w_ij cos(2 pi (theta_i - theta_j)), per replica. */
void orc_energy(int32_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                int32_t R, const double* theta, double* E)
{
    for (int32_t r = 0; r < R; ++r) {
        const double* th = theta + (int64_t)r * n;
        double acc = 0.0;
        for (int32_t i = 0; i < n; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int32_t j = col[e];
                if (j <= i) continue;
                acc += w[e] * cos(ORC_TWO_PI * (th[i] - th[j]));
            }
        E[r] = acc;
    }
}

/* Potential of the noise-free flow: V = (K/2pi) E - (Ks/(2 pi q)) sum_i cos(2 pi q theta_i).
 * Its negative gradient is f of Eq. 5, so V never increases along the flow. */
double orc_lyapunov(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col,
                    const double* w, const double* theta, double K, double Ks)
{
    double E;
    orc_energy(n, row_ptr, col, w, 1, theta, &E);
    double shil = 0.0;
    for (int32_t i = 0; i < n; ++i) shil += cos(ORC_TWO_PI * (double)q * theta[i]);
    return K / ORC_TWO_PI * E - Ks / (ORC_TWO_PI * (double)q) * shil;
}

/* Full simulation of R replicas for T steps (Algorithm 1).  Row r of theta[R][n]
 * is replica r0 + r of the run (its random streams use that index); when
 * init_given is zero theta is first filled from the INIT stream.  Every
 * readout_every steps (after the update of step t with (t+1) % readout_every == 0)
 * the FP64 readout and its score are written to trace[r*n_readouts + k].
 * Replicas are independent and run in parallel on nthreads host threads. */
int orc_run(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col, const double* w,
            const double* K, const double* Ks, const double* Kn, double dt, int64_t T,
            int32_t R, int64_t r0, uint64_t seed, uint32_t graph, int32_t init_given,
            double* theta, int64_t readout_every, double* trace, int32_t nthreads)
{
    if (n <= 0 || q < 2 || R <= 0 || T < 0 || r0 < 0) return -1;
    if (!init_given)
        for (int32_t r = 0; r < R; ++r)
            for (int32_t i = 0; i < n; ++i)
                theta[(int64_t)r * n + i] = orc_init_phase(seed, graph, i, r0 + r);
    int64_t n_readouts = (readout_every > 0) ? T / readout_every : 0;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t r = 0; r < R; ++r) {
        double* th = theta + (int64_t)r * n;
        double* scratch = (double*)malloc(sizeof(double) * (size_t)n);
        int8_t* sp = (int8_t*)malloc((size_t)n);
        if (!scratch || !sp) {
            failed = 1;
        } else {
            int64_t k = 0;
            for (int64_t t = 0; t < T; ++t) {
                orc_step_one(n, q, row_ptr, col, w, K[t], Ks[t], Kn[t], dt, seed, graph, t, r0 + r,
                             th, scratch);
                if (readout_every > 0 && (t + 1) % readout_every == 0 && trace) {
                    for (int32_t i = 0; i < n; ++i) sp[i] = (int8_t)orc_spin_f64(th[i], q);
                    trace[(int64_t)r * n_readouts + k] = orc_score_one(n, q, row_ptr, col, w, sp);
                    ++k;
                }
            }
        }
        free(scratch);
        free(sp);
    }
    return failed ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive solvers for tiny graphs (ground truth for the heuristics).     */
/* ------------------------------------------------------------------------ */

/* Max-cut by enumeration of all 2^(n-1) two-colourings (node n-1 fixed to side 0). */
double orc_bruteforce_maxcut(int32_t n, const int64_t* row_ptr, const int32_t* col,
                             const double* w, int8_t* best_spins)
{
    if (n <= 0 || n > 30) return NAN;
    int8_t* s = (int8_t*)calloc((size_t)n, 1);
    double best = -INFINITY;
    uint64_t count = (uint64_t)1 << (n - 1);
    for (uint64_t m = 0; m < count; ++m) {
        for (int32_t i = 0; i < n; ++i) s[i] = (int8_t)((m >> i) & 1u);
        double c = orc_score_one(n, 2, row_ptr, col, w, s);
        if (c > best) {
            best = c;
            if (best_spins) memcpy(best_spins, s, (size_t)n);
        }
    }
    free(s);
    return best;
}

/* Minimum (weighted) number of monochromatic edges over all q-colourings,
 * by enumeration of q^(n-1) colourings (node 0 fixed to colour 0). */
double orc_bruteforce_min_conflicts(int32_t n, int32_t q, const int64_t* row_ptr,
                                    const int32_t* col, const double* w, int8_t* best_spins)
{
    if (n <= 0 || q < 2) return NAN;
    double total = pow((double)q, (double)(n - 1));
    if (total > 5e8) return NAN;
    int8_t* s = (int8_t*)calloc((size_t)n, 1);
    double best = INFINITY;
    int64_t count = (int64_t)total;
    for (int64_t m = 0; m < count; ++m) {
        int64_t x = m;
        s[0] = 0;
        for (int32_t i = 1; i < n; ++i) { s[i] = (int8_t)(x % q); x /= q; }
        double c = orc_score_one(n, q < 3 ? 3 : q, row_ptr, col, w, s);
        if (c < best) {
            best = c;
            if (best_spins) memcpy(best_spins, s, (size_t)n);
        }
    }
    free(s);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the discrete forward-Euler map, for the gradient of the        */
/* relaxed loss L = (1/R) sum_r E(theta_T^r) (Eq. 6 on the final phases)     */
/* with respect to the per-step schedules K_t, Ks_t, Kn_t.                   */
/*                                                                           */
/* theta_{t+1} = wrap(theta_t + dt f(theta_t; K_t, Ks_t) + Kn_t sqrt(dt) xi_t) */
/* The wrap has unit derivative (every function of the phases is 1-periodic). */
/* lambda_T = dL/dtheta_T = -(2 pi / R) D(theta_T);                          */
/* lambda_t = lambda_{t+1} + dt J_f(theta_t)^T lambda_{t+1}, where           */
/*   df_i/dtheta_i = 2 pi K sum_k w_ik cos(2pi(theta_i-theta_k))             */
/*                   - 2 pi q Ks cos(2 pi q theta_i),                        */
/*   df_i/dtheta_j = -2 pi K w_ij cos(2pi(theta_i-theta_j))  (j in row i);   */
/* dL/dK_t  = dt sum_i lambda_{t+1,i} D_i(theta_t),                          */
/* dL/dKs_t = -dt sum_i lambda_{t+1,i} sin(2 pi q theta_{t,i}),              */
/* dL/dKn_t = sqrt(dt) sum_i lambda_{t+1,i} xi_{t,i}.                        */
/* The forward trajectory of each replica is stored whole.                   */
/* ------------------------------------------------------------------------ */
int orc_adjoint(int32_t n, int32_t q, const int64_t* row_ptr, const int32_t* col, const double* w,
                const double* K, const double* Ks, const double* Kn, double dt, int64_t T,
                int32_t R, uint64_t seed, uint32_t graph, int32_t init_given, const double* theta0,
                double* dK, double* dKs, double* dKn, double* loss, int32_t nthreads)
{
    if (n <= 0 || q < 2 || R <= 0 || T < 0) return -1;
    double* gK = (double*)calloc((size_t)R * (size_t)(T > 0 ? T : 1), sizeof(double));
    double* gS = (double*)calloc((size_t)R * (size_t)(T > 0 ? T : 1), sizeof(double));
    double* gN = (double*)calloc((size_t)R * (size_t)(T > 0 ? T : 1), sizeof(double));
    double* Er = (double*)calloc((size_t)R, sizeof(double));
    if (!gK || !gS || !gN || !Er) { free(gK); free(gS); free(gN); free(Er); return -2; }
    int failed = 0;
    double sdt = sqrt(dt);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t r = 0; r < R; ++r) {
        double* traj = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(T + 1));
        double* D = (double*)malloc(sizeof(double) * (size_t)n);
        double* lam = (double*)malloc(sizeof(double) * (size_t)n);
        double* lam_new = (double*)malloc(sizeof(double) * (size_t)n);
        if (!traj || !D || !lam || !lam_new) {
            failed = 1;
        } else {
            /* forward, keeping every state */
            for (int32_t i = 0; i < n; ++i)
                traj[i] = init_given ? theta0[(int64_t)r * n + i] : orc_init_phase(seed, graph, i, r);
            for (int64_t t = 0; t < T; ++t) {
                double* cur = traj + (size_t)t * n;
                double* nxt = traj + (size_t)(t + 1) * n;
                memcpy(nxt, cur, sizeof(double) * (size_t)n);
                orc_step_one(n, q, row_ptr, col, w, K[t], Ks[t], Kn[t], dt, seed, graph, t, r,
                             nxt, D);
            }
            const double* thT = traj + (size_t)T * n;
            orc_energy(n, row_ptr, col, w, 1, thT, &Er[r]);
            /* terminal adjoint */
            orc_coupling(n, row_ptr, col, w, thT, D);
            for (int32_t i = 0; i < n; ++i) lam[i] = -ORC_TWO_PI * D[i] / (double)R;
            /* backward sweep */
            for (int64_t t = T - 1; t >= 0; --t) {
                const double* th = traj + (size_t)t * n;
                orc_coupling(n, row_ptr, col, w, th, D);
                double aK = 0.0, aS = 0.0, aN = 0.0;
                for (int32_t i = 0; i < n; ++i) {
                    aK += lam[i] * D[i];
                    aS += lam[i] * sin(ORC_TWO_PI * (double)q * th[i]);
                    aN += lam[i] * orc_noise(seed, graph, i, t, r);
                }
                gK[(int64_t)r * T + t] = dt * aK;
                gS[(int64_t)r * T + t] = -dt * aS;
                gN[(int64_t)r * T + t] = sdt * aN;
                for (int32_t j = 0; j < n; ++j) {
                    double self = 0.0, cross = 0.0;
                    for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
                        int32_t k = col[e];
                        double cj = cos(ORC_TWO_PI * (th[j] - th[k]));
                        self += w[e] * cj;
                        cross += lam[k] * w[e] * cj;
                    }
                    double diag = ORC_TWO_PI * K[t] * self
                                  - ORC_TWO_PI * (double)q * Ks[t] * cos(ORC_TWO_PI * (double)q * th[j]);
                    lam_new[j] = lam[j] + dt * (lam[j] * diag - ORC_TWO_PI * K[t] * cross);
                }
                memcpy(lam, lam_new, sizeof(double) * (size_t)n);
            }
        }
        free(traj); free(D); free(lam); free(lam_new);
    }
    if (!failed) {
        for (int64_t t = 0; t < T; ++t) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int32_t r = 0; r < R; ++r) {
                a += gK[(int64_t)r * T + t];
                b += gS[(int64_t)r * T + t];
                c += gN[(int64_t)r * T + t];
            }
            dK[t] = a; dKs[t] = b; dKn[t] = c;
        }
        double L = 0.0;
        for (int32_t r = 0; r < R; ++r) L += Er[r];
        *loss = L / (double)R;
    }
    free(gK); free(gS); free(gN); free(Er);
    return failed ? -2 : 0;
}

/* Algorithm 1's annealing waveform for the injection strength (Sec. III-D): Ks
 * ramps linearly from 0 up to Ks_max and back to 0, `periods` times over `steps`
 * steps.  With x = periods * t / steps, Ks_t = Ks_max * (1 - |2 frac(x) - 1|). */
void orc_triangular(int64_t steps, double ks_max, int32_t periods, double* out)
{
    for (int64_t t = 0; t < steps; ++t) {
        double x = (double)periods * (double)t / (double)steps;
        double f = x - floor(x);
        out[t] = ks_max * (1.0 - fabs(2.0 * f - 1.0));
    }
}
