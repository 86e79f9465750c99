/* Leap-frog steps of eqs. 14-15 (eqs. 3-6) in plain C, FP64, caller numbering: a compiled copy
 * of the oracle's step (oracle/leapfrog.py) for timing the CPU baseline on the host cores.
 *
 * Oracle: test infrastructure only.  It takes the oracle's own CSR operators (L_B, eq. 3: one
 * row per unknown edge, entries +-1/d_i at R and L; L_E, eq. 4: one row per triangle, entries
 * -s |e| / S) and applies, per step,
 *   1. j = ((1 - nu dt/2) j + dt nbar E) / (1 + nu dt/2)        (plasma media, eq. 5)
 *   2. E = E + dt (L_B B - j)                                     (eqs. 3, 6, 14)
 *      E[src] += dt amp g(t), t = (n + 1/2) dt                    (soft source)
 *   3. B = B + dt L_E E                                           (eqs. 4, 15)
 * in the same order of operations as the numpy oracle (row sums in CSR order).  Each row is
 * computed on its own, so results do not depend on the number of threads.  No code is shared
 * with the library.  Parity: tests/test_oracle_cstep.py pins it to oracle/leapfrog.py. */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double source_g(double t, double w0, double t0, double tau) {
    const double x = (t - t0) / tau;
    return sin(w0 * t) * exp(-x * x);
}

/* Returns the number of threads used. */
int ue_oracle_steps(int64_t n_ei, int64_t n_t, const int64_t* lb_ptr, const int64_t* lb_col,
                    const double* lb_val, const int64_t* le_ptr, const int64_t* le_col,
                    const double* le_val, double* E, double* B, double* j, const double* nbar,
                    double nu, int64_t n_src, const int64_t* src_col, const double* src_amp,
                    double w0, double t0, double tau, double dt, int64_t n0, int64_t n_steps,
                    int threads) {
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#else
    (void)threads;
#endif
    const double ja = 1.0 - 0.5 * nu * dt, jb = 1.0 + 0.5 * nu * dt;
    for (int64_t s = 0; s < n_steps; ++s) {
        if (nbar) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n_ei; ++i) j[i] = (ja * j[i] + dt * nbar[i] * E[i]) / jb;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n_ei; ++i) {
            double acc = 0.0;
            for (int64_t p = lb_ptr[i]; p < lb_ptr[i + 1]; ++p) acc += lb_val[p] * B[lb_col[p]];
            E[i] = E[i] + dt * (acc - (nbar ? j[i] : 0.0));
        }
        if (n_src > 0) {
            const double g = source_g(((double)(n0 + s) + 0.5) * dt, w0, t0, tau);
            for (int64_t q = 0; q < n_src; ++q) E[src_col[q]] += dt * src_amp[q] * g;
        }
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < n_t; ++t) {
            double acc = 0.0;
            for (int64_t p = le_ptr[t]; p < le_ptr[t + 1]; ++p) acc += le_val[p] * E[le_col[p]];
            B[t] = B[t] + dt * acc;
        }
    }
    return used;
}
