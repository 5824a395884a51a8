/*
 * FP64 direct evaluation of the Laplace N-body sum, Eq. (1) ("The Fast
 * Multipole Method" section):
 *
 *     phi_j = sum_{i != j} q_i / (4 pi |x_i - x_j|)
 *
 * and of its gradient with respect to the target position (the field is
 * minus this):
 *
 *     grad_j = sum_{i != j} q_i (x_i - y_j) / (4 pi |x_i - y_j|^3)
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the CPU oracle that the
 * tests, the smoke check and the benchmark's CPU baseline use to judge the
 * CUDA path.  The product path never links, loads or calls it.
 *
 * Reading of "i != j": a pair whose distance is exactly zero is skipped.
 * With sources == targets this is the i == j term; coincident distinct
 * points contribute nothing instead of infinity.
 *
 * Layout: src, tgt are row-major (n, 3) doubles; q is row-major (ns, nrhs);
 * phi is row-major (nt, nrhs), grad row-major (nt, nrhs, 3); both are
 * overwritten.  Sums run in source order per target, one OpenMP thread per
 * block of targets.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_direct_sum(const double *src, const double *q, int64_t ns,
                       int nrhs, const double *tgt, int64_t nt, double *phi) {
    const double inv4pi = 1.0 / (4.0 * M_PI);
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)nrhs);
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < nt; ++j) {
            const double xj = tgt[3 * j], yj = tgt[3 * j + 1], zj = tgt[3 * j + 2];
            for (int r = 0; r < nrhs; ++r) acc[r] = 0.0;
            for (int64_t i = 0; i < ns; ++i) {
                const double dx = src[3 * i] - xj;
                const double dy = src[3 * i + 1] - yj;
                const double dz = src[3 * i + 2] - zj;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0.0) continue;
                const double inv_r = 1.0 / sqrt(r2);
                const double *qi = q + i * (int64_t)nrhs;
                for (int r = 0; r < nrhs; ++r) acc[r] += qi[r] * inv_r;
            }
            for (int r = 0; r < nrhs; ++r) phi[j * (int64_t)nrhs + r] = acc[r] * inv4pi;
        }
        free(acc);
    }
}

void oracle_direct_gradient(const double *src, const double *q, int64_t ns, int nrhs,
                            const double *tgt, int64_t nt, double *grad) {
    const double inv4pi = 1.0 / (4.0 * M_PI);
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 3 * (size_t)nrhs);
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < nt; ++j) {
            const double xj = tgt[3 * j], yj = tgt[3 * j + 1], zj = tgt[3 * j + 2];
            for (int r = 0; r < 3 * nrhs; ++r) acc[r] = 0.0;
            for (int64_t i = 0; i < ns; ++i) {
                const double dx = src[3 * i] - xj;
                const double dy = src[3 * i + 1] - yj;
                const double dz = src[3 * i + 2] - zj;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0.0) continue;
                const double inv_r = 1.0 / sqrt(r2);
                const double inv_r3 = inv_r * inv_r * inv_r;
                const double *qi = q + i * (int64_t)nrhs;
                for (int r = 0; r < nrhs; ++r) {
                    const double w = qi[r] * inv_r3;
                    acc[3 * r] += w * dx;
                    acc[3 * r + 1] += w * dy;
                    acc[3 * r + 2] += w * dz;
                }
            }
            for (int r = 0; r < 3 * nrhs; ++r) grad[j * 3 * (int64_t)nrhs + r] = acc[r] * inv4pi;
        }
        free(acc);
    }
}
