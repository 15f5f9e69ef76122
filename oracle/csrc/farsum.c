/* Far-field layer-potential sums by direct summation (oracle, FP64).
 *
 * Test infrastructure only: linked by the oracle's Python loader, never by
 * the CUDA library.
 *
 * For each requested target i and each density sigma_r this evaluates the
 * Nystrom far sums of Section 4 (the target-independent smooth rule over all
 * sources outside Near(i)):
 *
 *   out[r][k][t] = sum_{j : patch(j) not in Near(i)} w_j K_k(x_i, y_j) sigma_r[j]
 *
 * for the kernels k = 0..3 = S, D, S', S''+D' of Section 3 (d = x - y):
 *   S      = 1/(4 pi r)
 *   D      = n_y.d/(4 pi r^3)
 *   S'     = -n_x.d/(4 pi r^3)
 *   S''+D' = [3 (n_x.d)((n_x - n_y).d)/r^2 - (1 - n_x.n_y)]/(4 pi r^3)
 *
 * Sources are the N nodes themselves (node j belongs to patch j / np), or,
 * for the oversampled far rule of Section 4, Ns given points y_s with their
 * own normals, weights and densities (point s belongs to patch s / nps).  A
 * plain double loop, parallel over targets with OpenMP.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Sources given explicitly: Ns points Y with normals ny, weights wy and
 * densities sigma_src [nrhs][Ns]; source s lies on patch s / nps.  Targets
 * are nodes of the surface (X, n, near lists over its patches). */
int oracle_far_sums_src(int64_t N, const double *X, const double *n, const int64_t *near_ptr,
                        const int32_t *near_patch, int64_t npatch, int64_t Ns, int64_t nps,
                        const double *Y, const double *ny, const double *wy, int nrhs,
                        const double *sigma_src, int64_t ntgt, const int64_t *targets, double *out)
{
    const double four_pi = 4.0 * 3.14159265358979323846;
    int bad = 0;
    (void)N;
#pragma omp parallel
    {
        char *is_near = (char *)calloc((size_t)npatch, 1);
        double *acc = (double *)malloc(sizeof(double) * 4 * (size_t)nrhs);
        if (!is_near || !acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < ntgt; ++t) {
            if (!is_near || !acc) continue;
            const int64_t i = targets[t];
            for (int64_t b = near_ptr[i]; b < near_ptr[i + 1]; ++b) is_near[near_patch[b]] = 1;
            memset(acc, 0, sizeof(double) * 4 * (size_t)nrhs);
            const double xi0 = X[3 * i], xi1 = X[3 * i + 1], xi2 = X[3 * i + 2];
            const double nx0 = n[3 * i], nx1 = n[3 * i + 1], nx2 = n[3 * i + 2];
            for (int64_t j = 0; j < Ns; ++j) {
                if (is_near[j / nps]) continue;
                const double d0 = xi0 - Y[3 * j], d1 = xi1 - Y[3 * j + 1], d2 = xi2 - Y[3 * j + 2];
                const double ny0 = ny[3 * j], ny1 = ny[3 * j + 1], ny2 = ny[3 * j + 2];
                const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                const double r = sqrt(r2);
                const double g = 1.0 / (four_pi * r);
                const double g3 = g / r2;
                const double nxd = nx0 * d0 + nx1 * d1 + nx2 * d2;
                const double nyd = ny0 * d0 + ny1 * d1 + ny2 * d2;
                const double nxny = nx0 * ny0 + nx1 * ny1 + nx2 * ny2;
                const double kS = g;
                const double kD = nyd * g3;
                const double kSp = -nxd * g3;
                const double kSD = (3.0 * nxd * (nxd - nyd) / r2 - (1.0 - nxny)) * g3;
                for (int r_ = 0; r_ < nrhs; ++r_) {
                    const double q = wy[j] * sigma_src[(int64_t)r_ * Ns + j];
                    acc[4 * r_ + 0] += kS * q;
                    acc[4 * r_ + 1] += kD * q;
                    acc[4 * r_ + 2] += kSp * q;
                    acc[4 * r_ + 3] += kSD * q;
                }
            }
            for (int r_ = 0; r_ < nrhs; ++r_)
                for (int k = 0; k < 4; ++k)
                    out[((int64_t)r_ * 4 + k) * ntgt + t] = acc[4 * r_ + k];
            for (int64_t b = near_ptr[i]; b < near_ptr[i + 1]; ++b) is_near[near_patch[b]] = 0;
        }
        free(is_near);
        free(acc);
    }
    return bad ? -1 : 0;
}

/* The nodes themselves as sources (the base far rule). */
int oracle_far_sums(int64_t N, int64_t np_, const double *X, const double *n,
                    const double *w, const int64_t *near_ptr, const int32_t *near_patch,
                    int nrhs, const double *sigma, int64_t ntgt, const int64_t *targets,
                    double *out)
{
    return oracle_far_sums_src(N, X, n, near_ptr, near_patch, N / np_, N, np_, X, n, w, nrhs, sigma, ntgt,
                               targets, out);
}

/* Near-field correction sums (Section 4, the corrected Nystrom form): for
 * each requested target i, each density r and each kernel k = S, D, S', S''+D'
 *
 *   out[r][k][t] = sum_{b in row i} sum_q vals[b][k][q] sigma_r[patch(b) * np + q]
 *
 * over the row's blocks b (near_ptr[i] .. near_ptr[i+1]-1), patch(b) =
 * near_patch[b].  vals is [nnzb][4][np].  A plain loop, parallel over
 * targets. */
int oracle_near_apply(int64_t N, int64_t np_, const int64_t *near_ptr, const int32_t *near_patch,
                      const double *vals, int nrhs, const double *sigma, int64_t ntgt,
                      const int64_t *targets, double *out)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < ntgt; ++t) {
        const int64_t i = targets[t];
        for (int r_ = 0; r_ < nrhs; ++r_) {
            const double *sig = sigma + (int64_t)r_ * N;
            for (int k = 0; k < 4; ++k) {
                double acc = 0.0;
                for (int64_t b = near_ptr[i]; b < near_ptr[i + 1]; ++b) {
                    const double *v = vals + (b * 4 + k) * np_;
                    const double *s = sig + (int64_t)near_patch[b] * np_;
                    for (int64_t q = 0; q < np_; ++q) acc += v[q] * s[q];
                }
                out[((int64_t)r_ * 4 + k) * ntgt + t] = acc;
            }
        }
    }
    return 0;
}
