/*
 * FP64 direct sum of the DCIM-approximated layered Green's function (oracle).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the CPU baseline, never by
 * the CUDA library.
 *
 * Sec. 3.1, eq. ``totalinteraction``: for a target r_i in layer l,
 *   Phi(r_i) = sum_{j in layer l, r_j != r_i} q_j h0(k_l |r_i - r_j|)
 *            + sum_{l'} sum_j q_j (u^up_{l l'} + u^down_{l l'})(r_i, r_j),
 * with the factor i k_l / (4 pi) omitted (Sec. 3.1) and h0(z) = e^{iz}/(iz).
 * The same-layer reaction field is the DCIM image sum of Sec. 3.2, Step 3
 * (eq. ``closedformgreen``), written with the image distance
 *   zeta = sz*z + szp*z' + c,   R_j = sqrt(rho^2 + (zeta - zeta_min - Z_j)^2),
 * each image contributing A_j h0(k_l R_j).  The self pair is excluded from the
 * free-space part only, and only for bit-identical coordinates.
 *
 * Plain C99 complex arithmetic, one OpenMP thread per block of targets.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>

static inline double complex h0c(double complex kR) {
    return cexp(I * kR) / (I * kR);
}

void oracle_direct_sum(int64_t ns, const double *sx, const double *sy, const double *sz,
                       const double *q, const int *slay,
                       int64_t nt, const double *tx, const double *ty, const double *tz,
                       const int *tlay,
                       const double *kre, const double *kim,
                       int nimg, const int *img_layer, const double *img_sz,
                       const double *img_szp, const double *img_c, const double *img_zmin,
                       const double *img_are, const double *img_aim,
                       const double *img_zre, const double *img_zim,
                       int include_free, int include_reaction, double *phi)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        const int l = tlay[i];
        const double complex k = kre[l] + I * kim[l];
        double complex acc = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            if (slay[j] != l) continue;
            const double complex qj = q[2 * j] + I * q[2 * j + 1];
            const double dx = tx[i] - sx[j], dy = ty[i] - sy[j], dz = tz[i] - sz[j];
            const double rho2 = dx * dx + dy * dy;
            if (include_free && !(tx[i] == sx[j] && ty[i] == sy[j] && tz[i] == sz[j])) {
                const double r = sqrt(rho2 + dz * dz);
                acc += qj * h0c(k * r);
            }
            if (include_reaction) {
                for (int m = 0; m < nimg; ++m) {
                    if (img_layer[m] != l) continue;
                    const double zeta = img_sz[m] * tz[i] + img_szp[m] * sz[j] + img_c[m];
                    const double complex Z = img_zre[m] + I * img_zim[m];
                    const double complex A = img_are[m] + I * img_aim[m];
                    const double complex w = zeta - img_zmin[m] - Z;
                    const double complex R = csqrt(rho2 + w * w);
                    acc += qj * A * h0c(k * R);
                }
            }
        }
        phi[2 * i] = creal(acc);
        phi[2 * i + 1] = cimag(acc);
    }
}
