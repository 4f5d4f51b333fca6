/*
 * FP64 direct sum of the DCIM-approximated layered Green's function (oracle).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests and the CPU baseline, never by
 * the CUDA library.
 *
 * Sec. 3.2, eq. ``totalinteraction``: for a target r_i in layer l,
 *   Phi(r_i) = sum_{j in layer l, r_j != r_i} q_j h0(k_l |r_i - r_j|)
 *            + sum_{l'} sum_j q_j (u^up_{l l'} + u^down_{l l'})(r_i, r_j),
 * with the factor i k_l / (4 pi) omitted (Sec. 3.1) and h0(z) = e^{iz}/(iz).
 * The same-layer reaction field is the DCIM image sum of Sec. 3.3, Step 3
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

/*
 * Cross-layer part of Phi at each target by reciprocity (Sec. 3.3 fits, one per
 * target).  For a target r_i in layer l and sources in layer l' != l,
 *   u_{l l'}(r_i; r') = (k_l' / k_l)^2 u_{l' l}(r'; r_i),
 * and u_{l' l}(r'; r_i) (the field in layer l' of a source at r_i) is the
 * image sum  sum_m A_m h0(k_l' sqrt(rho^2 + (W(z') - W_min - Z_m)^2)),
 * W(z') = z' - d_l' (up-going part) or d_{l'-1} - z' (down-going part).
 * Fit f of target i (fit_first[i] <= f < fit_first[i+1]) applies to the
 * sources of layer fit_layer[f] with part fit_part[f] (0 up, 1 down), shift
 * fit_wmin[f], factor fit_fre + i fit_fim, images img_first[f] .. img_first[f+1].
 */
void oracle_cross_sum(int64_t ns, const double *sx, const double *sy, const double *sz,
                      const double *q, const int *slay,
                      int64_t nt, const double *tx, const double *ty,
                      const int64_t *fit_first, const int *fit_layer, const int *fit_part,
                      const double *fit_wmin, const double *fit_fre, const double *fit_fim,
                      const int64_t *img_first, const double *are, const double *aim,
                      const double *zre, const double *zim,
                      const double *kre, const double *kim, const double *d, double *phi)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nt; ++i) {
        double complex acc = 0.0;
        for (int64_t f = fit_first[i]; f < fit_first[i + 1]; ++f) {
            const int lp = fit_layer[f];
            const double complex k = kre[lp] + I * kim[lp];
            const double complex fac = fit_fre[f] + I * fit_fim[f];
            double complex part = 0.0;
            for (int64_t j = 0; j < ns; ++j) {
                if (slay[j] != lp) continue;
                const double complex qj = q[2 * j] + I * q[2 * j + 1];
                const double dx = tx[i] - sx[j], dy = ty[i] - sy[j];
                const double rho2 = dx * dx + dy * dy;
                const double W = fit_part[f] == 0 ? sz[j] - d[lp] : d[lp - 1] - sz[j];
                double complex s = 0.0;
                for (int64_t m = img_first[f]; m < img_first[f + 1]; ++m) {
                    const double complex w = W - fit_wmin[f] - (zre[m] + I * zim[m]);
                    const double complex R = csqrt(rho2 + w * w);
                    s += (are[m] + I * aim[m]) * h0c(k * R);
                }
                part += qj * s;
            }
            acc += fac * part;
        }
        phi[2 * i] = creal(acc);
        phi[2 * i + 1] = cimag(acc);
    }
}

/*
 * Cross-layer part of Phi with the images in the TARGET layer l (Sec. 3.3:
 * the source-box z'-expansion of the density, eq. ``layermediumdensity``, and
 * the image form of each z'-derivative, eq. ``closedformgreen``).  Sources are
 * grouped in narrow z'-bins; a source at z' = zc_b + delta (bin b) contributes
 *   q sum_{k3'=0..K} delta^{k3'} sum_m A_m h0(k_l sqrt(rho^2 + (W(z) - W_min - Z_m)^2)),
 * with the fit of Theta^{k3'} at zc_b, W(z) = z - d_l (up) or d_{l-1} - z (down).
 * Fit of (target layer l, bin b, part, k3') is
 *   f = ((l * nbin + b) * 2 + part) * (K + 1) + k3',
 * its images img_first[f] .. img_first[f+1]; wmin[2 l + part] is W_min.
 * Only the layer pairs with use[l * nl + l'] != 0 are summed here.
 */
void oracle_cross_sum_binned(int64_t ns, const double *sx, const double *sy, const double *q,
                             const int *slay, const int *sbin, const double *sdelta,
                             int64_t nt, const double *tx, const double *ty, const double *tz,
                             const int *tlay, int nl, const int *use, int nbin, int K,
                             const int64_t *img_first, const double *are, const double *aim,
                             const double *zre, const double *zim, const double *wmin,
                             const double *kre, const double *kim, const double *d, double *phi)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nt; ++i) {
        const int l = tlay[i];
        const double complex k = kre[l] + I * kim[l];
        double complex acc = 0.0;
        for (int part = 0; part < 2; ++part) {
            if (part == 0 ? l >= nl - 1 : l == 0) continue;
            const double W = part == 0 ? tz[i] - d[l] : d[l - 1] - tz[i];
            const double Wr = W - wmin[2 * l + part];
            for (int64_t j = 0; j < ns; ++j) {
                const int lp = slay[j];
                if (lp == l || !use[l * nl + lp]) continue;
                const double dx = tx[i] - sx[j], dy = ty[i] - sy[j];
                const double rho2 = dx * dx + dy * dy;
                const int64_t f0 = ((int64_t)(l * nbin + sbin[j]) * 2 + part) * (K + 1);
                double complex s = 0.0;
                double pw = 1.0;
                for (int k3p = 0; k3p <= K; ++k3p) {
                    double complex t = 0.0;
                    for (int64_t m = img_first[f0 + k3p]; m < img_first[f0 + k3p + 1]; ++m) {
                        const double complex w = Wr - (zre[m] + I * zim[m]);
                        const double complex R = csqrt(rho2 + w * w);
                        t += (are[m] + I * aim[m]) * h0c(k * R);
                    }
                    s += pw * t;
                    pw *= sdelta[j];
                }
                acc += (q[2 * j] + I * q[2 * j + 1]) * s;
            }
        }
        phi[2 * i] = creal(acc);
        phi[2 * i + 1] = cimag(acc);
    }
}
