/*
 * Raw IF-cube synthesiser for point scatterers seen from a rotating FMCW radar.
 *
 * Sensor model of arXiv 2309.08038, Sec. II-B, Eq. (10): pulse n, ADC sample m,
 *   raw[n][m] += A * p(theta) * exp(j*2*pi*[tau*K*(m*t_s + T_start) + fc*tau]),
 *   tau = 2*R/c,  R = |scatterer - phase centre n|,
 *   p(theta) = cos(theta) = (boresight . (scatterer - phase centre)) / R  when positive, else 0
 *   (Eq. (8) with Eq. (15)).
 * The phase-centre positions (px, py) and bore-sight unit vectors (ux, uy) are
 * supplied per pulse, so rotation jitter (Eq. (37)) is the caller's draw.
 *
 * This is an input generator, not part of the imaging path: it accumulates in
 * double precision and the caller casts the cube to complex64.  The per-sample
 * phase advances by a complex rotation that is re-anchored with an exact
 * sin/cos every 64 samples, which keeps the result within ~1e-13 of direct
 * evaluation.  Pulses are independent and run in parallel under OpenMP.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

static inline double frac_part(double x) { return x - floor(x); }

int synth_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out: [n_az][L] interleaved (re, im) doubles, accumulated into (caller zeroes it). */
void synth_raw_cube(int n_az, int L, int n_sc,
                    const double *sx, const double *sy, const double *a_re, const double *a_im,
                    const double *px, const double *py, const double *ux, const double *uy,
                    double fc, double slope, double t_s, double t_start, double c,
                    double *out, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 2)
#endif
    for (int n = 0; n < n_az; ++n) {
        double *row = out + (size_t)n * (size_t)L * 2;
        for (int t = 0; t < n_sc; ++t) {
            const double dx = sx[t] - px[n], dy = sy[t] - py[n];
            const double R = sqrt(dx * dx + dy * dy);
            const double proj = dx * ux[n] + dy * uy[n];
            double p;
            if (R == 0.0) p = 1.0;
            else if (proj <= 0.0) continue;
            else p = proj / R;
            const double tau = 2.0 * R / c;
            const double ph0 = frac_part(tau * (slope * t_start + fc));   /* cycles at m = 0 */
            const double dph = tau * slope * t_s;                          /* cycles per sample */
            const double are = a_re[t] * p, aim = a_im[t] * p;
            /* four interleaved chains z_{m+4} = z_m * rot^4 keep the recurrence off the critical path */
            const double r1r = cos(TWO_PI * dph), r1i = sin(TWO_PI * dph);
            const double r4r = cos(TWO_PI * 4.0 * dph), r4i = sin(TWO_PI * 4.0 * dph);
            for (int m0 = 0; m0 < L; m0 += 64) {
                const double ph = TWO_PI * frac_part(ph0 + dph * (double)m0);
                const double cr = cos(ph), ci = sin(ph);
                double zr[4], zi[4];
                zr[0] = are * cr - aim * ci;
                zi[0] = are * ci + aim * cr;
                for (int c = 1; c < 4; ++c) {
                    zr[c] = zr[c - 1] * r1r - zi[c - 1] * r1i;
                    zi[c] = zr[c - 1] * r1i + zi[c - 1] * r1r;
                }
                const int m1 = (m0 + 64 < L) ? m0 + 64 : L;
                int m = m0;
                for (; m + 4 <= m1; m += 4) {
                    for (int c = 0; c < 4; ++c) {
                        row[2 * (m + c)] += zr[c];
                        row[2 * (m + c) + 1] += zi[c];
                        const double nr = zr[c] * r4r - zi[c] * r4i;
                        zi[c] = zr[c] * r4i + zi[c] * r4r;
                        zr[c] = nr;
                    }
                }
                for (int c = 0; m < m1; ++m, ++c) {
                    row[2 * m] += zr[c];
                    row[2 * m + 1] += zi[c];
                }
            }
        }
    }
}
