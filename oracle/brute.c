/* Brute-force TACAW evaluation for tiny inputs, in long double.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/ to pin the NumPy oracle; never
 * linked into the CUDA library.
 *
 * For each pixel k (time series psi[n*npix + k], n = 0..T-1) and energy bin j,
 * evaluates the plain definition with four nested loops:
 *   mu      = (1/T) sum_n psi[n]            (only if subtract_mean)
 *   Psi_j   = sum_n w_n (psi[n] - mu) exp(-2 pi i frac(c_j n))
 *   I[j*npix + k] = |Psi_j|^2
 * The phase is reduced with fmodl in long double, independently of the NumPy path.
 */
#include <math.h>

void tacaw_brute_intensity(const double *psi_re, const double *psi_im, int T, int npix,
                           const double *w, const double *c, int nw, int subtract_mean,
                           double *out_I)
{
    const long double two_pi = 6.283185307179586476925286766559L;
    for (int k = 0; k < npix; ++k) {
        long double mr = 0.0L, mi = 0.0L;
        if (subtract_mean) {
            for (int n = 0; n < T; ++n) {
                mr += psi_re[(long)n * npix + k];
                mi += psi_im[(long)n * npix + k];
            }
            mr /= T;
            mi /= T;
        }
        for (int j = 0; j < nw; ++j) {
            long double sr = 0.0L, si = 0.0L;
            for (int n = 0; n < T; ++n) {
                long double yr = w[n] * ((long double)psi_re[(long)n * npix + k] - mr);
                long double yi = w[n] * ((long double)psi_im[(long)n * npix + k] - mi);
                long double x = (long double)c[j] * (long double)n;
                long double f = fmodl(x, 1.0L);
                if (f < 0) f += 1.0L;
                long double th = two_pi * f;
                long double cs = cosl(th), sn = sinl(th);
                /* (yr + i yi) (cs - i sn) */
                sr += yr * cs + yi * sn;
                si += yi * cs - yr * sn;
            }
            out_I[(long)j * npix + k] = (double)(sr * sr + si * si);
        }
    }
}
