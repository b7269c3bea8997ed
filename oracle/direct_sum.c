/*
 * Test infrastructure: part of the CPU oracle.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.
 *
 * Plain direct-sum evaluation of a 3D discrete convolution with a kernel that
 * is even in each coordinate (the discrete Green's function of Sec. 2, eq.
 * discreteConvolution):
 *
 *     out[o] = scale * sum_{k in src box} T[|o0-k0|][|o1-k1|][|o2-k2|] * src[k]
 *
 * T is stored as its octant [0, L]^3 (index (l0*(L+1)+l1)*(L+1)+l2).  The
 * source box starts at integer point slo and has extent sn; the output box
 * starts at olo with extent on.  Both arrays are dense with axis 2 fastest.
 * Returns 0 on success, 1 if some lag exceeds L (nothing is written then).
 */
#include <stdlib.h>

static long iabs_l(long v) { return v < 0 ? -v : v; }

int oracle_direct_sum(const double *T, int L,
                      const double *src, const int *slo, const int *sn,
                      double *out, const int *olo, const int *on, double scale)
{
    for (int d = 0; d < 3; ++d) {
        long lmax1 = iabs_l((long)olo[d] - (long)(slo[d] + sn[d] - 1));
        long lmax2 = iabs_l((long)(olo[d] + on[d] - 1) - (long)slo[d]);
        if (lmax1 > L || lmax2 > L) return 1;
    }
    const long Lp = (long)L + 1;
    long total = (long)on[0] * on[1];
#pragma omp parallel for schedule(dynamic, 1)
    for (long ab = 0; ab < total; ++ab) {
        long a = ab / on[1], b = ab % on[1];
        long o0 = olo[0] + a, o1 = olo[1] + b;
        for (long c = 0; c < on[2]; ++c) {
            long o2 = olo[2] + c;
            double acc = 0.0;
            for (long i = 0; i < sn[0]; ++i) {
                long l0 = iabs_l(o0 - (slo[0] + i));
                for (long j = 0; j < sn[1]; ++j) {
                    long l1 = iabs_l(o1 - (slo[1] + j));
                    const double *trow = T + (l0 * Lp + l1) * Lp;
                    const double *srow = src + (i * sn[1] + j) * (long)sn[2];
                    for (long k = 0; k < sn[2]; ++k) {
                        acc += trow[iabs_l(o2 - (slo[2] + k))] * srow[k];
                    }
                }
            }
            out[(a * on[1] + b) * (long)on[2] + c] = scale * acc;
        }
    }
    return 0;
}
