/* Brute-force demag sum (Sec. 4.4, the discrete convolution written out).
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle, never linked by the
 * product library.
 *
 *   h_i = - sum_j N(i - j) M_j          (positive-trace N, M = Ms m)
 *
 * Nt : 6 x (2nx-1) x (2ny-1) x (2nz-1) doubles, C order, components
 *      (xx, xy, xz, yy, yz, zz); entry [c][i+nx-1][j+ny-1][k+nz-1] is the
 *      component at cell offset (i, j, k).
 * M  : nx x ny x nz x 3 doubles (C order, vector component fastest).
 * h  : same layout as M, overwritten.
 * One OpenMP thread per target cell; each target sums its sources in a fixed
 * order, so the result does not depend on the thread count.
 */
#include <stddef.h>

void direct_demag(int nx, int ny, int nz, const double* Nt, const double* M, double* h)
{
    const long ox = 2L * nx - 1, oy = 2L * ny - 1, oz = 2L * nz - 1;
    const long comp = ox * oy * oz;
    const long ncell = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16)
    for (long t = 0; t < ncell; ++t) {
        const long i = t / ((long)ny * nz), j = (t / nz) % ny, k = t % nz;
        double hx = 0.0, hy = 0.0, hz = 0.0;
        for (long si = 0; si < nx; ++si)
            for (long sj = 0; sj < ny; ++sj)
                for (long sk = 0; sk < nz; ++sk) {
                    const long off = ((i - si + nx - 1) * oy + (j - sj + ny - 1)) * oz + (k - sk + nz - 1);
                    const double* m = M + 3 * ((si * ny + sj) * nz + sk);
                    const double nxx = Nt[off], nxy = Nt[comp + off], nxz = Nt[2 * comp + off];
                    const double nyy = Nt[3 * comp + off], nyz = Nt[4 * comp + off], nzz = Nt[5 * comp + off];
                    hx += nxx * m[0] + nxy * m[1] + nxz * m[2];
                    hy += nxy * m[0] + nyy * m[1] + nyz * m[2];
                    hz += nxz * m[0] + nyz * m[1] + nzz * m[2];
                }
        h[3 * t + 0] = -hx;
        h[3 * t + 1] = -hy;
        h[3 * t + 2] = -hz;
    }
}
