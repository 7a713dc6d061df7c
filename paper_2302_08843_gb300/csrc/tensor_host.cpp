// Host-side demag tensor (Sec. 4.4), double precision.
//
// Newell's cell-averaged tensor (Newell, Williams & Dunlop 1993, the formula
// Sec. 4.4 cites) within a Chebyshev cell distance p, the point dipole of
// Eq. dipole beyond.  Positive-trace convention: h = -N M.
//
// The spectrum on the padded periodic grid is real and needs only the
// non-negative octant of offsets: along an axis where a component is even,
//   F(k) = f(0) + 2 sum_{X=1}^{n-1} f(X) cos(2 pi k X / P),
// and where it is odd (f(0) = 0),
//   F(k) = -i * 2 sum_{X=1}^{n-1} f(X) sin(2 pi k X / P);
// off-diagonal components are odd along two axes, so the two factors of -i
// give an overall -1.  The wrapped entries between n-1 and P-n+1 are zero.
// The transform is applied axis by axis (x, then y, then z), each as a small
// dense matrix product with an OpenMP loop over the other two axes.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tensor_host.h"

namespace mm {

static inline double asinh_ratio(double num, double den) { return std::asinh(num / den); }

// Newell f, even in every argument; vanishing-prefactor terms are zero.
static double newell_f(double x, double y, double z) {
    x = std::fabs(x); y = std::fabs(y); z = std::fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = std::sqrt(x2 + y2 + z2);
    double r = (2.0 * x2 - y2 - z2) * R / 6.0;
    const double rxz = std::sqrt(x2 + z2), rxy = std::sqrt(x2 + y2);
    if (y > 0.0 && rxz > 0.0) r += 0.5 * y * (z2 - x2) * asinh_ratio(y, rxz);
    if (z > 0.0 && rxy > 0.0) r += 0.5 * z * (y2 - x2) * asinh_ratio(z, rxy);
    if (x > 0.0 && y > 0.0 && z > 0.0) r -= x * y * z * std::atan(y * z / (x * R));
    return r;
}

// Newell g, odd in x and y, even in z.
static double newell_g(double x, double y, double z) {
    const double sgn = ((x < 0.0) != (y < 0.0)) ? -1.0 : 1.0;
    if (x == 0.0 || y == 0.0) {
        // every term carries a factor x or y (the asinh/atan terms vanish with them)
        return 0.0;
    }
    x = std::fabs(x); y = std::fabs(y); z = std::fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = std::sqrt(x2 + y2 + z2);
    double r = -x * y * R / 3.0;
    r += y / 6.0 * (3.0 * z2 - y2) * asinh_ratio(x, std::sqrt(y2 + z2));
    r += x / 6.0 * (3.0 * z2 - x2) * asinh_ratio(y, std::sqrt(x2 + z2));
    if (z > 0.0) {
        r += x * y * z * asinh_ratio(z, std::sqrt(x2 + y2));
        r -= z * z2 / 6.0 * std::atan(x * y / (z * R));
        r -= z * y2 / 2.0 * std::atan(x * z / (y * R));
        r -= z * x2 / 2.0 * std::atan(y * z / (x * R));
    }
    return sgn * r;
}

typedef double (*gen_fn)(double, double, double);

// 27-point combination with weights prod_i (2 if e_i == 0 else -1), / (4 pi V)
static double newell_stencil(gen_fn fn, double X, double Y, double Z, double a, double b, double c) {
    double acc = 0.0;
    for (int i = -1; i <= 1; ++i) {
        const double wi = i == 0 ? 2.0 : -1.0;
        for (int j = -1; j <= 1; ++j) {
            const double wj = j == 0 ? 2.0 : -1.0;
            for (int k = -1; k <= 1; ++k) {
                const double wk = k == 0 ? 2.0 : -1.0;
                acc += wi * wj * wk * fn(X + i * a, Y + j * b, Z + k * c);
            }
        }
    }
    return acc / (4.0 * M_PI * a * b * c);
}

// component order: 0 xx, 1 xy, 2 xz, 3 yy, 4 yz, 5 zz
static double newell_comp(int comp, double X, double Y, double Z, double a, double b, double c) {
    switch (comp) {
        case 0: return newell_stencil(newell_f, X, Y, Z, a, b, c);
        case 3: return newell_stencil(newell_f, Y, X, Z, b, a, c);
        case 5: return newell_stencil(newell_f, Z, Y, X, c, b, a);
        case 1: return newell_stencil(newell_g, X, Y, Z, a, b, c);
        case 2: return newell_stencil(newell_g, X, Z, Y, a, c, b);
        default: return newell_stencil(newell_g, Y, Z, X, b, c, a);
    }
}

static double dipole_comp(int comp, double X, double Y, double Z, double V) {
    static const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    const double r2 = X * X + Y * Y + Z * Z;
    const double r = std::sqrt(r2);
    const double v[3] = {X, Y, Z};
    const double delta = ia[comp] == ib[comp] ? 1.0 : 0.0;
    return -V / (4.0 * M_PI * r2 * r) * (3.0 * v[ia[comp]] * v[ib[comp]] / r2 - delta);
}

void tensor_octant(const int n[3], const double d[3], int p, std::vector<double>& oct) {
    const int nx = n[0], ny = n[1], nz = n[2];
    const size_t cnt = (size_t)nx * ny * nz;
    oct.assign(6 * cnt, 0.0);
    const double V = d[0] * d[1] * d[2];
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int cheb = i > j ? (i > k ? i : k) : (j > k ? j : k);
                const bool near = p < 0 || cheb <= p;
                const double X = i * d[0], Y = j * d[1], Z = k * d[2];
                const size_t o = ((size_t)k * ny + j) * nx + i;
                for (int c = 0; c < 6; ++c)
                    oct[c * cnt + o] = near ? newell_comp(c, X, Y, Z, d[0], d[1], d[2])
                                            : dipole_comp(c, X, Y, Z, V);
            }
}

// parity of each component along (x, y, z): true = odd
static const bool kOdd[6][3] = {{false, false, false}, {true, true, false}, {true, false, true},
                                {false, false, false}, {false, true, true}, {false, false, false}};

void tensor_full_offsets(const int n[3], const double d[3], int p, double* out) {
    std::vector<double> oct;
    tensor_octant(n, d, p, oct);
    const int nx = n[0], ny = n[1], nz = n[2];
    const long ox = 2L * nx - 1, oy = 2L * ny - 1, oz = 2L * nz - 1;
    const size_t cnt = (size_t)nx * ny * nz;
    for (int c = 0; c < 6; ++c)
        for (long a = 0; a < ox; ++a)
            for (long b = 0; b < oy; ++b)
                for (long e = 0; e < oz; ++e) {
                    const long i = a - (nx - 1), j = b - (ny - 1), k = e - (nz - 1);
                    double s = 1.0;
                    if (kOdd[c][0] && i < 0) s = -s;
                    if (kOdd[c][1] && j < 0) s = -s;
                    if (kOdd[c][2] && k < 0) s = -s;
                    const size_t o = ((size_t)std::labs(k) * ny + std::labs(j)) * nx + std::labs(i);
                    out[((c * ox + a) * oy + b) * oz + e] = s * oct[c * cnt + o];
                }
}

// cos and sin of 2 pi m / P with exact symmetry: reduce m to the first octant.
static void unit_root(long P, long m, double* c, double* s) {
    m %= P;
    if (m < 0) m += P;
    // angle = 2 pi m / P; use quadrant and octant reduction on the integer
    const long q4 = 4 * m;                 // angle in units of (pi/2)/P
    long quad = q4 / P;                    // 0..3
    long rem = q4 - quad * P;              // in [0, P): fraction of a quadrant, times P
    double cc, ss;
    if (2 * rem <= P) {
        const double a = (M_PI / 2.0) * (double)rem / (double)P;
        cc = std::cos(a); ss = std::sin(a);
    } else {
        const double a = (M_PI / 2.0) * (double)(P - rem) / (double)P;
        cc = std::sin(a); ss = std::cos(a);
    }
    if (rem == 0) { cc = 1.0; ss = 0.0; }
    switch (quad & 3) {
        case 0: *c = cc; *s = ss; break;
        case 1: *c = -ss; *s = cc; break;
        case 2: *c = -cc; *s = -ss; break;
        default: *c = ss; *s = -cc; break;
    }
}

// table[k * n + X] for k in [0, K), X in [0, n): even -> (X == 0 ? 1 : 2 cos),
// odd -> (X == 0 ? 0 : 2 sin); the odd-axis -i factors are applied by the caller.
static void axis_table(int n, int P, int K, bool odd, std::vector<double>& t) {
    t.assign((size_t)K * n, 0.0);
    for (int k = 0; k < K; ++k)
        for (int X = 0; X < n; ++X) {
            double c, s;
            unit_root(P, (long)k * X, &c, &s);
            double v;
            if (X == 0) v = odd ? 0.0 : 1.0;
            else v = odd ? 2.0 * s : 2.0 * c;
            t[(size_t)k * n + X] = v;
        }
}

void tensor_spectrum(const int n[3], const double d[3], int p, const int P[3], int kx_stride,
                     std::vector<double>& spec) {
    const int nx = n[0], ny = n[1], nz = n[2];
    const int KX = P[0] / 2 + 1, KY = P[1] / 2 + 1, KZ = P[2] / 2 + 1;
    std::vector<double> oct;
    tensor_octant(n, d, p, oct);
    const size_t cnt = (size_t)nx * ny * nz;
    const size_t out_cnt = (size_t)KZ * KY * kx_stride;
    spec.assign(6 * out_cnt, 0.0);
    const double scale = -1.0 / ((double)P[0] * (double)P[1] * (double)P[2]);
    std::vector<double> tx[2], ty[2], tz[2];
    for (int o = 0; o < 2; ++o) {
        axis_table(nx, P[0], KX, o == 1, tx[o]);
        axis_table(ny, P[1], KY, o == 1, ty[o]);
        axis_table(nz, P[2], KZ, o == 1, tz[o]);
    }
    std::vector<double> a((size_t)nz * ny * KX), b((size_t)nz * KY * KX);
    for (int c = 0; c < 6; ++c) {
        const double* f = oct.data() + c * cnt;
        const std::vector<double>& Tx = tx[kOdd[c][0]];
        const std::vector<double>& Ty = ty[kOdd[c][1]];
        const std::vector<double>& Tz = tz[kOdd[c][2]];
        // x: a[z][y][kx] = sum_X Tx[kx][X] f[z][y][X]
#pragma omp parallel for schedule(static)
        for (long row = 0; row < (long)nz * ny; ++row) {
            const double* fr = f + row * nx;
            double* ar = a.data() + row * KX;
            for (int kx = 0; kx < KX; ++kx) {
                const double* t = Tx.data() + (size_t)kx * nx;
                double acc = 0.0;
                for (int X = 0; X < nx; ++X) acc += t[X] * fr[X];
                ar[kx] = acc;
            }
        }
        // y: b[z][ky][kx] = sum_Y Ty[ky][Y] a[z][Y][kx]
#pragma omp parallel for schedule(static) collapse(2)
        for (int z = 0; z < nz; ++z)
            for (int ky = 0; ky < KY; ++ky) {
                double* br = b.data() + ((size_t)z * KY + ky) * KX;
                for (int kx = 0; kx < KX; ++kx) br[kx] = 0.0;
                for (int Y = 0; Y < ny; ++Y) {
                    const double w = Ty[(size_t)ky * ny + Y];
                    if (w == 0.0) continue;
                    const double* ar = a.data() + ((size_t)z * ny + Y) * KX;
                    for (int kx = 0; kx < KX; ++kx) br[kx] += w * ar[kx];
                }
            }
        // z: out[kz][ky][kx] = sum_Z Tz[kz][Z] b[Z][ky][kx], times the sign of the
        // odd factors and the inverse-FFT normalisation
        const int nodd = (int)kOdd[c][0] + (int)kOdd[c][1] + (int)kOdd[c][2];
        const double sg = (nodd == 2 ? -1.0 : 1.0) * scale;
        double* outc = spec.data() + c * out_cnt;
#pragma omp parallel for schedule(static) collapse(2)
        for (int kz = 0; kz < KZ; ++kz)
            for (int ky = 0; ky < KY; ++ky) {
                double* orow = outc + ((size_t)kz * KY + ky) * kx_stride;
                for (int kx = 0; kx < KX; ++kx) orow[kx] = 0.0;
                for (int Z = 0; Z < nz; ++Z) {
                    const double w = Tz[(size_t)kz * nz + Z];
                    if (w == 0.0) continue;
                    const double* br = b.data() + ((size_t)Z * KY + ky) * KX;
                    for (int kx = 0; kx < KX; ++kx) orow[kx] += w * br[kx];
                }
                for (int kx = 0; kx < KX; ++kx) orow[kx] *= sg;
            }
    }
}

// ------------------------------------------------ non-equidistant layers ----
// Cell average between boxes of different thickness: along z, where equal
// cells combine 2 F(Z) - F(Z + c) - F(Z - c), a target box of thickness hi and
// a source box of thickness hj whose lower faces are Z0 apart combine
// F(Z0) - F(Z0 + hi) - F(Z0 - hj) + F(Z0 + hi - hj); the sum is divided by the
// target volume.  z is the third argument of f / g for xx, yy, xy, the first
// for zz and the second for xz, yz (the same permutations as newell_comp).
static double layer_comp(int comp, double X, double Y, double Z0, double a, double b, double hi, double hj) {
    const double zs[4] = {Z0, Z0 + hi, Z0 - hj, Z0 + hi - hj};
    const double wz[4] = {1.0, -1.0, -1.0, 1.0};
    double acc = 0.0;
    for (int i = -1; i <= 1; ++i) {
        const double wi = i == 0 ? 2.0 : -1.0;
        const double x = X + i * a;
        for (int j = -1; j <= 1; ++j) {
            const double wj = j == 0 ? 2.0 : -1.0;
            const double y = Y + j * b;
            for (int k = 0; k < 4; ++k) {
                const double z = zs[k];
                double v;
                switch (comp) {
                    case 0: v = newell_f(x, y, z); break;
                    case 3: v = newell_f(y, x, z); break;
                    case 5: v = newell_f(z, y, x); break;
                    case 1: v = newell_g(x, y, z); break;
                    case 2: v = newell_g(x, z, y); break;
                    default: v = newell_g(y, z, x); break;
                }
                acc += wi * wj * wz[k] * v;
            }
        }
    }
    return acc / (4.0 * M_PI * a * b * hi);
}

// lateral parity of each component (x, y): true = odd
static const bool kOddL[6][2] = {{false, false}, {true, true}, {true, false},
                                 {false, false}, {false, true}, {false, false}};

void tensor_layers_spectrum(int nx, int ny, int nz, double dx, double dy, const double* h, int p, int Px, int Py,
                            int kx_stride, std::vector<double>& spec) {
    const int KX = Px / 2 + 1, KY = Py / 2 + 1;
    const int npair = nz * (nz + 1) / 2;
    std::vector<double> z0(nz, 0.0);
    for (int k = 1; k < nz; ++k) z0[k] = z0[k - 1] + h[k - 1];
    // real-space entries at X, Y >= 0 for every stored pair: oct[c][q][Y][X]
    const size_t cnt = (size_t)nx * ny;
    std::vector<double> oct((size_t)6 * npair * cnt, 0.0);
    std::vector<int> qi(npair), qj(npair);
    for (int i = 0, q = 0; i < nz; ++i)
        for (int j = i; j < nz; ++j, ++q) { qi[q] = i; qj[q] = j; }
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int q = 0; q < npair; ++q)
        for (int Y = 0; Y < ny; ++Y)
            for (int X = 0; X < nx; ++X) {
                const int i = qi[q], j = qj[q];
                const int lat = X > Y ? X : Y;
                const int cheb = lat > (j - i) ? lat : (j - i);
                const bool near = p < 0 || cheb <= p;
                const double Xm = X * dx, Ym = Y * dy, Z0 = z0[i] - z0[j];
                const double Zc = Z0 + 0.5 * (h[i] - h[j]);       // centre offset for the dipole
                for (int c = 0; c < 6; ++c)
                    oct[((size_t)c * npair + q) * cnt + (size_t)Y * nx + X] =
                        near ? layer_comp(c, Xm, Ym, Z0, dx, dy, h[i], h[j])
                             : dipole_comp(c, Xm, Ym, Zc, dx * dy * h[j]);
            }
    const size_t out_cnt = (size_t)KY * kx_stride;
    spec.assign((size_t)6 * npair * out_cnt, 0.0);
    const double scale = -1.0 / ((double)Px * (double)Py);
    std::vector<double> tx[2], ty[2];
    for (int o = 0; o < 2; ++o) {
        axis_table(nx, Px, KX, o == 1, tx[o]);
        axis_table(ny, Py, KY, o == 1, ty[o]);
    }
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int c = 0; c < 6; ++c)
        for (int q = 0; q < npair; ++q) {
            const double* f = oct.data() + ((size_t)c * npair + q) * cnt;
            const std::vector<double>& Tx = tx[kOddL[c][0]];
            const std::vector<double>& Ty = ty[kOddL[c][1]];
            std::vector<double> a((size_t)ny * KX);
            for (int Y = 0; Y < ny; ++Y)
                for (int kx = 0; kx < KX; ++kx) {
                    const double* t = Tx.data() + (size_t)kx * nx;
                    double acc = 0.0;
                    for (int X = 0; X < nx; ++X) acc += t[X] * f[(size_t)Y * nx + X];
                    a[(size_t)Y * KX + kx] = acc;
                }
            // two odd axes: (-i)^2 = -1; one odd axis: the -i stays with the kernel
            const double sg = (kOddL[c][0] && kOddL[c][1] ? -1.0 : 1.0) * scale;
            double* outc = spec.data() + ((size_t)c * npair + q) * out_cnt;
            for (int ky = 0; ky < KY; ++ky) {
                double* orow = outc + (size_t)ky * kx_stride;
                for (int Y = 0; Y < ny; ++Y) {
                    const double w = Ty[(size_t)ky * ny + Y];
                    if (w == 0.0) continue;
                    const double* ar = a.data() + (size_t)Y * KX;
                    for (int kx = 0; kx < KX; ++kx) orow[kx] += w * ar[kx];
                }
                for (int kx = 0; kx < KX; ++kx) orow[kx] *= sg;
            }
        }
}

void twiddle_entry(int L, int m, double* re, double* im) {
    double c, s;
    unit_root(L, m, &c, &s);
    *re = c;
    *im = -s;       // exp(-2 pi i m / L)
}

void twiddle_table(int L, std::vector<double>& re, std::vector<double>& im) {
    re.resize(L);
    im.resize(L);
    for (int m = 0; m < L; ++m) {
        double c, s;
        unit_root(L, m, &c, &s);
        re[m] = c;
        im[m] = -s;     // exp(-2 pi i m / L)
    }
}

}  // namespace mm
