// Host-side demag tensor builder (Sec. 4.4), double precision.
#pragma once
#include <vector>

namespace mm {

// Tensor for offsets 0..n-1 per axis: oct[c][k][j][i], components
// (xx, xy, xz, yy, yz, zz).  Newell where max(i, j, k) <= p (p < 0: always),
// point dipole elsewhere.
void tensor_octant(const int n[3], const double d[3], int p, std::vector<double>& oct);

// All offsets, 6 x (2nx-1) x (2ny-1) x (2nz-1), offset (i,j,k) at
// [c][i+nx-1][j+ny-1][k+nz-1] (same rule as tensor_octant).
void tensor_full_offsets(const int n[3], const double d[3], int p, double* out);

// Real spectrum of the six components on the padded grid P, octant of
// wave numbers kz <= Pz/2, ky <= Py/2, kx <= Px/2, layout
// spec[c][kz][ky][kx] with row stride kx_stride, scaled by -1/(Px Py Pz).
void tensor_spectrum(const int n[3], const double d[3], int p, const int P[3], int kx_stride,
                     std::vector<double>& spec);

// exp(-2 pi i m / L), m in [0, L), with exact octant symmetry.
void twiddle_table(int L, std::vector<double>& re, std::vector<double>& im);
void twiddle_entry(int L, int m, double* re, double* im);

}  // namespace mm
