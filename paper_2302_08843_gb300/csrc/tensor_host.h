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

// Non-equidistant layers (Sec. 4.4): tensor between a target cell of layer i
// and a source cell of layer j (thicknesses h[i], h[j], stacked without gaps)
// at lateral offset (X dx, Y dy), transformed over the two lateral axes of the
// padded grid Px x Py.  Only pairs i <= j are stored (the rest follow from
// h_i N_ij(r) = h_j N_ji(-r)); pair index q(i, j) = i nz - i (i - 1) / 2 + j - i.
// Layout spec[c][q][ky][kx], ky <= Py/2, kx <= Px/2, row stride kx_stride,
// scaled by -1/(Px Py).  xx, xy, yy, zz are the real spectra; for xz and yz
// (odd along one lateral axis) the stored t gives the spectrum -i t.  Newell
// where max(|X|, |Y|, |i - j|) <= p (p < 0: always), the point dipole of the
// source cell beyond.
void tensor_layers_spectrum(int nx, int ny, int nz, double dx, double dy, const double* h, int p, int Px, int Py,
                            int kx_stride, std::vector<double>& spec);

// exp(-2 pi i m / L), m in [0, L), with exact octant symmetry.
void twiddle_table(int L, std::vector<double>& re, std::vector<double>& im);
void twiddle_entry(int L, int m, double* re, double* im);

}  // namespace mm
