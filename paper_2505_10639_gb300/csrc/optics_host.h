// Plan-time optics on the host (double precision): pupil masks, Zernike and
// Karhunen-Loeve bases, Kolmogorov covariance, exact OTF supports.
// Sec. 3.1 of the paper defines the generalised pupil (Eq. 20) and the modal
// wavefront (Eq. 22) over a Zernike or KL basis; the sampling readings are
// documented in mfbd.h.
#pragma once

#include <cstdint>
#include <vector>

namespace mfbd_host {

// Binary aperture [n][n] (1 inside), centre (n-1)/2, radius diam/2 (computed
// in double from the float diameter), optional central obscuration.
std::vector<uint8_t> pupil_mask(int n, float diam_px, float obscuration);

// Noll index j >= 1 -> radial order n and azimuthal order m >= 0.
void noll_to_nm(int j, int* n, int* m);

// Noll-normalised Zernike Z_j at (rho, theta); even j -> cos, odd j -> sin.
double zernike(int j, double rho, double theta);

// Covariance of Noll-normalised Zernike coefficients of a Kolmogorov phase
// screen, in units of (D/r0)^(5/3) rad^2 (Noll 1976), row-major [nj][nj].
std::vector<double> noll_covariance(const std::vector<int>& noll);

struct ModalBasis {
    std::vector<double> modes;    // [M][n][n], zero outside the pupil
    std::vector<double> variance; // [M], units of (D/r0)^(5/3)
};

// Zernike modes Noll 2..M+1 sampled on the pupil.
ModalBasis zernike_basis(int n, float diam_px, float obscuration, int n_modes);

// KL modes: block-diagonalised Noll covariance over Zernike 2..J_max (J_max
// closes the smallest complete radial order holding 4M+1 modes), sorted by
// decreasing variance, sampled on the pupil and re-orthonormalised by
// modified Gram-Schmidt on the discrete pupil (unit mean square).
ModalBasis kl_basis(int n, float diam_px, float obscuration, int n_modes);

// Exact OTF support: u on the n x n torus with a nonzero circular
// autocorrelation of the mask; returned for the half spectrum [n][n/2+1].
std::vector<uint8_t> otf_support_half(const std::vector<uint8_t>& mask, int n);

}  // namespace mfbd_host
