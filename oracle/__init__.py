"""FP64 CPU oracle for the MOMFBD loss, Wiener object and gradient.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (``paper_2505_10639_gb300``) never imports, links or
executes anything here, and this package imports nothing from the product
except the seeded input generators in ``paper_2505_10639_gb300.synth`` (which
hold none of the method's arithmetic).

It is a plain, slow, obviously correct restatement of the paper
(Asensio Ramos et al., torchmfbd, arXiv:2505.10639):

* ``dft``    -- its own radix-2 FFT and naive DFTs (no library FFT is used).
* ``optics`` -- pupil masks, Noll-indexed Zernike modes, the Kolmogorov
  covariance of Zernike coefficients and the Karhunen-Loeve basis
  (Sec. 3.1), OTF support masks.
* ``mfbd``   -- wavefront, pupil, PSF, OTF (Sec. 3.1, Eqs. 20-22), the
  Wiener object and the object-eliminated loss (Sec. 2.2.1, Eqs. 11-12), and
  the analytic gradient of that loss with respect to the modal coefficients.
* ``patches`` -- the patch grid, mean-subtracted modified-Hanning
  apodisation, data spectra of patches and the weighted merge of patch
  objects into a mosaic (Sec. 5.2), and the top-hat / cosine object filter
  (Sec. 4.1.1).
* ``filters`` -- the Lofdahl-Scharmer object filter (Sec. 4.1.1, Eq. 25):
  threshold, 3 x 3 median and connectivity to the zero frequency.

Every function computes in float64/complex128. Each one is pinned by tests
in ``tests/test_oracle_*.py`` against closed forms, invariants, brute force
and published tables; none is "parity unpinned".
"""

from . import dft, optics, mfbd, patches, filters  # noqa: F401
