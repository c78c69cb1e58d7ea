"""FP64 CPU oracle for the propagation of a 4D cross-spectral density (PyWolf, arXiv 2203.02734).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
anything in this package.  The product path (the CUDA library behind
``include/pywolf_gb.h`` and its Python binding) never imports it, and this
package imports nothing from the product: the two share no code.  The only
shared module is ``workloads`` (seeded input generators, none of the method's
arithmetic).

Everything here is plain NumPy in complex128 / float64, written from the
paper's definitions and algorithms (section, equation and algorithm cited in
each docstring), slow on purpose, so that a reader can check it by eye.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):

* ``axis_coords``, ``output_sampling``      -- pinned by the paper's printed worked
  numbers (Sec. 5.1, 5.3, 5.4; ``tests/golden/paper_numbers.json``).
* ``propagate_direct``                      -- brute-force quadrature of Eq. W_general;
  pinned by the GSM closed form (continuous Gaussian integral) and by Parseval.
* ``propagate_fft``                         -- Algorithm 2 route; pinned by
  ``propagate_direct`` (brute force, N <= 8), by the GSM closed form at N = 64..128,
  by the separable per-axis quadrature, by Hermiticity / Parseval / trace, and by the
  thin-lens identity q(f) q*(f) = 1 (Eq. qprop3).
* ``gsm_source``, ``circle_aperture``, ``thin_lens`` -- pinned by closed-form special
  cases (S = A exp(-r^2/(2 sigma_S^2)), mu = exp(-d^2/(2 sigma_mu^2))) and integer counts.
* ``spectral_density``, ``degree_of_coherence`` -- pinned by definitions checked on
  rank-one (coherent) inputs where |mu| = 1 exactly.
* ``propagate_adjoint``                     -- pinned by the dot-product test and by
  central finite differences of a real loss.
* ``propagate_padded``                      -- zero padding with cropped output (Sec. 3.2);
  pinned by brute-force quadrature at the padded output samples (``propagate_direct`` with
  ``Nz``) and reduces exactly to ``propagate_fft`` at Nz = N.
* ``padded_dft_matrix``, ``propagate_rows_gsm_padded`` -- the pruned transform as dense matrices,
  for large N; pinned by ``propagate_padded`` row by row and by the GSM closed form at the padded
  output sampling (``gsm_closed_form`` with ``Nz``).
* ``gsm_closed_form``                       -- pinned by Mandel-Wolf beam-expansion
  factor Delta(z) and radius of curvature R(z) (independent textbook forms).

``oracle.plain_fp32`` (imported on its own, not re-exported here) is not a reference: it is the
timed multi-threaded complex64 CPU baseline of the benchmark, checked against this FP64 oracle in
``tests/test_plain_fp32.py``.
"""
from .csd import *  # noqa: F401,F403
