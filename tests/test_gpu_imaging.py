"""Multi-plane system on the GPU (Sec. 2.3): source plane A -> Fresnel R1 -> thin lens (and an
optional pupil) in plane B -> Fresnel R2 -> image plane C, by chaining propagations through the
C ABI with the lens recorded on the propagated plane.  Against the paper's imaging result
S_C = C' S_A on the inverted grid (unit magnification, lens law) and against the FP64 oracle's
chain (with a finite pupil, where the image is no longer exact)."""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from gpu_cases import rel

pytestmark = pytest.mark.gpu

N, D, LAM, F = 64, 20e-6, 633e-9, 0.2
TOL = 1e-5


def _source():
    m = WL.to_c64(WL.amplitude_mask(N, seed=5) * (np.arange(N)[:, None] < 40))
    return m


def _gpu_chain(m, R1, R2, pupil=None):
    import torch
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(N, D, LAM)
    mt = torch.from_numpy(m).cuda()
    c.source_gsm(0.1e-3, 0.05e-3, 1.0)
    c.source_mask(mt)
    SA = c.spectral_density().cpu().numpy().astype(np.float64)
    c.propagate_fresnel(R1)
    c.source_lens(F)
    if pupil:
        c.source_aperture(pupil)
    c.propagate_fresnel(R2)
    SC = c.spectral_density()
    torch.cuda.synchronize()
    out = dict(SA=SA, SC=SC.cpu().numpy().astype(np.float64), W=c.W.cpu().numpy().astype(np.complex128),
               dx=c.sampling())
    c.close()
    return out


def test_unit_magnification_image_is_inverted_source():
    m = _source()
    out = _gpu_chain(m, 2 * F, 2 * F)
    assert abs(out["dx"] / D - 1) < 1e-12
    W0 = O.apply_mask(O.gsm_source(N, D, 0.1e-3, 0.05e-3, 1.0), m.astype(np.complex128))
    SA = np.real(O.spectral_density(W0))
    rev = (-np.arange(N)) % N
    assert rel(out["SA"], SA) < TOL
    assert rel(out["SC"], SA[rev][:, rev]) < TOL


def test_finite_pupil_against_oracle_chain():
    m = _source()
    pupil = 0.3e-3
    out = _gpu_chain(m, 1.5 * F, 3 * F, pupil=pupil)
    W0 = O.apply_mask(O.gsm_source(N, D, 0.1e-3, 0.05e-3, 1.0), m.astype(np.complex128))
    WB, dB = O.propagate_fft(W0, D, LAM, 1.5 * F)
    T = O.thin_lens(N, dB, LAM, F) * O.circle_aperture(N, dB, pupil)
    WC, dC = O.propagate_fft(O.apply_mask(WB, T), dB, LAM, 3 * F)
    assert abs(out["dx"] / dC - 1) < 1e-12
    assert rel(out["W"], WC) < TOL
    assert rel(out["SC"], np.real(O.spectral_density(WC))) < TOL
