"""Zero padding with cropped output (Sec. 3.2) and grid sizes without an FFT plan: the dense path
(four axis contractions, FP32 on the CUDA cores or split-BF16x3 on the tensor cores) against the
FP64 oracle's padded route, element by element at small N, by row probes at the paper's
N = 200 / Nz = 512, and the paper's own padded examples of Sec. 5.1 and 5.2 (N = 200, Nz = 512,
the paper's parameters) against their closed forms (GPU)."""
import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

D, LAM, SS, SM = 20e-6, 633e-9, 0.1e-3, 0.05e-3
MODES = pytest.mark.parametrize("mode", [1, 2], ids=["fp32", "tc_bf16x3"])  # PW_DFT_FP32, PW_DFT_TC_BF16X3


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _gpu(N, Nz, setup, z, farfield=False, dxi=D, lam=LAM, mode=1):
    import torch
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(N, dxi, lam)
    pw.pw_csd_set_padding(c.h, Nz)
    pw.pw_csd_set_dft_mode(c.h, mode)
    assert pw.pw_csd_get_padding(c.h) == Nz
    keep = setup(c, pw, torch)
    (c.propagate_farfield if farfield else c.propagate_fresnel)(z)
    S = c.spectral_density().cpu().numpy().astype(np.float64)
    mu = c.degree_of_coherence(N // 2, N // 2).cpu().numpy().astype(np.complex128)
    W = c.W.cpu().numpy().astype(np.complex128)
    dx = c.sampling()
    pw.pw_csd_check(c.h)
    c.close()
    del keep
    return W, S, mu, dx


def _check(W, S, mu, dx, Wr, dxr, name=None):
    """W, S and mu (where S >= 1e-4 max S) within a relative L2 error of 1e-5 of the oracle."""
    from gpu_cases import record
    N = W.shape[0]
    assert dx == pytest.approx(dxr, rel=1e-12)
    eW = rel(W, Wr)
    Sr = np.real(O.spectral_density(Wr))
    eS = rel(S, Sr)
    mur = O.degree_of_coherence(Wr, N // 2, N // 2)
    keep = Sr >= 1e-4 * Sr.max()
    emu = rel(mu[keep], mur[keep])
    if name:
        record(name, W=eW, S=eS, mu=emu)
    assert eW < 1e-5, eW
    assert eS < 1e-5, eS
    assert emu < 1e-5, emu


@MODES
@pytest.mark.parametrize("N,Nz,farfield", [(16, 24, False), (16, 40, True), (12, 30, False), (40, 64, False)])
def test_padded_gsm_aperture_lens(N, Nz, farfield, mode):
    radius, f, z = 0.3 * N * D, 0.3, 0.4

    def setup(c, pw, torch):
        c.source_gsm(SS, SM, 1.0)
        c.source_aperture(radius)
        c.source_lens(f)
    W, S, mu, dx = _gpu(N, Nz, setup, z, farfield, mode=mode)
    m = O.circle_aperture(N, D, radius) * O.thin_lens(N, D, LAM, f)
    Wr, dxr = O.propagate_padded(O.apply_mask(O.gsm_source(N, D, SS, SM), m), D, LAM, z, Nz, farfield)
    _check(W, S, mu, dx, Wr, dxr, name="padded_n%d_nz%d_%s_mode%d" % (N, Nz, "ff" if farfield else "fr", mode))


@MODES
def test_no_fft_plan_grid_unpadded(mode):
    # N = 20 has no FFT plan: the dense path computes Algorithm 2's result at size N
    N = 20

    def setup(c, pw, torch):
        c.source_gsm(SS, SM, 1.0)
        c.source_aperture(0.3 * N * D)
    W, S, mu, dx = _gpu(N, N, setup, 0.5, mode=mode)
    Wr, dxr = O.propagate_fft(O.apply_mask(O.gsm_source(N, D, SS, SM), O.circle_aperture(N, D, 0.3 * N * D)),
                              D, LAM, 0.5)
    _check(W, S, mu, dx, Wr, dxr, name="dense_n20_mode%d" % mode)


@MODES
def test_padded_uploaded_non_hermitian_array(mode):
    N, Nz = 12, 20
    rng = np.random.default_rng(11)
    W0 = (rng.standard_normal((N,) * 4) + 1j * rng.standard_normal((N,) * 4)).astype(np.complex64)

    def setup(c, pw, torch):
        c.W.copy_(torch.from_numpy(W0).cuda())
        pw.pw_source_array(c.h, c.W.data_ptr(), False)
    W, S, mu, dx = _gpu(N, Nz, setup, 0.5, mode=mode)
    Wr, dxr = O.propagate_padded(W0.astype(np.complex128), D, LAM, 0.5, Nz)
    assert dx == pytest.approx(dxr, rel=1e-12)
    assert rel(W, Wr) < 1e-5


@MODES
def test_padded_diagonal_source(mode):
    N, Nz = 16, 28
    d = WL.amplitude_mask(N, seed=5).real.astype(np.float32)

    def setup(c, pw, torch):
        dd = torch.from_numpy(d).cuda()
        pw.pw_source_diagonal(c.h, dd.data_ptr(), 1.0)
        return dd
    W, S, mu, dx = _gpu(N, Nz, setup, 2.0, farfield=True, mode=mode)
    W0 = np.zeros((N,) * 4, dtype=np.complex128)
    i = np.arange(N)
    W0[i[:, None], i[None, :], i[:, None], i[None, :]] = d
    Wr, dxr = O.propagate_padded(W0, D, LAM, 2.0, Nz, farfield=True)
    _check(W, S, mu, dx, Wr, dxr, name="padded_diag_mode%d" % mode)


def test_padded_two_plane_chain():
    # the padded output plane (sampling lambda z / (Nz dxi)) is the source of a second propagation
    import torch
    import paper_2203_02734_gb300 as pw
    N, Nz = 12, 20
    c = pw.CSD(N, D, LAM)
    pw.pw_csd_set_padding(c.h, Nz)
    c.source_gsm(SS, SM, 1.0)
    c.propagate_fresnel(0.3)
    dx1 = c.sampling()
    c.source_aperture(0.35 * N * dx1)
    c.propagate_fresnel(0.2)
    W = c.W.cpu().numpy().astype(np.complex128)
    dx2 = c.sampling()
    c.close()
    W1, dxr1 = O.propagate_padded(O.gsm_source(N, D, SS, SM), D, LAM, 0.3, Nz)
    W1 = O.apply_mask(W1, O.circle_aperture(N, dxr1, 0.35 * N * dxr1))
    Wr, dxr2 = O.propagate_padded(W1, dxr1, LAM, 0.2, Nz)
    assert dx1 == pytest.approx(dxr1, rel=1e-12) and dx2 == pytest.approx(dxr2, rel=1e-12)
    assert rel(W, Wr) < 1e-5


def test_padding_arguments():
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(16, D, LAM)
    for bad in (8, 17, 1 << 21):
        with pytest.raises(pw.PwError, match="PW_EINVAL"):
            pw.pw_csd_set_padding(c.h, bad)
    pw.pw_csd_set_padding(c.h, 0)
    assert pw.pw_csd_get_padding(c.h) == 16
    c.close()


def _paper_handle(N, Nz, dxi, lam, mode=1):
    import paper_2203_02734_gb300 as pw
    c = pw.CSD(N, dxi, lam)
    pw.pw_csd_set_padding(c.h, Nz)
    pw.pw_csd_set_dft_mode(c.h, mode)
    return c, pw


@MODES
def test_paper_dark_spot_n200_nz512(mode):
    """Sec. 5.1 at the paper's parameters: N = 200, Nz = 512, dxi = 0.0351 um, omega0 = 1.2566e19
    rad/s, a coherent square of Na = 57 pixels (Eq. Na: sqrt(2 pi Nz) = 56.7), R = the dark-spot
    distance (Eq. darkspot).  S against the discrete FP64 answer (the field is separable: a 1D
    pruned transform per axis) and against the Fresnel-integral intensity of a square aperture
    (measured difference of the normalised profiles on the CPU: 2.5e-3)."""
    sp = pytest.importorskip("scipy.special")
    import torch
    N, Nz, dxi, Na = 200, 512, 0.0351e-6, 57
    lam = 2 * np.pi * WL.C_LIGHT / 1.2566e19
    R = (Na * dxi) ** 2 / (2 * np.pi * lam)
    i0 = N // 2 - Na // 2
    m1 = np.zeros(N)
    m1[i0:i0 + Na] = 1.0
    c, pw = _paper_handle(N, Nz, dxi, lam, mode)
    c.source_gsm(1e3, 1e3, 1.0)  # coherence widths of a kilometre: a coherent source
    mt = torch.from_numpy(np.outer(m1, m1).astype(np.complex64)).cuda()
    c.source_mask(mt)
    c.propagate_fresnel(R)
    S = c.spectral_density().cpu().numpy().astype(np.float64)
    dx = c.sampling()
    pw.pw_csd_check(c.h)
    c.close()
    assert dx == pytest.approx(lam * R / (Nz * dxi), rel=1e-12)
    x, _ = O.axis_coords(N, dxi)
    X, _ = O.axis_coords(N, dx)
    u = O.q(R, X ** 2, lam) * (O.padded_dft_matrix(N, Nz, -1) @ (m1 * O.q(R, x ** 2, lam)))
    Sd = np.outer(np.abs(u) ** 2, np.abs(u) ** 2) * O.propagation_scale(dxi, lam, R)
    assert np.abs(S - Sd).max() < 1e-5 * Sd.max()
    lo, hi = x[i0] - dxi / 2, x[i0 + Na - 1] + dxi / 2
    s = np.sqrt(2 / (lam * R))
    S1, C1 = sp.fresnel(s * (lo - X))
    S2, C2 = sp.fresnel(s * (hi - X))
    f = 0.5 * ((C2 - C1) ** 2 + (S2 - S1) ** 2)
    I = np.outer(f, f)
    Sn = S / S.max()
    assert np.abs(Sn - I / I.max()).max() < 0.01
    assert Sn[N // 2, N // 2] < 0.5  # the dark spot at the centre


def test_paper_annulus_n200_nz512():
    """Sec. 5.2 at the paper's parameters: N = 200, Nz = 512, dxi = 1 mm, omega0 = 3.7699e15 rad/s,
    an incoherent annulus Ni = 5, No = 11 (circ = 1/2 on the circle), far field at R = 5 m.  mu(0, x)
    against the discrete FP64 answer (S is uniform; W(0, x) is the pruned 2D transform of the
    annulus) and against the van Cittert-Zernike form (measured on the CPU: 0.024)."""
    sp = pytest.importorskip("scipy.special")
    import torch
    N, Nz, dxi, z, Ni, No = 200, 512, 1e-3, 5.0, 5, 11
    lam = 2 * np.pi * WL.C_LIGHT / 3.7699e15
    x, y = O.axis_coords(N, dxi)
    r2 = np.rint((x[:, None] ** 2 + y[None, :] ** 2) / dxi ** 2)

    def circ(n):
        return np.where(r2 < n * n, 1.0, np.where(r2 == n * n, 0.5, 0.0))
    d = circ(No) - circ(Ni)
    c, pw = _paper_handle(N, Nz, dxi, lam)
    dd = torch.from_numpy(d.astype(np.float32)).cuda()
    pw.pw_source_diagonal(c.h, dd.data_ptr(), 1.0)
    c.propagate_farfield(z)
    mu = c.degree_of_coherence(N // 2, N // 2).cpu().numpy().astype(np.complex128)
    dx = c.sampling()
    pw.pw_csd_check(c.h)
    c.close()
    X, Y = O.axis_coords(N, dx)
    E = O.padded_dft_matrix(N, Nz, -1)
    qX = O.q(z, X[:, None] ** 2 + Y[None, :] ** 2, lam)
    mud = qX * (E @ d @ E.T) / d.sum()  # q*(0) = 1 at P1 = 0
    assert np.abs(mu - mud).max() < 1e-5
    k = 2 * np.pi / lam
    b = np.sqrt(X[:, None] ** 2 + Y[None, :] ** 2)

    def jinc(u):
        safe = np.where(u == 0, 1.0, u)
        return np.where(u == 0, 1.0, 2 * sp.j1(safe) / safe)
    ao, ai = No * dxi, Ni * dxi
    mut = (ao ** 2 * jinc(k * ao * b / z) - ai ** 2 * jinc(k * ai * b / z)) / (ao ** 2 - ai ** 2)
    mr = mu * np.conj(qX)
    assert np.abs(mr.imag).max() < 1e-5
    assert np.abs(mr.real - mut).max() < 0.04


@MODES
def test_phase_screen_rows_n200_nz512(mode):
    # the GSM x phase-screen source at the paper's padded size, three rows against the oracle's
    # pruned-transform probes; Hermiticity on sampled columns
    import torch
    N, Nz, z = 200, 512, 0.5
    m = WL.phase_screen(N, seed=WL.SEED, corr_px=3.0)
    c, pw = _paper_handle(N, Nz, D, LAM, mode)
    c.source_gsm(SS, SM, 1.0)
    mt = torch.from_numpy(WL.to_c64(m)).cuda()
    c.source_mask(mt)
    c.propagate_fresnel(z)
    rows = [(100, 100), (93, 108), (111, 97)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    cols = [c.W[:, :, a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    pw.pw_csd_check(c.h)
    c.close()
    ref = O.propagate_rows_gsm_padded(m, N, D, LAM, z, SS, SM, 1.0, rows, Nz)
    for r in range(len(rows)):
        assert rel(Wrows[r], ref[r]) < 1e-5
        assert np.linalg.norm(cols[r] - np.conj(Wrows[r])) < 1e-5 * np.linalg.norm(ref[r])


def test_tensor_core_single_a_tile_n240():
    # N = 240 (Np = 240): the tensor-core contraction's shared memory holds one A tile only
    import torch
    N, Nz, z = 240, 320, 0.4
    m = WL.phase_screen(N, seed=WL.SEED + 2, corr_px=3.0)
    c, pw = _paper_handle(N, Nz, D, LAM, 2)
    c.source_gsm(SS, SM, 1.0)
    mt = torch.from_numpy(WL.to_c64(m)).cuda()
    c.source_mask(mt)
    c.propagate_fresnel(z)
    rows = [(120, 120), (101, 133)]
    Wrows = [c.W[a, b].cpu().numpy().astype(np.complex128) for a, b in rows]
    pw.pw_csd_check(c.h)
    c.close()
    ref = O.propagate_rows_gsm_padded(m, N, D, LAM, z, SS, SM, 1.0, rows, Nz)
    for r in range(len(rows)):
        assert rel(Wrows[r], ref[r]) < 1e-5


@pytest.mark.parametrize("stall", [1, -2], ids=["b_copy_left_out", "a_tile_left_out"])
def test_tensor_core_wait_timeout_is_reported_and_recovers(stall):
    # failure detection without a GPU fault: CTA 0 never copies operand chunk 1 (stall = 1), or never
    # announces A tile 2 while that chunk's B copy is in flight (stall = -2); the bounded wait gives
    # up (~1 s), the kernel drains what it started, pw_csd_check reports PW_ETIMEOUT, and the next
    # propagation is right
    import paper_2203_02734_gb300 as pw
    N, Nz, z = 40, 64, 0.4  # Np = 48: three operand chunks
    c = pw.CSD(N, D, LAM)
    pw.pw_csd_set_padding(c.h, Nz)
    pw.pw_csd_set_dft_mode(c.h, pw.PW_DFT_TC_BF16X3)
    c.source_gsm(SS, SM, 1.0)
    pw.pw_csd_inject_stall(c.h, stall)
    c.propagate_fresnel(z)
    with pytest.raises(pw.PwError, match="PW_ETIMEOUT"):
        pw.pw_csd_check(c.h)
    pw.pw_csd_check(c.h)  # the condition was cleared
    pw.pw_csd_reset(c.h, D)
    c.source_gsm(SS, SM, 1.0)
    c.propagate_fresnel(z)
    pw.pw_csd_check(c.h)
    W = c.W.cpu().numpy().astype(np.complex128)
    c.close()
    Wr, _ = O.propagate_padded(O.gsm_source(N, D, SS, SM), D, LAM, z, Nz)
    assert rel(W, Wr) < 1e-5
