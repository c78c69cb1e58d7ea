"""The hand-written adjoint (GPU) against the FP64 oracle's adjoint gradient, which is itself
pinned by central finite differences (tests/test_oracle_pins.py): losses on S alone and on S and
mu together, gradients in the GSM parameters and the amplitude mask (reduced in the adjoint's
second pass) and in an uploaded W0 (stored); the C entry point's argument checks; and a short
fit."""
import numpy as np
import pytest

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

DXI, LAM, SS, SM = 20e-6, 633e-9, 0.1e-3, 0.05e-3


def _grads(N, z, farfield, seed):
    import torch
    from paper_2203_02734_gb300.autograd import GSMIntensity
    rng = np.random.default_rng(seed)
    amask = WL.to_c64(WL.amplitude_mask(N, seed=seed)).real.astype(np.float64)
    target = O.s_loss(1.2 * SS, 0.8 * SM, 1.1, WL.amplitude_mask(N, seed=seed + 1).real, N, DXI, LAM, z,
                      np.zeros((N, N)), np.ones((N, N)), farfield)[1]
    weight = 1.0 + rng.random((N, N))
    model = GSMIntensity(N, DXI, LAM, z, farfield)
    sS = torch.tensor(SS, dtype=torch.float64, requires_grad=True)
    sM = torch.tensor(SM, dtype=torch.float64, requires_grad=True)
    A = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    am = torch.tensor(amask, dtype=torch.float32, device="cuda", requires_grad=True)
    S = model(sS, sM, A, am)
    t = torch.tensor(target, dtype=torch.float64, device="cuda")
    w = torch.tensor(weight, dtype=torch.float64, device="cuda")
    L = torch.sum(w * (S.double() - t) ** 2)
    L.backward()
    model.close()
    ref = O.s_loss_gradient(SS, SM, 1.0, amask, N, DXI, LAM, z, target, weight, farfield)
    return (float(L), float(sS.grad), float(sM.grad), float(A.grad), am.grad.cpu().numpy().astype(np.float64)), ref


@pytest.mark.parametrize("N,z,farfield", [(16, 0.6, False), (16, 0.6, True), (32, 1.0, False)])
def test_adjoint_gradient_matches_oracle(N, z, farfield):
    got, ref = _grads(N, z, farfield, 7 + N)
    assert abs(got[0] / ref[0] - 1) < 1e-5
    for k in (1, 2, 3):
        assert abs(got[k] - ref[k]) < 1e-4 * abs(ref[k]), (k, got[k], ref[k])
    assert np.linalg.norm(got[4] - ref[4]) < 1e-4 * np.linalg.norm(ref[4])


def test_adjoint_gradient_n96_amplitude_mask():
    """The differentiable workload: N = 96, z = 1 m, amplitude mask uniform in [0.5, 1]."""
    cfg = WL.INVERSE_N96
    got, ref = _grads(cfg["N"], cfg["z"], False, 11)
    for k in (1, 2, 3):
        assert abs(got[k] - ref[k]) < 1e-4 * abs(ref[k]), (k, got[k], ref[k])
    assert np.linalg.norm(got[4] - ref[4]) < 1e-4 * np.linalg.norm(ref[4])


def test_fit_decreases_loss():
    """A few Adam steps on (sigma_S, sigma_mu, mask) towards a target S reduce the loss."""
    import torch
    from paper_2203_02734_gb300.autograd import GSMIntensity
    N, z = 32, 1.0
    model = GSMIntensity(N, DXI, LAM, z)
    a_true = torch.tensor(WL.amplitude_mask(N).real, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        target = model(torch.tensor(SS, dtype=torch.float64), torch.tensor(SM, dtype=torch.float64),
                       torch.tensor(1.0, dtype=torch.float64), a_true).double()
    lsS = torch.tensor(np.log(1.3 * SS), dtype=torch.float64, requires_grad=True)
    lsM = torch.tensor(np.log(1.3 * SM), dtype=torch.float64, requires_grad=True)
    am = torch.full((N, N), 0.75, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([lsS, lsM, am], lr=0.02)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        S = model(torch.exp(lsS), torch.exp(lsM), torch.tensor(1.0, dtype=torch.float64), am)
        L = torch.sum((S.double() - target) ** 2) / torch.sum(target ** 2)
        L.backward()
        opt.step()
        losses.append(float(L))
    model.close()
    assert losses[-1] < 0.2 * losses[0], losses


def _sm_targets(N, seed):
    S_t = 1e-3 * (0.5 + WL.uniform01(seed, N * N).reshape(N, N))
    mu_t = 0.3 * np.exp(2j * np.pi * WL.uniform01(seed + 1, N * N).reshape(N, N))
    wS = 1e6 * (0.5 + WL.uniform01(seed + 2, N * N).reshape(N, N))
    wmu = 0.5 + WL.uniform01(seed + 3, N * N).reshape(N, N)
    return S_t, wS, mu_t, wmu


def _torch_loss(S, mu, S_t, wS, mu_t, wmu):
    import torch
    t = lambda x: torch.tensor(x, device="cuda")  # noqa: E731
    return torch.sum(t(wS) * (S.double() - t(S_t)) ** 2) + torch.sum(t(wmu) * torch.abs(mu.cdouble() - t(mu_t)) ** 2)


@pytest.mark.parametrize("N,z,farfield", [(16, 0.6, False), (16, 0.6, True), (32, 1.0, False), (64, 0.8, True)])
def test_s_and_mu_loss_gradient_matches_oracle(N, z, farfield):
    """A loss on S and mu(P1, .): the single adjoint call's parameter and mask gradients against the
    oracle's adjoint (reading R22), 1e-4 relative."""
    import torch
    from paper_2203_02734_gb300.autograd import GSMPropagation
    P1 = (N // 2 - 1, N // 2 + 2)
    amask = WL.to_c64(WL.amplitude_mask(N, seed=N)).real.astype(np.float64)
    S_t, wS, mu_t, wmu = _sm_targets(N, 300 + N)
    model = GSMPropagation(N, DXI, LAM, z, P1=P1, farfield=farfield)
    sS = torch.tensor(SS, dtype=torch.float64, requires_grad=True)
    sM = torch.tensor(SM, dtype=torch.float64, requires_grad=True)
    A = torch.tensor(1.2, dtype=torch.float64, requires_grad=True)
    am = torch.tensor(amask, dtype=torch.float32, device="cuda", requires_grad=True)
    S, mu = model(sS, sM, A, am)
    L = _torch_loss(S, mu, S_t, wS, mu_t, wmu)
    L.backward()
    model.close()
    ref = O.sm_loss_gradient(SS, SM, 1.2, amask, N, DXI, LAM, z, P1, S_t, wS, mu_t, wmu, farfield)
    from gpu_cases import record
    got = (float(sS.grad), float(sM.grad), float(A.grad))
    errs = [abs(got[k] - ref[1 + k]) / abs(ref[1 + k]) for k in range(3)]
    emask = np.linalg.norm(am.grad.cpu().numpy() - ref[4]) / np.linalg.norm(ref[4])
    record("sm_grad_n%d_%s" % (N, "ff" if farfield else "fr"), sigma_S=errs[0], sigma_mu=errs[1], A=errs[2],
           mask=emask)
    assert abs(float(L) / ref[0] - 1) < 1e-4
    assert max(errs) < 1e-4, errs
    assert emask < 1e-4, emask


@pytest.mark.parametrize("with_mu", [False, True], ids=["S_loss", "S_and_mu_loss"])
@pytest.mark.parametrize("farfield", [False, True])
def test_w0_gradient_matches_oracle(with_mu, farfield):
    """dL/dRe W0 + i dL/dIm W0 of an uploaded Hermitian W0 (N = 16): the adjoint stored by the single
    call (Hermitian for an S-loss; the general, non-Hermitian adjoint with a mu term) against the
    oracle's 2 P^H(dL/dW_B*), element by element."""
    import torch
    from paper_2203_02734_gb300.autograd import CSDPropagation
    N, z = 16, 0.45
    P1 = (7, 9)
    R = WL.random_csd(N, seed=21, n_modes=3)
    W0 = (O.gsm_source(N, DXI, SS, SM) + 0.1 * R / np.abs(R).max()).astype(np.complex64)
    S_t, wS, mu_t, wmu = _sm_targets(N, 500)
    W064 = W0.astype(np.complex128)
    # the mu term is weighted where S >= 1e-4 max S (the comparison region of mu, reading R13): its
    # gradient carries 1/S(x) (reading R22), which amplifies the FP32 error of the forward's S and mu
    # where the spectral density is small
    Sref = np.real(O.spectral_density(O.propagate_fft(W064, DXI, LAM, z, farfield)[0]))
    wmu = np.where(Sref >= 1e-4 * Sref.max(), wmu, 0.0) if with_mu else np.zeros_like(wmu)
    model = CSDPropagation(N, DXI, LAM, z, P1=P1, farfield=farfield)
    W0t = torch.tensor(W0, device="cuda", requires_grad=True)
    S, mu = model(W0t)
    L = torch.sum(torch.tensor(wS, device="cuda") * (S.double() - torch.tensor(S_t, device="cuda")) ** 2)
    if with_mu:
        L = L + torch.sum(torch.tensor(wmu, device="cuda") * torch.abs(mu.cdouble() - torch.tensor(mu_t, device="cuda")) ** 2)
    L.backward()
    g = W0t.grad.cpu().numpy().astype(np.complex128)
    model.close()
    L0, WB, S0, mu0 = O.sm_loss(W064, DXI, LAM, z, P1, S_t, wS, mu_t, wmu, farfield)
    Y = O.adjoint_source(WB, P1, 2.0 * wS * (S0 - S_t), 2.0 * wmu * (mu0 - mu_t))
    gref = 2.0 * O.propagate_adjoint(Y, DXI, LAM, z, farfield)
    e = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    from gpu_cases import record
    record("w0_grad_%s_%s" % ("smu" if with_mu else "s", "ff" if farfield else "fr"), W0grad=e)
    assert abs(float(L) / L0 - 1) < 1e-4
    assert e < 1e-4, e
    # with a mu term the gradient is not Hermitian (the P1 row has no mirrored column)
    M = gref.reshape(N * N, N * N)
    herm = np.linalg.norm(M - M.conj().T) / np.linalg.norm(M)
    assert (herm > 1e-3) == with_mu


def test_adjoint_entry_point_rejects_bad_arguments():
    import torch
    import paper_2203_02734_gb300 as pw
    N = 16
    c = pw.CSD(N, DXI, LAM)
    g3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    dS = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    dmu = torch.zeros((N, N), dtype=torch.complex64, device="cuda")

    def call(**kw):
        a = pw.pw_adjoint()
        a.sigma_S_m, a.sigma_mu_m, a.amplitude = SS, SM, 1.0
        for k, v in kw.items():
            setattr(a, k, v)
        with pytest.raises(pw.PwError) as e:
            pw.pw_propagate_fresnel_adjoint(c.h, 0.5, a)
        return str(e.value)
    assert "no upstream gradient" in call(dev_grad3=g3.data_ptr())
    assert "no gradient requested" in call(dev_dS=dS.data_ptr())
    assert "needs the output plane" in call(dev_dmu=dmu.data_ptr(), dev_grad3=g3.data_ptr())
    assert "outside" in call(dev_dmu=dmu.data_ptr(), dev_S=dS.data_ptr(), dev_mu=dmu.data_ptr(), iP=N,
                             dev_grad3=g3.data_ptr())
    assert "misaligned" in call(dev_dS=dS.data_ptr() + 2, dev_grad3=g3.data_ptr())
    assert "GSM parameters" in call(dev_dS=dS.data_ptr(), dev_grad3=g3.data_ptr(), sigma_S_m=-1.0)
    pw.pw_csd_set_padding(c.h, 24)
    assert "PW_EUNSUPPORTED" in call(dev_dS=dS.data_ptr(), dev_grad3=g3.data_ptr())
    c.close()


@pytest.mark.parametrize("N,farfield", [(64, False), (128, False), (128, True)])
def test_adjoint_dot_product_identity_direct_pass_a(N, farfield):
    """The adjoint call at N = 64 and 128, whose first pass writes V directly from the sparse
    adjoint source (plane waves per slice plus the transformed P1 row): for the linear loss
    L(W_B) = Re <2 Y, W_B> with Y the adjoint source of (dL/dS, dL/dmu) (reading R22), the
    gradient in a general W0 is 2 P^H(Y), so Re <dL/dW0, W0> equals Re <2 Y, P(W0)>: the left side
    from the N^4 gradient the call writes, the right side from S and the P1 row of the forward
    (FP64 sums on both sides).  W0 = GSM x phase screen."""
    import torch
    import paper_2203_02734_gb300 as pw
    dxi, lam, z, sS, sM, A = 20e-6, 633e-9, 0.5, 0.1e-3, 0.05e-3, 1.3
    P1 = (N // 2 - 3, N // 2 + 2)
    mask = WL.to_c64(WL.phase_screen(N, seed=WL.SEED + 11, corr_px=3.0))
    c = pw.CSD(N, dxi, lam)
    mt = torch.from_numpy(mask).cuda()
    c.source_gsm(sS, sM, A)
    c.source_mask(mt)
    (c.propagate_farfield if farfield else c.propagate_fresnel)(z)
    S = c.spectral_density()
    mu = c.degree_of_coherence(*P1)
    row = c.W[P1[0], P1[1]].clone()
    torch.cuda.synchronize()
    Sh0 = S.cpu().numpy().astype(np.float64)
    gS_h = 0.5 + 0.5 * WL.uniform01(81, N * N).reshape(N, N)
    u = WL.uniform01(82, 2 * N * N).reshape(2, N, N) - 0.5
    region = Sh0 >= 1e-4 * Sh0.max()
    scale = 0.01 * np.sum(gS_h * Sh0) / max(float(np.sum(np.abs(mu.cpu().numpy())[region])), 1e-30)
    gS = torch.tensor(gS_h, dtype=torch.float32, device="cuda")
    gmu = torch.tensor(np.where(region, scale * (u[0] + 1j * u[1]), 0.0), dtype=torch.complex64, device="cuda")
    adj = pw.pw_adjoint()
    adj.dev_dS, adj.dev_dmu, adj.iP, adj.jP = gS.data_ptr(), gmu.data_ptr(), P1[0], P1[1]
    adj.dev_S, adj.dev_mu, adj.grad_W0 = S.data_ptr(), mu.data_ptr(), 1
    (pw.pw_propagate_farfield_adjoint if farfield else pw.pw_propagate_fresnel_adjoint)(c.h, z, adj)
    pw.pw_csd_check(c.h)
    x, _ = O.axis_coords(N, dxi)
    gax = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (4 * sS ** 2) - (x[:, None] - x[None, :]) ** 2 / (2 * sM ** 2))
    gt = torch.tensor(gax, dtype=torch.float64, device="cuda")
    m64 = torch.tensor(mask.astype(np.complex128), device="cuda")
    left = 0.0
    for a in range(N):  # W0[a, b, c, d] = A conj(m[a, b]) g[a, c] g[b, d] m[c, d]
        blk = (A * torch.conj(m64[a])[:, None, None] * gt[a][None, :, None] * gt[:, None, :]) * m64[None]
        left += float(torch.sum(torch.conj(c.W[a].cdouble()) * blk).real)
    c.close()
    Sh = S.cpu().numpy().astype(np.float64)
    muh = mu.cpu().numpy().astype(np.complex128)
    rowh = row.cpu().numpy().astype(np.complex128)
    gSh = gS.cpu().numpy().astype(np.float64)
    gmuh = gmu.cpu().numpy().astype(np.complex128)
    sp = Sh[P1]
    ok = sp * Sh > 0
    D = np.sqrt(np.where(ok, sp * Sh, 1.0))
    r = np.where(ok, np.real(np.conj(gmuh) * muh), 0.0)
    dS = gSh - np.where(ok & (Sh > 0), r / (2 * np.where(Sh > 0, Sh, 1.0)), 0.0)
    dS[P1] -= r.sum() / (2 * sp)
    gw = np.where(ok, gmuh / D, 0.0)
    right = float(np.sum(dS * Sh) + np.real(np.sum(np.conj(gw) * rowh)))
    e = abs(left - right) / abs(right)
    from gpu_cases import record
    record("adjoint_dot_n%d%s" % (N, "_ff" if farfield else ""), left=left, right=right, rel=e)
    assert e < 1e-5, (left, right, e)
