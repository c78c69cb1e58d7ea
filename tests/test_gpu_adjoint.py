"""The hand-written adjoint (GPU) against the FP64 oracle's adjoint gradient, which is itself
pinned by central finite differences (tests/test_oracle_pins.py); and a short fit."""
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
