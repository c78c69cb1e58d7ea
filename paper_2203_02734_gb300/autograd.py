"""torch.autograd bridge: S at distance z of the amplitude-masked GSM source, with the hand-written
adjoint of include/pywolf_gb.h (pw_source_diagonal + pw_propagate_fresnel + pw_gsm_gradient) as
its backward.  Forward and backward both run in the library's kernels; torch supplies the buffers
and the loss arithmetic the caller writes on S."""
import torch

from . import abi
from .csd import CSD


class GSMIntensity:
    """S(x) at distance z (Fresnel, or far field) of W0 = A a(xi1) a(xi2) G(xi1, xi2; sigma_S,
    sigma_mu), differentiable in sigma_S, sigma_mu, A and the amplitude mask a (N x N, real).
    One instance owns the two N^4 device buffers and the handles, reused by every call."""

    def __init__(self, N, dxi, lam, z, farfield=False, device=None):
        self.N, self.dxi, self.lam, self.z, self.farfield = N, float(dxi), float(lam), float(z), bool(farfield)
        self.dx = self.lam * self.z / (N * self.dxi)
        self.csd = CSD(N, self.dxi, self.lam, device=device)
        dev = self.csd.W.device
        self.mask_c = torch.zeros((N, N), dtype=torch.complex64, device=dev)
        self.S = torch.empty((N, N), dtype=torch.float32, device=dev)
        self.g3 = torch.zeros(3, dtype=torch.float64, device=dev)
        self.gmask = torch.empty((N, N), dtype=torch.float32, device=dev)

    def __call__(self, sigma_S, sigma_mu, A, amask):
        return _GSMIntensityFn.apply(sigma_S, sigma_mu, A, amask, self)

    def close(self):
        self.csd.close()


class _GSMIntensityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_S, sigma_mu, A, amask, m):
        h = m.csd.h
        am = amask.detach().to(torch.float32).contiguous()
        m.mask_c.real.copy_(am)  # the amplitude mask as a complex mask (argument marshalling)
        abi.pw_csd_reset(h, m.dxi)
        abi.pw_source_gsm(h, float(sigma_S), float(sigma_mu), float(A))
        abi.pw_source_mask(h, m.mask_c.data_ptr())
        (abi.pw_propagate_farfield if m.farfield else abi.pw_propagate_fresnel)(h, m.z)
        abi.pw_spectral_density(h, m.S.data_ptr())
        ctx.m = m
        ctx.params = (float(sigma_S), float(sigma_mu), float(A))
        ctx.like = [(x.device, x.dtype) if torch.is_tensor(x) else None for x in (sigma_S, sigma_mu, A)]
        ctx.save_for_backward(am)
        return m.S.clone()

    @staticmethod
    def backward(ctx, gS):
        m = ctx.m
        (am,) = ctx.saved_tensors
        sS, sM, A = ctx.params
        h = m.csd.h
        d = gS.detach().to(torch.float32).contiguous()
        # adjoint of S = Re diag W_B: dL/dW_B* = (1/2) diag(dL/dS), propagated from the output plane
        abi.pw_csd_reset(h, m.dx)
        abi.pw_source_diagonal(h, d.data_ptr(), 0.5)
        abi.pw_propagate_fresnel(h, m.z)
        abi.pw_gsm_gradient(h, sS, sM, A, am.data_ptr(), m.lam, m.z, m.farfield, m.g3.data_ptr(),
                            m.gmask.data_ptr())
        g = m.g3.clone()
        out = [None if lk is None else g[k].to(device=lk[0], dtype=lk[1]) for k, lk in enumerate(ctx.like)]
        return out[0], out[1], out[2], m.gmask.clone().to(dtype=am.dtype), None
