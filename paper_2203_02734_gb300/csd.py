"""Convenience wrapper: one C-ABI handle plus the torch device buffers it runs on."""
import torch

from . import abi


def _ptr(t):
    return 0 if t is None else t.data_ptr()


class CSD:
    """An N^4 complex64 CSDA on the current CUDA device (torch buffers) and its handle.

    Methods mirror the C calls (pw_source_*, pw_propagate_*, pw_spectral_density,
    pw_degree_of_coherence) and enqueue on `stream` (default: torch's current stream)."""

    def __init__(self, N, dxi, lam, W=None, work=None, stream=None, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        shape = (N, N, N, N)
        self.W = W if W is not None else torch.empty(shape, dtype=torch.complex64, device=dev)
        self.work = work if work is not None else torch.empty(shape, dtype=torch.complex64, device=dev)
        for t in (self.W, self.work):
            if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("W and work must be contiguous complex64 CUDA tensors")
        self.N = N
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        nb = self.W.numel() * 8
        self.h = abi.pw_csd_create(N, dxi, lam, self.W.data_ptr(), nb, self.work.data_ptr(),
                                   self.work.numel() * 8, self.stream.cuda_stream)
        self._keep = []

    def close(self):
        if self.h:
            abi.pw_csd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, dxi):
        abi.pw_csd_reset(self.h, dxi)
        self._keep = []

    def source_gsm(self, sigma_S, sigma_mu, A=1.0):
        abi.pw_source_gsm(self.h, sigma_S, sigma_mu, A)

    def source_aperture(self, radius):
        abi.pw_source_aperture(self.h, radius)

    def source_lens(self, f):
        abi.pw_source_lens(self.h, f)

    def source_mask(self, mask):
        if mask is not None:
            if mask.dtype != torch.complex64 or not mask.is_cuda or mask.shape != (self.N, self.N):
                raise ValueError("mask must be a complex64 CUDA tensor of shape (N, N)")
            mask = mask.contiguous()
            self._keep.append(mask)
        abi.pw_source_mask(self.h, _ptr(mask))

    def source_array(self, W0, hermitian=True):
        if W0.dtype != torch.complex64 or not W0.is_cuda or not W0.is_contiguous() or W0.numel() != self.N ** 4:
            raise ValueError("W0 must be a contiguous complex64 CUDA tensor with N^4 elements")
        self._keep.append(W0)
        abi.pw_source_array(self.h, W0.data_ptr(), hermitian)

    def propagate_fresnel(self, z):
        abi.pw_propagate_fresnel(self.h, z)
        self._keep = []

    def propagate_farfield(self, z):
        abi.pw_propagate_farfield(self.h, z)
        self._keep = []

    def sampling(self):
        return abi.pw_get_sampling(self.h)

    def spectral_density(self, out=None):
        out = out if out is not None else torch.empty((self.N, self.N), dtype=torch.float32, device=self.W.device)
        abi.pw_spectral_density(self.h, out.data_ptr())
        return out

    def degree_of_coherence(self, iP, jP, out=None):
        out = out if out is not None else torch.empty((self.N, self.N), dtype=torch.complex64, device=self.W.device)
        abi.pw_degree_of_coherence(self.h, iP, jP, out.data_ptr())
        return out
