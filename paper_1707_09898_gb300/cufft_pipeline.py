"""The plain cuFFT pipeline (libtopomag_cufft.so), kept only as a speed comparison.

Same objective and adjoint gradient as Magnet.objective_and_gradient, done with
explicit zero padding, 3-D cuFFT R2C/C2R and the full complex64 tensor. The
tensor values come from the main library (same float32 numbers), so only the
way the convolution is evaluated differs. Not used on the product path.
"""

import ctypes
import os

import torch

from . import _lib
from .magnet import Magnet, _ptr, _stream

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtopomag_cufft.so")
_blib = None


def blib():
    global _blib
    if _blib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtopomag_cufft.so not built ({LIB_PATH})")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.tmb_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, _lib.c_int3, ctypes.c_int, _lib.c_int3]
        L.tmb_destroy.argtypes = [vp]
        L.tmb_destroy.restype = None
        L.tmb_set_tensor.argtypes = [vp, vp]
        L.tmb_set_M0.argtypes = [vp, _lib.c_double3, ctypes.c_double]
        L.tmb_objective_and_gradient.argtypes = [vp, vp, vp, _lib.c_float3, _lib.c_float3, vp, vp]
        L.tmb_get_objective.argtypes = [vp, ctypes.POINTER(ctypes.c_double), vp]
        _blib = L
    return _blib


def plain_length(n):
    """Padded length of the plain pipeline: the smallest even 2^a 3^b (b <= 2, >= 8) >= 2 n,
    which cuFFT transforms directly (no replacement of 288 or 384 by 512)."""
    L = max(8, 2 * n)
    while True:
        r = L
        while r % 2 == 0:
            r //= 2
        b = 0
        while r % 3 == 0:
            r //= 3
            b += 1
        if L % 2 == 0 and r == 1 and b <= 2:
            return L
        L += 1


class CufftMagnet:
    def __init__(self, n_out, nzd, cellsize, M0, p=3.0, device=0):
        self.m = Magnet(n_out, nzd, cellsize, M0=M0, p=p, device=device,
                        fft_lengths=tuple(plain_length(int(n)) for n in n_out))
        self.device = self.m.device
        self.design_shape, self.out_shape = self.m.design_shape, self.m.out_shape
        L = self.m.fft_lengths()
        spec = self.m.tensor_spectrum()
        self.B = blib()
        h = ctypes.c_void_p()
        rc = self.B.tmb_create(ctypes.byref(h), self.device.index or 0, _lib.c_int3(*n_out), int(nzd), _lib.c_int3(*L))
        if rc != 0:
            raise RuntimeError(f"tmb_create failed: {rc}")
        self.h = h
        if self.B.tmb_set_tensor(self.h, ctypes.c_void_p(spec.ctypes.data)) != 0:
            raise RuntimeError("tmb_set_tensor failed")
        self.B.tmb_set_M0(self.h, _lib.c_double3(*[float(v) for v in M0]), float(p))

    def fft_lengths(self):
        return self.m.fft_lengths()

    def objective_and_gradient(self, rho, mask, Ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, 1.0), G=None, sync=True, **_):
        if G is None:
            G = torch.empty(self.design_shape, dtype=torch.float32, device=self.device)
        rc = self.B.tmb_objective_and_gradient(self.h, _ptr(rho), _ptr(mask), _lib.c_float3(*Ht_const),
                                               _lib.c_float3(*w), _ptr(G), _stream(self.device))
        if rc != 0:
            raise RuntimeError(f"tmb_objective_and_gradient failed: {rc}")
        return (self.objective() if sync else None), G

    def objective(self):
        J = ctypes.c_double(0.0)
        self.B.tmb_get_objective(self.h, ctypes.byref(J), _stream(self.device))
        return J.value

    def optimize_step(self, rho, G, alpha, normalize=True):
        return self.m.optimize_step(rho, G, alpha, normalize)

    def close(self):
        if getattr(self, "h", None):
            self.B.tmb_destroy(self.h)
            self.h = None
        self.m.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
