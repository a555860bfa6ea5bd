"""Python face of libtopomag: a context object and torch.autograd Functions.

Every step of the computation runs in the CUDA library; this module only
marshals device pointers, sizes and the current torch stream.

Method: Abert et al., "A fast finite-difference algorithm for topology
optimization of permanent magnets" (arXiv:1707.09898): M = rho^p M0
(Sec. "Methodology", Eq. 2), H = D[M] by the FFT-accelerated convolution with
the demagnetization tensor (Sec. "Discretization", Eqs. (convolution) and
(demag_tensor)), objective J(H(rho), rho) (Eq. (objective_function)) and its
adjoint gradient (Eqs. (adjoint1)-(adjoint2)).
"""

import ctypes

import torch

from . import _lib

F32, U8 = torch.float32, torch.uint8


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Magnet:
    """One grid: output box n_out = (nx, ny, nz), design slab z < nzd, cell size in metres."""

    def __init__(self, n_out, nzd, cellsize=(1e-3, 1e-3, 1e-3), M0=(0.0, 0.0, 1.0 / (4e-7 * 3.141592653589793)),
                 p=3.0, device=0, tensor=True, fft_lengths=None):
        self.L = _lib.lib()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        h = ctypes.c_void_p()
        _lib.check(None, self.L.tm_create(ctypes.byref(h), self.device.index or 0))
        self.h = h
        self.n_out = tuple(int(v) for v in n_out)
        self.nzd = int(nzd)
        self.cellsize = tuple(float(v) for v in cellsize)
        if fft_lengths is None:
            self._ck(self.L.tm_set_grid(self.h, _lib.c_int3(*self.n_out), self.nzd, _lib.c_double3(*self.cellsize)))
        else:  # chosen padded lengths (0: the default for that axis)
            self._ck(self.L.tm_set_grid_lengths(self.h, _lib.c_int3(*self.n_out), self.nzd,
                                                _lib.c_double3(*self.cellsize), _lib.c_int3(*fft_lengths)))
        self._ck(self.L.tm_set_penalty(self.h, float(p)))
        self.p = float(p)
        self.set_M0(M0)
        if tensor:
            self.set_tensor()

    # -- plumbing ------------------------------------------------------------
    def _ck(self, code):
        _lib.check(self.h, code)

    def close(self):
        if getattr(self, "h", None):
            self.L.tm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def design_shape(self):
        return (self.nzd, self.n_out[1], self.n_out[0])

    @property
    def out_shape(self):
        return (self.n_out[2], self.n_out[1], self.n_out[0])

    def fft_lengths(self):
        L = _lib.c_int3()
        self._ck(self.L.tm_get_fft_lengths(self.h, L))
        return tuple(L)

    def _dev(self, t, dtype, shape, name):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise TypeError(f"{name} must be a {dtype} tensor on {self.device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return t.contiguous()

    # -- setup ---------------------------------------------------------------
    def set_M0(self, M0):
        """Constant M0 (3 numbers, A/m) or a varying field (3, nzd, ny, nx) float32 on the device."""
        if isinstance(M0, torch.Tensor) and M0.dim() == 4:
            m = self._dev(M0, F32, (3,) + self.design_shape, "M0")
            self._ck(self.L.tm_set_M0(self.h, _ptr(m), _lib.c_double3(0.0, 0.0, 0.0), _stream(self.device)))
            self.M0 = m
        else:
            v = [float(x) for x in (M0.tolist() if isinstance(M0, torch.Tensor) else M0)]
            self._ck(self.L.tm_set_M0(self.h, None, _lib.c_double3(*v), _stream(self.device)))
            self.M0 = tuple(v)

    def set_tensor(self):
        self._ck(self.L.tm_set_tensor(self.h, _stream(self.device)))

    # -- operators -----------------------------------------------------------
    def stray_field(self, rho, out=None):
        rho = self._dev(rho, F32, self.design_shape, "rho")
        H = torch.empty((3,) + self.out_shape, dtype=F32, device=self.device) if out is None else out
        self._ck(self.L.tm_stray_field(self.h, _ptr(rho), _ptr(H), _stream(self.device)))
        return H

    def stray_field_adjoint(self, rho, gH, out=None):
        rho = self._dev(rho, F32, self.design_shape, "rho")
        gH = self._dev(gH, F32, (3,) + self.out_shape, "gH")
        G = torch.empty(self.design_shape, dtype=F32, device=self.device) if out is None else out
        self._ck(self.L.tm_stray_field_adjoint(self.h, _ptr(rho), _ptr(gH), _ptr(G), _stream(self.device)))
        return G

    def objective_and_gradient(self, rho, mask, Ht=None, Ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, 1.0), G=None,
                               H_out=None, sync=True):
        """(J, dJ/drho) of J = sum_mask sum_c w_c (H_c - Ht_c)^2. J is a float if sync else None."""
        rho = self._dev(rho, F32, self.design_shape, "rho")
        mask = self._dev(mask, U8, self.out_shape, "mask")
        if Ht is not None:
            Ht = self._dev(Ht, F32, (3,) + self.out_shape, "Ht")
        if G is None:
            G = torch.empty(self.design_shape, dtype=F32, device=self.device)
        J = ctypes.c_double(0.0)
        self._ck(self.L.tm_objective_and_gradient(
            self.h, _ptr(rho), _ptr(mask), _ptr(Ht), _lib.c_float3(*[float(v) for v in Ht_const]),
            _lib.c_float3(*[float(v) for v in w]), ctypes.byref(J) if sync else None, _ptr(G), _ptr(H_out),
            _stream(self.device)))
        return (J.value if sync else None), G

    def set_target(self, mask, Ht=None, Ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, 1.0)):
        """Prepare J = sum_mask sum_c w_c (H_c - Ht_c)^2 for repeated evaluate() calls."""
        mask = self._dev(mask, U8, self.out_shape, "mask")
        if Ht is not None:
            Ht = self._dev(Ht, F32, (3,) + self.out_shape, "Ht")
        self._ck(self.L.tm_set_target(self.h, _ptr(mask), _ptr(Ht), _lib.c_float3(*[float(v) for v in Ht_const]),
                                      _lib.c_float3(*[float(v) for v in w]), _stream(self.device)))

    def set_fused(self, on=True):
        """Prepared path: fuse the y transform with the direct z sum (default) or not."""
        self._ck(self.L.tm_set_fused(self.h, int(bool(on))))

    def set_stencil_objective(self, row_ptr, comp, cell, a, c):
        """Prepare J = sum_k c_k (sum_e a_e H[comp_e][cell_e])^2 for evaluate() (host arrays:
        row_ptr [K+1], per entry comp, cell = z*ny*nx + y*nx + x, a; per row c)."""
        import numpy as np

        rp = np.ascontiguousarray(row_ptr, np.int64)
        arrs = (np.ascontiguousarray(comp, np.int32), np.ascontiguousarray(cell, np.int64),
                np.ascontiguousarray(a, np.float64), np.ascontiguousarray(c, np.float64))
        K = len(rp) - 1
        ptr = [x.ctypes.data_as(ctypes.c_void_p) for x in (rp,) + arrs]
        self._ck(self.L.tm_set_stencil_objective(self.h, K, *ptr, _stream(self.device)))

    def evaluate(self, rho, G=None, sync=True):
        """(J, dJ/drho) for the prepared target. J is a float if sync else None."""
        rho = self._dev(rho, F32, self.design_shape, "rho")
        if G is None:
            G = torch.empty(self.design_shape, dtype=F32, device=self.device)
        J = ctypes.c_double(0.0)
        self._ck(self.L.tm_evaluate(self.h, _ptr(rho), ctypes.byref(J) if sync else None, _ptr(G),
                                    _stream(self.device)))
        return (J.value if sync else None), G

    def objective(self):
        J = ctypes.c_double(0.0)
        self._ck(self.L.tm_get_objective(self.h, ctypes.byref(J), _stream(self.device)))
        return J.value

    def copy_objective(self, out):
        """Enqueue a copy of the last J into out (a float64 tensor element, pinned host or
        device memory) on the current stream; returns at once (wait on an event)."""
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or out.numel() != 1:
            raise TypeError("out must be a one-element float64 tensor")
        if out.device.type == "cpu" and not out.is_pinned():
            raise ValueError("a host destination must be pinned memory")
        self._ck(self.L.tm_copy_objective(self.h, _ptr(out), _stream(self.device)))

    def optimize_step(self, rho, G, alpha, normalize=True, reuse_max=False):
        """rho <- clip(rho - alpha G / max|G|, 0, 1) (normalize) or clip(rho - alpha G, 0, 1).
        reuse_max: take max|G| from the evaluation that wrote G (G unchanged since)."""
        mode = (2 if reuse_max else 1) if normalize else 0
        self._ck(self.L.tm_optimize_step(self.h, _ptr(rho), _ptr(G), float(alpha), mode, _stream(self.device)))
        return rho

    def evaluate_step(self, rho, G, alpha, normalize=True, reuse_max=True, sync=True):
        """One projected-gradient iteration: optimize_step(rho, G, alpha, ...) on the
        gradient G holds, then evaluate(rho, G) at the new rho (G overwritten), in one
        call; for 512-point x transforms of one spectrum the step runs inside the
        evaluation's first pass. Returns (J, G) as evaluate."""
        for t, name in ((rho, "rho"), (G, "G")):
            if isinstance(t, torch.Tensor) and not t.is_contiguous():
                raise ValueError(f"{name} is updated in place and must be contiguous")
        rho = self._dev(rho, F32, self.design_shape, "rho")
        G = self._dev(G, F32, self.design_shape, "G")
        mode = (2 if reuse_max else 1) if normalize else 0
        J = ctypes.c_double(0.0)
        self._ck(self.L.tm_evaluate_step(self.h, _ptr(rho), float(alpha), mode, ctypes.byref(J) if sync else None,
                                         _ptr(G), _stream(self.device)))
        return (J.value if sync else None), G

    def check_design(self, rho):
        """Raise TopomagError (TM_ERR_ARG) if rho has entries that are NaN or outside [0, 1]."""
        rho = self._dev(rho, F32, self.design_shape, "rho")
        n = ctypes.c_longlong(0)
        self._ck(self.L.tm_check_design(self.h, _ptr(rho), ctypes.byref(n), _stream(self.device)))
        return 0

    def iteration_stats(self, rho, G):
        """(max|G|, volume fraction sum(rho)/N, share of cells with 0.1 < rho < 0.9)."""
        rho = self._dev(rho, F32, self.design_shape, "rho")
        G = self._dev(G, F32, self.design_shape, "G")
        out = (ctypes.c_double * 3)()
        self._ck(self.L.tm_iteration_stats(self.h, _ptr(rho), _ptr(G), out, _stream(self.device)))
        return tuple(out)

    def selftest_wait_timeout(self, polls=300):
        """Run the bounded-wait self-test; returns the library's return code (TM_ERR_TIMEOUT expected)."""
        return self.L.tm_selftest_wait_timeout(self.h, int(polls), _stream(self.device))

    # -- per-kernel event timing ---------------------------------------------
    KINDS = ("x_forward", "y_forward", "z_pass", "y_inverse", "x_inverse", "other", "yz_forward", "zy_adjoint",
             "objective")

    def profile(self, on=True):
        self._ck(self.L.tm_profile(self.h, int(bool(on))))

    def profile_read(self):
        """{kind: (total ms, launches)} over the launches recorded since profile(True)."""
        ms = (ctypes.c_double * 9)()
        n = (ctypes.c_int * 9)()
        self._ck(self.L.tm_profile_read(self.h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KINDS)}

    # -- inspection (tests) --------------------------------------------------
    def tensor_octant(self):
        import numpy as np
        nx, ny, nz = self.n_out
        out = np.empty((6, nz, ny, nx), dtype=np.float64)
        self._ck(self.L.tm_debug_tensor_octant(self.h, ctypes.c_void_p(out.ctypes.data), _stream(self.device)))
        return out

    def tensor_spectrum(self):
        import numpy as np
        Lx, Ly, Lz = self.fft_lengths()
        out = np.empty((6, Lz // 2 + 1, Ly // 2 + 1, Lx // 2 + 1), dtype=np.float32)
        self._ck(self.L.tm_debug_tensor_spectrum(self.h, ctypes.c_void_p(out.ctypes.data), _stream(self.device)))
        return out


class StrayField(torch.autograd.Function):
    """H = D[rho^p M0]; backward: dL/drho = p rho^(p-1) M0 . D(dL/dH) (hand-written adjoint kernels)."""

    @staticmethod
    def forward(ctx, rho, magnet):
        ctx.magnet = magnet
        ctx.save_for_backward(rho)
        return magnet.stray_field(rho.detach())

    @staticmethod
    def backward(ctx, gH):
        (rho,) = ctx.saved_tensors
        return ctx.magnet.stray_field_adjoint(rho.detach(), gH.contiguous()), None


class TopoObjective(torch.autograd.Function):
    """J(rho) = sum_mask sum_c w_c (H_c - Ht_c)^2 with its fused adjoint gradient."""

    @staticmethod
    def forward(ctx, rho, magnet, mask, Ht=None, Ht_const=(0.0, 0.0, 0.0), w=(0.0, 0.0, 1.0)):
        J, G = magnet.objective_and_gradient(rho.detach(), mask, Ht, Ht_const, w)
        ctx.save_for_backward(G)
        return torch.tensor(J, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, gJ):
        (G,) = ctx.saved_tensors
        return (gJ.to(G.dtype) * G), None, None, None, None, None
