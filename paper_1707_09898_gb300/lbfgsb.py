"""L-BFGS-B on the GPU (include/topomag_lbfgsb.h): argument marshalling and the
reverse-communication loop. The paper minimises its objective with L-BFGS-B over
0 <= rho <= 1 (Sec. "Discretization"; Table I counts its iterations).

    res = minimize(fg, x0)                   # fg(x) -> (f, g), x and g device tensors
    res = optimize_magnet(magnet, rho0)      # the prepared objective of a Magnet

Defaults are SciPy's: m = 10, factr = 1e7, pgtol = 1e-5, maxls = 20,
maxiter = maxfun = 15000.
"""

import ctypes
from dataclasses import dataclass, field
from typing import List

import torch

from . import _lib

FG, NEW_X, CONV_PGTOL, CONV_REL_F, ABNORMAL = 1, 2, 3, 4, 5
MESSAGES = {CONV_PGTOL: "CONVERGENCE: NORM OF PROJECTED GRADIENT <= PGTOL",
            CONV_REL_F: "CONVERGENCE: RELATIVE REDUCTION OF F <= FACTR*EPSMCH",
            ABNORMAL: "ABNORMAL: LINE SEARCH FAILED", -1: "STOP: TOTAL NO. OF ITERATIONS REACHED LIMIT",
            -2: "STOP: TOTAL NO. OF F AND G EVALUATIONS EXCEEDS LIMIT"}


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@dataclass
class Result:
    x: torch.Tensor
    fun: float
    nit: int
    nfev: int
    status: int
    message: str
    history: List[float] = field(default_factory=list)   # f after each iteration (f(x0) first)


class LBFGSB:
    """One optimizer state on the device (n variables, constant bounds)."""

    def __init__(self, n, lower=0.0, upper=1.0, m=10, factr=1e7, pgtol=1e-5, maxls=20, device=0):
        self.L = _lib.lib()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        h = ctypes.c_void_p()
        code = self.L.tm_lbfgsb_create(ctypes.byref(h), self.device.index or 0, int(n), int(m), float(lower),
                                       float(upper), float(factr), float(pgtol), int(maxls))
        if code != 0:
            raise _lib.TopomagError(code, "tm_lbfgsb_create failed")
        self.h, self.n = h, int(n)
        self.task = ctypes.c_int(0)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.tm_lbfgsb_destroy(self.h)
            self.h = None

    def _ck(self, code):
        if code != 0:
            raise _lib.TopomagError(code, self.L.tm_lbfgsb_last_error(self.h).decode())

    @staticmethod
    def _pair(t):
        if t is None:
            return None, None
        if t.dtype == torch.float32:
            return _p(t), None
        if t.dtype == torch.float64:
            return None, _p(t)
        raise TypeError("float32 or float64 device tensors only")

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def start(self, x0, xeval):
        a32, a64 = self._pair(x0)
        e32, e64 = self._pair(xeval)
        self._ck(self.L.tm_lbfgsb_start(self.h, a32, a64, e32, e64, ctypes.byref(self.task), self._stream()))
        return self.task.value

    def iterate(self, f, g, xeval):
        g32, g64 = self._pair(g)
        e32, e64 = self._pair(xeval)
        self._ck(self.L.tm_lbfgsb_iterate(self.h, float(f), g32, g64, e32, e64, ctypes.byref(self.task),
                                          self._stream()))
        return self.task.value

    def info(self):
        c, v = (ctypes.c_longlong * 5)(), (ctypes.c_double * 3)()
        self._ck(self.L.tm_lbfgsb_info(self.h, c, v))
        return {"nit": c[0], "nfev": c[1], "pairs": c[2], "breakpoints": c[3], "free": c[4], "f": v[0],
                "projg": v[1], "theta": v[2]}


def minimize(fg, x0, lower=0.0, upper=1.0, m=10, factr=1e7, pgtol=1e-5, maxls=20, maxiter=15000, maxfun=15000,
             callback=None):
    """Minimise fg over lower <= x <= upper from x0 (a float32 or float64 device tensor; the
    evaluation point has the same dtype). fg(x) returns (f, g) with g a device tensor of
    x's shape (float32 or float64). callback(x, f) after each iteration."""
    x0 = x0.contiguous()
    opt = LBFGSB(x0.numel(), lower, upper, m, factr, pgtol, maxls, x0.device)
    x = torch.empty_like(x0)
    task = opt.start(x0, x)
    nfev, nit, f, hist = 0, 0, None, []
    status = 0
    while True:
        if task == FG:
            if nfev >= maxfun:
                status = -2
                break
            f, g = fg(x)
            nfev += 1
            if not hist:
                hist.append(float(f))
            task = opt.iterate(f, g.contiguous(), x)
        elif task == NEW_X:
            nit += 1
            hist.append(float(f))
            if callback is not None:
                callback(x, f)
            if nit >= maxiter:
                status = -1
                break
            task = opt.iterate(0.0, None, x)
        else:
            status = task
            break
    info = opt.info()
    return Result(x=x, fun=info["f"], nit=info["nit"], nfev=nfev, status=status,
                  message=MESSAGES.get(status, str(status)), history=hist)


def optimize_magnet(magnet, rho0, **kw):
    """L-BFGS-B on the objective prepared by magnet.set_target (tm_evaluate), from rho0
    (float32 design-grid tensor)."""
    G = torch.empty_like(rho0)

    def fg(rho):
        J, _ = magnet.evaluate(rho, G=G)
        return J, G

    return minimize(fg, rho0.contiguous(), **kw)
