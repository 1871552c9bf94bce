"""Thin ctypes binding of the warm-start neural operator (include/nop.h).

Argument marshalling only: forward, backward, the Adam step and the
hand-off to the solver all run in the CUDA library.  Device arrays are torch
CUDA tensors (float32, contiguous, NHWC); host arrays are numpy.
"""
import ctypes as ct

import numpy as np

from . import lbmib

NOP_EXPORTS = ["nop_config_default", "nop_create", "nop_destroy", "nop_last_error", "nop_param_count",
               "nop_init_params", "nop_set_params", "nop_get_params", "nop_forward", "nop_backward",
               "nop_train_step", "nop_infer_into", "nop_set_fp32"]


class NopConfig(ct.Structure):
    _fields_ = [("struct_size", ct.c_size_t), ("height", ct.c_int), ("width", ct.c_int),
                ("max_batch", ct.c_int), ("in_channels", ct.c_int), ("out_channels", ct.c_int),
                ("channels", ct.c_int * 4), ("device", ct.c_int), ("stream", ct.c_void_p)]


_SET = False


def _lib():
    global _SET
    L = lbmib.lib()
    if not _SET:
        vp = ct.c_void_p
        L.nop_config_default.argtypes = [ct.POINTER(NopConfig)]
        L.nop_create.argtypes = [ct.POINTER(NopConfig), ct.POINTER(vp)]
        L.nop_destroy.argtypes = [vp]
        L.nop_destroy.restype = None
        L.nop_last_error.argtypes = [vp]
        L.nop_last_error.restype = ct.c_char_p
        L.nop_param_count.argtypes = [vp]
        L.nop_param_count.restype = ct.c_longlong
        L.nop_init_params.argtypes = [vp, ct.c_ulonglong]
        L.nop_set_params.argtypes = [vp, ct.c_int, vp]
        L.nop_get_params.argtypes = [vp, ct.c_int, vp]
        L.nop_forward.argtypes = [vp, ct.c_int, vp, vp]
        L.nop_backward.argtypes = [vp, ct.c_int, vp, vp, vp, vp]
        L.nop_set_fp32.argtypes = [vp, ct.c_int]
        L.nop_train_step.argtypes = [vp, ct.c_int, vp, vp, ct.c_float, ct.POINTER(ct.c_double)]
        L.nop_infer_into.argtypes = [vp, vp, vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        _SET = True
    return L


def _dev(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return ct.c_void_p(t.data_ptr())


def _ready():
    # the network runs on its own stream: work queued on torch's current
    # stream (copies into the argument tensors) must be complete first
    import torch
    torch.cuda.current_stream().synchronize()


class NeuralOperator:
    """The U-Net warm-start network on one GPU (nop_create ... nop_destroy)."""

    def __init__(self, height=256, width=512, max_batch=8, in_channels=3, out_channels=4,
                 channels=(32, 64, 96, 128), device=0):
        L = _lib()
        cfg = NopConfig()
        L.nop_config_default(ct.byref(cfg))
        cfg.height, cfg.width, cfg.max_batch = int(height), int(width), int(max_batch)
        cfg.in_channels, cfg.out_channels = int(in_channels), int(out_channels)
        for k in range(4):
            cfg.channels[k] = int(channels[k])
        cfg.device = int(device)
        h = ct.c_void_p()
        st = L.nop_create(ct.byref(cfg), ct.byref(h))
        if st:
            raise lbmib.LBMError(st, "nop_create failed")
        self.h = h
        self.cfg = cfg
        self.shape = (int(height), int(width))
        self.cin, self.cout = int(in_channels), int(out_channels)
        self.channels = tuple(int(c) for c in channels)
        self.n_params = int(L.nop_param_count(h))

    def _check(self, st):
        if st:
            raise lbmib.LBMError(st, _lib().nop_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            _lib().nop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_params(self, seed):
        self._check(_lib().nop_init_params(self.h, int(seed)))

    def set_params(self, theta):
        if hasattr(theta, "data_ptr"):
            _ready()
            self._check(_lib().nop_set_params(self.h, 1, _dev(theta)))
        else:
            a = np.ascontiguousarray(theta, dtype=np.float32)
            assert a.size == self.n_params
            self._check(_lib().nop_set_params(self.h, 0, a.ctypes.data_as(ct.c_void_p)))

    def params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._check(_lib().nop_get_params(self.h, 0, a.ctypes.data_as(ct.c_void_p)))
        return a

    def forward(self, x, y):
        _ready()
        self._check(_lib().nop_forward(self.h, int(x.shape[0]), _dev(x), _dev(y)))

    def backward(self, x, dy, dparams=None, dx=None):
        _ready()
        self._check(_lib().nop_backward(self.h, int(x.shape[0]), _dev(x), _dev(dy), _dev(dparams), _dev(dx)))

    def set_fp32(self, on=True):
        """Gradient-check mode: FP32-operand convolutions (slow; see
        nop_set_fp32 in include/nop.h)."""
        self._check(_lib().nop_set_fp32(self.h, 1 if on else 0))

    def train_step(self, x, target, lr):
        _ready()
        loss = ct.c_double()
        self._check(_lib().nop_train_step(self.h, int(x.shape[0]), _dev(x), _dev(target), float(lr),
                                          ct.byref(loss)))
        return loss.value

    def infer_into(self, solver, x, offset, scale):
        _ready()
        off = (ct.c_double * 4)(*[float(v) for v in offset])
        sc = (ct.c_double * 4)(*[float(v) for v in scale])
        self._check(_lib().nop_infer_into(self.h, solver.h, _dev(x), off, sc))
