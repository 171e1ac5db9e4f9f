"""ctypes binding of the learned warm-start network (include/vlb_nn.h).

Argument marshalling only: the forward and backward passes, the loss and the
optimizer run in the CUDA library. Device arrays are passed as raw pointers
(for example torch tensors' data_ptr()); parameters and gradients travel as
host FP32 arrays.
"""
import ctypes as C

import numpy as np

from . import vlb as _vlb

VLB_NN_F32, VLB_NN_BF16 = 0, 1
_done = False


def load():
    global _done
    lib = _vlb.load()
    if not _done:
        vp = C.c_void_p
        sig = {
            "vlb_nn_create": ([C.c_int32] * 6 + [C.c_int32, C.c_uint64, C.POINTER(vp)], C.c_int),
            "vlb_nn_num_params": ([vp, C.POINTER(C.c_int64)], C.c_int),
            "vlb_nn_get_params": ([vp, vp], C.c_int),
            "vlb_nn_set_params": ([vp, vp], C.c_int),
            "vlb_nn_forward": ([vp, vp, vp, C.c_int32], C.c_int),
            "vlb_nn_set_tensor_cores": ([vp, C.c_int32], C.c_int),
            "vlb_nn_mse": ([vp, vp, vp, vp, C.c_int32, C.POINTER(C.c_double)], C.c_int),
            "vlb_nn_backward": ([vp, vp, C.c_int32], C.c_int),
            "vlb_nn_get_grads": ([vp, vp], C.c_int),
            "vlb_nn_adam": ([vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int64], C.c_int),
            "vlb_nn_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _done = True
    return lib


def _check(rc, what):
    if rc != 0:
        raise _vlb.VlbError(rc, what, _vlb.load().vlb_last_error().decode())


class Net:
    """The U-Net of include/vlb_nn.h."""

    def __init__(self, in_ch, out_ch, width, H, W, max_batch, storage=VLB_NN_F32, seed=1):
        lib = load()
        h = C.c_void_p()
        _check(lib.vlb_nn_create(in_ch, out_ch, width, H, W, max_batch, storage, seed, C.byref(h)),
               "vlb_nn_create")
        self.h = h
        self.shape = (in_ch, out_ch, width, H, W, max_batch)
        n = C.c_int64()
        _check(lib.vlb_nn_num_params(h, C.byref(n)), "vlb_nn_num_params")
        self.nparams = n.value

    def params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _check(load().vlb_nn_get_params(self.h, p.ctypes.data), "vlb_nn_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load().vlb_nn_set_params(self.h, p.ctypes.data), "vlb_nn_set_params")

    def grads(self):
        g = np.zeros(self.nparams, dtype=np.float32)
        _check(load().vlb_nn_get_grads(self.h, g.ctypes.data), "vlb_nn_get_grads")
        return g

    def set_tensor_cores(self, enable):
        _check(load().vlb_nn_set_tensor_cores(self.h, 1 if enable else 0), "vlb_nn_set_tensor_cores")

    def forward(self, d_x, d_y, batch):
        _check(load().vlb_nn_forward(self.h, d_x, d_y, batch), "vlb_nn_forward")

    def mse(self, d_y, d_t, d_dy, batch):
        loss = C.c_double()
        _check(load().vlb_nn_mse(self.h, d_y, d_t, d_dy, batch, C.byref(loss)), "vlb_nn_mse")
        return loss.value

    def backward(self, d_dy, batch):
        _check(load().vlb_nn_backward(self.h, d_dy, batch), "vlb_nn_backward")

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load().vlb_nn_adam(self.h, lr, beta1, beta2, eps, t), "vlb_nn_adam")

    def close(self):
        if getattr(self, "h", None):
            load().vlb_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def layer_shapes(in_ch, out_ch, w):
    """(Cout, Cin, k) of the 11 layers, in parameter order."""
    return [(w, in_ch, 3), (w, w, 3), (2 * w, w, 3), (2 * w, 2 * w, 3), (4 * w, 2 * w, 3),
            (4 * w, 4 * w, 3), (2 * w, 6 * w, 3), (2 * w, 2 * w, 3), (w, 3 * w, 3), (w, w, 3),
            (out_ch, w, 1)]
