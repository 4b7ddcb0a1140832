"""ctypes binding of the warm-start network (include/dtt_net.h): argument marshalling only.

Every method maps to one C entry point of the same name in libdtt; the forward, backward
and optimiser steps run in the library's CUDA kernels.
"""
import ctypes as C

import numpy as np

from . import dtt

NET_CIN = 16
EXPORTS = ["dtt_net_create", "dtt_net_destroy", "dtt_net_num_params", "dtt_net_get_params", "dtt_net_set_params",
           "dtt_net_loss_grad", "dtt_net_forward", "dtt_net_features", "dtt_net_train_step", "dtt_net_predict",
           "dtt_net_set_loss", "dtt_net_set_increment", "dtt_net_increment_features", "dtt_net_train_increment",
           "dtt_net_predict_increment", "dtt_net_loss_grad_increment", "dtt_net_layer_trace", "dtt_net_grad_increment",
           "dtt_net_apply_grad", "dtt_net_grad_step"]
_bound = False


def _lib():
    global _bound
    L = dtt.lib()
    if not _bound:
        P, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        L.dtt_net_create.argtypes = [C.POINTER(P), i32, i32, i32, C.c_uint64, P]
        L.dtt_net_destroy.argtypes = [P]
        L.dtt_net_destroy.restype = None
        L.dtt_net_num_params.argtypes = [P]
        L.dtt_net_num_params.restype = i64
        L.dtt_net_get_params.argtypes = [P, P]
        L.dtt_net_set_params.argtypes = [P, P]
        L.dtt_net_loss_grad.argtypes = [P, i32, i32, i32, P, P, C.POINTER(C.c_double), P]
        L.dtt_net_forward.argtypes = [P, i32, i32, i32, P, P]
        L.dtt_net_features.argtypes = [P, P, P]
        L.dtt_net_train_step.argtypes = [P, P, P, f32, C.POINTER(C.c_double)]
        L.dtt_net_predict.argtypes = [P, P]
        L.dtt_net_set_loss.argtypes = [P, f32]
        L.dtt_net_set_increment.argtypes = [P, f32, f32, i32, i32]
        L.dtt_net_increment_features.argtypes = [P, P, P, P, P, P]
        L.dtt_net_train_increment.argtypes = [P, P, P, P, P, P, P, f32, C.POINTER(C.c_double)]
        L.dtt_net_grad_increment.argtypes = [P, P, P, P, P, P, P, P, C.POINTER(C.c_double)]
        L.dtt_net_apply_grad.argtypes = [P, P, f32, f32]
        L.dtt_net_grad_step.argtypes = [P, P, P, P, C.POINTER(C.c_double)]
        L.dtt_net_predict_increment.argtypes = [P, P, P, P, P]
        L.dtt_net_loss_grad_increment.argtypes = [P, i32, i32, i32, P, P, P, C.POINTER(C.c_double), P]
        L.dtt_net_layer_trace.argtypes = [P, i32, i32, i32, P, P, i32, P, P, P, P, P]
        for name in ("dtt_net_create", "dtt_net_get_params", "dtt_net_set_params", "dtt_net_loss_grad",
                     "dtt_net_forward", "dtt_net_features", "dtt_net_train_step", "dtt_net_predict",
                     "dtt_net_set_loss", "dtt_net_set_increment", "dtt_net_increment_features",
                     "dtt_net_train_increment", "dtt_net_predict_increment", "dtt_net_loss_grad_increment",
                     "dtt_net_layer_trace"):
            getattr(L, name).restype = i32
        _bound = True
    return L


def layer_shapes(c1=16, c2=32, c3=64):
    """(cin, cout) of the eleven convolutions in the order of include/dtt_net.h."""
    return [(16, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c2), (c2, c2), (c2, c1), (c1, c1),
            (c1, 16)]


def _torch():
    import torch
    return torch


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Net:
    """dtt_net: channels (c1, c2, c3) at full, 1/2 and 1/4 resolution."""

    def __init__(self, c1=16, c2=32, c3=64, seed=0, stream=None):
        L = _lib()
        self._h = C.c_void_p()
        dtt._check(L.dtt_net_create(C.byref(self._h), int(c1), int(c2), int(c3), int(seed),
                                    C.c_void_p(stream) if stream else None))
        self.channels = (c1, c2, c3)

    def close(self):
        if self._h:
            _lib().dtt_net_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(_lib().dtt_net_num_params(self._h))

    def get_params(self):
        p = np.zeros(self.num_params, np.float32)
        dtt._check(_lib().dtt_net_get_params(self._h, p.ctypes.data_as(C.c_void_p)))
        return p

    def set_params(self, p):
        p = _f32(p)
        assert p.size == self.num_params
        dtt._check(_lib().dtt_net_set_params(self._h, p.ctypes.data_as(C.c_void_p)))

    def set_loss(self, grad_weight):
        dtt._check(_lib().dtt_net_set_loss(self._h, float(grad_weight)))

    def loss_grad(self, x, target):
        """x: [nz, ny, nx, 16], target: [nz, ny, nx, 3] -> (loss, grad[num_params])."""
        x, t = _f32(x), _f32(target)
        nz, ny, nx = x.shape[:3]
        loss = C.c_double()
        g = np.zeros(self.num_params, np.float32)
        dtt._check(_lib().dtt_net_loss_grad(self._h, nx, ny, nz, x.ctypes.data_as(C.c_void_p),
                                            t.ctypes.data_as(C.c_void_p), C.byref(loss),
                                            g.ctypes.data_as(C.c_void_p)))
        return loss.value, g

    def layer_trace(self, x, target, layer):
        """For layer `layer` of the loss_grad pass on (x, target): its input activation
        [nz', ny', nx', cin], the output gradient through its ReLU [nz', ny', nx', cout] (both
        the BF16 values the kernels used), its gradients (W [27, cout, cin], b [cout]) and the
        gradient with respect to its input [nz', ny', nx', cin], at the layer's level."""
        x, t = _f32(x), _f32(target)
        nz, ny, nx = x.shape[:3]
        lvl = 2 if layer in (4, 5) else (1 if 2 <= layer <= 7 else 0)
        dims = (nz, ny, nx)
        for _ in range(lvl):
            dims = tuple((v + 1) // 2 for v in dims)
        cin, cout = layer_shapes(*self.channels)[layer]
        a = np.zeros(dims + (cin,), np.float32)
        dz = np.zeros(dims + (cout,), np.float32)
        gw = np.zeros((27, cout, cin), np.float32)
        gb = np.zeros(cout, np.float32)
        gx = np.zeros(dims + (cin,), np.float32)
        dtt._check(_lib().dtt_net_layer_trace(self._h, nx, ny, nz, x.ctypes.data_as(C.c_void_p),
                                              t.ctypes.data_as(C.c_void_p), int(layer),
                                              a.ctypes.data_as(C.c_void_p), dz.ctypes.data_as(C.c_void_p),
                                              gw.ctypes.data_as(C.c_void_p), gb.ctypes.data_as(C.c_void_p),
                                              gx.ctypes.data_as(C.c_void_p)))
        return a, dz, gw, gb, gx

    def forward(self, x):
        x = _f32(x)
        nz, ny, nx = x.shape[:3]
        out = np.zeros((nz, ny, nx, 3), np.float32)
        dtt._check(_lib().dtt_net_forward(self._h, nx, ny, nz, x.ctypes.data_as(C.c_void_p),
                                          out.ctypes.data_as(C.c_void_p)))
        return out

    def features(self, grid):
        nn = grid.node_shape   # (nz, ny, nx)
        x = np.zeros(tuple(nn) + (NET_CIN,), np.float32)
        dtt._check(_lib().dtt_net_features(self._h, grid._h, x.ctypes.data_as(C.c_void_p)))
        return x

    def train_step(self, grid, u_target, lr):
        """u_target: (3,) + node_shape float64 (the solver's converged u~)."""
        u = np.ascontiguousarray(u_target, dtype=np.float64)
        loss = C.c_double()
        dtt._check(_lib().dtt_net_train_step(self._h, grid._h, u.ctypes.data_as(C.c_void_p), float(lr),
                                             C.byref(loss)))
        return loss.value

    def grad_step(self, grid, u_target, grad):
        """Loss of one grid; its gradient goes into grad (a float32 CUDA tensor of num_params
        values), the parameters stay as they are."""
        if grad.dtype != _torch().float32 or grad.numel() != self.num_params:
            raise ValueError("grad: float32 CUDA tensor of num_params values")
        u = np.ascontiguousarray(u_target, dtype=np.float64)
        loss = C.c_double()
        dtt._check(_lib().dtt_net_grad_step(self._h, grid._h, u.ctypes.data_as(C.c_void_p), self._dev(grad),
                                            C.byref(loss)))
        return loss.value

    def predict(self, grid):
        """Writes the network's guess of u~ into the grid (solve with init=INIT_GUESS)."""
        dtt._check(_lib().dtt_net_predict(self._h, grid._h))

    # ---- increment mode (include/dtt_net.h): device arrays are torch CUDA tensors, complete
    # before the call (the library reads them on its own stream)
    def set_increment(self, pressure_weight=1.0, active_threshold=0.05, window_lateral=0, window_depth=0):
        dtt._check(_lib().dtt_net_set_increment(self._h, float(pressure_weight), float(active_threshold),
                                                int(window_lateral), int(window_depth)))
        self.window = (int(window_lateral), int(window_depth))

    @staticmethod
    def _dev(t):
        if t is None:
            return None
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
            raise ValueError("increment-mode arrays are contiguous CUDA tensors")
        return C.c_void_p(t.data_ptr())

    def increment_features(self, grid, u_prev2, fn_prev, depth):
        """Features of the window (the whole grid unless set_increment gave one, the
        contact face being the top z face)."""
        lat, dep = getattr(self, "window", (0, 0))
        nz, ny, nx = grid.node_shape
        shape = (dep if 0 < dep < nz else nz, lat if 0 < lat < ny else ny, lat if 0 < lat < nx else nx)
        x = np.zeros(shape + (NET_CIN,), np.float32)
        d = np.ascontiguousarray(depth, dtype=np.float64)
        dtt._check(_lib().dtt_net_increment_features(self._h, grid._h, self._dev(u_prev2), self._dev(fn_prev),
                                                     d.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p)))
        return x

    def train_increment(self, grid, u_prev2, fn_prev, depth, u_target, fn_target, lr):
        d = np.ascontiguousarray(depth, dtype=np.float64)
        loss = C.c_double()
        dtt._check(_lib().dtt_net_train_increment(self._h, grid._h, self._dev(u_prev2), self._dev(fn_prev),
                                                  d.ctypes.data_as(C.c_void_p), self._dev(u_target),
                                                  self._dev(fn_target), float(lr), C.byref(loss)))
        return loss.value

    def grad_increment(self, grid, u_prev2, fn_prev, depth, u_target, fn_target, grad):
        """Loss of increment k; its gradient goes into grad (a float32 CUDA tensor of
        num_params values), the parameters stay as they are."""
        if grad.dtype != _torch().float32 or grad.numel() != self.num_params:
            raise ValueError("grad: float32 CUDA tensor of num_params values")
        d = np.ascontiguousarray(depth, dtype=np.float64)
        loss = C.c_double()
        dtt._check(_lib().dtt_net_grad_increment(self._h, grid._h, self._dev(u_prev2), self._dev(fn_prev),
                                                 d.ctypes.data_as(C.c_void_p), self._dev(u_target),
                                                 self._dev(fn_target), self._dev(grad), C.byref(loss)))
        return loss.value

    def apply_grad(self, grad, scale, lr):
        """One Adam step with the gradient scale * grad (a float32 CUDA tensor of num_params
        values, e.g. the sum of the ranks' gradients with scale 1 / their number).  Torch's
        current stream is synchronised first, since the library reads grad on its own."""
        if grad.dtype != _torch().float32 or grad.numel() != self.num_params:
            raise ValueError("grad: float32 CUDA tensor of num_params values")
        p = self._dev(grad)
        _torch().cuda.current_stream().synchronize()
        dtt._check(_lib().dtt_net_apply_grad(self._h, p, float(scale), float(lr)))

    def predict_increment(self, grid, u_prev2, fn_prev, depth):
        d = np.ascontiguousarray(depth, dtype=np.float64)
        dtt._check(_lib().dtt_net_predict_increment(self._h, grid._h, self._dev(u_prev2), self._dev(fn_prev),
                                                    d.ctypes.data_as(C.c_void_p)))

    def loss_grad_increment(self, x, target, pmask):
        """x: [nz, ny, nx, 16], target: [nz, ny, nx, 4], pmask: [nz, ny, nx] -> (loss, grad)."""
        x, t, m = _f32(x), _f32(target), _f32(pmask)
        nz, ny, nx = x.shape[:3]
        loss = C.c_double()
        g = np.zeros(self.num_params, np.float32)
        dtt._check(_lib().dtt_net_loss_grad_increment(self._h, nx, ny, nz, x.ctypes.data_as(C.c_void_p),
                                                      t.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                                      C.byref(loss), g.ctypes.data_as(C.c_void_p)))
        return loss.value, g
