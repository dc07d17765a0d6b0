"""Python binding of the warm-start network (include/spirit_gb_unet.h).

Argument marshalling only: every forward, backward and update step runs in
the CUDA library.  BF16 tensors are passed as their bit patterns.
"""
import ctypes as C

import numpy as np
import torch

from .binding import SpinError, _ptr, _stream, lib

SP_ERR_ARG = -1


def _p(t):
    return C.c_void_p(0) if t is None else _ptr(t)


def _check_cuda(t, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dtype))


def set_conv_kernel(name):
    """'tcgen05_halo' (default: the input of a band of image rows staged once
    per channel chunk, the nine taps as offsets into it, for rows of at least
    64 pixels; 'tcgen05' below), 'tcgen05' (tensor-memory accumulators, a
    four-stage pipeline of one tap x 32 channels), 'tcgen05_ws' (the same
    with warp-specialised loads and MMA issue) or 'mma' (mma.sync)."""
    rc = lib().sp_conv3x3_set_kernel({"mma": 0, "tcgen05": 1, "tcgen05_ws": 2, "tcgen05_halo": 3}[name])
    if rc:
        raise SpinError(rc, "bad kernel name")


def conv_kernel():
    return {0: "mma", 1: "tcgen05", 2: "tcgen05_ws", 3: "tcgen05_halo"}[lib().sp_conv3x3_get_kernel()]


def check_device_error():
    """Raise if a convolution CTA gave up a bounded wait since the last check."""
    rc = lib().sp_unet_device_error()
    if rc:
        raise SpinError(rc, "a tensor-core pipeline wait timed out (outputs not written)")


def set_wait_limit(cycles=1 << 32):
    """Cycles a pipeline wait of the tcgen05 convolution polls before its CTA
    gives up (0: at once); the default is 2^32."""
    rc = lib().sp_conv3x3_set_wait_limit(int(cycles))
    if rc:
        raise SpinError(rc, "bad wait limit")


def n_params():
    return int(lib().sp_unet_n_params())


def layer(index):
    """(cout, cin, weight offset, bias offset) of convolution `index` (14 = head)."""
    co, ci, wo, bo = C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong()
    rc = lib().sp_unet_layer(index, C.byref(co), C.byref(ci), C.byref(wo), C.byref(bo))
    if rc:
        raise SpinError(rc, "no layer %d" % index)
    return co.value, ci.value, wo.value, bo.value


class UNet:
    """The network for L x L lattices and batches of at most `batch_max`."""

    def __init__(self, L, batch_max, params=None):
        h = C.c_void_p()
        rc = lib().sp_unet_create(C.byref(h), int(L), int(batch_max))
        if rc:
            raise SpinError(rc, "sp_unet_create(L=%d, batch_max=%d) failed" % (L, batch_max))
        self._h = h
        self.L = int(L)
        self.batch_max = int(batch_max)
        self.n_params = n_params()
        self._loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.steps = 0
        if params is not None:
            self.set_params(params)

    def _check(self, rc):
        if rc:
            raise SpinError(rc, lib().sp_unet_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().sp_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(lib().sp_unet_set_params(self._h, flat.ctypes.data_as(C.c_void_p), flat.size))
        self.steps = 0

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._check(lib().sp_unet_get_params(self._h, out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def predict(self, spins, features, out=None):
        """spins [B, L*L, 4] float32 CUDA, features [B, 4] -> [B, L*L, 4]."""
        _check_cuda(spins, torch.float32, "spins")
        _check_cuda(features, torch.float32, "features")
        out = torch.empty_like(spins) if out is None else out
        self._check(lib().sp_unet_predict(self._h, _ptr(spins), _ptr(features), spins.shape[0], _ptr(out), _stream()))
        return out

    def loss_grad(self, spins, features, target, grad=None):
        """Loss (device double tensor of 1) and, if `grad` is given, the flat
        FP32 gradient copied into it."""
        for t, n in ((spins, "spins"), (features, "features"), (target, "target")):
            _check_cuda(t, torch.float32, n)
        self._check(lib().sp_unet_loss_grad(self._h, _ptr(spins), _ptr(features), _ptr(target), spins.shape[0],
                                            _ptr(self._loss), _p(grad), _stream()))
        return self._loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.steps += 1
        self._check(lib().sp_unet_adam(self._h, float(lr), float(beta1), float(beta2), float(eps), self.steps,
                                       _stream()))

    def train_step(self, spins, features, target, lr, **kw):
        loss = self.loss_grad(spins, features, target)
        self.adam(lr, **kw)
        return loss


# ------------------------------------------------------------------ single kernels
def conv3x3_forward(src0, W, bias=None, relu=False, mask=None, src1=None, up0=False, cout=None):
    """src0 [B, h, w, C0] bf16 (h = H/2 when up0), src1 [B, H, W, C1] or None,
    W [Cout, 9, C0 + C1] bf16 -> [B, H, W, Cout] bf16."""
    B = src0.shape[0]
    H, Wd = (src0.shape[1] * 2, src0.shape[2] * 2) if up0 else (src0.shape[1], src0.shape[2])
    C0 = src0.shape[3]
    C1 = 0 if src1 is None else src1.shape[3]
    cout = W.shape[0] if cout is None else cout
    out = torch.empty((B, H, Wd, cout), dtype=torch.bfloat16, device=src0.device)
    rc = lib().sp_conv3x3_forward(_ptr(src0), C0, int(bool(up0)), _p(src1), C1, _ptr(W), _p(bias), int(bool(relu)),
                                  _p(mask), B, H, Wd, cout, _ptr(out), _stream())
    if rc:
        raise SpinError(rc, "sp_conv3x3_forward rejected the shapes")
    return out


def conv3x3_transpose(W):
    Co, _, Ci = W.shape
    Wt = torch.empty((Ci, 9, Co), dtype=torch.bfloat16, device=W.device)
    rc = lib().sp_conv3x3_transpose(_ptr(W), Co, Ci, _ptr(Wt), _stream())
    if rc:
        raise SpinError(rc, "sp_conv3x3_transpose failed")
    return Wt


def conv3x3_wgrad(src0, dz, src1=None, up0=False, bias_grad=True):
    """(dW [Cout, 9, Cin] float32, db [Cout] float32 or None)."""
    B, H, Wd, Cout = dz.shape
    C0 = src0.shape[3]
    C1 = 0 if src1 is None else src1.shape[3]
    ws_bytes = int(lib().sp_conv3x3_wgrad_workspace(B, H, Wd, C0 + C1, Cout))
    ws = torch.empty(max(ws_bytes // 4, 1), dtype=torch.float32, device=dz.device)
    dW = torch.empty((Cout, 9, C0 + C1), dtype=torch.float32, device=dz.device)
    db = torch.empty(Cout, dtype=torch.float32, device=dz.device) if bias_grad else None
    rc = lib().sp_conv3x3_wgrad(_ptr(src0), C0, int(bool(up0)), _p(src1), C1, _ptr(dz), B, H, Wd, Cout, _ptr(dW),
                                _p(db), _ptr(ws), ws_bytes, _stream())
    if rc:
        raise SpinError(rc, "sp_conv3x3_wgrad rejected the shapes")
    return dW, db
