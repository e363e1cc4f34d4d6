"""ctypes binding of the surrogate network (include/sde_mlp.h) and its training loop.

The network, its gradients and the Adam updates run in libsde.so's kernels;
this module marshals arguments, draws the minibatch order on the device
(torch.randperm) and schedules the learning rate.  There is no CPU fallback.
"""
import ctypes
import math

import numpy as np

from . import engine

NPARAMS = 137992
IN, OUT = 7, 2
_sig_done = False


def _lib():
    global _sig_done
    L = engine.lib()
    if not _sig_done:
        P = ctypes.c_void_p
        f = ctypes.c_float
        sig = {
            "sde_mlp_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_uint64, P]),
            "sde_mlp_set_maps": (ctypes.c_int, [P, P, P, ctypes.c_uint32, P, P]),
            "sde_mlp_set_params": (ctypes.c_int, [P, P]),
            "sde_mlp_get_params": (ctypes.c_int, [P, P]),
            "sde_mlp_forward": (ctypes.c_int, [P, P, ctypes.c_uint64, P]),
            "sde_mlp_gradients": (ctypes.c_int, [P, P, P, ctypes.c_uint64, P,
                                                 ctypes.POINTER(ctypes.c_double)]),
            "sde_mlp_train_step": (ctypes.c_int, [P, P, P, ctypes.c_uint64, f, f, f, f, P]),
            "sde_mlp_fit": (ctypes.c_int, [P, P, P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                           f, f, f, f, f, ctypes.c_uint64, P]),
            "sde_mlp_gemm_bf16": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_uint32,
                                                 P, ctypes.c_uint32, P, ctypes.c_uint32]),
            "sde_guided_flags": (ctypes.c_int, [P, P, P, P, ctypes.c_uint32, ctypes.c_uint32, f, f, f,
                                                f, f, P, P]),
            "sde_mlp_set_tensor_path": (ctypes.c_int, [P, ctypes.c_int]),
            "sde_mlp_sync": (ctypes.c_int, [P]),
            "sde_mlp_destroy": (None, [P]),
            "sde_mlp_last_error": (ctypes.c_char_p, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sig_done = True
    return L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Surrogate:
    """MLP 7 -> 256 -> 256 -> 256 -> 2 (SiLU), BF16 tensor-core kernels, FP32 master weights."""

    def __init__(self, seed=0, stream=None):
        self._L = _lib()
        self._net = ctypes.c_void_p()
        rc = self._L.sde_mlp_create(ctypes.byref(self._net), int(seed), engine._stream_handle(stream))
        if rc != 0:
            raise engine.SdeError(rc, self._L.sde_mlp_last_error(None).decode())

    def _check(self, rc):
        if rc != 0:
            raise engine.SdeError(rc, self._L.sde_mlp_last_error(self._net).decode())

    def close(self):
        if self._net:
            self._L.sde_mlp_destroy(self._net)
            self._net = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_maps(self, shift, scale, log_mask, out_shift, out_scale):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (shift, scale, out_shift, out_scale)]
        self._maps = (a, int(log_mask))
        self._check(self._L.sde_mlp_set_maps(self._net, a[0].ctypes.data, a[1].ctypes.data,
                                             int(log_mask), a[2].ctypes.data, a[3].ctypes.data))

    def set_tensor_path(self, use_tcgen05):
        """1: the 256 x 256 forward layers on tcgen05 (default); 0: mma.sync."""
        self._check(self._L.sde_mlp_set_tensor_path(self._net, int(use_tcgen05)))

    def sync(self):
        """Wait for the stream; raises if a tensor-core wait ran out."""
        self._check(self._L.sde_mlp_sync(self._net))

    def get_params(self):
        out = np.zeros(NPARAMS, dtype=np.float32)
        self._check(self._L.sde_mlp_get_params(self._net, out.ctypes.data))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == NPARAMS
        self._check(self._L.sde_mlp_set_params(self._net, p.ctypes.data))

    def forward(self, x):
        """x: CUDA float32 tensor [M, 7] of raw parameters -> CUDA float32 [M, 2]."""
        import torch
        x = x.contiguous()
        y = torch.empty((x.shape[0], OUT), dtype=torch.float32, device=x.device)
        self._check(self._L.sde_mlp_forward(self._net, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def gradients(self, x, t):
        g = np.zeros(NPARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._L.sde_mlp_gradients(self._net, _ptr(x.contiguous()), _ptr(t.contiguous()),
                                              x.shape[0], g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, loss_out=None):
        self._check(self._L.sde_mlp_train_step(
            self._net, _ptr(x), _ptr(t), x.shape[0], float(lr), float(beta1), float(beta2),
            float(eps), _ptr(loss_out) if loss_out is not None else None))

    def fit(self, X, T, steps=8000, batch=512, lr=2e-3, lr_final=2e-5, seed=0,
            beta1=0.9, beta2=0.999, eps=1e-8):
        """Adam with a cosine learning-rate decay over `steps` minibatches drawn
        (on the device) from epochs in shuffled order, the whole loop in one
        sde_mlp_fit call.  X, T: CUDA float32 [N, 7] and [N, 2].  Returns the
        batch losses (numpy, one per step)."""
        import torch
        X = X.contiguous()
        T = T.contiguous()
        n = X.shape[0]
        batch = min(batch, n)
        losses = torch.zeros(steps, dtype=torch.float32, device=X.device)
        self._check(self._L.sde_mlp_fit(self._net, _ptr(X), _ptr(T), n, int(steps), int(batch), float(lr),
                                        float(lr_final), float(beta1), float(beta2), float(eps), int(seed),
                                        _ptr(losses)))
        return losses.cpu().numpy()

    def gemm_bf16(self, a_layout, b_layout, M, N, K, A, B):
        """Test helper: C = op(A) op(B) on the tensor cores (A, B CUDA bfloat16)."""
        import torch
        C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
        self._check(self._L.sde_mlp_gemm_bf16(self._net, int(a_layout), int(b_layout), M, N, K,
                                              _ptr(A), A.shape[1], _ptr(B), B.shape[1], _ptr(C), N))
        return C
