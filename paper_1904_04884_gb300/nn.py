"""ctypes binding of the warm-start network's layer operations (rihv_nn.h).

Argument marshalling only: tensors in, raw pointers out, status checked. BF16
tensors are torch.bfloat16 CUDA tensors (passed as their bit patterns).
"""
from __future__ import annotations

import ctypes

from .rihv import RihvError, load_library

_sigs_done = False


def _lib():
    global _sigs_done
    L = load_library()
    if not _sigs_done:
        vp, i, f, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        sig = {
            "rihv_nn_conv3d": (i, [vp, vp, vp, vp, i, i, i, i, i, i, i, vp, vp]),
            "rihv_nn_conv3d_dgrad": (i, [vp, vp, vp, i, i, i, i, i, i, vp, vp]),
            "rihv_nn_conv3d_wgrad_workspace": (sz, [i, i, i, i, i]),
            "rihv_nn_conv3d_wgrad": (i, [vp, vp, vp, i, i, i, i, i, vp, sz, vp, vp]),
            "rihv_nn_bias_grad": (i, [vp, vp, sz, i, vp, vp]),
            "rihv_nn_relu_grad": (i, [vp, vp, vp, sz, vp]),
            "rihv_nn_avgpool2": (i, [vp, vp, i, i, i, i, vp]),
            "rihv_nn_avgpool2_grad": (i, [vp, vp, i, i, i, i, vp]),
            "rihv_nn_upsample2": (i, [vp, vp, i, i, i, i, vp]),
            "rihv_nn_upsample2_grad": (i, [vp, vp, i, i, i, i, vp]),
            "rihv_nn_add": (i, [vp, vp, vp, sz, vp]),
            "rihv_nn_concat": (i, [vp, vp, vp, sz, i, i, vp]),
            "rihv_nn_split": (i, [vp, vp, vp, sz, i, i, vp]),
            "rihv_nn_pack_input": (i, [vp, vp, sz, i, f, vp]),
            "rihv_nn_unpack_output": (i, [vp, vp, f, vp, sz, i, f, vp]),
            "rihv_nn_mse_grad": (i, [vp, vp, vp, vp, sz, i, f, vp, vp]),
            "rihv_nn_adam": (i, [vp, vp, vp, vp, vp, sz, f, f, f, f, i, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sigs_done = True
    return L


def _p(t):
    return None if t is None else t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ok(st, what):
    if st != 0:
        raise RihvError(st, what)


def conv3d(x, w, bias, y, dims, c_in, c_out, relu, err):
    d, h, wd = dims
    _ok(_lib().rihv_nn_conv3d(_p(x), _p(w), _p(bias), _p(y), d, h, wd, c_in, c_out, int(relu),
                              int(y.dtype.is_floating_point and y.element_size() == 4), _p(err),
                              _stream()), "rihv_nn_conv3d")


def conv3d_dgrad(gy, w, gx, dims, c_in, c_out, err):
    d, h, wd = dims
    _ok(_lib().rihv_nn_conv3d_dgrad(_p(gy), _p(w), _p(gx), d, h, wd, c_in, c_out,
                                    int(gx.element_size() == 4), _p(err), _stream()),
        "rihv_nn_conv3d_dgrad")


def wgrad_workspace_bytes(dims, c_in, c_out):
    d, h, wd = dims
    return int(_lib().rihv_nn_conv3d_wgrad_workspace(d, h, wd, c_in, c_out))


def conv3d_wgrad(x, gy, gw, dims, c_in, c_out, work, err):
    d, h, wd = dims
    _ok(_lib().rihv_nn_conv3d_wgrad(_p(x), _p(gy), _p(gw), d, h, wd, c_in, c_out, _p(work),
                                    work.numel() * work.element_size(), _p(err), _stream()),
        "rihv_nn_conv3d_wgrad")


def bias_grad(gy, gb, voxels, c, work):
    _ok(_lib().rihv_nn_bias_grad(_p(gy), _p(gb), voxels, c, _p(work), _stream()), "rihv_nn_bias_grad")


def relu_grad(g, y, out):
    _ok(_lib().rihv_nn_relu_grad(_p(g), _p(y), _p(out), g.numel(), _stream()), "rihv_nn_relu_grad")


def avgpool2(x, y, dims, c):
    _ok(_lib().rihv_nn_avgpool2(_p(x), _p(y), *dims, c, _stream()), "rihv_nn_avgpool2")


def avgpool2_grad(gy, gx, dims, c):
    _ok(_lib().rihv_nn_avgpool2_grad(_p(gy), _p(gx), *dims, c, _stream()), "rihv_nn_avgpool2_grad")


def upsample2(x, y, dims, c):
    _ok(_lib().rihv_nn_upsample2(_p(x), _p(y), *dims, c, _stream()), "rihv_nn_upsample2")


def upsample2_grad(gy, gx, dims, c):
    _ok(_lib().rihv_nn_upsample2_grad(_p(gy), _p(gx), *dims, c, _stream()), "rihv_nn_upsample2_grad")


def add(a, b, out):
    _ok(_lib().rihv_nn_add(_p(a), _p(b), _p(out), a.numel(), _stream()), "rihv_nn_add")


def concat(a, b, out, voxels, ca, cb):
    _ok(_lib().rihv_nn_concat(_p(a), _p(b), _p(out), voxels, ca, cb, _stream()), "rihv_nn_concat")


def split(g, ga, gb, voxels, ca, cb):
    _ok(_lib().rihv_nn_split(_p(g), _p(ga), _p(gb), voxels, ca, cb, _stream()), "rihv_nn_split")


def pack_input(vol, out, voxels, c, scale):
    _ok(_lib().rihv_nn_pack_input(_p(vol), _p(out), voxels, c, float(scale), _stream()),
        "rihv_nn_pack_input")


def unpack_output(y, vol, voxels, c, scale, base=None, base_scale=0.0):
    _ok(_lib().rihv_nn_unpack_output(_p(y), _p(base), float(base_scale), _p(vol), voxels, c,
                                     float(scale), _stream()), "rihv_nn_unpack_output")


def mse_grad(y, target, gy, loss, voxels, c, scale, work):
    _ok(_lib().rihv_nn_mse_grad(_p(y), _p(target), _p(gy), _p(loss), voxels, c, float(scale),
                                _p(work), _stream()), "rihv_nn_mse_grad")


def adam(param, grad, m, v, param_bf16, lr, beta1, beta2, eps, step):
    _ok(_lib().rihv_nn_adam(_p(param), _p(grad), _p(m), _p(v), _p(param_bf16), param.numel(),
                            float(lr), float(beta1), float(beta2), float(eps), int(step), _stream()),
        "rihv_nn_adam")
