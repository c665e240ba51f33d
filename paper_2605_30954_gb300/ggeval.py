"""Python binding of the ggeval C ABI (include/ggeval.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library ``_lib/libggeval.so``.  PyTorch tensors provide device memory,
pinned host memory and streams.  Importing this module without the built
library raises ImportError; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libggeval.so")

OK, ERR_ARG, ERR_TEMPLATE, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_CHECKED, ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
LAYOUT_HEAP, LAYOUT_PREFIX = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
F_GRAPH, F_EXACT, F_GRAD_MSE, F_PROFILE, F_POW, F_NO_FOLD, F_TEST_STALL = 1, 2, 4, 8, 16, 32, 64
NSTAT = 25
MAX_HEIGHT = 8

#: every symbol the header declares
SYMBOLS = ("ggeval_create_dataset", "ggeval_destroy", "ggeval_eval_batch", "ggeval_eval_rows",
           "ggeval_eval_plain", "ggeval_grad_batch", "ggeval_adam_step", "ggeval_autotune",
           "ggeval_sync", "ggeval_last_error", "ggeval_batch_stats", "ggeval_pack_host",
           "ggeval_pack_device",
           "ggeval_version", "ggeval_profile_read", "ggeval_eval_batch_noalloc",
           "ggeval_eval_batch_masked", "ggeval_gom_donate", "ggeval_gom_changed",
           "ggeval_gom_accept", "ggeval_trial_sizes", "ggeval_dataset_info",
           "ggeval_tile_config", "ggeval_pipe_rates", "ggeval_evaluate", "ggeval_tuning_save",
           "ggeval_tuning_load")


class GGEvalError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ggeval status {status}: {msg}")
        self.status = status


class Outputs(ctypes.Structure):
    _fields_ = [("smse", ctypes.c_void_p), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("mse", ctypes.c_void_p), ("nmse", ctypes.c_void_p), ("size", ctypes.c_void_p),
                ("size_evaluated", ctypes.c_void_p)]


class Batch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("max_height", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("memory", ctypes.c_int32),
                ("op", ctypes.c_void_p), ("cval", ctypes.c_void_p),
                ("height", ctypes.c_void_p)]


def load_library(path: str = LIB_PATH, strict: bool = True):
    """Load the library at `path`; with strict False, entry points the build
    does not export are left out (an older build)."""
    if not os.path.exists(path):
        raise ImportError(f"ggeval CUDA library not built: {path} is missing "
                          "(run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32, u32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                              ctypes.c_float, ctypes.c_uint32)
    bp = ctypes.POINTER(Batch)
    sig = {
        "ggeval_create_dataset": [vp, vp, i64, i32, i32, i32, vp, ctypes.POINTER(vp)],
        "ggeval_destroy": [vp],
        "ggeval_eval_batch": [vp, bp, u32, vp, vp, vp, vp, vp],
        "ggeval_eval_rows": [vp, bp, u32, vp, vp],
        "ggeval_eval_plain": [vp, bp, u32, vp, vp, vp, vp, vp],
        "ggeval_grad_batch": [vp, bp, u32, vp, vp, vp],
        "ggeval_adam_step": [bp, vp, vp, vp, vp, i32, f32, f32, f32, f32, vp],
        "ggeval_autotune": [vp, bp, u32, vp],
        "ggeval_sync": [vp, vp],
        "ggeval_last_error": [],
        "ggeval_batch_stats": [bp, i32, vp],
        "ggeval_pack_host": [bp, i32, i32, vp, vp, vp, i32, vp],
        "ggeval_pack_device": [vp, bp, u32, vp, vp, vp, i32, vp],
        "ggeval_version": [],
        "ggeval_profile_read": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)],
        "ggeval_eval_batch_noalloc": [vp, bp, vp, vp, vp, vp, vp],
        "ggeval_eval_batch_masked": [vp, bp, vp, u32, vp, vp, vp, vp, vp],
        "ggeval_gom_donate": [i32, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, i32, vp],
        "ggeval_gom_changed": [bp, vp, vp, i32, vp, vp],
        "ggeval_gom_accept": [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "ggeval_trial_sizes": [bp, i32, vp, vp],
        "ggeval_tile_config": [vp, bp, u32, vp, vp],
        "ggeval_pipe_rates": [i32, i32, vp],
        "ggeval_tuning_save": [vp, ctypes.c_char_p],
        "ggeval_tuning_load": [vp, ctypes.c_char_p, ctypes.POINTER(i32)],
        "ggeval_evaluate": [vp, bp, u32, ctypes.POINTER(Outputs), vp],
        "ggeval_dataset_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        if not strict and not hasattr(lib, name):
            continue
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ggeval_destroy.restype = None
    lib.ggeval_last_error.restype = ctypes.c_char_p
    lib.ggeval_version.restype = ctypes.c_char_p
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(status):
    if status != OK:
        raise GGEvalError(status, lib().ggeval_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_batch(op: torch.Tensor, cval: torch.Tensor, heights=None, max_height: int | None = None,
               layout: int = LAYOUT_HEAP) -> Batch:
    """Describe trial arrays as a ggeval_batch.  op uint8 [n, stride],
    cval float32 [n, stride], heights int8 [n] or None; all on one device
    (or all on the host, preferably pinned)."""
    n, stride = op.shape
    if max_height is None:
        max_height = (stride + 1).bit_length() - 2
    if (1 << (max_height + 1)) - 1 != stride:
        raise ValueError(f"stride {stride} is not 2**(h+1)-1")
    if op.dtype != torch.uint8 or cval.dtype != torch.float32 or tuple(cval.shape) != (n, stride):
        raise ValueError("op must be uint8 and cval float32 of the same shape")
    if not (op.is_contiguous() and cval.is_contiguous()):
        raise ValueError("op and cval must be contiguous")
    if heights is not None and (heights.dtype != torch.int8 or heights.numel() != n
                                or not heights.is_contiguous()):
        raise ValueError("heights must be contiguous int8 [n]")
    mem = MEM_DEVICE if op.is_cuda else MEM_HOST
    for t in (cval, heights):
        if t is not None and t.is_cuda != op.is_cuda:
            raise ValueError("batch arrays must all be on the device or all on the host")
    return Batch(n, max_height, layout, mem, op.data_ptr(), cval.data_ptr(),
                 None if heights is None else heights.data_ptr())


class Dataset:
    """A dataset resident on one GPU: X (N x F) and y (N), both float32."""

    def __init__(self, X: torch.Tensor, y: torch.Tensor, device: int | None = None,
                 stream=None):
        if X.dtype != torch.float32 or y.dtype != torch.float32:
            raise ValueError("X and y must be float32")
        X = X.contiguous()
        y = y.contiguous()
        if device is None:
            device = X.device.index if X.is_cuda else torch.cuda.current_device()
        self.device = device
        self.N, self.F = X.shape
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            _check(lib().ggeval_create_dataset(_ptr(X), _ptr(y), self.N, self.F, 1, device,
                                               _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().ggeval_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- evaluation ---------------------------------------------------------
    def _outs(self, n, like, want):
        kw = dict(dtype=torch.float32, device=like.device)
        if not like.is_cuda:
            kw["pin_memory"] = True
        return [torch.empty(n, **kw) if w else None for w in want]

    def eval_batch(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None,
                   out=None, want=(True, True, True, True)):
        """Scaled MSE, a, b and MSE of every trial (tensors on op's device)."""
        b = make_batch(op, cval, heights, layout=layout)
        outs = out if out is not None else self._outs(b.n, op, want)
        _check(lib().ggeval_eval_batch(self._h, ctypes.byref(b), flags, *map(_ptr, outs),
                                       _stream_handle(stream)))
        return outs

    #: the outputs of evaluate(), in the order of ggeval_outputs
    OUTPUTS = ("smse", "a", "b", "mse", "nmse", "size", "size_evaluated")

    def evaluate(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None,
                 want=OUTPUTS, out=None):
        """Every objective of every trial in one launch sequence: a dict
        name -> tensor [n] (float32; int32 for the sizes) on op's device,
        for the names in ``want`` (``out`` may supply the tensors)."""
        b = make_batch(op, cval, heights, layout=layout)
        kw = dict(device=op.device)
        if not op.is_cuda:
            kw["pin_memory"] = True
        res = dict(out or {})
        for name in want:
            if name not in res:
                dt = torch.int32 if name.startswith("size") else torch.float32
                res[name] = torch.empty(b.n, dtype=dt, **kw)
        o = Outputs(*[_ptr(res.get(name)) for name in self.OUTPUTS])
        _check(lib().ggeval_evaluate(self._h, ctypes.byref(b), flags, ctypes.byref(o),
                                     _stream_handle(stream)))
        return res

    def eval_plain(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None,
                   out=None):
        b = make_batch(op, cval, heights, layout=layout)
        outs = out if out is not None else self._outs(b.n, op, (True, True, True, True))
        _check(lib().ggeval_eval_plain(self._h, ctypes.byref(b), flags, *map(_ptr, outs),
                                       _stream_handle(stream)))
        return outs

    def eval_rows(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None):
        """Per-row values [n, N] from the configuration eval_batch would run
        with these flags."""
        b = make_batch(op, cval, heights, layout=layout)
        kw = dict(dtype=torch.float32, device=op.device)
        if not op.is_cuda:
            kw["pin_memory"] = True
        f = torch.empty((b.n, self.N), **kw)
        _check(lib().ggeval_eval_rows(self._h, ctypes.byref(b), flags, _ptr(f),
                                      _stream_handle(stream)))
        return f

    def tile_config(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, set=None):
        """(variant, rows per tile, trials per item, warps per CTA) that
        eval_batch uses for this batch shape; with ``set`` that tuple is
        checked and kept first."""
        b = make_batch(op, cval, heights, layout=layout)
        got = (ctypes.c_int32 * 4)()
        arr = None if set is None else (ctypes.c_int32 * 4)(*[int(x) for x in set])
        _check(lib().ggeval_tile_config(self._h, ctypes.byref(b), flags, arr, got))
        return tuple(got)

    def grad_batch(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None,
                   smse=None, dcval=None):
        """(smse [n], d fitness / d cval [n, stride])."""
        b = make_batch(op, cval, heights, layout=layout)
        kw = dict(dtype=torch.float32, device=op.device)
        if not op.is_cuda:
            kw["pin_memory"] = True
        if smse is None:
            smse = torch.empty(b.n, **kw)
        if dcval is None:
            dcval = torch.empty(tuple(cval.shape), **kw)
        _check(lib().ggeval_grad_batch(self._h, ctypes.byref(b), flags, _ptr(smse), _ptr(dcval),
                                       _stream_handle(stream)))
        return smse, dcval

    def eval_batch_masked(self, op, cval, mask, heights=None, layout=LAYOUT_HEAP, flags=0,
                          stream=None, out=None):
        """Evaluate only trials with mask != 0 (uint8 device tensor); the
        other entries of ``out`` are left as they are."""
        b = make_batch(op, cval, heights, layout=layout)
        outs = out if out is not None else self._outs(b.n, op, (True, True, True, True))
        _check(lib().ggeval_eval_batch_masked(self._h, ctypes.byref(b), _ptr(mask), flags,
                                              *map(_ptr, outs), _stream_handle(stream)))
        return outs

    def pack_device(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None):
        """The device packer's programs: (words uint32 [n, cap], consts
        float32 [n, cap], len int32 [n]), cap = the template stride."""
        b = make_batch(op, cval, heights, layout=layout)
        cap = op.shape[1]
        words = torch.zeros((b.n, cap), dtype=torch.int32)
        consts = torch.zeros((b.n, cap), dtype=torch.float32)
        ln = torch.zeros(b.n, dtype=torch.int32)
        _check(lib().ggeval_pack_device(self._h, ctypes.byref(b), flags, _ptr(words),
                                        _ptr(consts), _ptr(ln), cap, _stream_handle(stream)))
        return words.numpy().view("uint32"), consts.numpy(), ln.numpy()

    def autotune(self, op, cval, heights=None, layout=LAYOUT_HEAP, flags=0, stream=None):
        b = make_batch(op, cval, heights, layout=layout)
        _check(lib().ggeval_autotune(self._h, ctypes.byref(b), flags, _stream_handle(stream)))

    def tuning_save(self, path):
        """Write the autotuner's choices for this dataset to `path` (JSON lines)."""
        _check(lib().ggeval_tuning_save(self._h, os.fsencode(path)))

    def tuning_load(self, path):
        """Take the matching choices from `path`; returns how many."""
        n = ctypes.c_int32()
        _check(lib().ggeval_tuning_load(self._h, os.fsencode(path), ctypes.byref(n)))
        return n.value

    def sync(self, stream=None):
        _check(lib().ggeval_sync(self._h, _stream_handle(stream)))

    def info(self):
        """(rows, features, mean y, Var y) of the stored dataset."""
        n, f = ctypes.c_int64(), ctypes.c_int32()
        m, v = ctypes.c_double(), ctypes.c_double()
        _check(lib().ggeval_dataset_info(self._h, ctypes.byref(n), ctypes.byref(f),
                                         ctypes.byref(m), ctypes.byref(v)))
        return n.value, f.value, m.value, v.value

    def profile_read(self):
        """(total forward-kernel ms, launches) since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().ggeval_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


PIPE_KINDS = ("ffma", "ffma2", "rsqrt", "ex2", "lg2", "sin")


def pipe_rates(device=0, iters=1 << 14):
    """Operations per second of the issue-rate microbenchmarks, by kind
    (see ggeval_pipe_rates)."""
    out = (ctypes.c_double * len(PIPE_KINDS))()
    _check(lib().ggeval_pipe_rates(int(device), int(iters), out))
    return dict(zip(PIPE_KINDS, list(out)))


def adam_step(op, cval, grad, m, v, t, lr=0.05, beta1=0.9, beta2=0.999, eps=1e-8,
              stream=None):
    """One in-place Adam step on the ERC constants of a device batch."""
    b = make_batch(op, cval)
    _check(lib().ggeval_adam_step(ctypes.byref(b), _ptr(cval), _ptr(grad), _ptr(m), _ptr(v),
                                  int(t), lr, beta1, beta2, eps, _stream_handle(stream)))


def gom_donate(op, cval, pop_op, pop_cval, donor, subset, fos_offsets, fos_nodes, stream=None):
    """O_j[FOS[subset_j]] <- P_donor_j[FOS[subset_j]], in place (device tensors;
    donor, subset, fos_offsets, fos_nodes int32)."""
    n, stride = op.shape
    h = (stride + 1).bit_length() - 2
    _check(lib().ggeval_gom_donate(n, h, _ptr(op), _ptr(cval), _ptr(pop_op), _ptr(pop_cval),
                                   pop_op.shape[0], _ptr(donor), _ptr(subset), _ptr(fos_offsets),
                                   _ptr(fos_nodes), fos_offsets.numel() - 1,
                                   _stream_handle(stream)))


def gom_changed(op, cval, bop, bcval, n_features, heights=None, layout=LAYOUT_HEAP,
                stream=None):
    """uint8 [n]: 1 where an active part of the offspring differs from its backup."""
    b = make_batch(op, cval, heights, layout=layout)
    changed = torch.empty(b.n, dtype=torch.uint8, device=op.device)
    _check(lib().ggeval_gom_changed(ctypes.byref(b), _ptr(bop), _ptr(bcval), n_features,
                                    _ptr(changed), _stream_handle(stream)))
    return changed


def gom_accept(op, cval, bop, bcval, f_new, f_old, changed=None, stream=None):
    """Accept (backup <- offspring, f_old <- f_new) or revert (offspring <-
    backup) every trial in place; returns the uint8 accepted flags."""
    n, stride = op.shape
    h = (stride + 1).bit_length() - 2
    acc = torch.empty(n, dtype=torch.uint8, device=op.device)
    _check(lib().ggeval_gom_accept(n, h, _ptr(op), _ptr(cval), _ptr(bop), _ptr(bcval),
                                   _ptr(changed), _ptr(f_new), _ptr(f_old), _ptr(acc),
                                   _stream_handle(stream)))
    return acc


def trial_sizes(op, cval, n_features, heights=None, layout=LAYOUT_HEAP, stream=None):
    """int32 [n]: active node count of every trial (device batch)."""
    b = make_batch(op, cval, heights, layout=layout)
    size = torch.empty(b.n, dtype=torch.int32, device=op.device)
    _check(lib().ggeval_trial_sizes(ctypes.byref(b), n_features, _ptr(size),
                                    _stream_handle(stream)))
    return size


def batch_stats(op, cval, heights=None, layout=LAYOUT_HEAP, n_features=223):
    """int64 [n, NSTAT] node counts of a host batch (see the header)."""
    b = make_batch(op, cval, heights, layout=layout)
    out = torch.zeros((b.n, NSTAT), dtype=torch.int64)
    _check(lib().ggeval_batch_stats(ctypes.byref(b), n_features, _ptr(out)))
    return out


def pack_host(op, cval, index, heights=None, layout=LAYOUT_HEAP, n_features=223):
    """The packer on the CPU: (words, consts, template positions) of one trial."""
    b = make_batch(op, cval, heights, layout=layout)
    cap = op.shape[1]
    words = torch.zeros(cap, dtype=torch.int32)
    consts = torch.zeros(cap, dtype=torch.float32)
    tpos = torch.zeros(cap, dtype=torch.int32)
    n = ctypes.c_int32()
    _check(lib().ggeval_pack_host(ctypes.byref(b), index, n_features, _ptr(words), _ptr(consts),
                                  _ptr(tpos), cap, ctypes.byref(n)))
    L = n.value
    return words[:L].numpy().view("uint32"), consts[:L].numpy(), tpos[:L].numpy()


class ScaledMSE(torch.autograd.Function):
    """Scaled MSE of every trial as a differentiable function of cval.

    forward evaluates the fitness only (ggeval_eval_batch); backward runs
    the adjoint (ggeval_grad_batch, which evaluates the trials again on the
    way), so the adjoint costs nothing unless a gradient is asked for."""

    @staticmethod
    def forward(ctx, cval, op, dataset, heights=None, layout=LAYOUT_HEAP, flags=0):
        c = cval.detach().contiguous()
        smse = dataset.eval_batch(op, c, heights, layout, flags,
                                  want=(True, False, False, False))[0]
        ctx.save_for_backward(c, op)
        ctx.dataset, ctx.heights, ctx.layout, ctx.flags = dataset, heights, layout, flags
        return smse

    @staticmethod
    def backward(ctx, g):
        c, op = ctx.saved_tensors
        _, dc = ctx.dataset.grad_batch(op, c, ctx.heights, ctx.layout, ctx.flags)
        return dc * g[:, None], None, None, None, None, None
