"""Torch-facing binding of the TASER C ABI (argument marshalling only)."""
import ctypes

import torch

import numpy as np

from ._native import UnevenTuning, check, lib

BPSK, QPSK, JED_BPSK, JED_QPSK = 0, 1, 2, 3
KINDS = {"mimo_bpsk": BPSK, "mimo_qpsk": QPSK, "jed_bpsk": JED_BPSK, "jed_qpsk": JED_QPSK, BPSK: BPSK, QPSK: QPSK,
         JED_BPSK: JED_BPSK, JED_QPSK: JED_QPSK}
JED_KINDS = (JED_BPSK, JED_QPSK)
PRECISIONS = {"fp32": 0, "bf16_tc": 1, "fp16_tc": 2, "fixed14": 3}
LNN_MODES = {"fixed": 0, "literal": 1}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def problem_size(kind, U_or_K):
    return lib().taser_problem_size(KINDS[kind], int(U_or_K))


def build_T(kind, H_or_Y, y=None, alpha=0.5, out=None, stream=None, with_tau=True):
    """T~, D, tau (and ||T~||_2, flags) per instance from complex64 H [n,B,U] and
    y [n,B] (MIMO) or Y [n,B,K] (JED).  Returns a dict of device tensors.  With
    with_tau=False the step size is skipped (see step_size)."""
    k = KINDS[kind]
    X = _dev(H_or_Y, torch.complex64, "H_or_Y")
    n, B, M = X.shape
    if k not in JED_KINDS:
        _dev(y, torch.complex64, "y")
        if tuple(y.shape) != (n, B):
            raise ValueError("y must have shape [n, B]")
    N = problem_size(k, M)
    dev = X.device
    if out is None:
        out = {"T_tilde": torch.empty((n, N, N), device=dev, dtype=torch.float32),
               "D": torch.empty((n, N), device=dev, dtype=torch.float32),
               "tau": torch.empty((n,), device=dev, dtype=torch.float32),
               "spec_norm": torch.empty((n,), device=dev, dtype=torch.float32),
               "flags": torch.zeros((n,), device=dev, dtype=torch.int32)}
    st = lib().taser_build_T(k, n, B, M, _ptr(X), _ptr(y if k not in JED_KINDS else None), float(alpha),
                             _ptr(out["T_tilde"]), _ptr(out["D"]), _ptr(out["tau"] if with_tau else None),
                             _ptr(out.get("spec_norm")), _ptr(out.get("flags")), _stream(stream))
    check(st, "taser_build_T")
    return out


GENERIC = -1


def step_size(T_tilde, alpha=0.5, structure=GENERIC, tau=None, spec_norm=None, stream=None):
    """tau = alpha / ||T~||_2.  `structure`: a problem kind (what taser_build_T produced)
    or GENERIC.  Returns (tau, spec_norm)."""
    T = _dev(T_tilde, torch.float32, "T_tilde")
    n, N, _ = T.shape
    tau = tau if tau is not None else torch.empty((n,), device=T.device, dtype=torch.float32)
    nrm = spec_norm if spec_norm is not None else torch.empty((n,), device=T.device, dtype=torch.float32)
    s = KINDS[structure] if structure != GENERIC else GENERIC
    check(lib().taser_step_size(n, N, _ptr(T), s, float(alpha), _ptr(tau), _ptr(nrm), _stream(stream)),
          "taser_step_size")
    return tau, nrm


def detect(T_tilde, D, tau, t_max, precision="fp32", lnn_mode="fixed", want_L=True, flags=None,
           out_s=None, out_L=None, stream=None):
    """Algorithm 1 on every instance.  Returns (s_hat int8 [n,N-1], L or None, flags)."""
    T = _dev(T_tilde, torch.float32, "T_tilde")
    n, N, _ = T.shape
    _dev(D, torch.float32, "D")
    _dev(tau, torch.float32, "tau")
    s = out_s if out_s is not None else torch.empty((n, N - 1), device=T.device, dtype=torch.int8)
    L = out_L if out_L is not None else (
        torch.empty((n, N, N), device=T.device, dtype=torch.float32) if want_L else None)
    if flags is None:
        flags = torch.zeros((n,), device=T.device, dtype=torch.int32)
    st = lib().taser_detect(n, N, _ptr(T), _ptr(D), _ptr(tau), int(t_max), PRECISIONS[precision],
                            LNN_MODES[lnn_mode], _ptr(L), _ptr(s), _ptr(flags), _stream(stream))
    check(st, "taser_detect")
    return s, L, flags


FLAG_ASCENT = 1 << 6


def detect_monitored(T_tilde, D, tau, t_max, precision="fp32", ascent_tol=1e-5, lnn_mode="fixed", want_L=True,
                     want_objective=True, flags=None, stream=None):
    """detect() that also traces f(L~(t)) = Tr(L~ T~ L~^T), t = 0..t_max, and sets
    FLAG_ASCENT where it rose by more than ascent_tol |f|.  Returns (s_hat, L or None,
    flags, objective float64 [n, t_max + 1] or None)."""
    T = _dev(T_tilde, torch.float32, "T_tilde")
    n, N, _ = T.shape
    _dev(D, torch.float32, "D")
    _dev(tau, torch.float32, "tau")
    s = torch.empty((n, N - 1), device=T.device, dtype=torch.int8)
    L = torch.empty((n, N, N), device=T.device, dtype=torch.float32) if want_L else None
    obj = torch.empty((n, int(t_max) + 1), device=T.device, dtype=torch.float64) if want_objective else None
    if flags is None:
        flags = torch.zeros((n,), device=T.device, dtype=torch.int32)
    st = lib().taser_detect_monitored(n, N, _ptr(T), _ptr(D), _ptr(tau), int(t_max), PRECISIONS[precision],
                                      LNN_MODES[lnn_mode], float(ascent_tol), _ptr(obj), _ptr(L), _ptr(s),
                                      _ptr(flags), _stream(stream))
    check(st, "taser_detect_monitored")
    return s, L, flags, obj


def host_workspace_bytes(kind, batch, B, U_or_K):
    return int(lib().taser_host_workspace_bytes(KINDS[kind], int(batch), int(B), int(U_or_K)))


def run_host(kind, H_or_Y, y, alpha, t_max, precision, workspace, s_hat, flags=None, lnn_mode="fixed",
             stream=None):
    """End to end from host (ideally pinned) complex64 inputs to host int8 decisions.
    `workspace` is a uint8 CUDA tensor of at least host_workspace_bytes(...) bytes."""
    k = KINDS[kind]
    n, B, M = H_or_Y.shape
    for name, t in (("H_or_Y", H_or_Y), ("s_hat", s_hat)) + ((("y", y),) if k not in JED_KINDS else ()):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous host tensor" % name)
    _dev(workspace, torch.uint8, "workspace")
    st = lib().taser_run_host(k, n, B, M, _ptr(H_or_Y), _ptr(y if k not in JED_KINDS else None), float(alpha),
                              int(t_max), PRECISIONS[precision], LNN_MODES[lnn_mode], _ptr(workspace),
                              workspace.numel(), _ptr(s_hat), _ptr(flags), _stream(stream))
    check(st, "taser_run_host")


def run_host_static(kind, H_or_Y, y, alpha, t_max, precision, s_hat, flags=None, lnn_mode="fixed", stream=None):
    """run_host for callers that cannot allocate device memory: the workspace is the
    library's static device scratch (a batch must fit in it; see include/taser.h)."""
    k = KINDS[kind]
    n, B, M = H_or_Y.shape
    for name, t in (("H_or_Y", H_or_Y), ("s_hat", s_hat)) + ((("y", y),) if k not in JED_KINDS else ()):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous host tensor" % name)
    st = lib().taser_run_host_static(k, n, B, M, _ptr(H_or_Y), _ptr(y if k not in JED_KINDS else None), float(alpha),
                                     int(t_max), PRECISIONS[precision], LNN_MODES[lnn_mode], _ptr(s_hat),
                                     _ptr(flags), _stream(stream))
    check(st, "taser_run_host_static")


def unfolded_forward(T_tilde, D, inv_norm, alpha_t, c, want_ckpt=True, precision="fp32", stream=None):
    """Unfolded TASER forward (tau_t = alpha_t * inv_norm).  Returns (soft, s_hat, ckpt)."""
    T = _dev(T_tilde, torch.float32, "T_tilde")
    n, N, _ = T.shape
    for name, t in (("D", D), ("inv_norm", inv_norm), ("alpha_t", alpha_t)):
        _dev(t, torch.float32, name)
    t_max = alpha_t.numel()
    n_ck = -(-t_max // c)
    ckpt = torch.empty((n, n_ck, N, N), device=T.device, dtype=torch.float32) if want_ckpt else None
    soft = torch.empty((n, N - 1), device=T.device, dtype=torch.float32)
    s_hat = torch.empty((n, N - 1), device=T.device, dtype=torch.int8)
    check(lib().taser_unfolded_forward(n, N, _ptr(T), _ptr(D), _ptr(inv_norm), _ptr(alpha_t), t_max, int(c),
                                       PRECISIONS[precision], _ptr(ckpt), _ptr(soft), _ptr(s_hat), _stream(stream)),
          "taser_unfolded_forward")
    return soft, s_hat, ckpt


def unfolded_backward(T_tilde, D, inv_norm, alpha_t, c, ckpt, grad_soft, precision="fp32", stream=None):
    """Adjoint of unfolded_forward.  Returns (grad_tau [n, t_max], grad_alpha [t_max])."""
    T = _dev(T_tilde, torch.float32, "T_tilde")
    n, N, _ = T.shape
    t_max = alpha_t.numel()
    grad_soft = _dev(grad_soft.contiguous(), torch.float32, "grad_soft")
    grad_tau = torch.empty((n, t_max), device=T.device, dtype=torch.float32)
    grad_alpha = torch.empty((t_max,), device=T.device, dtype=torch.float32)
    check(lib().taser_unfolded_backward(n, N, _ptr(T), _ptr(D), _ptr(inv_norm), _ptr(alpha_t), t_max, int(c),
                                        PRECISIONS[precision], _ptr(ckpt), _ptr(grad_soft), _ptr(grad_tau),
                                        _ptr(grad_alpha), _stream(stream)), "taser_unfolded_backward")
    return grad_tau, grad_alpha


class UnfoldedTASER(torch.autograd.Function):
    """soft = UnfoldedTASER.apply(alpha_t, T_tilde, D, inv_norm, c[, precision]): the soft
    last row of unfolded TASER with learnable per-iteration steps alpha_t (gradient to
    alpha_t only; the decisions sign(soft) stay hard).  Checkpoints every c iterations."""

    @staticmethod
    def forward(ctx, alpha_t, T_tilde, D, inv_norm, c, precision="fp32"):
        a = alpha_t.detach().contiguous()
        soft, _, ckpt = unfolded_forward(T_tilde, D, inv_norm, a, c, want_ckpt=True, precision=precision)
        ctx.save_for_backward(a, T_tilde, D, inv_norm, ckpt)
        ctx.c = c
        ctx.precision = precision
        return soft

    @staticmethod
    def backward(ctx, grad_soft):
        a, T_tilde, D, inv_norm, ckpt = ctx.saved_tensors
        _, grad_alpha = unfolded_backward(T_tilde, D, inv_norm, a, ctx.c, ckpt, grad_soft, precision=ctx.precision)
        return grad_alpha, None, None, None, None, None


# taser_item of include/taser.h (40 bytes, naturally aligned).
ITEM_DTYPE = np.dtype([("N", "<i4"), ("t_max", "<i4"), ("t_off", "<i8"), ("d_off", "<i8"), ("s_off", "<i8"),
                       ("l_off", "<i8")])


def make_items(N, t_max, t_off, d_off, s_off, l_off=None):
    """Host array of taser_item from per-item arrays (l_off None -> no L output)."""
    n = len(N)
    it = np.zeros(n, dtype=ITEM_DTYPE)
    it["N"], it["t_max"], it["t_off"], it["d_off"], it["s_off"] = N, t_max, t_off, d_off, s_off
    it["l_off"] = -1 if l_off is None else l_off
    return it


def uneven_workspace_bytes(n_items):
    return int(lib().taser_uneven_workspace_bytes(int(n_items)))


def tuning(blocks_per_sm=(0, 0, 0, 0), pop=(0, 0, 0, 0)):
    t = UnevenTuning()
    for b in range(4):
        t.blocks_per_sm[b] = int(blocks_per_sm[b])
        t.pop[b] = int(pop[b])
    return t


def detect_uneven(items, T_pool, D_pool, tau, s_pool, workspace, precision="fp32", lnn_mode="fixed", L_pool=None,
                  flags=None, tune=None, stream=None):
    """Algorithm 1 on an uneven batch.  `items` is a CUDA uint8 tensor holding taser_item
    records (see make_items); pools are CUDA tensors addressed by the items' offsets."""
    n = items.numel() // ITEM_DTYPE.itemsize
    _dev(items, torch.uint8, "items")
    for name, t in (("T_pool", T_pool), ("D_pool", D_pool), ("tau", tau)):
        _dev(t, torch.float32, name)
    _dev(s_pool, torch.int8, "s_pool")
    _dev(workspace, torch.uint8, "workspace")
    st = lib().taser_detect_uneven(n, _ptr(items), _ptr(T_pool), _ptr(D_pool), _ptr(tau), PRECISIONS[precision],
                                   LNN_MODES[lnn_mode], _ptr(L_pool), _ptr(s_pool), _ptr(flags), _ptr(workspace),
                                   workspace.numel(), ctypes.byref(tune) if tune is not None else None,
                                   _stream(stream))
    check(st, "taser_detect_uneven")


def debug_report():
    """Counters of the bounds-checked library (TASER_LIBRARY=debug), read and cleared:
    {"fails", "nonfinite", "first": None or {"source", "line", "index"}}.  Raises
    TaserError (TASER_ERR_UNSUPPORTED) on the release library."""
    from .build import source_of
    fails, first, nonfinite = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().taser_debug_report(ctypes.byref(fails), ctypes.byref(first), ctypes.byref(nonfinite)),
          "taser_debug_report")
    rec = None
    if fails.value:
        f = first.value
        rec = {"source": source_of(f >> 56), "line": (f >> 32) & 0xffffff, "index": f & 0xffffffff}
    return {"fails": fails.value, "nonfinite": nonfinite.value, "first": rec}


def debug_drop_copy(instance, chunk):
    """Debug library only: later TMA-staged build_T calls withhold the staging copy of
    16-antenna chunk `chunk` of `instance` (instance < 0: off); see taser_debug_drop_copy."""
    check(lib().taser_debug_drop_copy(int(instance), int(chunk)), "taser_debug_drop_copy")
