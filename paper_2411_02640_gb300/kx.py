"""Python binding of libkx (ctypes): argument marshalling only.

Every computation happens in the library's CUDA kernels.  Tensors are
torch CUDA float64 tensors in the library's layout (T[n], p[n],
Y[N_s, ld], outputs likewise); the work is enqueued on the current torch
stream (or the stream given).  There is no CPU fallback: if libkx.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

from . import build as _build

_lib: Optional[ctypes.CDLL] = None

FP64, MIXED = 0, 1
KX_ERR_NONFINITE_INPUT = 9   # kx_last_point_status: a point outside the domain was recorded
_PREC = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}

KERNELS = ("wdot_fp64", "wdot_mixed", "rop_fp64", "rop_mixed", "thermo", "visc_fp64", "visc_mixed", "diff_fp64",
           "diff_mixed", "vjp", "wdot_fp64_noalloc", "wdot_fp64_wc", "vjp_wc")


class KxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"kx error {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("diff_mode", ctypes.c_int), ("kc_mode", ctypes.c_int), ("tr_mode", ctypes.c_int), ("rates_mode", ctypes.c_int),
                ("rates_arith", ctypes.c_int), ("tr_layout", ctypes.c_int), ("maxrreg", ctypes.c_int),
                ("block", ctypes.c_int), ("lazy", ctypes.c_int), ("verbose", ctypes.c_int),
                ("libmath", ctypes.c_int), ("compile_only", ctypes.c_int), ("rates_layout", ctypes.c_int),
                ("rates_group", ctypes.c_int), ("vjp_form", ctypes.c_int), ("vjp_layout", ctypes.c_int), ("rates_negligible", ctypes.c_int),
                ("cache_dir", ctypes.c_char_p)]


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libkx.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libkx.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        L.kx_load_mechanism.argtypes = [ctypes.c_char_p, ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.kx_free_mechanism.argtypes = [vp]
        L.kx_mechanism_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]
        L.kx_production_rates.argtypes = [vp, dp, dp, dp, i64, dp, i64, ctypes.c_int, vp]
        L.kx_production_rates_noalloc.argtypes = [vp, dp, dp, dp, i64, dp, i64, vp]
        L.kx_last_point_status.argtypes = [vp, vp, ctypes.POINTER(i64)]
        L.kx_evaluate_host_bytes_per_state.argtypes = [vp, ctypes.c_int]
        L.kx_evaluate_host_bytes_per_state.restype = i64
        L.kx_evaluate_host.argtypes = [vp, dp, dp, dp, i64, dp, dp, dp, dp, dp, dp, i64, i64, ctypes.c_int, ctypes.c_int,
                                       vp, ctypes.c_size_t, i64, vp, vp]
        L.kx_rates_of_progress.argtypes = [vp, dp, dp, dp, i64, dp, i64, ctypes.c_int, vp]
        L.kx_thermo.argtypes = [vp, dp, dp, dp, i64, dp, dp, i64, vp]
        L.kx_transport.argtypes = [vp, dp, dp, dp, i64, dp, dp, dp, i64, ctypes.c_int, vp]
        L.kx_viscosity_conductivity.argtypes = [vp, dp, dp, dp, i64, dp, dp, i64, ctypes.c_int, vp]
        L.kx_diffusion.argtypes = [vp, dp, dp, dp, i64, dp, i64, ctypes.c_int, vp]
        L.kx_production_rates_vjp.argtypes = [vp, dp, dp, dp, i64, dp, dp, dp, i64, vp]
        L.kx_kernel_info.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.kx_kernel_op_counts.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
        L.kx_kernel_source_hash.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint64)]
        L.kx_kernel_source.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.kx_copy_rows_async.argtypes = [vp, i64, vp, i64, i64, i64, vp]
        L.kx_probe_pipe.argtypes = [ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, dp, vp, ctypes.POINTER(ctypes.c_double)]
        L.kx_status_string.argtypes = [ctypes.c_int]
        L.kx_status_string.restype = ctypes.c_char_p
        L.kx_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        L = lib()
        raise KxError(status, (L.kx_last_error() or b"").decode() or L.kx_status_string(status).decode())


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Mechanism:
    """A mechanism compiled into GPU kernels.

    ``Mechanism(path, diff_mode=..., kc_mode=..., block=..., libmath=...,
    lazy=..., verbose=..., compile_only=..., cache_dir=...)``."""

    def __init__(self, path: str, **opts):
        L = lib()
        o = Options()
        for k, v in opts.items():
            if k == "cache_dir":
                o.cache_dir = v.encode() if v else None
            else:
                setattr(o, k, int(v))
        self._opts = o
        h = ctypes.c_void_p()
        _check(L.kx_load_mechanism(path.encode(), ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        ns, nr = ctypes.c_int(), ctypes.c_int()
        _check(L.kx_mechanism_info(h, ctypes.byref(ns), ctypes.byref(nr), None))
        self.n_species, self.n_reactions = ns.value, nr.value
        W = (ctypes.c_double * ns.value)()
        _check(L.kx_mechanism_info(h, None, None, W))
        self.W = list(W)
        self.path = path

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().kx_free_mechanism(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- helpers
    def _state(self, T, p, Y):
        import torch
        for t in (T, p, Y):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
                raise TypeError("T, p and Y must be CUDA float64 tensors")
        n = T.shape[0]
        if p.shape[0] != n or Y.dim() != 2 or Y.shape[0] != self.n_species or Y.shape[1] < n:
            raise ValueError("expected T[n], p[n], Y[N_s, >= n]")
        if n == 0:
            return 0, 0
        if not (T.is_contiguous() and p.is_contiguous() and Y.stride(1) == 1):
            raise ValueError("T and p must be contiguous and Y point-contiguous")
        return n, Y.stride(0)

    def _alloc(self, rows, n, ld, like):
        import torch
        if rows is None:
            return torch.empty(n, dtype=torch.float64, device=like.device)
        return torch.empty((rows, ld if n > 0 else 0), dtype=torch.float64, device=like.device)

    # -------------------------------------------------------------- calls
    def production_rates(self, T, p, Y, out=None, precision="fp64", stream=None):
        n, ld = self._state(T, p, Y)
        out = out if out is not None else self._alloc(self.n_species, n, ld, T)
        assert out.shape[0] == self.n_species and (n == 0 or out.stride(0) == ld)
        _check(lib().kx_production_rates(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(out), n, _PREC[precision],
                                          _stream(stream)))
        return out

    def production_rates_noalloc(self, T, p, Y, out, stream=None):
        """kx_production_rates_noalloc: float64-accurate production rates into a
        preallocated ``out`` with no device allocation by the call."""
        n, ld = self._state(T, p, Y)
        assert out.shape[0] == self.n_species and (n == 0 or out.stride(0) == ld)
        _check(lib().kx_production_rates_noalloc(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(out), n, _stream(stream)))
        return out

    OUT_WDOT, OUT_THERMO, OUT_TRANSPORT = 1, 2, 4

    def evaluate_host_bytes_per_state(self, outputs: int) -> int:
        return int(lib().kx_evaluate_host_bytes_per_state(self.h, outputs))

    def evaluate_host(self, T, p, Y, out: dict, outputs: int = 7, precision="fp64", workspace=None,
                      max_chunk: int = 0, streams=None):
        """kx_evaluate_host: host (pinned) states in, host outputs out, the
        copies overlapped with the kernels in chunks.  ``out``
        holds host tensors under the keys wdot, cp, h, mu, lam, Dk (those of
        the selected outputs); ``workspace`` a device uint8 tensor; ``streams``
        two torch streams.  Returns after enqueueing; synchronise both streams."""
        import torch
        if not all(isinstance(t, torch.Tensor) and t.dtype == torch.float64 and not t.is_cuda for t in (T, p, Y)):
            raise TypeError("T, p and Y must be host float64 tensors (pinned for asynchronous copies)")
        if not (T.dim() == 1 and p.shape == T.shape and Y.dim() == 2 and Y.shape[0] == self.n_species
                and Y.shape[1] == T.shape[0] and T.is_contiguous() and p.is_contiguous() and Y.stride(1) == 1):
            raise ValueError("T, p [n] contiguous and Y [n_species, n] point-contiguous expected")
        n, ld = T.shape[0], Y.stride(0)
        get = lambda k: _ptr(out[k]) if k in out else None
        ldo = out["wdot"].stride(0) if "wdot" in out else (out["Dk"].stride(0) if "Dk" in out else n)
        _check(lib().kx_evaluate_host(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, get("wdot"), get("cp"), get("h"), get("mu"),
                                      get("lam"), get("Dk"), ldo, n, _PREC[precision], outputs, workspace.data_ptr(),
                                      workspace.numel(), max_chunk, _stream(streams[0]), _stream(streams[1])))
        return out

    def rates_of_progress(self, T, p, Y, out=None, precision="fp64", stream=None):
        n, ld = self._state(T, p, Y)
        out = out if out is not None else self._alloc(self.n_reactions, n, ld, T)
        assert out.shape[0] == self.n_reactions and (n == 0 or out.stride(0) == ld)
        _check(lib().kx_rates_of_progress(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(out), n, _PREC[precision],
                                           _stream(stream)))
        return out

    def thermo(self, T, p, Y, out: Optional[Tuple] = None, stream=None):
        n, ld = self._state(T, p, Y)
        cp, h = out if out is not None else (self._alloc(None, n, ld, T), self._alloc(None, n, ld, T))
        _check(lib().kx_thermo(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(cp), _ptr(h), n, _stream(stream)))
        return cp, h

    def transport(self, T, p, Y, out: Optional[Tuple] = None, precision="fp64", stream=None):
        n, ld = self._state(T, p, Y)
        if out is None:
            out = (self._alloc(None, n, ld, T), self._alloc(None, n, ld, T), self._alloc(self.n_species, n, ld, T))
        mu, lam, D = out
        assert n == 0 or D.stride(0) == ld
        _check(lib().kx_transport(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(mu), _ptr(lam), _ptr(D), n,
                                  _PREC[precision], _stream(stream)))
        return mu, lam, D

    def viscosity_conductivity(self, T, p, Y, out: Optional[Tuple] = None, precision="fp64", stream=None):
        n, ld = self._state(T, p, Y)
        mu, lam = out if out is not None else (self._alloc(None, n, ld, T), self._alloc(None, n, ld, T))
        _check(lib().kx_viscosity_conductivity(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(mu), _ptr(lam), n,
                                               _PREC[precision], _stream(stream)))
        return mu, lam

    def diffusion(self, T, p, Y, out=None, precision="fp64", stream=None):
        n, ld = self._state(T, p, Y)
        D = out if out is not None else self._alloc(self.n_species, n, ld, T)
        assert n == 0 or D.stride(0) == ld
        _check(lib().kx_diffusion(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(D), n, _PREC[precision], _stream(stream)))
        return D

    def production_rates_vjp(self, T, p, Y, v, out: Optional[Tuple] = None, stream=None):
        """gT[n] = sum_k v_k d wdot_k/dT, gY[N_s, ld] = sum_k v_k d wdot_k/dY_j (p fixed)."""
        n, ld = self._state(T, p, Y)
        assert v.shape[0] == self.n_species and v.dtype == Y.dtype and (n == 0 or v.stride(0) == ld)
        if out is None:
            out = (self._alloc(None, n, ld, T), self._alloc(self.n_species, n, ld, T))
        gT, gY = out
        assert n == 0 or gY.stride(0) == ld
        _check(lib().kx_production_rates_vjp(self.h, _ptr(T), _ptr(p), _ptr(Y), ld, _ptr(v), _ptr(gT), _ptr(gY), n,
                                             _stream(stream)))
        return gT, gY

    def last_point_status(self, stream=None) -> int:
        """kx_last_point_status: the smallest index of a point outside the
        domain seen by this handle's calls since the last check (-1 if none);
        waits for ``stream`` and resets the record."""
        first = ctypes.c_int64()
        st = lib().kx_last_point_status(self.h, _stream(stream), ctypes.byref(first))
        if st != KX_ERR_NONFINITE_INPUT:
            _check(st)
        return first.value

    def source_hash(self, name: str) -> str:
        h = ctypes.c_uint64()
        _check(lib().kx_kernel_source_hash(self.h, name.encode(), ctypes.byref(h)))
        return f"{h.value:016x}"

    def kernel_source(self, name: str) -> str:
        """The emitted CUDA C++ source of one kernel."""
        n = ctypes.c_size_t()
        _check(lib().kx_kernel_source(self.h, name.encode(), None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(lib().kx_kernel_source(self.h, name.encode(), buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def op_counts(self, name: str) -> dict:
        """Per-point operation counts the emitter tallied for one kernel."""
        c = (ctypes.c_double * 8)()
        _check(lib().kx_kernel_op_counts(self.h, name.encode(), c))
        return dict(zip(("fp64", "fp32", "exp64", "log64", "div64", "exp32", "log32", "div32"), list(c)))

    def kernel_info(self, name: str) -> dict:
        r, lb = ctypes.c_int(), ctypes.c_int()
        cs, f64, f32, ex = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().kx_kernel_info(self.h, name.encode(), ctypes.byref(r), ctypes.byref(lb), ctypes.byref(cs),
                                    ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(ex)))
        return dict(registers=r.value, local_bytes=lb.value, compile_seconds=cs.value, fp64_ops=f64.value,
                    fp32_ops=f32.value, exps=ex.value)


PROBE_OPS = ("dfma", "ffma", "mufu_ex2", "exp64", "log64", "div64")


def probe_pipe(op: str, iters: int, blocks: int, threads: int, sink, stream=None) -> float:
    """Enqueue one arithmetic-pipe probe launch (kx_probe_pipe) on the stream;
    returns the number of operations it performs.  sink: a CUDA float64
    tensor of at least blocks * threads elements."""
    assert sink.dtype.is_floating_point and sink.element_size() == 8 and sink.numel() >= blocks * threads
    ops = ctypes.c_double()
    st = lib().kx_probe_pipe(PROBE_OPS.index(op), iters, blocks, threads, sink.data_ptr(), _stream(stream),
                             ctypes.byref(ops))
    if st != 0:
        raise KxError(st, f"kx_probe_pipe({op}) failed")
    return ops.value


def copy_rows(dst, src, stream=None) -> None:
    """dst[:, :] = src[:, :] for float64 2-D tensors with unit column stride
    (host or device, any row stride), one asynchronous 2-D copy."""
    rows, n = src.shape
    assert dst.shape[0] == rows and dst.shape[1] == n and src.stride(1) == 1 and dst.stride(1) == 1
    _check(lib().kx_copy_rows_async(dst.data_ptr(), dst.stride(0), src.data_ptr(), src.stride(0), rows, n,
                                    _stream(stream)))
