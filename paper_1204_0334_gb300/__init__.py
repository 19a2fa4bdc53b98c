"""Python binding of the GB300 LDPC library (``include/ldpc.h``).

Argument marshalling only: every step of decoding runs in the CUDA kernels of
``libldpc_gb300.so``.  PyTorch supplies device memory and streams.  There is no
CPU fallback: importing works without the library (so the package can be
inspected on a machine without a GPU), but every call raises if the shared
library has not been built.

The functions carry the C names (``ldpc_code_create``, ``ldpc_decode``,
``ldpc_channel``, ``ldpc_ber_sim`` ...).  Tensors are passed by data pointer;
``stream`` defaults to the current torch stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libldpc_gb300.so")

ALGO_SP, ALGO_MS, ALGO_NOMS = 0, 1, 2
MSG_F32, MSG_F16, MSG_I8 = 0, 1, 2
CODEWORDS_ZERO, CODEWORDS_RANDOM = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "device wait timed out",
          5: "unsupported"}


class LdpcError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class DecodeOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("early_stop", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("msg", ctypes.c_int32), ("clip", ctypes.c_float), ("frac_bits", ctypes.c_int32),
                ("noms_params", ctypes.c_void_p), ("codewords", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class BerResult(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("frame_errors", ctypes.c_int64), ("bit_errors", ctypes.c_int64),
                ("iters_sum", ctypes.c_int64), ("undetected", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("bit_errors_sq", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
P = ctypes.c_void_p

# (name, restype, argtypes) of every exported entry point
_SIGNATURES = [
    ("ldpc_default_opts", None, [P]),
    ("ldpc_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("ldpc_last_error", ctypes.c_char_p, []),
    ("ldpc_code_create", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]),
    ("ldpc_code_create_sparse", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P, P, P]),
    ("ldpc_code_destroy", ctypes.c_int, [P]),
    ("ldpc_code_dims", ctypes.c_int, [P, P, P, P, P]),
    ("ldpc_decode", ctypes.c_int, [P, P, ctypes.c_int32, P, P, P, P, P, P]),
    ("ldpc_decode_noalloc", ctypes.c_int, [P, P, ctypes.c_int32, P, P, P, P, P, P]),
    ("ldpc_batch_create", ctypes.c_int, [P, ctypes.c_int32, P, P, P]),
    ("ldpc_batch_decode", ctypes.c_int, [P, P, P, P, P, P]),
    ("ldpc_batch_info", ctypes.c_int, [P, P, P, P]),
    ("ldpc_batch_destroy", ctypes.c_int, [P]),
    ("ldpc_batch_moved", ctypes.c_int, [P, P]),
    ("ldpc_batch_set_compaction", ctypes.c_int, [P, ctypes.c_int32]),
    ("ldpc_batch_compaction", ctypes.c_int, [P, P, P]),
    ("ldpc_channel", ctypes.c_int, [P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, P, P]),
    ("ldpc_ber_sim", ctypes.c_int, [P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int32, P, P, P]),
    ("ldpc_code_info_set", ctypes.c_int, [P, P, P]),
    ("ldpc_encode", ctypes.c_int, [P, P, ctypes.c_int32, P, P]),
    ("ldpc_random_codewords", ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, P, P, P]),
    ("ldpc_channel_codewords", ctypes.c_int, [P, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32,
                                              P, P, P]),
    ("ldpccc_create", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, P]),
    ("ldpccc_create_tanner", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, P]),
    ("ldpccc_destroy", ctypes.c_int, [P]),
    ("ldpccc_dims", ctypes.c_int, [P, P, P, P, P]),
    ("ldpccc_reset", ctypes.c_int, [P]),
    ("ldpccc_decode_window", ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_float, P, P, P, P, P]),
    ("ldpccc_channel", ctypes.c_int, [P, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, P, P]),
    ("ldpc_noms_forward", ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_float, P, P, P]),
    ("ldpc_noms_backward", ctypes.c_int, [P, P, P, P]),
    ("ldpc_phi_eval", ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_int32, P]),
    ("ldpc_profile_enable", ctypes.c_int, [ctypes.c_int32]),
    ("ldpc_profile_read", ctypes.c_int, [P]),
    ("ldpc_bandwidth_probe", ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P, P]),
    ("ldpc_sync_probe", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, P, P]),
    ("ldpc_tune_slots", ctypes.c_int, [P, ctypes.c_double, ctypes.c_uint64, P, P, P, P]),
]


def exported_names() -> list[str]:
    return [n for n, _, _ in _SIGNATURES]


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1204_0334_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise LdpcError(status, where, lib().ldpc_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def default_opts(**kw) -> DecodeOpts:
    o = DecodeOpts()
    lib().ldpc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------- C-named calls
def ldpc_code_create(shifts, p: int) -> int:
    """shifts: J x L integer matrix (-1 = zero block).  Returns the opaque handle."""
    import numpy as np

    a = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32))
    J, L = a.shape
    h = ctypes.c_void_p()
    _check(lib().ldpc_code_create(a.ctypes.data_as(P), J, L, p, ctypes.byref(h)), "ldpc_code_create")
    return h.value


def ldpc_code_create_sparse(row_ptr, col_idx, N: int) -> int:
    """A general LDPC code from H in compressed-row form (row_ptr [M+1], col_idx [E]).  Returns the handle."""
    import numpy as np

    rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int32))
    ci = np.ascontiguousarray(np.asarray(col_idx, dtype=np.int32))
    h = ctypes.c_void_p()
    _check(lib().ldpc_code_create_sparse(len(rp) - 1, N, rp.ctypes.data_as(P), ci.ctypes.data_as(P), ctypes.byref(h)),
           "ldpc_code_create_sparse")
    return h.value


def ldpc_code_destroy(code: int):
    _check(lib().ldpc_code_destroy(code), "ldpc_code_destroy")


def ldpc_code_dims(code: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().ldpc_code_dims(code, *[ctypes.byref(x) for x in v]), "ldpc_code_dims")
    return dict(zip(["N", "M", "E", "K"], [x.value for x in v]))


def ldpc_decode(code: int, llr, opts: DecodeOpts, post=None, hard=None, iters=None, ok=None, stream=None):
    gamma = llr.shape[0]
    _check(lib().ldpc_decode(code, _ptr(llr), gamma, ctypes.byref(opts), _ptr(post), _ptr(hard), _ptr(iters),
                             _ptr(ok), _stream(stream)), "ldpc_decode")


def ldpc_decode_noalloc(code: int, llr, opts: DecodeOpts, post=None, hard=None, iters=None, ok=None, stream=None):
    """ldpc_decode with the library's fixed scratch instead of allocated workspace (device buffers only)."""
    gamma = llr.shape[0]
    _check(lib().ldpc_decode_noalloc(code, _ptr(llr), gamma, ctypes.byref(opts), _ptr(post), _ptr(hard),
                                     _ptr(iters), _ptr(ok), _stream(stream)), "ldpc_decode_noalloc")


def ldpc_channel(code: int, ebn0_db: float, seed: int, first_frame: int, out, stream=None):
    _check(lib().ldpc_channel(code, ebn0_db, seed, first_frame, out.shape[0], _ptr(out), _stream(stream)),
           "ldpc_channel")


def ldpc_ber_sim(code: int, ebn0_db: float, seed: int, first_frame: int, max_frames: int, target_frame_errors: int,
                 gamma: int, opts: DecodeOpts, stream=None) -> dict:
    r = BerResult()
    _check(lib().ldpc_ber_sim(code, ebn0_db, seed, first_frame, max_frames, target_frame_errors, gamma,
                              ctypes.byref(opts), ctypes.byref(r), _stream(stream)), "ldpc_ber_sim")
    return r.as_dict()


def ldpc_code_info_set(code: int):
    """(k, info_pos): the code's dimension and its information positions (numpy int32 [k])."""
    import numpy as np

    k = ctypes.c_int64()
    _check(lib().ldpc_code_info_set(code, ctypes.byref(k), None), "ldpc_code_info_set")
    pos = np.zeros(k.value, dtype=np.int32)
    if k.value:
        _check(lib().ldpc_code_info_set(code, ctypes.byref(k), pos.ctypes.data_as(ctypes.c_void_p)),
               "ldpc_code_info_set")
    return k.value, pos


def ldpc_encode(code: int, info, cw, stream=None):
    """cw[gamma][N] (uint8, device) = codewords of info[gamma][k] (uint8, device)."""
    _check(lib().ldpc_encode(code, _ptr(info), cw.shape[0], _ptr(cw), _stream(stream)), "ldpc_encode")


def ldpc_random_codewords(code: int, seed: int, first_frame: int, cw, info=None, stream=None):
    _check(lib().ldpc_random_codewords(code, seed, first_frame, cw.shape[0], _ptr(info), _ptr(cw), _stream(stream)),
           "ldpc_random_codewords")


def ldpc_channel_codewords(code: int, ebn0_db: float, seed: int, first_frame: int, cw, out, stream=None):
    _check(lib().ldpc_channel_codewords(code, ebn0_db, seed, first_frame, out.shape[0], _ptr(cw), _ptr(out),
                                        _stream(stream)), "ldpc_channel_codewords")


def ldpc_phi_eval(x, variant: int = 0, stream=None):
    """phi(x) = -ln tanh(x/2) evaluated on the device by the decoder's kernel code."""
    import torch

    y = torch.empty_like(x)
    _check(lib().ldpc_phi_eval(_ptr(x), _ptr(y), x.numel(), variant, _stream(stream)), "ldpc_phi_eval")
    return y


def ldpccc_create(shifts, p: int, I: int, gamma: int) -> int:
    import numpy as np

    a = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32))
    J, L = a.shape
    h = ctypes.c_void_p()
    _check(lib().ldpccc_create(a.ctypes.data_as(P), J, L, p, I, gamma, ctypes.byref(h)), "ldpccc_create")
    return h.value


def ldpccc_create_tanner(shifts, p: int, I: int, gamma: int) -> int:
    """Time-invariant LDPCCC with delays D^{a_jl}; frames of p time instants."""
    import numpy as np

    a = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32))
    J, L = a.shape
    h = ctypes.c_void_p()
    _check(lib().ldpccc_create_tanner(a.ctypes.data_as(P), J, L, p, I, gamma, ctypes.byref(h)),
           "ldpccc_create_tanner")
    return h.value


def ldpccc_destroy(cc: int):
    _check(lib().ldpccc_destroy(cc), "ldpccc_destroy")


def ldpccc_dims(cc: int) -> dict:
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().ldpccc_dims(cc, *[ctypes.byref(x) for x in v]), "ldpccc_dims")
    return dict(zip(["c", "b", "ms", "Lambda"], [x.value for x in v]))


def ldpccc_reset(cc: int):
    _check(lib().ldpccc_reset(cc), "ldpccc_reset")


def ldpccc_decode_window(cc: int, llr, clip: float = 30.0, hard=None, post=None, stream=None):
    """llr: [gamma][T][c] float32.  Returns (first decided frame or -1, number decided)."""
    first = ctypes.c_int64()
    n = ctypes.c_int32()
    T = llr.shape[1]
    _check(lib().ldpccc_decode_window(cc, _ptr(llr), T, clip, _ptr(hard), _ptr(post), ctypes.byref(first),
                                      ctypes.byref(n), _stream(stream)), "ldpccc_decode_window")
    return first.value, n.value


def ldpccc_channel(cc: int, ebn0_db: float, seed: int, first_frame: int, out, stream=None):
    _check(lib().ldpccc_channel(cc, ebn0_db, seed, first_frame, out.shape[1], _ptr(out), _stream(stream)),
           "ldpccc_channel")


class LDPCCC:
    """Owning wrapper of an ldpccc handle."""

    def __init__(self, shifts, p: int, I: int, gamma: int, tanner: bool = False):
        """tanner: the time-invariant code with delays D^{a_jl} instead of the Sec. II-D unwrapping."""
        self.handle = (ldpccc_create_tanner if tanner else ldpccc_create)(shifts, p, I, gamma)
        d = ldpccc_dims(self.handle)
        self.c, self.b, self.ms, self.Lambda = d["c"], d["b"], d["ms"], d["Lambda"]
        self.I, self.gamma = I, gamma

    def close(self):
        if getattr(self, "handle", None):
            ldpccc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def channel(self, ebn0_db, seed, first_frame, T, device="cuda", stream=None):
        import torch

        out = torch.empty((self.gamma, T, self.c), dtype=torch.float32, device=device)
        ldpccc_channel(self.handle, ebn0_db, seed, first_frame, out, stream)
        return out

    def window(self, llr, clip=30.0, want_post=True, stream=None):
        """llr: [gamma][T][c] tensor on the device.  Returns (first, n, hard[:, :n], post[:, :n])."""
        import torch

        g, T, c = llr.shape
        hard = torch.empty((g, T, c), dtype=torch.uint8, device=llr.device)
        post = torch.empty((g, T, c), dtype=torch.float32, device=llr.device) if want_post else None
        first, n = ldpccc_decode_window(self.handle, llr.contiguous(), clip, hard, post, stream)
        return first, n, hard[:, :n], (post[:, :n] if post is not None else None)


def ldpc_noms_forward(code: int, llr, params, msg: int = MSG_F32, ckpt_every: int = 1, clip: float = 30.0,
                      want_post: bool = False, stream=None):
    """Training forward pass; returns (loss tensor [1], post^(T) [B][N] or None)."""
    import torch

    B = llr.shape[0]
    T = params.shape[0]
    loss = torch.empty(1, dtype=torch.float32, device=llr.device)
    post = torch.empty_like(llr) if want_post else None
    _check(lib().ldpc_noms_forward(code, _ptr(llr), B, T, _ptr(params), msg, ckpt_every, clip, _ptr(loss),
                                   _ptr(post), _stream(stream)), "ldpc_noms_forward")
    return loss, post


def ldpc_noms_backward(code: int, params, grad, stream=None):
    _check(lib().ldpc_noms_backward(code, _ptr(params), _ptr(grad), _stream(stream)), "ldpc_noms_backward")


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def ldpc_batch_create(codes, gammas, opts: DecodeOpts) -> int:
    """codes: list of ldpc_code handles (or QCCode objects); gammas: frames per code."""
    hs = (ctypes.c_void_p * len(codes))(*[getattr(c, "handle", c) for c in codes])
    g = (ctypes.c_int32 * len(gammas))(*gammas)
    h = ctypes.c_void_p()
    _check(lib().ldpc_batch_create(hs, len(codes), g, ctypes.byref(opts), ctypes.byref(h)), "ldpc_batch_create")
    return h.value


def ldpc_batch_decode(batch: int, llrs, hards=None, iters=None, oks=None, stream=None):
    """llrs / hards / iters / oks: lists (one device tensor per code) or None."""
    la = _ptr_array(llrs)
    ha = _ptr_array(hards) if hards is not None else None
    ia = _ptr_array(iters) if iters is not None else None
    oa = _ptr_array(oks) if oks is not None else None
    _check(lib().ldpc_batch_decode(batch, la, ha, ia, oa, _stream(stream)), "ldpc_batch_decode")


def ldpc_batch_info(batch: int) -> dict:
    tr, tg = ctypes.c_int32(), ctypes.c_int32()
    ms = (ctypes.c_double * 3)()
    _check(lib().ldpc_batch_info(batch, ctypes.byref(tr), ctypes.byref(tg), ms), "ldpc_batch_info")
    return {"tile_rows": tr.value, "tile_groups": tg.value, "tune_ms": list(ms)}


def ldpc_batch_moved(batch: int, ncodes: int) -> list:
    """Frames of each code the last decode moved to the code's second package area."""
    out = (ctypes.c_int32 * ncodes)()
    _check(lib().ldpc_batch_moved(batch, out), "ldpc_batch_moved")
    return list(out)


def ldpc_batch_set_compaction(batch: int, after_iter: int):
    """Compaction after iteration after_iter (0: never, -1: autotuned by the next decode)."""
    _check(lib().ldpc_batch_set_compaction(batch, int(after_iter)), "ldpc_batch_set_compaction")


def ldpc_batch_compaction(batch: int) -> dict:
    k = ctypes.c_int32(0)
    ms = (ctypes.c_double * 4)()
    _check(lib().ldpc_batch_compaction(batch, ctypes.byref(k), ms), "ldpc_batch_compaction")
    return {"after_iter": k.value, "tune_ms": dict(zip((0, 8, 12, 16), list(ms)))}


def ldpc_batch_destroy(batch: int):
    _check(lib().ldpc_batch_destroy(batch), "ldpc_batch_destroy")


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("cn_launches", ctypes.c_int64), ("cn_ms", ctypes.c_double),
                ("vn_launches", ctypes.c_int64), ("vn_ms", ctypes.c_double)]


def ldpc_profile_enable(on: bool = True):
    _check(lib().ldpc_profile_enable(int(on)), "ldpc_profile_enable")


def ldpc_profile_read() -> dict:
    r = Profile()
    _check(lib().ldpc_profile_read(ctypes.byref(r)), "ldpc_profile_read")
    return {k: getattr(r, k) for k, _ in Profile._fields_}


TUNE_SLOTS = (16384, 8192, 4096, 2048, 1024)


def ldpc_tune_slots(code: int, ebn0_db: float, seed: int, opts: DecodeOpts, stream=None) -> dict:
    """The slot count the library's autotuner picks for this code and opts, with each candidate's Mbit/s."""
    g = ctypes.c_int32(0)
    rates = (ctypes.c_double * len(TUNE_SLOTS))()
    _check(lib().ldpc_tune_slots(ctypes.c_void_p(code), float(ebn0_db), int(seed), ctypes.byref(opts),
                                 ctypes.byref(g), rates, _stream(stream)), "ldpc_tune_slots")
    return {"gamma": int(g.value), "candidates": dict(zip(TUNE_SLOTS, list(rates)))}


def ldpc_bandwidth_probe(src, dst, reps: int, mode: int, stream=None) -> float:
    """GB/s of the library's streaming probe: mode 0 reads src through L2, mode 1 copies src to dst."""
    out = ctypes.c_double(0.0)
    nbytes = src.numel() * src.element_size()
    _check(lib().ldpc_bandwidth_probe(_ptr(src), _ptr(dst), nbytes, int(reps), int(mode), ctypes.byref(out),
                                      _stream(stream)), "ldpc_bandwidth_probe")
    return out.value


def ldpc_sync_probe(boundaries: int = 120, reps: int = 100) -> dict:
    """Microseconds per phase boundary: a CUDA graph of empty launches against grid barriers in one
    cooperative kernel (no work in either)."""
    g, c = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().ldpc_sync_probe(int(boundaries), int(reps), ctypes.byref(g), ctypes.byref(c)), "ldpc_sync_probe")
    return {"graph_us": g.value, "cooperative_us": c.value}


# ----------------------------------------------------------------- convenience
@dataclass
class QCCode:
    """Owning wrapper of an ldpc_code handle."""

    shifts: object
    p: int

    def __post_init__(self):
        self.handle = ldpc_code_create(self.shifts, self.p)
        d = ldpc_code_dims(self.handle)
        self.N, self.M, self.E, self.K = d["N"], d["M"], d["E"], d["K"]

    def close(self):
        if getattr(self, "handle", None):
            ldpc_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, llr, max_iter=30, early_stop=False, algo=ALGO_SP, msg=None, clip=30.0, frac_bits=2,
               want_post=True, stream=None):
        """Decode a [gamma][N] float32 tensor; returns (post, hard, iters, ok) on llr's device."""
        import torch

        if msg is None:
            msg = MSG_I8 if algo == ALGO_MS else MSG_F32
        gamma = llr.shape[0]
        dev = llr.device
        post = torch.empty((gamma, self.N), dtype=torch.float32, device=dev) if want_post else None
        hard = torch.empty((gamma, self.N), dtype=torch.uint8, device=dev)
        iters = torch.empty(gamma, dtype=torch.int32, device=dev)
        ok = torch.empty(gamma, dtype=torch.int32, device=dev)
        o = default_opts(max_iter=max_iter, early_stop=int(early_stop), algo=algo, msg=msg, clip=clip,
                         frac_bits=frac_bits)
        ldpc_decode(self.handle, llr.contiguous(), o, post, hard, iters, ok, stream)
        return post, hard, iters, ok

    def channel(self, ebn0_db, seed, first_frame, gamma, device="cuda", stream=None):
        import torch

        out = torch.empty((gamma, self.N), dtype=torch.float32, device=device)
        ldpc_channel(self.handle, ebn0_db, seed, first_frame, out, stream)
        return out

    def info_set(self):
        """(k, info_pos) of the systematic encoder."""
        return ldpc_code_info_set(self.handle)

    def encode(self, info, stream=None):
        import torch

        cw = torch.empty((info.shape[0], self.N), dtype=torch.uint8, device=info.device)
        ldpc_encode(self.handle, info.contiguous(), cw, stream)
        return cw

    def random_codewords(self, seed, first_frame, gamma, device="cuda", want_info=True, stream=None):
        """(info[gamma][k], cw[gamma][N]) as uint8 device tensors (info None unless want_info)."""
        import torch

        k, _ = self.info_set()
        cw = torch.empty((gamma, self.N), dtype=torch.uint8, device=device)
        info = torch.empty((gamma, k), dtype=torch.uint8, device=device) if want_info and k else None
        ldpc_random_codewords(self.handle, seed, first_frame, cw, info, stream)
        return info, cw

    def channel_codewords(self, ebn0_db, seed, first_frame, cw, stream=None):
        import torch

        out = torch.empty((cw.shape[0], self.N), dtype=torch.float32, device=cw.device)
        ldpc_channel_codewords(self.handle, ebn0_db, seed, first_frame, cw.contiguous(), out, stream)
        return out

    def ber_sim(self, ebn0_db, seed=1, first_frame=0, max_frames=4096, target_frame_errors=100, gamma=4096,
                stream=None, **opt):
        return ldpc_ber_sim(self.handle, ebn0_db, seed, first_frame, max_frames, target_frame_errors, gamma,
                            default_opts(**opt), stream)


class SparseCode(QCCode):
    """Owning wrapper of a general (index-table) code: H in compressed-row form."""

    def __init__(self, row_ptr, col_idx, N: int):
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.handle = ldpc_code_create_sparse(row_ptr, col_idx, N)
        d = ldpc_code_dims(self.handle)
        self.N, self.M, self.E, self.K = d["N"], d["M"], d["E"], d["K"]
