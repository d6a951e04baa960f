"""Plain CPU reference (oracle) for the Viterbi decoder — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The decoder library never does; it
shares no code with it.

The arithmetic lives in ``viterbi_oracle.c`` (plain C, int64 / fp64 metrics,
radix-2, Algorithms 1 and 2 of arXiv 2011.13579, frames with overlap as in
Sec. III).  This module compiles it with gcc into ``oracle/_build`` and wraps
it with ctypes over numpy arrays.

Every function is pinned by ``tests/test_oracle_pins.py`` against facts that
do not come from the oracle itself (noiseless channel, brute-force maximum
likelihood, re-encoding, the paper's trellis theorems, textbook code facts).
The per-frame canonical metric vector of ``decode(want_pm=True)`` and the
``min_gap`` / ``max_abs_pm`` outputs of ``decode_f64`` are pinned by
enumerating every path of small frames.  Parity unpinned: absolute BER
values (the paper prints none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "viterbi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_BETA = 4
MAX_PERIOD = 8


class _Code(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int),
        ("beta", ctypes.c_int),
        ("gens", ctypes.c_uint32 * MAX_BETA),
        ("period", ctypes.c_int),
        ("punct", (ctypes.c_uint8 * MAX_PERIOD) * MAX_BETA),
    ]


def build(force: bool = False) -> str:
    """Compiles the C oracle (gcc, portable flags: no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        i64, i32, u32, u8, dbl = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.c_uint8, ctypes.c_double)
        lib.or_decode_i64.argtypes = [P(_Code), P(i32), i64, ctypes.c_int, ctypes.c_int,
                                      i64, i64, P(u32), P(i64), ctypes.c_int]
        lib.or_decode_i64.restype = ctypes.c_int
        lib.or_decode_f64.argtypes = [P(_Code), P(dbl), i64, ctypes.c_int, ctypes.c_int,
                                      i64, i64, P(u32), P(dbl), P(dbl), ctypes.c_int]
        lib.or_decode_f64.restype = ctypes.c_int
        lib.or_depuncture_i32.argtypes = [P(_Code), P(i32), i64, i64, P(i32)]
        lib.or_depuncture_i32.restype = i64
        lib.or_depuncture_f64.argtypes = [P(_Code), P(dbl), i64, i64, P(dbl)]
        lib.or_depuncture_f64.restype = i64
        lib.or_encode.argtypes = [P(_Code), P(u8), i64, P(u8)]
        lib.or_encode.restype = None
        lib.or_encode_from.argtypes = [P(_Code), u32, P(u8), i64, P(u8)]
        lib.or_encode_from.restype = None
        lib.or_num_windows.argtypes = [i64, i64]
        lib.or_num_windows.restype = i64
        lib.or_trace_full_i64.argtypes = [P(_Code), P(i32), i64, ctypes.c_int, ctypes.c_int,
                                          i64, i64, i64, P(u8), P(u32), P(i64), P(i64)]
        lib.or_trace_full_i64.restype = i64
        lib.or_decode_frames_i64.argtypes = [P(_Code), P(i32), i64, ctypes.c_int, ctypes.c_int,
                                             i64, i64, P(i64), i64, P(u8), P(i64)]
        lib.or_decode_frames_i64.restype = ctypes.c_int
        lib.or_decode_hard.argtypes = [P(_Code), P(u8), i64, ctypes.c_int, ctypes.c_int, i64, i64, P(u32)]
        lib.or_decode_hard.restype = ctypes.c_int
        u64 = ctypes.c_uint64
        lib.or_philox4x64.argtypes = [P(u64), P(u64), P(u64)]
        lib.or_philox4x64.restype = None
        lib.or_transmit.argtypes = [P(_Code), P(u8), i64, ctypes.c_int, dbl, u64, u64, P(dbl), i64]
        lib.or_transmit.restype = i64
        lib.or_decode_packets_i64.argtypes = [P(_Code), P(_Packet), i64, P(ctypes.c_int8), P(u32), ctypes.c_int]
        lib.or_decode_packets_i64.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class _Packet(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("terminated", ctypes.c_int32), ("start_unknown", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("kept_off", ctypes.c_int64), ("n_info", ctypes.c_int64),
                ("f", ctypes.c_int64), ("v", ctypes.c_int64), ("out_word_off", ctypes.c_int64)]


class Code:
    """A convolutional code (k, beta generators, optional puncture pattern).

    gens are given in octal notation as Python ints written in octal, e.g.
    ``0o171``; the leftmost binary digit of a generator taps the current
    input (Sec. II-A).  ``puncture`` is a beta x period 0/1 matrix, rows =
    output bit b, columns = stage phase t mod period.
    """

    def __init__(self, K, gens, puncture=None):
        self.K = int(K)
        self.gens = [int(g) for g in gens]
        self.beta = len(self.gens)
        if not (1 <= self.beta <= MAX_BETA):
            raise ValueError("beta out of range")
        if puncture is None:
            puncture = np.ones((self.beta, 1), dtype=np.uint8)
        self.puncture = np.asarray(puncture, dtype=np.uint8)
        if self.puncture.shape[0] != self.beta or not (1 <= self.puncture.shape[1] <= MAX_PERIOD):
            raise ValueError("bad puncture pattern shape")
        self.period = self.puncture.shape[1]
        c = _Code()
        c.K = self.K
        c.beta = self.beta
        for b, g in enumerate(self.gens):
            c.gens[b] = g
        c.period = self.period
        for b in range(self.beta):
            for p in range(self.period):
                c.punct[b][p] = int(self.puncture[b, p])
        self._c = c

    @property
    def n_states(self):
        return 1 << (self.K - 1)

    def kept_per_period(self):
        return int(self.puncture.sum())

    def n_kept(self, T):
        """Number of transmitted LLRs for T stages."""
        full, rem = divmod(T, self.period)
        return full * self.kept_per_period() + int(self.puncture[:, :rem].sum())


def n_stages(code: Code, n_info: int, terminated: bool) -> int:
    return int(n_info) + (code.K - 1 if terminated else 0)


def depuncture(code: Code, kept, T: int):
    """Kept-only stream -> [T, beta] array with 0 at erased positions."""
    lib = _load()
    if np.issubdtype(np.asarray(kept).dtype, np.floating):
        src = np.ascontiguousarray(kept, dtype=np.float64)
        out = np.zeros((T, code.beta), dtype=np.float64)
        r = lib.or_depuncture_f64(ctypes.byref(code._c), _ptr(src, ctypes.c_double), src.size, T,
                                  _ptr(out, ctypes.c_double))
    else:
        src = np.ascontiguousarray(kept, dtype=np.int32)
        out = np.zeros((T, code.beta), dtype=np.int32)
        r = lib.or_depuncture_i32(ctypes.byref(code._c), _ptr(src, ctypes.c_int32), src.size, T,
                                  _ptr(out, ctypes.c_int32))
    if r < 0:
        raise ValueError("received stream too short for the puncture pattern")
    return out


def decode(code: Code, llr, n_info: int, f: int, v: int, terminated=False,
           start_unknown=False, threads: int = 1, want_pm=False):
    """Segmented (or full-length) decode with int64 metrics.

    ``llr`` is the depunctured [T, beta] integer array.  Returns packed
    LSB-first uint32 words, and with ``want_pm`` also the per-frame canonical
    final path metrics (lambda - min lambda), shape [n_windows, 2^(k-1)].
    """
    lib = _load()
    T = n_stages(code, n_info, terminated)
    llr = np.ascontiguousarray(llr, dtype=np.int32).reshape(-1)
    if llr.size != T * code.beta:
        raise ValueError(f"llr has {llr.size} values, expected {T * code.beta}")
    out = np.zeros(max(1, (n_info + 31) // 32), dtype=np.uint32)
    nwin = lib.or_num_windows(n_info, f)
    pm = np.zeros((max(nwin, 1), code.n_states), dtype=np.int64) if want_pm else None
    rc = lib.or_decode_i64(ctypes.byref(code._c), _ptr(llr, ctypes.c_int32), n_info,
                           int(bool(terminated)), int(bool(start_unknown)), f, v,
                           _ptr(out, ctypes.c_uint32),
                           _ptr(pm, ctypes.c_int64) if want_pm else None, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle decode failed ({rc})")
    out = out[: (n_info + 31) // 32]
    return (out, pm[:nwin]) if want_pm else out


def decode_full(code: Code, llr, n_info: int, terminated=False, start_unknown=False):
    """Full-length Viterbi: one frame over all stages (f >= n_info, v >= k-1)."""
    return decode(code, llr, n_info, f=max(n_info, 1), v=code.K - 1 + n_info,
                  terminated=terminated, start_unknown=start_unknown)


def decode_packets(codes, code_id, kept_off, n_info, f, v, terminated, start_unknown, out_word_off,
                   arena_s8, n_words, threads: int = 1):
    """Decodes a batch of packets (decode() per packet, after depuncturing
    its kept int8 values from ``arena_s8``), spread over host threads.
    Returns the packed output words (n_words)."""
    lib = _load()
    n = len(n_info)
    cs = (_Code * max(len(codes), 1))(*[c._c for c in codes])
    pk = (_Packet * max(n, 1))()
    for i in range(n):
        pk[i].code = int(code_id[i])
        pk[i].terminated = int(bool(terminated[i]))
        pk[i].start_unknown = int(bool(start_unknown[i]))
        pk[i].kept_off = int(kept_off[i])
        pk[i].n_info = int(n_info[i])
        pk[i].f = int(f[i])
        pk[i].v = int(v[i])
        pk[i].out_word_off = int(out_word_off[i])
    arena = np.ascontiguousarray(arena_s8, dtype=np.int8)
    out = np.zeros(max(int(n_words), 1), dtype=np.uint32)
    rc = lib.or_decode_packets_i64(cs, pk, n, _ptr(arena, ctypes.c_int8), _ptr(out, ctypes.c_uint32), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle decode_packets failed ({rc})")
    return out[: int(n_words)]


def decode_f64(code: Code, llr, n_info: int, f: int, v: int, terminated=False,
               start_unknown=False, threads: int = 1):
    """Segmented decode in fp64.  Returns (packed words, min_gap[nwin], max_abs_pm[nwin])."""
    lib = _load()
    T = n_stages(code, n_info, terminated)
    llr = np.ascontiguousarray(llr, dtype=np.float64).reshape(-1)
    if llr.size != T * code.beta:
        raise ValueError("llr size mismatch")
    out = np.zeros(max(1, (n_info + 31) // 32), dtype=np.uint32)
    nwin = lib.or_num_windows(n_info, f)
    gap = np.zeros(max(nwin, 1), dtype=np.float64)
    mx = np.zeros(max(nwin, 1), dtype=np.float64)
    rc = lib.or_decode_f64(ctypes.byref(code._c), _ptr(llr, ctypes.c_double), n_info,
                           int(bool(terminated)), int(bool(start_unknown)), f, v,
                           _ptr(out, ctypes.c_uint32), _ptr(gap, ctypes.c_double),
                           _ptr(mx, ctypes.c_double), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle decode_f64 failed ({rc})")
    return out[: (n_info + 31) // 32], gap[:nwin], mx[:nwin]


def depuncture_hard(code: Code, kept_bits, T: int):
    """Kept-only hard decisions (0/1) -> [T, beta] uint8 with 2 at erased positions."""
    kept = np.ascontiguousarray(kept_bits, dtype=np.int32).reshape(-1)
    full = depuncture(code, kept + 1, T)          # erased positions come back as 0
    return np.where(full == 0, 2, full - 1).astype(np.uint8)


def decode_hard(code: Code, rx, n_info: int, f: int, v: int, terminated=False, start_unknown=False):
    """Hard-decision decode (minimum Hamming distance, Sec. II-C).  ``rx`` is
    [T, beta] uint8: 0/1 received bits, 2 at erased positions.  Returns
    packed LSB-first uint32 words."""
    lib = _load()
    T = n_stages(code, n_info, terminated)
    rx = np.ascontiguousarray(rx, dtype=np.uint8).reshape(-1)
    if rx.size != T * code.beta:
        raise ValueError("rx size mismatch")
    out = np.zeros(max(1, (n_info + 31) // 32), dtype=np.uint32)
    rc = lib.or_decode_hard(ctypes.byref(code._c), _ptr(rx, ctypes.c_uint8), n_info,
                            int(bool(terminated)), int(bool(start_unknown)), f, v,
                            _ptr(out, ctypes.c_uint32))
    if rc != 0:
        raise RuntimeError(f"oracle decode_hard failed ({rc})")
    return out[: (n_info + 31) // 32]


def philox4x64(counter, key):
    """Philox4x64-10 of a 4-word counter and a 2-word key -> 4 uint64 words."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib.or_philox4x64(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def transmit(code: Code, bits, n_info: int, terminated: bool, sigma: float, seed: int, stream_id: int = 0):
    """Received samples y (float64, kept positions only) of the verification
    system (Sec. IX-B): encoder -> puncture -> BPSK -> AWGN with Philox4x64-10
    normals (key = (seed, stream_id), counter block k // 4 for value k)."""
    lib = _load()
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    T = n_stages(code, n_info, terminated)
    y = np.zeros(max(code.n_kept(T), 1), dtype=np.float64)
    n = lib.or_transmit(ctypes.byref(code._c), _ptr(b, ctypes.c_uint8), n_info, int(bool(terminated)),
                        float(sigma), int(seed) & (2**64 - 1), int(stream_id) & (2**64 - 1),
                        _ptr(y, ctypes.c_double), y.size)
    if n < 0:
        raise RuntimeError("oracle transmit failed")
    return y[:n]


def quantise(y, llr_type: str, sigma: float = 1.0):
    """The quantisers of the received samples: 's8' clip(rint(32 y), +-127),
    's4' clip(rint(2 y), +-7), 'f16' half(2 y / sigma^2), 'hard' (y < 0)."""
    y = np.asarray(y, dtype=np.float64)
    if llr_type == "s8":
        return np.clip(np.rint(32.0 * y), -127, 127).astype(np.int8)
    if llr_type == "s4":
        return np.clip(np.rint(2.0 * y), -7, 7).astype(np.int8)
    if llr_type == "f16":
        return (2.0 * y / (sigma * sigma)).astype(np.float16)
    if llr_type == "hard":
        return (y < 0.0).astype(np.uint8)
    raise ValueError(llr_type)


def decode_frames(code: Code, llr, n_info: int, f: int, v: int, frames, terminated=False,
                  start_unknown=False, want_pm=False):
    """Decodes only the listed frames.  Returns bits [n_sel, f] (uint8; only
    the first e-o of each row are meaningful) and optionally final metrics."""
    lib = _load()
    T = n_stages(code, n_info, terminated)
    llr = np.ascontiguousarray(llr, dtype=np.int32).reshape(-1)
    if llr.size != T * code.beta:
        raise ValueError("llr size mismatch")
    fr = np.ascontiguousarray(frames, dtype=np.int64)
    bits = np.zeros((fr.size, f), dtype=np.uint8)
    pm = np.zeros((fr.size, code.n_states), dtype=np.int64) if want_pm else None
    rc = lib.or_decode_frames_i64(ctypes.byref(code._c), _ptr(llr, ctypes.c_int32), n_info,
                                  int(bool(terminated)), int(bool(start_unknown)), f, v,
                                  _ptr(fr, ctypes.c_int64), fr.size, _ptr(bits, ctypes.c_uint8),
                                  _ptr(pm, ctypes.c_int64) if want_pm else None)
    if rc != 0:
        raise RuntimeError(f"oracle decode_frames failed ({rc})")
    return (bits, pm) if want_pm else bits


def encode(code: Code, bits):
    """FSM encoder from state 0 (bits already include any tail).  -> [n, beta] uint8."""
    lib = _load()
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.zeros((b.size, code.beta), dtype=np.uint8)
    lib.or_encode(ctypes.byref(code._c), _ptr(b, ctypes.c_uint8), b.size, _ptr(out, ctypes.c_uint8))
    return out


def encode_from(code: Code, state: int, bits):
    lib = _load()
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.zeros((b.size, code.beta), dtype=np.uint8)
    lib.or_encode_from(ctypes.byref(code._c), int(state), _ptr(b, ctypes.c_uint8), b.size,
                       _ptr(out, ctypes.c_uint8))
    return out


def trace_full(code: Code, llr, n_info: int, f: int, v: int, s: int, terminated=False,
               start_unknown=False):
    """Survivor path of frame s traced back to the frame's first stage.

    Returns (path_bits[W], origin_state, end_metric, init_metric, a) where a
    is the first stage of the frame.
    """
    lib = _load()
    T = n_stages(code, n_info, terminated)
    llr = np.ascontiguousarray(llr, dtype=np.int32).reshape(-1)
    path = np.zeros(T + 1, dtype=np.uint8)
    org = ctypes.c_uint32(0)
    em = ctypes.c_int64(0)
    im = ctypes.c_int64(0)
    W = lib.or_trace_full_i64(ctypes.byref(code._c), _ptr(llr, ctypes.c_int32), n_info,
                              int(bool(terminated)), int(bool(start_unknown)), f, v, s,
                              _ptr(path, ctypes.c_uint8), ctypes.byref(org), ctypes.byref(em),
                              ctypes.byref(im))
    if W < 0:
        raise ValueError("bad frame")
    a = max(0, s * f - v)
    return path[:W].copy(), int(org.value), int(em.value), int(im.value), a


def unpack_bits(words, n):
    """LSB-first packed words -> uint8 bit array of length n."""
    w = np.asarray(words, dtype=np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    return bits.reshape(-1)[:n]


def pack_bits(bits):
    """uint8 bits -> LSB-first packed uint32 words."""
    b = np.asarray(bits, dtype=np.uint8)
    n = b.size
    nw = (n + 31) // 32
    pad = np.zeros(nw * 32, dtype=np.uint64)
    pad[:n] = b
    w = (pad.reshape(nw, 32) << np.arange(32, dtype=np.uint64)[None, :]).sum(axis=1)
    return w.astype(np.uint32)
