"""Python binding of libvd, the GB300 soft-decision Viterbi decoder.

Thin ctypes layer over the C ABI declared in ``include/vd.h``: the functions
here carry the same names and only marshal arguments (torch tensors -> device
pointers, the current CUDA stream -> cudaStream_t).  Every step of decoding
runs in the library's CUDA kernels; there is no Python or CPU fallback, and
importing a function whose library is missing raises.

Method: arXiv 2011.13579 (parallel Viterbi decoding over overlapped frames,
radix-2 and radix-4 add-compare-select).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "VD_OK", "VD_EINVAL", "VD_ENOMEM", "VD_ECUDA", "VD_EUNSUPPORTED", "VD_ETIMEOUT", "VD_EBOUNDS",
    "VD_LLR_S8", "VD_LLR_S4", "VD_LLR_F16", "VD_LLR_HARD", "VD_TERMINATED", "VD_START_UNKNOWN",
    "VdError", "VdTune", "build", "lib", "vd_code_create", "vd_code_destroy", "vd_code_supported",
    "vd_decode", "vd_decode_batch", "vd_batch_plan_create", "vd_batch_plan_launch",
    "vd_batch_plan_info", "vd_batch_plan_packet_tune", "vd_batch_plan_status", "vd_batch_plan_destroy",
    "VdPacket", "VdBatchInfo", "BatchPlan", "VdServerConfig", "VdCompletion", "VdServerStats",
    "Server", "vd_server_create", "vd_server_submit", "vd_server_poll", "vd_server_stats_get",
    "vd_server_destroy", "vd_server_replay", "vd_server_submit_device", "vd_server_submit_many", "vd_bm_gate", "vd_decode_each", "vd_decode_tc", "vd_decode_host", "vd_decode_radix", "vd_int_peak", "vd_transmit", "vd_transmit_bytes", "transmit", "vd_get_tune", "vd_decode_noalloc", "vd_noalloc_scratch_limit", "vd_sync", "vd_num_frames", "vd_num_kept", "vd_scratch_bytes", "vd_release_scratch",
    "vd_last_error", "vd_version", "Code", "decode",
]

VD_OK, VD_EINVAL, VD_ENOMEM, VD_ECUDA, VD_EUNSUPPORTED, VD_ETIMEOUT, VD_EBOUNDS = 0, -1, -2, -3, -4, -5, -6
VD_LLR_S8, VD_LLR_S4, VD_LLR_F16, VD_LLR_HARD = 0, 1, 2, 3
VD_TERMINATED, VD_START_UNKNOWN = 1, 2

_STATUS = {0: "VD_OK", -1: "VD_EINVAL", -2: "VD_ENOMEM", -3: "VD_ECUDA", -4: "VD_EUNSUPPORTED",
           -5: "VD_ETIMEOUT", -6: "VD_EBOUNDS"}


class VdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class VdTune(ctypes.Structure):
    _fields_ = [("f", ctypes.c_int32), ("v", ctypes.c_int32), ("radix", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("form", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class VdPacket(ctypes.Structure):
    _fields_ = [("code_id", ctypes.c_int32), ("llr_type", ctypes.c_int32),
                ("llr_offset", ctypes.c_int64), ("n_info", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("f", ctypes.c_int32), ("v", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("out_word_offset", ctypes.c_int64)]


class VdBatchInfo(ctypes.Structure):
    _fields_ = [("n_packets", ctypes.c_int64), ("n_frames", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("resident_warps", ctypes.c_int64), ("lanes", ctypes.c_int32),
                ("radix", ctypes.c_int32), ("n_launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class VdServerConfig(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_packet_bits", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("radix", ctypes.c_int32), ("f7", ctypes.c_int32),
                ("v7", ctypes.c_int32), ("f9", ctypes.c_int32), ("v9", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class VdCompletion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_words", ctypes.c_int32),
                ("word_offset", ctypes.c_int64), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class VdServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("bits_decoded", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("arena_used", ctypes.c_int64), ("error", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles libvd.so for sm_103a (nvcc) in-tree."""
    return _build.build(force=force)


def lib():
    """The loaded libvd.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libvd.so is not built ({_build.LIB}); call build() first")
        L = ctypes.CDLL(_build.LIB)
        P = ctypes.POINTER
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
        L.vd_code_create.argtypes = [P(vp), i32, i32, P(u32), i32, i32, P(ctypes.c_uint8), i32]
        L.vd_code_create.restype = i32
        L.vd_code_destroy.argtypes = [vp]
        L.vd_code_destroy.restype = None
        L.vd_code_supported.argtypes = [i32, i32, P(u32)]
        L.vd_code_supported.restype = i32
        L.vd_decode.argtypes = [vp, vp, i32, i64, i32, i32, i32, u32, vp, vp, P(VdTune), vp]
        L.vd_decode.restype = i32
        L.vd_num_frames.argtypes = [i64, i32]
        L.vd_num_frames.restype = i64
        L.vd_num_kept.argtypes = [vp, i64]
        L.vd_num_kept.restype = i64
        L.vd_scratch_bytes.argtypes = [vp, i64, i32, i32, i32, P(VdTune)]
        L.vd_scratch_bytes.restype = i64
        L.vd_decode_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, u32, vp, vp]
        L.vd_decode_noalloc.restype = i32
        L.vd_noalloc_scratch_limit.argtypes = []
        L.vd_noalloc_scratch_limit.restype = i64
        L.vd_batch_plan_create.argtypes = [P(vp), P(vp), i32, P(VdPacket), i64, P(VdTune), vp]
        L.vd_batch_plan_create.restype = i32
        L.vd_batch_plan_launch.argtypes = [vp, vp, vp, vp]
        L.vd_batch_plan_launch.restype = i32
        L.vd_batch_plan_launch_graph.argtypes = [vp, vp, vp, vp]
        L.vd_batch_plan_launch_graph.restype = i32
        L.vd_batch_plan_launch_chained.argtypes = [vp, vp, vp, vp]
        L.vd_batch_plan_launch_chained.restype = i32
        L.vd_batch_plan_info.argtypes = [vp, P(VdBatchInfo)]
        L.vd_batch_plan_info.restype = i32
        L.vd_batch_plan_packet_tune.argtypes = [vp, P(ctypes.c_int32), P(ctypes.c_int32)]
        L.vd_batch_plan_packet_tune.restype = i32
        L.vd_batch_plan_status.argtypes = [vp, vp]
        L.vd_batch_plan_status.restype = i32
        L.vd_batch_plan_destroy.argtypes = [vp]
        L.vd_batch_plan_destroy.restype = None
        L.vd_decode_batch.argtypes = [P(vp), i32, P(VdPacket), i64, vp, vp, P(VdTune), vp]
        L.vd_decode_batch.restype = i32
        L.vd_server_create.argtypes = [P(vp), P(vp), i32, P(VdServerConfig)]
        L.vd_server_create.restype = i32
        L.vd_server_submit.argtypes = [vp, i32, i32, vp, i64, i64, u32, ctypes.c_uint64]
        L.vd_server_submit.restype = i32
        L.vd_server_poll.argtypes = [vp, P(VdCompletion), i64, P(u32), i64]
        L.vd_server_poll.restype = i64
        L.vd_server_stats_get.argtypes = [vp, P(VdServerStats)]
        L.vd_server_stats_get.restype = i32
        L.vd_server_destroy.argtypes = [vp]
        L.vd_server_destroy.restype = None
        L.vd_server_replay.argtypes = [vp, i64, P(i32), P(i32), vp, P(i64), P(i64), P(i64), P(u32), P(i64),
                                       i64, P(i64), P(u32), P(i64), P(i64)]
        L.vd_server_replay.restype = i32
        L.vd_server_replay_device.argtypes = L.vd_server_replay.argtypes
        L.vd_server_replay_device.restype = i32
        L.vd_server_submit_device.argtypes = [vp, i32, i32, vp, i64, i64, u32, ctypes.c_uint64]
        L.vd_server_submit_device.restype = i32
        L.vd_server_submit_many.argtypes = [vp, i64, P(ctypes.c_int32), P(ctypes.c_int32), vp, P(i64), P(i64),
                                            P(i64), P(u32), P(ctypes.c_uint64)]
        L.vd_server_submit_many.restype = i32
        L.vd_get_tune.argtypes = [vp, i32, i32, i32, i32, P(VdTune)]
        L.vd_get_tune.restype = i32
        L.vd_bm_gate.argtypes = [i32, vp, i64, i32, vp, vp, vp]
        L.vd_bm_gate.restype = i32
        L.vd_decode_host.argtypes = [vp, i32, P(vp), i32, i64, i32, i32, i32, u32, P(vp), vp]
        L.vd_decode_host.restype = i32
        L.vd_decode_radix.argtypes = [vp, vp, i64, i32, i32, i32, u32, vp, vp]
        L.vd_decode_radix.restype = i32
        L.vd_decode_tc.argtypes = [vp, vp, i64, i32, i32, u32, vp, vp]
        L.vd_decode_tc.restype = i32
        L.vd_decode_each.argtypes = [P(vp), i32, P(VdPacket), i64, vp, vp, i32, P(vp), i32]
        L.vd_decode_each.restype = i32
        L.vd_int_peak.argtypes = [i32, i64, i32, vp, vp, vp]
        L.vd_int_peak.restype = i32
        L.vd_transmit.argtypes = [vp, vp, i64, u32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, i32, vp, vp]
        L.vd_transmit.restype = i32
        L.vd_transmit_bytes.argtypes = [vp, i64, u32, i32]
        L.vd_transmit_bytes.restype = i64
        L.vd_sync.argtypes = [vp]
        L.vd_sync.restype = i32
        L.vd_release_scratch.argtypes = []
        L.vd_release_scratch.restype = i32
        L.vd_last_error.argtypes = []
        L.vd_last_error.restype = ctypes.c_char_p
        L.vd_version.argtypes = []
        L.vd_version.restype = i32
        _lib = L
        return L


def _check(status):
    if status != VD_OK:
        raise VdError(status, vd_last_error())
    return status


def _u32_array(vals):
    arr = (ctypes.c_uint32 * len(vals))(*[int(v) for v in vals])
    return arr


def vd_last_error() -> str:
    return (lib().vd_last_error() or b"").decode()


def vd_version() -> int:
    return lib().vd_version()


def vd_code_supported(K, gens) -> bool:
    return bool(lib().vd_code_supported(int(K), len(gens), _u32_array(gens)))


def vd_code_create(K, gens, rate=None, puncture=None):
    """Returns an opaque handle (int) to a new code object; raises VdError."""
    beta = len(gens)
    if puncture is not None:
        rows = [list(map(int, r)) for r in puncture]
        period = len(rows[0])
        flat = [x for r in rows for x in r]
        pbuf = (ctypes.c_uint8 * len(flat))(*flat)
        kept = sum(flat)
        rn, rd = rate if rate is not None else (period, kept)
    else:
        pbuf, period = None, 1
        rn, rd = rate if rate is not None else (1, beta)
    h = ctypes.c_void_p()
    _check(lib().vd_code_create(ctypes.byref(h), int(K), beta, _u32_array(gens), int(rn), int(rd),
                                pbuf, int(period)))
    return h.value


def vd_code_destroy(handle) -> None:
    if handle:
        lib().vd_code_destroy(ctypes.c_void_p(handle))


def vd_num_frames(n_info, f) -> int:
    return int(lib().vd_num_frames(int(n_info), int(f)))


def vd_num_kept(handle, T) -> int:
    return int(lib().vd_num_kept(ctypes.c_void_p(handle), int(T)))


def vd_scratch_bytes(handle, n_info, f, v, radix=2, tune=None) -> int:
    return int(lib().vd_scratch_bytes(ctypes.c_void_p(handle), int(n_info), int(f), int(v), int(radix),
                                      ctypes.byref(tune) if tune is not None else None))


def vd_sync(stream=None) -> None:
    """Waits for the stream and raises VdError if a kernel reported a device-side error."""
    _check(lib().vd_sync(_stream_handle(stream)))


def vd_bm_gate(variant, llr_words, n_pairs, n_stages, checksum, metrics=None, stream=None) -> None:
    """Branch-metric gate kernels (0: CUDA cores, 1: tensor cores) on device tensors."""
    _check(lib().vd_bm_gate(int(variant), ctypes.c_void_p(llr_words.data_ptr()), int(n_pairs), int(n_stages),
                            ctypes.c_void_p(checksum.data_ptr()),
                            ctypes.c_void_p(metrics.data_ptr()) if metrics is not None else None,
                            _stream_handle(stream)))


def vd_decode_host(handle, host_llrs, n_info, f, v, radix, flags, host_outs, stream=None,
                   llr_type=VD_LLR_S8) -> None:
    """vd_decode from host buffers: ``host_llrs`` / ``host_outs`` are lists of
    (preferably pinned) CPU tensors or numpy arrays, one per stream."""
    def ptr(x):
        return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    n = len(host_llrs)
    ins = (ctypes.c_void_p * n)(*[ptr(x) for x in host_llrs])
    outs = (ctypes.c_void_p * n)(*[ptr(x) for x in host_outs])
    _check(lib().vd_decode_host(ctypes.c_void_p(handle), n, ins, int(llr_type), int(n_info), int(f), int(v),
                                int(radix), int(flags), outs, _stream_handle(stream)))


def vd_decode_radix(handle, llr, n_info, f, v, rho, flags, out, stream=None) -> None:
    """The general radix-2^rho (Sec. VI) variant on device tensors."""
    _check(lib().vd_decode_radix(ctypes.c_void_p(handle), ctypes.c_void_p(llr.data_ptr()), int(n_info), int(f),
                                 int(v), int(rho), int(flags), ctypes.c_void_p(out.data_ptr()),
                                 _stream_handle(stream)))


def vd_decode_tc(handle, llr, n_info, f, v, flags, out, stream=None) -> None:
    """The tensor-core (Sec. VIII) radix-4 variant on device tensors."""
    _check(lib().vd_decode_tc(ctypes.c_void_p(handle), ctypes.c_void_p(llr.data_ptr()), int(n_info), int(f),
                              int(v), int(flags), ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))


def vd_decode_each(codes, packets, llr_arena, out_arena, radix, streams) -> None:
    """One vd_decode per packet from C (packets: VdPacket array or dict with
    f > 0 per packet), round-robin over ``streams`` (torch streams)."""
    arr, n = _packet_array(packets)
    sh = (ctypes.c_void_p * len(streams))(*[s.cuda_stream for s in streams])
    _check(lib().vd_decode_each(_code_handles(codes), len(codes), arr, n, ctypes.c_void_p(llr_arena.data_ptr()),
                                ctypes.c_void_p(out_arena.data_ptr()), int(radix), sh, len(streams)))


def vd_int_peak(variant, iters, n_blocks, cycles, sink, stream=None) -> None:
    """Integer-issue microbenchmark on device tensors: cycles (int64
    [n_blocks]) receives each block's SM-clock span, sink (int32
    [n_blocks * 1024]) the folded chains."""
    _check(lib().vd_int_peak(int(variant), int(iters), int(n_blocks), ctypes.c_void_p(cycles.data_ptr()),
                             ctypes.c_void_p(sink.data_ptr()), _stream_handle(stream)))


def vd_transmit(handle, bits, n_info, flags, sigma, seed, stream_id, llr_type, out, stream=None) -> None:
    """GPU transmitter and channel on device tensors: ``bits`` (packed info
    words), ``out`` (vd_transmit_bytes() bytes)."""
    _check(lib().vd_transmit(ctypes.c_void_p(handle), ctypes.c_void_p(bits.data_ptr()) if n_info else None,
                             int(n_info), int(flags), float(sigma), ctypes.c_uint64(int(seed) & (2**64 - 1)),
                             ctypes.c_uint64(int(stream_id) & (2**64 - 1)), int(llr_type),
                             ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))


def vd_transmit_bytes(handle, n_info, flags, llr_type) -> int:
    n = int(lib().vd_transmit_bytes(ctypes.c_void_p(handle), int(n_info), int(flags), int(llr_type)))
    if n < 0:
        raise VdError(VD_EINVAL, "vd_transmit_bytes: bad arguments")
    return n


def transmit(code, bits_words, n_info, sigma, seed, stream_id=0, terminated=False, llr_type=VD_LLR_S8,
             stream=None):
    """Allocates the received-value buffer (torch uint8, on the bits' device)
    and fills it with vd_transmit."""
    import torch
    flags = VD_TERMINATED if terminated else 0
    nb = vd_transmit_bytes(code.handle, n_info, flags, llr_type)
    out = torch.empty(max(nb, 1), dtype=torch.uint8, device=bits_words.device)
    vd_transmit(code.handle, bits_words, n_info, flags, sigma, seed, stream_id, llr_type, out, stream)
    return out[:nb]


def vd_get_tune(handle, llr_type, f, v, radix) -> "VdTune":
    """The kernel configuration vd_decode uses with tune=None."""
    t = VdTune()
    _check(lib().vd_get_tune(ctypes.c_void_p(handle), int(llr_type), int(f), int(v), int(radix),
                             ctypes.byref(t)))
    return t


def vd_release_scratch() -> None:
    _check(lib().vd_release_scratch())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def vd_decode(handle, llr, llr_type, n_info, f, v, radix, flags, out, pm=None, tune=None, stream=None):
    """Calls vd_decode on device tensors ``llr`` (received values) and ``out``
    (ceil(n_info/32) int32/uint32 words), optional ``pm`` (int32 frames x 2^(K-1))."""
    for name, t in (("llr", llr), ("out", out), ("pm", pm)):
        if t is not None and not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t is not None and not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    _check(lib().vd_decode(ctypes.c_void_p(handle), ctypes.c_void_p(llr.data_ptr()), int(llr_type),
                           int(n_info), int(f), int(v), int(radix), int(flags),
                           ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(pm.data_ptr()) if pm is not None else None,
                           ctypes.byref(tune) if tune is not None else None,
                           _stream_handle(stream)))


def vd_decode_noalloc(handle, llr, n_info, f, v, radix, flags, out, stream=None):
    """Calls vd_decode_noalloc: the stream decode with no device allocation
    (fixed scratch of vd_noalloc_scratch_limit() bytes; int8, unpunctured)."""
    for name, t in (("llr", llr), ("out", out)):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
    _check(lib().vd_decode_noalloc(ctypes.c_void_p(handle), ctypes.c_void_p(llr.data_ptr()),
                                   int(n_info), int(f), int(v), int(radix), int(flags),
                                   ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))


def vd_noalloc_scratch_limit() -> int:
    return int(lib().vd_noalloc_scratch_limit())


def _packet_array(packets):
    """packets: a ctypes VdPacket array, or a dict of equal-length numpy arrays
    with keys code_id, llr_type, llr_offset, n_info, flags, f, v, out_word_offset."""
    if isinstance(packets, ctypes.Array):
        return packets, len(packets)
    import numpy as np
    n = len(packets["n_info"])
    dt = np.dtype([("code_id", "<i4"), ("llr_type", "<i4"), ("llr_offset", "<i8"), ("n_info", "<i8"),
                   ("flags", "<u4"), ("f", "<i4"), ("v", "<i4"), ("reserved", "<i4"),
                   ("out_word_offset", "<i8")])
    assert dt.itemsize == ctypes.sizeof(VdPacket)
    rec = np.zeros(n, dtype=dt)
    for k in ("code_id", "llr_type", "llr_offset", "n_info", "flags", "f", "v", "out_word_offset"):
        if k in packets:
            rec[k] = packets[k]
    arr = (VdPacket * n).from_buffer_copy(rec.tobytes()) if n else (VdPacket * 0)()
    return arr, n


def _code_handles(codes):
    hs = [c.handle if isinstance(c, Code) else c for c in codes]
    return (ctypes.c_void_p * len(hs))(*hs)


def vd_batch_plan_create(codes, packets, tune=None, stream=None):
    arr, n = _packet_array(packets)
    h = ctypes.c_void_p()
    _check(lib().vd_batch_plan_create(ctypes.byref(h), _code_handles(codes), len(codes), arr, n,
                                      ctypes.byref(tune) if tune is not None else None,
                                      _stream_handle(stream)))
    return h.value


def vd_batch_plan_launch(plan, llr_arena, out_arena, stream=None, graph=False, chained=False):
    """graph: replay a captured CUDA graph; chained: vd_batch_plan_launch_chained
    (may overlap the kernel before it on the stream)."""
    if graph and chained:
        raise ValueError("graph and chained launches are exclusive")
    fn = (lib().vd_batch_plan_launch_graph if graph else
          lib().vd_batch_plan_launch_chained if chained else lib().vd_batch_plan_launch)
    _check(fn(ctypes.c_void_p(plan), ctypes.c_void_p(llr_arena.data_ptr()),
              ctypes.c_void_p(out_arena.data_ptr()), _stream_handle(stream)))


def vd_batch_plan_info(plan) -> VdBatchInfo:
    info = VdBatchInfo()
    _check(lib().vd_batch_plan_info(ctypes.c_void_p(plan), ctypes.byref(info)))
    return info


def vd_batch_plan_packet_tune(plan, n_packets):
    import numpy as np
    f = np.zeros(n_packets, dtype=np.int32)
    v = np.zeros(n_packets, dtype=np.int32)
    _check(lib().vd_batch_plan_packet_tune(ctypes.c_void_p(plan),
                                           f.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return f, v


def vd_batch_plan_status(plan, stream=None) -> None:
    _check(lib().vd_batch_plan_status(ctypes.c_void_p(plan), _stream_handle(stream)))


def vd_batch_plan_destroy(plan) -> None:
    if plan:
        lib().vd_batch_plan_destroy(ctypes.c_void_p(plan))


def vd_decode_batch(codes, packets, llr_arena, out_arena, tune=None, stream=None):
    arr, n = _packet_array(packets)
    _check(lib().vd_decode_batch(_code_handles(codes), len(codes), arr, n,
                                 ctypes.c_void_p(llr_arena.data_ptr()),
                                 ctypes.c_void_p(out_arena.data_ptr()),
                                 ctypes.byref(tune) if tune is not None else None,
                                 _stream_handle(stream)))


class BatchPlan:
    """Owning wrapper of a vd_batch_plan."""

    def __init__(self, codes, packets, tune=None, stream=None):
        self.codes = list(codes)
        self.n_packets = len(packets["n_info"]) if isinstance(packets, dict) else len(packets)
        self.handle = vd_batch_plan_create(self.codes, packets, tune=tune, stream=stream)

    def launch(self, llr_arena, out_arena, stream=None, graph=False, chained=False):
        vd_batch_plan_launch(self.handle, llr_arena, out_arena, stream=stream, graph=graph, chained=chained)

    def info(self):
        return vd_batch_plan_info(self.handle)

    def packet_tune(self):
        return vd_batch_plan_packet_tune(self.handle, self.n_packets)

    def status(self, stream=None):
        vd_batch_plan_status(self.handle, stream)

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            vd_batch_plan_destroy(h)

    def __del__(self):
        self.close()


def vd_server_create(codes, cfg=None):
    h = ctypes.c_void_p()
    _check(lib().vd_server_create(ctypes.byref(h), _code_handles(codes), len(codes),
                                  ctypes.byref(cfg) if cfg is not None else None))
    return h.value


def vd_server_submit(server, code_id, llr_type, host_llr, n_values, n_info, flags, tag):
    """host_llr: a contiguous numpy array (int8 values, or packed 4-bit bytes)."""
    _check(lib().vd_server_submit(ctypes.c_void_p(server), int(code_id), int(llr_type),
                                  ctypes.c_void_p(host_llr.ctypes.data), int(n_values), int(n_info),
                                  int(flags), ctypes.c_uint64(int(tag))))


def vd_server_poll(server, max_completions=4096, words_cap=1 << 22):
    """Returns a list of (VdCompletion, numpy uint32 words) for finished packets."""
    import numpy as np
    comp = (VdCompletion * max_completions)()
    words = np.empty(words_cap, dtype=np.uint32)
    n = lib().vd_server_poll(ctypes.c_void_p(server), comp, max_completions,
                             words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), words_cap)
    out = []
    for i in range(n):
        c = comp[i]
        out.append((c, words[c.word_offset:c.word_offset + c.n_words].copy()))
    return out


def vd_server_stats_get(server) -> VdServerStats:
    st = VdServerStats()
    _check(lib().vd_server_stats_get(ctypes.c_void_p(server), ctypes.byref(st)))
    return st


def vd_server_destroy(server) -> None:
    if server:
        lib().vd_server_destroy(ctypes.c_void_p(server))


def vd_server_submit_many(server, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, tags):
    """host_llr: a contiguous numpy array; the other arguments numpy arrays of
    one entry per packet (offsets in bytes)."""
    import numpy as np
    P = ctypes.POINTER
    arrs = [np.ascontiguousarray(code_id, np.int32), np.ascontiguousarray(llr_type, np.int32),
            np.ascontiguousarray(llr_offset, np.int64), np.ascontiguousarray(n_values, np.int64),
            np.ascontiguousarray(n_info, np.int64), np.ascontiguousarray(flags, np.uint32),
            np.ascontiguousarray(tags, np.uint64)]
    types = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
             ctypes.c_uint64]
    ptrs = [a.ctypes.data_as(P(t)) for a, t in zip(arrs, types)]
    _check(lib().vd_server_submit_many(ctypes.c_void_p(server), len(arrs[0]), ptrs[0], ptrs[1],
                                       ctypes.c_void_p(host_llr.ctypes.data), ptrs[2], ptrs[3], ptrs[4], ptrs[5],
                                       ptrs[6]))


def vd_server_submit_device(server, code_id, llr_type, d_llr, n_values, n_info, flags, tag):
    """d_llr: a contiguous CUDA tensor (or a device address) holding the packet's values."""
    addr = d_llr if isinstance(d_llr, int) else d_llr.data_ptr()
    _check(lib().vd_server_submit_device(ctypes.c_void_p(server), int(code_id), int(llr_type),
                                         ctypes.c_void_p(addr), int(n_values), int(n_info), int(flags),
                                         ctypes.c_uint64(int(tag))))


def vd_server_replay(server, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, arrival_ns,
                     timeout_ms=0, word_offset=None):
    """Open-loop replay: packet i is submitted arrival_ns[i] ns after the start.
    host_llr is one contiguous uint8/int8 numpy array holding every packet's
    values at llr_offset[i] — or a CUDA tensor, whose packets are then
    submitted in place (vd_server_replay_device).  Returns (latency_ns int64
    array, words uint32 array or None, span_ns)."""
    import numpy as np
    n = len(n_info)
    a_code = np.ascontiguousarray(code_id, dtype=np.int32)
    a_type = np.ascontiguousarray(llr_type, dtype=np.int32)
    a_off = np.ascontiguousarray(llr_offset, dtype=np.int64)
    a_nv = np.ascontiguousarray(n_values, dtype=np.int64)
    a_ni = np.ascontiguousarray(n_info, dtype=np.int64)
    a_fl = np.ascontiguousarray(flags, dtype=np.uint32)
    a_arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    device = hasattr(host_llr, "is_cuda") and host_llr.is_cuda
    if device:
        if not host_llr.is_contiguous():
            raise ValueError("the device LLR tensor must be contiguous")
        base = ctypes.c_void_p(host_llr.data_ptr())
    else:
        host = np.ascontiguousarray(host_llr)
        base = ctypes.c_void_p(host.ctypes.data)
    lat = np.empty(n, dtype=np.int64)
    words = None
    a_wo = None
    if word_offset is not None:
        a_wo = np.ascontiguousarray(word_offset, dtype=np.int64)
        total = int((a_wo + (a_ni + 31) // 32).max()) if n else 0
        words = np.zeros(max(total, 1), dtype=np.uint32)
    span = ctypes.c_int64(0)
    P = ctypes.POINTER

    def ptr(a, t):
        return a.ctypes.data_as(P(t)) if a is not None else None

    fn = lib().vd_server_replay_device if device else lib().vd_server_replay
    _check(fn(ctypes.c_void_p(server), n, ptr(a_code, ctypes.c_int32), ptr(a_type, ctypes.c_int32), base,
              ptr(a_off, ctypes.c_int64), ptr(a_nv, ctypes.c_int64), ptr(a_ni, ctypes.c_int64),
              ptr(a_fl, ctypes.c_uint32), ptr(a_arr, ctypes.c_int64), int(timeout_ms), ptr(lat, ctypes.c_int64),
              ptr(words, ctypes.c_uint32), ptr(a_wo, ctypes.c_int64), ctypes.byref(span)))
    return lat, words, int(span.value)


class Server:
    """Owning wrapper of a vd_server (continuous-batching decoder)."""

    def __init__(self, codes, cfg=None):
        self.codes = list(codes)
        self.handle = vd_server_create(self.codes, cfg)

    def submit(self, code_id, llr_type, host_llr, n_values, n_info, flags, tag):
        vd_server_submit(self.handle, code_id, llr_type, host_llr, n_values, n_info, flags, tag)

    def poll(self, max_completions=4096, words_cap=1 << 22):
        return vd_server_poll(self.handle, max_completions, words_cap)

    def stats(self):
        return vd_server_stats_get(self.handle)

    def replay(self, *args, **kw):
        return vd_server_replay(self.handle, *args, **kw)

    def submit_device(self, code_id, llr_type, d_llr, n_values, n_info, flags, tag):
        vd_server_submit_device(self.handle, code_id, llr_type, d_llr, n_values, n_info, flags, tag)

    def submit_many(self, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, tags):
        vd_server_submit_many(self.handle, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, tags)

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            vd_server_destroy(h)

    def __del__(self):
        self.close()


class Code:
    """Owning wrapper of a vd_code handle."""

    def __init__(self, K, gens, rate=None, puncture=None):
        self.K = int(K)
        self.gens = tuple(int(g) for g in gens)
        self.beta = len(self.gens)
        self.puncture = puncture
        self.handle = vd_code_create(K, gens, rate=rate, puncture=puncture)

    @property
    def n_states(self):
        return 1 << (self.K - 1)

    def n_kept(self, T):
        return vd_num_kept(self.handle, T)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            vd_code_destroy(h)


def decode(code: Code, llr, n_info, f, v, radix=2, terminated=False, start_unknown=False,
           llr_type=VD_LLR_S8, want_pm=False, lanes=0, stream=None, out=None):
    """Allocates the output words (torch, on llr's device) and decodes."""
    import torch
    nw = (int(n_info) + 31) // 32
    if out is None:
        out = torch.empty(max(nw, 1), dtype=torch.int32, device=llr.device)
    pm = None
    if want_pm:
        pm = torch.empty((max(vd_num_frames(n_info, f), 1), code.n_states), dtype=torch.int32,
                         device=llr.device)
    flags = (VD_TERMINATED if terminated else 0) | (VD_START_UNKNOWN if start_unknown else 0)
    tune = None
    if lanes:
        tune = VdTune()
        tune.lanes = int(lanes)
    vd_decode(code.handle, llr, llr_type, n_info, f, v, radix, flags, out, pm, tune, stream)
    return (out[:nw], pm) if want_pm else out[:nw]
