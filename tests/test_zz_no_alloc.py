"""vd_decode_noalloc: the decode entry point for callers that may not
allocate device memory while they run (a real-time receiver thread that
cannot wait for cudaMalloc, a program whose device memory is fixed up front
by another allocator or budget).  Its survivor scratch is a fixed device
array inside the library, shared by every call.

Its output must equal vd_decode's, bit for bit — the same tolerance as every
integer decode test here — on two calls in a row, since every call reuses
the same array; at the largest stream the array holds it must equal the
oracle's bits.  The call must leave the device's free memory unchanged, and
vd_sync must read its status word.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2011_13579_gb300 as vd  # noqa: E402
from paper_2011_13579_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vd.build()
    yield


def _flags(terminated=False, start_unknown=False):
    return (vd.VD_TERMINATED if terminated else 0) | (vd.VD_START_UNKNOWN if start_unknown else 0)


def _decode_both(code, llr, n, f, v, radix, flags):
    nw = (n + 31) // 32
    ref = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    vd.vd_decode(code.handle, llr, vd.VD_LLR_S8, n, f, v, radix, flags, ref)
    outs = []
    for _ in range(2):   # two calls in a row share the fixed scratch
        o = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
        vd.vd_decode_noalloc(code.handle, llr, n, f, v, radix, flags, o)
        outs.append(o)
    vd.vd_sync()         # reads the noalloc status word: no device-side error
    return ref.cpu().numpy(), [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("radix", [2, 4])
def test_noalloc_matches_vd_decode_k7(radix):
    code = vd.Code(7, synth.K7_GENS)
    n = (1 << 20) + 77
    llr = torch.from_numpy(synth.segmented_stream(2.0, n_info=n).s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 256, 42, radix, 0)
    for o in outs:
        assert np.array_equal(o, ref)


@pytest.mark.parametrize("radix", [2, 4])
def test_noalloc_matches_vd_decode_k9_terminated(radix):
    code = vd.Code(9, synth.K9_GENS)
    rng = np.random.Generator(np.random.PCG64(77))
    n = 100_000
    st = synth.make_stream(rng, 9, synth.K9_GENS, n, 1.5, True)
    llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 512, 64, radix, _flags(terminated=True))
    for o in outs:
        assert np.array_equal(o, ref)


@pytest.mark.parametrize("radix", [2, 4])
def test_noalloc_unknown_start(radix):
    code = vd.Code(7, synth.K7_GENS)
    rng = np.random.Generator(np.random.PCG64(78))
    n = 50_000 + 13
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 1.0, False)
    llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 256, 42, radix, _flags(start_unknown=True))
    for o in outs:
        assert np.array_equal(o, ref)


@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (9, synth.K9_GENS)])
def test_noalloc_single_frame(K, gens):
    """f >= n_info: one full-length frame (terminated), so the frame spans the
    whole stream."""
    code = vd.Code(K, gens)
    rng = np.random.Generator(np.random.PCG64(79 + K))
    n = 3001
    st = synth.make_stream(rng, K, gens, n, 2.0, True)
    llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 4096, 0, 2, _flags(terminated=True))
    for o in outs:
        assert np.array_equal(o, ref)


def test_noalloc_allocates_nothing():
    """After the set-up call (n_info = 0) and with the library's scratch pool
    released, two decodes leave the device's free memory exactly unchanged;
    their output equals vd_decode's, which runs only afterwards."""
    code = vd.Code(7, synth.K7_GENS)
    n = 300_000
    llr = torch.from_numpy(synth.segmented_stream(3.0, n_info=n).s8().view(np.uint8)).cuda()
    nw = (n + 31) // 32
    outs = [torch.full((nw,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    vd.vd_decode_noalloc(code.handle, llr, 0, 256, 42, 2, 0, outs[0])   # set-up only
    vd.vd_release_scratch()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for o in outs:
        vd.vd_decode_noalloc(code.handle, llr, n, 256, 42, 2, 0, o)
    vd.vd_sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    vd.vd_decode(code.handle, llr, vd.VD_LLR_S8, n, 256, 42, 2, 0, ref)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)


def _accepted(code, llr, n, out):
    try:
        vd.vd_decode_noalloc(code.handle, llr, n, 256, 42, 2, 0, out)
        return True
    except vd.VdError as e:
        assert e.status == vd.VD_EINVAL
        return False


def test_noalloc_largest_stream_matches_oracle():
    """The largest K=7 stream (f=256, v=42) whose scratch fits the fixed array
    — found by the entry point's own acceptance — decodes to the oracle's
    bits on two calls in a row; one more bit is rejected."""
    code = vd.Code(7, synth.K7_GENS)
    hi = 1 << 23
    st = synth.segmented_stream(2.5, n_info=hi)
    llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
    probe = torch.empty(hi // 32, dtype=torch.int32, device="cuda")
    lo = 1 << 16
    assert _accepted(code, llr, lo, probe) and not _accepted(code, llr, hi, probe)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _accepted(code, llr, mid, probe):
            lo = mid
        else:
            hi = mid
    n = lo
    torch.cuda.synchronize()
    q = st.s8()[: 2 * n].reshape(n, 2).astype(np.int32)
    want = oracle.decode(oracle.Code(7, synth.K7_GENS), q, n, 256, 42, threads=16)
    nw = (n + 31) // 32
    for _ in range(2):
        o = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
        vd.vd_decode_noalloc(code.handle, llr, n, 256, 42, 2, 0, o)
        vd.vd_sync()
        assert np.array_equal(o.cpu().numpy().view(np.uint32), want)
    assert not _accepted(code, llr, n + 1, probe)


def test_noalloc_rejects_streams_beyond_its_scratch():
    code = vd.Code(7, synth.K7_GENS)
    n = 1 << 24   # needs ~180 MB of survivor scratch
    llr = torch.zeros(2 * n, dtype=torch.int8, device="cuda")
    out = torch.zeros(n // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(vd.VdError) as e:
        vd.vd_decode_noalloc(code.handle, llr, n, 256, 42, 2, 0, out)
    assert e.value.status == vd.VD_EINVAL
    assert str(vd.vd_noalloc_scratch_limit()) in str(e.value)
