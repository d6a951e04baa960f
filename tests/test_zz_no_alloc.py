"""vd_decode_noalloc: the decode entry point for callers that may not
allocate device memory while they run (its survivor scratch is a fixed
device array inside the library).  Its output must equal vd_decode's, bit for
bit — the same tolerance as every integer decode test here — on two calls in
a row, since every call reuses the same array.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2011_13579_gb300 as vd  # noqa: E402
from paper_2011_13579_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vd.build()
    yield


def _decode_both(code, llr, n, f, v, radix, flags):
    nw = (n + 31) // 32
    ref = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    vd.vd_decode(code.handle, llr, vd.VD_LLR_S8, n, f, v, radix, flags, ref)
    outs = []
    for _ in range(2):   # two calls in a row share the fixed scratch
        o = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
        vd.vd_decode_noalloc(code.handle, llr, n, f, v, radix, flags, o)
        outs.append(o)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("radix", [2, 4])
def test_noalloc_matches_vd_decode_k7(radix):
    code = vd.Code(7, synth.K7_GENS)
    n = (1 << 20) + 77
    llr = torch.from_numpy(synth.segmented_stream(2.0, n_info=n).s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 256, 42, radix, 0)
    for o in outs:
        assert np.array_equal(o, ref)


def test_noalloc_matches_vd_decode_k9_terminated():
    code = vd.Code(9, synth.K9_GENS)
    rng = np.random.Generator(np.random.PCG64(77))
    n = 100_000
    st = synth.make_stream(rng, 9, synth.K9_GENS, n, 1.5, True)
    llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
    ref, outs = _decode_both(code, llr, n, 512, 64, 2, vd.VD_TERMINATED)
    for o in outs:
        assert np.array_equal(o, ref)


def test_noalloc_rejects_streams_beyond_its_scratch():
    code = vd.Code(7, synth.K7_GENS)
    n = 1 << 24   # needs ~180 MB of survivor scratch
    llr = torch.zeros(2 * n, dtype=torch.int8, device="cuda")
    out = torch.zeros(n // 32, dtype=torch.int32, device="cuda")
    with pytest.raises(vd.VdError) as e:
        vd.vd_decode_noalloc(code.handle, llr, n, 256, 42, 2, 0, out)
    assert e.value.status == vd.VD_EINVAL
    assert str(vd.vd_noalloc_scratch_limit()) in str(e.value)
