"""vd_decode_host: decoding straight from host memory through the C ABI (the
library uploads, decodes and downloads, overlapping one stream's upload with
another's decode).  Its words must equal vd_decode's bit for bit, for several
streams per call, on repeated calls (cached plans) and after the stream
configuration changes; one stream is also checked against the oracle."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2011_13579_gb300 as vd  # noqa: E402
from paper_2011_13579_gb300 import synth  # noqa: E402

THREADS = max(1, len(os.sched_getaffinity(0)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vd.build()
    yield


def _run(code, qs, n, f, v, radix, flags):
    ins = [torch.from_numpy(np.ascontiguousarray(q).view(np.uint8)).pin_memory() for q in qs]
    outs = [torch.full(((n + 31) // 32,), -1, dtype=torch.int32).pin_memory() for _ in qs]
    s = torch.cuda.Stream()
    vd.vd_decode_host(code.handle, ins, n, f, v, radix, flags, outs, stream=s)
    s.synchronize()
    vd.vd_sync(s)
    return [o.numpy().view(np.uint32).copy() for o in outs]


def _device(code, q, n, f, v, radix, flags):
    llr = torch.from_numpy(np.ascontiguousarray(q).view(np.uint8)).cuda()
    out = vd.decode(code, llr, n, f, v, radix=radix, terminated=bool(flags & vd.VD_TERMINATED))
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("radix", [2, 4])
def test_host_matches_device_decode(radix):
    code = vd.Code(7, synth.K7_GENS)
    n = 300_000 + 32 * 7
    qs = [synth.segmented_stream(e, n_info=n).s8() for e in (1.0, 2.5, 4.0)]
    for _ in range(2):   # the second call reuses the cached plans and device copies
        got = _run(code, qs, n, 256, 42, radix, 0)
        for q, g in zip(qs, got):
            assert np.array_equal(g, _device(code, q, n, 256, 42, radix, 0))


def test_host_config_change_and_oracle():
    code = vd.Code(7, synth.K7_GENS)
    rng = np.random.Generator(np.random.PCG64(1500))
    n = 100_003
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 2.0, True)
    q = st.s8()
    got = _run(code, [q, q], n, 128, 30, 2, vd.VD_TERMINATED)
    want = oracle.decode(oracle.Code(7, synth.K7_GENS), q.reshape(st.T, 2).astype(np.int32), n, 128, 30,
                         terminated=True, threads=THREADS)
    assert np.array_equal(got[0], want) and np.array_equal(got[1], want)
    # a different configuration on the same stream rebuilds the plans
    got = _run(code, [q], n, 256, 42, 2, vd.VD_TERMINATED)
    assert np.array_equal(got[0], _device(code, q, n, 256, 42, 2, vd.VD_TERMINATED))


def test_host_k9():
    code = vd.Code(9, synth.K9_GENS)
    n = 200_000
    q = synth.precision_stream(1.0, n_info=n).s8()
    got = _run(code, [q], n, 512, 64, 2, 0)
    assert np.array_equal(got[0], _device(code, q, n, 512, 64, 2, 0))
