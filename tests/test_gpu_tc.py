"""The tensor-core variant (vd_decode_tc: the paper's D = Theta_hat L + Lambda
radix-4 formulation, Sec. VIII) against the CPU oracle, bit for bit: frames
of several lengths and overlaps, terminated and unknown-start streams, odd
frame lengths (one radix-2 stage first), single-frame streams, and a full
2^24-bit stream of the segmented workload."""
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


def _tc(code, q, n, f, v, flags):
    llr = torch.from_numpy(np.ascontiguousarray(q).view(np.uint8)).cuda()
    out = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    vd.vd_decode_tc(code.handle, llr, n, f, v, flags, out)
    vd.vd_sync()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,f,v", [(5000, 256, 42), (4099, 128, 21), (3000, 64, 7), (777, 1024, 10),
                                   (10_000, 256, 0), (2048, 32, 33)])
@pytest.mark.parametrize("terminated,start_unknown", [(False, False), (True, False), (False, True)])
def test_tc_matches_oracle(n, f, v, terminated, start_unknown):
    rng = np.random.Generator(np.random.PCG64(1300 + n + f + v + 7 * terminated + 3 * start_unknown))
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 2.0, terminated)
    q = st.s8()
    code = vd.Code(7, synth.K7_GENS)
    flags = (vd.VD_TERMINATED if terminated else 0) | (vd.VD_START_UNKNOWN if start_unknown else 0)
    got = _tc(code, q, n, f, v, flags)
    want = oracle.decode(oracle.Code(7, synth.K7_GENS), q.reshape(st.T, 2).astype(np.int32), n, f, v,
                         terminated=terminated, start_unknown=start_unknown, threads=THREADS)
    assert np.array_equal(got, want)


def test_tc_adversarial_ties_and_saturation():
    """All-zero LLRs (every candidate ties) and saturated +-127 LLRs."""
    code = vd.Code(7, synth.K7_GENS)
    oc = oracle.Code(7, synth.K7_GENS)
    rng = np.random.Generator(np.random.PCG64(1399))
    n = 3001
    for q in (np.zeros(2 * n, np.int8), rng.choice(np.array([-127, 127], np.int8), size=2 * n),
              rng.choice(np.array([-1, 0, 1], np.int8), size=2 * n)):
        for flags in (0, vd.VD_START_UNKNOWN):
            got = _tc(code, q, n, 256, 42, flags)
            want = oracle.decode(oc, q.reshape(n, 2).astype(np.int32), n, 256, 42,
                                 start_unknown=bool(flags), threads=THREADS)
            assert np.array_equal(got, want), flags


def test_tc_full_stream_matches_vd_decode():
    n = 1 << 24
    q = synth.segmented_stream(2.0).s8()
    code = vd.Code(7, synth.K7_GENS)
    got = _tc(code, q, n, 256, 42, 0)
    ref = vd.decode(code, torch.from_numpy(q.view(np.uint8)).cuda(), n, 256, 42).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)


def test_tc_rejects_unsupported():
    k9 = vd.Code(9, synth.K9_GENS)
    x = torch.zeros(3 * 1000, dtype=torch.int8, device="cuda")
    o = torch.zeros(32, dtype=torch.int32, device="cuda")
    with pytest.raises(vd.VdError) as e:
        vd.vd_decode_tc(k9.handle, x, 1000, 256, 42, 0, o)
    assert e.value.status == vd.VD_EUNSUPPORTED
