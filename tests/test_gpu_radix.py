"""The general radix-2^rho variant (vd_decode_radix, Sec. VI, Eq. general:S)
against the CPU oracle, bit for bit, for rho = 1, 2, 3 (radix 2, 4, 8) on
both codes: frame lengths that are and are not multiples of rho (radix-2
steps first), terminated and unknown-start streams, single frames, ties."""
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


def _radix(code, q, n, f, v, rho, flags):
    llr = torch.from_numpy(np.ascontiguousarray(q).view(np.uint8)).cuda()
    out = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    vd.vd_decode_radix(code.handle, llr, n, f, v, rho, flags, out)
    vd.vd_sync()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (9, synth.K9_GENS)])
@pytest.mark.parametrize("rho", [1, 2, 3])
@pytest.mark.parametrize("n,f,v,terminated,start_unknown", [(4001, 256, 42, False, False),
                                                            (3000, 128, 20, True, False),
                                                            (2500, 96, 13, False, True),
                                                            (701, 4096, 0, True, False)])
def test_radix_matches_oracle(K, gens, rho, n, f, v, terminated, start_unknown):
    rng = np.random.Generator(np.random.PCG64(1700 + K + rho + n))
    st = synth.make_stream(rng, K, gens, n, 1.5, terminated)
    q = st.s8()
    code = vd.Code(K, gens)
    flags = (vd.VD_TERMINATED if terminated else 0) | (vd.VD_START_UNKNOWN if start_unknown else 0)
    got = _radix(code, q, n, f, v, rho, flags)
    want = oracle.decode(oracle.Code(K, gens), q.reshape(st.T, len(gens)).astype(np.int32), n, f, v,
                         terminated=terminated, start_unknown=start_unknown, threads=THREADS)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("rho", [1, 2, 3])
def test_radix_ties(rho):
    """Erasure-heavy small LLRs: many equal candidates, decided by the tie order."""
    code = vd.Code(7, synth.K7_GENS)
    rng = np.random.Generator(np.random.PCG64(1790 + rho))
    n = 3001
    q = rng.choice(np.array([-1, 0, 0, 0, 1], np.int8), size=2 * n)
    got = _radix(code, q, n, 256, 42, rho, 0)
    want = oracle.decode(oracle.Code(7, synth.K7_GENS), q.reshape(n, 2).astype(np.int32), n, 256, 42,
                         threads=THREADS)
    assert np.array_equal(got, want)


def test_radix_rejects_bad_rho():
    code = vd.Code(7, synth.K7_GENS)
    x = torch.zeros(2000, dtype=torch.int8, device="cuda")
    o = torch.zeros(32, dtype=torch.int32, device="cuda")
    with pytest.raises(vd.VdError) as e:
        vd.vd_decode_radix(code.handle, x, 1000, 256, 42, 4, 0, o)
    assert e.value.status == vd.VD_EINVAL
