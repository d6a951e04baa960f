"""The benchmarked launch configurations at their full sizes.

* six 2^24-bit K=7 streams (f=256, v=42) as one persistent batch plan with
  the autotuned kernel shape — every stream bit-exact against the oracle;
* 65,536 uneven terminated packets (r1/2, r2/3, r3/4) as one autotuned plan
  replayed from a CUDA graph — every packet bit-exact against the oracle at
  the f/v the plan chose.
"""
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


def test_six_full_streams_one_plan_match_oracle():
    n = 1 << 24
    ebn0s = (1.0, 2.0, 3.0, 4.0, 5.0, 6.0)
    qs = [synth.segmented_stream(e).s8() for e in ebn0s]
    arena = torch.from_numpy(np.concatenate(qs).view(np.uint8)).cuda()
    k7 = vd.Code(7, synth.K7_GENS)
    pk = {"code_id": np.zeros(6, np.int32), "llr_type": np.zeros(6, np.int32),
          "llr_offset": np.arange(6) * 2 * n, "n_info": np.full(6, n), "flags": np.zeros(6, np.uint32),
          "f": np.full(6, 256, np.int32), "v": np.full(6, 42, np.int32),
          "out_word_offset": np.arange(6) * (n // 32)}
    tune = vd.VdTune()
    tune.radix = 2   # lanes left to the autotuner, as in the benchmark
    plan = vd.BatchPlan([k7], pk, tune=tune)
    out = torch.full((6 * n // 32,), -1, dtype=torch.int32, device="cuda")
    plan.launch(arena, out)
    plan.status()
    got = out.cpu().numpy().view(np.uint32).reshape(6, n // 32)
    oc = oracle.Code(7, synth.K7_GENS)
    for i, q in enumerate(qs):
        want = oracle.decode(oc, q.reshape(n, 2).astype(np.int32), n, 256, 42, threads=THREADS)
        assert np.array_equal(got[i], want), ebn0s[i]
    plan.close()


def test_full_packet_batch_every_packet_matches_oracle():
    batch = synth.uneven_packets()            # 65,536 packets
    pats = (None, synth.PUNCT_R23, synth.PUNCT_R34)
    codes = [vd.Code(7, synth.K7_GENS, puncture=None if p is None else p.tolist()) for p in pats]
    n = batch.n_packets
    pk = {"code_id": batch.rate_id.astype(np.int32), "llr_type": np.zeros(n, np.int32),
          "llr_offset": batch.llr_offset, "n_info": batch.n_info,
          "flags": np.full(n, vd.VD_TERMINATED, np.uint32), "f": np.zeros(n, np.int32),
          "v": np.zeros(n, np.int32), "out_word_offset": batch.out_word_offset}
    s = torch.cuda.Stream()
    plan = vd.BatchPlan(codes, pk, stream=s)
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).cuda()
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    out = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    plan.launch(llr, out, stream=s, graph=True)
    plan.launch(llr, out, stream=s, graph=True)   # a replay
    plan.status(stream=s)
    got = out.cpu().numpy().view(np.uint32)
    f, v = plan.packet_tune()
    plan.close()
    ocodes = [oracle.Code(7, synth.K7_GENS, puncture=p) for p in pats]
    want = oracle.decode_packets(ocodes, batch.rate_id, batch.llr_offset, batch.n_info, f, v, np.ones(n),
                                 np.zeros(n), batch.out_word_offset, batch.llr_s8, nw, threads=THREADS)
    if not np.array_equal(got, want):
        bad = [i for i in range(n) if not np.array_equal(
            got[batch.out_word_offset[i]: batch.out_word_offset[i] + (batch.n_info[i] + 31) // 32],
            want[batch.out_word_offset[i]: batch.out_word_offset[i] + (batch.n_info[i] + 31) // 32])]
        raise AssertionError(f"{len(bad)} of {n} packets differ, e.g. {bad[:5]}")


@pytest.mark.parametrize("radix", [2, 4])
def test_long_stream_persistent_decode_matches_oracle(radix):
    """A stream long enough for vd_decode's persistent form (at least one
    task per resident warp): 2^26 + 1000 info bits, K=7, f=256, v=42,
    terminated — whole stream bit-exact against the oracle."""
    n = (1 << 26) + 1000
    rng = np.random.Generator(np.random.PCG64(2026 + radix))
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 2.5, True)
    q = st.s8()
    oc = oracle.Code(7, synth.K7_GENS)
    want = oracle.decode(oc, q.reshape(st.T, 2).astype(np.int32), n, 256, 42, terminated=True,
                         threads=THREADS)
    code = vd.Code(7, synth.K7_GENS)
    got = vd.decode(code, torch.from_numpy(q.view(np.uint8)).cuda(), n, 256, 42, radix=radix,
                    terminated=True).cpu().numpy().view(np.uint32)
    vd.vd_sync()
    assert np.array_equal(got, want)
