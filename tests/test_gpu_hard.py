"""Hard-decision input (Sec. II-C, hard-decision mode) on the GPU vs the
hard-decision oracle (minimum Hamming distance), bit for bit, through the
C ABI: stream decodes (K=7 and K=9, punctured, radix 2 and 4, terminated
and unknown start) and a batch that mixes hard-decision and int8 packets.
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


def _pat(name):
    return {"r12": None, "r23": synth.PUNCT_R23, "r34": synth.PUNCT_R34}[name]


@pytest.mark.parametrize("K,gens,pat", [(7, synth.K7_GENS, "r12"), (7, synth.K7_GENS, "r23"),
                                         (7, synth.K7_GENS, "r34"), (9, synth.K9_GENS, "r12")])
@pytest.mark.parametrize("radix", [2, 4])
@pytest.mark.parametrize("terminated,start_unknown", [(True, False), (False, True)])
def test_hard_stream_matches_oracle(K, gens, pat, radix, terminated, start_unknown):
    pattern = _pat(pat)
    rng = np.random.Generator(np.random.PCG64(9100 + K + radix + 3 * terminated))
    n = 40_000 + 77
    f, v = (256, 42) if K == 7 else (512, 64)
    st = synth.make_stream(rng, K, gens, n, 4.0, terminated, pattern=pattern)
    hard = st.hard()
    code = vd.Code(K, gens, puncture=None if pattern is None else pattern.tolist())
    oc = oracle.Code(K, gens, puncture=pattern)
    llr = torch.from_numpy(synth.pack_hard(hard)).cuda()
    got = vd.decode(code, llr, n, f, v, radix=radix, terminated=terminated, start_unknown=start_unknown,
                    llr_type=vd.VD_LLR_HARD).cpu().numpy().view(np.uint32)
    vd.vd_sync()
    want = oracle.decode_hard(oc, oracle.depuncture_hard(oc, hard, st.T), n, f, v, terminated=terminated,
                              start_unknown=start_unknown)
    assert np.array_equal(got, want)


def test_hard_and_int8_packets_in_one_batch():
    """A batch of K=7 packets, half hard-decision and half int8, r1/2 and
    r3/4: each packet equals its own oracle (hard or soft) at the plan's f/v."""
    rng = np.random.Generator(np.random.PCG64(9200))
    pats = (None, synth.PUNCT_R34)
    codes = [vd.Code(7, synth.K7_GENS, puncture=None if p is None else p.tolist()) for p in pats]
    n_pk = 300
    lens = synth.packet_lengths(rng, n_pk, lo=96, hi=3000)
    arena, meta = [], []
    byte_off, word_off = 0, 0
    for i in range(n_pk):
        cid = i % 2
        hard = (i // 2) % 2 == 0
        st = synth.make_stream(rng, 7, synth.K7_GENS, int(lens[i]), 3.0, True, pattern=pats[cid])
        raw = synth.pack_hard(st.hard()) if hard else st.s8().view(np.uint8)
        pad = (-len(raw)) % 16
        arena.append(np.concatenate([raw, np.zeros(pad, np.uint8)]))
        meta.append((cid, hard, byte_off, word_off, st))
        byte_off += len(raw) + pad
        word_off += (int(lens[i]) + 31) // 32
    pk = {"code_id": np.array([m[0] for m in meta], np.int32),
          "llr_type": np.array([vd.VD_LLR_HARD if m[1] else vd.VD_LLR_S8 for m in meta], np.int32),
          "llr_offset": np.array([8 * m[2] if m[1] else m[2] for m in meta], np.int64),
          "n_info": lens.astype(np.int64), "flags": np.full(n_pk, vd.VD_TERMINATED, np.uint32),
          "f": np.zeros(n_pk, np.int32), "v": np.zeros(n_pk, np.int32),
          "out_word_offset": np.array([m[3] for m in meta], np.int64)}
    plan = vd.BatchPlan(codes, pk)
    f, v = plan.packet_tune()
    llr = torch.from_numpy(np.concatenate(arena)).cuda()
    out = torch.full((word_off,), -1, dtype=torch.int32, device="cuda")
    plan.launch(llr, out)
    plan.status()
    got = out.cpu().numpy().view(np.uint32)
    plan.close()
    for i, (cid, hard, _, wo, st) in enumerate(meta):
        oc = oracle.Code(7, synth.K7_GENS, puncture=pats[cid])
        n = int(lens[i])
        if hard:
            want = oracle.decode_hard(oc, oracle.depuncture_hard(oc, st.hard(), st.T), n, int(f[i]), int(v[i]),
                                      terminated=True)
        else:
            full = oracle.depuncture(oc, st.s8().astype(np.int32), st.T)
            want = oracle.decode(oc, full, n, int(f[i]), int(v[i]), terminated=True)
        assert np.array_equal(got[wo: wo + want.size], want), i
