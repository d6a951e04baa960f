"""Batched persistent decode vs the CPU oracle, packet by packet.

A batch shaped like the uneven-packet workload (log-uniform lengths, r1/2,
r2/3, r3/4 round-robin, terminated, int8) is decoded by one plan and checked
bit for bit against the oracle at the f/v the plan chose for each packet;
mixed K=7/K=9 batches with 4-bit packets, CUDA-graph replay, and the
one-launch-per-packet form must all give the same bits.
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
PATTERNS = (None, synth.PUNCT_R23, synth.PUNCT_R34)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vd.build()
    yield


@pytest.fixture(scope="module")
def k7_codes():
    return [vd.Code(7, synth.K7_GENS, puncture=None if p is None else p.tolist()) for p in PATTERNS]


def packets_of(batch, f=0, v=0):
    n = batch.n_packets
    return {"code_id": batch.rate_id.astype(np.int32), "llr_type": np.zeros(n, np.int32),
            "llr_offset": batch.llr_offset, "n_info": batch.n_info,
            "flags": np.full(n, vd.VD_TERMINATED, np.uint32), "f": np.full(n, f, np.int32),
            "v": np.full(n, v, np.int32), "out_word_offset": batch.out_word_offset}


def oracle_packet(batch, i, f, v):
    pat = PATTERNS[batch.rate_id[i]]
    oc = oracle.Code(7, synth.K7_GENS, puncture=pat)
    n = int(batch.n_info[i])
    T = n + 6
    kept = batch.llr_s8[batch.llr_offset[i]: batch.llr_offset[i] + batch.n_kept[i]].astype(np.int32)
    full = oracle.depuncture(oc, kept, T)
    return oracle.decode(oc, full, n, int(f), int(v), terminated=True)


def words_of(out, batch, i):
    o = int(batch.out_word_offset[i])
    return out[o: o + (int(batch.n_info[i]) + 31) // 32]


@pytest.mark.parametrize("radix", [2, 4])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_uneven_packets_match_oracle(k7_codes, radix, lanes):
    batch = synth.uneven_packets(n_packets=300, index=1, lo=96, hi=4000)
    tune = vd.VdTune()
    tune.radix = radix
    tune.lanes = lanes
    plan = vd.BatchPlan(k7_codes, packets_of(batch), tune=tune)
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).cuda()
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    out = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    plan.launch(llr, out)
    plan.status()
    got = out.cpu().numpy().view(np.uint32)
    f, v = plan.packet_tune()
    info = plan.info()
    assert info.n_packets == batch.n_packets and info.n_frames >= batch.n_packets
    for i in range(batch.n_packets):
        want = oracle_packet(batch, i, f[i], v[i])
        assert np.array_equal(words_of(got, batch, i), want), (i, int(batch.n_info[i]), f[i], v[i])
    # packets no longer than the tuned frame are decoded whole (exact maximum likelihood)
    assert np.all((f >= batch.n_info) | (f % 32 == 0))
    plan.close()


def test_graph_replay_and_one_launch_per_packet_agree(k7_codes):
    batch = synth.uneven_packets(n_packets=200, index=2, lo=96, hi=2000)
    plan = vd.BatchPlan(k7_codes, packets_of(batch))
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).cuda()
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    s = torch.cuda.Stream()
    outs = []
    for graph in (False, True, True):
        out = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(s):
            plan.launch(llr, out, stream=s, graph=graph)
        s.synchronize()
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    # the plain form: one vd_decode launch per packet with the same f and v
    f, v = plan.packet_tune()
    plain = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    for i in range(batch.n_packets):
        code = k7_codes[batch.rate_id[i]]
        a, n = int(batch.llr_offset[i]), int(batch.n_info[i])
        o = int(batch.out_word_offset[i])
        vd.vd_decode(code.handle, llr[a: a + int(batch.n_kept[i])], vd.VD_LLR_S8, n, int(f[i]), int(v[i]),
                     2, vd.VD_TERMINATED, plain[o: o + (n + 31) // 32])
    torch.cuda.synchronize()
    assert np.array_equal(plain.cpu().numpy(), outs[0])
    plan.close()


def test_mixed_codes_and_4bit_packets():
    """K=7 int8 and 4-bit packets and K=9 4-bit packets in one plan (two
    persistent launches), checked against the oracle; explicit and tuned f."""
    rng = np.random.Generator(np.random.PCG64(404))
    k7 = vd.Code(7, synth.K7_GENS)
    k9 = vd.Code(9, synth.K9_GENS)
    arena, recs, truth = [], [], []
    byte_off, out_off = 0, 0
    for i in range(90):
        kind = i % 3            # 0: K=7 int8, 1: K=7 4-bit, 2: K=9 4-bit
        K, gens, code_id = (7, synth.K7_GENS, 0) if kind < 2 else (9, synth.K9_GENS, 1)
        n = int(rng.integers(40, 2500))
        term = bool(i % 4 != 3)
        st = synth.make_stream(rng, K, gens, n, 2.5, term)
        if kind == 0:
            q = st.s8()
            data, ltype, voff = q.view(np.uint8), vd.VD_LLR_S8, byte_off
        else:
            q = st.s4()
            data, ltype, voff = synth.pack_s4(q), vd.VD_LLR_S4, 2 * byte_off
        f = 0 if i % 2 == 0 else 512
        v = 0 if f == 0 else 40
        recs.append((code_id, ltype, voff, n, vd.VD_TERMINATED if term else 0, f, v, out_off))
        truth.append((K, gens, q.astype(np.int32), n, term))
        arena.append(data)
        byte_off += data.size + (data.size % 2)
        if data.size % 2:
            arena.append(np.zeros(1, np.uint8))
        out_off += (n + 31) // 32
    pk = {k: np.array([r[j] for r in recs]) for j, k in enumerate(
        ("code_id", "llr_type", "llr_offset", "n_info", "flags", "f", "v", "out_word_offset"))}
    plan = vd.BatchPlan([k7, k9], pk)
    llr = torch.from_numpy(np.concatenate(arena)).cuda()
    out = torch.full((out_off,), -1, dtype=torch.int32, device="cuda")
    plan.launch(llr, out)
    plan.status()
    got = out.cpu().numpy().view(np.uint32)
    ff, vv = plan.packet_tune()
    assert plan.info().n_launches >= 3   # pre-pass + one kernel per code kind
    for i, (K, gens, q, n, term) in enumerate(truth):
        oc = oracle.Code(K, gens)
        T = n + (K - 1 if term else 0)
        want = oracle.decode(oc, q.reshape(T, len(gens)), n, int(ff[i]), int(vv[i]), terminated=term)
        o = recs[i][7]
        assert np.array_equal(got[o: o + (n + 31) // 32], want), i
    plan.close()


def test_batch_of_whole_streams_matches_stream_decode():
    """Six 2^20-bit segmented streams as six packets of one plan give the same
    bits as six vd_decode calls."""
    k7 = vd.Code(7, synth.K7_GENS)
    n = 1 << 20
    qs = [synth.segmented_stream(e, n_info=n).s8() for e in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0)]
    arena = torch.from_numpy(np.concatenate(qs).view(np.uint8)).cuda()
    pk = {"code_id": np.zeros(6, np.int32), "llr_type": np.zeros(6, np.int32),
          "llr_offset": np.arange(6) * 2 * n, "n_info": np.full(6, n), "flags": np.zeros(6, np.uint32),
          "f": np.full(6, 256, np.int32), "v": np.full(6, 42, np.int32),
          "out_word_offset": np.arange(6) * (n // 32)}
    plan = vd.BatchPlan([k7], pk)
    out = torch.full((6 * n // 32,), -1, dtype=torch.int32, device="cuda")
    plan.launch(arena, out)
    ref = torch.full((6 * n // 32,), -1, dtype=torch.int32, device="cuda")
    for i in range(6):
        vd.vd_decode(k7.handle, arena[2 * n * i: 2 * n * (i + 1)], vd.VD_LLR_S8, n, 256, 42, 2, 0,
                     ref[i * (n // 32): (i + 1) * (n // 32)])
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    plan.close()


def test_autotuned_shape_gives_the_same_bits(k7_codes):
    """A plan built without a tune measures the candidate kernel shapes and
    keeps one; its output equals an explicitly shaped plan's bit for bit."""
    batch = synth.uneven_packets(n_packets=400, index=4, lo=96, hi=5000)
    pk = packets_of(batch, f=256, v=42)
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).cuda()
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    auto = vd.BatchPlan(k7_codes, pk)
    info = auto.info()
    assert info.radix in (2, 4) and info.lanes in (1, 2)
    fixed_tune = vd.VdTune()
    fixed_tune.radix = 4 if info.radix == 2 else 2
    fixed_tune.lanes = 2 if info.lanes == 1 else 1
    fixed = vd.BatchPlan(k7_codes, pk, tune=fixed_tune)
    out_a = torch.full((nw,), -1, dtype=torch.int32, device="cuda")
    out_f = torch.full((nw,), -2, dtype=torch.int32, device="cuda")
    auto.launch(llr, out_a)
    fixed.launch(llr, out_f)
    auto.status()
    fixed.status()
    assert torch.equal(out_a, out_f)
    auto.close()
    fixed.close()
