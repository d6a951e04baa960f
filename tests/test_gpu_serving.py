"""Continuous-batching server: every packet decoded in the mix equals the
same packet decoded alone (same frames, integer arithmetic: bit for bit),
a subset equals the CPU oracle, and admission by device memory holds packets
back without losing any when the arena is small."""
import time

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


def make_codes():
    return [vd.Code(K, gens, puncture=None if pat is None else pat.tolist())
            for (K, gens, pat) in synth.SERVING_CODES]


def serve_all(server, pkts, timeout_s=60.0):
    for i, p in enumerate(pkts):
        server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, p.n_info, vd.VD_TERMINATED, i)
    got, recs = {}, {}
    t_end = time.time() + timeout_s
    while len(got) < len(pkts) and time.time() < t_end:
        for c, w in server.poll():
            assert c.status == vd.VD_OK
            got[c.tag] = w
            recs[c.tag] = (c.submit_ns, c.admit_ns, c.done_ns)
        time.sleep(0.001)
    assert len(got) == len(pkts), f"only {len(got)} of {len(pkts)} packets completed"
    return got, recs


def alone(codes, p):
    K = synth.SERVING_CODES[p.code_id][0]
    F, V = (256, 42) if K == 7 else (512, 64)
    f = min(p.n_info, F)
    llr = torch.from_numpy(p.llr_s8.view(np.uint8)).cuda()
    out = vd.decode(codes[p.code_id], llr, p.n_info, f, V, terminated=True)
    return out.cpu().numpy().view(np.uint32), f, V


@pytest.mark.parametrize("arena_mb,streams,max_batch", [(64, 3, 4096), (2, 2, 16), (8, 4, 64)])
def test_mix_equals_alone_and_oracle(arena_mb, streams, max_batch):
    codes = make_codes()
    cfg = vd.VdServerConfig()
    cfg.device_bytes = arena_mb << 20
    cfg.n_streams = streams
    cfg.max_batch = max_batch
    server = vd.Server(codes, cfg)
    pkts = synth.serving_packets(400, index=arena_mb)
    got, recs = serve_all(server, pkts)
    st = server.stats()
    assert st.completed == len(pkts) and st.pending == 0 and st.error == 0
    assert st.batches >= (2 if max_batch < 400 else 1)
    for i, p in enumerate(pkts):
        want, f, v = alone(codes, p)
        assert np.array_equal(got[i], want), i
        s, a, d = recs[i]
        assert s <= a <= d
        if i % 25 == 0:
            K, gens, pat = synth.SERVING_CODES[p.code_id]
            oc = oracle.Code(K, gens, puncture=pat)
            T = p.n_info + K - 1
            full = oracle.depuncture(oc, p.llr_s8.astype(np.int32), T)
            assert np.array_equal(got[i], oracle.decode(oc, full, p.n_info, f, v, terminated=True)), i
    server.close()


def test_arrivals_while_busy_overlap():
    """Packets submitted while earlier batches run are admitted into later
    batches (more than one batch), and all results match decoding alone."""
    codes = make_codes()
    cfg = vd.VdServerConfig()
    cfg.n_streams = 3
    cfg.max_batch = 32
    server = vd.Server(codes, cfg)
    pkts = synth.serving_packets(300, index=77)
    got = {}
    for i, p in enumerate(pkts):
        server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, p.n_info, vd.VD_TERMINATED, i)
        if i % 20 == 0:
            time.sleep(0.0005)
            for c, w in server.poll():
                got[c.tag] = w
    t_end = time.time() + 60
    while len(got) < len(pkts) and time.time() < t_end:
        for c, w in server.poll():
            got[c.tag] = w
        time.sleep(0.001)
    assert len(got) == len(pkts)
    assert server.stats().batches > 2
    for i in range(0, len(pkts), 7):
        want, _, _ = alone(codes, pkts[i])
        assert np.array_equal(got[i], want), i
    server.close()


def test_submit_validation():
    codes = make_codes()
    server = vd.Server(codes)
    p = synth.serving_packets(1, index=5)[0]
    with pytest.raises(vd.VdError):
        server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size - 1, p.n_info, vd.VD_TERMINATED, 0)
    with pytest.raises(vd.VdError):
        server.submit(9, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, p.n_info, vd.VD_TERMINATED, 0)
    with pytest.raises(vd.VdError):
        server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, 20000, vd.VD_TERMINATED, 0)
    server.close()


def test_replay_open_loop_matches_alone():
    """Trace replay (Poisson arrivals): every packet completes with a positive
    latency and decodes to the same bits as alone; a busy server is refused."""
    codes = make_codes()
    server = vd.Server(codes)
    pkts = synth.serving_packets(300, index=91)
    fl = synth.flatten_packets(pkts)
    n = len(pkts)
    arr = synth.poisson_arrivals(np.random.Generator(np.random.PCG64(5)), n, 20000.0)
    lat, words, span = server.replay(fl["code_id"], np.zeros(n, np.int32), fl["llr"], fl["llr_offset"],
                                     fl["n_values"], fl["n_info"], np.full(n, vd.VD_TERMINATED, np.uint32),
                                     arr, timeout_ms=60000, word_offset=fl["word_offset"])
    assert (lat > 0).all() and span > 0
    for i in range(0, n, 5):
        want, _, _ = alone(codes, pkts[i])
        o = int(fl["word_offset"][i])
        assert np.array_equal(words[o:o + want.size], want), i
    # a packet left unpolled makes the server busy for a replay
    p = pkts[0]
    server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, p.n_info, vd.VD_TERMINATED, 0)
    with pytest.raises(vd.VdError):
        server.replay(fl["code_id"][:1], np.zeros(1, np.int32), fl["llr"], fl["llr_offset"][:1],
                      fl["n_values"][:1], fl["n_info"][:1], np.full(1, vd.VD_TERMINATED, np.uint32),
                      np.zeros(1, np.int64))
    server.close()


def test_device_resident_packets_match_alone():
    """Packets whose values are already in device memory (read in place, no
    upload; punctured ones expanded into the arena) decode to the same bits
    as alone, mixed with host packets and through the device replay."""
    codes = make_codes()
    cfg = vd.VdServerConfig()
    cfg.max_batch = 64
    server = vd.Server(codes, cfg)
    pkts = synth.serving_packets(240, index=93)
    fl = synth.flatten_packets(pkts)
    dev = torch.from_numpy(fl["llr"].view(np.uint8)).cuda()
    got = {}
    for i, p in enumerate(pkts):
        if i % 3 == 0:
            server.submit(p.code_id, vd.VD_LLR_S8, p.llr_s8, p.llr_s8.size, p.n_info, vd.VD_TERMINATED, i)
        else:
            server.submit_device(p.code_id, vd.VD_LLR_S8, dev.data_ptr() + int(fl["llr_offset"][i]),
                                 p.llr_s8.size, p.n_info, vd.VD_TERMINATED, i)
    t_end = time.time() + 60
    while len(got) < len(pkts) and time.time() < t_end:
        for c, w in server.poll():
            assert c.status == vd.VD_OK
            got[c.tag] = w
        time.sleep(0.001)
    assert len(got) == len(pkts)
    for i in range(0, len(pkts), 3):
        want, _, _ = alone(codes, pkts[i])
        assert np.array_equal(got[i], want), i
    for i in range(1, len(pkts), 3):
        want, _, _ = alone(codes, pkts[i])
        assert np.array_equal(got[i], want), i
    n = len(pkts)
    arr = synth.poisson_arrivals(np.random.Generator(np.random.PCG64(6)), n, 50000.0)
    lat, words, span = server.replay(fl["code_id"], np.zeros(n, np.int32), dev, fl["llr_offset"],
                                     fl["n_values"], fl["n_info"], np.full(n, vd.VD_TERMINATED, np.uint32),
                                     arr, timeout_ms=60000, word_offset=fl["word_offset"])
    assert (lat > 0).all() and span > 0
    for i in range(0, n, 4):
        o = int(fl["word_offset"][i])
        assert np.array_equal(words[o:o + got[i].size], got[i]), i
    server.close()


def test_submit_many_equals_alone():
    """Packets queued by one vd_server_submit_many call (host values copied
    into staging, uploaded into the device arena by the batch) decode to the
    same bits as each packet decoded alone; a bad packet in the list queues
    nothing."""
    codes = make_codes()
    server = vd.Server(codes)
    pkts = synth.serving_packets(300, index=9)
    flat = synth.flatten_packets(pkts)
    n = len(pkts)
    types = np.zeros(n, np.int32)
    flags = np.full(n, vd.VD_TERMINATED, np.uint32)
    bad_vals = flat["n_values"].copy()
    bad_vals[7] += 1
    with pytest.raises(vd.VdError):
        server.submit_many(flat["code_id"], types, flat["llr"], flat["llr_offset"], bad_vals, flat["n_info"],
                           flags, np.arange(n, dtype=np.uint64))
    assert server.stats().submitted == 0
    server.submit_many(flat["code_id"], types, flat["llr"], flat["llr_offset"], flat["n_values"], flat["n_info"],
                       flags, np.arange(n, dtype=np.uint64))
    got = {}
    t_end = time.time() + 60
    while len(got) < n and time.time() < t_end:
        for c, w in server.poll():
            assert c.status == vd.VD_OK
            got[c.tag] = w
        time.sleep(0.001)
    assert len(got) == n
    for i, p in enumerate(pkts):
        want, _, _ = alone(codes, p)
        assert np.array_equal(got[i], want), i
    server.close()
