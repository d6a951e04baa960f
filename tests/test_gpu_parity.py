"""GPU decoder vs the CPU oracle, element by element, through the C ABI.

Bit-exact on decoded bits (integer path), and on each frame's canonical final
path metrics (lambda - min lambda) where the oracle's metrics are all finite
(frames with at least K-1 stages).  Sizes span several frames and a ragged
tail; the full-size segmented stream of the workload is checked whole for
K=7 and on sampled frames for K=9.
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


_codes = {}


def gpu_code(K, gens, pattern=None):
    key = (K, tuple(gens), None if pattern is None else np.asarray(pattern).tobytes())
    if key not in _codes:
        _codes[key] = vd.Code(K, gens, puncture=None if pattern is None else np.asarray(pattern).tolist())
    return _codes[key]


def run_gpu(code, kept, n_info, f, v, radix=2, terminated=False, start_unknown=False,
            llr_type=vd.VD_LLR_S8, lanes=0, offset=0):
    """kept: numpy int8 (or packed 4-bit uint8) received stream."""
    raw = np.ascontiguousarray(kept).view(np.uint8)
    buf = torch.zeros(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size] = torch.from_numpy(raw).cuda()
    llr = buf[offset:offset + raw.size]
    out, pm = vd.decode(code, llr, n_info, f, v, radix=radix, terminated=terminated,
                        start_unknown=start_unknown, llr_type=llr_type, want_pm=True, lanes=lanes)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32), pm.cpu().numpy()


def run_oracle(ocode, full_llr, n_info, f, v, terminated=False, start_unknown=False):
    return oracle.decode(ocode, full_llr, n_info, f, v, terminated=terminated,
                         start_unknown=start_unknown, threads=THREADS, want_pm=True)


def check(gw, gpm, ow, opm, K, n_info, f, v, T, terminated, start_unknown, check_pm=True):
    assert gw.shape == ow.shape
    if not np.array_equal(gw, ow):
        gb, ob = oracle.unpack_bits(gw, n_info), oracle.unpack_bits(ow, n_info)
        bad = np.nonzero(gb != ob)[0]
        raise AssertionError(f"{bad.size} decoded bits differ, first at stage {bad[:8]} "
                             f"(frame {bad[0] // f})")
    if not check_pm:
        return
    nwin = opm.shape[0]
    for s in range(nwin):
        a = max(0, s * f - v)
        b = min(T, (s + 1) * f + v)
        if b - a < K - 1 and a == 0 and not start_unknown:
            continue   # oracle metrics hold -infinity
        if not np.array_equal(gpm[s].astype(np.int64), opm[s]):
            raise AssertionError(f"frame {s}: canonical metrics differ")


def full_llr_of(ocode, kept, T):
    """Depunctured [T, beta] int32 for the oracle (identity when unpunctured)."""
    kept32 = np.asarray(kept, dtype=np.int32).reshape(-1)
    if ocode.period == 1 and ocode.puncture.all():
        return kept32.reshape(T, ocode.beta)
    return oracle.depuncture(ocode, kept32, T)


# -------------------------------------------------- the plain small workload

@pytest.mark.parametrize("radix", [2, 4])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_plain_small_full_length(radix, lanes):
    st = synth.plain_small()
    q = st.s8()
    oc = oracle.Code(7, synth.K7_GENS)
    T = st.T
    f, v = st.n_info, st.K - 1
    ow, opm = run_oracle(oc, q.reshape(T, 2).astype(np.int32), st.n_info, f, v, terminated=True)
    gw, gpm = run_gpu(gpu_code(7, synth.K7_GENS), q, st.n_info, f, v, radix=radix, terminated=True,
                      lanes=lanes)
    check(gw, gpm, ow, opm, 7, st.n_info, f, v, T, True, False)
    # the plain full-length decode recovers the data at 3 dB nearly perfectly
    ber = np.mean(oracle.unpack_bits(gw, st.n_info) != st.bits)
    assert ber < 1e-2


# ------------------------------------------------------ segmented K=7 stream

@pytest.mark.parametrize("ebn0", [1.0, 3.0, 6.0])
@pytest.mark.parametrize("radix", [2, 4])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_segmented_k7(ebn0, radix, lanes):
    n = (1 << 14) + 77                # several frames and a ragged tail
    st = synth.segmented_stream(ebn0, n_info=n)
    q = st.s8()
    oc = oracle.Code(7, synth.K7_GENS)
    ow, opm = run_oracle(oc, q.reshape(n, 2).astype(np.int32), n, 256, 42)
    gw, gpm = run_gpu(gpu_code(7, synth.K7_GENS), q, n, 256, 42, radix=radix, lanes=lanes)
    check(gw, gpm, ow, opm, 7, n, 256, 42, n, False, False)


# ---------------------------------------------------- K=9 precision workload

@pytest.mark.parametrize("ebn0", [0.0, 2.0, 4.0])
@pytest.mark.parametrize("radix", [2, 4])
@pytest.mark.parametrize("lanes", [4, 8])
@pytest.mark.parametrize("llr_kind", ["s8", "s4"])
def test_segmented_k9(ebn0, radix, lanes, llr_kind):
    n = (1 << 12) * 3 + 5
    st = synth.precision_stream(ebn0, n_info=n)
    oc = oracle.Code(9, synth.K9_GENS)
    if llr_kind == "s8":
        q = st.s8()
        kept, ltype = q, vd.VD_LLR_S8
    else:
        q = st.s4()
        kept, ltype = synth.pack_s4(q), vd.VD_LLR_S4
    ow, opm = run_oracle(oc, q.reshape(n, 3).astype(np.int32), n, 512, 64)
    gw, gpm = run_gpu(gpu_code(9, synth.K9_GENS), kept, n, 512, 64, radix=radix, lanes=lanes,
                      llr_type=ltype)
    check(gw, gpm, ow, opm, 9, n, 512, 64, n, False, False)


# ---------------------------------------------------------------- edge cases

EDGE = [
    # n, f, v, terminated, start_unknown
    (1, 32, 6, False, False),
    (1, 32, 6, True, False),
    (5, 64, 0, False, False),
    (31, 32, 6, True, False),
    (32, 32, 6, False, True),
    (33, 32, 6, False, False),
    (100, 1000, 0, True, False),       # single frame, f not a multiple of 32
    (255, 64, 1, False, False),
    (257, 64, 42, True, False),
    (1000, 96, 300, False, False),     # overlap longer than the frame
    (1000, 32, 5, True, True),         # overlap shorter than K-1
    (4099, 4096, 6, True, False),      # one full frame plus a 3-bit tail frame
]


@pytest.mark.parametrize("n,f,v,term,unk", EDGE)
@pytest.mark.parametrize("kind", ["noisy", "zeros", "saturated", "erasures"])
@pytest.mark.parametrize("radix", [2, 4])
def test_edge_cases_k7(n, f, v, term, unk, kind, radix):
    rng = np.random.Generator(np.random.PCG64(1000 + n + f + v))
    oc = oracle.Code(7, synth.K7_GENS)
    T = n + (6 if term else 0)
    if kind == "noisy":
        st = synth.make_stream(rng, 7, synth.K7_GENS, n, 2.0, term)
        q = st.s8()
    elif kind == "zeros":
        q = np.zeros(2 * T, np.int8)             # every comparison is a tie
    elif kind == "saturated":
        q = (127 * (1 - 2 * rng.integers(0, 2, 2 * T))).astype(np.int8)
    else:
        q = rng.integers(-127, 128, 2 * T).astype(np.int8)
        q[rng.random(2 * T) < 0.6] = 0
    ow, opm = run_oracle(oc, q.reshape(T, 2).astype(np.int32), n, f, v, term, unk)
    for lanes in (1, 4):
        gw, gpm = run_gpu(gpu_code(7, synth.K7_GENS), q, n, f, v, radix=radix, terminated=term,
                          start_unknown=unk, lanes=lanes)
        check(gw, gpm, ow, opm, 7, n, f, v, T, term, unk)


@pytest.mark.parametrize("kind", ["saturated", "noisy"])
def test_head_start_near_normalisation_k7(kind):
    """The first frame's head-start stage swept over every residue of the
    metric normalisation period (18 stages for the K=7 integer form): the
    overlap v moves the start of the first frame inside its padded pair, so
    some resets fall within K-1 stages before a normalisation, where states
    not yet reachable from state 0 sit lowest.  Saturated LLRs make the
    metric spread as large as the bound allows."""
    oc = oracle.Code(7, synth.K7_GENS)
    code = gpu_code(7, synth.K7_GENS)
    n, f = 600, 64
    for v in range(6, 42):
        rng = np.random.Generator(np.random.PCG64(3000 + v))
        for term in (False, True):
            T = n + (6 if term else 0)
            if kind == "saturated":
                q = (127 * (1 - 2 * rng.integers(0, 2, 2 * T))).astype(np.int8)
            else:
                q = synth.make_stream(rng, 7, synth.K7_GENS, n, 1.0, term).s8()
            ow, opm = run_oracle(oc, q.reshape(T, 2).astype(np.int32), n, f, v, term)
            gw, gpm = run_gpu(code, q, n, f, v, terminated=term, lanes=1)
            check(gw, gpm, ow, opm, 7, n, f, v, T, term, False)


def _path_outputs(K, gens, s, inputs):
    """Output bits (stage-major, generator order) of the encoder path that
    starts in state s (register r = (u << (K-1)) | s, next state
    (u << (K-2)) | (s >> 1), as in the oracle's trellis)."""
    out = []
    for u in inputs:
        r = (u << (K - 1)) | s
        out += [bin(g & r).count("1") & 1 for g in gens]
        s = (u << (K - 2)) | (s >> 1)
    return out


@pytest.mark.parametrize("K,D", [(7, 51), (7, 1), (7, 32), (7, 63), (9, 191), (9, 1), (9, 229)])
def test_head_start_adversarial(K, D):
    """The frame that starts from the reset state: its first K-1 stages carry
    saturated LLRs that match the path from start state D != 0 (zero inputs),
    so that path leads the path from state 0 with the same inputs by 254 per
    differing output bit (2540 for D = 51 with the 171/133 code and 4826 for
    D = 191 with 557/663/711, the largest lead any start state can take).
    The oracle starts the other states at
    -infinity; the GPU's finite head start must keep the path from state 0
    ahead, which the frame's final canonical metrics show (the decoded bits
    cannot: both paths carry the same inputs).  The reset stage is swept over
    every position within a chunk of the kernel's unrolled stages."""
    gens = synth.K7_GENS if K == 7 else synth.K9_GENS
    beta, lanes = len(gens), (1 if K == 7 else 4)
    oc = oracle.Code(K, gens)
    code = gpu_code(K, gens)
    lead = np.array(_path_outputs(K, gens, D, [0] * (K - 1)))
    U = 6 if K == 7 else 8   # stages per unrolled chunk of the kernel
    cases = [(600 + i, 4096, 6) for i in range(U)] + [(700, 64, v) for v in range(6, 6 + U)]
    for n, f, v in cases:
        rng = np.random.Generator(np.random.PCG64(4000 + 17 * D + n + v))
        q = synth.make_stream(rng, K, gens, n, 2.0, False).s8().copy()
        q[:beta * (K - 1)] = np.where(lead == 0, 127, -127).astype(np.int8)
        ow, opm = run_oracle(oc, q.reshape(n, beta).astype(np.int32), n, f, v)
        gw, gpm = run_gpu(code, q, n, f, v, lanes=lanes)
        check(gw, gpm, ow, opm, K, n, f, v, n, False, False)


@pytest.mark.parametrize("n,f,v,term", [(1, 32, 8, True), (5, 32, 8, False), (7, 64, 0, False),
                                        (70, 64, 3, False), (2000, 512, 64, True),
                                        (2049, 1024, 700, False)])
@pytest.mark.parametrize("kind", ["noisy", "zeros", "saturated", "erasures"])
def test_edge_cases_k9(n, f, v, term, kind):
    rng = np.random.Generator(np.random.PCG64(2000 + n + f + v))
    oc = oracle.Code(9, synth.K9_GENS)
    T = n + (8 if term else 0)
    if kind == "noisy":
        q = synth.make_stream(rng, 9, synth.K9_GENS, n, 1.0, term).s8()
    elif kind == "zeros":
        q = np.zeros(3 * T, np.int8)
    elif kind == "saturated":
        q = (127 * (1 - 2 * rng.integers(0, 2, 3 * T))).astype(np.int8)
    else:
        q = rng.integers(-127, 128, 3 * T).astype(np.int8)
        q[rng.random(3 * T) < 0.6] = 0
    ow, opm = run_oracle(oc, q.reshape(T, 3).astype(np.int32), n, f, v, term)
    for radix in (2, 4):
        gw, gpm = run_gpu(gpu_code(9, synth.K9_GENS), q, n, f, v, radix=radix, terminated=term, lanes=4)
        check(gw, gpm, ow, opm, 9, n, f, v, T, term, False)


@pytest.mark.parametrize("offset", [1, 2, 3, 5])
def test_unaligned_llr_pointer(offset):
    n = 3000
    st = synth.segmented_stream(2.0, n_info=n)
    q = st.s8()
    oc = oracle.Code(7, synth.K7_GENS)
    ow, opm = run_oracle(oc, q.reshape(n, 2).astype(np.int32), n, 256, 42)
    gw, gpm = run_gpu(gpu_code(7, synth.K7_GENS), q, n, 256, 42, offset=offset)
    check(gw, gpm, ow, opm, 7, n, 256, 42, n, False, False)


@pytest.mark.parametrize("pat", ["r23", "r34"])
@pytest.mark.parametrize("f,v", [(256, 42), (10 ** 6, 6)])
def test_punctured_terminated_k7(pat, f, v):
    pattern = synth.PUNCT_R23 if pat == "r23" else synth.PUNCT_R34
    rng = np.random.Generator(np.random.PCG64(31 + len(pat) + v))
    n = 3001
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 4.0, True, pattern=pattern)
    kept = st.s8()
    oc = oracle.Code(7, synth.K7_GENS, puncture=pattern)
    T = st.T
    full = full_llr_of(oc, kept, T)
    ff = min(f, n)
    ow, opm = run_oracle(oc, full, n, ff, v, terminated=True)
    for radix in (2, 4):
        gw, gpm = run_gpu(gpu_code(7, synth.K7_GENS, pattern), kept, n, ff, v, radix=radix,
                          terminated=True)
        check(gw, gpm, ow, opm, 7, n, ff, v, T, True, False)


# ------------------------------------------------------- full-size workloads

def test_full_size_segmented_k7_radix2_radix4():
    """2^24 info bits, f=256, v=42 (the segmented-stream workload): whole
    stream bit-exact vs the oracle, and radix-4 identical to radix-2."""
    n = 1 << 24
    st = synth.segmented_stream(3.0)
    q = st.s8()
    oc = oracle.Code(7, synth.K7_GENS)
    ow = oracle.decode(oc, q.reshape(n, 2).astype(np.int32), n, 256, 42, threads=THREADS)
    code = gpu_code(7, synth.K7_GENS)
    llr = torch.from_numpy(q.view(np.uint8)).cuda()
    g2 = vd.decode(code, llr, n, 256, 42, radix=2).cpu().numpy().view(np.uint32)
    g4 = vd.decode(code, llr, n, 256, 42, radix=4).cpu().numpy().view(np.uint32)
    assert np.array_equal(g2, ow)
    assert np.array_equal(g4, g2)


def test_full_size_segmented_k9_sampled_frames():
    """2^24 info bits, K=9, f=512, v=64: sampled frames (first, last, spread)
    bit-exact with their canonical metrics."""
    n = 1 << 24
    f, v = 512, 64
    st = synth.precision_stream(2.0)
    q = st.s8()
    oc = oracle.Code(9, synth.K9_GENS)
    nwin = vd.vd_num_frames(n, f)
    code = gpu_code(9, synth.K9_GENS)
    llr = torch.from_numpy(q.view(np.uint8)).cuda()
    out, pm = vd.decode(code, llr, n, f, v, radix=2, want_pm=True)
    gbits = oracle.unpack_bits(out.cpu().numpy().view(np.uint32), n)
    gpm = pm.cpu().numpy()
    frames = np.unique(np.concatenate([[0, 1, nwin - 2, nwin - 1],
                                       np.random.Generator(np.random.PCG64(9)).integers(0, nwin, 60)]))
    obits, opm = oracle.decode_frames(oc, q.reshape(n, 3).astype(np.int32), n, f, v, frames, want_pm=True)
    for k, s in enumerate(frames):
        e = min(n, (s + 1) * f)
        assert np.array_equal(gbits[s * f:e], obits[k, :e - s * f]), s
        assert np.array_equal(gpm[s].astype(np.int64), opm[k]), s


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("K,gens,f,v,lanes,kind", [(7, synth.K7_GENS, 256, 42, 1, "s8"),
                                                   (7, synth.K7_GENS, 128, 30, 2, "s4"),
                                                   (9, synth.K9_GENS, 512, 64, 4, "s8")])
def test_both_vd_decode_forms(K, gens, f, v, lanes, kind, form):
    """vd_decode's persistent form (1) and one-wave form (2), forced through
    vd_tune.form, give the oracle's bits and canonical metrics, with a
    terminated ragged end and a pm output."""
    rng = np.random.Generator(np.random.PCG64(300 + K + form))
    n = 150_000 + 777
    st = synth.make_stream(rng, K, gens, n, 2.0, True)
    q = st.s8() if kind == "s8" else st.s4()
    kept = q if kind == "s8" else synth.pack_s4(q)
    code = gpu_code(K, gens)
    t = vd.VdTune()
    t.lanes = lanes
    t.form = form
    llr = torch.from_numpy(np.ascontiguousarray(kept).view(np.uint8)).cuda()
    nw = (n + 31) // 32
    out = torch.zeros(nw, dtype=torch.int32, device="cuda")
    pm = torch.zeros((vd.vd_num_frames(n, f), 1 << (K - 1)), dtype=torch.int32, device="cuda")
    vd.vd_decode(code.handle, llr, vd.VD_LLR_S8 if kind == "s8" else vd.VD_LLR_S4, n, f, v, 2,
                 vd.VD_TERMINATED, out, pm, t)
    vd.vd_sync()
    ocode = oracle.Code(K, gens)
    ow, opm = run_oracle(ocode, full_llr_of(ocode, q, st.T), n, f, v, terminated=True)
    check(out.cpu().numpy().view(np.uint32), pm.cpu().numpy(), ow, opm, K, n, f, v, st.T, True, False)
