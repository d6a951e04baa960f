"""fp16 LLRs with fp32 path metrics vs the FP64 oracle on the same fp16 values.

fp32 accumulation is not exact, so the rule is a tie margin: a frame's
decoded bits may differ from the FP64 oracle's only if the oracle's traced
survivor path in that frame has an add-compare-select decision whose two
candidates are within tau = 4 W 2^-24 M_w of each other, or a final-argmax gap
that small (W: the frame's trellis stages, M_w: the largest |metric| in it).
Any other disagreement fails.  The integer forms are checked bit-exact in
test_gpu_parity.py.
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


def check_margin(code, gbits, obits, gap, mx, n, f, v, T):
    bad = 0
    disagree_frames = 0
    for s in range(len(gap)):
        o, e = s * f, min(n, (s + 1) * f)
        a, b = max(0, o - v), min(T, (s + 1) * f + v)
        if np.array_equal(gbits[o:e], obits[o:e]):
            continue
        disagree_frames += 1
        tau = 4.0 * (b - a) * 2.0 ** -24 * max(mx[s], 1.0)
        if not gap[s] <= tau:
            bad += 1
    return bad, disagree_frames


@pytest.mark.parametrize("K,ebn0,f,v,lanes", [(9, 0.0, 512, 64, 8), (9, 2.0, 512, 64, 8),
                                               (9, 4.0, 512, 64, 8), (7, 1.0, 256, 42, 2),
                                               (7, 4.0, 256, 42, 2)])
def test_fp16_fp32_within_tie_margin(K, ebn0, f, v, lanes):
    n = 3 * 4096 + 5
    st = (synth.precision_stream if K == 9 else synth.segmented_stream)(ebn0, n_info=n)
    gens = synth.K9_GENS if K == 9 else synth.K7_GENS
    h = st.f16()
    code = vd.Code(K, gens)
    llr = torch.from_numpy(h.view(np.uint16)).cuda()
    gw = vd.decode(code, llr, n, f, v, llr_type=vd.VD_LLR_F16, lanes=lanes).cpu().numpy().view(np.uint32)
    oc = oracle.Code(K, gens)
    ow, gap, mx = oracle.decode_f64(oc, h.astype(np.float64).reshape(n, len(gens)), n, f, v, threads=THREADS)
    gb, ob = oracle.unpack_bits(gw, n), oracle.unpack_bits(ow, n)
    bad, frames = check_margin(oc, gb, ob, gap, mx, n, f, v, n)
    assert bad == 0, f"{bad} frames disagree with no near-tie ({frames} disagree in all)"
    # at these lengths the fp32 form agrees with FP64 on nearly every bit
    assert np.mean(gb != ob) < 1e-3


@pytest.mark.parametrize("term", [False, True])
def test_fp16_edges_and_reset(term):
    """Short streams, a single frame, terminated ends and the reset start."""
    rng = np.random.Generator(np.random.PCG64(88 + term))
    for K, gens, lanes in ((7, synth.K7_GENS, 2), (9, synth.K9_GENS, 8)):
        code = vd.Code(K, gens)
        oc = oracle.Code(K, gens)
        for n, f, v in ((1, 32, 6), (40, 64, 8), (700, 128, 30), (1000, 1000, 0)):
            st = synth.make_stream(rng, K, gens, n, 3.0, term)
            h = st.f16()
            T = st.T
            gw = vd.decode(code, torch.from_numpy(h.view(np.uint16)).cuda(), n, f, v, terminated=term,
                           llr_type=vd.VD_LLR_F16, lanes=lanes).cpu().numpy().view(np.uint32)
            ow, gap, mx = oracle.decode_f64(oc, h.astype(np.float64).reshape(T, len(gens)), n, f, v,
                                            terminated=term)
            gb, ob = oracle.unpack_bits(gw, n), oracle.unpack_bits(ow, n)
            bad, _ = check_margin(oc, gb, ob, gap, mx, n, f, v, T)
            assert bad == 0, (K, n, f, v)


def test_k9_full_size_fp16_within_tie_margin():
    """The precision-study configuration at full size: 2^24 K=9 r1/3 bits
    (f=512, v=64, Eb/N0 = 1 dB) in fp16 with fp32 metrics, every frame within
    the tie margin of the FP64 oracle on the same fp16 values."""
    n, f, v = 1 << 24, 512, 64
    st = synth.precision_stream(1.0, n_info=n)
    h = st.f16()
    code = vd.Code(9, synth.K9_GENS)
    gw = vd.decode(code, torch.from_numpy(h.view(np.uint16)).cuda(), n, f, v,
                   llr_type=vd.VD_LLR_F16).cpu().numpy().view(np.uint32)
    vd.vd_sync()
    oc = oracle.Code(9, synth.K9_GENS)
    ow, gap, mx = oracle.decode_f64(oc, h.astype(np.float64).reshape(n, 3), n, f, v, threads=THREADS)
    gb, ob = oracle.unpack_bits(gw, n), oracle.unpack_bits(ow, n)
    bad, frames = check_margin(oc, gb, ob, gap, mx, n, f, v, n)
    assert bad == 0, f"{bad} frames disagree with no near-tie ({frames} disagree in all)"


def test_k9_full_size_4bit_bit_exact():
    """The precision-study configuration at full size in 4-bit LLRs: 2^24
    K=9 r1/3 bits, every decoded bit equal to the int64 oracle's on the same
    4-bit values."""
    n, f, v = 1 << 24, 512, 64
    st = synth.precision_stream(2.0, n_info=n)
    q4 = st.s4()
    code = vd.Code(9, synth.K9_GENS)
    gw = vd.decode(code, torch.from_numpy(synth.pack_s4(q4)).cuda(), n, f, v,
                   llr_type=vd.VD_LLR_S4).cpu().numpy().view(np.uint32)
    vd.vd_sync()
    want = oracle.decode(oracle.Code(9, synth.K9_GENS), q4.reshape(n, 3).astype(np.int32), n, f, v,
                         threads=THREADS)
    assert np.array_equal(gw, want)
