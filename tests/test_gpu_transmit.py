"""GPU transmitter and channel (vd_transmit, Sec. IX-B) vs the oracle's.

Both sides implement the same published generator (Philox4x64-10) and the
Box-Muller transform in double precision, but with different libraries for
log/cos/sin, so a sample may differ in its last bits.  The quantised values
must be equal everywhere except where the oracle's sample sits within a
hair of a rounding boundary of the quantiser; such places are counted and
must be (practically) absent.
"""
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


TYPES = {"s8": vd.VD_LLR_S8, "s4": vd.VD_LLR_S4, "f16": vd.VD_LLR_F16, "hard": vd.VD_LLR_HARD}


def _near_boundary(y, kind, sigma):
    """Samples whose quantised value a last-bit difference could change."""
    if kind in ("s8", "s4"):
        s = 32.0 * y if kind == "s8" else 2.0 * y
        return np.abs(np.abs(s - np.floor(s)) - 0.5) < 1e-9
    if kind == "hard":
        return np.abs(y) < 1e-12
    v = 2.0 * y / (sigma * sigma)
    h = v.astype(np.float16).astype(np.float64)
    other = np.nextafter(v.astype(np.float16), np.where(v > h, np.inf, -np.inf).astype(np.float16)).astype(np.float64)
    mid = 0.5 * (h + other)
    return np.abs(v - mid) <= 1e-10 * np.abs(v)


def _unpack(raw, kind, n):
    if kind == "s8":
        return raw.view(np.int8)[:n]
    if kind == "s4":
        lo = (raw & 0x0F).astype(np.int8)
        hi = (raw >> 4).astype(np.int8)
        v = np.stack([lo, hi], axis=1).reshape(-1)[:n]
        return np.where(v > 7, v - 16, v).astype(np.int8)
    if kind == "hard":
        return np.unpackbits(raw, bitorder="little")[:n]
    return raw.view(np.float16)[:n]


@pytest.mark.parametrize("K,gens,pat,terminated", [(7, synth.K7_GENS, None, False), (7, synth.K7_GENS, "r23", True),
                                                   (7, synth.K7_GENS, "r34", True), (9, synth.K9_GENS, None, True)])
@pytest.mark.parametrize("kind", ["s8", "s4", "f16", "hard"])
def test_transmit_matches_oracle(K, gens, pat, terminated, kind):
    pattern = {None: None, "r23": synth.PUNCT_R23, "r34": synth.PUNCT_R34}[pat]
    rng = np.random.Generator(np.random.PCG64(800 + K))
    n = 100_003
    bits = synth.random_bits(rng, n)
    rate = synth.code_rate(len(gens), pattern)
    sigma = synth.sigma_for(2.0, rate)
    seed, sid = 2011135790 + K, 17
    code = vd.Code(K, gens, puncture=None if pattern is None else pattern.tolist())
    d_bits = torch.from_numpy(oracle.pack_bits(bits).view(np.int32)).cuda()
    got_raw = vd.transmit(code, d_bits, n, sigma, seed, sid, terminated=terminated, llr_type=TYPES[kind])
    oc = oracle.Code(K, gens, puncture=pattern)
    y = oracle.transmit(oc, bits, n, terminated, sigma, seed, sid)
    want = oracle.quantise(y, kind, sigma)
    got = _unpack(got_raw.cpu().numpy(), kind, y.size)
    if kind == "f16":
        got, want = got.view(np.uint16), want.view(np.uint16)
    diff = got != want
    edge = _near_boundary(y, kind, sigma)
    assert not np.any(diff & ~edge), np.nonzero(diff & ~edge)[0][:10]
    assert edge.sum() <= 2


def test_transmit_then_decode_on_the_gpu():
    """A stream made by vd_transmit and decoded by vd_decode, both on the
    device: bit-exact with the oracle's decode of the oracle's own samples
    (quantised equal), and error-free at 6 dB."""
    rng = np.random.Generator(np.random.PCG64(801))
    n = 1 << 18
    bits = synth.random_bits(rng, n)
    code = vd.Code(7, synth.K7_GENS)
    d_bits = torch.from_numpy(oracle.pack_bits(bits).view(np.int32)).cuda()
    for ebn0 in (2.0, 6.0):
        sigma = synth.sigma_for(ebn0, 0.5)
        llr = vd.transmit(code, d_bits, n, sigma, seed=99, stream_id=int(ebn0))
        got = vd.decode(code, llr, n, 256, 42).cpu().numpy().view(np.uint32)
        y = oracle.transmit(oracle.Code(7, synth.K7_GENS), bits, n, False, sigma, 99, int(ebn0))
        q = oracle.quantise(y, "s8").reshape(n, 2).astype(np.int32)
        want = oracle.decode(oracle.Code(7, synth.K7_GENS), q, n, 256, 42, threads=8)
        assert np.array_equal(got, want)
        ber = np.mean(oracle.unpack_bits(got, n) != bits)
        if ebn0 == 6.0:
            assert ber < 1e-5
