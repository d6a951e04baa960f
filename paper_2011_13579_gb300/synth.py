"""Seeded synthetic channel data: the transmitter side of the verification
system of arXiv 2011.13579, Sec. IX-B (uniform random bits -> convolutional
encoder -> BPSK -> AWGN), plus puncturing and LLR quantisation.

This module is the only code shared by the oracle tests and the CUDA path:
it produces inputs and holds no decoding arithmetic (no branch metric, no
add-compare-select, no traceback).  Every array is derived from NumPy's
``Generator(PCG64(seed))``; bits come from ``integers(0, 2)`` and noise from
``standard_normal``.

Conventions (the paper is silent on them):
  * generator polynomials are written in octal; the leftmost binary digit
    taps the current input (Eq. encoder, with 171/133 = 1111001/1011011);
  * BPSK maps bit 0 to +1, so a positive LLR means bit 0 (Sec. II-C);
  * noise: sigma = sqrt(1 / (2 R 10^(EbN0/10))) with R the nominal code rate
    after puncturing.  For R = 1/2 this is 10^(-EbN0/20); the printed formula
    in Sec. IX-B is garbled;
  * hard decision = 1 where y < 0 (packed eight per byte, bit 0 first);
  * int8 LLR  = clip(rint(32 y), -127, 127);
    4-bit LLR = clip(rint(2 y), -7, 7), two per byte, low nibble first;
    fp16 LLR  = half(2 y / sigma^2); fp64 LLR = 2 y / sigma^2;
    ``rint`` rounds half to even;
  * puncturing: pattern rows are output bits b, columns are stage phases
    (t mod period, phase 0 at the first stage of the stream or packet, running
    on through the tail); only kept positions are transmitted, stage-major
    with b ascending.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20111357900

# codes used by the workloads
K7_GENS = (0o171, 0o133)
K9_GENS = (0o557, 0o663, 0o711)
PUNCT_R23 = np.array([[1, 1], [1, 0]], dtype=np.uint8)
PUNCT_R34 = np.array([[1, 1, 0], [1, 0, 1]], dtype=np.uint8)


def seed_for(config: int, index: int) -> int:
    """Seed of input set ``index`` of workload ``config`` (1..5)."""
    return SEED_BASE + 100 * int(config) + int(index)


def rng_for(config: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, index)))


def random_bits(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(0, 2, size=int(n), dtype=np.uint8)


def conv_encode(K: int, gens, bits: np.ndarray) -> np.ndarray:
    """Convolutional encoder of Sec. II-A from the all-zero state.

    Output bit b at stage t is the XOR over m of g_b[m] * in[t - (K-1) + m]
    (bit K-1 of g_b taps the current input).  Implemented as a binary
    convolution; returns [n, beta] uint8.
    """
    bits = np.asarray(bits, dtype=np.uint8)
    n = bits.size
    out = np.empty((n, len(gens)), dtype=np.uint8)
    for b, g in enumerate(gens):
        taps = np.array([(g >> (K - 1 - d)) & 1 for d in range(K)], dtype=np.int32)
        acc = np.zeros(n, dtype=np.int32)
        for d in range(min(K, n)):
            if taps[d]:
                acc[d:] += bits[: n - d]
        out[:, b] = (acc & 1).astype(np.uint8)
    return out


def puncture_mask(pattern: np.ndarray, T: int) -> np.ndarray:
    """[T, beta] bool mask of transmitted positions (phase 0 at stage 0)."""
    pattern = np.asarray(pattern, dtype=bool)
    period = pattern.shape[1]
    reps = -(-T // period)
    return np.tile(pattern.T, (reps, 1))[:T]


def code_rate(beta: int, pattern=None) -> float:
    if pattern is None:
        return 1.0 / beta
    pattern = np.asarray(pattern)
    return pattern.shape[1] / float(pattern.sum())


def sigma_for(ebn0_db: float, rate: float) -> float:
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def quantise_s8(y: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(32.0 * y), -127, 127).astype(np.int8)


def quantise_s4(y: np.ndarray) -> np.ndarray:
    """4-bit values in [-7, 7] as int8 (unpacked)."""
    return np.clip(np.rint(2.0 * y), -7, 7).astype(np.int8)


def pack_s4(q: np.ndarray) -> np.ndarray:
    """Packs 4-bit values two per byte, low nibble = earlier value."""
    q = np.asarray(q, dtype=np.int8).reshape(-1)
    if q.size % 2:
        q = np.concatenate([q, np.zeros(1, dtype=np.int8)])
    lo = (q[0::2].astype(np.uint8) & 0x0F)
    hi = (q[1::2].astype(np.uint8) & 0x0F)
    return (lo | (hi << 4)).astype(np.uint8)


def llr_f64(y: np.ndarray, sigma: float) -> np.ndarray:
    return 2.0 * y / (sigma * sigma)


def hard_decide(y: np.ndarray) -> np.ndarray:
    """Hard decisions (Sec. II-C hard-decision mode): bit 1 where the sample
    is negative (BPSK sends bit 0 as +1), as uint8 0/1."""
    return (np.asarray(y) < 0.0).astype(np.uint8)


def pack_hard(bits: np.ndarray) -> np.ndarray:
    """Packs hard decisions eight per byte, earliest value in bit 0."""
    return np.packbits(np.asarray(bits, dtype=np.uint8).reshape(-1), bitorder="little")


@dataclass
class Stream:
    """One received stream: info bits, and the kept (transmitted) samples."""
    K: int
    gens: tuple
    n_info: int
    terminated: bool
    ebn0_db: float
    sigma: float
    bits: np.ndarray                 # [n_info] uint8
    y: np.ndarray                    # kept received samples (float64), stage-major
    pattern: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def beta(self):
        return len(self.gens)

    @property
    def T(self):
        return self.n_info + (self.K - 1 if self.terminated else 0)

    def s8(self):
        return quantise_s8(self.y)

    def s4(self):
        return quantise_s4(self.y)

    def f16(self):
        return llr_f64(self.y, self.sigma).astype(np.float16)

    def f64(self):
        return llr_f64(self.y, self.sigma)

    def hard(self):
        """Hard decisions of the kept samples, uint8 0/1 (unpacked)."""
        return hard_decide(self.y)


def make_stream(rng, K, gens, n_info, ebn0_db, terminated, pattern=None) -> Stream:
    """bits -> encoder (+ K-1 zero tail if terminated) -> puncture -> BPSK + AWGN."""
    bits = random_bits(rng, n_info)
    tx_bits = bits if not terminated else np.concatenate([bits, np.zeros(K - 1, np.uint8)])
    coded = conv_encode(K, gens, tx_bits)
    T = coded.shape[0]
    if pattern is not None:
        kept = coded[puncture_mask(pattern, T)]
    else:
        kept = coded.reshape(-1)
    rate = code_rate(len(gens), pattern)
    sigma = sigma_for(ebn0_db, rate)
    y = (1.0 - 2.0 * kept.astype(np.float64)) + sigma * rng.standard_normal(kept.size)
    return Stream(K, tuple(gens), int(n_info), bool(terminated), float(ebn0_db), sigma,
                  bits, y, None if pattern is None else np.asarray(pattern, np.uint8))


# ----------------------------------------------------------------- workloads

def plain_small(index: int = 0) -> Stream:
    """K=7 r1/2 171/133, one terminated frame of 4096 info bits, Eb/N0 = 3 dB."""
    return make_stream(rng_for(1, index), 7, K7_GENS, 4096, 3.0, terminated=True)


def segmented_stream(ebn0_db: float, n_info: int = 1 << 24, index: int | None = None) -> Stream:
    """K=7 r1/2 171/133 unterminated stream (default 2^24 info bits)."""
    idx = int(round(ebn0_db)) if index is None else index
    return make_stream(rng_for(2, idx), 7, K7_GENS, n_info, ebn0_db, terminated=False)


def precision_stream(ebn0_db: float, n_info: int = 1 << 24, index: int | None = None) -> Stream:
    """K=9 r1/3 557/663/711 unterminated stream (default 2^24 info bits)."""
    idx = int(round(ebn0_db)) if index is None else index
    return make_stream(rng_for(3, idx), 9, K9_GENS, n_info, ebn0_db, terminated=False)


@dataclass
class PacketBatch:
    """Uneven terminated packets, K=7 171/133 at r1/2, r2/3, r3/4 round-robin."""
    n_info: np.ndarray        # [P] int64
    rate_id: np.ndarray       # [P] 0 = r1/2, 1 = r2/3, 2 = r3/4
    ebn0_db: np.ndarray       # [P]
    llr_offset: np.ndarray    # [P] int64, offset of the packet's kept LLRs in the arena
    n_kept: np.ndarray        # [P] int64
    out_word_offset: np.ndarray  # [P] int64
    llr_s8: np.ndarray        # arena of kept int8 LLRs
    bits: np.ndarray          # concatenated info bits
    bit_offset: np.ndarray    # [P] int64

    @property
    def n_packets(self):
        return int(self.n_info.size)

    @property
    def total_bits(self):
        return int(self.n_info.sum())


RATE_PATTERNS = (None, PUNCT_R23, PUNCT_R34)


def packet_lengths(rng, n_packets, lo=96, hi=12000) -> np.ndarray:
    u = rng.uniform(math.log(lo), math.log(hi), size=n_packets)
    return np.floor(np.exp(u)).astype(np.int64)


def uneven_packets(n_packets: int = 65536, index: int = 0, lo: int = 96, hi: int = 12000,
                   K: int = 7, gens=K7_GENS) -> PacketBatch:
    """Batched workload: log-uniform info lengths in [lo, hi], Eb/N0 ~ U(2, 7)."""
    rng = rng_for(4, index)
    n_info = packet_lengths(rng, n_packets, lo, hi)
    rate_id = np.arange(n_packets, dtype=np.int64) % 3
    ebn0 = rng.uniform(2.0, 7.0, size=n_packets)
    beta = len(gens)
    # all packets' bits, each followed by its K-1 zero tail; since every tail
    # returns the encoder to state 0, one pass encodes every packet correctly
    total_info = int(n_info.sum())
    bits = random_bits(rng, total_info)
    T = n_info + (K - 1)
    stage_off = np.concatenate([[0], np.cumsum(T)[:-1]]).astype(np.int64)
    bit_off = np.concatenate([[0], np.cumsum(n_info)[:-1]]).astype(np.int64)
    tx = np.zeros(int(T.sum()), dtype=np.uint8)
    # scatter info bits into their stage slots
    pkt_of_bit = np.repeat(np.arange(n_packets), n_info)
    pos_in_pkt = np.arange(total_info, dtype=np.int64) - np.repeat(bit_off, n_info)
    tx[stage_off[pkt_of_bit] + pos_in_pkt] = bits
    coded = conv_encode(K, gens, tx)            # [sum T, beta]
    # keep mask: phase restarts at every packet's first stage
    pkt_of_stage = np.repeat(np.arange(n_packets), T)
    phase_in_pkt = np.arange(tx.size, dtype=np.int64) - np.repeat(stage_off, T)
    keep = np.ones((tx.size, beta), dtype=bool)
    for rid, pat in enumerate(RATE_PATTERNS):
        if pat is None:
            continue
        sel = rate_id[pkt_of_stage] == rid
        ph = phase_in_pkt[sel] % pat.shape[1]
        keep[sel] = pat.T.astype(bool)[ph]
    kept_bits = coded[keep]
    n_kept = np.bincount(pkt_of_stage, weights=keep.sum(axis=1), minlength=n_packets).astype(np.int64)
    llr_off = np.concatenate([[0], np.cumsum(n_kept)[:-1]]).astype(np.int64)
    rates = np.array([code_rate(beta, p) for p in RATE_PATTERNS])[rate_id]
    sig = np.sqrt(1.0 / (2.0 * rates * 10.0 ** (ebn0 / 10.0)))
    sig_per = np.repeat(sig, n_kept)
    llr = np.empty(kept_bits.size, dtype=np.int8)
    chunk = 1 << 24
    for s in range(0, kept_bits.size, chunk):
        e = min(kept_bits.size, s + chunk)
        y = (1.0 - 2.0 * kept_bits[s:e].astype(np.float64)) + sig_per[s:e] * rng.standard_normal(e - s)
        llr[s:e] = quantise_s8(y)
    out_words = (n_info + 31) // 32
    out_off = np.concatenate([[0], np.cumsum(out_words)[:-1]]).astype(np.int64)
    return PacketBatch(n_info, rate_id, ebn0, llr_off, n_kept, out_off, llr, bits, bit_off)


@dataclass
class ServingPacket:
    code_id: int          # 0: K=7 r1/2, 1: K=7 r3/4 (punctured), 2: K=9 r1/3
    n_info: int
    ebn0_db: float
    llr_s8: np.ndarray    # kept values, int8
    bits: np.ndarray


SERVING_CODES = ((7, K7_GENS, None), (7, K7_GENS, PUNCT_R34), (9, K9_GENS, None))


def serving_packets(n_packets: int, index: int = 0, punctured_share: float = 0.5):
    """Serving mix: payloads uniform in 40..1500 bytes (n_info = 8 x bytes),
    80% K=7 171/133 (a share of them punctured to r3/4), 20% K=9 557/663/711,
    Eb/N0 uniform in 1..6 dB, terminated, int8 LLRs."""
    rng = rng_for(5, index)
    out = []
    for _ in range(n_packets):
        nbytes = int(rng.integers(40, 1501))
        n = 8 * nbytes
        if rng.random() < 0.8:
            cid = 1 if rng.random() < punctured_share else 0
        else:
            cid = 2
        K, gens, pat = SERVING_CODES[cid]
        e = float(rng.uniform(1.0, 6.0))
        st = make_stream(rng, K, gens, n, e, True, pattern=pat)
        out.append(ServingPacket(cid, n, e, st.s8(), st.bits))
    return out


def flatten_packets(pkts):
    """The packets' int8 values in one array with per-packet offsets, counts and
    output word offsets (the layout the server's trace replay takes)."""
    n_values = np.array([p.llr_s8.size for p in pkts], dtype=np.int64)
    llr_offset = np.concatenate([[0], np.cumsum(n_values)[:-1]]).astype(np.int64)
    n_info = np.array([p.n_info for p in pkts], dtype=np.int64)
    words = (n_info + 31) // 32
    word_offset = np.concatenate([[0], np.cumsum(words)[:-1]]).astype(np.int64)
    llr = np.concatenate([p.llr_s8 for p in pkts]) if pkts else np.zeros(0, np.int8)
    return {"code_id": np.array([p.code_id for p in pkts], dtype=np.int32), "llr": llr,
            "llr_offset": llr_offset, "n_values": n_values, "n_info": n_info, "word_offset": word_offset}


def poisson_arrivals(rng, n, rate_per_s):
    """Arrival times (ns, from 0) of a Poisson process of the given rate."""
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    return np.floor(np.cumsum(gaps) * 1e9).astype(np.int64)
