"""Pins for the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against one of: values the paper prints
(tests/golden/paper_trellis_facts.json), a brute-force maximum-likelihood
search, a noiseless channel, re-encoding of the survivor path, textbook
properties of the codes, or a symmetry of linear codes.  A dropped term, a
wrong sign, an off-by-one in the frame geometry or a swapped tie rule in the
oracle fails at least one of them.
"""
import heapq
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2011_13579_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


K7 = oracle.Code(7, synth.K7_GENS)
K9 = oracle.Code(9, synth.K9_GENS)


# ------------------------------------------------------------ trellis facts

def _branch_out(code, state, u):
    """alpha_out of the branch (state, u) via the oracle's FSM encoder."""
    return tuple(int(x) for x in oracle.encode_from(code, state, [u])[0])


def _next_state_from_history(K, state, u):
    """Shift-register definition (Sec. II-A): the state is the previous K-1
    inputs, most recent first; independent of the oracle's formula."""
    hist = [(state >> (K - 2 - k)) & 1 for k in range(K - 1)]   # in_{t-1}, in_{t-2}, ...
    new = [u] + hist[:-1]
    return sum(b << (K - 2 - k) for k, b in enumerate(new))


@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
def test_trellis_matches_independent_encoder(code):
    """Branch outputs of the oracle's FSM equal the convolution encoder's
    output for the input history that defines the state (Eq. encoder)."""
    K = code.K
    for s in range(code.n_states):
        hist = [(s >> (K - 2 - k)) & 1 for k in range(K - 1)]     # in_{t-1} ..
        for u in (0, 1):
            seq = np.array(hist[::-1] + [u], dtype=np.uint8)        # oldest first
            ref = synth.conv_encode(K, code.gens, seq)[-1]
            assert _branch_out(code, s, u) == tuple(int(x) for x in ref)


def test_generator_binary_reading():
    g = _golden("paper_trellis_facts.json")["code_k7"]
    assert [format(x, "b") for x in synth.K7_GENS] == g["gens_binary"]
    assert [format(x, "o") for x in synth.K7_GENS] == g["gens_octal"]


@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
def test_theorem1_butterflies(code):
    """Thm. 1 (Eq. radix2:S): left states 2f, 2f+1 reach exactly f and f+2^(k-2)."""
    K = code.K
    for f in range(1 << (K - 2)):
        reach = {_next_state_from_history(K, i, u) for i in (2 * f, 2 * f + 1) for u in (0, 1)}
        assert reach == {f, f + (1 << (K - 2))}


@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
def test_corollary_msb_lsb_generators(code):
    """Corollary (Eq. radix2:boRelatNot): with MSB = LSB = 1 in every
    generator, outer branches share an output and inner branches carry its
    complement."""
    K = code.K
    half = 1 << (K - 2)
    for f in range(half):
        i0, i1 = 2 * f, 2 * f + 1
        a00 = _branch_out(code, i0, 0)       # i0 -> j0 (input 0 leads to j0 = f)
        a11 = _branch_out(code, i1, 1)       # i1 -> j1
        a01 = _branch_out(code, i0, 1)       # i0 -> j1
        a10 = _branch_out(code, i1, 0)       # i1 -> j0
        assert a00 == a11
        assert a01 == tuple(1 - x for x in a00)
        assert a10 == tuple(1 - x for x in a00)


def test_radix2_theta_classes():
    """Sec. V-B: for k=7 (171,133), 32 butterflies over 4 distinct Theta, 8 each."""
    g = _golden("paper_trellis_facts.json")["radix2_theta_classes"]
    mains = [_branch_out(K7, 2 * f, 0) for f in range(1 << (K7.K - 2))]
    assert len(mains) == g["n_butterflies"]
    counts = {}
    for m in mains:
        counts[m] = counts.get(m, 0) + 1
    assert len(counts) == g["n_distinct"]
    assert set(counts.values()) == {g["per_class"]}


def _super_branch(code, i, j):
    """All two-stage paths i -> m -> j: list of (m, 2*beta output bits)."""
    K = code.K
    paths = []
    for u1 in (0, 1):
        m = _next_state_from_history(K, i, u1)
        for u2 in (0, 1):
            if _next_state_from_history(K, m, u2) == j:
                paths.append((m, _branch_out(code, i, u1) + _branch_out(code, m, u2)))
    return paths


def _dragonfly_states(K, f):
    """Eq. radix4:S."""
    q = 1 << (K - 3)
    left = [4 * f + y for y in range(4)]
    right = [f + y * q for y in range(4)]
    mid = [2 * f, 2 * f + 1, 2 * f + (1 << (K - 2)), 2 * f + (1 << (K - 2)) + 1]
    return left, mid, right


@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
def test_radix4_unique_paths(code):
    """Sec. VII theorem: exactly one two-stage path joins every left and right
    state of a radix-4 dragonfly, through the middle states of Eq. radix4:S."""
    K = code.K
    for f in range(1 << (K - 3)):
        left, mid, right = _dragonfly_states(K, f)
        for i in left:
            for j in right:
                p = _super_branch(code, i, j)
                assert len(p) == 1
                assert p[0][0] in mid


def _theta_hat(code, f):
    left, _, right = _dragonfly_states(code.K, f)
    return [[_super_branch(code, i, j)[0][1] for i in left] for j in right]   # P_j blocks


def test_radix4_theta_hat_distinct():
    """Sec. VIII-D-1: for k=7 (171,133) all 16 main super-branch outputs differ."""
    g = _golden("paper_trellis_facts.json")["radix4_theta_hat"]
    mains = [_theta_hat(K7, f)[0][0] for f in range(1 << (K7.K - 3))]
    assert len(mains) == g["n_dragonflies"]
    assert len(set(mains)) == g["n_distinct"]


def test_dragonfly_groups():
    """Sec. VIII-D-2: dragonflies whose P_j blocks are the same sets (up to a
    common permutation of left states) form exactly DG0..DG3."""
    g = _golden("paper_trellis_facts.json")["dragonfly_groups"]
    keys = {}
    for f in range(16):
        th = _theta_hat(K7, f)
        key = tuple(frozenset(block) for block in th)
        keys.setdefault(key, []).append(f)
    groups = sorted(sorted(v) for v in keys.values())
    assert groups == sorted([g["DG0"], g["DG1"], g["DG2"], g["DG3"]])
    # and one common permutation of left states maps every member onto the first
    for members in groups:
        base = _theta_hat(K7, members[0])
        for f in members[1:]:
            th = _theta_hat(K7, f)
            perms = [p for p in itertools.permutations(range(4))
                     if all([th[j][p[y]] for y in range(4)] == base[j] for j in range(4))]
            assert perms


def test_bit_extract_and_general_state_formula():
    """Eq. bit example (39 -> 3, 7) and Eq. general:S read with the
    post-bubble taken as the low rho-x bits of y, checked against the
    trellis: it reproduces the radix-4 indices of Eq. radix4:S and the
    dragonfly connectivity for rho = 1, 2, 3."""
    ex = _golden("paper_trellis_facts.json")["bit_extract_example"]

    def bits(x, b, a):
        return (x >> a) & ((1 << (b - a)) - 1)

    for b, a, want in ex["cases"]:
        assert bits(ex["x"], b, a) == want

    def s_general(K, rho, f, x, y):
        pre = bits(y, rho, rho - x) << (K - x - 1)
        bub = f << (rho - x)
        post = bits(y, rho - x, 0)
        return pre + bub + post

    for K in (5, 7):
        # rho = 2 matches Eq. radix4:S
        for f in range(1 << (K - 3)):
            left, mid, right = _dragonfly_states(K, f)
            assert [s_general(K, 2, f, 0, y) for y in range(4)] == left
            assert sorted(s_general(K, 2, f, 1, y) for y in range(4)) == sorted(mid)
            assert [s_general(K, 2, f, 2, y) for y in range(4)] == right
        # for every rho, stage x+1 states are exactly the successors of stage x states
        for rho in (1, 2, 3):
            for f in range(1 << (K - 1 - rho)):
                for x in range(rho):
                    cur = {s_general(K, rho, f, x, y) for y in range(1 << rho)}
                    nxt = {s_general(K, rho, f, x + 1, y) for y in range(1 << rho)}
                    succ = {_next_state_from_history(K, s, u) for s in cur for u in (0, 1)}
                    assert succ == nxt


def _free_distance(K, gens):
    """Smallest Hamming weight of a path leaving state 0 and returning to it
    (Dijkstra over the shift-register trellis; independent of the oracle)."""
    NS = 1 << (K - 1)

    def out_weight(s, u):
        hist = [(s >> (K - 2 - k)) & 1 for k in range(K - 1)]
        seq = np.array(hist[::-1] + [u], dtype=np.uint8)
        return int(synth.conv_encode(K, gens, seq)[-1].sum())

    start = _next_state_from_history(K, 0, 1)
    dist = {start: out_weight(0, 1)}
    heap = [(dist[start], start)]
    while heap:
        d, s = heapq.heappop(heap)
        if s == 0:
            return d
        if d > dist.get(s, 1 << 30):
            continue
        for u in (0, 1):
            t = _next_state_from_history(K, s, u)
            nd = d + out_weight(s, u)
            if nd < dist.get(t, 1 << 30):
                dist[t] = nd
                heapq.heappush(heap, (nd, t))
    assert NS > 0
    return None


def test_free_distances_textbook():
    facts = _golden("code_facts.json")
    assert _free_distance(7, synth.K7_GENS) == facts["k7_171_133_free_distance"]["value"]
    assert _free_distance(9, synth.K9_GENS) == facts["k9_557_663_711_free_distance"]["value"]


# ------------------------------------------------------------- P1 noiseless

def _noiseless_llr(code, bits, terminated, amp=127):
    tx = bits if not terminated else np.concatenate([bits, np.zeros(code.K - 1, np.uint8)])
    c = synth.conv_encode(code.K, code.gens, tx)
    return (amp * (1 - 2 * c.astype(np.int32))).astype(np.int32)


@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
@pytest.mark.parametrize("terminated", [False, True])
def test_noiseless_returns_message(code, terminated):
    rng = np.random.Generator(np.random.PCG64(12345))
    n = 3000
    bits = synth.random_bits(rng, n)
    llr = _noiseless_llr(code, bits, terminated)
    want = oracle.pack_bits(bits)
    assert np.array_equal(oracle.decode_full(code, llr, n, terminated=terminated), want)
    for f, v in ((256, 42), (96, code.K - 1), (100, 2 * code.K), (64, 0) if not terminated else (64, 7)):
        got = oracle.decode(code, llr, n, f=f, v=v, terminated=terminated, threads=3)
        if v < code.K - 1:
            continue   # with no overlap the frame edges are guesses; checked elsewhere
        assert np.array_equal(got, want), (f, v)
    # closed form: the final maximum metric is 127 * beta * T at the true end state
    path, org, em, im, a = oracle.trace_full(code, llr, n, f=n, v=code.K, s=0, terminated=terminated)
    T = oracle.n_stages(code, n, terminated)
    assert em == 127 * code.beta * T
    assert org == 0 and im == 0
    assert np.array_equal(path[:n], bits)


# --------------------------------------------------------- P2 brute force ML

def _all_messages(n):
    return ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def _batch_encode(K, gens, msgs):
    n = msgs.shape[1]
    out = np.zeros((msgs.shape[0], n, len(gens)), dtype=np.uint8)
    for b, g in enumerate(gens):
        acc = np.zeros(msgs.shape, dtype=np.int32)
        for d in range(K):
            if (g >> (K - 1 - d)) & 1:
                acc[:, d:] += msgs[:, : n - d]
        out[:, :, b] = acc & 1
    return out


def _brute_force(code, llr, n, terminated):
    msgs = _all_messages(n)
    tx = msgs if not terminated else np.concatenate(
        [msgs, np.zeros((msgs.shape[0], code.K - 1), np.uint8)], axis=1)
    cw = _batch_encode(code.K, code.gens, tx)                 # [M, T, beta]
    corr = ((1 - 2 * cw.astype(np.int64)) * llr[None, :, :].astype(np.int64)).sum(axis=(1, 2))
    return msgs, corr


@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (5, (0o23, 0o35)), (4, (0o13, 0o15, 0o17))])
@pytest.mark.parametrize("terminated", [False, True])
@pytest.mark.parametrize("kind", ["random", "erasures", "tiny"])
def test_brute_force_ml(K, gens, terminated, kind):
    code = oracle.Code(K, gens)
    rng = np.random.Generator(np.random.PCG64(777 + K + 10 * terminated))
    n = 12
    T = oracle.n_stages(code, n, terminated)
    for trial in range(6):
        if kind == "random":
            llr = rng.integers(-127, 128, size=(T, code.beta)).astype(np.int32)
        elif kind == "erasures":
            llr = rng.integers(-127, 128, size=(T, code.beta)).astype(np.int32)
            llr[rng.random((T, code.beta)) < 0.6] = 0
        else:
            llr = rng.integers(-2, 3, size=(T, code.beta)).astype(np.int32)
        msgs, corr = _brute_force(code, llr, n, terminated)
        best = corr.max()
        path, org, em, im, a = oracle.trace_full(code, llr, n, f=n, v=K, s=0, terminated=terminated)
        assert em == best, (kind, trial)
        dec = oracle.unpack_bits(oracle.decode_full(code, llr, n, terminated=terminated), n)
        idx = int((dec.astype(np.int64) << np.arange(n)).sum())
        assert corr[idx] == best
        if (corr == best).sum() == 1:
            assert idx == int(np.argmax(corr))


# ------------------------------------------------------------- P3 re-encode

@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
@pytest.mark.parametrize("terminated", [False, True])
def test_reencode_survivor_attains_metric(code, terminated):
    """Tracing any frame's survivor back to its first stage and re-encoding it
    from its origin state reproduces end metric - initial metric exactly."""
    rng = np.random.Generator(np.random.PCG64(99 + code.K))
    n = 700
    T = oracle.n_stages(code, n, terminated)
    llr = rng.integers(-127, 128, size=(T, code.beta)).astype(np.int32)
    llr[rng.random((T, code.beta)) < 0.3] = 0
    f, v = 128, 20
    for s in range(oracle._load().or_num_windows(n, f)):
        path, org, em, im, a = oracle.trace_full(code, llr, n, f=f, v=v, s=s, terminated=terminated)
        W = path.size
        hist = [(org >> k) & 1 for k in range(code.K - 1)]          # oldest first
        seq = np.concatenate([np.array(hist, np.uint8), path])
        cw = synth.conv_encode(code.K, code.gens, seq)[code.K - 1:]
        corr = int(((1 - 2 * cw.astype(np.int64)) * llr[a:a + W].astype(np.int64)).sum())
        assert corr == em - im, s
        if a == 0:
            assert org == 0 and im == 0
    # full length, terminated: the optimal correlation over all codewords
    path, org, em, im, a = oracle.trace_full(code, llr, n, f=n, v=code.K, s=0, terminated=terminated)
    cw = synth.conv_encode(code.K, code.gens, path)
    assert int(((1 - 2 * cw.astype(np.int64)) * llr.astype(np.int64)).sum()) == em


# --------------------------------------------- per-frame brute force (geometry)

def _brute_window(code, llr, n, T, f, v, s, terminated, start_unknown):
    """ML path over one frame by enumeration, with the frame rules stated in
    Sec. III (frames of f, v extra stages on each side, clipped) and the
    start/end rules; returns the decided bits of stages [o, e)."""
    K = code.K
    o, e = s * f, min(n, (s + 1) * f)
    a, b = max(0, o - v), min(T, (s + 1) * f + v)
    W = b - a
    starts = [0] if (a == 0 and not start_unknown) else list(range(code.n_states))
    best, arg = None, None
    for st in starts:
        hist = np.array([(st >> k) & 1 for k in range(K - 1)], np.uint8)
        msgs = _all_messages(W)
        seqs = np.concatenate([np.repeat(hist[None, :], msgs.shape[0], 0), msgs], axis=1)
        cw = _batch_encode(K, code.gens, seqs)[:, K - 1:]
        corr = ((1 - 2 * cw.astype(np.int64)) * llr[a:b][None].astype(np.int64)).sum(axis=(1, 2))
        if terminated and b == T:
            endst = np.zeros(msgs.shape[0], dtype=np.int64)
            for k in range(K - 1):
                endst |= seqs[:, -1 - k].astype(np.int64) << (K - 2 - k)
            corr = np.where(endst == 0, corr, np.iinfo(np.int64).min // 2)
        i = int(np.argmax(corr))
        if best is None or corr[i] > best:
            best, arg = corr[i], msgs[i]
            tie = (corr == corr[i]).sum() > 1
        elif corr[i] == best:
            tie = True
    return arg[o - a:e - a], tie


@pytest.mark.parametrize("terminated,start_unknown", [(False, False), (True, False), (False, True)])
def test_frame_geometry_brute_force(terminated, start_unknown):
    """Every frame of a segmented decode equals the maximum-likelihood path of
    that frame alone (no ties: wide-range LLRs), so the frame boundaries,
    the start rule and the end rule are all pinned."""
    code = oracle.Code(4, (0o13, 0o15))
    rng = np.random.Generator(np.random.PCG64(4242 + terminated + 2 * start_unknown))
    n, f, v = 21, 5, 3
    T = oracle.n_stages(code, n, terminated)
    for trial in range(3):
        llr = rng.integers(-100000, 100001, size=(T, code.beta)).astype(np.int32)
        got = oracle.unpack_bits(oracle.decode(code, llr, n, f=f, v=v, terminated=terminated,
                                               start_unknown=start_unknown), n)
        for s in range(-(-n // f)):
            want, tie = _brute_window(code, llr, n, T, f, v, s, terminated, start_unknown)
            if not tie:
                assert np.array_equal(got[s * f: s * f + want.size], want), (trial, s)


# ------------------------------------------------------ tie rules (Alg. 1/2)

def test_tie_rules_on_erased_stream():
    """With every LLR zero all candidates tie.  Algorithm 1's strict '>'
    keeps the second predecessor p1 = 2f+1 everywhere and Algorithm 2's
    argmax takes state 0, so the traceback walks state 0 -> 1 -> 3 -> 7 ...
    i.e. the decoded input at stage t is bit (k-2) of ((1 << (steps+1)) - 1)."""
    code = K7
    n = 40
    llr = np.zeros((n, 2), np.int32)
    got = oracle.unpack_bits(oracle.decode_full(code, llr, n), n)
    # walking back from state 0: states 0, 1, 3, 7, 15, 31, 63, 63, ... so the
    # decoded bit (MSB of the state after stage t) is 1 for all but the last
    # K-2+1 stages counted from the end
    js, want = 0, np.zeros(n, np.uint8)
    for t in range(n - 1, -1, -1):
        want[t] = js >> (code.K - 2)
        js = ((js << 1) & (code.n_states - 1)) | 1
    assert np.array_equal(got, want)
    assert got[-1] == 0 and got[0] == 1


# ----------------------------------------------------------- P9 symmetry

@pytest.mark.parametrize("code", [K7, K9], ids=["k7", "k9"])
@pytest.mark.parametrize("f,v", [(10 ** 6, 10), (64, 20)])
def test_linear_code_symmetry_fp64(code, f, v):
    """Flipping LLR signs along the codeword of m0 flips the decode by m0
    (continuous noise, so ties have probability zero)."""
    rng = np.random.Generator(np.random.PCG64(31337 + code.K))
    n = 900
    st = synth.make_stream(rng, code.K, code.gens, n, 2.0, terminated=True)
    llr = st.f64().reshape(-1, code.beta)
    m0 = synth.random_bits(rng, n)
    c0 = synth.conv_encode(code.K, code.gens, np.concatenate([m0, np.zeros(code.K - 1, np.uint8)]))
    llr2 = llr * (1 - 2 * c0.astype(np.float64))
    ff = min(f, n)
    d1, _, _ = oracle.decode_f64(code, llr, n, f=ff, v=v, terminated=True)
    d2, _, _ = oracle.decode_f64(code, llr2, n, f=ff, v=v, terminated=True)
    assert np.array_equal(oracle.unpack_bits(d2, n), oracle.unpack_bits(d1, n) ^ m0)


def test_f64_matches_i64_on_integer_inputs():
    """The fp64 oracle equals the int64 oracle on integer LLRs whose decisions
    are not ties (fp64 sums of small integers are exact)."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = 2000
    for code in (K7, K9):
        T = oracle.n_stages(code, n, False)
        llr = rng.integers(-127, 128, size=(T, code.beta)).astype(np.int32)
        a = oracle.decode(code, llr, n, f=256, v=42)
        b, gap, mx = oracle.decode_f64(code, llr.astype(np.float64), n, f=256, v=42)
        assert np.array_equal(a, b)
        assert np.all(mx > 0)


# ---------------------------------------------------------- P10 BER sanity

def test_ber_falls_with_snr_and_segmentation_costs():
    n = 1 << 15
    floor = _golden("paper_trellis_facts.json")["ber_validity"]["factor"] / n
    full_ber, seg_ber = [], []
    for ebn0 in (1.0, 2.0, 3.0):
        st = synth.segmented_stream(ebn0, n_info=n)
        llr = st.s8().reshape(-1, 2).astype(np.int32)
        full = oracle.unpack_bits(oracle.decode_full(K7, llr, n), n)
        seg = oracle.unpack_bits(oracle.decode(K7, llr, n, f=32, v=6, threads=4), n)
        full_ber.append(np.mean(full != st.bits))
        seg_ber.append(np.mean(seg != st.bits))
    assert full_ber[0] > full_ber[1] > full_ber[2]
    assert full_ber[0] > floor
    # a short overlap (v = k-1) costs BER at every point
    for fb, sb in zip(full_ber, seg_ber):
        assert sb >= fb


# ------------------------------------------------------------- depuncture

def test_depuncture_roundtrip():
    rng = np.random.Generator(np.random.PCG64(8))
    for pat in (synth.PUNCT_R23, synth.PUNCT_R34):
        code = oracle.Code(7, synth.K7_GENS, puncture=pat)
        T = 57
        full = rng.integers(-127, 128, size=(T, 2)).astype(np.int32)
        mask = synth.puncture_mask(pat, T)
        kept = full[mask]
        assert kept.size == code.n_kept(T)
        back = oracle.depuncture(code, kept, T)
        assert np.array_equal(back[mask], full[mask])
        assert np.all(back[~mask] == 0)
        with pytest.raises(ValueError):
            oracle.depuncture(code, kept[:-1], T)


def test_decode_frames_matches_full_decode():
    """The frame-subset entry point returns the same bits and metrics as the
    whole-stream decode for the frames it is asked for."""
    rng = np.random.Generator(np.random.PCG64(17))
    code = K7
    n, f, v = 3000, 256, 42
    llr = rng.integers(-127, 128, size=(n, 2)).astype(np.int32)
    words, pm = oracle.decode(code, llr, n, f=f, v=v, want_pm=True)
    allbits = oracle.unpack_bits(words, n)
    frames = [0, 3, 11]
    bits, pm_sel = oracle.decode_frames(code, llr, n, f, v, frames, want_pm=True)
    for k, s in enumerate(frames):
        e = min(n, (s + 1) * f)
        assert np.array_equal(bits[k, : e - s * f], allbits[s * f: e])
        assert np.array_equal(pm_sel[k], pm[s])


# ------------------------------------- metric vector and fp64 gaps, brute force

def _enumerate_window(code, llr, starts):
    """Every path through a window: for each start state in ``starts`` and
    each input sequence of the window's W stages, the cumulative correlation
    after l stages (l = 0..W) and the state after l stages.  Built from the
    shift-register definition of Sec. II-A with this file's own encoder,
    nothing from the oracle.  Returns (inputs [M, W], corr [M, W+1],
    state [M, W+1])."""
    K, beta = code.K, code.beta
    W = llr.shape[0]
    msgs = _all_messages(W)
    hists, ins = [], []
    for st in starts:
        hist = np.array([(st >> k) & 1 for k in range(K - 1)], np.uint8)   # oldest first
        hists.append(np.repeat(hist[None, :], msgs.shape[0], 0))
        ins.append(msgs)
    hist = np.concatenate(hists)
    u = np.concatenate(ins)
    seqs = np.concatenate([hist, u], axis=1)
    cw = _batch_encode(K, code.gens, seqs)[:, K - 1:]                       # [M, W, beta]
    per_stage = ((1 - 2 * cw.astype(np.float64)) * llr[None].astype(np.float64)).sum(axis=2)
    corr = np.concatenate([np.zeros((seqs.shape[0], 1)), np.cumsum(per_stage, axis=1)], axis=1)
    state = np.zeros((seqs.shape[0], W + 1), dtype=np.int64)
    for l in range(W + 1):
        # state after l stages: the last K-1 inputs, most recent as the MSB
        for k in range(K - 1):
            state[:, l] |= seqs[:, K - 2 + l - k].astype(np.int64) << (K - 2 - k)
    return u, corr, state


def _metric_vectors(code, corr, state):
    """lambda_j after l stages = the best correlation of any path in state j
    (Eq. PM unrolled: the maximum over whole paths), -inf if none reaches j."""
    NS = code.n_states
    L = np.full((corr.shape[1], NS), -np.inf)
    for l in range(corr.shape[1]):
        np.maximum.at(L[l], state[:, l], corr[:, l])
    return L


@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (5, (0o23, 0o35)), (4, (0o13, 0o15, 0o17))])
@pytest.mark.parametrize("start_unknown", [False, True])
@pytest.mark.parametrize("kind", ["random", "erasures"])
def test_final_metric_vector_brute_force(K, gens, start_unknown, kind):
    """The canonical final metric vector the oracle reports per frame
    (lambda - min lambda after the frame's last stage, Eq. PM) equals the
    best correlation of every path ending in each state, found by
    enumerating all paths of the frame, minus its minimum.  Frames in the
    middle of a stream start from any state (all-zero metrics, Algorithm 1);
    the first frame from state 0 unless the start is unknown."""
    code = oracle.Code(K, gens)
    rng = np.random.Generator(np.random.PCG64(9001 + K + 7 * start_unknown + (kind == "erasures")))
    n, f, v = 18, 6, 3                      # windows of up to f + 2v = 12 stages
    T = oracle.n_stages(code, n, False)
    for trial in range(3):
        llr = rng.integers(-127, 128, size=(T, code.beta)).astype(np.int32)
        if kind == "erasures":
            llr[rng.random((T, code.beta)) < 0.6] = 0
        _, pm = oracle.decode(code, llr, n, f=f, v=v, start_unknown=start_unknown, want_pm=True)
        for s in range(-(-n // f)):
            a, b = max(0, s * f - v), min(T, (s + 1) * f + v)
            starts = [0] if (a == 0 and not start_unknown) else list(range(code.n_states))
            _, corr, state = _enumerate_window(code, llr[a:b], starts)
            lam = _metric_vectors(code, corr, state)[-1]
            assert np.all(np.isfinite(lam))     # W >= K-1: every state is reachable
            want = (lam - lam.min()).astype(np.int64)
            assert np.array_equal(pm[s], want), (trial, s)


def test_final_metric_vector_full_length_closed_form():
    """Full length from state 0 on a noiseless codeword of amplitude 127:
    the canonical vector equals the enumerated best correlation per end
    state minus its minimum, the true end state holds the closed-form
    maximum 127 * beta * T, and every other state is strictly below it."""
    code = K7
    rng = np.random.Generator(np.random.PCG64(4711))
    n = 13
    bits = synth.random_bits(rng, n)
    llr = _noiseless_llr(code, bits, False)
    _, pm = oracle.decode(code, llr, n, f=n, v=code.K, want_pm=True)
    _, corr, state = _enumerate_window(code, llr, [0])
    lam = _metric_vectors(code, corr, state)[-1]
    assert np.array_equal(pm[0], (lam - lam.min()).astype(np.int64))
    end = 0
    for k in range(code.K - 1):
        end |= int(bits[n - 1 - k]) << (code.K - 2 - k)
    assert lam[end] == 127 * code.beta * n
    assert np.all(np.delete(lam, end) < lam[end])


@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (5, (0o23, 0o35))])
@pytest.mark.parametrize("terminated,start_unknown", [(False, False), (True, False), (False, True)])
def test_f64_gap_and_max_metric_brute_force(K, gens, terminated, start_unknown):
    """The fp64 oracle's per-frame min_gap and max_abs_pm, pinned by
    enumeration on continuous LLRs (no ties):
      * the traced path is the best path into the traceback start state;
      * at each traced stage t in [o, b) with state j after it, the decision
        gap is |c1 - c0|, c_x = lambda_{p_x}(t) + delta(p_x -> j), where
        lambda_{p_x}(t) + delta is the best correlation of the paths into j
        whose previous state is p_x (Eq. PM / Eq. SP0);
      * unless the frame ends at a terminated end, the best final metric
        minus the runner-up is also a gap;
      * max_abs_pm is the largest |lambda_j| of any reachable state after
        any stage of the frame."""
    code = oracle.Code(K, gens)
    rng = np.random.Generator(np.random.PCG64(1234 + K + 2 * terminated + 5 * start_unknown))
    n, f, v = 14, 5, 3
    T = oracle.n_stages(code, n, terminated)
    mask = code.n_states - 1
    for trial in range(3):
        llr = rng.normal(0.0, 2.0, size=(T, code.beta))
        _, gap, mx = oracle.decode_f64(code, llr, n, f=f, v=v, terminated=terminated,
                                       start_unknown=start_unknown)
        for s in range(-(-n // f)):
            o = s * f
            a, b = max(0, o - v), min(T, (s + 1) * f + v)
            starts = [0] if (a == 0 and not start_unknown) else list(range(code.n_states))
            u, corr, state = _enumerate_window(code, llr[a:b], starts)
            lam = _metric_vectors(code, corr, state)          # [W+1, NS]
            W = b - a
            want_mx = max(abs(x) for x in lam[1:].reshape(-1) if np.isfinite(x))
            assert mx[s] == pytest.approx(want_mx, rel=1e-12, abs=1e-12), (trial, s)
            gaps = []
            if terminated and b == T:
                js = 0
            else:
                fin = lam[W]
                js = int(np.argmax(fin))
                gaps.append(fin[js] - np.max(np.delete(fin, js)))
            # the best path into js at the last stage, and its states
            into = np.nonzero(state[:, W] == js)[0]
            best = into[np.argmax(corr[into, W])]
            path_states = state[best]
            for t in range(b - 1, o - 1, -1):
                l = t - a                      # stages done before stage t
                j = int(path_states[l + 1])
                p0 = (j << 1) & mask
                c = []
                for p in (p0, p0 | 1):
                    sel = np.nonzero((state[:, l] == p) & (state[:, l + 1] == j))[0]
                    c.append(np.max(corr[sel, l + 1]) if sel.size else -np.inf)
                gaps.append(abs(c[1] - c[0]))
            want_gap = min(gaps)
            assert gap[s] == pytest.approx(want_gap, rel=1e-9, abs=1e-9), (trial, s)


# --------------------------------------------------- hard decisions (Sec. II-C)

@pytest.mark.parametrize("K,gens", [(7, synth.K7_GENS), (5, (0o23, 0o35)), (4, (0o13, 0o15, 0o17))])
@pytest.mark.parametrize("terminated", [False, True])
@pytest.mark.parametrize("erasures", [False, True])
def test_hard_decision_brute_force_min_distance(K, gens, terminated, erasures):
    """Full-length hard-decision decoding returns a message whose codeword is
    at the minimum Hamming distance from the received bits (over the
    positions not erased), found by enumerating all 2^n messages; the
    argmin itself when it is unique."""
    code = oracle.Code(K, gens)
    rng = np.random.Generator(np.random.PCG64(606 + K + 2 * terminated + 4 * erasures))
    n = 12
    T = oracle.n_stages(code, n, terminated)
    msgs = _all_messages(n)
    tx = msgs if not terminated else np.concatenate(
        [msgs, np.zeros((msgs.shape[0], K - 1), np.uint8)], axis=1)
    cw = _batch_encode(K, gens, tx)                                   # [M, T, beta]
    for trial in range(6):
        rx = rng.integers(0, 2, size=(T, code.beta)).astype(np.uint8)
        if erasures:
            rx[rng.random((T, code.beta)) < 0.4] = 2
        dist = ((cw != rx[None]) & (rx[None] < 2)).sum(axis=(1, 2))
        dec = oracle.unpack_bits(oracle.decode_hard(code, rx, n, f=n, v=K + n, terminated=terminated), n)
        idx = int((dec.astype(np.int64) << np.arange(n)).sum())
        assert dist[idx] == dist.min(), trial
        if (dist == dist.min()).sum() == 1:
            assert idx == int(np.argmin(dist))


@pytest.mark.parametrize("pat", [None, synth.PUNCT_R23, synth.PUNCT_R34])
def test_hard_decision_noiseless_and_segmented(pat):
    """Received bits equal to the (punctured) codeword decode to the message,
    full length and segmented (f=256, v=42)."""
    rng = np.random.Generator(np.random.PCG64(607))
    code = oracle.Code(7, synth.K7_GENS, puncture=pat)
    n = 3000
    bits = synth.random_bits(rng, n)
    tx = np.concatenate([bits, np.zeros(6, np.uint8)])
    cw = synth.conv_encode(7, synth.K7_GENS, tx)
    T = cw.shape[0]
    kept = cw[synth.puncture_mask(pat, T)] if pat is not None else cw.reshape(-1)
    rx = oracle.depuncture_hard(code, kept, T)
    want = oracle.pack_bits(bits)
    assert np.array_equal(oracle.decode_hard(code, rx, n, f=n, v=n + 7, terminated=True), want)
    assert np.array_equal(oracle.decode_hard(code, rx, n, f=256, v=42, terminated=True), want)
    if pat is not None:
        assert np.all(rx[~synth.puncture_mask(pat, T)] == 2)


def test_hard_decision_equals_unit_llr_correlation():
    """Minimising the Hamming distance is maximising the correlation with
    +-1 LLRs (Eq. BM gives beta - 2 d per unerased stage): the hard-decision
    decode equals the soft decode of the same decisions as LLRs +1 / -1 / 0
    (erased), frame by frame, including the tie rules."""
    rng = np.random.Generator(np.random.PCG64(608))
    code = oracle.Code(7, synth.K7_GENS, puncture=synth.PUNCT_R34)
    n = 4000
    st = synth.make_stream(rng, 7, synth.K7_GENS, n, 1.0, True, pattern=synth.PUNCT_R34)
    rx = oracle.depuncture_hard(code, st.hard(), st.T)
    llr = np.where(rx == 2, 0, 1 - 2 * rx.astype(np.int32)).astype(np.int32)
    for f, v in ((256, 42), (64, 6), (n, n + 7)):
        a = oracle.decode_hard(code, rx, n, f=f, v=v, terminated=True)
        b = oracle.decode(code, llr, n, f=f, v=v, terminated=True)
        assert np.array_equal(a, b), (f, v)


# ------------------------------------------- transmitter and channel (Sec. IX-B)

@pytest.mark.parametrize("seed,sid", [(0, 0), (1, 2), (2011135790, 7), (2**64 - 1, 2**63 + 5)])
def test_philox4x64_matches_numpy(seed, sid):
    """The oracle's Philox4x64-10 equals NumPy's Philox bit generator, which
    advances its 256-bit counter before each block (so NumPy counter q - 1
    yields block q; q = 0 wraps around from all ones)."""
    for q in (0, 1, 2, 3, 1000, 2**40 + 3):
        prev = (q - 1) % 2**256
        ctr = np.array([(prev >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(key=np.array([seed, sid], dtype=np.uint64), counter=ctr)
        assert np.array_equal(oracle.philox4x64([q, 0, 0, 0], [seed, sid]), bg.random_raw(4)), q


@pytest.mark.parametrize("K,gens,pat,terminated", [(7, synth.K7_GENS, None, False), (7, synth.K7_GENS, "r23", True),
                                                   (7, synth.K7_GENS, "r34", True), (9, synth.K9_GENS, None, True)])
def test_transmit_noiseless_is_bpsk_of_the_codeword(K, gens, pat, terminated):
    """sigma = 0: the received samples are the BPSK symbols (bit 0 -> +1) of
    the punctured codeword of this file's independent encoder."""
    pattern = {None: None, "r23": synth.PUNCT_R23, "r34": synth.PUNCT_R34}[pat]
    code = oracle.Code(K, gens, puncture=pattern)
    rng = np.random.Generator(np.random.PCG64(700 + K))
    n = 1001
    bits = synth.random_bits(rng, n)
    tx = bits if not terminated else np.concatenate([bits, np.zeros(K - 1, np.uint8)])
    cw = synth.conv_encode(K, gens, tx)
    kept = cw[synth.puncture_mask(pattern, cw.shape[0])] if pattern is not None else cw.reshape(-1)
    y = oracle.transmit(code, bits, n, terminated, 0.0, seed=5)
    assert np.array_equal(y, 1.0 - 2.0 * kept.astype(np.float64))


def test_transmit_noise_is_standard_normal():
    """y - x over 400k samples is standard normal (Kolmogorov-Smirnov), and
    the samples do not depend on sigma except through the scale."""
    scipy_stats = pytest.importorskip("scipy.stats")
    code = oracle.Code(7, synth.K7_GENS)
    rng = np.random.Generator(np.random.PCG64(701))
    n = 200_000
    bits = synth.random_bits(rng, n)
    x = oracle.transmit(code, bits, n, False, 0.0, seed=11, stream_id=3)
    y = oracle.transmit(code, bits, n, False, 0.7, seed=11, stream_id=3)
    z = (y - x) / 0.7
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size) and abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / z.size)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    y2 = oracle.transmit(code, bits, n, False, 1.4, seed=11, stream_id=3)
    assert np.allclose((y2 - x) / 1.4, z, rtol=0, atol=1e-12)
    other = oracle.transmit(code, bits, n, False, 0.7, seed=11, stream_id=4)
    assert not np.array_equal(other, y)


def test_quantisers_match_the_synthetic_recipe():
    """The oracle's quantisers equal the input generator's (an independent
    implementation of the same recipe)."""
    rng = np.random.Generator(np.random.PCG64(702))
    y = rng.normal(0.0, 3.0, size=50_000)
    y[:8] = [0.0, -0.0, 1.0 / 64, -1.0 / 64, 0.25, -0.75, 200.0, -200.0]
    sigma = 0.8
    assert np.array_equal(oracle.quantise(y, "s8"), synth.quantise_s8(y))
    assert np.array_equal(oracle.quantise(y, "s4"), synth.quantise_s4(y))
    assert np.array_equal(oracle.quantise(y, "f16", sigma).view(np.uint16),
                          synth.llr_f64(y, sigma).astype(np.float16).view(np.uint16))
    assert np.array_equal(oracle.quantise(y, "hard"), synth.hard_decide(y))
