"""vd_batch_plan_launch_chained: back-to-back launches that may overlap.

Every chained launch must give the bits of an isolated vd_batch_plan_launch
(itself checked against the oracle in test_gpu_batch.py and, at full size,
in test_gpu_fullsize.py): for the same buffers, for alternating input and
output arenas, for consecutive launches that write the same output words from
different inputs (the later one must win), mixed with ordinary launches, for
K=9, and for a plan with a pre-pass, which launches as an ordinary one.
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


N = 1 << 20
NS = 4


def _plan(code, beta, f, v, n=N, ns=NS):
    pk = {"code_id": np.zeros(ns, np.int32), "llr_type": np.zeros(ns, np.int32),
          "llr_offset": np.arange(ns, dtype=np.int64) * beta * n, "n_info": np.full(ns, n, np.int64),
          "flags": np.zeros(ns, np.uint32), "f": np.full(ns, f, np.int32), "v": np.full(ns, v, np.int32),
          "out_word_offset": np.arange(ns, dtype=np.int64) * (n // 32)}
    return vd.BatchPlan([code], pk)


# buffers are made on the default stream and used on another: synchronise
def _arena(make, ebn0s):
    a = torch.from_numpy(np.concatenate([make(e).s8() for e in ebn0s]).view(np.uint8)).cuda()
    torch.cuda.synchronize()
    return a


def _isolated(plan, arena, s):
    out = _new_out()
    plan.launch(arena, out, stream=s)
    s.synchronize()
    return out.clone()


def _new_out(words=NS * N // 32):
    o = torch.full((words,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    return o


@pytest.fixture(scope="module")
def k7_setup():
    code = vd.Code(7, synth.K7_GENS)
    a = _arena(lambda e: synth.segmented_stream(e, n_info=N), (1.0, 2.0, 3.0, 4.0))
    b = _arena(lambda e: synth.segmented_stream(e, n_info=N, index=7), (1.5, 2.5, 3.5, 6.0))
    plan = _plan(code, 2, 256, 42)
    s = torch.cuda.Stream()
    ref_a, ref_b = _isolated(plan, a, s), _isolated(plan, b, s)
    assert not torch.equal(ref_a, ref_b)
    yield code, plan, s, a, b, ref_a, ref_b
    plan.close()


def test_chained_same_buffers_match_isolated(k7_setup):
    _, plan, s, a, _, ref_a, _ = k7_setup
    out = _new_out()
    for _ in range(6):
        plan.launch(a, out, stream=s, chained=True)
    s.synchronize()
    assert torch.equal(out, ref_a)


def test_chained_alternating_arenas(k7_setup):
    _, plan, s, a, b, ref_a, ref_b = k7_setup
    oa, ob = _new_out(), _new_out()
    for _ in range(4):
        plan.launch(a, oa, stream=s, chained=True)
        plan.launch(b, ob, stream=s, chained=True)
    s.synchronize()
    assert torch.equal(oa, ref_a) and torch.equal(ob, ref_b)


def test_chained_later_launch_wins_shared_output(k7_setup):
    """Consecutive launches write the same words from different inputs: each
    waits for the one before to complete before its first output word."""
    _, plan, s, a, b, ref_a, ref_b = k7_setup
    for last, ref in ((b, ref_b), (a, ref_a)):
        out = _new_out()
        for _ in range(3):
            plan.launch(a, out, stream=s, chained=True)
            plan.launch(b, out, stream=s, chained=True)
        plan.launch(last, out, stream=s, chained=True)
        s.synchronize()
        assert torch.equal(out, ref)


def test_chained_mixed_with_ordinary_launches(k7_setup):
    _, plan, s, a, b, ref_a, ref_b = k7_setup
    seq = [(a, False), (b, True), (a, True), (b, False), (a, True), (a, True), (b, False), (b, True)]
    outs = []
    for arena, chained in seq:
        o = _new_out()
        plan.launch(arena, o, stream=s, chained=chained)
        outs.append(o)
    s.synchronize()
    for (arena, _), o in zip(seq, outs):
        assert torch.equal(o, ref_a if arena is a else ref_b)
    assert vd.vd_batch_plan_info(plan.handle).scratch_bytes > 0


def test_chained_matches_oracle_on_a_sampled_stream(k7_setup):
    code, plan, s, a, _, _, _ = k7_setup
    out = _new_out()
    for _ in range(3):
        plan.launch(a, out, stream=s, chained=True)
    s.synchronize()
    st = synth.segmented_stream(2.0, n_info=N)
    want = oracle.decode(oracle.Code(7, synth.K7_GENS), st.s8().reshape(-1, 2).astype(np.int32), N, 256, 42,
                         threads=8)
    got = out.cpu().numpy().view(np.uint32)[N // 32: 2 * N // 32]
    assert np.array_equal(got, want)


def test_chained_k9():
    code = vd.Code(9, synth.K9_GENS)
    a = _arena(lambda e: synth.precision_stream(e, n_info=N), (0.0, 1.0, 2.0, 3.0))
    plan = _plan(code, 3, 512, 64)
    s = torch.cuda.Stream()
    ref = _isolated(plan, a, s)
    out = _new_out()
    for _ in range(4):
        plan.launch(a, out, stream=s, chained=True)
    s.synchronize()
    assert torch.equal(out, ref)
    plan.close()


def test_chained_with_prepass_launches_as_ordinary():
    code = vd.Code(7, synth.K7_GENS, puncture=synth.PUNCT_R34.tolist())
    rng = np.random.Generator(np.random.PCG64(4242))
    n = 1 << 16
    streams = [synth.make_stream(rng, 7, synth.K7_GENS, n, 3.0, False, synth.PUNCT_R34).s8() for _ in range(NS)]
    kept = streams[0].size
    arena = torch.from_numpy(np.concatenate(streams).view(np.uint8)).cuda()
    torch.cuda.synchronize()
    pk = {"code_id": np.zeros(NS, np.int32), "llr_type": np.zeros(NS, np.int32),
          "llr_offset": np.arange(NS, dtype=np.int64) * kept, "n_info": np.full(NS, n, np.int64),
          "flags": np.zeros(NS, np.uint32), "f": np.full(NS, 256, np.int32), "v": np.full(NS, 42, np.int32),
          "out_word_offset": np.arange(NS, dtype=np.int64) * (n // 32)}
    plan = vd.BatchPlan([code], pk)
    s = torch.cuda.Stream()
    ref = _new_out(NS * n // 32)
    plan.launch(arena, ref, stream=s)
    out = _new_out(NS * n // 32)
    for _ in range(3):
        plan.launch(arena, out, stream=s, chained=True)
    s.synchronize()
    assert torch.equal(out, ref)
    plan.close()


def test_chained_mixed_code_kinds():
    """A plan of K=7 and K=9 packets launches one kernel per code kind; chained,
    the second kernel of a launch may also start beside the first."""
    k7, k9 = vd.Code(7, synth.K7_GENS), vd.Code(9, synth.K9_GENS)
    n = 1 << 18
    s7 = [synth.segmented_stream(e, n_info=n).s8() for e in (1.0, 3.0)]
    s9 = [synth.precision_stream(e, n_info=n).s8() for e in (0.0, 2.0)]
    vals = s7 + s9
    offs = np.concatenate([[0], np.cumsum([v.size for v in vals])[:-1]]).astype(np.int64)
    arena = torch.from_numpy(np.concatenate(vals).view(np.uint8)).cuda()
    torch.cuda.synchronize()
    pk = {"code_id": np.array([0, 0, 1, 1], np.int32), "llr_type": np.zeros(4, np.int32),
          "llr_offset": offs, "n_info": np.full(4, n, np.int64), "flags": np.zeros(4, np.uint32),
          "f": np.array([256, 256, 512, 512], np.int32), "v": np.array([42, 42, 64, 64], np.int32),
          "out_word_offset": np.arange(4, dtype=np.int64) * (n // 32)}
    plan = vd.BatchPlan([k7, k9], pk)
    s = torch.cuda.Stream()
    ref = _new_out(4 * n // 32)
    plan.launch(arena, ref, stream=s)
    s.synchronize()
    outs = [_new_out(4 * n // 32) for _ in range(3)]
    for _ in range(2):
        for o in outs:
            plan.launch(arena, o, stream=s, chained=True)
    s.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    plan.close()
