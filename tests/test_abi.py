"""The C-ABI library builds, loads, exports every symbol include/vd.h declares,
and validates arguments on the host (no GPU needed: nothing here launches)."""
import ctypes
import os
import re
import subprocess

import pytest

import oracle
import paper_2011_13579_gb300 as vd
from paper_2011_13579_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    vd.build()
    return vd.lib()


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(vd_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "vd_decode" in names and "vd_code_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", vd._build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(vd_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_version_and_counts(lib):
    assert vd.vd_version() >= 100
    assert vd.vd_num_frames(0, 256) == 0
    assert vd.vd_num_frames(1, 256) == 1
    assert vd.vd_num_frames(1 << 24, 256) == 65536
    assert vd.vd_num_frames(257, 256) == 2


@pytest.mark.parametrize("pat", [None, synth.PUNCT_R23, synth.PUNCT_R34])
def test_num_kept_matches_oracle(lib, pat):
    c = vd.Code(7, synth.K7_GENS, puncture=pat)
    oc = oracle.Code(7, synth.K7_GENS, puncture=pat)
    for T in (0, 1, 2, 3, 5, 100, 4102, 12006):
        assert c.n_kept(T) == oc.n_kept(T)


def test_code_create_validation(lib):
    with pytest.raises(vd.VdError) as e:
        vd.vd_code_create(10, (0o171, 0o133))
    assert e.value.status == vd.VD_EINVAL and "K=10" in str(e.value)
    with pytest.raises(vd.VdError) as e:
        vd.vd_code_create(7, (0o71, 0o133))     # does not tap the current input
    assert e.value.status == vd.VD_EINVAL
    with pytest.raises(vd.VdError) as e:
        vd.vd_code_create(7, (0o171, 0o133), rate=(2, 3))   # rate does not match pattern
    assert e.value.status == vd.VD_EINVAL
    with pytest.raises(vd.VdError) as e:
        vd.vd_code_create(7, (0o171, 0o133), puncture=[[1, 0], [0, 0]])   # empty column
    assert e.value.status == vd.VD_EINVAL
    with pytest.raises(vd.VdError) as e:
        vd.vd_code_create(7, (0o171, 0o133, 0o165))           # valid but not built
    assert e.value.status == vd.VD_EUNSUPPORTED
    h = vd.vd_code_create(7, (0o171, 0o133), rate=(2, 3), puncture=synth.PUNCT_R23)
    vd.vd_code_destroy(h)
    assert vd.vd_code_supported(9, synth.K9_GENS)
    assert not vd.vd_code_supported(9, (0o561, 0o753))


def test_decode_argument_validation(lib):
    """Bad arguments are rejected on the host before any CUDA call."""
    c = vd.Code(7, synth.K7_GENS)
    L = vd.lib()
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first

    def call(n_info, f, v, radix, flags, llr_type=vd.VD_LLR_S8, llr=fake, out=fake):
        return L.vd_decode(ctypes.c_void_p(c.handle), llr, llr_type, n_info, f, v, radix, flags,
                           out, None, None, None)

    assert call(100, 0, 6, 2, 0) == vd.VD_EINVAL
    assert call(100, 64, -1, 2, 0) == vd.VD_EINVAL
    assert call(100, 64, 6, 3, 0) == vd.VD_EINVAL
    assert call(100, 64, 6, 2, 0x80) == vd.VD_EINVAL
    assert call(100, 48, 6, 2, 0) == vd.VD_EINVAL          # f not a multiple of 32
    assert "multiple of 32" in vd.vd_last_error()
    assert call(100, 64, 6, 2, 0, llr_type=7) == vd.VD_EINVAL
    assert call(100, 64, 6, 2, 0, llr=None) == vd.VD_EINVAL
    assert call(-1, 64, 6, 2, 0) == vd.VD_EINVAL
    assert call(0, 64, 6, 2, 0, llr=None, out=None) == vd.VD_OK   # empty stream: no-op
    assert L.vd_decode(None, fake, 0, 10, 64, 6, 2, 0, fake, None, None, None) == vd.VD_EINVAL


def test_no_cpu_fallback_in_package():
    """The product path never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2011_13579_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "viterbi_oracle" not in text, fn


def test_get_tune_reports_the_decode_configuration():
    code = vd.Code(7, synth.K7_GENS)
    t = vd.vd_get_tune(code.handle, vd.VD_LLR_S8, 256, 42, 4)
    assert (t.f, t.v, t.radix, t.lanes, t.threads) == (256, 42, 4, 1, 128)
    t = vd.vd_get_tune(code.handle, vd.VD_LLR_F16, 256, 42, 4)
    assert t.radix == 2 and t.lanes == 2
    k9 = vd.Code(9, synth.K9_GENS)
    assert vd.vd_get_tune(k9.handle, vd.VD_LLR_S4, 512, 64, 2).lanes == 4
    with pytest.raises(vd.VdError):
        vd.vd_get_tune(code.handle, vd.VD_LLR_S8, 0, 42, 2)
    with pytest.raises(vd.VdError):
        vd.vd_get_tune(code.handle, vd.VD_LLR_S8, 256, 42, 3)


def test_chained_launch_validates_on_the_host(lib):
    """vd_batch_plan_launch_chained checks its arguments before any device work,
    and the binding keeps graph replay and chained launches apart."""
    assert lib.vd_batch_plan_launch_chained(None, None, None, None) == vd.VD_EINVAL
    with pytest.raises(ValueError):
        vd.vd_batch_plan_launch(0, None, None, graph=True, chained=True)
