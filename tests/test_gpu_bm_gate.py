"""Branch-metric gate: the CUDA-core and tensor-core (mma.sync) forms of
Eq. BM give exactly the metrics of the definition, in the decoder's layout."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2011_13579_gb300 as vd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vd.build()
    yield


@pytest.mark.parametrize("n_pairs,n_stages", [(32, 1), (96, 7), (4096, 33)])
def test_both_forms_equal_definition(n_pairs, n_stages):
    rng = np.random.Generator(np.random.PCG64(n_pairs + n_stages))
    llr = rng.integers(-127, 128, size=(n_stages, n_pairs, 2, 2), dtype=np.int8)
    llr[0, 0] = 127
    llr[-1, -1] = -127
    words = torch.from_numpy(llr.reshape(-1).view(np.uint32).copy()).cuda()
    # Eq. BM: metric of output pattern x = sum_b (-1)^{x_b} l_b, per frame half
    l = llr.astype(np.int64)
    want = np.empty((n_stages, 4, n_pairs), dtype=np.uint32)
    for x in range(4):
        s0 = (-1) ** (x & 1)
        s1 = (-1) ** ((x >> 1) & 1)
        m = s0 * l[..., 0] + s1 * l[..., 1]          # [stage, pair, half]
        h = (m & 0xFFFF).astype(np.uint32)
        want[:, x, :] = h[:, :, 0] | (h[:, :, 1] << 16)
    sums = []
    for variant in (0, 1):
        cs = torch.zeros(n_pairs, dtype=torch.int32, device="cuda")
        out = torch.zeros(n_stages * 4 * n_pairs, dtype=torch.int32, device="cuda")
        vd.vd_bm_gate(variant, words, n_pairs, n_stages, cs, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(n_stages, 4, n_pairs)
        assert np.array_equal(got, want), variant
        sums.append(cs.cpu().numpy())
    assert np.array_equal(sums[0], sums[1])


def test_gate_rejects_bad_arguments():
    words = torch.zeros(64, dtype=torch.int32, device="cuda")
    cs = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(vd.VdError):
        vd.vd_bm_gate(2, words, 32, 1, cs)
    with pytest.raises(vd.VdError):
        vd.vd_bm_gate(0, words, 33, 1, cs)
