"""The finite head start of a frame that starts from the reset state.

The decoder gives state 0 a lead HT over all other states instead of the
-infinity of a known start (Sec. II-B, Algorithm 1 with a known encoder
state).  That is exact when no path from another start state can overtake
the path from state 0 where they meet.  This brute force enumerates every
pair of trellis paths (any inputs) that start in state 0 and in a state
D != 0 and meet in one state within K-1 stages, and takes the largest number
of output bits in which they differ: with saturated LLRs of magnitude 127
the lead of the other path is 254 per differing bit.  For the (2,1,7)
171/133 code that is 10 bits, so HT = 254 * 10 + 1 = 2541 is the least head
start that keeps state 0's path strictly ahead; the K=9 557/663/711 code
gives 19 bits.  The GPU side of the same bound is the adversarial case in
test_gpu_parity.py.
"""
import itertools

import pytest


def _walk(K, gens, s, inputs):
    outs = []
    for u in inputs:
        r = (u << (K - 1)) | s
        outs += [bin(g & r).count("1") & 1 for g in gens]
        s = (u << (K - 2)) | (s >> 1)
    return s, outs


def max_differing_bits(K, gens):
    best = 0
    for k in range(1, K):
        from_zero = {}
        for u in itertools.product((0, 1), repeat=k):
            end, outs = _walk(K, gens, 0, u)
            from_zero[end] = outs
        for D in range(1, 1 << (K - 1)):
            for u in itertools.product((0, 1), repeat=k):
                end, outs = _walk(K, gens, D, u)
                if end in from_zero:
                    best = max(best, sum(a != b for a, b in zip(outs, from_zero[end])))
    return best


@pytest.mark.parametrize("K,gens,bits", [(7, (0o171, 0o133), 10), (9, (0o557, 0o663, 0o711), 19)])
def test_largest_lead_of_another_start_state(K, gens, bits):
    assert max_differing_bits(K, gens) == bits


def test_paths_that_meet_carry_the_same_inputs():
    """Within K-1 stages two paths can only meet if their inputs agree (the
    state holds the last K-1 inputs), so only the start-state bits still in
    the register make outputs differ."""
    K, gens = 7, (0o171, 0o133)
    for k in range(1, K):
        for D in range(1, 1 << (K - 1)):
            for u in itertools.product((0, 1), repeat=k):
                for w in itertools.product((0, 1), repeat=k):
                    if _walk(K, gens, D, u)[0] == _walk(K, gens, 0, w)[0]:
                        assert u == w


def test_kernel_constants_match_the_brute_force(tmp_path):
    """The decoder's compile-time DMAX and HT (Code<> in vd_device.cuh) equal
    the brute-force bound above: a host-only program prints them (nvcc, no
    GPU needed)."""
    import os
    import shutil
    import subprocess
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and not shutil.which(nvcc):
        pytest.skip("nvcc not found")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "ht.cu"
    src.write_text(
        '#include <cstdio>\n'
        '#include "vd_device.cuh"\n'
        'using C7 = vd::Code<7, 2, (uint64_t)0171 | ((uint64_t)0133 << 16)>;\n'
        'using C9 = vd::Code<9, 3, (uint64_t)0557 | ((uint64_t)0663 << 16) | ((uint64_t)0711 << 32)>;\n'
        'int main() { std::printf("%d %d %d %d\\n", C7::DMAX, C7::HT, C9::DMAX, C9::HT); return 0; }\n')
    exe = tmp_path / "ht"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(root, "paper_2011_13579_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    d7, ht7, d9, ht9 = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                text=True).stdout.split())
    assert (d7, d9) == (max_differing_bits(7, (0o171, 0o133)), max_differing_bits(9, (0o557, 0o663, 0o711)))
    assert (ht7, ht9) == (254 * d7 + 1, 254 * d9 + 1)
