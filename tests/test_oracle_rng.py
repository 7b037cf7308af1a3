"""Pins of the oracle's counter-based RNG (Philox4x32-10) and its uniform mapping.

The Philox pin is a library routine, not a retyping: Triton's Philox4x32-10 (the
`tl.philox` primitive, run on the CPU by Triton's interpreter) in a subprocess.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = textwrap.dedent(r"""
    import json, os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed_lo, seed_hi, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 0 + i * 4)
        c1 = tl.load(c_ptr + 1 + i * 4)
        c2 = tl.load(c_ptr + 2 + i * 4)
        c3 = tl.load(c_ptr + 3 + i * 4)
        seed = (seed_hi.to(tl.uint64) << 32) | seed_lo.to(tl.uint64)
        r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 0 + i * 4, r0)
        tl.store(out_ptr + 1 + i * 4, r1)
        tl.store(out_ptr + 2 + i * 4, r2)
        tl.store(out_ptr + 3 + i * 4, r3)

    cases = json.loads(sys.stdin.read())
    res = []
    for key, ctrs in cases:
        c = torch.tensor([x for ctr in ctrs for x in ctr], dtype=torch.int64).to(torch.uint32)
        out = torch.zeros_like(c)
        k[(1,)](c, out, key[0], key[1], N=len(ctrs))
        o = out.to(torch.int64).tolist()
        res.append([o[4 * j:4 * j + 4] for j in range(len(ctrs))])
    print(json.dumps(res))
""")


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(1)
    cases = []
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0xA4093822, 0x299F31D0],
                [int(x) for x in rng.integers(0, 2**32, 2)]):
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
        ctrs += [[int(x) for x in rng.integers(0, 2**32, 4)] for _ in range(5)]
        cases.append((key, ctrs))
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (key, ctrs), outs in zip(cases, ref):
        for ctr, want in zip(ctrs, outs):
            assert oracle.philox4x32_10(ctr, key) == [w & 0xFFFFFFFF for w in want], (key, ctr)


def test_uniform_is_exact_24bit_grid():
    u = oracle.uniform_batch(np.arange(20000), 3, 1, np.arange(20000) % 16, 12345)
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    scaled = u * 2.0**24
    assert np.all(scaled == np.floor(scaled))
    # the same value is representable in float32 (both sides see identical uniforms)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_uniform_keying_selects_words():
    # dims 4j..4j+3 are the four words of one Philox call with counter word 3 = j
    seed = (7 << 32) | 99
    for dim in range(12):
        out = oracle.philox4x32_10([11, 22, 33, dim >> 2], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.uniform(11, 22, 33, dim, seed) == (out[dim & 3] >> 8) / 2.0**24


def test_uniform_statistics():
    n = 200_000
    pix = np.arange(n) % 4096
    smp = np.arange(n) // 4096
    u = oracle.uniform_batch(pix, smp, 2, 5, 0)
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.002
    counts, _ = np.histogram(u, bins=256, range=(0, 1))
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, 255) > 1e-4
    # neighbouring dimensions and neighbouring pixels are uncorrelated
    v = oracle.uniform_batch(pix, smp, 2, 6, 0)
    w = oracle.uniform_batch(pix + 1, smp, 2, 5, 0)
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.01
    assert abs(np.corrcoef(u, w)[0, 1]) < 0.01
