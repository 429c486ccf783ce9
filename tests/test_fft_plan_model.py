"""The mixed-radix Stockham line FFT of the FFT kernels, restated in NumPy
with the per-pass twiddle tables laid out as the kernels lay them out, and
checked against numpy.fft for every configured length (the unitary 2-D FFT
of A = R F, Sec. 5.4, is a row pass and a column pass of these lines).

A pass of radix R after P points already transformed takes butterfly i
(i < N/R) over elements i + q N/R, multiplies input q by w_N^(q k N/(P R))
with k = i mod P, runs an R-point DFT and writes output q to
(i / P) P R + k + q P.  The factors of the pass come from its own table,
[q - 1][k], which starts at entry P - R0 (R0 the first radix), filled from
the global table w_N^j = exp(-2 pi i j / N).  The configured plans are read
from the kernels' header.
"""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1411_5057_gb300", "csrc", "fft.cuh")


def plans():
    out = []
    for m in re.finditer(r"FIRLS_FFT_CFG\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)",
                         open(HDR).read()):
        n, e, npass = int(m.group(1)), int(m.group(2)), int(m.group(3))
        radices = [int(m.group(4 + p)) for p in range(npass)]
        out.append((n, e, radices))
    return out


def pass_tables(N, radices):
    twg = np.exp(-2j * np.pi * np.arange(N) / N)
    tw = np.full(N + 1, np.nan, complex)
    P = radices[0]
    for R in radices[1:]:
        step, off = N // (P * R), P - radices[0]
        for i in range((R - 1) * P):
            q, k = i // P + 1, i % P
            assert np.isnan(tw[off + i])  # the tables do not overlap
            tw[off + i] = twg[q * k * step]
        P *= R
    return tw


def line_fft(x, radices, direction):
    N = len(x)
    tw = pass_tables(N, radices)
    v = x.astype(complex)
    P = 1
    for R in radices:
        out = np.empty(N, complex)
        dft = np.exp(direction * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        for i in range(N // R):
            k = i % P
            a = np.array([v[i + q * (N // R)] for q in range(R)])
            if P > 1:
                for q in range(1, R):
                    w = tw[(P - radices[0]) + (q - 1) * P + k]
                    a[q] *= w if direction < 0 else np.conj(w)
            A = dft @ a
            j = (i // P) * P * R + k
            out[j + np.arange(R) * P] = A
        v = out
        P *= R
    return v


@pytest.mark.parametrize("n,e,radices", plans(), ids=[str(p[0]) for p in plans()])
def test_plan_matches_numpy_fft(n, e, radices):
    assert int(np.prod(radices)) == n and n % e == 0
    assert all(e % r == 0 for r in radices)  # every radix divides the per-thread element count
    # the per-pass tables together hold N - R0 entries: they fit the N-entry table
    P, total = radices[0], 0
    for r in radices[1:]:
        total += (r - 1) * P
        P *= r
    assert total == n - radices[0]
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(line_fft(x, radices, -1), np.fft.fft(x), atol=1e-10 * n)
    assert np.allclose(line_fft(x, radices, +1), n * np.fft.ifft(x), atol=1e-10 * n)


def test_every_plan_is_present():
    assert sorted(p[0] for p in plans()) == [16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512]
