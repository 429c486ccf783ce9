"""The in-place schedule of the one-launch wavelet term u = Phi^T (w o Phi x)
(Sec. 3.1: Phi orthogonal, Mallat pyramid), restated in NumPy and checked
against the oracle's wavedec2 / waverec2.

The kernel splits a slice into C blocks of R = n/C rows (one CTA each) and
runs every level in place:
* level l keeps its row r at local row r * 2^(l-1);
* a row step stores a row as [lowpass | highpass];
* a column step streams down a column, split into equal pair ranges (one
  thread each), and leaves pair k as rows 2k, 2k+1;
* the Daubechies-4 column steps take two rows of the neighbouring block (its
  first two rows forward, its last pair inverse);
* a coefficient is scaled by its weight as soon as it is final;
* the range that reads the halo does every other pair first.
Every position ends holding exactly one coefficient, whose Mallat row is
given by the coefficient-row map.  This model follows that schedule
step by step (ranges run one after the other, which any interleaving after
the boundary reads is equivalent to) so that a wrong index, order or halo
fails here, without a GPU.
"""
import math

import numpy as np
import pytest

from oracle import firls_oracle as O


def rows_per_block(n, L):
    """The shape rule of the one-launch form: most blocks (at most 8) with an
    even number of rows per block at every level, at most 32 rows."""
    if n % 8 or n > 256 or L < 1 or L > 5 or (n >> L) % 4:
        return 0
    for C in range(8, 0, -1):
        if n % (C << L) == 0 and n // C <= 32:
            return n // C
    return 0


def coef_row(rho, j, n, L, R, blk):
    """Mallat row of the coefficient at local row rho, column j of block blk."""
    for l in range(1, L + 1):
        m, r = n >> (l - 1), rho >> (l - 1)
        k = blk * ((R >> (l - 1)) // 2) + (r >> 1)
        if r & 1:
            return m // 2 + k
        if j >= m // 2 or l == L:
            return k
    raise AssertionError


def model(x, w, kind, L, threads):
    n = x.shape[0]
    R = rows_per_block(n, L)
    C = n // R
    h, g = O.wavelet_filters(kind)
    K = len(h)

    def fwd(xs):
        return sum(h[t] * xs[t] for t in range(K)), sum(g[t] * xs[t] for t in range(K))

    def inv(am, dm, al, dl):
        if K == 2:
            return h[0] * al + g[0] * dl, h[1] * al + g[1] * dl
        return (h[0] * al + g[0] * dl + h[2] * am + g[2] * dm,
                h[1] * al + g[1] * dl + h[3] * am + g[3] * dm)

    D = [x[b * R:(b + 1) * R].astype(np.complex128) for b in range(C)]
    Wm = [np.array([[w[coef_row(rho, j, n, L, R, b), j] for j in range(n)] for rho in range(R)]) for b in range(C)]

    def rows(Dk, sr, Rl, m, inverse):
        half = m // 2
        for rr in range(Rl):
            row = Dk[rr * sr, :m].copy()
            out = np.empty(m, complex)
            for k in range(half):
                if not inverse:
                    out[k], out[half + k] = fwd([row[(2 * k + t) % m] for t in range(K)])
                else:
                    km = k - 1 if k else half - 1
                    out[2 * k], out[2 * k + 1] = inv(row[km], row[half + km], row[k], row[half + k])
            Dk[rr * sr, :m] = out

    def pairs(Dk, b, sr, m, k0, k1, e0, e1, inverse, last_level):
        """Pairs [k0, k1) of every column (vectorised over columns);
        forward (e0, e1) are rows 2 k1, 2 k1 + 1, inverse pair k0 - 1."""
        lo_final = np.array([last_level or j >= m // 2 for j in range(m)])

        def sc(v, rho, lowpass):
            f = Wm[b][rho, :m]
            return np.where(lo_final, v * f, v) if lowpass else v * f

        R_ = lambda rr: Dk[rr * sr, :m].copy()
        if K == 2:
            for kk in range(k0, k1):
                a0, a1 = R_(2 * kk), R_(2 * kk + 1)
                if not inverse:
                    o0, o1 = fwd([a0, a1])
                    o0, o1 = sc(o0, 2 * kk * sr, True), sc(o1, (2 * kk + 1) * sr, False)
                else:
                    o0, o1 = inv(None, None, a0, a1)
                Dk[2 * kk * sr, :m], Dk[(2 * kk + 1) * sr, :m] = o0, o1
        elif not inverse:
            for kk in range(k0, k1):
                r2 = R_(2 * kk + 2) if kk + 1 < k1 else e0
                r3 = R_(2 * kk + 3) if kk + 1 < k1 else e1
                a, d = fwd([R_(2 * kk), R_(2 * kk + 1), r2, r3])
                Dk[2 * kk * sr, :m] = sc(a, 2 * kk * sr, True)
                Dk[(2 * kk + 1) * sr, :m] = sc(d, (2 * kk + 1) * sr, False)
        else:
            am, dm = e0, e1
            for kk in range(k0, k1):
                al, dl = R_(2 * kk), R_(2 * kk + 1)
                Dk[2 * kk * sr, :m], Dk[(2 * kk + 1) * sr, :m] = inv(am, dm, al, dl)
                am, dm = al, dl

    def cols(l, m, Rl, sr, inverse, halos):
        npair = Rl // 2
        parts = 1
        while parts * 2 * m <= threads and npair % (parts * 2) == 0:
            parts *= 2
        per = npair // parts
        # every range reads its neighbour's boundary rows first
        pre = {}
        for b in range(C):
            for p in range(parts):
                k0 = p * per
                if not inverse and p + 1 < parts:
                    pre[b, p] = (Dk_row(b, 2 * (k0 + per), sr, m), Dk_row(b, 2 * (k0 + per) + 1, sr, m))
                if inverse and p > 0:
                    pre[b, p] = (Dk_row(b, 2 * k0 - 2, sr, m), Dk_row(b, 2 * k0 - 1, sr, m))
        for b in range(C):
            order = range(parts) if inverse else reversed(range(parts))
            for p in order:
                k0, k1 = p * per, p * per + per
                edge = K == 4 and (p == 0 if inverse else p + 1 == parts)
                if not edge:
                    e0, e1 = pre.get((b, p), (None, None))
                    pairs(D[b], b, sr, m, k0, k1, e0, e1, inverse, l == L)
                elif not inverse:  # all but the last pair, then the last with the halo
                    if k1 - k0 >= 2:
                        pairs(D[b], b, sr, m, k0, k1 - 1, Dk_row(b, 2 * (k1 - 1), sr, m),
                              Dk_row(b, 2 * (k1 - 1) + 1, sr, m), False, l == L)
                    pairs(D[b], b, sr, m, k1 - 1, k1, halos[b][0], halos[b][1], False, l == L)
                else:  # pairs after the first, then the first with the halo
                    if k1 - k0 >= 2:
                        pairs(D[b], b, sr, m, k0 + 1, k1, Dk_row(b, 2 * k0, sr, m),
                              Dk_row(b, 2 * k0 + 1, sr, m), True, False)
                    pairs(D[b], b, sr, m, k0, k0 + 1, halos[b][0], halos[b][1], True, False)

    def Dk_row(b, rr, sr, m):
        return D[b][rr * sr, :m].copy()

    for l in range(1, L + 1):
        m, Rl, sr = n >> (l - 1), R >> (l - 1), 1 << (l - 1)
        for b in range(C):
            rows(D[b], sr, Rl, m, False)
        halos = [(Dk_row((b + 1) % C, 0, sr, m), Dk_row((b + 1) % C, 1, sr, m)) for b in range(C)]
        cols(l, m, Rl, sr, False, halos)
    for l in range(L, 0, -1):
        m, Rl, sr = n >> (l - 1), R >> (l - 1), 1 << (l - 1)
        halos = [(Dk_row((b - 1) % C, Rl - 2, sr, m), Dk_row((b - 1) % C, Rl - 1, sr, m)) for b in range(C)]
        cols(l, m, Rl, sr, True, halos)
        for b in range(C):
            rows(D[b], sr, Rl, m, True)
    return np.concatenate(D, axis=0)


@pytest.mark.parametrize("n,L,kind,threads", [
    (256, 4, O.PSI_DB4, 512),    # the specialised shape: 8 blocks of 32 rows, 2..4 ranges per column
    (64, 3, O.PSI_DB4, 256),     # 8 blocks of 8 rows
    (64, 4, O.PSI_DB4, 256),     # 4 blocks of 16 rows
    (96, 3, O.PSI_DB4, 256),     # 6 blocks of 16 rows
    (192, 3, O.PSI_HAAR, 256),   # 8 blocks of 24 rows: odd pair counts at the coarse level
    (128, 4, O.PSI_DB4, 256),
])
def test_schedule_reproduces_phi_t_w_phi(n, L, kind, threads):
    assert rows_per_block(n, L) > 0
    rng = np.random.default_rng(n + L)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w = rng.random((n, n)) + 0.5
    ref = O.waverec2(w * O.wavedec2(x, kind, L), kind, L)
    got = model(x, w, kind, L, threads)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_coefficient_row_map_is_a_partition():
    """Every Mallat position is held by exactly one (block, local row, column)."""
    for n, L in ((256, 4), (64, 3), (96, 3), (192, 4)):
        R = rows_per_block(n, L)
        C = n // R
        seen = np.zeros((n, n), int)
        for b in range(C):
            for rho in range(R):
                for j in range(n):
                    seen[coef_row(rho, j, n, L, R, b), j] += 1
        assert (seen == 1).all(), (n, L)


def test_shape_rule():
    assert rows_per_block(256, 4) == 32       # 8 blocks
    assert rows_per_block(192, 4) == 32       # 6 blocks
    assert rows_per_block(512, 5) == 0        # too large for one cluster's shared memory
    assert rows_per_block(64, 5) == 0         # the coarsest level would be narrower than 4
    assert math.gcd(256 // rows_per_block(256, 4), 8) == 8
