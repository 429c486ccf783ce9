"""The row-scan form of the TV preconditioner's L U sweeps (Sec. 4.2, the
printed factors L = I + L_P D^-1, U = D + U_P of P, Eq. ptv), restated in
NumPy and checked against the oracle's sparse triangular solves.

The ILU kernel runs a sweep row by row:
* The coupling to the row above (forward) or below (backward) is
  elementwise.
* Along the row, y_c = t_c + g_c y_{c-1} is a first-order recurrence. Each
  of 32 lanes holds E = ceil(n/32) consecutive columns and composes them into
  one affine map y -> A y + B.
* An exclusive Kogge-Stone scan of those maps across the lanes gives the
  value entering every segment.
* Each lane then applies its columns.

The backward sweep is the same in reverse order.  ia = 1/diag(P) and the
coefficients come from P's own off-diagonals, so the model checks the
decomposition, not the weight formula (the oracle's own tests pin that).
"""
import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O


def lane_scan_exclusive(A, B, reverse):
    """Exclusive scan over 32 lanes of maps y -> A y + B (composition in lane
    order, or from lane 31 down), by doubling; the entry value is 0."""
    A, B = A.copy(), B.copy()
    lanes = len(A)
    off = 1
    while off < lanes:
        An, Bn = A.copy(), B.copy()
        for L in range(lanes):
            src = L + off if reverse else L - off
            if 0 <= src < lanes:
                # the lane's map after the one `off` lanes earlier
                Bn[L] = A[L] * B[src] + B[L]
                An[L] = A[L] * A[src]
        A, B = An, Bn
        off *= 2
    vin = np.zeros_like(B)
    for L in range(lanes):
        src = L + 1 if reverse else L - 1
        if 0 <= src < lanes:
            vin[L] = B[src]  # inclusive value of the previous lane, applied to 0
    return vin


def sweep_rows(n, t_of_row, g, reverse):
    """Row-scan sweep: rows in order (reverse: from the last), each row
    y_c = t_c + g_c y_{c -/+ 1} through 32 lane segments."""
    E = -(-n // 32)
    width = 32 * E
    out = np.zeros((n, n), complex)
    rows = range(n - 1, -1, -1) if reverse else range(n)
    prev = None
    for k in rows:
        t = np.zeros(width, complex)
        gg = np.zeros(width)
        t[:n] = t_of_row(k, prev)
        gg[:n] = g[k]
        seg_t, seg_g = t.reshape(32, E), gg.reshape(32, E)
        A = np.ones(32)
        B = np.zeros(32, complex)
        order = range(E - 1, -1, -1) if reverse else range(E)
        for e in order:  # the lane's segment as one map
            B = seg_g[:, e] * B + seg_t[:, e]
            A = A * seg_g[:, e]
        v = lane_scan_exclusive(A, B, reverse)
        y = np.zeros((32, E), complex)
        for e in order:
            v = seg_g[:, e] * v + seg_t[:, e]
            y[:, e] = v
        out[k] = y.reshape(-1)[:n]
        prev = out[k]
    return out


def ilu_model(P, r, n):
    P = P.tocsr()
    a = P.diagonal()
    ia = (1.0 / a).reshape(n, n)
    N = n * n
    off = lambda i, j: P[i, j] if 0 <= j < N else 0.0
    # forward: y_i = r_i - P[i,i-1] ia_{i-1} y_{i-1} - P[i,i-n] ia_{i-n} y_{i-n}
    gf = np.zeros((n, n))
    hf = np.zeros((n, n))
    gb = np.zeros((n, n))
    hb = np.zeros((n, n))
    for k in range(n):
        for c in range(n):
            i = k * n + c
            if c > 0:
                gf[k, c] = -off(i, i - 1) * ia.reshape(-1)[i - 1]
            if k > 0:
                hf[k, c] = -off(i, i - n) * ia.reshape(-1)[i - n]
            if c < n - 1:
                gb[k, c] = -off(i, i + 1) * ia.reshape(-1)[i]
            if k < n - 1:
                hb[k, c] = -off(i, i + n) * ia.reshape(-1)[i]
    y = sweep_rows(n, lambda k, above: r[k] + (hf[k] * above if above is not None else 0), gf, False)
    # backward: z_i = ia_i y_i - P[i,i+1] ia_i z_{i+1} - P[i,i+n] ia_i z_{i+n}
    z = sweep_rows(n, lambda k, below: ia[k] * y[k] + (hb[k] * below if below is not None else 0), gb, True)
    return z


@pytest.mark.parametrize("n", [32, 64, 96])
def test_row_scan_sweeps_equal_triangular_solves(n):
    mask = fs.vd_mask(n, 0.25, 3)
    sysm = O.System(mask, False, O.PSI_TV, 0, 0.0, 8e-4)
    rng = np.random.default_rng(n)
    x = fs.complex_phantom(n, 4) + 0.05 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sysm.update_weights(x)
    r = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    z = ilu_model(sysm.P, r, n)
    ref = sysm.apply_Pinv(r).reshape(n, n)
    assert np.max(np.abs(z - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_exclusive_scan_is_the_sequential_recurrence():
    rng = np.random.default_rng(1)
    A = rng.uniform(-1, 1, 32)
    B = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    for reverse in (False, True):
        vin = lane_scan_exclusive(A, B, reverse)
        v = 0
        for L in (range(31, -1, -1) if reverse else range(32)):
            assert abs(vin[L] - v) < 1e-12
            v = A[L] * v + B[L]
