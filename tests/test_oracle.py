"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself:
brute-force definitions on tiny inputs, closed forms, invariants (adjoints,
orthogonality, Theorem 2 monotonicity, Theorem 3 stationarity), published
values (Daubechies-4 taps, Fig. 1 group examples) and special cases that
reduce to textbook solutions (soft thresholding).
"""
import math
import os

import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed=0):
    return np.random.default_rng(seed)


def crandn(r, *shape):
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def dense_op(f, n, dtype=complex):
    """Matrix of a linear map on n x n images (column j = f(e_j))."""
    N = n * n
    cols = []
    for j in range(N):
        e = np.zeros(N, dtype=dtype)
        e[j] = 1
        cols.append(np.asarray(f(e.reshape(n, n))).reshape(-1))
    return np.stack(cols, axis=1)


# --------------------------------------------------------------- FFT / A ---

@pytest.mark.parametrize("n", [8, 12, 20])
def test_fft_matches_naive_dft(n):
    """Unitary DFT against the O(N^2) definition, radix 2, 3 and 5 sizes."""
    x = crandn(rng(n), n, n)
    k = np.arange(n)
    Wn = np.exp(-2j * np.pi * np.outer(k, k) / n) / math.sqrt(n)
    naive = np.zeros((n, n), complex)
    for a in range(n):
        for b in range(n):
            naive[a, b] = np.sum(Wn[a, :, None] * Wn[b, None, :] * x)
    assert np.allclose(O.fft2u(x), naive, atol=1e-12, rtol=0)
    assert np.allclose(O.ifft2u(naive), x, atol=1e-12, rtol=0)
    # Parseval
    assert abs(np.linalg.norm(naive) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("real", [False, True])
def test_A_adjoint(real):
    n = 16
    r = rng(1)
    mask = fs.vd_mask(n, 0.3, 5).astype(float)
    x = r.standard_normal((n, n)) if real else crandn(r, n, n)
    y = mask * crandn(r, n, n)
    lhs = np.real(np.vdot(O.op_A(x, mask), y))
    rhs = np.real(np.vdot(x, O.op_AH(y, mask, real)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_AHA_diagonal_equals_sampling_ratio():
    """Every diagonal entry of F^H R^T R F is M/N (Sec. 5.4: abar = ratio)."""
    n = 8
    mask = fs.vd_mask(n, 0.4, 3).astype(float)
    S = dense_op(lambda e: O.op_AH(O.op_A(e, mask), mask, False), n)
    M = mask.sum()
    assert np.allclose(np.diag(S), M / (n * n), atol=1e-13)
    assert O.a_bar(mask) == M / (n * n)


# ------------------------------------------------------------- wavelets ---

def test_db4_taps_match_published_values():
    vals = [float(l) for l in open(os.path.join(GOLDEN, "db4_taps.txt")) if l.strip() and not l.startswith("#")]
    h, g = O.wavelet_filters(O.PSI_DB4)
    assert np.allclose(h, vals, atol=5e-15)
    # orthonormality to even shifts and two vanishing moments of g
    assert abs(np.sum(h) - math.sqrt(2)) < 1e-14
    assert abs(np.sum(h * h) - 1) < 1e-14
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-15
    t = np.arange(4)
    assert abs(np.sum(g)) < 1e-14 and abs(np.sum(g * t)) < 1e-14


def test_haar_2x2_closed_form():
    x = np.array([[1.0, 2.0], [3.0, 5.0]])
    c = O.wavedec2(x, O.PSI_HAAR, 1)
    a, b, cc, d = x[0, 0], x[0, 1], x[1, 0], x[1, 1]
    expect = np.array([[a + b + cc + d, a - b + cc - d],
                       [a + b - cc - d, a - b - cc + d]]) / 2
    assert np.allclose(c, expect, atol=1e-15)


@pytest.mark.parametrize("kind,levels", [(O.PSI_HAAR, 1), (O.PSI_HAAR, 4), (O.PSI_DB4, 1), (O.PSI_DB4, 2), (O.PSI_DB4, 3)])
def test_wavelet_orthogonal_dense(kind, levels):
    n = 16
    Phi = dense_op(lambda e: O.wavedec2(e, kind, levels), n, dtype=float)
    I = np.eye(n * n)
    assert np.allclose(Phi.T @ Phi, I, atol=1e-12)
    assert np.allclose(Phi @ Phi.T, I, atol=1e-12)
    PhiT = dense_op(lambda e: O.waverec2(e, kind, levels), n, dtype=float)
    assert np.allclose(PhiT, Phi.T, atol=1e-12)


def test_db4_level1_bruteforce():
    """One level against a_{k,l} = sum_{s,t} h_s h_t x_{2k+s, 2l+t} (periodic)."""
    n = 12
    x = rng(2).standard_normal((n, n))
    h, g = O.wavelet_filters(O.PSI_DB4)
    c = O.wavedec2(x, O.PSI_DB4, 1)
    half = n // 2
    for k in range(half):
        for l in range(half):
            acc = {"LL": 0.0, "LH": 0.0, "HL": 0.0, "HH": 0.0}
            for s in range(4):
                for t in range(4):
                    v = x[(2 * k + s) % n, (2 * l + t) % n]
                    acc["LL"] += h[s] * h[t] * v
                    acc["LH"] += h[s] * g[t] * v   # vertical low, horizontal high
                    acc["HL"] += g[s] * h[t] * v
                    acc["HH"] += g[s] * g[t] * v
            assert abs(c[k, l] - acc["LL"]) < 1e-13
            assert abs(c[k, half + l] - acc["LH"]) < 1e-13
            assert abs(c[half + k, l] - acc["HL"]) < 1e-13
            assert abs(c[half + k, half + l] - acc["HH"]) < 1e-13


def test_haar_multilevel_closed_form():
    """Two and three Haar levels in closed form (Mallat pyramid on the LL band).

    With h = (1, 1)/sqrt2 and g = (1, -1)/sqrt2 every level-l coefficient is
    a signed sum over a 2^l x 2^l block divided by 2^l: LL the plain sum,
    the horizontal detail left half minus right half, the vertical detail
    top half minus bottom half, the diagonal detail the checkerboard of the
    four quadrants.  A recursion on another quadrant than LL, or a band
    stored in the other off-diagonal quadrant, fails here.
    """
    x = rng(5).standard_normal((16, 16))
    for levels in (1, 2, 3):
        c = O.wavedec2(x, O.PSI_HAAR, levels)
        n = 16
        for l in range(1, levels + 1):
            b = 1 << l           # block side at level l
            h = n >> l           # side of each level-l band
            hb = b // 2
            for p in range(h):
                for q in range(h):
                    blk = x[p * b:(p + 1) * b, q * b:(q + 1) * b]
                    tl, tr = blk[:hb, :hb].sum(), blk[:hb, hb:].sum()
                    bl, br = blk[hb:, :hb].sum(), blk[hb:, hb:].sum()
                    assert abs(c[p, h + q] - (tl + bl - tr - br) / b) < 1e-12      # horizontal detail
                    assert abs(c[h + p, q] - (tl + tr - bl - br) / b) < 1e-12      # vertical detail
                    assert abs(c[h + p, h + q] - (tl - tr - bl + br) / b) < 1e-12  # diagonal detail
                    if l == levels:
                        assert abs(c[p, q] - blk.sum() / b) < 1e-12                # LL of the last level


def _db4_taps_from_golden():
    vals = [float(l) for l in open(os.path.join(GOLDEN, "db4_taps.txt")) if l.strip() and not l.startswith("#")]
    h = np.array(vals)
    g = np.array([(-1) ** t * h[3 - t] for t in range(4)])
    return h, g


def _analysis_rows_bruteforce(n, levels, h, g):
    """1-D level-l scaling (type 0) and wavelet (type 1) functionals by loops.

    Level 1: row k of the lowpass is e_i -> sum_t h_t [i == (2k + t) mod n].
    Level l: row k is sum_t f_t * (level l-1 scaling row (2k + t) mod m),
    m = n / 2^(l-1), with f = h (scaling) or g (wavelet).
    Returns rows[l][type] as arrays [n / 2^l][n].
    """
    rows = {}
    prev = np.eye(n)   # level-0 scaling rows: the unit vectors
    for l in range(1, levels + 1):
        m = n >> (l - 1)
        lo = np.zeros((m // 2, n))
        hi = np.zeros((m // 2, n))
        for k in range(m // 2):
            for t in range(len(h)):
                lo[k] += h[t] * prev[(2 * k + t) % m]
                hi[k] += g[t] * prev[(2 * k + t) % m]
        rows[l] = (lo, hi)
        prev = lo
    return rows


@pytest.mark.parametrize("n,levels", [(16, 2), (16, 3), (32, 4)])
def test_db4_multilevel_bruteforce(n, levels):
    """Every coefficient of the multi-level D4 pyramid against a brute-force
    separable sum of level-l functionals built from the published taps.

    The level-l band (vertical type br, horizontal type bc) at rows
    [br h, br h + h) and columns [bc h, bc h + h), h = n / 2^l, holds
    c[p, q] = sum_{i,j} R_{l,br}[p, i] R_{l,bc}[q, j] x[i, j]; the LL band
    of the last level sits at the top-left.  Checks the recursion quadrant,
    the band placement and the row/column roles at every level.
    """
    h, g = _db4_taps_from_golden()
    rows = _analysis_rows_bruteforce(n, levels, h, g)
    x = rng(6).standard_normal((n, n)) + 1j * rng(7).standard_normal((n, n))
    c = O.wavedec2(x, O.PSI_DB4, levels)
    expect = np.full((n, n), np.nan, dtype=complex)
    for l in range(1, levels + 1):
        hh = n >> l
        for br, bc in ((0, 1), (1, 0), (1, 1)):
            expect[br * hh:(br + 1) * hh, bc * hh:(bc + 1) * hh] = rows[l][br] @ x @ rows[l][bc].T
    hh = n >> levels
    expect[:hh, :hh] = rows[levels][0] @ x @ rows[levels][0].T
    assert not np.isnan(expect).any()
    assert np.max(np.abs(c - expect)) < 1e-12 * np.max(np.abs(expect))


@pytest.mark.parametrize("kind,levels", [(O.PSI_HAAR, 2), (O.PSI_HAAR, 3), (O.PSI_DB4, 2), (O.PSI_DB4, 3)])
def test_wavelet_diag_bruteforce(kind, levels):
    """diag(Phi^T W Phi) against the dense product at n = 16."""
    n = 16
    Phi = dense_op(lambda e: O.wavedec2(e, kind, levels), n, dtype=float)
    w = rng(3).random(n * n) * 10
    brute = np.diag(Phi.T @ np.diag(w) @ Phi)
    assert np.allclose(O.wavelet_diag(w, n, kind, levels).reshape(-1), brute, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------- TV ---

def test_tv_matrices_stencil_and_adjoint():
    n = 5
    x = crandn(rng(4), n, n)
    D1, D2 = O.tv_matrices(n)
    g1 = (D1 @ x.reshape(-1)).reshape(n, n)
    g2 = (D2 @ x.reshape(-1)).reshape(n, n)
    for r in range(n):
        for c in range(n):
            assert abs(g1[r, c] - (x[r, c] - (x[r, c - 1] if c > 0 else 0))) < 1e-14
            assert abs(g2[r, c] - (x[r, c] - (x[r - 1, c] if r > 0 else 0))) < 1e-14
    # unit diagonal, -1 on sub-diagonals 1 and n (printed form, Sec. 4.1)
    assert np.all(D1.diagonal() == 1) and np.all(D2.diagonal() == 1)
    assert np.all(D2.diagonal(-n) == -1)
    d1 = D1.diagonal(-1)
    assert np.all(d1[np.arange(1, n * n) % n != 0] == -1)


def test_tv_system_is_pentadiagonal_with_closed_form_entries():
    """D1^T W D1 + D2^T W D2: symmetric, bands 0, +-1, +-n (Sec. 4.2)."""
    n = 6
    W = rng(5).random(n * n) + 0.1
    D1, D2 = O.tv_matrices(n)
    import scipy.sparse as sp
    T = (D1.T @ sp.diags(W) @ D1 + D2.T @ sp.diags(W) @ D2).toarray()
    assert np.allclose(T, T.T)
    Wm = W.reshape(n, n)
    for i in range(n * n):
        r, c = divmod(i, n)
        a = 2 * Wm[r, c] + (Wm[r, c + 1] if c < n - 1 else 0) + (Wm[r + 1, c] if r < n - 1 else 0)
        assert abs(T[i, i] - a) < 1e-13
        if c < n - 1:
            assert abs(T[i, i + 1] + Wm[r, c + 1]) < 1e-13
        if r < n - 1:
            assert abs(T[i, i + n] + Wm[r + 1, c]) < 1e-13
        nz = {j for j in range(n * n) if abs(T[i, j]) > 0}
        assert nz <= {i, i - 1, i + 1, i - n, i + n}


def test_tv_ilu_factor_identity():
    """The printed L, U satisfy LU = P + L_P diag(a)^-1 U_P and LU = L D L^T."""
    n = 6
    mask = fs.vd_mask(n, 0.3, 1)
    sysm = O.System(mask, False, O.PSI_TV, 0, 0.0, 0.5)
    sysm.update_weights(crandn(rng(6), n, n))
    P = sysm.P.toarray()
    L = sysm.L.toarray()
    U = sysm.U.toarray()
    a = np.diag(P)
    LP, UP = np.tril(P, -1), np.triu(P, 1)
    assert np.allclose(L @ U - P, LP @ np.diag(1 / a) @ UP, atol=1e-12)
    assert np.allclose(np.tril(L, -1) * 0 + np.diag(L), 1)
    LU = L @ U
    assert np.allclose(LU, LU.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(LU) > 0)
    r = crandn(rng(7), n, n)
    z = sysm.apply_Pinv(r).reshape(-1)
    assert np.allclose(LU @ z, r.reshape(-1), atol=1e-10)


# --------------------------------------------------------------- groups ---

def _fig1():
    rows = []
    for line in open(os.path.join(GOLDEN, "fig1_groups.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, size, groups = [s.strip() for s in line.split("|")]
        groups = [[int(v) - 1 for v in g.split(",")] for g in groups.split(";")]
        rows.append((name, int(size), np.array(groups, dtype=np.int32)))
    return rows


@pytest.mark.parametrize("name,size,groups", _fig1())
def test_fig1_group_matrices(name, size, groups):
    G, sizes = O.group_matrix(groups, 8)
    Gd = G.toarray()
    assert Gd.shape == (groups.size, 8) and np.all(sizes == size)
    # every row of G is a row of the identity
    assert np.all(Gd.sum(axis=1) == 1) and set(np.unique(Gd)) <= {0.0, 1.0}
    r = 0
    for gi in groups:
        for j in gi:
            assert Gd[r, j] == 1
            r += 1
    # G^T W G is diagonal; its diagonal sums the weights of the groups holding j
    Wg = np.arange(1, len(groups) + 1, dtype=float)
    M = Gd.T @ np.diag(np.repeat(Wg, sizes)) @ Gd
    assert np.allclose(M, np.diag(np.diag(M)))
    expect = np.zeros(8)
    for k, gi in enumerate(groups):
        expect[gi] += Wg[k]
    assert np.allclose(O.gwg_diag(Wg, G, sizes), expect)


def test_singleton_weights_are_irls_weights():
    """Singleton groups give W_i = (|c_i|^2 + eps)^-1/2 (Sec. 3.1 remark)."""
    c = crandn(rng(8), 64)
    G, sizes = O.group_matrix(None, 64)
    Wg = O.group_weights(c, G, sizes)
    assert np.allclose(Wg, 1 / np.sqrt(np.abs(c) ** 2 + O.EPS), rtol=1e-14)


def test_tree_groups_structure():
    n, L = 16, 3
    gr = fs.tree_groups(n, L)
    N, nLL = n * n, (n >> L) ** 2
    assert gr.shape == (N - nLL, 2) and gr.dtype == np.int32
    assert np.all(np.diff(gr[:, 0]) > 0)
    counts = np.bincount(gr.reshape(-1), minlength=N).reshape(n, n)
    h1 = n >> 1
    fine = np.zeros((n, n), bool)
    fine[:, h1:] = True
    fine[h1:, :] = True
    ll = np.zeros((n, n), bool)
    ll[: n >> L, : n >> L] = True
    assert np.all(counts[fine] == 1)
    assert np.all(counts[ll] == 3)
    assert np.all(counts[~fine & ~ll] == 5)
    # brute-force parent rule for a few coefficients
    for (c, p) in gr[:: max(1, len(gr) // 50)]:
        r, cc = divmod(int(c), n)
        pr, pc = divmod(int(p), n)
        lvl = next(l for l in range(1, L + 1) if max(r, cc) >= (n >> l))
        h = n >> lvl
        br, bc = r // h, cc // h
        if lvl < L:
            assert (pr // (h // 2), pc // (h // 2)) == (br, bc)
            assert (pr % (h // 2), pc % (h // 2)) == ((r % h) // 2, (cc % h) // 2)
        else:
            assert (pr, pc) == (r % h, cc % h)


def test_inverse_group_map_bruteforce():
    n, L = 8, 2
    gr = fs.tree_groups(n, L)
    off, ids = O.inverse_group_map(gr, n * n)
    for j in range(n * n):
        expect = [k for k in range(len(gr)) if j in gr[k]]
        assert list(ids[off[j]:off[j + 1]]) == expect


def test_tree_weights_dense():
    """Overlapping tree groups: diag(G^T W G) against the dense product."""
    n, L = 8, 2
    gr = fs.tree_groups(n, L)
    c = crandn(rng(9), n * n)
    G, sizes = O.group_matrix(gr, n * n)
    Wg = O.group_weights(c, G, sizes)
    for k in range(len(gr)):
        assert abs(Wg[k] - (np.sum(np.abs(c[gr[k]]) ** 2) + O.EPS) ** -0.5) < 1e-12 * Wg[k]
    Gd = G.toarray()
    assert np.allclose(O.gwg_diag(Wg, G, sizes), np.diag(Gd.T @ np.diag(np.repeat(Wg, 2)) @ Gd))


# ------------------------------------------------------------------ PCG ---

def _system(n, psi, real=False, groups=None, levels=2, ratio=0.3, seed=0, precond="paper"):
    mask = fs.vd_mask(n, ratio, seed)
    s = O.System(mask, real, psi, levels, 0.05, 0.02, groups, precond=precond)
    r = rng(seed + 10)
    x = r.standard_normal((n, n)) if real else crandn(r, n, n)
    s.update_weights(x)
    return s, mask


@pytest.mark.parametrize("precond", O.PRECONDS)
@pytest.mark.parametrize("psi", [O.PSI_HAAR, O.PSI_DB4, O.PSI_TV, O.PSI_TV | O.PSI_DB4, O.PSI_TV_ANISO])
def test_pcg_matches_dense_direct_solve(psi, precond):
    """PCG with the proposed P, with Jacobi and without a preconditioner (plain
    CG) reaches the dense direct solve of S x = rhs (S Hermitian positive
    definite, so PCG with any SPD P converges in at most 2N real dimensions)."""
    n = 8
    if precond == "ilu0" and not psi & O.PSI_ANY_TV:
        pytest.skip("ILU(0) factors the TV preconditioner")
    s, mask = _system(n, psi, precond=precond)
    Sd = dense_op(s.apply_S, n)
    assert np.allclose(Sd, Sd.conj().T, atol=1e-12)        # Hermitian
    rhs = crandn(rng(11), n, n)
    x_direct = np.linalg.solve(Sd, rhs.reshape(-1)).reshape(n, n)
    x, steps = O.pcg(s, rhs, np.zeros((n, n), complex), 4 * n * n, 1e-14, np.linalg.norm(rhs))
    assert np.linalg.norm(x - x_direct) <= 1e-9 * np.linalg.norm(x_direct)


@pytest.mark.parametrize("psi,groups", [(O.PSI_HAAR, None), (O.PSI_DB4, "tree"), (O.PSI_TV, None),
                                         (O.PSI_TV | O.PSI_DB4, None)])
def test_jacobi_preconditioner_is_the_dense_diagonal(psi, groups):
    """Jacobi PCG (Sec. 5.2) divides by diag(S); diag(S) equals the diagonal of
    the dense S built column by column from apply_S, for a real unknown too."""
    n = 8
    gr = fs.tree_groups(n, 2) if groups == "tree" else None
    for real in (False, True):
        if real and psi & O.PSI_TV:
            continue
        s, _ = _system(n, psi, real=real, groups=gr, precond="jacobi")
        Sd = dense_op(s.apply_S, n, dtype=float if real else complex)
        assert np.allclose(s.diag_S(), np.real(np.diag(Sd)), rtol=1e-12, atol=1e-12)
        r = crandn(rng(12), n, n)
        assert np.allclose(s.apply_Pinv(r), r / np.real(np.diag(Sd)).reshape(n, n), rtol=1e-12)
    s, _ = _system(n, psi, groups=gr, precond="none")
    r = crandn(rng(13), n, n)
    assert np.array_equal(s.apply_Pinv(r), r)


@pytest.mark.parametrize("tv", [O.PSI_TV, O.PSI_TV_ANISO])
def test_irls_system_is_the_gradient_of_F_eps(tv):
    """S(W(x)) x - A^H b equals the gradient of the eps-smoothed objective at
    x (central differences of F_eps alone): the weights of Eq. wi (or the l1
    weights of Eq. l1) and the assembly of S agree with the objective."""
    n = 6
    p = fs.make_problem(n, 0.4, 0.01, 11, real=False, psi=tv | O.PSI_HAAR, levels=1, lam=5e-3, lam_tv=1e-2)
    eps = 1e-4
    x = fs.complex_phantom(n, 3) + 0.05 * crandn(rng(14), n, n)
    s = O.System(p.mask, False, p.psi, p.levels, p.lam, p.lam_tv, None, eps)
    s.update_weights(x)
    g_irls = s.apply_S(x) - O.op_AH(p.b, p.mask.astype(float), False)
    F = lambda z: O.objective(z, p.b, p.mask, False, p.psi, p.levels, p.lam, p.lam_tv, None, eps)
    h = 1e-6
    for i in range(n * n):
        for e, part in ((1.0, "re"), (1j, "im")):
            zp, zm = x.copy().reshape(-1), x.copy().reshape(-1)
            zp[i] += h * e
            zm[i] -= h * e
            fd = (F(zp.reshape(n, n)) - F(zm.reshape(n, n))) / (2 * h)
            got = g_irls.reshape(-1)[i]
            got = got.real if part == "re" else got.imag
            assert abs(fd - got) < 1e-5 * (1 + abs(fd)), (i, part, fd, got)


@pytest.mark.parametrize("psi", [O.PSI_TV, O.PSI_TV_ANISO, O.PSI_TV | O.PSI_DB4, O.PSI_TV_ANISO | O.PSI_HAAR])
def test_ilu0_reproduces_P_on_its_pattern(psi):
    """ILU(0) (zero fill, updated pivots): L U equals P at every position of
    P's sparsity pattern, the diagonal included, and differs only at the
    fill positions; all pivots are positive (P is a diagonally dominant
    M-matrix).  The printed factors of Sec. 4.2 differ on the diagonal."""
    n = 6
    s, _ = _system(n, psi, levels=1, precond="ilu0")
    P = s.P.toarray()
    LU = (s.L @ s.U).toarray()
    pattern = P != 0
    assert np.allclose(LU[pattern], P[pattern], rtol=1e-12, atol=1e-14)
    assert np.all(s.U.diagonal() > 0)
    printed, _ = _system(n, psi, levels=1, precond="paper")
    LU_p = (printed.L @ printed.U).toarray()
    assert not np.allclose(np.diag(LU_p), np.diag(P), rtol=1e-9)


def test_S_is_gradient_of_quadratic_model():
    """S equals the Hessian of Q(x, W) (Eq. GWx / Gx) by finite differences."""
    n = 6
    s, mask = _system(n, O.PSI_TV | O.PSI_DB4, levels=1)
    Wd = s.Wtv

    def Q(x):
        xf = x.reshape(-1)
        val = 0.5 * np.sum(np.abs(O.op_A(x, mask)) ** 2)
        c = O.wavedec2(x, s.kind, s.levels).reshape(-1)
        val += 0.5 * s.lam * np.sum(s.w * np.abs(c) ** 2)
        val += 0.5 * s.lam_tv * np.sum(Wd * (np.abs(s.D1 @ xf) ** 2 + np.abs(s.D2 @ xf) ** 2))
        return val

    x = crandn(rng(12), n, n)
    d = crandn(rng(13), n, n)
    h = 1e-3
    # Q is quadratic: second difference is exact up to rounding
    curv = (Q(x + h * d) - 2 * Q(x) + Q(x - h * d)) / h ** 2
    assert abs(curv - np.real(np.vdot(d, s.apply_S(d)))) < 1e-6 * abs(curv)


def test_full_mask_wavelet_pcg_one_step():
    """Full mask: A^H A = I, so S = P exactly and PCG converges in one step."""
    n = 16
    mask = np.ones((n, n), np.uint8)
    s = O.System(mask, False, O.PSI_DB4, 2, 0.1, 0.0)
    s.update_weights(crandn(rng(14), n, n))
    rhs = crandn(rng(15), n, n)
    x, _ = O.pcg(s, rhs, np.zeros((n, n), complex), 1, 0.0, 1.0)
    assert np.linalg.norm(s.apply_S(x) - rhs) < 1e-12 * np.linalg.norm(rhs)


# ---------------------------------------------------------------- FIRLS ---

@pytest.mark.parametrize("inner", [1, 3, 20])
@pytest.mark.parametrize("which", ["haar_real", "tv_db4", "tree", "tv", "tv_l1", "tv_l1_db4_ilu0"])
def test_theorem2_monotone_decrease(which, inner):
    if which == "haar_real":
        p = fs.make_problem(32, 0.25, 0.01, 1, real=True, psi=O.PSI_HAAR, levels=3, lam=1e-3)
    elif which == "tv_db4":
        p = fs.make_problem(32, 0.2, 0.01, 2, real=False, psi=O.PSI_TV | O.PSI_DB4, levels=2, lam=5e-4, lam_tv=1e-3)
    elif which == "tree":
        p = fs.make_problem(32, 0.15, 0.005, 3, real=False, psi=O.PSI_DB4, levels=3, lam=2e-4, tree=True)
    elif which == "tv":
        p = fs.make_problem(32, 0.2, 0.01, 4, real=False, psi=O.PSI_TV, levels=0, lam=0.0, lam_tv=1e-3)
    elif which == "tv_l1":
        p = fs.make_problem(32, 0.2, 0.01, 4, real=False, psi=O.PSI_TV_ANISO, levels=0, lam=0.0, lam_tv=1e-3)
    else:
        p = fs.make_problem(32, 0.2, 0.01, 5, real=False, psi=O.PSI_TV_ANISO | O.PSI_DB4, levels=2, lam=5e-4,
                            lam_tv=1e-3)
    pre = "ilu0" if which == "tv_l1_db4_ilu0" else "paper"
    _, info = O.firls_problem(p, outer=8, inner=inner, record=True, precond=pre)
    F = info["F_eps"]
    for k in range(len(F) - 1):
        assert F[k + 1] <= F[k] * (1 + 1e-12), (k, F[k], F[k + 1])
    assert F[-1] < F[0]


def test_soft_threshold_special_case():
    """Full mask + Haar + singletons + real x separates in the wavelet domain.

    The minimiser of 1/2||x - y||^2 + lam sum sqrt(c^2 + eps) has, per
    coefficient, the root of c - v + lam c / sqrt(c^2 + eps) = 0 (v = Phi y);
    as eps -> 0 it is soft thresholding of v by lam.
    """
    n, lam = 16, 0.05
    r = rng(16)
    x0 = np.round(r.standard_normal((n, n)), 1)
    mask = np.ones((n, n), np.uint8)
    b = O.fft2u(x0) + 0.01 * crandn(r, n, n)
    x, info = O.firls(b, mask, real=True, psi=O.PSI_HAAR, levels=3, lam=lam, outer=300, inner=5)
    v = O.wavedec2(np.real(O.ifft2u(b)), O.PSI_HAAR, 3).reshape(-1)
    roots = np.empty_like(v)
    for i, vi in enumerate(v):           # 1-D bisection on a monotone function
        lo, hi = -abs(vi) - 1, abs(vi) + 1
        f = lambda c: c - vi + lam * c / math.sqrt(c * c + O.EPS)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) > 0:
                hi = mid
            else:
                lo = mid
        roots[i] = 0.5 * (lo + hi)
    c = O.wavedec2(x, O.PSI_HAAR, 3).reshape(-1)
    assert np.max(np.abs(c - roots)) < 1e-6
    soft = np.sign(v) * np.maximum(np.abs(v) - lam, 0)
    assert np.max(np.abs(c - soft)) < 10 * math.sqrt(O.EPS)


@pytest.mark.parametrize("tv", [O.PSI_TV, O.PSI_TV_ANISO])
def test_theorem3_stationarity_by_finite_differences(tv):
    """At convergence the gradient of F_eps vanishes (Thm 3), checked with
    central differences of the objective alone (forward operators only), for
    isotropic (Eq. iso) and l1 (Eq. l1) TV."""
    n = 6
    p = fs.make_problem(n, 0.4, 0.01, 7, real=False, psi=tv | O.PSI_DB4, levels=1, lam=5e-3, lam_tv=1e-2)
    # eps = 1e-6 keeps the objective's curvature scale (sqrt eps) well above
    # the difference step, so central differences are accurate
    eps = 1e-6
    x, _ = O.firls(p.b, p.mask, real=False, psi=p.psi, levels=p.levels, lam=p.lam, lam_tv=p.lam_tv,
                   outer=400, inner=40, eps=eps)
    F = lambda z: O.objective(z, p.b, p.mask, False, p.psi, p.levels, p.lam, p.lam_tv, None, eps)

    def grad(z):
        gr = np.zeros(2 * n * n)
        h = 1e-7
        for i in range(n * n):
            for part, e in enumerate((1.0, 1j)):
                zp = z.copy().reshape(-1)
                zm = z.copy().reshape(-1)
                zp[i] += h * e
                zm[i] -= h * e
                gr[2 * i + part] = (F(zp.reshape(n, n)) - F(zm.reshape(n, n))) / (2 * h)
        return gr

    g_star = grad(x)
    g_init = grad(O.op_AH(p.b, p.mask, False))
    assert np.linalg.norm(g_star) < 1e-5 * np.linalg.norm(g_init)


def test_objective_eps_bound():
    p = fs.make_problem(16, 0.3, 0.01, 8, real=False, psi=O.PSI_TV | O.PSI_DB4, levels=2, lam=1e-3, lam_tv=1e-3)
    x = O.op_AH(p.b, p.mask, False)
    F0 = O.objective(x, p.b, p.mask, False, p.psi, p.levels, p.lam, p.lam_tv)
    Fe = O.objective(x, p.b, p.mask, False, p.psi, p.levels, p.lam, p.lam_tv, None, O.EPS)
    s = 16 * 16
    assert 0 <= Fe - F0 <= (p.lam + p.lam_tv) * s * math.sqrt(O.EPS)


# ------------------------------------------------------------- generator ---

def test_mask_generator():
    n = 64
    m = fs.vd_mask(n, 0.25, 1)
    assert m.dtype == np.uint8 and m[0, 0] == 1
    assert int(m.sum()) == round(0.25 * n * n)
    k = np.arange(n)
    k = np.where(k >= n // 2, k - n, k)
    rad = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    assert m[rad < n / 8].mean() > 2 * m[rad > n / 4].mean()
    assert np.array_equal(m, fs.vd_mask(n, 0.25, 1))
