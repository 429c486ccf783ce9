"""FP64 CPU oracle for the FIRLS hot path (arXiv 1411.5057).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA library (no kernels, headers, tables or
helpers); the only thing both sides use is the seeded input generator
``firls_synth``, which holds none of the method's arithmetic.

Plain, slow and written to be checked against the paper by eye: every step
is the paper's formula with numpy/scipy library primitives (FFT, sparse
products, sparse triangular solves) and no blocking or fusion.

Problem (Eq. anapro / probogs / iso):
    min_x  1/2 ||A x - b||^2 + lam_W ||G Phi x||_{2,1} + lam_TV ||[D1 x, D2 x]||_{2,1}
with A = R F (R: sampling mask, F: unitary 2-D DFT), Phi an orthogonal
periodic wavelet (Haar or Daubechies-4, Mallat layout), G a group map
(rows of the identity) and D1/D2 first-order differences.

Readings where the paper is silent or garbled (each listed in the design
notes of the repository):
  * F is the unitary DFT, so mean(diag(A^H A)) equals the sampling ratio
    (Sec. 5.4 states the two are identical).
  * A real unknown uses A^T y = Re(F^H R^T y); a complex unknown uses the
    Hermitian adjoint and the real inner product Re <u, v>.
  * Group norms of complex coefficients use the complex modulus.
  * eps = 1e-10 is added to the squared norm (Eq. gw, Eq. wi).
  * Haar taps (1, 1)/sqrt 2; Daubechies-4 = the 4-tap, two-vanishing-moment
    orthogonal filter; periodic extension; a_k = sum_t h_t x_{2k+t},
    d_k = sum_t g_t x_{2k+t}, g_t = (-1)^t h_{K-1-t}; standard separable
    Mallat pyramid on the LL band; every coefficient (LL included) is
    regularised when groups are singletons.
  * D1 (offset 1) and D2 (offset n) act on the row-major image with zero
    extension: the printed -1 that would wrap across a row seam is dropped.
  * The TV preconditioner factors are the printed ones,
    L = I + L_P diag(a)^-1 and U = diag(a) + U_P (Sec. 4.2).
  * TV plus wavelet (both regularisers) sums both terms in S; P is the TV
    penta-diagonal P with a_i increased by lam_W diag(Phi^T W Phi)_i.
  * PCG restarts every outer step (d = z), warm-started at x^k; it stops
    when ||r|| / ||A^H b|| <= pcg_tol or after ``inner`` steps.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

EPS = 1e-10
PSI_HAAR, PSI_DB4, PSI_TV, PSI_TV_ANISO = 1, 2, 4, 8
PSI_ANY_TV = PSI_TV | PSI_TV_ANISO


# ---------------------------------------------------------------------------
# A = R F and its adjoint (Sec. 5.4: A = RF, R a selection of M rows of I)
# ---------------------------------------------------------------------------

def fft2u(x):
    """Unitary 2-D DFT F (library primitive)."""
    return np.fft.fft2(x, norm="ortho")


def ifft2u(y):
    """F^H, the inverse of the unitary 2-D DFT (library primitive)."""
    return np.fft.ifft2(y, norm="ortho")


def op_A(x, mask):
    """A x = R F x, kept on the full grid with zeros off the mask."""
    return mask * fft2u(x)


def op_AH(y, mask, real):
    """A^H y = F^H R^T y (real unknown: Re F^H R^T y)."""
    out = ifft2u(mask * y)
    return out.real if real else out


def a_bar(mask):
    """mean(diag(A^H A)) = M / N, the sampling ratio (Sec. 5.4, Eq. pog)."""
    return float(np.count_nonzero(mask)) / mask.size


# ---------------------------------------------------------------------------
# Phi: orthogonal periodic wavelet, direct convolution filter bank
# ---------------------------------------------------------------------------

def wavelet_filters(kind):
    """Lowpass h and highpass g of the orthogonal wavelet (Sec. 3.1: Phi)."""
    if kind == PSI_HAAR:
        h = np.array([1.0, 1.0]) / math.sqrt(2.0)
    elif kind == PSI_DB4:
        s3 = math.sqrt(3.0)
        h = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4.0 * math.sqrt(2.0))
    else:
        raise ValueError("unknown wavelet kind")
    K = len(h)
    g = np.array([(-1) ** t * h[K - 1 - t] for t in range(K)])
    return h, g


def dwt1(x, h, g, axis):
    """One periodic analysis level along ``axis``: returns (lowpass, highpass).

    a_k = sum_t h_t x_{(2k+t) mod m},  d_k = sum_t g_t x_{(2k+t) mod m}.
    """
    a = 0
    d = 0
    for t in range(len(h)):
        xs = np.take(np.roll(x, -t, axis=axis), np.arange(0, x.shape[axis], 2), axis=axis)
        a = a + h[t] * xs
        d = d + g[t] * xs
    return a, d


def idwt1(a, d, h, g, axis):
    """Inverse (= adjoint, Phi orthogonal) of ``dwt1`` along ``axis``.

    x_i = sum_k h_{i-2k} a_k + g_{i-2k} d_k  (indices mod m).
    """
    shape = list(a.shape)
    shape[axis] *= 2
    ua = np.zeros(shape, dtype=np.result_type(a, d))
    ud = np.zeros(shape, dtype=np.result_type(a, d))
    idx = [slice(None)] * len(shape)
    idx[axis] = slice(0, shape[axis], 2)
    ua[tuple(idx)] = a
    ud[tuple(idx)] = d
    x = 0
    for t in range(len(h)):
        x = x + h[t] * np.roll(ua, t, axis=axis) + g[t] * np.roll(ud, t, axis=axis)
    return x


def wavedec2(x, kind, levels):
    """Phi x: multi-level 2-D transform in Mallat layout (LL top-left)."""
    h, g = wavelet_filters(kind)
    c = np.array(x, dtype=np.complex128 if np.iscomplexobj(x) else np.float64, copy=True)
    n = c.shape[0]
    for l in range(levels):
        m = n >> l
        blk = c[:m, :m]
        lo, hi = dwt1(blk, h, g, axis=1)           # along each row
        row = np.concatenate([lo, hi], axis=1)
        lo, hi = dwt1(row, h, g, axis=0)           # along each column
        c[:m, :m] = np.concatenate([lo, hi], axis=0)
    return c


def waverec2(c, kind, levels):
    """Phi^T c = Phi^{-1} c (orthogonal)."""
    h, g = wavelet_filters(kind)
    x = np.array(c, copy=True)
    n = x.shape[0]
    for l in reversed(range(levels)):
        m = n >> l
        blk = x[:m, :m]
        half = m // 2
        col = idwt1(blk[:half, :], blk[half:, :], h, g, axis=0)
        x[:m, :m] = idwt1(col[:, :half], col[:, half:], h, g, axis=1)
    return x


def wavelet_kind(psi):
    if psi & PSI_HAAR:
        return PSI_HAAR
    if psi & PSI_DB4:
        return PSI_DB4
    return 0


# ---------------------------------------------------------------------------
# G and the group weights (Eq. gw, Eq. Wog; G^T W G is diagonal)
# ---------------------------------------------------------------------------

def group_matrix(groups, N):
    """G: N' x N binary matrix whose rows are rows of the identity (Fig. 1).

    ``groups`` is int32 [n_groups][g] (uniform size), a tuple
    (offsets [n_groups+1], members) for groups of varying size (Sec. 3.1:
    variant-size groups), or None for singletons.  Returns (G, sizes).
    """
    if groups is None:
        return sp.identity(N, format="csr"), np.ones(N, dtype=np.int64)
    if isinstance(groups, tuple):
        off, idx = (np.asarray(a) for a in groups)
        M = len(idx)
        G = sp.csr_matrix((np.ones(M), (np.arange(M), idx)), shape=(M, N))
        return G, np.diff(off).astype(np.int64)
    groups = np.asarray(groups)
    s, g = groups.shape
    rows = np.arange(s * g)
    G = sp.csr_matrix((np.ones(s * g), (rows, groups.reshape(-1))), shape=(s * g, N))
    return G, np.full(s, g, dtype=np.int64)


def group_weights(c_flat, G, sizes, eps=EPS):
    """W_{g_i} = (||(G Phi x)_{g_i}||^2 + eps)^(-1/2)  (Eq. gw)."""
    gc = G @ c_flat
    sq = np.abs(gc) ** 2
    ends = np.cumsum(sizes)
    norms2 = np.add.reduceat(sq, ends - sizes)
    return (norms2 + eps) ** -0.5


def duplicated_weights(Wg, sizes):
    """Diagonal of the N' x N' matrix W: each W_{g_i} repeated |g_i| times (Eq. Wog)."""
    return np.repeat(Wg, sizes)


def gwg_diag(Wg, G, sizes):
    """diag(G^T W G); G^T W G is diagonal for any G built from rows of I (Sec. 3.2)."""
    M = G.T @ sp.diags(duplicated_weights(Wg, sizes)) @ G
    return np.asarray(M.diagonal())


def group_l21(c_flat, G, sizes, eps=0.0):
    """sum_i sqrt(||(G c)_{g_i}||^2 + eps)  (Eq. l21; eps=0 gives the plain norm)."""
    sq = np.abs(G @ c_flat) ** 2
    ends = np.cumsum(sizes)
    return float(np.sum(np.sqrt(np.add.reduceat(sq, ends - sizes) + eps)))


# ---------------------------------------------------------------------------
# TV: D1, D2 (Sec. 4.1) as sparse matrices on the row-major image
# ---------------------------------------------------------------------------

def tv_matrices(n):
    """D1 (offset 1) and D2 (offset n): unit diagonal, -1 on the sub-diagonal.

    Zero extension: the entries of D1 that would couple the last pixel of a
    row with the first pixel of the next row are removed.
    """
    N = n * n
    sub1 = -np.ones(N - 1)
    sub1[np.arange(1, N) % n == 0] = 0.0       # row seams
    D1 = sp.diags([np.ones(N), sub1], [0, -1], format="csr")
    D2 = sp.diags([np.ones(N), -np.ones(N - n)], [0, -n], format="csr")
    return D1, D2


def tv_weights(x_flat, D1, D2, eps=EPS):
    """W_i = 1 / sqrt((grad_1 x_i)^2 + (grad_2 x_i)^2 + eps)  (Eq. wi)."""
    g1 = D1 @ x_flat
    g2 = D2 @ x_flat
    return (np.abs(g1) ** 2 + np.abs(g2) ** 2 + eps) ** -0.5


def tv_iso(x_flat, D1, D2, eps=0.0):
    """||[D1 x, D2 x]||_{2,1} (Eq. iso), eps-smoothed when eps > 0."""
    g1 = D1 @ x_flat
    g2 = D2 @ x_flat
    return float(np.sum(np.sqrt(np.abs(g1) ** 2 + np.abs(g2) ** 2 + eps)))


def tv_weights_aniso(x_flat, D1, D2, eps=EPS):
    """l1 TV (Eq. l1): every entry of D1 x and of D2 x is its own group, so
    W1_i = (|(D1 x)_i|^2 + eps)^(-1/2) and W2_i = (|(D2 x)_i|^2 + eps)^(-1/2)
    (Sec. 4.1: the l1 form follows the isotropic derivation)."""
    return (np.abs(D1 @ x_flat) ** 2 + eps) ** -0.5, (np.abs(D2 @ x_flat) ** 2 + eps) ** -0.5


def tv_l1(x_flat, D1, D2, eps=0.0):
    """||D1 x||_1 + ||D2 x||_1 (Eq. l1), eps-smoothed when eps > 0."""
    return float(np.sum(np.sqrt(np.abs(D1 @ x_flat) ** 2 + eps)) + np.sum(np.sqrt(np.abs(D2 @ x_flat) ** 2 + eps)))


def ilu0_pivots(P, n):
    """Pivots d of the incomplete LU factorisation with zero fill, ILU(0), of
    the penta-diagonal P (offsets 1 and n): d_i = a_i - sum over the lower
    neighbours j in {i-1, i-n} of P_ij^2 / d_j, so that L U equals P on P's
    sparsity pattern with L = I + L_P diag(d)^-1, U = diag(d) + U_P."""
    P = sp.csr_matrix(P)
    N = P.shape[0]
    d = np.zeros(N)
    for i in range(N):
        di = P[i, i]
        for j in (i - 1, i - n):
            if j >= 0:
                pij = P[i, j]
                if pij != 0.0:
                    di -= pij * pij / d[j]
        d[i] = di
    return d


# ---------------------------------------------------------------------------
# diag(Phi^T W Phi) for the combined preconditioner (exact diagonal)
# ---------------------------------------------------------------------------

def _analysis_matrices_1d(n, kind, levels):
    """Rows of the 1-D level-l scaling functions S_l and wavelets V_l (periodic).

    S_0 = I_n; S_l = H_l S_{l-1}; V_l = G_l S_{l-1}, with H_l, G_l the
    one-level periodic analysis matrices on length n / 2^(l-1).
    """
    h, g = wavelet_filters(kind)
    S = [np.eye(n)]
    V = [None]
    for l in range(1, levels + 1):
        m = n >> (l - 1)
        Hm, Gm = dwt1(np.eye(m), h, g, axis=0)   # columns = responses to unit impulses
        S.append(Hm @ S[-1])
        V.append(Gm @ S[-2])
    return S, V


def wavelet_diag(w, n, kind, levels):
    """diag(Phi^T diag(w) Phi)_i = sum_j w_j Phi_{j,i}^2 for a Mallat array w.

    Each 2-D basis function of the separable pyramid is an outer product of
    1-D level-l functions, so the sum splits per subband into
    (X_l^2)^T w_band (Y_l^2) with X, Y in {S_l, V_l}.
    """
    S, V = _analysis_matrices_1d(n, kind, levels)
    w = np.asarray(w, dtype=np.float64).reshape(n, n)
    out = np.zeros((n, n))
    for l in range(1, levels + 1):
        h = n >> l
        for (br, bc) in ((0, 1), (1, 0), (1, 1)):
            R = (S[l] if br == 0 else V[l]) ** 2
            C = (S[l] if bc == 0 else V[l]) ** 2
            out += R.T @ w[br * h:(br + 1) * h, bc * h:(bc + 1) * h] @ C
    h = n >> levels
    out += (S[levels] ** 2).T @ w[:h, :h] @ (S[levels] ** 2)
    return out


# ---------------------------------------------------------------------------
# The system S and the preconditioners
# ---------------------------------------------------------------------------

PRECONDS = ("paper", "jacobi", "none", "ilu0")


class System:
    """S = A^H A + lam_W Phi^T G^T W G Phi + lam_TV (D1^T W D1 + D2^T W D2)
    (Eq. subprob, Eq. sub) and its preconditioner P.

    ``precond`` selects P for the comparison of Sec. 5.2 (Fig. 2 and the TV
    figure): "paper" is the proposed P (Eq. pog, Eq. ptv with the printed L
    U factors), "jacobi" is P = diag(S) (conventional Jacobi PCG), "none" is
    P = I (standard CG), "ilu0" (TV only) factors the penta-diagonal P of
    Eq. ptv by ILU(0) with updated pivots instead of the printed factors.
    ``psi`` may hold PSI_TV (isotropic, Eq. iso) or PSI_TV_ANISO (l1, Eq. l1).
    """

    def __init__(self, mask, real, psi, levels, lam, lam_tv, groups=None, eps=EPS, precond="paper"):
        if precond not in PRECONDS:
            raise ValueError("unknown preconditioner")
        if precond == "ilu0" and not (psi & PSI_ANY_TV):
            raise ValueError("ILU(0) factors the TV preconditioner")
        self.precond = precond
        self.eps = float(eps)
        self.mask = np.asarray(mask).astype(np.float64)
        self.n = self.mask.shape[0]
        self.N = self.n * self.n
        self.real = bool(real)
        self.psi = int(psi)
        self.kind = wavelet_kind(psi)
        self.levels = int(levels)
        self.lam = float(lam)
        self.tv = bool(psi & PSI_ANY_TV)
        self.aniso = bool(psi & PSI_TV_ANISO)
        self.lam_tv = float(lam_tv) if self.tv else 0.0
        self.abar = a_bar(mask)
        self.G, self.sizes = group_matrix(groups, self.N)
        if self.tv:
            self.D1, self.D2 = tv_matrices(self.n)
        self.w = None        # diag(G^T W G) (wavelet part)
        self.Wtv = None      # TV weights (isotropic); W1, W2 below for both forms
        self.W1 = self.W2 = None
        self.L = self.U = None
        self.pinv = None

    # -- weights (Alg. 2 / Alg. 3: "Update W^k") --
    def update_weights(self, x):
        xf = x.reshape(-1)
        if self.kind:
            c = wavedec2(x, self.kind, self.levels).reshape(-1)
            Wg = group_weights(c, self.G, self.sizes, self.eps)
            self.w = gwg_diag(Wg, self.G, self.sizes)
        if self.aniso:
            self.W1, self.W2 = tv_weights_aniso(xf, self.D1, self.D2, self.eps)
        elif self.tv:
            self.Wtv = tv_weights(xf, self.D1, self.D2, self.eps)
            self.W1 = self.W2 = self.Wtv
        self._build_preconditioner()

    def tv_term(self):
        """D1^T W1 D1 + D2^T W2 D2 (W1 = W2 = W for isotropic TV, Eq. sub)."""
        return self.D1.T @ sp.diags(self.W1) @ self.D1 + self.D2.T @ sp.diags(self.W2) @ self.D2

    def diag_S(self):
        """diag(S): abar (every diagonal entry of A^H A, Sec. 5.4) plus
        lam_W diag(Phi^T W Phi) plus lam_TV diag(D1^T W D1 + D2^T W D2)."""
        d = np.full(self.N, self.abar)
        if self.kind:
            d = d + self.lam * wavelet_diag(self.w, self.n, self.kind, self.levels).reshape(-1)
        if self.tv:
            d = d + self.lam_tv * self.tv_term().diagonal()
        return d

    def _build_preconditioner(self):
        if self.precond == "jacobi":
            self.jacobi = 1.0 / self.diag_S()
            return
        if self.precond == "none":
            return
        if self.tv:
            # P = abar I + lam (D1^T W D1 + D2^T W D2)  (Eq. ptv), penta-diagonal
            P = self.abar * sp.identity(self.N) + self.lam_tv * self.tv_term()
            P = sp.csr_matrix(P)
            if self.kind:
                P = P + sp.diags(self.lam * wavelet_diag(self.w, self.n, self.kind, self.levels).reshape(-1))
            self.P = sp.csr_matrix(P)
            # printed factors: L = I + L_P diag(a)^-1, U = diag(a) + U_P with
            # a = diag(P); ILU(0) uses the updated pivots instead of a
            a = ilu0_pivots(self.P, self.n) if self.precond == "ilu0" else self.P.diagonal()
            LP = sp.tril(self.P, -1)
            UP = sp.triu(self.P, 1)
            self.L = sp.csr_matrix(sp.identity(self.N) + LP @ sp.diags(1.0 / a))
            self.U = sp.csr_matrix(sp.diags(a) + UP)
        else:
            # P^-1 = Phi^T (abar I + lam G^T W G)^-1 Phi  (Eq. pog and below)
            self.pinv = 1.0 / (self.abar + self.lam * self.w)

    # -- operators --
    def AHA(self, x):
        return op_AH(op_A(x, self.mask), self.mask, self.real)

    def apply_S(self, x):
        out = self.AHA(x)
        if self.kind:
            c = wavedec2(x, self.kind, self.levels)
            out = out + self.lam * waverec2(self.w.reshape(self.n, self.n) * c, self.kind, self.levels)
        if self.tv:
            xf = x.reshape(-1)
            t = self.D1.T @ (self.W1 * (self.D1 @ xf)) + self.D2.T @ (self.W2 * (self.D2 @ xf))
            out = out + self.lam_tv * t.reshape(self.n, self.n)
        return out

    def apply_Pinv(self, r):
        if self.precond == "jacobi":
            return (self.jacobi * np.asarray(r).reshape(-1)).reshape(self.n, self.n)
        if self.precond == "none":
            return np.array(r, copy=True)
        if self.tv:
            rf = r.reshape(-1)
            y = spl.spsolve_triangular(self.L, rf, lower=True)
            z = spl.spsolve_triangular(self.U, y, lower=False)
            return z.reshape(self.n, self.n)
        c = wavedec2(r, self.kind, self.levels)
        return waverec2(self.pinv.reshape(self.n, self.n) * c, self.kind, self.levels)


def rdot(u, v):
    """Real inner product Re <u, v> on R^N or C^N (= R^{2N})."""
    return float(np.real(np.vdot(u, v)))


def pcg(system, rhs, x, inner, tol, rhs_norm):
    """Preconditioned CG on S x = rhs from the warm start x (Saad, Alg. 9.1).

    Returns (x, steps).  Stops when ||r|| / ||rhs|| <= tol or after ``inner``
    steps.
    """
    x = x.copy()
    r = rhs - system.apply_S(x)
    z = system.apply_Pinv(r)
    d = z.copy()
    rho = rdot(r, z)
    steps = 0
    for j in range(inner):
        q = system.apply_S(d)
        alpha = rho / rdot(d, q)
        x = x + alpha * d
        r = r - alpha * q
        steps += 1
        if tol > 0 and math.sqrt(rdot(r, r)) <= tol * rhs_norm:
            break
        if j == inner - 1:
            break
        z = system.apply_Pinv(r)
        rho_new = rdot(r, z)
        beta = rho_new / rho
        d = z + beta * d
        rho = rho_new
    return x, steps


def objective(x, b, mask, real, psi, levels, lam, lam_tv, groups=None, eps=0.0):
    """F(x) (eps = 0, Eq. anapro / iso) or its smoothed form F_eps (eps > 0)."""
    mask = np.asarray(mask).astype(np.float64)
    n = mask.shape[0]
    N = n * n
    res = op_A(x, mask) - mask * b
    val = 0.5 * float(np.sum(np.abs(res) ** 2))
    kind = wavelet_kind(psi)
    if kind:
        G, sizes = group_matrix(groups, N)
        c = wavedec2(x, kind, levels).reshape(-1)
        val += lam * group_l21(c, G, sizes, eps)
    if psi & PSI_TV_ANISO:
        D1, D2 = tv_matrices(n)
        val += lam_tv * tv_l1(np.asarray(x).reshape(-1), D1, D2, eps)
    elif psi & PSI_TV:
        D1, D2 = tv_matrices(n)
        val += lam_tv * tv_iso(np.asarray(x).reshape(-1), D1, D2, eps)
    return val


def firls(b, mask, *, real, psi, levels, lam, lam_tv=0.0, groups=None, outer=50, inner=20,
          pcg_tol=0.0, outer_tol=0.0, x_init=None, record=False, eps=EPS, precond="paper"):
    """FIRLS outer loop (Alg. 2 FIRLS_OG / Alg. 3 FIRLS_TV).

    x^1 = A^H b unless ``x_init`` is given (Sec. 3.3: x^0 = A^T b).  Each outer
    step updates W^k from x^k, rebuilds P and runs PCG on S x = A^H b
    warm-started at x^k.  Returns (x, info) with per-step history.
    """
    mask = np.asarray(mask)
    system = System(mask, real, psi, levels, lam, lam_tv, groups, eps, precond)
    rhs = op_AH(mask * b, mask.astype(np.float64), real)
    rhs_norm = math.sqrt(rdot(rhs, rhs))
    x = rhs.copy() if x_init is None else np.array(x_init, copy=True)
    info = dict(pcg_steps=[], rel_change=[], F_eps=[], outer_done=0)
    if record:
        info["F_eps"].append(objective(x, b, mask, real, psi, levels, lam, lam_tv, groups, eps))
    for k in range(outer):
        system.update_weights(x)
        x_new, steps = pcg(system, rhs, x, inner, pcg_tol, rhs_norm)
        dx = x_new - x
        nx = math.sqrt(rdot(x, x))
        rel = math.sqrt(rdot(dx, dx)) / nx if nx > 0 else float("inf")
        x = x_new
        info["pcg_steps"].append(steps)
        info["rel_change"].append(rel)
        info["outer_done"] = k + 1
        if record:
            info["F_eps"].append(objective(x, b, mask, real, psi, levels, lam, lam_tv, groups, eps))
        if outer_tol > 0 and rel <= outer_tol:
            break
    return x, info


def firls_problem(p, outer=50, inner=20, pcg_tol=0.0, outer_tol=0.0, x_init=None, record=False, precond="paper"):
    """Convenience wrapper over a ``firls_synth.Problem``."""
    return firls(p.b, p.mask, real=p.real, psi=p.psi, levels=p.levels, lam=p.lam,
                 lam_tv=p.lam_tv, groups=p.groups, outer=outer, inner=inner,
                 pcg_tol=pcg_tol, outer_tol=outer_tol, x_init=x_init, record=record, precond=precond)


def inverse_group_map(groups, N):
    """Coefficient -> groups map (CSR): offsets [N+1] and group ids, ascending.

    The integer structure the library derives from G at set-up; compared bit
    for bit.  ``groups`` as in ``group_matrix``.
    """
    if isinstance(groups, tuple):
        off, coef = (np.asarray(a) for a in groups)
        gid = np.repeat(np.arange(len(off) - 1), np.diff(off))
    else:
        groups = np.asarray(groups)
        s, g = groups.shape
        coef = groups.reshape(-1)
        gid = np.repeat(np.arange(s), g)
    order = np.lexsort((gid, coef))
    counts = np.bincount(coef, minlength=N)
    off = np.zeros(N + 1, dtype=np.int32)
    off[1:] = np.cumsum(counts)
    return off, gid[order].astype(np.int32)


# ---------------------------------------------------------------------------
# Multi-contrast reconstruction (Sec. 5.6: FIRLS_MT, FIRLS_JTV)
# ---------------------------------------------------------------------------

class JointSystem:
    """T contrasts x_1..x_T of one cross section, each with its own sampling
    mask, sharing the regulariser's weights (Sec. 5.6):

    * wavelet joint sparsity (FIRLS_MT): the group of coefficient j holds
      (Phi x_t)_j of every contrast, W_j = (sum_t |(Phi x_t)_j|^2 + eps)^(-1/2)
      (Eq. gw with non-overlapping groups across contrasts);
    * joint TV (FIRLS_JTV): W_i = (sum_t |grad_1 x_t,i|^2 + |grad_2 x_t,i|^2
      + eps)^(-1/2) (Eq. wi summed over contrasts).

    Given W the system is block diagonal: S = blockdiag_t(A_t^H A_t + lam
    Phi^T W Phi + lam_TV (D1^T W D1 + D2^T W D2)), and so is P (each block
    the single-contrast P of Eq. pog / Eq. ptv with that contrast's abar).
    PCG runs on the stacked system (one alpha, beta, rho for all contrasts),
    as Alg. 2 / Alg. 3 on the stacked unknown.
    """

    def __init__(self, masks, psi, levels, lam, lam_tv, eps=EPS):
        self.T = len(masks)
        self.eps = float(eps)
        self.psi = int(psi)
        self.kind = wavelet_kind(psi)
        self.tv = bool(psi & PSI_TV)
        if psi & PSI_TV_ANISO:
            raise ValueError("joint TV is the isotropic form")
        self.levels = int(levels)
        self.lam = float(lam)
        self.lam_tv = float(lam_tv) if self.tv else 0.0
        self.parts = [System(m, False, psi, levels, lam, lam_tv, None, eps) for m in masks]

    def update_weights(self, xs):
        if self.kind:
            sq = sum(np.abs(wavedec2(x, self.kind, self.levels).reshape(-1)) ** 2 for x in xs)
            w = (sq + self.eps) ** -0.5
            for p in self.parts:
                p.w = w
        if self.tv:
            D1, D2 = self.parts[0].D1, self.parts[0].D2
            sq = sum(np.abs(D1 @ x.reshape(-1)) ** 2 + np.abs(D2 @ x.reshape(-1)) ** 2 for x in xs)
            W = (sq + self.eps) ** -0.5
            for p in self.parts:
                p.Wtv = W
                p.W1 = p.W2 = W
        for p in self.parts:
            p._build_preconditioner()

    def apply_S(self, xs):
        return [p.apply_S(x) for p, x in zip(self.parts, xs)]

    def apply_Pinv(self, rs):
        return [p.apply_Pinv(r) for p, r in zip(self.parts, rs)]


def rdot_joint(us, vs):
    """Real inner product of stacked contrasts: sum_t Re <u_t, v_t>."""
    return sum(rdot(u, v) for u, v in zip(us, vs))


def pcg_joint(system, rhs, xs, inner, tol, rhs_norm):
    """PCG (Saad, Alg. 9.1) on the stacked block system from the warm start xs."""
    xs = [x.copy() for x in xs]
    r = [b - s for b, s in zip(rhs, system.apply_S(xs))]
    z = system.apply_Pinv(r)
    d = [v.copy() for v in z]
    rho = rdot_joint(r, z)
    steps = 0
    for j in range(inner):
        q = system.apply_S(d)
        alpha = rho / rdot_joint(d, q)
        xs = [x + alpha * v for x, v in zip(xs, d)]
        r = [a - alpha * v for a, v in zip(r, q)]
        steps += 1
        if tol > 0 and math.sqrt(rdot_joint(r, r)) <= tol * rhs_norm:
            break
        if j == inner - 1:
            break
        z = system.apply_Pinv(r)
        rho_new = rdot_joint(r, z)
        beta = rho_new / rho
        d = [a + beta * v for a, v in zip(z, d)]
        rho = rho_new
    return xs, steps


def objective_joint(xs, bs, masks, psi, levels, lam, lam_tv, eps=0.0):
    """sum_t 1/2 ||A_t x_t - b_t||^2 + lam sum_j sqrt(sum_t |(Phi x_t)_j|^2 + eps)
    + lam_TV sum_i sqrt(sum_t |grad x_t,i|^2 + eps)."""
    val = 0.0
    for x, b, m in zip(xs, bs, masks):
        m = np.asarray(m).astype(np.float64)
        val += 0.5 * float(np.sum(np.abs(op_A(x, m) - m * b) ** 2))
    kind = wavelet_kind(psi)
    if kind:
        sq = sum(np.abs(wavedec2(x, kind, levels)) ** 2 for x in xs)
        val += lam * float(np.sum(np.sqrt(sq + eps)))
    if psi & PSI_TV:
        n = np.asarray(masks[0]).shape[0]
        D1, D2 = tv_matrices(n)
        sq = sum(np.abs(D1 @ np.asarray(x).reshape(-1)) ** 2 + np.abs(D2 @ np.asarray(x).reshape(-1)) ** 2 for x in xs)
        val += lam_tv * float(np.sum(np.sqrt(sq + eps)))
    return val


def firls_joint(bs, masks, *, psi, levels, lam, lam_tv=0.0, outer=50, inner=20, pcg_tol=0.0, outer_tol=0.0,
                x_init=None, record=False, eps=EPS):
    """FIRLS_MT / FIRLS_JTV (Sec. 5.6): Alg. 2 / Alg. 3 on the stacked
    contrasts with joint weights.  Returns (list of x_t, info)."""
    system = JointSystem(masks, psi, levels, lam, lam_tv, eps)
    rhs = [op_AH(np.asarray(m) * b, np.asarray(m).astype(np.float64), False) for b, m in zip(bs, masks)]
    rhs_norm = math.sqrt(rdot_joint(rhs, rhs))
    xs = [r.copy() for r in rhs] if x_init is None else [np.array(x, copy=True) for x in x_init]
    info = dict(pcg_steps=[], rel_change=[], F_eps=[], outer_done=0)
    if record:
        info["F_eps"].append(objective_joint(xs, bs, masks, psi, levels, lam, lam_tv, eps))
    for k in range(outer):
        system.update_weights(xs)
        x_new, steps = pcg_joint(system, rhs, xs, inner, pcg_tol, rhs_norm)
        dx = [a - b for a, b in zip(x_new, xs)]
        nx = math.sqrt(rdot_joint(xs, xs))
        rel = math.sqrt(rdot_joint(dx, dx)) / nx if nx > 0 else float("inf")
        xs = x_new
        info["pcg_steps"].append(steps)
        info["rel_change"].append(rel)
        info["outer_done"] = k + 1
        if record:
            info["F_eps"].append(objective_joint(xs, bs, masks, psi, levels, lam, lam_tv, eps))
        if outer_tol > 0 and rel <= outer_tol:
            break
    return xs, info
