"""Planted mistakes in the oracle, on the CPU.

Each case puts one plausible slip into one oracle function (a dropped term or
factor, a wrong sign, index, offset or band, a transposed or swapped
operand) and then runs the pins named beside it, which are the tests of
test_oracle.py, test_oracle_joint.py, test_oracle_dense.py and
test_cnn_oracle.py called directly.  At least one of them must fail: a pin
set that let the slip through would not be pinning that part of the oracle.
Where a slip keeps an invariant (a consistent band swap or a recursion on the
wrong quadrant keeps Phi orthogonal), the case names the invariant's pin as
well and checks that it alone would not have caught the slip.  Nothing of the
CUDA library is involved.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import test_cnn_oracle as TC
import test_oracle as TO
import test_oracle_dense as TD
import test_oracle_joint as TJ
from oracle import cnn_oracle as C
from oracle import dense_oracle as D
from oracle import firls_oracle as O

_orig_System = {name: getattr(O.System, name) for name in ("apply_S", "apply_Pinv", "_build_preconditioner")}


def _fails(pin):
    try:
        pin()
    except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError, ZeroDivisionError):
        return True
    return False


# ------------------------------------------------------------------ mutants --

def _wavelet_pair(block_of, permute):
    """A consistent analysis / synthesis pair with the level-l working block
    chosen by ``block_of(n, m)`` (its top-left corner) and each level's four
    bands rearranged by ``permute`` (and back on synthesis): Phi stays
    orthogonal and Phi^T stays its transpose."""
    def dec(x, kind, levels):
        h, g = O.wavelet_filters(kind)
        c = np.array(x, dtype=np.complex128 if np.iscomplexobj(x) else np.float64, copy=True)
        n = c.shape[0]
        for l in range(levels):
            m = n >> l
            o = block_of(n, m)
            blk = c[o:o + m, o:o + m]
            lo, hi = O.dwt1(blk, h, g, axis=1)
            row = np.concatenate([lo, hi], axis=1)
            lo, hi = O.dwt1(row, h, g, axis=0)
            c[o:o + m, o:o + m] = permute(np.concatenate([lo, hi], axis=0), False)
        return c

    def rec(c, kind, levels):
        h, g = O.wavelet_filters(kind)
        x = np.array(c, copy=True)
        n = x.shape[0]
        for l in reversed(range(levels)):
            m = n >> l
            o = block_of(n, m)
            blk = permute(x[o:o + m, o:o + m], True)
            half = m // 2
            col = O.idwt1(blk[:half, :], blk[half:, :], h, g, axis=0)
            x[o:o + m, o:o + m] = O.idwt1(col[:, :half], col[:, half:], h, g, axis=1)
        return x

    return dec, rec


def _swap_details(b, inverse):
    """Horizontal and vertical details in each other's quadrant."""
    b = b.copy()
    h = b.shape[0] // 2
    tr, bl = b[:h, h:].copy(), b[h:, :h].copy()
    b[:h, h:], b[h:, :h] = bl, tr
    return b


def _identity(b, inverse):
    return b


def _mut_pcg(slip):
    """PCG (the oracle's iteration) with one slip: 'beta' inverts rho_new / rho,
    'resid' adds alpha q to the residual, 'xr' steps x along r instead of d."""
    def pcg(system, rhs, x, inner, tol, rhs_norm):
        x = x.copy()
        r = rhs - system.apply_S(x)
        z = system.apply_Pinv(r)
        d = z.copy()
        rho = O.rdot(r, z)
        steps = 0
        for j in range(inner):
            q = system.apply_S(d)
            alpha = rho / O.rdot(d, q)
            x = x + alpha * (r if slip == "xr" else d)
            r = r + alpha * q if slip == "resid" else r - alpha * q
            steps += 1
            if tol > 0 and math.sqrt(O.rdot(r, r)) <= tol * rhs_norm:
                break
            if j == inner - 1:
                break
            z = system.apply_Pinv(r)
            rho_new = O.rdot(r, z)
            beta = rho / rho_new if slip == "beta" else rho_new / rho
            d = z + beta * d
            rho = rho_new
        return x, steps
    return pcg


def _apply_S_mut(slip):
    """S d with one slip: 'lam' drops lam from the wavelet term, 'tvsign'
    subtracts the TV term."""
    def apply_S(self, x):
        out = self.AHA(x)
        if self.kind:
            c = O.wavedec2(x, self.kind, self.levels)
            lam = 1.0 if slip == "lam" else self.lam
            out = out + lam * O.waverec2(self.w.reshape(self.n, self.n) * c, self.kind, self.levels)
        if self.tv:
            xf = x.reshape(-1)
            t = self.D1.T @ (self.W1 * (self.D1 @ xf)) + self.D2.T @ (self.W2 * (self.D2 @ xf))
            sgn = -1.0 if slip == "tvsign" else 1.0
            out = out + sgn * self.lam_tv * t.reshape(self.n, self.n)
        return out
    return apply_S


def _pinv_swapped(self, r):
    """Wavelet P^-1 with analysis and synthesis exchanged: Phi pinv Phi^T."""
    if self.precond != "paper" or self.tv:
        return _orig_System["apply_Pinv"](self, r)
    c = O.waverec2(r, self.kind, self.levels)
    return O.wavedec2(self.pinv.reshape(self.n, self.n) * c, self.kind, self.levels)


def _precond_mut(slip):
    """The preconditioner with one slip: 'nolam' leaves lam out of the wavelet
    pinv, 'printedL' forms L = I + L_P (without diag(a)^-1)."""
    def build(self):
        _orig_System["_build_preconditioner"](self)
        if slip == "nolam" and self.pinv is not None:
            self.pinv = 1.0 / (self.abar + self.w)
        if slip == "printedL" and self.L is not None:
            self.L = sp.csr_matrix(sp.identity(self.N) + sp.tril(self.P, -1))
    return build


def _objective_mut(slip):
    """F with one slip: 'half' drops the 1/2 of the data term, 'tvl1' evaluates
    isotropic TV as the l1 form."""
    def objective(x, b, mask, real, psi, levels, lam, lam_tv, groups=None, eps=0.0):
        mask = np.asarray(mask).astype(np.float64)
        n = mask.shape[0]
        res = O.op_A(x, mask) - mask * b
        val = (1.0 if slip == "half" else 0.5) * float(np.sum(np.abs(res) ** 2))
        kind = O.wavelet_kind(psi)
        if kind:
            G, sizes = O.group_matrix(groups, n * n)
            val += lam * O.group_l21(O.wavedec2(x, kind, levels).reshape(-1), G, sizes, eps)
        D1, D2 = O.tv_matrices(n)
        xf = np.asarray(x).reshape(-1)
        if psi & O.PSI_TV_ANISO or (psi & O.PSI_TV and slip == "tvl1"):
            val += lam_tv * O.tv_l1(xf, D1, D2, eps)
        elif psi & O.PSI_TV:
            val += lam_tv * O.tv_iso(xf, D1, D2, eps)
        return val
    return objective


def _tv_matrices_mut(slip):
    """D1, D2 with one slip: 'seam' keeps the -1 across row seams, 'offset'
    puts D2's -1 at offset n - 1."""
    def tv_matrices(n):
        N = n * n
        sub1 = -np.ones(N - 1)
        if slip != "seam":
            sub1[np.arange(1, N) % n == 0] = 0.0
        D1 = sp.diags([np.ones(N), sub1], [0, -1], format="csr")
        k = n - 1 if slip == "offset" else n
        D2 = sp.diags([np.ones(N), -np.ones(N - k)], [0, -k], format="csr")
        return D1, D2
    return tv_matrices


def _gwg_first_only(Wg, G, sizes):
    """diag(G^T W G) keeping one group per coefficient (overlaps dropped)."""
    out = np.zeros(G.shape[1])
    out[G.indices] = O.duplicated_weights(Wg, sizes)
    return out


def _ilu0_plus(P, n):
    P = sp.csr_matrix(P)
    d = np.zeros(P.shape[0])
    for i in range(P.shape[0]):
        di = P[i, i]
        for j in (i - 1, i - n):
            if j >= 0 and P[i, j] != 0.0:
                di += P[i, j] ** 2 / d[j]
        d[i] = di
    return d


def _wavelet_diag_swapped(w, n, kind, levels):
    """diag(Phi^T W Phi) with the row and column functionals of the mixed
    bands exchanged."""
    S, V = O._analysis_matrices_1d(n, kind, levels)
    w = np.asarray(w, dtype=np.float64).reshape(n, n)
    out = np.zeros((n, n))
    for l in range(1, levels + 1):
        h = n >> l
        for (br, bc) in ((0, 1), (1, 0), (1, 1)):
            R = (S[l] if bc == 0 else V[l]) ** 2
            Cm = (S[l] if br == 0 else V[l]) ** 2
            out += R.T @ w[br * h:(br + 1) * h, bc * h:(bc + 1) * h] @ Cm
    h = n >> levels
    out += (S[levels] ** 2).T @ w[:h, :h] @ (S[levels] ** 2)
    return out


def _joint_weights_per_contrast(self, xs):
    """Each contrast weighted by its own coefficients (no sum over contrasts)."""
    for p, x in zip(self.parts, xs):
        p.update_weights(x)


def _conv_flipped(a, w, b):
    return _orig_conv(a, w[::-1, ::-1], b)


_orig_conv = C.conv3x3


def _conv_backward_unflipped(a, w, dz):
    """da formed with the kernel's taps at the forward positions (the
    correlation's adjoint needs them mirrored)."""
    da, dw, db = _orig_conv_bwd(a, w, dz)
    B, H, W, _ = a.shape
    dzp = np.pad(dz, ((0, 0), (1, 1), (1, 1), (0, 0)))
    da2 = np.zeros_like(a, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            da2 += np.einsum("bhwo,io->bhwi", dzp[:, ky:ky + H, kx:kx + W, :], w[ky, kx])
    return da2, dw, db


_orig_conv_bwd = C.conv3x3_backward


def _idwt1_shift(a, d, h, g, axis):
    """Synthesis with the taps rolled the wrong way (not the adjoint)."""
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
        x = x + h[t] * np.roll(ua, -t, axis=axis) + g[t] * np.roll(ud, -t, axis=axis)
    return x


def _inverse_map_descending(groups, N):
    """Coefficient -> groups map with each coefficient's groups in descending order."""
    groups = np.asarray(groups)
    s, g = groups.shape
    coef = groups.reshape(-1)
    gid = np.repeat(np.arange(s), g)
    order = np.lexsort((-gid, coef))
    off = np.zeros(N + 1, dtype=np.int32)
    off[1:] = np.cumsum(np.bincount(coef, minlength=N))
    return off, gid[order].astype(np.int32)


def _wavelet_diag_no_LL(w, n, kind, levels):
    """diag(Phi^T W Phi) without the coarsest scaling band."""
    S, V = O._analysis_matrices_1d(n, kind, levels)
    w = np.asarray(w, dtype=np.float64).reshape(n, n)
    out = np.zeros((n, n))
    for l in range(1, levels + 1):
        h = n >> l
        for (br, bc) in ((0, 1), (1, 0), (1, 1)):
            R = (S[l] if br == 0 else V[l]) ** 2
            Cm = (S[l] if bc == 0 else V[l]) ** 2
            out += R.T @ w[br * h:(br + 1) * h, bc * h:(bc + 1) * h] @ Cm
    return out


def _objective_joint_unsummed(xs, bs, masks, psi, levels, lam, lam_tv, eps=0.0):
    """Joint F with the wavelet norm taken per contrast (no sum under the root)."""
    val = 0.0
    for x, b, m in zip(xs, bs, masks):
        m = np.asarray(m).astype(np.float64)
        val += 0.5 * float(np.sum(np.abs(O.op_A(x, m) - m * b) ** 2))
    kind = O.wavelet_kind(psi)
    if kind:
        val += lam * sum(float(np.sum(np.sqrt(np.abs(O.wavedec2(x, kind, levels)) ** 2 + eps))) for x in xs)
    if psi & O.PSI_TV:
        n = np.asarray(masks[0]).shape[0]
        D1, D2 = O.tv_matrices(n)
        sq = sum(np.abs(D1 @ np.asarray(x).reshape(-1)) ** 2 + np.abs(D2 @ np.asarray(x).reshape(-1)) ** 2
                 for x in xs)
        val += lam_tv * float(np.sum(np.sqrt(sq + eps)))
    return val


def _forward_relu_last(params, inp):
    """The CNN with ReLU on its last layer too."""
    acts = [inp]
    a = inp
    for w, b in params:
        a = np.maximum(C.conv3x3(a, w, b), 0.0)
        acts.append(a)
    return acts


def _adam_no_bias_correction(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    state["t"] += 1
    out = []
    for i, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((w, gw), (b, gb))):
            m = state["m"][2 * i + j] = beta1 * state["m"][2 * i + j] + (1 - beta1) * g
            v = state["v"][2 * i + j] = beta2 * state["v"][2 * i + j] + (1 - beta2) * g * g
            new.append(p - lr * m / (np.sqrt(v) + eps))
        out.append(tuple(new))
    return out


# (target, attribute, replacement, pins that must catch it, invariant pins it passes)
CASES = {
    "dft_unnormalised": [(O, "fft2u", lambda x: np.fft.fft2(x)), (O, "ifft2u", lambda y: np.fft.ifft2(y))],
    "dft_sign": [(O, "fft2u", lambda x: np.fft.ifft2(x, norm="ortho")),
                 (O, "ifft2u", lambda y: np.fft.fft2(y, norm="ortho"))],
    "real_adjoint_imag": [(O, "op_AH", lambda y, mask, real: (lambda o: o.imag if real else o)(
        O.ifft2u(mask * y)))],
    "abar_over_side": [(O, "a_bar", lambda mask: float(np.count_nonzero(mask)) / mask.shape[0])],
    "highpass_no_alternation": [(O, "wavelet_filters", lambda kind: (lambda hg: (hg[0], hg[0][::-1].copy()))(
        _filters(kind)))],
    "odd_phase": [(O, "dwt1", lambda x, h, g, axis: _dwt1_phase(x, h, g, axis, 1))],
    "details_swapped": [(O, "wavedec2", _wavelet_pair(lambda n, m: 0, _swap_details)[0]),
                        (O, "waverec2", _wavelet_pair(lambda n, m: 0, _swap_details)[1])],
    "recursion_on_HH": [(O, "wavedec2", _wavelet_pair(lambda n, m: n - m, _identity)[0]),
                        (O, "waverec2", _wavelet_pair(lambda n, m: n - m, _identity)[1])],
    "synthesis_levels_forward": [(O, "waverec2", lambda c, kind, levels: _waverec_forward(c, kind, levels))],
    "weights_no_sqrt": [(O, "group_weights", lambda c, G, sizes, eps=O.EPS: (
        np.add.reduceat(np.abs(G @ c) ** 2, np.cumsum(sizes) - sizes) + eps) ** -1.0)],
    "overlap_dropped": [(O, "gwg_diag", _gwg_first_only)],
    "tv_seam_kept": [(O, "tv_matrices", _tv_matrices_mut("seam"))],
    "tv_offset": [(O, "tv_matrices", _tv_matrices_mut("offset"))],
    "tv_weight_one_direction": [(O, "tv_weights", lambda x, D1, D2, eps=O.EPS: (
        np.abs(D1 @ x) ** 2 + eps) ** -0.5)],
    "ilu0_pivot_sign": [(O, "ilu0_pivots", _ilu0_plus)],
    "printed_L_unscaled": [(O.System, "_build_preconditioner", _precond_mut("printedL"))],
    "pinv_no_lambda": [(O.System, "_build_preconditioner", _precond_mut("nolam"))],
    "pinv_analysis_synthesis_swapped": [(O.System, "apply_Pinv", _pinv_swapped)],
    "S_wavelet_no_lambda": [(O.System, "apply_S", _apply_S_mut("lam"))],
    "S_tv_sign": [(O.System, "apply_S", _apply_S_mut("tvsign"))],
    "pcg_beta_inverted": [(O, "pcg", _mut_pcg("beta")), (D, "pcg", _mut_pcg("beta"))],
    "pcg_residual_sign": [(O, "pcg", _mut_pcg("resid")), (D, "pcg", _mut_pcg("resid"))],
    "pcg_x_along_r": [(O, "pcg", _mut_pcg("xr")), (D, "pcg", _mut_pcg("xr"))],
    "objective_no_half": [(O, "objective", _objective_mut("half"))],
    "objective_tv_as_l1": [(O, "objective", _objective_mut("tvl1"))],
    "wavelet_diag_bands_swapped": [(O, "wavelet_diag", _wavelet_diag_swapped)],
    "joint_weights_per_contrast": [(O.JointSystem, "update_weights", _joint_weights_per_contrast)],
    "joint_rdot_first_contrast": [(O, "rdot_joint", lambda us, vs: O.rdot(us[0], vs[0]))],
    "dense_abar_over_M": [(D.DenseSystem, "__init__", lambda self, *a, **k: _dense_init_M(self, *a, **k))],
    "dense_jacobi_no_weights": [(D.DenseSystem, "p_diag", lambda self: (
        self.diag_AtA if self.precond == "jacobi" else _orig_p_diag(self)))],
    "dense_weights_no_sqrt": [(D.DenseSystem, "update_weights", lambda self, x: setattr(
        self, "w", (np.asarray(x, dtype=np.float64) ** 2 + self.eps) ** -1.0))],
    "cnn_kernel_flipped": [(C, "conv3x3", _conv_flipped)],
    "cnn_backward_unflipped": [(C, "conv3x3_backward", _conv_backward_unflipped)],
    "synthesis_taps_rolled_back": [(O, "idwt1", _idwt1_shift)],
    "inverse_map_descending": [(O, "inverse_group_map", _inverse_map_descending)],
    "wavelet_diag_no_LL": [(O, "wavelet_diag", _wavelet_diag_no_LL)],
    "l1_tv_weights_swapped": [(O, "tv_weights_aniso", lambda x, D1, D2, eps=O.EPS: tuple(reversed(
        _orig_aniso(x, D1, D2, eps))))],
    "joint_objective_unsummed": [(O, "objective_joint", _objective_joint_unsummed)],
    "dense_objective_no_half": [(D, "objective", lambda x, A, b, lam, eps=0.0: 2.0 * _orig_dense_obj(
        x, A, b, lam, eps) - lam * float(np.sum(np.sqrt(np.asarray(x, dtype=np.float64) ** 2 + eps))))],
    "cnn_relu_on_output": [(C, "forward", _forward_relu_last)],
    "adam_no_bias_correction": [(C, "adam_step", _adam_no_bias_correction)],
}

_orig_aniso = O.tv_weights_aniso
_orig_dense_obj = D.objective

_filters = O.wavelet_filters
_orig_p_diag = D.DenseSystem.p_diag
_orig_dense_init = D.DenseSystem.__init__


def _dense_init_M(self, A, lam, precond="paper", eps=O.EPS):
    _orig_dense_init(self, A, lam, precond, eps)
    self.abar = float(np.trace(self.A.T @ self.A)) / self.A.shape[0]


def _dwt1_phase(x, h, g, axis, phase):
    a = 0
    d = 0
    m = x.shape[axis]
    for t in range(len(h)):
        xs = np.take(np.roll(x, -t, axis=axis), np.arange(phase, m, 2), axis=axis)
        a = a + h[t] * xs
        d = d + g[t] * xs
    return a, d


def _waverec_forward(c, kind, levels):
    h, g = O.wavelet_filters(kind)
    x = np.array(c, copy=True)
    n = x.shape[0]
    for l in range(levels):
        m = n >> l
        blk = x[:m, :m]
        half = m // 2
        col = O.idwt1(blk[:half, :], blk[half:, :], h, g, axis=0)
        x[:m, :m] = O.idwt1(col[:, :half], col[:, half:], h, g, axis=1)
    return x


PINS = {
    "dft_unnormalised": [lambda: TO.test_fft_matches_naive_dft(8), lambda: TO.test_A_adjoint(False)],
    "dft_sign": [lambda: TO.test_fft_matches_naive_dft(8)],
    "real_adjoint_imag": [lambda: TO.test_A_adjoint(True)],
    "abar_over_side": [TO.test_AHA_diagonal_equals_sampling_ratio],
    "highpass_no_alternation": [TO.test_db4_taps_match_published_values],
    "odd_phase": [TO.test_haar_2x2_closed_form, TO.test_db4_level1_bruteforce],
    "details_swapped": [TO.test_haar_multilevel_closed_form, lambda: TO.test_db4_multilevel_bruteforce(16, 2)],
    "recursion_on_HH": [TO.test_haar_multilevel_closed_form, lambda: TO.test_db4_multilevel_bruteforce(16, 3)],
    "synthesis_levels_forward": [lambda: TO.test_wavelet_orthogonal_dense(O.PSI_DB4, 3)],
    "weights_no_sqrt": [TO.test_singleton_weights_are_irls_weights, TO.test_tree_weights_dense],
    "overlap_dropped": [TO.test_tree_weights_dense],
    "tv_seam_kept": [TO.test_tv_matrices_stencil_and_adjoint],
    "tv_offset": [TO.test_tv_matrices_stencil_and_adjoint],
    "tv_weight_one_direction": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV)],
    "ilu0_pivot_sign": [lambda: TO.test_ilu0_reproduces_P_on_its_pattern(O.PSI_TV)],
    "printed_L_unscaled": [TO.test_tv_ilu_factor_identity],
    "pinv_no_lambda": [TO.test_full_mask_wavelet_pcg_one_step],
    "pinv_analysis_synthesis_swapped": [TO.test_full_mask_wavelet_pcg_one_step],
    "S_wavelet_no_lambda": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV),
                            TO.test_S_is_gradient_of_quadratic_model],
    "S_tv_sign": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV)],
    "pcg_beta_inverted": [lambda: TO.test_pcg_matches_dense_direct_solve(O.PSI_DB4, "paper"),
                          lambda: TD.test_pcg_matches_dense_direct_solve("jacobi")],
    "pcg_residual_sign": [lambda: TO.test_pcg_matches_dense_direct_solve(O.PSI_HAAR, "paper"),
                          lambda: TD.test_pcg_matches_dense_direct_solve("paper")],
    "pcg_x_along_r": [lambda: TO.test_pcg_matches_dense_direct_solve(O.PSI_TV, "paper"),
                      lambda: TD.test_pcg_matches_dense_direct_solve("none")],
    "objective_no_half": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV)],
    "objective_tv_as_l1": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV)],
    "wavelet_diag_bands_swapped": [lambda: TO.test_wavelet_diag_bruteforce(O.PSI_DB4, 2)],
    "joint_weights_per_contrast": [lambda: TJ.test_identical_contrasts_reduce_to_one_with_scaled_lambda(
        O.PSI_DB4, 2e-3, 0.0)],
    "joint_rdot_first_contrast": [TJ.test_joint_pcg_matches_dense_block_solve],
    "dense_abar_over_M": [TD.test_abar_of_orthonormal_rows_is_M_over_N],
    "dense_jacobi_no_weights": [TD.test_jacobi_diagonal_is_diag_of_dense_S],
    "dense_weights_no_sqrt": [TD.test_system_is_gradient_of_F_eps],
    "cnn_kernel_flipped": [TC.test_conv_matches_bruteforce],
    "cnn_backward_unflipped": [TC.test_conv_backward_is_the_adjoint],
    "synthesis_taps_rolled_back": [lambda: TO.test_wavelet_orthogonal_dense(O.PSI_DB4, 1)],
    "inverse_map_descending": [TO.test_inverse_group_map_bruteforce],
    "wavelet_diag_no_LL": [lambda: TO.test_wavelet_diag_bruteforce(O.PSI_HAAR, 2)],
    "l1_tv_weights_swapped": [lambda: TO.test_irls_system_is_the_gradient_of_F_eps(O.PSI_TV_ANISO)],
    "joint_objective_unsummed": [lambda: TJ.test_joint_system_is_the_gradient_of_joint_F_eps(O.PSI_HAAR, 5e-3,
                                                                                              0.0)],
    "dense_objective_no_half": [TD.test_system_is_gradient_of_F_eps],
    "cnn_relu_on_output": [TC.test_network_gradients_by_finite_differences],
    "adam_no_bias_correction": [TC.test_adam_matches_closed_form_first_step],
}

# slips that keep an invariant: the invariant's pin passes, the other pins fail
INVARIANT_PINS = {
    "details_swapped": [lambda: TO.test_wavelet_orthogonal_dense(O.PSI_DB4, 2)],
    "recursion_on_HH": [lambda: TO.test_wavelet_orthogonal_dense(O.PSI_HAAR, 4)],
    "dft_sign": [lambda: TO.test_A_adjoint(False), TO.test_AHA_diagonal_equals_sampling_ratio],
}


def test_every_case_has_pins():
    assert set(CASES) == set(PINS)
    assert set(INVARIANT_PINS) <= set(CASES)


def test_pins_pass_unmutated():
    """The harness calls the pins as the suite does: unmutated, they pass."""
    for name in ("dft_unnormalised", "details_swapped", "pcg_beta_inverted", "dense_abar_over_M",
                 "joint_rdot_first_contrast", "cnn_backward_unflipped"):
        for pin in PINS[name] + INVARIANT_PINS.get(name, []):
            assert not _fails(pin), name


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    for target, attr, repl in CASES[name]:
        monkeypatch.setattr(target, attr, repl)
    for pin in INVARIANT_PINS.get(name, []):
        assert not _fails(pin), f"{name}: the invariant pin should not see this slip"
    caught = [i for i, pin in enumerate(PINS[name]) if _fails(pin)]
    assert caught, f"planted mistake '{name}' passed every pin named for it"
