"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types an oracle formula: each checks the oracle against an
independent fact (complex-arithmetic identities, closed forms derived by hand,
exhaustive search, optimality of a projection, finite differences, invariants).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import taser_oracle as O
from synth import make_jed, make_mimo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_signs(rng, n, N):
    s = rng.choice([-1.0, 1.0], size=(n, N))
    s[:, -1] = 1.0
    return s


# ---------------------------------------------------------------- T (Sec. II) ----
@pytest.mark.parametrize("const", ["bpsk", "qpsk"])
def test_T_mimo_equals_residual_norm(const):
    """s~^T T s~ = ||y - H s||^2 for every s~ = [s_bar; 1] (Eq. 1 vs Eq. 2), computed
    here with complex arithmetic, independent of the real decomposition."""
    w = make_mimo(16, 12, 5, 8.0, const, seed=11)
    T = O.T_mimo(w["H"], w["y"], const)
    U = 5
    rng = np.random.default_rng(0)
    H = w["H"].astype(np.complex128)
    y = w["y"].astype(np.complex128)
    for _ in range(20):
        s_t = _random_signs(rng, 16, T.shape[1])
        if const == "qpsk":
            s_c = (s_t[:, :U] + 1j * s_t[:, U:2 * U]) / np.sqrt(2.0)
        else:
            s_c = s_t[:, :U].astype(np.complex128)
        resid = y - np.einsum("nbu,nu->nb", H, s_c)
        lhs = np.einsum("ni,nij,nj->n", s_t, T, s_t)
        np.testing.assert_allclose(lhs, np.sum(np.abs(resid) ** 2, axis=1), rtol=1e-12)


def test_T_jed_equals_minus_energy():
    """s~^T T s~ = -||Y s||^2 with s_0 = +1 (Eq. 4 vs Eq. 5), complex arithmetic."""
    w = make_jed(16, 6, 7, 5.0, seed=3)
    T = O.T_jed_bpsk(w["Y"])
    Y = w["Y"].astype(np.complex128)
    rng = np.random.default_rng(1)
    for _ in range(20):
        s_t = _random_signs(rng, 16, T.shape[1])       # [s_1..s_{K-1}, 1]
        s_full = np.concatenate([np.ones((16, 1)), s_t[:, :-1]], axis=1)
        energy = np.sum(np.abs(np.einsum("nbk,nk->nb", Y, s_full)) ** 2, axis=1)
        lhs = np.einsum("ni,nij,nj->n", s_t, T, s_t)
        np.testing.assert_allclose(lhs, -energy, rtol=1e-12)


def test_T_jed_qpsk_equals_minus_energy():
    """s~^T T s~ = -||Y s||^2 for QPSK JED with the pilot s_0 = (1 + j)/sqrt2 and data
    s_k = (a_k + j b_k)/sqrt2, s~ = [a; b; 1] (Eq. 4 vs Eq. 5, readings R1, R16), in
    complex arithmetic."""
    n, B, K = 12, 6, 5
    w = make_jed(n, B, K, 5.0, seed=13, constellation="qpsk")
    T = O.T_jed_qpsk(w["Y"])
    assert T.shape[1] == O.problem_size("jed_qpsk", K) == 2 * K - 1
    Y = w["Y"].astype(np.complex128)
    rng = np.random.default_rng(2)
    for _ in range(20):
        a = _random_signs(rng, n, K)[:, :-1]
        b = _random_signs(rng, n, K)[:, :-1]
        s_full = np.concatenate([np.full((n, 1), (1 + 1j) / np.sqrt(2.0)), (a + 1j * b) / np.sqrt(2.0)], axis=1)
        s_t = np.concatenate([a, b, np.ones((n, 1))], axis=1)
        energy = np.sum(np.abs(np.einsum("nbk,nk->nb", Y, s_full)) ** 2, axis=1)
        lhs = np.einsum("ni,nij,nj->n", s_t, T, s_t)
        np.testing.assert_allclose(lhs, -energy, rtol=1e-12)


def test_noise_free_jed_qpsk_equals_ml_and_truth():
    """Y = h s^H without noise: the exhaustive ML over the data slots and TASER both return
    the transmitted QPSK symbols (the pilot fixes the phase ambiguity of Sec. II-B)."""
    w = make_jed(20, 16, 5, 400.0, seed=21, constellation="qpsk")
    r = O.detect("jed_qpsk", w["Y"], None, 0.45, 50)
    truth = np.concatenate([w["bits_re"][:, 1:], w["bits_im"][:, 1:]], axis=1)
    ml, _ = O.brute_force_ml(r["T"])
    np.testing.assert_array_equal(ml, truth)
    np.testing.assert_array_equal(r["s_hat"], truth)
    re, im = O.map_back_qpsk(r["s_hat"])
    np.testing.assert_array_equal(re, w["bits_re"][:, 1:])
    np.testing.assert_array_equal(im, w["bits_im"][:, 1:])


def test_T_structure_and_preconditioning():
    """T symmetric, PSD (MIMO) / NSD (JED); T~ has a +-1 diagonal and D^2 = |diag T|
    (Sec. III-C)."""
    w = make_mimo(8, 16, 4, 3.0, "qpsk", seed=5)
    T = O.T_mimo(w["H"], w["y"], "qpsk")
    np.testing.assert_allclose(T, np.transpose(T, (0, 2, 1)), atol=0)
    ev = np.linalg.eigvalsh(T)
    assert (ev > -1e-10 * ev.max(axis=1, keepdims=True)).all()
    Tt, D, flags = O.jacobi_precondition(T)
    np.testing.assert_allclose(np.diagonal(Tt, axis1=1, axis2=2), 1.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(D ** 2, np.abs(np.diagonal(T, axis1=1, axis2=2)), rtol=1e-14)
    assert (flags == 0).all()
    wj = make_jed(8, 8, 6, 3.0, seed=6)
    Tj = O.T_jed_bpsk(wj["Y"])
    evj = np.linalg.eigvalsh(Tj)
    assert (evj < 1e-10 * np.abs(evj).max(axis=1, keepdims=True)).all()
    Ttj, Dj, _ = O.jacobi_precondition(Tj)
    np.testing.assert_allclose(np.diagonal(Ttj, axis1=1, axis2=2), -1.0, atol=1e-15)


def test_zero_diagonal_is_flagged():
    """A user whose channel column is zero gives T_kk = 0: D_kk = 1 and a flag (R3)."""
    w = make_mimo(2, 8, 3, 10.0, "bpsk", seed=2)
    H = w["H"].copy()
    H[0, :, 1] = 0
    T = O.T_mimo(H, w["y"], "bpsk")
    Tt, D, flags = O.jacobi_precondition(T)
    assert flags[0] & O.FLAG_ZERO_DIAG and flags[1] == 0
    assert D[0, 1] == 1.0 and np.all(Tt[0, 1, :] == 0)


# ------------------------------------------------------- ||T~||_2 (Sec. III-B) ----
def test_spectral_norm_closed_forms():
    # 2x2 [[1, c], [c, 1]]: eigenvalues 1 +- c
    c = np.array([0.3, -0.7, 0.0])
    Tt = np.stack([np.array([[1, x], [x, 1]]) for x in c])
    np.testing.assert_allclose(O.spectral_norm(Tt), 1 + np.abs(c), rtol=1e-15)
    # bordered identity [[I, b], [b^T, 1]]: eigenvalues 1 (N-2 times) and 1 +- ||b||
    rng = np.random.default_rng(4)
    b = rng.uniform(-0.3, 0.3, size=(5, 8))
    M = np.zeros((5, 9, 9))
    M[:, np.arange(9), np.arange(9)] = 1.0
    M[:, :8, 8] = b
    M[:, 8, :8] = b
    np.testing.assert_allclose(O.spectral_norm(M), 1 + np.linalg.norm(b, axis=1), rtol=1e-14)
    # negative rank one: -s s^T has norm N
    s = _random_signs(rng, 4, 7)
    np.testing.assert_allclose(O.spectral_norm(-np.einsum("ni,nj->nij", s, s)), 7.0, rtol=1e-14)


def test_spectral_norm_is_the_operator_norm():
    """||T~ x|| <= ||T~|| ||x|| for all x, with equality approached by maximisation."""
    w = make_mimo(6, 32, 8, 6.0, "bpsk", seed=9)
    Tt, _, _ = O.jacobi_precondition(O.T_mimo(w["H"], w["y"], "bpsk"))
    nrm = O.spectral_norm(Tt)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 4000, 9))
    ratio = np.linalg.norm(np.einsum("nij,nkj->nki", Tt, x), axis=2) / np.linalg.norm(x, axis=2)
    assert (ratio.max(axis=1) <= nrm * (1 + 1e-12)).all()
    # singular values (a different factorisation) agree
    np.testing.assert_allclose(np.linalg.svd(Tt, compute_uv=False)[:, 0], nrm, rtol=1e-12)


# ------------------------------------------- gradient and prox (Sec. III-B/C) ----
def test_gradient_matches_finite_differences():
    """The gradient step uses tril(grad f) with f(L) = Tr(L T~ L^T): compare with
    central differences of f on every lower-triangular entry."""
    rng = np.random.default_rng(7)
    N = 5
    A = rng.standard_normal((1, N, N))
    Tt = A + np.transpose(A, (0, 2, 1))
    L = np.tril(rng.standard_normal((1, N, N)))
    G = O.gradient(L, Tt)
    h = 1e-6
    for i in range(N):
        for j in range(i + 1):
            E = np.zeros_like(L)
            E[0, i, j] = h
            fd = (O.objective(L + E, Tt) - O.objective(L - E, Tt)) / (2 * h)
            assert abs(fd[0] - G[0, i, j]) < 1e-6 * max(1.0, abs(fd[0]))
    assert np.all(np.triu(G[0], 1) == 0)


def test_prox_is_the_nearest_point():
    """prox rescales every column to norm D_kk; that is the closest point of the
    sphere of radius D_kk (Eq. 9 with the characteristic function g~)."""
    rng = np.random.default_rng(8)
    N = 6
    V = np.tril(rng.standard_normal((3, N, N)))
    V[:, -1, -1] = np.abs(V[:, -1, -1]) + 0.1
    D = rng.uniform(0.5, 3.0, size=(3, N))
    P, flags = O.prox(V, D, "literal")
    np.testing.assert_allclose(np.linalg.norm(P, axis=1), D, rtol=1e-14)
    for k in range(N - 1):
        col = V[:, k:, k]
        dist = np.linalg.norm(P[:, k:, k] - col, axis=1)
        z = rng.standard_normal((3, 500, N - k))
        z = z / np.linalg.norm(z, axis=2, keepdims=True) * D[:, k, None, None]
        other = np.linalg.norm(z - col[:, None, :], axis=2).min(axis=1)
        assert (dist <= other + 1e-12).all()


# ------------------------------------------------- Algorithm 1 closed forms ----
def test_N2_first_iterate_and_ml_sign():
    """N = 2 (one BPSK user).  T~ = [[1, c], [c, 1]], L~(0) = D.  By hand, one
    iteration gives V_11 = D_1 (1 - 2 tau), V_21 = -2 tau c D_2, so
    L~(1)_21 = -D_1 2 tau c D_2 / sqrt(D_1^2 (1 - 2tau)^2 + 4 tau^2 c^2 D_2^2), and
    for 2 tau < 1 the sign of V_21 stays -sign(c) = sign(Re h^H y) (the ML decision)
    for every later t."""
    w = make_mimo(64, 8, 1, 0.0, "bpsk", seed=21)
    r = O.detect("mimo_bpsk", w["H"], w["y"], 0.45, 1)
    Tt, D, tau = r["T_tilde"], r["D"], r["tau"]
    c = Tt[:, 0, 1]
    L21 = -D[:, 0] * 2 * tau * c * D[:, 1] / np.sqrt(
        D[:, 0] ** 2 * (1 - 2 * tau) ** 2 + 4 * tau ** 2 * c ** 2 * D[:, 1] ** 2)
    np.testing.assert_allclose(r["L"][:, 1, 0], L21, rtol=1e-12)
    H = w["H"].astype(np.complex128)[:, :, 0]
    ml = np.where(np.real(np.sum(np.conj(H) * w["y"], axis=1)) >= 0, 1, -1)
    for t_max in (1, 2, 7, 30):
        r = O.detect("mimo_bpsk", w["H"], w["y"], 0.45, t_max)
        np.testing.assert_array_equal(r["s_hat"][:, 0], ml)


def _orthogonal_channel(n, B, U, rng):
    Q = np.linalg.qr(rng.standard_normal((n, 2 * B, 2 * B)))[0]
    # columns of a complex H whose real form has orthogonal columns: take H = Q1 + j Q2
    # with [Q1; Q2] orthonormal columns of a real 2B x U matrix (BPSK: Hunder^T Hunder = I)
    cols = Q[:, :, :U] * rng.uniform(0.5, 2.0, size=(n, 1, U))
    return cols[:, :B, :] + 1j * cols[:, B:, :]


def test_orthogonal_channel_gives_ml():
    """BPSK with orthogonal real channel columns: the user block of T~ is I, and for
    2 tau < 1 the decisions equal sign(Hunder^T ybar), which is the exact ML
    decision there (checked against exhaustive search), for every t."""
    rng = np.random.default_rng(12)
    n, B, U = 40, 10, 6
    H = _orthogonal_channel(n, B, U, rng)
    s = rng.choice([-1.0, 1.0], size=(n, U))
    y = np.einsum("nbu,nu->nb", H, s) + 1.5 * (rng.standard_normal((n, B)) + 1j * rng.standard_normal((n, B)))
    T = O.T_mimo(H, y, "bpsk")
    Tt, D, _ = O.jacobi_precondition(T)
    np.testing.assert_allclose(Tt[:, :U, :U], np.broadcast_to(np.eye(U), (n, U, U)), atol=1e-12)
    ml, _ = O.brute_force_ml(T)
    mf = np.where(np.einsum("nbu,nb->nu", np.concatenate([H.real, H.imag], 1),
                            np.concatenate([y.real, y.imag], 1)) >= 0, 1, -1)
    np.testing.assert_array_equal(ml, mf)
    tau = O.step_size(Tt, 0.45)
    for t_max in (1, 3, 20):
        L, _ = O.taser(Tt, D, tau, t_max)
        np.testing.assert_array_equal(O.decisions(L), ml)


def test_noise_free_jed_recovers_symbols():
    """Y = h s^T: T~ = -s~ s~^T and the decisions equal the transmitted slots."""
    w = make_jed(30, 16, 12, 300.0, seed=4)
    r = O.detect("jed_bpsk", w["Y"], None, 0.45, 5)
    np.testing.assert_array_equal(r["s_hat"], w["s"][:, 1:])
    s_t = np.concatenate([w["s"][:, 1:], np.ones((30, 1))], axis=1).astype(np.float64)
    np.testing.assert_allclose(r["T_tilde"], -np.einsum("ni,nj->nij", s_t, s_t), atol=1e-5)
    np.testing.assert_allclose(r["tau"], 0.45 / 12, rtol=1e-5)


@pytest.mark.parametrize("const,U", [("bpsk", 4), ("bpsk", 6), ("qpsk", 2), ("qpsk", 3)])
def test_noise_free_tall_channel_equals_ml_and_truth(const, U):
    """Noise-free, well-conditioned (B >= 8U): TASER = exhaustive ML = transmitted."""
    B = 8 * U
    w = make_mimo(25, B, U, 400.0, const, seed=30 + U)
    r = O.detect("mimo_" + const, w["H"], w["y"], 0.45, 50)
    truth = w["bits_re"] if const == "bpsk" else np.concatenate([w["bits_re"], w["bits_im"]], 1)
    ml, _ = O.brute_force_ml(r["T"])
    np.testing.assert_array_equal(ml, truth)
    np.testing.assert_array_equal(r["s_hat"], truth)


def test_brute_force_ml_is_exhaustive():
    """brute_force_ml agrees with a plain loop over all sign vectors (tiny N)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 6, 6))
    T = A @ np.transpose(A, (0, 2, 1))
    s, v = O.brute_force_ml(T)
    for i in range(3):
        best = min((np.array(list(c) + [1.0]) @ T[i] @ np.array(list(c) + [1.0]), c)
                   for c in itertools.product((-1.0, 1.0), repeat=5))
        assert abs(best[0] - v[i]) < 1e-12
        np.testing.assert_array_equal(s[i], np.array(best[1]))


# --------------------------------------------- invariants (Sec. III-C, III-E) ----
def test_iterate_invariants_and_descent():
    """Every iterate: lower-triangular, column norms D_kk, L~_NN = D_NN (mode fixed);
    the objective does not increase for alpha < 1/2 (Prop. 1 step-size regime with the
    Lipschitz constant 2||T~|| of tril(2 L T~))."""
    for kind, w in (("mimo_qpsk", make_mimo(40, 32, 8, 4.0, "qpsk", seed=40)),
                    ("mimo_bpsk", make_mimo(40, 16, 12, 2.0, "bpsk", seed=41))):
        r = O.detect(kind, w["H"], w["y"], 0.45, 1)
        Tt, D, tau = r["T_tilde"], r["D"], r["tau"]
        L, _, Ls = O.taser(Tt, D, tau, 40, history=True)
        f_prev = O.objective(Ls[0], Tt)
        for Lt in Ls[1:]:
            assert np.all(np.triu(Lt, 1) == 0)
            np.testing.assert_allclose(np.linalg.norm(Lt, axis=1), D, rtol=1e-12)
            np.testing.assert_array_equal(Lt[:, -1, -1], D[:, -1])
            f = O.objective(Lt, Tt)
            assert np.all(f <= f_prev + 1e-9 * np.abs(f_prev))
            f_prev = f


def test_convergence_to_a_fixed_point():
    """Prop. 1: the iterates converge; ||L~(t) - L~(t-1)||_F -> 0."""
    w = make_mimo(10, 32, 6, 5.0, "bpsk", seed=42)
    r = O.detect("mimo_bpsk", w["H"], w["y"], 0.45, 1)
    L, _, Ls = O.taser(r["T_tilde"], r["D"], r["tau"], 1500, history=True)
    step = np.linalg.norm(Ls[-1] - Ls[-2], axis=(1, 2)) / np.linalg.norm(Ls[-1], axis=(1, 2))
    assert (step < 1e-9).all()


def test_literal_prox_of_the_last_column_is_the_nearest_point():
    """Literal mode (reading R7) on the branch V_NN <= 0.  The last column of a lower-
    triangular V holds V_NN alone, so its sphere of radius D_NN (Eq. 9) is the two-point
    set {-D_NN, +D_NN}; the nearest point of a negative V_NN is -D_NN, and at the tie
    V_NN = 0 the reading sign(0) = +1 picks +D_NN.  Every such step is flagged."""
    rng = np.random.default_rng(81)
    N = 5
    vnn = np.array([-2.5, -1e-9, 0.0, 1e-9, 0.7, -0.3])
    n = len(vnn)
    V = np.tril(rng.standard_normal((n, N, N)))
    V[:, -1, -1] = vnn
    D = rng.uniform(0.5, 3.0, size=(n, N))
    P, flags = O.prox(V, D, "literal")
    cand = np.stack([-D[:, -1], D[:, -1]], axis=1)                       # the 1-D sphere
    best = cand[np.arange(n), np.argmin(np.abs(cand - vnn[:, None]), axis=1)]
    tie = vnn == 0.0
    np.testing.assert_array_equal(P[~tie, -1, -1], best[~tie])
    np.testing.assert_array_equal(P[tie, -1, -1], D[tie, -1])
    np.testing.assert_array_equal((flags & O.FLAG_LNN_SIGN) != 0, vnn <= 0.0)
    Pf, ff = O.prox(V, D, "fixed")
    np.testing.assert_array_equal(Pf[:, -1, -1], D[:, -1])                # mode C: always +D_NN
    np.testing.assert_array_equal(ff, flags)
    np.testing.assert_array_equal(Pf[:, :, :-1], P[:, :, :-1])            # other columns unaffected


def test_literal_mode_is_symmetric_under_negating_the_last_row():
    """S = L^T L (the relaxed SDR variable) does not change when the whole last row of L~
    is negated (its entries enter S only as products L_Nj L_Nk), and neither do the
    decisions sign(S_Nk) = sign(L~_NN) sign(L~_Nk) of literal mode.  One literal step maps
    the negated state to the negated step: the gradient row N is linear in row N, the
    column norms only see squares, and the last column's prox follows sign(V_NN).  Checked
    on states of real trajectories in which V_NN <= 0 occurs (the unpinned branch)."""
    w = make_mimo(64, 8, 6, 0.0, "bpsk", seed=82)                 # N = 7, 0 dB, B = 8
    r = O.detect("mimo_bpsk", w["H"], w["y"], 0.95, 1)
    Tt, D, tau = r["T_tilde"], r["D"], r["tau"]
    L, flags, Ls = O.taser(Tt, D, tau, 12, lnn_mode="literal", history=True)
    hit = (flags & O.FLAG_LNN_SIGN) != 0
    assert hit.sum() >= 5
    assert (np.array([Lt[:, -1, -1] for Lt in Ls]) < 0).any(axis=0)[hit].sum() >= 5
    for Lt in Ls[1:]:
        R = Lt.copy()
        R[:, -1, :] *= -1.0
        np.testing.assert_allclose(np.matmul(np.transpose(R, (0, 2, 1)), R),
                                   np.matmul(np.transpose(Lt, (0, 2, 1)), Lt), rtol=0, atol=1e-12)
        np.testing.assert_array_equal(O.decisions(R, "literal"), O.decisions(Lt, "literal"))
        step, _ = O.prox(Lt - tau[:, None, None] * O.gradient(Lt, Tt), D, "literal")
        step_r, _ = O.prox(R - tau[:, None, None] * O.gradient(R, Tt), D, "literal")
        mirrored = step.copy()
        mirrored[:, -1, :] *= -1.0
        # the mirror holds exactly wherever V_NN != 0 (sign(0) = +1 breaks the symmetry)
        vnn = (Lt - tau[:, None, None] * O.gradient(Lt, Tt))[:, -1, -1]
        ok = vnn != 0.0
        np.testing.assert_allclose(step_r[ok], mirrored[ok], rtol=0, atol=1e-12)


def test_modes_agree_while_vnn_positive():
    """Reading R7: literal and fixed modes coincide whenever V_NN > 0."""
    w = make_mimo(30, 64, 8, 8.0, "qpsk", seed=43)
    r = O.detect("mimo_qpsk", w["H"], w["y"], 0.45, 20)
    rl = O.detect("mimo_qpsk", w["H"], w["y"], 0.45, 20, lnn_mode="literal")
    ok = (r["flags"] & O.FLAG_LNN_SIGN) == 0
    assert ok.sum() > 20
    np.testing.assert_array_equal(r["L"][ok], rl["L"][ok])
    np.testing.assert_array_equal(r["s_hat"], rl["s_hat"])


# --------------------------------------------------------- Table I (Sec. V-B) ----
def _triangular_array_mults(N):
    """Count multiplications of one iteration by walking the triangular array of
    Sec. IV-A: row i (1-based) has i PEs and finishes after i MAC cycles; each PE
    squares its V once and scales once; the scale unit of each column multiplies once."""
    count = 0
    for i in range(1, N + 1):
        for j in range(1, i + 1):
            count += i          # matrix-multiplication mode
            count += 1          # squared-norm mode
            count += 1          # scaling mode
    count += N                  # D_jj * rsqrt(.) in the column scale units
    return count


def test_table1_multiplication_counts():
    with open(os.path.join(GOLDEN, "table1_complexity.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for const, U, t_max, value in rows:
        U, t_max, value = int(U), int(t_max), int(value)
        N = U + 1 if const == "bpsk" else 2 * U + 1
        assert _triangular_array_mults(N) * t_max == value
        assert abs(O.table1_mults(const, U, t_max) - value) < 1e-9


# ------------------------------------------------- unfolded adjoint (R13) ----
def test_unfolded_adjoint_matches_finite_differences():
    w = make_mimo(3, 16, 4, 6.0, "qpsk", seed=50)     # N = 9
    r = O.detect("mimo_qpsk", w["H"], w["y"], 0.4, 1)
    Tt, D = r["T_tilde"], r["D"]
    t_max = 6
    rng = np.random.default_rng(1)
    tau_t = r["tau"][:, None] * rng.uniform(0.6, 1.2, size=(3, t_max))
    s_bar = np.concatenate([w["bits_re"], w["bits_im"]], 1).astype(np.float64)

    def loss(tt):
        L, _ = O.unfolded_forward(Tt, D, tt)
        return O.mse_loss(L, D, s_bar)

    L, Ls = O.unfolded_forward(Tt, D, tau_t)
    x = O.soft_output(L, D)
    g_soft = 2.0 * (x - s_bar) / x.size
    g = O.unfolded_backward(Tt, D, tau_t, Ls, g_soft)
    h = 1e-6
    for i in range(3):
        for t in range(t_max):
            e = np.zeros_like(tau_t)
            e[i, t] = h * tau_t[i, t]
            fd = (loss(tau_t + e) - loss(tau_t - e)) / (2 * e[i, t])
            assert abs(fd - g[i, t]) <= 1e-6 * max(abs(fd), 1e-8) + 1e-12, (i, t, fd, g[i, t])


def test_unfolded_adjoint_dot_product():
    """<J v, w> = <v, J^T w> with J = d(soft output)/d(tau_t), J v by central differences."""
    w = make_mimo(2, 12, 4, 3.0, "bpsk", seed=51)     # N = 5
    r = O.detect("mimo_bpsk", w["H"], w["y"], 0.4, 1)
    Tt, D = r["T_tilde"], r["D"]
    t_max = 5
    rng = np.random.default_rng(2)
    tau_t = r["tau"][:, None] * rng.uniform(0.7, 1.1, size=(2, t_max))
    v = rng.standard_normal(tau_t.shape)
    wv = rng.standard_normal((2, 4))
    h = 1e-6
    xp = O.soft_output(O.unfolded_forward(Tt, D, tau_t + h * v)[0], D)
    xm = O.soft_output(O.unfolded_forward(Tt, D, tau_t - h * v)[0], D)
    Jv = (xp - xm) / (2 * h)
    _, Ls = O.unfolded_forward(Tt, D, tau_t)
    JTw = O.unfolded_backward(Tt, D, tau_t, Ls, wv)
    lhs, rhs = np.sum(Jv * wv), np.sum(v * JTw)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
