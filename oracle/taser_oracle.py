"""FP64 CPU oracle for TASER (Castaneda, Goldstein, Studer, arXiv:1609.01797).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or runs this
module: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may use it.  It shares no code with the CUDA path; the only thing both
sides consume is the seeded input generator in ``synth`` (which holds none of the
method's arithmetic).

Everything is plain numpy in float64, batched over a leading instance axis ``n``.
Batching over independent instances is the only restructuring; every step follows
the paper's definitions in the paper's order:

  * real-valued decomposition and the matrix T          (Sec. II-A, Eq. 2; Sec. II-B, Eq. 5)
  * Jacobi preconditioning  D = diag(sqrt T_kk), T~ = D^-1 T D^-1   (Sec. III-C)
  * step size  tau = alpha / ||T~||_2                   (Sec. III-B, Algorithm 1 inputs)
  * Algorithm 1 (TASER): L~(0) = D; V = L~ - tril(2 tau L~ T~); L~ = prox(V)
  * decisions  s_k = sign(L~_{N,k}), k < N              (Algorithm 1 outputs)

Readings taken where the paper is silent or ambiguous (the identifiers are shared with
the project's design notes):
  R1  QPSK symbols are (+-1 +-j)/sqrt2: T is built from the effective channel H/sqrt2
      so that the relaxed vector is exactly in {+-1}^N.
  R2  The augmented "1" coordinate is the last index N; for JED the pilot column
      y_0 s_0 (s_0 = +1) is moved to the end, so N = K when K counts the pilot slot.
  R16 JED with QPSK: the pilot is s_0 = (1 + j)/sqrt2, the data slots use the effective
      Y_r / sqrt2 (as R1), and N = 2K - 1 when K counts the pilot slot.
  R3  D_kk = sqrt(|T_kk|) (T_kk < 0 for JED); D_kk = 0 is replaced by 1 and flagged.
  R7  Sign of L~_NN: mode "fixed" (default) keeps L~_NN = D_NN, mode "literal" applies
      the prox to the last column as well, L~_NN = D_NN sign(V_NN), and multiplies
      the decisions by sign(L~_NN).
  R8  sign(0) = +1.
  R9  ||T~||_2 is the exact largest |eigenvalue| (symmetric eigensolver).
  R13 Unfolded TASER: per-iteration steps tau_t; soft output x_k = L~_{N,k} / D_kk.

Parity status: every function below is pinned by tests in tests/test_oracle_pins.py
(closed forms, identities, brute force, invariants, finite differences).  The BER /
VER curves of Sec. V-A are *parity unpinned* against the paper (its plots are not
available as numbers).
"""
import itertools

import numpy as np

# Per-instance flag bits (same meaning as the C-ABI flags).
FLAG_ZERO_DIAG = 1 << 0      # some T_kk == 0; D_kk replaced by 1
FLAG_NONFINITE = 1 << 1      # non-finite value in the input
FLAG_ZERO_COLUMN = 1 << 2    # a column of V had zero norm during the prox
FLAG_LNN_SIGN = 1 << 3       # V_NN <= 0 was seen (mode "fixed" keeps L~_NN = D_NN)

QPSK_SCALE = 1.0 / np.sqrt(2.0)


def problem_size(kind, U_or_K):
    """N of the real-valued problem: BPSK U+1, QPSK 2U+1 (Sec. II-A); JED BPSK N = K
    when K counts the pilot slot (Sec. II-B with reading R2)."""
    if kind == "mimo_bpsk":
        return U_or_K + 1
    if kind == "mimo_qpsk":
        return 2 * U_or_K + 1
    if kind == "jed_bpsk":
        return U_or_K
    if kind == "jed_qpsk":
        return 2 * U_or_K - 1
    raise ValueError(kind)


# ----------------------------------------------------------------------------------
# Sec. II-A: coherent MU-MIMO, real-valued decomposition (Eq. 2)
# ----------------------------------------------------------------------------------
def real_decomposition_mimo(H, y, constellation):
    """Explicit real-valued model of Sec. II-A.

    QPSK: ybar = [Re y; Im y], Hbar = [[Re H, -Im H], [Im H, Re H]] (2B x 2U) of the
          effective channel H/sqrt2 (reading R1).
    BPSK: ybar = [Re y; Im y], Hunder = [Re H; Im H] (2B x U).
    H complex [n, B, U], y complex [n, B]. Returns (Hbar [n, 2B, M], ybar [n, 2B]).
    """
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    ybar = np.concatenate([y.real, y.imag], axis=1)
    if constellation == "qpsk":
        He = H * QPSK_SCALE
        top = np.concatenate([He.real, -He.imag], axis=2)
        bot = np.concatenate([He.imag, He.real], axis=2)
        Hbar = np.concatenate([top, bot], axis=1)
    elif constellation == "bpsk":
        Hbar = np.concatenate([H.real, H.imag], axis=1)
    else:
        raise ValueError(constellation)
    return Hbar, ybar


def T_mimo(H, y, constellation):
    """T = [Hbar^T Hbar, -Hbar^T ybar; -ybar^T Hbar, ybar^T ybar] (Sec. II-A, Eq. 2).

    Formed as A^T A with A = [Hbar, -ybar], which is that block matrix written out.
    """
    Hbar, ybar = real_decomposition_mimo(H, y, constellation)
    A = np.concatenate([Hbar, -ybar[:, :, None]], axis=2)
    return np.matmul(np.transpose(A, (0, 2, 1)), A)


def T_jed_bpsk(Y):
    """SIMO JED with BPSK (Sec. II-B, Eq. 5).

    Y complex [n, B, K]; column 0 is the pilot slot with s_0 = +1 (reading R2).
    Hunder = [Re Y_r; Im Y_r] (2B x (K-1)), ybar = [Re(y_0 s_0); Im(y_0 s_0)],
    T = -[Hunder^T Hunder, Hunder^T ybar; ybar^T Hunder, ybar^T ybar] = -A^T A with
    A = [Hunder, ybar].  N = K.
    """
    Y = np.asarray(Y, dtype=np.complex128)
    s0 = 1.0
    y0 = Y[:, :, 0] * s0
    Yr = Y[:, :, 1:]
    Hunder = np.concatenate([Yr.real, Yr.imag], axis=1)
    ybar = np.concatenate([y0.real, y0.imag], axis=1)
    A = np.concatenate([Hunder, ybar[:, :, None]], axis=2)
    return -np.matmul(np.transpose(A, (0, 2, 1)), A)


QPSK_PILOT = (1.0 + 1.0j) / np.sqrt(2.0)


def T_jed_qpsk(Y):
    """SIMO JED with QPSK (Sec. II-B, Eq. 5).

    Y complex [n, B, K]; column 0 is the pilot slot, s_0 = (1 + j)/sqrt2 (reading R16).
    ybar = [Re(y_0 s_0); Im(y_0 s_0)], Hbar = [[Re Y_r, -Im Y_r], [Im Y_r, Re Y_r]] of the
    effective Y_r / sqrt2 (reading R1), and
    T = -[Hbar^T Hbar, Hbar^T ybar; ybar^T Hbar, ybar^T ybar] = -A^T A with A = [Hbar, ybar].
    N = 2(K - 1) + 1 = 2K - 1 (the paper's 2K + 1 with its K = our K - 1 data slots).
    """
    Y = np.asarray(Y, dtype=np.complex128)
    y0 = Y[:, :, 0] * QPSK_PILOT
    Yr = Y[:, :, 1:] * QPSK_SCALE
    ybar = np.concatenate([y0.real, y0.imag], axis=1)
    top = np.concatenate([Yr.real, -Yr.imag], axis=2)
    bot = np.concatenate([Yr.imag, Yr.real], axis=2)
    Hbar = np.concatenate([top, bot], axis=1)
    A = np.concatenate([Hbar, ybar[:, :, None]], axis=2)
    return -np.matmul(np.transpose(A, (0, 2, 1)), A)


def build_T(kind, H_or_Y, y=None):
    if kind == "mimo_bpsk":
        return T_mimo(H_or_Y, y, "bpsk")
    if kind == "mimo_qpsk":
        return T_mimo(H_or_Y, y, "qpsk")
    if kind == "jed_bpsk":
        return T_jed_bpsk(H_or_Y)
    if kind == "jed_qpsk":
        return T_jed_qpsk(H_or_Y)
    raise ValueError(kind)


# ----------------------------------------------------------------------------------
# Sec. III-C: Jacobi preconditioning
# ----------------------------------------------------------------------------------
def jacobi_precondition(T):
    """D = diag(sqrt |T_kk|) and T~ = D^-1 T D^-1 (Sec. III-C; reading R3).

    Returns (T_tilde [n,N,N], D [n,N], flags uint32 [n]).
    """
    T = np.asarray(T, dtype=np.float64)
    n = T.shape[0]
    flags = np.zeros(n, dtype=np.uint32)
    diag = np.abs(np.diagonal(T, axis1=1, axis2=2))
    zero = diag == 0.0
    flags[zero.any(axis=1)] |= FLAG_ZERO_DIAG
    D = np.sqrt(np.where(zero, 1.0, diag))
    flags[~np.isfinite(T).all(axis=(1, 2))] |= FLAG_NONFINITE
    Tt = T / D[:, :, None] / D[:, None, :]
    return Tt, D, flags


def spectral_norm(Tt):
    """||T~||_2 of a symmetric matrix: the largest |eigenvalue| (reading R9)."""
    ev = np.linalg.eigvalsh(np.asarray(Tt, dtype=np.float64))
    return np.max(np.abs(ev), axis=1)


def step_size(Tt, alpha):
    """tau = alpha / ||T~||_2 with 0 < alpha < 1 (Sec. III-B, Algorithm 1 inputs)."""
    return alpha / spectral_norm(Tt)


# ----------------------------------------------------------------------------------
# Sec. III-B/III-D: objective, gradient, prox, Algorithm 1
# ----------------------------------------------------------------------------------
def objective(L, Tt):
    """f(L~) = Tr(L~ T~ L~^T) (Eq. 8 after preconditioning)."""
    return np.einsum("nij,njk,nik->n", L, Tt, L)


def gradient(L, Tt):
    """Gradient of f restricted to lower-triangular L~: tril(2 L~ T~) (Sec. III-B)."""
    return np.tril(2.0 * np.matmul(L, Tt))


def prox(V, D, lnn_mode="fixed"):
    """prox_g~ of Sec. III-C: column k is rescaled to Euclidean norm D_kk.

    The last column holds only the (N,N) entry.  Mode "fixed" (reading R7) pins it
    to +D_NN; mode "literal" applies the prox to it as well (D_NN sign(V_NN)).
    A column with zero norm is left at zero and flagged.
    Returns (L_new, flags).
    """
    n, N, _ = V.shape
    flags = np.zeros(n, dtype=np.uint32)
    norms = np.sqrt(np.sum(V * V, axis=1))              # column norms, [n, N]
    zero = norms == 0.0
    flags[zero[:, : N - 1].any(axis=1)] |= FLAG_ZERO_COLUMN
    scale = np.where(zero, 0.0, D / np.where(zero, 1.0, norms))
    L = V * scale[:, None, :]
    vnn = V[:, N - 1, N - 1]
    flags[vnn <= 0.0] |= FLAG_LNN_SIGN
    if lnn_mode == "fixed":
        L[:, N - 1, N - 1] = D[:, N - 1]
    elif lnn_mode == "literal":
        L[:, N - 1, N - 1] = D[:, N - 1] * np.where(vnn >= 0.0, 1.0, -1.0)
    else:
        raise ValueError(lnn_mode)
    return L, flags


def taser(Tt, D, tau, t_max, lnn_mode="fixed", history=False):
    """Algorithm 1 (TASER).

    Inputs T~ [n,N,N], D [n,N], tau [n] (or [n, t_max] for per-iteration steps, as
    used by unfolded TASER), t_max >= 1.
    L~(0) = D; for t = 1..t_max: V = L~ - tril(2 tau L~ T~); L~ = prox(V).
    Returns (L [n,N,N], flags [n]) or, with history=True, (L, flags, Ls) where
    Ls[t] is L~(t) for t = 0..t_max.
    """
    if t_max < 1:
        raise ValueError("t_max must be >= 1")
    Tt = np.asarray(Tt, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    n, N, _ = Tt.shape
    tau = np.asarray(tau, dtype=np.float64)
    if tau.ndim == 1:
        tau = np.repeat(tau[:, None], t_max, axis=1)
    L = np.zeros((n, N, N))
    L[:, np.arange(N), np.arange(N)] = D
    flags = np.zeros(n, dtype=np.uint32)
    Ls = [L.copy()] if history else None
    for t in range(t_max):
        V = L - tau[:, t, None, None] * gradient(L, Tt)
        L, f = prox(V, D, lnn_mode)
        flags |= f
        if history:
            Ls.append(L.copy())
    if history:
        return L, flags, Ls
    return L, flags


def decisions(L, lnn_mode="fixed"):
    """s_k = sign(L~_{N,k}) for k = 1..N-1 (Algorithm 1 outputs), sign(0) = +1.
    In mode "literal" the row is multiplied by sign(L~_NN) (reading R7). int8 [n, N-1]."""
    row = L[:, -1, :-1]
    s = np.where(row >= 0.0, 1, -1).astype(np.int8)
    if lnn_mode == "literal":
        s = s * np.where(L[:, -1, -1] >= 0.0, 1, -1).astype(np.int8)[:, None]
    return s


def map_back_qpsk(s_bar):
    """Sec. II-A: [s_hat]_i = [s_bar]_i + j [s_bar]_{i+U}; returns (re, im) +-1 int8."""
    U = s_bar.shape[1] // 2
    return s_bar[:, :U], s_bar[:, U:]


def detect(kind, H_or_Y, y, alpha, t_max, lnn_mode="fixed"):
    """End to end: T, preconditioning, tau, Algorithm 1, decisions."""
    T = build_T(kind, H_or_Y, y)
    Tt, D, f0 = jacobi_precondition(T)
    tau = step_size(Tt, alpha)
    L, f1 = taser(Tt, D, tau, t_max, lnn_mode)
    return {"T": T, "T_tilde": Tt, "D": D, "tau": tau, "L": L,
            "s_hat": decisions(L, lnn_mode), "flags": f0 | f1}


# ----------------------------------------------------------------------------------
# Eq. 2 / Eq. 5 by exhaustive search (tiny instances only)
# ----------------------------------------------------------------------------------
def brute_force_ml(T):
    """argmin over s~ in {+-1}^(N-1) x {+1} of s~^T T s~ (Eq. 2 / Eq. 5).
    Returns (s_bar int8 [n, N-1], min value [n])."""
    T = np.asarray(T, dtype=np.float64)
    n, N, _ = T.shape
    if N - 1 > 16:
        raise ValueError("brute force limited to N-1 <= 16")
    cand = np.array(list(itertools.product((-1.0, 1.0), repeat=N - 1)))
    cand = np.concatenate([cand, np.ones((cand.shape[0], 1))], axis=1)   # [C, N]
    vals = np.einsum("ci,nij,cj->nc", cand, T, cand)
    best = np.argmin(vals, axis=1)
    return cand[best, :-1].astype(np.int8), vals[np.arange(n), best]


# ----------------------------------------------------------------------------------
# Unfolded TASER (reading R13): soft output, MSE loss and its reverse-mode adjoint
# ----------------------------------------------------------------------------------
def soft_output(L, D):
    """x_k = L~_{N,k} / D_kk = L_{N,k} (last row of the unit-column factor), k < N."""
    return L[:, -1, :-1] / D[:, :-1]


def mse_loss(L, D, s_bar):
    """mean over (instances, k) of (x_k - s_k)^2."""
    x = soft_output(L, D)
    return np.mean((x - s_bar) ** 2)


def unfolded_forward(Tt, D, tau_t):
    """Algorithm 1 with per-iteration steps tau_t [n, t_max], mode "fixed".
    Returns (L_final, Ls) with Ls[t] = L~(t), t = 0..t_max."""
    tau_t = np.asarray(tau_t, dtype=np.float64)
    L, _, Ls = taser(Tt, D, tau_t, tau_t.shape[1], "fixed", history=True)
    return L, Ls


def unfolded_backward(Tt, D, tau_t, Ls, grad_soft):
    """Reverse-mode adjoint of unfolded TASER (mode "fixed").

    grad_soft [n, N-1] = dloss/dx.  Returns dloss/dtau_t [n, t_max].
    Per step t (in reverse), with V_t = L~(t-1) - tau_t tril(2 L~(t-1) T~):
      Lbar(t)[:, N-1] is ignored (L~_NN is a constant), for k < N-1:
        u_k = V_t[:, k] / ||V_t[:, k]||,
        Vbar[:, k] = (D_k / ||V_t[:, k]||) (Lbar[:, k] - u_k (u_k . Lbar[:, k]))
      taubar_t = -sum_{i>=j} Vbar_ij (2 L~(t-1) T~)_ij
      Lbar(t-1) = tril(Vbar - tau_t Vbar (2 T~))
    """
    Tt = np.asarray(Tt, dtype=np.float64)
    n, N, _ = Tt.shape
    t_max = tau_t.shape[1]
    Lbar = np.zeros((n, N, N))
    Lbar[:, -1, :-1] = grad_soft / D[:, :-1]
    gtau = np.zeros((n, t_max))
    for t in range(t_max - 1, -1, -1):
        Lprev = Ls[t]
        G = gradient(Lprev, Tt)                       # tril(2 L T)
        V = Lprev - tau_t[:, t, None, None] * G
        nv = np.sqrt(np.sum(V * V, axis=1))           # [n, N]
        U = V / nv[:, None, :]
        proj = np.sum(U * Lbar, axis=1)               # [n, N]
        Vbar = (D / nv)[:, None, :] * (Lbar - U * proj[:, None, :])
        Vbar[:, :, -1] = 0.0
        Vbar = np.tril(Vbar)
        gtau[:, t] = -np.sum(Vbar * G, axis=(1, 2))
        Lbar = np.tril(Vbar - tau_t[:, t, None, None] * 2.0 * np.matmul(Vbar, Tt))
    return gtau


# ----------------------------------------------------------------------------------
# Table I: multiplications per iteration of the triangular array
# ----------------------------------------------------------------------------------
def table1_mults(constellation, U, t_max=1):
    """Real multiplications for t_max iterations as printed in Table I."""
    if constellation == "bpsk":
        return t_max * (U ** 3 / 3 + 5 * U ** 2 / 2 + 37 * U / 6 + 4)
    return t_max * (8 * U ** 3 / 3 + 10 * U ** 2 + 37 * U / 3 + 4)
