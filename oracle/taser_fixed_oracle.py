"""Fixed-point TASER oracle: the 14-bit datapath of the paper's VLSI designs, emulated
exactly in integer arithmetic (Sec. IV-B operation modes; Sec. IV-D fixed-point design
parameters and inverse square-root LUT).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or runs this
module: only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may use it.  It shares no code with the CUDA path.

What the paper fixes (Sec. IV-D): 14-bit fixed-point numbers; L~_ij and V_ij use 8
fraction bits except in the bottom row (row N), which uses 7; L~_NN sits in a register
with 5 fraction bits and stays constant (the hardware keeps L~_NN = D_NN, i.e. the
"fixed" L~_NN mode); the inverse square root of the squared column norm comes from a
LUT of 2^11 entries of 14 bits, 13 of them fraction bits, and the scale unit multiplies
it by D_jj (Sec. IV-A/B).

Readings where the paper is silent (F1-F7; the identifiers are shared with the
project's design notes):
  F1  Numbers are two's complement and saturate to [-2^13, 2^13 - 1].
  F2  Rounding to a narrower format is round-half-up on the integer grid:
      (a + 2^(k-1)) >> k with an arithmetic (flooring) shift.
  F3  T^ = 2 tau T~ uses 12 fraction bits (|T^_ij| <= 2 tau ||T~||_2 = 2 alpha < 2, so
      one integer bit suffices).  D_jj (j < N) uses the 8 fraction bits of the diagonal
      PEs it initialises; D_NN uses the 5 of the L~_NN register.  Inputs are quantised
      from the FP32 T~, D, tau: T^ from the FP32 product fl(2 tau) * T~_ij, then
      floor(x 2^f + 1/2) and saturation.
  F4  The MAC accumulates exactly (wide accumulator): row i < N accumulates at 20
      fraction bits, row N at 19 (the L~_NN T^_Nj term is aligned by 2 bits); V is the
      accumulator rounded to the PE's format and saturated.
  F5  The squared column norm is exact: sum over rows j..N of V_ij^2 at 16 fraction
      bits (the 7-bit bottom-row entry is aligned to 8 bits first).
  F6  The LUT is indexed after normalising the squared norm x = m 4^e with m in [1, 4):
      index i = floor(512 m) in [512, 2048) (the top 11 bits); the entry is the
      inverse square root at the bin centre, LUT[i] = round(2^13 / sqrt((i + 1/2)/512)).
      The power-of-two part 2^-e is applied as a shift.
  F7  The scale factor D_jj * LUT[i] is kept at full width with its shift; the PE product
      V_ij * scale is rounded once to the PE's format (F2) and saturated.
  Only mode "fixed" exists (the register holding L~_NN is constant); V_NN <= 0 is still
  flagged.  A saturation anywhere raises FLAG_SATURATED.

Integer ranges (default formats): |L~|, |V|, |T^| <= 2^13, so every product is below
2^26 and every accumulator below 2^33; int64 is exact.  Wider formats (used by the pins
to compare with the FP64 oracle) switch to Python integers.

Parity status: pinned by tests/test_fixed_oracle_pins.py -- the LUT against exact
integer rounding, the datapath against the FP64 oracle at wide formats, invariants, and
the paper's own statement that the fixed-point design loses little against floating
point (Sec. V-A).
"""
import numpy as np

FLAG_ZERO_COLUMN = 1 << 2
FLAG_LNN_SIGN = 1 << 3
FLAG_SATURATED = 1 << 5

# Sec. IV-D, with the readings above.
PAPER_FORMATS = dict(bits=14, frac_l=8, frac_last=7, frac_lnn=5, frac_t=12, lut_index_bits=11, lut_frac=13)


def _dtype(fmt):
    """int64 when every intermediate provably fits, else Python integers."""
    wide = max(fmt["frac_l"], fmt["frac_last"], fmt["frac_lnn"]) + fmt["frac_t"] + 2 * (fmt["bits"] - 14)
    return np.int64 if (wide <= 24 and fmt["bits"] <= 16 and fmt["lut_frac"] <= 16) else object


def round_shift(a, k):
    """round(a / 2^k), ties toward +infinity, for integer arrays a and k >= 0 (F2)."""
    if k == 0:
        return a
    return (a + (1 << (k - 1))) >> k


def saturate(a, bits):
    """Clip to the two's complement range of `bits` bits; returns (a, saturated mask) (F1)."""
    lo, hi = -(1 << (bits - 1)), (1 << (bits - 1)) - 1
    sat = (a < lo) | (a > hi)
    return np.where(a < lo, lo, np.where(a > hi, hi, a)), sat


def quantize(x, frac, bits, dtype):
    """Float -> integer code: floor(x 2^frac + 1/2), saturated; NaN -> 0 (saturated) (F3)."""
    x = np.asarray(x, dtype=np.float64)
    v = np.floor(x * 2.0 ** frac + 0.5)
    nan = np.isnan(v)
    lim = float(1 << (bits - 1))
    sat = nan | (v < -lim) | (v > lim - 1)
    v = np.where(nan, 0.0, np.clip(v, -lim, lim - 1))
    out = v.astype(np.int64)
    if dtype is object:
        out = out.astype(object)
    return out, sat


def inverse_sqrt_lut(index_bits=11, frac=13):
    """F6: entries i in [2^(b-2), 2^b) stand for m = i / 2^(b-2) in [1, 4);
    LUT[i] = round(2^frac / sqrt((i + 1/2) / 2^(b-2))).  Entries below 2^(b-2) are unused (0)."""
    q = 1 << (index_bits - 2)
    i = np.arange(1 << index_bits, dtype=np.float64)
    lut = np.floor(2.0 ** frac / np.sqrt((i + 0.5) / q) + 0.5)
    lut[:q] = 0.0
    return lut.astype(np.int64)


def lut_index_and_shift(x, index_bits=11):
    """Normalise integer x >= 1 as m 2^s, s even, m in [1, 4) (F6).
    Returns (index floor(m 2^(b-2)), s)."""
    b = index_bits - 2
    idx = np.zeros(x.shape, dtype=np.int64)
    s = np.zeros(x.shape, dtype=np.int64)
    for pos, v in np.ndenumerate(x):
        v = int(v)
        if v <= 0:
            continue
        e = ((v.bit_length() - 1) // 2) * 2
        idx[pos] = (v >> (e - b)) if e >= b else (v << (b - e))
        s[pos] = e
    return idx, s


def quantize_inputs(Tt, D, tau, fmt=PAPER_FORMATS):
    """F3: T^ = Q(fl32(fl32(2 tau) T~)) with frac_t bits, d_j = Q(D_j) with frac_l bits
    (j < N), d_N = Q(D_N) with frac_lnn bits.  Inputs are the FP32 arrays the detector
    receives.  Returns (That [n,N,N], d [n,N], saturated [n])."""
    dt = _dtype(fmt)
    Tt = np.asarray(Tt, dtype=np.float32)
    D = np.asarray(D, dtype=np.float32)
    tau = np.asarray(tau, dtype=np.float32)
    two_tau = (tau + tau).astype(np.float32)                  # exact doubling in FP32
    prod = (two_tau[:, None, None] * Tt).astype(np.float32)     # IEEE single product
    That, st = quantize(prod, fmt["frac_t"], fmt["bits"], dt)
    dv, sd = quantize(D[:, :-1], fmt["frac_l"], fmt["bits"], dt)
    dn, sn = quantize(D[:, -1:], fmt["frac_lnn"], fmt["bits"], dt)
    d = np.concatenate([dv, dn], axis=1)
    sat = st.any(axis=(1, 2)) | sd.any(axis=1) | sn.any(axis=1)
    return That, d, sat


def taser_fixed(Tt, D, tau, t_max, fmt=PAPER_FORMATS):
    """Algorithm 1 on the fixed-point datapath (Sec. IV-B, Sec. IV-D; readings F1-F7).

    Inputs are the FP32 T~ [n,N,N], D [n,N], tau [n]; t_max >= 1.
    Returns dict with integer codes `L` [n,N,N] (row N at frac_last bits, L~_NN at
    frac_lnn bits, other rows at frac_l bits), their real values `L_real`, decisions
    `s_hat` int8 [n,N-1] and `flags` [n]."""
    if t_max < 1:
        raise ValueError("t_max must be >= 1")
    bits, fl, fN, fnn, ft = fmt["bits"], fmt["frac_l"], fmt["frac_last"], fmt["frac_lnn"], fmt["frac_t"]
    dt = _dtype(fmt)
    That, d, sat0 = quantize_inputs(Tt, D, tau, fmt)
    n, N, _ = That.shape
    lut = inverse_sqrt_lut(fmt["lut_index_bits"], fmt["lut_frac"])
    flags = np.where(sat0, FLAG_SATURATED, 0).astype(np.uint32)
    last = N - 1

    # Initialisation L~(0) = D (diagonal PEs take D_jj; the L~_NN register takes D_NN).
    L = np.zeros((n, N, N), dtype=dt)
    for j in range(N):
        L[:, j, j] = d[:, j]
    lnn = d[:, last].copy()
    below = np.tril(np.ones((N, N), dtype=bool))

    for _t in range(t_max):
        # Gradient step V = L~ - tril(L~ T^) in matrix-multiplication mode: the accumulator starts at L~_ij and the
        # products L~_ik T^_kj are subtracted; exact, at frac_l + frac_t bits (rows < N)
        # or frac_last + frac_t bits (row N, L~_NN term aligned) (F4).
        P = np.matmul(L, That)                                 # exact integer products
        acc = L * (1 << ft) - P
        # Row N: the k = N product used L~_NN at frac_lnn bits; align it to frac_last.
        acc[:, last, :] = (L[:, last, :] * (1 << ft)
                           - (P[:, last, :] - L[:, last, last, None] * That[:, last, :])
                           - (lnn[:, None] * That[:, last, :]) * (1 << (fN - fnn)))
        vnn_acc = (lnn * (1 << (ft + fN - fnn))
                   - (P[:, last, last] - L[:, last, last] * That[:, last, last])
                   - lnn * That[:, last, last] * (1 << (fN - fnn)))
        flags[np.asarray(vnn_acc <= 0, dtype=bool)] |= FLAG_LNN_SIGN
        acc[:, :, last] = 0                                      # L~_NN has no PE
        V, s1 = saturate(round_shift(acc, ft), bits)
        V = np.where(below, V, 0)
        sat = (s1 & below).any(axis=(1, 2))

        # Prox, squared-norm mode (exact, 2 frac_l bits; the bottom row aligned) (F5).
        Vn = V.copy()
        Vn[:, last, :] = Vn[:, last, :] * (1 << (fl - fN))
        x = np.sum(Vn[:, :, :last] * Vn[:, :, :last], axis=1)   # [n, N-1], rows j..N
        # Scale unit: LUT inverse square root times D_jj (F6, F7).
        idx, s = lut_index_and_shift(np.asarray(x, dtype=object), fmt["lut_index_bits"])
        zero = np.asarray(x == 0, dtype=bool)
        flags[zero.any(axis=1)] |= FLAG_ZERO_COLUMN
        c = np.where(zero, 0, d[:, :last] * lut[idx].astype(dt))
        # 1/sqrt(x 2^-2frac_l) D_j = d_j LUT[i] 2^-(lut_frac + s/2): one shift per column.
        sh = (fmt["lut_frac"] + s // 2).astype(dt)[:, None, :]
        # Scaling mode: every PE rounds V_ij * scale_j to its own format (F7).
        prod = V[:, :, :last] * c[:, None, :]
        q, s2 = saturate((prod + (np.ones_like(sh) << (sh - 1))) >> sh, bits)
        Lnew = np.zeros_like(L)
        Lnew[:, :, :last] = np.where(below[None, :, :last], q, 0)
        sat |= (s2 & below[None, :, :last]).any(axis=(1, 2))
        Lnew[:, last, last] = lnn                                # the constant register
        L = Lnew
        flags[sat] |= FLAG_SATURATED

    row = np.asarray(L[:, last, :last], dtype=np.int64)
    s_hat = np.where(row >= 0, 1, -1).astype(np.int8)
    frac = np.full((N, N), fl, dtype=np.int64)
    frac[last, :] = fN
    frac[last, last] = fnn
    L_real = np.asarray(L, dtype=np.float64) * np.exp2(-frac.astype(np.float64))
    return {"L": L, "L_real": L_real, "s_hat": s_hat, "flags": flags, "That": That, "d": d}
