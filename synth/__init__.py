"""Seeded synthetic workloads for TASER detection experiments.

This module only draws random channels, symbols and noise (numpy PCG64, or a seeded
torch generator on the GPU for workloads that need fresh instances at every step); it
holds none of the detector's arithmetic, so both the FP64 oracle and the CUDA path can
consume the same inputs.

Models (Sec. II-A and II-B of the paper):
  * MU-MIMO uplink  y = H s + n,  H i.i.d. CN(0, 1), n i.i.d. CN(0, N0),
    N0 = U / SNR with unit-energy symbols (BPSK +-1, QPSK (+-1 +-j)/sqrt 2).
  * SIMO block fading  Y = h s^H + N over K slots, h ~ CN(0, I_B) constant over the
    slots, slot 0 a known pilot (+1 for BPSK, (1 + j)/sqrt2 for QPSK), N0 = 1 / SNR per
    receive antenna.

Arrays are complex64 (what the C-ABI consumes). Bits are returned as +-1 int8.
"""
import numpy as np

__all__ = ["rng_for", "make_mimo", "make_jed", "make_uneven", "UNEVEN_SHAPES", "make_mimo_device"]


def rng_for(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _cn(rng, shape):
    """i.i.d. CN(0, 1) samples, complex128."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def _pm1(rng, shape):
    return (rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1).astype(np.int8)


def make_mimo(n, B, U, snr_db, constellation="qpsk", seed=0):
    """n independent MU-MIMO instances with B receive antennas and U users.

    snr_db: scalar or per-instance array. Returns a dict with
      H  complex64 [n, B, U], y complex64 [n, B],
      bits_re, bits_im  int8 [n, U] (+-1; bits_im is zero for BPSK),
      N0 float64 [n], snr_db float64 [n].
    """
    if constellation not in ("bpsk", "qpsk"):
        raise ValueError("constellation must be 'bpsk' or 'qpsk'")
    rng = rng_for(seed)
    snr_db = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (n,)).copy()
    H = _cn(rng, (n, B, U))
    bits_re = _pm1(rng, (n, U))
    if constellation == "qpsk":
        bits_im = _pm1(rng, (n, U))
        s = (bits_re + 1j * bits_im) / np.sqrt(2.0)
    else:
        bits_im = np.zeros((n, U), dtype=np.int8)
        s = bits_re.astype(np.complex128)
    N0 = U / 10.0 ** (snr_db / 10.0)
    noise = _cn(rng, (n, B)) * np.sqrt(N0)[:, None]
    y = np.einsum("nbu,nu->nb", H, s) + noise
    return {
        "H": np.ascontiguousarray(H.astype(np.complex64)),
        "y": np.ascontiguousarray(y.astype(np.complex64)),
        "bits_re": bits_re,
        "bits_im": bits_im,
        "N0": N0,
        "snr_db": snr_db,
        "constellation": constellation,
        "B": B,
        "U": U,
    }


def make_jed(n, B, K, snr_db, seed=0, constellation="bpsk"):
    """n independent SIMO JED instances over K slots, Y = h s^H + noise (slot 0 is the pilot).

    BPSK: s int8 [n, K] of +-1 with s[:, 0] == +1.
    QPSK: s complex [n, K] of (+-1 +-j)/sqrt2 with s[:, 0] == (1 + j)/sqrt2, plus bits_re,
          bits_im int8 [n, K] (the signs of its real and imaginary parts).
    Returns Y complex64 [n, B, K], s, N0, snr_db (N0 = 1/SNR per receive antenna).
    """
    rng = rng_for(seed)
    snr_db = np.broadcast_to(np.asarray(snr_db, dtype=np.float64), (n,)).copy()
    h = _cn(rng, (n, B))
    out = {}
    if constellation == "bpsk":
        s = _pm1(rng, (n, K))
        s[:, 0] = 1
        sym = s.astype(np.float64)
        out["s"] = s
    elif constellation == "qpsk":
        bits_re = _pm1(rng, (n, K))
        bits_im = _pm1(rng, (n, K))
        bits_re[:, 0] = 1
        bits_im[:, 0] = 1
        sym = (bits_re + 1j * bits_im) / np.sqrt(2.0)
        out.update(s=sym, bits_re=bits_re, bits_im=bits_im)
    else:
        raise ValueError(constellation)
    N0 = 1.0 / 10.0 ** (snr_db / 10.0)
    noise = _cn(rng, (n, B, K)) * np.sqrt(N0)[:, None, None]
    Y = h[:, :, None] * np.conj(sym)[:, None, :] + noise
    out.update(Y=np.ascontiguousarray(Y.astype(np.complex64)), N0=N0, snr_db=snr_db, B=B, K=K,
               constellation=constellation)
    return out


# (B, U) pairs of the uneven QPSK batch: N = 2U + 1 = 9, 17, 33, 65.
UNEVEN_SHAPES = ((32, 4), (64, 8), (128, 16), (256, 32))


def make_uneven(n, seed=0, shapes=UNEVEN_SHAPES, snr_range=(4.0, 16.0), t_max_choices=(10, 20)):
    """Item list of an uneven QPSK batch: per item a shape index, an SNR and a t_max.

    Returns dict with shape_idx int32 [n], snr_db float64 [n], t_max int32 [n] and the
    per-shape instance payloads generated per shape with derived seeds.
    """
    rng = rng_for(seed)
    shape_idx = rng.integers(0, len(shapes), size=n).astype(np.int32)
    snr_db = rng.uniform(snr_range[0], snr_range[1], size=n)
    t_max = np.asarray(t_max_choices, dtype=np.int32)[rng.integers(0, len(t_max_choices), size=n)]
    per_shape = []
    for si, (B, U) in enumerate(shapes):
        sel = np.nonzero(shape_idx == si)[0]
        w = make_mimo(len(sel), B, U, snr_db[sel], "qpsk", seed=seed * 7919 + 101 + si)
        w["items"] = sel
        per_shape.append(w)
    return {"shape_idx": shape_idx, "snr_db": snr_db, "t_max": t_max, "per_shape": per_shape,
            "shapes": tuple(shapes)}


def make_mimo_device(n, B, U, snr_db, constellation="qpsk", seed=0, device="cuda", generator=None):
    """make_mimo's recipe drawn on a CUDA device with a seeded torch generator, for
    workloads that need fresh instances at every step (a different random stream from
    make_mimo's PCG64, same distributions).

    snr_db: a scalar, or a (lo, hi) pair for SNRs drawn uniformly per instance.  generator:
    a torch CUDA generator to draw from (then `seed` is unused; its state advances, which
    also keeps the draw capturable in a CUDA graph with the default generator), or None for
    a fresh generator seeded with `seed`.  Returns H complex64 [n, B, U], y complex64 [n, B]
    and the transmitted signs int8 [n, M] in decision order (BPSK: M = U; QPSK: real parts
    then imaginary parts, M = 2U), all on the device.
    """
    import torch
    if constellation not in ("bpsk", "qpsk"):
        raise ValueError("constellation must be 'bpsk' or 'qpsk'")
    if generator is not None:
        gen = generator
    else:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
    half = 0.5 ** 0.5

    def cn(shape):
        return torch.view_as_complex(torch.normal(0.0, half, tuple(shape) + (2,), generator=gen, device=device))

    if isinstance(snr_db, (tuple, list)):
        lo, hi = snr_db
        snr = lo + (hi - lo) * torch.rand((n,), generator=gen, device=device, dtype=torch.float64)
    else:
        snr = torch.full((n,), float(snr_db), device=device, dtype=torch.float64)
    H = cn((n, B, U))
    bre = torch.randint(0, 2, (n, U), generator=gen, device=device, dtype=torch.int8) * 2 - 1
    if constellation == "qpsk":
        bim = torch.randint(0, 2, (n, U), generator=gen, device=device, dtype=torch.int8) * 2 - 1
        s = torch.complex(bre.float(), bim.float()) * half
        truth = torch.cat([bre, bim], dim=1)
    else:
        s = torch.complex(bre.float(), torch.zeros_like(bre, dtype=torch.float32))
        truth = bre
    n0 = (U / 10.0 ** (snr / 10.0)).float()
    y = torch.bmm(H, s.unsqueeze(2)).squeeze(2) + cn((n, B)) * n0.sqrt()[:, None]
    return H.contiguous(), y.contiguous(), truth
