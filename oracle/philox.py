"""Philox4x32-10 counter-based generator and the uniform draws built on it.

TEST INFRASTRUCTURE ONLY: this module is part of the CPU oracle. Only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.

The paper only says that each coordinate of a multi-index is drawn
independently from its factor's leverage-score distribution (proof of Thm 4.5,
"sample each coordinate independently"); it fixes no generator. The reading used
here (and, independently re-implemented, by the CUDA sampler):

* Generator: Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror and
  Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11). A round maps the
  counter (x0, x1, x2, x3) under key (k0, k1) to
  (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
  with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
  Weyl constants (0x9E3779B9, 0xBB67AE85) modulo 2^32.
* Key: (seed mod 2^32, seed >> 32 mod 2^32).
* Counter for draw t, Philox call k (one call serves two consecutive modes of the
  draw's mode list), factor row ``row`` (the Tucker factor-row index; 0 for a
  plain regression) and call id: (t mod 2^32, t >> 32, k + 256*row, call_id mod 2^32).
* Uniform from two 32-bit words (wa, wb): u = (((wa << 32) | wb) >> 11) * 2^-53,
  an exact double in [0, 1). Mode 2k uses words (w0, w1) of call k, mode 2k+1 uses
  (w2, w3).

Parity status: pinned by bit equality with NVIDIA's cuRAND Philox4_32_10 host
generator, run as a library on the CPU (its block j is Philox at counter
(j div 65536, 0, j mod 65536, 0) under key (seed lo, seed hi)), and by statistical
tests (uniformity, independence across modes).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_LO = np.uint64(0xFFFFFFFF)
_SH32 = np.uint64(32)
_SH11 = np.uint64(11)


def philox4x32_10(x0, x1, x2, x3, k0, k1):
    """Apply the 10-round Philox4x32 bijection to counters (arrays) under key (k0, k1).

    Returns four uint32 arrays. Arithmetic is done in uint64 so that the 32x32->64
    products are exact.
    """
    x0 = np.asarray(x0, dtype=np.uint64) & _LO
    x1 = np.asarray(x1, dtype=np.uint64) & _LO
    x2 = np.asarray(x2, dtype=np.uint64) & _LO
    x3 = np.asarray(x3, dtype=np.uint64) & _LO
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        y0 = (p1 >> _SH32) ^ x1 ^ np.uint64(k0)
        y1 = p1 & _LO
        y2 = (p0 >> _SH32) ^ x3 ^ np.uint64(k1)
        y3 = p0 & _LO
        x0, x1, x2, x3 = y0, y1, y2, y3
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def words_to_uniform(wa, wb):
    """53-bit uniform in [0, 1) from two 32-bit words (exact in binary64)."""
    v = (np.asarray(wa, dtype=np.uint64) << _SH32) | np.asarray(wb, dtype=np.uint64)
    return (v >> _SH11).astype(np.float64) * (2.0 ** -53)


def draw_uniforms(seed, call_id, t, n_modes, row=0):
    """Uniforms u[m, j] for draws t[j] and positions m = 0..n_modes-1 of the mode list.

    ``t`` is an array of non-negative draw indices (< 2^64).
    """
    t = np.asarray(t, dtype=np.uint64)
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    c0 = t & _LO
    c1 = t >> _SH32
    c3 = np.uint64(int(call_id) & 0xFFFFFFFF)
    out = np.empty((n_modes, t.shape[0]), dtype=np.float64)
    for k in range((n_modes + 1) // 2):
        c2 = np.uint64((k + 256 * int(row)) & 0xFFFFFFFF)
        w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, c3, k0, k1)
        out[2 * k] = words_to_uniform(w0, w1)
        if 2 * k + 1 < n_modes:
            out[2 * k + 1] = words_to_uniform(w2, w3)
    return out
