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
* Counter for draw t, Philox call k, factor row ``row`` (the Tucker factor-row
  index; 0 for a plain regression) and call id: (t mod 2^32, t >> 32, k + 256*row,
  call_id mod 2^32).
* Draws of 3 or 4 coordinates take ONE call (k = 0): its 128 bits, w0 first (most
  significant), are cut from the top into n chunks of floor(128 / n) bits (42 for
  n = 3, 32 for n = 4), and coordinate m's uniform is chunk_m * 2^-floor(128/n), an
  exact double on a grid of 2^-42 (2^-32) instead of 2^-53: it moves a row's
  probability by at most one grid step, far below any leverage-score difference that
  matters to the method, and saves a Philox evaluation per draw.
* Otherwise one call serves two consecutive coordinates: the uniform from two 32-bit
  words (wa, wb) is u = (((wa << 32) | wb) >> 11) * 2^-53, an exact double in [0, 1);
  coordinate 2k uses words (w0, w1) of call k, coordinate 2k+1 uses (w2, w3).

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


def one_call_chunks(w0, w1, w2, w3, n):
    """The n = 3 or 4 chunks (uint64 arrays) of floor(128 / n) bits cut from the top of
    the 128-bit value w0 w1 w2 w3 (w0 most significant)."""
    w = [np.asarray(v, dtype=np.uint64) for v in (w0, w1, w2, w3)]
    if n == 4:
        return w
    hi = (w[0] << _SH32) | w[1]
    lo = (w[2] << _SH32) | w[3]
    m42 = np.uint64((1 << 42) - 1)
    m22 = np.uint64((1 << 22) - 1)
    return [hi >> np.uint64(22), ((hi & m22) << np.uint64(20)) | (lo >> np.uint64(44)), (lo >> np.uint64(2)) & m42]


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
    if n_modes in (3, 4):
        c2 = np.uint64((256 * int(row)) & 0xFFFFFFFF)
        w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, c3, k0, k1)
        for m, c in enumerate(one_call_chunks(w0, w1, w2, w3, n_modes)):
            out[m] = c.astype(np.float64) * (2.0 ** -(128 // n_modes))
        return out
    for k in range((n_modes + 1) // 2):
        c2 = np.uint64((k + 256 * int(row)) & 0xFFFFFFFF)
        w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, c3, k0, k1)
        out[2 * k] = words_to_uniform(w0, w1)
        if 2 * k + 1 < n_modes:
            out[2 * k + 1] = words_to_uniform(w2, w3)
    return out
