"""Philox4x32-10, written from its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).  Test infrastructure only.

The step draws every random number from (key, counter) so that a decision replays
exactly and does not depend on thread order:

    key     = (seed low 32 bits, (seed high bits << 8 | purpose) mod 2^32)
    counter = (id low 32, id high 32, step, draw >> 2); word (draw & 3) of the output
    U       = ((word >> 8) + 0.5) * 2^-24            (exact in f32 and f64, never 0 or 1)
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# purposes of the draws (one key per purpose)
EMIT, PAIR, ION, SCAT, DFI, EVAP, SPUT = 1, 2, 3, 4, 5, 6, 7
# Cu2+ channels: scattering of double ionization; pairing, draws and scattering of the
# ionization of Cu+ (the Coulomb passes with Cu2+ keep their purposes in coulomb.py)
SCAT2, PAIR_IZ, ION_IZ, SCAT_IZ = 22, 23, 24, 25


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on a (broadcastable) batch of counters; returns 4 uint32 arrays."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    c = list(np.broadcast_arrays(*c))
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [(p1 >> _S32) ^ c[1] ^ np.uint64(k0),
             p1 & _MASK,
             (p0 >> _S32) ^ c[3] ^ np.uint64(k1),
             p0 & _MASK]
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return [x.astype(np.uint32) for x in c]


def key_of(seed, purpose):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (((seed >> 32) << 8) | int(purpose)) & 0xFFFFFFFF


def words(seed, purpose, ident, step, draw):
    """uint32 word `draw` of the stream (purpose, ident, step).  Arrays broadcast."""
    ident = np.asarray(ident, dtype=np.uint64)
    draw = np.asarray(draw, dtype=np.uint64)
    k0, k1 = key_of(seed, purpose)
    out = philox4x32_10(ident & _MASK, ident >> _S32, np.uint64(int(step) & 0xFFFFFFFF),
                        draw >> np.uint64(2), k0, k1)
    sel = (draw & np.uint64(3)).astype(np.int64)
    stacked = np.stack(np.broadcast_arrays(*out), axis=0)
    sel = np.broadcast_to(sel, stacked.shape[1:])
    return np.take_along_axis(stacked, sel[None], axis=0)[0]


def uniform(seed, purpose, ident, step, draw):
    """U in (0,1) with 24 random bits, as float64 (exactly representable in float32)."""
    w = words(seed, purpose, ident, step, draw).astype(np.uint64)
    return ((w >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0 ** -24


def uniform_index(seed, purpose, ident, step, draw, n):
    """floor(U * n) computed exactly in integers: ((2 (w>>8) + 1) n) >> 25."""
    w = words(seed, purpose, ident, step, draw).astype(np.uint64)
    u24 = w >> np.uint64(8)
    return (((np.uint64(2) * u24 + np.uint64(1)) * np.asarray(n, dtype=np.uint64)) >> np.uint64(25)).astype(np.int64)
