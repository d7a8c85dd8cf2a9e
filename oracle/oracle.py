"""ctypes wrapper of the C oracle (blowchoc_oracle.c). Test infrastructure only.

The wrapper marshals numpy arrays; every step of the method runs in the C
file, which states each formula with its section or equation of the paper.
"""
import ctypes
import math

import numpy as np

from . import build as _build

COST_MIX, COST_LA, COST_EXP, COST_TABLE = 0, 1, 2, 3
GOLDEN_RATIO = (1.0 + math.sqrt(5.0)) / 2.0

_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    u64, u32, i32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    lib.orc_splitmix64_next.argtypes = [_u64p]
    lib.orc_splitmix64_next.restype = u64
    lib.orc_hash.argtypes = [u64, u64, u64]
    lib.orc_hash.restype = u64
    lib.orc_derive_multipliers.argtypes = [u64, u64, u32, u32, vp, vp]
    lib.orc_derive_multipliers.restype = i32
    lib.orc_cost.argtypes = [i32, dbl, u32, u32, u32]
    lib.orc_cost.restype = dbl
    lib.orc_bit_positions.argtypes = [vp, u32, u64, vp]
    lib.orc_bit_positions.restype = u32
    lib.orc_insert.argtypes = [vp, u64, u32, u32, i32, dbl, vp, vp, vp, u64, u64,
                               vp, _u64p, _u64p]
    lib.orc_insert.restype = i32
    lib.orc_query.argtypes = [vp, u64, u32, u32, vp, vp, vp, u64, vp, vp]
    lib.orc_query.restype = i32
    lib.orc_histogram.argtypes = [vp, u64, vp]
    lib.orc_histogram.restype = u64
    lib.orc_block_terms.argtypes = [vp, u64, vp, u32, u64,
                                    ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.orc_block_terms.restype = None
    lib.orc_set_cost_table.argtypes = [vp, u32]
    lib.orc_set_cost_table.restype = None
    lib.orc_set_bitsel.argtypes = [i32]
    lib.orc_set_bitsel.restype = None
    lib.orc_distinct_from_raw.argtypes = [vp, u32, vp]
    lib.orc_distinct_from_raw.restype = None
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64_next(state: int):
    """One splitmix64 step; returns (new_state, output)."""
    s = ctypes.c_uint64(state)
    out = _load().orc_splitmix64_next(ctypes.byref(s))
    return s.value, out


def hash_lin(a: int, x: int, b: int) -> int:
    """Linear hash of Section 3.4 (top bits / xor-fold / plain mod)."""
    return int(_load().orc_hash(a, x, b))


def cost(kind: int, param: float, k: int, j: int, a: int) -> float:
    """cost^MIX (Eq. 5), cost^LA (Eq. 6) or cost^EXP (Eq. 4) in double."""
    return float(_load().orc_cost(kind, param, k, j, a))


def derive_multipliers(seed: int, M: int, k: int, c: int, bitsel: int = 0):
    """Hash multipliers (a_1..a_c, a'_1..a'_k) drawn from the seed."""
    a_block = np.zeros(3, dtype=np.uint64)
    a_bit = np.zeros(32, dtype=np.uint64)
    _load().orc_set_bitsel(int(bitsel))
    rc = _load().orc_derive_multipliers(seed, M, k, c, _ptr(a_block), _ptr(a_bit))
    if rc != 0:
        raise ValueError("bad filter parameters")
    return a_block[:c].copy(), a_bit[:k].copy()


def bit_positions(a_bit, x: int, bitsel: int = 0):
    """Sorted distinct positions F(x) (Eq. 3)."""
    a_bit = np.ascontiguousarray(a_bit, dtype=np.uint64)
    out = np.zeros(32, dtype=np.uint32)
    _load().orc_set_bitsel(int(bitsel))
    n = _load().orc_bit_positions(_ptr(a_bit), len(a_bit), x, _ptr(out))
    return out[:n].copy()


def distinct_from_raw(raw):
    """Appendix B's shift rule on given raw values (raw[i] in [512 - i])."""
    raw = np.ascontiguousarray(raw, dtype=np.uint32)
    out = np.zeros(len(raw), dtype=np.uint32)
    _load().orc_distinct_from_raw(_ptr(raw), len(raw), _ptr(out))
    return out


class OracleFilter:
    """A BlowChoc filter held in host memory and updated by the C oracle.

    M blocks of 512 bits, k bit hashes, c choices, cost kind and parameter
    (sigma, mu or beta), batch size B of the batch-synchronous insertion
    (B = 1: the paper's sequential insertion).
    """

    def __init__(self, M, k, c, cost_kind=COST_EXP, cost_param=GOLDEN_RATIO,
                 seed=0, batch=1, a_block=None, a_bit=None, bitsel=0):
        self.M, self.k, self.c = int(M), int(k), int(c)
        self.cost_kind, self.cost_param = int(cost_kind), float(cost_param)
        self.batch = int(batch)
        self.bitsel = int(bitsel)
        if a_block is None:
            a_block, a_bit = derive_multipliers(seed, self.M, self.k, self.c, self.bitsel)
        self.a_block = np.zeros(3, dtype=np.uint64)
        self.a_block[:self.c] = a_block
        self.a_bit = np.zeros(32, dtype=np.uint64)
        self.a_bit[:self.k] = a_bit
        self.words = np.zeros(8 * self.M, dtype=np.uint64)
        self.inserted = 0
        self.skipped = 0

    def set_cost_table(self, table):
        """Use costs table[L * (k + 1) + a] (a table cost, e.g. a learned one)."""
        self.cost_kind = COST_TABLE
        self.table = np.ascontiguousarray(table, dtype=np.float64).copy()
        assert self.table.shape == (513 * (self.k + 1),)

    def insert(self, keys, batch=None, return_choices=False):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        _load().orc_set_bitsel(self.bitsel)
        if self.cost_kind == COST_TABLE:
            _load().orc_set_cost_table(_ptr(self.table), self.k)
        B = self.batch if batch is None else int(batch)
        n = len(keys)
        choices = np.empty(max(n, 1), dtype=np.int8) if return_choices else None
        ins, skp = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = _load().orc_insert(_ptr(self.words), self.M, self.k, self.c,
                                self.cost_kind, self.cost_param,
                                _ptr(self.a_block), _ptr(self.a_bit),
                                _ptr(keys), n, B,
                                _ptr(choices) if return_choices else None,
                                ctypes.byref(ins), ctypes.byref(skp))
        if rc != 0:
            raise ValueError("oracle insert failed")
        self.inserted += ins.value
        self.skipped += skp.value
        if return_choices:
            return choices[:n]
        return None

    def query(self, keys, return_first=False):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        _load().orc_set_bitsel(self.bitsel)
        n = len(keys)
        bitmap = np.zeros(max((n + 63) // 64, 1), dtype=np.uint64)
        first = np.zeros(max(n, 1), dtype=np.uint8) if return_first else None
        rc = _load().orc_query(_ptr(self.words), self.M, self.k, self.c,
                               _ptr(self.a_block), _ptr(self.a_bit), _ptr(keys), n,
                               _ptr(bitmap), _ptr(first) if return_first else None)
        if rc != 0:
            raise ValueError("oracle query failed")
        bitmap = bitmap[:(n + 63) // 64]
        if return_first:
            return bitmap, first[:n]
        return bitmap

    def histogram(self):
        """(hist[0..512], total set bits): blocks per load (Fig. 8)."""
        hist = np.zeros(513, dtype=np.uint64)
        total = _load().orc_histogram(_ptr(self.words), self.M, _ptr(hist))
        return hist, int(total)

    def block_terms(self, block, x):
        """(|F'|, |F(x) minus F'|) of block `block` for key x (Section 3.2)."""
        _load().orc_set_bitsel(self.bitsel)
        L, a = ctypes.c_uint32(0), ctypes.c_uint32(0)
        _load().orc_block_terms(_ptr(self.words), block, _ptr(self.a_bit), self.k, x,
                                ctypes.byref(L), ctypes.byref(a))
        return L.value, a.value

    def candidates(self, x):
        """Block addresses h_1(x)..h_c(x)."""
        return [hash_lin(int(self.a_block[i]), int(x), self.M) for i in range(self.c)]


def bits_of_bitmap(bitmap, n):
    """Unpack an LSB-first u64 bitmap into a bool array of length n."""
    b = np.ascontiguousarray(bitmap, dtype=np.uint64).view(np.uint8)
    return np.unpackbits(b, bitorder="little")[:n].astype(bool)
