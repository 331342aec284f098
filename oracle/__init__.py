"""Sequential CPU oracle for compact cuckoo and compact iceberg hash tables.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It wraps the plain C
restatement of the paper's algorithms in ``oracle.c`` (Algorithm 4 and the
Section 4.4 lookup for cuckoo, Algorithm 5 and the Section 2.3 lookup for
iceberg, enumeration by k = pi^-1(a . r) of Section 2.4) and shares no code with
the CUDA library.

Parity status per function (see the tests that pin each one):
  perm / perm_inv / address / remainder: pinned by brute-force bijectivity over
      every key of a 16-bit space and by the round trip of Section 2.4; the
      round function itself is a design reading (Section 4.3 does not fix it).
  prec: pinned by the worked ranks of the slot-ordering figure (Appendix A).
  iceberg_fop: pinned by Theorem 1 (a)-(e) on brute-force tiny tables and by
      agreement with an independent restatement of Algorithm 1.
  cuckoo_insert / cuckoo_find: pinned by set semantics on brute-force tiny
      tables, the H=1 closed form (a plain bucketed table), and the exhaustive
      lookup.
  check_prefix / check_entries / check_order_property / check_cuckoo_chain /
      check_duplicates: pinned by hand-built tables that break one invariant
      a known number of times (exact counts) and by a plain restatement of
      Definition 1 on perturbed tables.
  insert_concurrent (host-threaded model of the packed-word claim): pinned by
      equality with the sequential operations on one thread and by Theorem 1
      and key conservation under real races on many threads.
  A mutation check plants plausible mistakes in all of the above; each is
  caught by these pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NOT_FOUND, FOUND, PUT, FULL, INVALID = 0, 1, 2, 3, 4
CUCKOO, ICEBERG = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with the host C compiler."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                           "-pthread", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


class Cfg(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("compact", ctypes.c_int),
        ("key_bits", ctypes.c_int),
        ("num_hashes", ctypes.c_int),
        ("max_chain", ctypes.c_int),
        ("wpb", ctypes.c_int),
        ("fpw", ctypes.c_int * 2),
        ("nb", ctypes.c_uint64 * 2),
        ("seed", ctypes.c_uint64),
        ("stash", ctypes.c_uint64),
    ]


_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_cfgp = ctypes.POINTER(Cfg)
_sz = ctypes.c_size_t


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, i = ctypes.c_uint64, ctypes.c_int
            sig = {
                "orc_cfg_check": (i, [_cfgp]),
                "orc_perm": (u64, [_cfgp, i, i, u64]),
                "orc_perm_inv": (u64, [_cfgp, i, i, u64]),
                "orc_address": (u64, [_cfgp, i, i, u64]),
                "orc_remainder": (u64, [_cfgp, i, i, u64]),
                "orc_key_from": (u64, [_cfgp, i, i, u64, u64]),
                "orc_perm_many": (None, [_cfgp, i, i, _u64p, _sz, _u64p, _u64p, _u64p, _u64p]),
                "orc_prec": (i, [i, i, i, i]),
                "orc_table_words": (u64, [_cfgp, i]),
                "orc_slots_per_bucket": (i, [_cfgp, i]),
                "orc_get_slot": (u64, [_cfgp, i, _u64p, u64, i]),
                "orc_cuckoo_insert": (None, [_cfgp, _u64p, _u64p, _sz, _u8p, _u64p, _u64p, _u64p]),
                "orc_cuckoo_find": (None, [_cfgp, _u64p, _u64p, _sz, _u8p, _u64p]),
                "orc_cuckoo_find_exhaustive": (None, [_cfgp, _u64p, _u64p, _sz, _u8p]),
                "orc_iceberg_fop": (None, [_cfgp, _u64p, _u64p, _u64p, _sz, _u8p, _u64p, _u64p]),
                "orc_iceberg_find": (None, [_cfgp, _u64p, _u64p, _u64p, _sz, _u8p, _u64p]),
                "orc_enumerate": (u64, [_cfgp, _u64p, _u64p, _u64p, u64]),
                "orc_iceberg_locate": (None, [_cfgp, _u64p, _u64p, _u64p, _sz, _u64p]),
                "orc_check_prefix": (u64, [_cfgp, i, _u64p]),
                "orc_check_entries": (u64, [_cfgp, _u64p, _u64p]),
                "orc_check_order_property": (u64, [_cfgp, _u64p, _u64p]),
                "orc_check_cuckoo_chain": (u64, [_cfgp, _u64p]),
                "orc_check_duplicates": (u64, [_cfgp, _u64p, _u64p]),
                "orc_check_stash": (u64, [_cfgp, _u64p, _u64p]),
                "orc_stash_home": (u64, [_cfgp, u64]),
                "orc_set_slot": (None, [_cfgp, i, _u64p, u64, i, u64]),
                "orc_entry_of": (u64, [_cfgp, i, u64]),
                "orc_bucket_of": (u64, [_cfgp, i, u64]),
                "orc_concurrent_insert": (i, [_cfgp, _u64p, _u64p, _u64p, _sz, _u8p, _u64p, i,
                                              _u64p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _p8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u8p)


def _keys(keys) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(keys).astype(np.uint64))


def make_cfg(kind: int, key_bits: int, nb0: int, nb1: int = 0, *,
             compact: bool = True, fpw0: int = 1, fpw1: int = 1, wpb: int = 16,
             num_hashes: int = 3, max_chain: int = 128, seed: int = 0, stash: int = 0) -> Cfg:
    c = Cfg()
    c.kind, c.compact, c.key_bits = kind, int(compact), key_bits
    c.num_hashes, c.max_chain, c.wpb = num_hashes, max_chain, wpb
    c.fpw[0], c.fpw[1] = fpw0, (fpw1 if kind == ICEBERG else 1)
    c.nb[0], c.nb[1] = nb0, (nb1 if kind == ICEBERG else 0)
    c.seed = seed & 0xFFFFFFFFFFFFFFFF
    c.stash = stash if kind == ICEBERG else 0
    return c


def check_cfg(*args, **kw) -> int:
    """0 if the configuration (same arguments as Table) is usable."""
    return int(lib().orc_cfg_check(ctypes.byref(make_cfg(*args, **kw))))


class Table:
    """A host-resident table of either kind, operated on sequentially.

    kind: CUCKOO or ICEBERG. compact: quotiented remainders (True) or whole
    keys in 64-bit slots. nb0 / nb1: bucket counts of level 0 (the cuckoo
    table or iceberg primary) and level 1 (iceberg secondary). fpw0 / fpw1:
    fields per 64-bit word. wpb: 64-bit words per bucket (16 = 128 bytes).
    stash: iceberg level-3 overflow slots (0 = none, else a power of two),
    kept after the secondary level in t1.
    """

    def __init__(self, kind: int, key_bits: int, nb0: int, nb1: int = 0, *,
                 compact: bool = True, fpw0: int = 1, fpw1: int = 1, wpb: int = 16,
                 num_hashes: int = 3, max_chain: int = 128, seed: int = 0, stash: int = 0):
        c = make_cfg(kind, key_bits, nb0, nb1, compact=compact, fpw0=fpw0, fpw1=fpw1,
                     wpb=wpb, num_hashes=num_hashes, max_chain=max_chain, seed=seed,
                     stash=stash)
        self.cfg = c
        self._cp = ctypes.byref(c)
        L = lib()
        err = int(L.orc_cfg_check(self._cp))
        if err:
            raise ValueError(f"oracle: invalid table configuration (check {err})")
        self.t0 = np.zeros(int(L.orc_table_words(self._cp, 0)), dtype=np.uint64)
        n1 = int(L.orc_table_words(self._cp, 1)) if kind == ICEBERG else 0
        self.t1 = np.zeros(max(n1, 1), dtype=np.uint64)
        self.probes = 0
        self.writes = 0

    # -- permutation -------------------------------------------------------
    def perm(self, level: int, j: int, k: int) -> int:
        return int(lib().orc_perm(self._cp, level, j, k))

    def perm_inv(self, level: int, j: int, p: int) -> int:
        return int(lib().orc_perm_inv(self._cp, level, j, p))

    def address(self, level: int, j: int, k: int) -> int:
        return int(lib().orc_address(self._cp, level, j, k))

    def remainder(self, level: int, j: int, k: int) -> int:
        return int(lib().orc_remainder(self._cp, level, j, k))

    def key_from(self, level: int, j: int, a: int, r: int) -> int:
        return int(lib().orc_key_from(self._cp, level, j, a, r))

    def perm_many(self, level: int, j: int, keys):
        """Vectorised (perm, address, remainder, perm_inv(perm)) over keys."""
        k = _keys(keys)
        outs = [np.zeros(len(k), dtype=np.uint64) for _ in range(4)]
        lib().orc_perm_many(self._cp, level, j, _p64(k), len(k), *[_p64(o) for o in outs])
        return tuple(outs)

    def slots_per_bucket(self, level: int) -> int:
        return int(lib().orc_slots_per_bucket(self._cp, level))

    def slot(self, level: int, bucket: int, y: int) -> int:
        t = self.t0 if level == 0 else self.t1
        return int(lib().orc_get_slot(self._cp, level, _p64(t), bucket, y))

    def set_slot(self, level: int, bucket: int, y: int, value: int) -> None:
        """Overwrite one slot (tests plant invariant violations with it)."""
        t = self.t0 if level == 0 else self.t1
        lib().orc_set_slot(self._cp, level, _p64(t), bucket, y, value)

    def entry_of(self, x: int, k: int) -> int:
        """Encoded entry of key k under choice x (cuckoo: hash index j;
        iceberg: 0 primary, 1 / 2 the secondary choices)."""
        return int(lib().orc_entry_of(self._cp, x, k))

    def bucket_of(self, x: int, k: int) -> int:
        """Bucket of key k under choice x (same x as entry_of)."""
        return int(lib().orc_bucket_of(self._cp, x, k))

    # -- operations --------------------------------------------------------
    def insert(self, keys):
        """Cuckoo: Algorithm 4 per key. Iceberg: find-or-put. Returns
        (status, dropped) for cuckoo and status for iceberg."""
        k = _keys(keys)
        st = np.zeros(len(k), dtype=np.uint8)
        p, w = ctypes.c_uint64(0), ctypes.c_uint64(0)
        if self.cfg.kind == CUCKOO:
            dr = np.zeros(len(k), dtype=np.uint64)
            lib().orc_cuckoo_insert(self._cp, _p64(self.t0), _p64(k), len(k), _p8(st),
                                    _p64(dr), ctypes.byref(p), ctypes.byref(w))
            self.probes, self.writes = p.value, w.value
            return st, dr
        lib().orc_iceberg_fop(self._cp, _p64(self.t0), _p64(self.t1), _p64(k), len(k),
                              _p8(st), ctypes.byref(p), ctypes.byref(w))
        self.probes, self.writes = p.value, w.value
        return st

    def find_or_put(self, keys):
        assert self.cfg.kind == ICEBERG
        return self.insert(keys)

    def insert_concurrent(self, keys, threads: int):
        """The host-threaded model: the kind's write operation (iceberg
        find-or-put, cuckoo put) on `threads` threads at once, with
        field-level compare-and-swap claims on packed words. Returns (status,
        dropped, threads that ran concurrently, lost compare-and-swaps);
        status 5 marks a key whose bounded retry gave up."""
        k = _keys(keys)
        st = np.zeros(len(k), dtype=np.uint8)
        dr = np.zeros(len(k), dtype=np.uint64)
        fails = ctypes.c_uint64(0)
        ran = lib().orc_concurrent_insert(self._cp, _p64(self.t0), _p64(self.t1), _p64(k),
                                          len(k), _p8(st), _p64(dr), threads,
                                          ctypes.byref(fails))
        if ran < 0:
            raise ValueError("oracle: bad arguments to the threaded model")
        return st, dr, int(ran), int(fails.value)

    def find(self, keys):
        k = _keys(keys)
        st = np.zeros(len(k), dtype=np.uint8)
        p = ctypes.c_uint64(0)
        if self.cfg.kind == CUCKOO:
            lib().orc_cuckoo_find(self._cp, _p64(self.t0), _p64(k), len(k), _p8(st),
                                  ctypes.byref(p))
        else:
            lib().orc_iceberg_find(self._cp, _p64(self.t0), _p64(self.t1), _p64(k), len(k),
                                   _p8(st), ctypes.byref(p))
        self.probes = p.value
        return st

    def locate(self, keys) -> np.ndarray:
        """Slot index of each key (iceberg): a * B0 + y at level 0,
        nb0 * B0 + a * B1 + y at level 1; 2^64 - 1 if absent or invalid."""
        assert self.cfg.kind == ICEBERG
        k = _keys(keys)
        out = np.zeros(len(k), dtype=np.uint64)
        lib().orc_iceberg_locate(self._cp, _p64(self.t0), _p64(self.t1), _p64(k), len(k),
                                 _p64(out))
        return out

    def find_exhaustive(self, keys):
        assert self.cfg.kind == CUCKOO
        k = _keys(keys)
        st = np.zeros(len(k), dtype=np.uint8)
        lib().orc_cuckoo_find_exhaustive(self._cp, _p64(self.t0), _p64(k), len(k), _p8(st))
        return st

    def enumerate(self) -> np.ndarray:
        L = lib()
        n = int(L.orc_enumerate(self._cp, _p64(self.t0), _p64(self.t1), None, 0))
        out = np.zeros(max(n, 1), dtype=np.uint64)
        L.orc_enumerate(self._cp, _p64(self.t0), _p64(self.t1), _p64(out), n)
        return out[:n]

    # -- invariants --------------------------------------------------------
    def check_prefix(self) -> int:
        L = lib()
        bad = int(L.orc_check_prefix(self._cp, 0, _p64(self.t0)))
        if self.cfg.kind == ICEBERG:
            bad += int(L.orc_check_prefix(self._cp, 1, _p64(self.t1)))
        return bad

    def check_entries(self) -> int:
        return int(lib().orc_check_entries(self._cp, _p64(self.t0), _p64(self.t1)))

    def check_order_property(self) -> int:
        assert self.cfg.kind == ICEBERG
        return int(lib().orc_check_order_property(self._cp, _p64(self.t0), _p64(self.t1)))

    def check_cuckoo_chain(self) -> int:
        assert self.cfg.kind == CUCKOO
        return int(lib().orc_check_cuckoo_chain(self._cp, _p64(self.t0)))

    def check_duplicates(self) -> int:
        return int(lib().orc_check_duplicates(self._cp, _p64(self.t0), _p64(self.t1)))

    def check_stash(self) -> int:
        return int(lib().orc_check_stash(self._cp, _p64(self.t0), _p64(self.t1)))

    def stash_home(self, k: int) -> int:
        return int(lib().orc_stash_home(self._cp, k))

    @property
    def stash(self) -> np.ndarray:
        """The level-3 stash (whole keys, 0 = empty), a view into t1."""
        c = self.cfg
        off = c.nb[1] * c.wpb
        return self.t1[off: off + c.stash]

    def check_prefix_level(self, level: int) -> int:
        t = self.t0 if level == 0 else self.t1
        return int(lib().orc_check_prefix(self._cp, level, _p64(t)))

    def load_words(self, t0: np.ndarray, t1: np.ndarray | None = None):
        """Replace the table contents with a dump (e.g. of a device table)."""
        self.t0[:] = np.asarray(t0, dtype=np.uint64).reshape(-1)[: len(self.t0)]
        if t1 is not None and self.cfg.kind == ICEBERG:
            self.t1[:] = np.asarray(t1, dtype=np.uint64).reshape(-1)[: len(self.t1)]


def prec(x1: int, y1: int, x2: int, y2: int) -> bool:
    """Definition 1: (x1, y1) strictly precedes (x2, y2)."""
    return bool(lib().orc_prec(x1, y1, x2, y2))
