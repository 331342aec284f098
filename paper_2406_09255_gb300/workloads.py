"""Seeded synthetic workloads shaped like the paper's benchmarks.

This module holds only input generation: unique uniform keys, present/absent
query mixes, duplicate-heavy find-or-put streams, log-uniform batch sizes and
Poisson arrival times. It contains none of the hash-table method's arithmetic
(no table permutation, no slot layout) and is the one module that both the
CUDA path's tests and the CPU oracle's tests draw inputs from.

Keys are produced by a keyed bijection G_s on w-bit integers: a 4-round
balanced Feistel network whose round function is the splitmix64 finaliser
(Steele, Lea and Flood 2014), with cycle-walking for odd w. Key number i is
G_s(i'), where i' skips the single index that maps to 0, so keys are unique by
construction, uniform in [1, 2^w), and "absent" keys are simply those with an
index at or beyond the number inserted. Everything is written with int64 torch
ops (wrapping multiply, masked logical shifts) so the same code runs on the CPU
and on the GPU and gives identical values.
"""
from __future__ import annotations

import ctypes
import functools
import math
import os

import numpy as np
import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

#: per-workload seeds (workload number c -> base seed)
SEED_BASE = 0x2406_0925_5000


def _s64(x: int) -> int:
    """Unsigned 64-bit python int -> the int64 value with the same bits."""
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _u64(x: int) -> int:
    return x & MASK64


# --- scalar (python int) versions, used for inverses and cross-checks -------

def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def splitmix(seed: int, idx: int) -> int:
    return mix64(seed + (idx + 1) * GAMMA)


@functools.lru_cache(maxsize=4096)
def _round_keys(seed: int) -> tuple[int, ...]:
    return tuple(splitmix(seed ^ 0x5EED_0F_FE15, r) for r in range(4))


def _feistel_scalar(x: int, bits: int, rk: list[int], inverse: bool) -> int:
    h = bits // 2
    m = (1 << h) - 1
    L, R = x >> h, x & m
    if not inverse:
        for k in rk:
            L, R = R, L ^ (mix64(R + k) & m)
    else:
        for k in reversed(rk):
            L, R = R ^ (mix64(L + k) & m), L
    return (L << h) | R


def _walk_bits(w: int) -> int:
    return w + (w & 1)


def g_scalar(i: int, w: int, seed: int, inverse: bool = False) -> int:
    """G_s (or its inverse) on one w-bit value."""
    rk = _round_keys(seed)
    bits = _walk_bits(w)
    y = _feistel_scalar(i, bits, rk, inverse)
    while y >> w:
        y = _feistel_scalar(y, bits, rk, inverse)
    return y


# --- tensor versions --------------------------------------------------------

def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    if s == 0:
        return x
    return (x >> s) & ((1 << (64 - s)) - 1)


def mix64_t(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def _feistel_t(x: torch.Tensor, bits: int, rk: list[int]) -> torch.Tensor:
    h = bits // 2
    m = (1 << h) - 1
    L, R = _srl(x, h), x & m
    for k in rk:
        L, R = R, L ^ (mix64_t(R + _s64(k)) & m)
    return (L << h) | R


def _bijection_t(x: torch.Tensor, w: int, seed: int) -> torch.Tensor:
    """Cycle-walking Feistel bijection on [0, 2^w) applied elementwise."""
    rk = _round_keys(seed)
    bits = _walk_bits(w)
    y = _feistel_t(x, bits, rk)
    if bits != w:
        lim = 1 << w
        bad = y >= lim
        while bool(bad.any()):
            y = torch.where(bad, _feistel_t(y, bits, rk), y)
            bad = y >= lim
    return y


@functools.lru_cache(maxsize=4096)
def key_index_skip(w: int, seed: int) -> int:
    """The one index i with G_s(i) = 0; it is skipped when numbering keys."""
    return g_scalar(0, w, seed, inverse=True)


def unique_keys(start: int, count: int, key_bits: int, seed: int,
                device="cpu") -> torch.Tensor:
    """Keys number start .. start+count-1 of seed's key sequence (int64).

    Unique across all indices, uniform in [1, 2^key_bits)."""
    if count <= 0:
        return torch.empty(0, dtype=torch.int64, device=device)
    assert 2 <= key_bits <= 62
    assert start + count <= (1 << key_bits) - 1
    z = key_index_skip(key_bits, seed)
    idx = torch.arange(start, start + count, dtype=torch.int64, device=device)
    idx = idx + (idx >= z).to(torch.int64)
    return _bijection_t(idx, key_bits, seed)


def keys_at(indices: torch.Tensor, key_bits: int, seed: int) -> torch.Tensor:
    """Keys at arbitrary key indices (int64 tensor of indices)."""
    z = key_index_skip(key_bits, seed)
    idx = indices.to(torch.int64)
    idx = idx + (idx >= z).to(torch.int64)
    return _bijection_t(idx, key_bits, seed)


def permutation(n: int, seed: int, device="cpu", start: int = 0,
                count: int | None = None) -> torch.Tensor:
    """Entries start..start+count-1 of a seeded permutation of [0, n)."""
    if count is None:
        count = n - start
    if n <= 1:
        return torch.zeros(count, dtype=torch.int64, device=device)
    bits = max(2, math.ceil(math.log2(n)))
    rk_seed = seed ^ 0xB1_7EC7_10
    x = torch.arange(start, start + count, dtype=torch.int64, device=device)
    # cycle-walk on [0, 2^bits) until the value falls inside [0, n)
    rk = _round_keys(rk_seed)
    wb = _walk_bits(bits)
    y = _feistel_t(x, wb, rk)
    bad = y >= n
    while bool(bad.any()):
        y = torch.where(bad, _feistel_t(y, wb, rk), y)
        bad = y >= n
    return y


def find_queries(n_inserted: int, n_queries: int, hit_rate: float,
                 key_bits: int, seed: int, absent_base: int,
                 device="cpu", shuffle_seed: int | None = None
                 ) -> tuple[torch.Tensor, torch.Tensor]:
    """A shuffled mix of present and absent lookup keys.

    Keys come from the key sequence of `seed` (the one the table was filled
    from). floor(hit_rate * n_queries) queries are distinct inserted keys (key
    indices below n_inserted, chosen by a seeded permutation); the rest are
    distinct keys with indices from absent_base upward, which were never
    inserted. shuffle_seed (default: seed) only varies which keys are picked
    and their order. Returns (keys int64, expected_present bool)."""
    n_hit = int(math.floor(hit_rate * n_queries + 1e-9))
    assert n_hit <= n_inserted
    assert absent_base >= n_inserted
    ss = seed if shuffle_seed is None else shuffle_seed
    idx = torch.empty(n_queries, dtype=torch.int64, device=device)
    if n_hit:
        idx[:n_hit] = permutation(n_inserted, ss + 1, device, 0, n_hit)
    if n_queries - n_hit:
        idx[n_hit:] = torch.arange(absent_base, absent_base + n_queries - n_hit,
                                   dtype=torch.int64, device=device)
    present = torch.zeros(n_queries, dtype=torch.bool, device=device)
    present[:n_hit] = True
    pos = permutation(n_queries, ss + 2, device)
    q = torch.empty_like(idx)
    q[pos] = idx
    pr = torch.empty_like(present)
    pr[pos] = present
    return keys_at(q, key_bits, seed), pr


def to_u32(keys: torch.Tensor) -> torch.Tensor:
    """int64 keys < 2^32 -> int32 tensor holding the same 32 bits."""
    assert keys.dtype == torch.int64
    return (keys - ((keys >> 31) & 1) * (1 << 32)).to(torch.int32)


def duplicate_stream(n_ops: int, distinct: int, key_bits: int, seed: int,
                     dup_frac: float, device="cpu") -> torch.Tensor:
    """n_ops keys: `distinct` fresh keys plus duplicates of them, shuffled.

    Duplicates are uniform picks among the fresh keys. Used for multi-table
    find-or-put batches (a share of the keys repeats)."""
    fresh = unique_keys(0, distinct, key_bits, seed, device)
    n_dup = n_ops - distinct
    g = torch.Generator(device="cpu").manual_seed(seed & 0x7FFFFFFF)
    pick = torch.randint(0, max(distinct, 1), (max(n_dup, 0),), generator=g).to(device)
    allk = torch.cat([fresh, fresh[pick]]) if n_dup > 0 else fresh
    pos = permutation(len(allk), seed + 7, device)
    out = torch.empty_like(allk)
    out[pos] = allk
    return out


def zipf_recency_stream(n_ops: int, key_bits: int, seed: int, *,
                        fresh_frac: float = 0.5, zipf_s: float = 0.99,
                        find_frac: float = 0.2, rng_seed: int = 0,
                        max_distinct: int | None = None):
    """A model-checking-like operation stream (host side, numpy).

    Each op is a find-or-put (share 1 - find_frac) or a pure find. A share
    fresh_frac of keys are first-seen keys (next index of the key sequence);
    the rest repeat an already-seen key whose recency rank follows a Zipf(s)
    law (rank 1 = the most recently introduced key). Once max_distinct keys
    have been introduced, fresh draws become repeats.
    Returns (key_index int64 array, is_find bool array, distinct count)."""
    rng = np.random.default_rng(rng_seed)
    is_fresh = rng.random(n_ops) < fresh_frac
    is_find = rng.random(n_ops) < find_frac
    # fresh keys used by finds are lookups of never-inserted keys: they take a
    # separate index range so that they stay absent
    fop_fresh = is_fresh & ~is_find
    counter = np.cumsum(fop_fresh) - fop_fresh  # fresh index for this op
    if max_distinct is not None:
        over = fop_fresh & (counter >= max_distinct)
        is_fresh = is_fresh & ~over
        fop_fresh = fop_fresh & ~over
        counter = np.minimum(counter, max_distinct)
    n_seen = np.cumsum(fop_fresh) - fop_fresh  # keys introduced before this op
    # Zipf ranks (bounded by what has been seen); sample by inverse CDF on a
    # truncated harmonic approximation of the power law
    u = rng.random(n_ops)
    cap = np.maximum(n_seen, 1).astype(np.float64)
    a = 1.0 - zipf_s
    rank = np.floor(((cap ** a - 1.0) * u + 1.0) ** (1.0 / a)).astype(np.int64)
    rank = np.clip(rank, 1, np.maximum(n_seen, 1))
    rep_idx = n_seen - rank
    idx = np.where(fop_fresh, counter, rep_idx)
    absent_base = (1 << 40) if key_bits > 41 else (1 << (key_bits - 1))
    find_fresh = is_fresh & is_find
    idx = np.where(find_fresh, absent_base + np.arange(n_ops), idx)
    # before any key is seen, a repeat has nothing to repeat: make it a miss
    idx = np.where((~is_fresh) & (n_seen == 0), absent_base + np.arange(n_ops), idx)
    return idx.astype(np.int64), is_find, int(fop_fresh.sum())


def fop_stream(n_ops: int, key_bits: int, seed: int, *, fresh_frac: float = 0.5,
               zipf_s: float = 0.99, find_frac: float = 0.2, max_distinct: int | None = None,
               rng_seed: int = 0, device="cpu"):
    """The same model-checking-like stream as zipf_recency_stream, generated
    with torch on `device` (for streams of hundreds of millions of ops).

    Returns (keys int64, is_find bool, fresh_before int64): fresh_before[i] is
    the number of distinct keys introduced by find-or-puts before op i."""
    g = torch.Generator(device=device)
    g.manual_seed(rng_seed)
    is_find = torch.rand(n_ops, generator=g, device=device) < find_frac
    is_fresh = torch.rand(n_ops, generator=g, device=device) < fresh_frac
    fop_fresh = is_fresh & ~is_find
    counter = torch.cumsum(fop_fresh.to(torch.int64), 0) - fop_fresh.to(torch.int64)
    if max_distinct is not None:
        fop_fresh &= counter < max_distinct
        counter.clamp_(max=max_distinct)
    n_seen = counter  # keys introduced before this op
    u = torch.rand(n_ops, generator=g, device=device, dtype=torch.float64)
    a = 1.0 - zipf_s
    cap = n_seen.clamp(min=1).to(torch.float64)
    rank = torch.floor(((cap ** a - 1.0) * u + 1.0) ** (1.0 / a)).to(torch.int64)
    rank = torch.minimum(rank.clamp(min=1), n_seen.clamp(min=1))
    idx = torch.where(fop_fresh, counter, n_seen - rank)
    absent_base = 1 << (key_bits - 2)
    miss = (is_fresh & is_find) | ((~fop_fresh) & (n_seen == 0))
    idx = torch.where(miss, absent_base + torch.arange(n_ops, device=device), idx)
    return keys_at(idx, key_bits, seed), is_find, counter


def log_uniform_sizes(n: int, lo: int, hi: int, rng_seed: int) -> np.ndarray:
    rng = np.random.default_rng(rng_seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), n))).astype(np.int64).clip(lo, hi)


def poisson_arrivals(n: int, rate_per_s: float, rng_seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(rng_seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def multi_table_spec(count: int = 256, lo_exp: int = 8, hi_exp: int = 18,
                     min_batch: int = 1000, max_batch: int = 1_000_000,
                     distinct_frac: float = 0.7, slots_per_primary: int = 32,
                     slots_per_backyard: int = 32, fill_cap: float = 0.85,
                     rng_seed: int = SEED_BASE + 4):
    """Shape of a many-table find-or-put workload.

    Table i has 2^e_i primary buckets (e_i uniform in [lo_exp, hi_exp]) and
    2^(e_i - 3) secondary buckets, and receives one batch whose size is
    log-uniform in [min_batch, max_batch], capped so that its distinct keys
    (distinct_frac of the batch) stay below fill_cap of the table's slots.
    Returns a list of (primary_exp, batch_size, distinct) tuples."""
    rng = np.random.default_rng(rng_seed)
    exps = rng.integers(lo_exp, hi_exp + 1, count)
    sizes = log_uniform_sizes(count, min_batch, max_batch, rng_seed + 1)
    out = []
    for e, s in zip(exps, sizes):
        slots = (1 << int(e)) * slots_per_primary + (1 << (int(e) - 3)) * slots_per_backyard
        cap = int(fill_cap * slots / distinct_frac)
        s = int(min(s, cap))
        out.append((int(e), s, int(distinct_frac * s)))
    return out


# --- request keys of the served benchmark -----------------------------------
# A request's keys are n_fresh keys at consecutive indices from fresh_base,
# then n - n_fresh re-queries: index floor(h * re_hi / 2^64) with h the j-th
# output of the splitmix64 sequence of re_seed (j = 0, 1, ...), or, when
# re_hi is 0 (a table with nothing given yet), consecutive indices from
# miss_base. Keys are G_s at those indices (keys_at). The same definition is
# computed here with torch (request_keys) and on the device by the generator
# kernel of gen/keygen.cu (request_keys_device), so that a served run holds
# only the keys of admitted requests.

def _mulhi_small(h: torch.Tensor, m: int) -> torch.Tensor:
    """floor(h * m / 2^64) for int64 tensors h holding 64-bit unsigned bits
    and 0 <= m < 2^31."""
    assert 0 <= m < (1 << 31)
    h0 = h & 0xFFFFFFFF
    h1 = _srl(h, 32)
    t = h1 * m + _srl(h0 * m, 32)
    return _srl(t, 32)


def request_indices(n: int, n_fresh: int, fresh_base: int, re_hi: int, re_seed: int,
                    miss_base: int, device="cpu") -> torch.Tensor:
    """The key indices of one request (see above)."""
    fresh = torch.arange(fresh_base, fresh_base + n_fresh, dtype=torch.int64, device=device)
    n_re = n - n_fresh
    if n_re <= 0:
        return fresh
    j = torch.arange(n_re, dtype=torch.int64, device=device)
    if re_hi:
        h = mix64_t(_s64(re_seed) + (j + 1) * _s64(GAMMA))
        re = _mulhi_small(h, re_hi)
    else:
        re = miss_base + j
    return torch.cat([fresh, re])


def request_keys(n: int, n_fresh: int, fresh_base: int, re_hi: int, re_seed: int,
                 miss_base: int, key_bits: int, seed: int, device="cpu") -> torch.Tensor:
    """The keys of one request, computed with torch (int64)."""
    return keys_at(request_indices(n, n_fresh, fresh_base, re_hi, re_seed, miss_base, device),
                   key_bits, seed)


class _GenReq(ctypes.Structure):
    """One request descriptor of the device generator (gen/keygen.cu)."""
    _fields_ = [("out_off", ctypes.c_uint64), ("n", ctypes.c_uint64),
                ("n_fresh", ctypes.c_uint64), ("fresh_base", ctypes.c_uint64),
                ("re_hi", ctypes.c_uint64), ("re_seed", ctypes.c_uint64),
                ("miss_base", ctypes.c_uint64), ("rk", ctypes.c_uint64 * 4),
                ("skip", ctypes.c_uint64), ("key_bits", ctypes.c_int32), ("pad", ctypes.c_int32)]


_gen_lib = None


def _gen():
    global _gen_lib
    if _gen_lib is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libchtgen.so")
        if not os.path.exists(path):
            raise RuntimeError("libchtgen.so is missing: build the package first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        L.keygen_request_keys.restype = ctypes.c_int
        L.keygen_request_keys.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        assert L.keygen_req_bytes() == ctypes.sizeof(_GenReq)
        _gen_lib = L
    return _gen_lib


def request_keys_device(reqs: list, out: torch.Tensor, stream=None) -> None:
    """Write the keys of several requests into the int64 device tensor out.

    reqs: dicts with out_off (position in out, ascending), n, n_fresh,
    fresh_base, re_hi, re_seed, miss_base, key_bits, seed. One kernel launch
    per 128 requests, on stream (default: the current stream)."""
    import ctypes
    L = _gen()
    per = L.keygen_req_per_launch()
    s = stream if stream is not None else torch.cuda.current_stream(out.device)
    sms = torch.cuda.get_device_properties(out.device).multi_processor_count
    for i0 in range(0, len(reqs), per):
        part = reqs[i0: i0 + per]
        arr = (_GenReq * len(part))()
        for d, r in zip(arr, part):
            d.out_off, d.n, d.n_fresh = r["out_off"], r["n"], r["n_fresh"]
            d.fresh_base, d.re_hi = r["fresh_base"], r["re_hi"]
            d.re_seed, d.miss_base = _u64(r["re_seed"]), r["miss_base"]
            for k, v in enumerate(_round_keys(r["seed"])):
                d.rk[k] = v
            d.skip = key_index_skip(r["key_bits"], r["seed"])
            d.key_bits = r["key_bits"]
        base = part[0]["out_off"]
        total = part[-1]["out_off"] + part[-1]["n"] - base
        # positions are relative to the first request of this launch
        for d in arr:
            d.out_off -= base
        if total == 0:
            continue
        code = L.keygen_request_keys(ctypes.addressof(arr), len(part), total,
                                     out.data_ptr() + 8 * base, sms,
                                     ctypes.c_void_p(s.cuda_stream))
        if code:
            raise RuntimeError(f"request key generator launch failed (CUDA error {code})")
