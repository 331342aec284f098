// cht_device.cuh - device-side building blocks of the compact hash tables:
// the quotienting permutation (Section 2.4, Section 4.3), the packed bucket
// layout, cooperative-tile primitives (Section 4.1: Any / Count / First /
// Shuffle over a tile of T threads that owns one bucket) and the field-level
// compare-and-swap and swap used by Algorithms 1 and 4.
//
// Bucket layout: a bucket is WPB little-endian 64-bit words: 16 (128 bytes,
// one cache line, Section 4.5; the default), or 8 or 4 (64- or 32-byte
// buckets, the smaller bucket sizes of Section 5.1). A level stores fpw
// fields per word, each
// S = 64 / fpw bits wide; slot y is field y % fpw of word y / fpw. The
// all-zero field is EMPTY. Entries:
//   cuckoo            (body << 2) | (j + 1)   j = hash index (Section 2.2)
//   iceberg primary   (body << 1) | 1         one occupancy bit (Section 5.1)
//   iceberg secondary (body << 2) | (i + 1)   i = secondary choice (Algorithm 1)
// where body is the remainder r_j(k) for compact tables and k itself for
// whole-key tables.
//
// In a tile of T threads lane l owns words [l * W, l * W + W), W = WPB / T,
// i.e. slots [l * W * fpw, (l + 1) * W * fpw): slot order runs lane by lane,
// so "the first empty slot" is found with one ballot plus a local scan.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cht {

constexpr int kWordsPerBucket = 16;  // the default bucket: one 128-byte line
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// status bytes (mirror include/cht.h)
constexpr uint8_t ST_NOT_FOUND = 0, ST_FOUND = 1, ST_PUT = 2, ST_FULL = 3,
                  ST_INVALID = 4, ST_ERROR = 5;
// internal, never left in a caller's status array: an iceberg key whose
// level-1 step found its primary bucket full and that awaits level 2
constexpr uint8_t ST_PENDING = 6;

// bits of the table header's error word: a key reported ST_ERROR (a bounded
// retry loop gave up), or a kernel's loop bound ran out
constexpr uint32_t kErrRetry = 1u, kErrLoopBound = 2u;

// One level of a table (cuckoo table, iceberg primary or iceberg secondary).
struct Level {
    uint64_t *words;  // bucket b starts at words + 16 * b
    uint64_t nb;      // bucket count
    int n;            // address bits, ceil(log2 nb)
    int R;            // remainder bits, w - n
    int pow2;         // nb == 2^n
    int fpw;          // fields per word (also a template parameter)
    uint64_t A[3];    // Feistel round-function multipliers (odd), per hash
    uint64_t B[3];    // Feistel round-function offsets, per hash
};

// Everything a kernel needs about a table, passed by value (216 bytes; a
// batch descriptor of the fused launch embeds it).
struct TableArgs {
    Level lv[2];
    int16_t w;                // key bits
    int16_t key_bytes;        // 4 or 8
    int16_t H;                // cuckoo hash count
    int16_t wpb;              // words per bucket: 4, 8 or 16 (32, 64 or 128 bytes)
    int C;                    // cuckoo chain bound
    int16_t compact;          // 1: remainders, 0: whole keys
    int16_t retry_limit;      // iceberg: lost claims a key may retry (0 = built-in bound)
    int max_tiles;            // 0 = unbounded
    uint32_t *err;            // header error word
    unsigned long long *ctr;  // optional cht_counters (probes, writes, cas_fail, ops)
    uint64_t stash_slots;     // iceberg level-3 stash: 0 = none, else a power of two
    uint64_t stash_key;       // constant of the stash's home hash
};

// Lost claims an iceberg find-or-put may retry before it reports ST_ERROR.
// Every lost claim means another key filled a slot of the same buckets, and
// fields are never emptied, so a key can lose at most once per slot of its
// three buckets (Appendix A, termination); the bound adds a margin to that.
// A table configured with retry_limit > 0 uses that instead.
__host__ __device__ __forceinline__ int iceberg_retry_bound(const TableArgs &ta, int B0, int B1) {
    return ta.retry_limit > 0 ? ta.retry_limit : 4 * (B0 + 2 * B1) + 16;
}

// ---------------------------------------------------------------------------
// splitmix64 (Steele, Lea and Flood 2014)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t splitmix(uint64_t s, uint64_t idx) {
    return mix64(s + (idx + 1) * kGamma);
}

// ---------------------------------------------------------------------------
// Level 3: the overflow stash of an iceberg table (Section 2.3 describes a
// third level; the paper's implementation leaves it out, so the design here
// is this library's). stash_slots whole keys follow the secondary level's
// buckets; 0 is EMPTY. A key is placed there only when its primary and both
// secondary buckets are full, by linear probing from its home position
// mix64(k ^ stash_key) mod stash_slots; a claim is a 64-bit compare-and-swap
// EMPTY -> k. Positions never become empty again, so every thread probing
// for k walks the same filled prefix of k's probe sequence: of concurrent
// puts of k exactly one claims a position and the others then find k there.
// ---------------------------------------------------------------------------
struct StashResult {
    uint8_t status;  // FOUND / PUT / FULL (puts), FOUND / NOT_FOUND (lookups)
    uint64_t pos;    // the position that holds k when FOUND or PUT
};

__device__ __forceinline__ uint64_t *stash_words(const TableArgs &ta) {
    return ta.lv[1].words + ta.lv[1].nb * (uint64_t)ta.wpb;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// find-or-put of k in the stash; the probe sequence is bounded by the
// stash's size, so the loop always ends
__device__ __forceinline__ StashResult stash_find_or_put(const TableArgs &ta, uint64_t k,
                                                         int &fails) {
    uint64_t *st = stash_words(ta);
    const uint64_t mask = ta.stash_slots - 1;
    const uint64_t h = mix64(k ^ ta.stash_key) & mask;
    for (uint64_t i = 0; i < ta.stash_slots; ++i) {
        const uint64_t p = (h + i) & mask;
        uint64_t v = ld_relaxed_u64(st + p);
        if (v == 0) {
            const unsigned long long old =
                atomicCAS(reinterpret_cast<unsigned long long *>(st + p), 0ull,
                          static_cast<unsigned long long>(k));
            if (old == 0ull) return {ST_PUT, p};
            fails++;
            v = old;
        }
        if (v == k) return {ST_FOUND, p};
    }
    return {ST_FULL, ~0ull};
}

// lookup of k in the stash: it ends at k or at the first empty position
__device__ __forceinline__ StashResult stash_find(const TableArgs &ta, uint64_t k) {
    const uint64_t *st = stash_words(ta);
    const uint64_t mask = ta.stash_slots - 1;
    const uint64_t h = mix64(k ^ ta.stash_key) & mask;
    for (uint64_t i = 0; i < ta.stash_slots; ++i) {
        const uint64_t p = (h + i) & mask;
        const uint64_t v = ld_relaxed_u64(st + p);
        if (v == k) return {ST_FOUND, p};
        if (v == 0) break;
    }
    return {ST_NOT_FOUND, ~0ull};
}

// ---------------------------------------------------------------------------
// Permutation pi_j and quotient (Section 2.4). One-round Feistel: the low R
// bits r of k pass through, the high n bits are XORed with f_j(r), a
// multiply-shift hash of r. a = the high n bits of pi_j(k), remainder = r.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t round_fn(const Level &L, int j, uint64_t r) {
    // select the constants without indexing the parameter block dynamically
    const uint64_t A = j == 0 ? L.A[0] : (j == 1 ? L.A[1] : L.A[2]);
    const uint64_t B = j == 0 ? L.B[0] : (j == 1 ? L.B[1] : L.B[2]);
    return L.n ? (A * r + B) >> (64 - L.n) : 0ull;
}

__device__ __forceinline__ uint64_t low_mask(int bits) {
    return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
}

struct Quot {
    uint64_t a;  // bucket address
    uint64_t r;  // remainder
};

__device__ __forceinline__ Quot quotient(const Level &L, int w, int j, uint64_t k) {
    uint64_t r = k & low_mask(L.R);
    uint64_t hi = (k >> L.R) ^ round_fn(L, j, r);
    if (L.pow2) return {hi, r};
    // bucket count not a power of two (whole-key tables): scale pi_j(k) onto [0, nb)
    uint64_t p = (hi << L.R) | r;
    uint64_t lo = p * L.nb, h = __umul64hi(p, L.nb);
    return {(h << (64 - w)) | (lo >> w), r};
}

// k = pi_j^-1(a . r)
__device__ __forceinline__ uint64_t unquotient(const Level &L, int j, uint64_t a, uint64_t r) {
    return ((a ^ round_fn(L, j, r)) << L.R) | r;
}

// ---------------------------------------------------------------------------
// Fields
// ---------------------------------------------------------------------------
template <int FPW>
struct Fields {
    static constexpr int S = 64 / FPW;
    static constexpr uint64_t M = (S >= 64) ? ~0ull : ((1ull << S) - 1ull);
    __device__ __forceinline__ static uint64_t get(uint64_t word, int f) {
        return (word >> (f * S)) & M;
    }
};

// ---------------------------------------------------------------------------
// Bucket chunk loads. Concurrent writers exist during insert / find-or-put,
// so those loads are relaxed at GPU scope (each 64-bit element single-copy
// atomic; a snapshot may be torn across words, which the algorithms
// tolerate: a stale EMPTY only makes a later CAS fail). Static lookups use
// the read-only path.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void load_relaxed(const uint64_t *p, uint64_t (&v)[W]) {
    if constexpr (W == 1) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v[0]) : "l"(p) : "memory");
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
            asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
                         : "=l"(v[i]), "=l"(v[i + 1])
                         : "l"(p + i)
                         : "memory");
    }
}

template <int W>
__device__ __forceinline__ void load_readonly(const uint64_t *p, uint64_t (&v)[W]) {
    if constexpr (W == 1) {
        v[0] = __ldg(reinterpret_cast<const unsigned long long *>(p));
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) {
            ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2 *>(p + i));
            v[i] = x.x;
            v[i + 1] = x.y;
        }
    }
}

// read-only data that will not be reused soon: non-coherent path, no L1
// allocation (random bucket lines would only evict each other)
template <int W>
__device__ __forceinline__ void load_stream(const uint64_t *p, uint64_t (&v)[W]) {
    if constexpr (W == 1) {
        asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v[0]) : "l"(p));
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
            asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
                         : "=l"(v[i]), "=l"(v[i + 1])
                         : "l"(p + i));
    }
}

// load_stream under a predicate: when p is false no load is issued and v keeps
// its previous contents
template <int W>
__device__ __forceinline__ void load_stream_if(bool p, const uint64_t *ptr, uint64_t (&v)[W]) {
    const unsigned pr = p ? 1u : 0u;
    if constexpr (W == 1) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
            "@q ld.global.nc.L1::no_allocate.u64 %0, [%1];\n\t}"
            : "+l"(v[0])
            : "l"(ptr), "r"(pr));
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
                "@q ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];\n\t}"
                : "+l"(v[i]), "+l"(v[i + 1])
                : "l"(ptr + i), "r"(pr));
    }
}

// load_relaxed under a predicate, for callers that ignore v when p is false
// (v is then left unspecified)
template <int W>
__device__ __forceinline__ void load_relaxed_or_skip(bool p, const uint64_t *ptr,
                                                     uint64_t (&v)[W]) {
    const unsigned pr = p ? 1u : 0u;
    if constexpr (W == 1) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
            "@q ld.relaxed.gpu.global.u64 %0, [%1];\n\t}"
            : "=l"(v[0])
            : "l"(ptr), "r"(pr)
            : "memory");
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
                "@q ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];\n\t}"
                : "=l"(v[i]), "=l"(v[i + 1])
                : "l"(ptr + i), "r"(pr)
                : "memory");
    }
}

// load_stream under a predicate, for callers that ignore v when p is false:
// v is then left unspecified, which saves initialising it
template <int W>
__device__ __forceinline__ void load_stream_or_skip(bool p, const uint64_t *ptr,
                                                    uint64_t (&v)[W]) {
    const unsigned pr = p ? 1u : 0u;
    if constexpr (W == 1) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
            "@q ld.global.nc.L1::no_allocate.u64 %0, [%1];\n\t}"
            : "=l"(v[0])
            : "l"(ptr), "r"(pr));
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2)
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
                "@q ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];\n\t}"
                : "=l"(v[i]), "=l"(v[i + 1])
                : "l"(ptr + i), "r"(pr));
    }
}

// ---------------------------------------------------------------------------
// Tile primitives. A tile is T consecutive lanes of a warp; every lane of the
// warp executes these together (full-warp masks), each tile reading its own
// bits.
// ---------------------------------------------------------------------------
template <int T>
__device__ __forceinline__ uint32_t tile_bits(uint32_t warp_ballot) {
    const int lane = threadIdx.x & 31;
    const uint32_t m = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
    return (warp_ballot >> (lane & ~(T - 1))) & m;
}
template <int T>
__device__ __forceinline__ uint32_t tile_ballot(bool p) {
    return tile_bits<T>(__ballot_sync(0xffffffffu, p));
}
// value of v held by tile lane src (src relative to the tile)
template <int T, typename V>
__device__ __forceinline__ V tile_shfl(V v, int src) {
    return __shfl_sync(0xffffffffu, v, src, T);
}
template <int T>
__device__ __forceinline__ bool tile_shfl(bool v, int src) {
    return __shfl_sync(0xffffffffu, (int)v, src, T) != 0;
}

// Zero-field test on a packed word (the "has a zero byte" bit trick, widened
// to S-bit fields): (x - LOWS) & ~x & HIGHS has the top bit of field f set
// when field f is zero and lies below every other zero field; fields above
// the lowest zero one may be flagged spuriously (a borrow), which neither
// "any field zero" nor "lowest zero field" can see. No field value in
// [1, 2^S) is ever flagged without a zero field below it.
template <int FPW>
struct Swar {
    static constexpr int S = 64 / FPW;
    static constexpr uint64_t LOWS = FPW == 1 ? 1ull
                                   : FPW == 2 ? 0x0000000100000001ull
                                   : FPW == 3 ? ((1ull << 42) | (1ull << 21) | 1ull)
                                              : 0x0001000100010001ull;
    static constexpr uint64_t HIGHS = LOWS << (S - 1);
    __device__ __forceinline__ static uint64_t zeros(uint64_t x) {
        return (x - LOWS) & ~x & HIGHS;
    }
    // entry replicated into every field of a word
    __device__ __forceinline__ static uint64_t spread(uint64_t entry) { return entry * LOWS; }
};

// per-lane scan of the owned fields: whether one equals `entry`, and the local
// index at which to claim: W * FPW minus the number of EMPTY fields, or -1 if
// none is empty.
//
// Filled slots of a bucket form a prefix, so in a consistent snapshot this is
// the first empty field (and the zero-field mask is then exact, one flag per
// empty field). A snapshot torn across words may show stale empties; since a
// field never becomes empty again, the snapshot's empty fields include every
// field that is truly empty, so the index is never past the true first empty
// slot: a claim there either hits exactly the first empty slot or finds its
// field taken and fails, as any lost race does.
template <int W, int FPW>
__device__ __forceinline__ void scan_chunk(const uint64_t (&v)[W], uint64_t entry, bool &match,
                                           int &first_empty) {
    using Z = Swar<FPW>;
    const uint64_t pat = Z::spread(entry);
    uint64_t hit = 0;
    int empties = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        hit |= Z::zeros(v[i] ^ pat);
        empties += __popcll(Z::zeros(v[i]));
    }
    match = hit != 0;
    first_empty = empties ? W * FPW - empties : -1;
}

// lookup form of the scan: whether some owned field equals `entry`, and
// whether the lane's last field is EMPTY. Filled slots of a bucket always
// form a prefix (a claim only succeeds on the first empty slot and no field
// is ever emptied), so the bucket has room exactly when its last slot,
// owned by the tile's last lane, is empty.
template <int W, int FPW>
__device__ __forceinline__ void probe_chunk(const uint64_t (&v)[W], uint64_t entry, bool &match,
                                            bool &last_empty) {
    using Z = Swar<FPW>;
    const uint64_t pat = Z::spread(entry);
    uint64_t hm = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) hm |= Z::zeros(v[i] ^ pat);
    match = hm != 0;
    last_empty = Fields<FPW>::get(v[W - 1], FPW - 1) == 0;
}

// probe_chunk / scan_chunk that also give the local field index of the match
// (-1 if none) from the same zero-field masks: the first word with a flag is
// picked with selects, then one find-first-set gives its lowest flagged field
template <int FPW>
__device__ __forceinline__ int first_flag_field(uint64_t zsel, int wsel) {
    const int b = __ffsll((long long)zsel) - 1;  // -1 when zsel == 0
    return zsel ? wsel * FPW + b / Swar<FPW>::S : -1;
}
template <int W, int FPW>
__device__ __forceinline__ void probe_chunk_pos(const uint64_t (&v)[W], uint64_t entry,
                                                bool &match, bool &last_empty, int &pos) {
    using Z = Swar<FPW>;
    const uint64_t pat = Z::spread(entry);
    uint64_t zsel = 0;
    int wsel = 0;
#pragma unroll
    for (int i = W - 1; i >= 0; --i) {
        const uint64_t z = Z::zeros(v[i] ^ pat);
        wsel = z ? i : wsel;
        zsel = z ? z : zsel;
    }
    pos = first_flag_field<FPW>(zsel, wsel);
    match = zsel != 0;
    last_empty = Fields<FPW>::get(v[W - 1], FPW - 1) == 0;
}
template <int W, int FPW>
__device__ __forceinline__ void scan_chunk_pos(const uint64_t (&v)[W], uint64_t entry, bool &match,
                                               int &first_empty, int &pos) {
    using Z = Swar<FPW>;
    const uint64_t pat = Z::spread(entry);
    int empties = 0;
    uint64_t zsel = 0;
    int wsel = 0;
#pragma unroll
    for (int i = W - 1; i >= 0; --i) {
        const uint64_t z = Z::zeros(v[i] ^ pat);
        wsel = z ? i : wsel;
        zsel = z ? z : zsel;
        empties += __popcll(Z::zeros(v[i]));
    }
    pos = first_flag_field<FPW>(zsel, wsel);
    match = zsel != 0;
    first_empty = empties ? W * FPW - empties : -1;
}

template <int W>
__device__ __forceinline__ void scan_chunk_rt_pos(const uint64_t (&v)[W], uint64_t entry, int fpw,
                                                  bool &match, int &first_empty, int &pos) {
    switch (fpw) {
        case 1: scan_chunk_pos<W, 1>(v, entry, match, first_empty, pos); break;
        case 2: scan_chunk_pos<W, 2>(v, entry, match, first_empty, pos); break;
        case 3: scan_chunk_pos<W, 3>(v, entry, match, first_empty, pos); break;
        default: scan_chunk_pos<W, 4>(v, entry, match, first_empty, pos); break;
    }
}

// local field index (word * FPW + field) of the owned field equal to entry,
// or -1: the lowest flagged field of the first word with a flag is exact
// (see Swar), and a table holds an entry at most once
template <int W, int FPW>
__device__ __forceinline__ int match_field(const uint64_t (&v)[W], uint64_t entry) {
    using Z = Swar<FPW>;
    const uint64_t pat = Z::spread(entry);
    int r = -1;
#pragma unroll
    for (int i = W - 1; i >= 0; --i) {
        const uint64_t z = Z::zeros(v[i] ^ pat);
        if (z) r = i * FPW + (__ffsll((long long)z) - 1) / Z::S;
    }
    return r;
}
template <int W>
__device__ __forceinline__ int match_field_rt(const uint64_t (&v)[W], uint64_t entry, int fpw) {
    switch (fpw) {
        case 1: return match_field<W, 1>(v, entry);
        case 2: return match_field<W, 2>(v, entry);
        case 3: return match_field<W, 3>(v, entry);
        default: return match_field<W, 4>(v, entry);
    }
}

// the same with the packing known only at run time (fpw in 1..4)
template <int W>
__device__ __forceinline__ void scan_chunk_rt(const uint64_t (&v)[W], uint64_t entry, int fpw,
                                              bool &match, int &first_empty) {
    switch (fpw) {
        case 1: scan_chunk<W, 1>(v, entry, match, first_empty); break;
        case 2: scan_chunk<W, 2>(v, entry, match, first_empty); break;
        case 3: scan_chunk<W, 3>(v, entry, match, first_empty); break;
        default: scan_chunk<W, 4>(v, entry, match, first_empty); break;
    }
}

// ---------------------------------------------------------------------------
// Field-level compare-and-swap EMPTY -> entry on field f of *wp, emulated on
// the narrowest naturally aligned atomic that contains the field: 16-bit and
// 32-bit fields use native sub-word CAS, 21-bit fields a 64-bit CAS that is
// retried while only neighbouring fields changed (fields only ever go from
// EMPTY to filled, so the retry count is bounded by the fields per word).
// Returns true if this thread wrote the entry; otherwise *seen holds the
// field value that won.
// ---------------------------------------------------------------------------
template <int FPW>
__device__ __forceinline__ bool claim_field(uint64_t *wp, int f, uint64_t snap_word,
                                            uint64_t entry, uint64_t &seen, int &fails) {
    using F = Fields<FPW>;
    if constexpr (FPW == 1) {
        unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long *>(wp), 0ull,
                                           static_cast<unsigned long long>(entry));
        seen = old;
        if (old != 0ull) fails++;
        return old == 0ull;
    } else if constexpr (FPW == 2) {
        unsigned int *hp = reinterpret_cast<unsigned int *>(wp) + f;
        unsigned int old = atomicCAS(hp, 0u, static_cast<unsigned int>(entry));
        seen = old;
        if (old != 0u) fails++;
        return old == 0u;
    } else if constexpr (FPW == 4) {
        unsigned short *hp = reinterpret_cast<unsigned short *>(wp) + f;
        unsigned short old = atomicCAS(hp, static_cast<unsigned short>(0),
                                       static_cast<unsigned short>(entry));
        seen = old;
        if (old != 0) fails++;
        return old == 0;
    } else {
        uint64_t expected = snap_word & ~(F::M << (f * F::S));
        for (int it = 0; it < 64; ++it) {
            uint64_t desired = expected | (entry << (f * F::S));
            unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long *>(wp),
                                               expected, desired);
            if (old == expected) return true;
            fails++;
            uint64_t fld = F::get(old, f);
            if (fld != 0) {
                seen = fld;
                return false;
            }
            expected = old;
        }
        seen = 0;  // gave up on this word; the caller re-reads the bucket
        return false;
    }
}

__device__ __forceinline__ bool claim_field_rt(int fpw, uint64_t *wp, int f, uint64_t snap_word,
                                               uint64_t entry, uint64_t &seen, int &fails);

// Atomic swap of field f of *wp with `entry` (Algorithm 4's Swap). Returns the
// previous field value; sets ok = false if a bounded retry loop gave up.
template <int FPW>
__device__ __forceinline__ uint64_t swap_field(uint64_t *wp, int f, uint64_t snap_word,
                                               uint64_t entry, bool &ok) {
    using F = Fields<FPW>;
    ok = true;
    if constexpr (FPW == 1) {
        return atomicExch(reinterpret_cast<unsigned long long *>(wp),
                          static_cast<unsigned long long>(entry));
    } else if constexpr (FPW == 2) {
        return atomicExch(reinterpret_cast<unsigned int *>(wp) + f,
                          static_cast<unsigned int>(entry));
    } else {
        uint64_t expected = snap_word;
        for (int it = 0; it < 4096; ++it) {
            uint64_t desired = (expected & ~(F::M << (f * F::S))) | (entry << (f * F::S));
            unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long *>(wp),
                                               expected, desired);
            if (old == expected) return F::get(old, f);
            expected = old;
        }
        ok = false;
        return 0;
    }
}

// The same two operations split in two phases, so that a thread can have the
// atomics of several buckets in flight: field_op_issue makes the first
// attempt (a claim when `swap` is false, else a swap) and returns the value
// the atomic saw together with the value it expected; field_op_finish reads
// the outcome and, in the rare case where only a neighbouring field of a
// packed word changed, continues with the retry loops above.
template <int FPW>
__device__ __forceinline__ uint64_t field_op_issue(bool swap, uint64_t *wp, int f, uint64_t snap_word,
                                                   uint64_t entry, uint64_t &expected) {
    using F = Fields<FPW>;
    if constexpr (FPW == 1) {
        expected = 0ull;
        if (swap) {
            const uint64_t old = atomicExch(reinterpret_cast<unsigned long long *>(wp),
                                            static_cast<unsigned long long>(entry));
            expected = old;
            return old;
        }
        return atomicCAS(reinterpret_cast<unsigned long long *>(wp), 0ull,
                         static_cast<unsigned long long>(entry));
    } else if constexpr (FPW == 2) {
        unsigned int *hp = reinterpret_cast<unsigned int *>(wp) + f;
        if (swap) {
            const uint64_t old = atomicExch(hp, static_cast<unsigned int>(entry));
            expected = old;
            return old;
        }
        expected = 0;
        return atomicCAS(hp, 0u, static_cast<unsigned int>(entry));
    } else {
        if (FPW == 4 && !swap) {
            unsigned short *hp = reinterpret_cast<unsigned short *>(wp) + f;
            expected = 0;
            return atomicCAS(hp, static_cast<unsigned short>(0), static_cast<unsigned short>(entry));
        }
        expected = snap_word & ~(F::M << (f * F::S));
        if (swap) expected = snap_word;
        const uint64_t desired = (snap_word & ~(F::M << (f * F::S))) | (entry << (f * F::S));
        return atomicCAS(reinterpret_cast<unsigned long long *>(wp), expected, desired);
    }
}

// outcome of a claim: true if written, else seen = the field value that won
template <int FPW>
__device__ __forceinline__ bool claim_finish(uint64_t *wp, int f, uint64_t old, uint64_t expected,
                                             uint64_t entry, uint64_t &seen, int &fails) {
    using F = Fields<FPW>;
    if (old == expected) return true;
    fails++;
    if constexpr (FPW == 1 || FPW == 2 || FPW == 4) {
        seen = old;  // a whole-field CAS: the winner's value
        return false;
    } else {
        const uint64_t fld = F::get(old, f);
        if (fld != 0) {
            seen = fld;
            return false;
        }
        return claim_field<FPW>(wp, f, old, entry, seen, fails);  // a neighbour changed
    }
}

// outcome of a swap: the previous field value; ok = false if the retry gave up
template <int FPW>
__device__ __forceinline__ uint64_t swap_finish(uint64_t *wp, int f, uint64_t old,
                                                uint64_t expected, uint64_t entry, bool &ok) {
    using F = Fields<FPW>;
    ok = true;
    if constexpr (FPW == 1 || FPW == 2) {
        return old;  // a native exchange always succeeds
    } else {
        if (old == expected) return F::get(old, f);
        return swap_field<FPW>(wp, f, old, entry, ok);
    }
}

__device__ __forceinline__ bool claim_field_rt(int fpw, uint64_t *wp, int f, uint64_t snap_word,
                                               uint64_t entry, uint64_t &seen, int &fails) {
    switch (fpw) {
        case 1: return claim_field<1>(wp, f, snap_word, entry, seen, fails);
        case 2: return claim_field<2>(wp, f, snap_word, entry, seen, fails);
        case 3: return claim_field<3>(wp, f, snap_word, entry, seen, fails);
        default: return claim_field<4>(wp, f, snap_word, entry, seen, fails);
    }
}

// ---------------------------------------------------------------------------
// Values of the key-value extension: a caller array of nstore values of
// vbytes (4, 8 or 16) indexed by slot. A put copies value i of its batch to
// the key's slot; a get copies the slot's value to output i (zero when the
// key has no slot).
// ---------------------------------------------------------------------------
struct KVArgs {
    const void *vin;  // put: the batch's values
    void *vout;       // get: output values
    void *store;      // the value array (null: no value moves)
    uint64_t nstore;  // its length in values
    int vbytes;
};

// one value as two words (4-byte values use lo only)
struct KVal {
    uint64_t lo, hi;
};
__device__ __forceinline__ KVal kv_read(const void *base, uint64_t i, int vbytes) {
    if (vbytes == 4) return {static_cast<const uint32_t *>(base)[i], 0};
    if (vbytes == 8) return {static_cast<const uint64_t *>(base)[i], 0};
    const ulonglong2 v = static_cast<const ulonglong2 *>(base)[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void kv_write(void *base, uint64_t i, int vbytes, KVal v) {
    if (vbytes == 4)
        static_cast<uint32_t *>(base)[i] = static_cast<uint32_t>(v.lo);
    else if (vbytes == 8)
        static_cast<uint64_t *>(base)[i] = v.lo;
    else
        static_cast<ulonglong2 *>(base)[i] = make_ulonglong2(v.lo, v.hi);
}

__device__ __forceinline__ void kv_move(const KVArgs &kv, bool put, uint64_t i, uint64_t slot) {
    const bool has = slot < kv.nstore;
    switch (kv.vbytes) {
        case 4: {
            uint32_t *st = static_cast<uint32_t *>(kv.store);
            if (put) {
                if (has) st[slot] = static_cast<const uint32_t *>(kv.vin)[i];
            } else {
                static_cast<uint32_t *>(kv.vout)[i] = has ? st[slot] : 0u;
            }
            break;
        }
        case 8: {
            uint64_t *st = static_cast<uint64_t *>(kv.store);
            if (put) {
                if (has) st[slot] = static_cast<const uint64_t *>(kv.vin)[i];
            } else {
                static_cast<uint64_t *>(kv.vout)[i] = has ? st[slot] : 0ull;
            }
            break;
        }
        default: {
            ulonglong2 *st = static_cast<ulonglong2 *>(kv.store);
            if (put) {
                if (has) st[slot] = static_cast<const ulonglong2 *>(kv.vin)[i];
            } else {
                static_cast<ulonglong2 *>(kv.vout)[i] = has ? st[slot] : make_ulonglong2(0, 0);
            }
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t load_key(const void *keys, int key_bytes, uint64_t i) {
    if (key_bytes == 8) return __ldg(static_cast<const unsigned long long *>(keys) + i);
    return __ldg(static_cast<const unsigned int *>(keys) + i);
}
__device__ __forceinline__ void store_key(void *out, int key_bytes, uint64_t i, uint64_t k) {
    if (key_bytes == 8)
        static_cast<unsigned long long *>(out)[i] = k;
    else
        static_cast<unsigned int *>(out)[i] = static_cast<unsigned int>(k);
}
__device__ __forceinline__ bool valid_key(uint64_t k, int w) {
    return k != 0 && (k >> w) == 0;
}

// add a per-thread counter into the table's counters, one atomic per warp
__device__ __forceinline__ void flush_counter(unsigned long long *ctr, int idx, uint64_t v) {
    unsigned long long s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr + idx, s);
}

// ---------------------------------------------------------------------------
// Work distribution (Algorithm 3, cooperative work sharing). Each tile takes
// chunks of T * items consecutive keys, stages them in shared memory and
// processes them one at a time in input order; statuses are staged too and
// written back per chunk. The per-tile state machine advances every tile of a
// warp in lock step so that ballots and shuffles see full warps.
// ---------------------------------------------------------------------------
template <int T>
struct TileWork {
    uint64_t *s_keys;  // T * items keys of this tile
    uint8_t *s_st;     // T * items status bytes
    uint64_t chunk, nchunks, stride;
    uint64_t base;
    int q, qn, items;
    bool done;

    __device__ __forceinline__ void init(uint64_t *smem_keys, uint8_t *smem_st, int items_,
                                         uint64_t n, int max_tiles) {
        const int tiles_per_block = blockDim.x / T;
        const int tib = threadIdx.x / T;
        items = items_;
        s_keys = smem_keys + (size_t)tib * T * items;
        s_st = smem_st ? smem_st + (size_t)tib * T * items : nullptr;
        const uint64_t tile_id = (uint64_t)blockIdx.x * tiles_per_block + tib;
        uint64_t ntiles = (uint64_t)gridDim.x * tiles_per_block;
        if (max_tiles > 0 && ntiles > (uint64_t)max_tiles) ntiles = max_tiles;
        const uint64_t per = (uint64_t)T * items;
        nchunks = (n + per - 1) / per;
        stride = ntiles;
        chunk = tile_id;
        done = (tile_id >= ntiles) || (chunk >= nchunks);
        q = qn = 0;
        base = 0;
    }

    // stage the next chunk's keys (called with q >= qn by every lane of the tile)
    __device__ __forceinline__ void refill(const void *keys, int key_bytes, uint64_t n,
                                           uint8_t *status) {
        const int tl = threadIdx.x & (T - 1);
        const uint64_t per = (uint64_t)T * items;
        if (qn > 0) {
            for (int i = 0; i < items; ++i) {
                int idx = i * T + tl;
                if (idx < qn) status[base + idx] = s_st[idx];
            }
            chunk += stride;
        }
        if (chunk >= nchunks) {
            done = true;
            qn = q = 0;
            return;
        }
        base = chunk * per;
        uint64_t rem = n - base;
        qn = rem < per ? (int)rem : (int)per;
        q = 0;
        for (int i = 0; i < items; ++i) {
            int idx = i * T + tl;
            if (idx < qn) s_keys[idx] = load_key(keys, key_bytes, base + idx);
        }
    }

    // stage the next chunk's keys for kernels that write statuses directly
    // (no staged statuses to flush); called with q >= qn by every lane of
    // the tile
    __device__ __forceinline__ void stage(const void *keys, int key_bytes, uint64_t n) {
        const int tl = threadIdx.x & (T - 1);
        const uint64_t per = (uint64_t)T * items;
        if (qn > 0) chunk += stride;
        if (chunk >= nchunks) {
            done = true;
            qn = q = 0;
            return;
        }
        base = chunk * per;
        uint64_t rem = n - base;
        qn = rem < per ? (int)rem : (int)per;
        q = 0;
        for (int i = 0; i < items; ++i) {
            int idx = i * T + tl;
            if (idx < qn) s_keys[idx] = load_key(keys, key_bytes, base + idx);
        }
    }
};

}  // namespace cht
