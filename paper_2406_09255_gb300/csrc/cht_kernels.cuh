// cht_kernels.cuh - the hot-path kernels, templated on the tile width T
// (threads per bucket) and the packing FPW (fields per 64-bit word).
//
// Every kernel is persistent: tiles loop over chunks of keys (TileWork), and
// each loop iteration performs at most one bucket probe step per tile. All
// lanes of a warp run the loop body together; what differs between tiles is
// carried in predicates, so every ballot and shuffle is a full-warp one.
#pragma once

#include <type_traits>

#include "cht_device.cuh"

namespace cht {

template <int W>
__device__ __forceinline__ uint64_t pick_word(const uint64_t (&v)[W], int i) {
    uint64_t r = v[0];
#pragma unroll
    for (int k = 1; k < W; ++k)
        if (i == k) r = v[k];
    return r;
}

// shared memory bytes per block: keys (8 B) and status (1 B) per staged key
__host__ __device__ inline size_t smem_bytes(int cta_threads, int items) {
    return (size_t)cta_threads * items * 9;
}

// ===========================================================================
// Compact cuckoo put, Algorithm 4. Per key: probe a_j(k); if the bucket has
// an empty slot, CAS the first one; otherwise swap (r, j) into the slot chosen
// from (k, c) and continue with the evicted key under hash (j' + 1) mod H. A
// failed CAS also consumes a step. After C steps the put reports FULL and the
// key in hand is the dropped one.
// ===========================================================================
template <int T, int FPW, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256)
    k_cuckoo_insert(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                    uint8_t *__restrict__ status, uint64_t *__restrict__ dropped, int items) {
    constexpr int W = WPB / T;
    constexpr int LF = W * FPW;  // fields per lane
    constexpr int B = WPB * FPW;
    extern __shared__ uint64_t smem[];
    TileWork<T> tw;
    tw.init(smem, reinterpret_cast<uint8_t *>(smem + (size_t)blockDim.x * items), items, n,
            ta.max_tiles);
    const int tl = threadIdx.x & (T - 1);
    const Level &L = ta.lv[0];
    uint64_t cur = 0;
    int j = 0, c = 0;
    bool fresh = true;
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    while (__any_sync(0xffffffffu, !tw.done)) {
        if (!tw.done && tw.q >= tw.qn) tw.refill(keys, ta.key_bytes, n, status);
        __syncwarp();
        const bool act = !tw.done;
        if (act && fresh) {
            cur = tw.s_keys[tw.q];
            j = 0;
            c = 1;
            fresh = false;
        }
        const bool inval = act && !valid_key(cur, ta.w);
        const bool probe = act && !inval;

        const Quot qt = quotient(L, ta.w, j, cur);
        const uint64_t entry = ((ta.compact ? qt.r : cur) << 2) | (uint64_t)(j + 1);
        uint64_t *bp = L.words + qt.a * WPB + tl * W;
        uint64_t v[W] = {};
        if (probe) load_relaxed<W>(bp, v);
        bool m;
        int fe;
        scan_chunk<W, FPW>(v, entry, m, fe);
        const uint32_t be = tile_ballot<T>(probe && fe >= 0);
        const int cl = be ? __ffs(be) - 1 : 0;
        // slot to evict if the bucket is full: "pseudorandomly, based on c, k"
        const int y = (int)(((splitmix(cur, (uint64_t)c) >> 32) * (uint64_t)B) >> 32);
        const int el = y / LF, ef = y - el * LF;

        bool claimed = false, swap_ok = true;
        uint64_t seen = 0, evicted = 0;
        if (probe && be && tl == cl)
            claimed = claim_field<FPW>(bp + fe / FPW, fe % FPW, pick_word<W>(v, fe / FPW), entry,
                                       seen, n_fail);
        if (probe && !be && tl == el)
            evicted = swap_field<FPW>(bp + ef / FPW, ef % FPW, pick_word<W>(v, ef / FPW), entry,
                                      swap_ok);
        claimed = tile_shfl<T>(claimed, cl);
        evicted = tile_shfl<T>(evicted, el);
        swap_ok = tile_shfl<T>(swap_ok, el);

        if (act) {
            bool fin = false;
            uint8_t st = ST_PUT;
            if (inval) {
                fin = true;
                st = ST_INVALID;
            } else {
                n_probe++;
                if (be) {
                    if (claimed) {
                        fin = true;
                        n_write++;
                    } else if (++c > ta.C) {
                        fin = true;
                        st = ST_FULL;
                    }
                } else if (!swap_ok) {
                    fin = true;
                    st = ST_ERROR;
                } else {
                    n_write++;
                    if (evicted == 0) {
                        fin = true;  // the chosen slot held nothing: placed
                    } else {
                        const int jo = (int)(evicted & 3) - 1;
                        cur = ta.compact ? unquotient(L, jo, qt.a, evicted >> 2) : (evicted >> 2);
                        j = (jo + 1 == ta.H) ? 0 : jo + 1;
                        if (++c > ta.C) {
                            fin = true;
                            st = ST_FULL;
                        }
                    }
                }
            }
            if (fin) {
                if (tl == 0) {
                    tw.s_st[tw.q] = st;
                    if (st == ST_FULL && dropped) dropped[tw.base + tw.q] = cur;
                    if (st == ST_ERROR) atomicOr(ta.err, 1u);
                    n_ops++;
                }
                tw.q++;
                fresh = true;
            }
        }
        __syncwarp();
    }
    if (ta.ctr) {
        if (tl != 0) n_probe = n_write = 0;
        flush_counter(ta.ctr, 0, n_probe);
        flush_counter(ta.ctr, 1, n_write);
        flush_counter(ta.ctr, 2, (uint64_t)n_fail);
        flush_counter(ta.ctr, 3, n_ops);
    }
}

// ===========================================================================
// Compact cuckoo lookup, Section 4.4: probe a_0, a_1, ... for (r_j, j); stop
// at the first bucket that holds it (FOUND) or that is not full (NOT_FOUND).
//
// Work sharing as in Algorithm 3, with the per-key arithmetic taken out of
// the tile: every lane loads one key of the warp's 32 and computes its own
// bucket address and entry; then each tile of T lanes walks the keys of its
// own lanes, one per round. It broadcasts the key's bucket index and entry
// (Shuffle), loads the bucket (for T = 8 one 16-byte read per lane, so one
// warp load instruction fetches four whole lines) and answers with two
// ballots (Any match, last slot empty). A key whose bucket was full and did
// not hold it moves to hash j + 1 in the next pass. The table is not written
// while a lookup runs (static table), so buckets are read through the
// non-coherent path without L1 allocation.
//
// This form keeps one bucket load in flight per tile; the stream form below
// is the fast path and this one its plain counterpart.
// ===========================================================================
template <int T, int FPW, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, 6)
    k_cuckoo_find(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                  uint8_t *__restrict__ status) {
    constexpr int W = WPB / T;
    // compact entries fit 32 bits when fields are at most 32 bits wide
    using Entry = typename std::conditional<(FPW >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tbase = lane & ~(T - 1);
    const uint32_t tmask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << tbase;
    const uint32_t last_lane = 1u << (tbase + T - 1);
    const Level &L = ta.lv[0];
    const uint64_t *words = L.words + tl * W;  // this lane's part of every bucket
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) << 5;
    uint64_t n_probe = 0, n_ops = 0;
    uint64_t v[W];
#pragma unroll
    for (int i = 0; i < W; ++i) v[i] = 0;

    uint64_t base = warp * 32;
    uint64_t k_next = (base + lane < n) ? load_key(keys, ta.key_bytes, base + lane) : 0;
    for (; base < n; base += stride) {
        const uint64_t idx = base + lane;
        const bool has = idx < n;
        const uint64_t k = k_next;
        // fetch the next chunk's key now; it arrives while this chunk runs
        const uint64_t nidx = idx + stride;
        k_next = (nidx < n) ? load_key(keys, ta.key_bytes, nidx) : 0;
        bool pending = has && valid_key(k, ta.w);
        uint8_t st = pending ? ST_NOT_FOUND : ST_INVALID;
        int j = 0;
        while (__any_sync(0xffffffffu, pending)) {
            uint32_t addr = 0;  // bucket index (a table has fewer than 2^32 buckets)
            Entry entry = 0;
            if (pending) {
                const Quot qt = quotient(L, ta.w, j, k);
                addr = (uint32_t)qt.a;
                entry = (Entry)((((ta.compact ? qt.r : k)) << 2) | (uint64_t)(j + 1));
            }
            // this pass: every key of the tile still pending, at its own hash j
            uint32_t pm = __ballot_sync(0xffffffffu, pending) & tmask;
            int r = pm ? __ffs(pm) - 1 - tbase : -1;
            pm &= pm - 1;
            Entry e = tile_shfl<T>(entry, r & (T - 1));
            {
                const uint32_t a = tile_shfl<T>(addr, r & (T - 1));
                load_stream_if<W>(r >= 0, words + (uint64_t)a * WPB, v);
            }
            while (__any_sync(0xffffffffu, r >= 0)) {
                bool m, le;
                probe_chunk<W, FPW>(v, e, m, le);
                const bool live = r >= 0;
                const uint32_t bm = __ballot_sync(0xffffffffu, live && m) & tmask;
                const uint32_t be = __ballot_sync(0xffffffffu, live && le) & last_lane;
                if (tl == r) {
                    n_probe++;
                    if (bm) {
                        st = ST_FOUND;
                        pending = false;
                    } else if (be || j + 1 >= ta.H) {
                        pending = false;
                    } else {
                        j++;  // probe a_{j+1} in the next pass
                    }
                }
                r = pm ? __ffs(pm) - 1 - tbase : -1;
                pm &= pm - 1;
                e = tile_shfl<T>(entry, r & (T - 1));
                const uint32_t a = tile_shfl<T>(addr, r & (T - 1));
                load_stream_if<W>(r >= 0, words + (uint64_t)a * WPB, v);
            }
        }
        if (has) status[idx] = st;
        n_ops += has ? 1 : 0;
    }
    if (ta.ctr) {
        flush_counter(ta.ctr, 0, n_probe);
        flush_counter(ta.ctr, 3, n_ops);
    }
}

// ===========================================================================
// The lookup of Section 4.4 as a stream of probe rounds (the fast path).
// Each lane holds one key at a time with its current hash index j. In every
// round each tile probes all of its lanes' keys on a fixed schedule: tile
// lane s's key goes in slot s, and Q bucket loads are issued back to back
// before any is inspected (Q lines in flight per tile), with no search for
// pending keys. Match flags are gathered per lane as bit s of a mask and
// OR-reduced over the tile once per round; the last lane's "last slot empty"
// flags come back in one broadcast. A lane whose key is answered writes the
// status and takes the next key of the warp's stream (the warp's grid-stride
// 32-key chunks in order) for the next round, so every round is fully packed
// whatever mix of j the keys are at: the waiting lanes are ranked with one
// ballot and served from two chunks of keys held one per lane and read ahead
// of use. Probes per key, and so the answers and probe counts, are those of
// the per-round form.
// ===========================================================================
template <int T, int FPW, int Q, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, 3)
    k_cuckoo_find_stream(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                         uint8_t *__restrict__ status) {
    constexpr int W = WPB / T;
    constexpr int QE = Q < T ? Q : T;
    static_assert(T % QE == 0, "slots split evenly into load groups");
    using Entry = typename std::conditional<(FPW >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const uint32_t lt_mask = (1u << lane) - 1u;
    const Level &L = ta.lv[0];
    const uint64_t *words = L.words + tl * W;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) << 5;
    uint64_t n_probe = 0, n_ops = 0;

    // key buffers: chunk A at baseA (next key at offset o), chunk B at baseA + stride
    uint64_t baseA = warp * 32;
    uint64_t kA = (baseA + lane < n) ? load_key(keys, ta.key_bytes, baseA + lane) : 0;
    uint64_t kB = (baseA + stride + lane < n) ? load_key(keys, ta.key_bytes, baseA + stride + lane)
                                              : 0;
    int o = 0;
    uint64_t k = 0, idx = 0;
    int j = 0;
    bool live = false;
    while (true) {
        // refill the lanes without a key, in rank order
        const uint32_t need = __ballot_sync(0xffffffffu, !live);
        if (need) {
            const int src = o + __popc(need & lt_mask);
            const uint64_t ka = __shfl_sync(0xffffffffu, kA, src & 31);
            const uint64_t kb = __shfl_sync(0xffffffffu, kB, src & 31);
            if (!live) {
                idx = src < 32 ? baseA + src : baseA + stride + (src - 32);
                if (idx < n) {
                    k = src < 32 ? ka : kb;
                    j = 0;
                    n_ops++;
                    if (valid_key(k, ta.w))
                        live = true;
                    else
                        status[idx] = ST_INVALID;
                }
            }
            o += __popc(need);
            if (o >= 32) {
                o -= 32;
                baseA += stride;
                kA = kB;
                const uint64_t nb = baseA + stride + lane;
                kB = nb < n ? load_key(keys, ta.key_bytes, nb) : 0;
            }
        }
        if (!__any_sync(0xffffffffu, live)) {
            if (baseA >= n) break;  // the warp's stream is exhausted
            continue;               // a round of invalid keys only
        }
        uint32_t addr = 0;
        Entry entry = 0;
        if (live) {
            const Quot qt = quotient(L, ta.w, j, k);
            addr = (uint32_t)qt.a;
            entry = (Entry)(((ta.compact ? qt.r : k) << 2) | (uint64_t)(j + 1));
        }
        const uint32_t pb = tile_ballot<T>(live);
        uint32_t mbits = 0, lbits = 0;
#pragma unroll
        for (int s0 = 0; s0 < T; s0 += QE) {
            uint64_t v[QE][W];
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const uint32_t a = tile_shfl<T>(addr, s0 + q);
                load_stream_or_skip<W>((pb >> (s0 + q)) & 1u,
                                       words + (uint64_t)a * WPB, v[q]);
            }
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const Entry e = tile_shfl<T>(entry, s0 + q);
                bool m, le;
                probe_chunk<W, FPW>(v[q], e, m, le);
                mbits |= (m ? 1u : 0u) << (s0 + q);
                lbits |= (le ? 1u : 0u) << (s0 + q);
            }
        }
#pragma unroll
        for (int off = 1; off < T; off <<= 1) mbits |= __shfl_xor_sync(0xffffffffu, mbits, off);
        lbits = tile_shfl<T>(lbits, T - 1);
        if (live) {
            n_probe++;
            if ((mbits >> tl) & 1u) {
                status[idx] = ST_FOUND;
                live = false;
            } else if (((lbits >> tl) & 1u) || j + 1 >= ta.H) {
                status[idx] = ST_NOT_FOUND;
                live = false;
            } else {
                j++;
            }
        }
    }
    if (ta.ctr) {
        flush_counter(ta.ctr, 0, n_probe);
        flush_counter(ta.ctr, 3, n_ops);
    }
}

// ===========================================================================
// Compact iceberg find-or-put, Algorithm 1 (cooperative form of Algorithm 2).
// Level 1: snapshot the primary bucket; FOUND if it holds r_0(k); if it has
// an empty slot CAS the first one (PUT, or re-inspect the value that won);
// if it is full go to level 2. Level 2: snapshot both secondary buckets;
// FOUND if either holds (r_i(k), i - 1); otherwise pick the one whose first
// empty slot comes first in the slot order of Definition 1 (the strictly less
// full one, ties to the second), FULL if it has none, else CAS its first
// empty slot. A failed CAS re-inspects the winning value and, unless it is
// k's own entry, re-reads the buckets; the termination lemma of Appendix A
// bounds the retries by the slots involved.
// With LOOKUP set the engine is the Section 2.3 lookup instead.
//
// This engine processes each tile's keys strictly in input order; it serves
// runs with a bounded number of tiles (max_tiles > 0, e.g. the sequential
// single-tile run). Unordered runs use the warp-batched engine of
// cht_warp.cuh. The primary packing FPW0 is a template parameter; the
// secondary level, visited only by keys whose primary bucket is full, reads
// its packing at run time.
// ===========================================================================

// work source over one table: TileWork plus the table's arguments
template <int T>
struct SingleWork : TileWork<T> {
    const TableArgs *tap;
    const void *keys;
    uint64_t n;
    uint8_t *status;
    uint64_t *slots;  // optional slot index per key (iceberg key-value handle)
    const KVArgs *kv;  // optional value moves (key-value extension)
    __device__ __forceinline__ const TableArgs &ta() const { return *tap; }
    __device__ __forceinline__ void next() { this->refill(keys, tap->key_bytes, n, status); }
};

// one (table, keys, statuses) triple of a fused multi-table launch
struct BatchDesc {
    TableArgs ta;
    const void *keys;
    uint64_t n;
    uint8_t *status;
};

template <int T, int FPW0, bool LOOKUP, class Work, int WPB = kWordsPerBucket>
__device__ __forceinline__ void iceberg_engine(Work &tw, unsigned long long *ctr) {
    constexpr int W = WPB / T;
    const int tl = threadIdx.x & (T - 1);
    uint64_t cur = 0;
    int lvl = 1, it = 0;
    bool fresh = true;
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    while (__any_sync(0xffffffffu, !tw.done)) {
        if (!tw.done && tw.q >= tw.qn) tw.next();
        __syncwarp();
        const TableArgs &ta = tw.ta();
        const Level &L0 = ta.lv[0];
        const Level &L1 = ta.lv[1];
        const int FPW1 = L1.fpw;
        const int LF1 = W * FPW1;
        const int B1 = WPB * FPW1;
        const bool act = !tw.done;
        if (act && fresh) {
            cur = tw.s_keys[tw.q];
            lvl = 1;
            it = 0;
            fresh = false;
        }
        const bool inval = act && !valid_key(cur, ta.w);
        const bool probe = act && !inval;
        const bool p1 = probe && lvl == 1, p2 = probe && lvl == 2;

        const Quot q0 = quotient(L0, ta.w, 0, cur);
        const Quot qa = quotient(L1, ta.w, 0, cur);
        const Quot qb = quotient(L1, ta.w, 1, cur);
        const uint64_t e0 = ((ta.compact ? q0.r : cur) << 1) | 1ull;
        const uint64_t ea = ((ta.compact ? qa.r : cur) << 2) | 1ull;
        const uint64_t eb = ((ta.compact ? qb.r : cur) << 2) | 2ull;
        uint64_t *p0 = L0.words + q0.a * WPB + tl * W;
        uint64_t *pa = L1.words + qa.a * WPB + tl * W;
        uint64_t *pb = L1.words + qb.a * WPB + tl * W;
        uint64_t v0[W] = {}, va[W] = {}, vb[W] = {};
        if (p1) load_relaxed<W>(p0, v0);
        if (p2) {
            load_relaxed<W>(pa, va);
            load_relaxed<W>(pb, vb);
        }
        bool m0, ma, mb;
        int f0, fa, fb;
        scan_chunk<W, FPW0>(v0, e0, m0, f0);
        scan_chunk_rt<W>(va, ea, FPW1, ma, fa);
        scan_chunk_rt<W>(vb, eb, FPW1, mb, fb);
        const uint32_t bfound = tile_ballot<T>((p1 && m0) || (p2 && (ma || mb)));
        const uint32_t be0 = tile_ballot<T>(p1 && f0 >= 0);
        const uint32_t bea = tile_ballot<T>(p2 && fa >= 0);
        const uint32_t beb = tile_ballot<T>(p2 && fb >= 0);
        // where a match sits (slot outputs only): the first matching lane and
        // its local field, and whether it is in secondary bucket b
        int mlane = 0, mloc = -1;
        bool min_b = false;
        const bool want_slots = tw.slots || tw.kv->store;
        if (want_slots) {
            const uint32_t bma = tile_ballot<T>(p2 && ma);
            const int ml = p1 ? match_field<W, FPW0>(v0, e0)
                              : (ma ? match_field_rt<W>(va, ea, FPW1) : match_field_rt<W>(vb, eb, FPW1));
            min_b = p2 && !bma;
            mlane = bfound ? __ffs(bfound) - 1 : 0;
            mloc = tile_shfl<T>(ml, mlane);
        }
        // first empty slot index of each snapshot (B1 if none)
        const int la0 = be0 ? __ffs(be0) - 1 : 0;
        const int laa = bea ? __ffs(bea) - 1 : 0;
        const int lab = beb ? __ffs(beb) - 1 : 0;
        const int fea = tile_shfl<T>(fa, laa);
        const int feb = tile_shfl<T>(fb, lab);
        const int loada = bea ? laa * LF1 + fea : B1;
        const int loadb = beb ? lab * LF1 + feb : B1;
        // Definition 1: (1, y) precedes (2, y') iff y < y'; ties go to the second
        const bool pick_a = loada < loadb;
        const int load2 = pick_a ? loada : loadb;

        bool want_claim = false;
        int cl = 0;
        if (!LOOKUP && !bfound) {
            if (p1 && be0) {
                want_claim = true;
                cl = la0;
            } else if (p2 && load2 < B1) {
                want_claim = true;
                cl = pick_a ? laa : lab;
            }
        }
        bool claimed = false;
        uint64_t seen = 0;
        if (!LOOKUP && want_claim && tl == cl) {
            if (lvl == 1)
                claimed = claim_field<FPW0>(p0 + f0 / FPW0, f0 % FPW0, pick_word<W>(v0, f0 / FPW0),
                                            e0, seen, n_fail);
            else if (pick_a)
                claimed = claim_field_rt(FPW1, pa + fa / FPW1, fa % FPW1,
                                         pick_word<W>(va, fa / FPW1), ea, seen, n_fail);
            else
                claimed = claim_field_rt(FPW1, pb + fb / FPW1, fb % FPW1,
                                         pick_word<W>(vb, fb / FPW1), eb, seen, n_fail);
        }
        claimed = tile_shfl<T>(claimed, cl);
        seen = tile_shfl<T>(seen, cl);
        int cloc = 0;  // the claimed slot's local field in lane cl (slot outputs only)
        if (want_slots) cloc = tile_shfl<T>(lvl == 1 ? f0 : (pick_a ? fa : fb), cl);
        // level 3: a key whose three buckets are all full goes to the stash
        // (find-or-put), or is looked up there (lookup: only if both
        // secondaries are full, as full buckets stay full); the tile's first
        // lane probes and broadcasts the outcome
        const bool to_stash = ta.stash_slots && p2 && !bfound &&
                              (LOOKUP ? (!bea && !beb) : load2 >= B1);
        StashResult sr{LOOKUP ? ST_NOT_FOUND : ST_FULL, ~0ull};
        if (to_stash && tl == 0)
            sr = LOOKUP ? stash_find(ta, cur) : stash_find_or_put(ta, cur, n_fail);
        sr.status = (uint8_t)tile_shfl<T>((int)sr.status, 0);
        sr.pos = tile_shfl<T>(sr.pos, 0);

        if (act) {
            bool fin = true;
            uint8_t st = ST_NOT_FOUND;
            if (inval) {
                st = ST_INVALID;
            } else {
                n_probe += (lvl == 1) ? 1 : 2;
                if (bfound) {
                    st = ST_FOUND;
                } else if (LOOKUP) {
                    if (lvl == 1 && !be0) {
                        fin = false;
                        lvl = 2;
                    } else if (to_stash) {
                        st = sr.status;
                    }
                } else if (lvl == 1 && !be0) {
                    fin = false;
                    lvl = 2;
                } else if (lvl == 2 && load2 >= B1) {
                    st = sr.status;  // FULL, or the stash's answer
                    if (st == ST_PUT) n_write++;
                } else if (claimed) {
                    st = ST_PUT;
                    n_write++;
                } else {
                    const uint64_t mine = (lvl == 1) ? e0 : (pick_a ? ea : eb);
                    const int max_iter = iceberg_retry_bound(ta, WPB * FPW0, B1);
                    if (seen == mine) {
                        st = ST_FOUND;  // another thread inserted k first
                    } else if (++it > max_iter) {
                        st = ST_ERROR;
                    } else {
                        fin = false;  // re-read the bucket(s) at this level
                    }
                }
            }
            if (fin) {
                if (tl == 0) {
                    tw.s_st[tw.q] = st;
                    if (st == ST_ERROR) atomicOr(ta.err, 1u);
                    n_ops++;
                    if (want_slots) {
                        // FOUND by a match: the matching slot; PUT, or FOUND
                        // after losing the claim to k itself: the claimed slot
                        const uint64_t B0 = (uint64_t)WPB * FPW0;
                        uint64_t slot = ~0ull;
                        if (to_stash && (st == ST_FOUND || st == ST_PUT)) {
                            slot = L0.nb * B0 + L1.nb * (uint64_t)B1 + sr.pos;
                        } else if (st == ST_FOUND || st == ST_PUT) {
                            const bool bym = st == ST_FOUND && bfound;
                            const int ln = bym ? mlane : cl;
                            const int loc = bym ? mloc : cloc;
                            if (lvl == 1) {
                                slot = q0.a * B0 + (uint64_t)(ln * W * FPW0 + loc);
                            } else {
                                const bool inb = bym ? min_b : !pick_a;
                                slot = L0.nb * B0 + (inb ? qb.a : qa.a) * (uint64_t)B1 +
                                       (uint64_t)(ln * LF1 + loc);
                            }
                        }
                        if (tw.slots) tw.slots[tw.base + tw.q] = slot;
                        if (tw.kv->store) kv_move(*tw.kv, !LOOKUP, tw.base + tw.q, slot);
                    }
                }
                tw.q++;
                fresh = true;
            }
        }
        __syncwarp();
    }
    if (ctr) {
        if (tl != 0) n_probe = n_write = 0;
        flush_counter(ctr, 0, n_probe);
        flush_counter(ctr, 1, n_write);
        flush_counter(ctr, 2, (uint64_t)n_fail);
        flush_counter(ctr, 3, n_ops);
    }
}

template <int T, int FPW0, bool LOOKUP, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256)
    k_iceberg(TableArgs ta, const void *__restrict__ keys, uint64_t n,
              uint8_t *__restrict__ status, uint64_t *__restrict__ slots, KVArgs kv, int items) {
    extern __shared__ uint64_t smem[];
    SingleWork<T> tw;
    tw.init(smem, reinterpret_cast<uint8_t *>(smem + (size_t)blockDim.x * items), items, n,
            ta.max_tiles);
    tw.tap = &ta;
    tw.keys = keys;
    tw.n = n;
    tw.status = status;
    tw.slots = slots;
    tw.kv = &kv;
    iceberg_engine<T, FPW0, LOOKUP, SingleWork<T>, WPB>(tw, ta.ctr);
}

}  // namespace cht
