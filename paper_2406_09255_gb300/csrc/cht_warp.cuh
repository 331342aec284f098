// cht_warp.cuh - warp-batched iceberg find-or-put and lookup (Algorithm 1,
// Section 2.3) for unordered runs: the work sharing of Algorithm 3 with the
// per-key arithmetic taken out of the tile.
//
// A warp takes chunks of 32 * I keys (I = items per lane). Every lane holds I
// keys and computes their primary address and entry itself, once. Tiles of T
// lanes then walk the pending keys of their own lanes in passes: a level-1
// pass probes the primary bucket of every key still at level 1 (claiming its
// first empty slot, Algorithm 1 lines for level 1), a level-2 pass probes both
// secondary buckets of every key at level 2 (the secondary addresses are
// computed only for keys that get there). In one round a tile takes the next
// pending key of each of its I item slots, broadcasts their addresses
// (Shuffle), issues the I bucket loads back to back, and answers each with
// ballots (Any match, First empty); the lane owning the first empty slot does
// the compare-and-swap and broadcasts the outcome to the key's lane. A key
// whose claim lost a race is retried in the next pass at the same level, so
// each key still follows Algorithm 1 step by step; keys of different lanes
// interleave freely, as concurrent find-or-puts do.
#pragma once

#include <type_traits>

#include "cht_kernels.cuh"

namespace cht {

// a warp's share of the keys: up to 32 * I keys of one table
struct WarpChunk {
    const TableArgs *ta;
    const void *keys;
    uint8_t *status;
    uint64_t *slots;  // optional slot index per key (iceberg key-value handle)
    const KVArgs *kv;  // optional value moves (key-value extension)
    uint64_t base;
    int count;
};

// chunks of one table
struct SingleSource {
    const TableArgs *ta;
    const void *keys;
    uint8_t *status;
    uint64_t *slots;
    const KVArgs *kv;
    uint64_t n;
    uint64_t per;  // keys per chunk
    __device__ __forceinline__ uint64_t nchunks() const { return (n + per - 1) / per; }
    __device__ __forceinline__ WarpChunk get(uint64_t c) const {
        const uint64_t base = c * per;
        const uint64_t rem = n - base;
        return {ta, keys, status, slots, kv, base, (int)(rem < per ? rem : per)};
    }
};

// chunks of many tables: table t owns chunks [prefix[t], prefix[t+1])
struct BatchSource {
    const BatchDesc *bd;
    const uint64_t *prefix;
    int count;
    uint64_t per;
    __device__ __forceinline__ uint64_t nchunks() const { return prefix[count]; }
    __device__ __forceinline__ WarpChunk get(uint64_t c) const {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const BatchDesc &d = bd[lo];
        const uint64_t base = (c - prefix[lo]) * per;
        const uint64_t rem = d.n - base;
        return {&d.ta, d.keys, d.status, nullptr, nullptr, base, (int)(rem < per ? rem : per)};
    }
};

// SLOTS: also write each FOUND / PUT key's slot index to the chunk's slots
// array (the key-value extension); a separate instantiation, so that plain
// runs pay nothing for it
// RESUME: take only the keys whose status is ST_PENDING (left by the level-1
// stream kernel), start them at level 2, and write only their statuses
template <int T, int FPW0, int I, bool LOOKUP, class Src, bool SLOTS = false,
          int WPB = kWordsPerBucket, bool RESUME = false>
__device__ __forceinline__ void iceberg_warp(const Src &src, unsigned long long *ctr) {
    constexpr int W = WPB / T;
    constexpr uint32_t TM = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
    using E0 = typename std::conditional<(FPW0 >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tbase = lane & ~(T - 1);
    const uint32_t tmask = TM << tbase;
    const uint32_t last_lane = 1u << (tbase + T - 1);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    for (uint64_t c = warp; c < src.nchunks(); c += nwarps) {
        const WarpChunk ch = src.get(c);
        const TableArgs &ta = *ch.ta;
        const Level &L0 = ta.lv[0];
        const Level &L1 = ta.lv[1];
        const int FPW1 = L1.fpw;
        const int LF1 = W * FPW1;
        const int B1 = WPB * FPW1;
        const int max_iter = iceberg_retry_bound(ta, WPB * FPW0, B1);
        const uint64_t *w0 = L0.words + tl * W;
        const uint64_t *w1 = L1.words + tl * W;

        uint64_t k[I];
        uint32_t a0[I];
        E0 e0[I];
        bool pending[I], lvl2[I], lvl3[I];
        uint8_t st[I];
        int it[I];
        uint64_t slot_of[I];  // slot of a FOUND / PUT key (slot outputs only)
        // value moves: a put's value is read with the key, a get's value as
        // soon as the key is found, so both loads overlap the probe passes
        KVal vpre[I];
        const bool moves = SLOTS && ch.kv->store != nullptr;
        constexpr bool want_slots = SLOTS;
        const uint64_t B0 = (uint64_t)WPB * FPW0;
#pragma unroll
        for (int i = 0; i < I; ++i) {
            slot_of[i] = ~0ull;
            vpre[i] = KVal{0, 0};
            const int pos = i * 32 + lane;
            bool has = pos < ch.count;
            if constexpr (RESUME) has = has && ch.status[ch.base + pos] == ST_PENDING;
            k[i] = has ? load_key(ch.keys, ta.key_bytes, ch.base + pos) : 0;
            if (!LOOKUP && moves && has) vpre[i] = kv_read(ch.kv->vin, ch.base + pos, ch.kv->vbytes);
            pending[i] = has && valid_key(k[i], ta.w);
            st[i] = pending[i] ? ST_NOT_FOUND : ST_INVALID;
            lvl2[i] = RESUME;
            lvl3[i] = false;
            it[i] = 0;
            const Quot q = quotient(L0, ta.w, 0, k[i]);
            a0[i] = (uint32_t)q.a;
            e0[i] = (E0)(((ta.compact ? q.r : k[i]) << 1) | 1ull);
        }

        bool any_pending = false;
#pragma unroll
        for (int i = 0; i < I; ++i) any_pending |= pending[i];
        // every pass resolves each pending key or counts one of its lost
        // claims (at most max_iter per level, two levels and the stash), so
        // 2 * max_iter + 8 passes bound a chunk; past that the keys still
        // pending report ST_ERROR and kErrLoopBound is recorded
        int passes = 0;
        while (__any_sync(0xffffffffu, any_pending)) {
            if (++passes > 2 * max_iter + 8) {
#pragma unroll
                for (int i = 0; i < I; ++i)
                    if (pending[i]) {
                        st[i] = ST_ERROR;
                        pending[i] = false;
                    }
                if (lane == 0) atomicOr(ta.err, kErrLoopBound);
                break;
            }
            // ---- level-1 pass: the primary bucket of every key still at level 1
            uint32_t pm[I];
            bool more = false;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                pm[i] = __ballot_sync(0xffffffffu, pending[i] && !lvl2[i]) & tmask;
                more |= pm[i] != 0;
            }
            while (__any_sync(0xffffffffu, more)) {
                int r[I];
                E0 e[I];
                uint64_t v[I][W];
                const uint64_t *p[I];
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    r[i] = pm[i] ? __ffs(pm[i]) - 1 - tbase : -1;
                    pm[i] &= pm[i] - 1;
                    const int sl = r[i] & (T - 1);
                    const uint32_t a = tile_shfl<T>(a0[i], sl);
                    e[i] = tile_shfl<T>(e0[i], sl);
                    p[i] = w0 + (uint64_t)a * WPB;
#pragma unroll
                    for (int x = 0; x < W; ++x) v[i][x] = 0;
                    if (r[i] >= 0) load_relaxed<W>(p[i], v[i]);
                }
                more = false;
                // claims of all I items are issued before any outcome is read
                uint64_t old[I], expd[I];
                int fei[I], cli[I], y1[I];
                uint32_t bmv = 0, bev = 0;
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    more |= pm[i] != 0;
                    const bool live = r[i] >= 0;
                    if constexpr (LOOKUP) {
                        bool m, le;
                        int mpos = -1;
                        if constexpr (SLOTS)
                            probe_chunk_pos<W, FPW0>(v[i], e[i], m, le, mpos);
                        else
                            probe_chunk<W, FPW0>(v[i], e[i], m, le);
                        const uint32_t bm = __ballot_sync(0xffffffffu, live && m) & tmask;
                        const uint32_t be = __ballot_sync(0xffffffffu, live && le) & last_lane;
                        int y = 0;  // the matching slot's position in the bucket
                        if (want_slots) {
                            const int lm = bm ? __ffs(bm) - 1 - tbase : 0;
                            y = lm * W * FPW0 + tile_shfl<T>(mpos, lm);
                        }
                        if (tl == r[i]) {
                            n_probe++;
                            if (bm) {
                                st[i] = ST_FOUND;
                                pending[i] = false;
                                slot_of[i] = (uint64_t)a0[i] * B0 + (uint64_t)y;
                                if (moves && slot_of[i] < ch.kv->nstore)
                                    vpre[i] = kv_read(ch.kv->store, slot_of[i], ch.kv->vbytes);
                            } else if (be) {
                                pending[i] = false;  // NOT_FOUND
                            } else {
                                lvl2[i] = true;
                            }
                        }
                    } else {
                        bool m;
                        int fe, mpos = -1;
                        if constexpr (SLOTS)
                            scan_chunk_pos<W, FPW0>(v[i], e[i], m, fe, mpos);
                        else
                            scan_chunk<W, FPW0>(v[i], e[i], m, fe);
                        const uint32_t bm = __ballot_sync(0xffffffffu, live && m) & tmask;
                        const uint32_t be = __ballot_sync(0xffffffffu, live && fe >= 0) & tmask;
                        cli[i] = be ? __ffs(be) - 1 - tbase : 0;
                        fei[i] = fe;
                        y1[i] = 0;
                        if (want_slots) {
                            // the slot that answers: the match, else the one claimed
                            const int src = bm ? __ffs(bm) - 1 - tbase : cli[i];
                            y1[i] = src * W * FPW0 + tile_shfl<T>(bm ? mpos : fe, src);
                        }
                        bmv |= (bm ? 1u : 0u) << i;
                        bev |= (be ? 1u : 0u) << i;
                        old[i] = expd[i] = 0;
                        if (live && !bm && be && tl == cli[i])
                            old[i] = field_op_issue<FPW0>(
                                false, const_cast<uint64_t *>(p[i]) + fe / FPW0, fe % FPW0,
                                pick_word<W>(v[i], fe / FPW0), e[i], expd[i]);
                    }
                }
                if constexpr (!LOOKUP) {
#pragma unroll
                    for (int i = 0; i < I; ++i) {
                        const bool live = r[i] >= 0;
                        const bool bm = (bmv >> i) & 1u, be = (bev >> i) & 1u;
                        int outcome = 0;  // 1: written, 2: the same key won the slot, 0: lost
                        if (live && !bm && be && tl == cli[i]) {
                            uint64_t seen = 0;
                            const bool won = claim_finish<FPW0>(
                                const_cast<uint64_t *>(p[i]) + fei[i] / FPW0, fei[i] % FPW0, old[i],
                                expd[i], e[i], seen, n_fail);
                            outcome = won ? 1 : (seen == (uint64_t)e[i] ? 2 : 0);
                        }
                        outcome = tile_shfl<T>(outcome, cli[i]);
                        if (tl == r[i]) {
                            n_probe++;
                            const uint64_t at = (uint64_t)a0[i] * B0 + (uint64_t)y1[i];
                            if (bm) {
                                st[i] = ST_FOUND;
                                pending[i] = false;
                                slot_of[i] = at;
                            } else if (!be) {
                                lvl2[i] = true;  // level 1 is full for good
                            } else if (outcome == 1) {
                                st[i] = ST_PUT;
                                pending[i] = false;
                                n_write++;
                                slot_of[i] = at;
                            } else if (outcome == 2) {
                                st[i] = ST_FOUND;  // another thread put k first
                                pending[i] = false;
                                slot_of[i] = at;
                            } else if (++it[i] > max_iter) {
                                st[i] = ST_ERROR;
                                pending[i] = false;
                                atomicOr(ta.err, 1u);
                            }
                        }
                    }
                }
            }

            // ---- level-2 pass: both secondary buckets of every key at level 2
            uint32_t aa[I], ab[I];
            uint64_t ea[I], eb[I];
            more = false;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const bool at2 = pending[i] && lvl2[i] && !lvl3[i];
                pm[i] = __ballot_sync(0xffffffffu, at2) & tmask;
                more |= pm[i] != 0;
                aa[i] = ab[i] = 0;
                ea[i] = eb[i] = 0;
                if (at2) {
                    const Quot qa = quotient(L1, ta.w, 0, k[i]);
                    const Quot qb = quotient(L1, ta.w, 1, k[i]);
                    aa[i] = (uint32_t)qa.a;
                    ab[i] = (uint32_t)qb.a;
                    ea[i] = ((ta.compact ? qa.r : k[i]) << 2) | 1ull;
                    eb[i] = ((ta.compact ? qb.r : k[i]) << 2) | 2ull;
                }
            }
            while (__any_sync(0xffffffffu, more)) {
                more = false;
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    const int r = pm[i] ? __ffs(pm[i]) - 1 - tbase : -1;
                    pm[i] &= pm[i] - 1;
                    more |= pm[i] != 0;
                    const bool live = r >= 0;
                    const int sl = r & (T - 1);
                    const uint32_t xa = tile_shfl<T>(aa[i], sl), xb = tile_shfl<T>(ab[i], sl);
                    const uint64_t ya = tile_shfl<T>(ea[i], sl), yb = tile_shfl<T>(eb[i], sl);
                    uint64_t *pa = const_cast<uint64_t *>(w1) + (uint64_t)xa * WPB;
                    uint64_t *pb = const_cast<uint64_t *>(w1) + (uint64_t)xb * WPB;
                    uint64_t va[W] = {}, vb[W] = {};
                    if (live) {
                        load_relaxed<W>(pa, va);
                        load_relaxed<W>(pb, vb);
                    }
                    bool ma, mb;
                    int fa, fb, pa_pos = -1, pb_pos = -1;
                    if constexpr (SLOTS) {
                        scan_chunk_rt_pos<W>(va, ya, FPW1, ma, fa, pa_pos);
                        scan_chunk_rt_pos<W>(vb, yb, FPW1, mb, fb, pb_pos);
                    } else {
                        scan_chunk_rt<W>(va, ya, FPW1, ma, fa);
                        scan_chunk_rt<W>(vb, yb, FPW1, mb, fb);
                    }
                    const uint32_t bfound = __ballot_sync(0xffffffffu, live && (ma || mb)) & tmask;
                    // slot outputs: where the match sits (bucket b?, lane, field)
                    int mval = 0;
                    bool mb_side = false;
                    if (want_slots) {
                        const uint32_t bma = __ballot_sync(0xffffffffu, live && ma) & tmask;
                        mb_side = !bma;
                        mval = ma ? pa_pos : pb_pos;
                    }
                    const uint64_t lvl2_base = L0.nb * B0;
                    if constexpr (LOOKUP) {
                        int y = 0;
                        if (want_slots) {
                            const int lm = bfound ? __ffs(bfound) - 1 - tbase : 0;
                            y = lm * LF1 + tile_shfl<T>(mval, lm);
                        }
                        // level 3 holds k only if both secondaries were full
                        // when it was put, and full buckets stay full
                        bool both_full = false;
                        if (ta.stash_slots) {
                            const uint32_t bea = __ballot_sync(0xffffffffu, live && fa >= 0) & tmask;
                            const uint32_t beb = __ballot_sync(0xffffffffu, live && fb >= 0) & tmask;
                            both_full = !bea && !beb;
                        }
                        if (tl == r) {
                            n_probe += 2;
                            if (bfound) {
                                st[i] = ST_FOUND;
                                slot_of[i] = lvl2_base + (uint64_t)(mb_side ? ab[i] : aa[i]) * B1 +
                                        (uint64_t)y;
                                if (moves && slot_of[i] < ch.kv->nstore)
                                    vpre[i] = kv_read(ch.kv->store, slot_of[i], ch.kv->vbytes);
                            }
                            if (!bfound && both_full)
                                lvl3[i] = true;  // the stash, after this pass
                            else
                                pending[i] = false;
                        }
                    } else {
                        const uint32_t bea = __ballot_sync(0xffffffffu, live && fa >= 0) & tmask;
                        const uint32_t beb = __ballot_sync(0xffffffffu, live && fb >= 0) & tmask;
                        const int laa = bea ? __ffs(bea) - 1 - tbase : 0;
                        const int lab = beb ? __ffs(beb) - 1 - tbase : 0;
                        const int fea = tile_shfl<T>(fa, laa);
                        const int feb = tile_shfl<T>(fb, lab);
                        const int loada = bea ? laa * LF1 + fea : B1;
                        const int loadb = beb ? lab * LF1 + feb : B1;
                        // Definition 1: (1, y) precedes (2, y') iff y < y'; ties to the second
                        const bool pick_a = loada < loadb;
                        const int load2 = pick_a ? loada : loadb;
                        const int cl = pick_a ? laa : lab;
                        bool claimed = false;
                        uint64_t seen = 0;
                        if (live && !bfound && load2 < B1 && tl == cl) {
                            if (pick_a)
                                claimed = claim_field_rt(FPW1, pa + fa / FPW1, fa % FPW1,
                                                         pick_word<W>(va, fa / FPW1), ya, seen,
                                                         n_fail);
                            else
                                claimed = claim_field_rt(FPW1, pb + fb / FPW1, fb % FPW1,
                                                         pick_word<W>(vb, fb / FPW1), yb, seen,
                                                         n_fail);
                        }
                        claimed = tile_shfl<T>(claimed, cl);
                        seen = tile_shfl<T>(seen, cl);
                        int y = 0;
                        if (want_slots) {
                            // the slot that answers: the match, else the one claimed
                            const int src = bfound ? __ffs(bfound) - 1 - tbase : cl;
                            y = src * LF1 + tile_shfl<T>(bfound ? mval : (pick_a ? fa : fb), src);
                        }
                        const bool in_b = bfound ? mb_side : !pick_a;
                        const uint64_t at =
                            lvl2_base + (uint64_t)(in_b ? ab[i] : aa[i]) * B1 + (uint64_t)y;
                        if (tl == r) {
                            n_probe += 2;
                            if (bfound) {
                                st[i] = ST_FOUND;
                                pending[i] = false;
                                slot_of[i] = at;
                            } else if (load2 >= B1) {
                                if (ta.stash_slots) {
                                    lvl3[i] = true;  // the stash, after this pass
                                } else {
                                    st[i] = ST_FULL;
                                    pending[i] = false;
                                }
                            } else if (claimed) {
                                st[i] = ST_PUT;
                                pending[i] = false;
                                n_write++;
                                slot_of[i] = at;
                            } else if (seen == (pick_a ? ya : yb)) {
                                st[i] = ST_FOUND;
                                pending[i] = false;
                                slot_of[i] = at;
                            } else if (++it[i] > max_iter) {
                                st[i] = ST_ERROR;
                                pending[i] = false;
                                atomicOr(ta.err, 1u);
                            }
                        }
                    }
                }
            }
            // ---- level 3: keys whose three buckets are all full go to the
            // stash, each lane its own keys (rare: only near capacity)
            if (ta.stash_slots) {
                const uint64_t stash_base = L0.nb * B0 + L1.nb * (uint64_t)B1;
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    if (pending[i] && lvl3[i]) {
                        const StashResult sr = LOOKUP ? stash_find(ta, k[i])
                                                      : stash_find_or_put(ta, k[i], n_fail);
                        st[i] = sr.status;
                        pending[i] = false;
                        if (sr.status == ST_PUT) n_write++;
                        if (sr.status == ST_FOUND || sr.status == ST_PUT) {
                            slot_of[i] = stash_base + sr.pos;
                            if (LOOKUP && moves && slot_of[i] < ch.kv->nstore)
                                vpre[i] = kv_read(ch.kv->store, slot_of[i], ch.kv->vbytes);
                        }
                    }
                }
            }
            any_pending = false;
#pragma unroll
            for (int i = 0; i < I; ++i) any_pending |= pending[i];
        }
#pragma unroll
        for (int i = 0; i < I; ++i) {
            const int pos = i * 32 + lane;
            // a resumed run writes back only the keys it took (valid keys
            // reach the end with a final status: pending is false)
            if (pos < ch.count && (!RESUME || k[i] != 0)) {
                ch.status[ch.base + pos] = st[i];
                if constexpr (SLOTS) {
                    if (ch.slots) ch.slots[ch.base + pos] = slot_of[i];
                    if (moves) {
                        if (LOOKUP)
                            kv_write(ch.kv->vout, ch.base + pos, ch.kv->vbytes, vpre[i]);
                        else if (slot_of[i] < ch.kv->nstore)
                            kv_write(ch.kv->store, slot_of[i], ch.kv->vbytes, vpre[i]);
                    }
                }
            }
            n_ops += (!RESUME && pos < ch.count) ? 1 : 0;
        }
    }
    if (ctr) {
        flush_counter(ctr, 0, n_probe);
        flush_counter(ctr, 1, n_write);
        flush_counter(ctr, 2, (uint64_t)n_fail);
        flush_counter(ctr, 3, n_ops);
    }
}

// five blocks per SM (48 registers): measured 5-8 % faster than four blocks
// with fewer spills, and faster than six blocks with more
template <int T, int FPW0, int I, bool LOOKUP, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, 5)
    k_iceberg_warp(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                   uint8_t *__restrict__ status) {
    SingleSource src{&ta, keys, status, nullptr, nullptr, n, (uint64_t)32 * I};
    iceberg_warp<T, FPW0, I, LOOKUP, SingleSource, false, WPB>(src, ta.ctr);
}

// level 2 (and the stash) for the keys the level-1 stream kernel left
// pending; one key per lane, five blocks per SM as for the engine above
template <int T, int FPW0, bool LOOKUP, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, 5)
    k_iceberg_resume(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                     uint8_t *__restrict__ status) {
    SingleSource src{&ta, keys, status, nullptr, nullptr, n, 32};
    iceberg_warp<T, FPW0, 1, LOOKUP, SingleSource, false, WPB, true>(src, ta.ctr);
}

// with slot outputs and value moves (one key per lane); held to 64 registers
// so that four blocks share an SM, as for the plain engine
template <int T, int FPW0, bool LOOKUP>
__global__ void __launch_bounds__(256, 4)
    k_iceberg_warp_slots(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                         uint8_t *__restrict__ status, uint64_t *__restrict__ slots, KVArgs kv) {
    SingleSource src{&ta, keys, status, slots, &kv, n, 32};
    iceberg_warp<T, FPW0, 1, LOOKUP, SingleSource, true>(src, ta.ctr);
}

// one persistent launch over many tables; shared memory holds the prefix of
// the tables' chunk counts (chunks of 32 * I keys), scanned by the first warp
template <int T, int FPW0, int I, bool LOOKUP>
__device__ __forceinline__ void iceberg_batch_body(const BatchDesc *__restrict__ bd, int count,
                                                   unsigned long long *ctr) {
    extern __shared__ uint64_t smem[];
    uint64_t *prefix = smem;  // count + 1 entries
    const uint64_t per = (uint64_t)32 * I;
    if (threadIdx.x < 32) {
        uint64_t carry = 0;
        for (int b0 = 0; b0 < count; b0 += 32) {
            const int t = b0 + (int)threadIdx.x;
            const uint64_t cnt = t < count ? (bd[t].n + per - 1) / per : 0;
            uint64_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)threadIdx.x >= o) incl += y;
            }
            if (t < count) prefix[t] = carry + incl - cnt;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (threadIdx.x == 0) prefix[count] = carry;
    }
    __syncthreads();
    BatchSource src{bd, prefix, count, per};
    iceberg_warp<T, FPW0, I, LOOKUP>(src, ctr);
}

template <int T, int FPW0, int I, bool LOOKUP>
__global__ void __launch_bounds__(256)
    k_iceberg_batch(const BatchDesc *__restrict__ bd, int count, unsigned long long *ctr) {
    iceberg_batch_body<T, FPW0, I, LOOKUP>(bd, count, ctr);
}

// one key per lane: five blocks per SM, as for the single-table engine
template <int T, int FPW0, bool LOOKUP>
__global__ void __launch_bounds__(256, 5)
    k_iceberg_batch1(const BatchDesc *__restrict__ bd, int count, unsigned long long *ctr) {
    iceberg_batch_body<T, FPW0, 1, LOOKUP>(bd, count, ctr);
}

}  // namespace cht
