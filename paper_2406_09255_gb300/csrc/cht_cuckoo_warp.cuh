// cht_cuckoo_warp.cuh - compact cuckoo put (Algorithm 4) for unordered
// runs: the warp-batched chunk form described here, and the stream form
// (k_cuckoo_insert_stream, the default) described at its definition below.
//
// A warp takes chunks of 32 * I keys; every lane holds I keys "in hand", each
// with its hash index j and step count c. In each pass, tiles of T lanes
// probe the bucket a_j of every pending key of their lanes once, I keys per
// round in flight: if the snapshot has an empty slot, the lane owning the
// first one compare-and-swaps (r_j, j) into it; otherwise the lane owning the
// slot chosen from (k, c) swaps the entry in, and the evicted entry goes back
// to the key's lane, which decodes the evicted key, k' = pi_j'^-1(a . r'), and
// continues with it under hash j' + 1 in the next pass. A lost claim, like a
// swap, uses up one of the C steps; after C steps the put reports FULL and the
// key in hand is the dropped one.
#pragma once

#include <type_traits>

#include "cht_kernels.cuh"

namespace cht {

template <int T, int FPW, int I, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256)
    k_cuckoo_insert_warp(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                         uint8_t *__restrict__ status, uint64_t *__restrict__ dropped) {
    constexpr int W = WPB / T;
    constexpr int LF = W * FPW;               // fields per lane
    constexpr int B = WPB * FPW;  // slots per bucket
    constexpr uint32_t TM = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
    using Entry = typename std::conditional<(FPW >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tbase = lane & ~(T - 1);
    const uint32_t tmask = TM << tbase;
    const Level &L = ta.lv[0];
    const uint64_t *wl = L.words + tl * W;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t per = (uint64_t)32 * I;
    const uint64_t nchunks = (n + per - 1) / per;
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    for (uint64_t c0 = warp; c0 < nchunks; c0 += nwarps) {
        const uint64_t base = c0 * per;
        uint64_t cur[I];
        int j[I], c[I];
        bool pending[I];
        uint8_t st[I];
#pragma unroll
        for (int i = 0; i < I; ++i) {
            const uint64_t idx = base + i * 32 + lane;
            const bool has = idx < n;
            cur[i] = has ? load_key(keys, ta.key_bytes, idx) : 0;
            pending[i] = has && valid_key(cur[i], ta.w);
            st[i] = pending[i] ? ST_PUT : ST_INVALID;
            j[i] = 0;
            c[i] = 1;
        }
        bool any_pending = false;
#pragma unroll
        for (int i = 0; i < I; ++i) any_pending |= pending[i];
        while (__any_sync(0xffffffffu, any_pending)) {
            // this pass: one step of every pending key at its (k, j, c)
            uint32_t addr[I], pm[I];
            Entry ent[I];
            int ysl[I];
            bool more = false;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                addr[i] = 0;
                ent[i] = 0;
                ysl[i] = 0;
                if (pending[i]) {
                    const Quot q = quotient(L, ta.w, j[i], cur[i]);
                    addr[i] = (uint32_t)q.a;
                    ent[i] = (Entry)(((ta.compact ? q.r : cur[i]) << 2) | (uint64_t)(j[i] + 1));
                    // the slot to evict should the bucket be full: "based on c, k"
                    ysl[i] = (int)(((splitmix(cur[i], (uint64_t)c[i]) >> 32) * (uint64_t)B) >> 32);
                }
                pm[i] = __ballot_sync(0xffffffffu, pending[i]) & tmask;
                more |= pm[i] != 0;
            }
            while (__any_sync(0xffffffffu, more)) {
                int r[I];
                Entry e[I];
                uint64_t v[I][W];
                uint64_t *p[I];
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    r[i] = pm[i] ? __ffs(pm[i]) - 1 - tbase : -1;
                    pm[i] &= pm[i] - 1;
                    const int sl = r[i] & (T - 1);
                    const uint32_t a = tile_shfl<T>(addr[i], sl);
                    e[i] = tile_shfl<T>(ent[i], sl);
                    p[i] = const_cast<uint64_t *>(wl) + (uint64_t)a * WPB;
#pragma unroll
                    for (int x = 0; x < W; ++x) v[i][x] = 0;
                    if (r[i] >= 0) load_relaxed<W>(p[i], v[i]);
                }
                more = false;
#pragma unroll
                for (int i = 0; i < I; ++i) {
                    more |= pm[i] != 0;
                    const bool live = r[i] >= 0;
                    const int sl = r[i] & (T - 1);
                    const int y = tile_shfl<T>(ysl[i], sl);
                    bool m;
                    int fe;
                    scan_chunk<W, FPW>(v[i], e[i], m, fe);
                    const uint32_t be = __ballot_sync(0xffffffffu, live && fe >= 0) & tmask;
                    const int cl = be ? __ffs(be) - 1 - tbase : 0;
                    const int el = y / LF, ef = y - el * LF;
                    bool claimed = false, swap_ok = true;
                    uint64_t seen = 0, evicted = 0;
                    if (live && be && tl == cl)
                        claimed = claim_field<FPW>(p[i] + fe / FPW, fe % FPW,
                                                   pick_word<W>(v[i], fe / FPW), e[i], seen,
                                                   n_fail);
                    if (live && !be && tl == el)
                        evicted = swap_field<FPW>(p[i] + ef / FPW, ef % FPW,
                                                  pick_word<W>(v[i], ef / FPW), e[i], swap_ok);
                    claimed = tile_shfl<T>(claimed, cl);
                    evicted = tile_shfl<T>(evicted, el);
                    swap_ok = tile_shfl<T>(swap_ok, el);
                    if (tl == r[i]) {
                        n_probe++;
                        if (be) {
                            if (claimed) {
                                pending[i] = false;  // PUT
                                n_write++;
                            } else if (++c[i] > ta.C) {
                                pending[i] = false;
                                st[i] = ST_FULL;
                            }
                        } else if (!swap_ok) {
                            pending[i] = false;
                            st[i] = ST_ERROR;
                            atomicOr(ta.err, 1u);
                        } else {
                            n_write++;
                            if (evicted == 0) {
                                pending[i] = false;  // the chosen slot held nothing: placed
                            } else {
                                const int jo = (int)(evicted & 3) - 1;
                                cur[i] = ta.compact ? unquotient(L, jo, addr[i], evicted >> 2)
                                                    : (evicted >> 2);
                                j[i] = (jo + 1 == ta.H) ? 0 : jo + 1;
                                if (++c[i] > ta.C) {
                                    pending[i] = false;
                                    st[i] = ST_FULL;
                                }
                            }
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
            const uint64_t idx = base + i * 32 + lane;
            if (idx < n) {
                status[idx] = st[i];
                if (st[i] == ST_FULL && dropped) dropped[idx] = cur[i];
                n_ops++;
            }
        }
    }
    if (ta.ctr) {
        flush_counter(ta.ctr, 0, n_probe);
        flush_counter(ta.ctr, 1, n_write);
        flush_counter(ta.ctr, 2, (uint64_t)n_fail);
        flush_counter(ta.ctr, 3, n_ops);
    }
}

// ===========================================================================
// The put of Algorithm 4 as a stream of rounds. Each lane holds one key in
// hand (k, j, c) at a time. In every round each tile takes one step of all
// of its lanes' keys: tile lane s's key goes in slot s, and the buckets of Q
// slots are loaded back to back before any is inspected (Q lines in flight
// per tile). A slot's step is the same as above: claim the first empty slot
// of the snapshot, else swap the entry into the slot chosen from (k, c) and
// carry the evicted key on under hash j' + 1. A slot's snapshot may predate
// a claim made by an earlier slot of the same round; such a claim fails and
// is retried like any lost race. A lane whose put ended (PUT, FULL, ERROR)
// writes its status and takes the next key of the warp's stream (its
// grid-stride 32-key chunks in order) for the next round, so long eviction
// chains do not hold other lanes idle.
// ===========================================================================
template <int T, int FPW, int Q, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, 2)
    k_cuckoo_insert_stream(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                           uint8_t *__restrict__ status, uint64_t *__restrict__ dropped) {
    constexpr int W = WPB / T;
    constexpr int LF = W * FPW;               // fields per lane
    constexpr int B = WPB * FPW;  // slots per bucket
    constexpr int QE = Q < T ? Q : T;
    static_assert(T % QE == 0, "slots split evenly into load groups");
    constexpr uint32_t TM = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
    using Entry = typename std::conditional<(FPW >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tbase = lane & ~(T - 1);
    const uint32_t tmask = TM << tbase;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const Level &L = ta.lv[0];
    uint64_t *wl = L.words + tl * W;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) << 5;
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    uint64_t baseA = warp * 32;
    uint64_t kA = (baseA + lane < n) ? load_key(keys, ta.key_bytes, baseA + lane) : 0;
    uint64_t kB = (baseA + stride + lane < n) ? load_key(keys, ta.key_bytes, baseA + stride + lane)
                                              : 0;
    int o = 0;
    uint64_t cur = 0, idx = 0;
    int j = 0, c = 1;
    bool live = false;
    while (true) {
        const uint32_t need = __ballot_sync(0xffffffffu, !live);
        if (need) {
            const int src = o + __popc(need & lt_mask);
            const uint64_t ka = __shfl_sync(0xffffffffu, kA, src & 31);
            const uint64_t kb = __shfl_sync(0xffffffffu, kB, src & 31);
            if (!live) {
                idx = src < 32 ? baseA + src : baseA + stride + (src - 32);
                if (idx < n) {
                    cur = src < 32 ? ka : kb;
                    j = 0;
                    c = 1;
                    n_ops++;
                    if (valid_key(cur, ta.w))
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
            if (baseA >= n) break;
            continue;
        }
        // this round: one step of every lane's key at its (k, j, c)
        uint32_t addr = 0;
        Entry ent = 0;
        int ysl = 0;
        if (live) {
            const Quot q = quotient(L, ta.w, j, cur);
            addr = (uint32_t)q.a;
            ent = (Entry)(((ta.compact ? q.r : cur) << 2) | (uint64_t)(j + 1));
            // the slot to evict should the bucket be full: "based on c, k"
            ysl = (int)(((splitmix(cur, (uint64_t)c) >> 32) * (uint64_t)B) >> 32);
        }
        const uint32_t pb = tile_ballot<T>(live);
#pragma unroll
        for (int s0 = 0; s0 < T; s0 += QE) {
            uint64_t v[QE][W];
            uint32_t a[QE];
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                a[q] = tile_shfl<T>(addr, s0 + q);
                load_relaxed_or_skip<W>((pb >> (s0 + q)) & 1u, wl + (uint64_t)a[q] * WPB,
                                        v[q]);
            }
            // issue: per slot, the acting lane (owner of the first empty slot,
            // or of the slot to evict) starts its atomic; none waits yet
            uint64_t old[QE], expd[QE];
            uint32_t bes = 0;  // bit q: slot q's snapshot had an empty slot
            int fidx[QE], actor[QE];
            Entry es[QE];
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const int s = s0 + q;
                const bool on = (pb >> s) & 1u;  // the same for the whole tile
                const Entry e = tile_shfl<T>(ent, s);
                es[q] = e;
                const int y = tile_shfl<T>(ysl, s);
                bool m;
                int fe;
                scan_chunk<W, FPW>(v[q], e, m, fe);
                const uint32_t be = __ballot_sync(0xffffffffu, on && fe >= 0) & tmask;
                const int cl = be ? __ffs(be) - 1 - tbase : 0;
                const int el = y / LF, ef = y - el * LF;
                actor[q] = be ? cl : el;
                fidx[q] = be ? fe : ef;
                bes |= (be ? 1u : 0u) << q;
                old[q] = expd[q] = 0;
                if (on && tl == actor[q]) {
                    uint64_t *p = wl + (uint64_t)a[q] * WPB + fidx[q] / FPW;
                    old[q] = field_op_issue<FPW>(!be, p, fidx[q] % FPW,
                                                 pick_word<W>(v[q], fidx[q] / FPW), e, expd[q]);
                }
            }
            // finish: outcomes back to each key's lane
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const int s = s0 + q;
                const bool on = (pb >> s) & 1u;
                const bool be = (bes >> q) & 1u;
                bool claimed = false, swap_ok = true;
                uint64_t evicted = 0;
                if (on && tl == actor[q]) {
                    uint64_t *p = wl + (uint64_t)a[q] * WPB + fidx[q] / FPW;
                    if (be) {
                        uint64_t seen = 0;
                        claimed = claim_finish<FPW>(p, fidx[q] % FPW, old[q], expd[q], es[q],
                                                    seen, n_fail);
                    } else {
                        evicted = swap_finish<FPW>(p, fidx[q] % FPW, old[q], expd[q], es[q],
                                                   swap_ok);
                    }
                }
                const int flags = tile_shfl<T>((claimed ? 1 : 0) | (swap_ok ? 2 : 0), actor[q]);
                evicted = tile_shfl<T>(evicted, actor[q]);
                claimed = flags & 1;
                swap_ok = (flags & 2) != 0;
                if (on && tl == s) {
                    n_probe++;
                    uint8_t done = 0;  // status once the put has ended
                    if (be) {
                        if (claimed) {
                            done = ST_PUT;
                            n_write++;
                        } else if (++c > ta.C) {
                            done = ST_FULL;
                        }
                    } else if (!swap_ok) {
                        done = ST_ERROR;
                        atomicOr(ta.err, 1u);
                    } else {
                        n_write++;
                        if (evicted == 0) {
                            done = ST_PUT;  // the chosen slot held nothing: placed
                        } else {
                            const int jo = (int)(evicted & 3) - 1;
                            cur = ta.compact ? unquotient(L, jo, addr, evicted >> 2)
                                             : (evicted >> 2);
                            j = (jo + 1 == ta.H) ? 0 : jo + 1;
                            if (++c > ta.C) done = ST_FULL;
                        }
                    }
                    if (done) {
                        status[idx] = done;
                        if (done == ST_FULL && dropped) dropped[idx] = cur;
                        live = false;
                    }
                }
            }
        }
    }
    if (ta.ctr) {
        flush_counter(ta.ctr, 0, n_probe);
        flush_counter(ta.ctr, 1, n_write);
        flush_counter(ta.ctr, 2, (uint64_t)n_fail);
        flush_counter(ta.ctr, 3, n_ops);
    }
}

}  // namespace cht
