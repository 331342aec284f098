// cht_cuckoo_warp.cuh - warp-batched compact cuckoo put (Algorithm 4) for
// unordered runs.
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

template <int T, int FPW, int I>
__global__ void __launch_bounds__(256)
    k_cuckoo_insert_warp(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                         uint8_t *__restrict__ status, uint64_t *__restrict__ dropped) {
    constexpr int W = kWordsPerBucket / T;
    constexpr int LF = W * FPW;               // fields per lane
    constexpr int B = kWordsPerBucket * FPW;  // slots per bucket
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
                    p[i] = const_cast<uint64_t *>(wl) + (uint64_t)a * kWordsPerBucket;
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

}  // namespace cht
