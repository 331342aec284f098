// cht_iceberg_stream.cuh - level 1 of iceberg find-or-put (Algorithm 1) and
// of the lookup (Section 2.3) as a stream of fully packed rounds, the form
// of the cuckoo stream kernels applied to the primary level.
//
// Each lane holds one key at a time. In every round each tile takes one step
// of all of its lanes' keys: tile lane s's key goes in slot s, and the
// primary buckets of Q slots are loaded back to back before any is
// inspected (Q lines in flight per tile). A slot's step is Algorithm 1's
// level-1 step: the bucket holds k's entry -> FOUND; it has an empty slot ->
// compare-and-swap the first one (split in two phases: all of a group's
// claims are issued before any outcome is read) -> PUT, or FOUND when the
// value that won is k's own entry, or another round at level 1 when another
// key won; the bucket is full -> level 2. A lookup step ends at the match
// (FOUND) or at a bucket with room (NOT_FOUND), and goes to level 2 at a full
// bucket. A lane whose key is answered writes its status and takes the next
// key of the warp's stream (its grid-stride 32-key chunks in order).
//
// Keys that go to level 2 get the status ST_PENDING here; the level-2 pass
// (iceberg_warp with RESUME) then takes exactly those keys, from the status
// array, through both secondary buckets and the stash. Running the level-2
// steps of a batch after its level-1 steps is one more interleaving of
// concurrent operations, each of which still follows Algorithm 1 step by
// step, so Theorem 1 holds as for any other schedule.
#pragma once

#include <type_traits>

#include "cht_kernels.cuh"

namespace cht {

// lookups: three blocks per SM (85 registers), as for the cuckoo lookup
// stream; find-or-puts carry the claims' state and run two
template <int T, int FPW0, int Q, bool LOOKUP, int WPB = kWordsPerBucket>
__global__ void __launch_bounds__(256, LOOKUP ? 3 : 2)
    k_iceberg_stream(TableArgs ta, const void *__restrict__ keys, uint64_t n,
                     uint8_t *__restrict__ status) {
    constexpr int W = WPB / T;
    constexpr int QE = Q < T ? Q : T;
    static_assert(T % QE == 0, "slots split evenly into load groups");
    constexpr uint32_t TM = (T == 32) ? 0xffffffffu : ((1u << T) - 1u);
    using Entry = typename std::conditional<(FPW0 >= 2), uint32_t, uint64_t>::type;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tbase = lane & ~(T - 1);
    const uint32_t tmask = TM << tbase;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const Level &L = ta.lv[0];
    uint64_t *wl = L.words + tl * W;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) << 5;
    const int max_iter = iceberg_retry_bound(ta, WPB * FPW0, WPB * ta.lv[1].fpw);
    uint64_t n_probe = 0, n_write = 0, n_ops = 0;
    int n_fail = 0;

    // key buffers: chunk A at baseA (next key at offset o), chunk B at baseA + stride
    uint64_t baseA = warp * 32;
    uint64_t kA = (baseA + lane < n) ? load_key(keys, ta.key_bytes, baseA + lane) : 0;
    uint64_t kB = (baseA + stride + lane < n) ? load_key(keys, ta.key_bytes, baseA + stride + lane)
                                              : 0;
    int o = 0;
    uint64_t cur = 0, idx = 0;
    int it = 0;
    bool live = false;
    // a bound on the rounds this warp can need: every round takes one step
    // of each live key and a key takes at most max_iter + 1 steps; past it
    // the warp records kErrLoopBound and stops, leaving its remaining keys'
    // statuses unwritten
    const uint64_t warp_keys = (n + stride - 1) / stride * 32 + 64;
    const uint64_t max_rounds = warp_keys * (uint64_t)(max_iter + 2) + 64;
    uint64_t rounds = 0;
    while (true) {
        if (++rounds > max_rounds) {
            if (lane == 0) atomicOr(ta.err, kErrLoopBound);
            break;
        }
        // refill the lanes without a key, in rank order
        const uint32_t need = __ballot_sync(0xffffffffu, !live);
        if (need) {
            const int src = o + __popc(need & lt_mask);
            const uint64_t ka = __shfl_sync(0xffffffffu, kA, src & 31);
            const uint64_t kb = __shfl_sync(0xffffffffu, kB, src & 31);
            if (!live) {
                idx = src < 32 ? baseA + src : baseA + stride + (src - 32);
                if (idx < n) {
                    cur = src < 32 ? ka : kb;
                    it = 0;
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
            if (baseA >= n) break;  // the warp's stream is exhausted
            continue;               // a round of invalid keys only
        }
        uint32_t addr = 0;
        Entry ent = 0;
        if (live) {
            const Quot q = quotient(L, ta.w, 0, cur);
            addr = (uint32_t)q.a;
            ent = (Entry)(((ta.compact ? q.r : cur) << 1) | 1ull);
        }
        const uint32_t pb = tile_ballot<T>(live);
#pragma unroll
        for (int s0 = 0; s0 < T; s0 += QE) {
            uint64_t v[QE][W];
            uint32_t a[QE];
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                a[q] = tile_shfl<T>(addr, s0 + q);
                load_relaxed_or_skip<W>((pb >> (s0 + q)) & 1u, wl + (uint64_t)a[q] * WPB, v[q]);
            }
            // inspect each slot; for a put, the owner of the first empty
            // slot issues the claim, none waits yet
            uint64_t old[QE], expd[QE];
            uint32_t bms = 0, bes = 0;  // bit q: slot q matched / had an empty slot
            int fidx[QE], actor[QE];
            Entry es[QE];
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const int s = s0 + q;
                const bool on = (pb >> s) & 1u;  // the same for the whole tile
                const Entry e = tile_shfl<T>(ent, s);
                es[q] = e;
                bool m;
                int fe;
                if constexpr (LOOKUP) {
                    bool le;
                    probe_chunk<W, FPW0>(v[q], e, m, le);
                    fe = le ? 0 : -1;  // only "the bucket has room" is used
                } else {
                    scan_chunk<W, FPW0>(v[q], e, m, fe);
                }
                const uint32_t bm = __ballot_sync(0xffffffffu, on && m) & tmask;
                const uint32_t be = LOOKUP ? (__ballot_sync(0xffffffffu, on && fe >= 0) &
                                              (1u << (tbase + T - 1)))
                                           : (__ballot_sync(0xffffffffu, on && fe >= 0) & tmask);
                bms |= (bm ? 1u : 0u) << q;
                bes |= (be ? 1u : 0u) << q;
                actor[q] = be ? __ffs(be) - 1 - tbase : 0;
                fidx[q] = fe;
                old[q] = expd[q] = 0;
                if constexpr (!LOOKUP) {
                    if (on && !bm && be && tl == actor[q]) {
                        uint64_t *p = wl + (uint64_t)a[q] * WPB + fe / FPW0;
                        old[q] = field_op_issue<FPW0>(false, p, fe % FPW0,
                                                      pick_word<W>(v[q], fe / FPW0), e, expd[q]);
                    }
                }
            }
            // outcomes back to each key's lane
#pragma unroll
            for (int q = 0; q < QE; ++q) {
                const int s = s0 + q;
                const bool on = (pb >> s) & 1u;
                const bool bm = (bms >> q) & 1u, be = (bes >> q) & 1u;
                int outcome = 0;  // 1: written, 2: k's own entry won the slot, 0: lost
                if constexpr (!LOOKUP) {
                    if (on && !bm && be && tl == actor[q]) {
                        uint64_t *p = wl + (uint64_t)a[q] * WPB + fidx[q] / FPW0;
                        uint64_t seen = 0;
                        const bool won = claim_finish<FPW0>(p, fidx[q] % FPW0, old[q], expd[q],
                                                            es[q], seen, n_fail);
                        outcome = won ? 1 : (seen == (uint64_t)es[q] ? 2 : 0);
                    }
                    outcome = tile_shfl<T>(outcome, actor[q]);
                }
                if (on && tl == s) {
                    n_probe++;
                    // the level-1 step's outcome; fin: the key leaves this
                    // kernel (ST_NOT_FOUND is 0, so the status alone cannot
                    // say whether the step has ended)
                    bool fin = true;
                    uint8_t out = ST_NOT_FOUND;
                    if (bm) {
                        out = ST_FOUND;
                    } else if (!be) {
                        out = ST_PENDING;  // primary full: level 2
                    } else if (LOOKUP) {
                        out = ST_NOT_FOUND;  // the primary has room and no k
                    } else if (outcome == 1) {
                        out = ST_PUT;
                        n_write++;
                    } else if (outcome == 2) {
                        out = ST_FOUND;  // another thread put k first
                    } else if (++it > max_iter) {
                        out = ST_ERROR;
                        atomicOr(ta.err, kErrRetry);
                    } else {
                        fin = false;  // lost the claim to another key: next round
                    }
                    if (fin) {
                        status[idx] = out;
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
