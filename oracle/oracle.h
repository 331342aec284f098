/*
 * oracle.h - sequential CPU oracle for compact bucketed cuckoo hashing and
 * compact two-level iceberg hashing (Hegeman, Woeltgens, Wijs, Laarman,
 * "Compact Parallel Hash Tables on the GPU").
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may call this code. It shares no code with the CUDA
 * library: it has its own permutation, slot layout, encodings and algorithms,
 * written plainly and sequentially so that each step can be checked against
 * the paper by eye. Keys are processed strictly in input order.
 *
 * Table memory is an array of 64-bit words. A bucket is wpb words; 16 words
 * make one 128-byte cache line (Section 4.5), and smaller buckets (down to one
 * word) serve brute-force tests on tiny tables. Level 0 is the cuckoo table or the iceberg
 * primary level; level 1 is the iceberg secondary (backyard) level. Slot y of
 * a bucket lives in word y / fpw, bits [(y % fpw) * s, (y % fpw) * s + s),
 * where fpw is the number of fields per word and s = 64 / fpw.
 *
 * An iceberg table may have a third level (Section 2.3 describes it; the
 * paper's implementation leaves it out, Section 3): an overflow stash of
 * `stash` whole-key slots stored after the secondary level's words in the
 * level-1 array. A key goes there only when its primary and both secondary
 * buckets are full; the stash is an open-addressing table with linear
 * probing from a hash of the key (this library's design: the paper gives
 * none).
 */
#ifndef CHT_ORACLE_H
#define CHT_ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* per-key outcome codes (Section 3: found / put / full, plus lookups) */
enum {
    ORC_NOT_FOUND = 0,
    ORC_FOUND = 1,
    ORC_PUT = 2,
    ORC_FULL = 3,
    ORC_INVALID = 4
};

typedef struct {
    int kind;          /* 0 = bucketed cuckoo, 1 = two-level iceberg          */
    int compact;       /* 1 = quotiented remainders, 0 = whole key per slot    */
    int key_bits;      /* w: keys are integers in [1, 2^w)                     */
    int num_hashes;    /* cuckoo H (1..3); ignored for iceberg                 */
    int max_chain;     /* cuckoo C: eviction steps before a put reports full   */
    int wpb;           /* 64-bit words per bucket (16 = one 128-byte line)     */
    int fpw[2];        /* fields per 64-bit word, per level                    */
    uint64_t nb[2];    /* bucket counts, per level (nb[1] = 0 for cuckoo)      */
    uint64_t seed;     /* all permutation constants derive from this           */
    uint64_t stash;    /* iceberg level-3 overflow stash: 0 (none) or a power  */
                       /* of two, its slot count                               */
} orc_cfg;

/* 0 if the configuration is usable: every encoded entry fits its field, the
 * bucket counts are powers of two where quotienting needs them, and the sizes
 * are in range; otherwise a nonzero code naming the first failed check. */
int orc_cfg_check(const orc_cfg *c);

/* --- permutation and quotient (Section 2.4, Section 4.3) --- */
uint64_t orc_perm(const orc_cfg *c, int level, int j, uint64_t k);
uint64_t orc_perm_inv(const orc_cfg *c, int level, int j, uint64_t p);
uint64_t orc_address(const orc_cfg *c, int level, int j, uint64_t k);
uint64_t orc_remainder(const orc_cfg *c, int level, int j, uint64_t k);
uint64_t orc_key_from(const orc_cfg *c, int level, int j, uint64_t a, uint64_t r);

/* batch form of the above for tests: out_perm/out_addr/out_rem may be NULL */
void orc_perm_many(const orc_cfg *c, int level, int j, const uint64_t *keys,
                   size_t n, uint64_t *out_perm, uint64_t *out_addr,
                   uint64_t *out_rem, uint64_t *out_back);

/* --- slot order of Definition 1 (Appendix A) --- */
int orc_prec(int x1, int y1, int x2, int y2);

/* --- table geometry --- */
/* words of a level's array (level 1 includes the stash, if any) */
uint64_t orc_table_words(const orc_cfg *c, int level);
/* first stash position of key k (linear probing continues from it) */
uint64_t orc_stash_home(const orc_cfg *c, uint64_t k);
int orc_slots_per_bucket(const orc_cfg *c, int level);
uint64_t orc_get_slot(const orc_cfg *c, int level, const uint64_t *table,
                      uint64_t bucket, int y);
/* write slot y of a bucket (tests use it to plant invariant violations) */
void orc_set_slot(const orc_cfg *c, int level, uint64_t *table,
                  uint64_t bucket, int y, uint64_t v);
/* the encoded entry of key k under choice x, and the bucket it belongs in:
 * cuckoo x = hash index j (level 0); iceberg x = 0 primary, 1 and 2 the two
 * secondary choices (level 1) */
uint64_t orc_entry_of(const orc_cfg *c, int x, uint64_t k);
uint64_t orc_bucket_of(const orc_cfg *c, int x, uint64_t k);

/* --- operations (all sequential, keys in input order) --- */
/* Algorithm 4 read sequentially. status[i] in {PUT, FULL, INVALID}; when a put
 * runs out of chain steps, dropped[i] holds the key that was left without a
 * slot (it may differ from keys[i]). probes/writes count bucket reads and slot
 * writes summed over the batch. */
void orc_cuckoo_insert(const orc_cfg *c, uint64_t *table, const uint64_t *keys,
                       size_t n, uint8_t *status, uint64_t *dropped,
                       uint64_t *probes, uint64_t *writes);
/* Section 4.4 lookup with early stop. */
void orc_cuckoo_find(const orc_cfg *c, const uint64_t *table,
                     const uint64_t *keys, size_t n, uint8_t *status,
                     uint64_t *probes);
/* Lookup that inspects every slot of all H buckets (no early stop). */
void orc_cuckoo_find_exhaustive(const orc_cfg *c, const uint64_t *table,
                                const uint64_t *keys, size_t n,
                                uint8_t *status);
/* Algorithm 5 (simplified find-or-put) read sequentially. */
void orc_iceberg_fop(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                     const uint64_t *keys, size_t n, uint8_t *status,
                     uint64_t *probes, uint64_t *writes);
/* Section 2.3 lookup over levels 1 and 2. */
void orc_iceberg_find(const orc_cfg *c, const uint64_t *t0, const uint64_t *t1,
                      const uint64_t *keys, size_t n, uint8_t *status,
                      uint64_t *probes);
/* Slot index of each key in an iceberg table: level-0 slot y of bucket a is
 * a * B0 + y, level-1 slot y of bucket a is nb0 * B0 + a * B1 + y (B = slots
 * per bucket of the level); UINT64_MAX for absent or invalid keys. */
void orc_iceberg_locate(const orc_cfg *c, const uint64_t *t0, const uint64_t *t1,
                        const uint64_t *keys, size_t n, uint64_t *slot_out);
/* Decode every stored entry back to its key (k = pi^-1(a . r)). Writes at
 * most cap keys, returns the number of stored entries. */
uint64_t orc_enumerate(const orc_cfg *c, const uint64_t *t0,
                       const uint64_t *t1, uint64_t *out, uint64_t cap);

/* --- invariant checkers; each returns the number of violations --- */
/* filled slots of every bucket form a prefix (Section 3, Limitations) */
uint64_t orc_check_prefix(const orc_cfg *c, int level, const uint64_t *table);
/* every entry decodes to a key of the right address and a valid tag */
uint64_t orc_check_entries(const orc_cfg *c, const uint64_t *t0,
                           const uint64_t *t1);
/* iceberg order property of the well-formedness definition (Appendix A) */
uint64_t orc_check_order_property(const orc_cfg *c, const uint64_t *t0,
                                  const uint64_t *t1);
/* cuckoo: an entry stored under hash index j has buckets a_0..a_{j-1} full */
uint64_t orc_check_cuckoo_chain(const orc_cfg *c, const uint64_t *table);
/* level-3 stash: every stash key has its three buckets full without it, and
 * every position from its home up to its own holds another key */
uint64_t orc_check_stash(const orc_cfg *c, const uint64_t *t0, const uint64_t *t1);
/* stored entries minus distinct stored keys (0 when no key is held twice) */
uint64_t orc_check_duplicates(const orc_cfg *c, const uint64_t *t0,
                              const uint64_t *t1);

/* --- host-threaded model of the lockless operations on packed slots ---
 * The table kind's write operation (iceberg: Algorithm 1 find-or-put; cuckoo:
 * Algorithm 4 put) run by nthreads POSIX threads at once, thread t taking
 * keys t, t + nthreads, ...; every claim is a compare-and-swap of one field
 * of a 64-bit word, retried while only neighbouring fields changed. status
 * as for the sequential operations, plus 5 when a bounded retry loop gave
 * up. Returns the number of threads that ran concurrently, -1 on bad
 * arguments; *fails_out (may be NULL) counts lost compare-and-swaps. */
int orc_concurrent_insert(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                          const uint64_t *keys, size_t n, uint8_t *status,
                          uint64_t *dropped, int nthreads, uint64_t *fails_out);

#ifdef __cplusplus
}
#endif
#endif
