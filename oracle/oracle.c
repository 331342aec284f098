/*
 * oracle.c - sequential CPU oracle for compact bucketed cuckoo hashing and
 * compact two-level iceberg hashing (Hegeman et al., "Compact Parallel Hash
 * Tables on the GPU").
 *
 * TEST INFRASTRUCTURE: called only by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark. Shares no code with the CUDA library.
 * Every function is a plain sequential restatement of the paper's definition
 * or algorithm, cited beside it.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - Permutation (Section 4.3 says only "one-round Feistel"): with R = w - N,
 *     split k into L = k >> R (N bits) and r = k mod 2^R. Then
 *     pi(k) = ((L xor f(r)) << R) | r, with f(r) = (A*r + B) mod 2^64 >> (64-N),
 *     A odd. A and B come from the splitmix64 sequence of the table seed.
 *   - Address and remainder (Section 2.4): a(k) = first N bits of pi(k),
 *     r(k) = the other R bits. For a bucket count nb that is not a power of
 *     two (whole-key tables only) a(k) = (pi(k) * nb) >> w with N = ceil(log2 nb).
 *   - Slot contents: cuckoo (r << 2) | (j + 1) (Section 2.2 stores (k, j));
 *     iceberg primary (r << 1) | 1 (one bit marks occupancy, Section 5.1);
 *     iceberg secondary (r << 2) | (i + 1), i the secondary choice
 *     (Algorithm 1 stores (r_i(k), i - 1)). Whole-key tables store k in place
 *     of r. The all-zero field is EMPTY.
 *   - Cuckoo eviction choice (Algorithm 4: "pseudorandomly, or based on c, k"):
 *     slot = (hi32(splitmix64(k, c)) * B) >> 32, k the key in hand at step c.
 *   - Key 0 and keys >= 2^w are rejected as INVALID.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

/* splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014) */
static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* output number idx (0-based) of the splitmix64 sequence whose state starts at s */
static uint64_t orc_splitmix(uint64_t s, uint64_t idx)
{
    return orc_mix64(s + (idx + 1) * ORC_GAMMA);
}

static int orc_ceil_log2(uint64_t x)
{
    int n = 0;
    while (n < 64 && (1ULL << n) < x)
        n++;
    return n;
}

static uint64_t orc_low_mask(int bits)
{
    return bits >= 64 ? ~0ULL : ((1ULL << bits) - 1);
}

static int orc_valid_key(const orc_cfg *c, uint64_t k)
{
    return k != 0 && (c->key_bits >= 64 || (k >> c->key_bits) == 0);
}

/* ------------------------------------------------------------------------ */
/* Permutation pi_j and quotienting, Section 2.4 and Section 4.3             */
/* ------------------------------------------------------------------------ */

static int orc_addr_bits(const orc_cfg *c, int level)
{
    return orc_ceil_log2(c->nb[level]);
}

int orc_cfg_check(const orc_cfg *c)
{
    int levels = c->kind == 1 ? 2 : 1;
    if (c->kind != 0 && c->kind != 1)
        return 1;
    if (c->key_bits < 2 || c->key_bits > 62)
        return 2;
    if (c->wpb < 1 || c->wpb > 16)
        return 3;
    if (c->kind == 0 && (c->num_hashes < 1 || c->num_hashes > 3 || c->max_chain < 1))
        return 4;
    if (c->stash && (c->kind != 1 || (c->stash & (c->stash - 1)) || c->stash > (1ULL << 40)))
        return 9;
    for (int level = 0; level < levels; level++) {
        int fpw = c->fpw[level];
        uint64_t nb = c->nb[level];
        int n = orc_addr_bits(c, level);
        /* tag bits: cuckoo (j + 1) in 2 bits, iceberg primary 1, secondary 2 */
        int tag = (c->kind == 1 && level == 0) ? 1 : 2;
        int body = c->compact ? c->key_bits - n : c->key_bits;
        if (fpw < 1 || fpw > 4)
            return 5;
        if (nb < 1 || n >= c->key_bits)
            return 6;
        if (c->compact && (nb & (nb - 1)) != 0)
            return 7;
        if (body + tag > 64 / fpw)
            return 8;
    }
    return 0;
}

/* Feistel round function of permutation j on the given level */
static uint64_t orc_round(const orc_cfg *c, int level, int j, uint64_t r)
{
    int n = orc_addr_bits(c, level);
    uint64_t idx = 2 * (uint64_t)(4 * level + j);
    uint64_t A = orc_splitmix(c->seed, idx) | 1ULL;
    uint64_t B = orc_splitmix(c->seed, idx + 1);
    if (n == 0)
        return 0;
    return (A * r + B) >> (64 - n);
}

uint64_t orc_perm(const orc_cfg *c, int level, int j, uint64_t k)
{
    int R = c->key_bits - orc_addr_bits(c, level);
    uint64_t r = k & orc_low_mask(R);
    uint64_t L = k >> R;
    return ((L ^ orc_round(c, level, j, r)) << R) | r;
}

uint64_t orc_perm_inv(const orc_cfg *c, int level, int j, uint64_t p)
{
    int R = c->key_bits - orc_addr_bits(c, level);
    uint64_t r = p & orc_low_mask(R);
    uint64_t L = (p >> R) ^ orc_round(c, level, j, r);
    return (L << R) | r;
}

/* a_j(k): the first N bits of pi_j(k); for a bucket count that is not a
 * power of two, pi_j(k) scaled onto [0, nb) */
uint64_t orc_address(const orc_cfg *c, int level, int j, uint64_t k)
{
    uint64_t p = orc_perm(c, level, j, k);
    unsigned __int128 prod = (unsigned __int128)p * c->nb[level];
    return (uint64_t)(prod >> c->key_bits);
}

/* r_j(k): the remaining w - N bits of pi_j(k) */
uint64_t orc_remainder(const orc_cfg *c, int level, int j, uint64_t k)
{
    int R = c->key_bits - orc_addr_bits(c, level);
    return orc_perm(c, level, j, k) & orc_low_mask(R);
}

/* k = pi_j^-1(a . r), Section 2.4 */
uint64_t orc_key_from(const orc_cfg *c, int level, int j, uint64_t a,
                      uint64_t r)
{
    int R = c->key_bits - orc_addr_bits(c, level);
    return orc_perm_inv(c, level, j, (a << R) | r);
}

void orc_perm_many(const orc_cfg *c, int level, int j, const uint64_t *keys,
                   size_t n, uint64_t *out_perm, uint64_t *out_addr,
                   uint64_t *out_rem, uint64_t *out_back)
{
    for (size_t i = 0; i < n; i++) {
        uint64_t p = orc_perm(c, level, j, keys[i]);
        if (out_perm)
            out_perm[i] = p;
        if (out_addr)
            out_addr[i] = orc_address(c, level, j, keys[i]);
        if (out_rem)
            out_rem[i] = orc_remainder(c, level, j, keys[i]);
        if (out_back)
            out_back[i] = orc_perm_inv(c, level, j, p);
    }
}

/* ------------------------------------------------------------------------ */
/* Slot order, Definition 1 (Appendix A)                                     */
/* ------------------------------------------------------------------------ */

/* (x1, y1) strictly precedes (x2, y2). x = 0 is the primary bucket, x = 1 and
 * x = 2 the first and second secondary buckets. The definition lists the cases
 * in which the order holds; since it is a total order, (2, y) precedes (1, x)
 * exactly when (1, x) does not precede (2, y), i.e. when y <= x. */
int orc_prec(int x1, int y1, int x2, int y2)
{
    if (x1 == x2)
        return y1 < y2;
    if (x1 == 0)
        return 1;
    if (x2 == 0)
        return 0;
    if (x1 == 1) /* x2 == 2 */
        return y1 < y2;
    return y1 <= y2; /* x1 == 2, x2 == 1 */
}

/* ------------------------------------------------------------------------ */
/* Table geometry and slot access                                            */
/* ------------------------------------------------------------------------ */

uint64_t orc_table_words(const orc_cfg *c, int level)
{
    uint64_t w = c->nb[level] * (uint64_t)c->wpb;
    return level == 1 ? w + c->stash : w;
}

/* the stash: whole keys after the secondary level's words */
static uint64_t *orc_stash_ptr(const orc_cfg *c, const uint64_t *t1)
{
    return (uint64_t *)t1 + c->nb[1] * (uint64_t)c->wpb;
}

/* home position of k in the stash: the splitmix64 finaliser of k xor a
 * constant of the third level (output 16 of the seed's sequence, after the
 * permutation constants of levels 0 and 1) */
uint64_t orc_stash_home(const orc_cfg *c, uint64_t k)
{
    return orc_mix64(k ^ orc_splitmix(c->seed, 16)) & (c->stash - 1);
}

int orc_slots_per_bucket(const orc_cfg *c, int level)
{
    return (uint64_t)c->wpb * c->fpw[level];
}

uint64_t orc_get_slot(const orc_cfg *c, int level, const uint64_t *table,
                      uint64_t bucket, int y)
{
    int fpw = c->fpw[level];
    int s = 64 / fpw;
    uint64_t word = table[bucket * (uint64_t)c->wpb + (uint64_t)(y / fpw)];
    return (word >> ((y % fpw) * s)) & orc_low_mask(s);
}

void orc_set_slot(const orc_cfg *c, int level, uint64_t *table,
                  uint64_t bucket, int y, uint64_t v)
{
    int fpw = c->fpw[level];
    int s = 64 / fpw;
    int sh = (y % fpw) * s;
    uint64_t m = orc_low_mask(s) << sh;
    uint64_t *w = &table[bucket * (uint64_t)c->wpb + (uint64_t)(y / fpw)];
    *w = (*w & ~m) | ((v << sh) & m);
}

/* ------------------------------------------------------------------------ */
/* Entry encodings                                                           */
/* ------------------------------------------------------------------------ */

/* cuckoo slot content for key k placed through hash j: the pair (r_j(k), j) */
static uint64_t orc_cuckoo_entry(const orc_cfg *c, int j, uint64_t k)
{
    uint64_t body = c->compact ? orc_remainder(c, 0, j, k) : k;
    return (body << 2) | (uint64_t)(j + 1);
}

/* iceberg slot content r'_x(k) for x in {0, 1, 2} (Appendix A notation):
 * r'_0 = r_0(k), r'_{1+i} = (r_{1+i}(k), i) */
static uint64_t orc_iceberg_entry(const orc_cfg *c, int x, uint64_t k)
{
    if (x == 0) {
        uint64_t body = c->compact ? orc_remainder(c, 0, 0, k) : k;
        return (body << 1) | 1ULL;
    } else {
        uint64_t body = c->compact ? orc_remainder(c, 1, x - 1, k) : k;
        return (body << 2) | (uint64_t)x;
    }
}

/* bucket index and level of the (x, .) bucket of key k in an iceberg table */
static uint64_t orc_iceberg_bucket(const orc_cfg *c, int x, uint64_t k)
{
    return x == 0 ? orc_address(c, 0, 0, k) : orc_address(c, 1, x - 1, k);
}

static const uint64_t *orc_level_table(int x, const uint64_t *t0,
                                       const uint64_t *t1)
{
    return x == 0 ? t0 : t1;
}

/* the entry key k has under choice x and the bucket it goes to: for cuckoo x
 * is the hash index j (level 0); for iceberg x = 0 is the primary bucket and
 * x = 1, 2 the secondary ones */
uint64_t orc_entry_of(const orc_cfg *c, int x, uint64_t k)
{
    return c->kind == 0 ? orc_cuckoo_entry(c, x, k) : orc_iceberg_entry(c, x, k);
}

uint64_t orc_bucket_of(const orc_cfg *c, int x, uint64_t k)
{
    return c->kind == 0 ? orc_address(c, 0, x, k) : orc_iceberg_bucket(c, x, k);
}

static int orc_bucket_contains(const orc_cfg *c, int level,
                               const uint64_t *table, uint64_t bucket,
                               uint64_t entry)
{
    int B = orc_slots_per_bucket(c, level);
    for (int y = 0; y < B; y++)
        if (orc_get_slot(c, level, table, bucket, y) == entry)
            return 1;
    return 0;
}

static int orc_bucket_has_empty(const orc_cfg *c, int level,
                                const uint64_t *table, uint64_t bucket)
{
    int B = orc_slots_per_bucket(c, level);
    for (int y = 0; y < B; y++)
        if (orc_get_slot(c, level, table, bucket, y) == 0)
            return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cuckoo put, Algorithm 4, run sequentially                                 */
/* ------------------------------------------------------------------------ */

static uint64_t orc_evict_slot(uint64_t k, int step, int B)
{
    uint64_t h = orc_splitmix(k, (uint64_t)step) >> 32;
    return (h * (uint64_t)B) >> 32;
}

/* decode a cuckoo entry found in bucket a into (key, hash index) */
static uint64_t orc_cuckoo_decode(const orc_cfg *c, uint64_t a, uint64_t e,
                                  int *j_out)
{
    int j = (int)(e & 3) - 1;
    *j_out = j;
    if (c->compact)
        return orc_key_from(c, 0, j, a, e >> 2);
    return e >> 2;
}

static int orc_cuckoo_put(const orc_cfg *c, uint64_t *table, uint64_t k,
                          uint64_t *dropped, uint64_t *probes,
                          uint64_t *writes)
{
    int B = orc_slots_per_bucket(c, 0);
    int j = 0;
    for (int step = 1; step <= c->max_chain; step++) {
        uint64_t a = orc_address(c, 0, j, k);
        uint64_t e = orc_cuckoo_entry(c, j, k);
        int y_empty = -1;
        (*probes)++;
        for (int y = 0; y < B; y++) {
            if (orc_get_slot(c, 0, table, a, y) == 0) {
                y_empty = y;
                break;
            }
        }
        (*writes)++;
        if (y_empty >= 0) {
            /* an empty slot: claim the first one */
            orc_set_slot(c, 0, table, a, y_empty, e);
            return ORC_PUT;
        }
        /* bucket full: swap (r, j) with the chosen slot, continue with the
         * evicted key under its next hash function */
        int y = (int)orc_evict_slot(k, step, B);
        uint64_t old = orc_get_slot(c, 0, table, a, y);
        orc_set_slot(c, 0, table, a, y, e);
        int jo;
        k = orc_cuckoo_decode(c, a, old, &jo);
        j = (jo + 1) % c->num_hashes;
    }
    *dropped = k;
    return ORC_FULL;
}

void orc_cuckoo_insert(const orc_cfg *c, uint64_t *table, const uint64_t *keys,
                       size_t n, uint8_t *status, uint64_t *dropped,
                       uint64_t *probes, uint64_t *writes)
{
    uint64_t p = 0, w = 0;
    for (size_t i = 0; i < n; i++) {
        uint64_t d = 0;
        if (!orc_valid_key(c, keys[i])) {
            status[i] = ORC_INVALID;
        } else {
            status[i] = (uint8_t)orc_cuckoo_put(c, table, keys[i], &d, &p, &w);
        }
        if (dropped)
            dropped[i] = d;
    }
    if (probes)
        *probes = p;
    if (writes)
        *writes = w;
}

/* ------------------------------------------------------------------------ */
/* Cuckoo lookup, Section 4.4                                                */
/* ------------------------------------------------------------------------ */

void orc_cuckoo_find(const orc_cfg *c, const uint64_t *table,
                     const uint64_t *keys, size_t n, uint8_t *status,
                     uint64_t *probes)
{
    uint64_t p = 0;
    for (size_t i = 0; i < n; i++) {
        uint64_t k = keys[i];
        if (!orc_valid_key(c, k)) {
            status[i] = ORC_INVALID;
            continue;
        }
        status[i] = ORC_NOT_FOUND;
        for (int j = 0; j < c->num_hashes; j++) {
            uint64_t a = orc_address(c, 0, j, k);
            p++;
            if (orc_bucket_contains(c, 0, table, a, orc_cuckoo_entry(c, j, k))) {
                status[i] = ORC_FOUND;
                break;
            }
            /* a bucket with a free slot ends the search: k would have been
             * placed here before moving on to a_{j+1} */
            if (orc_bucket_has_empty(c, 0, table, a))
                break;
        }
    }
    if (probes)
        *probes = p;
}

void orc_cuckoo_find_exhaustive(const orc_cfg *c, const uint64_t *table,
                                const uint64_t *keys, size_t n,
                                uint8_t *status)
{
    for (size_t i = 0; i < n; i++) {
        uint64_t k = keys[i];
        if (!orc_valid_key(c, k)) {
            status[i] = ORC_INVALID;
            continue;
        }
        status[i] = ORC_NOT_FOUND;
        for (int j = 0; j < c->num_hashes; j++)
            if (orc_bucket_contains(c, 0, table, orc_address(c, 0, j, k),
                                    orc_cuckoo_entry(c, j, k)))
                status[i] = ORC_FOUND;
    }
}

/* ------------------------------------------------------------------------ */
/* Iceberg find-or-put, Algorithm 5 (Appendix A), run sequentially           */
/* ------------------------------------------------------------------------ */

/* Level 3, reached only when the primary and both secondary buckets are
 * full (Section 2.3): linear probing in the stash from k's home position;
 * k found -> FOUND, the first empty position takes k -> PUT, all positions
 * taken -> FULL. */
static int orc_stash_fop(const orc_cfg *c, uint64_t *t1, uint64_t k, uint64_t *writes)
{
    uint64_t *st = orc_stash_ptr(c, t1);
    uint64_t h = orc_stash_home(c, k);
    for (uint64_t i = 0; i < c->stash; i++) {
        uint64_t p = (h + i) & (c->stash - 1);
        if (st[p] == k)
            return ORC_FOUND;
        if (st[p] == 0) {
            st[p] = k;
            (*writes)++;
            return ORC_PUT;
        }
    }
    return ORC_FULL;
}

/* lookup in the stash: stops at k or at the first empty position */
static int orc_stash_find(const orc_cfg *c, const uint64_t *t1, uint64_t k, uint64_t *pos)
{
    const uint64_t *st = orc_stash_ptr(c, t1);
    uint64_t h = orc_stash_home(c, k);
    for (uint64_t i = 0; i < c->stash; i++) {
        uint64_t p = (h + i) & (c->stash - 1);
        if (st[p] == k) {
            if (pos)
                *pos = p;
            return 1;
        }
        if (st[p] == 0)
            return 0;
    }
    return 0;
}

static int orc_iceberg_fop1(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                            uint64_t k, uint64_t *probes, uint64_t *writes)
{
    int Bx[3] = {orc_slots_per_bucket(c, 0), orc_slots_per_bucket(c, 1),
                 orc_slots_per_bucket(c, 1)};
    uint64_t a[3], e[3];
    for (int x = 0; x < 3; x++) {
        a[x] = orc_iceberg_bucket(c, x, k);
        e[x] = orc_iceberg_entry(c, x, k);
    }
    /* bucket probes the method needs: the primary alone decides when it
     * holds k or has room (Algorithm 1, level 1); otherwise both secondaries */
    if (orc_bucket_contains(c, 0, t0, a[0], e[0]) ||
        orc_bucket_has_empty(c, 0, t0, a[0]))
        *probes += 1;
    else
        *probes += 3;

    /* found: some slot (x, y) of S holds r'_x(k) */
    for (int x = 0; x < 3; x++)
        for (int y = 0; y < Bx[x]; y++)
            if (orc_get_slot(c, x ? 1 : 0, orc_level_table(x, t0, t1), a[x],
                             y) == e[x])
                return ORC_FOUND;
    /* otherwise the prec-least empty slot of S, if any */
    int bx = -1, by = -1;
    for (int x = 0; x < 3; x++)
        for (int y = 0; y < Bx[x]; y++) {
            if (orc_get_slot(c, x ? 1 : 0, orc_level_table(x, t0, t1), a[x],
                             y) != 0)
                continue;
            if (bx < 0 || orc_prec(x, y, bx, by)) {
                bx = x;
                by = y;
            }
        }
    if (bx < 0)
        return c->stash ? orc_stash_fop(c, t1, k, writes) : ORC_FULL;
    orc_set_slot(c, bx ? 1 : 0, bx ? t1 : t0, a[bx], by, e[bx]);
    (*writes)++;
    return ORC_PUT;
}

void orc_iceberg_fop(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                     const uint64_t *keys, size_t n, uint8_t *status,
                     uint64_t *probes, uint64_t *writes)
{
    uint64_t p = 0, w = 0;
    for (size_t i = 0; i < n; i++) {
        if (!orc_valid_key(c, keys[i]))
            status[i] = ORC_INVALID;
        else
            status[i] = (uint8_t)orc_iceberg_fop1(c, t0, t1, keys[i], &p, &w);
    }
    if (probes)
        *probes = p;
    if (writes)
        *writes = w;
}

/* ------------------------------------------------------------------------ */
/* Iceberg lookup, Section 2.3 (levels 1 and 2)                              */
/* ------------------------------------------------------------------------ */

void orc_iceberg_find(const orc_cfg *c, const uint64_t *t0, const uint64_t *t1,
                      const uint64_t *keys, size_t n, uint8_t *status,
                      uint64_t *probes)
{
    uint64_t p = 0;
    for (size_t i = 0; i < n; i++) {
        uint64_t k = keys[i];
        if (!orc_valid_key(c, k)) {
            status[i] = ORC_INVALID;
            continue;
        }
        uint64_t a0 = orc_iceberg_bucket(c, 0, k);
        p++;
        if (orc_bucket_contains(c, 0, t0, a0, orc_iceberg_entry(c, 0, k))) {
            status[i] = ORC_FOUND;
            continue;
        }
        if (orc_bucket_has_empty(c, 0, t0, a0)) {
            status[i] = ORC_NOT_FOUND;
            continue;
        }
        p += 2;
        int hit = 0, room = 0;
        for (int x = 1; x <= 2; x++) {
            uint64_t a = orc_iceberg_bucket(c, x, k);
            if (orc_bucket_contains(c, 1, t1, a, orc_iceberg_entry(c, x, k)))
                hit = 1;
            room |= orc_bucket_has_empty(c, 1, t1, a);
        }
        /* level 3: k can be in the stash only if all three buckets were full
         * when it was put, and full buckets stay full */
        if (!hit && !room && c->stash)
            hit = orc_stash_find(c, t1, k, NULL);
        status[i] = hit ? ORC_FOUND : ORC_NOT_FOUND;
    }
    if (probes)
        *probes = p;
}

/* ------------------------------------------------------------------------ */
/* Slot index of a stored key (iceberg entries never move, Section 5.1, so   */
/* the index can address a value array: the key-value extension)            */
/* ------------------------------------------------------------------------ */

/* Level-0 slots are numbered a * B0 + y, level-1 slots nb0 * B0 + a * B1 + y,
 * with y the slot's position in bucket a, and stash position p is
 * nb0 * B0 + nb1 * B1 + p. Absent or invalid keys get UINT64_MAX. */
void orc_iceberg_locate(const orc_cfg *c, const uint64_t *t0, const uint64_t *t1,
                        const uint64_t *keys, size_t n, uint64_t *slot_out)
{
    int B0 = orc_slots_per_bucket(c, 0);
    int B1 = c->kind == 1 ? orc_slots_per_bucket(c, 1) : 0;
    for (size_t i = 0; i < n; i++) {
        uint64_t k = keys[i];
        slot_out[i] = UINT64_MAX;
        if (!orc_valid_key(c, k))
            continue;
        for (int x = 0; x <= 2 && slot_out[i] == UINT64_MAX; x++) {
            int level = x == 0 ? 0 : 1;
            uint64_t a = orc_iceberg_bucket(c, x, k);
            uint64_t e = orc_iceberg_entry(c, x, k);
            const uint64_t *t = orc_level_table(x, t0, t1);
            int B = level == 0 ? B0 : B1;
            for (int y = 0; y < B; y++) {
                if (orc_get_slot(c, level, t, a, y) == e) {
                    slot_out[i] = level == 0
                                      ? a * (uint64_t)B0 + (uint64_t)y
                                      : c->nb[0] * (uint64_t)B0 + a * (uint64_t)B1 + (uint64_t)y;
                    break;
                }
            }
        }
        uint64_t p;
        if (slot_out[i] == UINT64_MAX && c->stash && orc_stash_find(c, t1, k, &p))
            slot_out[i] = c->nb[0] * (uint64_t)B0 + c->nb[1] * (uint64_t)B1 + p;
    }
}

/* ------------------------------------------------------------------------ */
/* Enumerate: k = pi^-1(a . r) for every stored entry (Section 2.4)          */
/* ------------------------------------------------------------------------ */

/* key held by entry e found in bucket a of the given level; -1 tag on error */
static uint64_t orc_decode(const orc_cfg *c, int level, uint64_t a, uint64_t e,
                           int *x_out)
{
    if (c->kind == 0) {
        int j;
        uint64_t k = orc_cuckoo_decode(c, a, e, &j);
        *x_out = j;
        return k;
    }
    if (level == 0) {
        *x_out = 0;
        return c->compact ? orc_key_from(c, 0, 0, a, e >> 1) : e >> 1;
    }
    int x = (int)(e & 3);
    *x_out = x;
    if (x < 1 || x > 2)
        return 0;
    return c->compact ? orc_key_from(c, 1, x - 1, a, e >> 2) : e >> 2;
}

static int orc_levels(const orc_cfg *c)
{
    return c->kind == 1 ? 2 : 1;
}

uint64_t orc_enumerate(const orc_cfg *c, const uint64_t *t0,
                       const uint64_t *t1, uint64_t *out, uint64_t cap)
{
    uint64_t cnt = 0;
    for (int level = 0; level < orc_levels(c); level++) {
        const uint64_t *t = level ? t1 : t0;
        int B = orc_slots_per_bucket(c, level);
        for (uint64_t a = 0; a < c->nb[level]; a++)
            for (int y = 0; y < B; y++) {
                uint64_t e = orc_get_slot(c, level, t, a, y);
                if (e == 0)
                    continue;
                int x;
                uint64_t k = orc_decode(c, level, a, e, &x);
                if (cnt < cap)
                    out[cnt] = k;
                cnt++;
            }
    }
    if (c->kind == 1 && c->stash) {
        const uint64_t *st = orc_stash_ptr(c, t1);
        for (uint64_t p = 0; p < c->stash; p++) {
            if (st[p] == 0)
                continue;
            if (cnt < cap)
                out[cnt] = st[p];
            cnt++;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Invariant checkers                                                        */
/* ------------------------------------------------------------------------ */

uint64_t orc_check_prefix(const orc_cfg *c, int level, const uint64_t *table)
{
    uint64_t bad = 0;
    int B = orc_slots_per_bucket(c, level);
    for (uint64_t a = 0; a < c->nb[level]; a++) {
        int seen_empty = 0;
        for (int y = 0; y < B; y++) {
            uint64_t e = orc_get_slot(c, level, table, a, y);
            if (e == 0)
                seen_empty = 1;
            else if (seen_empty) {
                bad++;
                break;
            }
        }
    }
    return bad;
}

uint64_t orc_check_entries(const orc_cfg *c, const uint64_t *t0,
                           const uint64_t *t1)
{
    uint64_t bad = 0;
    for (int level = 0; level < orc_levels(c); level++) {
        const uint64_t *t = level ? t1 : t0;
        int B = orc_slots_per_bucket(c, level);
        for (uint64_t a = 0; a < c->nb[level]; a++)
            for (int y = 0; y < B; y++) {
                uint64_t e = orc_get_slot(c, level, t, a, y);
                if (e == 0)
                    continue;
                int x;
                uint64_t k = orc_decode(c, level, a, e, &x);
                int ok;
                if (c->kind == 0)
                    ok = x >= 0 && x < c->num_hashes && orc_valid_key(c, k) &&
                         orc_address(c, 0, x, k) == a &&
                         orc_cuckoo_entry(c, x, k) == e;
                else if (level == 0)
                    ok = (e & 1) && orc_valid_key(c, k) &&
                         orc_address(c, 0, 0, k) == a &&
                         orc_iceberg_entry(c, 0, k) == e;
                else
                    ok = x >= 1 && x <= 2 && orc_valid_key(c, k) &&
                         orc_iceberg_bucket(c, x, k) == a &&
                         orc_iceberg_entry(c, x, k) == e;
                if (!ok)
                    bad++;
            }
    }
    return bad;
}

/* order property: if slot (x, y) for k holds r'_x(k), every slot (x', y')
 * preceding it holds some other key's entry (neither EMPTY nor r'_{x'}(k)) */
uint64_t orc_check_order_property(const orc_cfg *c, const uint64_t *t0,
                                  const uint64_t *t1)
{
    uint64_t bad = 0;
    int Bx[3] = {orc_slots_per_bucket(c, 0), orc_slots_per_bucket(c, 1),
                 orc_slots_per_bucket(c, 1)};
    for (int level = 0; level < 2; level++) {
        const uint64_t *t = level ? t1 : t0;
        for (uint64_t a = 0; a < c->nb[level]; a++)
            for (int y = 0; y < Bx[level]; y++) {
                uint64_t e = orc_get_slot(c, level, t, a, y);
                if (e == 0)
                    continue;
                int x;
                uint64_t k = orc_decode(c, level, a, e, &x);
                /* k's three buckets and its entry for each */
                uint64_t kb[3], ke[3];
                for (int x2 = 0; x2 < 3; x2++) {
                    kb[x2] = orc_iceberg_bucket(c, x2, k);
                    ke[x2] = orc_iceberg_entry(c, x2, k);
                }
                int violated = 0;
                for (int x2 = 0; x2 < 3 && !violated; x2++)
                    for (int y2 = 0; y2 < Bx[x2]; y2++) {
                        if (!orc_prec(x2, y2, x, y))
                            continue;
                        uint64_t e2 = orc_get_slot(
                            c, x2 ? 1 : 0, orc_level_table(x2, t0, t1), kb[x2], y2);
                        if (e2 == 0 || e2 == ke[x2]) {
                            violated = 1;
                            break;
                        }
                    }
                bad += (uint64_t)violated;
            }
    }
    return bad;
}

uint64_t orc_check_cuckoo_chain(const orc_cfg *c, const uint64_t *table)
{
    uint64_t bad = 0;
    int B = orc_slots_per_bucket(c, 0);
    for (uint64_t a = 0; a < c->nb[0]; a++)
        for (int y = 0; y < B; y++) {
            uint64_t e = orc_get_slot(c, 0, table, a, y);
            if (e == 0)
                continue;
            int j;
            uint64_t k = orc_cuckoo_decode(c, a, e, &j);
            for (int jj = 0; jj < j; jj++)
                if (orc_bucket_has_empty(c, 0, table, orc_address(c, 0, jj, k))) {
                    bad++;
                    break;
                }
        }
    return bad;
}

uint64_t orc_check_stash(const orc_cfg *c, const uint64_t *t0,
                         const uint64_t *t1)
{
    uint64_t bad = 0;
    if (c->kind != 1 || !c->stash)
        return 0;
    const uint64_t *st = orc_stash_ptr(c, t1);
    for (uint64_t p = 0; p < c->stash; p++) {
        uint64_t k = st[p];
        if (k == 0)
            continue;
        int violated = !orc_valid_key(c, k);
        /* stash slots come after every bucket slot: all three buckets full,
         * none holding k */
        for (int x = 0; x < 3 && !violated; x++) {
            int level = x ? 1 : 0;
            const uint64_t *t = orc_level_table(x, t0, t1);
            uint64_t a = orc_iceberg_bucket(c, x, k);
            if (orc_bucket_has_empty(c, level, t, a) ||
                orc_bucket_contains(c, level, t, a, orc_iceberg_entry(c, x, k)))
                violated = 1;
        }
        /* linear probing: every position from home up to p holds another key */
        for (uint64_t q = orc_stash_home(c, k); q != p && !violated;
             q = (q + 1) & (c->stash - 1))
            if (st[q] == 0 || st[q] == k)
                violated = 1;
        bad += (uint64_t)violated;
    }
    return bad;
}

static int orc_cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* no key is stored twice (Appendix A, the no-duplicates lemma; for cuckoo the
 * set semantics of Section 3): the number of stored entries minus the number
 * of distinct keys they decode to */
uint64_t orc_check_duplicates(const orc_cfg *c, const uint64_t *t0,
                              const uint64_t *t1)
{
    uint64_t n = orc_enumerate(c, t0, t1, NULL, 0);
    if (n < 2)
        return 0;
    uint64_t *keys = malloc(n * sizeof *keys);
    if (!keys)
        return UINT64_MAX;
    orc_enumerate(c, t0, t1, keys, n);
    qsort(keys, n, sizeof *keys, orc_cmp_u64);
    uint64_t dup = 0;
    for (uint64_t i = 1; i < n; i++)
        if (keys[i] == keys[i - 1])
            dup++;
    free(keys);
    return dup;
}

/* ------------------------------------------------------------------------ */
/* Host-threaded model of the lockless operations on packed slots           */
/* ------------------------------------------------------------------------ */
/*
 * Algorithm 1 (iceberg find-or-put) and Algorithm 4 (cuckoo put) run by many
 * POSIX threads at once on one table. Section 4.5 observes that atomic
 * instructions are too coarse for small slots; here, as in the GPU kernels,
 * a slot is one field of a 64-bit word and a claim is a compare-and-swap of
 * the whole word that succeeds only if the target field is still EMPTY:
 *   - a snapshot reads a bucket word by word (each word atomically, the
 *     bucket as a whole possibly torn);
 *   - the claim index is the number of filled fields in the snapshot, which
 *     is never past the true first empty slot because fields only ever go
 *     from EMPTY to filled (Section 3, Limitations: filled slots form a
 *     prefix);
 *   - a failed compare-and-swap whose target field is still EMPTY (only a
 *     neighbouring field changed) is retried with the word it returned, at
 *     most 64 times; otherwise the field's new value decides: the key's own
 *     entry means another thread put it (FOUND), anything else means the
 *     bucket is read again;
 *   - a cuckoo swap is a compare-and-swap loop that exchanges one field.
 * Each retry loop has a bound; a key that exhausts it gets status 5 (error).
 * This is test infrastructure: it pins the packed-word claim protocol on the
 * CPU (no duplicate keys, one PUT per distinct key, conservation of keys),
 * and it shares no code with the CUDA library.
 */
#include <pthread.h>
#include <sched.h>

#define ORC_ERROR 5

static uint64_t mt_load(const uint64_t *p)
{
    return __atomic_load_n(p, __ATOMIC_RELAXED);
}

/* the fields of bucket a, read word by word; returns the number of filled
 * fields and sets *hit if one equals e */
static int mt_snapshot(const orc_cfg *c, int level, const uint64_t *table,
                       uint64_t a, uint64_t e, uint64_t *words, int *hit)
{
    int fpw = c->fpw[level], s = 64 / fpw, filled = 0;
    *hit = 0;
    for (int w = 0; w < c->wpb; w++) {
        words[w] = mt_load(&table[a * (uint64_t)c->wpb + (uint64_t)w]);
        for (int f = 0; f < fpw; f++) {
            uint64_t v = (words[w] >> (f * s)) & orc_low_mask(s);
            filled += v != 0;
            *hit |= v == e;
        }
    }
    return filled;
}

/* EMPTY -> e on field f of *wp; snap is the word as the snapshot saw it.
 * 1 if written; otherwise *seen is the value that won the field (0 if the
 * bounded retry gave up and the bucket has to be read again). */
static int mt_claim(uint64_t *wp, int f, int fpw, uint64_t snap, uint64_t e,
                    uint64_t *seen, uint64_t *fails)
{
    int s = 64 / fpw;
    uint64_t m = orc_low_mask(s) << (f * s);
    uint64_t expected = snap & ~m;
    for (int it = 0; it < 64; it++) {
        uint64_t old = expected;
        uint64_t desired = expected | (e << (f * s));
        if (__atomic_compare_exchange_n(wp, &old, desired, 0, __ATOMIC_RELAXED,
                                        __ATOMIC_RELAXED))
            return 1;
        (*fails)++;
        uint64_t fld = (old & m) >> (f * s);
        if (fld != 0) {
            *seen = fld;
            return 0;
        }
        expected = old; /* only a neighbouring field changed */
    }
    *seen = 0;
    return 0;
}

/* exchange field f of *wp with e; 1 and *prev = the old field on success,
 * 0 if the bounded retry gave up */
static int mt_swap(uint64_t *wp, int f, int fpw, uint64_t snap, uint64_t e,
                   uint64_t *prev)
{
    int s = 64 / fpw;
    uint64_t m = orc_low_mask(s) << (f * s);
    uint64_t expected = snap;
    for (int it = 0; it < 4096; it++) {
        uint64_t old = expected;
        uint64_t desired = (expected & ~m) | (e << (f * s));
        if (__atomic_compare_exchange_n(wp, &old, desired, 0, __ATOMIC_RELAXED,
                                        __ATOMIC_RELAXED)) {
            *prev = (expected & m) >> (f * s);
            return 1;
        }
        expected = old;
    }
    return 0;
}

static uint64_t *mt_word(const orc_cfg *c, int level, uint64_t *table,
                         uint64_t a, int y)
{
    return &table[a * (uint64_t)c->wpb + (uint64_t)(y / c->fpw[level])];
}

/* level 3 with compare-and-swap claims: linear probing from k's home; a
 * position that another thread filled first is read again (k itself means
 * FOUND) and otherwise passed */
static int mt_stash_fop(const orc_cfg *c, uint64_t *t1, uint64_t k, uint64_t *fails)
{
    uint64_t *st = orc_stash_ptr(c, t1);
    uint64_t h = orc_stash_home(c, k);
    for (uint64_t i = 0; i < c->stash; i++) {
        uint64_t *sp = &st[(h + i) & (c->stash - 1)];
        uint64_t v = mt_load(sp);
        if (v == 0) {
            uint64_t expected = 0;
            if (__atomic_compare_exchange_n(sp, &expected, k, 0, __ATOMIC_RELAXED,
                                            __ATOMIC_RELAXED))
                return ORC_PUT;
            (*fails)++;
            v = expected;
        }
        if (v == k)
            return ORC_FOUND;
    }
    return ORC_FULL;
}

/* Algorithm 1 for one key, with the claims above */
static int mt_iceberg_fop1(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                           uint64_t k, uint64_t *fails)
{
    int B0 = orc_slots_per_bucket(c, 0), B1 = orc_slots_per_bucket(c, 1);
    int max_iter = 4 * (B0 + 2 * B1) + 16;
    uint64_t w0[16], w1[16], w2[16];
    uint64_t a0 = orc_iceberg_bucket(c, 0, k), e0 = orc_iceberg_entry(c, 0, k);
    int it = 0, hit;
    /* level 1: the primary bucket */
    for (;;) {
        if (++it > max_iter)
            return ORC_ERROR;
        int y = mt_snapshot(c, 0, t0, a0, e0, w0, &hit);
        if (hit)
            return ORC_FOUND;
        if (y == B0)
            break;
        uint64_t seen = 0;
        int fpw = c->fpw[0];
        if (mt_claim(mt_word(c, 0, t0, a0, y), y % fpw, fpw, w0[y / fpw], e0,
                     &seen, fails))
            return ORC_PUT;
        if (seen == e0)
            return ORC_FOUND;
    }
    /* level 2: both secondary buckets, the less full one (ties to the
     * second: Definition 1) */
    uint64_t a1 = orc_iceberg_bucket(c, 1, k), e1 = orc_iceberg_entry(c, 1, k);
    uint64_t a2 = orc_iceberg_bucket(c, 2, k), e2 = orc_iceberg_entry(c, 2, k);
    for (;;) {
        if (++it > max_iter)
            return ORC_ERROR;
        int h1, h2;
        int y1 = mt_snapshot(c, 1, t1, a1, e1, w1, &h1);
        int y2 = mt_snapshot(c, 1, t1, a2, e2, w2, &h2);
        if (h1 || h2)
            return ORC_FOUND;
        int pick1 = y1 < y2;
        int y = pick1 ? y1 : y2;
        if (y == B1)
            return c->stash ? mt_stash_fop(c, t1, k, fails) : ORC_FULL;
        uint64_t a = pick1 ? a1 : a2, e = pick1 ? e1 : e2;
        uint64_t *snap = pick1 ? w1 : w2;
        uint64_t seen = 0;
        int fpw = c->fpw[1];
        if (mt_claim(mt_word(c, 1, t1, a, y), y % fpw, fpw, snap[y / fpw], e,
                     &seen, fails))
            return ORC_PUT;
        if (seen == e)
            return ORC_FOUND;
    }
}

/* Algorithm 4 for one key: a lost claim, like a swap, uses up a step */
static int mt_cuckoo_put(const orc_cfg *c, uint64_t *table, uint64_t k,
                         uint64_t *dropped, uint64_t *fails)
{
    int B = orc_slots_per_bucket(c, 0), fpw = c->fpw[0];
    uint64_t w[16];
    int j = 0, hit;
    for (int step = 1; step <= c->max_chain; step++) {
        uint64_t a = orc_address(c, 0, j, k);
        uint64_t e = orc_cuckoo_entry(c, j, k);
        int y = mt_snapshot(c, 0, table, a, e, w, &hit);
        if (y < B) {
            uint64_t seen = 0;
            if (mt_claim(mt_word(c, 0, table, a, y), y % fpw, fpw, w[y / fpw],
                         e, &seen, fails))
                return ORC_PUT;
            continue;
        }
        int ys = (int)orc_evict_slot(k, step, B);
        uint64_t prev = 0;
        if (!mt_swap(mt_word(c, 0, table, a, ys), ys % fpw, fpw, w[ys / fpw], e,
                     &prev))
            return ORC_ERROR;
        if (prev == 0)
            return ORC_PUT; /* the chosen slot held nothing */
        int jo;
        k = orc_cuckoo_decode(c, a, prev, &jo);
        j = (jo + 1) % c->num_hashes;
    }
    *dropped = k;
    return ORC_FULL;
}

typedef struct {
    const orc_cfg *c;
    uint64_t *t0, *t1;
    const uint64_t *keys;
    size_t n;
    uint8_t *status;
    uint64_t *dropped;
    int tid, nthreads;
    const int *go;
    uint64_t fails;
} mt_job;

static void *mt_worker(void *arg)
{
    mt_job *j = arg;
    while (!__atomic_load_n(j->go, __ATOMIC_ACQUIRE))
        sched_yield(); /* start together */
    /* thread t takes keys t, t + T, t + 2T, ...: copies of one key, and keys
     * of one bucket, land on different threads */
    for (size_t i = (size_t)j->tid; i < j->n; i += (size_t)j->nthreads) {
        uint64_t k = j->keys[i], d = 0;
        if (!orc_valid_key(j->c, k)) {
            j->status[i] = ORC_INVALID;
            continue;
        }
        if (j->c->kind == 1) {
            j->status[i] = (uint8_t)mt_iceberg_fop1(j->c, j->t0, j->t1, k, &j->fails);
        } else {
            j->status[i] = (uint8_t)mt_cuckoo_put(j->c, j->t0, k, &d, &j->fails);
            if (j->dropped)
                j->dropped[i] = d;
        }
    }
    return NULL;
}

/* Run the operation of the table's kind (iceberg find-or-put, cuckoo put)
 * on nthreads threads at once. Returns the number of threads that ran
 * concurrently (if some could not be started, their shares of the keys run
 * afterwards on the calling thread), or -1 on bad arguments. *fails_out (may
 * be NULL) counts compare-and-swaps that lost. */
int orc_concurrent_insert(const orc_cfg *c, uint64_t *t0, uint64_t *t1,
                          const uint64_t *keys, size_t n, uint8_t *status,
                          uint64_t *dropped, int nthreads, uint64_t *fails_out)
{
    if (nthreads < 1 || nthreads > 256 || c->wpb > 16)
        return -1;
    pthread_t th[256];
    int ok[256] = {0};
    mt_job jobs[256];
    int go = 0;
    for (int t = 0; t < nthreads; t++) {
        mt_job jb = {c, t0, t1, keys, n, status, dropped, t, nthreads, &go, 0};
        jobs[t] = jb;
    }
    int running = 1;
    for (int t = 1; t < nthreads; t++) {
        ok[t] = pthread_create(&th[t], NULL, mt_worker, &jobs[t]) == 0;
        running += ok[t];
    }
    __atomic_store_n(&go, 1, __ATOMIC_RELEASE);
    mt_worker(&jobs[0]);
    uint64_t fails = jobs[0].fails;
    for (int t = 1; t < nthreads; t++) {
        if (ok[t])
            pthread_join(th[t], NULL);
        else
            mt_worker(&jobs[t]);
        fails += jobs[t].fails;
    }
    if (fails_out)
        *fails_out = fails;
    return running;
}
