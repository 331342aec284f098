/*
 * cht.h - C ABI of the compact parallel hash table library (GB300, sm_103a).
 *
 * Batched, lockless insert, find and find-or-put on compact (quotiented)
 * bucketed hash tables, after Hegeman, Woeltgens, Wijs and Laarman, "Compact
 * Parallel Hash Tables on the GPU". Two table kinds:
 *
 *   CHT_CUCKOO   bucketed cuckoo hashing with H permutations (Section 2.2,
 *                Section 4.4, Algorithm 4): a static table, built from unique
 *                keys and then queried.
 *   CHT_ICEBERG  two-level iceberg hashing (Section 2.3, Section 3,
 *                Algorithm 1): a dynamic table whose find-or-put may run
 *                concurrently with other find-or-puts and lookups.
 *
 * Quotienting (Section 2.4): a permutation pi_j of the w-bit keys maps k to
 * pi_j(k) = a . r; the first N bits a address one of 2^N buckets and only the
 * remaining w - N bits r (plus a few tag bits) are stored, so more slots fit
 * in one 128-byte bucket. A "whole-key" table (compact = 0) stores k itself in
 * 64-bit slots and is the paper's non-compact baseline (Section 5.1).
 *
 * Conventions for every call below:
 *  - Pointers named d_* are addresses the current CUDA device can access:
 *    device memory, or page-locked host memory, which the kernels then read
 *    and write directly over the CPU-GPU link (for key, status, slot and
 *    value arrays; table storage must be device memory). The caller owns all
 *    memory: the table storage, key arrays and outputs. The library
 *    allocates no device memory.
 *  - stream is a cudaStream_t passed as an opaque pointer (NULL = the legacy
 *    default stream). Calls only enqueue work and return; results are valid
 *    once the stream has been synchronised.
 *  - Each call returns CHT_OK or one of the CHT_ERR_* codes; cht_last_error()
 *    then gives a message (thread-local). Argument errors are detected on the
 *    host before anything is enqueued. Per-key outcomes are status bytes.
 *  - Keys are unsigned integers of key_bytes (4 or 8) bytes, little-endian,
 *    in [1, 2^key_bits). Key 0 and keys >= 2^key_bits get status CHT_INVALID.
 */
#ifndef CHT_H
#define CHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- call return codes ---- */
#define CHT_OK 0
#define CHT_ERR_INVALID 1     /* bad argument or configuration                */
#define CHT_ERR_UNSUPPORTED 2 /* valid request this table kind does not offer */
#define CHT_ERR_CUDA 3        /* a CUDA runtime call failed                   */
#define CHT_ERR_CAPACITY 4    /* an output buffer is too small                */
#define CHT_ERR_TIMEOUT 5     /* a bounded device wait ran out                */

/* ---- per-key status bytes (Section 3: found / put / full) ---- */
#define CHT_NOT_FOUND 0 /* lookup: key absent                                */
#define CHT_FOUND 1     /* key present (find-or-put: it was already there)   */
#define CHT_PUT 2       /* this call inserted the key                        */
#define CHT_FULL 3      /* no slot available for the key                     */
#define CHT_INVALID 4   /* key 0 or key >= 2^key_bits                        */
#define CHT_ERROR 5     /* a bounded retry loop gave up (should not happen)  */

#define CHT_CUCKOO 0
#define CHT_ICEBERG 1

/* bytes of the table header at the start of the table storage */
#define CHT_HEADER_BYTES 256
/* bytes per bucket by default: 16 words of 64 bits, one cache line
 * (Section 4.5); see bucket_words for 32- and 64-byte buckets */
#define CHT_BUCKET_BYTES 128

typedef struct cht_table cht_table; /* opaque host handle */

/*
 * Table configuration. Zero-valued tuning fields select defaults.
 *
 * kind                  CHT_CUCKOO or CHT_ICEBERG.
 * compact               1: store remainders (quotienting, Section 2.4);
 *                       0: store whole keys, one 64-bit slot each.
 * key_bits              w, 2..62 (at most 32 when key_bytes = 4).
 * key_bytes             width of the caller's key arrays: 4 or 8.
 * num_buckets           buckets of the cuckoo table / iceberg primary level,
 *                       1..2^32. A power of two when compact = 1 (Section 4.5).
 * num_buckets_backyard  iceberg secondary-level buckets (ignored for cuckoo),
 *                       1..2^32.
 * fields_per_word       slots per 64-bit word of level 0, 1..4 (slot width
 *                       64/fields_per_word bits); 0 = the densest packing in
 *                       which every entry fits. Whole-key tables use 1.
 * fields_per_word_backyard  the same for the iceberg secondary level.
 * num_hashes            cuckoo H, 1..3 (0 = 3).
 * max_chain             cuckoo C, eviction steps before a put gives up
 *                       (Algorithm 4); 0 = 128.
 * seed                  all permutation constants derive from it.
 * tile                  threads cooperating on one bucket: 4, 8 or 16; 0 lets
 *                       each operation use its fastest width (cuckoo lookups
 *                       8, everything else 4).
 * items_per_thread      keys each thread holds per work chunk, 1..8 (0 = 1);
 *                       iceberg operations use 1, 2 or 4 (larger values
 *                       count as 4, 3 as 2).
 * cta_threads           threads per block, a multiple of 32 (0 = 256).
 * max_ctas              upper bound on blocks (0 = enough to fill the GPU).
 * max_tiles             upper bound on tiles that take work (0 = no bound).
 *                       With max_tiles = 1 a single tile processes the keys
 *                       strictly in input order (a sequential run).
 * lookups_in_flight     bucket loads a tile keeps in flight: 1, 4 or 8 (0 =
 *                       4 for cuckoo tables, 1 for iceberg tables). With 1
 *                       each tile walks its pending keys one load at a time
 *                       (chunks of items_per_thread keys per lane); with 4
 *                       or 8 every lane holds a key, each round takes one
 *                       step of all of a tile's keys with that many loads
 *                       issued back to back (puts and find-or-puts also
 *                       issue that many claims before reading any), and
 *                       answered lanes take the next key (a stream of fully
 *                       packed rounds). For iceberg find-or-put and lookups
 *                       the stream covers the primary level, and a second
 *                       pass takes the keys whose primary bucket was full
 *                       through level 2 (and the stash). Answers (lookups;
 *                       one PUT per absent key) are the same for every
 *                       value; runs with slot outputs or value moves use 1.
 * retry_limit           iceberg find-or-put: lost claims a key may retry
 *                       before it gives up with status CHT_ERROR, 0..32767
 *                       (0 = the built-in bound, which a correct run never
 *                       reaches: a key can lose at most once per slot of
 *                       its three buckets, Appendix A). A small value lets a
 *                       test drive the error path (CHT_ERROR statuses and
 *                       cht_error_flags) under contention; set it at
 *                       cht_create. Cuckoo tables ignore it.
 * stash_slots           iceberg level-3 overflow stash (Section 2.3 describes
 *                       a third level; the paper's implementation leaves it
 *                       out): 0 = none, else a power of two in [2, 2^30],
 *                       the number of whole-key slots. A key goes there only
 *                       when its primary and both secondary buckets are full
 *                       (a two-level table would report CHT_FULL); the stash
 *                       is an open-addressing table with linear probing from
 *                       a hash of the key, claimed by 64-bit compare-and-swap,
 *                       so find-or-put still reports exactly one CHT_PUT per
 *                       absent key and CHT_FULL only once the key's probe
 *                       sequence holds no free slot. Cuckoo tables must
 *                       leave it 0.
 * bucket_words          64-bit words per bucket, both levels: 16 (128 bytes,
 *                       one cache line; 0 selects it), 8 or 4 (64- or
 *                       32-byte buckets: with 32-bit slots the 16- and 8-slot
 *                       buckets that Section 5.1 sweeps beside 32). Smaller
 *                       buckets use tiles of bucket_words / 2 lanes (the tile
 *                       field must be 0 or that) and offer insert, find,
 *                       find-or-put and enumerate; slot outputs, key-value
 *                       calls and fused batches need 16.
 */
typedef struct cht_config {
    int32_t kind;
    int32_t compact;
    int32_t key_bits;
    int32_t key_bytes;
    uint64_t num_buckets;
    uint64_t num_buckets_backyard;
    int32_t fields_per_word;
    int32_t fields_per_word_backyard;
    int32_t num_hashes;
    int32_t max_chain;
    uint64_t seed;
    int32_t tile;
    int32_t items_per_thread;
    int32_t cta_threads;
    int32_t max_ctas;
    int32_t max_tiles;
    int32_t lookups_in_flight;
    int32_t retry_limit;
    int32_t stash_slots;
    int32_t bucket_words;
    int32_t reserved;
} cht_config;

/* Device counters a table can accumulate into (see cht_set_counters). */
typedef struct cht_counters {
    uint64_t probes;     /* bucket reads (one 128-byte line each)            */
    uint64_t writes;     /* successful slot claims and cuckoo swaps           */
    uint64_t cas_fail;   /* claims that lost a race and were retried          */
    uint64_t ops;        /* keys processed                                    */
} cht_counters;

/*
 * Resolve zero fields to defaults and validate. On CHT_OK, *out holds the
 * resolved configuration (out may alias cfg). Host only; no CUDA calls.
 */
int cht_resolve_config(const cht_config *cfg, cht_config *out);

/*
 * Bytes of device storage a table of this configuration needs:
 * CHT_HEADER_BYTES + (num_buckets + num_buckets_backyard) * 8 * bucket_words
 * (no backyard for cuckoo), plus 8 * stash_slots rounded up to a multiple of
 * CHT_BUCKET_BYTES for an iceberg stash. Returns 0 if the configuration is
 * invalid. Host only.
 */
size_t cht_table_bytes(const cht_config *cfg);

/*
 * Create a table handle over caller-owned device storage d_mem of at least
 * cht_table_bytes(cfg) bytes, 256-byte aligned. The storage is zeroed on
 * stream (an empty table). The handle does not own d_mem; the caller keeps it
 * alive until cht_destroy. *out receives the handle.
 */
int cht_create(const cht_config *cfg, void *d_mem, size_t bytes, void *stream,
               cht_table **out);

/* Free the host handle (the device storage stays the caller's). */
int cht_destroy(cht_table *t);

/* Empty the table again (zero its buckets and header) on stream. */
int cht_clear(cht_table *t, void *stream);

/* Copy the resolved configuration of a table into *out. Host only. */
int cht_get_config(const cht_table *t, cht_config *out);

/*
 * Change how later calls on the table are launched, leaving its contents and
 * layout alone: only the launch fields of *launch are read (tile,
 * items_per_thread, cta_threads, max_ctas, max_tiles, lookups_in_flight; zero
 * selects the default). Used by autotuners. Host only; validates like
 * cht_resolve_config and leaves the table unchanged on error.
 */
int cht_set_launch(cht_table *t, const cht_config *launch);

/*
 * Insert n keys (d_keys, key_bytes each). d_status[i] receives CHT_PUT,
 * CHT_FULL, CHT_INVALID or (iceberg) CHT_FOUND.
 * Cuckoo: Algorithm 4 per key. Keys must be unique within the table's
 *   lifetime (a static build, Section 1); a put that runs out of its
 *   max_chain eviction steps reports CHT_FULL and, when d_dropped is not
 *   NULL, d_dropped[i] receives the key that was left without a slot (it may
 *   be another key, evicted along the chain). d_dropped entries of keys whose
 *   status is not CHT_FULL are not written. Must not overlap a find or
 *   another insert on the same table.
 * Iceberg: the same as cht_find_or_put (d_dropped is ignored).
 */
int cht_insert(cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
               uint64_t *d_dropped, void *stream);

/*
 * Look up n keys. d_status[i] receives CHT_FOUND, CHT_NOT_FOUND or
 * CHT_INVALID. Cuckoo: probes a_0, a_1, ... and stops at the first bucket
 * that holds the key or has a free slot (Section 4.4). Iceberg: the primary
 * bucket, then both secondary buckets if the primary is full (Section 2.3).
 */
int cht_find(const cht_table *t, const void *d_keys, size_t n,
             uint8_t *d_status, void *stream);

/*
 * Iceberg find-or-put (Algorithm 1 per key): CHT_FOUND if the key was in the
 * table, otherwise CHT_PUT if this call inserted it, or CHT_FULL if its
 * primary and both secondary buckets are full. Duplicates within a batch and
 * concurrent calls are allowed: of several find-or-puts of one absent key
 * exactly one reports CHT_PUT and the others CHT_FOUND (Theorem 1).
 * Cuckoo tables return CHT_ERR_UNSUPPORTED (Section 4.4 gives no lockless
 * find-or-put for cuckoo hashing).
 */
int cht_find_or_put(cht_table *t, const void *d_keys, size_t n,
                    uint8_t *d_status, void *stream);

/*
 * Key-value extension (the paper names a key-value map as the natural next
 * step; iceberg entries never move once placed, Section 5.1, so a key's slot
 * is a stable handle that can index a caller-owned value array).
 *
 * cht_find_or_put_slots: cht_find_or_put, and also d_slots[i] = the slot that
 * holds key i after the call when its status is FOUND or PUT, else
 * UINT64_MAX. cht_find_slots: cht_find, with d_slots as above for FOUND keys.
 * Slot numbering: level-0 slot y of primary bucket a is a * B0 + y; level-1
 * slot y of secondary bucket a is nb0 * B0 + a * B1 + y, where B0 = 16 *
 * fields_per_word and B1 = 16 * fields_per_word_backyard are the slots per
 * bucket and y runs over a bucket's slots in slot order (word by word, field
 * by field); stash position p (level 3, when the table has a stash) is slot
 * nb0 * B0 + nb1 * B1 + p. There are nb0 * B0 + nb1 * B1 + stash_slots slots
 * in all. A key keeps its slot for the table's lifetime (until cht_clear). d_slots: n device uint64
 * (8-byte aligned), written. Iceberg tables only (CHT_ERR_UNSUPPORTED on
 * cuckoo tables, whose puts move entries); other arguments and errors as for
 * cht_find_or_put / cht_find.
 */
int cht_find_or_put_slots(cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                          uint64_t *d_slots, void *stream);
int cht_find_slots(const cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                   uint64_t *d_slots, void *stream);

/*
 * Value moves for the key-value extension. d_store is a caller-owned device
 * array of store_slots values (value_bytes = 4, 8 or 16 each), indexed by slot.
 * cht_values_scatter: d_store[d_slots[i]] = d_values[i] for every i with
 * d_slots[i] < store_slots (two keys of one call with the same slot: one of
 * the values lands, which one is unspecified). cht_values_gather: d_out[i] =
 * d_store[d_slots[i]], or zero when d_slots[i] >= store_slots (UINT64_MAX for
 * keys not found). d_slots: n device uint64; values aligned to value_bytes.
 * Asynchronous on stream; CHT_ERR_INVALID on bad arguments.
 */
int cht_values_scatter(const uint64_t *d_slots, size_t n, const void *d_values, int value_bytes,
                       void *d_store, uint64_t store_slots, void *stream);
int cht_values_gather(const uint64_t *d_slots, size_t n, const void *d_store, int value_bytes,
                      uint64_t store_slots, void *d_out, void *stream);

/*
 * Fused key-value put and get: one kernel each, the value move done by the
 * lane that answers the key. cht_kv_put = cht_find_or_put, then for every
 * FOUND or PUT key i d_store[slot(i)] = d_values[i] (insert or assign; a key
 * given twice in one call keeps one of its values, which one is unspecified;
 * FULL keys store nothing). cht_kv_get = cht_find, then d_out[i] =
 * d_store[slot(i)] for FOUND keys and zero otherwise. d_store holds
 * store_slots values of value_bytes (4, 8 or 16) and must cover the table's
 * slots (nb0 * B0 + nb1 * B1 + stash_slots, see above) for every key to have its value;
 * slots at or past store_slots are skipped. Iceberg tables only
 * (CHT_ERR_UNSUPPORTED otherwise); values aligned to value_bytes
 * (CHT_ERR_INVALID otherwise); keys, statuses and errors as for
 * cht_find_or_put / cht_find.
 * Ordering: a value is written by a plain store after its key's slot has
 * been claimed, and nothing orders the two for other threads. So a
 * cht_kv_get that runs concurrently with a cht_kv_put of the same key (other
 * streams) may find the key and read the slot's previous value (zero for a
 * fresh slot); order them on one stream for the new value. A 16-byte value
 * is written as one 16-byte store, whose two 8-byte halves are separate
 * single-copy atomic accesses: when a key is given twice in one cht_kv_put,
 * each half of the stored value comes from one of the copies, not
 * necessarily the same one. 4- and 8-byte values are written whole.
 */
int cht_kv_put(cht_table *t, const void *d_keys, size_t n, const void *d_values, int value_bytes,
               void *d_store, uint64_t store_slots, uint8_t *d_status, void *stream);
int cht_kv_get(const cht_table *t, const void *d_keys, size_t n, const void *d_store,
               int value_bytes, uint64_t store_slots, void *d_out, uint8_t *d_status,
               void *stream);

/*
 * Write every stored key, decoded as k = pi_j^-1(a . r) (Section 2.4), to
 * d_out (key_bytes each) in unspecified order, at most cap keys. *d_count (a
 * device uint64) receives the number of stored keys, which may exceed cap;
 * it is overwritten, not accumulated.
 */
int cht_enumerate(const cht_table *t, void *d_out, size_t cap,
                  uint64_t *d_count, void *stream);

/*
 * Attach a device cht_counters block (or NULL to detach). Later calls on the
 * table add their probe/write/retry/op counts into it with atomics. The
 * caller zeroes it. Counting costs a few instructions per key and one atomic
 * per warp.
 */
int cht_set_counters(cht_table *t, cht_counters *d_counters);

/*
 * Read the device error word of the table header (synchronises stream). A
 * nonzero value means something went wrong since the last clear: bit 0, some
 * key got CHT_ERROR status (a bounded retry loop gave up); bit 1, a kernel's
 * own bound on its loop ran out, and keys it had not answered may be left
 * with CHT_ERROR or unwritten statuses. Neither happens in a correct run.
 */
int cht_error_flags(const cht_table *t, uint32_t *flags, void *stream);

/* ------------------------------------------------------------------------ */
/* Fused multi-table batches                                                 */
/* ------------------------------------------------------------------------ */
/*
 * A batch applies one operation to many iceberg tables, each with its own key
 * array, in ONE persistent kernel launch: the chunks of all tables form one
 * index space that every tile walks, so small and large batches share the GPU
 * instead of each paying a launch and a tail. The operation is Algorithm 1
 * (find-or-put) or the Section 2.3 lookup, per key exactly as cht_find_or_put
 * and cht_find on that table.
 *
 * All tables of a batch must be iceberg tables on the current device with the
 * same primary packing (fields_per_word). Tables, key arrays and status arrays
 * must stay alive for as long as the batch is launched. In a find-or-put batch
 * no table may appear twice (CHT_ERR_INVALID); a lookup batch may list a table
 * several times, each entry with its own keys (lookups only read). A table may
 * be written by only one batch or call at a time.
 */
typedef struct cht_batch cht_batch; /* opaque host handle */

#define CHT_OP_FIND_OR_PUT 0
#define CHT_OP_FIND 1

/* Device scratch bytes a batch of count tables needs (its descriptors). */
size_t cht_batch_scratch_bytes(int count);

/*
 * Plan a batch: count (1..16384) entries of (tables[i], d_keys[i], n[i],
 * d_status[i]). The descriptors are written into the caller-owned device
 * scratch d_scratch (at least cht_batch_scratch_bytes(count) bytes, 16-byte
 * aligned) by small kernels enqueued on stream (the descriptors travel as
 * kernel parameters, so the call does not wait on the stream); the scratch
 * must stay untouched until cht_batch_destroy. Launch shape: tile 4, 1 item
 * per thread, 256 threads per block unless changed with
 * cht_batch_set_launch.
 */
int cht_batch_create(cht_table *const *tables, const void *const *d_keys, const size_t *n,
                     uint8_t *const *d_status, int count, int op, void *d_scratch,
                     size_t scratch_bytes, void *stream, cht_batch **out);

/* Change the launch shape (tile, items_per_thread, cta_threads, max_ctas of
 * *launch; zero = default). Drops a captured graph. Host only. */
int cht_batch_set_launch(cht_batch *b, const cht_config *launch);

/* Enqueue the fused launch on stream (capturable in a CUDA graph). */
int cht_batch_launch(const cht_batch *b, void *stream);

/*
 * Capture one fused launch into a CUDA graph owned by the batch (on an
 * internal stream; stream only orders the capture after earlier work) and
 * instantiate it. cht_batch_replay then launches the graph on any stream.
 */
int cht_batch_capture(cht_batch *b, void *stream);
int cht_batch_replay(const cht_batch *b, void *stream);

/* Empty every table of the batch (zero buckets and headers) in one launch. */
int cht_batch_clear(const cht_batch *b, void *stream);

/* Free the batch handle and its graph (the scratch stays the caller's). */
int cht_batch_destroy(cht_batch *b);

/*
 * Allocation-free fused find-or-put (the paper has no counterpart; this is a
 * convenience of this library). Same work as cht_batch_create with
 * CHT_OP_FIND_OR_PUT followed by cht_batch_launch, but for callers that must
 * not allocate device memory at all: code that runs while another thread
 * captures a CUDA graph in global capture mode (where cudaMalloc is an illegal
 * call), latency-critical loops that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause, and hosts where another
 * allocator has already reserved the GPU's memory so a fresh cudaMalloc fails.
 *
 * The batch descriptors live in a fixed array inside the library (device
 * memory that every GPU which loads the library holds until the process
 * exits) with room for CHT_STATIC_BATCH_MAX tables (240 bytes each, 60 KiB in
 * all); count above that is rejected with CHT_ERR_INVALID. Nothing is
 * allocated on any call: the descriptors travel to the array as the
 * parameters of small kernel launches on stream (so the host never waits),
 * then the fused kernel runs. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, and looks
 * it up again if the device's context has changed since (cudaDeviceReset);
 * make that first call before any stream capture. Every call shares the one
 * array and each call overwrites the descriptors it uses (nothing in it has
 * to start at zero), so calls whose work overlaps on the GPU (different
 * streams, or different host threads) race: order them on one stream.
 * Arguments and per-key results are as for cht_batch_create /
 * cht_find_or_put; all tables must be iceberg tables with the same primary
 * packing on the current device, and no table may be listed twice
 * (CHT_ERR_INVALID).
 */
#define CHT_STATIC_BATCH_MAX 256
int cht_batch_find_or_put_static(cht_table *const *tables, const void *const *d_keys,
                                 const size_t *n, uint8_t *const *d_status, int count,
                                 void *stream);

/* Message for the last failed call on this thread ("" if none). */
const char *cht_last_error(void);

/* Library version string. */
const char *cht_version(void);

/*
 * Measurement utility; the paper has no counterpart. Reads n_blocks blocks of
 * block_bytes (32, 64, 128 or 256) from d_buf at pseudo-random block indices
 * (splitmix64 of seed + i, masked to the block count) and XOR-folds the data
 * into *d_sink. One tile of lanes reads a block with one 16-byte (256: 32-byte)
 * load per lane, four blocks in flight per tile, on a grid that fills the
 * GPU. Timed with events on stream, it gives the random-access rate of the
 * memory behind d_buf: the ceiling for bucket probes, which are reads of one
 * 128-byte line at a data-dependent address. d_buf: device memory of
 * buf_bytes = block_bytes x a power of two, 32-byte aligned, only read;
 * d_sink: one 8-byte aligned device word, modified. Asynchronous on stream;
 * CHT_ERR_INVALID on bad arguments, CHT_ERR_CUDA if the launch fails.
 */
int cht_random_read(const void *d_buf, size_t buf_bytes, int block_bytes, uint64_t n_blocks,
                    uint64_t seed, uint64_t *d_sink, void *stream);

/*
 * Measurement utility; the paper has no counterpart. The access pattern of a
 * put that claims a slot in the first bucket it probes: for each of n_lines
 * pseudo-random 128-byte lines of d_buf (splitmix64 of seed + i, masked to
 * the line count), eight lanes read the line with 16-byte relaxed loads, then
 * the lane owning one of its words (chosen from the same hash) compare-and-
 * swaps that word from the value it read to that value + 1; four lines per
 * tile in flight, the four compare-and-swaps issued before any result is
 * read, as the put kernels do. Timed with events on stream, it gives the
 * rate at which this GPU's memory serves a line read plus the write-back of
 * the dirtied line: the ceiling for puts. d_buf: device memory of buf_bytes =
 * 128 x a power of two, 128-byte aligned, modified; d_sink: one 8-byte aligned
 * device word, modified. Asynchronous on stream; CHT_ERR_INVALID on bad
 * arguments, CHT_ERR_CUDA if the launch fails.
 */
int cht_random_claim(void *d_buf, size_t buf_bytes, uint64_t n_lines, uint64_t seed,
                     uint64_t *d_sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CHT_H */
