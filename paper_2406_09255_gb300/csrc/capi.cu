// capi.cu - the C ABI declared in include/cht.h: configuration planning and
// validation, table handles over caller-owned device storage, and dispatch
// of the hot-path kernels. No device memory is allocated here.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cht.h"
#include "cht_kernels.cuh"
#include "cht_scan.cuh"
#include "cht_launch.h"

using namespace cht;

struct cht_table {
    cht_config cfg;       // resolved
    TableArgs args;       // what the kernels see
    unsigned char *mem;   // caller's storage (header + buckets)
    size_t bytes;
    int device;
    int sms;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int ok() {
    g_err.clear();
    return CHT_OK;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(CHT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ceil_log2(uint64_t x) {
    int n = 0;
    while (n < 64 && (1ull << n) < x) n++;
    return n;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

// tag bits of an entry: cuckoo (j + 1) and iceberg secondary (i + 1) take 2,
// the iceberg primary occupancy flag 1
int tag_bits(int kind, int level) { return (kind == CHT_ICEBERG && level == 0) ? 1 : 2; }

int resolve_level(cht_config &c, int level, uint64_t nb, int32_t &fpw) {
    const char *lname = level ? "num_buckets_backyard" : "num_buckets";
    if (nb < 1) return fail(CHT_ERR_INVALID, "%s must be >= 1", lname);
    // the kernels carry bucket indices in 32 bits (2^32 buckets = 512 GiB)
    if (nb > (1ull << 32)) return fail(CHT_ERR_INVALID, "%s must be at most 2^32", lname);
    if (c.compact && !is_pow2(nb))
        return fail(CHT_ERR_INVALID, "%s = %llu must be a power of two for a compact table",
                    lname, (unsigned long long)nb);
    const int n = ceil_log2(nb);
    if (n >= c.key_bits)
        return fail(CHT_ERR_INVALID, "%s = 2^%d leaves no remainder bits for %d-bit keys", lname,
                    n, c.key_bits);
    const int body = c.compact ? c.key_bits - n : c.key_bits;
    const int need = body + tag_bits(c.kind, level);
    if (fpw == 0) {
        if (!c.compact) {
            fpw = 1;
        } else {
            for (int f = 4; f >= 1; --f)
                if (need <= 64 / f) {
                    fpw = f;
                    break;
                }
        }
    }
    if (fpw < 1 || fpw > 4)
        return fail(CHT_ERR_INVALID, "fields per word must be 1..4 (got %d)", fpw);
    if (need > 64 / fpw)
        return fail(CHT_ERR_INVALID,
                    "level %d entries need %d bits but %d fields per word give %d-bit slots",
                    level, need, fpw, 64 / fpw);
    return CHT_OK;
}

int resolve(const cht_config *in, cht_config *out) {
    if (!in || !out) return fail(CHT_ERR_INVALID, "null configuration pointer");
    cht_config c = *in;
    if (c.kind != CHT_CUCKOO && c.kind != CHT_ICEBERG)
        return fail(CHT_ERR_INVALID, "kind must be CHT_CUCKOO or CHT_ICEBERG");
    if (c.compact != 0 && c.compact != 1) return fail(CHT_ERR_INVALID, "compact must be 0 or 1");
    if (c.key_bytes != 4 && c.key_bytes != 8)
        return fail(CHT_ERR_INVALID, "key_bytes must be 4 or 8");
    if (c.key_bits < 2 || c.key_bits > 62 || c.key_bits > 8 * c.key_bytes)
        return fail(CHT_ERR_INVALID, "key_bits = %d out of range for %d-byte keys", c.key_bits,
                    c.key_bytes);
    if (c.kind == CHT_CUCKOO) {
        if (c.num_hashes == 0) c.num_hashes = 3;
        if (c.num_hashes < 1 || c.num_hashes > 3)
            return fail(CHT_ERR_INVALID, "num_hashes must be 1..3");
        if (c.max_chain == 0) c.max_chain = 128;
        if (c.max_chain < 1) return fail(CHT_ERR_INVALID, "max_chain must be >= 1");
        c.num_buckets_backyard = 0;
        c.fields_per_word_backyard = 0;
    } else {
        c.num_hashes = 0;
        c.max_chain = 0;
    }
    int e = resolve_level(c, 0, c.num_buckets, c.fields_per_word);
    if (e) return e;
    if (c.kind == CHT_ICEBERG) {
        e = resolve_level(c, 1, c.num_buckets_backyard, c.fields_per_word_backyard);
        if (e) return e;
    }
    if (c.bucket_words == 0) c.bucket_words = kWordsPerBucket;
    if (c.bucket_words != 4 && c.bucket_words != 8 && c.bucket_words != 16)
        return fail(CHT_ERR_INVALID, "bucket_words must be 4, 8 or 16 (got %d)", c.bucket_words);
    // tile 0 stays 0: each operation then uses its own best width
    if (c.bucket_words < kWordsPerBucket) {
        if (c.tile != 0 && c.tile != c.bucket_words / 2)
            return fail(CHT_ERR_INVALID, "tile must be 0 or %d for %d-word buckets",
                        c.bucket_words / 2, c.bucket_words);
    } else if (c.tile != 0 && c.tile != 4 && c.tile != 8 && c.tile != 16) {
        return fail(CHT_ERR_INVALID, "tile must be 4, 8 or 16 (got %d)", c.tile);
    }
    if (c.items_per_thread == 0) c.items_per_thread = 1;
    if (c.items_per_thread < 1 || c.items_per_thread > 8)
        return fail(CHT_ERR_INVALID, "items_per_thread must be 1..8");
    if (c.cta_threads == 0) c.cta_threads = 256;
    if (c.cta_threads < 32 || c.cta_threads > 256 || c.cta_threads % 32)
        return fail(CHT_ERR_INVALID, "cta_threads must be a multiple of 32 in [32, 256]");
    if (c.max_ctas < 0 || c.max_tiles < 0)
        return fail(CHT_ERR_INVALID, "max_ctas and max_tiles must be >= 0");
    if (c.retry_limit < 0 || c.retry_limit > 32767)
        return fail(CHT_ERR_INVALID, "retry_limit must be 0..32767");
    if (c.stash_slots != 0) {
        if (c.kind != CHT_ICEBERG)
            return fail(CHT_ERR_INVALID, "stash_slots: only iceberg tables have a stash");
        if (c.stash_slots < 2 || c.stash_slots > (1 << 30) ||
            !is_pow2((uint64_t)c.stash_slots))
            return fail(CHT_ERR_INVALID, "stash_slots must be 0 or a power of two in [2, 2^30]");
    }
    // cuckoo: the stream kernels; iceberg: the warp-batched chunk engine
    if (c.lookups_in_flight == 0) c.lookups_in_flight = c.kind == CHT_ICEBERG ? 1 : 4;
    if (c.lookups_in_flight != 1 && c.lookups_in_flight != 4 && c.lookups_in_flight != 8)
        return fail(CHT_ERR_INVALID, "lookups_in_flight must be 1, 4 or 8");
    *out = c;
    return CHT_OK;
}

// bytes of the stash region: 8 per slot, rounded up to whole 128-byte lines
uint64_t stash_bytes(const cht_config &c) {
    return ((uint64_t)c.stash_slots + 15) / 16 * CHT_BUCKET_BYTES;
}

size_t table_bytes(const cht_config &c) {
    uint64_t nb = c.num_buckets + (c.kind == CHT_ICEBERG ? c.num_buckets_backyard : 0);
    return CHT_HEADER_BYTES + (size_t)nb * 8 * (size_t)c.bucket_words + (size_t)stash_bytes(c);
}

void fill_level(Level &L, uint64_t *words, uint64_t nb, int key_bits, int fpw, uint64_t seed,
                int level) {
    L.words = words;
    L.nb = nb;
    L.n = ceil_log2(nb);
    L.R = key_bits - L.n;
    L.pow2 = is_pow2(nb);
    L.fpw = fpw;
    for (int j = 0; j < 3; ++j) {
        const uint64_t idx = 2ull * (uint64_t)(4 * level + j);
        L.A[j] = splitmix(seed, idx) | 1ull;
        L.B[j] = splitmix(seed, idx + 1);
    }
}

enum Op { kOpCuckooInsert, kOpCuckooFind, kOpIcebergFop, kOpIcebergFind };

// threads per bucket for an operation: the configured tile, or when it is 0
// the width measured fastest on GB300 for that operation. Cuckoo lookups use
// eight lanes, one 16-byte read each, so one warp load fetches four whole
// lines and their stream kernel keeps four of those in flight per tile.
// Everything else keeps four lanes per bucket: twice the keys per warp pass,
// which outweighs the second 16-byte read per lane for the puts and for the
// iceberg engine's passes.
int tile_for(const cht_table *t, Op op) {
    if (t->cfg.tile) return t->cfg.tile;
    switch (op) {
        case kOpCuckooInsert: return 4;
        case kOpCuckooFind: return 8;
        case kOpIcebergFop: return 4;
        case kOpIcebergFind: return 4;
    }
    return 4;
}

LaunchParams launch_params(const cht_table *t, void *stream) {
    LaunchParams lp;
    lp.cta = t->cfg.cta_threads;
    lp.items = t->cfg.items_per_thread;
    lp.max_ctas = t->cfg.max_ctas;
    lp.max_tiles = t->cfg.max_tiles;
    lp.in_flight = t->cfg.lookups_in_flight;
    lp.sms = t->sms;
    lp.stream = static_cast<cudaStream_t>(stream);
    return lp;
}

int check_keys(const cht_table *t, const void *d_keys, size_t n, const void *d_out) {
    if (!t) return fail(CHT_ERR_INVALID, "null table");
    if (n && (!d_keys || !d_out)) return fail(CHT_ERR_INVALID, "null key or output pointer");
    if ((uintptr_t)d_keys % t->cfg.key_bytes)
        return fail(CHT_ERR_INVALID, "key array not aligned to %d bytes", t->cfg.key_bytes);
    return CHT_OK;
}

int clear_storage(cht_table *t, cudaStream_t s) {
    const uint64_t n16 = t->bytes / 16;
    int blocks = (int)std::min<uint64_t>((n16 + 255) / 256, (uint64_t)t->sms * 8);
    if (blocks < 1) blocks = 1;
    k_clear<<<blocks, 256, 0, s>>>(reinterpret_cast<ulonglong2 *>(t->mem), n16);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CHT_OK : cuda_fail(e, "clear kernel launch");
}

}  // namespace

extern "C" {

int cht_resolve_config(const cht_config *cfg, cht_config *out) {
    int e = resolve(cfg, out);
    return e ? e : ok();
}

size_t cht_table_bytes(const cht_config *cfg) {
    cht_config c;
    if (resolve(cfg, &c)) return 0;
    return table_bytes(c);
}

int cht_create(const cht_config *cfg, void *d_mem, size_t bytes, void *stream, cht_table **out) {
    if (!out) return fail(CHT_ERR_INVALID, "null output handle pointer");
    *out = nullptr;
    cht_config c;
    int e = resolve(cfg, &c);
    if (e) return e;
    const size_t need = table_bytes(c);
    if (!d_mem) return fail(CHT_ERR_INVALID, "null table storage");
    if ((uintptr_t)d_mem % 256) return fail(CHT_ERR_INVALID, "table storage not 256-byte aligned");
    if (bytes < need)
        return fail(CHT_ERR_CAPACITY, "table storage of %zu bytes is below the %zu needed", bytes,
                    need);
    cht_table *t = new cht_table();
    t->cfg = c;
    t->mem = static_cast<unsigned char *>(d_mem);
    t->bytes = need;
    cudaError_t ce = cudaGetDevice(&t->device);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, t->device);
    if (ce != cudaSuccess) {
        delete t;
        return cuda_fail(ce, "device query");
    }
    TableArgs &a = t->args;
    memset(&a, 0, sizeof a);
    uint64_t *words0 = reinterpret_cast<uint64_t *>(t->mem + CHT_HEADER_BYTES);
    fill_level(a.lv[0], words0, c.num_buckets, c.key_bits, c.fields_per_word, c.seed, 0);
    if (c.kind == CHT_ICEBERG)
        fill_level(a.lv[1], words0 + c.num_buckets * (uint64_t)c.bucket_words, c.num_buckets_backyard,
                   c.key_bits, c.fields_per_word_backyard, c.seed, 1);
    a.w = (int16_t)c.key_bits;
    a.key_bytes = (int16_t)c.key_bytes;
    a.H = (int16_t)c.num_hashes;
    a.wpb = (int16_t)c.bucket_words;
    a.C = c.max_chain;
    a.compact = (int16_t)c.compact;
    a.retry_limit = (int16_t)c.retry_limit;
    a.max_tiles = c.max_tiles;
    a.err = reinterpret_cast<uint32_t *>(t->mem);
    a.ctr = nullptr;
    a.stash_slots = (uint64_t)c.stash_slots;
    // output 16 of the seed's splitmix64 sequence, after the permutation
    // constants of levels 0 and 1 (outputs 0..13)
    a.stash_key = splitmix(c.seed, 16);
    e = clear_storage(t, static_cast<cudaStream_t>(stream));
    if (e) {
        delete t;
        return e;
    }
    *out = t;
    return ok();
}

int cht_destroy(cht_table *t) {
    delete t;
    return ok();
}

int cht_clear(cht_table *t, void *stream) {
    if (!t) return fail(CHT_ERR_INVALID, "null table");
    int e = clear_storage(t, static_cast<cudaStream_t>(stream));
    return e ? e : ok();
}

int cht_get_config(const cht_table *t, cht_config *out) {
    if (!t || !out) return fail(CHT_ERR_INVALID, "null argument");
    *out = t->cfg;
    return ok();
}

int cht_set_launch(cht_table *t, const cht_config *launch) {
    if (!t || !launch) return fail(CHT_ERR_INVALID, "null argument");
    cht_config c = t->cfg;
    c.tile = launch->tile;
    c.items_per_thread = launch->items_per_thread;
    c.cta_threads = launch->cta_threads;
    c.max_ctas = launch->max_ctas;
    c.max_tiles = launch->max_tiles;
    c.lookups_in_flight = launch->lookups_in_flight;
    cht_config r;
    int e = resolve(&c, &r);
    if (e) return e;
    t->cfg = r;
    t->args.max_tiles = r.max_tiles;
    return ok();
}

int cht_insert(cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
               uint64_t *d_dropped, void *stream) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    cudaError_t ce;
    if (t->cfg.bucket_words < kWordsPerBucket)
        ce = launch_small_buckets(t->cfg.kind == CHT_CUCKOO ? kSmallCuckooInsert : kSmallIcebergFop,
                                  t->cfg.bucket_words, t->cfg.fields_per_word, lp, t->args,
                                  d_keys, n, d_status, d_dropped);
    else if (t->cfg.kind == CHT_CUCKOO)
        ce = launch_cuckoo_insert(tile_for(t, kOpCuckooInsert), t->cfg.fields_per_word, lp, t->args, d_keys, n,
                                  d_status, d_dropped);
    else
        ce = launch_iceberg(tile_for(t, kOpIcebergFop), t->cfg.fields_per_word, false, lp, t->args, d_keys, n,
                            d_status);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "insert kernel launch");
}

int cht_find(const cht_table *t, const void *d_keys, size_t n, uint8_t *d_status, void *stream) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    cudaError_t ce;
    if (t->cfg.bucket_words < kWordsPerBucket)
        ce = launch_small_buckets(t->cfg.kind == CHT_CUCKOO ? kSmallCuckooFind : kSmallIcebergFind,
                                  t->cfg.bucket_words, t->cfg.fields_per_word, lp, t->args,
                                  d_keys, n, d_status, nullptr);
    else if (t->cfg.kind == CHT_CUCKOO)
        ce = launch_cuckoo_find(tile_for(t, kOpCuckooFind), t->cfg.fields_per_word, lp, t->args, d_keys, n,
                                d_status);
    else
        ce = launch_iceberg(tile_for(t, kOpIcebergFind), t->cfg.fields_per_word, true, lp, t->args, d_keys, n,
                            d_status);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "find kernel launch");
}

int cht_find_or_put_slots(cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                          uint64_t *d_slots, void *stream) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (t->cfg.kind != CHT_ICEBERG)
        return fail(CHT_ERR_UNSUPPORTED, "slot indices are stable in iceberg tables only");
    if (t->cfg.bucket_words != kWordsPerBucket)
        return fail(CHT_ERR_UNSUPPORTED, "slot outputs need 16-word (128-byte) buckets");
    if (!d_slots || (uintptr_t)d_slots % 8) return fail(CHT_ERR_INVALID, "d_slots must be 8-byte aligned");
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    cudaError_t ce = launch_iceberg(tile_for(t, kOpIcebergFop), t->cfg.fields_per_word, false, lp,
                                    t->args, d_keys, n, d_status, d_slots);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "find-or-put kernel launch");
}

int cht_find_slots(const cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                   uint64_t *d_slots, void *stream) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (t->cfg.kind != CHT_ICEBERG)
        return fail(CHT_ERR_UNSUPPORTED, "slot indices are stable in iceberg tables only");
    if (t->cfg.bucket_words != kWordsPerBucket)
        return fail(CHT_ERR_UNSUPPORTED, "slot outputs need 16-word (128-byte) buckets");
    if (!d_slots || (uintptr_t)d_slots % 8) return fail(CHT_ERR_INVALID, "d_slots must be 8-byte aligned");
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    cudaError_t ce = launch_iceberg(tile_for(t, kOpIcebergFind), t->cfg.fields_per_word, true, lp,
                                    t->args, d_keys, n, d_status, d_slots);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "find kernel launch");
}

static int values_call(bool scatter, const uint64_t *d_slots, size_t n, const void *src,
                       void *dst, int value_bytes, uint64_t store_slots, void *stream) {
    if (value_bytes != 4 && value_bytes != 8 && value_bytes != 16)
        return fail(CHT_ERR_INVALID, "value_bytes must be 4, 8 or 16");
    if (n == 0) return ok();
    if (!d_slots || !src || !dst) return fail(CHT_ERR_INVALID, "null pointer");
    if ((uintptr_t)d_slots % 8 || (uintptr_t)src % value_bytes || (uintptr_t)dst % value_bytes)
        return fail(CHT_ERR_INVALID, "misaligned slots or values");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = launch_values(scatter, d_slots, n, src, dst, value_bytes, store_slots, sms,
                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "value kernel launch");
}

int cht_values_scatter(const uint64_t *d_slots, size_t n, const void *d_values, int value_bytes,
                       void *d_store, uint64_t store_slots, void *stream) {
    return values_call(true, d_slots, n, d_values, d_store, value_bytes, store_slots, stream);
}

int cht_values_gather(const uint64_t *d_slots, size_t n, const void *d_store, int value_bytes,
                      uint64_t store_slots, void *d_out, void *stream) {
    return values_call(false, d_slots, n, d_store, d_out, value_bytes, store_slots, stream);
}

static int kv_check(const cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                    const void *values, int value_bytes, const void *store) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (t->cfg.kind != CHT_ICEBERG)
        return fail(CHT_ERR_UNSUPPORTED, "key-value maps need iceberg tables (stable slots)");
    if (t->cfg.bucket_words != kWordsPerBucket)
        return fail(CHT_ERR_UNSUPPORTED, "key-value maps need 16-word (128-byte) buckets");
    if (value_bytes != 4 && value_bytes != 8 && value_bytes != 16)
        return fail(CHT_ERR_INVALID, "value_bytes must be 4, 8 or 16");
    if (n && (!values || !store)) return fail(CHT_ERR_INVALID, "null value pointer");
    if ((uintptr_t)values % value_bytes || (uintptr_t)store % value_bytes)
        return fail(CHT_ERR_INVALID, "values not aligned to value_bytes");
    return CHT_OK;
}

int cht_kv_put(cht_table *t, const void *d_keys, size_t n, const void *d_values, int value_bytes,
               void *d_store, uint64_t store_slots, uint8_t *d_status, void *stream) {
    int e = kv_check(t, d_keys, n, d_status, d_values, value_bytes, d_store);
    if (e) return e;
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    const KVArgs kv{d_values, nullptr, d_store, store_slots, value_bytes};
    cudaError_t ce = launch_iceberg(tile_for(t, kOpIcebergFop), t->cfg.fields_per_word, false, lp,
                                    t->args, d_keys, n, d_status, nullptr, &kv);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "key-value put kernel launch");
}

int cht_kv_get(const cht_table *t, const void *d_keys, size_t n, const void *d_store,
               int value_bytes, uint64_t store_slots, void *d_out, uint8_t *d_status,
               void *stream) {
    int e = kv_check(t, d_keys, n, d_status, d_out, value_bytes, d_store);
    if (e) return e;
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    const KVArgs kv{nullptr, d_out, const_cast<void *>(d_store), store_slots, value_bytes};
    cudaError_t ce = launch_iceberg(tile_for(t, kOpIcebergFind), t->cfg.fields_per_word, true, lp,
                                    t->args, d_keys, n, d_status, nullptr, &kv);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "key-value get kernel launch");
}

int cht_find_or_put(cht_table *t, const void *d_keys, size_t n, uint8_t *d_status,
                    void *stream) {
    int e = check_keys(t, d_keys, n, d_status);
    if (e) return e;
    if (t->cfg.kind != CHT_ICEBERG)
        return fail(CHT_ERR_UNSUPPORTED,
                    "find-or-put is offered by iceberg tables only (cuckoo tables are static)");
    if (n == 0) return ok();
    const LaunchParams lp = launch_params(t, stream);
    cudaError_t ce =
        t->cfg.bucket_words < kWordsPerBucket
            ? launch_small_buckets(kSmallIcebergFop, t->cfg.bucket_words, t->cfg.fields_per_word,
                                   lp, t->args, d_keys, n, d_status, nullptr)
            : launch_iceberg(tile_for(t, kOpIcebergFop), t->cfg.fields_per_word, false, lp,
                             t->args, d_keys, n, d_status);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "find-or-put kernel launch");
}

int cht_enumerate(const cht_table *t, void *d_out, size_t cap, uint64_t *d_count, void *stream) {
    if (!t) return fail(CHT_ERR_INVALID, "null table");
    if (!d_count) return fail(CHT_ERR_INVALID, "null count pointer");
    if (cap && !d_out) return fail(CHT_ERR_INVALID, "null output with nonzero capacity");
    if ((uintptr_t)d_out % t->cfg.key_bytes)
        return fail(CHT_ERR_INVALID, "output not aligned to %d bytes", t->cfg.key_bytes);
    if ((uintptr_t)d_count % 8) return fail(CHT_ERR_INVALID, "count not 8-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto *cnt = reinterpret_cast<unsigned long long *>(d_count);
    k_zero_u64<<<1, 32, 0, s>>>(cnt);
    const uint64_t words = (t->cfg.num_buckets +
                            (t->cfg.kind == CHT_ICEBERG ? t->cfg.num_buckets_backyard : 0)) *
                               (uint64_t)t->cfg.bucket_words +
                           stash_bytes(t->cfg) / 8;
    uint64_t blocks = (words / 2 + 255) / 256;
    const uint64_t cap_blocks = (uint64_t)t->sms * 8;
    if (blocks > cap_blocks) blocks = cap_blocks;
    if (blocks < 1) blocks = 1;
    k_enumerate<<<(int)blocks, 256, 0, s>>>(t->args, t->cfg.kind, d_out, cap, cnt);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "enumerate kernel launch");
}

int cht_set_counters(cht_table *t, cht_counters *d_counters) {
    if (!t) return fail(CHT_ERR_INVALID, "null table");
    if ((uintptr_t)d_counters % 8) return fail(CHT_ERR_INVALID, "counters not 8-byte aligned");
    t->args.ctr = reinterpret_cast<unsigned long long *>(d_counters);
    return ok();
}

int cht_error_flags(const cht_table *t, uint32_t *flags, void *stream) {
    if (!t || !flags) return fail(CHT_ERR_INVALID, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t ce = cudaMemcpyAsync(flags, t->args.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "reading the error word");
}

const char *cht_last_error(void) { return g_err.c_str(); }

const char *cht_version(void) { return "cht 0.1 (sm_103a)"; }

int cht_random_read(const void *d_buf, size_t buf_bytes, int block_bytes, uint64_t n_blocks,
                    uint64_t seed, uint64_t *d_sink, void *stream) {
    if (block_bytes != 32 && block_bytes != 64 && block_bytes != 128 && block_bytes != 256)
        return fail(CHT_ERR_INVALID, "block_bytes must be 32, 64, 128 or 256");
    if (!d_buf || !d_sink) return fail(CHT_ERR_INVALID, "null buffer");
    if ((reinterpret_cast<uintptr_t>(d_buf) % 32) || (reinterpret_cast<uintptr_t>(d_sink) % 8))
        return fail(CHT_ERR_INVALID, "d_buf must be 32-byte and d_sink 8-byte aligned");
    if (buf_bytes % (size_t)block_bytes || !is_pow2(buf_bytes / (size_t)block_bytes))
        return fail(CHT_ERR_INVALID, "buf_bytes must be block_bytes times a power of two");
    if (n_blocks == 0) return ok();
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = launch_random_read(d_buf, buf_bytes, block_bytes, n_blocks, seed,
                               reinterpret_cast<unsigned long long *>(d_sink), sms,
                               static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "random read kernel launch");
}

int cht_random_claim(void *d_buf, size_t buf_bytes, uint64_t n_lines, uint64_t seed,
                     uint64_t *d_sink, void *stream) {
    if (!d_buf || !d_sink) return fail(CHT_ERR_INVALID, "null buffer");
    if ((reinterpret_cast<uintptr_t>(d_buf) % 128) || (reinterpret_cast<uintptr_t>(d_sink) % 8))
        return fail(CHT_ERR_INVALID, "d_buf must be 128-byte and d_sink 8-byte aligned");
    if (buf_bytes % 128 || !is_pow2(buf_bytes / 128))
        return fail(CHT_ERR_INVALID, "buf_bytes must be 128 times a power of two");
    if (n_lines == 0) return ok();
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = launch_random_claim(d_buf, buf_bytes, n_lines, seed,
                                reinterpret_cast<unsigned long long *>(d_sink), sms,
                                static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ok() : cuda_fail(e, "random claim kernel launch");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fused multi-table batches
// ---------------------------------------------------------------------------
struct cht_batch {
    std::vector<BatchDesc> host;   // descriptors as uploaded
    BatchDesc *dev;                // caller's scratch
    int count;
    int op;
    int fpw0;
    int device;
    int sms;
    cht_config launch;             // tile, items_per_thread, cta_threads, max_ctas
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

int batch_launch_params(const cht_batch *b, void *stream, LaunchParams &lp, int &T,
                        uint64_t &chunks) {
    lp.cta = b->launch.cta_threads ? b->launch.cta_threads : 256;
    lp.items = b->launch.items_per_thread ? b->launch.items_per_thread : 1;
    lp.max_ctas = b->launch.max_ctas;
    lp.max_tiles = 0;
    lp.in_flight = 1;
    lp.sms = b->sms;
    lp.stream = static_cast<cudaStream_t>(stream);
    T = b->launch.tile ? b->launch.tile : 4;
    const uint64_t per = (uint64_t)32 * batch_items(lp.items);
    chunks = 0;
    for (const BatchDesc &d : b->host) chunks += (d.n + per - 1) / per;
    return CHT_OK;
}

void drop_graph(cht_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

int check_batch_launch(const cht_config &l) {
    if (l.tile != 0 && l.tile != 4 && l.tile != 8 && l.tile != 16)
        return fail(CHT_ERR_INVALID, "tile must be 4, 8 or 16 (got %d)", l.tile);
    if (l.items_per_thread < 0 || l.items_per_thread > 8)
        return fail(CHT_ERR_INVALID, "items_per_thread must be 1..8");
    if (l.cta_threads != 0 && (l.cta_threads < 32 || l.cta_threads > 256 || l.cta_threads % 32))
        return fail(CHT_ERR_INVALID, "cta_threads must be a multiple of 32 in [32, 256]");
    if (l.max_ctas < 0) return fail(CHT_ERR_INVALID, "max_ctas must be >= 0");
    return CHT_OK;
}

}  // namespace

extern "C" {

size_t cht_batch_scratch_bytes(int count) {
    if (count < 1 || count > 16384) return 0;
    return (size_t)count * sizeof(BatchDesc);
}

int cht_batch_create(cht_table *const *tables, const void *const *d_keys, const size_t *n,
                     uint8_t *const *d_status, int count, int op, void *d_scratch,
                     size_t scratch_bytes, void *stream, cht_batch **out) {
    if (!out) return fail(CHT_ERR_INVALID, "null output handle pointer");
    *out = nullptr;
    if (!tables || !d_keys || !n || !d_status)
        return fail(CHT_ERR_INVALID, "null batch array");
    if (count < 1 || count > 16384) return fail(CHT_ERR_INVALID, "count must be 1..16384");
    if (op != CHT_OP_FIND_OR_PUT && op != CHT_OP_FIND)
        return fail(CHT_ERR_INVALID, "op must be CHT_OP_FIND_OR_PUT or CHT_OP_FIND");
    if (!d_scratch || (uintptr_t)d_scratch % 16)
        return fail(CHT_ERR_INVALID, "scratch must be a 16-byte aligned device pointer");
    if (scratch_bytes < cht_batch_scratch_bytes(count))
        return fail(CHT_ERR_CAPACITY, "scratch of %zu bytes is below the %zu needed",
                    scratch_bytes, cht_batch_scratch_bytes(count));
    cht_batch *b = new cht_batch();
    b->count = count;
    b->op = op;
    b->dev = static_cast<BatchDesc *>(d_scratch);
    b->graph = nullptr;
    b->exec = nullptr;
    memset(&b->launch, 0, sizeof b->launch);
    b->host.resize(count);
    for (int i = 0; i < count; ++i) {
        const cht_table *t = tables[i];
        if (!t) {
            delete b;
            return fail(CHT_ERR_INVALID, "null table at batch entry %d", i);
        }
        if (t->cfg.kind != CHT_ICEBERG) {
            delete b;
            return fail(CHT_ERR_UNSUPPORTED, "batch entry %d is not an iceberg table", i);
        }
        if (t->cfg.bucket_words != kWordsPerBucket) {
            delete b;
            return fail(CHT_ERR_UNSUPPORTED, "batch entry %d has %d-word buckets (fused batches "
                        "need 16)", i, t->cfg.bucket_words);
        }
        if (i == 0) {
            b->fpw0 = t->cfg.fields_per_word;
            b->device = t->device;
            b->sms = t->sms;
        } else if (t->cfg.fields_per_word != b->fpw0 || t->device != b->device) {
            delete b;
            return fail(CHT_ERR_UNSUPPORTED,
                        "batch entry %d differs in primary packing or device from entry 0", i);
        }
        if (n[i] && (!d_keys[i] || !d_status[i])) {
            delete b;
            return fail(CHT_ERR_INVALID, "null keys or statuses at batch entry %d", i);
        }
        if ((uintptr_t)d_keys[i] % t->cfg.key_bytes) {
            delete b;
            return fail(CHT_ERR_INVALID, "keys of batch entry %d not aligned", i);
        }
        b->host[i].ta = t->args;
        b->host[i].ta.max_tiles = 0;
        b->host[i].ta.ctr = nullptr;
        b->host[i].keys = d_keys[i];
        b->host[i].n = n[i];
        b->host[i].status = d_status[i];
    }
    if (op == CHT_OP_FIND_OR_PUT) {
        // concurrent writes from two entries of one table would race
        std::vector<const cht_table *> seen(tables, tables + count);
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
            delete b;
            return fail(CHT_ERR_INVALID, "a find-or-put batch lists a table twice");
        }
    }
    // descriptors travel as kernel parameters (kDescPerLaunch per launch): the
    // upload is asynchronous and leaves no host buffer to keep alive
    cudaError_t ce = cudaSuccess;
    for (int i0 = 0; i0 < count && ce == cudaSuccess; i0 += kDescPerLaunch) {
        const int m = std::min(kDescPerLaunch, count - i0);
        DescBlock blk;
        memcpy(blk.d, b->host.data() + i0, sizeof(BatchDesc) * m);
        k_write_desc<<<1, 128, 0, static_cast<cudaStream_t>(stream)>>>(b->dev + i0, blk, m);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        delete b;
        return cuda_fail(ce, "uploading batch descriptors");
    }
    *out = b;
    return ok();
}

int cht_batch_set_launch(cht_batch *b, const cht_config *launch) {
    if (!b || !launch) return fail(CHT_ERR_INVALID, "null argument");
    int e = check_batch_launch(*launch);
    if (e) return e;
    b->launch = *launch;
    drop_graph(b);
    return ok();
}

int cht_batch_launch(const cht_batch *b, void *stream) {
    if (!b) return fail(CHT_ERR_INVALID, "null batch");
    LaunchParams lp;
    int T;
    uint64_t chunks;
    batch_launch_params(b, stream, lp, T, chunks);
    if (chunks == 0) return ok();
    cudaError_t ce = launch_iceberg_batch(T, b->fpw0, b->op == CHT_OP_FIND, lp, b->dev, b->count,
                                          chunks, nullptr);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "batch kernel launch");
}

int cht_batch_capture(cht_batch *b, void *stream) {
    if (!b) return fail(CHT_ERR_INVALID, "null batch");
    drop_graph(b);
    cudaStream_t cs;
    cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(ce, "creating the capture stream");
    // order the capture after the caller's earlier work (descriptor upload)
    ce = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(ce, "beginning the capture");
    }
    int e = cht_batch_launch(b, cs);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "ending the capture");
    cudaGraphExec_t x = nullptr;
    ce = cudaGraphInstantiate(&x, g, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ce, "instantiating the graph");
    }
    b->graph = g;
    b->exec = x;
    return ok();
}

int cht_batch_replay(const cht_batch *b, void *stream) {
    if (!b) return fail(CHT_ERR_INVALID, "null batch");
    if (!b->exec) return fail(CHT_ERR_INVALID, "batch has no captured graph");
    cudaError_t ce = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "graph launch");
}

int cht_batch_clear(const cht_batch *b, void *stream) {
    if (!b) return fail(CHT_ERR_INVALID, "null batch");
    k_clear_batch<<<b->sms * 4, 256, 0, static_cast<cudaStream_t>(stream)>>>(b->dev, b->count);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "batch clear launch");
}

int cht_batch_destroy(cht_batch *b) {
    if (b) drop_graph(b);
    delete b;
    return ok();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free fused find-or-put: the batch descriptors live in a fixed
// array of this library instead of caller scratch (the paper has no
// counterpart; see the declaration in cht.h for who needs it).
// ---------------------------------------------------------------------------
namespace {

// the descriptor layout the documented limit is stated in (256 x 240 bytes)
static_assert(sizeof(BatchDesc) == 240, "batch descriptor size changed: update cht.h");

// room for CHT_STATIC_BATCH_MAX descriptors; held by every GPU that loads the
// library until the process exits
static __device__ __align__(256) unsigned char
    g_static_batch[CHT_STATIC_BATCH_MAX * sizeof(BatchDesc)];

// Driver calls that identify the current context, looked up through the
// runtime so that the library needs no link-time dependency on the driver.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
struct StaticAddr {
    unsigned long long ctx;  // id of the context the address belongs to (0: none)
    void *addr;
};
StaticAddr g_static_addr[kMaxDevices];

// id of the current context, or 0 if there is none or it cannot be read
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0)
        return 0;
    return id;
}

// The array's device address on device dev (current). It is looked up with
// cudaGetSymbolAddress on the first call on the device and again whenever the
// device's context has changed since (after cudaDeviceReset the module is
// loaded anew and the array may move); otherwise the cached address is used.
int static_batch_address(int dev, void **out) {
    std::lock_guard<std::mutex> g(g_static_mu);
    const unsigned long long ctx = current_context_id();
    StaticAddr &c = g_static_addr[dev];
    if (!c.addr || ctx == 0 || c.ctx != ctx) {
        void *p = nullptr;
        cudaError_t ce = cudaGetSymbolAddress(&p, g_static_batch);
        if (ce != cudaSuccess) return cuda_fail(ce, "looking up the static batch array");
        c.addr = p;
        // the lookup made the primary context current if it was not yet
        c.ctx = ctx ? ctx : current_context_id();
    }
    *out = c.addr;
    return CHT_OK;
}

}  // namespace

extern "C" int cht_batch_find_or_put_static(cht_table *const *tables, const void *const *d_keys,
                                            const size_t *n, uint8_t *const *d_status, int count,
                                            void *stream) {
    if (!tables || !d_keys || !n || !d_status) return fail(CHT_ERR_INVALID, "null batch array");
    if (count < 1 || count > CHT_STATIC_BATCH_MAX)
        return fail(CHT_ERR_INVALID,
                    "count = %d: the allocation-free batch takes 1..%d tables (its fixed array "
                    "holds %d descriptors)",
                    count, CHT_STATIC_BATCH_MAX, CHT_STATIC_BATCH_MAX);
    int cur = -1;
    cudaError_t ce = cudaGetDevice(&cur);
    if (ce != cudaSuccess) return cuda_fail(ce, "device query");
    if (cur < 0 || cur >= kMaxDevices) return fail(CHT_ERR_UNSUPPORTED, "device id %d", cur);
    int fpw0 = 0, sms = 0;
    uint64_t total_chunks = 0;
    const uint64_t per = (uint64_t)32 * kStaticBatchItems;
    for (int i = 0; i < count; ++i) {
        const cht_table *t = tables[i];
        if (!t) return fail(CHT_ERR_INVALID, "null table at batch entry %d", i);
        if (t->cfg.kind != CHT_ICEBERG)
            return fail(CHT_ERR_UNSUPPORTED, "batch entry %d is not an iceberg table", i);
        if (t->cfg.bucket_words != kWordsPerBucket)
            return fail(CHT_ERR_UNSUPPORTED, "batch entry %d has %d-word buckets (fused batches "
                        "need 16)", i, t->cfg.bucket_words);
        if (t->device != cur)
            return fail(CHT_ERR_INVALID, "batch entry %d is not on the current device", i);
        if (i == 0) {
            fpw0 = t->cfg.fields_per_word;
            sms = t->sms;
        } else if (t->cfg.fields_per_word != fpw0) {
            return fail(CHT_ERR_UNSUPPORTED, "batch entry %d differs in primary packing", i);
        }
        if (n[i] && (!d_keys[i] || !d_status[i]))
            return fail(CHT_ERR_INVALID, "null keys or statuses at batch entry %d", i);
        if ((uintptr_t)d_keys[i] % t->cfg.key_bytes)
            return fail(CHT_ERR_INVALID, "keys of batch entry %d not aligned", i);
        total_chunks += (n[i] + per - 1) / per;
    }
    {
        // a table listed twice would have its writes race (as in
        // cht_batch_create); the check sorts a copy on the stack
        const cht_table *seen[CHT_STATIC_BATCH_MAX];
        std::copy(tables, tables + count, seen);
        std::sort(seen, seen + count);
        if (std::adjacent_find(seen, seen + count) != seen + count)
            return fail(CHT_ERR_INVALID, "a find-or-put batch lists a table twice");
    }
    void *dst = nullptr;
    int e = static_batch_address(cur, &dst);
    if (e) return e;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchDesc *dev_desc = static_cast<BatchDesc *>(dst);
    // descriptors travel as kernel parameters, kDescPerLaunch per launch (a
    // block of 64 x 240 bytes = 15 KiB on the stack), as in cht_batch_create:
    // the upload is an ordinary asynchronous launch on stream
    for (int i0 = 0; i0 < count; i0 += kDescPerLaunch) {
        const int m = std::min(kDescPerLaunch, count - i0);
        DescBlock blk;
        for (int i = 0; i < m; ++i) {
            const cht_table *t = tables[i0 + i];
            BatchDesc &d = blk.d[i];
            d.ta = t->args;
            d.ta.max_tiles = 0;
            d.ta.ctr = nullptr;
            d.keys = d_keys[i0 + i];
            d.n = n[i0 + i];
            d.status = d_status[i0 + i];
        }
        k_write_desc<<<1, 128, 0, s>>>(dev_desc + i0, blk, m);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return cuda_fail(ce, "writing the static batch descriptors");
    }
    if (total_chunks == 0) return ok();
    ce = launch_iceberg_batch_noalloc(fpw0, s, sms, dev_desc, count, total_chunks);
    return ce == cudaSuccess ? ok() : cuda_fail(ce, "static batch kernel launch");
}
