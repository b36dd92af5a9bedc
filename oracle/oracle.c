/*
 * CPU oracle for the DIM^3 Join-Project hot path. TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. The product path never calls it.
 *
 * It computes, plainly and slowly, what the GPU path computes quickly:
 *
 *   Eq. 1 (Section 1):  Pi_{x,z}( R(x,y) join_y S(z,y) ),
 *   the set { (x,z) : exists y with (x,y) in R and (z,y) in S }, with R and S
 *   taken as sets of tuples, listed in canonical order (x ascending, then z
 *   ascending, both compared as signed 32-bit integers);
 *
 *   Join-Aggregate with COUNT as the aggregate (Section 4.1, group-by
 *   attributes from both tables): for every (x,z) in that set, the number of
 *   distinct y it is joined through.
 *
 * The algorithm is the paper's "classical solution" (Section 1.1): a hash
 * join of R and S on y, then hash-based duplicate elimination of the projected
 * (x,z) tuples, then a sort into canonical order. Input tuples are first
 * de-duplicated (set semantics). While joining it counts the join tuples, so
 * it also reports |OUT_J|.
 *
 * The order-preserving value mapping used by the GPU path is checked against
 * oracle_rank_map(): the id of a value is the number of distinct smaller values
 * in its column (sort, unique, binary search).
 *
 * Shares no code with the CUDA path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- hashing */

static uint64_t mix64(uint64_t v) {
    /* splitmix64 finaliser (Steele, Lea and Flood, 2014) */
    v ^= v >> 30;
    v *= 0xbf58476d1ce4e5b9ULL;
    v ^= v >> 27;
    v *= 0x94d049bb133111ebULL;
    v ^= v >> 31;
    return v;
}

static uint64_t pack(int32_t a, int32_t b) {
    return ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
}

static int64_t pow2_at_least(int64_t n) {
    int64_t c = 16;
    while (c < n) c <<= 1;
    return c;
}

/* Open-addressing hash map from a 64-bit key to a 64-bit value, linear probing.
 * A separate occupancy byte means every key value is usable. */
typedef struct {
    uint64_t *keys;
    int64_t *vals;
    uint8_t *used;
    int64_t cap; /* power of two */
    int64_t size;
} hmap;

static int hmap_init(hmap *h, int64_t expected) {
    h->cap = pow2_at_least(2 * expected + 16);
    h->size = 0;
    h->keys = (uint64_t *)malloc((size_t)h->cap * sizeof(uint64_t));
    h->vals = (int64_t *)malloc((size_t)h->cap * sizeof(int64_t));
    h->used = (uint8_t *)calloc((size_t)h->cap, 1);
    return (h->keys && h->vals && h->used) ? 0 : -1;
}

static void hmap_free(hmap *h) {
    free(h->keys);
    free(h->vals);
    free(h->used);
    h->keys = NULL;
    h->vals = NULL;
    h->used = NULL;
}

static int hmap_grow(hmap *h) {
    hmap n;
    n.cap = h->cap * 2;
    n.size = 0;
    n.keys = (uint64_t *)malloc((size_t)n.cap * sizeof(uint64_t));
    n.vals = (int64_t *)malloc((size_t)n.cap * sizeof(int64_t));
    n.used = (uint8_t *)calloc((size_t)n.cap, 1);
    if (!n.keys || !n.vals || !n.used) {
        hmap_free(&n);
        return -1;
    }
    for (int64_t i = 0; i < h->cap; ++i) {
        if (!h->used[i]) continue;
        int64_t s = (int64_t)(mix64(h->keys[i]) & (uint64_t)(n.cap - 1));
        while (n.used[s]) s = (s + 1) & (n.cap - 1);
        n.used[s] = 1;
        n.keys[s] = h->keys[i];
        n.vals[s] = h->vals[i];
        n.size++;
    }
    hmap_free(h);
    *h = n;
    return 0;
}

/* Returns the slot of key, inserting it with value init if absent.
 * *inserted tells which happened. Returns -1 on allocation failure. */
static int64_t hmap_upsert(hmap *h, uint64_t key, int64_t init, int *inserted) {
    if (2 * (h->size + 1) > h->cap) {
        if (hmap_grow(h) != 0) return -1;
    }
    int64_t s = (int64_t)(mix64(key) & (uint64_t)(h->cap - 1));
    while (h->used[s]) {
        if (h->keys[s] == key) {
            *inserted = 0;
            return s;
        }
        s = (s + 1) & (h->cap - 1);
    }
    h->used[s] = 1;
    h->keys[s] = key;
    h->vals[s] = init;
    h->size++;
    *inserted = 1;
    return s;
}

static int64_t hmap_find(const hmap *h, uint64_t key) {
    int64_t s = (int64_t)(mix64(key) & (uint64_t)(h->cap - 1));
    while (h->used[s]) {
        if (h->keys[s] == key) return s;
        s = (s + 1) & (h->cap - 1);
    }
    return -1;
}

/* ------------------------------------------------------------- results */

typedef struct {
    int64_t n;      /* |OUT_P| */
    int64_t out_j;  /* |OUT_J|: join tuples enumerated (after input dedup) */
    int32_t *x;
    int32_t *z;
    int64_t *cnt;
} oracle_result;

static int cmp_u64(const void *a, const void *b) {
    uint64_t u = *(const uint64_t *)a, v = *(const uint64_t *)b;
    return (u > v) - (u < v);
}

/* Order-preserving code of a signed pair: flipping the sign bits makes the
 * unsigned order of the packed word equal to the signed (x, z) order. */
static uint64_t order_code(uint64_t packed_xz) {
    return packed_xz ^ 0x8000000080000000ULL;
}

/*
 * The classical solution. x_filter (sorted or not, may be NULL) restricts R to
 * the tuples whose x is in the filter set: the result is then exactly the rows
 * of the full result with those x (used to check large inputs row by row).
 */
oracle_result *oracle_join(const int32_t *r_key, const int32_t *r_val, int64_t nr,
                           const int32_t *s_key, const int32_t *s_val, int64_t ns,
                           const int32_t *x_filter, int64_t n_filter) {
    oracle_result *res = (oracle_result *)calloc(1, sizeof(oracle_result));
    if (!res) return NULL;
    hmap xf = {0}, sdedup = {0}, rdedup = {0}, ybucket = {0}, outset = {0};
    int64_t *next = NULL, *head = NULL;
    uint64_t *codes = NULL;
    int ins;
    int ok = 0;

    if (x_filter) {
        if (hmap_init(&xf, n_filter) != 0) goto done;
        for (int64_t i = 0; i < n_filter; ++i)
            if (hmap_upsert(&xf, (uint64_t)(uint32_t)x_filter[i], 0, &ins) < 0) goto done;
    }

    /* Build side: S, de-duplicated, chained by y. ybucket maps y -> bucket id;
     * head[bucket] is the first S tuple of the bucket, next[] links the rest. */
    if (hmap_init(&sdedup, ns) != 0 || hmap_init(&ybucket, ns) != 0) goto done;
    next = (int64_t *)malloc((size_t)(ns + 1) * sizeof(int64_t));
    head = (int64_t *)malloc((size_t)(ns + 1) * sizeof(int64_t));
    if (!next || !head) goto done;
    int64_t nbuckets = 0;
    for (int64_t j = 0; j < ns; ++j) {
        if (hmap_upsert(&sdedup, pack(s_val[j], s_key[j]), 0, &ins) < 0) goto done;
        if (!ins) continue; /* duplicate S tuple */
        int64_t s = hmap_upsert(&ybucket, (uint64_t)(uint32_t)s_key[j], nbuckets, &ins);
        if (s < 0) goto done;
        if (ins) head[nbuckets++] = -1;
        int64_t b = ybucket.vals[s];
        next[j] = head[b];
        head[b] = j;
    }

    /* Probe side: R, de-duplicated; every join tuple (x,y,z) projects to
     * (x,z), which goes into the output hash map (value = its count). */
    if (hmap_init(&rdedup, nr) != 0 || hmap_init(&outset, 1024) != 0) goto done;
    for (int64_t i = 0; i < nr; ++i) {
        if (x_filter && hmap_find(&xf, (uint64_t)(uint32_t)r_val[i]) < 0) continue;
        if (hmap_upsert(&rdedup, pack(r_val[i], r_key[i]), 0, &ins) < 0) goto done;
        if (!ins) continue; /* duplicate R tuple */
        int64_t s = hmap_find(&ybucket, (uint64_t)(uint32_t)r_key[i]);
        if (s < 0) continue; /* no S tuple with this y */
        for (int64_t j = head[ybucket.vals[s]]; j >= 0; j = next[j]) {
            res->out_j++;
            int64_t o = hmap_upsert(&outset, pack(r_val[i], s_val[j]), 0, &ins);
            if (o < 0) goto done;
            outset.vals[o] += 1;
        }
    }

    /* Sort the distinct (x,z) into canonical order. */
    res->n = outset.size;
    codes = (uint64_t *)malloc((size_t)(res->n + 1) * sizeof(uint64_t));
    res->x = (int32_t *)malloc((size_t)(res->n + 1) * sizeof(int32_t));
    res->z = (int32_t *)malloc((size_t)(res->n + 1) * sizeof(int32_t));
    res->cnt = (int64_t *)malloc((size_t)(res->n + 1) * sizeof(int64_t));
    if (!codes || !res->x || !res->z || !res->cnt) goto done;
    int64_t k = 0;
    for (int64_t s = 0; s < outset.cap; ++s)
        if (outset.used[s]) codes[k++] = order_code(outset.keys[s]);
    qsort(codes, (size_t)res->n, sizeof(uint64_t), cmp_u64);
    for (int64_t t = 0; t < res->n; ++t) {
        uint64_t packed = order_code(codes[t]);
        res->x[t] = (int32_t)(uint32_t)(packed >> 32);
        res->z[t] = (int32_t)(uint32_t)(packed & 0xFFFFFFFFULL);
        res->cnt[t] = outset.vals[hmap_find(&outset, packed)];
    }
    ok = 1;

done:
    hmap_free(&xf);
    hmap_free(&sdedup);
    hmap_free(&rdedup);
    hmap_free(&ybucket);
    hmap_free(&outset);
    free(next);
    free(head);
    free(codes);
    if (!ok) {
        free(res->x);
        free(res->z);
        free(res->cnt);
        free(res);
        return NULL;
    }
    return res;
}

int64_t oracle_result_size(const oracle_result *r) { return r->n; }
int64_t oracle_result_out_j(const oracle_result *r) { return r->out_j; }

void oracle_result_copy(const oracle_result *r, int32_t *x, int32_t *z, int64_t *cnt) {
    if (x) memcpy(x, r->x, (size_t)r->n * sizeof(int32_t));
    if (z) memcpy(z, r->z, (size_t)r->n * sizeof(int32_t));
    if (cnt) memcpy(cnt, r->cnt, (size_t)r->n * sizeof(int64_t));
}

void oracle_result_free(oracle_result *r) {
    if (!r) return;
    free(r->x);
    free(r->z);
    free(r->cnt);
    free(r);
}

/* ------------------------------------------------------------- mapping */

static int cmp_i32(const void *a, const void *b) {
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    return (u > v) - (u < v);
}

/*
 * Order-preserving mapping of a column to consecutive natural numbers
 * (Section 2.2 maps every distinct value to a natural number; the rank order
 * is this library's reading of which number). ids[i] = number of distinct
 * values smaller than vals[i]; dict[0..d) = the distinct values ascending.
 * Returns d, or -1 on allocation failure.
 */
int64_t oracle_rank_map(const int32_t *vals, int64_t n, int32_t *ids, int32_t *dict) {
    int32_t *sorted = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!sorted) return -1;
    memcpy(sorted, vals, (size_t)n * sizeof(int32_t));
    qsort(sorted, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t d = 0;
    for (int64_t i = 0; i < n; ++i)
        if (i == 0 || sorted[i] != sorted[i - 1]) sorted[d++] = sorted[i];
    for (int64_t i = 0; i < n; ++i) {
        int64_t lo = 0, hi = d; /* first index with sorted[idx] >= vals[i] */
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (sorted[mid] < vals[i]) lo = mid + 1; else hi = mid;
        }
        ids[i] = (int32_t)lo;
    }
    if (dict) memcpy(dict, sorted, (size_t)d * sizeof(int32_t));
    free(sorted);
    return d;
}
