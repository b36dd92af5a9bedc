/*
 * dim3.h -- C ABI of the GB300 (sm_103a) DIM^3 Join-Project library.
 *
 * The library computes the Join-Project of Eq. 1 (Section 1),
 *     Pi_{x,z}( R(x,y) join_y S(z,y) ),
 * and the Join-Aggregate COUNT of Section 4.1, on one GPU, with every step
 * of Algorithm 1 (mapping, CSR construction, intersection-free partitioning,
 * SparseBMM, DenseEC, union of the disjoint results) in CUDA kernels.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Tables are int32 column pairs in DEVICE memory: R is (r_key = y,
 *   r_val = x), S is (s_key = y, s_val = z), each of n rows. Rows may repeat
 *   and come in any order: tables are sets (duplicates collapse).
 * - Output pairs are the original int32 values, distinct, in canonical order:
 *   x ascending, then z ascending, comparing signed 32-bit integers.
 * - The caller owns every input and output buffer. The library owns its
 *   context, its plans and the scratch memory they allocate (stream-ordered
 *   cudaMallocAsync on the call's stream).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Work is enqueued on it. Calls that return sizes in host memory
 *   (counts, distinct counts, plan info) synchronise that stream before they
 *   return.
 * - Every call returns a dim3_status. No C++ exception crosses the ABI.
 *   On failure dim3_last_error() returns a message for the calling thread.
 * - Sizes are int64. Null pointers with a nonzero size, or negative sizes,
 *   give DIM3_ERR_ARG. n = 0 is legal and yields an empty result.
 * - A context is bound to one device and may be used by one host thread at
 *   a time. It owns a second stream on which independent partition steps
 *   (the z mapping, the (y, z) pair sort) run beside the caller's stream;
 *   the caller's stream is made to wait for them before the call returns or
 *   enqueues anything that reads their results.
 * - Bounded device waits (decoupled look-back of sorts and of the one-pass
 *   compaction, tensor-core pipeline barriers) give up after 2 s; the call
 *   that observes it returns DIM3_ERR_TIMEOUT.
 * - Self-joins: when R and S are passed as the same column pointers, the
 *   values are mapped once (the x map serves as the z map). Results equal
 *   those of separate copies of the same tables.
 */
#ifndef DIM3_H
#define DIM3_H

#include <stdint.h>

#if defined(__GNUC__)
#define DIM3_API __attribute__((visibility("default")))
#else
#define DIM3_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DIM3_OK = 0,
    DIM3_ERR_ARG = -1,         /* bad argument (null pointer, negative size, bad range) */
    DIM3_ERR_CUDA = -2,        /* a CUDA runtime/driver call failed */
    DIM3_ERR_NOMEM = -3,       /* device allocation failed */
    DIM3_ERR_CAPACITY = -4,    /* output capacity smaller than the result; count is set */
    DIM3_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    DIM3_ERR_OVERFLOW = -6,    /* a size exceeds what the library supports */
    DIM3_ERR_UNSUPPORTED = -7  /* option or device not supported */
} dim3_status;

typedef struct dim3_ctx dim3_ctx;
typedef struct dim3_plan dim3_plan;
typedef struct dim3_cache dim3_cache;

/* Sizes of a partitioned input, returned by dim3_partition (host struct). */
typedef struct {
    int64_t n_r;          /* input R rows */
    int64_t n_s;          /* input S rows */
    int64_t n_r_kept;     /* distinct R tuples whose y occurs in S.y (Section 2.2, Opt. 2) */
    int64_t n_s_distinct; /* distinct S tuples */
    int64_t n_x;          /* |X|: distinct x of the kept R tuples */
    int64_t n_y;          /* |Y|: distinct S.y */
    int64_t n_z;          /* |Z|: distinct S.z */
    int64_t n_z_dense;    /* |Z_d|: z columns judged dense (Section 2.3) */
    int64_t n_y_dense;    /* distinct y of the dense S tuples (K of the DenseEC contraction) */
    int64_t n_s_sparse;   /* S tuples in S_sparse */
    int64_t n_y_bitmap;   /* S_sparse rows held as z-bitmaps (SparseBMM's wide rows) */
    int64_t out_j;        /* |OUT_J| = sum over y of deg_R(y) * deg_S(y) (cached z excluded) */
    int64_t n_z_cached;   /* z served from a partial result cache (Section 3), else 0 */
    int32_t theta_z;      /* degree threshold used: z dense iff m_z >= theta_z */
    int32_t dense_variant;/* DenseEC variant that will run (dim3_dense_variant) */
} dim3_plan_info;

/* One instance of a batch: device columns as for dim3_join_project. */
typedef struct {
    const int32_t *r_key, *r_val; /* R(x, y): key = y, value = x */
    int64_t nr;
    const int32_t *s_key, *s_val; /* S(z, y): key = y, value = z */
    int64_t ns;
} dim3_instance;

/* One relation R_i(x_i, x_{i+1}) of a multi-way join (device int32 columns). */
typedef struct {
    const int32_t *d_a;  /* x_i */
    const int32_t *d_b;  /* x_{i+1} */
    int64_t n;
} dim3_edge_table;

/* DenseEC bitmap-intersection variants (Algorithm 3; the choice is the role
 * of f3 in Section 2.6). All give identical results. */
typedef enum {
    DIM3_DENSE_AUTO = 0,   /* tuned choice */
    DIM3_DENSE_TC = 1,     /* 0/1 tile product on tcgen05 tensor cores, then > 0 */
    DIM3_DENSE_POPC = 2,   /* bit-packed AND + popc on CUDA cores */
    DIM3_DENSE_PROBE = 3   /* per x, probe each y of R[x] in S_dense (non-SIMD method) */
} dim3_dense_variant;

/* Join-Aggregate (Section 4.1): the aggregate and the function f(R.v, S.u). */
typedef enum {
    DIM3_AGG_COUNT = 0,  /* join tuples of the group (int64) */
    DIM3_AGG_SUM = 1,    /* sum of f (int64, wrapping modulo 2^64) */
    DIM3_AGG_MIN = 2,    /* int64 */
    DIM3_AGG_MAX = 3,    /* int64 */
    DIM3_AGG_AVG = 4     /* (double)SUM / (double)COUNT */
} dim3_agg;
typedef enum {
    DIM3_FN_MUL = 0,     /* v * u (int64) */
    DIM3_FN_ADD = 1,     /* v + u */
    DIM3_FN_LEFT = 2,    /* v */
    DIM3_FN_RIGHT = 3    /* u */
} dim3_agg_fn;

/* Context options (dim3_ctx_set_option). */
typedef enum {
    DIM3_OPT_THETA_Z = 1,       /* z dense iff m_z >= value; <0: tuned (default) */
    DIM3_OPT_DENSE_VARIANT = 2, /* a dim3_dense_variant (default AUTO) */
    DIM3_OPT_BITMAP_ROW_MIN = 3,/* S_sparse rows with at least this many z are held as bitmaps; <0: |Z|/32 */
    DIM3_OPT_LIGHT_ROW_MAX = 4, /* x rows with at most this many join tuples dedup in shared memory by sort; <0: default */
    DIM3_OPT_TIMING = 5,        /* nonzero: record CUDA events around each phase (dim3_ctx_timing) */
    DIM3_OPT_EMIT_ROWS = 6,     /* x rows per CTA in the emitting SparseBMM pass: 1, 2, 4; 0: automatic */
    DIM3_OPT_TWO_PASS = 7,      /* nonzero: always count before emitting (no single-pass look-back, no
                                   staged z values: the emitting pass rebuilds the bitmaps) */
    DIM3_OPT_ID_CHUNK_MAX = 8,  /* emitting pass: a 4096-z chunk of one x row holding at most this many
                                   pairs is written through staged z ids, a denser one group by group;
                                   0: always group by group; <0: default (512); at most 1024 */
    DIM3_OPT_PATH = 9,          /* dim3_join_project / dim3_join_count: 0 (default) f1 of Section 2.6
                                   chooses, 1 the hybrid DIM^3 path, 2 the classical solution */
    DIM3_OPT_TILE_WORDS = 10,   /* 32-bit words per z tile, 1024..12288, of the bitmap over z ranges wider
                                   than 393,216 z and of Join-Count's packed counters; 0 (default): the
                                   fewest tiles of at most 12,288 (bitmap) / 7,168 (counters) words */
    DIM3_OPT_DENSE_TILE_N = 11, /* tensor-core DenseEC: dense z per CTA tile, 128 or 256; 0 (default): 256 */
    DIM3_OPT_EMIT_PIPELINE = 12 /* single-pass emission with two x rows per CTA: 1 = persistent CTAs that
                                   build the next row group while the previous one's offset resolves;
                                   0 (default) = one group per CTA */
} dim3_option;

/* Phases timed under DIM3_OPT_TIMING. */
typedef enum {
    DIM3_PHASE_MAP = 0,          /* dim3_map */
    DIM3_PHASE_PARTITION = 1,    /* mapping + CSR + split of dim3_partition / dim3_join_* */
    DIM3_PHASE_DENSE_EC = 2,     /* DenseEC kernels */
    DIM3_PHASE_SPARSE_COUNT = 3, /* SparseBMM + union, counting pass */
    DIM3_PHASE_SPARSE_EMIT = 4,  /* SparseBMM + union + compaction, emitting pass */
    DIM3_PHASE_DENSE_TC = 5      /* the tcgen05 DenseEC kernel alone (inside DIM3_PHASE_DENSE_EC) */
} dim3_phase;

/* Library version as major*10000 + minor*100 + patch (library plumbing; no
 * passage of the paper). */
DIM3_API int dim3_version(void);

/* Message of the last failed call on this host thread ("" if none). */
DIM3_API const char *dim3_last_error(void);

/* Create a context on CUDA device `device`. *out receives the handle.
 * Contexts, options, timing and errors are library plumbing: the paper's
 * Algorithm 1 defines the steps they drive, not these calls. */
DIM3_API int dim3_ctx_create(dim3_ctx **out, int device);

/* Destroy a context. Plans made with it must be destroyed first. */
DIM3_API int dim3_ctx_destroy(dim3_ctx *ctx);

/*
 * dim3_selftest_wait_timeout -- failure detection without a GPU fault: one
 * warp runs the decoupled look-back of the one-pass compaction against a
 * predecessor that never publishes, with a limit of `seconds` (0 < seconds
 * <= 2). Returns DIM3_ERR_TIMEOUT when the wait gave up and reported it (the
 * expected outcome; the context stays usable), DIM3_ERR_CUDA if it did not.
 * Synchronises the stream. Library plumbing, not a step of the paper.
 */
DIM3_API int dim3_selftest_wait_timeout(dim3_ctx *ctx, double seconds, void *stream);

/* Set a dim3_option. Returns DIM3_ERR_ARG for an unknown option. */
DIM3_API int dim3_ctx_set_option(dim3_ctx *ctx, int option, int64_t value);

/* Accumulated device time (CUDA events on the launching stream) and number of
 * timed intervals of a dim3_phase since the last reset, while DIM3_OPT_TIMING
 * is on. Waits for the recorded events. reset != 0 clears all phases after
 * reading. Not a paper operation: instrumentation for roofline measurement. */
DIM3_API int dim3_ctx_timing(dim3_ctx *ctx, int phase, double *total_ms, int64_t *launches, int reset);

/* Number of CUDA kernels this library has launched in this process. */
DIM3_API int dim3_launch_count(int64_t *out);

/*
 * Strategy selection f1 (Section 2.6): a one-call join under DIM3_OPT_PATH 0
 * maps y first, counts |OUT_J| of the input bags from the y ids (S rows per
 * y, summed over R's rows) and evaluates
 *   f1 = 2 (|R| + |S|) t_map + |OUT_J| t_randRW - |OUT_J| t_hash;
 * f1 > 0 stops the mapping and runs the classical solution (hash join +
 * dedup; here a sort-based join and a radix-sort dedup), else the hybrid path
 * continues with the y ids already made. The constants
 * are seconds per input row (mapping), per join tuple in SparseBMM and per
 * join tuple in the classical path; the defaults were measured on GB300.
 * dim3_ctx_last_path returns the path of the context's last one-call join
 * (1 hybrid, 2 classical, 0 none yet).
 */
DIM3_API int dim3_ctx_set_f1_costs(dim3_ctx *ctx, double t_map, double t_rand, double t_hash);
DIM3_API int dim3_ctx_last_path(const dim3_ctx *ctx);

/*
 * dim3_map -- order-preserving mapping of one column to dense ids.
 * Section 2.2 maps every distinct value of a column to a natural number; this
 * library gives each value its rank among the column's distinct values, so id
 * order is value order (the reason canonical output order needs no sort).
 *   d_vals     [n] int32 device, the column.
 *   d_ids      [n] int32 device, out: d_ids[i] = #distinct values < d_vals[i].
 *   d_dict     [n] int32 device, out: the first *n_distinct entries are the
 *              distinct values ascending (d_dict[d_ids[i]] == d_vals[i]).
 *   n_distinct host, out.
 * Synchronises the stream.
 */
DIM3_API int dim3_map(dim3_ctx *ctx, const int32_t *d_vals, int64_t n, int32_t *d_ids,
             int32_t *d_dict, int64_t *n_distinct, void *stream);

/*
 * dim3_map_noalloc -- dim3_map for callers that may not allocate device
 * memory (a host engine that fixed its GPU memory budget at start-up and
 * forbids later allocations, code living under another framework's allocator,
 * or latency-critical code that must not enter the allocator). It returns the
 * same rank ids and dictionary as dim3_map. This allocation-free entry point
 * is an interface variant: the paper has no counterpart.
 *   d_vals, d_ids, d_dict, n_distinct: as for dim3_map; n <= 65536.
 * No context. Runs on the current device and stream. All scratch lives in one
 * fixed 2,883,840-byte device array inside the library (held by every GPU
 * that loads it until the process exits); the calls themselves allocate and
 * free nothing. With lazy module loading (the CUDA default) the library's
 * module, and with it that array, is placed on a device by the first call
 * there, which can fail for lack of memory: an engine with a fixed budget
 * should make one call per device at start-up. That first call also looks up
 * the array's device address, so it should come before any stream capture.
 * The address is kept per device index for the life of the process: after
 * cudaDeviceReset the cached address is stale, so do not use this entry
 * point on a device that was reset. Every call reuses the same array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. n > 65536 gives DIM3_ERR_OVERFLOW.
 * Synchronises the stream.
 */
DIM3_API int dim3_map_noalloc(const int32_t *d_vals, int64_t n, int32_t *d_ids, int32_t *d_dict,
                              int64_t *n_distinct, void *stream);

/*
 * dim3_partition -- Algorithm 1 up to the compute steps: map y from S.y and
 * drop R tuples whose y is not in S.y (Section 2.2, Opt. 2); map x and z;
 * build R_CSR by x (Section 2.5); split S by z into S_sparse (CSR by y) and
 * S_dense (bitmaps / 0-1 tiles) so that the two results are disjoint
 * (Section 2.3). z is dense iff m_z >= theta_z (theta_z < 0: the context's
 * option, else tuned).
 *   *plan_out  receives a plan that owns the device-resident tables.
 *   info       host, out (may be NULL).
 * Inputs may be freed or reused once the call returns. Synchronises the stream.
 */
DIM3_API int dim3_partition(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                   const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns,
                   int32_t theta_z, dim3_plan **plan_out, dim3_plan_info *info, void *stream);

/*
 * dim3_partition_ids -- dim3_partition for columns that already hold natural
 * numbers, with the mapping step skipped (Section 2.2, Optimization 1: auto-
 * increment keys, dictionary-encoded strings, or ids from dim3_map_tuples).
 *   d_r_y, d_r_x [nr] int32 device: R's y and x ids; d_s_y, d_s_z [ns]: S's.
 *   n_x, n_y, n_z: the id ranges; every id must be < its range.
 * A negative id removes its tuple from the input (e.g. an R tuple whose y is
 * missing from S's dictionary). Ids are used as they are: the plan's x and z
 * dictionaries are the identity, so the emitted pairs are ids, in id order
 * (canonical order), and the bitmaps span the declared ranges, however few
 * ids occur. R tuples whose y no S tuple holds stay in R_CSR with an empty S
 * row (the semi-join of Optimization 2 belongs to the caller's mapping).
 * An id >= its range gives DIM3_ERR_ARG and no plan; ranges above 2^31 - 1
 * too. Synchronises the stream.
 */
DIM3_API int dim3_partition_ids(dim3_ctx *ctx, const int32_t *d_r_y, const int32_t *d_r_x, int64_t nr,
                                const int32_t *d_s_y, const int32_t *d_s_z, int64_t ns, int64_t n_x,
                                int64_t n_y, int64_t n_z, int32_t theta_z, dim3_plan **plan_out,
                                dim3_plan_info *info, void *stream);

/*
 * dim3_map_tuples -- mapping of several attributes together (Section 2.2,
 * "Supporting Wider Range of Join-Project Operations"): Pi_{a,b,c,d,e}(R(a,b,
 * c,d) join_{c,d} S(c,d,e,f)) runs as Pi_{x,z}(R(x,y) join_y S(z,y)) with
 * x = (a,b), y = (c,d), z = (c,d,e). Rows of k int32 columns (1 <= k <= 8) are
 * numbered by the rank of their tuple among the distinct tuples in
 * lexicographic order (column 0 most significant).
 *   d_cols        host array of k device pointers, each [n] int32.
 *   unsigned_mask bit c set: column c compares as unsigned 32-bit, else as
 *                 signed (an int64 key is (high word signed, low word unsigned)).
 *   d_ids         [n] int32 device, out: the tuple rank of each row.
 *   d_first       [n] int32 device, out: the first *n_distinct entries give,
 *                 per id, the smallest row holding that tuple (gather the
 *                 columns there to translate ids back, e.g. dim3_gather_i32).
 *   n_distinct    host, out.
 * Ids from one call over R's and S's join columns together share a numbering,
 * ready for dim3_partition_ids. n < 2^31. Synchronises the stream.
 */
DIM3_API int dim3_map_tuples(dim3_ctx *ctx, const int32_t *const *d_cols, int k, uint32_t unsigned_mask,
                             int64_t n, int32_t *d_ids, int32_t *d_first, int64_t *n_distinct, void *stream);

/*
 * dim3_gather_i32 -- d_dst[i] = d_src[d_idx[i]] for i < n (int32 device
 * arrays; d_src has n_src entries). Translates ids back to attribute values
 * through dim3_map_tuples' d_first (the inverse of the multi-attribute
 * mapping of Section 2.2). An index outside [0, n_src) gives
 * DIM3_ERR_ARG, with d_dst[i] = -1 there. Synchronises the stream.
 */
DIM3_API int dim3_gather_i32(dim3_ctx *ctx, const int32_t *d_src, int64_t n_src, const int32_t *d_idx, int64_t n,
                             int32_t *d_dst, void *stream);

/*
 * Partial result caching (Section 3). A cache holds, for a set Z_cached of z
 * values, the x of their results (x, z): per z either the x themselves or,
 * when they are more than half of X, the complement in X. A plan built with a
 * cache omits the S tuples of cached z from S_sparse and S_dense and adds the
 * cached results in the union step, so its results are those of the plain
 * plan. The cache stays valid while the tables do not change (the caller
 * rebuilds it otherwise, as the section prescribes).
 */
typedef struct {
    int64_t n_entries;  /* cached z */
    int64_t n_list;     /* stored x values over all entries */
    int64_t space;      /* sum of space(z) = 2 + min(k, |X| - k) over the entries */
    int64_t n_x;        /* |X| of the tables */
} dim3_cache_info;

/*
 * dim3_cache_build -- score every z and cache the best within a budget.
 *   tables        as for dim3_partition (device int32 columns).
 *   theta_z       the threshold the queries will use (z dense iff m_z >=
 *                 theta_z; < 0: the context's option), which decides cost(z).
 *   budget        cache space in entries (Section 3's units: an entry costs
 *                 2 + min(k, |X| - k), k = the z's result size).
 *   t_sparse      cost of one join tuple in SparseBMM (seconds or any unit);
 *   t_dense       cost of one (x, z) evaluation in DenseEC (same unit).
 *                 cost(z) = n_join(z) * t_sparse for a sparse z, n_join(z) =
 *                 sum over S(z) of deg_R(y); |X| * t_dense for a dense z.
 *                 Measured on GB300: about 1.2e-12 s and 1.1e-11 s.
 * CacheScore(z) = cost(z) / space(z) in double precision; z are taken by
 * descending score (ties: ascending z) while the running space fits budget.
 *   *cache_out    receives a device-resident cache; info (may be NULL) its sizes.
 * Negative budget or cost constants: DIM3_ERR_ARG. Synchronises the stream.
 */
DIM3_API int dim3_cache_build(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                              const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns, int32_t theta_z,
                              int64_t budget, double t_sparse, double t_dense, dim3_cache **cache_out,
                              dim3_cache_info *info, void *stream);

/*
 * dim3_cache_export -- copy a cache's entries (Section 3: per cached z, its
 * x list or the complement of it in X) to device buffers sized from its info: d_z [n_entries] int32 (ascending z values), d_size [n_entries]
 * int64 (k, or k - |X| for a complement entry), d_complement [n_entries]
 * uint8 (1 = complement; also marks k = |X|, whose size is 0), d_offsets
 * [n_entries + 1] int64, d_xs [n_list] int32 (entry e's x values, ascending,
 * at d_offsets[e] .. d_offsets[e + 1]). Any pointer may be NULL to skip it.
 */
DIM3_API int dim3_cache_export(dim3_ctx *ctx, const dim3_cache *cache, int32_t *d_z, int64_t *d_size,
                               uint8_t *d_complement, int64_t *d_offsets, int32_t *d_xs, void *stream);

/* Free a cache's device memory (Section 3's cache; stream-ordered). */
DIM3_API int dim3_cache_destroy(dim3_cache *cache);

/*
 * dim3_partition_cached -- dim3_partition with a cache built on the same
 * tables (Section 3: cached z are left out of S_sparse and S_dense and their
 * stored results are output in addition): the dictionaries are those of the full tables, the S tuples of
 * cached z are dropped after mapping, and the plan's Join-Project results
 * include the cached pairs (info.n_z_cached = entries). Join-Count on such a
 * plan gives DIM3_ERR_UNSUPPORTED (the cache holds pairs, not counts). A
 * cache whose values do not occur in the tables, or whose |X| differs, gives
 * DIM3_ERR_ARG. Synchronises the stream.
 */
DIM3_API int dim3_partition_cached(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                                   const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns,
                                   const dim3_cache *cache, int32_t theta_z, dim3_plan **plan_out,
                                   dim3_plan_info *info, void *stream);

/*
 * dim3_join_aggregate -- Join-Aggregate with group-by attributes from both
 * tables (Section 4.1): G_{x,z} agg(f(R.v, S.u)) over R(x, y, v) join_y
 * S(z, y, u). R and S are bags of rows (every pair of rows with equal y is a
 * join tuple, duplicates included, as in SQL).
 *   d_r_key, d_r_val, d_r_v [nr] int32 device: R's y, x and v columns.
 *   d_s_key, d_s_val, d_s_u [ns] int32 device: S's y, z and u columns.
 *   agg, fn    a dim3_agg and a dim3_agg_fn (fn is ignored for COUNT).
 *   d_out_x, d_out_z [capacity] int32 device, out: the groups (x, z) with at
 *              least one join tuple, canonical order (the Join-Project pairs).
 *   d_out_val  [capacity] device, out: int64 per group, or double for AVG.
 *   count      host, out: number of groups; always set.
 * capacity < count: DIM3_ERR_CAPACITY, nothing written (capacity 0 sizes).
 * Unknown agg or fn: DIM3_ERR_ARG. Synchronises the stream.
 */
DIM3_API int dim3_join_aggregate(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, const int32_t *d_r_v,
                                 int64_t nr, const int32_t *d_s_key, const int32_t *d_s_val, const int32_t *d_s_u,
                                 int64_t ns, int agg, int fn, int32_t *d_out_x, int32_t *d_out_z, void *d_out_val,
                                 int64_t capacity, int64_t *count, void *stream);

/*
 * dim3_groupby_aggregate -- Join-Aggregate with the group-by attribute from
 * one table (Section 4.1): G_x agg(z) over R(x, y) join_y S(z, y), computed by
 * the section's rewrite: per-y aggregates of S first (count, sum, min, max of
 * its z values), then one fold per x over R's rows. Bags as above (COUNT
 * counts join tuples). To group by z instead, swap the tables.
 *   d_out_x    [capacity] int32 device, out: every x with a join tuple, ascending.
 *   d_out_val  [capacity] device, out: int64, or double for AVG.
 *   count      host, out. Capacity protocol and errors as dim3_join_aggregate.
 */
DIM3_API int dim3_groupby_aggregate(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                                    const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns, int agg,
                                    int32_t *d_out_x, void *d_out_val, int64_t capacity, int64_t *count,
                                    void *stream);

/*
 * Multi-way joins with projection, MJP (Section 4.2): the line query
 *   Pi_{x_1, x_{k+1}}(R_1(x_1, x_2) join R_2(x_2, x_3) join ... join R_k(x_k, x_{k+1}))
 * over a left-deep plan, relations as sets.
 *
 * dim3_mjp_sizes -- |OUT_J_i| (join paths through R_1 .. R_i) and |OUT_P_i|
 * (distinct (x_1, x_{i+1})) for i = 1..k, exact (path counts in double,
 * exact below 2^53); out_j, out_p host arrays of k entries.
 *
 * dim3_mjp_plan -- the dynamic programme of Section 4.2 on the sizes:
 *   DP_1 = 0, DP_i = min_{j<i} DP_j + sum_{h=j+1}^{i-1} JoinCost_h + JPCost_i,
 * input sizes after a deduplication at j scaled by |OUT_P_j| / |OUT_J_j|; with
 *   JoinCost(l, r, out)  = c[0] (l + r) + c[1] out             (bag join)
 *   JPCost(l, r, oj, op) = c[2] (l + r) + c[3] oj + c[4] op    (Join-Project).
 * Ties take the smaller j. dedup[i] = 1 when a deduplication follows the
 * join with table i (0-based; dedup[0] = 0, dedup[k-1] = 1); *cost = DP_k.
 * Host only (no context, no device work).
 *
 * dim3_mjp_execute -- run a placement: joins flagged in dedup are Join-
 * Projects of this library, the others bag joins (every running pair joins).
 * The result pairs (x_1, x_{k+1}) in canonical order go to d_out_x, d_out_z;
 * capacity protocol as dim3_join_project. dedup[k-1] must be 1.
 */
DIM3_API int dim3_mjp_sizes(dim3_ctx *ctx, int k, const dim3_edge_table *tables, double *out_j, double *out_p,
                            void *stream);
DIM3_API int dim3_mjp_plan(int k, const double *r_size, const double *out_j, const double *out_p,
                           const double *c, int *dedup, double *cost);
DIM3_API int dim3_mjp_execute(dim3_ctx *ctx, int k, const dim3_edge_table *tables, const int *dedup,
                              int32_t *d_out_x, int32_t *d_out_z, int64_t capacity, int64_t *count, void *stream);

/* Copy of the plan's sizes: |X|, |Y|, |Z|, |Z_dense|, |OUT_J| and the other
 * quantities of Algorithm 1's partition steps (Sections 2.2-2.4). */
DIM3_API int dim3_plan_get_info(const dim3_plan *plan, dim3_plan_info *info);

/*
 * dim3_plan_row_counts -- per-x output sizes for the x-id range
 * [x_begin, x_end): d_counts[i] = |{z : (x_begin + i, z) in result}|
 * (int64 device, x_end - x_begin entries): the per-x popcounts of the union
 * of Algorithm 1's sparse and dense results. Useful to size x-range chunks.
 */
DIM3_API int dim3_plan_row_counts(dim3_ctx *ctx, dim3_plan *plan, int64_t x_begin, int64_t x_end,
                         int64_t *d_counts, void *stream);

/*
 * dim3_plan_join_project -- SparseBMM (Algorithm 2) and DenseEC (Algorithm 3)
 * over the x-id range [x_begin, x_end) of a plan, and their union
 * (Algorithm 1, last step: disjoint, so no dedup), compacted into
 *   d_out_x, d_out_z  [capacity] int32 device, out: pairs of the range in
 *                     canonical order (x ids are rank-ordered, so ranges
 *                     concatenate into the full canonical result).
 *   count             host, out: pairs of the range; always set.
 * If capacity < count, DIM3_ERR_CAPACITY is returned and the contents of the
 * output buffers are unspecified (a single-pass emission may have written a
 * prefix). capacity = 0 (or null buffers) only sizes the range: it runs a
 * counting pass that the plan keeps, so the next call for the same range
 * emits without counting again. Memory: on a single instance whose z range
 * spans several shared-memory tiles, or whose light rows are sorted, that
 * counting pass also keeps every row's z values for the emitting pass (a
 * staging buffer of 4 bytes per min(join tuples of the row, |Z|) entry,
 * taken only when it fits a quarter of the free device memory, else the
 * emitting pass recomputes), released with the plan or by the next range's
 * count; dim3_plan_row_counts never stages.
 * x_begin = 0, x_end = n_x covers everything. Synchronises the stream.
 */
DIM3_API int dim3_plan_join_project(dim3_ctx *ctx, dim3_plan *plan, int64_t x_begin, int64_t x_end,
                           int32_t *d_out_x, int32_t *d_out_z, int64_t capacity,
                           int64_t *count, void *stream);

/*
 * dim3_plan_join_count -- as dim3_plan_join_project, plus
 *   d_out_cnt [capacity] int32 device, out: COUNT(x,z) = number of distinct y
 *             joining x and z (Join-Aggregate, Section 4.1, with COUNT).
 */
DIM3_API int dim3_plan_join_count(dim3_ctx *ctx, dim3_plan *plan, int64_t x_begin, int64_t x_end,
                         int32_t *d_out_x, int32_t *d_out_z, int32_t *d_out_cnt,
                         int64_t capacity, int64_t *count, void *stream);

/*
 * Batches of independent instances (Eq. 1 for each), run through one pass
 * of the path: the columns are gathered with an instance tag, mapping ranks
 * (instance, value) pairs, so each instance owns a contiguous block of ids and
 * no join crosses instances; SparseBMM works in each x's own z window and
 * DenseEC computes only the block diagonal. Not a paper operation as such:
 * the data-parallel outer x loop of Section 6 (OpenMP) extended across
 * instances.
 *
 * dim3_batch_partition -- as dim3_partition for n_inst instances (host array
 *   of dim3_instance with device columns). The plan's x ids list instance 0's
 *   x first, then instance 1's, ...; info holds the batch totals.
 * dim3_plan_instance_ranges -- x_lo[t] .. x_lo[t+1] (host, n_inst + 1 entries)
 *   is instance t's x-id range, for x-range calls on a batch plan.
 * dim3_batch_join_project / dim3_batch_join_count -- the whole path for a
 *   batch: pairs of instance 0 in canonical order, then instance 1's, ...;
 *   inst_counts (host, n_inst entries, may be NULL) receives each instance's
 *   number of pairs, count their sum. Capacity protocol as dim3_join_project.
 * All synchronise the stream.
 */
DIM3_API int dim3_batch_partition(dim3_ctx *ctx, int n_inst, const dim3_instance *inst, int32_t theta_z,
                                  dim3_plan **plan_out, dim3_plan_info *info, void *stream);
DIM3_API int dim3_plan_instance_ranges(const dim3_plan *plan, int64_t *x_lo);
DIM3_API int dim3_batch_join_project(dim3_ctx *ctx, int n_inst, const dim3_instance *inst, int32_t *d_out_x,
                                     int32_t *d_out_z, int64_t capacity, int64_t *inst_counts, int64_t *count,
                                     void *stream);
DIM3_API int dim3_batch_join_count(dim3_ctx *ctx, int n_inst, const dim3_instance *inst, int32_t *d_out_x,
                                   int32_t *d_out_z, int32_t *d_out_cnt, int64_t capacity, int64_t *inst_counts,
                                   int64_t *count, void *stream);

/* Tables a plan can export (dim3_plan_export), for inspection and tests. */
typedef enum {
    DIM3_TABLE_DICT_X = 1,    /* int32 [n_x]   distinct x ascending */
    DIM3_TABLE_DICT_Y = 2,    /* int32 [n_y]   distinct S.y ascending */
    DIM3_TABLE_DICT_Z = 3,    /* int32 [n_z]   distinct S.z ascending */
    DIM3_TABLE_R_ROWPTR = 4,  /* int64 [n_x+1] R_CSR row pointers */
    DIM3_TABLE_R_COL = 5,     /* int32 [n_r_kept] R_CSR y ids, ascending per row */
    DIM3_TABLE_M_Z = 6,       /* int32 [n_z]   m_z */
    DIM3_TABLE_DENSE_Z = 7,   /* uint8 [n_z]   1 if z is dense */
    DIM3_TABLE_SS_ROWPTR = 8, /* int64 [n_y+1] S_sparse row pointers by y id */
    DIM3_TABLE_SS_COL = 9,    /* int32 [n_s_sparse] S_sparse z ids, ascending per row */
    DIM3_TABLE_DEG_S = 10,    /* int32 [n_y]   deg_S(y) */
    DIM3_TABLE_OUTJ_X = 11    /* int64 [n_x]   join tuples per x: sum over y in R[x] of deg_S(y) */
} dim3_table;

/* Copy table `which` (a structure of Algorithm 1: dictionaries, R_CSR,
 * S_sparse, degrees, the dense split) into d_dst (device), which holds
 * `bytes` bytes. */
DIM3_API int dim3_plan_export(dim3_plan *plan, int which, void *d_dst, int64_t bytes, void *stream);

/* Free a plan's device tables (stream-ordered on the plan's stream; library
 * plumbing). */
DIM3_API int dim3_plan_destroy(dim3_plan *plan);

/*
 * dim3_join_project -- the whole hot path of Eq. 1 in one call: partition,
 * SparseBMM + DenseEC, union, compaction.
 *   d_out_x, d_out_z [capacity] int32 device, out.
 *   count            host, out: |OUT_P|; always set, also on DIM3_ERR_CAPACITY
 *                    (then the buffers' contents are unspecified).
 * Synchronises the stream.
 */
DIM3_API int dim3_join_project(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                      const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns,
                      int32_t *d_out_x, int32_t *d_out_z, int64_t capacity, int64_t *count,
                      void *stream);

/*
 * dim3_join_count -- Join-Aggregate COUNT (Section 4.1): as dim3_join_project
 * plus d_out_cnt [capacity] int32 device, COUNT(x,z) for every output pair.
 */
DIM3_API int dim3_join_count(dim3_ctx *ctx, const int32_t *d_r_key, const int32_t *d_r_val, int64_t nr,
                    const int32_t *d_s_key, const int32_t *d_s_val, int64_t ns,
                    int32_t *d_out_x, int32_t *d_out_z, int32_t *d_out_cnt, int64_t capacity,
                    int64_t *count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DIM3_H */
