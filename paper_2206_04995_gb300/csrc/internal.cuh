// Internal plan structures and step launchers.
#pragma once

#include "common.cuh"

namespace dimcube {

// ----------------------------------------------------------------- mapping
// An order-preserving map of one column's values to dense ids (ranks among
// the distinct values). The hash table stays alive so other columns can be
// probed against it (semi-join of Section 2.2, Optimization 2).
struct ValueMap {
    DevBuf table;  // uint64 slots: 0 = empty, else (1 << 32) | uint32(value)
    DevBuf rank;   // uint32 per slot: rank of the slot's value
    DevBuf count;  // int64: the distinct count on the device
    uint32_t mask = 0;
    int64_t n_distinct = 0;  // -1 until read (resolve_counts)
};

// Map vals[0..n) (rows with pred[i] < 0 are skipped and get id -1).
// ids_out [n]; dict_out [n] capacity, first n_distinct ascending.
void build_value_map(const int32_t* vals, const int32_t* pred, int64_t n, ValueMap& vm,
                     int32_t* ids_out, int32_t* dict_out, cudaStream_t s);
// Batched form: row i belongs to instance tags[i] (0 <= tag < n_tags); ids
// rank the (instance, value) pairs; dict_tag_out[id] = the id's instance.
// With read_count false the distinct count is left on the device
// (n_distinct = -1) for resolve_counts.
void build_value_map(const int32_t* vals, const int32_t* tags, int n_tags, const int32_t* pred, int64_t n,
                     ValueMap& vm, int32_t* ids_out, int32_t* dict_out, int32_t* dict_tag_out, cudaStream_t s,
                     bool read_count = true);
// Reads the unresolved distinct counts of maps[0..n_maps) and, if extra is not
// null, *extra into *extra_out, with one synchronisation.
int64_t resolve_counts(ValueMap* const* maps, int n_maps, const int64_t* extra, int64_t* extra_out, cudaStream_t s);
// ids_out[i] = id of (tags[i], vals[i]) in vm (tags may be null), or -1 if absent.
void probe_value_map(const ValueMap& vm, const int32_t* vals, const int32_t* tags, int64_t n, int32_t* ids_out,
                     cudaStream_t s);

// Partial result cache (Section 3): entries for the cached z values
// (ascending), each holding the x of that z's results, or, when they are more
// than half of X, the complement in X. Values, not ids, so that a plan built
// later on the same tables can attach it. Device resident.
struct ResultCache {
    int64_t n_x = 0;     // |X| of the tables it was built on
    int64_t n_c = 0;     // entries
    int64_t n_list = 0;  // stored x values over all entries
    int64_t space = 0;   // sum of 2 + min(k, |X| - k) over the entries
    DevBuf z;            // int32 [n_c]: cached z values, ascending
    DevBuf size;         // int64 [n_c]: k, or k - |X| for a complement entry
    DevBuf comp;         // uint8 [n_c]: 1 = complement entry
    DevBuf off;          // int64 [n_c + 1]: entry e's x values are xs[off[e], off[e + 1])
    DevBuf xs;           // int32 [n_list]: x values, ascending within an entry
};

// Input of the plan builder: one instance (tags null, n_inst 1) or a batch of
// n_inst instances concatenated, row i of R belonging to instance r_tag[i].
struct PlanInput {
    const int32_t *r_key = nullptr, *r_val = nullptr, *r_tag = nullptr;
    int64_t nr = 0;
    const int32_t *s_key = nullptr, *s_val = nullptr, *s_tag = nullptr;
    int64_t ns = 0;
    int n_inst = 1;
    // Section 2.2, Optimization 1: the columns already hold natural numbers
    // (x ids < n_x, y ids < n_y, z ids < n_z; a negative id drops its tuple)
    // and the mapping step is skipped
    bool premapped = false;
    int64_t n_x = 0, n_y = 0, n_z = 0;
    // Section 3: omit the cache's z from S_sparse and S_dense and add the
    // cached results in the union step (single instance, mapped columns)
    const ResultCache* cache = nullptr;
};

// -------------------------------------------------------------------- plan
// f1 constants measured on GB300 (seconds)
constexpr double kF1TMap = 4.0e-10;
constexpr double kF1TRand = 1.0e-12;
constexpr double kF1THash = 2.0e-11;

struct Options {
    int64_t theta_z = -1;
    int64_t dense_variant = DIM3_DENSE_AUTO;
    int64_t bitmap_row_min = -1;
    int64_t light_row_max = -1;
    int64_t emit_rows = 0;  // x rows per CTA in the emitting pass (0: automatic)
    int64_t two_pass = 0;   // nonzero: always a counting pass before the emitting pass
    int64_t id_chunk_max = -1;  // pairs per 4096-z chunk written through staged ids (<0: 512)
    int64_t path = 0;           // one-call joins: 0 f1 decides, 1 hybrid, 2 classical
    int64_t tile_words = 0;     // z-tiled rows: bitmap words per tile (0: automatic)
    int64_t dense_tile_n = 0;   // tensor-core DenseEC: dense z per CTA tile (128 or 256; 0: 256)
    int64_t emit_pipe = 0;      // single pass, two rows per CTA: persistent pipelined kernel (1) or not (0)
    // f1 constants (Section 2.6), seconds: t_map per input row, t_randRW per
    // join tuple of the hybrid path, t_hash per join tuple of the classical path
    double f1c[3] = {kF1TMap, kF1TRand, kF1THash};
};

struct Plan {
    dim3_plan_info info{};
    cudaStream_t stream = nullptr;
    int device = 0;
    Options opt;
    // mapping
    DevBuf dict_x, dict_y, dict_z;  // int32
    // R_CSR by x id
    DevBuf r_rowptr;  // int64 [n_x + 1]
    DevBuf r_col;     // int32 [n_r_kept], y ids ascending per row
    DevBuf outj_x;    // int64 [n_x], join tuples per x
    // degrees
    DevBuf m_z;       // int32 [n_z]
    DevBuf deg_s;     // int32 [n_y]
    DevBuf dense_z;   // uint8 [n_z]
    // S_sparse CSR by y id
    DevBuf ss_rowptr;   // int64 [n_y + 1]
    DevBuf ss_col;      // int32 [n_s_sparse], z ids ascending per row
    DevBuf bm_row_of_y; // int32 [n_y], bitmap row or -1
    DevBuf bm_off;      // int64 [n_y_bitmap + 1]: first word of each bitmap row in ss_bits
    DevBuf ss_bits;     // uint32, bitmap row b covers the z window of its instance
    int64_t zw = 0;     // words of the widest z window
    // batches: per-instance ranges (n_inst + 1 entries) and the instance of each x
    int n_inst = 1;
    DevBuf x_tag;       // int32 [n_x] (batches only)
    DevBuf y_tag;       // int32 [n_y] (batches only)
    // z-tiled SparseBMM: start of every tile in each S_sparse row, per pass kind
    DevBuf tile_ptr[2];
    int64_t tile_ptr_bits[2] = {0, 0}, tile_cols[2] = {0, 0};
    DevBuf inst_x_lo;   // int64 [n_inst + 1]: x ids of instance i are [lo[i], lo[i+1])
    DevBuf inst_z_lo;   // int64 [n_inst + 1]: z ids
    DevBuf inst_zd_lo;  // int64 [n_inst + 1]: dense z indices
    std::vector<int64_t> h_inst_x_lo, h_inst_z_lo, h_inst_zd_lo;
    // S_dense
    DevBuf zd_list;     // int32 [n_zd]: dense index -> z id (ascending)
    DevBuf kidx_of_y;   // int32 [n_y]: y id -> K index or -1
    DevBuf b_tc;        // uint8 [n_zd_pad][k_pad]: e4m3 0/1, K-major (tensor-core operand)
    DevBuf b_bits;      // uint32 [n_zd][kw]: Bitmap_z over K (AND+popc operand)
    DevBuf sdt_bits;    // uint32 [n_yd][zdw_op]: S_dense rows by y over dense index (probe operand)
    int64_t k_pad = 0, kw = 0, n_zd_pad = 0;
    int64_t zdw_op = 0;  // words of the dense z index in the operands
    // Dense-result rows [rows][zdw]: the dense z index [0, n_z_dense) and, for
    // a plan with a partial result cache, the cached z at [zc_off, zc_off +
    // n_zc) (zc_off = n_zd_pad, a whole number of words); zd_list maps every
    // index to its z id. n_zd_total = zc_off + n_zc (= n_z_dense uncached).
    int64_t zdw = 0, n_zd_total = 0;
    int64_t n_zc = 0, zc_off = 0, zc_nlist = 0;
    DevBuf zc_zid;      // int32 [n_zc]: z id of every cache entry
    DevBuf zc_cmask;    // uint32 [ceil(n_zc / 32)]: complement entries' bits
    DevBuf zc_comp;     // uint8 [n_zc]
    DevBuf zc_xid;      // int32 [zc_nlist]: x ids of the entries' lists
    DevBuf zc_ent;      // int32 [zc_nlist]: entry of each list element
    // light rows (few join tuples on a wide z range): dedup by sorting their
    // z ids instead of a |Z|-bit SPA; light_n < 0: not decided yet
    DevBuf light;        // uint8 [n_x]
    int64_t light_n = -1;
    // cached row offsets of the last counting pass
    int64_t cache_begin = -1, cache_end = -1;
    int cache_kind = -1;
    DevBuf cache_off;  // int64 [rows + 1]
    DevBuf cache_dbits; // dense bits of the cached range
    DevBuf cache_dcnt;  // dense counts of the cached range
    // z-tiled single instance (or light rows beside bitmap rows): the rows the
    // cached range sweeps over the z tiles
    DevBuf cache_units;     // int32 [cache_n_list]: rows run over the z tiles (null: every row)
    int64_t cache_n_list = 0, cache_tile_bits = 0;
    // z-tiled single instance, counted for an emitting call: every row's z
    // values, deduplicated and ascending, at cache_slot[r] of cache_vals (a
    // slot of min(|OUT_J| of the row, |Z|) entries rounded up to a multiple
    // of four); the emitting pass then only places them (null: not staged)
    DevBuf cache_vals;      // int32 [cache_slot[rows]]
    DevBuf cache_slot;      // int64 [rows + 1]
    int64_t max_mx = -1;  // largest |R[x]| (the bound of a pair's count), -1 until computed
};

// Per-phase CUDA-event timing (DIM3_OPT_TIMING). Events are recorded on the
// launching stream around a phase and resolved when the caller asks.
enum Phase { PH_MAP = 0, PH_PARTITION = 1, PH_DENSE = 2, PH_COUNT = 3, PH_EMIT = 4, PH_DENSE_TC = 5, PH_N = 6 };
struct Stats {
    bool on = false;
    double ms[PH_N] = {};
    int64_t n[PH_N] = {};
    struct Pending {
        int ph;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    void resolve();
    void reset();
};
struct PhaseScope {
    Stats* st = nullptr;
    int ph = 0;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseScope(Stats* stats, int phase, cudaStream_t stream);
    ~PhaseScope();
};

struct Ctx {
    Stats* stats = nullptr;  // owned by the ABI context
    // second stream for independent steps (the z map runs beside the y and x
    // maps), with the events that fork work onto it and join it back
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int sm_count = 152;
    int smem_optin = 227 * 1024;
    int cc_major = 0, cc_minor = 0;
    Options opt;
};

// Bounded-wait self-test (selftest.cu): 1 if a look-back whose predecessor
// never publishes gave up after `seconds` and reported it, else 0.
int wait_selftest(double seconds, cudaStream_t s);

// prefer_classical non-null (a single instance of value columns): after the
// y mapping, evaluate f1 (Section 2.6); when it favours the classical
// solution, set *prefer_classical and return nullptr without finishing.
Plan* build_plan(const Ctx& ctx, const PlanInput& in, int64_t theta_z, cudaStream_t s,
                 bool* prefer_classical = nullptr);

// Output of a join over an x-id range: counts pass + scan + emit pass.
// kind 0 = project, 1 = count. Returns the number of pairs; writes only when
// capacity >= pairs (else throws DIM3_ERR_CAPACITY after setting *count).
int64_t plan_join(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int kind, int32_t* out_x,
                  int32_t* out_z, int32_t* out_cnt, int64_t capacity, int64_t* count, cudaStream_t s);
void plan_row_counts(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int64_t* d_counts,
                     cudaStream_t s);

// DenseEC over rows [x_begin, x_begin + rows): dense result bits [rows][zdw]
// (kind 0) or dense counts [rows][n_zd] int32 (kind 1).
void dense_ec(const Ctx& ctx, const Plan& p, int64_t x_begin, int64_t rows, int kind, uint32_t* d_bits,
              int32_t* d_cnt, cudaStream_t s);
void dense_build_operands(const Ctx& ctx, Plan& p, const uint64_t* s_keys_u64, const uint32_t* s_keys_u32,
                          int64_t n_s, int bz, const int32_t* zd_index, cudaStream_t s);

// Batches (batch.cu): plan over n_inst instances; per-instance pair counts
// after a join over all x of that plan.
Plan* build_batch_plan(const Ctx& ctx, int n_inst, const dim3_instance* inst, int64_t theta_z, cudaStream_t s);
void batch_instance_counts(const Plan& p, int64_t* host_counts, cudaStream_t s);

// Multi-attribute mapping (tuples.cu): ranks of k-column tuples in
// lexicographic order (column c unsigned when bit c of unsigned_mask is set),
// first row of every distinct tuple; returns the number of distinct tuples.
constexpr int kMaxTupleCols = 8;
int64_t map_tuples(const int32_t* const* cols, int k, uint32_t unsigned_mask, int64_t n, int32_t* ids, int32_t* first,
                   cudaStream_t s);
// dst[i] = src[idx[i]]; false (dst[i] = -1 there) when an index is outside [0, n_src).
bool gather_i32(const int32_t* src, int64_t n_src, const int32_t* idx, int64_t n, int32_t* dst, cudaStream_t s);

// Partial result caching (cache.cu): statistics of the tables, CacheScore
// selection under a budget (space units), entries; attach to a plan being
// built; expand into dense-result rows [rows][zdw].
ResultCache* build_result_cache(const Ctx& ctx, const PlanInput& in, int64_t theta_z, int64_t budget,
                                double t_sparse, double t_dense, cudaStream_t s);
void attach_cache_ids(Plan& p, const ResultCache& c, int32_t* sz_id, int64_t ns, cudaStream_t s);
void finish_cache_index(Plan& p, cudaStream_t s);
void cache_expand(const Plan& p, int64_t x_begin, int64_t rows, uint32_t* d_bits, cudaStream_t s);

// Join-Aggregate (aggregate.cu), Section 4.1: G_{x,z} agg(f(R.v, S.u)) and
// the one-table G_x agg(z). out_val is int64 (COUNT, SUM, MIN, MAX) or
// double (AVG). *count = the number of groups (also returned); a smaller
// capacity throws DIM3_ERR_CAPACITY with nothing written.
int64_t join_aggregate(const Ctx& ctx, const PlanInput& in, const int32_t* r_v, const int32_t* s_u, int agg, int fn,
                       int32_t* out_x, int32_t* out_z, void* out_val, int64_t capacity, int64_t* count,
                       cudaStream_t s);
int64_t groupby_aggregate(const Ctx& ctx, const PlanInput& in, int agg, int32_t* out_x, void* out_val,
                          int64_t capacity, int64_t* count, cudaStream_t s);

// The classical solution (classical.cu): distinct tuples sorted by y, join by
// binary search, dedup by radix sort (kind 0 project, 1 count); f1 of Section
// 2.6 (> 0: classical).
int64_t classical_join(const Ctx& ctx, const PlanInput& in, int kind, int32_t* out_x, int32_t* out_z,
                       int32_t* out_cnt, int64_t capacity, int64_t* count, cudaStream_t s);
double f1_value(int64_t nr, int64_t ns, int64_t out_j, const double* c);
// the bag join (R's rows all kept, S distinct, results not deduplicated) into
// buffers it allocates; returns the number of pairs
int64_t bag_join_into(const Ctx& ctx, const PlanInput& in, DevBuf& out_x, DevBuf& out_z, cudaStream_t s);
// the distinct (a, b) pairs of two columns, canonical order
int64_t distinct_pairs(const int32_t* a, const int32_t* b, int64_t n, int32_t* out_a, int32_t* out_b,
                       int64_t capacity, int64_t* count, cudaStream_t s);

// Multi-way joins with projection (mjp.cu), Section 4.2: the deduplication-
// placement DP (host), exact chain sizes, and the execution of a placement.
double mjp_dp(int k, const double* r_size, const double* out_j, const double* out_p, const double* c, int* dedup);
void mjp_sizes(const Ctx& ctx, int k, const dim3_edge_table* t, double* out_j, double* out_p, cudaStream_t s);
int64_t mjp_execute(const Ctx& ctx, int k, const dim3_edge_table* t, const int* dedup, int32_t* out_x,
                    int32_t* out_z, int64_t capacity, int64_t* count, cudaStream_t s);

// Value mapping with all scratch in a fixed device array (noalloc.cu).
void map_noalloc(const int32_t* d_vals, int64_t n, int32_t* d_ids, int32_t* d_dict, int64_t* n_distinct,
                 cudaStream_t s);

}  // namespace dimcube
