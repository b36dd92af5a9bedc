// The C ABI (include/dim3.h): argument checks, device selection, error
// reporting, and the order of the steps of Algorithm 1.
#include <atomic>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "internal.cuh"

struct dim3_ctx {
    dimcube::Ctx c;
    dimcube::Stats stats;
    int last_path = 0;  // path of the last one-call join: 1 hybrid, 2 classical
    ~dim3_ctx() {
        stats.resolve();
        if (c.aux) cudaStreamDestroy(c.aux);
        if (c.ev_fork) cudaEventDestroy(c.ev_fork);
        if (c.ev_join) cudaEventDestroy(c.ev_join);
    }
};

namespace dimcube {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void Stats::resolve() {
    for (auto& e : pending) {
        float ms_f = 0.f;
        if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms_f, e.a, e.b) == cudaSuccess) {
            ms[e.ph] += ms_f;
            n[e.ph] += 1;
        }
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    pending.clear();
}

void Stats::reset() {
    resolve();
    for (int i = 0; i < PH_N; ++i) {
        ms[i] = 0.0;
        n[i] = 0;
    }
}

PhaseScope::PhaseScope(Stats* stats, int phase, cudaStream_t stream)
    : st(stats && stats->on ? stats : nullptr), ph(phase), s(stream) {
    if (!st) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
}

PhaseScope::~PhaseScope() {
    if (!st) return;
    if (cudaEventRecord(b, s) == cudaSuccess) {
        st->pending.push_back({ph, a, b});
    } else {
        cudaGetLastError();
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
}

}  // namespace dimcube
struct dim3_plan {
    std::unique_ptr<dimcube::Plan> p;
};

struct dim3_cache {
    std::unique_ptr<dimcube::ResultCache> c;
};

namespace {

thread_local std::string g_last_error;

template <class F>
int guarded(F&& f) {
    try {
        f();
        dimcube::raise_if_wait_fault();
        g_last_error.clear();
        return DIM3_OK;
    } catch (const dimcube::Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return DIM3_ERR_NOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return DIM3_ERR_CUDA;
    } catch (...) {
        g_last_error = "unknown error";
        return DIM3_ERR_CUDA;
    }
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        DIM3_CUDA(cudaGetDevice(&prev));
        if (prev != dev) DIM3_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void check_table(const int32_t* k, const int32_t* v, int64_t n, const char* name) {
    DIM3_REQUIRE(n >= 0, DIM3_ERR_ARG, std::string(name) + ": negative row count");
    DIM3_REQUIRE(n == 0 || (k && v), DIM3_ERR_ARG, std::string(name) + ": null column pointer");
    DIM3_REQUIRE(n < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, std::string(name) + ": more than 2^31 - 1 rows");
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

dimcube::PlanInput single_input(const int32_t* rk, const int32_t* rv, int64_t nr, const int32_t* sk, const int32_t* sv,
                                int64_t ns) {
    dimcube::PlanInput in;
    in.r_key = rk;
    in.r_val = rv;
    in.nr = nr;
    in.s_key = sk;
    in.s_val = sv;
    in.ns = ns;
    in.n_inst = 1;
    return in;
}

}  // namespace

extern "C" {

int dim3_version(void) { return 100; }

const char* dim3_last_error(void) { return g_last_error.c_str(); }

int dim3_ctx_create(dim3_ctx** out, int device) {
    return guarded([&] {
        DIM3_REQUIRE(out != nullptr, DIM3_ERR_ARG, "out is null");
        *out = nullptr;
        int n = 0;
        DIM3_CUDA(cudaGetDeviceCount(&n));
        DIM3_REQUIRE(device >= 0 && device < n, DIM3_ERR_ARG, "no such CUDA device");
        std::unique_ptr<dim3_ctx> c(new dim3_ctx());
        c->c.stats = &c->stats;
        c->c.device = device;
        cudaDeviceProp prop;
        DIM3_CUDA(cudaGetDeviceProperties(&prop, device));
        c->c.sm_count = prop.multiProcessorCount;
        c->c.smem_optin = (int)prop.sharedMemPerBlockOptin;
        c->c.cc_major = prop.major;
        c->c.cc_minor = prop.minor;
        DIM3_REQUIRE(prop.major == 10 && prop.minor == 3, DIM3_ERR_UNSUPPORTED,
                     "this library is built for sm_103a (GB300) only; device is sm_" + std::to_string(prop.major) +
                         std::to_string(prop.minor));
        // keep freed stream-ordered memory in the pool between calls
        DeviceGuard g(device);
        cudaMemPool_t pool;
        DIM3_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        DIM3_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        DIM3_CUDA(cudaStreamCreateWithFlags(&c->c.aux, cudaStreamNonBlocking));
        DIM3_CUDA(cudaEventCreateWithFlags(&c->c.ev_fork, cudaEventDisableTiming));
        DIM3_CUDA(cudaEventCreateWithFlags(&c->c.ev_join, cudaEventDisableTiming));
        *out = c.release();
    });
}

int dim3_selftest_wait_timeout(dim3_ctx* ctx, double seconds, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx, DIM3_ERR_ARG, "ctx is null");
        DeviceGuard g(ctx->c.device);
        const int gave_up = dimcube::wait_selftest(seconds, as_stream(stream));
        DIM3_REQUIRE(gave_up, DIM3_ERR_CUDA, "self-test: the bounded wait did not report giving up");
        throw dimcube::Error(DIM3_ERR_TIMEOUT, "self-test: the bounded wait gave up as intended");
    });
}

int dim3_ctx_destroy(dim3_ctx* ctx) {
    return guarded([&] { delete ctx; });
}

int dim3_ctx_set_option(dim3_ctx* ctx, int option, int64_t value) {
    return guarded([&] {
        DIM3_REQUIRE(ctx, DIM3_ERR_ARG, "ctx is null");
        switch (option) {
            case DIM3_OPT_THETA_Z: ctx->c.opt.theta_z = value; break;
            case DIM3_OPT_DENSE_VARIANT:
                DIM3_REQUIRE(value >= DIM3_DENSE_AUTO && value <= DIM3_DENSE_PROBE, DIM3_ERR_ARG, "bad DenseEC variant");
                ctx->c.opt.dense_variant = value;
                break;
            case DIM3_OPT_BITMAP_ROW_MIN: ctx->c.opt.bitmap_row_min = value; break;
            case DIM3_OPT_LIGHT_ROW_MAX: ctx->c.opt.light_row_max = value; break;
            case DIM3_OPT_TIMING: ctx->stats.on = value != 0; break;
            case DIM3_OPT_TWO_PASS: ctx->c.opt.two_pass = value; break;
            case DIM3_OPT_EMIT_PIPELINE:
                DIM3_REQUIRE(value == 0 || value == 1, DIM3_ERR_ARG, "emit pipeline must be 0 or 1");
                ctx->c.opt.emit_pipe = value;
                break;
            case DIM3_OPT_DENSE_TILE_N:
                DIM3_REQUIRE(value == 0 || value == 128 || value == 256, DIM3_ERR_ARG,
                             "dense tile width must be 0, 128 or 256");
                ctx->c.opt.dense_tile_n = value;
                break;
            case DIM3_OPT_TILE_WORDS:
                DIM3_REQUIRE(value == 0 || (value >= 1024 && value <= 12288), DIM3_ERR_ARG,
                             "tile words must be 0 or in [1024, 12288]");
                ctx->c.opt.tile_words = value;
                break;
            case DIM3_OPT_PATH:
                DIM3_REQUIRE(value >= 0 && value <= 2, DIM3_ERR_ARG, "path must be 0 (f1), 1 (hybrid) or 2 (classical)");
                ctx->c.opt.path = value;
                break;
            case DIM3_OPT_ID_CHUNK_MAX:
                DIM3_REQUIRE(value <= 1024, DIM3_ERR_ARG, "id chunk maximum above 1024");
                ctx->c.opt.id_chunk_max = value;
                break;
            case DIM3_OPT_EMIT_ROWS:
                DIM3_REQUIRE(value == 0 || value == 1 || value == 2 || value == 4, DIM3_ERR_ARG,
                             "emit rows per CTA must be 0 (auto), 1, 2 or 4");
                ctx->c.opt.emit_rows = value;
                break;
            default: throw dimcube::Error(DIM3_ERR_ARG, "unknown option " + std::to_string(option));
        }
    });
}

int dim3_ctx_set_f1_costs(dim3_ctx* ctx, double t_map, double t_rand, double t_hash) {
    return guarded([&] {
        DIM3_REQUIRE(ctx, DIM3_ERR_ARG, "null ctx");
        DIM3_REQUIRE(t_map >= 0.0 && t_rand >= 0.0 && t_hash >= 0.0, DIM3_ERR_ARG, "negative cost constant");
        ctx->c.opt.f1c[0] = t_map;
        ctx->c.opt.f1c[1] = t_rand;
        ctx->c.opt.f1c[2] = t_hash;
    });
}

int dim3_ctx_last_path(const dim3_ctx* ctx) { return ctx ? ctx->last_path : 0; }

int dim3_map(dim3_ctx* ctx, const int32_t* d_vals, int64_t n, int32_t* d_ids, int32_t* d_dict, int64_t* n_distinct,
             void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && n_distinct, DIM3_ERR_ARG, "null ctx or n_distinct");
        DIM3_REQUIRE(n >= 0 && (n == 0 || (d_vals && d_ids && d_dict)), DIM3_ERR_ARG, "bad column arguments");
        DIM3_REQUIRE(n < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "more than 2^31 - 1 rows");
        DeviceGuard g(ctx->c.device);
        cudaStream_t s = as_stream(stream);
        dimcube::ValueMap vm;
        {
            dimcube::PhaseScope ps(ctx->c.stats, dimcube::PH_MAP, s);
            dimcube::build_value_map(d_vals, nullptr, n, vm, d_ids, d_dict, s);
        }
        DIM3_CUDA(cudaStreamSynchronize(s));
        *n_distinct = vm.n_distinct;
    });
}

int dim3_map_noalloc(const int32_t* d_vals, int64_t n, int32_t* d_ids, int32_t* d_dict, int64_t* n_distinct,
                     void* stream) {
    return guarded([&] { dimcube::map_noalloc(d_vals, n, d_ids, d_dict, n_distinct, as_stream(stream)); });
}

int dim3_ctx_timing(dim3_ctx* ctx, int phase, double* total_ms, int64_t* launches, int reset) {
    return guarded([&] {
        DIM3_REQUIRE(ctx, DIM3_ERR_ARG, "ctx is null");
        DIM3_REQUIRE(phase >= 0 && phase < dimcube::PH_N, DIM3_ERR_ARG, "unknown phase");
        DeviceGuard g(ctx->c.device);
        ctx->stats.resolve();
        if (total_ms) *total_ms = ctx->stats.ms[phase];
        if (launches) *launches = ctx->stats.n[phase];
        if (reset) ctx->stats.reset();
    });
}

int dim3_launch_count(int64_t* out) {
    return guarded([&] {
        DIM3_REQUIRE(out, DIM3_ERR_ARG, "out is null");
        *out = dimcube::g_launches.load();
    });
}

static int64_t resolve_theta(const dim3_ctx* ctx, int32_t theta_z) {
    if (theta_z >= 0) return theta_z;
    return ctx->c.opt.theta_z;  // < 0 means the tuned default inside the plan builder
}

int dim3_partition(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr, const int32_t* d_s_key,
                   const int32_t* d_s_val, int64_t ns, int32_t theta_z, dim3_plan** plan_out, dim3_plan_info* info,
                   void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan_out, DIM3_ERR_ARG, "null ctx or plan_out");
        *plan_out = nullptr;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DeviceGuard g(ctx->c.device);
        std::unique_ptr<dim3_plan> pl(new dim3_plan());
        pl->p.reset(dimcube::build_plan(ctx->c, single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns),
                                        resolve_theta(ctx, theta_z), as_stream(stream)));
        if (info) *info = pl->p->info;
        *plan_out = pl.release();
    });
}

int dim3_partition_ids(dim3_ctx* ctx, const int32_t* d_r_y, const int32_t* d_r_x, int64_t nr, const int32_t* d_s_y,
                       const int32_t* d_s_z, int64_t ns, int64_t n_x, int64_t n_y, int64_t n_z, int32_t theta_z,
                       dim3_plan** plan_out, dim3_plan_info* info, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan_out, DIM3_ERR_ARG, "null ctx or plan_out");
        *plan_out = nullptr;
        check_table(d_r_y, d_r_x, nr, "R");
        check_table(d_s_y, d_s_z, ns, "S");
        DeviceGuard g(ctx->c.device);
        dimcube::PlanInput in = single_input(d_r_y, d_r_x, nr, d_s_y, d_s_z, ns);
        in.premapped = true;
        in.n_x = n_x;
        in.n_y = n_y;
        in.n_z = n_z;
        std::unique_ptr<dim3_plan> pl(new dim3_plan());
        pl->p.reset(dimcube::build_plan(ctx->c, in, resolve_theta(ctx, theta_z), as_stream(stream)));
        if (info) *info = pl->p->info;
        *plan_out = pl.release();
    });
}

int dim3_map_tuples(dim3_ctx* ctx, const int32_t* const* d_cols, int k, uint32_t unsigned_mask, int64_t n,
                    int32_t* d_ids, int32_t* d_first, int64_t* n_distinct, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && n_distinct, DIM3_ERR_ARG, "null ctx or n_distinct");
        DIM3_REQUIRE(k >= 1 && k <= dimcube::kMaxTupleCols, DIM3_ERR_ARG, "k must be 1..8");
        DIM3_REQUIRE(n >= 0, DIM3_ERR_ARG, "negative row count");
        DIM3_REQUIRE(n < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "more than 2^31 - 1 rows");
        if (n > 0) {
            DIM3_REQUIRE(d_cols && d_ids && d_first, DIM3_ERR_ARG, "null column or output pointer");
            for (int c = 0; c < k; ++c) DIM3_REQUIRE(d_cols[c], DIM3_ERR_ARG, "null column pointer");
        }
        DeviceGuard g(ctx->c.device);
        cudaStream_t s = as_stream(stream);
        int64_t d = 0;
        {
            dimcube::PhaseScope ps(ctx->c.stats, dimcube::PH_MAP, s);
            d = dimcube::map_tuples(d_cols, k, unsigned_mask, n, d_ids, d_first, s);
        }
        DIM3_CUDA(cudaStreamSynchronize(s));
        *n_distinct = d;
    });
}

int dim3_gather_i32(dim3_ctx* ctx, const int32_t* d_src, int64_t n_src, const int32_t* d_idx, int64_t n,
                    int32_t* d_dst, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx, DIM3_ERR_ARG, "null ctx");
        DIM3_REQUIRE(n >= 0 && n_src >= 0, DIM3_ERR_ARG, "negative length");
        DIM3_REQUIRE(n == 0 || (d_idx && d_dst && (n_src == 0 || d_src)), DIM3_ERR_ARG, "null pointer");
        DeviceGuard g(ctx->c.device);
        const bool ok = dimcube::gather_i32(d_src, n_src, d_idx, n, d_dst, as_stream(stream));
        DIM3_REQUIRE(ok, DIM3_ERR_ARG, "an index lies outside [0, n_src)");
    });
}

int dim3_cache_build(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr, const int32_t* d_s_key,
                     const int32_t* d_s_val, int64_t ns, int32_t theta_z, int64_t budget, double t_sparse,
                     double t_dense, dim3_cache** cache_out, dim3_cache_info* info, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && cache_out, DIM3_ERR_ARG, "null ctx or cache_out");
        *cache_out = nullptr;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DeviceGuard g(ctx->c.device);
        std::unique_ptr<dim3_cache> c(new dim3_cache());
        c->c.reset(dimcube::build_result_cache(ctx->c, single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns),
                                               resolve_theta(ctx, theta_z), budget, t_sparse, t_dense,
                                               as_stream(stream)));
        if (info) *info = dim3_cache_info{c->c->n_c, c->c->n_list, c->c->space, c->c->n_x};
        *cache_out = c.release();
    });
}

int dim3_cache_export(dim3_ctx* ctx, const dim3_cache* cache, int32_t* d_z, int64_t* d_size, uint8_t* d_complement,
                      int64_t* d_offsets, int32_t* d_xs, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && cache, DIM3_ERR_ARG, "null ctx or cache");
        DeviceGuard g(ctx->c.device);
        const dimcube::ResultCache& c = *cache->c;
        cudaStream_t s = as_stream(stream);
        auto cp = [&](void* dst, const dimcube::DevBuf& src, size_t bytes) {
            if (dst && bytes) DIM3_CUDA(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToDevice, s));
        };
        cp(d_z, c.z, (size_t)c.n_c * 4);
        cp(d_size, c.size, (size_t)c.n_c * 8);
        cp(d_complement, c.comp, (size_t)c.n_c);
        cp(d_offsets, c.off, (size_t)(c.n_c + 1) * 8);
        cp(d_xs, c.xs, (size_t)c.n_list * 4);
        DIM3_CUDA(cudaStreamSynchronize(s));
    });
}

int dim3_cache_destroy(dim3_cache* cache) {
    return guarded([&] { delete cache; });
}

int dim3_partition_cached(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr,
                          const int32_t* d_s_key, const int32_t* d_s_val, int64_t ns, const dim3_cache* cache,
                          int32_t theta_z, dim3_plan** plan_out, dim3_plan_info* info, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan_out && cache, DIM3_ERR_ARG, "null ctx, cache or plan_out");
        *plan_out = nullptr;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DeviceGuard g(ctx->c.device);
        dimcube::PlanInput in = single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns);
        in.cache = cache->c.get();
        std::unique_ptr<dim3_plan> pl(new dim3_plan());
        pl->p.reset(dimcube::build_plan(ctx->c, in, resolve_theta(ctx, theta_z), as_stream(stream)));
        if (info) *info = pl->p->info;
        *plan_out = pl.release();
    });
}

int dim3_join_aggregate(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, const int32_t* d_r_v,
                        int64_t nr, const int32_t* d_s_key, const int32_t* d_s_val, const int32_t* d_s_u, int64_t ns,
                        int agg, int fn, int32_t* d_out_x, int32_t* d_out_z, void* d_out_val, int64_t capacity,
                        int64_t* count, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && count, DIM3_ERR_ARG, "null ctx or count");
        *count = 0;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DIM3_REQUIRE(nr == 0 || d_r_v, DIM3_ERR_ARG, "R: null value column");
        DIM3_REQUIRE(ns == 0 || d_s_u, DIM3_ERR_ARG, "S: null value column");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        DeviceGuard g(ctx->c.device);
        dimcube::join_aggregate(ctx->c, single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns), d_r_v, d_s_u, agg,
                                fn, d_out_x, d_out_z, d_out_val, capacity, count, as_stream(stream));
    });
}

int dim3_groupby_aggregate(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr,
                           const int32_t* d_s_key, const int32_t* d_s_val, int64_t ns, int agg, int32_t* d_out_x,
                           void* d_out_val, int64_t capacity, int64_t* count, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && count, DIM3_ERR_ARG, "null ctx or count");
        *count = 0;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        DeviceGuard g(ctx->c.device);
        dimcube::groupby_aggregate(ctx->c, single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns), agg, d_out_x,
                                   d_out_val, capacity, count, as_stream(stream));
    });
}

static void check_edges(int k, const dim3_edge_table* t) {
    DIM3_REQUIRE(k >= 1 && t, DIM3_ERR_ARG, "need at least one table");
    for (int i = 0; i < k; ++i) check_table(t[i].d_a, t[i].d_b, t[i].n, "R_i");
}

int dim3_mjp_sizes(dim3_ctx* ctx, int k, const dim3_edge_table* tables, double* out_j, double* out_p, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && out_j && out_p, DIM3_ERR_ARG, "null ctx or output");
        check_edges(k, tables);
        DeviceGuard g(ctx->c.device);
        dimcube::mjp_sizes(ctx->c, k, tables, out_j, out_p, as_stream(stream));
    });
}

int dim3_mjp_plan(int k, const double* r_size, const double* out_j, const double* out_p, const double* c, int* dedup,
                  double* cost) {
    return guarded([&] {
        DIM3_REQUIRE(k >= 1 && r_size && out_j && out_p && c && dedup, DIM3_ERR_ARG, "null argument");
        for (int i = 0; i < 5; ++i) DIM3_REQUIRE(c[i] >= 0.0, DIM3_ERR_ARG, "negative cost constant");
        const double v = dimcube::mjp_dp(k, r_size, out_j, out_p, c, dedup);
        if (cost) *cost = v;
    });
}

int dim3_mjp_execute(dim3_ctx* ctx, int k, const dim3_edge_table* tables, const int* dedup, int32_t* d_out_x,
                     int32_t* d_out_z, int64_t capacity, int64_t* count, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && count && dedup, DIM3_ERR_ARG, "null ctx, dedup or count");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        *count = 0;
        check_edges(k, tables);
        DeviceGuard g(ctx->c.device);
        dimcube::mjp_execute(ctx->c, k, tables, dedup, d_out_x, d_out_z, capacity, count, as_stream(stream));
    });
}

int dim3_plan_get_info(const dim3_plan* plan, dim3_plan_info* info) {
    return guarded([&] {
        DIM3_REQUIRE(plan && info, DIM3_ERR_ARG, "null plan or info");
        *info = plan->p->info;
    });
}

int dim3_plan_row_counts(dim3_ctx* ctx, dim3_plan* plan, int64_t x_begin, int64_t x_end, int64_t* d_counts,
                         void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan, DIM3_ERR_ARG, "null ctx or plan");
        DIM3_REQUIRE(x_end == x_begin || d_counts, DIM3_ERR_ARG, "null d_counts");
        DeviceGuard g(ctx->c.device);
        dimcube::plan_row_counts(ctx->c, *plan->p, x_begin, x_end, d_counts, as_stream(stream));
        DIM3_CUDA(cudaStreamSynchronize(as_stream(stream)));
    });
}

int dim3_plan_join_project(dim3_ctx* ctx, dim3_plan* plan, int64_t x_begin, int64_t x_end, int32_t* d_out_x,
                           int32_t* d_out_z, int64_t capacity, int64_t* count, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan && count, DIM3_ERR_ARG, "null ctx, plan or count");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        *count = 0;
        DeviceGuard g(ctx->c.device);
        dimcube::plan_join(ctx->c, *plan->p, x_begin, x_end, 0, d_out_x, d_out_z, nullptr, capacity, count,
                           as_stream(stream));
    });
}

int dim3_plan_join_count(dim3_ctx* ctx, dim3_plan* plan, int64_t x_begin, int64_t x_end, int32_t* d_out_x,
                         int32_t* d_out_z, int32_t* d_out_cnt, int64_t capacity, int64_t* count, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan && count, DIM3_ERR_ARG, "null ctx, plan or count");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        *count = 0;
        DeviceGuard g(ctx->c.device);
        dimcube::plan_join(ctx->c, *plan->p, x_begin, x_end, 1, d_out_x, d_out_z, d_out_cnt, capacity, count,
                           as_stream(stream));
    });
}

int dim3_plan_export(dim3_plan* plan, int which, void* d_dst, int64_t bytes, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(plan, DIM3_ERR_ARG, "null plan");
        const dimcube::Plan& p = *plan->p;
        const dim3_plan_info& in = p.info;
        const void* src = nullptr;
        int64_t need = 0;
        switch (which) {
            case DIM3_TABLE_DICT_X: src = p.dict_x.p; need = in.n_x * 4; break;
            case DIM3_TABLE_DICT_Y: src = p.dict_y.p; need = in.n_y * 4; break;
            case DIM3_TABLE_DICT_Z: src = p.dict_z.p; need = in.n_z * 4; break;
            case DIM3_TABLE_R_ROWPTR: src = p.r_rowptr.p; need = (in.n_x + 1) * 8; break;
            case DIM3_TABLE_R_COL: src = p.r_col.p; need = in.n_r_kept * 4; break;
            case DIM3_TABLE_M_Z: src = p.m_z.p; need = in.n_z * 4; break;
            case DIM3_TABLE_DENSE_Z: src = p.dense_z.p; need = in.n_z; break;
            case DIM3_TABLE_SS_ROWPTR: src = p.ss_rowptr.p; need = (in.n_y + 1) * 8; break;
            case DIM3_TABLE_SS_COL: src = p.ss_col.p; need = in.n_s_sparse * 4; break;
            case DIM3_TABLE_DEG_S: src = p.deg_s.p; need = in.n_y * 4; break;
            case DIM3_TABLE_OUTJ_X: src = p.outj_x.p; need = in.n_x * 8; break;
            default: throw dimcube::Error(DIM3_ERR_ARG, "unknown table " + std::to_string(which));
        }
        DIM3_REQUIRE(bytes >= need, DIM3_ERR_CAPACITY, "destination smaller than the table");
        if (need == 0) return;
        DIM3_REQUIRE(d_dst, DIM3_ERR_ARG, "null destination");
        DeviceGuard g(p.device);
        DIM3_CUDA(cudaMemcpyAsync(d_dst, src, (size_t)need, cudaMemcpyDeviceToDevice, as_stream(stream)));
        DIM3_CUDA(cudaStreamSynchronize(as_stream(stream)));
    });
}

int dim3_plan_destroy(dim3_plan* plan) {
    return guarded([&] {
        if (!plan) return;
        DeviceGuard g(plan->p->device);
        cudaStream_t s = plan->p->stream;
        delete plan;
        DIM3_CUDA(cudaStreamSynchronize(s));
    });
}

static int join_common(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr,
                       const int32_t* d_s_key, const int32_t* d_s_val, int64_t ns, int32_t* d_out_x, int32_t* d_out_z,
                       int32_t* d_out_cnt, int64_t capacity, int64_t* count, void* stream, int kind) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && count, DIM3_ERR_ARG, "null ctx or count");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        *count = 0;
        check_table(d_r_key, d_r_val, nr, "R");
        check_table(d_s_key, d_s_val, ns, "S");
        DeviceGuard g(ctx->c.device);
        cudaStream_t s = as_stream(stream);
        const dimcube::PlanInput in = single_input(d_r_key, d_r_val, nr, d_s_key, d_s_val, ns);
        const int64_t path = ctx->c.opt.path;
        std::unique_ptr<dimcube::Plan> p;
        bool classical = path == 2;
        if (!classical) {
            // path 0: f1 (Section 2.6), evaluated right after the y mapping,
            // may hand the join to the classical solution
            p.reset(dimcube::build_plan(ctx->c, in, resolve_theta(ctx, -1), s, path == 0 ? &classical : nullptr));
        }
        ctx->last_path = classical ? 2 : 1;
        if (classical) {
            dimcube::classical_join(ctx->c, in, kind, d_out_x, d_out_z, d_out_cnt, capacity, count, s);
            return;
        }
        try {
            dimcube::plan_join(ctx->c, *p, 0, p->info.n_x, kind, d_out_x, d_out_z, d_out_cnt, capacity, count, s);
        } catch (...) {
            p.reset();
            cudaStreamSynchronize(s);
            throw;
        }
        p.reset();
        DIM3_CUDA(cudaStreamSynchronize(s));
    });
}

int dim3_batch_partition(dim3_ctx* ctx, int n_inst, const dim3_instance* inst, int32_t theta_z, dim3_plan** plan_out,
                         dim3_plan_info* info, void* stream) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && plan_out && inst && n_inst >= 1, DIM3_ERR_ARG, "null ctx, plan_out or instances");
        *plan_out = nullptr;
        DeviceGuard g(ctx->c.device);
        std::unique_ptr<dim3_plan> pl(new dim3_plan());
        pl->p.reset(dimcube::build_batch_plan(ctx->c, n_inst, inst, resolve_theta(ctx, theta_z), as_stream(stream)));
        if (info) *info = pl->p->info;
        *plan_out = pl.release();
    });
}

int dim3_plan_instance_ranges(const dim3_plan* plan, int64_t* x_lo) {
    return guarded([&] {
        DIM3_REQUIRE(plan && x_lo, DIM3_ERR_ARG, "null plan or x_lo");
        const auto& v = plan->p->h_inst_x_lo;
        std::copy(v.begin(), v.end(), x_lo);
    });
}

static int batch_common(dim3_ctx* ctx, int n_inst, const dim3_instance* inst, int32_t* d_out_x, int32_t* d_out_z,
                        int32_t* d_out_cnt, int64_t capacity, int64_t* inst_counts, int64_t* count, void* stream,
                        int kind) {
    return guarded([&] {
        DIM3_REQUIRE(ctx && count && inst && n_inst >= 1, DIM3_ERR_ARG, "null ctx, count or instances");
        DIM3_REQUIRE(capacity >= 0, DIM3_ERR_ARG, "negative capacity");
        *count = 0;
        DeviceGuard g(ctx->c.device);
        cudaStream_t s = as_stream(stream);
        std::unique_ptr<dimcube::Plan> p(dimcube::build_batch_plan(ctx->c, n_inst, inst, resolve_theta(ctx, -1), s));
        try {
            dimcube::plan_join(ctx->c, *p, 0, p->info.n_x, kind, d_out_x, d_out_z, d_out_cnt, capacity, count, s);
            if (inst_counts) dimcube::batch_instance_counts(*p, inst_counts, s);
        } catch (const dimcube::Error& e) {
            if (e.status == DIM3_ERR_CAPACITY && inst_counts) dimcube::batch_instance_counts(*p, inst_counts, s);
            p.reset();
            cudaStreamSynchronize(s);
            throw;
        } catch (...) {
            p.reset();
            cudaStreamSynchronize(s);
            throw;
        }
        p.reset();
        DIM3_CUDA(cudaStreamSynchronize(s));
    });
}

int dim3_batch_join_project(dim3_ctx* ctx, int n_inst, const dim3_instance* inst, int32_t* d_out_x, int32_t* d_out_z,
                            int64_t capacity, int64_t* inst_counts, int64_t* count, void* stream) {
    return batch_common(ctx, n_inst, inst, d_out_x, d_out_z, nullptr, capacity, inst_counts, count, stream, 0);
}

int dim3_batch_join_count(dim3_ctx* ctx, int n_inst, const dim3_instance* inst, int32_t* d_out_x, int32_t* d_out_z,
                          int32_t* d_out_cnt, int64_t capacity, int64_t* inst_counts, int64_t* count, void* stream) {
    return batch_common(ctx, n_inst, inst, d_out_x, d_out_z, d_out_cnt, capacity, inst_counts, count, stream, 1);
}

int dim3_join_project(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr, const int32_t* d_s_key,
                      const int32_t* d_s_val, int64_t ns, int32_t* d_out_x, int32_t* d_out_z, int64_t capacity,
                      int64_t* count, void* stream) {
    return join_common(ctx, d_r_key, d_r_val, nr, d_s_key, d_s_val, ns, d_out_x, d_out_z, nullptr, capacity, count,
                       stream, 0);
}

int dim3_join_count(dim3_ctx* ctx, const int32_t* d_r_key, const int32_t* d_r_val, int64_t nr, const int32_t* d_s_key,
                    const int32_t* d_s_val, int64_t ns, int32_t* d_out_x, int32_t* d_out_z, int32_t* d_out_cnt,
                    int64_t capacity, int64_t* count, void* stream) {
    return join_common(ctx, d_r_key, d_r_val, nr, d_s_key, d_s_val, ns, d_out_x, d_out_z, d_out_cnt, capacity, count,
                       stream, 1);
}

}  // extern "C"
