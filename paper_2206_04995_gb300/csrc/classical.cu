// The classical solution (Section 1.1) on the GPU, the strategy choice f1
// between it and the hybrid path (Section 2.6), and the bag join that the
// multi-way plans of Section 4.2 use between deduplications.
//
// GPU form: sorting instead of hashing. The distinct input tuples of R and S
// are radix-sorted as 64-bit (y, value) keys (values with the sign bit flipped,
// so key order is signed value order). Both tables are then sorted by y, and
// every R tuple finds the S tuples of its y by binary search: a counting pass,
// a scan and an emitting pass (one warp per R tuple, lanes over its S range)
// materialise the join results as packed (x, z) keys. Deduplication is a radix
// sort of those keys and a unique (the sorted order is the canonical order);
// Join-Count is the run length of each key.
#include <algorithm>
#include <memory>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

#define GRID_STRIDE(i, n)                                                        \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

__host__ __device__ __forceinline__ uint32_t flip(int32_t v) { return (uint32_t)v ^ 0x80000000u; }
__host__ __device__ __forceinline__ int32_t unflip(uint32_t v) { return (int32_t)(v ^ 0x80000000u); }

__global__ void k_pack_yv(const int32_t* __restrict__ y, const int32_t* __restrict__ v, int64_t n, uint64_t* keys) {
    GRID_STRIDE(i, n) keys[i] = ((uint64_t)flip(y[i]) << 32) | flip(v[i]);
}

// the (y, value) tuples of a table, ascending; distinct unless keep_dups
static int64_t sorted_tuples(const int32_t* y, const int32_t* v, int64_t n, DevBuf& out, cudaStream_t s,
                             bool keep_dups = false) {
    DevBuf keys, alt;
    keys.alloc((size_t)std::max<int64_t>(n, 1) * 8, s);
    alt.alloc((size_t)std::max<int64_t>(n, 1) * 8, s);
    if (n > 0) {
        k_pack_yv<<<grid_for(n), kThreads, 0, s>>>(y, v, n, keys.as<uint64_t>());
        DIM3_LAUNCHED();
    }
    radix_sort_u64(keys.as<uint64_t>(), nullptr, alt.as<uint64_t>(), nullptr, n, 64, s);
    if (keep_dups) {
        out = std::move(keys);
        return n;
    }
    out.alloc((size_t)std::max<int64_t>(n, 1) * 8, s);
    return n > 0 ? unique_sorted_u64(keys.as<uint64_t>(), out.as<uint64_t>(), n, s) : 0;
}

// S range of the y of every R tuple (lower bounds on the y half of the keys)
__global__ void k_join_ranges(const uint64_t* __restrict__ rk, int64_t nr, const uint64_t* __restrict__ sk, int64_t ns,
                              int64_t* lo, int64_t* cnt) {
    GRID_STRIDE(i, nr) {
        const uint64_t y = rk[i] >> 32;
        const int64_t a = lower_bound_dev<uint64_t>(sk, 0, ns, y << 32);
        const int64_t b = y == 0xffffffffull ? ns : lower_bound_dev<uint64_t>(sk, a, ns, (y + 1) << 32);
        lo[i] = a;
        cnt[i] = b - a;
    }
}

// join results as packed (x, z) keys, or (when split) as two int32 columns
__global__ void k_join_emit(const uint64_t* __restrict__ rk, int64_t nr, const uint64_t* __restrict__ sk,
                            const int64_t* __restrict__ lo, const int64_t* __restrict__ off, uint64_t* out_keys,
                            int32_t* out_x, int32_t* out_z) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < nr; r += warps) {
        const uint32_t xf = (uint32_t)rk[r];
        const int64_t a = lo[r], o = off[r], c = off[r + 1] - o;
        for (int64_t j = lane; j < c; j += 32) {
            const uint32_t zf = (uint32_t)sk[a + j];
            if (out_keys) {
                out_keys[o + j] = ((uint64_t)xf << 32) | zf;
            } else {
                out_x[o + j] = unflip(xf);
                out_z[o + j] = unflip(zf);
            }
        }
    }
}

// Join of the distinct tuples: returns |OUT_J|; when emit, the results
struct JoinSides {
    DevBuf rk, sk, lo, off;
    int64_t nr = 0, ns = 0, out_j = 0;
};

static void join_sides(const PlanInput& in, JoinSides& j, cudaStream_t s, bool r_bag = false) {
    j.nr = sorted_tuples(in.r_key, in.r_val, in.nr, j.rk, s, r_bag);
    j.ns = sorted_tuples(in.s_key, in.s_val, in.ns, j.sk, s);
    DevBuf cnt;
    j.lo.alloc((size_t)std::max<int64_t>(j.nr, 1) * 8, s);
    cnt.alloc((size_t)std::max<int64_t>(j.nr, 1) * 8, s);
    j.off.alloc((size_t)(j.nr + 1) * 8, s);
    if (j.nr > 0) {
        k_join_ranges<<<grid_for(j.nr), kThreads, 0, s>>>(j.rk.as<uint64_t>(), j.nr, j.sk.as<uint64_t>(), j.ns,
                                                           j.lo.as<int64_t>(), cnt.as<int64_t>());
        DIM3_LAUNCHED();
    }
    exclusive_scan_i64(cnt.as<int64_t>(), j.off.as<int64_t>(), j.nr, s);
    j.out_j = read_i64(j.off.as<int64_t>() + j.nr, s);
}

static unsigned warp_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads / 32), 152 * 32));
}

__global__ void k_run_flags(const uint64_t* __restrict__ k, int64_t n, int32_t* flag) {
    GRID_STRIDE(i, n) flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

__global__ void k_runs_out(const uint64_t* __restrict__ k, const int32_t* __restrict__ flag,
                           const int64_t* __restrict__ pos, int64_t n, int64_t n_runs, int32_t* out_x, int32_t* out_z,
                           int32_t* out_cnt) {
    GRID_STRIDE(i, n) {
        if (!flag[i]) continue;
        const int64_t r = pos[i];
        out_x[r] = unflip((uint32_t)(k[i] >> 32));
        out_z[r] = unflip((uint32_t)k[i]);
        if (out_cnt) {
            // run length: distance to the next run start (or to the end)
            int64_t e = i + 1;
            while (e < n && !flag[e]) ++e;
            out_cnt[r] = (int32_t)(e - i);
        }
    }
}

int64_t classical_join(const Ctx& ctx, const PlanInput& in, int kind, int32_t* out_x, int32_t* out_z,
                       int32_t* out_cnt, int64_t capacity, int64_t* count, cudaStream_t s) {
    DIM3_REQUIRE(in.n_inst <= 1 && !in.premapped && !in.cache, DIM3_ERR_ARG, "the classical path takes one instance");
    PhaseScope phase(ctx.stats, PH_EMIT, s);
    JoinSides j;
    join_sides(in, j, s);
    const int64_t m = j.out_j;
    DevBuf keys, alt;
    keys.alloc((size_t)std::max<int64_t>(m, 1) * 8, s);
    alt.alloc((size_t)std::max<int64_t>(m, 1) * 8, s);
    if (j.nr > 0 && m > 0) {
        k_join_emit<<<warp_grid(j.nr), kThreads, 0, s>>>(j.rk.as<uint64_t>(), j.nr, j.sk.as<uint64_t>(),
                                                          j.lo.as<int64_t>(), j.off.as<int64_t>(), keys.as<uint64_t>(),
                                                          nullptr, nullptr);
        DIM3_LAUNCHED();
    }
    radix_sort_u64(keys.as<uint64_t>(), nullptr, alt.as<uint64_t>(), nullptr, m, 64, s);
    DevBuf flag, pos;
    flag.alloc((size_t)std::max<int64_t>(m, 1) * 4, s);
    pos.alloc((size_t)(m + 1) * 8, s);
    int64_t n_out = 0;
    if (m > 0) {
        k_run_flags<<<grid_for(m), kThreads, 0, s>>>(keys.as<uint64_t>(), m, flag.as<int32_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos.as<int64_t>(), m, s);
        n_out = read_i64(pos.as<int64_t>() + m, s);
    }
    if (count) *count = n_out;
    if (n_out > capacity)
        throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) + " < result size " +
                                           std::to_string(n_out));
    if (n_out > 0) {
        DIM3_REQUIRE(out_x && out_z && (kind == 0 || out_cnt), DIM3_ERR_ARG, "null output buffer");
        k_runs_out<<<grid_for(m), kThreads, 0, s>>>(keys.as<uint64_t>(), flag.as<int32_t>(), pos.as<int64_t>(), m,
                                                     n_out, out_x, out_z, kind ? out_cnt : nullptr);
        DIM3_LAUNCHED();
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
    return n_out;
}

__global__ void k_unpack_pairs(const uint64_t* __restrict__ k, int64_t n, int32_t* a, int32_t* b) {
    GRID_STRIDE(i, n) {
        a[i] = unflip((uint32_t)(k[i] >> 32));
        b[i] = unflip((uint32_t)k[i]);
    }
}

int64_t distinct_pairs(const int32_t* a, const int32_t* b, int64_t n, int32_t* out_a, int32_t* out_b,
                       int64_t capacity, int64_t* count, cudaStream_t s) {
    DevBuf keys;
    const int64_t m = sorted_tuples(a, b, n, keys, s);  // keyed (a, b): canonical order
    if (count) *count = m;
    if (m > capacity)
        throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) + " < result size " +
                                           std::to_string(m));
    if (m > 0) {
        DIM3_REQUIRE(out_a && out_b, DIM3_ERR_ARG, "null output buffer");
        k_unpack_pairs<<<grid_for(m), kThreads, 0, s>>>(keys.as<uint64_t>(), m, out_a, out_b);
        DIM3_LAUNCHED();
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
    return m;
}

int64_t bag_join_into(const Ctx& ctx, const PlanInput& in, DevBuf& out_x, DevBuf& out_z, cudaStream_t s) {
    PhaseScope phase(ctx.stats, PH_EMIT, s);
    JoinSides j;
    join_sides(in, j, s, true);
    out_x.alloc((size_t)std::max<int64_t>(j.out_j, 1) * 4, s);
    out_z.alloc((size_t)std::max<int64_t>(j.out_j, 1) * 4, s);
    if (j.out_j > 0) {
        k_join_emit<<<warp_grid(j.nr), kThreads, 0, s>>>(j.rk.as<uint64_t>(), j.nr, j.sk.as<uint64_t>(),
                                                          j.lo.as<int64_t>(), j.off.as<int64_t>(), nullptr,
                                                          out_x.as<int32_t>(), out_z.as<int32_t>());
        DIM3_LAUNCHED();
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
    return j.out_j;
}

double f1_value(int64_t nr, int64_t ns, int64_t out_j, const double* c) {
    // f1 = 2 (|R| + |S|) t_map + |OUT_J| t_randRW - |OUT_J| t_hash (Section 2.6)
    return 2.0 * (double)(nr + ns) * c[0] + (double)out_j * c[1] - (double)out_j * c[2];
}

}  // namespace dimcube
