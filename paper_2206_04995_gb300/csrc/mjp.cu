// Multi-way joins with projection, MJP (Section 4.2): the line query
// Pi_{x_1, x_{k+1}}(R_1(x_1, x_2) join R_2(x_2, x_3) join ... join R_k(x_k, x_{k+1}))
// as a left-deep plan whose deduplications are placed by the section's
// dynamic programme.
//
// Execution: the running result is a pair list (x_1, x_i). A join with a
// deduplication after it is one Join-Project of this library (the running
// result as R(x = x_1, y = x_i), R_i as S(z = x_{i+1}, y = x_i)); a join
// without one is the bag join (every running pair joins, nothing is removed).
//
// Sizes for the programme: |OUT_J_i| counts the join paths through the
// first i tables (path counts per end value, carried table by table: a
// gather of the previous counts along R_i's edges and a segmented sum by the
// new end value, in double, exact below 2^53), |OUT_P_i| the distinct (x_1,
// x_{i+1}) after each table (a chain of Join-Projects).
#include <algorithm>
#include <memory>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

#define GRID_STRIDE(i, n)                                                        \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------- DP
double mjp_dp(int k, const double* r_size, const double* out_j, const double* out_p, const double* c, int* dedup) {
    for (int i = 0; i < k; ++i) dedup[i] = 0;
    if (k < 2) return 0.0;
    std::vector<double> rho(k), best(k, 0.0);
    std::vector<int> arg(k, -1);
    for (int i = 0; i < k; ++i) rho[i] = out_j[i] > 0.0 ? out_p[i] / out_j[i] : 0.0;
    for (int i = 1; i < k; ++i) {
        bool have = false;
        double cand = 0.0;
        for (int j = 0; j < i; ++j) {
            double total = best[j];
            for (int h = j + 1; h < i; ++h)  // joins without deduplication
                total += c[0] * (rho[j] * out_j[h - 1] + r_size[h]) + c[1] * (rho[j] * out_j[h]);
            total += c[2] * (rho[j] * out_j[i - 1] + r_size[i]) + c[3] * (rho[j] * out_j[i]) + c[4] * out_p[i];
            if (!have || total < cand) {
                cand = total;
                arg[i] = j;
                have = true;
            }
        }
        best[i] = cand;
    }
    for (int i = k - 1; i > 0; i = arg[i]) dedup[i] = 1;
    return best[k - 1];
}

// -------------------------------------------------------------- pairs
struct PairList {
    DevBuf a, b;  // int32 columns
    int64_t n = 0;
};

static void copy_pairs(const int32_t* a, const int32_t* b, int64_t n, PairList& out, cudaStream_t s) {
    out.a.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
    out.b.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
    if (n > 0) {
        DIM3_CUDA(cudaMemcpyAsync(out.a.p, a, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        DIM3_CUDA(cudaMemcpyAsync(out.b.p, b, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    out.n = n;
}

// one step of the chain: cur (x_1, x_i) joined with R_i (x_i, x_{i+1})
static void chain_step(const Ctx& ctx, const PairList& cur, const dim3_edge_table& t, bool dedup, PairList& next,
                       cudaStream_t s) {
    PlanInput in;
    in.r_key = cur.b.as<int32_t>();
    in.r_val = cur.a.as<int32_t>();
    in.nr = cur.n;
    in.s_key = t.d_a;
    in.s_val = t.d_b;
    in.ns = t.n;
    int64_t m = 0;
    if (dedup) {
        std::unique_ptr<Plan> p(build_plan(ctx, in, -1, s));
        const int64_t n_x = p->info.n_x;
        if (n_x > 0) {
            DevBuf cnt, off;
            cnt.alloc((size_t)n_x * 8, s);
            off.alloc((size_t)(n_x + 1) * 8, s);
            plan_row_counts(ctx, *p, 0, n_x, cnt.as<int64_t>(), s);
            exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), n_x, s);
            m = read_i64(off.as<int64_t>() + n_x, s);
        }
        next.a.alloc((size_t)std::max<int64_t>(m, 1) * 4, s);
        next.b.alloc((size_t)std::max<int64_t>(m, 1) * 4, s);
        int64_t got = 0;
        if (m > 0) plan_join(ctx, *p, 0, n_x, 0, next.a.as<int32_t>(), next.b.as<int32_t>(), nullptr, m, &got, s);
        DIM3_REQUIRE(got == m, DIM3_ERR_CUDA, "MJP: inconsistent Join-Project size");
    } else {
        m = bag_join_into(ctx, in, next.a, next.b, s);
    }
    next.n = m;
}

int64_t mjp_execute(const Ctx& ctx, int k, const dim3_edge_table* t, const int* dedup, int32_t* out_x,
                    int32_t* out_z, int64_t capacity, int64_t* count, cudaStream_t s) {
    DIM3_REQUIRE(k >= 1, DIM3_ERR_ARG, "at least one table");
    DIM3_REQUIRE(k == 1 || dedup[k - 1], DIM3_ERR_ARG, "the last join must deduplicate (the query's projection)");
    if (k == 1)  // the projection of one relation: its distinct pairs
        return distinct_pairs(t[0].d_a, t[0].d_b, t[0].n, out_x, out_z, capacity, count, s);
    // relations are sets: the running result starts as R_1's distinct pairs
    PairList cur;
    cur.a.alloc((size_t)std::max<int64_t>(t[0].n, 1) * 4, s);
    cur.b.alloc((size_t)std::max<int64_t>(t[0].n, 1) * 4, s);
    distinct_pairs(t[0].d_a, t[0].d_b, t[0].n, cur.a.as<int32_t>(), cur.b.as<int32_t>(), t[0].n, &cur.n, s);
    for (int i = 1; i < k; ++i) {
        PairList next;
        chain_step(ctx, cur, t[i], dedup[i] != 0, next, s);
        cur = std::move(next);
    }
    if (count) *count = cur.n;
    if (cur.n > capacity)
        throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) + " < result size " +
                                           std::to_string(cur.n));
    if (cur.n > 0) {
        DIM3_REQUIRE(out_x && out_z, DIM3_ERR_ARG, "null output buffer");
        DIM3_CUDA(cudaMemcpyAsync(out_x, cur.a.p, (size_t)cur.n * 4, cudaMemcpyDeviceToDevice, s));
        DIM3_CUDA(cudaMemcpyAsync(out_z, cur.b.p, (size_t)cur.n * 4, cudaMemcpyDeviceToDevice, s));
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
    return cur.n;
}

// ---------------------------------------------------------------- sizes
__global__ void k_pack_edge(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n, uint64_t* keys) {
    GRID_STRIDE(i, n) keys[i] = ((uint64_t)((uint32_t)a[i] ^ 0x80000000u) << 32) | ((uint32_t)b[i] ^ 0x80000000u);
}

// path counts after one more table: for every distinct edge (u, v), the count
// of u (binary search among the previous end values) is added to v's slot
// (v's position among the distinct new end values)
__global__ void k_carry_paths(const uint64_t* __restrict__ edges, int64_t ne, const uint32_t* __restrict__ ends,
                              const double* __restrict__ cnt, int64_t n_ends, const uint32_t* __restrict__ new_ends,
                              int64_t n_new, double* new_cnt) {
    GRID_STRIDE(i, ne) {
        const uint32_t u = (uint32_t)(edges[i] >> 32), v = (uint32_t)edges[i];
        const int64_t j = lower_bound_dev<uint32_t>(ends, 0, n_ends, u);
        if (j < n_ends && ends[j] == u) {
            const int64_t q = lower_bound_dev<uint32_t>(new_ends, 0, n_new, v);
            atomicAdd(new_cnt + q, cnt[j]);
        }
    }
}

__global__ void k_add_one_by_end(const uint64_t* __restrict__ edges, int64_t ne, const uint32_t* __restrict__ ends,
                                 int64_t n_ends, double* cnt) {
    GRID_STRIDE(i, ne) atomicAdd(cnt + lower_bound_dev<uint32_t>(ends, 0, n_ends, (uint32_t)edges[i]), 1.0);
}

__global__ void k_low_words(const uint64_t* __restrict__ k, int64_t n, uint32_t* out) {
    GRID_STRIDE(i, n) out[i] = (uint32_t)k[i];
}

__global__ void k_sum_doubles(const double* __restrict__ v, int64_t n, double* total) {
    // single block: deterministic order is not needed (integers below 2^53)
    __shared__ double s[kThreads];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s[0];
}

void mjp_sizes(const Ctx& ctx, int k, const dim3_edge_table* t, double* out_j, double* out_p, cudaStream_t s) {
    DIM3_REQUIRE(k >= 1, DIM3_ERR_ARG, "at least one table");
    // distinct edges of every table, sorted by (u, v)
    std::vector<DevBuf> edges(k);
    std::vector<int64_t> ne(k);
    for (int i = 0; i < k; ++i) {
        DevBuf keys, alt;
        keys.alloc((size_t)std::max<int64_t>(t[i].n, 1) * 8, s);
        alt.alloc((size_t)std::max<int64_t>(t[i].n, 1) * 8, s);
        if (t[i].n > 0) {
            k_pack_edge<<<grid_for(t[i].n), kThreads, 0, s>>>(t[i].d_a, t[i].d_b, t[i].n, keys.as<uint64_t>());
            DIM3_LAUNCHED();
        }
        radix_sort_u64(keys.as<uint64_t>(), nullptr, alt.as<uint64_t>(), nullptr, t[i].n, 64, s);
        edges[i].alloc((size_t)std::max<int64_t>(t[i].n, 1) * 8, s);
        ne[i] = t[i].n > 0 ? unique_sorted_u64(keys.as<uint64_t>(), edges[i].as<uint64_t>(), t[i].n, s) : 0;
    }
    // OUT_J: path counts per end value, table by table
    auto end_values = [&](const DevBuf& e, int64_t n, DevBuf& vals) -> int64_t {
        DevBuf low, alt;
        low.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
        alt.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
        if (n > 0) {
            k_low_words<<<grid_for(n), kThreads, 0, s>>>(e.as<uint64_t>(), n, low.as<uint32_t>());
            DIM3_LAUNCHED();
        }
        radix_sort_u32(low.as<uint32_t>(), nullptr, alt.as<uint32_t>(), nullptr, n, 32, s);
        vals.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
        return n > 0 ? unique_sorted_u32(low.as<uint32_t>(), vals.as<uint32_t>(), n, s) : 0;
    };
    DevBuf ends, cnt, tot;
    tot.alloc(8, s);
    int64_t n_ends = end_values(edges[0], ne[0], ends);
    cnt.alloc((size_t)std::max<int64_t>(n_ends, 1) * 8, s);
    DIM3_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes, s));
    if (ne[0] > 0) {  // one path per distinct edge of R_1, counted at its end value
        k_add_one_by_end<<<grid_for(ne[0]), kThreads, 0, s>>>(edges[0].as<uint64_t>(), ne[0], ends.as<uint32_t>(),
                                                               n_ends, cnt.as<double>());
        DIM3_LAUNCHED();
    }
    out_j[0] = (double)ne[0];
    out_p[0] = (double)ne[0];
    for (int i = 1; i < k; ++i) {
        DevBuf new_ends, new_cnt;
        const int64_t n_new = end_values(edges[i], ne[i], new_ends);
        new_cnt.alloc((size_t)std::max<int64_t>(n_new, 1) * 8, s);
        DIM3_CUDA(cudaMemsetAsync(new_cnt.p, 0, new_cnt.bytes, s));
        if (ne[i] > 0 && n_ends > 0) {
            k_carry_paths<<<grid_for(ne[i]), kThreads, 0, s>>>(edges[i].as<uint64_t>(), ne[i], ends.as<uint32_t>(),
                                                               cnt.as<double>(), n_ends, new_ends.as<uint32_t>(),
                                                               n_new, new_cnt.as<double>());
            DIM3_LAUNCHED();
        }
        k_sum_doubles<<<1, kThreads, 0, s>>>(new_cnt.as<double>(), n_new, tot.as<double>());
        DIM3_LAUNCHED();
        DIM3_CUDA(cudaMemcpyAsync(&out_j[i], tot.p, 8, cudaMemcpyDeviceToHost, s));
        DIM3_CUDA(cudaStreamSynchronize(s));
        ends = std::move(new_ends);
        cnt = std::move(new_cnt);
        n_ends = n_new;
    }
    // OUT_P: the chain of Join-Projects
    PairList cur;
    copy_pairs(t[0].d_a, t[0].d_b, t[0].n, cur, s);
    for (int i = 1; i < k; ++i) {
        PairList next;
        chain_step(ctx, cur, t[i], true, next, s);
        cur = std::move(next);
        out_p[i] = (double)cur.n;
    }
}

}  // namespace dimcube
