// Join-Aggregate (Section 4.1).
//
// Group-by attributes from both tables, G_{x,z} agg(f(R.v, S.u)): the SPA of
// SparseBMM holds an aggregate per z instead of a bit. Rows are bags, so the
// join tuples of a group (x, z) are, for every y they share, all pairs of an
// R row (x, y, v) and an S row (z, y, u). Each distinct (x, y) of R_CSR and
// (y, z) of S_sparse carries the count, sum, min and max of its rows' values,
// and the per-y contribution follows from those: COUNT adds cnt_R * cnt_S;
// SUM of v * u adds sum_R * sum_S, of v + u cnt_S * sum_R + cnt_R * sum_S, of
// v cnt_S * sum_R, of u cnt_R * sum_S; MIN and MAX of v * u take the extreme
// of the four corner products, of v + u min_R + min_S (max_R + max_S), of v or
// u that side's extreme; AVG keeps SUM and COUNT and divides at the end. All
// integer work is int64 (sums wrap modulo 2^64, so any order gives the same
// bits). Every z goes through the list path: the paper's dense alternative
// for aggregates is a plain dense product, and an exact int64 product has no
// tensor-core form on this GPU.
//
// Group-by attribute from one table, G_x agg(z): the rewrite of Section 4.1,
// SG(y, z') = per-y count, sum, min and max of S's z values, then every x
// folds its R_CSR row against SG (one value per y, so no deduplication).
#include <algorithm>
#include <memory>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

constexpr int kAggTile = 2048;  // z per SPA tile: 2 x 16 KiB of int64 accumulators (static shared memory)

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

#define GRID_STRIDE(i, n)                                                        \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// Per distinct pair: count, sum, min, max of its rows' values.
struct PairStats {
    DevBuf cnt;  // int64
    DevBuf sum;  // int64
    DevBuf mn;   // int32
    DevBuf mx;   // int32
};

__global__ void k_find_row_ids(const int32_t* __restrict__ dict, int64_t n_dict, const int32_t* __restrict__ vals,
                               const int32_t* __restrict__ pred, int64_t n, int32_t* __restrict__ ids) {
    GRID_STRIDE(i, n) {
        int32_t id = -1;
        if (!pred || pred[i] >= 0) {
            const int32_t v = vals[i];
            const int64_t j = lower_bound_dev<int32_t>(dict, 0, n_dict, v);
            if (j < n_dict && dict[j] == v) id = (int32_t)j;
        }
        ids[i] = id;
    }
}

__global__ void k_pack_kv(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                          const int32_t* __restrict__ v, int64_t n, int shift, uint64_t* keys, uint32_t* vals,
                          unsigned long long* counter) {
    __shared__ unsigned long long s_cnt[kThreads / 32 + 2];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (n + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        int32_t av = -1, bv = -1;
        if (i < n) {
            av = a[i];
            bv = b[i];
        }
        const bool ok = av >= 0 && bv >= 0;
        const unsigned long long pos = block_append<kThreads>(ok, counter, s_cnt);
        if (ok) {
            keys[pos] = ((uint64_t)(uint32_t)av << shift) | (uint64_t)(uint32_t)bv;
            vals[pos] = v ? (uint32_t)v[i] : 0u;
        }
    }
}

__global__ void k_seg_flags(const uint64_t* __restrict__ keys, int64_t n, int32_t* flag) {
    GRID_STRIDE(i, n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_seg_init(int64_t n, int64_t* cnt, int64_t* sum, int32_t* mn, int32_t* mx) {
    GRID_STRIDE(i, n) {
        cnt[i] = 0;
        sum[i] = 0;
        mn[i] = INT32_MAX;
        mx[i] = INT32_MIN;
    }
}

__global__ void k_seg_reduce(const int64_t* __restrict__ pos, const int32_t* __restrict__ flag,
                             const uint32_t* __restrict__ vals, int64_t n, int64_t* cnt, int64_t* sum, int32_t* mn,
                             int32_t* mx) {
    GRID_STRIDE(i, n) {
        const int64_t sgm = pos[i] + flag[i] - 1;
        const int32_t v = (int32_t)vals[i];
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + sgm), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(sum + sgm), (unsigned long long)(int64_t)v);
        atomicMin(mn + sgm, v);
        atomicMax(mx + sgm, v);
    }
}

// Stats of the distinct (a, b) pairs in ascending (a, b) order; rows with a
// negative id are skipped. Returns the number of distinct pairs.
static int64_t pair_stats(const int32_t* a, const int32_t* b, const int32_t* v, int64_t n, int shift, int bits,
                          PairStats& out, cudaStream_t s) {
    DevBuf keys, vals, keys_alt, vals_alt, counter;
    keys.alloc((size_t)std::max<int64_t>(n, 1) * 8, s);
    vals.alloc((size_t)std::max<int64_t>(n, 1) * 4, s);
    counter.alloc(8, s);
    DIM3_CUDA(cudaMemsetAsync(counter.p, 0, 8, s));
    if (n > 0) {
        k_pack_kv<<<grid_for(n), kThreads, 0, s>>>(a, b, v, n, shift, keys.as<uint64_t>(), vals.as<uint32_t>(),
                                                    counter.as<unsigned long long>());
        DIM3_LAUNCHED();
    }
    const int64_t m = read_i64(counter.as<int64_t>(), s);
    keys_alt.alloc((size_t)std::max<int64_t>(m, 1) * 8, s);
    vals_alt.alloc((size_t)std::max<int64_t>(m, 1) * 4, s);
    radix_sort_u64(keys.as<uint64_t>(), vals.as<uint32_t>(), keys_alt.as<uint64_t>(), vals_alt.as<uint32_t>(), m, bits,
                   s);
    DevBuf flag, pos;
    flag.alloc((size_t)std::max<int64_t>(m, 1) * 4, s);
    pos.alloc((size_t)(m + 1) * 8, s);
    int64_t d = 0;
    if (m > 0) {
        k_seg_flags<<<grid_for(m), kThreads, 0, s>>>(keys.as<uint64_t>(), m, flag.as<int32_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos.as<int64_t>(), m, s);
        d = read_i64(pos.as<int64_t>() + m, s);
    }
    out.cnt.alloc((size_t)std::max<int64_t>(d, 1) * 8, s);
    out.sum.alloc((size_t)std::max<int64_t>(d, 1) * 8, s);
    out.mn.alloc((size_t)std::max<int64_t>(d, 1) * 4, s);
    out.mx.alloc((size_t)std::max<int64_t>(d, 1) * 4, s);
    if (d > 0) {
        k_seg_init<<<grid_for(d), kThreads, 0, s>>>(d, out.cnt.as<int64_t>(), out.sum.as<int64_t>(),
                                                     out.mn.as<int32_t>(), out.mx.as<int32_t>());
        DIM3_LAUNCHED();
        k_seg_reduce<<<grid_for(m), kThreads, 0, s>>>(pos.as<int64_t>(), flag.as<int32_t>(), vals.as<uint32_t>(), m,
                                                       out.cnt.as<int64_t>(), out.sum.as<int64_t>(),
                                                       out.mn.as<int32_t>(), out.mx.as<int32_t>());
        DIM3_LAUNCHED();
    }
    return d;
}

struct AggArgs {
    int64_t n_z;
    const int64_t* r_rowptr;
    const int32_t* r_col;
    const int64_t* rc;
    const int64_t* rs;
    const int32_t* rmn;
    const int32_t* rmx;
    const int64_t* ss_rowptr;
    const int32_t* ss_col;
    const int64_t* sc;
    const int64_t* su;
    const int32_t* smn;
    const int32_t* smx;
    const int32_t* dict_x;
    const int32_t* dict_z;
    const int64_t* off;
    int agg, fn;
    int32_t* out_x;
    int32_t* out_z;
    int64_t* out_i;
    double* out_f;
};

__device__ __forceinline__ int64_t mul_wrap(int64_t a, int64_t b) {
    return (int64_t)((uint64_t)a * (uint64_t)b);
}

// the contribution of one shared y to a group (SUM part / extreme part)
__device__ __forceinline__ int64_t contrib_sum(int fn, int64_t cr, int64_t sr, int64_t cs, int64_t ss) {
    switch (fn) {
        case DIM3_FN_MUL: return mul_wrap(sr, ss);
        case DIM3_FN_ADD: return (int64_t)((uint64_t)mul_wrap(cs, sr) + (uint64_t)mul_wrap(cr, ss));
        case DIM3_FN_LEFT: return mul_wrap(cs, sr);
        default: return mul_wrap(cr, ss);
    }
}

__device__ __forceinline__ int64_t contrib_ext(int fn, bool want_min, int64_t rmn, int64_t rmx, int64_t smn,
                                               int64_t smx) {
    switch (fn) {
        case DIM3_FN_MUL: {
            const int64_t a = rmn * smn, b = rmn * smx, c = rmx * smn, d = rmx * smx;  // |.| < 2^62
            return want_min ? min64(min64(a, b), min64(c, d)) : max64(max64(a, b), max64(c, d));
        }
        case DIM3_FN_ADD: return want_min ? rmn + smn : rmx + smx;
        case DIM3_FN_LEFT: return want_min ? rmn : rmx;
        default: return want_min ? smn : smx;
    }
}

__global__ void __launch_bounds__(kThreads) k_xrow_agg(const AggArgs a) {
    __shared__ int64_t acc[kAggTile];
    __shared__ int64_t acc2[kAggTile];  // AVG: count
    __shared__ uint32_t pres[kAggTile / 32];
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    const int64_t x = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    const int64_t init = a.agg == DIM3_AGG_MIN ? INT64_MAX : (a.agg == DIM3_AGG_MAX ? INT64_MIN : 0);
    int64_t out_pos = a.off[x];
    const int32_t xv = a.dict_x[x];
    for (int64_t zt0 = 0; zt0 < a.n_z; zt0 += kAggTile) {
        const int64_t zt1 = min64(zt0 + kAggTile, a.n_z);
        const int tz = (int)(zt1 - zt0);
        for (int i = tid; i < tz; i += kThreads) {
            acc[i] = init;
            acc2[i] = 0;
        }
        for (int i = tid; i < kAggTile / 32; i += kThreads) pres[i] = 0u;
        __syncthreads();
        // one warp per distinct (x, y) of R_CSR; lanes walk S_sparse row y
        for (int64_t q = r0 + warp; q < r1; q += kThreads / 32) {
            const int32_t y = a.r_col[q];
            const int64_t cr = a.rc[q], sr = a.rs[q];
            const int64_t rmn = a.rmn[q], rmx = a.rmx[q];
            int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            if (zt0 > 0 || zt1 < a.n_z) {
                s0 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt0);
                s1 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt1);
            }
            for (int64_t j = s0 + lane; j < s1; j += 32) {
                const int z = a.ss_col[j] - (int)zt0;
                atomicOr(&pres[z >> 5], 1u << (z & 31));
                if (a.agg == DIM3_AGG_COUNT) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[z]), (unsigned long long)mul_wrap(cr, a.sc[j]));
                } else if (a.agg == DIM3_AGG_SUM || a.agg == DIM3_AGG_AVG) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[z]),
                              (unsigned long long)contrib_sum(a.fn, cr, sr, a.sc[j], a.su[j]));
                    if (a.agg == DIM3_AGG_AVG)
                        atomicAdd(reinterpret_cast<unsigned long long*>(&acc2[z]),
                                  (unsigned long long)mul_wrap(cr, a.sc[j]));
                } else {
                    const bool mn = a.agg == DIM3_AGG_MIN;
                    const int64_t c = contrib_ext(a.fn, mn, rmn, rmx, a.smn[j], a.smx[j]);
                    if (mn) atomicMin(reinterpret_cast<long long*>(&acc[z]), (long long)c);
                    else atomicMax(reinterpret_cast<long long*>(&acc[z]), (long long)c);
                }
            }
        }
        __syncthreads();
        // emit the groups of this tile in z order
        const int nw = (tz + 31) >> 5;
        for (int w0 = 0; w0 < nw; w0 += kThreads) {
            const int w = w0 + tid;
            uint32_t bits = w < nw ? pres[w] : 0u;
            int64_t total;
            const int64_t pre = block_exclusive_scan<int64_t, kThreads>(__popc(bits), &total, s_warp);
            int64_t o = out_pos + pre;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int zi = (w << 5) + b;
                a.out_x[o] = xv;
                a.out_z[o] = a.dict_z[zt0 + zi];
                if (a.agg == DIM3_AGG_AVG) a.out_f[o] = (double)acc[zi] / (double)acc2[zi];
                else a.out_i[o] = acc[zi];
                ++o;
            }
            out_pos += total;
        }
        __syncthreads();
    }
}

__global__ void k_y_stats(const int32_t* __restrict__ y_id, const int32_t* __restrict__ z_val, int64_t n, int64_t* cnt,
                          int64_t* sum, int32_t* mn, int32_t* mx) {
    GRID_STRIDE(i, n) {
        const int32_t y = y_id[i];
        if (y < 0) continue;
        const int32_t v = z_val[i];
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + y), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(sum + y), (unsigned long long)(int64_t)v);
        atomicMin(mn + y, v);
        atomicMax(mx + y, v);
    }
}

// one warp per x: fold its R_CSR row against the per-y aggregates of S
__global__ void k_groupby_fold(const int64_t* __restrict__ r_rowptr, const int32_t* __restrict__ r_col,
                               const int64_t* __restrict__ rc, int64_t n_x, const int64_t* __restrict__ yc,
                               const int64_t* __restrict__ ys, const int32_t* __restrict__ ymn,
                               const int32_t* __restrict__ ymx, const int32_t* __restrict__ dict_x, int agg,
                               int32_t* out_x, int64_t* out_i, double* out_f) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < n_x; x += warps) {
        uint64_t c = 0, sm = 0;
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int64_t q = r_rowptr[x] + lane; q < r_rowptr[x + 1]; q += 32) {
            const int32_t y = r_col[q];
            const uint64_t k = (uint64_t)rc[q];
            c += k * (uint64_t)yc[y];
            sm += k * (uint64_t)ys[y];
            mn = min64(mn, ymn[y]);
            mx = max64(mx, ymx[y]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(kFull, c, o);
            sm += __shfl_xor_sync(kFull, sm, o);
            mn = min64(mn, (int64_t)__shfl_xor_sync(kFull, (long long)mn, o));
            mx = max64(mx, (int64_t)__shfl_xor_sync(kFull, (long long)mx, o));
        }
        if (lane == 0) {
            out_x[x] = dict_x[x];
            switch (agg) {
                case DIM3_AGG_COUNT: out_i[x] = (int64_t)c; break;
                case DIM3_AGG_SUM: out_i[x] = (int64_t)sm; break;
                case DIM3_AGG_MIN: out_i[x] = mn; break;
                case DIM3_AGG_MAX: out_i[x] = mx; break;
                default: out_f[x] = (double)(int64_t)sm / (double)(int64_t)c; break;
            }
        }
    }
}

// ids of every input row against the plan's dictionaries (the plan keeps only
// the distinct pairs): y from S.y (R rows with an absent y get -1), x, z
static void row_ids(const Plan& p, const PlanInput& in, DevBuf& ry, DevBuf& rx, DevBuf& sy, DevBuf& sz,
                    cudaStream_t s) {
    ry.alloc((size_t)std::max<int64_t>(in.nr, 1) * 4, s);
    rx.alloc((size_t)std::max<int64_t>(in.nr, 1) * 4, s);
    sy.alloc((size_t)std::max<int64_t>(in.ns, 1) * 4, s);
    sz.alloc((size_t)std::max<int64_t>(in.ns, 1) * 4, s);
    if (in.nr > 0) {
        k_find_row_ids<<<grid_for(in.nr), kThreads, 0, s>>>(p.dict_y.as<int32_t>(), p.info.n_y, in.r_key, nullptr,
                                                             in.nr, ry.as<int32_t>());
        DIM3_LAUNCHED();
        k_find_row_ids<<<grid_for(in.nr), kThreads, 0, s>>>(p.dict_x.as<int32_t>(), p.info.n_x, in.r_val,
                                                             ry.as<int32_t>(), in.nr, rx.as<int32_t>());
        DIM3_LAUNCHED();
    }
    if (in.ns > 0) {
        k_find_row_ids<<<grid_for(in.ns), kThreads, 0, s>>>(p.dict_y.as<int32_t>(), p.info.n_y, in.s_key, nullptr,
                                                             in.ns, sy.as<int32_t>());
        DIM3_LAUNCHED();
        k_find_row_ids<<<grid_for(in.ns), kThreads, 0, s>>>(p.dict_z.as<int32_t>(), p.info.n_z, in.s_val, nullptr,
                                                             in.ns, sz.as<int32_t>());
        DIM3_LAUNCHED();
    }
}

int64_t join_aggregate(const Ctx& ctx, const PlanInput& in, const int32_t* r_v, const int32_t* s_u, int agg, int fn,
                       int32_t* out_x, int32_t* out_z, void* out_val, int64_t capacity, int64_t* count,
                       cudaStream_t s) {
    DIM3_REQUIRE(agg >= DIM3_AGG_COUNT && agg <= DIM3_AGG_AVG, DIM3_ERR_ARG, "unknown aggregate");
    DIM3_REQUIRE(fn >= DIM3_FN_MUL && fn <= DIM3_FN_RIGHT, DIM3_ERR_ARG, "unknown aggregate function");
    std::unique_ptr<Plan> p(build_plan(ctx, in, INT32_MAX, s));  // every z on the list path
    const int64_t n_x = p->info.n_x;
    // the groups are the Join-Project pairs: their counts give the offsets
    DevBuf cnt, off;
    cnt.alloc((size_t)std::max<int64_t>(n_x, 1) * 8, s);
    off.alloc((size_t)(n_x + 1) * 8, s);
    if (n_x > 0) plan_row_counts(ctx, *p, 0, n_x, cnt.as<int64_t>(), s);
    exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), n_x, s);
    const int64_t total = read_i64(off.as<int64_t>() + n_x, s);
    *count = total;
    if (total > capacity)
        throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) + " < result size " +
                                           std::to_string(total));
    if (total == 0) return 0;
    DIM3_REQUIRE(out_x && out_z && out_val, DIM3_ERR_ARG, "null output buffer");
    DIM3_REQUIRE(n_x < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "too many x");
    PhaseScope phase(ctx.stats, PH_EMIT, s);
    DevBuf ry, rx, sy, sz;
    row_ids(*p, in, ry, rx, sy, sz, s);
    const int bx = bits_for(p->info.n_x), by = bits_for(p->info.n_y), bz = bits_for(p->info.n_z);
    PairStats rst, sst;
    const int64_t dr = pair_stats(rx.as<int32_t>(), ry.as<int32_t>(), r_v, in.nr, by, bx + by, rst, s);
    const int64_t ds = pair_stats(sy.as<int32_t>(), sz.as<int32_t>(), s_u, in.ns, bz, by + bz, sst, s);
    DIM3_REQUIRE(dr == p->info.n_r_kept && ds == p->info.n_s_sparse, DIM3_ERR_CUDA,
                 "aggregate statistics do not line up with the plan");
    AggArgs a{};
    a.n_z = p->info.n_z;
    a.r_rowptr = p->r_rowptr.as<int64_t>();
    a.r_col = p->r_col.as<int32_t>();
    a.rc = rst.cnt.as<int64_t>();
    a.rs = rst.sum.as<int64_t>();
    a.rmn = rst.mn.as<int32_t>();
    a.rmx = rst.mx.as<int32_t>();
    a.ss_rowptr = p->ss_rowptr.as<int64_t>();
    a.ss_col = p->ss_col.as<int32_t>();
    a.sc = sst.cnt.as<int64_t>();
    a.su = sst.sum.as<int64_t>();
    a.smn = sst.mn.as<int32_t>();
    a.smx = sst.mx.as<int32_t>();
    a.dict_x = p->dict_x.as<int32_t>();
    a.dict_z = p->dict_z.as<int32_t>();
    a.off = off.as<int64_t>();
    a.agg = agg;
    a.fn = fn;
    a.out_x = out_x;
    a.out_z = out_z;
    a.out_i = agg == DIM3_AGG_AVG ? nullptr : static_cast<int64_t*>(out_val);
    a.out_f = agg == DIM3_AGG_AVG ? static_cast<double*>(out_val) : nullptr;
    k_xrow_agg<<<(unsigned)n_x, kThreads, 0, s>>>(a);
    DIM3_LAUNCHED();
    DIM3_CUDA(cudaStreamSynchronize(s));
    return total;
}

int64_t groupby_aggregate(const Ctx& ctx, const PlanInput& in, int agg, int32_t* out_x, void* out_val,
                          int64_t capacity, int64_t* count, cudaStream_t s) {
    DIM3_REQUIRE(agg >= DIM3_AGG_COUNT && agg <= DIM3_AGG_AVG, DIM3_ERR_ARG, "unknown aggregate");
    std::unique_ptr<Plan> p(build_plan(ctx, in, INT32_MAX, s));
    const int64_t n_x = p->info.n_x, n_y = p->info.n_y;
    *count = n_x;
    if (n_x > capacity)
        throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) + " < result size " +
                                           std::to_string(n_x));
    if (n_x == 0) return 0;
    DIM3_REQUIRE(out_x && out_val, DIM3_ERR_ARG, "null output buffer");
    PhaseScope phase(ctx.stats, PH_EMIT, s);
    DevBuf ry, rx, sy, sz;
    row_ids(*p, in, ry, rx, sy, sz, s);
    const int bx = bits_for(p->info.n_x), by = bits_for(p->info.n_y);
    PairStats rst;
    const int64_t dr = pair_stats(rx.as<int32_t>(), ry.as<int32_t>(), nullptr, in.nr, by, bx + by, rst, s);
    DIM3_REQUIRE(dr == p->info.n_r_kept, DIM3_ERR_CUDA, "aggregate statistics do not line up with the plan");
    // SG(y, z'): count, sum, min, max of the z values of S's rows, per y
    DevBuf yc, ys, ymn, ymx;
    yc.alloc((size_t)n_y * 8, s);
    ys.alloc((size_t)n_y * 8, s);
    ymn.alloc((size_t)n_y * 4, s);
    ymx.alloc((size_t)n_y * 4, s);
    k_seg_init<<<grid_for(n_y), kThreads, 0, s>>>(n_y, yc.as<int64_t>(), ys.as<int64_t>(), ymn.as<int32_t>(),
                                                   ymx.as<int32_t>());
    DIM3_LAUNCHED();
    if (in.ns > 0) {
        k_y_stats<<<grid_for(in.ns), kThreads, 0, s>>>(sy.as<int32_t>(), in.s_val, in.ns, yc.as<int64_t>(),
                                                        ys.as<int64_t>(), ymn.as<int32_t>(), ymx.as<int32_t>());
        DIM3_LAUNCHED();
    }
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_x, kThreads / 32), 152 * 16));
    k_groupby_fold<<<g, kThreads, 0, s>>>(p->r_rowptr.as<int64_t>(), p->r_col.as<int32_t>(), rst.cnt.as<int64_t>(), n_x,
                                           yc.as<int64_t>(), ys.as<int64_t>(), ymn.as<int32_t>(), ymx.as<int32_t>(),
                                           p->dict_x.as<int32_t>(), agg, out_x,
                                           agg == DIM3_AGG_AVG ? nullptr : static_cast<int64_t*>(out_val),
                                           agg == DIM3_AGG_AVG ? static_cast<double*>(out_val) : nullptr);
    DIM3_LAUNCHED();
    DIM3_CUDA(cudaStreamSynchronize(s));
    return n_x;
}

}  // namespace dimcube
