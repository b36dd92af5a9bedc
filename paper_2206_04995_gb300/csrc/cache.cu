// Partial result caching (Section 3).
//
// Building a cache: the per-z statistics come from a plan of the transposed
// query Pi_{z,x}(S(z,y) join_y R(x,y)), whose rows are the z: its counting
// pass gives k(z) = |{x : (x, z) in the result}| and its per-row join-tuple
// counts give n_join(z) = sum over S(z) of deg_R(y). CacheScore(z) =
// cost(z) / space(z) in float64 with space(z) = 2 + min(k, |X| - k) and
// cost(z) = n_join(z) * t_sparse for a sparse z, |X| * t_dense for a dense z
// (m_z >= theta_z, one DenseEC evaluation per x). The z are radix-sorted by
// descending score (stable, so ties stay in ascending z order) and the longest
// prefix whose running space fits the budget is cached. The entries come from
// a second transposed plan restricted to the cached z: the x list of a z, or,
// when k > |X| / 2, its complement in X (from a bitmap over X per entry).
//
// Using a cache: the plan builder drops the S tuples of cached z after mapping
// and appends the cached z to the dense z index, so the union step of every
// SparseBMM kernel picks them up from the dense-result rows; cache_expand
// fills those columns (complement columns set, then list members set or, for
// complements, cleared).
#include <algorithm>
#include <cmath>
#include <cstring>
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

static int read_flag(const DevBuf& f, cudaStream_t s) {
    int h = 0;
    DIM3_CUDA(cudaMemcpyAsync(&h, f.p, 4, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    return h;
}

// ids[i] = position of vals[i] in the ascending dict; a value missing from it
// sets *bad (and gets -1)
__global__ void k_find_ids(const int32_t* __restrict__ dict, int64_t n_dict, const int32_t* __restrict__ vals,
                           int64_t n, int32_t* __restrict__ ids, int* bad) {
    GRID_STRIDE(i, n) {
        const int32_t v = vals[i];
        const int64_t j = lower_bound_dev<int32_t>(dict, 0, n_dict, v);
        if (j < n_dict && dict[j] == v) {
            ids[i] = (int32_t)j;
        } else {
            ids[i] = -1;
            *bad = 1;
        }
    }
}

__global__ void k_mark_ids(const int32_t* __restrict__ ids, int64_t n, uint8_t* flag) {
    GRID_STRIDE(i, n) flag[ids[i]] = 1;
}

__global__ void k_drop_marked(int32_t* col, int64_t n, const uint8_t* __restrict__ flag) {
    GRID_STRIDE(i, n) {
        const int32_t v = col[i];
        if (v >= 0 && flag[v]) col[i] = -1;
    }
}

// entry of list element j: the e with off[e] <= j < off[e + 1]
__global__ void k_entry_of(const int64_t* __restrict__ off, int64_t n_c, int64_t n_list, int32_t* ent) {
    GRID_STRIDE(j, n_list) ent[j] = (int32_t)(lower_bound_dev<int64_t>(off, 0, n_c + 1, j + 1) - 1);
}

void attach_cache_ids(Plan& p, const ResultCache& c, int32_t* sz_id, int64_t ns, cudaStream_t s) {
    DIM3_REQUIRE(c.n_x == p.info.n_x, DIM3_ERR_ARG, "the cache was built on other tables (|X| differs)");
    const int64_t n_z = p.info.n_z;
    DevBuf bad, flag;
    bad.alloc(4, s);
    DIM3_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    p.n_zc = c.n_c;
    p.zc_nlist = c.n_list;
    p.zc_zid.alloc((size_t)std::max<int64_t>(c.n_c, 1) * 4, s);
    if (c.n_c > 0) {
        k_find_ids<<<grid_for(c.n_c), kThreads, 0, s>>>(p.dict_z.as<int32_t>(), n_z, c.z.as<int32_t>(), c.n_c,
                                                         p.zc_zid.as<int32_t>(), bad.as<int>());
        DIM3_LAUNCHED();
    }
    p.zc_xid.alloc((size_t)std::max<int64_t>(c.n_list, 1) * 4, s);
    p.zc_ent.alloc((size_t)std::max<int64_t>(c.n_list, 1) * 4, s);
    if (c.n_list > 0) {
        k_find_ids<<<grid_for(c.n_list), kThreads, 0, s>>>(p.dict_x.as<int32_t>(), p.info.n_x, c.xs.as<int32_t>(),
                                                            c.n_list, p.zc_xid.as<int32_t>(), bad.as<int>());
        DIM3_LAUNCHED();
        k_entry_of<<<grid_for(c.n_list), kThreads, 0, s>>>(c.off.as<int64_t>(), c.n_c, c.n_list,
                                                            p.zc_ent.as<int32_t>());
        DIM3_LAUNCHED();
    }
    DIM3_REQUIRE(read_flag(bad, s) == 0, DIM3_ERR_ARG, "the cache was built on other tables (a value is missing)");
    p.zc_comp.alloc((size_t)std::max<int64_t>(c.n_c, 1), s);
    if (c.n_c > 0) {
        DIM3_CUDA(cudaMemcpyAsync(p.zc_comp.p, c.comp.p, (size_t)c.n_c, cudaMemcpyDeviceToDevice, s));
        flag.alloc((size_t)std::max<int64_t>(n_z, 1), s);
        DIM3_CUDA(cudaMemsetAsync(flag.p, 0, (size_t)std::max<int64_t>(n_z, 1), s));
        k_mark_ids<<<grid_for(c.n_c), kThreads, 0, s>>>(p.zc_zid.as<int32_t>(), c.n_c, flag.as<uint8_t>());
        DIM3_LAUNCHED();
        if (ns > 0) {
            k_drop_marked<<<grid_for(ns), kThreads, 0, s>>>(sz_id, ns, flag.as<uint8_t>());
            DIM3_LAUNCHED();
        }
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_extend_zd_list(const int32_t* __restrict__ old, int64_t n_zd, int64_t zc_off,
                                 const int32_t* __restrict__ zc_zid, int64_t total, int32_t* out) {
    GRID_STRIDE(i, total) out[i] = i < n_zd ? old[i] : (i < zc_off ? -1 : zc_zid[i - zc_off]);
}

__global__ void k_comp_mask(const uint8_t* __restrict__ comp, int64_t n_c, uint32_t* mask, int64_t n_w) {
    GRID_STRIDE(w, n_w) {
        uint32_t m = 0u;
        for (int b = 0; b < 32; ++b) {
            const int64_t e = w * 32 + b;
            if (e < n_c && comp[e]) m |= 1u << b;
        }
        mask[w] = m;
    }
}

void finish_cache_index(Plan& p, cudaStream_t s) {
    const int64_t n_zd = p.info.n_z_dense;
    p.zc_off = n_zd > 0 ? p.n_zd_pad : 0;  // a multiple of the tensor-core tile: whole words
    const int64_t total = p.zc_off + p.n_zc;
    p.n_zd_total = total;
    p.zdw = ceil_div(total, 32);
    p.info.n_z_cached = p.n_zc;
    DevBuf zl;
    zl.alloc((size_t)std::max<int64_t>(total, 1) * 4, s);
    if (total > 0) {
        k_extend_zd_list<<<grid_for(total), kThreads, 0, s>>>(p.zd_list.as<int32_t>(), n_zd, p.zc_off,
                                                               p.zc_zid.as<int32_t>(), total, zl.as<int32_t>());
        DIM3_LAUNCHED();
    }
    p.zd_list = std::move(zl);
    p.h_inst_zd_lo.assign(2, 0);
    p.h_inst_zd_lo[1] = total;
    store_i64_pair(p.inst_zd_lo.as<int64_t>(), 0, total, s);
    const int64_t n_w = ceil_div(p.n_zc, 32);
    p.zc_cmask.alloc((size_t)std::max<int64_t>(n_w, 1) * 4, s);
    if (n_w > 0) {
        k_comp_mask<<<grid_for(n_w), kThreads, 0, s>>>(p.zc_comp.as<uint8_t>(), p.n_zc, p.zc_cmask.as<uint32_t>(), n_w);
        DIM3_LAUNCHED();
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
}

// complement columns: every row starts with the bit set
__global__ void k_cache_fill(uint32_t* d_bits, int64_t rows, int64_t zdw, int64_t w0, int64_t n_w,
                             const uint32_t* __restrict__ mask) {
    GRID_STRIDE(i, rows * n_w) {
        const int64_t r = i / n_w, w = i - r * n_w;
        const uint32_t m = mask[w];
        if (m) d_bits[r * zdw + w0 + w] |= m;
    }
}

// list members: set (list entry) or clear (complement entry) their bit
__global__ void k_cache_scatter(const int32_t* __restrict__ xid, const int32_t* __restrict__ ent, int64_t n_list,
                                const uint8_t* __restrict__ comp, int64_t x_begin, int64_t rows, int64_t zc_off,
                                int64_t zdw, uint32_t* d_bits) {
    GRID_STRIDE(j, n_list) {
        const int64_t x = xid[j];
        if (x < x_begin || x >= x_begin + rows) continue;
        const int32_t e = ent[j];
        const int64_t col = zc_off + e;
        uint32_t* wp = d_bits + (x - x_begin) * zdw + (col >> 5);
        const uint32_t bit = 1u << (col & 31);
        if (comp[e]) atomicAnd(wp, ~bit);
        else atomicOr(wp, bit);
    }
}

void cache_expand(const Plan& p, int64_t x_begin, int64_t rows, uint32_t* d_bits, cudaStream_t s) {
    if (p.n_zc == 0 || rows <= 0) return;
    const int64_t w0 = p.zc_off >> 5, n_w = ceil_div(p.n_zc, 32);
    k_cache_fill<<<grid_for(rows * n_w), kThreads, 0, s>>>(d_bits, rows, p.zdw, w0, n_w, p.zc_cmask.as<uint32_t>());
    DIM3_LAUNCHED();
    if (p.zc_nlist > 0) {
        k_cache_scatter<<<grid_for(p.zc_nlist), kThreads, 0, s>>>(p.zc_xid.as<int32_t>(), p.zc_ent.as<int32_t>(),
                                                                   p.zc_nlist, p.zc_comp.as<uint8_t>(), x_begin, rows,
                                                                   p.zc_off, p.zdw, d_bits);
        DIM3_LAUNCHED();
    }
}

// ------------------------------------------------------------------ build
// k and n_join of the original plan's z from the transposed plan's rows
__global__ void k_scatter_stats(const int32_t* __restrict__ t_dict, const int64_t* __restrict__ t_cnt,
                                const int64_t* __restrict__ t_outj, int64_t rows_t, const int32_t* __restrict__ dict_z,
                                int64_t n_z, int64_t* k, int64_t* n_join, int* bad) {
    GRID_STRIDE(r, rows_t) {
        const int32_t v = t_dict[r];
        const int64_t j = lower_bound_dev<int32_t>(dict_z, 0, n_z, v);
        if (j < n_z && dict_z[j] == v) {
            k[j] = t_cnt[r];
            n_join[j] = t_outj[r];
        } else {
            *bad = 1;
        }
    }
}

// CacheScore per z and the sort key of the ranking (descending score: the
// bits of a non-negative double, inverted)
__global__ void k_scores(const int64_t* __restrict__ k, const int64_t* __restrict__ n_join,
                         const uint8_t* __restrict__ dense, int64_t n_z, int64_t n_x, double t_sparse, double t_dense,
                         int64_t* space, uint64_t* key, uint32_t* idx) {
    GRID_STRIDE(z, n_z) {
        const int64_t kz = k[z];
        const int64_t sp = 2 + min64(kz, n_x - kz);
        double cost;
        if (dense[z]) cost = __dmul_rn((double)n_x, t_dense);
        else cost = __dmul_rn((double)n_join[z], t_sparse);
        const double score = __ddiv_rn(cost, (double)sp);
        space[z] = sp;
        key[z] = ~(uint64_t)__double_as_longlong(score);
        idx[z] = (uint32_t)z;
    }
}

__global__ void k_gather_space(const uint32_t* __restrict__ idx, const int64_t* __restrict__ space, int64_t n,
                               int64_t* out) {
    GRID_STRIDE(i, n) out[i] = space[idx[i]];
}

// number of ranked z whose running space (incl[i] = cum[i + 1]) is <= budget
__global__ void k_prefix_fit(const int64_t* cum, int64_t n, int64_t budget, int64_t* n_take) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t lo = 0, hi = n;  // first i with cum[i + 1] > budget
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid + 1] <= budget) lo = mid + 1;
            else hi = mid;
        }
        *n_take = lo;
    }
}

__global__ void k_select_flags(const uint32_t* __restrict__ idx, int64_t n_take, int32_t* flag) {
    GRID_STRIDE(i, n_take) flag[idx[i]] = 1;
}

__global__ void k_entries(const int32_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n_z,
                          const int64_t* __restrict__ k, const int32_t* __restrict__ dict_z, int64_t n_x,
                          int32_t* zval, int32_t* zidx, int64_t* size, uint8_t* comp, int64_t* len, int64_t* space) {
    GRID_STRIDE(z, n_z) {
        if (!flag[z]) continue;
        const int64_t e = pos[z];
        const int64_t kz = k[z];
        const bool c = 2 * kz > n_x;
        zval[e] = dict_z[z];
        zidx[e] = (int32_t)z;
        size[e] = c ? kz - n_x : kz;
        comp[e] = c ? 1 : 0;
        len[e] = c ? n_x - kz : kz;
        space[e] = 2 + min64(kz, n_x - kz);
    }
}

// S rows whose z is cached (binary search in the ascending cached values)
__global__ void k_flag_cached_s(const int32_t* __restrict__ s_val, int64_t ns, const int32_t* __restrict__ zval,
                                int64_t n_c, int32_t* flag) {
    GRID_STRIDE(i, ns) {
        const int32_t v = s_val[i];
        const int64_t j = lower_bound_dev<int32_t>(zval, 0, n_c, v);
        flag[i] = (j < n_c && zval[j] == v) ? 1 : 0;
    }
}

__global__ void k_compact_pair(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n,
                               const int32_t* __restrict__ flag, const int64_t* __restrict__ pos, int32_t* oa,
                               int32_t* ob) {
    GRID_STRIDE(i, n) {
        if (flag[i]) {
            oa[pos[i]] = a[i];
            ob[pos[i]] = b[i];
        }
    }
}

// row r of the restricted transposed plan -> its entry; list entries copy the
// row's x values, complement entries mark them in their bitmap over X
__global__ void k_fill_lists(const int32_t* __restrict__ c_dict, int64_t rows_c, const int64_t* __restrict__ roff,
                             const int32_t* __restrict__ pair_x, const int32_t* __restrict__ zval, int64_t n_c,
                             const uint8_t* __restrict__ comp, const int64_t* __restrict__ comp_pos,
                             const int64_t* __restrict__ off, const int32_t* __restrict__ dict_x, int64_t n_x,
                             int32_t* xs, uint32_t* cbits, int64_t xw, int* bad) {
    for (int64_t r = blockIdx.x; r < rows_c; r += gridDim.x) {
        const int32_t zv = c_dict[r];
        const int64_t e = lower_bound_dev<int32_t>(zval, 0, n_c, zv);
        if (e >= n_c || zval[e] != zv) {
            if (threadIdx.x == 0) *bad = 1;
            continue;
        }
        const int64_t q0 = roff[r], q1 = roff[r + 1];
        if (!comp[e]) {
            if (q1 - q0 != off[e + 1] - off[e]) {
                if (threadIdx.x == 0) *bad = 1;
                continue;
            }
            for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) xs[off[e] + (q - q0)] = pair_x[q];
        } else {
            uint32_t* bm = cbits + comp_pos[e] * xw;
            for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                const int32_t v = pair_x[q];
                const int64_t j = lower_bound_dev<int32_t>(dict_x, 0, n_x, v);
                if (j < n_x && dict_x[j] == v) atomicOr(&bm[j >> 5], 1u << (j & 31));
                else *bad = 1;
            }
        }
    }
}

// complement entries: the x of X whose bit is clear, ascending
__global__ void __launch_bounds__(kThreads) k_emit_complements(const uint8_t* __restrict__ comp,
                                                               const int64_t* __restrict__ comp_pos, int64_t n_c,
                                                               const uint32_t* __restrict__ cbits, int64_t xw,
                                                               int64_t n_x, const int32_t* __restrict__ dict_x,
                                                               const int64_t* __restrict__ off, int32_t* xs, int* bad) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    for (int64_t e = blockIdx.x; e < n_c; e += gridDim.x) {
        if (!comp[e]) continue;
        const uint32_t* bm = cbits + comp_pos[e] * xw;
        int64_t base = off[e];
        for (int64_t w0 = 0; w0 < xw; w0 += kThreads) {
            const int64_t w = w0 + threadIdx.x;
            uint32_t free_bits = 0u;
            if (w < xw) {
                free_bits = ~bm[w];
                const int64_t hi = n_x - w * 32;  // valid bits in this word
                if (hi < 32) free_bits &= (1u << hi) - 1u;
            }
            int64_t total;
            const int64_t pre = block_exclusive_scan<int64_t, kThreads>(__popc(free_bits), &total, s_warp);
            int64_t o = base + pre;
            while (free_bits) {
                const int b = __ffs(free_bits) - 1;
                free_bits &= free_bits - 1;
                xs[o++] = dict_x[w * 32 + b];
            }
            base += total;
        }
        if (threadIdx.x == 0 && base != off[e + 1]) *bad = 1;
    }
}

ResultCache* build_result_cache(const Ctx& ctx, const PlanInput& in, int64_t theta_z, int64_t budget,
                                double t_sparse, double t_dense, cudaStream_t s) {
    DIM3_REQUIRE(in.n_inst <= 1 && !in.premapped && !in.cache, DIM3_ERR_ARG, "a cache is built on one instance");
    DIM3_REQUIRE(budget >= 0, DIM3_ERR_ARG, "negative cache budget");
    DIM3_REQUIRE(std::isfinite(t_sparse) && std::isfinite(t_dense) && t_sparse >= 0.0 && t_dense >= 0.0,
                 DIM3_ERR_ARG, "cost constants must be finite and non-negative");
    std::unique_ptr<Plan> p(build_plan(ctx, in, theta_z, s));
    const int64_t n_x = p->info.n_x, n_z = p->info.n_z;
    std::unique_ptr<ResultCache> c(new ResultCache());
    c->n_x = n_x;
    DevBuf bad;
    bad.alloc(4, s);
    DIM3_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));

    // per-z statistics from the transposed plan: rows are the z
    DevBuf k, nj;
    k.alloc((size_t)std::max<int64_t>(n_z, 1) * 8, s);
    nj.alloc((size_t)std::max<int64_t>(n_z, 1) * 8, s);
    DIM3_CUDA(cudaMemsetAsync(k.p, 0, k.bytes, s));
    DIM3_CUDA(cudaMemsetAsync(nj.p, 0, nj.bytes, s));
    {
        PlanInput t;
        t.r_key = in.s_key;
        t.r_val = in.s_val;
        t.nr = in.ns;
        t.s_key = in.r_key;
        t.s_val = in.r_val;
        t.ns = in.nr;
        std::unique_ptr<Plan> pt(build_plan(ctx, t, INT32_MAX, s));
        const int64_t rows_t = pt->info.n_x;
        if (rows_t > 0) {
            DevBuf cnt;
            cnt.alloc((size_t)rows_t * 8, s);
            plan_row_counts(ctx, *pt, 0, rows_t, cnt.as<int64_t>(), s);
            k_scatter_stats<<<grid_for(rows_t), kThreads, 0, s>>>(pt->dict_x.as<int32_t>(), cnt.as<int64_t>(),
                                                                   pt->outj_x.as<int64_t>(), rows_t,
                                                                   p->dict_z.as<int32_t>(), n_z, k.as<int64_t>(),
                                                                   nj.as<int64_t>(), bad.as<int>());
            DIM3_LAUNCHED();
            DIM3_CUDA(cudaStreamSynchronize(s));
        }
    }

    // ranking and selection
    int64_t n_take = 0;
    DevBuf flag, pos;
    flag.alloc((size_t)std::max<int64_t>(n_z, 1) * 4, s);
    pos.alloc((size_t)(n_z + 1) * 8, s);
    DIM3_CUDA(cudaMemsetAsync(flag.p, 0, flag.bytes, s));
    if (n_z > 0) {
        DevBuf space, key, idx, key_alt, idx_alt, ranked, cum, take;
        space.alloc((size_t)n_z * 8, s);
        key.alloc((size_t)n_z * 8, s);
        idx.alloc((size_t)n_z * 4, s);
        key_alt.alloc((size_t)n_z * 8, s);
        idx_alt.alloc((size_t)n_z * 4, s);
        k_scores<<<grid_for(n_z), kThreads, 0, s>>>(k.as<int64_t>(), nj.as<int64_t>(), p->dense_z.as<uint8_t>(), n_z,
                                                     n_x, t_sparse, t_dense, space.as<int64_t>(), key.as<uint64_t>(),
                                                     idx.as<uint32_t>());
        DIM3_LAUNCHED();
        radix_sort_u64(key.as<uint64_t>(), idx.as<uint32_t>(), key_alt.as<uint64_t>(), idx_alt.as<uint32_t>(), n_z, 64,
                       s);
        ranked.alloc((size_t)n_z * 8, s);
        cum.alloc((size_t)(n_z + 1) * 8, s);
        take.alloc(8, s);
        k_gather_space<<<grid_for(n_z), kThreads, 0, s>>>(idx.as<uint32_t>(), space.as<int64_t>(), n_z,
                                                           ranked.as<int64_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i64(ranked.as<int64_t>(), cum.as<int64_t>(), n_z, s);
        k_prefix_fit<<<1, 32, 0, s>>>(cum.as<int64_t>(), n_z, budget, take.as<int64_t>());
        DIM3_LAUNCHED();
        n_take = read_i64(take.as<int64_t>(), s);
        if (n_take > 0) {
            k_select_flags<<<grid_for(n_take), kThreads, 0, s>>>(idx.as<uint32_t>(), n_take, flag.as<int32_t>());
            DIM3_LAUNCHED();
        }
        exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos.as<int64_t>(), n_z, s);
    }
    const int64_t n_c = n_take;
    c->n_c = n_c;
    c->z.alloc((size_t)std::max<int64_t>(n_c, 1) * 4, s);
    c->size.alloc((size_t)std::max<int64_t>(n_c, 1) * 8, s);
    c->comp.alloc((size_t)std::max<int64_t>(n_c, 1), s);
    c->off.alloc((size_t)(n_c + 1) * 8, s);
    DIM3_CUDA(cudaMemsetAsync(c->off.p, 0, 8, s));
    if (n_c == 0) {
        c->xs.alloc(4, s);
        DIM3_REQUIRE(read_flag(bad, s) == 0, DIM3_ERR_CUDA, "cache statistics: inconsistent transposed plan");
        return c.release();
    }
    DevBuf zidx, len, espace, esum;
    zidx.alloc((size_t)n_c * 4, s);
    len.alloc((size_t)n_c * 8, s);
    espace.alloc((size_t)n_c * 8, s);
    k_entries<<<grid_for(n_z), kThreads, 0, s>>>(flag.as<int32_t>(), pos.as<int64_t>(), n_z, k.as<int64_t>(),
                                                  p->dict_z.as<int32_t>(), n_x, c->z.as<int32_t>(), zidx.as<int32_t>(),
                                                  c->size.as<int64_t>(), c->comp.as<uint8_t>(), len.as<int64_t>(),
                                                  espace.as<int64_t>());
    DIM3_LAUNCHED();
    exclusive_scan_i64(len.as<int64_t>(), c->off.as<int64_t>(), n_c, s);
    esum.alloc((size_t)(n_c + 1) * 8, s);
    exclusive_scan_i64(espace.as<int64_t>(), esum.as<int64_t>(), n_c, s);
    c->space = read_i64(esum.as<int64_t>() + n_c, s);
    c->n_list = read_i64(c->off.as<int64_t>() + n_c, s);
    c->xs.alloc((size_t)std::max<int64_t>(c->n_list, 1) * 4, s);

    // complement entries: one bitmap over X each
    DevBuf cflag, cpos;
    cflag.alloc((size_t)n_c * 4, s);
    cpos.alloc((size_t)(n_c + 1) * 8, s);
    {
        std::vector<uint8_t> hc((size_t)n_c);
        DIM3_CUDA(cudaMemcpyAsync(hc.data(), c->comp.p, (size_t)n_c, cudaMemcpyDeviceToHost, s));
        DIM3_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> hf(hc.begin(), hc.end());
        DIM3_CUDA(cudaMemcpyAsync(cflag.p, hf.data(), (size_t)n_c * 4, cudaMemcpyHostToDevice, s));
        DIM3_CUDA(cudaStreamSynchronize(s));
    }
    exclusive_scan_i32_to_i64(cflag.as<int32_t>(), cpos.as<int64_t>(), n_c, s);
    const int64_t n_comp = read_i64(cpos.as<int64_t>() + n_c, s);
    const int64_t xw = ceil_div(n_x, 32);
    DIM3_REQUIRE((double)n_comp * (double)xw * 4.0 < 32e9, DIM3_ERR_OVERFLOW, "complement bitmaps too large");
    DevBuf cbits;
    cbits.alloc((size_t)std::max<int64_t>(n_comp * xw, 1) * 4, s);
    DIM3_CUDA(cudaMemsetAsync(cbits.p, 0, cbits.bytes, s));

    // the cached z's results: transposed plan over the S tuples of cached z
    {
        DevBuf sflag, spos, sy, sz;
        const int64_t ns = in.ns;
        sflag.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        spos.alloc((size_t)(ns + 1) * 8, s);
        int64_t nsc = 0;
        if (ns > 0) {
            k_flag_cached_s<<<grid_for(ns), kThreads, 0, s>>>(in.s_val, ns, c->z.as<int32_t>(), n_c,
                                                               sflag.as<int32_t>());
            DIM3_LAUNCHED();
            exclusive_scan_i32_to_i64(sflag.as<int32_t>(), spos.as<int64_t>(), ns, s);
            nsc = read_i64(spos.as<int64_t>() + ns, s);
        }
        sy.alloc((size_t)std::max<int64_t>(nsc, 1) * 4, s);
        sz.alloc((size_t)std::max<int64_t>(nsc, 1) * 4, s);
        if (nsc > 0) {
            k_compact_pair<<<grid_for(ns), kThreads, 0, s>>>(in.s_key, in.s_val, ns, sflag.as<int32_t>(),
                                                              spos.as<int64_t>(), sy.as<int32_t>(), sz.as<int32_t>());
            DIM3_LAUNCHED();
            PlanInput t;
            t.r_key = sy.as<int32_t>();
            t.r_val = sz.as<int32_t>();
            t.nr = nsc;
            t.s_key = in.r_key;
            t.s_val = in.r_val;
            t.ns = in.nr;
            std::unique_ptr<Plan> pc(build_plan(ctx, t, INT32_MAX, s));
            const int64_t rows_c = pc->info.n_x;
            if (rows_c > 0) {
                DevBuf cnt, roff, pz, px;
                cnt.alloc((size_t)rows_c * 8, s);
                roff.alloc((size_t)(rows_c + 1) * 8, s);
                plan_row_counts(ctx, *pc, 0, rows_c, cnt.as<int64_t>(), s);
                exclusive_scan_i64(cnt.as<int64_t>(), roff.as<int64_t>(), rows_c, s);
                const int64_t n_pairs = read_i64(roff.as<int64_t>() + rows_c, s);
                pz.alloc((size_t)std::max<int64_t>(n_pairs, 1) * 4, s);
                px.alloc((size_t)std::max<int64_t>(n_pairs, 1) * 4, s);
                int64_t got = 0;
                if (n_pairs > 0)
                    plan_join(ctx, *pc, 0, rows_c, 0, pz.as<int32_t>(), px.as<int32_t>(), nullptr, n_pairs, &got, s);
                DIM3_REQUIRE(got == n_pairs, DIM3_ERR_CUDA, "cache entries: inconsistent pair count");
                const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows_c, 152 * 8));
                k_fill_lists<<<g, kThreads, 0, s>>>(pc->dict_x.as<int32_t>(), rows_c, roff.as<int64_t>(),
                                                     px.as<int32_t>(), c->z.as<int32_t>(), n_c, c->comp.as<uint8_t>(),
                                                     cpos.as<int64_t>(), c->off.as<int64_t>(), p->dict_x.as<int32_t>(),
                                                     n_x, c->xs.as<int32_t>(), cbits.as<uint32_t>(), xw,
                                                     bad.as<int>());
                DIM3_LAUNCHED();
            }
        }
    }
    if (n_comp > 0) {
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n_c, 152 * 8));
        k_emit_complements<<<g, kThreads, 0, s>>>(c->comp.as<uint8_t>(), cpos.as<int64_t>(), n_c, cbits.as<uint32_t>(),
                                                   xw, n_x, p->dict_x.as<int32_t>(), c->off.as<int64_t>(),
                                                   c->xs.as<int32_t>(), bad.as<int>());
        DIM3_LAUNCHED();
    }
    DIM3_REQUIRE(read_flag(bad, s) == 0, DIM3_ERR_CUDA, "cache entries: inconsistent transposed plans");
    return c.release();
}

}  // namespace dimcube
