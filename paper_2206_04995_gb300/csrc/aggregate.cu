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

// z per SPA tile: 2048 (16 KiB of int64, 32 KiB for AVG's pairs; six CTAs
// per SM) for ranges up to 2^18 z, else 8192 (fewer tiles per row on a wide
// range, empty ones skipped)
constexpr int kAggTile = 2048;
constexpr int kAggTileWide = 8192;
constexpr int64_t kAggWideZ = int64_t(1) << 18;
constexpr int kAggLight = 512;            // join tuples of a light row (sorted in shared memory)
constexpr int kAggLightWarps = 4;         // light rows: warps per CTA

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
    const uint8_t* light;  // per x: handled by the light-row kernel (or null)
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

// the contribution of one join path group (R entry q, S entry j) to its z
struct Contribution {
    int64_t v;   // SUM / COUNT / AVG sum part, or the MIN / MAX extreme
    int64_t c;   // AVG: count part
};

__device__ __forceinline__ Contribution contribution(const AggArgs& a, int64_t q, int64_t j) {
    Contribution r{0, 0};
    const int64_t cr = a.rc[q];
    if (a.agg == DIM3_AGG_COUNT) {
        r.v = mul_wrap(cr, a.sc[j]);
    } else if (a.agg == DIM3_AGG_SUM || a.agg == DIM3_AGG_AVG) {
        r.v = contrib_sum(a.fn, cr, a.rs[q], a.sc[j], a.su[j]);
        r.c = mul_wrap(cr, a.sc[j]);
    } else {
        r.v = contrib_ext(a.fn, a.agg == DIM3_AGG_MIN, a.rmn[q], a.rmx[q], a.smn[j], a.smx[j]);
    }
    return r;
}

__device__ __forceinline__ void combine_smem(int agg, int64_t* acc, int64_t* acc2, int i, const Contribution& c) {
    if (agg == DIM3_AGG_MIN) {
        atomicMin(reinterpret_cast<long long*>(acc + i), (long long)c.v);
    } else if (agg == DIM3_AGG_MAX) {
        atomicMax(reinterpret_cast<long long*>(acc + i), (long long)c.v);
    } else {
        atomicAdd(reinterpret_cast<unsigned long long*>(acc + i), (unsigned long long)c.v);
        if (agg == DIM3_AGG_AVG) atomicAdd(reinterpret_cast<unsigned long long*>(acc2 + i), (unsigned long long)c.c);
    }
}

// Heavy rows: one CTA per x, an SPA of kAggTile z per pass (dynamic shared
// memory: accumulators, AVG counts, presence bits). Rows flagged light skip.
// Emission: a scan of the tile's presence words gives every word its output
// position; each warp then writes its words lane by bit, so a dense word
// becomes 32 consecutive outputs.
template <bool kWide>
__global__ void __launch_bounds__(kThreads) k_xrow_agg(const AggArgs a) {
    constexpr int tile = kWide ? kAggTileWide : kAggTile;
    extern __shared__ __align__(16) int64_t agg_smem[];
    int64_t* acc = agg_smem;
    int64_t* acc2 = acc + tile;  // AVG only
    uint32_t* pres = reinterpret_cast<uint32_t*>(acc + (a.agg == DIM3_AGG_AVG ? 2 * tile : tile));
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    __shared__ int32_t s_pre[tile / 32 + 1];
    const int64_t x = blockIdx.x;
    if (a.light && a.light[x]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    const int64_t init = a.agg == DIM3_AGG_MIN ? INT64_MAX : (a.agg == DIM3_AGG_MAX ? INT64_MIN : 0);
    int64_t out_pos = a.off[x];
    const int32_t xv = a.dict_x[x];
    for (int64_t zt0 = 0; zt0 < a.n_z; zt0 += tile) {
        const int64_t zt1 = min64(zt0 + (int64_t)tile, a.n_z);
        const int tz = (int)(zt1 - zt0);
        const bool part = zt0 > 0 || zt1 < a.n_z;
        if (kWide && part) {  // skip a tile none of the row's S rows reaches
            int any = 0;
            if (lane == 0) {
                for (int64_t q = r0 + warp; q < r1 && !any; q += kThreads / 32) {
                    const int32_t y = a.r_col[q];
                    const int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
                    const int64_t b0 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt0);
                    any = b0 < s1 && a.ss_col[b0] < zt1;
                }
            }
            if (!__syncthreads_or(any)) continue;
        }
        for (int i = tid; i < tz; i += kThreads) {
            acc[i] = init;
            if (a.agg == DIM3_AGG_AVG) acc2[i] = 0;
        }
        for (int i = tid; i < (tz + 31) / 32; i += kThreads) pres[i] = 0u;
        __syncthreads();
        // one warp per distinct (x, y) of R_CSR; lanes walk S_sparse row y
        for (int64_t q = r0 + warp; q < r1; q += kThreads / 32) {
            const int32_t y = a.r_col[q];
            int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            if (part) {
                s0 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt0);
                s1 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt1);
            }
            for (int64_t j = s0 + lane; j < s1; j += 32) {
                const int z = a.ss_col[j] - (int)zt0;
                atomicOr(&pres[z >> 5], 1u << (z & 31));
                combine_smem(a.agg, acc, acc2, z, contribution(a, q, j));
            }
        }
        __syncthreads();
        // emit the groups of this tile in z order
        const int nw = (tz + 31) >> 5;  // <= kThreads
        {
            const uint32_t bits = tid < nw ? pres[tid] : 0u;
            int64_t total;
            const int64_t pre = block_exclusive_scan<int64_t, kThreads>(__popc(bits), &total, s_warp);
            if (tid < nw) s_pre[tid] = (int32_t)pre;
            __syncthreads();
            const unsigned lt = lanemask_lt();
            for (int w = warp; w < nw; w += kThreads / 32) {
                const uint32_t word = pres[w];
                if (!((word >> lane) & 1u)) continue;
                const int64_t o = out_pos + s_pre[w] + __popc(word & lt);
                const int zi = (w << 5) + lane;
                a.out_x[o] = xv;
                a.out_z[o] = a.dict_z[zt0 + zi];
                if (a.agg == DIM3_AGG_AVG) a.out_f[o] = (double)acc[zi] / (double)acc2[zi];
                else a.out_i[o] = acc[zi];
            }
            out_pos += total;
        }
        __syncthreads();
    }
}

// Light rows (at most kAggLight join tuples): one warp per x gathers its
// tuples as (z id, tuple number) keys, sorts them (bitonic), numbers the
// distinct z and accumulates every tuple's contribution at its z's number.
constexpr int kAggLightWarpBytes = kAggLight * (8 + 8 + 8 + 4 + 4 + 4);  // key, acc, acc2, q, j, rank

__global__ void __launch_bounds__(kAggLightWarps * 32) k_light_agg(const AggArgs a, const int32_t* rows, int64_t n) {
    extern __shared__ __align__(16) uint64_t light_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* key = light_smem + (size_t)warp * (kAggLightWarpBytes / 8);
    int64_t* acc = reinterpret_cast<int64_t*>(key + kAggLight);
    int64_t* acc2 = acc + kAggLight;
    int32_t* tq = reinterpret_cast<int32_t*>(acc2 + kAggLight);
    int32_t* tj = tq + kAggLight;
    int32_t* rank = tj + kAggLight;
    const unsigned lt = lanemask_lt();
    const int64_t init = a.agg == DIM3_AGG_MIN ? INT64_MAX : (a.agg == DIM3_AGG_MAX ? INT64_MIN : 0);
    for (int64_t i = blockIdx.x * (int64_t)kAggLightWarps + warp; i < n; i += (int64_t)gridDim.x * kAggLightWarps) {
        const int64_t x = rows[i];
        int m = 0;
        for (int64_t q = a.r_rowptr[x]; q < a.r_rowptr[x + 1]; ++q) {
            const int32_t y = a.r_col[q];
            const int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            for (int64_t j = s0 + lane; j < s1; j += 32) {
                const int t = m + (int)(j - s0);
                key[t] = ((uint64_t)(uint32_t)a.ss_col[j] << 32) | (uint32_t)t;
                tq[t] = (int32_t)q;
                tj[t] = (int32_t)j;
            }
            m += (int)(s1 - s0);
        }
        int pw = 1;
        while (pw < m) pw <<= 1;
        for (int t = m + lane; t < pw; t += 32) key[t] = ~0ull;
        __syncwarp();
        for (int k = 2; k <= pw; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < (pw >> 1); t += 32) {
                    const int lo = (t / j) * 2 * j + (t % j), hi = lo + j;
                    const uint64_t u = key[lo], v = key[hi];
                    if ((u > v) == ((lo & k) == 0)) {
                        key[lo] = v;
                        key[hi] = u;
                    }
                }
                __syncwarp();
            }
        }
        // number the distinct z (run starts 0, 1, ...; every element takes
        // its run's number by a running max), initialise their accumulators
        int groups = 0, carry = -1;
        for (int base = 0; base < m; base += 32) {
            const int t = base + lane;
            const bool first = t < m && (t == 0 || (key[t - 1] >> 32) != (key[t] >> 32));
            const unsigned bal = __ballot_sync(kFull, first);
            const int g = groups + __popc(bal & lt);
            if (first) {
                acc[g] = init;
                acc2[g] = 0;
            }
            int r = first ? g : -1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, r, o);
                if (lane >= o) r = max(r, u);
            }
            r = max(r, carry);
            if (t < m) rank[t] = r;
            carry = __shfl_sync(kFull, r, 31);
            groups += __popc(bal);
        }
        __syncwarp();
        for (int t = lane; t < m; t += 32) {
            const int src = (int)(uint32_t)key[t];
            combine_smem(a.agg, acc, acc2, rank[t], contribution(a, tq[src], tj[src]));
        }
        __syncwarp();
        const int64_t o = a.off[x];
        const int32_t xv = a.dict_x[x];
        for (int base = 0; base < m; base += 32) {
            const int t = base + lane;
            const bool first = t < m && (t == 0 || (key[t - 1] >> 32) != (key[t] >> 32));
            if (first) {
                const int g = rank[t];
                a.out_x[o + g] = xv;
                a.out_z[o + g] = a.dict_z[(int64_t)(key[t] >> 32)];
                if (a.agg == DIM3_AGG_AVG) a.out_f[o + g] = (double)acc[g] / (double)acc2[g];
                else a.out_i[o + g] = acc[g];
            }
        }
        __syncwarp();
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

__global__ void k_light_agg_flags(const int64_t* __restrict__ outj_x, int64_t n_x, uint8_t* light, int32_t* flag) {
    GRID_STRIDE(x, n_x) {
        const bool l = outj_x[x] <= kAggLight;
        light[x] = l ? 1 : 0;
        flag[x] = l ? 1 : 0;
    }
}

__global__ void k_light_agg_list(const int32_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n,
                                 int32_t* rows) {
    GRID_STRIDE(x, n) {
        if (flag[x]) rows[pos[x]] = (int32_t)x;
    }
}

static void set_agg_attrs(const Ctx& ctx) {
    static bool done[64] = {false};
    bool& d = done[ctx.device & 63];
    if (d) return;
    const int heavy = kAggTileWide * 16 + (kAggTileWide / 32) * 4;
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_agg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, heavy));
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_agg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, heavy));
    DIM3_CUDA(cudaFuncSetAttribute(k_light_agg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kAggLightWarps * kAggLightWarpBytes));
    d = true;
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
    // light rows: at most kAggLight join tuples (outj_x counts them exactly:
    // every z is on the list path)
    DevBuf light, lflag, lpos, lrows;
    light.alloc((size_t)n_x, s);
    lflag.alloc((size_t)n_x * 4, s);
    lpos.alloc((size_t)(n_x + 1) * 8, s);
    k_light_agg_flags<<<grid_for(n_x), kThreads, 0, s>>>(p->outj_x.as<int64_t>(), n_x, light.as<uint8_t>(),
                                                          lflag.as<int32_t>());
    DIM3_LAUNCHED();
    exclusive_scan_i32_to_i64(lflag.as<int32_t>(), lpos.as<int64_t>(), n_x, s);
    const int64_t n_light = read_i64(lpos.as<int64_t>() + n_x, s);
    a.light = n_light > 0 ? light.as<uint8_t>() : nullptr;
    set_agg_attrs(ctx);
    const bool wide = a.n_z >= kAggWideZ;
    const int tile = wide ? kAggTileWide : kAggTile;
    const size_t smem = (size_t)tile * (agg == DIM3_AGG_AVG ? 16 : 8) + (size_t)(tile / 32) * 4;
    if (n_light < n_x) {
        if (wide) k_xrow_agg<true><<<(unsigned)n_x, kThreads, smem, s>>>(a);
        else k_xrow_agg<false><<<(unsigned)n_x, kThreads, smem, s>>>(a);
        DIM3_LAUNCHED();
    }
    if (n_light > 0) {
        lrows.alloc((size_t)n_light * 4, s);
        k_light_agg_list<<<grid_for(n_x), kThreads, 0, s>>>(lflag.as<int32_t>(), lpos.as<int64_t>(), n_x,
                                                             lrows.as<int32_t>());
        DIM3_LAUNCHED();
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_light, kAggLightWarps),
                                                                            152 * 32));
        k_light_agg<<<g, kAggLightWarps * 32, (size_t)kAggLightWarps * kAggLightWarpBytes, s>>>(a, lrows.as<int32_t>(),
                                                                                            n_light);
        DIM3_LAUNCHED();
    }
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
