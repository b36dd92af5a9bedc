// Steps 2-3 of Algorithm 1: R_CSR by x, degrees, and the intersection-free
// partition of S by z (Section 2.3) into S_sparse (CSR by y, Section 2.4) and
// S_dense (Section 2.5).
//
// Tuples are packed into one integer key (row id in the high bits, column id
// in the low bits) and radix-sorted; adjacent duplicates are dropped, which
// applies set semantics, and CSR row pointers come from binary searches over
// the sorted keys. Every z is judged once (dense iff m_z >= theta_z), so all
// tuples of one z land on the same side and the two results are disjoint.
#include <algorithm>
#include <climits>
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

// Append key = (a << shift) | b for rows with a >= 0 and b >= 0 (unordered;
// a sort follows).
template <typename K>
__global__ void k_pack_pairs(const int32_t* a, const int32_t* b, int64_t n, int shift, K* keys,
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
        if (ok) keys[pos] = ((K)(uint32_t)av << shift) | (K)(uint32_t)bv;
    }
}

template <typename K>
__global__ void k_split_low(const K* keys, int64_t n, K mask, int32_t* col) {
    GRID_STRIDE(i, n) col[i] = (int32_t)(keys[i] & mask);
}

template <typename K>
__global__ void k_hist_low(const K* keys, int64_t n, K mask, int32_t* hist) {
    GRID_STRIDE(i, n) atomicAdd(&hist[(int64_t)(keys[i] & mask)], 1);
}

__global__ void k_row_len(const int64_t* rowptr, int64_t n_rows, int32_t* len) {
    GRID_STRIDE(r, n_rows) len[r] = (int32_t)(rowptr[r + 1] - rowptr[r]);
}

// join tuples per x: sum of deg_S(y) over y in R[x]
// one warp per x (rows are power-law in graphs: a thread per row stalls on hubs)
__global__ void k_outj_x(const int64_t* r_rowptr, const int32_t* r_col, int64_t n_x, const int32_t* deg_s,
                         int64_t* outj_x) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < n_x; x += warps) {
        int64_t acc = 0;
        for (int64_t p = r_rowptr[x] + lane; p < r_rowptr[x + 1]; p += 32) acc += deg_s[r_col[p]];
        acc = warp_sum(acc);
        if (lane == 0) outj_x[x] = acc;
    }
}

__global__ void k_dense_flags(const int32_t* m_z, int64_t n_z, int64_t theta, uint8_t* dense_u8, int32_t* flag) {
    GRID_STRIDE(z, n_z) {
        const bool d = (int64_t)m_z[z] >= theta;
        dense_u8[z] = d ? 1 : 0;
        flag[z] = d ? 1 : 0;
    }
}

// dense index of every dense z (order-preserving compaction of the flags)
__global__ void k_zd_list(const int32_t* flag, const int64_t* pos, int64_t n_z, int32_t* zd_list, int32_t* zd_index) {
    GRID_STRIDE(z, n_z) {
        if (flag[z]) {
            zd_list[pos[z]] = (int32_t)z;
            zd_index[z] = (int32_t)pos[z];
        } else {
            zd_index[z] = -1;
        }
    }
}

template <typename K>
__global__ void k_sparse_flags(const K* keys, int64_t n, K zmask, const uint8_t* dense_u8, int32_t* flag) {
    GRID_STRIDE(i, n) flag[i] = dense_u8[(int64_t)(keys[i] & zmask)] ? 0 : 1;
}

template <typename K>
__global__ void k_compact(const K* in, int64_t n, const int32_t* flag, const int64_t* pos, K* out) {
    GRID_STRIDE(i, n) if (flag[i]) out[pos[i]] = in[i];
}

// word window of instance t: [floor32(z_lo[t]), z_lo[t + 1])
__device__ __forceinline__ int64_t window_words(const int64_t* z_lo, int t) {
    const int64_t lo = z_lo[t] & ~int64_t(31);
    return (z_lo[t + 1] - lo + 31) >> 5;
}

// Wide S_sparse rows: flag and words of the bitmap of every wide row.
__global__ void k_wide_rows(const int64_t* rowptr, int64_t n_rows, const int32_t* y_tag, const int64_t* z_lo,
                            int64_t fixed_min, int64_t mult, int32_t* flag, int64_t* words) {
    GRID_STRIDE(r, n_rows) {
        const int t = y_tag ? y_tag[r] : 0;
        const int64_t ww = window_words(z_lo, t);
        const int64_t thr = fixed_min >= 0 ? fixed_min * mult : max64(ww, 8) * mult;
        const bool wide = (rowptr[r + 1] - rowptr[r]) >= max64(thr, 1);
        flag[r] = wide ? 1 : 0;
        words[r] = wide ? ww : 0;
    }
}

// bm_off[b] = first word of wide row b (b = position among the flagged rows)
__global__ void k_row_offsets(const int32_t* flag, const int64_t* pos, const int64_t* wpos, int64_t n, int64_t* off) {
    GRID_STRIDE(r, n + 1) {
        if (r == n) off[pos[n]] = wpos[n];
        else if (flag[r]) off[pos[r]] = wpos[r];
    }
}

// per-instance id ranges of a tag array sorted ascending: lo[t] = first index with tag >= t
__global__ void k_tag_ranges(const int32_t* tags, int64_t n, int n_inst, int64_t* lo) {
    GRID_STRIDE(t, (int64_t)n_inst + 1) {
        int64_t a = 0, b = n;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (tags[m] < t) a = m + 1; else b = m;
        }
        lo[t] = a;
    }
}

__global__ void k_gather_tags(const int32_t* idx, int64_t n, const int32_t* tag_of, int32_t* out) {
    GRID_STRIDE(i, n) out[i] = tag_of[idx[i]];
}

__global__ void k_index_from_flags(const int32_t* flag, const int64_t* pos, int64_t n, int32_t* idx) {
    GRID_STRIDE(i, n) idx[i] = flag[i] ? (int32_t)pos[i] : -1;
}

// bitmap rows of the wide S_sparse rows
template <typename K>
__global__ void k_fill_row_bits(const K* keys, int64_t n, int bz, K zmask, const int32_t* row_of_y,
                                const int64_t* bm_off, const int32_t* y_tag, const int64_t* z_lo, uint32_t* bits) {
    GRID_STRIDE(i, n) {
        const K k = keys[i];
        const int64_t y = (int64_t)(k >> bz);
        const int32_t b = row_of_y[y];
        if (b >= 0) {
            const int t = y_tag ? y_tag[y] : 0;
            const int64_t z = (int64_t)(k & zmask) - (z_lo[t] & ~int64_t(31));
            atomicOr(&bits[bm_off[b] + (z >> 5)], 1u << (z & 31));
        }
    }
}

template <typename K>
__global__ void k_mark_dense_y(const K* keys, int64_t n, int bz, K zmask, const uint8_t* dense_u8, int32_t* flag_y) {
    GRID_STRIDE(i, n) {
        const K k = keys[i];
        if (dense_u8[(int64_t)(k & zmask)]) flag_y[(int64_t)(k >> bz)] = 1;
    }
}

// ------------------------------------------------------------------------
template <typename K>
struct SortedPairs {
    DevBuf keys;  // sorted unique
    int64_t n = 0;
};

// Distinct packed pairs, sorted, with their count still on the device
// (everything enqueued, nothing read back).
template <typename K>
struct PendingPairs {
    DevBuf keys, alt, counter, pos;
    const int64_t* count = nullptr;
    void adopt(cudaStream_t st) {
        keys.adopt(st);
        alt.adopt(st);
        counter.adopt(st);
        pos.adopt(st);
    }
};

template <typename K>
static void sort_unique_pairs_enqueue(const int32_t* a, const int32_t* b, int64_t n, int shift, int bits,
                                      PendingPairs<K>& pp, cudaStream_t s) {
    pp.keys.alloc((size_t)std::max<int64_t>(n, 1) * sizeof(K), s);
    pp.counter.alloc(8, s);
    DIM3_CUDA(cudaMemsetAsync(pp.counter.p, 0, 8, s));
    if (n > 0) {
        k_pack_pairs<K><<<grid_for(n), kThreads, 0, s>>>(a, b, n, shift, pp.keys.template as<K>(),
                                                          pp.counter.template as<unsigned long long>());
        DIM3_LAUNCHED();
    }
    // the count of packed pairs stays on the device: sort and unique take it
    // from there
    const int64_t* m_dev = pp.counter.template as<int64_t>();
    pp.alt.alloc((size_t)std::max<int64_t>(n, 1) * sizeof(K), s);
    if constexpr (sizeof(K) == 4) {
        radix_sort_u32(pp.keys.template as<uint32_t>(), nullptr, pp.alt.template as<uint32_t>(), nullptr, n, bits, s, m_dev);
        pp.count = unique_sorted_u32_async(pp.keys.template as<uint32_t>(), pp.alt.template as<uint32_t>(), n, s, m_dev, pp.pos);
    } else {
        radix_sort_u64(pp.keys.template as<uint64_t>(), nullptr, pp.alt.template as<uint64_t>(), nullptr, n, bits, s, m_dev);
        pp.count = unique_sorted_u64_async(pp.keys.template as<uint64_t>(), pp.alt.template as<uint64_t>(), n, s, m_dev, pp.pos);
    }
}

// One host read: the unique pairs end in out (the unique keys are in alt).
template <typename K>
static void sort_unique_pairs_finish(PendingPairs<K>& pp, SortedPairs<K>& out, cudaStream_t s) {
    out.n = read_i64(pp.count, s);
    out.keys = std::move(pp.alt);
}

template <typename K>
static void sort_unique_pairs(const int32_t* a, const int32_t* b, int64_t n, int shift, int bits,
                              SortedPairs<K>& out, cudaStream_t s) {
    PendingPairs<K> pp;
    sort_unique_pairs_enqueue<K>(a, b, n, shift, bits, pp, s);
    sort_unique_pairs_finish<K>(pp, out, s);
}

template <typename K>
static void rowptr_sorted(const K* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr, cudaStream_t s) {
    if constexpr (sizeof(K) == 4)
        rowptr_from_sorted_u32(keys, n, shift, n_rows, rowptr, s);
    else
        rowptr_from_sorted_u64(keys, n, shift, n_rows, rowptr, s);
}

// R side: CSR of the kept distinct R tuples by x id.
template <typename K>
static void build_r_side(Plan& p, const int32_t* rx_id, const int32_t* ry_id, int64_t nr, int bx, int by,
                         cudaStream_t s) {
    SortedPairs<K> r;
    sort_unique_pairs<K>(rx_id, ry_id, nr, by, bx + by, r, s);
    const int64_t n_x = p.info.n_x;
    p.info.n_r_kept = r.n;
    p.r_col.alloc((size_t)std::max<int64_t>(r.n, 1) * 4, s);
    p.r_rowptr.alloc((size_t)(n_x + 1) * 8, s);
    if (r.n > 0) {
        k_split_low<K><<<grid_for(r.n), kThreads, 0, s>>>(r.keys.template as<K>(), r.n, (K)((K(1) << by) - 1),
                                                           p.r_col.as<int32_t>());
        DIM3_LAUNCHED();
    }
    rowptr_sorted<K>(r.keys.template as<K>(), r.n, by, n_x, p.r_rowptr.as<int64_t>(), s);
}

// S side: everything that depends on the distinct S tuples sorted by (y, z).
// pending: the (y, z) pairs already sorted (on any stream that s has been
// made to wait for), or null to sort them here.
template <typename K>
static void build_s_side(const Ctx& ctx, Plan& p, const int32_t* sy_id, const int32_t* sz_id, int64_t ns,
                         int by, int bz, int64_t theta, const int32_t* y_tag_dev, const int32_t* z_tag_dev,
                         cudaStream_t s, PendingPairs<K>* pending = nullptr) {
    const int64_t n_y = p.info.n_y, n_z = p.info.n_z, n_x = p.info.n_x;
    const K zmask = (K)((K(1) << bz) - 1);
    SortedPairs<K> sp;
    if (pending)
        sort_unique_pairs_finish<K>(*pending, sp, s);
    else
        sort_unique_pairs<K>(sy_id, sz_id, ns, bz, by + bz, sp, s);
    p.info.n_s_distinct = sp.n;
    const K* keys = sp.keys.template as<K>();

    // deg_S(y) and m_z
    DevBuf s_rowptr;
    s_rowptr.alloc((size_t)(n_y + 1) * 8, s);
    rowptr_sorted<K>(keys, sp.n, bz, n_y, s_rowptr.as<int64_t>(), s);
    p.deg_s.alloc((size_t)std::max<int64_t>(n_y, 1) * 4, s);
    if (n_y > 0) {
        k_row_len<<<grid_for(n_y), kThreads, 0, s>>>(s_rowptr.as<int64_t>(), n_y, p.deg_s.as<int32_t>());
        DIM3_LAUNCHED();
    }
    p.m_z.alloc((size_t)std::max<int64_t>(n_z, 1) * 4, s);
    DIM3_CUDA(cudaMemsetAsync(p.m_z.p, 0, (size_t)std::max<int64_t>(n_z, 1) * 4, s));
    if (sp.n > 0) {
        k_hist_low<K><<<grid_for(sp.n), kThreads, 0, s>>>(keys, sp.n, zmask, p.m_z.as<int32_t>());
        DIM3_LAUNCHED();
    }

    // join tuples per x and |OUT_J|
    DevBuf outj_sc;
    p.outj_x.alloc((size_t)std::max<int64_t>(n_x, 1) * 8, s);
    if (n_x > 0) {
        k_outj_x<<<grid_for(n_x * 32), kThreads, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(), n_x,
                                                     p.deg_s.as<int32_t>(), p.outj_x.as<int64_t>());
        DIM3_LAUNCHED();
        // |OUT_J| is read together with the next host read (below)
        outj_sc.alloc((size_t)(n_x + 1) * 8, s);
        exclusive_scan_i64(p.outj_x.as<int64_t>(), outj_sc.as<int64_t>(), n_x, s);
    } else {
        outj_sc.alloc(8, s);
        DIM3_CUDA(cudaMemsetAsync(outj_sc.p, 0, 8, s));
    }
    const int64_t* outj_dev = outj_sc.as<int64_t>() + (n_x > 0 ? n_x : 0);
    bool outj_read = false;

    // intersection-free split: z dense iff m_z >= theta
    if (theta < 0) theta = INT32_MAX;  // tuned choice made by the caller; default all sparse
    p.info.theta_z = (int32_t)std::min<int64_t>(theta, INT32_MAX);
    p.dense_z.alloc((size_t)std::max<int64_t>(n_z, 1), s);
    DevBuf zflag, zpos, zd_index;
    zflag.alloc((size_t)std::max<int64_t>(n_z, 1) * 4, s);
    zpos.alloc((size_t)(n_z + 1) * 8, s);
    zd_index.alloc((size_t)std::max<int64_t>(n_z, 1) * 4, s);
    int64_t n_zd = 0;
    // m_z counts distinct S tuples, so theta above their number leaves every z
    // sparse: no flags, no scan, no host read
    const bool any_dense = theta <= sp.n;
    if (n_z > 0 && !any_dense) {
        DIM3_CUDA(cudaMemsetAsync(p.dense_z.p, 0, (size_t)n_z, s));
        p.zd_list.alloc(4, s);
    } else if (n_z > 0) {
        k_dense_flags<<<grid_for(n_z), kThreads, 0, s>>>(p.m_z.as<int32_t>(), n_z, theta, p.dense_z.as<uint8_t>(),
                                                          zflag.as<int32_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(zflag.as<int32_t>(), zpos.as<int64_t>(), n_z, s);
        const int64_t* src[2] = {zpos.as<int64_t>() + n_z, outj_dev};
        int64_t got[2];
        read_i64_n(src, 2, got, s);
        n_zd = got[0];
        p.info.out_j = got[1];
        outj_read = true;
        p.zd_list.alloc((size_t)std::max<int64_t>(n_zd, 1) * 4, s);
        k_zd_list<<<grid_for(n_z), kThreads, 0, s>>>(zflag.as<int32_t>(), zpos.as<int64_t>(), n_z,
                                                      p.zd_list.as<int32_t>(), zd_index.as<int32_t>());
        DIM3_LAUNCHED();
    }
    p.info.n_z_dense = n_zd;
    p.n_zd_total = n_zd;
    // dense index range of every instance
    p.inst_zd_lo.alloc((size_t)(p.n_inst + 1) * 8, s);
    p.h_inst_zd_lo.assign(p.n_inst + 1, 0);
    if (p.n_inst > 1 && n_zd > 0) {
        DevBuf zd_tag;
        zd_tag.alloc((size_t)n_zd * 4, s);
        k_gather_tags<<<grid_for(n_zd), kThreads, 0, s>>>(p.zd_list.as<int32_t>(), n_zd, z_tag_dev,
                                                           zd_tag.as<int32_t>());
        DIM3_LAUNCHED();
        k_tag_ranges<<<grid_for(p.n_inst + 1), kThreads, 0, s>>>(zd_tag.as<int32_t>(), n_zd, p.n_inst,
                                                                  p.inst_zd_lo.as<int64_t>());
        DIM3_LAUNCHED();
        DIM3_CUDA(cudaMemcpyAsync(p.h_inst_zd_lo.data(), p.inst_zd_lo.p, (size_t)(p.n_inst + 1) * 8,
                                  cudaMemcpyDeviceToHost, s));
        DIM3_CUDA(cudaStreamSynchronize(s));
    } else {
        for (int t = 1; t <= p.n_inst; ++t) p.h_inst_zd_lo[t] = n_zd;
        if (p.n_inst == 1) {
            store_i64_pair(p.inst_zd_lo.as<int64_t>(), 0, n_zd, s);
        } else {
            DIM3_CUDA(cudaMemcpyAsync(p.inst_zd_lo.p, p.h_inst_zd_lo.data(), (size_t)(p.n_inst + 1) * 8,
                                      cudaMemcpyHostToDevice, s));
            DIM3_CUDA(cudaStreamSynchronize(s));
        }
    }

    // S_sparse: the distinct tuples of sparse z, still sorted by (y, z) (all
    // of them when no z is dense)
    DevBuf sflag, spos, skeys_buf;
    int64_t n_ss = n_zd > 0 ? 0 : sp.n;
    if (sp.n > 0 && n_zd > 0) {
        sflag.alloc((size_t)sp.n * 4, s);
        spos.alloc((size_t)(sp.n + 1) * 8, s);
        k_sparse_flags<K><<<grid_for(sp.n), kThreads, 0, s>>>(keys, sp.n, zmask, p.dense_z.as<uint8_t>(),
                                                               sflag.as<int32_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(sflag.as<int32_t>(), spos.as<int64_t>(), sp.n, s);
        n_ss = read_i64(spos.as<int64_t>() + sp.n, s);
    }
    p.info.n_s_sparse = n_ss;
    const K* skeys = keys;
    if (n_zd > 0) {
        skeys_buf.alloc((size_t)std::max<int64_t>(n_ss, 1) * sizeof(K), s);
        if (n_ss > 0) {
            k_compact<K><<<grid_for(sp.n), kThreads, 0, s>>>(keys, sp.n, sflag.as<int32_t>(), spos.as<int64_t>(),
                                                              skeys_buf.as<K>());
            DIM3_LAUNCHED();
        }
        skeys = skeys_buf.as<K>();
    }
    p.ss_col.alloc((size_t)std::max<int64_t>(n_ss, 1) * 4, s);
    p.ss_rowptr.alloc((size_t)(n_y + 1) * 8, s);
    if (n_ss > 0) {
        k_split_low<K><<<grid_for(n_ss), kThreads, 0, s>>>(skeys, n_ss, zmask, p.ss_col.as<int32_t>());
        DIM3_LAUNCHED();
    }
    rowptr_sorted<K>(skeys, n_ss, bz, n_y, p.ss_rowptr.as<int64_t>(), s);

    // wide S_sparse rows held as z-bitmaps over the z window of their
    // instance (all of Z for a single instance): a row is wide when it holds
    // at least max(8, window words) z, times a factor that doubles until the
    // bitmaps fit 4 GiB
    const int32_t* y_tag = p.n_inst > 1 ? y_tag_dev : nullptr;
    p.zw = 1;
    for (int t = 0; t < p.n_inst; ++t) {
        const int64_t lo = p.h_inst_z_lo[t] & ~int64_t(31);
        p.zw = std::max<int64_t>(p.zw, ceil_div(p.h_inst_z_lo[t + 1] - lo, 32));
    }
    p.bm_row_of_y.alloc((size_t)std::max<int64_t>(n_y, 1) * 4, s);
    int64_t n_bm = 0, n_words = 0;
    if (n_y > 0) {
        DevBuf yflag, ypos, words, wpos;
        yflag.alloc((size_t)n_y * 4, s);
        ypos.alloc((size_t)(n_y + 1) * 8, s);
        words.alloc((size_t)n_y * 8, s);
        wpos.alloc((size_t)(n_y + 1) * 8, s);
        const int64_t budget_words = (int64_t(4) << 30) / 4;
        for (int64_t mult = 1;; mult *= 2) {
            k_wide_rows<<<grid_for(n_y), kThreads, 0, s>>>(p.ss_rowptr.as<int64_t>(), n_y, y_tag,
                                                            p.inst_z_lo.as<int64_t>(), p.opt.bitmap_row_min, mult,
                                                            yflag.as<int32_t>(), words.as<int64_t>());
            DIM3_LAUNCHED();
            exclusive_scan_i64(words.as<int64_t>(), wpos.as<int64_t>(), n_y, s);
            exclusive_scan_i32_to_i64(yflag.as<int32_t>(), ypos.as<int64_t>(), n_y, s);
            const int64_t* src[3] = {wpos.as<int64_t>() + n_y, ypos.as<int64_t>() + n_y, outj_dev};
            int64_t got[3];
            read_i64_n(src, outj_read ? 2 : 3, got, s);
            n_words = got[0];
            n_bm = got[1];
            if (!outj_read) p.info.out_j = got[2];
            outj_read = true;
            if (n_words <= budget_words) break;
        }
        k_index_from_flags<<<grid_for(n_y), kThreads, 0, s>>>(yflag.as<int32_t>(), ypos.as<int64_t>(), n_y,
                                                               p.bm_row_of_y.as<int32_t>());
        DIM3_LAUNCHED();
        p.bm_off.alloc((size_t)(n_bm + 1) * 8, s);
        k_row_offsets<<<grid_for(n_y + 1), kThreads, 0, s>>>(yflag.as<int32_t>(), ypos.as<int64_t>(),
                                                              wpos.as<int64_t>(), n_y, p.bm_off.as<int64_t>());
        DIM3_LAUNCHED();
    } else {
        p.bm_off.alloc(8, s);
        DIM3_CUDA(cudaMemsetAsync(p.bm_off.p, 0, 8, s));
    }
    if (!outj_read) p.info.out_j = read_i64(outj_dev, s);
    p.info.n_y_bitmap = n_bm;
    p.ss_bits.alloc((size_t)std::max<int64_t>(n_words, 1) * 4, s);
    if (n_bm > 0) {
        DIM3_CUDA(cudaMemsetAsync(p.ss_bits.p, 0, (size_t)n_words * 4, s));
        k_fill_row_bits<K><<<grid_for(n_ss), kThreads, 0, s>>>(skeys, n_ss, bz, zmask,
                                                                p.bm_row_of_y.as<int32_t>(), p.bm_off.as<int64_t>(),
                                                                y_tag, p.inst_z_lo.as<int64_t>(),
                                                                p.ss_bits.as<uint32_t>());
        DIM3_LAUNCHED();
    }

    // S_dense: K = distinct y of the dense tuples
    p.kidx_of_y.alloc((size_t)std::max<int64_t>(n_y, 1) * 4, s);
    p.info.n_y_dense = 0;
    if (n_zd > 0 && sp.n > 0) {
        DevBuf yflag, ypos;
        yflag.alloc((size_t)n_y * 4, s);
        ypos.alloc((size_t)(n_y + 1) * 8, s);
        DIM3_CUDA(cudaMemsetAsync(yflag.p, 0, (size_t)n_y * 4, s));
        k_mark_dense_y<K><<<grid_for(sp.n), kThreads, 0, s>>>(keys, sp.n, bz, zmask, p.dense_z.as<uint8_t>(),
                                                               yflag.as<int32_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(yflag.as<int32_t>(), ypos.as<int64_t>(), n_y, s);
        p.info.n_y_dense = read_i64(ypos.as<int64_t>() + n_y, s);
        k_index_from_flags<<<grid_for(n_y), kThreads, 0, s>>>(yflag.as<int32_t>(), ypos.as<int64_t>(), n_y,
                                                               p.kidx_of_y.as<int32_t>());
        DIM3_LAUNCHED();
        if constexpr (sizeof(K) == 8)
            dense_build_operands(ctx, p, keys, nullptr, sp.n, bz, zd_index.as<int32_t>(), s);
        else
            dense_build_operands(ctx, p, nullptr, keys, sp.n, bz, zd_index.as<int32_t>(), s);
    }
}

// lo[t] for t = 0..n_inst: first id whose instance is >= t (ids are ordered
// by instance); a single instance gets {0, n}.
static void instance_ranges(const int32_t* tag_dev, int64_t n, int n_inst, DevBuf& lo_dev, std::vector<int64_t>& lo,
                            cudaStream_t s) {
    lo_dev.alloc((size_t)(n_inst + 1) * 8, s);
    lo.assign(n_inst + 1, 0);
    if (n_inst > 1 && n > 0) {
        k_tag_ranges<<<grid_for(n_inst + 1), kThreads, 0, s>>>(tag_dev, n, n_inst, lo_dev.as<int64_t>());
        DIM3_LAUNCHED();
        DIM3_CUDA(cudaMemcpyAsync(lo.data(), lo_dev.p, (size_t)(n_inst + 1) * 8, cudaMemcpyDeviceToHost, s));
        DIM3_CUDA(cudaStreamSynchronize(s));
    } else {
        for (int t = 1; t <= n_inst; ++t) lo[t] = n;
        if (n_inst == 1) {
            store_i64_pair(lo_dev.as<int64_t>(), 0, n, s);
        } else {
            DIM3_CUDA(cudaMemcpyAsync(lo_dev.p, lo.data(), (size_t)(n_inst + 1) * 8, cudaMemcpyHostToDevice, s));
            DIM3_CUDA(cudaStreamSynchronize(s));
        }
    }
}

__global__ void k_ids_above(const int32_t* v, int64_t n, int64_t limit, int* flag) {
    GRID_STRIDE(i, n) {
        if ((int64_t)v[i] >= limit) *flag = 1;
    }
}

__global__ void k_iota(int32_t* out, int64_t n) { GRID_STRIDE(i, n) out[i] = (int32_t)i; }

// Skipped mapping (Section 2.2, Optimization 1): check every id column
// against its range, and make the dictionaries the identity.
static void premapped_ids(Plan& p, const PlanInput& in, cudaStream_t s) {
    DIM3_REQUIRE(in.n_inst <= 1, DIM3_ERR_ARG, "pre-mapped ids take a single instance");
    DIM3_REQUIRE(in.n_x >= 0 && in.n_y >= 0 && in.n_z >= 0 && in.n_x <= INT32_MAX && in.n_y <= INT32_MAX &&
                     in.n_z <= INT32_MAX,
                 DIM3_ERR_ARG, "id ranges must lie in [0, 2^31 - 1]");
    DevBuf flag;
    flag.alloc(4, s);
    DIM3_CUDA(cudaMemsetAsync(flag.p, 0, 4, s));
    const struct {
        const int32_t* v;
        int64_t n, lim;
    } cols[4] = {{in.r_val, in.nr, in.n_x}, {in.r_key, in.nr, in.n_y}, {in.s_key, in.ns, in.n_y}, {in.s_val, in.ns, in.n_z}};
    for (const auto& c : cols) {
        if (c.n <= 0) continue;
        k_ids_above<<<grid_for(c.n), kThreads, 0, s>>>(c.v, c.n, c.lim, flag.as<int>());
        DIM3_LAUNCHED();
    }
    int h = 0;
    DIM3_CUDA(cudaMemcpyAsync(&h, flag.p, 4, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    DIM3_REQUIRE(h == 0, DIM3_ERR_ARG, "an id is not below its declared range");
    p.info.n_x = in.n_x;
    p.info.n_y = in.n_y;
    p.info.n_z = in.n_z;
    DevBuf* dicts[3] = {&p.dict_x, &p.dict_y, &p.dict_z};
    const int64_t lens[3] = {in.n_x, in.n_y, in.n_z};
    for (int d = 0; d < 3; ++d) {
        dicts[d]->alloc((size_t)std::max<int64_t>(lens[d], 1) * 4, s);
        if (lens[d] > 0) {
            k_iota<<<grid_for(lens[d]), kThreads, 0, s>>>(dicts[d]->as<int32_t>(), lens[d]);
            DIM3_LAUNCHED();
        }
    }
}

// cnt[v] += occurrences of v; lanes holding the same id add once (skewed
// columns put many equal ids in one warp)
__global__ void k_count_ids(const int32_t* __restrict__ ids, int64_t n, unsigned long long* cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (n + stride - 1) / stride;
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t i = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int32_t v = i < n ? ids[i] : -1;
        const unsigned peers = __match_any_sync(kFull, v);
        if (v >= 0 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(cnt + v, (unsigned long long)__popc(peers));
    }
}

// sum over R rows (with a y id) of the S rows of that y: |OUT_J| of the bags
__global__ void k_sum_deg(const int32_t* __restrict__ ids, int64_t n, const unsigned long long* __restrict__ deg,
                          unsigned long long* total) {
    __shared__ unsigned long long s_warp[kThreads / 32 + 1];
    unsigned long long acc = 0;
    GRID_STRIDE(i, n) {
        const int32_t v = ids[i];
        if (v >= 0) acc += deg[v];
    }
    acc = block_sum<unsigned long long, kThreads>(acc, s_warp);
    if (threadIdx.x == 0 && acc) atomicAdd(total, acc);
}

// Armed when work is forked from stream s onto stream `from`: join() records
// the event on `from` (after everything enqueued there so far) and makes s
// wait for it. Joins when it goes out of scope too, so an exception thrown
// half-way through the forked work still orders s after it (s frees buffers
// that work reads).
struct StreamJoin {
    cudaStream_t s = nullptr, from = nullptr;
    cudaEvent_t ev = nullptr;
    void arm(cudaStream_t st, cudaStream_t other, cudaEvent_t e) {
        s = st;
        from = other;
        ev = e;
    }
    cudaError_t join() {
        if (!ev) return cudaSuccess;
        cudaEvent_t e = ev;
        ev = nullptr;
        cudaError_t r = cudaEventRecord(e, from);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(s, e, 0);
        return r;
    }
    ~StreamJoin() { join(); }
};

struct SideArgs {
    const int32_t *rx, *ry;
    int64_t nr;
    const int32_t *sy, *sz;
    int64_t ns;
    int bx, by, bz;
    int64_t theta_z;
    const int32_t *y_tag, *z_tag;
};

// R_CSR and the S side; the (y, z) pairs are sorted on the context's second
// stream while the R side is built on s.
template <typename KR, typename KS>
static void build_sides(const Ctx& ctx, Plan& p, const SideArgs& a, cudaStream_t s) {
    PendingPairs<KS> spp;
    StreamJoin sjoin;
    cudaStream_t ss = s;
    if (ctx.aux && ctx.ev_fork && ctx.ev_join) {
        DIM3_CUDA(cudaEventRecord(ctx.ev_fork, s));
        DIM3_CUDA(cudaStreamWaitEvent(ctx.aux, ctx.ev_fork, 0));
        ss = ctx.aux;
        sjoin.arm(s, ss, ctx.ev_join);
    }
    sort_unique_pairs_enqueue<KS>(a.sy, a.sz, a.ns, a.bz, a.by + a.bz, spp, ss);
    build_r_side<KR>(p, a.rx, a.ry, a.nr, a.bx, a.by, s);
    DIM3_CUDA(sjoin.join());
    spp.adopt(s);
    build_s_side<KS>(ctx, p, a.sy, a.sz, a.ns, a.by, a.bz, a.theta_z, a.y_tag, a.z_tag, s, &spp);
}

Plan* build_plan(const Ctx& ctx, const PlanInput& in, int64_t theta_z, cudaStream_t s, bool* prefer_classical) {
    PhaseScope phase(ctx.stats, PH_PARTITION, s);
    std::unique_ptr<Plan> p(new Plan());
    const int64_t nr = in.nr, ns = in.ns;
    const bool batch = in.n_inst > 1;
    p->stream = s;
    p->device = ctx.device;
    p->opt = ctx.opt;
    p->n_inst = std::max(in.n_inst, 1);
    p->info.n_r = nr;
    p->info.n_s = ns;

    DevBuf sy_id, sz_id, ry_id, rx_id, y_tag, z_tag;
    const int32_t *rx = nullptr, *ry = nullptr, *sy = nullptr, *sz = nullptr;
    DIM3_REQUIRE(!in.cache || (!in.premapped && !batch), DIM3_ERR_ARG,
                 "a partial result cache attaches to a single instance of mapped columns");
    if (in.premapped) {
        premapped_ids(*p, in, s);
        rx = in.r_val;
        ry = in.r_key;
        sy = in.s_key;
        sz = in.s_val;
    } else {
        sy_id.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        sz_id.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        ry_id.alloc((size_t)std::max<int64_t>(nr, 1) * 4, s);
        rx_id.alloc((size_t)std::max<int64_t>(nr, 1) * 4, s);
        if (batch) {
            y_tag.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
            z_tag.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
            p->x_tag.alloc((size_t)std::max<int64_t>(nr, 1) * 4, s);
        }
        // The three maps leave their distinct counts on the device; they are
        // read together (with f1's |OUT_J| when that is asked for). The z map
        // depends on neither of the others and runs on the context's second
        // stream meanwhile; `zjoin` makes s wait for it before anything that
        // reads its results, and on every way out of this block (buffers the
        // z map writes are freed in s's order).
        //
        // A self-join (R and S given by the same column pointers) maps once:
        // every R.y occurs in S.y, so R's y ids are S's, no tuple is dropped,
        // and the x map (over R.x) is the z map (over S.z).
        const bool self_join = in.r_key == in.s_key && in.r_val == in.s_val && nr == ns && in.r_tag == in.s_tag;
        ValueMap ymap, xmap, zmap;
        p->dict_y.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        p->dict_x.alloc((size_t)std::max<int64_t>(nr, 1) * 4, s);
        p->dict_z.alloc((size_t)std::max<int64_t>(ns, 1) * 4, s);
        StreamJoin zjoin;
        if (!self_join) {
            cudaStream_t zs = s;
            if (ctx.aux && ctx.ev_fork && ctx.ev_join) {
                DIM3_CUDA(cudaEventRecord(ctx.ev_fork, s));
                DIM3_CUDA(cudaStreamWaitEvent(ctx.aux, ctx.ev_fork, 0));
                zs = ctx.aux;
                zjoin.arm(s, zs, ctx.ev_join);
            }
            build_value_map(in.s_val, in.s_tag, p->n_inst, nullptr, ns, zmap, sz_id.as<int32_t>(),
                            p->dict_z.as<int32_t>(), z_tag.as<int32_t>(), zs, false);
        }
        {
            // y from S.y; R tuples whose y is absent from S.y get id -1 (dropped)
            build_value_map(in.s_key, in.s_tag, p->n_inst, nullptr, ns, ymap, sy_id.as<int32_t>(),
                            p->dict_y.as<int32_t>(), y_tag.as<int32_t>(), s, false);
            if (self_join)
                DIM3_CUDA(cudaMemcpyAsync(ry_id.p, sy_id.p, (size_t)nr * 4, cudaMemcpyDeviceToDevice, s));
            else
                probe_value_map(ymap, in.r_key, in.r_tag, nr, ry_id.as<int32_t>(), s);
        }
        if (prefer_classical) {
            // f1 (Section 2.6) from the y ids just made: |OUT_J| of the bags
            DevBuf deg, tot;
            deg.alloc((size_t)std::max<int64_t>(ns, 1) * 8, s);  // y ids < |Y| <= |S|
            tot.alloc(8, s);
            DIM3_CUDA(cudaMemsetAsync(deg.p, 0, deg.bytes, s));
            DIM3_CUDA(cudaMemsetAsync(tot.p, 0, 8, s));
            if (ns > 0) {
                k_count_ids<<<grid_for(ns), kThreads, 0, s>>>(sy_id.as<int32_t>(), ns, deg.as<unsigned long long>());
                DIM3_LAUNCHED();
            }
            if (nr > 0) {
                k_sum_deg<<<grid_for(nr), kThreads, 0, s>>>(ry_id.as<int32_t>(), nr, deg.as<unsigned long long>(),
                                                             tot.as<unsigned long long>());
                DIM3_LAUNCHED();
            }
            int64_t out_j = 0;
            ValueMap* ym = &ymap;
            resolve_counts(&ym, 1, tot.as<int64_t>(), &out_j, s);
            *prefer_classical = f1_value(nr, ns, out_j, ctx.opt.f1c) > 0.0;
            if (*prefer_classical) return nullptr;
        }
        build_value_map(in.r_val, in.r_tag, p->n_inst, ry_id.as<int32_t>(), nr, xmap, rx_id.as<int32_t>(),
                        p->dict_x.as<int32_t>(), p->x_tag.as<int32_t>(), s, false);
        DIM3_CUDA(zjoin.join());
        ValueMap* maps[3] = {&ymap, &xmap, &zmap};
        resolve_counts(maps, self_join ? 2 : 3, nullptr, nullptr, s);
        if (self_join) {
            zmap.n_distinct = xmap.n_distinct;
            const size_t b = (size_t)std::max<int64_t>(ns, 1) * 4;
            DIM3_CUDA(cudaMemcpyAsync(sz_id.p, rx_id.p, b, cudaMemcpyDeviceToDevice, s));
            DIM3_CUDA(cudaMemcpyAsync(p->dict_z.p, p->dict_x.p, (size_t)std::max<int64_t>(xmap.n_distinct, 1) * 4,
                                      cudaMemcpyDeviceToDevice, s));
            if (batch) DIM3_CUDA(cudaMemcpyAsync(z_tag.p, p->x_tag.p, b, cudaMemcpyDeviceToDevice, s));
        }
        DIM3_REQUIRE(ymap.n_distinct >= 0 && ymap.n_distinct <= ns && xmap.n_distinct >= 0 &&
                         xmap.n_distinct <= nr && zmap.n_distinct >= 0 && zmap.n_distinct <= ns,
                     DIM3_ERR_CUDA, "value map: inconsistent distinct count");
        p->info.n_y = ymap.n_distinct;
        p->info.n_x = xmap.n_distinct;
        p->info.n_z = zmap.n_distinct;
        // Section 3: the S tuples of cached z leave after mapping, so the
        // dictionaries (and X) stay those of the full tables
        if (in.cache) attach_cache_ids(*p, *in.cache, sz_id.as<int32_t>(), ns, s);
        rx = rx_id.as<int32_t>();
        ry = ry_id.as<int32_t>();
        sy = sy_id.as<int32_t>();
        sz = sz_id.as<int32_t>();
    }
    instance_ranges(p->x_tag.as<int32_t>(), p->info.n_x, p->n_inst, p->inst_x_lo, p->h_inst_x_lo, s);
    instance_ranges(z_tag.as<int32_t>(), p->info.n_z, p->n_inst, p->inst_z_lo, p->h_inst_z_lo, s);
    const int bx = bits_for(p->info.n_x), by = bits_for(p->info.n_y), bz = bits_for(p->info.n_z);
    const SideArgs sa{rx, ry, nr, sy, sz, ns, bx, by, bz, theta_z, y_tag.as<int32_t>(), z_tag.as<int32_t>()};
    if (bx + by <= 32) {
        if (by + bz <= 32) build_sides<uint32_t, uint32_t>(ctx, *p, sa, s);
        else build_sides<uint32_t, uint64_t>(ctx, *p, sa, s);
    } else {
        if (by + bz <= 32) build_sides<uint64_t, uint32_t>(ctx, *p, sa, s);
        else build_sides<uint64_t, uint64_t>(ctx, *p, sa, s);
    }
    if (in.cache) finish_cache_index(*p, s);
    if (batch) p->y_tag = std::move(y_tag);
    DIM3_CUDA(cudaStreamSynchronize(s));
    return p.release();
}

}  // namespace dimcube
