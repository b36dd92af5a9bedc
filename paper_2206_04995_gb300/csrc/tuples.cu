// Multi-attribute mapping (Section 2.2, "Supporting Wider Range of
// Join-Project Operations"): the rows of k int32 columns are numbered by the
// rank of their tuple among the distinct tuples in lexicographic order, so a
// query such as Pi_{a,b,c,d,e}(R(a,b,c,d) join_{c,d} S(c,d,e,f)) runs as
// Pi_{x,z}(R(x,y) join_y S(z,y)) over x = (a,b), y = (c,d), z = (c,d,e).
//
// GPU form: LSD over the columns. A row permutation is radix-sorted stably by
// the last column's 32-bit key, then by the column before it, and so on to
// column 0 (signed columns get their sign bit flipped so that unsigned key
// order is signed value order). Stability leaves equal tuples in ascending
// row order. A sorted position whose tuple differs from its predecessor's
// starts a new id; a scan of those flags gives every position its rank, and
// the first position of each id names the smallest row with that tuple.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

struct ColSet {
    const int32_t* c[kMaxTupleCols];
    uint32_t flip[kMaxTupleCols];  // 0x80000000 for signed columns, 0 for unsigned
    int k;
};

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

// keys[i] = column value of row perm[i] (row i when perm is null), as an
// order-preserving unsigned key; perm_out[i] = that row (starts the permutation)
__global__ void k_tuple_keys(const int32_t* __restrict__ col, uint32_t flip, const uint32_t* perm, int64_t n,
                             uint32_t* __restrict__ keys, uint32_t* perm_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = perm ? perm[i] : (uint32_t)i;
        keys[i] = (uint32_t)col[r] ^ flip;
        if (!perm) perm_out[i] = r;
    }
}

// flag[i] = 1 when sorted position i starts a new tuple
__global__ void k_tuple_flags(ColSet cs, const uint32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int f = i == 0;
        if (!f) {
            const uint32_t a = perm[i], b = perm[i - 1];
            for (int c = 0; c < cs.k; ++c) f |= cs.c[c][a] != cs.c[c][b];
        }
        flag[i] = f;
    }
}

__global__ void k_tuple_ids(const uint32_t* __restrict__ perm, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ flag, int64_t n, int32_t* __restrict__ ids,
                            int32_t* __restrict__ first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(off[i] + flag[i] - 1);
        ids[perm[i]] = r;
        if (flag[i]) first[r] = (int32_t)perm[i];
    }
}

int64_t map_tuples(const int32_t* const* cols, int k, uint32_t unsigned_mask, int64_t n, int32_t* ids, int32_t* first,
                   cudaStream_t s) {
    if (n == 0) return 0;
    ColSet cs{};
    cs.k = k;
    for (int c = 0; c < k; ++c) {
        cs.c[c] = cols[c];
        cs.flip[c] = ((unsigned_mask >> c) & 1u) ? 0u : 0x80000000u;
    }
    DevBuf keys, perm, keys_alt, perm_alt;
    keys.alloc((size_t)n * 4, s);
    perm.alloc((size_t)n * 4, s);
    keys_alt.alloc((size_t)n * 4, s);
    perm_alt.alloc((size_t)n * 4, s);
    for (int c = k - 1; c >= 0; --c) {
        const bool start = c == k - 1;
        // the key gather reads perm and, at the start, writes it
        k_tuple_keys<<<grid_for(n), kThreads, 0, s>>>(cs.c[c], cs.flip[c], start ? nullptr : perm.as<uint32_t>(), n,
                                                        keys.as<uint32_t>(), perm.as<uint32_t>());
        DIM3_LAUNCHED();
        radix_sort_u32(keys.as<uint32_t>(), perm.as<uint32_t>(), keys_alt.as<uint32_t>(), perm_alt.as<uint32_t>(), n,
                       32, s);
    }
    DevBuf flag, off;
    flag.alloc((size_t)n * 4, s);
    off.alloc((size_t)(n + 1) * 8, s);
    k_tuple_flags<<<grid_for(n), kThreads, 0, s>>>(cs, perm.as<uint32_t>(), n, flag.as<int32_t>());
    DIM3_LAUNCHED();
    exclusive_scan_i32_to_i64(flag.as<int32_t>(), off.as<int64_t>(), n, s);
    k_tuple_ids<<<grid_for(n), kThreads, 0, s>>>(perm.as<uint32_t>(), off.as<int64_t>(), flag.as<int32_t>(), n, ids,
                                                  first);
    DIM3_LAUNCHED();
    return read_i64(off.as<int64_t>() + n, s);
}

__global__ void k_gather_i32(const int32_t* __restrict__ src, int64_t n_src, const int32_t* __restrict__ idx,
                             int64_t n, int32_t* __restrict__ dst, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = idx[i];
        if (j < 0 || (int64_t)j >= n_src) {
            dst[i] = -1;
            *bad = 1;
        } else {
            dst[i] = src[j];
        }
    }
}

bool gather_i32(const int32_t* src, int64_t n_src, const int32_t* idx, int64_t n, int32_t* dst, cudaStream_t s) {
    if (n == 0) return true;
    DevBuf bad;
    bad.alloc(4, s);
    DIM3_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
    k_gather_i32<<<grid_for(n), kThreads, 0, s>>>(src, n_src, idx, n, dst, bad.as<int>());
    DIM3_LAUNCHED();
    int h = 0;
    DIM3_CUDA(cudaMemcpyAsync(&h, bad.p, 4, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    return h == 0;
}

}  // namespace dimcube
