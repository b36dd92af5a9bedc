// Device-wide primitives: exclusive scan, LSD radix sort, unique, CSR row
// pointers. They carry no Join-Project arithmetic; the mapping and partition
// steps are built from them.
#include <algorithm>

#include "common.cuh"
#include "device.cuh"

namespace dimcube {

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

template <typename Tin>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const Tin* in, int64_t n, int64_t* partial) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kThreads) {
        int64_t idx = base + i;
        if (idx < n) acc += (int64_t)in[idx];
    }
    acc = block_sum<int64_t, kThreads>(acc, s_warp);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// single block: exclusive scan of partial[0..nb) in place; total -> *total_out
__global__ void __launch_bounds__(kThreads) k_scan_partials(int64_t* partial, int64_t nb, int64_t* total_out) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kThreads) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? partial[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<int64_t, kThreads>(v, &tot, s_warp);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename Tin>
__global__ void __launch_bounds__(kThreads) k_scan_down(const Tin* in, int64_t* out, int64_t n,
                                                        const int64_t* partial) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t idx = base + j;
        v[j] = idx < n ? (int64_t)in[idx] : 0;
        sum += v[j];
    }
    int64_t tot;
    int64_t run = block_exclusive_scan<int64_t, kThreads>(sum, &tot, s_warp) + partial[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t idx = base + j;
        if (idx < n) out[idx] = run;
        run += v[j];
    }
}

template <typename Tin>
static void exclusive_scan_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        fill_i64(out, 0, 1, s);
        return;
    }
    const int64_t nb = ceil_div(n, kScanTile);
    DevBuf partial;
    partial.alloc((size_t)nb * sizeof(int64_t), s);
    k_scan_reduce<Tin><<<(unsigned)nb, kThreads, 0, s>>>(in, n, partial.as<int64_t>());
    DIM3_LAUNCHED();
    k_scan_partials<<<1, kThreads, 0, s>>>(partial.as<int64_t>(), nb, out + n);
    DIM3_LAUNCHED();
    k_scan_down<Tin><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, partial.as<int64_t>());
    DIM3_LAUNCHED();
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan_impl<int64_t>(in, out, n, s);
}
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan_impl<int32_t>(in, out, n, s);
}

__global__ void k_fill_i64(int64_t* p, int64_t v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, kThreads), 4096);
    k_fill_i64<<<g, kThreads, 0, s>>>(p, v, n);
    DIM3_LAUNCHED();
}

int64_t read_i64(const int64_t* d, cudaStream_t s) {
    int64_t h = 0;
    DIM3_CUDA(cudaMemcpyAsync(&h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    return h;
}

// ------------------------------------------------------------ radix sort
// LSD radix sort, 8-bit digits. Per pass: a per-tile digit histogram, an
// exclusive scan of the digit-major histogram table (global digit offsets per
// tile), and a stable scatter. Ranks inside a tile come from warp-level
// __match_any_sync groups and per-warp digit counters in shared memory, so the
// scatter is stable (element order: tile, warp, chunk, lane).
constexpr int kRadixIpt = 16;
constexpr int kRadixTile = kThreads * kRadixIpt;
constexpr int kWarps = kThreads / 32;

template <typename K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K* keys, int64_t n, int shift,
                                                         int32_t* hist, int64_t nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += kThreads) {
        int64_t idx = base + i;
        bool valid = idx < n;
        unsigned d = valid ? (unsigned)((keys[idx] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        if (valid && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = (int32_t)h[threadIdx.x];
}

template <typename K, bool kVals>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const K* __restrict__ keys,
                                                            const uint32_t* __restrict__ vals,
                                                            K* __restrict__ okeys,
                                                            uint32_t* __restrict__ ovals, int64_t n,
                                                            int shift, const int64_t* offs, int64_t nb) {
    __shared__ uint32_t wcount[kWarps][256];
    __shared__ int64_t base[256];
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&wcount[0][0])[i] = 0;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const unsigned lane = lane_id();
    const unsigned warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t wbase = (int64_t)blockIdx.x * kRadixTile + (int64_t)warp * (kRadixTile / kWarps);
    K k[kRadixIpt];
    uint32_t v[kRadixIpt];
    uint32_t rk[kRadixIpt];
    unsigned dg[kRadixIpt];
#pragma unroll
    for (int j = 0; j < kRadixIpt; ++j) {
        int64_t idx = wbase + j * 32 + lane;
        bool valid = idx < n;
        k[j] = valid ? keys[idx] : K(0);
        if (kVals) v[j] = valid ? vals[idx] : 0u;
        unsigned d = valid ? (unsigned)((k[j] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(kFull, d);
        int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && (int)lane == leader) {
            before = wcount[warp][d];
            wcount[warp][d] = before + (uint32_t)__popc(peers);
        }
        before = __shfl_sync(kFull, before, leader);
        rk[j] = before + (uint32_t)__popc(peers & lt);
        dg[j] = d;
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t t = wcount[w][d];
            wcount[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRadixIpt; ++j) {
        if (dg[j] < 256u) {
            int64_t pos = base[dg[j]] + wcount[warp][dg[j]] + rk[j];
            okeys[pos] = k[j];
            if (kVals) ovals[pos] = v[j];
        }
    }
}

template <typename K>
static void radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                            int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    const int64_t nb = ceil_div(n, kRadixTile);
    DevBuf hist, offs;
    hist.alloc((size_t)nb * 256 * sizeof(int32_t), s);
    offs.alloc(((size_t)nb * 256 + 1) * sizeof(int64_t), s);
    const int passes = (bits + 7) / 8;
    K* src = keys;
    K* dst = keys_alt;
    uint32_t* sv = vals;
    uint32_t* dv = vals_alt;
    for (int p = 0; p < passes; ++p) {
        k_radix_hist<K><<<(unsigned)nb, kThreads, 0, s>>>(src, n, 8 * p, hist.as<int32_t>(), nb);
        DIM3_LAUNCHED();
        exclusive_scan_i32_to_i64(hist.as<int32_t>(), offs.as<int64_t>(), nb * 256, s);
        if (vals)
            k_radix_scatter<K, true><<<(unsigned)nb, kThreads, 0, s>>>(src, sv, dst, dv, n, 8 * p,
                                                                       offs.as<int64_t>(), nb);
        else
            k_radix_scatter<K, false><<<(unsigned)nb, kThreads, 0, s>>>(src, nullptr, dst, nullptr, n,
                                                                        8 * p, offs.as<int64_t>(), nb);
        DIM3_LAUNCHED();
        std::swap(src, dst);
        std::swap(sv, dv);
    }
    if (src != keys) {
        DIM3_CUDA(cudaMemcpyAsync(keys, src, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        if (vals)
            DIM3_CUDA(cudaMemcpyAsync(vals, sv, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

void radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int64_t n,
                    int bits, cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, s);
}
void radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                    int bits, cudaStream_t s) {
    radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, bits, s);
}

// ------------------------------------------------------------------ unique
template <typename K>
__global__ void k_unique_flags(const K* in, int64_t n, int32_t* flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || in[i] != in[i - 1]) ? 1 : 0;
}

template <typename K>
__global__ void k_unique_scatter(const K* in, int64_t n, const int32_t* flags, const int64_t* pos, K* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i]) out[pos[i]] = in[i];
}

template <typename K>
static int64_t unique_impl(const K* in, K* out, int64_t n, cudaStream_t s) {
    if (n == 0) return 0;
    DevBuf flags, pos;
    flags.alloc((size_t)n * sizeof(int32_t), s);
    pos.alloc(((size_t)n + 1) * sizeof(int64_t), s);
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n, kThreads), 8192);
    k_unique_flags<K><<<g, kThreads, 0, s>>>(in, n, flags.as<int32_t>());
    DIM3_LAUNCHED();
    exclusive_scan_i32_to_i64(flags.as<int32_t>(), pos.as<int64_t>(), n, s);
    k_unique_scatter<K><<<g, kThreads, 0, s>>>(in, n, flags.as<int32_t>(), pos.as<int64_t>(), out);
    DIM3_LAUNCHED();
    return read_i64(pos.as<int64_t>() + n, s);
}

int64_t unique_sorted_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    return unique_impl<uint32_t>(in, out, n, s);
}
int64_t unique_sorted_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s) {
    return unique_impl<uint64_t>(in, out, n, s);
}

// ----------------------------------------------------------------- rowptr
template <typename K>
__global__ void k_rowptr(const K* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(keys[mid] >> shift) < r) lo = mid + 1; else hi = mid;
        }
        rowptr[r] = lo;
    }
}

void rowptr_from_sorted_u32(const uint32_t* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr,
                            cudaStream_t s) {
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n_rows + 1, kThreads), 8192);
    k_rowptr<uint32_t><<<g, kThreads, 0, s>>>(keys, n, shift, n_rows, rowptr);
    DIM3_LAUNCHED();
}
void rowptr_from_sorted_u64(const uint64_t* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr,
                            cudaStream_t s) {
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n_rows + 1, kThreads), 8192);
    k_rowptr<uint64_t><<<g, kThreads, 0, s>>>(keys, n, shift, n_rows, rowptr);
    DIM3_LAUNCHED();
}

}  // namespace dimcube
