// Device-wide primitives: exclusive scan, LSD radix sort, unique, CSR row
// pointers. They carry no Join-Project arithmetic; the mapping and partition
// steps are built from them.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "device.cuh"

namespace dimcube {

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

// Single-pass exclusive scan: one launch whatever n. Every CTA scans one
// tile of kScanTile items and finds the tile's offset by decoupled look-back
// over the tiles before it (logical tile numbers from a ticket, so a CTA only
// waits on tiles already running; a wait that runs past 2 s gives up, stores 1
// to the process-wide wait-fault flag, which fails the call with
// DIM3_ERR_TIMEOUT after its next synchronisation). The last tile writes the
// total to out[n].
constexpr uint64_t kScanWaitNs = 2000000000ull;

template <typename Tin>
__global__ void __launch_bounds__(kThreads) k_scan_lb(const Tin* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                                                      int64_t n_tiles, unsigned long long* status,
                                                      unsigned long long* ticket, int* err, int* fault) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    __shared__ int64_t s_blk, s_pre;
    if (threadIdx.x == 0) s_blk = (int64_t)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t b = s_blk;
    const int64_t base = b * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t idx = base + j;
        v[j] = idx < n ? (int64_t)in[idx] : 0;
        sum += v[j];
    }
    int64_t tot;
    const int64_t ex = block_exclusive_scan<int64_t, kThreads>(sum, &tot, s_warp);
    if ((threadIdx.x >> 5) == 0) {
        const int64_t pre = lookback_prefix(status, b, tot, err, kScanWaitNs);
        if ((threadIdx.x & 31) == 0) {
            s_pre = pre < 0 ? 0 : pre;
            if (pre < 0) *static_cast<volatile int*>(fault) = 1;
        }
    }
    __syncthreads();
    int64_t run = s_pre + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t idx = base + j;
        if (idx < n) out[idx] = run;
        run += v[j];
    }
    if (b == n_tiles - 1 && threadIdx.x == 0) out[n] = s_pre + tot;
}

template <typename Tin>
static void exclusive_scan_impl(const Tin* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        fill_i64(out, 0, 1, s);
        return;
    }
    const int64_t nb = ceil_div(n, kScanTile);
    DIM3_REQUIRE(nb < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "scan too long");
    DevBuf st;  // ticket, error word, then one status word per tile
    st.alloc((size_t)(nb + 2) * sizeof(unsigned long long), s);
    DIM3_CUDA(cudaMemsetAsync(st.p, 0, st.bytes, s));
    unsigned long long* w = st.as<unsigned long long>();
    k_scan_lb<Tin><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, nb, w + 2, w, reinterpret_cast<int*>(w + 1),
                                                     wait_fault_flag());
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

__global__ void k_store_pair(int64_t* p, int64_t a, int64_t b) {
    if (threadIdx.x == 0) {
        p[0] = a;
        p[1] = b;
    }
}

void store_i64_pair(int64_t* p, int64_t a, int64_t b, cudaStream_t s) {
    k_store_pair<<<1, 32, 0, s>>>(p, a, b);
    DIM3_LAUNCHED();
}

// Pinned staging for synchronising reads: a copy into pageable memory would
// block on its own, so several values could not share one synchronisation.
constexpr int kReadSlots = 16;
static int64_t* read_slots() {
    thread_local struct Slots {
        int64_t* p = nullptr;
        ~Slots() {
            if (p) cudaFreeHost(p);
        }
    } slots;
    if (!slots.p) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, kReadSlots * sizeof(int64_t), cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            throw Error(DIM3_ERR_NOMEM, "pinned allocation of the read slots failed");
        }
        slots.p = static_cast<int64_t*>(h);
    }
    return slots.p;
}

void read_i64_n(const int64_t* const* d, int n, int64_t* h, cudaStream_t s) {
    DIM3_REQUIRE(n >= 0 && n <= kReadSlots, DIM3_ERR_ARG, "too many values in one read");
    int64_t* slot = read_slots();
    for (int i = 0; i < n; ++i)
        DIM3_CUDA(cudaMemcpyAsync(slot + i, d[i], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    raise_if_wait_fault();
    for (int i = 0; i < n; ++i) h[i] = slot[i];
}

int64_t read_i64(const int64_t* d, cudaStream_t s) {
    int64_t h = 0;
    read_i64_n(&d, 1, &h, s);
    return h;
}

// ------------------------------------------------------------ radix sort
// LSD radix sort with 8-bit digits in the one-sweep form (Adinets and Merrill,
// "Onesweep: A Faster Least Significant Digit Radix Sort for GPUs", 2022): one
// kernel counts the digits of every pass at once; then each pass is ONE kernel
// whose tiles (taken in dispatch order from a ticket) rank their keys, publish
// their per-digit counts, find the counts of the tiles before them by
// decoupled look-back (one thread per digit), reorder the tile by digit in
// shared memory and write each digit's run contiguously. Ranks inside a tile
// come from __match_any_sync groups and per-warp digit counters, so every pass
// is stable (element order: tile, warp, chunk, lane).
constexpr int kRadixIpt = 16;
constexpr int kRadixTile = kThreads * kRadixIpt;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxPasses = 8;
constexpr uint64_t kSortWaitNs = 2000000000ull;  // give up on a predecessor tile after 2 s

namespace {
std::once_flag g_fault_once;
int* g_fault_host = nullptr;  // pinned, mapped: device stores are read by the host after a sync
int* g_fault_dev = nullptr;   // the device's address of the same word
}  // namespace

int* wait_fault_flag() {
    std::call_once(g_fault_once, [] {
        void* h = nullptr;
        void* d = nullptr;
        if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
            cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            if (h) cudaFreeHost(h);
            return;
        }
        *static_cast<volatile int*>(h) = 0;
        g_fault_host = static_cast<int*>(h);
        g_fault_dev = static_cast<int*>(d);
    });
    DIM3_REQUIRE(g_fault_dev, DIM3_ERR_NOMEM, "pinned allocation of the wait-fault flag failed");
    return g_fault_dev;
}

void raise_if_wait_fault() {
    if (!g_fault_host) return;
    volatile int* f = g_fault_host;
    if (*f) {
        *f = 0;
        throw Error(DIM3_ERR_TIMEOUT, "a device-side wait on another thread block gave up after 2 s");
    }
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_os_hist(const K* __restrict__ keys, int64_t n, const int64_t* n_dev,
                                                      int passes, unsigned long long* ghist) {
    __shared__ uint32_t h[kMaxPasses][256];
    if (n_dev) n = min64(n, *n_dev);
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = h[p][threadIdx.x];
        if (v) atomicAdd(&ghist[p * 256 + threadIdx.x], (unsigned long long)v);
    }
}

// status[tile * 256 + digit]: flag in the top two bits (0 none yet, 1 the
// tile's own count, 2 the inclusive count over tiles 0..tile), count below.
// status_next (the buffer of the following pass) is cleared tile by tile.
template <typename K, bool kVals>
__global__ void __launch_bounds__(kThreads) k_os_pass(const K* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                      K* __restrict__ okeys, uint32_t* __restrict__ ovals, int64_t n,
                                                      const int64_t* n_dev, int pass,
                                                      const unsigned long long* __restrict__ ghist,
                                                      unsigned long long* status, unsigned long long* status_next,
                                                      unsigned long long* ticket, int* fault) {
    extern __shared__ __align__(16) unsigned char os_smem[];
    K* s_keys = reinterpret_cast<K*>(os_smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(os_smem + (size_t)kRadixTile * sizeof(K));
    __shared__ uint32_t wcount[kWarps][256];
    __shared__ int64_t s_goff[256];
    __shared__ uint32_t s_lstart[256];
    __shared__ uint32_t s_w32[kWarps + 1];
    __shared__ unsigned long long s_w64[kWarps + 1];
    __shared__ int64_t s_tile;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(ticket, 1ull);
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int64_t t = s_tile;
    // with a device-side count the grid covers the largest count; tiles past
    // the actual one have nothing to do and nobody waits on them
    if (n_dev) n = min64(n, *n_dev);
    if (t * kRadixTile >= n) return;
    const int shift = 8 * pass;
    const unsigned lane = lane_id();
    const unsigned warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t tbase = t * kRadixTile;
    const int64_t wbase = tbase + (int64_t)warp * (kRadixTile / kWarps);
    K k[kRadixIpt];
    uint32_t v[kRadixIpt];
    uint32_t rk[kRadixIpt];
#pragma unroll
    for (int j = 0; j < kRadixIpt; ++j) {
        const int64_t idx = wbase + j * 32 + lane;
        const bool valid = idx < n;
        k[j] = valid ? keys[idx] : K(0);
        if (kVals) v[j] = valid ? vals[idx] : 0u;
        const unsigned d = valid ? ((unsigned)(k[j] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && (int)lane == leader) {
            before = wcount[warp][d];
            wcount[warp][d] = before + (uint32_t)__popc(peers);
        }
        before = __shfl_sync(kFull, before, leader);
        rk[j] = valid ? before + (uint32_t)__popc(peers & lt) : 0xffffffffu;
        __syncwarp();
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcount[w][d];
        wcount[w][d] = cnt;
        cnt += c;
    }
    // publish this tile's count of digit d before anything else
    unsigned long long* my = status + t * 256 + d;
    atomicExch(my, (t == 0 ? kLbInc : kLbAgg) | (unsigned long long)cnt);
    if (status_next) status_next[t * 256 + d] = 0ull;
    uint32_t ltot;
    const uint32_t lstart = block_exclusive_scan<uint32_t, kThreads>(cnt, &ltot, s_w32);
    unsigned long long gtot;
    const unsigned long long gbase = block_exclusive_scan<unsigned long long, kThreads>(ghist[pass * 256 + d], &gtot, s_w64);
    // decoupled look-back over the tiles before this one, digit d only; the
    // words of kLbBatch predecessors are loaded at once, so a walk through
    // tiles that have only published their own counts costs one load latency
    // per kLbBatch tiles (before tile -1 reads as an inclusive zero)
    constexpr int kLbBatch = 8;
    int64_t prefix = 0;
    if (t > 0) {
        int64_t j = t - 1;
        const uint64_t t0 = global_ns();
        uint32_t polls = 0;
        while (true) {
            unsigned long long w[kLbBatch];
#pragma unroll
            for (int q = 0; q < kLbBatch; ++q) w[q] = j - q >= 0 ? ld_relaxed_u64(status + (j - q) * 256 + d) : kLbInc;
            int used = 0;
            bool done = false;
#pragma unroll
            for (int q = 0; q < kLbBatch; ++q) {
                if (done || used < q) continue;  // stop at the first word not yet published
                const unsigned long long f = w[q] >> 62;
                if (f == 0ull) continue;
                prefix += (int64_t)(w[q] & kLbVal);
                used = q + 1;
                done = f == 2ull;
            }
            if (done) break;
            j -= used;
            if (used == 0 && (++polls & 63u) == 0u && global_ns() - t0 > kSortWaitNs) {
                *static_cast<volatile int*>(fault) = 1;
                break;
            }
        }
        atomicExch(my, kLbInc | (unsigned long long)(prefix + cnt));
    }
    s_goff[d] = (int64_t)gbase + prefix - (int64_t)lstart;
    s_lstart[d] = lstart;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRadixIpt; ++j) {
        if (rk[j] != 0xffffffffu) {
            const unsigned dg = (unsigned)(k[j] >> shift) & 255u;
            const uint32_t li = s_lstart[dg] + wcount[warp][dg] + rk[j];
            s_keys[li] = k[j];
            if (kVals) s_vals[li] = v[j];
        }
    }
    __syncthreads();
    const int tn = (int)min64((int64_t)kRadixTile, n - tbase);
    for (int i = threadIdx.x; i < tn; i += kThreads) {
        const K key = s_keys[i];
        const int64_t pos = s_goff[(unsigned)(key >> shift) & 255u] + i;
        okeys[pos] = key;
        if (kVals) ovals[pos] = s_vals[i];
    }
}

template <typename K, bool kVals>
static void os_pass_launch(const K* src, const uint32_t* sv, K* dst, uint32_t* dv, int64_t n, const int64_t* n_dev,
                           int pass,
                           const unsigned long long* ghist, unsigned long long* st, unsigned long long* st_next,
                           unsigned long long* ticket, int* fault, cudaStream_t s) {
    constexpr size_t smem = (size_t)kRadixTile * (sizeof(K) + (kVals ? 4 : 0));
    static bool attr_done[64] = {false};
    int dev = 0;
    DIM3_CUDA(cudaGetDevice(&dev));
    if (!attr_done[dev & 63]) {
        DIM3_CUDA(cudaFuncSetAttribute(k_os_pass<K, kVals>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done[dev & 63] = true;
    }
    k_os_pass<K, kVals><<<(unsigned)ceil_div(n, kRadixTile), kThreads, smem, s>>>(src, sv, dst, dv, n, n_dev, pass, ghist,
                                                                                  st, st_next, ticket, fault);
    DIM3_LAUNCHED();
}

template <typename K>
static void radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n, int bits,
                            cudaStream_t s, const int64_t* n_dev) {
    if (n <= 1 || bits <= 0) return;
    const int passes = std::min<int>((bits + 7) / 8, (int)sizeof(K));
    const int64_t tiles = ceil_div(n, kRadixTile);
    int* fault = wait_fault_flag();
    // scratch: tickets [kMaxPasses], digit counts [kMaxPasses][256], two status buffers [tiles][256]
    const size_t head = (size_t)kMaxPasses * (1 + 256);
    const size_t stw = (size_t)tiles * 256;
    DevBuf scratch;
    scratch.alloc((head + 2 * stw) * sizeof(unsigned long long), s);
    unsigned long long* ticket = scratch.as<unsigned long long>();
    unsigned long long* ghist = ticket + kMaxPasses;
    unsigned long long* st[2] = {ghist + (size_t)kMaxPasses * 256, ghist + (size_t)kMaxPasses * 256 + stw};
    DIM3_CUDA(cudaMemsetAsync(scratch.p, 0, (head + stw) * sizeof(unsigned long long), s));
    const unsigned hg = (unsigned)std::min<int64_t>(ceil_div(n, kThreads * 8), (int64_t)kSms * 8);
    k_os_hist<K><<<hg, kThreads, 0, s>>>(keys, n, n_dev, passes, ghist);
    DIM3_LAUNCHED();
    K* src = keys;
    K* dst = keys_alt;
    uint32_t* sv = vals;
    uint32_t* dv = vals_alt;
    for (int p = 0; p < passes; ++p) {
        unsigned long long* next = p + 1 < passes ? st[(p + 1) & 1] : nullptr;
        if (vals)
            os_pass_launch<K, true>(src, sv, dst, dv, n, n_dev, p, ghist, st[p & 1], next, ticket + p, fault, s);
        else
            os_pass_launch<K, false>(src, nullptr, dst, nullptr, n, n_dev, p, ghist, st[p & 1], next, ticket + p, fault,
                                     s);
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
                    int bits, cudaStream_t s, const int64_t* n_dev) {
    radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, s, n_dev);
}
void radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                    int bits, cudaStream_t s, const int64_t* n_dev) {
    radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, bits, s, n_dev);
}

// ------------------------------------------------------------------ unique
// Drop adjacent duplicates in one launch: every CTA flags the first key of
// each run in its tile of kScanTile keys, finds the tile's output offset by
// decoupled look-back (as k_scan_lb) and scatters its kept keys; the last tile
// writes the number kept to *count. Keys at or past *m_dev (when given) are
// ignored.
template <typename K>
__global__ void __launch_bounds__(kThreads) k_unique_lb(const K* __restrict__ in, int64_t n, const int64_t* m_dev,
                                                        K* __restrict__ out, int64_t* count, int64_t n_tiles,
                                                        unsigned long long* status, unsigned long long* ticket,
                                                        int* err, int* fault) {
    __shared__ int64_t s_warp[kThreads / 32 + 1];
    __shared__ int64_t s_blk, s_pre;
    if (threadIdx.x == 0) s_blk = (int64_t)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t b = s_blk;
    const int64_t m = m_dev ? min64(n, *m_dev) : n;
    const int64_t base = b * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned keep = 0u;
    int c = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        if (i < m && (i == 0 || in[i] != in[i - 1])) {
            keep |= 1u << j;
            ++c;
        }
    }
    int64_t tot;
    const int64_t ex = block_exclusive_scan<int64_t, kThreads>((int64_t)c, &tot, s_warp);
    if ((threadIdx.x >> 5) == 0) {
        const int64_t pre = lookback_prefix(status, b, tot, err, kScanWaitNs);
        if ((threadIdx.x & 31) == 0) {
            s_pre = pre < 0 ? 0 : pre;
            if (pre < 0) *static_cast<volatile int*>(fault) = 1;
        }
    }
    __syncthreads();
    int64_t pos = s_pre + ex;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if ((keep >> j) & 1u) out[pos++] = in[base + j];
    if (b == n_tiles - 1 && threadIdx.x == 0) *count = s_pre + tot;
}

template <typename K>
static const int64_t* unique_enqueue(const K* in, K* out, int64_t n, cudaStream_t s, const int64_t* n_dev,
                                     DevBuf& pos) {
    if (n == 0) {
        pos.alloc(sizeof(int64_t), s);
        fill_i64(pos.as<int64_t>(), 0, 1, s);
        return pos.as<int64_t>();
    }
    const int64_t nb = ceil_div(n, kScanTile);
    DIM3_REQUIRE(nb < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "unique input too long");
    // count, ticket, error word, then one status word per tile
    pos.alloc((size_t)(nb + 3) * sizeof(unsigned long long), s);
    DIM3_CUDA(cudaMemsetAsync(pos.p, 0, pos.bytes, s));
    unsigned long long* w = pos.as<unsigned long long>();
    k_unique_lb<K><<<(unsigned)nb, kThreads, 0, s>>>(in, n, n_dev, out, pos.as<int64_t>(), nb, w + 3, w + 1,
                                                     reinterpret_cast<int*>(w + 2), wait_fault_flag());
    DIM3_LAUNCHED();
    return pos.as<int64_t>();
}

template <typename K>
static int64_t unique_impl(const K* in, K* out, int64_t n, cudaStream_t s, const int64_t* n_dev) {
    if (n == 0) return 0;
    DevBuf pos;
    return read_i64(unique_enqueue<K>(in, out, n, s, n_dev, pos), s);
}

const int64_t* unique_sorted_u32_async(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s,
                                       const int64_t* n_dev, DevBuf& pos) {
    return unique_enqueue<uint32_t>(in, out, n, s, n_dev, pos);
}
const int64_t* unique_sorted_u64_async(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                                       const int64_t* n_dev, DevBuf& pos) {
    return unique_enqueue<uint64_t>(in, out, n, s, n_dev, pos);
}

int64_t unique_sorted_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s, const int64_t* n_dev) {
    return unique_impl<uint32_t>(in, out, n, s, n_dev);
}
int64_t unique_sorted_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s, const int64_t* n_dev) {
    return unique_impl<uint64_t>(in, out, n, s, n_dev);
}

// ----------------------------------------------------------------- rowptr
// Position i (0..n) writes rowptr[r] = i for the rows r in (row(i-1), row(i)]
// (row(-1) = -1, row(n) = n_rows): one coalesced pass over the keys, every
// row pointer written once; rows without keys take the next row's start.
template <typename K>
__global__ void k_rowptr(const K* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = i == 0 ? -1 : min64((int64_t)(keys[i - 1] >> shift), n_rows);
        const int64_t cur = i == n ? n_rows : min64((int64_t)(keys[i] >> shift), n_rows);
        for (int64_t r = prev + 1; r <= cur; ++r) rowptr[r] = i;
    }
}

void rowptr_from_sorted_u32(const uint32_t* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr,
                            cudaStream_t s) {
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n + 1, kThreads), 8192);
    k_rowptr<uint32_t><<<g, kThreads, 0, s>>>(keys, n, shift, n_rows, rowptr);
    DIM3_LAUNCHED();
}
void rowptr_from_sorted_u64(const uint64_t* keys, int64_t n, int shift, int64_t n_rows, int64_t* rowptr,
                            cudaStream_t s) {
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(n + 1, kThreads), 8192);
    k_rowptr<uint64_t><<<g, kThreads, 0, s>>>(keys, n, shift, n_rows, rowptr);
    DIM3_LAUNCHED();
}

}  // namespace dimcube
