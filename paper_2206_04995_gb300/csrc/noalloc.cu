// dim3_map_noalloc: the order-preserving value mapping for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocator) at the time they
// need a mapping: a host engine that hands the GPU a fixed memory budget at
// start-up and forbids later device allocations, code running inside another
// framework's allocator regime, or latency-critical code that must not take
// the allocator's locks or trigger its synchronisations. For them this entry
// point keeps all of its scratch in one file-scope device array of fixed size
// (below), shared by every call; the caller passes only the input column and
// the two output buffers.
//
// The work is the same as dim3_map (hash insert of every value, collection
// of the distinct values, LSD radix sort, ranks), done by ONE CTA of 1024
// threads whose phases are separated by __syncthreads, so no second kernel
// launch or grid-wide synchronisation is needed. Columns are limited to
// kNoAllocMaxN values.
#include <mutex>

#include "common.cuh"
#include "device.cuh"

namespace dimcube {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 16;     // values per call
constexpr int64_t kNaSlots = 2 * kNoAllocMaxN;         // hash slots (power of two)
constexpr int kNaThreads = 1024;
// layout of the scratch array (bytes)
constexpr size_t kNaTableOff = 0;                                      // uint64 [kNaSlots]
constexpr size_t kNaRankOff = kNaTableOff + kNaSlots * 8;              // uint32 [kNaSlots]
constexpr size_t kNaSlotOff = kNaRankOff + kNaSlots * 4;               // uint32 [kNoAllocMaxN]
constexpr size_t kNaKeysOff = kNaSlotOff + kNoAllocMaxN * 4;           // uint32 [2][kNoAllocMaxN]
constexpr size_t kNaValsOff = kNaKeysOff + 2 * kNoAllocMaxN * 4;       // uint32 [2][kNoAllocMaxN]
constexpr size_t kNaCountOff = kNaValsOff + 2 * kNoAllocMaxN * 4;      // int64 distinct count
constexpr size_t kNaBytes = kNaCountOff + 256;                         // 2,883,840 bytes

// The scratch of every dim3_map_noalloc call on a device; each GPU that loads
// the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_map_scratch[kNaBytes];

__global__ void __launch_bounds__(kNaThreads, 1) k_map_noalloc(const int32_t* __restrict__ vals, int n,
                                                               int32_t* __restrict__ ids, int32_t* __restrict__ dict,
                                                               unsigned char* scratch) {
    unsigned long long* table = reinterpret_cast<unsigned long long*>(scratch + kNaTableOff);
    uint32_t* rank = reinterpret_cast<uint32_t*>(scratch + kNaRankOff);
    uint32_t* slot = reinterpret_cast<uint32_t*>(scratch + kNaSlotOff);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(scratch + kNaKeysOff),
                         reinterpret_cast<uint32_t*>(scratch + kNaKeysOff) + kNoAllocMaxN};
    uint32_t* pay[2] = {reinterpret_cast<uint32_t*>(scratch + kNaValsOff),
                        reinterpret_cast<uint32_t*>(scratch + kNaValsOff) + kNoAllocMaxN};
    int64_t* count_out = reinterpret_cast<int64_t*>(scratch + kNaCountOff);

    __shared__ uint32_t s_cnt;
    __shared__ uint32_t dig_off[256];
    __shared__ uint32_t tile_tot[256];
    __shared__ uint32_t wcnt[kNaThreads / 32][256];
    const int tid = threadIdx.x;
    const unsigned lane = lane_id(), warp = tid >> 5;

    uint32_t slots = 64;
    while ((int64_t)slots < 2 * (int64_t)n) slots <<= 1;
    const uint32_t mask = slots - 1;

    // the array keeps the previous call's contents: clear the table first
    for (uint32_t i = tid; i < slots; i += kNaThreads) table[i] = 0ull;
    if (tid == 0) s_cnt = 0;
    __syncthreads();

    // 1. insert every value; remember its slot
    for (int i = tid; i < n; i += kNaThreads) {
        const int32_t v = vals[i];
        const unsigned long long key = (1ull << 32) | (uint32_t)v;
        uint32_t h = fmix32((uint32_t)v) & mask;
        for (uint32_t step = 0; step <= mask; ++step) {
            const unsigned long long cur = table[h];
            if (cur == key) break;
            if (cur == 0ull) {
                const unsigned long long old = atomicCAS(&table[h], 0ull, key);
                if (old == 0ull || old == key) break;
            }
            h = (h + 1) & mask;
        }
        slot[i] = h;
    }
    __syncthreads();

    // 2. collect the distinct values as (order key, slot)
    for (uint32_t s = tid; s < slots; s += kNaThreads) {
        const unsigned long long t = table[s];
        if (t) {
            const uint32_t p = atomicAdd(&s_cnt, 1u);
            keys[0][p] = ((uint32_t)t) ^ 0x80000000u;
            pay[0][p] = s;
        }
    }
    __syncthreads();
    const int d = (int)s_cnt;

    // 3. stable LSD radix sort of the d keys, 8-bit digits, tiles of 1024
    for (int pass = 0; pass < 4; ++pass) {
        const int src = pass & 1, dst = src ^ 1, shift = 8 * pass;
        if (tid < 256) dig_off[tid] = 0;
        __syncthreads();
        for (int i = tid; i < d; i += kNaThreads) atomicAdd(&dig_off[(keys[src][i] >> shift) & 255u], 1u);
        __syncthreads();
        if (tid == 0) {
            uint32_t run = 0;
            for (int b = 0; b < 256; ++b) {
                const uint32_t c = dig_off[b];
                dig_off[b] = run;
                run += c;
            }
        }
        __syncthreads();
        for (int t0 = 0; t0 < d; t0 += kNaThreads) {
            for (int i = tid; i < (kNaThreads / 32) * 256; i += kNaThreads) (&wcnt[0][0])[i] = 0u;
            __syncthreads();
            const int idx = t0 + tid;
            const bool valid = idx < d;
            const uint32_t k = valid ? keys[src][idx] : 0u;
            const uint32_t pv = valid ? pay[src][idx] : 0u;
            const unsigned dg = valid ? ((k >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(kFull, dg);
            const uint32_t in_warp = (uint32_t)__popc(peers & lanemask_lt());
            if (valid && (int)lane == __ffs(peers) - 1) wcnt[warp][dg] = (uint32_t)__popc(peers);
            __syncthreads();
            if (tid < 256) {
                uint32_t run = 0;
                for (int w = 0; w < kNaThreads / 32; ++w) {
                    const uint32_t c = wcnt[w][tid];
                    wcnt[w][tid] = run;
                    run += c;
                }
                tile_tot[tid] = run;
            }
            __syncthreads();
            if (valid) {
                const uint32_t pos = dig_off[dg] + wcnt[warp][dg] + in_warp;
                keys[dst][pos] = k;
                pay[dst][pos] = pv;
            }
            __syncthreads();
            if (tid < 256) dig_off[tid] += tile_tot[tid];
            __syncthreads();
        }
    }

    // 4. ranks (four passes leave the sorted data in buffer 0) and the dictionary
    for (int p = tid; p < d; p += kNaThreads) {
        rank[pay[0][p]] = (uint32_t)p;
        dict[p] = (int32_t)(keys[0][p] ^ 0x80000000u);
    }
    __syncthreads();
    for (int i = tid; i < n; i += kNaThreads) ids[i] = (int32_t)rank[slot[i]];
    if (tid == 0) *count_out = d;
}

// Device address of g_map_scratch, looked up once per device with that device current.
static unsigned char* scratch_on_current_device() {
    static std::mutex mu;
    static unsigned char* addr[64] = {nullptr};
    int dev = 0;
    DIM3_CUDA(cudaGetDevice(&dev));
    DIM3_REQUIRE(dev >= 0 && dev < 64, DIM3_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        DIM3_CUDA(cudaGetSymbolAddress(&p, g_map_scratch));
        DIM3_REQUIRE(p != nullptr, DIM3_ERR_CUDA, "no device address for the mapping scratch");
        addr[dev] = static_cast<unsigned char*>(p);
    }
    return addr[dev];
}

void map_noalloc(const int32_t* d_vals, int64_t n, int32_t* d_ids, int32_t* d_dict, int64_t* n_distinct,
                 cudaStream_t s) {
    DIM3_REQUIRE(n >= 0 && (n == 0 || (d_vals && d_ids && d_dict)) && n_distinct, DIM3_ERR_ARG,
                 "bad column arguments");
    DIM3_REQUIRE(n <= kNoAllocMaxN, DIM3_ERR_OVERFLOW,
                 "dim3_map_noalloc takes at most " + std::to_string(kNoAllocMaxN) + " values; got " +
                     std::to_string(n) + " (use dim3_map)");
    unsigned char* scratch = scratch_on_current_device();
    if (n == 0) {
        *n_distinct = 0;
        return;
    }
    k_map_noalloc<<<1, kNaThreads, 0, s>>>(d_vals, (int)n, d_ids, d_dict, scratch);
    DIM3_LAUNCHED();
    DIM3_CUDA(cudaMemcpyAsync(n_distinct, scratch + kNaCountOff, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dimcube
