// Step 1 of Algorithm 1: mapping column values to consecutive natural
// numbers (Section 2.2).
//
// GPU form: an open-addressing linear-probing hash table (the paper's
// Optimization 3 uses linear probing too) is filled by all threads at once;
// the distinct keys are collected and radix-sorted, and each distinct value's
// id is its rank. Ranks, unlike first-seen numbering, do not depend on the
// order in which threads reach the table, so the mapping is deterministic and
// order-preserving (id order = signed value order).
//
// Batches of independent instances map (instance, value) pairs instead of
// values: the instance index is part of the key and the most significant
// part of the sort order, so the ids of instance i form one contiguous block
// that precedes instance i + 1's, and equal values of different instances
// never share an id (hence never join).
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

constexpr uint32_t kNoSlot = 0xffffffffu;

// slot content: occupied flag | instance | value
__device__ __forceinline__ unsigned long long table_key(int32_t v, int32_t tag) {
    return (1ull << 63) | ((unsigned long long)(uint32_t)tag << 32) | (unsigned long long)(uint32_t)v;
}

__device__ __forceinline__ uint32_t slot_hash(int32_t v, int32_t tag) {
    return fmix32((uint32_t)v ^ ((uint32_t)tag * 0x9E3779B9u));
}

// Insert every value (rows with pred < 0 skipped); slot_out[i] = its slot.
__global__ void k_hash_insert(const int32_t* __restrict__ vals, const int32_t* __restrict__ tags,
                              const int32_t* __restrict__ pred, int64_t n, unsigned long long* table, uint32_t mask,
                              uint32_t* __restrict__ slot_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (pred && pred[i] < 0) {
            slot_out[i] = kNoSlot;
            continue;
        }
        const int32_t v = vals[i];
        const int32_t tg = tags ? tags[i] : 0;
        const unsigned long long key = table_key(v, tg);
        uint32_t h = slot_hash(v, tg) & mask;
        // The table holds at least twice as many slots as rows, so the probe
        // sequence always reaches the key or an empty slot within mask+1 steps.
        for (uint32_t step = 0; step <= mask; ++step) {
            unsigned long long cur = table[h];
            if (cur == key) break;
            if (cur == 0ull) {
                unsigned long long old = atomicCAS(&table[h], 0ull, key);
                if (old == 0ull || old == key) break;
            }
            h = (h + 1) & mask;
        }
        slot_out[i] = h;
    }
}

// Append every occupied slot's (order key, slot) to the output arrays. The
// order key compares like (instance, signed value).
template <typename K>
__global__ void k_hash_collect(const unsigned long long* table, int64_t cap, K* okeys, uint32_t* oslots,
                               unsigned long long* counter) {
    __shared__ unsigned long long s_cnt[kThreads / 32 + 2];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t iters = (cap + stride - 1) / stride;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t s = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const unsigned long long t = s < cap ? table[s] : 0ull;
        const bool occ = t != 0ull;
        const unsigned long long pos = block_append<kThreads>(occ, counter, s_cnt);
        if (occ) {
            const uint64_t tag = (t >> 32) & 0x7fffffffull;
            okeys[pos] = (K)((tag << 32) | (uint64_t)(((uint32_t)t) ^ 0x80000000u));
            oslots[pos] = (uint32_t)s;
        }
    }
}

template <typename K>
__global__ void k_hash_rank(const K* skeys, const uint32_t* sslots, int64_t d, const int64_t* d_dev, uint32_t* rank,
                            int32_t* dict_out, int32_t* dict_tag_out) {
    if (d_dev) d = min64(d, *d_dev);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < d;
         p += (int64_t)gridDim.x * blockDim.x) {
        rank[sslots[p]] = (uint32_t)p;
        const uint64_t k = (uint64_t)skeys[p];
        dict_out[p] = (int32_t)(((uint32_t)k) ^ 0x80000000u);
        if (dict_tag_out) dict_tag_out[p] = (int32_t)(k >> 32);
    }
}

__global__ void k_gather_rank(const uint32_t* slot, int64_t n, const uint32_t* rank, int32_t* ids) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = slot[i];
        ids[i] = s == kNoSlot ? -1 : (int32_t)rank[s];
    }
}

__global__ void k_hash_probe(const int32_t* __restrict__ vals, const int32_t* __restrict__ tags, int64_t n,
                             const unsigned long long* table, uint32_t mask, const uint32_t* __restrict__ rank,
                             int32_t* __restrict__ ids) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = vals[i];
        const int32_t tg = tags ? tags[i] : 0;
        const unsigned long long key = table_key(v, tg);
        uint32_t h = slot_hash(v, tg) & mask;
        int32_t id = -1;
        for (uint32_t step = 0; step <= mask; ++step) {
            const unsigned long long cur = table[h];
            if (cur == key) {
                id = (int32_t)rank[h];
                break;
            }
            if (cur == 0ull) break;
            h = (h + 1) & mask;
        }
        ids[i] = id;
    }
}

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

// With read_count the distinct count is read at once (one synchronisation);
// otherwise it stays on the device (vm.count) and the sort and the ranking
// take it from there, so that several maps can share one host read.
template <typename K>
static void collect_sort_rank(ValueMap& vm, int64_t cap, int64_t n, int tag_bits, int32_t* dict_out,
                              int32_t* dict_tag_out, bool read_count, cudaStream_t s) {
    DevBuf keys, sl, keys_alt, sl_alt;
    vm.count.alloc(8, s);
    DIM3_CUDA(cudaMemsetAsync(vm.count.p, 0, 8, s));
    keys.alloc((size_t)n * sizeof(K), s);
    sl.alloc((size_t)n * 4, s);
    k_hash_collect<K><<<grid_for(cap), kThreads, 0, s>>>(vm.table.as<unsigned long long>(), cap, keys.as<K>(),
                                                          sl.as<uint32_t>(), vm.count.as<unsigned long long>());
    DIM3_LAUNCHED();
    int64_t d = n;  // bound (distinct values <= rows)
    const int64_t* d_dev = vm.count.as<int64_t>();
    vm.n_distinct = -1;
    if (read_count) {
        d = read_i64(d_dev, s);
        DIM3_REQUIRE(d >= 0 && d <= n, DIM3_ERR_CUDA, "value map: inconsistent distinct count");
        vm.n_distinct = d;
        d_dev = nullptr;
    }
    keys_alt.alloc((size_t)std::max<int64_t>(d, 1) * sizeof(K), s);
    sl_alt.alloc((size_t)std::max<int64_t>(d, 1) * 4, s);
    if constexpr (sizeof(K) == 4)
        radix_sort_u32(keys.as<uint32_t>(), sl.as<uint32_t>(), keys_alt.as<uint32_t>(), sl_alt.as<uint32_t>(), d, 32,
                       s, d_dev);
    else
        radix_sort_u64(keys.as<uint64_t>(), sl.as<uint32_t>(), keys_alt.as<uint64_t>(), sl_alt.as<uint32_t>(), d,
                       32 + tag_bits, s, d_dev);
    k_hash_rank<K><<<grid_for(d), kThreads, 0, s>>>(keys.as<K>(), sl.as<uint32_t>(), d, d_dev, vm.rank.as<uint32_t>(),
                                                     dict_out, dict_tag_out);
    DIM3_LAUNCHED();
}

int64_t resolve_counts(ValueMap* const* maps, int n_maps, const int64_t* extra, int64_t* extra_out, cudaStream_t s) {
    DIM3_REQUIRE(n_maps >= 0 && n_maps <= 7, DIM3_ERR_ARG, "resolve_counts: at most 7 maps");
    const int64_t* src[8];
    int64_t got[8];
    int k = 0;
    for (int i = 0; i < n_maps; ++i)
        if (maps[i]->n_distinct < 0) src[k++] = maps[i]->count.as<int64_t>();
    const int n_counts = k;
    if (extra) src[k++] = extra;
    if (k == 0) return 0;
    read_i64_n(src, k, got, s);
    k = 0;
    for (int i = 0; i < n_maps; ++i)
        if (maps[i]->n_distinct < 0) maps[i]->n_distinct = got[k++];
    if (extra) *extra_out = got[n_counts];
    return n_counts;
}

void build_value_map(const int32_t* vals, const int32_t* tags, int n_tags, const int32_t* pred, int64_t n,
                     ValueMap& vm, int32_t* ids_out, int32_t* dict_out, int32_t* dict_tag_out, cudaStream_t s,
                     bool read_count) {
    int64_t cap = 64;
    while (cap < 2 * n) cap <<= 1;
    DIM3_REQUIRE(cap <= (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "column too long for the value map");
    vm.mask = (uint32_t)(cap - 1);
    vm.table.alloc((size_t)cap * 8, s);
    vm.rank.alloc((size_t)cap * 4, s);
    DIM3_CUDA(cudaMemsetAsync(vm.table.p, 0, (size_t)cap * 8, s));
    vm.n_distinct = 0;
    if (n == 0) return;
    DevBuf slots;
    slots.alloc((size_t)n * 4, s);
    k_hash_insert<<<grid_for(n), kThreads, 0, s>>>(vals, tags, pred, n, vm.table.as<unsigned long long>(), vm.mask,
                                                    slots.as<uint32_t>());
    DIM3_LAUNCHED();
    if (tags && n_tags > 1)
        collect_sort_rank<uint64_t>(vm, cap, n, bits_for(n_tags), dict_out, dict_tag_out, read_count, s);
    else
        collect_sort_rank<uint32_t>(vm, cap, n, 0, dict_out, dict_tag_out, read_count, s);
    k_gather_rank<<<grid_for(n), kThreads, 0, s>>>(slots.as<uint32_t>(), n, vm.rank.as<uint32_t>(), ids_out);
    DIM3_LAUNCHED();
}

void build_value_map(const int32_t* vals, const int32_t* pred, int64_t n, ValueMap& vm, int32_t* ids_out,
                     int32_t* dict_out, cudaStream_t s) {
    build_value_map(vals, nullptr, 1, pred, n, vm, ids_out, dict_out, nullptr, s);
}

void probe_value_map(const ValueMap& vm, const int32_t* vals, const int32_t* tags, int64_t n, int32_t* ids_out,
                     cudaStream_t s) {
    if (n == 0) return;
    k_hash_probe<<<grid_for(n), kThreads, 0, s>>>(vals, tags, n, vm.table.as<unsigned long long>(), vm.mask,
                                                   vm.rank.as<uint32_t>(), ids_out);
    DIM3_LAUNCHED();
}

}  // namespace dimcube
