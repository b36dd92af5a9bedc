// Device-side building blocks: warp/block scans, hashing, lane masks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dimcube {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(kFull, v, o);
        if (lane >= (unsigned)o) v += n;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Exclusive scan over a block of NT threads. `s_warp` is shared scratch of
// NT/32 + 1 elements. Returns this thread's exclusive prefix; *total gets the
// block total. Contains __syncthreads (call from all threads).
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* s_warp) {
    constexpr int NW = NT / 32;
    const unsigned lane = lane_id();
    const unsigned w = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < (unsigned)NW ? s_warp[lane] : T(0);
        T ti = warp_inclusive_scan(t);
        if (lane < (unsigned)NW) s_warp[lane] = ti - t;
        if (lane == NW - 1) s_warp[NW] = ti;
    }
    __syncthreads();
    T res = s_warp[w] + inc - v;
    *total = s_warp[NW];
    __syncthreads();
    return res;
}

template <typename T, int NT>
__device__ __forceinline__ T block_sum(T v, T* s_warp) {
    constexpr int NW = NT / 32;
    const unsigned lane = lane_id();
    const unsigned w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) s_warp[w] = v;
    __syncthreads();
    if (w == 0) {
        T t = lane < (unsigned)NW ? s_warp[lane] : T(0);
        t = warp_sum(t);
        if (lane == 0) s_warp[NW] = t;
    }
    __syncthreads();
    T r = s_warp[NW];
    __syncthreads();
    return r;
}

// Block-aggregated append: every thread with `want` gets a distinct slot in
// [base, base + block total) of a global counter, with ONE atomicAdd per block
// (instead of one per warp). Call from all threads of the block; s_cnt is
// shared scratch of NT/32 + 2 entries.
template <int NT>
__device__ __forceinline__ unsigned long long block_append(bool want, unsigned long long* counter,
                                                           unsigned long long* s_cnt) {
    constexpr int NW = NT / 32;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(kFull, want);
    if (lane == 0) s_cnt[w] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < NW; ++i) {
            const unsigned long long c = s_cnt[i];
            s_cnt[i] = run;
            run += c;
        }
        s_cnt[NW] = run ? atomicAdd(counter, run) : 0ull;
    }
    __syncthreads();
    const unsigned long long pos = s_cnt[NW] + s_cnt[w] + __popc(b & lanemask_lt());
    __syncthreads();
    return pos;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Decoupled look-back (single-pass prefix sum across CTAs). status[b] holds a
// flag in its top two bits (0 none yet, 1 aggregate of block b, 2 inclusive
// prefix up to b) and the value in the rest. Blocks take logical numbers in
// dispatch order (a ticket), so a block only waits on blocks that are already
// running. Called by one whole warp; returns the exclusive prefix of block b
// (the same in every lane), or -1 if a predecessor did not publish within
// wait_ns (then *err is set and a placeholder is published so that the blocks
// after this one do not wait either).
constexpr unsigned long long kLbAgg = 1ull << 62, kLbInc = 2ull << 62, kLbVal = (1ull << 62) - 1;

__device__ __forceinline__ int64_t lookback_prefix(unsigned long long* status, int64_t b, int64_t aggregate, int* err,
                                                   uint64_t wait_ns) {
    const int lane = lane_id();
    if (b == 0) {
        if (lane == 0) atomicExch(&status[0], kLbInc | (unsigned long long)aggregate);
        return 0;
    }
    if (lane == 0) atomicExch(&status[b], kLbAgg | (unsigned long long)aggregate);
    int64_t prefix = 0, j = b - 1;
    const uint64_t t0 = global_ns();
    uint32_t polls = 0;
    while (true) {
        const int64_t idx = j - lane;
        const unsigned long long v = idx >= 0 ? ld_relaxed_u64(&status[idx]) : kLbInc;
        if (!__all_sync(kFull, (v >> 62) != 0ull)) {
            const bool late = ((++polls & 63u) == 0u) && (global_ns() - t0 > wait_ns);
            if (__any_sync(kFull, late)) {
                if (lane == 0) atomicExch(err, 1);
                prefix = -1;
                break;
            }
            continue;
        }
        const unsigned inc = __ballot_sync(kFull, (v >> 62) == 2ull);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        prefix += warp_sum(lane <= stop ? (int64_t)(v & kLbVal) : (int64_t)0);
        if (inc) break;
        j -= 32;
    }
    if (lane == 0) atomicExch(&status[b], kLbInc | (unsigned long long)((prefix < 0 ? 0 : prefix) + aggregate));
    return prefix;
}

// Split form of lookback_prefix for blocks that publish their aggregate and
// resolve their prefix later (with other work in between): lookback_publish
// stores block b's aggregate (block 0: its inclusive prefix); lookback_resolve
// (one whole warp) then waits for the predecessors as lookback_prefix does
// and stores b's inclusive prefix. Same return and failure behaviour.
__device__ __forceinline__ void lookback_publish(unsigned long long* status, int64_t b, int64_t aggregate) {
    atomicExch(&status[b], (b == 0 ? kLbInc : kLbAgg) | (unsigned long long)aggregate);
}

__device__ __forceinline__ int64_t lookback_resolve(unsigned long long* status, int64_t b, int64_t aggregate, int* err,
                                                    uint64_t wait_ns) {
    const int lane = lane_id();
    if (b == 0) return 0;
    int64_t prefix = 0, j = b - 1;
    const uint64_t t0 = global_ns();
    uint32_t polls = 0;
    while (true) {
        const int64_t idx = j - lane;
        const unsigned long long v = idx >= 0 ? ld_relaxed_u64(&status[idx]) : kLbInc;
        if (!__all_sync(kFull, (v >> 62) != 0ull)) {
            const bool late = ((++polls & 63u) == 0u) && (global_ns() - t0 > wait_ns);
            if (__any_sync(kFull, late)) {
                if (lane == 0) atomicExch(err, 1);
                prefix = -1;
                break;
            }
            continue;
        }
        const unsigned inc = __ballot_sync(kFull, (v >> 62) == 2ull);
        const int stop = inc ? __ffs(inc) - 1 : 31;
        prefix += warp_sum(lane <= stop ? (int64_t)(v & kLbVal) : (int64_t)0);
        if (inc) break;
        j -= 32;
    }
    if (lane == 0) atomicExch(&status[b], kLbInc | (unsigned long long)((prefix < 0 ? 0 : prefix) + aggregate));
    return prefix;
}

// 32-bit finaliser of MurmurHash3 (Appleby): spreads keys over table slots.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// first index in [lo, hi) with a[i] >= v (a ascending)
template <typename T>
__device__ __forceinline__ int64_t lower_bound_dev(const T* a, int64_t lo, int64_t hi, T v) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace dimcube
