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
