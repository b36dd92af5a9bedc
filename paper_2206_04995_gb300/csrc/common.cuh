// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dim3.h"

namespace dimcube {

// Error carried from deep inside the library to the C ABI boundary.
struct Error : std::runtime_error {
    int status;
    Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define DIM3_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            int st_ = (e_ == cudaErrorMemoryAllocation) ? DIM3_ERR_NOMEM : DIM3_ERR_CUDA;  \
            throw ::dimcube::Error(st_, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)

// Every kernel launch of the library is followed by DIM3_LAUNCHED(): it checks
// the launch and counts it (dim3_launch_count).
void count_launch();
#define DIM3_LAUNCHED()                 \
    do {                                \
        ::dimcube::count_launch();      \
        DIM3_CUDA(cudaGetLastError());  \
    } while (0)

#define DIM3_REQUIRE(cond, status, msg)                 \
    do {                                                \
        if (!(cond)) throw ::dimcube::Error((status), (msg)); \
    } while (0)

constexpr int kThreads = 256;
constexpr int kSms = 152;  // GB300; the real count is queried at context creation

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int bits_for(int64_t n) {  // bits needed to store values 0..n-1 (at least 1)
    int b = 1;
    while (b < 62 && (int64_t(1) << b) < n) ++b;
    return b;
}

// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; s = o.s;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t n, cudaStream_t st) {
        release();
        s = st;
        bytes = n;
        if (n == 0) return;
        cudaError_t e = cudaMallocAsync(&p, n, st);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            throw Error(DIM3_ERR_NOMEM, "device allocation of " + std::to_string(n) +
                                            " bytes failed: " + cudaGetErrorString(e));
        }
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
    // free in stream st's order from now on (after st has been made to wait
    // for the stream the buffer was last used on)
    void adopt(cudaStream_t st) { s = st; }
};

// ---------------------------------------------------------------- launchers
// primitives (prims.cu)
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);  // out[n+1]
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
void fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t s);
// p[0] = a, p[1] = b in stream order (no host synchronisation, unlike a copy
// from pageable host memory)
void store_i64_pair(int64_t* p, int64_t a, int64_t b, cudaStream_t s);
int64_t read_i64(const int64_t* d, cudaStream_t s);  // synchronising read of one device value
// h[i] = *d[i] for i < n (n <= 16) with ONE synchronisation
void read_i64_n(const int64_t* const* d, int n, int64_t* h, cudaStream_t s);
// A bounded device wait that gives up stores 1 to this process-wide flag
// (pinned, mapped host memory); raise_if_wait_fault(), called after
// synchronisations (read_i64, the end of every C-ABI call), turns it into
// DIM3_ERR_TIMEOUT once and clears it.
int* wait_fault_flag();
void raise_if_wait_fault();
// LSD radix sort of n keys (32- or 64-bit) on their low `bits` bits, with an
// optional uint32 payload. Results end in keys/vals (the alt buffers are scratch).
// Stable; one-sweep passes (a tile that waits on its predecessors for more than
// 2 s gives up and sets the wait-fault flag). With n_dev, the count is
// min(n, *n_dev) read on the device (n then only bounds it), so no host read
// has to precede the sort.
void radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                    int64_t n, int bits, cudaStream_t s, const int64_t* n_dev = nullptr);
void radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                    int64_t n, int bits, cudaStream_t s, const int64_t* n_dev = nullptr);
// Drop adjacent duplicates of sorted keys; returns the count (synchronising).
// With n_dev the input is in[0, min(n, *n_dev)).
int64_t unique_sorted_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s,
                          const int64_t* n_dev = nullptr);
int64_t unique_sorted_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                          const int64_t* n_dev = nullptr);
// Enqueue-only forms: no host read; the count is left on the device at the
// returned address (inside pos, which the caller keeps alive).
const int64_t* unique_sorted_u32_async(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s,
                                       const int64_t* n_dev, DevBuf& pos);
const int64_t* unique_sorted_u64_async(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                                       const int64_t* n_dev, DevBuf& pos);
// rowptr[r] = first index i with (keys[i] >> shift) >= r, for r = 0..n_rows
void rowptr_from_sorted_u32(const uint32_t* keys, int64_t n, int shift, int64_t n_rows,
                            int64_t* rowptr, cudaStream_t s);
void rowptr_from_sorted_u64(const uint64_t* keys, int64_t n, int shift, int64_t n_rows,
                            int64_t* rowptr, cudaStream_t s);

}  // namespace dimcube
