// Self-test of failure detection without a GPU fault: a decoupled look-back
// (the wait of the one-pass compaction) whose predecessor never publishes
// must give up after its limit, report it, and leave the context usable.
#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

// One warp looks back from block 1 while block 0's status stays 0 (nothing
// ever sets it): lookback_prefix polls until wait_ns has passed, sets *err
// and returns -1, which is stored in *result.
__global__ void k_wait_selftest(unsigned long long* status, int* err, long long* result, uint64_t wait_ns) {
    if (threadIdx.x >= 32) return;
    const int64_t pre = lookback_prefix(status, 1, 0, err, wait_ns);
    if (threadIdx.x == 0) *result = pre;
}

int wait_selftest(double seconds, cudaStream_t s) {
    DIM3_REQUIRE(seconds > 0.0 && seconds <= 2.0, DIM3_ERR_ARG, "self-test wait must lie in (0, 2] s");
    DevBuf status, err, result;
    status.alloc(2 * sizeof(unsigned long long), s);
    err.alloc(8, s);
    result.alloc(8, s);
    DIM3_CUDA(cudaMemsetAsync(status.p, 0, 2 * sizeof(unsigned long long), s));
    DIM3_CUDA(cudaMemsetAsync(err.p, 0, 8, s));
    DIM3_CUDA(cudaMemsetAsync(result.p, 0, 8, s));
    k_wait_selftest<<<1, 32, 0, s>>>(status.as<unsigned long long>(), err.as<int>(), result.as<long long>(),
                                     (uint64_t)(seconds * 1e9));
    DIM3_LAUNCHED();
    const int64_t* src[2] = {err.as<int64_t>(), result.as<int64_t>()};
    int64_t got[2];
    read_i64_n(src, 2, got, s);
    return (got[0] != 0 && got[1] == -1) ? 1 : 0;
}

}  // namespace dimcube
