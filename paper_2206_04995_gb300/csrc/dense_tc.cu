// DenseEC on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Algorithm 3 asks, for each x and each dense z, whether Bitmap_x AND
// Bitmap_z has a set bit; the MM formulation of Section 1.1 gives the same
// answer as C[x][z] = sum_y R[x][y] * S[y][z] > 0. Here R_dense and S_dense
// are stored as 0/1 e4m3 bytes (K-major) and multiplied with
// tcgen05.mma.kind::f8f6f4 into FP32 accumulators in tensor memory. The
// accumulation is exact (at most K < 2^24 ones), so C is the exact count of
// common y: thresholded > 0 it is DenseEC's answer, read as is it is the
// Join-Count. The paper's early stop has no tensor-core analog; the tile
// runs over all of K.
//
// One CTA computes a 128 x N tile of C (128 TMEM lanes x N FP32 columns, N =
// 256 or 128, the DIM3_OPT_DENSE_TILE_N option):
//   warp 0, one lane : TMA producer, a ring of (A 16 KB, B N x 128 B) tiles
//                      (4 stages for N = 256, 6 for N = 128) with 128-byte
//                      swizzle, one mbarrier pair per stage;
//   warp 1, one lane : MMA issuer, 4 x (M128 N K32) per stage, commits to
//                      the stage's "empty" barrier and finally to "done";
//   warps 0-3        : epilogue, each warp reads its 32 TMEM lanes with
//                      tcgen05.ld and writes result bits (or counts).
// Every mbarrier wait is bounded; a wait that gives up records an error flag
// that the host turns into DIM3_ERR_TIMEOUT, and TMEM is always freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dense_tc.cuh"
#include "device.cuh"

namespace dimcube {

constexpr int kTcThreads = 128;
constexpr uint32_t kStageBytesA = kTcTileM * kTcBlockK;  // 16 KiB
constexpr uint32_t kWaitLimit = 1u << 26;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kGroupM = 16;  // row tiles per raster group (see k_dense_tc)

// Pipeline shape of a CTA computing a 128 x N tile (N = 256 or 128): the B
// tile of a stage is N rows of 128 K bytes; narrower tiles afford more stages.
template <int N>
struct TcShape {
    static constexpr int kStages = N == 256 ? 4 : 6;
    static constexpr uint32_t kStageBytesB = (uint32_t)N * kTcBlockK;
    static constexpr uint32_t kStageBytes = kStageBytesA + kStageBytesB;
    static constexpr uint32_t kTmemCols = N;  // one FP32 column per output column
    static constexpr uint32_t kSmem = kStages * kStageBytes + 1024 + 256;
    // Instruction descriptor of tcgen05.mma.kind::f8f6f4: D = F32 (bits 4-5 =
    // 1), A = B = E4M3 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0),
    // N >> 3 in bits 17-22, M >> 4 in bits 24-28.
    static constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) |
                                       ((uint32_t)(kTcTileM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on the phase with the given parity: gives up (returns false)
// after kWaitNs nanoseconds of wall time or kWaitLimit polls, whichever first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int32_t c0, int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row swizzle atoms 1024 bytes apart
// (stride byte offset), descriptor version 1, layout code 2 (SWIZZLE_128B).
// The leading byte offset is unused for swizzled K-major tiles.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Tile order: without a tile list the CTAs run down groups of kGroupM row
// tiles, the row tile changing fastest (b = group * kGroupM * n_n + n * gm +
// m_in_group), so CTAs that run together share their B tiles (each read by
// up to kGroupM CTAs in a row) and a group's A tiles stay in L2 while it
// sweeps every column tile.
template <int kKind, int N>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dense_tc(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b, int64_t rows,
               int64_t n_zd, int num_kb, uint32_t* __restrict__ d_bits, int64_t zdw, int32_t* __restrict__ d_cnt,
               int* err, const int2* __restrict__ tiles, int n_m, int n_n) {
    using Sh = TcShape<N>;
    constexpr int kStages = Sh::kStages;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kStageBytesA;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * Sh::kStageBytesB);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tm, tn;
    if (tiles) {
        // batches compute only the tiles of the block-diagonal (tile list)
        tm = tiles[blockIdx.x].x;
        tn = tiles[blockIdx.x].y;
    } else {
        const int b = (int)blockIdx.x, per_group = kGroupM * n_n;
        const int g = b / per_group, r = b - g * per_group;
        const int first = g * kGroupM, gm = min(kGroupM, n_m - first);
        tm = first + r % gm;
        tn = r / gm;
    }
    const int64_t m0 = (int64_t)tm * kTcTileM;
    const int64_t n0 = (int64_t)tn * N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap_b)) : "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, Sh::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        for (int kb = 0; kb < num_kb; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) {
                s_abort = 1;
                atomicExch(err, 1);
                break;
            }
            if (s_abort) break;
            mbar_expect_tx(&full[s], Sh::kStageBytes);
            tma_load_2d(sA + s * kStageBytesA, &tmap_a, &full[s], kb * kTcBlockK, (int32_t)m0);
            tma_load_2d(sB + s * Sh::kStageBytesB, &tmap_b, &full[s], kb * kTcBlockK, (int32_t)n0);
        }
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < num_kb; ++kb) {
            const int s = kb % kStages;
            const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                s_abort = 1;
                atomicExch(err, 2);
                break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sA + s * kStageBytesA);
            const uint32_t b_addr = smem_u32(sB + s * Sh::kStageBytesB);
#pragma unroll
            for (int k = 0; k < kTcBlockK / 32; ++k)
                tc_mma(tmem, smem_desc_sw128(a_addr + 32u * k), smem_desc_sw128(b_addr + 32u * k), Sh::kIdesc,
                       (kb | k) != 0 ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        tc_commit(done);
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes (= tile rows) 32w .. 32w + 31
    bool ok = mbar_wait(done, 0);
    ok = __all_sync(kFull, ok && !s_abort);
    tc_fence_after();
    if (ok) {
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
            if (kKind == 0) {
                uint32_t word = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) word |= (__uint_as_float(v[j]) > 0.0f ? 1u : 0u) << j;
                const int64_t wi = (n0 + c0) >> 5;
                if (row < rows && wi < zdw) d_bits[row * zdw + wi] = word;
            } else {
                if (row < rows) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t col = n0 + c0 + j;
                        if (col < n_zd) d_cnt[row * n_zd + col] = (int32_t)__uint_as_float(v[j]);
                    }
                }
            }
        }
    } else if (lane == 0) {
        atomicExch(err, 3);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, Sh::kTmemCols);
    }
}

// ----------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        DIM3_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        DIM3_REQUIRE(q == cudaDriverEntryPointSuccess && p, DIM3_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D K-major uint8 tensor [outer][inner], box = (kTcBlockK, box_outer), 128B swizzle.
static CUtensorMap make_map(const uint8_t* ptr, int64_t inner, int64_t outer, uint32_t box_outer) {
    DIM3_REQUIRE((reinterpret_cast<uintptr_t>(ptr) & 15u) == 0, DIM3_ERR_ARG, "tensor map base not 16-byte aligned");
    DIM3_REQUIRE(inner % kTcBlockK == 0 && outer % box_outer == 0, DIM3_ERR_ARG, "tensor map extents not padded");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner};
    cuuint32_t box[2] = {(cuuint32_t)kTcBlockK, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(ptr), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    DIM3_REQUIRE(r == CUDA_SUCCESS, DIM3_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

bool tc_supported(const Ctx& ctx) { return ctx.cc_major == 10 && ctx.cc_minor == 3; }

int tc_tile_n(const Ctx& ctx) { return ctx.opt.dense_tile_n == 128 ? 128 : 256; }

template <int N>
static void launch_tc(const Ctx& ctx, const uint8_t* A, int64_t rows, int64_t rows_pad, const uint8_t* B,
                      int64_t n_zd, int64_t n_pad, int64_t k_pad, int kind, uint32_t* d_bits, int64_t zdw,
                      int32_t* d_cnt, const int2* tiles, int64_t n_tiles, int* err, cudaStream_t s) {
    using Sh = TcShape<N>;
    static bool attr_done[64] = {false};
    if (!attr_done[ctx.device & 63]) {
        DIM3_CUDA(cudaFuncSetAttribute(k_dense_tc<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::kSmem));
        DIM3_CUDA(cudaFuncSetAttribute(k_dense_tc<1, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::kSmem));
        attr_done[ctx.device & 63] = true;
    }
    DIM3_REQUIRE(n_pad % N == 0, DIM3_ERR_ARG, "dense operand not padded to the tile width");
    const CUtensorMap ma = make_map(A, k_pad, rows_pad, kTcTileM);
    const CUtensorMap mb = make_map(B, k_pad, n_pad, N);
    const int n_m = (int)(rows_pad / kTcTileM), n_n = (int)(n_pad / N);
    const int64_t blocks = tiles ? n_tiles : (int64_t)n_m * n_n;
    DIM3_REQUIRE(blocks < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "too many DenseEC tiles");
    const int num_kb = (int)(k_pad / kTcBlockK);
    PhaseScope phase(ctx.stats, PH_DENSE_TC, s);
    if (kind == 0)
        k_dense_tc<0, N><<<(unsigned)blocks, kTcThreads, Sh::kSmem, s>>>(ma, mb, rows, n_zd, num_kb, d_bits, zdw,
                                                                         nullptr, err, tiles, n_m, n_n);
    else
        k_dense_tc<1, N><<<(unsigned)blocks, kTcThreads, Sh::kSmem, s>>>(ma, mb, rows, n_zd, num_kb, nullptr, zdw,
                                                                         d_cnt, err, tiles, n_m, n_n);
    DIM3_LAUNCHED();
}

void tc_dense_product(const Ctx& ctx, const uint8_t* A, int64_t rows, int64_t rows_pad, const uint8_t* B, int64_t n_zd,
                      int64_t n_pad, int64_t k_pad, int kind, uint32_t* d_bits, int64_t zdw, int32_t* d_cnt,
                      const int2* tiles, int64_t n_tiles, cudaStream_t s) {
    if (rows <= 0 || n_zd <= 0 || (tiles && n_tiles <= 0)) return;
    DIM3_REQUIRE(tc_supported(ctx), DIM3_ERR_UNSUPPORTED, "tensor-core DenseEC needs an sm_103 device");
    DIM3_REQUIRE(k_pad > 0 && k_pad < kTcMaxK, DIM3_ERR_OVERFLOW, "DenseEC K exceeds the exact FP32 range");
    DevBuf err;
    err.alloc(sizeof(int), s);
    DIM3_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    if (tc_tile_n(ctx) == 128)
        launch_tc<128>(ctx, A, rows, rows_pad, B, n_zd, n_pad, k_pad, kind, d_bits, zdw, d_cnt, tiles, n_tiles,
                       err.as<int>(), s);
    else
        launch_tc<256>(ctx, A, rows, rows_pad, B, n_zd, n_pad, k_pad, kind, d_bits, zdw, d_cnt, tiles, n_tiles,
                       err.as<int>(), s);
    int h = 0;
    DIM3_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    DIM3_REQUIRE(h == 0, DIM3_ERR_TIMEOUT, "tensor-core DenseEC: a pipeline wait gave up (code " + std::to_string(h) + ")");
}

}  // namespace dimcube
