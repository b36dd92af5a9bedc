// DenseEC (Algorithm 3): for every x and every dense z, is there a common y?
// (Join-Count: how many?) Three interchangeable variants, the role f3 plays
// in Section 2.6:
//   POPC  -- Bitmap_x AND Bitmap_z over K = |Y_d| bits, 32 bits per AND+popc
//            (the paper's SIMD AND, on CUDA cores; no early stop, the tile
//            runs to the end of K).
//   PROBE -- for each y of R[x], look up S_dense's row of y (a bitmap over the
//            dense z index) and OR it in: the non-SIMD method of Algorithm 3
//            with the loops over z and y exchanged, so each probe answers 32
//            z at once.
//   TC    -- the 0/1 product on tcgen05 tensor cores (dense_tc.cu).
// All produce dense result bits [rows][zdw] (or counts [rows][n_zd]).
#include <algorithm>

#include "dense_tc.cuh"
#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

static unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

#define GRID_STRIDE(i, n)                                                        \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------ operands of S
template <typename K>
__global__ void k_dense_operands(const K* keys, int64_t n, int bz, const int32_t* zd_index, const int32_t* kidx,
                                 int variant, uint32_t* b_bits, int64_t kw, uint32_t* sdt, int64_t zdw,
                                 uint8_t* b_tc, int64_t k_pad) {
    const K zmask = (K)((K(1) << bz) - 1);
    GRID_STRIDE(i, n) {
        const K key = keys[i];
        const int32_t d = zd_index[(int64_t)(key & zmask)];
        if (d < 0) continue;
        const int32_t k = kidx[(int64_t)(key >> bz)];
        if (variant == DIM3_DENSE_POPC) atomicOr(&b_bits[(int64_t)d * kw + (k >> 5)], 1u << (k & 31));
        else if (variant == DIM3_DENSE_PROBE) atomicOr(&sdt[(int64_t)k * zdw + (d >> 5)], 1u << (d & 31));
        else b_tc[(int64_t)d * k_pad + k] = kE4m3One;
    }
}

void dense_build_operands(const Ctx& ctx, Plan& p, const uint64_t* keys64, const uint32_t* keys32, int64_t n,
                          int bz, const int32_t* zd_index, cudaStream_t s) {
    int variant = (int)p.opt.dense_variant;
    if (variant == DIM3_DENSE_AUTO) variant = DIM3_DENSE_TC;
    if (variant == DIM3_DENSE_TC && !tc_supported(ctx)) variant = DIM3_DENSE_POPC;
    DIM3_REQUIRE(variant >= DIM3_DENSE_TC && variant <= DIM3_DENSE_PROBE, DIM3_ERR_ARG, "unknown DenseEC variant");
    p.info.dense_variant = variant;
    const int64_t n_zd = p.info.n_z_dense, K = p.info.n_y_dense;
    p.zdw_op = ceil_div(n_zd, 32);
    p.zdw = p.zdw_op;  // widened by a partial result cache after the split
    p.kw = ceil_div(K, 32);
    p.k_pad = ceil_div(K, kTcBlockK) * kTcBlockK;
    p.n_zd_pad = ceil_div(n_zd, kTcPadN) * kTcPadN;
    if (variant == DIM3_DENSE_POPC) {
        p.b_bits.alloc((size_t)(n_zd * p.kw) * 4, s);
        DIM3_CUDA(cudaMemsetAsync(p.b_bits.p, 0, p.b_bits.bytes, s));
    } else if (variant == DIM3_DENSE_PROBE) {
        p.sdt_bits.alloc((size_t)(K * p.zdw_op) * 4, s);
        DIM3_CUDA(cudaMemsetAsync(p.sdt_bits.p, 0, p.sdt_bits.bytes, s));
    } else {
        const double bytes = (double)p.n_zd_pad * (double)p.k_pad;
        DIM3_REQUIRE(bytes < 64e9, DIM3_ERR_OVERFLOW, "dense operand too large");
        p.b_tc.alloc((size_t)(p.n_zd_pad * p.k_pad), s);
        DIM3_CUDA(cudaMemsetAsync(p.b_tc.p, 0, p.b_tc.bytes, s));
    }
    if (n == 0) return;
    if (keys64)
        k_dense_operands<uint64_t><<<grid_for(n), kThreads, 0, s>>>(
            keys64, n, bz, zd_index, p.kidx_of_y.as<int32_t>(), variant, p.b_bits.as<uint32_t>(), p.kw,
            p.sdt_bits.as<uint32_t>(), p.zdw_op, p.b_tc.as<uint8_t>(), p.k_pad);
    else
        k_dense_operands<uint32_t><<<grid_for(n), kThreads, 0, s>>>(
            keys32, n, bz, zd_index, p.kidx_of_y.as<int32_t>(), variant, p.b_bits.as<uint32_t>(), p.kw,
            p.sdt_bits.as<uint32_t>(), p.zdw_op, p.b_tc.as<uint8_t>(), p.k_pad);
    DIM3_LAUNCHED();
}

// ------------------------------------------------------------ operands of R
// Bitmap_x over K for rows [x_begin, x_begin + rows) (Algorithm 3, line 2).
__global__ void k_a_bits(const int64_t* r_rowptr, const int32_t* r_col, const int32_t* kidx, int64_t x_begin,
                         int64_t rows, uint32_t* a, int64_t kw) {
    GRID_STRIDE(xr, rows) {
        const int64_t x = x_begin + xr;
        for (int64_t q = r_rowptr[x]; q < r_rowptr[x + 1]; ++q) {
            const int32_t k = kidx[r_col[q]];
            if (k >= 0) a[xr * kw + (k >> 5)] |= 1u << (k & 31);
        }
    }
}

__global__ void k_a_tc(const int64_t* r_rowptr, const int32_t* r_col, const int32_t* kidx, int64_t x_begin,
                       int64_t rows, uint8_t* a, int64_t k_pad) {
    GRID_STRIDE(xr, rows) {
        const int64_t x = x_begin + xr;
        for (int64_t q = r_rowptr[x]; q < r_rowptr[x + 1]; ++q) {
            const int32_t k = kidx[r_col[q]];
            if (k >= 0) a[xr * k_pad + k] = kE4m3One;
        }
    }
}

// ------------------------------------------------------------------ POPC
// 64 x 64 output tile per CTA, K in chunks of 32 words staged in shared
// memory. Thread (warp ty, lane tx) owns rows ty*8..ty*8+7, columns tx, tx+32.
template <bool kCount>
__global__ void __launch_bounds__(kThreads) k_dense_popc(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                                         int64_t rows, int64_t n_zd, int64_t kw, uint32_t* D,
                                                         int64_t zdw, int32_t* C, const int2* __restrict__ tiles) {
    __shared__ uint32_t As[64][33];
    __shared__ uint32_t Bs[32][65];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // batches compute only the tiles of the block diagonal (tile list)
    const int64_t row0 = (int64_t)(tiles ? tiles[blockIdx.x].x : (int)blockIdx.y) * 64;
    const int64_t col0 = (int64_t)(tiles ? tiles[blockIdx.x].y : (int)blockIdx.x) * 64;
    int acc[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = 0;
    for (int64_t k0 = 0; k0 < kw; k0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += kThreads) {
            const int r = e >> 5, k = e & 31;
            const int64_t gr = row0 + r, gk = k0 + k;
            As[r][k] = (gr < rows && gk < kw) ? A[gr * kw + gk] : 0u;
            const int64_t gc = col0 + r;
            Bs[k][r] = (gc < n_zd && gk < kw) ? B[gc * kw + gk] : 0u;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const uint32_t b0 = Bs[k][tx], b1 = Bs[k][tx + 32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t av = As[ty * 8 + i][k];
                if (kCount) {
                    acc[i][0] += __popc(av & b0);
                    acc[i][1] += __popc(av & b1);
                } else {
                    acc[i][0] |= (int)(av & b0);
                    acc[i][1] |= (int)(av & b1);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = row0 + ty * 8 + i;
        if (kCount) {
            if (r < rows) {
                if (col0 + tx < n_zd) C[r * n_zd + col0 + tx] = acc[i][0];
                if (col0 + tx + 32 < n_zd) C[r * n_zd + col0 + tx + 32] = acc[i][1];
            }
        } else {
            const unsigned w0 = __ballot_sync(kFull, acc[i][0] != 0);
            const unsigned w1 = __ballot_sync(kFull, acc[i][1] != 0);
            if (tx == 0 && r < rows) {
                const int64_t cw = col0 >> 5;
                if (cw < zdw) D[r * zdw + cw] = w0;
                if (cw + 1 < zdw) D[r * zdw + cw + 1] = w1;
            }
        }
    }
}

// ----------------------------------------------------------------- PROBE
// One CTA per x; each thread owns words of the result row. sdw = words of an
// S_dense row (the dense z index), zdw = words of a result row (sdw, or more
// when a partial result cache adds its columns after the dense index).
template <bool kCount>
__global__ void __launch_bounds__(128) k_dense_probe(const int64_t* r_rowptr, const int32_t* r_col, const int32_t* kidx,
                                                     int64_t x_begin, int64_t rows, const uint32_t* __restrict__ sdt,
                                                     int64_t sdw, int64_t zdw, int64_t n_zd, uint32_t* D, int32_t* C,
                                                     const int32_t* x_tag, const int64_t* zd_lo) {
    const int64_t xr = blockIdx.x;
    if (xr >= rows) return;
    const int64_t x = x_begin + xr;
    const int64_t q0 = r_rowptr[x], q1 = r_rowptr[x + 1];
    // words of the dense indices of x's instance (batches; all words otherwise)
    const int tg = x_tag ? x_tag[x] : 0;
    const int64_t w0 = x_tag ? (zd_lo[tg] >> 5) : 0, w1 = x_tag ? ((zd_lo[tg + 1] + 31) >> 5) : sdw;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        if (!kCount) {
            uint32_t acc = 0u;
            for (int64_t q = q0; q < q1; ++q) {
                const int32_t k = kidx[r_col[q]];
                if (k >= 0) acc |= sdt[(int64_t)k * sdw + w];
            }
            D[xr * zdw + w] = acc;
        } else {
            int c[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) c[j] = 0;
            for (int64_t q = q0; q < q1; ++q) {
                const int32_t k = kidx[r_col[q]];
                if (k < 0) continue;
                const uint32_t bits = sdt[(int64_t)k * sdw + w];
#pragma unroll
                for (int j = 0; j < 32; ++j) c[j] += (bits >> j) & 1u;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int64_t d = w * 32 + j;
                if (d < n_zd) C[xr * n_zd + d] = c[j];
            }
        }
    }
}

// Tiles (row tile, column tile) of size tm x tn that meet the block of some
// instance: its x rows within [x_begin, x_begin + rows) times its dense z.
// Uploaded to `out`; returns their number.
static int64_t upload_block_tiles(const Plan& p, int64_t x_begin, int64_t rows, int tm, int tn, DevBuf& out,
                                  cudaStream_t s) {
    std::vector<int64_t> keys;
    for (int t = 0; t < p.n_inst; ++t) {
        const int64_t r0 = std::max(p.h_inst_x_lo[t], x_begin) - x_begin;
        const int64_t r1 = std::min(p.h_inst_x_lo[t + 1], x_begin + rows) - x_begin;
        const int64_t c0 = p.h_inst_zd_lo[t], c1 = p.h_inst_zd_lo[t + 1];
        if (r1 <= r0 || c1 <= c0) continue;
        for (int64_t m = r0 / tm; m <= (r1 - 1) / tm; ++m)
            for (int64_t n = c0 / tn; n <= (c1 - 1) / tn; ++n) keys.push_back((m << 32) | n);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    std::vector<int2> tiles(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) tiles[i] = make_int2((int)(keys[i] >> 32), (int)(keys[i] & 0xffffffff));
    if (tiles.empty()) return 0;
    out.alloc(tiles.size() * sizeof(int2), s);
    DIM3_CUDA(cudaMemcpyAsync(out.p, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    DIM3_CUDA(cudaStreamSynchronize(s));  // the host vector goes out of scope
    return (int64_t)tiles.size();
}

static void dense_product(const Ctx& ctx, const Plan& p, int64_t x_begin, int64_t rows, int kind, uint32_t* d_bits,
                          int32_t* d_cnt, cudaStream_t s);

void dense_ec(const Ctx& ctx, const Plan& p, int64_t x_begin, int64_t rows, int kind, uint32_t* d_bits, int32_t* d_cnt,
              cudaStream_t s) {
    const int64_t n_zd = p.info.n_z_dense;
    const bool cached = kind == 0 && p.n_zc > 0;
    if (rows <= 0 || (n_zd <= 0 && !cached)) return;
    const int variant = p.info.dense_variant;
    PhaseScope phase(ctx.stats, PH_DENSE, s);
    if (cached) {
        // the cache's columns are filled after the dense product; everything
        // the product does not write must be zero
        DIM3_CUDA(cudaMemsetAsync(d_bits, 0, (size_t)(rows * p.zdw) * 4, s));
        if (n_zd > 0) dense_product(ctx, p, x_begin, rows, kind, d_bits, d_cnt, s);
        cache_expand(p, x_begin, rows, d_bits, s);
        return;
    }
    dense_product(ctx, p, x_begin, rows, kind, d_bits, d_cnt, s);
}

static void dense_product(const Ctx& ctx, const Plan& p, int64_t x_begin, int64_t rows, int kind, uint32_t* d_bits,
                          int32_t* d_cnt, cudaStream_t s) {
    const int64_t n_zd = p.info.n_z_dense;
    const int variant = p.info.dense_variant;
    const bool batch = p.n_inst > 1;
    if (batch) {
        // only the block diagonal is computed: everything else is zero
        if (kind == 0) DIM3_CUDA(cudaMemsetAsync(d_bits, 0, (size_t)(rows * p.zdw) * 4, s));
        else DIM3_CUDA(cudaMemsetAsync(d_cnt, 0, (size_t)(rows * n_zd) * 4, s));
    }
    if (variant == DIM3_DENSE_PROBE) {
        DIM3_REQUIRE(rows < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "x range too long");
        const int32_t* xt = batch ? p.x_tag.as<int32_t>() : nullptr;
        if (kind == 0)
            k_dense_probe<false><<<(unsigned)rows, 128, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(),
                                                               p.kidx_of_y.as<int32_t>(), x_begin, rows,
                                                               p.sdt_bits.as<uint32_t>(), p.zdw_op, p.zdw, n_zd, d_bits,
                                                               nullptr,
                                                               xt, p.inst_zd_lo.as<int64_t>());
        else
            k_dense_probe<true><<<(unsigned)rows, 128, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(),
                                                              p.kidx_of_y.as<int32_t>(), x_begin, rows,
                                                              p.sdt_bits.as<uint32_t>(), p.zdw_op, p.zdw, n_zd, nullptr,
                                                              d_cnt,
                                                              xt, p.inst_zd_lo.as<int64_t>());
        DIM3_LAUNCHED();
    } else if (variant == DIM3_DENSE_POPC && batch) {
        DevBuf a;
        a.alloc((size_t)(rows * p.kw) * 4, s);
        DIM3_CUDA(cudaMemsetAsync(a.p, 0, a.bytes, s));
        k_a_bits<<<grid_for(rows), kThreads, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(),
                                                      p.kidx_of_y.as<int32_t>(), x_begin, rows, a.as<uint32_t>(), p.kw);
        DIM3_LAUNCHED();
        DevBuf tl;
        const int64_t nt = upload_block_tiles(p, x_begin, rows, 64, 64, tl, s);
        if (nt > 0) {
            if (kind == 0)
                k_dense_popc<false><<<(unsigned)nt, kThreads, 0, s>>>(a.as<uint32_t>(), p.b_bits.as<uint32_t>(), rows,
                                                                      n_zd, p.kw, d_bits, p.zdw, nullptr, tl.as<int2>());
            else
                k_dense_popc<true><<<(unsigned)nt, kThreads, 0, s>>>(a.as<uint32_t>(), p.b_bits.as<uint32_t>(), rows,
                                                                     n_zd, p.kw, nullptr, p.zdw, d_cnt, tl.as<int2>());
            DIM3_LAUNCHED();
        }
    } else if (variant == DIM3_DENSE_POPC) {
        DevBuf a;
        a.alloc((size_t)(rows * p.kw) * 4, s);
        DIM3_CUDA(cudaMemsetAsync(a.p, 0, a.bytes, s));
        k_a_bits<<<grid_for(rows), kThreads, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(),
                                                      p.kidx_of_y.as<int32_t>(), x_begin, rows, a.as<uint32_t>(), p.kw);
        DIM3_LAUNCHED();
        {
            const dim3 g((unsigned)ceil_div(n_zd, 64), (unsigned)ceil_div(rows, 64));
            DIM3_REQUIRE(ceil_div(rows, 64) < 65536, DIM3_ERR_OVERFLOW, "x range too long for one DenseEC launch");
            if (kind == 0)
                k_dense_popc<false><<<g, kThreads, 0, s>>>(a.as<uint32_t>(), p.b_bits.as<uint32_t>(), rows, n_zd, p.kw,
                                                           d_bits, p.zdw, nullptr, nullptr);
            else
                k_dense_popc<true><<<g, kThreads, 0, s>>>(a.as<uint32_t>(), p.b_bits.as<uint32_t>(), rows, n_zd, p.kw,
                                                          nullptr, p.zdw, d_cnt, nullptr);
            DIM3_LAUNCHED();
        }
    } else {
        const int64_t rows_pad = ceil_div(rows, kTcTileM) * kTcTileM;
        DevBuf a;
        a.alloc((size_t)(rows_pad * p.k_pad), s);
        DIM3_CUDA(cudaMemsetAsync(a.p, 0, a.bytes, s));
        k_a_tc<<<grid_for(rows), kThreads, 0, s>>>(p.r_rowptr.as<int64_t>(), p.r_col.as<int32_t>(),
                                                    p.kidx_of_y.as<int32_t>(), x_begin, rows, a.as<uint8_t>(), p.k_pad);
        DIM3_LAUNCHED();
        DevBuf tl;
        int64_t nt = 0;
        if (batch) {
            nt = upload_block_tiles(p, x_begin, rows, kTcTileM, tc_tile_n(ctx), tl, s);
            if (nt == 0) return;
        }
        tc_dense_product(ctx, a.as<uint8_t>(), rows, rows_pad, p.b_tc.as<uint8_t>(), n_zd, p.n_zd_pad, p.k_pad, kind,
                         d_bits, p.zdw, d_cnt, batch ? tl.as<int2>() : nullptr, nt, s);
    }
}

}  // namespace dimcube
