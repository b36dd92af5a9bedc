// DenseEC on tcgen05 tensor cores: shared constants and launcher.
#pragma once

#include "internal.cuh"

namespace dimcube {

// 0/1 operands are e4m3 values 0.0 (0x00) and 1.0 (0x38). Products are 0 or
// 1 and FP32 accumulation of at most K < 2^24 ones is exact, so C[x][z] is the
// exact number of common y (the Join-Count) and C > 0 is Algorithm 3's test.
constexpr uint8_t kE4m3One = 0x38;
constexpr int kTcTileM = 128;   // x rows per CTA (TMEM lanes)
constexpr int kTcPadN = 256;    // dense z padding of the operands (a multiple of every tile width)
constexpr int kTcBlockK = 128;  // K bytes per pipeline stage (one 128-byte swizzle span)
constexpr int64_t kTcMaxK = int64_t(1) << 24;

bool tc_supported(const Ctx& ctx);
// Dense z per CTA of the tensor-core product (TMEM FP32 columns): 256, or 128
// under DIM3_OPT_DENSE_TILE_N.
int tc_tile_n(const Ctx& ctx);

// C = A * B^T over K (both K-major e4m3 0/1), A [rows_pad][k_pad], B [n_pad][k_pad].
// kind 0: bits D[r][zdw] = (C > 0); kind 1: counts C[r][n_zd] (int32).
// tiles (device, n_tiles entries of (row tile, column tile)) restricts the
// product to those 128 x tc_tile_n tiles (batches: the block diagonal); null =
// all, in raster groups of row tiles.
void tc_dense_product(const Ctx& ctx, const uint8_t* A, int64_t rows, int64_t rows_pad, const uint8_t* B,
                      int64_t n_zd, int64_t n_pad, int64_t k_pad, int kind, uint32_t* d_bits, int64_t zdw,
                      int32_t* d_cnt, const int2* tiles, int64_t n_tiles, cudaStream_t s);

}  // namespace dimcube
