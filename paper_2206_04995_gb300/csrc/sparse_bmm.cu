// SparseBMM (Algorithm 2), the union with DenseEC's result (Algorithm 1, last
// step) and compaction into canonical order.
//
// GPU form. One CTA owns one x. Its SPA (Algorithm 2's z-vector) is a
// shared-memory bitmap over the z ids of a z tile: the paper's monotone
// "SPA[z] = x" tag avoids re-initialising a |Z|-long array per x; a bitmap of
// |Z|/8 bytes in shared memory is cheap to clear instead.
//   * Narrow S_sparse rows: a warp walks the row and sets bits (atomicOr).
//   * Wide S_sparse rows (held as z-bitmaps): the row is OR-ed in word by word,
//     |Z|/32 words instead of deg_S(y) bit updates.
//   * DenseEC's result bits (over the dense z index) are OR-ed in; the dense
//     and sparse z sets are disjoint (Section 2.3), so no dedup is needed.
// Because ids are ranks, scanning the bitmap in word order yields z ascending,
// and x ids processed in order yield the canonical (x, z) order. A counting
// pass gives per-x sizes, a scan gives offsets, an emitting pass rebuilds the
// bitmap and writes the pairs through a shared-memory staging buffer with
// 16-byte stores.
//
// Join-Count (Section 4.1): the SPA holds a 32-bit counter per z of the tile
// instead of a bit, every S_sparse row is walked as a list, and DenseEC's
// counts are added in.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

constexpr int kWarps = kThreads / 32;
// Passes of the row kernels over wide z ranges (k_tiled_rows, k_light_rows):
// count each row's pairs; emit them at the row offsets; or stage each row's
// z values at its slot of a buffer (and count them) for k_place_rows.
constexpr int kCountRows = 0, kEmitRows = 1, kStageRows = 2;
constexpr int kWarpStage = 1040;        // staged output values per warp (1024 + alignment shift, 16-byte multiple)
constexpr int kWarpStageIds = 528;      // staged z ids per warp in the one-row kernel (512 + shift)
constexpr int kWarpStageQ = 272;        // staged values per warp, quarter groups (256 + shift)
constexpr int64_t kMaxTileWords = 12 * 1024;   // 48 KiB bitmap tile = 393,216 z (three emitting CTAs per SM)
constexpr int kCntChunk = 4096;         // z per compaction chunk (count mode)
constexpr int64_t kMaxCntTile = 16 * 1024;     // counters per tile (64 KiB)
constexpr uint64_t kLookbackWaitNs = 2000000000ull;  // single pass: give up on a predecessor after 2 s

struct XRowArgs {
    int64_t x_begin, n_rows;
    int64_t n_z, zw, tile_bits;
    const int64_t* r_rowptr;
    const int32_t* r_col;
    const int64_t* ss_rowptr;
    const int32_t* ss_col;
    const int32_t* bm_row_of_y;
    const int64_t* bm_off;   // first word of each wide row's bitmap
    const uint32_t* ss_bits;
    const int32_t* x_tag;    // instance of each x (batches) or null
    const int64_t* z_lo;     // [n_inst + 1] z id range of each instance
    const int64_t* zd_lo;    // [n_inst + 1] dense index range of each instance
    const int64_t* tile_ptr; // tiled: [n_y][tile_cols] start of every z tile in each S_sparse row
    int64_t tile_cols;
    const uint32_t* d_bits;  // [n_rows][zdw] or null
    const int32_t* d_cnt;    // [n_rows][n_zd] or null
    int64_t zdw, n_zd;
    const int32_t* zd_list;
    const int32_t* dict_x;
    const int32_t* dict_z;
    int64_t* cnt;            // counting pass out
    // single pass (no counting pass): look-back status per logical block,
    // ticket counter, error flag and the output capacity
    unsigned long long* lb_status;
    unsigned long long* lb_ticket;
    int* lb_err;
    int64_t capacity;
    // one-row emitting kernel: staged entries per warp, kWarpStageIds (sparse
    // output, more CTAs per SM) or kWarpStage (dense output, whole groups)
    int stage_ints;
    int id_max;  // a 4096-z chunk with at most this many pairs goes through staged ids
    int flat_max;  // x rows (groups) with at most this many R entries take the one-phase build
    const uint8_t* light;  // per x id: handled by the light-row kernel (skip here), or null
    const int64_t* off;      // emitting pass: [n_rows + 1]
    int32_t* out_x;
    int32_t* out_z;
    int32_t* out_c;
    int vec_ok;
    // z-tiled single instance (k_tiled_rows): one CTA per listed row, n_tiles z tiles each
    const int64_t* slot;       // staging pass: each row's slot in the staging buffer (a.out_z)
    const int32_t* unit_rows;  // row numbers (x - x_begin) of the rows to run, or null (rows 0 .. n_list-1)
    int64_t n_list;            // rows in the list
    int n_tiles;               // z tiles per row
    // k_xrow_emit_g over a batch: groups of up to G rows of one instance,
    // (first row, rows) each; null = consecutive groups of G rows
    const int2* groups;
    int64_t n_groups;
};

// Fill out[o0, o1) with v using 16-byte stores where aligned.
__device__ __forceinline__ void fill_range(int32_t* out, int64_t o0, int64_t o1, int32_t v, bool vec_ok) {
    if (!vec_ok) {
        for (int64_t i = o0 + threadIdx.x; i < o1; i += blockDim.x) out[i] = v;
        return;
    }
    int64_t a = min64(o1, (o0 + 3) & ~int64_t(3));
    int64_t b = max64(a, o1 & ~int64_t(3));
    for (int64_t i = o0 + threadIdx.x; i < a; i += blockDim.x) out[i] = v;
    const int4 v4 = make_int4(v, v, v, v);
    for (int64_t i = a + 4 * (int64_t)threadIdx.x; i < b; i += 4 * (int64_t)blockDim.x)
        __stcs(reinterpret_cast<int4*>(out + i), v4);  // streaming: the output is not re-read
    for (int64_t i = b + threadIdx.x; i < o1; i += blockDim.x) out[i] = v;
}

// Copy stage[sh, sh + cnt) to dst[sh, sh + cnt) where dst + 0 is 16-byte
// aligned when vec_ok (the caller offsets dst by the global misalignment).
__device__ __forceinline__ void flush_stage(int32_t* dst, const int32_t* stage, int sh, int cnt, bool vec_ok) {
    const int end = sh + cnt;
    const int nv = (end + 3) >> 2;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const int s = v << 2;
        if (vec_ok && s >= sh && s + 4 <= end) {
            *reinterpret_cast<int4*>(dst + s) = *reinterpret_cast<const int4*>(stage + s);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = s + j;
                if (t >= sh && t < end) dst[t] = stage[t];
            }
        }
    }
}

// Warp-level version of flush_stage.
__device__ __forceinline__ void flush_warp(int32_t* dst, const int32_t* st, int sh, int cnt, bool vec_ok) {
    const int end = sh + cnt;
    const int nv = (end + 3) >> 2;
    const int lane = threadIdx.x & 31;
    for (int v = lane; v < nv; v += 32) {
        const int s = v << 2;
        if (vec_ok && s >= sh && s + 4 <= end) {
            __stcs(reinterpret_cast<int4*>(dst + s), *reinterpret_cast<const int4*>(st + s));
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = s + j;
                if (t >= sh && t < end) __stcs(dst + t, st[t]);
            }
        }
    }
}

// Write the z values of the set bits of one 32-word group (1024 z ids, lane j
// holding word j, excl = set bits in words < j) to st[sh + ...] in z order.
// Dense groups: lane l reads dictionary entry 32 j + l while word j is
// broadcast, so every load is one 128-byte line; only nonzero words are
// visited. Sparse groups: every lane writes its own word's few bits.
__device__ __forceinline__ void compact_group(int32_t* st, int sh, uint32_t word, int excl, int total_g,
                                              const int32_t* dz, int lane, unsigned lt) {
    constexpr int kSparseGroup = 64;
    if (total_g <= kSparseGroup) {
        int pos = sh + excl;
        uint32_t wv = word;
        while (wv) {
            const int b = __ffs(wv) - 1;
            wv &= wv - 1;
            st[pos++] = __ldg(dz + (lane << 5) + b);
        }
        return;
    }
    unsigned m = __ballot_sync(kFull, word != 0u);
    if (__popc(m) >= 24) {  // nearly every word set: a fixed, unrolled sweep
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const uint32_t wj = __shfl_sync(kFull, word, j);
            const int pj = __shfl_sync(kFull, excl, j);
            if ((wj >> lane) & 1u) st[sh + pj + __popc(wj & lt)] = __ldg(dz + (j << 5) + lane);
        }
        return;
    }
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t wj = __shfl_sync(kFull, word, j);
        const int pj = __shfl_sync(kFull, excl, j);
        if ((wj >> lane) & 1u) st[sh + pj + __popc(wj & lt)] = __ldg(dz + (j << 5) + lane);
    }
}

// Zero bm[0, n) with 16-byte stores (bm is 16-byte aligned).
__device__ __forceinline__ void clear_words(uint32_t* bm, int n) {
    const int n4 = n >> 2;
    uint4* b4 = reinterpret_cast<uint4*>(bm);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) b4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = (n4 << 2) + threadIdx.x; i < n; i += blockDim.x) bm[i] = 0u;
}

// This thread's share of the set bits of bm[0, n), read 16 bytes at a time.
__device__ __forceinline__ int64_t popc_words(const uint32_t* bm, int n) {
    const int n4 = n >> 2;
    const uint4* b4 = reinterpret_cast<const uint4*>(bm);
    int64_t c = 0;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const uint4 v = b4[i];
        c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    }
    for (int i = (n4 << 2) + threadIdx.x; i < n; i += blockDim.x) c += __popc(bm[i]);
    return c;
}

// flush_warp for a stage of z ids: dst[t] = dict_z[st[t]] for t in [sh, sh + cnt).
// Two 16-byte pieces per lane and round: their eight gathers are issued
// before either store, so a round costs one dictionary latency.
__device__ __forceinline__ void flush_warp_ids(int32_t* dst, const int32_t* st, int sh, int cnt,
                                               const int32_t* __restrict__ dict_z, bool vec_ok) {
    const int end = sh + cnt;
    const int nv = (end + 3) >> 2;
    const int lane = threadIdx.x & 31;
    if (vec_ok) {
        // whole pieces [v0, v1): v0 = first piece at or after sh, v1 = last full piece
        const int v0 = (sh + 3) >> 2, v1 = end >> 2;
        for (int v = v0 + lane; v < v1; v += 64) {
            const bool two = v + 32 < v1;
            const int4 ia = *reinterpret_cast<const int4*>(st + 4 * v);
            const int4 ib = two ? *reinterpret_cast<const int4*>(st + 4 * (v + 32)) : ia;
            const int4 a = make_int4(__ldg(dict_z + ia.x), __ldg(dict_z + ia.y), __ldg(dict_z + ia.z),
                                     __ldg(dict_z + ia.w));
            const int4 b = make_int4(__ldg(dict_z + ib.x), __ldg(dict_z + ib.y), __ldg(dict_z + ib.z),
                                     __ldg(dict_z + ib.w));
            __stcs(reinterpret_cast<int4*>(dst + 4 * v), a);
            if (two) __stcs(reinterpret_cast<int4*>(dst + 4 * (v + 32)), b);
        }
        // the partial pieces at both ends (at most three entries each)
        if (lane < 8) {
            const int t = lane < 4 ? sh + lane : 4 * v1 + (lane - 4);
            const bool head = lane < 4 && t < min(end, 4 * v0);
            const bool tail = lane >= 4 && t < end && v1 >= v0;
            if (head || tail) __stcs(dst + t, __ldg(dict_z + st[t]));
        }
        return;
    }
    for (int v = lane; v < nv; v += 32) {
        const int s = v << 2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = s + j;
            if (t >= sh && t < end) __stcs(dst + t, __ldg(dict_z + st[t]));
        }
    }
}

// Compaction of one warp's run of 32-word groups [g0, g1) of a z-tile bitmap
// (holding `mine` set bits) into out_z from position wpos, z ascending: the
// per-warp stage st collects z values (dense groups) or z ids (sparse 4096-z
// chunks) and is flushed with 16-byte stores. Called by a whole warp.
__device__ __forceinline__ void compact_run(const XRowArgs& a, const uint32_t* bm, int tw, int g0, int g1, int mine,
                                            int64_t zt0, int64_t wpos, int32_t* st) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    // Set bits are staged as z ids, group after group, and turned
    // into z values only when the stage is flushed: a sparse row
    // then costs one round of independent dictionary gathers per
    // ~1000 pairs instead of one dependent round per group.
    int sh = (int)(wpos & 3), sc = 0;  // stage holds pairs [wpos, wpos + sc) at st[sh ..]
    // Chunks of 4 groups (128 words, 4096 z): lane l first reads words
    // 4l .. 4l+3; a sparse chunk is extracted lane by lane in one step,
    // a dense one group by group with the transposed dictionary reads.
    // A dense run (an eighth of its bits set or more, large stage):
    // every group straight through compact_group, no chunk scan.
    const bool dense_run = a.stage_ints >= kWarpStage && (int64_t)mine * 8 >= (int64_t)(g1 - g0) * 1024;
    for (int g = g0; dense_run && g < g1; ++g) {
        const int w = (g << 5) + lane;
        const uint32_t word = w < tw ? bm[w] : 0u;
        const int c = __popc(word);
        const int incl = warp_inclusive_scan(c);
        const int total_g = __shfl_sync(kFull, incl, 31);
        if (total_g == 0) continue;
        sh = (int)(wpos & 3);
        compact_group(st, sh, word, incl - c, total_g, a.dict_z + zt0 + ((int64_t)g << 10), lane, lt);
        __syncwarp();
        flush_warp(a.out_z + (wpos - sh), st, sh, total_g, a.vec_ok);
        __syncwarp();
        wpos += total_g;
    }
    for (int gc = g0; !dense_run && gc < g1; gc += 4) {
        const int wl = (gc << 5) + (lane << 2);
        const int wlim = min(tw, g1 << 5);
        uint32_t wv[4];
        if (wl + 4 <= wlim) {
            // one 16-byte load per lane (wl is a multiple of 4 and bm 16-byte
            // aligned): no bank conflicts, unlike four stride-4 word loads
            const uint4 q = *reinterpret_cast<const uint4*>(bm + wl);
            wv[0] = q.x;
            wv[1] = q.y;
            wv[2] = q.z;
            wv[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) wv[k] = wl + k < wlim ? bm[wl + k] : 0u;
        }
        int c4 = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) c4 += __popc(wv[k]);
        const int incl4 = warp_inclusive_scan(c4);
        const int total_c = __shfl_sync(kFull, incl4, 31);
        if (total_c == 0) continue;
        if (total_c <= a.id_max) {
            if (sh + sc + total_c > a.stage_ints) {
                __syncwarp();
                flush_warp_ids(a.out_z + (wpos - sh), st, sh, sc, a.dict_z, a.vec_ok);
                __syncwarp();
                wpos += sc;
                sh = (int)(wpos & 3);
                sc = 0;
            }
            // one step per set bit of the lane's four words (the warp takes
            // as many steps as its fullest lane)
            int pos = sh + sc + incl4 - c4;
            int k = 0;
            uint32_t v = wv[0];
            for (int i = 0; i < c4; ++i) {
                while (v == 0u) {
                    ++k;
                    v = k == 1 ? wv[1] : k == 2 ? wv[2] : wv[3];
                }
                st[pos++] = (int32_t)(zt0 + ((int64_t)(wl + k) << 5) + __ffs(v) - 1);
                v &= v - 1;
            }
            sc += total_c;
            continue;
        }
        // dense chunk: write z values directly (coalesced dictionary
        // reads, lane l reading entry 32 j + l), one half-group (16
        // words, at most 512 pairs) per flush; pending ids go first
        if (sc) {
            __syncwarp();
            flush_warp_ids(a.out_z + (wpos - sh), st, sh, sc, a.dict_z, a.vec_ok);
            __syncwarp();
            wpos += sc;
            sc = 0;
        }
        // whole groups fit a large stage, half groups (512 pairs) the
        // 528-entry one, quarter groups (256 pairs) the 272-entry one
        const int per = a.stage_ints >= kWarpStage ? 1 : a.stage_ints >= kWarpStageIds ? 2 : 4;
        for (int h = gc * per; h < min(gc + 4, g1) * per; ++h) {
            const int g = h / per;
            const int w = (g << 5) + lane;
            const bool mine_part = per == 1 || lane / (32 / per) == h % per;
            const uint32_t word = (mine_part && w < tw) ? bm[w] : 0u;
            const int c = __popc(word);
            const int incl = warp_inclusive_scan(c);
            const int total_g = __shfl_sync(kFull, incl, 31);
            if (total_g == 0) continue;
            sh = (int)(wpos & 3);
            compact_group(st, sh, word, incl - c, total_g, a.dict_z + zt0 + ((int64_t)g << 10), lane, lt);
            __syncwarp();
            flush_warp(a.out_z + (wpos - sh), st, sh, total_g, a.vec_ok);
            __syncwarp();
            wpos += total_g;
        }
        sh = (int)(wpos & 3);
    }
    __syncwarp();
    if (sc) flush_warp_ids(a.out_z + (wpos - sh), st, sh, sc, a.dict_z, a.vec_ok);
    __syncwarp();
}

// Register caps: 32 for the counting instance (eight CTAs per SM), 64 for the
// emitting one (four, no spills); both are latency-bound. Measured on the
// 256-instance batch: the emitting instance at 64 registers 18.4 ms, at 48
// (spilling) 19.3 ms.
template <bool kEmit>
__global__ void __launch_bounds__(kThreads, kEmit ? 4 : 8) k_xrow_bits(const XRowArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t* stage = reinterpret_cast<int32_t*>(smem);           // emit: kWarps x a.stage_ints
    uint32_t* bm = smem + (kEmit ? kWarps * a.stage_ints : 0);  // tile words
    __shared__ int64_t s_scan[kThreads / 32 + 1];
    __shared__ int32_t s_list[kThreads];
    __shared__ int32_t s_ny[kThreads];
    __shared__ int64_t s_woff[kThreads];
    __shared__ int32_t s_wc[kThreads / 32 + 1];
    __shared__ int32_t s_cw[kWarps], s_cn[kWarps];
    __shared__ int64_t s_blk, s_prefix;

    // single pass (emitting kernel, one z tile): row number from a ticket
    int64_t xr = blockIdx.x;
    if (kEmit && a.lb_status) {
        if (threadIdx.x == 0) s_blk = (int64_t)atomicAdd(a.lb_ticket, 1ull);
        __syncthreads();
        xr = s_blk;
    }
    if (xr >= a.n_rows) return;
    const int64_t x = a.x_begin + xr;
    if (a.light && a.light[x]) return;  // the light-row kernel counts and writes it
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // z window of x's instance (all of Z for a single instance), from a
    // 32-aligned start so that bitmap words line up with the wide rows' words
    const int tg = a.x_tag ? a.x_tag[x] : 0;
    const int64_t zb = a.z_lo[tg] & ~int64_t(31), ze = a.z_lo[tg + 1];
    const bool tiled = a.tile_bits < ze - zb;
    int64_t total = 0;
    int64_t out_pos = 0;
    bool write = true;
    if (kEmit && !a.lb_status) {
        out_pos = a.off[xr];
        fill_range(a.out_x, out_pos, a.off[xr + 1], a.dict_x[x], a.vec_ok);
    }
    // At most kThreads R entries: sorted once into per-warp lists of narrow
    // rows (y) and wide rows (bitmap), then each tile is built in one
    // barrier-free phase (warps walk narrow rows while every thread ORs the
    // wide rows into its words, both with shared atomics).
    const bool flat = r1 - r0 <= a.flat_max;  // block-uniform
    if (flat) {
        const int64_t p = r0 + tid;
        int32_t y = -1, b = -1;
        if (p < r1) {
            y = a.r_col[p];
            b = a.bm_row_of_y[y];
        }
        const bool isw = b >= 0, isn = p < r1 && b < 0;
        const unsigned bw = __ballot_sync(kFull, isw), bn = __ballot_sync(kFull, isn);
        if (isw) s_woff[(warp << 5) + __popc(bw & lanemask_lt())] = a.bm_off[b];
        if (isn) s_ny[(warp << 5) + __popc(bn & lanemask_lt())] = y;
        if (lane == 0) {
            s_cw[warp] = __popc(bw);
            s_cn[warp] = __popc(bn);
        }
    }
    for (int64_t zt0 = zb; zt0 < ze; zt0 += a.tile_bits) {
        const int64_t zt1 = min64(zt0 + a.tile_bits, ze);
        const int tw = (int)((zt1 - zt0 + 31) >> 5);
        clear_words(bm, tw);
        __syncthreads();
        if (flat) {
            int n_nar = 0;
            unsigned wmask = 0u;  // warps whose list holds wide rows
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                n_nar += s_cn[w];
                wmask |= s_cw[w] > 0 ? 1u << w : 0u;
            }
            for (int e = warp; e < n_nar; e += kWarps) {
                int sg = 0, base = 0;
                while (e - base >= s_cn[sg]) base += s_cn[sg++];
                const int32_t y = s_ny[(sg << 5) + (e - base)];
                int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
                if (tiled) {
                    const int64_t* tp = a.tile_ptr + (int64_t)y * a.tile_cols + (zt0 - zb) / a.tile_bits;
                    s0 = tp[0];
                    s1 = tp[1];
                }
                for (int64_t q = s0 + lane; q < s1; q += 32) {
                    const int32_t z = a.ss_col[q] - (int32_t)zt0;
                    atomicOr(&bm[z >> 5], 1u << (z & 31));
                }
            }
            if (wmask) {
                const uint32_t* bits = a.ss_bits + ((zt0 - zb) >> 5);
                for (int w = tid; w < tw; w += kThreads) {
                    uint32_t acc = 0u;
                    for (unsigned m = wmask; m; m &= m - 1) {
                        const int sg = __ffs(m) - 1, c = s_cw[sg];
                        for (int i = sg << 5; i < (sg << 5) + c; ++i) acc |= __ldg(bits + s_woff[i] + w);
                    }
                    if (acc) atomicOr(&bm[w], acc);
                }
            }
        } else {
            // narrow S_sparse rows: one warp per y of R[x]
            for (int64_t p = r0 + warp; p < r1; p += kThreads / 32) {
                const int32_t y = a.r_col[p];
                if (a.bm_row_of_y[y] >= 0) continue;
                int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
                if (tiled) {
                    const int64_t* tp = a.tile_ptr + (int64_t)y * a.tile_cols + (zt0 - zb) / a.tile_bits;
                    s0 = tp[0];
                    s1 = tp[1];
                }
                for (int64_t q = s0 + lane; q < s1; q += 32) {
                    const int32_t z = a.ss_col[q] - (int32_t)zt0;
                    atomicOr(&bm[z >> 5], 1u << (z & 31));
                }
            }
            // wide S_sparse rows: gather up to kThreads bitmap rows, OR them word-wise
            for (int64_t base = r0; base < r1; base += kThreads) {
                const int64_t p = base + tid;
                const int32_t b = p < r1 ? a.bm_row_of_y[a.r_col[p]] : -1;
                const unsigned bal = __ballot_sync(kFull, b >= 0);
                if (lane == 0) s_wc[warp] = __popc(bal);
                __syncthreads();
                if (tid == 0) {
                    int run = 0;
                    for (int w = 0; w < kThreads / 32; ++w) {
                        const int c = s_wc[w];
                        s_wc[w] = run;
                        run += c;
                    }
                    s_wc[kThreads / 32] = run;
                }
                __syncthreads();
                if (b >= 0) s_list[s_wc[warp] + __popc(bal & lanemask_lt())] = b;
                __syncthreads();
                const int nl = s_wc[kThreads / 32];
                if (nl > 0) {
                    const uint32_t* bits = a.ss_bits + ((zt0 - zb) >> 5);
                    for (int w = tid; w < tw; w += kThreads) {
                        uint32_t acc = 0u;
                        for (int i = 0; i < nl; ++i) acc |= __ldg(bits + a.bm_off[s_list[i]] + w);
                        if (acc) bm[w] |= acc;
                    }
                }
                __syncthreads();
            }
        }
        // DenseEC result of this x (disjoint from the sparse z set), over the
        // dense indices of x's instance: one thread per index, so the result
        // word is a broadcast read and the z ids of set bits coalesced reads
        if (a.n_zd > 0) {
            const uint32_t* drow = a.d_bits + xr * a.zdw;
            const int64_t d1 = a.zd_lo[tg + 1];
            for (int64_t d = a.zd_lo[tg] + tid; d < d1; d += kThreads) {
                if ((drow[d >> 5] >> (d & 31)) & 1u) {
                    int32_t z = a.zd_list[d];
                    if (z >= zt0 && z < zt1) {
                        z -= (int32_t)zt0;
                        atomicOr(&bm[z >> 5], 1u << (z & 31));
                    }
                }
            }
        }
        __syncthreads();
        if (!kEmit) {
            int64_t c = 0;
            c = popc_words(bm, tw);
            total += block_sum<int64_t, kThreads>(c, s_scan);
        } else {
            // Each warp owns a run of 32-word groups (1024 z ids each). The
            // warps' output offsets come from one popcount pass; after that
            // every warp compacts and writes its run without block barriers.
            const int groups = (tw + 31) >> 5;
            const int gpw = (groups + kWarps - 1) / kWarps;  // chunk reads below are masked at g1
            const int g0 = warp * gpw, g1 = min(groups, g0 + gpw);
            int mine = 0;
            for (int g = g0; g < g1; ++g) {
                const int w = (g << 5) + lane;
                mine += w < tw ? __popc(bm[w]) : 0;
            }
            mine = warp_sum(mine);
            if (lane == 0) s_wc[warp] = mine;
            __syncthreads();
            if (a.lb_status) {
                int64_t agg = 0;
                for (int w = 0; w < kWarps; ++w) agg += s_wc[w];
                if (warp == 0) {
                    const int64_t pre = lookback_prefix(a.lb_status, xr, agg, a.lb_err, kLookbackWaitNs);
                    if (lane == 0) s_prefix = pre;
                }
                __syncthreads();
                const int64_t pre = s_prefix;
                write = pre >= 0 && pre + agg <= a.capacity;
                out_pos = pre;
                if (write) fill_range(a.out_x, pre, pre + agg, a.dict_x[x], a.vec_ok);
            }
            int64_t wpos = out_pos, tile_total = 0;
            for (int w = 0; w < kWarps; ++w) {
                const int c = s_wc[w];
                if (w < warp) wpos += c;
                tile_total += c;
            }
            if (write) compact_run(a, bm, tw, g0, g1, mine, zt0, wpos, stage + warp * a.stage_ints);
            out_pos += tile_total;
        }
        __syncthreads();
    }
    if (!kEmit && tid == 0) a.cnt[xr] = total;
}

// Emitting pass for G consecutive x rows per CTA. The rows' SPA bitmaps are
// built together (their R_CSR rows are adjacent, so one flattened entry list
// feeds the warps), and each 1024-entry slice of the z dictionary is loaded
// into registers half a slice at a time (lane l holds entries 32 j + l of 16
// words j) and used for all G rows, which divides the dictionary's L2 traffic
// and the block barriers per row by G; a half (at most 512 pairs) is staged
// and flushed, so the per-warp stage is 528 entries. The steps are device
// functions shared by the plain kernel and the pipelined persistent one.

// Build scratch of a row group.
struct GroupSmem {
    int32_t list[kThreads];
    int32_t lk[kThreads];
    int32_t ny[kThreads];
    int32_t nk[kThreads];
    int64_t woff[kThreads];
    int32_t wc[kWarps + 1];
    int32_t cw[kWarps], cn[kWarps];
};

// Row group number blk: its first row (relative to x_begin) and row count;
// false past the last group.
template <int G>
__device__ __forceinline__ bool g_locate(const XRowArgs& a, int64_t blk, int64_t& xr0, int& ng) {
    if (a.groups) {
        if (blk >= a.n_groups) return false;
        const int2 g = a.groups[blk];
        xr0 = g.x;
        ng = g.y;
        return true;
    }
    xr0 = blk * G;
    if (xr0 >= a.n_rows) return false;
    ng = (int)min64(G, a.n_rows - xr0);
    return true;
}

// Which of the group's rows holds R_CSR entry p (rb = the rows' starts).
template <int G>
__device__ __forceinline__ int g_row_of(int64_t p, const int64_t (&rb)[G + 1], int ng) {
    int k = 0;
#pragma unroll
    for (int q = 1; q < G; ++q) k += (q < ng && p >= rb[q]) ? 1 : 0;
    return k;
}

// At most flat_max R entries (the usual case): one thread per entry sorts
// them once into per-warp lists of narrow rows (y, row) and wide rows
// (bitmap, row); every tile then builds its bitmaps in ONE barrier-free phase,
// warps walking narrow rows while every thread ORs wide rows into its words
// (both with shared atomics). Returns whether the group is flat (block-
// uniform); the lists are ready after the next block barrier.
template <int G>
__device__ __forceinline__ bool g_prepare(const XRowArgs& a, const int64_t (&rb)[G + 1], int ng, GroupSmem& gs) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t n_ent = rb[G] - rb[0];
    const bool flat = n_ent <= a.flat_max;
    if (flat) {
        const int64_t p = rb[0] + tid;
        int32_t y = -1, b = -1;
        if (tid < n_ent) {
            y = a.r_col[p];
            b = a.bm_row_of_y[y];
        }
        const bool isw = b >= 0, isn = tid < n_ent && b < 0;
        const unsigned bw = __ballot_sync(kFull, isw), bn = __ballot_sync(kFull, isn);
        const int k = tid < n_ent ? g_row_of<G>(p, rb, ng) : 0;
        if (isw) {
            const int slot = (warp << 5) + __popc(bw & lt);
            gs.woff[slot] = a.bm_off[b];
            gs.lk[slot] = k;
        }
        if (isn) {
            const int slot = (warp << 5) + __popc(bn & lt);
            gs.ny[slot] = y;
            gs.nk[slot] = k;
        }
        if (lane == 0) {
            gs.cw[warp] = __popc(bw);
            gs.cn[warp] = __popc(bn);
        }
    }
    return flat;
}

// The group's bitmaps over z tile [zt0, zt1) (window start zb of instance tg):
// clear, narrow S rows, wide S rows, DenseEC bits. Ends with a block barrier.
template <int G>
__device__ __forceinline__ void g_build(const XRowArgs& a, const int64_t (&rb)[G + 1], int ng, bool flat, int tg,
                                        int64_t xr0, int64_t zb, int64_t zt0, int64_t zt1, bool tiled,
                                        uint32_t* bm_all, int64_t tile_words, GroupSmem& gs) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t r_end = rb[G];
    const int tw = (int)((zt1 - zt0 + 31) >> 5);
    clear_words(bm_all, (int)(ng * tile_words));
    __syncthreads();
    if (flat) {
        int n_nar = 0;
        unsigned wmask = 0u;  // warps whose list holds wide rows
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            n_nar += gs.cn[w];
            wmask |= gs.cw[w] > 0 ? 1u << w : 0u;
        }
        for (int e = warp; e < n_nar; e += kWarps) {
            int sg = 0, base = 0;
            while (e - base >= gs.cn[sg]) base += gs.cn[sg++];
            const int slot = (sg << 5) + (e - base);
            const int32_t y = gs.ny[slot];
            uint32_t* bm = bm_all + gs.nk[slot] * tile_words;
            int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            if (tiled) {
                s0 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt0);
                s1 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt1);
            }
            for (int64_t q = s0 + lane; q < s1; q += 32) {
                const int32_t z = a.ss_col[q] - (int32_t)zt0;
                atomicOr(&bm[z >> 5], 1u << (z & 31));
            }
        }
        if (wmask) {
            const uint32_t* bits = a.ss_bits + ((zt0 - zb) >> 5);
            for (int w = tid; w < tw; w += kThreads) {
                uint32_t acc[G];
#pragma unroll
                for (int k = 0; k < G; ++k) acc[k] = 0u;
                for (unsigned m = wmask; m; m &= m - 1) {
                    const int sg = __ffs(m) - 1, c = gs.cw[sg];
                    for (int i = sg << 5; i < (sg << 5) + c; ++i) {
                        const uint32_t v = __ldg(bits + gs.woff[i] + w);
                        const int k = gs.lk[i];
#pragma unroll
                        for (int q = 0; q < G; ++q) acc[q] |= (k == q) ? v : 0u;
                    }
                }
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (k < ng && acc[k]) atomicOr(&bm_all[k * tile_words + w], acc[k]);
            }
        }
    } else {
        // narrow S_sparse rows of all G rows: one warp per R entry
        for (int64_t p = rb[0] + warp; p < r_end; p += kWarps) {
            const int32_t y = a.r_col[p];
            if (a.bm_row_of_y[y] >= 0) continue;
            uint32_t* bm = bm_all + g_row_of<G>(p, rb, ng) * tile_words;
            int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            if (tiled) {
                s0 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt0);
                s1 = lower_bound_dev<int32_t>(a.ss_col, s0, s1, (int32_t)zt1);
            }
            for (int64_t q = s0 + lane; q < s1; q += 32) {
                const int32_t z = a.ss_col[q] - (int32_t)zt0;
                atomicOr(&bm[z >> 5], 1u << (z & 31));
            }
        }
        // wide S_sparse rows
        for (int64_t base = rb[0]; base < r_end; base += kThreads) {
            const int64_t p = base + tid;
            const int32_t b = p < r_end ? a.bm_row_of_y[a.r_col[p]] : -1;
            const unsigned bal = __ballot_sync(kFull, b >= 0);
            if (lane == 0) gs.wc[warp] = __popc(bal);
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int w = 0; w < kWarps; ++w) {
                    const int c = gs.wc[w];
                    gs.wc[w] = run;
                    run += c;
                }
                gs.wc[kWarps] = run;
            }
            __syncthreads();
            if (b >= 0) {
                const int slot = gs.wc[warp] + __popc(bal & lt);
                gs.list[slot] = b;
                gs.lk[slot] = g_row_of<G>(p, rb, ng);
            }
            __syncthreads();
            const int nl = gs.wc[kWarps];
            if (nl > 0) {
                const uint32_t* bits = a.ss_bits + ((zt0 - zb) >> 5);
                for (int w = tid; w < tw; w += kThreads) {
                    uint32_t acc[G];
#pragma unroll
                    for (int k = 0; k < G; ++k) acc[k] = 0u;
                    for (int i = 0; i < nl; ++i) {
                        const uint32_t v = __ldg(bits + a.bm_off[gs.list[i]] + w);
                        const int k = gs.lk[i];
#pragma unroll
                        for (int q = 0; q < G; ++q) acc[q] |= (k == q) ? v : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < G; ++k)
                        if (k < ng && acc[k]) bm_all[k * tile_words + w] |= acc[k];
                }
            }
            __syncthreads();
        }
    }
    if (a.n_zd > 0) {
        // DenseEC results, one thread per dense index of the instance (see k_xrow_bits)
        const int64_t d0 = a.x_tag ? a.zd_lo[tg] : 0, d1 = a.x_tag ? a.zd_lo[tg + 1] : a.n_zd;
        for (int k = 0; k < ng; ++k) {
            const uint32_t* drow = a.d_bits + (xr0 + k) * a.zdw;
            uint32_t* bm = bm_all + k * tile_words;
            for (int64_t d = d0 + tid; d < d1; d += kThreads) {
                if ((drow[d >> 5] >> (d & 31)) & 1u) {
                    int32_t z = a.zd_list[d];
                    if (z >= zt0 && z < zt1) {
                        z -= (int32_t)zt0;
                        atomicOr(&bm[z >> 5], 1u << (z & 31));
                    }
                }
            }
        }
    }
    __syncthreads();
}

// Per-warp segment sizes of every row of the group (warp w owns groups of 32
// words [g0, g1) of the tile). Ends with a block barrier.
template <int G>
__device__ __forceinline__ void g_counts(const uint32_t* bm_all, int64_t tile_words, int tw, int ng,
                                         int32_t (&seg)[G][kWarps]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int groups = (tw + 31) >> 5;
    const int gpw = (groups + kWarps - 1) / kWarps;
    const int g0 = warp * gpw, g1 = min(groups, g0 + gpw);
#pragma unroll
    for (int k = 0; k < G; ++k) {
        int mine = 0;
        if (k < ng) {
            const uint32_t* bm = bm_all + k * tile_words;
            for (int g = g0; g < g1; ++g) {
                const int w = (g << 5) + lane;
                mine += w < tw ? __popc(bm[w]) : 0;
            }
        }
        mine = warp_sum(mine);
        if (lane == 0) seg[k][warp] = mine;
    }
    __syncthreads();
}

// Compaction of the group's tile: every warp writes the z values of its run
// of 32-word groups for each row, row k's run starting at row_pos[k] plus the
// earlier warps' segments of that row. A dense 32-word group is staged and
// flushed in P parts of 32 / P words (at most 1024 / P pairs each), so the
// per-warp stage holds 1024 / P + 16 entries (stage_ints). No block barrier.
template <int G, int P>
__device__ __forceinline__ void g_emit(const XRowArgs& a, const uint32_t* bm_all, int64_t tile_words, int tw, int ng,
                                       int64_t zt0, const int32_t (&seg)[G][kWarps], const int64_t (&row_pos)[G],
                                       int32_t* stage, int stage_ints) {
    constexpr int W = 32 / P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int groups = (tw + 31) >> 5;
    const int gpw = (groups + kWarps - 1) / kWarps;
    const int g0 = warp * gpw, g1 = min(groups, g0 + gpw);
    int64_t wpos[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        int64_t before = 0;
        for (int w = 0; w < warp; ++w) before += seg[k][w];
        wpos[k] = (k < ng ? row_pos[k] : 0) + before;
    }
    int32_t* st = stage + warp * stage_ints;
    const int64_t zlim = a.n_z - zt0;
    for (int g = g0; g < g1; ++g) {
        const int w = (g << 5) + lane;
        uint32_t word[G];
        bool any = false;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            word[k] = (k < ng && w < tw) ? bm_all[k * tile_words + w] : 0u;
            any |= word[k] != 0u;
        }
        if (!__any_sync(kFull, any)) continue;
        const int64_t gb = (int64_t)g << 10;
        const int32_t* dz = a.dict_z + zt0 + gb;
        int excl[G], total[G], mid[G];  // mid: the count before word 16 (two parts)
        bool dense = false;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int c = __popc(word[k]);
            const int incl = warp_inclusive_scan(c);
            total[k] = __shfl_sync(kFull, incl, 31);
            mid[k] = P == 2 ? __shfl_sync(kFull, incl, 15) : 0;
            excl[k] = incl - c;
            if (total[k] > 64) {
                dense = true;
            } else if (total[k] > 0) {
                // few bits: each lane writes its own word's bits
                const int sh = (int)(wpos[k] & 3);
                int pos = sh + excl[k];
                uint32_t wv = word[k];
                while (wv) {
                    const int b = __ffs(wv) - 1;
                    wv &= wv - 1;
                    st[pos++] = __ldg(dz + (lane << 5) + b);
                }
                __syncwarp();
                flush_warp(a.out_z + (wpos[k] - sh), st, sh, total[k], a.vec_ok);
                __syncwarp();
                wpos[k] += total[k];
            }
        }
        if (!dense) continue;
        // dense rows: the group's dictionary slice is read once per part
        // (lane l holds entry 32 j + l of the W words j) and shared by the
        // rows; each part is staged and flushed
#pragma unroll
        for (int h = 0; h < P; ++h) {
            int32_t dreg[W];
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int64_t idx = gb + ((W * h + i) << 5) + lane;
                dreg[i] = idx < zlim ? __ldg(a.dict_z + zt0 + idx) : 0;
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                if (total[k] <= 64) continue;
                // the part's first pair and its end (lane 0's exclusive count is 0)
                const int base = h == 0 ? 0 : P == 2 ? mid[k] : __shfl_sync(kFull, excl[k], W * h);
                const int end = h + 1 == P ? total[k] : P == 2 ? mid[k] : __shfl_sync(kFull, excl[k], W * (h + 1));
                const int cnt = end - base;
                if (cnt == 0) continue;
                const int sh = (int)(wpos[k] & 3);
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const uint32_t wj = __shfl_sync(kFull, word[k], W * h + i);
                    const int pj = __shfl_sync(kFull, excl[k], W * h + i) - base;
                    if ((wj >> lane) & 1u) st[sh + pj + __popc(wj & lt)] = dreg[i];
                }
                __syncwarp();
                flush_warp(a.out_z + (wpos[k] - sh), st, sh, cnt, a.vec_ok);
                __syncwarp();
                wpos[k] += cnt;
            }
        }
    }
}

template <int G>
__global__ void __launch_bounds__(kThreads) k_xrow_emit_g(const XRowArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t* stage = reinterpret_cast<int32_t*>(smem);  // kWarps x kWarpStageIds
    uint32_t* bm_all = smem + kWarps * kWarpStageIds;   // G bitmaps of tile_words words
    __shared__ GroupSmem gs;
    __shared__ int32_t s_seg[G][kWarps];
    __shared__ int64_t s_blk, s_prefix;

    // single pass: logical block number from a ticket (dispatch order)
    int64_t blk = blockIdx.x;
    if (a.lb_status) {
        if (threadIdx.x == 0) s_blk = (int64_t)atomicAdd(a.lb_ticket, 1ull);
        __syncthreads();
        blk = s_blk;
    }
    int64_t xr0;
    int ng;
    if (!g_locate<G>(a, blk, xr0, ng)) return;
    const int64_t x0 = a.x_begin + xr0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile_words = a.tile_bits >> 5;
    // z window of the group's instance (all of Z for a single instance; the
    // rows of a group share their instance), from a 32-aligned start so that
    // bitmap words line up with the wide rows' words
    const int tg = a.x_tag ? a.x_tag[x0] : 0;
    const int64_t zb = a.z_lo[tg] & ~int64_t(31), ze = a.z_lo[tg + 1];
    const bool tiled = a.tile_bits < ze - zb;
    // R_CSR rows of the group are adjacent; rb is indexed only with unrolled
    // constants so that it stays in registers
    int64_t rb[G + 1];
#pragma unroll
    for (int k = 0; k <= G; ++k) rb[k] = a.r_rowptr[x0 + min(k, ng)];
    int64_t out_pos[G];
    bool write = true;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        out_pos[k] = 0;
        if (k < ng && !a.lb_status) {
            out_pos[k] = a.off[xr0 + k];
            fill_range(a.out_x, out_pos[k], a.off[xr0 + k + 1], a.dict_x[x0 + k], a.vec_ok);
        }
    }
    const bool flat = g_prepare<G>(a, rb, ng, gs);
    for (int64_t zt0 = zb; zt0 < ze; zt0 += a.tile_bits) {
        const int64_t zt1 = min64(zt0 + a.tile_bits, ze);
        const int tw = (int)((zt1 - zt0 + 31) >> 5);
        g_build<G>(a, rb, ng, flat, tg, xr0, zb, zt0, zt1, tiled, bm_all, tile_words, gs);
        g_counts<G>(bm_all, tile_words, tw, ng, s_seg);
        if (a.lb_status) {
            // single pass (one z tile): this block's rows start after all
            // earlier blocks' pairs
            int64_t agg = 0;
#pragma unroll
            for (int k = 0; k < G; ++k)
                for (int w = 0; w < kWarps; ++w) agg += k < ng ? s_seg[k][w] : 0;
            if (warp == 0) {
                const int64_t pre = lookback_prefix(a.lb_status, blk, agg, a.lb_err, kLookbackWaitNs);
                if (lane == 0) s_prefix = pre;
            }
            __syncthreads();
            const int64_t pre = s_prefix;
            write = pre >= 0 && pre + agg <= a.capacity;
            int64_t run = pre;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                int64_t ck = 0;
                for (int w = 0; w < kWarps; ++w) ck += k < ng ? s_seg[k][w] : 0;
                out_pos[k] = run;
                if (write && k < ng) fill_range(a.out_x, run, run + ck, a.dict_x[x0 + k], a.vec_ok);
                if (a.cnt && tid == 0 && k < ng) a.cnt[xr0 + k] = ck;  // the row counts, for later queries
                run += ck;
            }
        }
        if (write) g_emit<G, 2>(a, bm_all, tile_words, tw, ng, zt0, s_seg, out_pos, stage, kWarpStageIds);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            int64_t all = 0;
            for (int w = 0; w < kWarps; ++w) all += s_seg[k][w];
            if (k < ng) out_pos[k] += all;
        }
        __syncthreads();
    }
}

// Persistent single pass with one row group in flight per CTA. A CTA takes a
// ticket, builds that group's bitmaps and publishes its pair count (the
// look-back aggregate) at once; only then does it resolve the offset of the
// group it built in the previous round -- every earlier group has published
// on being built, so the wait is short -- and write that group, while the new
// one waits in the second bitmap buffer. Output writes no longer stall behind
// the look-back. Rows whose whole z window fits one bitmap only (the
// single-pass condition). Every earlier ticket belongs to a CTA that published
// before waiting on anything, so the waits end; each is bounded all the same.
template <int G>
__global__ void __launch_bounds__(kThreads) k_xrow_emit_pipe(const XRowArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t* stage = reinterpret_cast<int32_t*>(smem);   // kWarps x kWarpStageQ (quarter groups)
    const int64_t tile_words = a.tile_bits >> 5;
    // two buffers of G bitmaps; the second starts on a 16-byte boundary
    // (clear_words stores 16 bytes at a time)
    const int64_t buf_words = (G * tile_words + 3) & ~int64_t(3);
    uint32_t* bm_base = smem + kWarps * kWarpStageQ;
    __shared__ GroupSmem gs;
    __shared__ int32_t s_seg[2][G][kWarps];
    __shared__ int64_t s_blk, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int buf = 0;
    bool have_prev = false;
    int64_t p_blk = 0, p_xr0 = 0, p_agg = 0, p_zb = 0;
    int p_ng = 0, p_tw = 0;
    for (;;) {
        if (tid == 0) s_blk = (int64_t)atomicAdd(a.lb_ticket, 1ull);
        __syncthreads();
        const int64_t blk = s_blk;
        int64_t xr0 = 0, agg = 0, zb = 0;
        int ng = 0, tw = 0;
        const bool have_cur = g_locate<G>(a, blk, xr0, ng);
        if (have_cur) {
            const int64_t x0 = a.x_begin + xr0;
            const int tg = a.x_tag ? a.x_tag[x0] : 0;
            zb = a.z_lo[tg] & ~int64_t(31);
            const int64_t ze = a.z_lo[tg + 1];
            tw = (int)((ze - zb + 31) >> 5);
            int64_t rb[G + 1];
#pragma unroll
            for (int k = 0; k <= G; ++k) rb[k] = a.r_rowptr[x0 + min(k, ng)];
            uint32_t* bm = bm_base + (int64_t)buf * buf_words;
            const bool flat = g_prepare<G>(a, rb, ng, gs);
            g_build<G>(a, rb, ng, flat, tg, xr0, zb, zb, ze, false, bm, tile_words, gs);
            g_counts<G>(bm, tile_words, tw, ng, s_seg[buf]);
#pragma unroll
            for (int k = 0; k < G; ++k)
                for (int w = 0; w < kWarps; ++w) agg += k < ng ? s_seg[buf][k][w] : 0;
            if (tid == 0) lookback_publish(a.lb_status, blk, agg);
        }
        if (have_prev) {
            const int pb = buf ^ 1;
            if (warp == 0) {
                const int64_t pre = lookback_resolve(a.lb_status, p_blk, p_agg, a.lb_err, kLookbackWaitNs);
                if (lane == 0) s_prefix = pre;
            }
            __syncthreads();
            const int64_t pre = s_prefix;
            const bool write = pre >= 0 && pre + p_agg <= a.capacity;
            const int64_t px0 = a.x_begin + p_xr0;
            int64_t row_pos[G];
            int64_t run = pre;
#pragma unroll
            for (int k = 0; k < G; ++k) {
                int64_t ck = 0;
                for (int w = 0; w < kWarps; ++w) ck += k < p_ng ? s_seg[pb][k][w] : 0;
                row_pos[k] = run;
                if (write && k < p_ng) fill_range(a.out_x, run, run + ck, a.dict_x[px0 + k], a.vec_ok);
                if (a.cnt && tid == 0 && k < p_ng) a.cnt[p_xr0 + k] = ck;
                run += ck;
            }
            if (write)
                g_emit<G, 4>(a, bm_base + (int64_t)pb * buf_words, tile_words, p_tw, p_ng, p_zb, s_seg[pb], row_pos,
                             stage, kWarpStageQ);
            __syncthreads();
        }
        if (!have_cur) break;
        have_prev = true;
        p_blk = blk;
        p_xr0 = xr0;
        p_ng = ng;
        p_agg = agg;
        p_zb = zb;
        p_tw = tw;
        buf ^= 1;
    }
}

// Join-Count: counters per z of a tile.
template <bool kEmit>
__global__ void __launch_bounds__(kThreads) k_xrow_counts(const XRowArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t* stage_z = reinterpret_cast<int32_t*>(smem);          // kCntChunk + 8
    int32_t* stage_c = stage_z + (kCntChunk + 8);                  // kCntChunk + 8
    uint32_t* ctr = reinterpret_cast<uint32_t*>(stage_c + (kCntChunk + 8));  // tile counters
    __shared__ int64_t s_scan[kThreads / 32 + 1];

    const int64_t xr = blockIdx.x;
    if (xr >= a.n_rows) return;
    const int64_t x = a.x_begin + xr;
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tg = a.x_tag ? a.x_tag[x] : 0;
    const int64_t zb = a.z_lo[tg] & ~int64_t(31), ze = a.z_lo[tg + 1];  // z window of x's instance
    const bool tiled = a.tile_bits < ze - zb;
    int64_t total = 0;
    int64_t out_pos = 0;
    if (kEmit) {
        out_pos = a.off[xr];
        fill_range(a.out_x, out_pos, a.off[xr + 1], a.dict_x[x], a.vec_ok);
    }
    for (int64_t zt0 = zb; zt0 < ze; zt0 += a.tile_bits) {
        const int64_t zt1 = min64(zt0 + a.tile_bits, ze);
        const int tn = (int)(zt1 - zt0);
        for (int i = tid; i < tn; i += kThreads) ctr[i] = 0u;
        __syncthreads();
        for (int64_t p = r0 + warp; p < r1; p += kThreads / 32) {
            const int32_t y = a.r_col[p];
            int64_t s0 = a.ss_rowptr[y], s1 = a.ss_rowptr[y + 1];
            if (tiled) {
                const int64_t* tp = a.tile_ptr + (int64_t)y * a.tile_cols + (zt0 - zb) / a.tile_bits;
                s0 = tp[0];
                s1 = tp[1];
            }
            for (int64_t q = s0 + lane; q < s1; q += 32) atomicAdd(&ctr[a.ss_col[q] - (int32_t)zt0], 1u);
        }
        if (a.n_zd > 0) {
            const int32_t* crow = a.d_cnt + xr * a.n_zd;
            for (int64_t d = a.zd_lo[tg] + tid; d < a.zd_lo[tg + 1]; d += kThreads) {
                const int32_t c = crow[d];
                const int32_t z = a.zd_list[d];
                if (c > 0 && z >= zt0 && z < zt1) atomicAdd(&ctr[z - (int32_t)zt0], (uint32_t)c);
            }
        }
        __syncthreads();
        if (!kEmit) {
            int64_t c = 0;
            for (int i = tid; i < tn; i += kThreads) c += ctr[i] != 0u;
            total += block_sum<int64_t, kThreads>(c, s_scan);
        } else {
            constexpr int kPer = kCntChunk / kThreads;  // z per thread per chunk
            for (int c0 = 0; c0 < tn; c0 += kCntChunk) {
                const int i0 = c0 + tid * kPer;
                int n = 0;
#pragma unroll
                for (int j = 0; j < kPer; ++j) n += (i0 + j < tn && ctr[i0 + j] != 0u);
                int64_t ctot;
                const int64_t ex = block_exclusive_scan<int64_t, kThreads>(n, &ctot, s_scan);
                const int sh = (int)(out_pos & 3);
                int pos = sh + (int)ex;
#pragma unroll
                for (int j = 0; j < kPer; ++j) {
                    const int i = i0 + j;
                    if (i < tn) {
                        const uint32_t v = ctr[i];
                        if (v) {
                            stage_z[pos] = a.dict_z[zt0 + i];
                            stage_c[pos] = (int32_t)v;
                            ++pos;
                        }
                    }
                }
                __syncthreads();
                flush_stage(a.out_z + (out_pos - sh), stage_z, sh, (int)ctot, a.vec_ok);
                flush_stage(a.out_c + (out_pos - sh), stage_c, sh, (int)ctot, a.vec_ok);
                out_pos += ctot;
                __syncthreads();
            }
        }
        __syncthreads();
    }
    if (!kEmit && tid == 0) a.cnt[xr] = total;
}

// ------------------------------------------------------------- tiled rows
// A single instance whose z range spans several shared-memory tiles: one CTA
// per x row sweeps the row's z tiles, holding one tile's SPA bitmap at a
// time. The bitmap is built from the row's join tuples that fall in the tile:
// the tile boundaries of every S_sparse row are precomputed (tile_ptr), so
// each R entry y of the row names one segment of S_sparse[y]. Segments of at
// least 32 tuples (in power-law graphs nearly all join tuples lie in them:
// the neighbours of a vertex are biased towards hubs) are cut into pieces of
// up to 256 tuples, and the warps take the pieces in turn, each lane loading
// every 32nd tuple of a piece (coalesced, eight independent loads in flight).
// Shorter segments are walked by the thread that read their entry. (Laying
// all segments end to end and giving every thread eight consecutive tuples
// balances the threads but makes the loads uncoalesced: measured slower on
// both the power-law graph and Zipf tables.) The counting pass stores each
// row's pairs; the emitting pass writes them at the row's offset, tile after
// tile.
constexpr int kTileChunk = kThreads;      // R entries of a row per round (one per thread)
constexpr int kPiece = 256;               // tuples per warp work item
constexpr int kLongSeg = 32;              // segments from this length on go to the warps

// Shared memory of visit_segments.
struct ChunkSmem {
    uint32_t s0[kTileChunk];   // first tuple of the entry's segment in ss_col
    int32_t len[kTileChunk];   // its length
    int32_t pc[kTileChunk];    // exclusive scan of the pieces of long segments
    int32_t sc[kWarps + 1];
};

// Calls visit(z) for every z of the chunk's segments: thread i holds entry
// i's segment (first tuple in ss_col and length, 0 for none), nc entries.
// Long segments are cut into pieces of kPiece tuples taken by the warps in
// turn (coalesced, kPiece / 32 independent loads per lane); short ones are
// walked by the thread that holds them. Contains __syncthreads: call from
// every thread; the caller synchronises before sm is reused.
template <class Visit>
__device__ __forceinline__ void visit_segments(const XRowArgs& a, int nc, int len, uint32_t first, ChunkSmem& sm,
                                               Visit visit) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pc = len >= kLongSeg ? (len + kPiece - 1) / kPiece : 0;
    int n_pieces;
    const int ex = block_exclusive_scan<int, kThreads>(pc, &n_pieces, sm.sc);
    sm.pc[tid] = ex;
    sm.s0[tid] = first;
    sm.len[tid] = len;
    __syncthreads();
    // long segments: piece p of the chunk goes to warp p mod kWarps
    for (int p = warp; p < n_pieces; p += kWarps) {
        int lo = 0, hi = nc;  // the entry whose pieces hold p (the same search in every lane)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sm.pc[mid] <= p) lo = mid; else hi = mid;
        }
        const int off = (p - sm.pc[lo]) * kPiece;
        const int n = min(kPiece, sm.len[lo] - off);
        const int32_t* src = a.ss_col + sm.s0[lo] + off;
        int32_t zz[kPiece / 32];
#pragma unroll
        for (int u = 0; u < kPiece / 32; ++u) zz[u] = u * 32 + lane < n ? __ldg(src + u * 32 + lane) : -1;
#pragma unroll
        for (int u = 0; u < kPiece / 32; ++u)
            if (zz[u] >= 0) visit(zz[u]);
    }
    // short segments: the thread that holds the entry walks it
    if (len > 0 && len < kLongSeg) {
        const int32_t* src = a.ss_col + first;
        for (int q0 = 0; q0 < len; q0 += 4) {
            int32_t zz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) zz[u] = q0 + u < len ? __ldg(src + q0 + u) : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (zz[u] >= 0) visit(zz[u]);
        }
    }
}

// Calls visit(z) for every join tuple (y in R entries [c0, c0 + nc), z in
// S_sparse[y]) -- only the z of tile t when tile_ptr is set; one entry per
// thread (nc <= kTileChunk). Entries whose y is held as a bitmap row are
// skipped when `wide` is set and their bitmap rows appended to
// wide[*nwide++] instead. Contains __syncthreads (see visit_segments).
template <class Visit>
__device__ __forceinline__ void visit_chunk(const XRowArgs& a, int64_t c0, int nc, int t, ChunkSmem& sm,
                                            int32_t* wide, int* nwide, Visit visit) {
    const int tid = threadIdx.x;
    int len = 0;
    uint32_t first = 0u;
    if (tid < nc) {
        const int32_t y = a.r_col[c0 + tid];
        const int32_t b = wide ? a.bm_row_of_y[y] : -1;
        if (b >= 0) {
            wide[atomicAdd(nwide, 1)] = b;
        } else {
            int64_t s0, s1;
            if (a.tile_ptr) {
                const int64_t* tp = a.tile_ptr + (int64_t)y * a.tile_cols + t;
                s0 = tp[0];
                s1 = tp[1];
            } else {
                s0 = a.ss_rowptr[y];
                s1 = a.ss_rowptr[y + 1];
            }
            len = (int)(s1 - s0);
            first = (uint32_t)s0;
        }
    }
    visit_segments(a, nc, len, first, sm, visit);
}

// Set bits of a 16-byte bitmap word.
__device__ __forceinline__ int popc4(const uint4 v) {
    return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

// Block-wide flush of a stage of z ids: dst[t] = dict_z[st[t]] for t in
// [sh, sh + cnt), with 16-byte stores where dst + 0 is 16-byte aligned.
__device__ __forceinline__ void flush_block_ids(int32_t* dst, const int32_t* st, int sh, int cnt,
                                                const int32_t* __restrict__ dict_z, bool vec_ok) {
    const int end = sh + cnt;
    const int nv = (end + 3) >> 2;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const int s = v << 2;
        if (vec_ok && s >= sh && s + 4 <= end) {
            const int4 id = *reinterpret_cast<const int4*>(st + s);
            const int4 val = make_int4(__ldg(dict_z + id.x), __ldg(dict_z + id.y), __ldg(dict_z + id.z),
                                       __ldg(dict_z + id.w));
            __stcs(reinterpret_cast<int4*>(dst + s), val);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = s + j;
                if (t >= sh && t < end) __stcs(dst + t, __ldg(dict_z + st[t]));
            }
        }
    }
}

// 16-byte bitmap words per thread in the scan of a tile of tw4 of them: a
// contiguous run each, of odd length, so that the eight threads of one
// 128-byte phase of a 16-byte shared load start in distinct bank groups.
__device__ __forceinline__ int wide_run(int tw4) { return ((tw4 + kThreads - 1) / kThreads) | 1; }

// One CTA per x row, sweeping the row's z tiles in order with one tile's SPA
// bitmap (the tiles' pairs are consecutive in the output, so x is filled
// once and the offset runs on from tile to tile). Each tile's bitmap is built
// from the row's join tuples in that tile (visit_chunk over the tile starts
// of the S_sparse rows, wide S rows OR-ed in word by word, DenseEC bits).
// Then every thread takes a contiguous run of 16-byte bitmap words, counts
// its set bits, and one block scan places them: the counting pass only adds
// and zeroes; the emitting pass, when the tile's pairs fit the stage, writes
// the z ids of its bits into the stage in z order while zeroing its words
// (the next tile starts clean), and the block flushes the stage as z values
// with 16-byte stores. A denser tile is compacted warp run by warp run
// (compact_run) and cleared afterwards. The scan costs a few instructions
// per 128 z, whichever bits are set.
template <int kMode>
__global__ void __launch_bounds__(kThreads) k_tiled_rows(const XRowArgs a) {
    constexpr bool kWrite = kMode != kCountRows;  // emitting or staging: z values are written
    extern __shared__ __align__(16) uint32_t smem[];
    const int stage_cap = kWrite ? kWarps * a.stage_ints : 0;
    int32_t* stage = reinterpret_cast<int32_t*>(smem);
    uint32_t* bm = smem + stage_cap;
    uint4* b4 = reinterpret_cast<uint4*>(bm);
    __shared__ ChunkSmem cs;
    __shared__ int32_t s_wide[kTileChunk];   // bitmap rows of the chunk's wide S rows
    __shared__ int64_t s_scan[kWarps + 1];
    __shared__ int s_sc[kWarps + 1];
    __shared__ int s_nwide[2];  // wide rows of the current chunk; the two alternate between chunks

    const int64_t li = blockIdx.x;
    if (li >= a.n_list) return;
    const int64_t xr = a.unit_rows ? (int64_t)a.unit_rows[li] : li;
    const int64_t x = a.x_begin + xr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // emitting: the row's pairs go to out_z at its offset (x filled once);
    // staging: its z values go to a.out_z (the staging buffer) at its slot
    int64_t o = 0;
    if (kMode == kEmitRows) {
        o = a.off[xr];
        const int64_t o_end = a.off[xr + 1];
        if (o_end == o) return;
        fill_range(a.out_x, o, o_end, a.dict_x[x], a.vec_ok);
    } else if (kMode == kStageRows) {
        o = a.slot[xr];
    }
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    // A row of at most kTileChunk R entries (the common case) keeps them in
    // registers over its tiles: thread i holds entry i's y, the bitmap row of
    // a wide y (else -1) and the bounds of its segment in the current tile,
    // the next tile's end loaded while the current tile is processed.
    const bool one = r1 - r0 <= kTileChunk;
    int32_t my_y = -1, my_b = -1;
    int64_t seg0 = 0, seg1 = 0;
    if (one && tid < r1 - r0) {
        my_y = a.r_col[r0 + tid];
        my_b = a.bm_row_of_y[my_y];
        if (my_b < 0) {
            const int64_t* tp = a.tile_ptr + (int64_t)my_y * a.tile_cols;
            seg0 = tp[0];
            seg1 = tp[1];
        }
    }
    clear_words(bm, (int)(((a.tile_bits + 127) >> 7) << 2));
    if (tid == 0) s_nwide[0] = s_nwide[1] = 0;
    __syncthreads();
    if (one && my_b >= 0) s_wide[atomicAdd(&s_nwide[1], 1)] = my_b;  // final after the next barrier
    int64_t total = 0;
    // Every tile starts with a clean bitmap and s_nwide[0] = 0: both are
    // restored before the last block barrier of the previous tile.
    for (int t = 0; t < a.n_tiles; ++t) {
        const int64_t zt0 = (int64_t)t * a.tile_bits, zt1 = min64(zt0 + a.tile_bits, a.n_z);
        const int tw = (int)((zt1 - zt0 + 31) >> 5), tw4 = (tw + 3) >> 2;
        if (one) {
            const bool seg = my_y >= 0 && my_b < 0;
            const int64_t nxt = seg && t + 1 < a.n_tiles ? a.tile_ptr[(int64_t)my_y * a.tile_cols + t + 2] : seg1;
            visit_segments(a, (int)(r1 - r0), seg ? (int)(seg1 - seg0) : 0, (uint32_t)seg0, cs, [&](int32_t zid) {
                const int z = (int)(zid - zt0);
                atomicOr(&bm[z >> 5], 1u << (z & 31));
            });
            const int nw = s_nwide[1];  // the row's wide S rows: OR their bitmap words over the tile
            if (nw > 0) {
                const uint32_t* bits = a.ss_bits + (zt0 >> 5);
                for (int w = tid; w < tw; w += kThreads) {
                    uint32_t acc = 0u;
                    for (int i = 0; i < nw; ++i) acc |= __ldg(bits + a.bm_off[s_wide[i]] + w);
                    if (acc) atomicOr(&bm[w], acc);
                }
            }
            seg0 = seg1;
            seg1 = nxt;
        }
        for (int64_t c0 = r0, ck = 0; !one && c0 < r1; c0 += kTileChunk, ++ck) {
            const int nc = (int)min64(kTileChunk, r1 - c0);
            int* nwide = &s_nwide[ck & 1];
            if (tid == 0) s_nwide[(ck + 1) & 1] = 0;  // the next chunk's counter (the previous chunk's is done)
            visit_chunk(a, c0, nc, t, cs, s_wide, nwide, [&](int32_t zid) {
                const int z = (int)(zid - zt0);
                atomicOr(&bm[z >> 5], 1u << (z & 31));
            });
            // wide S rows of the chunk: OR their bitmap words over the tile
            const int nw = *nwide;
            if (nw > 0) {
                const uint32_t* bits = a.ss_bits + (zt0 >> 5);
                for (int w = tid; w < tw; w += kThreads) {
                    uint32_t acc = 0u;
                    for (int i = 0; i < nw; ++i) acc |= __ldg(bits + a.bm_off[s_wide[i]] + w);
                    if (acc) atomicOr(&bm[w], acc);
                }
            }
            __syncthreads();
        }
        if (a.n_zd > 0) {
            // DenseEC result of x over the dense index (see k_xrow_bits)
            const uint32_t* drow = a.d_bits + xr * a.zdw;
            for (int64_t d = tid; d < a.n_zd; d += kThreads) {
                if ((drow[d >> 5] >> (d & 31)) & 1u) {
                    int32_t z = a.zd_list[d];
                    if (z >= zt0 && z < zt1) {
                        z -= (int32_t)zt0;
                        atomicOr(&bm[z >> 5], 1u << (z & 31));
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_nwide[0] = 0;  // the build is done with it; the next barrier publishes it
        const int q = wide_run(tw4);
        const int u0 = min(tid * q, tw4), u1 = min(u0 + q, tw4);
        int c = 0;
        uint64_t nz = 0;  // emitting pass: the nonzero words of this thread's run (at most 52)
        for (int u = u0; u < u1; ++u) {
            const uint4 v = b4[u];
            c += popc4(v);
            if (kWrite) {
                const uint32_t m = (uint32_t)(v.x != 0u) | ((uint32_t)(v.y != 0u) << 1) |
                                   ((uint32_t)(v.z != 0u) << 2) | ((uint32_t)(v.w != 0u) << 3);
                nz |= (uint64_t)m << (4 * (u - u0));
            } else {
                b4[u] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (!kWrite) {
            total += block_sum<int64_t, kThreads>((int64_t)c, s_scan);
            continue;
        }
        // warp w's pairs follow warps 0 .. w-1 of the tile
        const int incl = warp_inclusive_scan(c);
        if (lane == 31) s_sc[warp] = incl;
        __syncthreads();
        int base = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const int n = s_sc[w];
            base += w < warp ? n : 0;
            tot += n;
        }
        if (tot == 0) continue;  // nothing set: the bitmap is clean
        const int64_t wpos = o + base;
        const int mine = __shfl_sync(kFull, incl, 31);
        const int sh = (int)(wpos & 3);
        int32_t* st = stage + warp * a.stage_ints;
        const bool lane_runs = sh + mine <= a.stage_ints;
        if (lane_runs) {
            // every lane writes the z ids of its run's bits in one flat loop
            // of c steps (one per set bit; a nonzero word is read and zeroed
            // when the previous one runs out), so the warp takes as many
            // steps as its fullest lane, not one per word
            int pos = sh + incl - c;
            __syncwarp();  // the warp's previous flush has read the stage
            uint32_t cur = 0u;
            int32_t zb = 0;
            for (int i = 0; i < c; ++i) {
                if (cur == 0u) {
                    const int w = 4 * u0 + __ffsll((long long)nz) - 1;
                    nz &= nz - 1;
                    cur = bm[w];
                    bm[w] = 0u;
                    zb = (int32_t)(zt0 + ((int64_t)w << 5));
                }
                st[pos++] = zb + __ffs(cur) - 1;
                cur &= cur - 1;
            }
        } else if (mine > 0) {
            // a dense run: group by group (compact_run), then zeroed
            const int groups = (tw + 31) >> 5;
            const int g0 = min(groups, warp * 4 * q), g1 = min(groups, (warp + 1) * 4 * q);
            compact_run(a, bm, tw, g0, g1, mine, zt0, wpos, st);
            for (int u = u0; u < u1; ++u) b4[u] = make_uint4(0u, 0u, 0u, 0u);
        }
        // every word is zero again before any warp builds the next tile; the
        // staged ids are flushed while the other warps go on building
        __syncthreads();
        if (lane_runs && mine > 0) {
            __syncwarp();
            flush_warp_ids(a.out_z + (wpos - sh), st, sh, mine, a.dict_z, a.vec_ok);
        }
        o += tot;
        total += tot;
    }
    if (kMode != kEmitRows && tid == 0) a.cnt[xr] = total;
}

// ------------------------------------------------- Join-Count, packed
// Join-Count rows of a single instance. The SPA holds one counter per z of a
// z tile, packed CB bits wide (8 when no x has more than 255 R entries, 16
// up to 65,535, else 32; a pair's count is at most |R[x]|, so it cannot carry
// into the next counter), which puts 4x (2x) as many z in a tile of shared
// memory. Join tuples come from visit_chunk (warp pieces of long S rows,
// threads on short ones) and add 1 << (CB * slot) with one shared atomic;
// DenseEC's counts are added the same way. Every warp then owns a run of the
// tile's counter words: it counts their nonzero counters and, in the
// emitting pass, writes (z, count) of each in z order straight to the output
// (one z per lane, ballot compaction) -- no block barrier between a warp's
// blocks and no staging.
constexpr int64_t kMaxPackedWords = 7168;   // counter words per tile (28 KiB)

template <int CB>
__device__ __forceinline__ uint32_t nonzero_slots(uint32_t w) {
    if (CB == 32) return w != 0u ? 1u : 0u;
    if (CB == 16) return ((w & 0xFFFFu) != 0u ? 1u : 0u) | ((w >> 16) != 0u ? 2u : 0u);
    const uint32_t m = __vcmpne4(w, 0u);  // 0xFF in every nonzero byte
    return ((m >> 7) & 1u) | ((m >> 14) & 2u) | ((m >> 21) & 4u) | ((m >> 28) & 8u);
}

template <int CB, bool kEmit>
__global__ void __launch_bounds__(kThreads) k_cnt_rows(const XRowArgs a) {
    constexpr int CPW = 32 / CB;
    constexpr int LCPW = CB == 8 ? 2 : CB == 16 ? 1 : 0;
    constexpr uint32_t CMASK = CB == 32 ? 0xFFFFFFFFu : ((1u << CB) - 1u);
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* ctr = smem;  // the tile's packed counters
    __shared__ ChunkSmem cs;
    __shared__ int32_t s_wc[kWarps];
    __shared__ int64_t s_scan[kWarps + 1];

    const int64_t xr = blockIdx.x;
    if (xr >= a.n_rows) return;
    const int64_t x = a.x_begin + xr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t r0 = a.r_rowptr[x], r1 = a.r_rowptr[x + 1];
    int64_t out_pos = 0, total = 0;
    if (kEmit) {
        out_pos = a.off[xr];
        if (a.off[xr + 1] == out_pos) return;
        fill_range(a.out_x, out_pos, a.off[xr + 1], a.dict_x[x], a.vec_ok);
    }
    for (int t = 0; t < a.n_tiles; ++t) {
        const int64_t zt0 = (int64_t)t * a.tile_bits, zt1 = min64(zt0 + a.tile_bits, a.n_z);
        const int tw = (int)((zt1 - zt0 + CPW - 1) / CPW);
        clear_words(ctr, tw);
        __syncthreads();
        for (int64_t c0 = r0; c0 < r1; c0 += kTileChunk) {
            visit_chunk(a, c0, (int)min64(kTileChunk, r1 - c0), t, cs, nullptr, nullptr, [&](int32_t zid) {
                const int z = (int)(zid - zt0);
                atomicAdd(&ctr[z >> LCPW], 1u << (CB * (z & (CPW - 1))));
            });
            __syncthreads();
        }
        if (a.n_zd > 0) {
            const int32_t* crow = a.d_cnt + xr * a.n_zd;
            for (int64_t d = tid; d < a.n_zd; d += kThreads) {
                const int32_t c = crow[d];
                const int32_t z = a.zd_list[d];
                if (c > 0 && z >= zt0 && z < zt1) {
                    const int zz = (int)(z - zt0);
                    atomicAdd(&ctr[zz >> LCPW], (uint32_t)c << (CB * (zz & (CPW - 1))));
                }
            }
        }
        __syncthreads();
        // warp w owns counter words [w0, w1) (whole 32-word groups but the last)
        const int wpw = ((tw + kWarps * 32 - 1) / (kWarps * 32)) * 32;
        const int w0 = min(tw, warp * wpw), w1 = min(tw, w0 + wpw);
        int mine = 0;
        for (int w = w0 + lane; w < w1; w += 32) mine += __popc(nonzero_slots<CB>(ctr[w]));
        mine = warp_sum(mine);
        if (!kEmit) {
            total += block_sum<int64_t, kThreads>(lane == 0 ? mine : 0, s_scan);
            continue;  // block_sum ends with a barrier: the tile can be cleared
        }
        if (lane == 0) s_wc[warp] = mine;
        __syncthreads();
        int64_t wpos = out_pos, tile_total = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (w < warp) wpos += s_wc[w];
            tile_total += s_wc[w];
        }
        // Round of 32 counter words (32 * CPW z), lane l holding word l:
        // blocks of 32 consecutive z, each lane taking one z (its word shuffled
        // in), the nonzero ones compacted by a ballot and written straight to
        // the output -- z values read coalesced from the dictionary, stores to
        // consecutive positions; blocks whose words are all zero are skipped.
        constexpr int WPB = 32 / CPW;  // counter words per 32-z block
        constexpr unsigned BMASK = WPB == 32 ? 0xFFFFFFFFu : ((1u << WPB) - 1u);
        for (int wb = w0; wb < w1; wb += 32) {
            const int w = wb + lane;
            const uint32_t word = w < w1 ? ctr[w] : 0u;
            const unsigned nzw = __ballot_sync(kFull, word != 0u);
            if (nzw == 0u) continue;
#pragma unroll
            for (int j = 0; j < CPW; ++j) {
                if (((nzw >> (j * WPB)) & BMASK) == 0u) continue;
                const uint32_t wv = __shfl_sync(kFull, word, j * WPB + lane / CPW);
                const uint32_t c = (wv >> (CB * (lane % CPW))) & CMASK;
                const unsigned m = __ballot_sync(kFull, c != 0u);
                if (c != 0u) {
                    const int64_t pos = wpos + __popc(m & lt);
                    const int64_t z = zt0 + (int64_t)(wb + j * WPB) * CPW + lane;
                    __stcs(a.out_z + pos, __ldg(a.dict_z + z));
                    __stcs(a.out_c + pos, (int32_t)c);
                }
                wpos += __popc(m);
            }
        }
        out_pos += tile_total;
        __syncthreads();
    }
    if (!kEmit && tid == 0) a.cnt[xr] = total;
}

__global__ void k_max_row(const int64_t* __restrict__ rowptr, int64_t n, unsigned long long* out) {
    __shared__ unsigned long long s_w[kThreads / 32 + 1];
    unsigned long long m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)(rowptr[i + 1] - rowptr[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = max(m, s_w[w]);
        atomicMax(out, m);
    }
}

// ----------------------------------------------------------------- host side
static size_t bits_smem(int64_t tile_bits, bool emit, int stage_ints) {
    return (emit ? (size_t)kWarps * stage_ints * 4 : 0) + (size_t)(tile_bits / 32) * 4;
}
static size_t cnt_smem(int64_t tile_bits) { return (size_t)(kCntChunk + 8) * 8 + (size_t)tile_bits * 4; }

static void setup_attrs(const Ctx& ctx) {
    // the largest dynamic shared memory any launch of these kernels asks for
    static bool done[64] = {false};
    const int d = ctx.device & 63;
    if (done[d]) return;
    const int bits_max = (int)bits_smem(kMaxTileWords * 32, true, kWarpStage);
    const int cnt_max = (int)cnt_smem(kMaxCntTile);
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_bits<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bits_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_bits<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bits_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_counts<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cnt_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_counts<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cnt_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_tiled_rows<kCountRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, bits_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_tiled_rows<kEmitRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, bits_max));
    DIM3_CUDA(cudaFuncSetAttribute(k_tiled_rows<kStageRows>, cudaFuncAttributeMaxDynamicSharedMemorySize, bits_max));
    done[d] = true;
}

// Project rows of a single instance whose z range needs several bitmap tiles
// (of at most kMaxTileWords words, or of the option's size) run one CTA per
// row over the tiles (k_tiled_rows).
static bool use_tiles(const Ctx& ctx, const Plan& p, int kind) {
    const int64_t lim = ctx.opt.tile_words > 0 ? std::min<int64_t>(ctx.opt.tile_words, kMaxTileWords) : kMaxTileWords;
    return kind == 0 && p.n_inst == 1 && p.zw > lim;
}

// Bitmap words per tile of k_tiled_rows: the option if set, else the fewest
// tiles of at most kMaxTileWords words, of equal size (a multiple of 32 words).
static int64_t tile_words_for(const Ctx& ctx, const Plan& p) {
    if (ctx.opt.tile_words > 0) return std::min<int64_t>(ctx.opt.tile_words, kMaxTileWords);
    const int64_t n_tiles = ceil_div(p.zw, kMaxTileWords);
    return std::min<int64_t>(kMaxTileWords, ceil_div(ceil_div(p.zw, n_tiles), 32) * 32);
}

// tile_ptr[y * cols + t] = first entry of S_sparse row y with z >= start of
// tile t of y's instance window (t = 0 .. cols - 1)
__global__ void k_tile_ptr(const int64_t* rowptr, const int32_t* col, int64_t n_y, const int32_t* y_tag,
                           const int64_t* z_lo, int64_t tile_bits, int64_t cols, int64_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_y * cols;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / cols, t = i % cols;
        const int tg = y_tag ? y_tag[y] : 0;
        const int64_t v = min64((z_lo[tg] & ~int64_t(31)) + t * tile_bits, (int64_t)INT32_MAX);
        out[i] = lower_bound_dev<int32_t>(col, rowptr[y], rowptr[y + 1], (int32_t)v);
    }
}

// Build (once per pass kind and tile size) the per-row tile starts of a z-tiled plan.
static void ensure_tile_ptr(Plan& p, int kind, int64_t tile_bits, cudaStream_t s) {
    if (p.tile_ptr_bits[kind] == tile_bits) return;
    int64_t n_tiles = 1;
    for (int t = 0; t < p.n_inst; ++t) {
        const int64_t w = p.h_inst_z_lo[t + 1] - (p.h_inst_z_lo[t] & ~int64_t(31));
        n_tiles = std::max<int64_t>(n_tiles, ceil_div(std::max<int64_t>(w, 1), tile_bits));
    }
    const int64_t cols = n_tiles + 1, n_y = p.info.n_y;
    p.tile_ptr[kind].alloc((size_t)std::max<int64_t>(n_y * cols, 1) * 8, s);
    if (n_y > 0) {
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_y * cols, kThreads), 152 * 16));
        k_tile_ptr<<<g, kThreads, 0, s>>>(p.ss_rowptr.as<int64_t>(), p.ss_col.as<int32_t>(), n_y,
                                          p.n_inst > 1 ? p.y_tag.as<int32_t>() : nullptr, p.inst_z_lo.as<int64_t>(),
                                          tile_bits, cols, p.tile_ptr[kind].as<int64_t>());
        DIM3_LAUNCHED();
    }
    p.tile_ptr_bits[kind] = tile_bits;
    p.tile_cols[kind] = cols;
}

static XRowArgs make_args(const Plan& p, int64_t x_begin, int64_t rows, int kind) {
    XRowArgs a{};
    a.x_begin = x_begin;
    a.n_rows = rows;
    a.n_z = p.info.n_z;
    a.zw = p.zw;
    if (kind == 0) {
        const int64_t tw = std::min<int64_t>(p.zw, kMaxTileWords);
        a.tile_bits = tw * 32;
    } else {
        a.tile_bits = std::min<int64_t>(std::max<int64_t>(p.zw * 32, 1), kMaxCntTile);
    }
    a.r_rowptr = p.r_rowptr.as<int64_t>();
    a.r_col = p.r_col.as<int32_t>();
    a.ss_rowptr = p.ss_rowptr.as<int64_t>();
    a.ss_col = p.ss_col.as<int32_t>();
    a.bm_row_of_y = p.bm_row_of_y.as<int32_t>();
    a.bm_off = p.bm_off.as<int64_t>();
    a.ss_bits = p.ss_bits.as<uint32_t>();
    a.x_tag = p.n_inst > 1 ? p.x_tag.as<int32_t>() : nullptr;
    a.z_lo = p.inst_z_lo.as<int64_t>();
    a.zd_lo = p.inst_zd_lo.as<int64_t>();
    a.zdw = p.zdw;
    a.n_zd = p.n_zd_total;  // dense z index plus a partial result cache's columns
    a.zd_list = p.zd_list.as<int32_t>();
    a.dict_x = p.dict_x.as<int32_t>();
    a.dict_z = p.dict_z.as<int32_t>();
    a.stage_ints = kWarpStageIds;
    a.id_max = 512;
    a.flat_max = kThreads;
    a.light = nullptr;
    return a;
}

// x rows per CTA of the emitting pass: the option if set (1, 2 or 4), else 2
// when the two bitmaps keep the CTA under 112 KiB of shared memory, else 1.
// (Measured on the 1M x 1M Zipf workload with the half-group dictionary: one
// pass 2 rows 7.82 ms, 4 rows 8.20 ms; two rows take 64 registers and 43 KiB,
// four CTAs per SM. Capping them at 48 registers for a fifth CTA made the
// kernel 12.98 ms.)
static int emit_rows_per_cta(const Ctx& ctx, int64_t tile_bits) {
    const int64_t want = ctx.opt.emit_rows;
    const int64_t stage = (int64_t)kWarps * kWarpStageIds * 4, bm = (tile_bits / 32) * 4;
    const int64_t cap = (int64_t)ctx.smem_optin - 4096;
    auto fits = [&](int64_t g, int64_t lim) { return stage + g * bm <= lim; };
    if (want == 1 || want == 2 || want == 4) return fits(want, cap) ? (int)want : 1;
    if (fits(2, 112 * 1024)) return 2;
    return 1;
}

// Groups of up to G consecutive rows of [x_begin, x_begin + rows) that stay
// inside one instance of a batch plan, as (first row - x_begin, rows), on the
// device in `out`; returns their number.
static int64_t group_list(const Plan& p, int64_t x_begin, int64_t rows, int G, DevBuf& out, cudaStream_t s) {
    std::vector<int2> g;
    g.reserve((size_t)(rows / G + p.n_inst + 1));
    const int64_t x_end = x_begin + rows;
    for (int t = 0; t < p.n_inst; ++t) {
        const int64_t lo = std::max(x_begin, p.h_inst_x_lo[t]), hi = std::min(x_end, p.h_inst_x_lo[t + 1]);
        for (int64_t r = lo; r < hi; r += G) g.push_back(make_int2((int)(r - x_begin), (int)std::min<int64_t>(G, hi - r)));
    }
    if (g.empty()) return 0;
    out.alloc(g.size() * sizeof(int2), s);
    DIM3_CUDA(cudaMemcpyAsync(out.p, g.data(), g.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    DIM3_CUDA(cudaStreamSynchronize(s));  // the host vector goes out of scope
    return (int64_t)g.size();
}

// Staged entries per warp for the one-row emitting kernel: the large stage
// (whole 1024-z groups per flush) when the range's output fills more than 2 %
// of its rows' z-window bits, else the small one (more CTAs per SM). `pairs`
// is the exact result size or an upper bound of it.
static int stage_for(const Plan& p, int64_t x_begin, int64_t rows, int64_t pairs) {
    double bits = 0.0;
    if (p.n_inst > 1) {
        const int64_t x_end = x_begin + rows;
        for (int t = 0; t < p.n_inst; ++t) {
            const int64_t lo = std::max(x_begin, p.h_inst_x_lo[t]), hi = std::min(x_end, p.h_inst_x_lo[t + 1]);
            if (hi > lo) bits += (double)(hi - lo) * (double)(p.h_inst_z_lo[t + 1] - p.h_inst_z_lo[t]);
        }
    } else {
        bits = (double)rows * (double)p.info.n_z;
    }
    return (double)pairs > 0.02 * bits ? kWarpStage : kWarpStageIds;
}

// Stage size and id-chunk threshold of an emitting launch; the threshold
// leaves room for a chunk plus the 16-byte alignment shift in an empty stage.
static void set_stage(const Ctx& ctx, const Plan& p, XRowArgs& a, int64_t pairs) {
    a.stage_ints = stage_for(p, a.x_begin, a.n_rows, pairs);
    const int64_t want = ctx.opt.id_chunk_max < 0 ? 512 : ctx.opt.id_chunk_max;
    a.id_max = (int)std::min<int64_t>(want, a.stage_ints - 4);
}

// make_args plus, for z-tiled plans, the per-row tile starts.
static XRowArgs prep_args(Plan& p, int64_t x_begin, int64_t rows, int kind, cudaStream_t s) {
    XRowArgs a = make_args(p, x_begin, rows, kind);
    if (p.zw * 32 > a.tile_bits) {
        ensure_tile_ptr(p, kind, a.tile_bits, s);
        a.tile_ptr = p.tile_ptr[kind].as<int64_t>();
        a.tile_cols = p.tile_cols[kind];
    }
    return a;
}

// ------------------------------------------------------------ light rows
// An x whose join tuples are few (|OUT_J| of the row <= kLightMax) on a wide z
// range pays more for clearing and scanning a |Z|-bit SPA than for its
// tuples. One warp per such row gathers the z ids of its join tuples into
// shared memory, sorts them (bitonic network) and keeps the first of each run:
// the same deduplicated, ascending z as the SPA gives.
constexpr int kLightMax = 1024;
constexpr int64_t kLightMinZ = 65536;  // z range from which light rows pay off

struct LightArgs {
    const int32_t* rows;  // row numbers (x - x_begin) of the light rows
    int64_t n, x_begin;
    const int64_t* r_rowptr;
    const int32_t* r_col;
    const int64_t* ss_rowptr;
    const int32_t* ss_col;
    const int32_t* dict_x;
    const int32_t* dict_z;
    int64_t* cnt;         // counting and staging passes out
    const int64_t* off;   // emitting pass: row offsets
    int32_t* out_x;
    int32_t* out_z;
    const int64_t* slot;  // staging pass: each row's slot in vals
    int32_t* vals;
};

template <int kMode>
__global__ void __launch_bounds__(kThreads) k_light_rows(const LightArgs a) {
    __shared__ int32_t s_buf[kWarps][kLightMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t* buf = s_buf[warp];
    const unsigned lt = lanemask_lt();
    for (int64_t i = blockIdx.x * (int64_t)kWarps + warp; i < a.n; i += (int64_t)gridDim.x * kWarps) {
        const int64_t xr = a.rows[i], x = a.x_begin + xr;
        // gather the row's join tuples' z ids: 32 R entries at a time, lane l
        // holding entry l's S row start and the exclusive scan of the row
        // lengths; lane l then copies tuples l, l + 32, ... of the batch, its
        // entry found by a binary search over the lanes (shuffles), so the
        // loads of all entries are independent
        int n = 0;
        const int64_t q1 = a.r_rowptr[x + 1];
        for (int64_t qb = a.r_rowptr[x]; qb < q1; qb += 32) {
            const int64_t q = qb + lane;
            int64_t s0 = 0;
            int len = 0;
            if (q < q1) {
                const int32_t y = a.r_col[q];
                s0 = a.ss_rowptr[y];
                len = (int)(a.ss_rowptr[y + 1] - s0);
            }
            const int incl = warp_inclusive_scan(len);
            const int ex = incl - len, m = __shfl_sync(kFull, incl, 31);
            for (int j0 = 0; j0 < m; j0 += 32) {
                const int j = j0 + lane;
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int e = __shfl_sync(kFull, ex, lo + step);
                    if (e <= j) lo += step;
                }
                const int64_t base = __shfl_sync(kFull, s0, lo);
                const int e_lo = __shfl_sync(kFull, ex, lo);
                if (j < m) buf[n + j] = __ldg(a.ss_col + base + (j - e_lo));
            }
            n += m;
        }
        int pw = 1;
        while (pw < n) pw <<= 1;
        for (int t = n + lane; t < pw; t += 32) buf[t] = INT32_MAX;
        __syncwarp();
        for (int k = 2; k <= pw; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < (pw >> 1); t += 32) {
                    const int lo = (t / j) * 2 * j + (t % j), hi = lo + j;
                    const int32_t u = buf[lo], v = buf[hi];
                    if ((u > v) == ((lo & k) == 0)) {
                        buf[lo] = v;
                        buf[hi] = u;
                    }
                }
                __syncwarp();
            }
        }
        // emitting: pairs at the row's offset; staging: z values at its slot
        int64_t o = kMode == kEmitRows ? a.off[xr] : kMode == kStageRows ? a.slot[xr] : 0;
        int run = 0;
        for (int base = 0; base < n; base += 32) {
            const int t = base + lane;
            const int32_t v = t < n ? buf[t] : 0;
            const bool first = t < n && (t == 0 || buf[t - 1] != v);
            const unsigned bal = __ballot_sync(kFull, first);
            if (kMode == kEmitRows && first) {
                const int64_t at = o + run + __popc(bal & lt);
                a.out_x[at] = a.dict_x[x];
                a.out_z[at] = a.dict_z[v];
            } else if (kMode == kStageRows && first) {
                a.vals[o + run + __popc(bal & lt)] = a.dict_z[v];
            }
            run += __popc(bal);
        }
        if (kMode != kEmitRows && lane == 0) a.cnt[xr] = run;
        __syncwarp();
    }
}

// Row classes: 1 light (at most lim join tuples), 0 the rest (bitmap rows).
__global__ void k_light_flags(const int64_t* __restrict__ outj_x, int64_t n_x, int64_t lim, uint8_t* light) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n_x; x += (int64_t)gridDim.x * blockDim.x)
        light[x] = outj_x[x] <= lim ? 1 : 0;
}

__global__ void k_light_range(const uint8_t* __restrict__ light, int64_t x_begin, int64_t rows, int want,
                              int32_t* flag) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = (light ? (int)light[x_begin + r] : 0) == want ? 1 : 0;
}

__global__ void k_light_list(const int32_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t rows,
                             int32_t* list) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) list[pos[r]] = (int32_t)r;
}

static unsigned blocks_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kThreads), 152 * 16));
}

__global__ void k_count_flags(const uint8_t* __restrict__ f, int64_t n, unsigned long long* total) {
    __shared__ unsigned long long s_warp[kThreads / 32 + 1];
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += f[i] != 0;
    c = block_sum<unsigned long long, kThreads>(c, s_warp);
    if (threadIdx.x == 0 && c) atomicAdd(total, c);
}

// Decide once per plan whether light rows apply: a single instance, no dense
// or cached columns (their bits would have to join the sort), a z range of at
// least kLightMinZ, and either a z-tiled plan or a quarter of the rows light
// (otherwise the one-row kernel and the two passes that light rows require
// cost the heavy rows more than the light rows save). Returns the flags or null.
static const uint8_t* ensure_light(const Ctx& ctx, Plan& p, cudaStream_t s) {
    if (p.light_n < 0) {
        p.light_n = 0;
        const int64_t lim = ctx.opt.light_row_max < 0 ? kLightMax : std::min<int64_t>(ctx.opt.light_row_max, kLightMax);
        if (lim > 0 && p.n_inst == 1 && p.n_zd_total == 0 && p.info.n_z >= kLightMinZ && p.info.n_x > 0) {
            p.light.alloc((size_t)p.info.n_x, s);
            k_light_flags<<<blocks_for(p.info.n_x), kThreads, 0, s>>>(p.outj_x.as<int64_t>(), p.info.n_x, lim,
                                                                     p.light.as<uint8_t>());
            DIM3_LAUNCHED();
            DevBuf tot;
            tot.alloc(8, s);
            DIM3_CUDA(cudaMemsetAsync(tot.p, 0, 8, s));
            k_count_flags<<<blocks_for(p.info.n_x), kThreads, 0, s>>>(p.light.as<uint8_t>(), p.info.n_x,
                                                                     tot.as<unsigned long long>());
            DIM3_LAUNCHED();
            const int64_t n_light = read_i64(tot.as<int64_t>(), s);
            const bool tiled = p.zw > kMaxTileWords;
            if (n_light > 0 && (tiled || 4 * n_light >= p.info.n_x)) p.light_n = n_light;
            else p.light.release();
        }
    }
    return p.light_n > 0 ? p.light.as<uint8_t>() : nullptr;
}

// Join-Project rows of a single instance that k_tiled_rows sweeps (one CTA
// per row, the counting pass staging z values for the emitting call): a z
// range wider than one tile, or light rows beside the others (the staging
// pass then sorts the light rows once instead of in both passes).
static bool row_sweep(const Ctx& ctx, Plan& p, int kind, cudaStream_t s) {
    return use_tiles(ctx, p, kind) || (kind == 0 && p.n_inst == 1 && ensure_light(ctx, p, s) != nullptr);
}

// Row numbers r of [x_begin, x_begin + rows) whose light flag equals `want`
// (flags null: every row is heavy) into `list`; returns their number.
static int64_t list_rows(const uint8_t* light, int64_t x_begin, int64_t rows, int want, DevBuf& list,
                         cudaStream_t s) {
    DevBuf flag, pos;
    flag.alloc((size_t)rows * 4, s);
    pos.alloc((size_t)(rows + 1) * 8, s);
    k_light_range<<<blocks_for(rows), kThreads, 0, s>>>(light, x_begin, rows, want, flag.as<int32_t>());
    DIM3_LAUNCHED();
    exclusive_scan_i32_to_i64(flag.as<int32_t>(), pos.as<int64_t>(), rows, s);
    const int64_t n = read_i64(pos.as<int64_t>() + rows, s);
    if (n == 0) return 0;
    list.alloc((size_t)n * 4, s);
    k_light_list<<<blocks_for(rows), kThreads, 0, s>>>(flag.as<int32_t>(), pos.as<int64_t>(), rows, list.as<int32_t>());
    DIM3_LAUNCHED();
    return n;
}

// The light rows (warp sorts) of [x_begin, x_begin + rows): counting (cnt),
// emitting (off, out_x, out_z) or staging (cnt, slot, vals).
static void launch_light(const Plan& p, int mode, int64_t x_begin, int64_t rows, int64_t* cnt, const int64_t* off,
                         int32_t* out_x, int32_t* out_z, const int64_t* slot, int32_t* vals, cudaStream_t s) {
    LightArgs la{};
    la.x_begin = x_begin;
    la.r_rowptr = p.r_rowptr.as<int64_t>();
    la.r_col = p.r_col.as<int32_t>();
    la.ss_rowptr = p.ss_rowptr.as<int64_t>();
    la.ss_col = p.ss_col.as<int32_t>();
    la.dict_x = p.dict_x.as<int32_t>();
    la.dict_z = p.dict_z.as<int32_t>();
    la.cnt = cnt;
    la.off = off;
    la.out_x = out_x;
    la.out_z = out_z;
    la.slot = slot;
    la.vals = vals;
    DevBuf list;
    const int64_t n = list_rows(p.light.as<uint8_t>(), x_begin, rows, 1, list, s);
    if (n > 0) {
        la.rows = list.as<int32_t>();
        la.n = n;
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kWarps), 152 * 8));
        if (mode == kEmitRows) k_light_rows<kEmitRows><<<g, kThreads, 0, s>>>(la);
        else if (mode == kStageRows) k_light_rows<kStageRows><<<g, kThreads, 0, s>>>(la);
        else k_light_rows<kCountRows><<<g, kThreads, 0, s>>>(la);
        DIM3_LAUNCHED();
    }
}

static void launch_rows(const Ctx& ctx, const XRowArgs& a, int kind, bool emit, cudaStream_t s) {
    if (a.n_rows <= 0 || a.n_z <= 0) return;
    setup_attrs(ctx);
    DIM3_REQUIRE(a.n_rows < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "x range too long");
    const unsigned g = (unsigned)a.n_rows;
    PhaseScope phase(ctx.stats, emit ? PH_EMIT : PH_COUNT, s);
    if (kind == 0) {
        const size_t sm = bits_smem(a.tile_bits, emit, a.stage_ints);
        // several rows per CTA share one z window: batches need a list of
        // groups that stay inside one instance (a.groups)
        const int grp = (emit && !a.light && (a.x_tag == nullptr || a.groups)) ? emit_rows_per_cta(ctx, a.tile_bits) : 1;
        if (emit && grp > 1) {
            const size_t smg = (size_t)kWarps * kWarpStageIds * 4 + (size_t)grp * (size_t)(a.tile_bits / 32) * 4;
            const unsigned gg = (unsigned)(a.groups ? a.n_groups : ceil_div(a.n_rows, grp));
            static int cur2[64] = {0}, cur4[64] = {0};
            int* cur = (grp == 2 ? cur2 : cur4) + (ctx.device & 63);
            if ((int)smg > *cur) {
                if (grp == 2)
                    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_emit_g<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg));
                else
                    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_emit_g<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg));
                *cur = (int)smg;
            }
            if (grp == 2 && a.lb_status && ctx.opt.emit_pipe) {
                // persistent, one group in flight per CTA: two bitmap buffers
                const size_t buf_words = ((size_t)2 * (size_t)(a.tile_bits / 32) + 3) & ~size_t(3);
                const size_t smp = (size_t)kWarps * kWarpStageQ * 4 + 2 * buf_words * 4;
                static int curp[64] = {0};
                if ((int)smp > curp[ctx.device & 63]) {
                    DIM3_CUDA(cudaFuncSetAttribute(k_xrow_emit_pipe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smp));
                    curp[ctx.device & 63] = (int)smp;
                }
                int per_sm = 0;
                DIM3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xrow_emit_pipe<2>, kThreads, smp));
                const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(gg, (int64_t)ctx.sm_count * std::max(per_sm, 1)));
                k_xrow_emit_pipe<2><<<gp, kThreads, smp, s>>>(a);
            } else if (grp == 2) {
                k_xrow_emit_g<2><<<gg, kThreads, smg, s>>>(a);
            } else {
                k_xrow_emit_g<4><<<gg, kThreads, smg, s>>>(a);
            }
        } else if (emit) {
            k_xrow_bits<true><<<g, kThreads, sm, s>>>(a);
        } else {
            k_xrow_bits<false><<<g, kThreads, sm, s>>>(a);
        }
    } else {
        const size_t sm = cnt_smem(a.tile_bits);
        if (emit) k_xrow_counts<true><<<g, kThreads, sm, s>>>(a);
        else k_xrow_counts<false><<<g, kThreads, sm, s>>>(a);
    }
    DIM3_LAUNCHED();
}

// Join-Count rows of a single instance go through k_cnt_rows.
static bool use_packed_counts(const Plan& p, int kind) { return kind == 1 && p.n_inst == 1; }

// Counter width of k_cnt_rows: the largest |R[x]| bounds every count.
static int counter_bits(Plan& p, cudaStream_t s) {
    if (p.max_mx < 0) {
        DevBuf m;
        m.alloc(8, s);
        DIM3_CUDA(cudaMemsetAsync(m.p, 0, 8, s));
        if (p.info.n_x > 0) {
            k_max_row<<<blocks_for(p.info.n_x), kThreads, 0, s>>>(p.r_rowptr.as<int64_t>(), p.info.n_x,
                                                                 m.as<unsigned long long>());
            DIM3_LAUNCHED();
        }
        p.max_mx = read_i64(m.as<int64_t>(), s);
    }
    return p.max_mx <= 255 ? 8 : p.max_mx <= 65535 ? 16 : 32;
}

// Arguments of k_cnt_rows: z per tile = counter words (at most kMaxPackedWords,
// equal tiles) x counters per word; tile starts when there are several tiles.
static XRowArgs cnt_args(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t rows, int cb, cudaStream_t s) {
    XRowArgs a = make_args(p, x_begin, rows, 1);
    const int64_t cpw = 32 / cb;
    const int64_t words = std::max<int64_t>(1, ceil_div(p.info.n_z, cpw));
    const int64_t max_words = ctx.opt.tile_words > 0 ? ctx.opt.tile_words : kMaxPackedWords;
    const int64_t n_tiles = ceil_div(words, max_words);
    a.tile_bits = ceil_div(words, n_tiles) * cpw;
    a.n_tiles = (int)ceil_div(std::max<int64_t>(p.info.n_z, 1), a.tile_bits);
    a.tile_ptr = nullptr;
    if (a.n_tiles > 1) {
        ensure_tile_ptr(p, 1, a.tile_bits, s);
        a.tile_ptr = p.tile_ptr[1].as<int64_t>();
        a.tile_cols = p.tile_cols[1];
    }
    return a;
}

static void launch_cnt(const Ctx& ctx, const XRowArgs& a, int cb, bool emit, cudaStream_t s) {
    if (a.n_rows <= 0 || a.n_z <= 0) return;
    static bool done[64] = {false};
    if (!done[ctx.device & 63]) {
        const int mx = (int)((size_t)12288 * 4);  // the largest tile option
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        DIM3_CUDA(cudaFuncSetAttribute(k_cnt_rows<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        done[ctx.device & 63] = true;
    }
    DIM3_REQUIRE(a.n_rows < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "x range too long");
    PhaseScope phase(ctx.stats, emit ? PH_EMIT : PH_COUNT, s);
    const size_t words = (size_t)ceil_div(a.tile_bits, 32 / cb);
    const size_t sm = words * 4;
    const unsigned g = (unsigned)a.n_rows;
#define DIM3_CNT_LAUNCH(CB)                                                 \
    do {                                                                    \
        if (emit) k_cnt_rows<CB, true><<<g, kThreads, sm, s>>>(a);          \
        else k_cnt_rows<CB, false><<<g, kThreads, sm, s>>>(a);              \
    } while (0)
    if (cb == 8) DIM3_CNT_LAUNCH(8);
    else if (cb == 16) DIM3_CNT_LAUNCH(16);
    else DIM3_CNT_LAUNCH(32);
#undef DIM3_CNT_LAUNCH
    DIM3_LAUNCHED();
}

// One CTA per listed row over its z tiles: counting (a.cnt), emitting
// (a.off) or staging (a.slot, a.cnt; a.out_z is the staging buffer).
static void launch_wide(const Ctx& ctx, const XRowArgs& a, int mode, cudaStream_t s) {
    if (a.n_list <= 0) return;
    DIM3_REQUIRE(a.n_list < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "x range too long");
    setup_attrs(ctx);
    PhaseScope phase(ctx.stats, mode == kEmitRows ? PH_EMIT : PH_COUNT, s);
    const size_t sm = bits_smem(a.tile_bits, mode != kCountRows, a.stage_ints);
    if (mode == kEmitRows) k_tiled_rows<kEmitRows><<<(unsigned)a.n_list, kThreads, sm, s>>>(a);
    else if (mode == kStageRows) k_tiled_rows<kStageRows><<<(unsigned)a.n_list, kThreads, sm, s>>>(a);
    else k_tiled_rows<kCountRows><<<(unsigned)a.n_list, kThreads, sm, s>>>(a);
    DIM3_LAUNCHED();
}

// Staged rows to their places: row r's z values from vals[slot[r] ..] to
// out_z[off[r] .. off[r + 1]) (16-byte stores where the output is aligned),
// x = dict_x[x_begin + r] beside them. One CTA per row, rows in turn.
__global__ void __launch_bounds__(kThreads) k_place_rows(const int64_t* __restrict__ off,
                                                         const int64_t* __restrict__ slot,
                                                         const int32_t* __restrict__ vals, int64_t rows,
                                                         int64_t x_begin, const int32_t* __restrict__ dict_x,
                                                         int32_t* out_x, int32_t* out_z, int vec_ok) {
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int64_t o0 = off[r], o1 = off[r + 1];
        if (o0 == o1) continue;
        const int64_t d = slot[r] - o0;  // vals index of output position o: o + d
        fill_range(out_x, o0, o1, dict_x[x_begin + r], vec_ok);
        if (!vec_ok) {
            for (int64_t o = o0 + threadIdx.x; o < o1; o += blockDim.x) __stcs(out_z + o, __ldcs(vals + o + d));
            continue;
        }
        const int64_t a = min64(o1, (o0 + 3) & ~int64_t(3)), b = max64(a, o1 & ~int64_t(3));
        for (int64_t o = o0 + threadIdx.x; o < a; o += blockDim.x) __stcs(out_z + o, __ldcs(vals + o + d));
        // 16-byte pieces [a, b), two per thread and round with all their loads
        // issued first; 16-byte loads too when source and output share their
        // alignment (d a multiple of four)
        const bool same = (d & 3) == 0;
        const int64_t step = 4 * (int64_t)blockDim.x;
        for (int64_t o = a + 4 * (int64_t)threadIdx.x; o < b; o += 2 * step) {
            const int64_t o2 = o + step;
            const bool two = o2 < b;
            const int32_t* v = vals + o + d;
            const int32_t* w = vals + (two ? o2 : o) + d;
            int4 p, q;
            if (same) {
                p = __ldcs(reinterpret_cast<const int4*>(v));
                q = __ldcs(reinterpret_cast<const int4*>(w));
            } else {
                p = make_int4(__ldcs(v), __ldcs(v + 1), __ldcs(v + 2), __ldcs(v + 3));
                q = make_int4(__ldcs(w), __ldcs(w + 1), __ldcs(w + 2), __ldcs(w + 3));
            }
            __stcs(reinterpret_cast<int4*>(out_z + o), p);
            if (two) __stcs(reinterpret_cast<int4*>(out_z + o2), q);
        }
        for (int64_t o = b + threadIdx.x; o < o1; o += blockDim.x) __stcs(out_z + o, __ldcs(vals + o + d));
    }
}

// slot length of row r: min(|OUT_J| of x_begin + r + extra, n_z), rounded
// up to a multiple of four (16-byte aligned slots); extra covers pairs that
// are no join tuples of the plan (a partial result cache's columns)
__global__ void k_slot_len(const int64_t* __restrict__ outj_x, int64_t x_begin, int64_t rows, int64_t extra,
                           int64_t n_z, int64_t* len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        len[r] = (min64(outj_x[x_begin + r] + extra, n_z) + 3) & ~int64_t(3);
}

// make_args with k_tiled_rows's tile size and tile starts (built once per size).
static XRowArgs tile_args(Plan& p, int64_t x_begin, int64_t rows, int64_t tile_bits, cudaStream_t s) {
    XRowArgs a = make_args(p, x_begin, rows, 0);
    a.tile_bits = tile_bits;
    ensure_tile_ptr(p, 0, tile_bits, s);
    a.tile_ptr = p.tile_ptr[0].as<int64_t>();
    a.tile_cols = p.tile_cols[0];
    a.n_tiles = (int)ceil_div(p.info.n_z, tile_bits);
    return a;
}

// Dense results and per-row counts of a range, cached on the plan so that a
// count query followed by the emitting call does the counting pass once.
// Slots of a staging pass over rows [x_begin, x_begin + rows) of a z-tiled
// plan (p.cache_slot, p.cache_vals): each row gets min(its |OUT_J| plus the
// partial result cache's columns, |Z|) entries, a bound of its pairs. Returns false (and allocates nothing) when
// the buffer would take more than a quarter of the free device memory.
static bool stage_slots(Plan& p, int64_t x_begin, int64_t rows, cudaStream_t s) {
    p.cache_slot.alloc((size_t)(rows + 1) * 8, s);
    {
        DevBuf len;
        len.alloc((size_t)rows * 8, s);
        k_slot_len<<<blocks_for(rows), kThreads, 0, s>>>(p.outj_x.as<int64_t>(), x_begin, rows, p.n_zc,
                                                         p.info.n_z, len.as<int64_t>());
        DIM3_LAUNCHED();
        exclusive_scan_i64(len.as<int64_t>(), p.cache_slot.as<int64_t>(), rows, s);
    }
    const int64_t n = read_i64(p.cache_slot.as<int64_t>() + rows, s);
    size_t free_b = 0, total_b = 0;
    DIM3_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if ((double)n * 4.0 > 0.25 * (double)free_b) {
        p.cache_slot.release();
        return false;
    }
    p.cache_vals.alloc((size_t)std::max<int64_t>(n, 4) * 4, s);
    return true;
}

// The counting pass of a range (row offsets in p.cache_off, dense results).
// With `stage` (an emitting call follows) a z-tiled plan also keeps every
// row's z values (p.cache_vals), so that the emitting pass only places them.
static void ensure_counts(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int kind, cudaStream_t s,
                          bool stage = false) {
    if (p.cache_begin == x_begin && p.cache_end == x_end && p.cache_kind == kind) return;
    p.cache_begin = p.cache_end = -1;
    p.cache_kind = -1;
    const int64_t rows = x_end - x_begin;
    p.cache_dbits.release();
    p.cache_dcnt.release();
    p.cache_vals.release();
    p.cache_slot.release();
    DIM3_REQUIRE(kind == 0 || p.n_zc == 0, DIM3_ERR_UNSUPPORTED,
                 "Join-Count on a plan with a partial result cache (the cache holds pairs, not counts)");
    if (p.n_zd_total > 0 && rows > 0) {
        if (kind == 0) {
            p.cache_dbits.alloc((size_t)(rows * p.zdw) * 4, s);
            dense_ec(ctx, p, x_begin, rows, 0, p.cache_dbits.as<uint32_t>(), nullptr, s);
        } else {
            p.cache_dcnt.alloc((size_t)(rows * p.info.n_z_dense) * 4, s);
            dense_ec(ctx, p, x_begin, rows, 1, nullptr, p.cache_dcnt.as<int32_t>(), s);
        }
    }
    DevBuf cnt;
    cnt.alloc((size_t)std::max<int64_t>(rows, 1) * 8, s);
    p.cache_off.alloc((size_t)(rows + 1) * 8, s);
    p.cache_units.release();
    p.cache_n_list = 0;
    if (rows > 0) {
        if (p.info.n_z <= 0 || p.info.n_r_kept == 0) {
            DIM3_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)rows * 8, s));
        } else if (use_packed_counts(p, kind)) {
            XRowArgs a = cnt_args(ctx, p, x_begin, rows, counter_bits(p, s), s);
            a.d_cnt = p.cache_dcnt.as<int32_t>();
            a.cnt = cnt.as<int64_t>();
            launch_cnt(ctx, a, counter_bits(p, s), false, s);
        } else if (row_sweep(ctx, p, kind, s)) {
            XRowArgs a = tile_args(p, x_begin, rows, tile_words_for(ctx, p) * 32, s);
            a.d_bits = p.cache_dbits.as<uint32_t>();
            const uint8_t* light = ensure_light(ctx, p, s);
            a.n_list = light ? list_rows(light, x_begin, rows, 0, p.cache_units, s) : rows;
            a.unit_rows = p.cache_units.as<int32_t>();
            a.cnt = cnt.as<int64_t>();
            DIM3_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)rows * 8, s));
            const int mode = stage && !ctx.opt.two_pass && stage_slots(p, x_begin, rows, s) ? kStageRows : kCountRows;
            if (mode == kStageRows) {
                a.slot = p.cache_slot.as<int64_t>();
                a.out_z = p.cache_vals.as<int32_t>();
                a.vec_ok = 1;
                set_stage(ctx, p, a, p.info.out_j);
            }
            launch_wide(ctx, a, mode, s);
            if (light) {
                PhaseScope phase(ctx.stats, PH_COUNT, s);
                launch_light(p, mode, x_begin, rows, cnt.as<int64_t>(), nullptr, nullptr, nullptr,
                             p.cache_slot.as<int64_t>(), p.cache_vals.as<int32_t>(), s);
            }
            p.cache_n_list = a.n_list;
            p.cache_tile_bits = a.tile_bits;
        } else {
            XRowArgs a = prep_args(p, x_begin, rows, kind, s);
            a.d_bits = p.cache_dbits.as<uint32_t>();
            a.d_cnt = p.cache_dcnt.as<int32_t>();
            a.cnt = cnt.as<int64_t>();
            a.light = kind == 0 ? ensure_light(ctx, p, s) : nullptr;
            launch_rows(ctx, a, kind, false, s);
            if (a.light) {
                PhaseScope phase(ctx.stats, PH_COUNT, s);
                launch_light(p, kCountRows, x_begin, rows, cnt.as<int64_t>(), nullptr, nullptr, nullptr, nullptr,
                             nullptr, s);
            }
        }
    }
    exclusive_scan_i64(cnt.as<int64_t>(), p.cache_off.as<int64_t>(), rows, s);
    p.cache_begin = x_begin;
    p.cache_end = x_end;
    p.cache_kind = kind;
}

static void check_range(const Plan& p, int64_t x_begin, int64_t x_end) {
    DIM3_REQUIRE(x_begin >= 0 && x_end >= x_begin && x_end <= p.info.n_x, DIM3_ERR_ARG,
                 "x range outside [0, n_x]");
}

__global__ void k_diff_i64(const int64_t* off, int64_t n, int64_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = off[i + 1] - off[i];
}

void plan_row_counts(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int64_t* d_counts, cudaStream_t s) {
    check_range(p, x_begin, x_end);
    ensure_counts(ctx, p, x_begin, x_end, 0, s);
    const int64_t rows = x_end - x_begin;
    if (rows > 0) {
        const unsigned g = (unsigned)std::min<int64_t>(ceil_div(rows, kThreads), 4096);
        k_diff_i64<<<g, kThreads, 0, s>>>(p.cache_off.as<int64_t>(), rows, d_counts);
        DIM3_LAUNCHED();
    }
}

// off[0] = 0, off[i + 1] = inclusive prefix published by row i
__global__ void k_status_to_offsets(const unsigned long long* status, int64_t rows, int64_t* off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= rows; i += (int64_t)gridDim.x * blockDim.x)
        off[i] = i == 0 ? 0 : (int64_t)(status[i - 1] & kLbVal);
}

// Join-Project of a range in ONE emitting pass (no counting pass): every CTA
// counts its rows' pairs, finds its output offset by decoupled look-back over
// the CTAs before it and writes at once. Used when each row's bitmap fits one
// z tile and the caller gave output buffers.
static int64_t plan_join_single_pass(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int32_t* out_x,
                                     int32_t* out_z, int64_t capacity, int64_t* count, cudaStream_t s) {
    const int64_t rows = x_end - x_begin;
    DevBuf dbits;
    if (p.n_zd_total > 0) {
        dbits.alloc((size_t)(rows * p.zdw) * 4, s);
        dense_ec(ctx, p, x_begin, rows, 0, dbits.as<uint32_t>(), nullptr, s);
    }
    XRowArgs a = prep_args(p, x_begin, rows, 0, s);
    a.d_bits = dbits.as<uint32_t>();
    a.out_x = out_x;
    a.out_z = out_z;
    a.vec_ok = ((reinterpret_cast<uintptr_t>(out_x) | reinterpret_cast<uintptr_t>(out_z)) & 15u) == 0;
    const int grp = emit_rows_per_cta(ctx, a.tile_bits);
    DevBuf groups, cnt;
    if (grp > 1 && a.x_tag) {
        a.n_groups = group_list(p, x_begin, rows, grp, groups, s);
        a.groups = groups.as<int2>();
    }
    if (grp > 1) {
        // several rows per block: each block also records its rows' counts
        cnt.alloc((size_t)rows * 8, s);
        a.cnt = cnt.as<int64_t>();
    }
    const int64_t nb = a.groups ? a.n_groups : ceil_div(rows, grp);
    DevBuf status, ticket, err;
    status.alloc((size_t)nb * 8, s);
    ticket.alloc(8, s);
    err.alloc(4, s);
    DIM3_CUDA(cudaMemsetAsync(status.p, 0, (size_t)nb * 8, s));
    DIM3_CUDA(cudaMemsetAsync(ticket.p, 0, 8, s));
    DIM3_CUDA(cudaMemsetAsync(err.p, 0, 4, s));
    a.lb_status = status.as<unsigned long long>();
    a.lb_ticket = ticket.as<unsigned long long>();
    a.lb_err = err.as<int>();
    a.capacity = capacity;
    set_stage(ctx, p, a, std::min<int64_t>(p.info.out_j, capacity));
    launch_rows(ctx, a, 0, true, s);
    unsigned long long last = 0;
    int h_err = 0;
    DIM3_CUDA(cudaMemcpyAsync(&last, status.as<unsigned long long>() + nb - 1, 8, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaMemcpyAsync(&h_err, err.p, 4, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    DIM3_REQUIRE(h_err == 0 && (last >> 62) == 2ull, DIM3_ERR_TIMEOUT,
                 "single-pass compaction: a block's offset was not published in time");
    const int64_t total = (int64_t)(last & kLbVal);
    {
        // the row offsets (the inclusive prefixes with one row per block, else
        // a scan of the recorded row counts) and the dense result become the
        // plan's counting-pass cache
        p.cache_off.alloc((size_t)(rows + 1) * 8, s);
        if (grp == 1) {
            const unsigned g = (unsigned)std::min<int64_t>(ceil_div(rows + 1, kThreads), 4096);
            k_status_to_offsets<<<g, kThreads, 0, s>>>(status.as<unsigned long long>(), rows,
                                                       p.cache_off.as<int64_t>());
            DIM3_LAUNCHED();
        } else {
            exclusive_scan_i64(cnt.as<int64_t>(), p.cache_off.as<int64_t>(), rows, s);
        }
        p.cache_dbits = std::move(dbits);
        p.cache_dcnt.release();
        p.cache_begin = x_begin;
        p.cache_end = x_end;
        p.cache_kind = 0;
        DIM3_CUDA(cudaStreamSynchronize(s));
    }
    if (count) *count = total;
    if (total > capacity)
        throw Error(DIM3_ERR_CAPACITY,
                    "output capacity " + std::to_string(capacity) + " < result size " + std::to_string(total));
    return total;
}

int64_t plan_join(const Ctx& ctx, Plan& p, int64_t x_begin, int64_t x_end, int kind, int32_t* out_x, int32_t* out_z,
                  int32_t* out_cnt, int64_t capacity, int64_t* count, cudaStream_t s) {
    check_range(p, x_begin, x_end);
    const bool cached = p.cache_begin == x_begin && p.cache_end == x_end && p.cache_kind == kind;
    if (!cached && kind == 0 && capacity > 0 && out_x && out_z && x_end > x_begin && p.info.n_z > 0 &&
        p.info.n_r_kept > 0 && !row_sweep(ctx, p, 0, s) && p.zw <= kMaxTileWords && !ctx.opt.two_pass &&
        !ensure_light(ctx, p, s))
        return plan_join_single_pass(ctx, p, x_begin, x_end, out_x, out_z, capacity, count, s);
    ensure_counts(ctx, p, x_begin, x_end, kind, s, true);
    const int64_t rows = x_end - x_begin;
    const int64_t total = read_i64(p.cache_off.as<int64_t>() + rows, s);
    if (count) *count = total;
    if (total > capacity) throw Error(DIM3_ERR_CAPACITY, "output capacity " + std::to_string(capacity) +
                                                             " < result size " + std::to_string(total));
    if (total > 0 && use_packed_counts(p, kind)) {
        DIM3_REQUIRE(out_x && out_z && out_cnt, DIM3_ERR_ARG, "null output buffer");
        const int cb = counter_bits(p, s);
        XRowArgs a = cnt_args(ctx, p, x_begin, rows, cb, s);
        a.d_cnt = p.cache_dcnt.as<int32_t>();
        a.off = p.cache_off.as<int64_t>();
        a.out_x = out_x;
        a.out_z = out_z;
        a.out_c = out_cnt;
        a.vec_ok = ((reinterpret_cast<uintptr_t>(out_x) | reinterpret_cast<uintptr_t>(out_z) |
                     reinterpret_cast<uintptr_t>(out_cnt)) & 15u) == 0;
        launch_cnt(ctx, a, cb, true, s);
    } else if (total > 0 && row_sweep(ctx, p, kind, s) && p.cache_vals.p) {
        // staged by the counting pass: place every row's z values
        DIM3_REQUIRE(out_x && out_z, DIM3_ERR_ARG, "null output buffer");
        PhaseScope phase(ctx.stats, PH_EMIT, s);
        const int vec_ok = ((reinterpret_cast<uintptr_t>(out_x) | reinterpret_cast<uintptr_t>(out_z)) & 15u) == 0;
        k_place_rows<<<(unsigned)std::min<int64_t>(rows, (int64_t)ctx.sm_count * 16), kThreads, 0, s>>>(
            p.cache_off.as<int64_t>(), p.cache_slot.as<int64_t>(), p.cache_vals.as<int32_t>(), rows, x_begin,
            p.dict_x.as<int32_t>(), out_x, out_z, vec_ok);
        DIM3_LAUNCHED();
    } else if (total > 0 && row_sweep(ctx, p, kind, s)) {
        DIM3_REQUIRE(out_x && out_z, DIM3_ERR_ARG, "null output buffer");
        XRowArgs a = tile_args(p, x_begin, rows, p.cache_tile_bits, s);
        a.d_bits = p.cache_dbits.as<uint32_t>();
        a.off = p.cache_off.as<int64_t>();
        a.out_x = out_x;
        a.out_z = out_z;
        a.vec_ok = ((reinterpret_cast<uintptr_t>(out_x) | reinterpret_cast<uintptr_t>(out_z)) & 15u) == 0;
        set_stage(ctx, p, a, total);
        a.unit_rows = p.cache_units.as<int32_t>();
        a.n_list = p.cache_n_list;
        launch_wide(ctx, a, kEmitRows, s);
        if (p.light_n > 0) {
            PhaseScope phase(ctx.stats, PH_EMIT, s);
            launch_light(p, kEmitRows, x_begin, rows, nullptr, a.off, out_x, out_z, nullptr, nullptr, s);
        }
    } else if (total > 0) {
        DIM3_REQUIRE(out_x && out_z && (kind == 0 || out_cnt), DIM3_ERR_ARG, "null output buffer");
        XRowArgs a = prep_args(p, x_begin, rows, kind, s);
        a.d_bits = p.cache_dbits.as<uint32_t>();
        a.d_cnt = p.cache_dcnt.as<int32_t>();
        a.off = p.cache_off.as<int64_t>();
        a.out_x = out_x;
        a.out_z = out_z;
        a.out_c = out_cnt;
        const uintptr_t al = reinterpret_cast<uintptr_t>(out_x) | reinterpret_cast<uintptr_t>(out_z) |
                             (kind ? reinterpret_cast<uintptr_t>(out_cnt) : 0);
        a.vec_ok = (al & 15u) == 0;
        set_stage(ctx, p, a, total);
        a.light = kind == 0 ? ensure_light(ctx, p, s) : nullptr;
        DevBuf groups;
        if (kind == 0 && a.x_tag && !a.light) {
            const int G = emit_rows_per_cta(ctx, a.tile_bits);
            if (G > 1) {
                a.n_groups = group_list(p, x_begin, rows, G, groups, s);
                a.groups = groups.as<int2>();
            }
        }
        launch_rows(ctx, a, kind, true, s);
        if (a.light) {
            PhaseScope phase(ctx.stats, PH_EMIT, s);
            launch_light(p, kEmitRows, x_begin, rows, nullptr, a.off, out_x, out_z, nullptr, nullptr, s);
        }
    }
    DIM3_CUDA(cudaStreamSynchronize(s));
    return total;
}

}  // namespace dimcube
