// Batched execution: many independent Join-Project instances of uneven
// sizes run through ONE pass of the path (the same launches a single
// instance uses), instead of one pass each.
//
// The instances' columns are gathered into concatenated arrays with an
// instance tag per row (one kernel). Mapping then ranks (instance, value)
// pairs, so every instance owns a contiguous block of x, y and z ids and no
// join crosses instances; SparseBMM works in each x's own z window and
// DenseEC computes only the block diagonal. The canonical per-instance results
// come out concatenated in instance order; per-instance sizes are differences
// of the x-row offsets at instance boundaries.
#include <algorithm>
#include <memory>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace dimcube {

struct InstCols {
    const int32_t* key;
    const int32_t* val;
    int64_t off;  // first row of this instance in the concatenation
};

// row i of the concatenation comes from instance t with off[t] <= i < off[t + 1]
__global__ void k_gather_batch(const InstCols* inst, int n_inst, int64_t total, int32_t* key, int32_t* val,
                               int32_t* tag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_inst;  // last t with inst[t].off <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (inst[mid].off <= i) lo = mid; else hi = mid;
        }
        const int64_t j = i - inst[lo].off;
        key[i] = inst[lo].key[j];
        val[i] = inst[lo].val[j];
        tag[i] = lo;
    }
}

__global__ void k_offsets_at(const int64_t* off, const int64_t* x_lo, int n, int64_t* out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n; t += gridDim.x * blockDim.x) out[t] = off[x_lo[t]];
}

static void gather(const std::vector<const int32_t*>& keys, const std::vector<const int32_t*>& vals,
                   const std::vector<int64_t>& lens, DevBuf& key, DevBuf& val, DevBuf& tag, int64_t& total,
                   cudaStream_t s) {
    const int n = (int)lens.size();
    std::vector<InstCols> h(n);
    total = 0;
    for (int t = 0; t < n; ++t) {
        h[t] = {keys[t], vals[t], total};
        total += lens[t];
    }
    DIM3_REQUIRE(total < (int64_t(1) << 31), DIM3_ERR_OVERFLOW, "batch holds more than 2^31 - 1 rows per table");
    key.alloc((size_t)std::max<int64_t>(total, 1) * 4, s);
    val.alloc((size_t)std::max<int64_t>(total, 1) * 4, s);
    tag.alloc((size_t)std::max<int64_t>(total, 1) * 4, s);
    if (total == 0) return;
    DevBuf d;
    d.alloc(h.size() * sizeof(InstCols), s);
    DIM3_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(InstCols), cudaMemcpyHostToDevice, s));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, kThreads), 152 * 16));
    k_gather_batch<<<g, kThreads, 0, s>>>(d.as<InstCols>(), n, total, key.as<int32_t>(), val.as<int32_t>(),
                                          tag.as<int32_t>());
    DIM3_LAUNCHED();
    DIM3_CUDA(cudaStreamSynchronize(s));  // h and d go out of scope
}

Plan* build_batch_plan(const Ctx& ctx, int n_inst, const dim3_instance* inst, int64_t theta_z, cudaStream_t s) {
    DIM3_REQUIRE(n_inst >= 1 && inst, DIM3_ERR_ARG, "empty batch");
    DIM3_REQUIRE(n_inst < (1 << 24), DIM3_ERR_OVERFLOW, "too many instances in one batch");
    std::vector<const int32_t*> rk, rv, sk, sv;
    std::vector<int64_t> nr, ns;
    for (int t = 0; t < n_inst; ++t) {
        const dim3_instance& q = inst[t];
        DIM3_REQUIRE(q.nr >= 0 && q.ns >= 0, DIM3_ERR_ARG, "negative row count in a batch instance");
        DIM3_REQUIRE((q.nr == 0 || (q.r_key && q.r_val)) && (q.ns == 0 || (q.s_key && q.s_val)), DIM3_ERR_ARG,
                     "null column in a batch instance");
        rk.push_back(q.r_key);
        rv.push_back(q.r_val);
        nr.push_back(q.nr);
        sk.push_back(q.s_key);
        sv.push_back(q.s_val);
        ns.push_back(q.ns);
    }
    DevBuf r_key, r_val, r_tag, s_key, s_val, s_tag;
    PlanInput in;
    gather(rk, rv, nr, r_key, r_val, r_tag, in.nr, s);
    gather(sk, sv, ns, s_key, s_val, s_tag, in.ns, s);
    in.r_key = r_key.as<int32_t>();
    in.r_val = r_val.as<int32_t>();
    in.r_tag = r_tag.as<int32_t>();
    in.s_key = s_key.as<int32_t>();
    in.s_val = s_val.as<int32_t>();
    in.s_tag = s_tag.as<int32_t>();
    in.n_inst = n_inst;
    return build_plan(ctx, in, theta_z, s);
}

// Pairs of every instance after a join over all x of a batch plan.
void batch_instance_counts(const Plan& p, int64_t* host_counts, cudaStream_t s) {
    DIM3_REQUIRE(p.cache_begin == 0 && p.cache_end == p.info.n_x, DIM3_ERR_ARG, "no counting pass over the batch");
    DevBuf at;
    at.alloc((size_t)(p.n_inst + 1) * 8, s);
    k_offsets_at<<<1, kThreads, 0, s>>>(p.cache_off.as<int64_t>(), p.inst_x_lo.as<int64_t>(), p.n_inst,
                                        at.as<int64_t>());
    DIM3_LAUNCHED();
    std::vector<int64_t> h(p.n_inst + 1);
    DIM3_CUDA(cudaMemcpyAsync(h.data(), at.p, h.size() * 8, cudaMemcpyDeviceToHost, s));
    DIM3_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t < p.n_inst; ++t) host_counts[t] = h[t + 1] - h[t];
}

}  // namespace dimcube
