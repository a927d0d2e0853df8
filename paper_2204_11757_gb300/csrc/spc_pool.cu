// Node-feature pooling onto the super-nodes, and its gradient: the graph-pooling layer built on
// the coarsening (the assignment held fixed).
//
// Definition 2's lift averages over the member pairs of two super-nodes (it divides by
// |u_c| |v_c|).  Its node counterpart is the mean over a super-node's members:
//   xc[U][f] = (sum over the members v of U of x[v][f]) / |U|.
// The paper has no node features, so the summation order is this library's: the members in
// ascending id, in chunks of kPoolChunk consecutive members; each chunk summed left to right
// from 0, then the chunk sums left to right from 0, all with IEEE adds in the feature type;
// then one IEEE division by |U|.  Gradient: grad_x[v][f] = grad_xc[c(v)][f] / |c(v)|.
//
// The members of every super-node are listed by a stable radix sort of the node ids by their
// super-node (stable, so ascending id inside each super-node); member and chunk offsets are
// exclusive scans of the counts.  One thread per (chunk, feature) sums a chunk, one thread per
// (super-node, feature) adds its chunk sums; consecutive threads take consecutive features, so
// member rows are read with coalesced loads, four members' loads in flight at a time while the
// additions stay in order.
#include "spc_internal.cuh"

namespace spc {

namespace {

template <class T> struct PoolOps;
template <> struct PoolOps<float> {
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float div(float a, int64_t c) { return __fdiv_rn(a, __ll2float_rn(c)); }
};
template <> struct PoolOps<double> {
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double div(double a, int64_t c) { return __ddiv_rn(a, __ll2double_rn(c)); }
};

// member counts; lift values outside [0, n_c) are reported and left out
__global__ void k_pool_counts(int64_t n, const int32_t* __restrict__ lift, int64_t n_c,
                              int32_t* __restrict__ cnt, uint32_t* __restrict__ status) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = lift[v];
        if (u < 0 || (int64_t)u >= n_c) {
            atomicOr(status, DEV_BAD_ARG);
            continue;
        }
        atomicAdd(cnt + u, 1);
    }
}

// sort input: key = super-node, value = node id (in ascending order, so the stable sort keeps
// ascending ids inside every super-node)
__global__ void k_pool_keys(int64_t n, const int32_t* __restrict__ lift,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = (uint32_t)lift[v];
        val[v] = (uint32_t)v;
    }
}

constexpr int64_t kPoolChunk = 256;

// chunks of every super-node
__global__ void k_pool_nchunks(int64_t n_c, const int32_t* __restrict__ cnt,
                               int32_t* __restrict__ nch) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        nch[u] = (int32_t)((cnt[u] + kPoolChunk - 1) / kPoolChunk);
}

__global__ void k_pool_owner(int64_t n_c, const int32_t* __restrict__ choff,
                             int32_t* __restrict__ owner) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        for (int32_t c = choff[u]; c < choff[u + 1]; ++c) owner[c] = (int32_t)u;
}

// one thread per (chunk, feature): the chunk's members summed left to right from 0
template <class T>
__global__ void __launch_bounds__(kThreads)
k_pool_partials(int64_t n_c, int64_t F, const int32_t* __restrict__ off,
                const int32_t* __restrict__ choff, const int32_t* __restrict__ owner,
                const uint32_t* __restrict__ members, const T* __restrict__ x,
                T* __restrict__ part, const uint32_t* status) {
    if (*status) return;
    const int64_t total = (int64_t)choff[n_c] * F;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / F;
        const int64_t f = t - c * F;
        const int32_t u = owner[c];
        const int64_t k0 = off[u] + (c - choff[u]) * kPoolChunk;
        const int64_t kend = k0 + kPoolChunk < off[u + 1] ? k0 + kPoolChunk : off[u + 1];
        T acc = T(0);
        int64_t k = k0;
        for (; k + 4 <= kend; k += 4) {
            const T a0 = x[(int64_t)members[k] * F + f];
            const T a1 = x[(int64_t)members[k + 1] * F + f];
            const T a2 = x[(int64_t)members[k + 2] * F + f];
            const T a3 = x[(int64_t)members[k + 3] * F + f];
            acc = PoolOps<T>::add(acc, a0);
            acc = PoolOps<T>::add(acc, a1);
            acc = PoolOps<T>::add(acc, a2);
            acc = PoolOps<T>::add(acc, a3);
        }
        for (; k < kend; ++k) acc = PoolOps<T>::add(acc, x[(int64_t)members[k] * F + f]);
        part[t] = acc;
    }
}

// one thread per (super-node, feature): the chunk sums left to right from 0, then the mean
template <class T>
__global__ void __launch_bounds__(kThreads)
k_pool_forward(int64_t n_c, int64_t F, const int32_t* __restrict__ cnt,
               const int32_t* __restrict__ choff, const T* __restrict__ part,
               T* __restrict__ xc, const uint32_t* status) {
    if (*status) return;
    const int64_t total = n_c * F;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = t / F;
        const int64_t f = t - u * F;
        T acc = T(0);
        for (int64_t c = choff[u]; c < choff[u + 1]; ++c)
            acc = PoolOps<T>::add(acc, part[c * F + f]);
        xc[t] = cnt[u] > 0 ? PoolOps<T>::div(acc, cnt[u]) : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads)
k_pool_backward(int64_t n, int64_t F, const int32_t* __restrict__ lift,
                const int32_t* __restrict__ cnt, const T* __restrict__ grad_xc,
                T* __restrict__ grad_x, const uint32_t* status) {
    if (*status) return;
    const int64_t total = n * F;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / F;
        const int64_t f = t - v * F;
        const int32_t u = lift[v];
        grad_x[t] = PoolOps<T>::div(grad_xc[(int64_t)u * F + f], cnt[u]);
    }
}

// member counts of every super-node, checked (a sync: the later kernels index with them)
spc_status pool_counts(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c) {
    Work& W = ctx->work;
    SPC_TRY(ensure(ctx, W.pool_cnt, (size_t)(n_c + 1) * 4));
    SPC_CUDA(cudaMemsetAsync(W.pool_cnt.p, 0, (size_t)(n_c + 1) * 4, ctx->stream));
    if (n > 0) {
        SPC_LAUNCH(ctx, k_pool_counts, grid_for(n, kThreads, ctx->num_sms * 8), kThreads, 0, n,
                   lift, n_c, W.pool_cnt.as<int32_t>(), ctx->d_status);
    }
    return sync_status(ctx);
}

template <class T>
spc_status pool_forward_typed(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                              int64_t F, const T* x, T* xc) {
    Work& W = ctx->work;
    SPC_TRY(pool_counts(ctx, n, lift, n_c));
    SPC_TRY(ensure(ctx, W.pool_off, (size_t)(n_c + 1) * 4));
    SPC_TRY(scan_i32(ctx, W.pool_cnt.as<int32_t>(), W.pool_off.as<int32_t>(), n_c));
    const size_t nb = (size_t)(n > 0 ? n : 1) * 4;
    SPC_TRY(ensure(ctx, W.pool_key, nb));
    SPC_TRY(ensure(ctx, W.pool_val, nb));
    SPC_TRY(ensure(ctx, W.pool_key2, nb));
    SPC_TRY(ensure(ctx, W.pool_val2, nb));
    int bits = 1;
    while ((1ll << bits) < n_c) ++bits;
    if (n > 0) {
        SPC_LAUNCH(ctx, k_pool_keys, grid_for(n, kThreads, ctx->num_sms * 8), kThreads, 0, n,
                   lift, W.pool_key.as<uint32_t>(), W.pool_val.as<uint32_t>());
        SPC_TRY(radix_sort_u32(ctx, W.pool_key.as<uint32_t>(), W.pool_val.as<uint32_t>(),
                               W.pool_key2.as<uint32_t>(), W.pool_val2.as<uint32_t>(), n, bits));
    }
    // chunks: counts, offsets, owners (at most n_c + n / kPoolChunk of them)
    const int64_t max_chunks = n_c + n / kPoolChunk + 1;
    SPC_TRY(ensure(ctx, W.pool_nch, (size_t)(n_c + 1) * 4));
    SPC_TRY(ensure(ctx, W.pool_choff, (size_t)(n_c + 1) * 4));
    SPC_TRY(ensure(ctx, W.pool_owner, (size_t)max_chunks * 4));
    SPC_TRY(ensure(ctx, W.pool_part, (size_t)max_chunks * F * sizeof(T)));
    const int gu = grid_for(n_c, kThreads, ctx->num_sms * 8);
    SPC_LAUNCH(ctx, k_pool_nchunks, gu, kThreads, 0, n_c, W.pool_cnt.as<int32_t>(),
               W.pool_nch.as<int32_t>());
    SPC_TRY(scan_i32(ctx, W.pool_nch.as<int32_t>(), W.pool_choff.as<int32_t>(), n_c));
    SPC_LAUNCH(ctx, k_pool_owner, gu, kThreads, 0, n_c, W.pool_choff.as<int32_t>(),
               W.pool_owner.as<int32_t>());
    // every feature of every member read once, the member list read once, one partial per
    // chunk and feature written
    note_bytes(ctx, (double)n * F * sizeof(T) + 4.0 * n + (double)max_chunks * F * sizeof(T));
    SPC_LAUNCH(ctx, k_pool_partials<T>, grid_for(max_chunks * F, kThreads, ctx->num_sms * 16),
               kThreads, 0, n_c, F, W.pool_off.as<int32_t>(), W.pool_choff.as<int32_t>(),
               W.pool_owner.as<int32_t>(), W.pool_val.as<uint32_t>(), x, W.pool_part.as<T>(),
               ctx->d_status);
    SPC_LAUNCH(ctx, k_pool_forward<T>, grid_for(n_c * F, kThreads, ctx->num_sms * 16), kThreads, 0,
               n_c, F, W.pool_cnt.as<int32_t>(), W.pool_choff.as<int32_t>(), W.pool_part.as<T>(),
               xc, ctx->d_status);
    return SPC_OK;
}

template <class T>
spc_status pool_backward_typed(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                               int64_t F, const T* grad_xc, T* grad_x) {
    SPC_TRY(pool_counts(ctx, n, lift, n_c));
    if (n == 0) return SPC_OK;
    // lift and counts, every coarse gradient once, every fine gradient written once
    note_bytes(ctx, 4.0 * n + 4.0 * n_c + (double)n_c * F * sizeof(T) +
                        (double)n * F * sizeof(T));
    SPC_LAUNCH(ctx, k_pool_backward<T>, grid_for(n * F, kThreads, ctx->num_sms * 16), kThreads, 0,
               n, F, lift, ctx->work.pool_cnt.as<int32_t>(), grad_xc, grad_x, ctx->d_status);
    return SPC_OK;
}

}  // namespace

spc_status run_pool_forward(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                            int64_t F, spc_dtype dt, const void* x, void* xc) {
    if (dt == SPC_F32)
        return pool_forward_typed<float>(ctx, n, lift, n_c, F, static_cast<const float*>(x),
                                         static_cast<float*>(xc));
    if (dt == SPC_F64)
        return pool_forward_typed<double>(ctx, n, lift, n_c, F, static_cast<const double*>(x),
                                          static_cast<double*>(xc));
    return SPC_ERR_INVALID_ARG;
}

spc_status run_pool_backward(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                             int64_t F, spc_dtype dt, const void* grad_xc, void* grad_x) {
    if (dt == SPC_F32)
        return pool_backward_typed<float>(ctx, n, lift, n_c, F,
                                          static_cast<const float*>(grad_xc),
                                          static_cast<float*>(grad_x));
    if (dt == SPC_F64)
        return pool_backward_typed<double>(ctx, n, lift, n_c, F,
                                           static_cast<const double*>(grad_xc),
                                           static_cast<double*>(grad_x));
    return SPC_ERR_INVALID_ARG;
}

}  // namespace spc
