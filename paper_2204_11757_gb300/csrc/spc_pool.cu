// Node-feature pooling onto the super-nodes, and its gradient: the graph-pooling layer built on
// the coarsening (the assignment held fixed).
//
// Definition 2's lift averages over the member pairs of two super-nodes (it divides by
// |u_c| |v_c|).  Its node counterpart is the mean over a super-node's members:
//   xc[U][f] = S(x[v][f] for the members v of U in ascending v) / |U|,
// with one IEEE division.  The paper has no node features, so the summation order S is this
// library's: a 256-ary tree -- a list of at most kPoolChunk items is summed left to right
// from 0 in the feature type; a longer list is replaced by the sums of its consecutive chunks
// of kPoolChunk, recursively.  Gradient: grad_x[v][f] = grad_xc[c(v)][f] / |c(v)|.
//
// The members of every super-node are listed by a stable radix sort of the node ids by their
// super-node (stable, so ascending id inside each super-node).  Each tree level is one pass:
// chunk counts and offsets (scan), the owner of every chunk, and one chunk sum per (chunk,
// feature).  Chunking a list of one item gives that item back (0 + t = t: a sum started at +0
// is never -0), so every super-node runs through the same number of levels, enough for the
// largest possible list.  Blocks are 32 features x 8 units: a warp reads 32 consecutive
// features of one row, so member rows are read with coalesced loads.
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

constexpr int64_t kPoolChunk = 256;
constexpr int kPoolRows = 8;  // units (rows, chunks, super-nodes) per block; 32 features each

// member counts; lift values outside [0, n_c) are reported and left out.  Runs of one
// super-node (a hub holds most nodes of a deep coarsening) are counted with one atomic per
// block or per warp.
__global__ void __launch_bounds__(kThreads)
k_pool_counts(int64_t n, const int32_t* __restrict__ lift, int64_t n_c,
              int32_t* __restrict__ cnt, uint32_t* __restrict__ status) {
    spc::pdl_wait();
    __shared__ int32_t sh_first;
    const int lane = threadIdx.x & 31;
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n;
         b0 += (int64_t)gridDim.x * blockDim.x) {  // uniform per block
        const int64_t v = b0 + threadIdx.x;
        int32_t u = v < n ? lift[v] : -1;
        if (v < n && (u < 0 || (int64_t)u >= n_c)) {
            atomicOr(status, DEV_BAD_ARG);
            u = -1;
        }
        if (threadIdx.x == 0) sh_first = u;
        __syncthreads();
        const int32_t first = sh_first;
        const bool all_same = __syncthreads_and(u == first || v >= n) != 0;
        if (all_same) {
            if (threadIdx.x == 0 && first >= 0) {
                const int64_t k = n - b0 < (int64_t)blockDim.x ? n - b0 : blockDim.x;
                atomicAdd(cnt + first, (int32_t)k);
            }
        } else {
            const unsigned peers = __match_any_sync(0xffffffffu, u);
            if (u >= 0 && lane == __ffs(peers) - 1) atomicAdd(cnt + u, __popc(peers));
        }
        __syncthreads();
    }
}

// sort input: key = super-node, value = node id (in ascending order, so the stable sort keeps
// ascending ids inside every super-node)
__global__ void k_pool_keys(int64_t n, const int32_t* __restrict__ lift,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = (uint32_t)lift[v];
        val[v] = (uint32_t)v;
    }
}

// chunks of every super-node's list at the next tree level
__global__ void k_pool_nchunks(int64_t n_c, const int32_t* __restrict__ items,
                               int32_t* __restrict__ nch) {
    spc::pdl_wait();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        nch[u] = (int32_t)((items[u] + kPoolChunk - 1) / kPoolChunk);
}

__global__ void k_pool_owner(int64_t n_c, const int32_t* __restrict__ choff,
                             int32_t* __restrict__ owner) {
    spc::pdl_wait();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        for (int32_t c = choff[u]; c < choff[u + 1]; ++c) owner[c] = (int32_t)u;
}

// One tree level: the sum of every chunk of kPoolChunk consecutive items of a super-node's
// list, left to right from 0.  Level 0 items are member rows of x (members[k]), later levels
// the previous level's sums (prev[k]).
template <class T>
__global__ void __launch_bounds__(32 * kPoolRows)
k_pool_level(int64_t n_c, int64_t F, const int32_t* __restrict__ ioff,
             const int32_t* __restrict__ icnt, const int32_t* __restrict__ choff,
             const int32_t* __restrict__ owner, const uint32_t* __restrict__ members,
             const T* __restrict__ x, const T* __restrict__ prev, T* __restrict__ part,
             const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    const int64_t nchunks = choff[n_c];
    for (int64_t c = (int64_t)blockIdx.x * kPoolRows + threadIdx.y; c < nchunks;
         c += (int64_t)gridDim.x * kPoolRows) {
        const int32_t u = owner[c];
        const int64_t k0 = ioff[u] + (c - choff[u]) * kPoolChunk;
        const int64_t iend = (int64_t)ioff[u] + icnt[u];
        const int64_t k1 = k0 + kPoolChunk < iend ? k0 + kPoolChunk : iend;
        for (int64_t f = threadIdx.x; f < F; f += 32) {
            T acc = T(0);
            int64_t k = k0;
            if (members) {
                for (; k + 4 <= k1; k += 4) {  // four rows in flight, additions in order
                    const T a0 = x[(int64_t)members[k] * F + f];
                    const T a1 = x[(int64_t)members[k + 1] * F + f];
                    const T a2 = x[(int64_t)members[k + 2] * F + f];
                    const T a3 = x[(int64_t)members[k + 3] * F + f];
                    acc = PoolOps<T>::add(acc, a0);
                    acc = PoolOps<T>::add(acc, a1);
                    acc = PoolOps<T>::add(acc, a2);
                    acc = PoolOps<T>::add(acc, a3);
                }
                for (; k < k1; ++k) acc = PoolOps<T>::add(acc, x[(int64_t)members[k] * F + f]);
            } else {
                for (; k < k1; ++k) acc = PoolOps<T>::add(acc, prev[k * F + f]);
            }
            part[c * F + f] = acc;
        }
    }
}

// the mean: the single sum left after the last level, divided by the member count
template <class T>
__global__ void __launch_bounds__(32 * kPoolRows)
k_pool_mean(int64_t n_c, int64_t F, const int32_t* __restrict__ cnt,
            const int32_t* __restrict__ off, const T* __restrict__ part, T* __restrict__ xc,
            const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    for (int64_t u = (int64_t)blockIdx.x * kPoolRows + threadIdx.y; u < n_c;
         u += (int64_t)gridDim.x * kPoolRows) {
        const int32_t c = cnt[u];
        for (int64_t f = threadIdx.x; f < F; f += 32)
            xc[u * F + f] = c > 0 ? PoolOps<T>::div(part[(int64_t)off[u] * F + f], c) : T(0);
    }
}

template <class T>
__global__ void __launch_bounds__(32 * kPoolRows)
k_pool_backward(int64_t n, int64_t F, const int32_t* __restrict__ lift,
                const int32_t* __restrict__ cnt, const T* __restrict__ grad_xc,
                T* __restrict__ grad_x, const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    for (int64_t v = (int64_t)blockIdx.x * kPoolRows + threadIdx.y; v < n;
         v += (int64_t)gridDim.x * kPoolRows) {
        const int32_t u = lift[v];
        const int32_t c = cnt[u];
        for (int64_t f = threadIdx.x; f < F; f += 32)
            grad_x[v * F + f] = PoolOps<T>::div(grad_xc[(int64_t)u * F + f], c);
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

int pool_grid(int64_t units, int num_sms) {
    return grid_for(units, kPoolRows, num_sms * 16);
}

template <class T>
spc_status pool_forward_typed(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                              int64_t F, const T* x, T* xc) {
    Work& W = ctx->work;
    SPC_TRY(pool_counts(ctx, n, lift, n_c));
    const size_t nb = (size_t)(n > 0 ? n : 1) * 4;
    SPC_TRY(ensure(ctx, W.pool_off, (size_t)(n_c + 1) * 4));
    SPC_TRY(ensure(ctx, W.pool_key, nb));
    SPC_TRY(ensure(ctx, W.pool_val, nb));
    SPC_TRY(ensure(ctx, W.pool_key2, nb));
    SPC_TRY(ensure(ctx, W.pool_val2, nb));
    // tree levels enough for a list of n items; chunk buffers at the level-0 bound
    int levels = 1;
    for (int64_t cap = kPoolChunk; cap < n; cap *= kPoolChunk) ++levels;
    const int64_t max_chunks = n_c + n / kPoolChunk + 1;
    SPC_TRY(ensure(ctx, W.pool_nch, (size_t)(n_c + 1) * 4 * 2));
    SPC_TRY(ensure(ctx, W.pool_choff, (size_t)(n_c + 1) * 4 * 2));
    SPC_TRY(ensure(ctx, W.pool_owner, (size_t)max_chunks * 4));
    SPC_TRY(ensure(ctx, W.pool_part, (size_t)max_chunks * F * sizeof(T) * 2));
    int32_t* cnt = W.pool_cnt.as<int32_t>();
    int32_t* off = W.pool_off.as<int32_t>();
    SPC_TRY(scan_i32(ctx, cnt, off, n_c));
    int bits = 1;
    while ((1ll << bits) < n_c) ++bits;
    if (n > 0) {
        SPC_LAUNCH(ctx, k_pool_keys, grid_for(n, kThreads, ctx->num_sms * 8), kThreads, 0, n,
                   lift, W.pool_key.as<uint32_t>(), W.pool_val.as<uint32_t>());
        SPC_TRY(radix_sort_u32(ctx, W.pool_key.as<uint32_t>(), W.pool_val.as<uint32_t>(),
                               W.pool_key2.as<uint32_t>(), W.pool_val2.as<uint32_t>(), n, bits));
    }
    const int gu = grid_for(n_c, kThreads, ctx->num_sms * 8);
    const dim3 blk(32, kPoolRows);
    const int32_t* icnt = cnt;   // items per super-node at this level
    const int32_t* ioff = off;   // their offsets
    const T* prev = nullptr;
    T* part = W.pool_part.as<T>();
    for (int l = 0; l < levels; ++l) {
        int32_t* nch = W.pool_nch.as<int32_t>() + (l & 1) * (n_c + 1);
        int32_t* choff = W.pool_choff.as<int32_t>() + (l & 1) * (n_c + 1);
        T* out = part + (size_t)(l & 1) * max_chunks * F;
        SPC_LAUNCH(ctx, k_pool_nchunks, gu, kThreads, 0, n_c, icnt, nch);
        SPC_TRY(scan_i32(ctx, nch, choff, n_c));
        SPC_LAUNCH(ctx, k_pool_owner, gu, kThreads, 0, n_c, choff, W.pool_owner.as<int32_t>());
        // level 0: every feature of every member read once, the member list read once,
        // one sum per chunk and feature written
        if (l == 0)
            note_bytes(ctx, (double)n * F * sizeof(T) + 4.0 * n +
                                (double)max_chunks * F * sizeof(T));
        SPC_LAUNCH(ctx, k_pool_level<T>, pool_grid(max_chunks, ctx->num_sms), blk, 0, n_c, F,
                   ioff, icnt, choff, W.pool_owner.as<int32_t>(),
                   l == 0 ? W.pool_val.as<uint32_t>() : nullptr, x, prev, out, ctx->d_status);
        icnt = nch;
        ioff = choff;
        prev = out;
    }
    SPC_LAUNCH(ctx, k_pool_mean<T>, pool_grid(n_c, ctx->num_sms), blk, 0, n_c, F, cnt, ioff,
               prev, xc, ctx->d_status);
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
    SPC_LAUNCH(ctx, k_pool_backward<T>, pool_grid(n, ctx->num_sms), dim3(32, kPoolRows), 0, n, F,
               lift, ctx->work.pool_cnt.as<int32_t>(), grad_xc, grad_x, ctx->d_status);
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
