// Adjacency reordering (an option of the multilevel driver).  The paper's closing section
// suggests graph adjacency reordering for the memory locality of the score walks; the order
// is this library's choice: the hop distance of every node from node 0 by breadth-first
// search (nodes that node 0 does not reach after all others), nodes renumbered by
// (distance, id).  Breadth-first levels of a geometric graph are shells, so the rows an edge's
// walk reads (its two end points, at most one level apart) sit close together in the
// renumbered CSR.  The coarsening then runs on the renumbered graph: node x of the caller's
// graph is node perm[x] there, and every result refers to the renumbered graph except the
// composed lift, which is read back in the caller's numbering.
#include "spc_scan.cuh"

namespace spc {

namespace {

constexpr int32_t kUnreached = 0x7fffffff;
constexpr int kShortRow = 32;  // rows ranked in registers; longer rows by a radix sort

__global__ void __launch_bounds__(kThreads)
k_bfs_init(int64_t n, int32_t* __restrict__ dist, int32_t* __restrict__ frontier,
           int32_t* __restrict__ counts) {
    spc::pdl_wait();
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t x = t0; x < n; x += (int64_t)gridDim.x * blockDim.x)
        dist[x] = x == 0 ? 0 : kUnreached;
    if (t0 == 0) {
        frontier[0] = 0;
        counts[0] = 1;
        counts[1] = 0;
        counts[2] = 0;
    }
}

// One breadth-first level: the unreached neighbours of the frontier get distance d1 and form
// the next frontier, appended by one atomic per warp and step.  Counts rotate over three
// words: this level reads counts[in], fills counts[out] and zeroes the third, which the level
// before read and the level after fills.
__global__ void __launch_bounds__(kThreads)
k_bfs_expand(const int32_t* __restrict__ frontier_in, const int32_t* in_count,
             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             int32_t* dist, int32_t d1, int32_t* __restrict__ frontier_out, int32_t* out_count,
             int32_t* spare_count) {
    spc::pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) *spare_count = 0;
    const int64_t cnt = *in_count;
    const int lane = threadIdx.x & 31;
    for (int64_t i = t0; i < cnt; i += stride) {
        const int32_t u = frontier_in[i];
        const int64_t r1 = rowptr[u + 1];
        for (int64_t j = rowptr[u]; j < r1; ++j) {
            const int32_t v = col[j];
            const bool found = dist[v] == kUnreached && atomicCAS(dist + v, kUnreached, d1) ==
                                                            kUnreached;
            const unsigned mask = __activemask();
            const unsigned b = __ballot_sync(mask, found);
            if (b) {
                const int leader = __ffs(b) - 1;
                int32_t base = 0;
                if (lane == leader) base = atomicAdd(out_count, __popc(b));
                base = __shfl_sync(mask, base, leader);
                if (found) frontier_out[base + __popc(b & ((1u << lane) - 1u))] = v;
            }
        }
    }
}

// sort keys: the distance (unreached nodes one past the largest), values: the node ids
__global__ void __launch_bounds__(kThreads)
k_bfs_keys(int64_t n, const int32_t* __restrict__ dist, uint32_t far,
           uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = dist[x];
        key[x] = d == kUnreached ? far : (uint32_t)d;
        val[x] = (uint32_t)x;
    }
}

__global__ void k_set_count(int32_t* c) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *c = 0;
}

// the lengths of the listed long rows
__global__ void __launch_bounds__(kThreads)
k_long_lengths(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ long_count,
               const uint32_t* __restrict__ order, const int64_t* __restrict__ rowptr,
               int64_t* __restrict__ len) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = order[long_rows[q]];
        len[q] = rowptr[x + 1] - rowptr[x];
    }
}

// perm[order[r]] = r; the renumbered rows' lengths
__global__ void __launch_bounds__(kThreads)
k_perm_rows(int64_t n, const uint32_t* __restrict__ order, const int64_t* __restrict__ rowptr,
            int32_t* __restrict__ perm, int32_t* __restrict__ deg_new) {
    spc::pdl_wait();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = order[r];
        perm[x] = (int32_t)r;
        deg_new[r] = (int32_t)(rowptr[x + 1] - rowptr[x]);
    }
}

// Renumbered row r (old row order[r]) of at most kShortRow entries: the new columns perm[y]
// ranked in registers and written in ascending order with their weights.  Longer rows are
// listed for the radix path.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_perm_short(int64_t n, const uint32_t* __restrict__ order, const int32_t* __restrict__ perm,
             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const WT* __restrict__ w, const int64_t* __restrict__ rowptr_new,
             int32_t* __restrict__ col_new, WT* __restrict__ w_new,
             int32_t* __restrict__ long_rows, int32_t* long_count) {
    spc::pdl_wait();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = order[r];
        const int64_t r0 = rowptr[x];
        const int d = (int)(rowptr[x + 1] - r0);
        if (d > kShortRow) {
            long_rows[atomicAdd(long_count, 1)] = (int32_t)r;
            continue;
        }
        int32_t c[kShortRow];
#pragma unroll
        for (int k = 0; k < kShortRow; ++k) c[k] = k < d ? perm[col[r0 + k]] : kUnreached;
        const int64_t base = rowptr_new[r];
#pragma unroll
        for (int k = 0; k < kShortRow; ++k) {
            if (k >= d) break;
            int rank = 0;
#pragma unroll
            for (int k2 = 0; k2 < kShortRow; ++k2) rank += c[k2] < c[k] ? 1 : 0;
            col_new[base + rank] = c[k];
            w_new[base + rank] = w[r0 + k];
        }
    }
}

// long rows, step 1: their entries gathered as keys (row r, new column) with the old entry
// index, one warp per long row (off: exclusive prefix of their lengths)
__global__ void __launch_bounds__(kThreads)
k_perm_long_keys(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ long_count,
                 const uint32_t* __restrict__ order, const int32_t* __restrict__ perm,
                 const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const int64_t* __restrict__ off, unsigned long long* __restrict__ key,
                 uint32_t* __restrict__ val) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < cnt;
         q += warps) {
        const int32_t r = long_rows[q];
        const uint32_t x = order[r];
        const int64_t r0 = rowptr[x], d = rowptr[x + 1] - r0;
        for (int64_t k = lane; k < d; k += 32) {
            key[off[q] + k] = ((unsigned long long)(uint32_t)r << 32) |
                              (uint32_t)perm[col[r0 + k]];
            val[off[q] + k] = (uint32_t)(r0 + k);
        }
    }
}

// long rows, step 2: the sorted entries of row r start at the first sorted position holding r
__global__ void __launch_bounds__(kThreads)
k_perm_long_heads(int64_t total, const unsigned long long* __restrict__ key,
                  int64_t* __restrict__ head) {
    spc::pdl_wait();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(key[k] >> 32);
        if (k == 0 || (uint32_t)(key[k - 1] >> 32) != r) head[r] = k;
    }
}

template <class WT>
__global__ void __launch_bounds__(kThreads)
k_perm_long_place(int64_t total, const unsigned long long* __restrict__ key,
                  const uint32_t* __restrict__ val, const int64_t* __restrict__ head,
                  const int64_t* __restrict__ rowptr_new, const WT* __restrict__ w,
                  int32_t* __restrict__ col_new, WT* __restrict__ w_new) {
    spc::pdl_wait();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(key[k] >> 32);
        const int64_t pos = rowptr_new[r] + (k - head[r]);
        col_new[pos] = (int32_t)(uint32_t)key[k];
        w_new[pos] = w[val[k]];
    }
}

// out[x] = in[perm[x]]: the renumbered graph's composed lift read in the caller's numbering
__global__ void __launch_bounds__(kThreads)
k_unpermute(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ in,
            int32_t* __restrict__ out) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        out[x] = in[perm[x]];
}

template <class WT>
spc_status reorder_typed(spc_context* ctx, const GraphView& g, GraphView& out) {
    Work& W = ctx->work;
    const int64_t n = g.n, nnz = g.nnz;
    const int maxb = ctx->num_sms * 8;
    const int gn = grid_for(n, kThreads, maxb);
    const size_t N = (size_t)n + 1;
    SPC_TRY(ensure(ctx, W.ro_dist, N * 4));
    SPC_TRY(ensure(ctx, W.ro_front[0], N * 4));
    SPC_TRY(ensure(ctx, W.ro_front[1], N * 4));
    SPC_TRY(ensure(ctx, W.ro_key, N * 4));
    SPC_TRY(ensure(ctx, W.ro_val, N * 4));
    SPC_TRY(ensure(ctx, W.ro_key2, N * 4));
    SPC_TRY(ensure(ctx, W.ro_val2, N * 4));
    SPC_TRY(ensure(ctx, W.ro_perm, N * 4));
    SPC_TRY(ensure(ctx, W.ro_deg, N * 4));
    SPC_TRY(ensure(ctx, W.ro_rowptr, (N + 1) * 8));
    SPC_TRY(ensure(ctx, W.ro_col, (size_t)(nnz + 1) * 4));
    SPC_TRY(ensure(ctx, W.ro_w, (size_t)(nnz + 1) * sizeof(WT)));
    int32_t* dist = W.ro_dist.as<int32_t>();
    int32_t* counts = W.counters.as<int32_t>() + 56;  // three rotating frontier counts
    out = g;
    if (n == 0) return SPC_OK;
    // ---- breadth-first levels from node 0 --------------------------------------------------
    SPC_LAUNCH(ctx, k_bfs_init, gn, kThreads, 0, n, dist, W.ro_front[0].as<int32_t>(), counts);
    int64_t cur = 1;
    int32_t d = 0;
    for (; cur > 0; ++d) {
        if (d >= n) return SPC_ERR_TIMEOUT;  // a BFS has at most n levels
        const int in = d % 3, o = (d + 1) % 3, spare = (d + 2) % 3;
        SPC_LAUNCH(ctx, k_bfs_expand, grid_for(cur, kThreads, maxb), kThreads, 0,
                   W.ro_front[d & 1].as<int32_t>(), counts + in, g.rowptr, g.col, dist,
                   (int32_t)(d + 1), W.ro_front[(d + 1) & 1].as<int32_t>(), counts + o,
                   counts + spare);
        SPC_TRY(read_loop_count(ctx, counts + o, &cur));
    }
    // d levels were expanded; the last one found nothing, so distances are at most d - 1
    const uint32_t far = (uint32_t)d;
    int bits = 1;
    while ((1ll << bits) <= (int64_t)far) ++bits;
    uint32_t* key = W.ro_key.as<uint32_t>();
    uint32_t* order = W.ro_val.as<uint32_t>();
    SPC_LAUNCH(ctx, k_bfs_keys, gn, kThreads, 0, n, dist, far, key, order);
    SPC_TRY(radix_sort_u32(ctx, key, order, W.ro_key2.as<uint32_t>(), W.ro_val2.as<uint32_t>(),
                           n, bits));
    // ---- the CSR in the new numbering -------------------------------------------------------
    int32_t* perm = W.ro_perm.as<int32_t>();
    int64_t* rowptr_new = W.ro_rowptr.as<int64_t>();
    int32_t* col_new = W.ro_col.as<int32_t>();
    WT* w_new = W.ro_w.as<WT>();
    SPC_LAUNCH(ctx, k_perm_rows, gn, kThreads, 0, n, order, g.rowptr, perm,
               W.ro_deg.as<int32_t>());
    SPC_TRY(scan_i64(ctx, W.ro_deg.as<int32_t>(), rowptr_new, n));
    int32_t* long_rows = W.long_rows.as<int32_t>();
    int32_t* long_count = W.counters.as<int32_t>() + 59;
    SPC_LAUNCH(ctx, k_set_count, 1, 32, 0, long_count);
    SPC_LAUNCH(ctx, k_perm_short<WT>, gn, kThreads, 0, n, order, perm, g.rowptr, g.col,
               static_cast<const WT*>(g.w), rowptr_new, col_new, w_new, long_rows,
               long_count);
    int64_t n_long = 0;
    SPC_TRY(read_i32(ctx, long_count, &n_long));
    if (n_long > 0) {
        int64_t* len = W.lr_len.as<int64_t>();
        int64_t* off = W.lr_eoff.as<int64_t>();
        SPC_LAUNCH(ctx, k_long_lengths, grid_for(n_long, kThreads, maxb), kThreads, 0,
                   long_rows, long_count, order, g.rowptr, len);
        SPC_TRY(scan_i64_i64(ctx, len, off, n_long));
        int64_t total = 0;
        SPC_TRY(read_i64(ctx, off + n_long, &total));
        SPC_TRY(ensure(ctx, W.ro_lkey, (size_t)(total + 1) * 8));
        SPC_TRY(ensure(ctx, W.ro_lkey2, (size_t)(total + 1) * 8));
        SPC_TRY(ensure(ctx, W.ro_lval, (size_t)(total + 1) * 4));
        SPC_TRY(ensure(ctx, W.ro_lval2, (size_t)(total + 1) * 4));
        SPC_TRY(ensure(ctx, W.ro_head, N * 8));
        unsigned long long* lkey = W.ro_lkey.as<unsigned long long>();
        uint32_t* lval = W.ro_lval.as<uint32_t>();
        SPC_LAUNCH(ctx, k_perm_long_keys, grid_for(n_long, kThreads / 32, maxb), kThreads, 0,
                   long_rows, long_count, order, perm, g.rowptr, g.col, off, lkey, lval);
        int nb = 1;
        while ((1ll << nb) < n) ++nb;
        SPC_TRY(radix_sort_u64(ctx, reinterpret_cast<uint64_t*>(lkey), lval,
                               W.ro_lkey2.as<uint64_t>(), W.ro_lval2.as<uint32_t>(), total,
                               32 + nb));
        const int gt = grid_for(total, kThreads, maxb);
        SPC_LAUNCH(ctx, k_perm_long_heads, gt, kThreads, 0, total, lkey,
                   W.ro_head.as<int64_t>());
        SPC_LAUNCH(ctx, k_perm_long_place<WT>, gt, kThreads, 0, total, lkey, lval,
                   W.ro_head.as<int64_t>(), rowptr_new, static_cast<const WT*>(g.w), col_new,
                   w_new);
    }
    out.rowptr = rowptr_new;
    out.col = col_new;
    out.w = w_new;
    return SPC_OK;
}

}  // namespace

spc_status run_reorder(spc_context* ctx, const GraphView& g, GraphView& out) {
    switch (g.wtype) {
        case SPC_I32: return reorder_typed<int32_t>(ctx, g, out);
        case SPC_F32: return reorder_typed<float>(ctx, g, out);
        case SPC_F64: return reorder_typed<double>(ctx, g, out);
    }
    return SPC_ERR_INVALID_ARG;
}

spc_status run_unpermute(spc_context* ctx, int64_t n, const int32_t* in, int32_t* out) {
    if (n <= 0) return SPC_OK;
    SPC_LAUNCH(ctx, k_unpermute, grid_for(n, kThreads, ctx->num_sms * 8), kThreads, 0, n,
               ctx->work.ro_perm.as<int32_t>(), in, out);
    return SPC_OK;
}

}  // namespace spc
