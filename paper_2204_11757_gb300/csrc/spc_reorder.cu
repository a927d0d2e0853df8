// Adjacency reordering (an option of the multilevel driver).  The paper's closing section
// suggests graph adjacency reordering for the memory locality of the score walks; the order
// is this library's choice: the hop distance of every node from node 0 by breadth-first
// search (nodes that node 0 does not reach after all others), nodes renumbered by
// (distance, id).  Breadth-first levels of a geometric graph are shells, so the rows an edge's
// walk reads (its two end points, at most one level apart) sit close together in the
// renumbered CSR.  The coarsening then runs on the renumbered graph: node x of the caller's
// graph is node perm[x] there, and every result refers to the renumbered graph except the
// composed lift, which is read back in the caller's numbering.
#include <atomic>

#include "spc_scan.cuh"

namespace spc {

namespace {

constexpr int32_t kUnreached = 0x7fffffff;
constexpr int kShortRow = 32;  // rows ranked in registers; longer rows by a radix sort
constexpr int kBarGen = 32;    // the grid barrier's generation word, 128 bytes past its counter

__global__ void __launch_bounds__(kThreads)
k_bfs_init(int64_t n, int32_t* __restrict__ dist, int32_t* __restrict__ flags,
           unsigned* __restrict__ bar) {
    spc::pdl_wait();
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t x = t0; x < n; x += (int64_t)gridDim.x * blockDim.x)
        dist[x] = x == 0 ? 0 : kUnreached;
    if (t0 == 0) {
        flags[0] = 0;
        flags[1] = 0;
        flags[2] = 0;
        bar[0] = 0u;
        bar[kBarGen] = 0u;
    }
}

// Grid-wide barrier of a cooperative launch (every block resident, so every wait ends); the
// waits are bounded by the context's wait limit all the same.  bar[0] counts the blocks that
// arrived, bar[kBarGen] (another 128-byte line, so the pollers do not contend with the
// arrivals) is the generation; the pollers back off between reads.  Returns false (and sets
// DEV_TIMEOUT) when a wait gave up.
__device__ bool grid_barrier(unsigned* bar, uint32_t* status) {
    __shared__ int sh_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + kBarGen;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + kBarGen, 1u);
        } else {
            const uint32_t lim = spin_limit(status);
            uint32_t spins = 0;
            while (*gen == g) {
                __nanosleep(32);
                if (++spins > lim) {
                    atomicOr(status, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        sh_ok = ok;
    }
    __syncthreads();
    return sh_ok != 0;
}

// Every breadth-first level in one cooperative launch.  At level d every node at distance d
// gives its unreached neighbours distance d + 1 (one compare-and-swap each).  The nodes of a
// level are found by scanning the distance array (4 bytes a node, resident in L2) rather than
// through a frontier queue, so no counter is shared by the whole grid; the reads bypass L1,
// where a line of an earlier level could be stale.  A block that reached a node sets the
// level's flag (three words rotate: level d sets flags[d % 3] and clears flags[(d + 1) % 3],
// last read two levels earlier); after the grid barrier every block reads the flag, and the
// first level that reached nothing ends the loop.  *levels_out = that level + 1, one past the
// largest distance.
__global__ void __launch_bounds__(kThreads)
k_bfs_all(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
          int32_t* dist, int32_t* flags, unsigned* bar, int32_t* levels_out, uint32_t* status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n4 = n >> 2;
    const int4* dist4 = reinterpret_cast<const int4*>(dist);
    constexpr int kScanUnroll = 8;  // groups of four distances in flight per thread
    int32_t d = 0;
    for (;; ++d) {
        if (t0 == 0) flags[(d + 1) % 3] = 0;
        bool any = false;
        auto expand = [&](int64_t x) {
            const int64_t r1 = rowptr[x + 1];
            for (int64_t j = rowptr[x]; j < r1; ++j) {
                const int32_t v = col[j];
                if (__ldcg(dist + v) == kUnreached &&
                    atomicCAS(dist + v, kUnreached, d + 1) == kUnreached)
                    any = true;
            }
        };
        for (int64_t g0 = t0; g0 < n4; g0 += (int64_t)kScanUnroll * stride) {
            int4 q[kScanUnroll];
#pragma unroll
            for (int u = 0; u < kScanUnroll; ++u) {
                const int64_t g = g0 + (int64_t)u * stride;
                q[u] = g < n4 ? __ldcg(dist4 + g) : make_int4(-1, -1, -1, -1);
            }
#pragma unroll
            for (int u = 0; u < kScanUnroll; ++u) {
                const int64_t x0 = (g0 + (int64_t)u * stride) << 2;
                if (q[u].x == d) expand(x0);
                if (q[u].y == d) expand(x0 + 1);
                if (q[u].z == d) expand(x0 + 2);
                if (q[u].w == d) expand(x0 + 3);
            }
        }
        // the last n mod 4 nodes
        if (t0 < (n & 3) && __ldcg(dist + (n4 << 2) + t0) == d) expand((n4 << 2) + t0);
        if (__syncthreads_or(any) && threadIdx.x == 0) flags[d % 3] = 1;
        if (!grid_barrier(bar, status)) break;
        if (*reinterpret_cast<volatile int32_t*>(flags + d % 3) == 0) break;
    }
    if (t0 == 0) *levels_out = d + 1;
}

// S0 row checks of the caller's graph before the renumbering indexes with it: row pointers
// monotone, columns strictly ascending inside [0, n), no self-loop, weights finite and > 0.
// (Symmetry is checked on the renumbered graph, whose first score walk checks every mirror.)
template <class WT> __device__ __forceinline__ bool weight_ok(WT w);
template <> __device__ __forceinline__ bool weight_ok<int32_t>(int32_t w) { return w > 0; }
template <> __device__ __forceinline__ bool weight_ok<float>(float w) {
    const int b = __float_as_int(w);
    return b > 0 && b < 0x7f800000;
}
template <> __device__ __forceinline__ bool weight_ok<double>(double w) {
    const long long b = __double_as_longlong(w);
    return b > 0 && b < 0x7ff0000000000000ll;
}

template <class WT>
__global__ void __launch_bounds__(kThreads)
k_check_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
             const int32_t* __restrict__ col, const WT* __restrict__ w, uint32_t* status) {
    spc::pdl_wait();
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) atomicOr(status, DEV_UNSORTED);
    for (int64_t x = t0; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        if (r0 < 0 || r1 < r0 || r1 > nnz) {
            atomicOr(status, DEV_UNSORTED);
            continue;
        }
        uint32_t bits = 0;
        int64_t prev = -1;
        for (int64_t j = r0; j < r1; ++j) {
            const int32_t y = col[j];
            if (y < 0 || (int64_t)y >= n || (int64_t)y <= prev) bits |= DEV_UNSORTED;
            if ((int64_t)y == x) bits |= DEV_SELF_LOOP;
            if (!weight_ok<WT>(w[j])) bits |= DEV_BAD_WEIGHT;
            prev = y;
        }
        if (bits) atomicOr(status, bits);
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

// the cooperative launch: as many blocks as fit on the device at once (all resident)
spc_status launch_bfs_all(spc_context* ctx, const GraphView& g, int32_t* dist, int32_t* flags,
                          unsigned* bar, int32_t* levels) {
    static std::atomic<unsigned long long> occ_devs{0};
    static int occ_blocks[64];
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(occ_devs.load() & bit)) {
        int b = 0;
        SPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bfs_all, kThreads, 0));
        occ_blocks[ctx->device & 63] = b;
        occ_devs.fetch_or(bit);
    }
    int per_sm = occ_blocks[ctx->device & 63];
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) return SPC_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctx->num_sms * per_sm));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the CSR's row pointers and columns read once, every distance written once
    note_bytes(ctx, 8.0 * (g.n + 1) + 4.0 * g.nnz + 4.0 * g.n);
    before_launch(ctx, "k_bfs_all");
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_bfs_all, g.n, g.rowptr, g.col, dist, flags, bar,
                                       levels, ctx->d_status);
    if (e == cudaSuccess) e = cudaGetLastError();
    after_launch(ctx, "k_bfs_all");
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "k_bfs_all", __FILE__, __LINE__);
        return SPC_ERR_CUDA;
    }
    return SPC_OK;
}

template <class WT>
spc_status check_rows_typed(spc_context* ctx, const GraphView& g) {
    SPC_LAUNCH(ctx, k_check_rows<WT>, grid_for(g.n, kThreads, ctx->num_sms * 8), kThreads, 0,
               g.n, g.nnz, g.rowptr, g.col, static_cast<const WT*>(g.w), ctx->d_status);
    return check_status(ctx);
}

template <class WT>
spc_status reorder_typed(spc_context* ctx, const GraphView& g, GraphView& out) {
    Work& W = ctx->work;
    const int64_t n = g.n, nnz = g.nnz;
    const int maxb = ctx->num_sms * 8;
    const int gn = grid_for(n, kThreads, maxb);
    const size_t N = (size_t)n + 1;
    SPC_TRY(ensure(ctx, W.ro_dist, N * 4));
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
    int32_t* flags = W.counters.as<int32_t>() + 56;  // three rotating level flags
    out = g;
    if (n == 0) return SPC_OK;
    // ---- breadth-first levels from node 0, all in one cooperative launch ----------------------
    SPC_TRY(ensure(ctx, W.ro_bar, 256));
    unsigned* bar = W.ro_bar.as<unsigned>();
    int32_t* levels = W.counters.as<int32_t>() + 62;
    SPC_LAUNCH(ctx, k_bfs_init, gn, kThreads, 0, n, dist, flags, bar);
    SPC_TRY(launch_bfs_all(ctx, g, dist, flags, bar, levels));
    int64_t d = 0;
    SPC_TRY(read_i32(ctx, levels, &d));
    SPC_TRY(check_status(ctx));  // a barrier that gave up
    // one past the largest distance: the key of the unreached nodes
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

spc_status run_check_rows(spc_context* ctx, const GraphView& g) {
    switch (g.wtype) {
        case SPC_I32: return check_rows_typed<int32_t>(ctx, g);
        case SPC_F32: return check_rows_typed<float>(ctx, g);
        case SPC_F64: return check_rows_typed<double>(ctx, g);
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
