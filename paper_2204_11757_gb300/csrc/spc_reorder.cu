// Adjacency reordering (an option of the multilevel driver).  The paper's closing section
// suggests graph adjacency reordering for the memory locality of the score walks; the order
// is this library's choice: L_k(x), the smallest node id within k hops of x (x included), by k
// synchronous rounds of L(x) <- min(L(x), min over the neighbours y of L(y)), and the nodes
// renumbered by (L_8(x), L_2(x), x).  Nodes that share their 8-hop label form clusters of
// nearby nodes (a few hundred on a geometric graph), ordered inside by the 2-hop label, so an
// edge's two rows mostly sit close together in the renumbered CSR; the rounds are independent
// of the graph's diameter.  The coarsening then runs on the renumbered graph: node x of the
// caller's graph is node perm[x] there, and every result refers to the renumbered graph except
// the composed lift, which is read back in the caller's numbering.

#include "spc_scan.cuh"

namespace spc {

namespace {

constexpr int kShortRow = 32;    // rows ranked in shared memory; longer rows by a radix sort
constexpr int kReorderHops = 8;  // the cluster label's hops
constexpr int kReorderSub = 2;   // the sub-cluster label's hops

// one synchronous round of the labels: out[x] = min(in[x], min over the row of x of in[y]);
// the round that makes the sub-cluster label also copies it to `sub` (may be null).  A row is
// read in batches of kLabelBatch columns whose label gathers are all in flight together.
constexpr int kLabelBatch = 8;

__global__ void __launch_bounds__(kThreads)
k_label_round(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
              const int32_t* __restrict__ in, int32_t* __restrict__ out,
              int32_t* __restrict__ sub) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = in ? in[x] : (int32_t)x;  // the first label round starts from the ids
        const int64_t r1 = rowptr[x + 1];
        for (int64_t j0 = rowptr[x]; j0 < r1; j0 += kLabelBatch) {
            int32_t y[kLabelBatch];
#pragma unroll
            for (int t = 0; t < kLabelBatch; ++t) y[t] = j0 + t < r1 ? col[j0 + t] : -1;
#pragma unroll
            for (int t = 0; t < kLabelBatch; ++t) {
                if (y[t] < 0) continue;
                const int32_t l = in ? in[y[t]] : y[t];
                m = l < m ? l : m;
            }
        }
        out[x] = m;
        if (sub) sub[x] = m;
    }
}

// sort keys (L_8(x) << nb) | L_2(x), values the node ids: a stable sort gives (L_8, L_2, x)
__global__ void __launch_bounds__(kThreads)
k_label_keys(int64_t n, int nb, const int32_t* __restrict__ lab, const int32_t* __restrict__ sub,
             uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        key[x] = ((uint64_t)(uint32_t)lab[x] << nb) | (uint32_t)sub[x];
        val[x] = (uint32_t)x;
    }
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

// Renumbered rows of at most kShortRow entries, one warp per 32 consecutive new rows (whose
// entries form one contiguous run of the new CSR).  The warp copies each of its rows into
// shared memory (lanes along the row: the old row's columns mapped through perm, its weights,
// and the row's index within the tile), then every entry is ranked among its row's entries
// (at most kShortRow comparisons) and written at its place: the stores of a warp instruction
// land in the few rows that 32 consecutive entries span.  Rows longer than kShortRow are listed
// for the radix path; a tile whose rows exceed kPermStage entries is ranked the same way from
// global memory.
constexpr int kPermStage = 512;  // entries staged per warp
// warps per block: the stage of 8 warps of binary64 weights would pass 48 KB
template <class WT>
__host__ __device__ constexpr int perm_warps() { return sizeof(WT) == 8 ? 4 : 8; }

template <class WT>
__global__ void __launch_bounds__(perm_warps<WT>() * 32)
k_perm_short(int64_t n, const uint32_t* __restrict__ order, const int32_t* __restrict__ perm,
             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const WT* __restrict__ w, const int64_t* __restrict__ rowptr_new,
             int32_t* __restrict__ col_new, WT* __restrict__ w_new,
             int32_t* __restrict__ long_rows, int32_t* long_count) {
    spc::pdl_wait();
    constexpr int kPermWarps = perm_warps<WT>();
    __shared__ int32_t s_col[kPermWarps][kPermStage];
    __shared__ WT s_w[kPermWarps][kPermStage];
    __shared__ uint8_t s_row[kPermWarps][kPermStage];
    __shared__ int32_t s_off[kPermWarps][33];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t* const sc = s_col[wib];
    WT* const sw = s_w[wib];
    uint8_t* const sr = s_row[wib];
    int32_t* const so = s_off[wib];
    const int64_t nwarps = (int64_t)gridDim.x * kPermWarps;
    for (int64_t r0 = ((int64_t)blockIdx.x * kPermWarps + wib) * 32; r0 < n; r0 += nwarps * 32) {
        const int64_t r = r0 + lane;
        int64_t rs = 0;
        int d = 0;
        if (r < n) {
            const uint32_t x = order[r];
            rs = rowptr[x];
            d = (int)(rowptr[x + 1] - rs);
            if (d > kShortRow) {
                long_rows[atomicAdd(long_count, 1)] = (int32_t)r;
                d = 0;
            }
        }
        // offsets of the short rows within the tile's run of the new CSR (a long row's entries
        // are placed by the radix path; its slot here is empty)
        int o = d;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, o, k);
            if (lane >= k) o += t;
        }
        const int total = __shfl_sync(0xffffffffu, o, 31);
        o -= d;
        if (total <= kPermStage) {
            so[lane] = o;
            if (lane == 31) so[32] = total;
            // the rows' old columns and weights, every copy in flight together
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {  // row k of the tile, lanes along it
                const int dk = __shfl_sync(0xffffffffu, d, k);
                const int ok = __shfl_sync(0xffffffffu, o, k);
                const int64_t rk = __shfl_sync(0xffffffffu, rs, k);
                if (lane < dk) {
                    cp_async_4(sc + ok + lane, col + rk + lane);
                    cp_async_elem(sw + ok + lane, w + rk + lane);
                    sr[ok + lane] = (uint8_t)k;
                }
            }
            cp_async_wait_all();
            __syncwarp();
            // the new columns: the gathers of perm, four per lane in flight
            for (int i0 = 0; i0 < total; i0 += 128) {
                int32_t y[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int i = i0 + 32 * t + lane;
                    y[t] = i < total ? perm[sc[i]] : 0;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int i = i0 + 32 * t + lane;
                    if (i < total) sc[i] = y[t];
                }
            }
            __syncwarp();
            for (int i = lane; i < total; i += 32) {
                const int k = sr[i];
                const int lo = so[k], hi = so[k + 1];
                const int32_t ci = sc[i];
                int rank = 0;
                for (int j = lo; j < hi; ++j) rank += sc[j] < ci ? 1 : 0;
                const int64_t dest = rowptr_new[r0 + k] + rank;
                col_new[dest] = ci;
                w_new[dest] = sw[i];
            }
        } else if (d > 0) {  // a tile too large for the stage: each lane ranks its own row
            const int64_t base = rowptr_new[r];
            for (int k = 0; k < d; ++k) {
                const int32_t ck = perm[col[rs + k]];
                int rank = 0;
                for (int j = 0; j < d; ++j) rank += perm[col[rs + j]] < ck ? 1 : 0;
                col_new[base + rank] = ck;
                w_new[base + rank] = w[rs + k];
            }
        }
        __syncwarp();  // the next tile overwrites the stage
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
    SPC_TRY(ensure(ctx, W.ro_key, N * 8));
    SPC_TRY(ensure(ctx, W.ro_val, N * 4));
    SPC_TRY(ensure(ctx, W.ro_key2, N * 8));
    SPC_TRY(ensure(ctx, W.ro_val2, N * 4));
    SPC_TRY(ensure(ctx, W.ro_perm, N * 4));
    SPC_TRY(ensure(ctx, W.ro_deg, N * 4));
    SPC_TRY(ensure(ctx, W.ro_rowptr, (N + 1) * 8));
    SPC_TRY(ensure(ctx, W.ro_col, (size_t)(nnz + 1) * 4));
    SPC_TRY(ensure(ctx, W.ro_w, (size_t)(nnz + 1) * sizeof(WT)));
    out = g;
    if (n == 0) return SPC_OK;
    // ---- the labels: kReorderHops rounds, ping-pong between two arrays ------------------------
    int32_t* lab[2] = {W.ro_dist.as<int32_t>(), W.ro_deg.as<int32_t>()};
    int32_t* sub = W.ro_perm.as<int32_t>();  // the 2-hop label (perm is written after the sort)
    // the CSR's row pointers and columns read once, every neighbour's label gathered, every
    // label written once
    for (int k = 1; k <= kReorderHops; ++k) {
        note_bytes(ctx, 8.0 * (n + 1) + 8.0 * nnz + 4.0 * n);
        SPC_LAUNCH(ctx, k_label_round, gn, kThreads, 0, n, g.rowptr, g.col,
                   k == 1 ? nullptr : lab[(k - 1) & 1], lab[k & 1],
                   k == kReorderSub ? sub : nullptr);
    }
    int nb = 1;
    while ((1ll << nb) < n) ++nb;
    uint64_t* key = W.ro_key.as<uint64_t>();
    uint32_t* order = W.ro_val.as<uint32_t>();
    SPC_LAUNCH(ctx, k_label_keys, gn, kThreads, 0, n, nb, lab[kReorderHops & 1], sub, key, order);
    SPC_TRY(radix_sort_u64(ctx, key, order, W.ro_key2.as<uint64_t>(), W.ro_val2.as<uint32_t>(),
                           n, 2 * nb));
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
    SPC_LAUNCH(ctx, k_perm_short<WT>, grid_for((n + 31) / 32, perm_warps<WT>(), maxb),
               perm_warps<WT>() * 32, 0, n, order, perm, g.rowptr, g.col,
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
