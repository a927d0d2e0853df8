// S0-S3: input checks, weighted degrees, normalised rows and the per-edge score.
//
// Score (Theorem 1; Algorithm 1 fitness loop; Section 2 "one norm per edge, O(d_u + d_v)"):
//   f(a, b) = || w_a / d_a - w_b / d_b ||_1 = sum over x in N(a) u N(b) of |p_ax - p_bx|,
// the union taken in ascending x and containing a and b themselves (p_aa = p_bb = 0).
// Every sum here runs sequentially in ascending column order with IEEE round-to-nearest adds
// (__dadd_rn / __fadd_rn, no FMA), and p = w / d is one IEEE division per stored entry, so
// the results are the same bits on every run and every schedule.
#include "spc_internal.cuh"

namespace spc {

template <class WT> struct Tr;
template <> struct Tr<int32_t> {
    using Acc = long long;
    using P = double;
    using Key = unsigned long long;
    __device__ static Acc add(Acc a, int32_t w) { return a + (Acc)w; }
    __device__ static P div(int32_t w, Acc d) { return __ddiv_rn((double)w, (double)d); }
    __device__ static bool ok(int32_t w) { return w > 0; }
    __device__ static uint64_t bits(int32_t w) { return (uint32_t)w; }
};
template <> struct Tr<float> {
    using Acc = float;
    using P = float;
    using Key = unsigned int;
    __device__ static Acc add(Acc a, float w) { return __fadd_rn(a, w); }
    __device__ static P div(float w, Acc d) { return __fdiv_rn(w, d); }
    __device__ static bool ok(float w) { return w > 0.f && !isinf(w); }
    __device__ static uint64_t bits(float w) { return __float_as_uint(w); }
};
template <> struct Tr<double> {
    using Acc = double;
    using P = double;
    using Key = unsigned long long;
    __device__ static Acc add(Acc a, double w) { return __dadd_rn(a, w); }
    __device__ static P div(double w, Acc d) { return __ddiv_rn(w, d); }
    __device__ static bool ok(double w) { return w > 0.0 && !isinf(w); }
    __device__ static uint64_t bits(double w) { return (uint64_t)__double_as_longlong(w); }
};

__device__ __forceinline__ double p_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float p_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double p_absdiff(double a, double b) { return fabs(__dsub_rn(a, b)); }
__device__ __forceinline__ float p_absdiff(float a, float b) { return fabsf(__fsub_rn(a, b)); }
__device__ __forceinline__ unsigned long long key_bits(double s) {
    return (unsigned long long)__double_as_longlong(s);
}
__device__ __forceinline__ unsigned int key_bits(float s) { return __float_as_uint(s); }

// S0 + S1: one thread per row.  Checks the row (when `validate`), sums the weighted degree in
// ascending column order, counts the entries below the diagonal and above it.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_rows_degree(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
              const int32_t* __restrict__ col, const WT* __restrict__ w, int validate,
              typename Tr<WT>::Acc* __restrict__ deg, int32_t* __restrict__ up_cnt,
              int32_t* __restrict__ nlow_out, uint32_t* __restrict__ status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (validate && blockIdx.x == 0 && threadIdx.x == 0) {
        if (rowptr[0] != 0 || rowptr[n] != nnz) atomicOr(status, DEV_UNSORTED);
    }
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        uint32_t bits = 0;
        if (r0 < 0 || r1 < r0 || r1 > nnz) {
            atomicOr(status, DEV_UNSORTED);
            deg[x] = 0;
            up_cnt[x] = 0;
            nlow_out[x] = 0;
            continue;
        }
        typename Tr<WT>::Acc acc = 0;
        int32_t nlow = 0;
        int64_t prev = -1;
        for (int64_t j = r0; j < r1; ++j) {
            const int32_t y = col[j];
            const WT wj = w[j];
            if (validate) {
                if (y < 0 || (int64_t)y >= n || (int64_t)y <= prev) bits |= DEV_UNSORTED;
                if ((int64_t)y == x) bits |= DEV_SELF_LOOP;
                if (!Tr<WT>::ok(wj)) bits |= DEV_BAD_WEIGHT;
                prev = y;
            }
            nlow += ((int64_t)y < x) ? 1 : 0;
            acc = Tr<WT>::add(acc, wj);
        }
        deg[x] = acc;
        nlow_out[x] = nlow;
        up_cnt[x] = (int32_t)(r1 - r0) - nlow;
        if (bits) atomicOr(status, bits);
    }
}

// S2 (+ the edge list): one thread per row.  p[j] = w[j] / d[x]; for the entries above the
// diagonal writes the undirected edge (x, y) at its edge id; when `validate`, looks up the
// mirror entry (y, x) by binary search and compares the weight bits.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_rows_edges(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const WT* __restrict__ w, int validate, const typename Tr<WT>::Acc* __restrict__ deg,
             const int32_t* __restrict__ nlow, const int32_t* __restrict__ up_ptr,
             typename Tr<WT>::P* __restrict__ p, int32_t* __restrict__ eu,
             int32_t* __restrict__ ev, WT* __restrict__ w_und, uint32_t* __restrict__ status) {
    if (*status) return;  // invalid input: nothing below may index with it
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        const typename Tr<WT>::Acc d = deg[x];
        const int64_t ubase = (int64_t)up_ptr[x] - (r0 + nlow[x]);
        uint32_t bits = 0;
        for (int64_t j = r0; j < r1; ++j) {
            const int32_t y = col[j];
            const WT wj = w[j];
            p[j] = Tr<WT>::div(wj, d);
            if (validate) {
                int64_t lo = rowptr[y], hi = rowptr[y + 1];
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if ((int64_t)col[mid] < x) lo = mid + 1; else hi = mid;
                }
                if (lo >= rowptr[y + 1] || (int64_t)col[lo] != x ||
                    Tr<WT>::bits(w[lo]) != Tr<WT>::bits(wj))
                    bits |= DEV_NOT_SYMMETRIC;
            }
            if ((int64_t)y > x) {
                const int64_t e = ubase + j;
                eu[e] = (int32_t)x;
                ev[e] = y;
                w_und[e] = wj;
            }
        }
        if (bits) atomicOr(status, bits);
    }
}

// S3, edge-tile schedule: one thread per undirected edge; consecutive threads take consecutive
// edge ids, which mostly share row a (cached), and walk rows a and b in step.
template <class PT, class KT>
__global__ void __launch_bounds__(kThreads)
k_score_edges(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
              const PT* __restrict__ p, KT* __restrict__ score, const uint32_t* status) {
    if (*status) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = eu[e], b = ev[e];
        int64_t i = rowptr[a];
        const int64_t ie = rowptr[a + 1];
        int64_t j = rowptr[b];
        const int64_t je = rowptr[b + 1];
        PT s = PT(0);
        while (i < ie && j < je) {
            const int32_t ca = col[i], cb = col[j];
            PT t;
            if (ca < cb) {
                t = p[i++];
            } else if (cb < ca) {
                t = p[j++];
            } else {
                t = p_absdiff(p[i], p[j]);
                ++i; ++j;
            }
            s = p_add(s, t);
        }
        while (i < ie) s = p_add(s, p[i++]);
        while (j < je) s = p_add(s, p[j++]);
        score[e] = key_bits(s);
    }
}

// S3, warp-per-row schedule: a warp owns row a, keeps its columns and p values in shared
// memory (up to kRowCache entries) and each lane scores one edge (a, b), b > a, walking row b
// from global memory.  Suits rows with many upper neighbours (hubs); same sums, same order.
constexpr int kRowCache = 512;

template <class PT, class KT>
__global__ void __launch_bounds__(kThreads)
k_score_warp_row(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const PT* __restrict__ p, const int32_t* __restrict__ up_ptr,
                 const int32_t* __restrict__ nlow, KT* __restrict__ score,
                 const uint32_t* status) {
    if (*status) return;
    __shared__ int32_t s_col[kThreads / 32][kRowCache];
    __shared__ PT s_p[kThreads / 32][kRowCache];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; a < n; a += warps) {
        const int64_t r0 = rowptr[a], r1 = rowptr[a + 1];
        const int64_t da = r1 - r0;
        const int64_t ufirst = r0 + nlow[a];
        const bool cached = da <= kRowCache;
        if (cached) {
            for (int64_t k = lane; k < da; k += 32) {
                s_col[wib][k] = col[r0 + k];
                s_p[wib][k] = p[r0 + k];
            }
        }
        __syncwarp();
        const int64_t e0 = up_ptr[a];
        for (int64_t jb = ufirst + lane; jb < r1; jb += 32) {
            const int32_t b = col[jb];
            int64_t i = 0;
            int64_t j = rowptr[b];
            const int64_t je = rowptr[b + 1];
            PT s = PT(0);
            while (i < da && j < je) {
                const int32_t ca = cached ? s_col[wib][i] : col[r0 + i];
                const int32_t cb = col[j];
                PT t;
                if (ca < cb) {
                    t = cached ? s_p[wib][i] : p[r0 + i];
                    ++i;
                } else if (cb < ca) {
                    t = p[j++];
                } else {
                    t = p_absdiff(cached ? s_p[wib][i] : p[r0 + i], p[j]);
                    ++i; ++j;
                }
                s = p_add(s, t);
            }
            while (i < da) {
                s = p_add(s, cached ? s_p[wib][i] : p[r0 + i]);
                ++i;
            }
            while (j < je) s = p_add(s, p[j++]);
            score[e0 + (jb - ufirst)] = key_bits(s);
        }
        __syncwarp();
    }
}

template <class WT>
static spc_status score_typed(spc_context* ctx, GraphView& g, bool validate, void* score,
                              int schedule) {
    using Acc = typename Tr<WT>::Acc;
    using P = typename Tr<WT>::P;
    using Key = typename Tr<WT>::Key;
    Work& W = ctx->work;
    const int64_t n = g.n;
    const int64_t nnz = g.nnz;
    const int maxb = ctx->num_sms * 8;
    uint32_t* status = ctx->d_status;
    const int gb = grid_for(n, kThreads, maxb);
    SPC_LAUNCH(ctx, k_rows_degree<WT>, gb, kThreads, 0, n, nnz, g.rowptr, g.col,
               static_cast<const WT*>(g.w), validate ? 1 : 0, W.deg.as<Acc>(),
               W.up_cnt.as<int32_t>(), W.first_up.as<int32_t>(), status);
    SPC_TRY(scan_i32(ctx, W.up_cnt.as<int32_t>(), W.up_ptr.as<int32_t>(), n));
    // one readback: the status word and the edge count
    SPC_CUDA(cudaMemcpyAsync(ctx->h_scalars, W.up_ptr.as<int32_t>() + n, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, ctx->stream));
    SPC_CUDA(cudaMemcpyAsync(ctx->h_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             ctx->stream));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (*ctx->h_status) return status_from_bits(*ctx->h_status);
    const int64_t m = *reinterpret_cast<int32_t*>(ctx->h_scalars);
    if (2 * m != nnz) return SPC_ERR_NOT_SYMMETRIC;
    g.m = m;
    SPC_LAUNCH(ctx, k_rows_edges<WT>, gb, kThreads, 0, n, g.rowptr, g.col,
               static_cast<const WT*>(g.w), validate ? 1 : 0, W.deg.as<Acc>(),
               W.first_up.as<int32_t>(), W.up_ptr.as<int32_t>(), W.p.as<P>(),
               W.eu.as<int32_t>(), W.ev.as<int32_t>(), W.w_und.as<WT>(), status);
    if (validate) SPC_TRY(sync_status(ctx));  // no later kernel runs on an asymmetric input
    if (score == nullptr || m == 0) return SPC_OK;
    if (schedule == 2) {
        const int warps_per_block = kThreads / 32;
        const int gw = grid_for(n, warps_per_block, maxb);
        SPC_LAUNCH(ctx, (k_score_warp_row<P, Key>), gw, kThreads, 0, n, g.rowptr, g.col,
                   W.p.as<P>(), W.up_ptr.as<int32_t>(), W.first_up.as<int32_t>(),
                   static_cast<Key*>(score), status);
    } else {
        SPC_LAUNCH(ctx, (k_score_edges<P, Key>), grid_for(m, kThreads, maxb), kThreads, 0, m,
                   W.eu.as<int32_t>(), W.ev.as<int32_t>(), g.rowptr, g.col, W.p.as<P>(),
                   static_cast<Key*>(score), status);
    }
    return SPC_OK;
}

spc_status run_score(spc_context* ctx, GraphView& g, bool validate, void* score, int schedule) {
    switch (g.wtype) {
        case SPC_I32: return score_typed<int32_t>(ctx, g, validate, score, schedule);
        case SPC_F32: return score_typed<float>(ctx, g, validate, score, schedule);
        case SPC_F64: return score_typed<double>(ctx, g, validate, score, schedule);
    }
    return SPC_ERR_INVALID_ARG;
}

}  // namespace spc
