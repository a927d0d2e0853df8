// S0-S3: input checks, weighted degrees, normalised rows and the per-edge score.
//
// Score (Theorem 1; the fitness loop of Algorithm 1, one norm per edge, Section 2):
//   f(a, b) = || w_a / d_a - w_b / d_b ||_1 = sum over x in N(a) u N(b) of |p_ax - p_bx|,
// the union taken in ascending x and containing a and b themselves.  A caller's graph has no
// diagonal (p_aa = p_bb = 0).  Under the self-mass reading of the multilevel driver a coarse
// graph holds the diagonal entry (x, x) = 2 mass(x) of every super-node with internal weight
// (the merged node of the proof of Theorem 2); it is an ordinary stored entry of row x, so the
// degree and the union walks include it with no special case.  `nlow` counts the entries of a
// row at or below its diagonal: the upper (edge) entries start after them.
// Every sum here runs sequentially in ascending column order with IEEE round-to-nearest adds
// (__dadd_rn / __fadd_rn, no FMA), and p = w / d is one IEEE division per stored entry, so
// the results are the same bits on every run and every schedule.
#include <algorithm>
#include <atomic>
#include <memory>

#include "spc_seqsum.cuh"

namespace spc {

// w / d for every entry of a row that shares the degree d, with y = RN(1/d) computed once per row:
// Markstein's theorem (IBM J. Res. Dev. 34(1), 1990; also Muller et al., Handbook of
// Floating-Point Arithmetic, ch. 4): if y is within half an ulp of 1/d and q0 within one ulp of
// w/d, then r = w - d*q0 is exact (one FMA) and RN(q0 + r*y) = RN(w/d).  q0 = RN(w*y) is within
// one ulp.  With w and d in [2^-400, 2^400) every intermediate is a normal number (q0 within
// (2^-800, 2^800), the residual a multiple of about 2^-505 or 0); outside that range the IEEE
// division is used directly.  The range tests read the exponent fields with integer
// instructions: GB300's FP64 pipe is narrow, and the divisions of a level are bound by it.
__device__ __forceinline__ bool mid_range(double v) {
    const unsigned e = ((unsigned)__double2hiint(v) >> 20) & 0x7ffu;
    return e - (1023u - 400u) < 800u;
}

__device__ __forceinline__ double div_row(double w, double d, double y, bool d_mid) {
    if (!(d_mid && mid_range(w))) return __ddiv_rn(w, d);
    const double q0 = __dmul_rn(w, y);
    const double r = __fma_rn(-d, q0, w);
    return __fma_rn(r, y, q0);
}

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
    // finite and > 0, tested on the bits (no floating-point compare)
    __device__ static bool ok(float w) {
        const int b = __float_as_int(w);
        return b > 0 && b < 0x7f800000;
    }
    __device__ static uint64_t bits(float w) { return __float_as_uint(w); }
};
template <> struct Tr<double> {
    using Acc = double;
    using P = double;
    using Key = unsigned long long;
    __device__ static Acc add(Acc a, double w) { return __dadd_rn(a, w); }
    __device__ static P div(double w, Acc d) { return __ddiv_rn(w, d); }
    // finite and > 0, tested on the bits (no FP64 compare)
    __device__ static bool ok(double w) {
        const long long b = __double_as_longlong(w);
        return b > 0 && b < 0x7ff0000000000000ll;
    }
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
// ascending column order, counts the entries at or below the diagonal and above it.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_rows_degree(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
              const int32_t* __restrict__ col, const WT* __restrict__ w, int validate,
              typename Tr<WT>::Acc* __restrict__ deg, int32_t* __restrict__ up_cnt,
              int32_t* __restrict__ nlow_out, int32_t* __restrict__ long_rows,
              int32_t* __restrict__ long_count, uint32_t* __restrict__ status) {
    spc::pdl_wait();
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
        if (r1 - r0 > kLongRow) {  // long rows: k_long_rows_meta and the per-binade tables
            long_rows[atomicAdd(long_count, 1)] = (int32_t)x;
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
            nlow += ((int64_t)y <= x) ? 1 : 0;
            acc = Tr<WT>::add(acc, wj);
        }
        deg[x] = acc;
        nlow_out[x] = nlow;
        up_cnt[x] = (int32_t)(r1 - r0) - nlow;
        if (bits) atomicOr(status, bits);
    }
}

// S0 for rows longer than kLongRow, part 1: one warp per row records the row as a sequence
// (base, length) for the exact degree sum (the per-binade tables of spc_seqtab.cu evaluate
// it) and counts its entries at or below the diagonal by a 32-way search for x among the
// sorted columns.  On an unsorted row the count is wrong but in range; part 2 reports the row.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_long_rows_meta(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const int32_t* __restrict__ long_rows, const int32_t* __restrict__ long_count,
                 typename Tr<WT>::Acc* __restrict__ deg, int32_t* __restrict__ up_cnt,
                 int32_t* __restrict__ nlow_out, int64_t* __restrict__ lr_base,
                 int64_t* __restrict__ lr_len, int64_t* __restrict__ lr_idx,
                 int32_t* __restrict__ heavy_count) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *heavy_count = 0;  // for k_score_hub
    const int32_t cnt = *long_count;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < cnt;
         i += warps) {
        const int64_t x = long_rows[i];
        const int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        // first position in [r0, r1] whose column is > x
        int64_t lo = r0, hi = r1;  // answer in [lo, hi]
        while (hi > lo) {
            const int64_t step = (hi - lo + 31) / 32;
            const int64_t probe = lo + (int64_t)lane * step;  // lane 0 probes lo itself
            const bool below = probe < hi && (int64_t)col[probe] <= x;
            const int nb = __popc(__ballot_sync(0xffffffffu, below));
            // columns up to x form a prefix of the probes
            if (nb == 0) { hi = lo; break; }
            lo = lo + (int64_t)(nb - 1) * step + 1;
            const int64_t cap = lo - 1 + step;
            hi = cap < hi ? cap : hi;
        }
        if (lane == 0) {
            const int32_t nl = (int32_t)(lo - r0);
            nlow_out[x] = nl;
            up_cnt[x] = (int32_t)(r1 - r0) - nl;
            lr_base[i] = r0;
            lr_len[i] = r1 - r0;
            lr_idx[i] = x;
            if constexpr (std::is_same<WT, int32_t>::value) deg[x] = 0;
        }
    }
}

// S0 (+ S1 for integer weights) for rows longer than kLongRow, part 2: one thread per entry,
// flat over all long rows (lr_eoff: exclusive prefix of the row lengths).  Checks every entry
// and, for integer weights, adds the row's weights into its degree (exact in any order).
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_long_rows_flat(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const WT* __restrict__ w, int validate, const int32_t* __restrict__ long_rows,
                 const int32_t* __restrict__ long_count, const int64_t* __restrict__ lr_eoff,
                 typename Tr<WT>::Acc* __restrict__ deg, uint32_t* __restrict__ status) {
    spc::pdl_wait();
    constexpr bool kInt = std::is_same<WT, int32_t>::value;
    const int32_t cnt = *long_count;
    const int64_t total = lr_eoff[cnt];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f0 = (int64_t)blockIdx.x * blockDim.x; f0 < total; f0 += stride) {
        const int64_t f = f0 + threadIdx.x;
        const bool act = f < total;
        int32_t row = 0;
        long long wsum = 0;
        if (act) {
            int32_t lo = 0, hi = cnt - 1;
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (lr_eoff[mid] <= f) lo = mid; else hi = mid - 1;
            }
            row = lo;
            const int64_t x = long_rows[lo];
            const int64_t r0 = rowptr[x];
            const int64_t j = r0 + (f - lr_eoff[lo]);
            const int32_t y = col[j];
            const WT wj = w[j];
            if (validate) {
                uint32_t bits = 0;
                if (y < 0 || (int64_t)y >= n || (j > r0 && col[j - 1] >= y)) bits |= DEV_UNSORTED;
                if ((int64_t)y == x) bits |= DEV_SELF_LOOP;
                if (!Tr<WT>::ok(wj)) bits |= DEV_BAD_WEIGHT;
                if (bits) atomicOr(status, bits);
            }
            if constexpr (kInt) wsum = (long long)wj;
        }
        if constexpr (kInt) {
            // lanes of one row add up first, one atomic per row and warp
            const unsigned peers = __match_any_sync(0xffffffffu, act ? row : -1);
            const int lane = threadIdx.x & 31;
            long long part = 0;
            for (unsigned m = peers; m; m &= m - 1)
                part += __shfl_sync(peers, wsum, __ffs(m) - 1);
            if (act && lane == __ffs(peers) - 1)
                atomicAdd(reinterpret_cast<unsigned long long*>(deg + long_rows[row]),
                          (unsigned long long)part);
        }
    }
}

// S2 + edge list for rows longer than kLongRow: one thread per entry, flat over all long rows.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_long_rows_edges(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const WT* __restrict__ w, int validate,
                  const typename Tr<WT>::Acc* __restrict__ deg, const int32_t* __restrict__ nlow,
                  const int32_t* __restrict__ up_ptr, const int32_t* __restrict__ long_rows,
                  const int32_t* __restrict__ long_count, const int64_t* __restrict__ lr_eoff,
                  typename Tr<WT>::P* __restrict__ p, int32_t* __restrict__ eu,
                  int32_t* __restrict__ ev, WT* __restrict__ w_und, uint32_t* __restrict__ status) {
    spc::pdl_wait();
    if (*status) return;
    const int32_t cnt = *long_count;
    const int64_t total = lr_eoff[cnt];
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (lr_eoff[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int64_t x = long_rows[lo];
        const int64_t r0 = rowptr[x];
        const int64_t j = r0 + (f - lr_eoff[lo]);
        const int32_t y = col[j];
        const WT wj = w[j];
        p[j] = Tr<WT>::div(wj, deg[x]);
        if (validate) {
            int64_t l2 = rowptr[y], h2 = rowptr[y + 1];
            while (l2 < h2) {
                int64_t mid = (l2 + h2) >> 1;
                if ((int64_t)col[mid] < x) l2 = mid + 1; else h2 = mid;
            }
            if (l2 >= rowptr[y + 1] || (int64_t)col[l2] != x ||
                Tr<WT>::bits(w[l2]) != Tr<WT>::bits(wj))
                atomicOr(status, DEV_NOT_SYMMETRIC);
        }
        if ((int64_t)y > x) {
            const int64_t e = (int64_t)up_ptr[x] + (j - (r0 + nlow[x]));
            eu[e] = (int32_t)x;
            ev[e] = y;
            w_und[e] = wj;
        }
    }
}

// S2 (+ the edge list): one thread per row.  p[j] = w[j] / d[x]; for the entries above the
// diagonal writes the undirected edge (x, y) at its edge id; when `validate` (set only when no
// score kernel follows: those check every upper entry's mirror on their walks), looks up the
// mirror entry (y, x) by binary search and compares the weight bits.
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_rows_edges(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const WT* __restrict__ w, int validate, const typename Tr<WT>::Acc* __restrict__ deg,
             const int32_t* __restrict__ nlow, const int32_t* __restrict__ up_ptr,
             typename Tr<WT>::P* __restrict__ p, int32_t* __restrict__ eu,
             int32_t* __restrict__ ev, WT* __restrict__ w_und, uint32_t* __restrict__ status) {
    spc::pdl_wait();
    if (*status) return;  // invalid input: nothing below may index with it
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        if (r1 - r0 > kLongRow) continue;  // k_long_rows_edges
        const typename Tr<WT>::Acc d = deg[x];
        const int64_t ubase = (int64_t)up_ptr[x] - (r0 + nlow[x]);
        // binary64 rows: one correctly rounded reciprocal per row, Markstein per entry
        double dd = 0.0, rcp = 0.0;
        bool d_mid = false;
        if constexpr (!std::is_same<WT, float>::value) {
            dd = (double)d;
            d_mid = mid_range(dd);
            rcp = d_mid ? __drcp_rn(dd) : 0.0;
        }
        uint32_t bits = 0;
        for (int64_t j = r0; j < r1; ++j) {
            const int32_t y = col[j];
            const WT wj = w[j];
            if constexpr (std::is_same<WT, float>::value) p[j] = Tr<WT>::div(wj, d);
            else p[j] = div_row((double)wj, dd, rcp, d_mid);
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

// Symmetry fingerprint (S0) of a binary32 graph: every stored entry (x, y, w) off the diagonal
// adds +H(min, max, bits of w) when x < y and -H(...) when x > y, modulo 2^64.  A symmetric
// graph pairs every upper entry with a lower one of the same (min, max, w), so the sum is 0
// whatever the order of the additions.  An asymmetric graph leaves a nonempty set of
// unpaired terms, whose signed sum is 0 only by a coincidence of the 64-bit keyed hash (about
// 2^-64 per input; the key is drawn at context creation).  H chains two rounds of the
// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014), keyed by k0 and k1.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sym_term(int64_t x, int32_t y, uint32_t wbits, uint64_t k0,
                                             uint64_t k1) {
    const uint64_t lo = (uint64_t)((int64_t)y < x ? y : x), hi = (uint64_t)((int64_t)y < x ? x : y);
    const uint64_t h = mix64(mix64(k0 ^ ((lo << 32) | hi)) ^ (wbits + k1));
    return (int64_t)y > x ? h : (uint64_t)0 - h;
}

// S2 (+ the edge list) for binary32 weights, flat over the stored entries: each block takes
// kFlatTile consecutive entries and marks the row of each in shared memory (tile_rows), so the
// columns, weights and p values of a warp are consecutive (the row-per-thread kernel reads 32
// rows at once).  p = w / d is one IEEE division per entry, exactly as k_rows_edges computes
// it.  `p` (may be null) receives p alone, `pk` the (column, p) pair of every entry.  Rows
// longer than kLongRow are left to k_long_rows_edges.  With `sym` (input validation), every
// entry of every row, long ones included, also adds its symmetry fingerprint term into *sym.
constexpr int64_t kFlatTile = 2048;

__global__ void __launch_bounds__(kThreads)
k_rows_edges_flat(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                  const int32_t* __restrict__ col, const float* __restrict__ w,
                  const float* __restrict__ deg, const int32_t* __restrict__ nlow,
                  const int32_t* __restrict__ up_ptr, float* __restrict__ p,
                  uint2* __restrict__ pk, int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                  float* __restrict__ w_und, unsigned long long* sym, uint64_t k0, uint64_t k1,
                  const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;  // invalid input: nothing below may index with it
    __shared__ int64_t s_rows[2];
    __shared__ int32_t s_row[kFlatTile];  // row of each entry of the tile minus the first row
    uint64_t fp = 0;                      // this thread's fingerprint terms
    for (int64_t base = (int64_t)blockIdx.x * kFlatTile; base < nnz;
         base += (int64_t)gridDim.x * kFlatTile) {
        const int64_t end = base + kFlatTile < nnz ? base + kFlatTile : nnz;
        const int64_t r_lo = tile_rows(rowptr, n, base, end, kLongRow, s_row, s_rows);
        for (int64_t j = base + threadIdx.x; j < end; j += blockDim.x) {
            const int32_t rel = s_row[j - base];
            const int64_t x = r_lo + (rel >= 0 ? rel : -2 - rel);
            const int32_t y = col[j];
            const float wj = w[j];
            if (sym && (int64_t)y != x) fp += sym_term(x, y, __float_as_uint(wj), k0, k1);
            if (rel < 0) continue;  // long row: k_long_rows_edges
            const float pj = __fdiv_rn(wj, deg[x]);
            if (p) p[j] = pj;
            // row x's pairs at pk[rowptr[x] + x ..], then its end marker
            pk[j + x] = make_uint2((uint32_t)y, __float_as_uint(pj));
            if (j + 1 == rowptr[x + 1]) pk[j + x + 1] = make_uint2(0x7fffffffu, 0u);
            if ((int64_t)y > x) {
                const int64_t e = (int64_t)up_ptr[x] + (j - (rowptr[x] + nlow[x]));
                eu[e] = (int32_t)x;
                ev[e] = y;
                w_und[e] = wj;
            }
        }
        __syncthreads();
    }
    if (sym) {
        for (int o = 16; o > 0; o >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, o);
        if ((threadIdx.x & 31) == 0 && fp) atomicAdd(sym, (unsigned long long)fp);
    }
}

// the verdict of the symmetry fingerprint: a nonzero sum is an asymmetric input (unless a row
// check already failed, in which case the flat kernel did not run and that error stands)
__global__ void k_sym_check(const unsigned long long* __restrict__ sym, uint32_t* status) {
    spc::pdl_wait();
    if (threadIdx.x == 0 && *status == 0u && *sym != 0ull) atomicOr(status, DEV_NOT_SYMMETRIC);
}

// Arithmetic count of a score launch, for the roofline: ops[0] += additions into the running
// sums (one per union coordinate), ops[1] += subtractions (one per coordinate present in both
// rows).  One atomic per warp; every lane of the block reaches it.
__device__ __forceinline__ void count_ops(unsigned long long* ops, uint32_t n_add,
                                          uint32_t n_sub) {
    if (!ops) return;
    const uint32_t a = __reduce_add_sync(0xffffffffu, n_add);
    const uint32_t b = __reduce_add_sync(0xffffffffu, n_sub);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(ops, (unsigned long long)a);
        atomicAdd(ops + 1, (unsigned long long)b);
    }
}

// raw bits of entry j of a weight array of wsize-byte elements (int32, binary32 or binary64)
__device__ __forceinline__ uint64_t weight_bits(const void* w, int wsize, int64_t j) {
    return wsize == 8 ? static_cast<const unsigned long long*>(w)[j]
                      : (uint64_t)static_cast<const unsigned int*>(w)[j];
}

// true if row [j0, j1) (sorted) holds column a with weight bits wb: the mirror of entry (a, .)
__device__ __forceinline__ bool has_mirror(const int32_t* __restrict__ col, const void* w,
                                           int wsize, int64_t j0, int64_t j1, int64_t a,
                                           uint64_t wb) {
    int64_t lo = j0, hi = j1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)col[mid] < a) lo = mid + 1; else hi = mid;
    }
    return lo < j1 && (int64_t)col[lo] == a && weight_bits(w, wsize, lo) == wb;
}

// S3, edge-tile schedule: one thread per undirected edge; consecutive threads take consecutive
// edge ids, which mostly share row a (cached), and walk rows a and b in step.
template <class PT, class KT, int K>
__global__ void __launch_bounds__(kThreads)
k_score_edges(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
              const PT* __restrict__ p, KT* __restrict__ score, const void* __restrict__ w,
              const void* __restrict__ w_und, int wsize, int validate, uint32_t* status,
              unsigned long long* __restrict__ ops) {
    spc::pdl_wait();
    if (*status) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t n_add = 0, n_sub = 0;  // union coordinates, coordinates in both rows
    bool asym = false;
    constexpr int32_t kEnd = 0x7fffffff;
    // K edges per thread walked together: K independent addition chains hide the latency of
    // the binary64 additions and of the row loads; each edge keeps its own order
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < m;
         e0 += (int64_t)K * stride) {
        int64_t e[K], i[K], ie[K], j[K], je[K];
        int32_t a[K], ca[K], cb[K];
        PT s[K];
        bool mirror[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            e[q] = e0 + (int64_t)q * stride;
            s[q] = PT(0);
            mirror[q] = false;
            ca[q] = kEnd;
            cb[q] = kEnd;
            i[q] = ie[q] = j[q] = je[q] = 0;
            a[q] = 0;
            if (e[q] >= m) {
                e[q] = -1;
                continue;
            }
            a[q] = eu[e[q]];
            const int32_t b = ev[e[q]];
            i[q] = rowptr[a[q]];
            ie[q] = rowptr[a[q] + 1];
            j[q] = rowptr[b];
            je[q] = rowptr[b + 1];
            if (ie[q] - i[q] > kLongRow || je[q] - j[q] > kLongRow) {  // hub edge: k_score_hub
                // a long row a has its mirrors checked with the long rows; a long row b only
                // holds the mirror of this entry, so it is looked up here
                if (validate && ie[q] - i[q] <= kLongRow)
                    asym = asym || !has_mirror(col, w, wsize, j[q], je[q], a[q],
                                               weight_bits(w_und, wsize, e[q]));
                e[q] = -1;
                continue;
            }
            ca[q] = i[q] < ie[q] ? col[i[q]] : kEnd;
            cb[q] = j[q] < je[q] ? col[j[q]] : kEnd;
        }
        // one uniform step per coordinate of each union: t = |pa - pb| with the missing side
        // read as 0 (exact: |x - 0| = x), so every live walk issues the same two FP operations.
        // S0's symmetry check rides on the walk: coordinate a of row b is the mirror entry of
        // (a, b), and its weight must have the same bits.
        for (;;) {
            bool any = false;
#pragma unroll
            for (int q = 0; q < K; ++q) {
                if (ca[q] == kEnd && cb[q] == kEnd) continue;
                any = true;
                const bool ta = ca[q] <= cb[q], tb = cb[q] <= ca[q];
                if (validate && tb && cb[q] == a[q])
                    mirror[q] = weight_bits(w, wsize, j[q]) == weight_bits(w_und, wsize, e[q]);
                const PT pa = ta ? p[i[q]] : PT(0);
                const PT pb = tb ? p[j[q]] : PT(0);
                s[q] = p_add(s[q], p_absdiff(pa, pb));
                ++n_add;
                n_sub += (ta && tb) ? 1u : 0u;
                if (ta) { ++i[q]; ca[q] = i[q] < ie[q] ? col[i[q]] : kEnd; }
                if (tb) { ++j[q]; cb[q] = j[q] < je[q] ? col[j[q]] : kEnd; }
            }
            if (!any) break;
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (e[q] < 0) continue;
            score[e[q]] = key_bits(s[q]);
            asym = asym || (validate && !mirror[q]);
        }
    }
    if (asym) atomicOr(status, DEV_NOT_SYMMETRIC);
    count_ops(ops, n_add, n_sub);
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
                 const void* __restrict__ w, const void* __restrict__ w_und, int wsize,
                 int validate, uint32_t* status, unsigned long long* __restrict__ ops) {
    spc::pdl_wait();
    if (*status) return;
    uint32_t n_add = 0, n_sub = 0;
    bool asym = false;
    __shared__ int32_t s_col[kThreads / 32][kRowCache];
    __shared__ PT s_p[kThreads / 32][kRowCache];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; a < n; a += warps) {
        const int64_t r0 = rowptr[a], r1 = rowptr[a + 1];
        const int64_t da = r1 - r0;
        if (da > kLongRow) continue;  // hub row: k_score_hub
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
            const int64_t e = e0 + (jb - ufirst);
            if (je - j > kLongRow) {  // hub edge: k_score_hub; the mirror sits in the long row
                if (validate)
                    asym = asym || !has_mirror(col, w, wsize, j, je, a,
                                               weight_bits(w_und, wsize, e));
                continue;
            }
            // the mirror entry (b, a) is where row b holds column a; its weight bits must match
            bool mirror = false;
            if (validate) {
                for (int64_t q = j; q < je; ++q) {
                    const int32_t c = col[q];
                    if ((int64_t)c >= a) {
                        mirror = (int64_t)c == a &&
                                 weight_bits(w, wsize, q) == weight_bits(w_und, wsize, e);
                        break;
                    }
                }
                asym = asym || !mirror;
            }
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
                    ++n_sub;
                }
                s = p_add(s, t);
                ++n_add;
            }
            n_add += (uint32_t)(da - i) + (uint32_t)(je - j);
            while (i < da) {
                s = p_add(s, cached ? s_p[wib][i] : p[r0 + i]);
                ++i;
            }
            while (j < je) s = p_add(s, p[j++]);
            score[e] = key_bits(s);
        }
        __syncwarp();
    }
    if (asym) atomicOr(status, DEV_NOT_SYMMETRIC);
    count_ops(ops, n_add, n_sub);
}


// S3, staged schedule: a warp takes 32 consecutive edges (one lane each) and first moves their
// rows into shared memory with coalesced bulk loads -- the rows a of the tile, which are one
// contiguous slice of the CSR, and the 32 rows b, each read by the whole warp with its loads
// for eight rows in flight together -- then every lane walks its edge's union from shared
// memory with the same uniform step and order as k_score_edges (the same bits).  Walking rows
// in place reads one element per step from wherever row b lives; on graphs whose rows b are
// scattered (random node order) the lines are evicted between the steps and each step reads a
// sector from DRAM again.  Rows b longer than kStageCap entries, or a tile whose rows a exceed
// kStageA entries, are walked in place.
constexpr int kStageCap = 32;
constexpr int kStageStr = kStageCap + 1;  // padded: lanes of one step hit different banks
constexpr int kStageA = 256;
constexpr int kStageWarps = 4;
constexpr int kStageRegion = kStageA + 32 * kStageStr;  // elements per warp

// binary64: the positions of each lane's common coordinates in rows a and b (split walk)
constexpr int kSplitBytes = 2 * 32 * kStageCap;  // per warp: i and j, one byte each

template <class PT>
constexpr size_t stage_smem_bytes() {
    return (size_t)kStageWarps * kStageRegion * (sizeof(PT) + sizeof(int32_t)) +
           (sizeof(PT) == 8 ? (size_t)kStageWarps * kSplitBytes : 0);
}

template <class PT, class KT>
__global__ void __launch_bounds__(kStageWarps * 32)
k_score_staged(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
               const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
               const PT* __restrict__ p, KT* __restrict__ score, const void* __restrict__ w,
               const void* __restrict__ w_und, int wsize, int validate, uint32_t* status,
               unsigned long long* __restrict__ ops) {
    spc::pdl_wait();
    if (*status) return;
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    PT* const sa_p = reinterpret_cast<PT*>(stage_raw) + (size_t)wib * kStageRegion;
    PT* const sb_p = sa_p + kStageA;
    int32_t* const sa_c = reinterpret_cast<int32_t*>(reinterpret_cast<PT*>(stage_raw) +
                                                     (size_t)kStageWarps * kStageRegion) +
                          (size_t)wib * kStageRegion;
    int32_t* const sb_c = sa_c + kStageA;
    // binary64 split walk: lane l's common positions at sp_i/sp_j[l * kStageCap + c]
    uint8_t* const sp_i = reinterpret_cast<uint8_t*>(reinterpret_cast<int32_t*>(
                              reinterpret_cast<PT*>(stage_raw) + (size_t)kStageWarps * kStageRegion) +
                          (size_t)kStageWarps * kStageRegion) + (size_t)wib * kSplitBytes;
    uint8_t* const sp_j = sp_i + 32 * kStageCap;
    constexpr bool kSplit = sizeof(PT) == 8;
    constexpr int32_t kEnd = 0x7fffffff;
    uint32_t n_add = 0, n_sub = 0;
    bool asym = false;
    const int64_t step_e = (int64_t)gridDim.x * kStageWarps * 32;
    for (int64_t e0 = ((int64_t)blockIdx.x * kStageWarps + wib) * 32; e0 < m; e0 += step_e) {
        const int64_t e = e0 + lane;
        const bool act = e < m;
        int32_t a = 0;
        int64_t ra = 0, da = 0, rb = 0, db = 0;
        if (act) {
            a = eu[e];
            const int32_t b = ev[e];
            ra = rowptr[a];
            da = rowptr[a + 1] - ra;
            rb = rowptr[b];
            db = rowptr[b + 1] - rb;
        }
        // the tile's rows a: entries [rowptr[a of lane 0], rowptr[a of the last lane + 1])
        const int lastl = (int)((m - e0 < 32 ? m - e0 : 32) - 1);
        const int64_t abase = __shfl_sync(0xffffffffu, ra, 0);
        const int64_t alen = __shfl_sync(0xffffffffu, ra + da, lastl) - abase;
        const bool a_staged = alen <= kStageA;
        // asynchronous copies straight into shared memory: the row-a slice and all 32 rows b
        // of the tile are in flight together
        if (a_staged) {
            for (int64_t i = lane; i < alen; i += 32) {
                cp_async_4(sa_c + i, col + abase + i);
                cp_async_elem(sa_p + i, p + abase + i);
            }
        }
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int64_t rbk = __shfl_sync(0xffffffffu, rb, k);
            const int64_t dbk = __shfl_sync(0xffffffffu, db, k);
            if (dbk <= kStageCap && lane < dbk) {
                cp_async_4(sb_c + k * kStageStr + lane, col + rbk + lane);
                cp_async_elem(sb_p + k * kStageStr + lane, p + rbk + lane);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        const bool hub = act && (da > kLongRow || db > kLongRow);
        // binary64 rows that are both staged take the split walk: the subtractions, which only
        // coordinates in both rows need, in a loop of their own, then the additions
        const bool split = kSplit && act && !hub && a_staged && db <= kStageCap;
        if constexpr (kSplit) {
            int nc = 0;
            const int32_t* Ac = sa_c + (ra - abase);
            PT* const Bp = sb_p + lane * kStageStr;
            if (split) {  // integers only: where the two rows share a coordinate
                const int32_t* Bc = sb_c + lane * kStageStr;
                int i = 0, j = 0;
                while (i < da && j < db) {
                    const int32_t ca = Ac[i], cb = Bc[j];
                    if (ca == cb) {
                        sp_i[lane * kStageCap + nc] = (uint8_t)i;
                        sp_j[lane * kStageCap + nc] = (uint8_t)j;
                        ++nc;
                    }
                    i += ca <= cb ? 1 : 0;
                    j += cb <= ca ? 1 : 0;
                }
            }
            // one subtraction per common coordinate, |p_a - p_b| written over p_b
            const int maxc = __reduce_max_sync(0xffffffffu, nc);
            const PT* Ap = sa_p + (ra - abase);
            for (int c = 0; c < maxc; ++c) {
                if (c < nc) {
                    const int i = sp_i[lane * kStageCap + c], j = sp_j[lane * kStageCap + c];
                    Bp[j] = p_absdiff(Ap[i], Bp[j]);
                }
            }
            n_sub += (uint32_t)nc;
            __syncwarp();
        }
        if (split) {
            // one addition per coordinate of the union: the term is p_a, p_b or the difference
            // already in p_b's place (|x - 0| = x, so the bits equal the uniform step's)
            const int32_t* Ac = sa_c + (ra - abase);
            const PT* Ap = sa_p + (ra - abase);
            const int32_t* Bc = sb_c + lane * kStageStr;
            const PT* Bp = sb_p + lane * kStageStr;
            int i = 0, j = 0;
            int32_t ca = da > 0 ? Ac[0] : kEnd;
            int32_t cb = db > 0 ? Bc[0] : kEnd;
            PT s = PT(0);
            bool mirror = false;
            while (ca != kEnd || cb != kEnd) {
                const bool ta = ca <= cb, tb = cb <= ca;
                if (validate && tb && cb == a)
                    mirror = weight_bits(w, wsize, rb + j) == weight_bits(w_und, wsize, e);
                s = p_add(s, tb ? Bp[j] : Ap[i]);
                ++n_add;
                if (ta) { ++i; ca = i < da ? Ac[i] : kEnd; }
                if (tb) { ++j; cb = j < db ? Bc[j] : kEnd; }
            }
            score[e] = key_bits(s);
            asym = asym || (validate && !mirror);
        } else if (act) {
            if (hub) {  // hub edge: k_score_hub
                if (validate && da <= kLongRow)
                    asym = asym || !has_mirror(col, w, wsize, rb, rb + db, a,
                                               weight_bits(w_und, wsize, e));
            } else {
                const int32_t* Ac = a_staged ? sa_c + (ra - abase) : col + ra;
                const PT* Ap = a_staged ? sa_p + (ra - abase) : p + ra;
                const int32_t* Bc = db <= kStageCap ? sb_c + lane * kStageStr : col + rb;
                const PT* Bp = db <= kStageCap ? sb_p + lane * kStageStr : p + rb;
                int64_t i = 0, j = 0;
                int32_t ca = da > 0 ? Ac[0] : kEnd;
                int32_t cb = db > 0 ? Bc[0] : kEnd;
                PT s = PT(0);
                bool mirror = false;
                // the uniform step of k_score_edges: t = |pa - pb| with a missing side read as 0
                while (ca != kEnd || cb != kEnd) {
                    const bool ta = ca <= cb, tb = cb <= ca;
                    if (validate && tb && cb == a)
                        mirror = weight_bits(w, wsize, rb + j) == weight_bits(w_und, wsize, e);
                    const PT pa = ta ? Ap[i] : PT(0);
                    const PT pb = tb ? Bp[j] : PT(0);
                    s = p_add(s, p_absdiff(pa, pb));
                    ++n_add;
                    n_sub += (ta && tb) ? 1u : 0u;
                    if (ta) { ++i; ca = i < da ? Ac[i] : kEnd; }
                    if (tb) { ++j; cb = j < db ? Bc[j] : kEnd; }
                }
                score[e] = key_bits(s);
                asym = asym || (validate && !mirror);
            }
        }
        __syncwarp();  // the next tile overwrites the stage
    }
    if (asym) atomicOr(status, DEV_NOT_SYMMETRIC);
    count_ops(ops, n_add, n_sub);
}

// S3, packed schedule for binary32 rows: the normalise kernel stores every entry as one 8-byte
// (column, p) pair, so a row is one contiguous run of bytes.  A warp takes 32 consecutive
// edges (one lane each): the tile's rows a, one contiguous slice, are copied by the whole warp,
// and every lane copies its own row b into the warp's area, the rows packed one after the other
// (a prefix sum of their lengths places them), all with 16-byte asynchronous copies.  A copy
// keeps each entry's position modulo two entries, so both of its ends are 16-byte aligned; a
// row that starts or ends inside a 16-byte chunk brings its neighbour along, never read.  Then
// every lane walks its edge's union from shared memory, one 8-byte load per step, with the
// uniform step of k_score_edges (the same bits).  Rows that do not fit are walked in place.
// Binary32 inputs have their symmetry checked by the fingerprint of the normalise kernel, so
// the walk carries no mirror check (and no arithmetic count, which serves binary64 only).
constexpr int kPkWarps = 8;
constexpr int kPkA = 192;  // entries of the tile's row-a slice staged per warp
constexpr int kPkB = 576;  // entries of the tile's 32 rows b staged per warp
constexpr int kPkRegion = kPkA + kPkB;
constexpr size_t kPkSmem = (size_t)kPkWarps * kPkRegion * sizeof(uint2);

// L2 eviction priority (createpolicy, sm_80 and later): the row pointers, read at random once
// per edge endpoint, are kept in L2 ahead of the rows, which are far larger than L2 on big graphs.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ int64_t ld_l2hint(const int64_t* ptr, uint64_t pol) {
    int64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

template <class KT>
__global__ void __launch_bounds__(kPkWarps * 32)
k_score_packed(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
               const int64_t* __restrict__ rowptr, const uint2* __restrict__ pk,
               KT* __restrict__ score, const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    extern __shared__ __align__(16) uint2 pk_stage[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint2* const sa = pk_stage + (size_t)wib * kPkRegion;
    uint2* const sb = sa + kPkA;
    const uint4* const pk16 = reinterpret_cast<const uint4*>(pk);
    constexpr int32_t kEnd = 0x7fffffff;  // the end marker's column
    const uint64_t keep = l2_policy_evict_last();
    const int64_t step_e = (int64_t)gridDim.x * kPkWarps * 32;
    for (int64_t e0 = ((int64_t)blockIdx.x * kPkWarps + wib) * 32; e0 < m; e0 += step_e) {
        const int64_t e = e0 + lane;
        const bool act = e < m;
        int32_t a = 0, b = 0;
        int64_t ra = 0, da = 0, rb = 0, db = 0;
        if (act) {
            a = eu[e];
            b = ev[e];
            ra = ld_l2hint(rowptr + a, keep);
            da = ld_l2hint(rowptr + a + 1, keep) - ra;
            rb = ld_l2hint(rowptr + b, keep);
            db = ld_l2hint(rowptr + b + 1, keep) - rb;
        }
        const bool hub = act && (da > kLongRow || db > kLongRow);
        // packed positions: row x's pairs start at rowptr[x] + x, its end marker follows them
        const int64_t pa0 = ra + a, pb0 = rb + b;
        // the rows a of the tile, end markers included: pairs [pa0 of lane 0, pa0 + da + 1
        // of the last lane), as 16-byte chunks [ac0, ac1)
        const int lastl = (int)((m - e0 < 32 ? m - e0 : 32) - 1);
        const int64_t ac0 = __shfl_sync(0xffffffffu, pa0, 0) >> 1;
        const int64_t ac1 = (__shfl_sync(0xffffffffu, pa0 + da + 1, lastl) + 1) >> 1;
        const bool a_staged = 2 * (ac1 - ac0) <= kPkA;
        if (a_staged)
            for (int64_t q = ac0 + lane; q < ac1; q += 32)
                cp_async_16(sa + 2 * (q - ac0), pk16 + q);
        // this lane's row b: its pairs, chunks [pb0 / 2, (pb0 + db + 1) / 2), placed after the
        // other lanes'; its end marker is written in shared memory (a random row fetches no
        // more than its pairs), in one more chunk of room when the pairs fill their last one
        const int64_t bc0 = pb0 >> 1;
        const int nch = (act && !hub) ? (int)(((pb0 + db + 1) >> 1) - bc0) : 0;
        const int nroom = nch + ((act && !hub && (pb0 & 1) + db == 2 * nch) ? 1 : 0);
        int choff = nroom;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, choff, d);
            if (lane >= d) choff += t;
        }
        choff -= nroom;
        const bool b_staged = 2 * (choff + nroom) <= kPkB;
        const int maxch = __reduce_max_sync(0xffffffffu, b_staged ? nch : 0);
        for (int k = 0; k < maxch; ++k)
            if (b_staged && k < nch) cp_async_16(sb + 2 * (choff + k), pk16 + bc0 + k);
        cp_async_wait_all();
        if (b_staged && act && !hub)
            sb[2 * choff + (pb0 & 1) + db] = make_uint2((uint32_t)kEnd, 0u);
        __syncwarp();
        if (act && !hub) {
            // both rows end in their marker: the walk advances without bounds
            const uint2* A = a_staged ? sa + (pa0 - 2 * ac0) : pk + pa0;
            const uint2* B = b_staged ? sb + 2 * choff + (pb0 & 1) : pk + pb0;
            uint2 xa = A[0], xb = B[0];
            float s = 0.f;
            for (;;) {
                const int32_t ca = (int32_t)xa.x, cb = (int32_t)xb.x;
                if (ca == kEnd && cb == kEnd) break;
                const bool ta = ca <= cb, tb = cb <= ca;
                const float pa = ta ? __uint_as_float(xa.y) : 0.f;
                const float pb = tb ? __uint_as_float(xb.y) : 0.f;
                s = p_add(s, p_absdiff(pa, pb));
                if (ta) xa = *++A;
                if (tb) xb = *++B;
            }
            score[e] = key_bits(s);
        }
        __syncwarp();  // the next tile overwrites the stage
    }
}

// ---- hub edges ----------------------------------------------------------------------------------
// An edge with an end point of more than kLongRow entries is scored from the larger row H (its
// "hub"; ties go to the smaller id).  The score is the same left-to-right sum over the union of
// the two rows, which reads as runs of plain H terms p_Hx (x not in the other row v) separated
// by the coordinates of v's row ("specials": an extra term p_vx, or |p_Hx - p_vx| where both
// rows have x).  Runs are evaluated exactly from per-binade prefix tables of H's row.

constexpr int kHeavySpecials = 32;  // edges whose other row is longer go to the warp kernel

// light hub edges: one thread per entry (H, v) of a hub row, flat over all hubs
// Column positions of the largest hub rows: for up to kMaxHubMaps hubs holding at least an
// eighth of the nodes (and 2048 entries), map[slot * n + x] = the first position of the hub's
// row whose column is >= x, so the hub kernels place a coordinate with one load instead of a
// binary search over the hub's row.
constexpr int kMaxHubMaps = 8;
struct HubMaps {
    const int32_t* map;   // nullptr: no maps on this level
    const int32_t* slot;  // per long row: its map slot or -1
    int64_t n;
};

__global__ void k_hub_slots(const int32_t* __restrict__ long_count,
                            const int64_t* __restrict__ lr_len, int64_t n, int maps,
                            int32_t* __restrict__ slot_of, int32_t* __restrict__ slot_hub,
                            int32_t* __restrict__ nslots) {
    spc::pdl_wait();
    __shared__ int32_t cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int32_t c = *long_count;
    for (int32_t i = threadIdx.x; i < c; i += blockDim.x) {
        int32_t sl = -1;
        const int64_t d = lr_len[i];
        if (d >= 2048 && d * 8 >= n) {
            const int32_t s = atomicAdd(&cnt, 1);
            if (s < maps) {
                sl = s;
                slot_hub[s] = i;
            }
        }
        slot_of[i] = sl;
    }
    __syncthreads();
    if (threadIdx.x == 0) *nslots = cnt < maps ? cnt : maps;
}

__global__ void __launch_bounds__(kThreads)
k_hub_posmap(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const int32_t* __restrict__ long_rows, const int32_t* __restrict__ slot_hub,
             const int32_t* __restrict__ nslots, int64_t n, int32_t* __restrict__ map) {
    spc::pdl_wait();
    const int64_t total = (int64_t)*nslots * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = (int32_t)(t / n);
        const int64_t x = t - (int64_t)s * n;
        const int64_t H = long_rows[slot_hub[s]];
        const int64_t r0 = rowptr[H];
        int64_t lo = 0, hi = rowptr[H + 1] - r0;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)col[r0 + mid] < x) lo = mid + 1; else hi = mid;
        }
        map[t] = (int32_t)lo;
    }
}

// Hub edge (H, v) where v's only entry is H (v has no diagonal): the union of the two rows is
// H's row with p_v[H] = w / w = 1 at H's own column position -- a term |0 - 1| = 1 inserted
// there, or, when H's row holds its diagonal entry, that entry's term |p_HH - 1| -- so every
// such edge of H has the same score.  A warp evaluates it once per hub.
template <class PT>
__global__ void __launch_bounds__(kThreads)
k_hub_leaf_score(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const PT* __restrict__ p, const int32_t* __restrict__ long_rows,
                 const int32_t* __restrict__ long_count, SeqTabView tab, PT* __restrict__ leaf) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < cnt;
         i += warps) {
        const int64_t H = long_rows[i];
        const int64_t rH = rowptr[H], dH = rowptr[H + 1] - rH;
        const int32_t* cH = col + rH;
        int64_t lo = 0, hi = dH;  // first position whose column is H or above
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)cH[mid] < H) lo = mid + 1; else hi = mid;
        }
        const bool diag = lo < dH && (int64_t)cH[lo] == H;
        const unsigned long long* P = tab.P + tab.tab_off[i];
        const int32_t* T = tab.T + tab.tab_off[i];
        PT s = tab_run_warp<PT>(PT(0), 0, lo, p + rH, P, T, tab.eblo[i], tab.nE[i], dH + 1);
        s = p_add(s, diag ? p_absdiff(p[rH + lo], PT(1)) : PT(1));
        s = tab_run_warp<PT>(s, diag ? lo + 1 : lo, dH, p + rH, P, T, tab.eblo[i], tab.nE[i],
                             dH + 1);
        if ((threadIdx.x & 31) == 0) leaf[i] = s;
    }
}

template <class PT, class KT>
__global__ void __launch_bounds__(kThreads)
k_score_hub(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
            const PT* __restrict__ p, const int32_t* __restrict__ up_ptr,
            const int32_t* __restrict__ nlow, const int32_t* __restrict__ long_rows,
            const int32_t* __restrict__ long_count, const int64_t* __restrict__ lr_eoff,
            SeqTabView tab, HubMaps hm, const PT* __restrict__ leaf, KT* __restrict__ score,
            int32_t* __restrict__ heavy, int32_t* __restrict__ heavy_count,
            const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    const int32_t cnt = *long_count;
    const int64_t total = lr_eoff[cnt];
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = cnt - 1;  // hub of flat entry f
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (lr_eoff[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int32_t i = lo;
        const int64_t H = long_rows[i];
        const int64_t rH = rowptr[H], dH = rowptr[H + 1] - rH;
        const int64_t k = f - lr_eoff[i];
        const int64_t v = col[rH + k];
        if (v == H) continue;  // H's diagonal entry is no edge
        const int64_t rv = rowptr[v], dv = rowptr[v + 1] - rv;
        if (dv > dH || (dv == dH && v < H)) continue;  // v's row is the hub of this edge
        if (dv == 1 && key_bits(p[rv]) == key_bits(PT(1))) {  // v a leaf of H: the hub's value
            const int64_t e = (H < v) ? (int64_t)up_ptr[H] + (k - nlow[H])
                                      : (int64_t)up_ptr[v] - nlow[v];
            score[e] = key_bits(leaf[i]);
            continue;
        }
        if (dv > kHeavySpecials) {                       // many specials: warp kernel
            heavy[atomicAdd(heavy_count, 1)] = (int32_t)f;
            continue;
        }
        const int32_t* cH = col + rH;
        const PT* pH = p + rH;
        const unsigned long long* P = tab.P + tab.tab_off[i];
        const int32_t* T = tab.T + tab.tab_off[i];
        const int eblo = tab.eblo[i], nE = tab.nE[i];
        const int32_t* hmap = (hm.map && hm.slot[i] >= 0) ? hm.map + (int64_t)hm.slot[i] * hm.n
                                                          : nullptr;
        PT s = PT(0);
        int64_t a = 0;
        int64_t jH = -1;  // position of H in v's row
        for (int64_t j = 0; j < dv; ++j) {
            const int32_t x = col[rv + j];
            if ((int64_t)x == H) jH = j;
            int64_t l2 = a, h2 = dH;  // first position >= a in H's row with column >= x
            if (hmap) {
                l2 = hmap[x];
                if (l2 < a) l2 = a;
            } else {
                while (l2 < h2) {
                    const int64_t mid = (l2 + h2) >> 1;
                    if (cH[mid] < x) l2 = mid + 1; else h2 = mid;
                }
            }
            s = tab_run<PT>(s, a, l2, pH, P, T, eblo, nE, dH + 1);
            PT t;
            if (l2 < dH && cH[l2] == x) {
                t = p_absdiff(pH[l2], p[rv + j]);
                a = l2 + 1;
            } else {
                t = p[rv + j];
                a = l2;
            }
            s = p_add(s, t);
        }
        s = tab_run<PT>(s, a, dH, pH, P, T, eblo, nE, dH + 1);
        const int64_t e = (H < v) ? (int64_t)up_ptr[H] + (k - nlow[H])
                                  : (int64_t)up_ptr[v] + (jH - nlow[v]);
        score[e] = key_bits(s);
    }
}

// heavy hub edges: one warp per edge.  Lanes take 32 specials at a time: each finds its
// position in H's row; then, inside the running sum's binade, the whole group advances as one
// integer prefix sum over (run before special j, special j) pairs -- the run's increment read
// from H's tables, the special's as its grid-rounded value.  The first pair that crosses the
// binade or holds a tie is finished exactly (tab_run / one native add) and the group restarts.
template <class PT, class KT>
__global__ void __launch_bounds__(kThreads)
k_score_hub_heavy(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const PT* __restrict__ p, const int32_t* __restrict__ up_ptr,
                  const int32_t* __restrict__ nlow, const int32_t* __restrict__ long_rows,
                  const int32_t* __restrict__ long_count, const int64_t* __restrict__ lr_eoff,
                  SeqTabView tab, HubMaps hm, const int32_t* __restrict__ heavy,
                  const int32_t* __restrict__ heavy_count, KT* __restrict__ score,
                  const uint32_t* status) {
    spc::pdl_wait();
    if (*status) return;
    const int lane = threadIdx.x & 31;
    const int32_t cnt = *long_count;
    const int32_t nheavy = *heavy_count;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t hq = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); hq < nheavy;
         hq += warps) {
        const int64_t f = heavy[hq];
        int32_t lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (lr_eoff[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int32_t i = lo;
        const int64_t H = long_rows[i];
        const int64_t rH = rowptr[H], dH = rowptr[H + 1] - rH;
        const int64_t k = f - lr_eoff[i];
        const int64_t v = col[rH + k];
        const int64_t rv = rowptr[v], dv = rowptr[v + 1] - rv;
        const int32_t* cH = col + rH;
        const PT* pH = p + rH;
        const unsigned long long* P = tab.P + tab.tab_off[i];
        const int32_t* T = tab.T + tab.tab_off[i];
        const int eblo = tab.eblo[i], nE = tab.nE[i];
        const int32_t* hmap = (hm.map && hm.slot[i] >= 0) ? hm.map + (int64_t)hm.slot[i] * hm.n
                                                          : nullptr;
        const int64_t d1 = dH + 1;
        PT s = PT(0);
        int64_t a = 0;      // next unread position of H's row
        int64_t jH = -1;
        int64_t j0 = 0;     // next special
        while (j0 < dv) {
            const int64_t j = j0 + lane;
            const bool act = j < dv;
            int32_t x = 0;
            int64_t pos = dH;
            bool common = false;
            PT t = PT(0);
            if (act) {
                x = col[rv + j];
                int64_t l2 = a, h2 = dH;
                if (hmap) {
                    l2 = hmap[x];
                    if (l2 < a) l2 = a;
                } else {
                    while (l2 < h2) {
                        const int64_t mid = (l2 + h2) >> 1;
                        if (cH[mid] < x) l2 = mid + 1; else h2 = mid;
                    }
                }
                pos = l2;
                common = pos < dH && cH[pos] == x;
                t = common ? p_absdiff(pH[pos], p[rv + j]) : p[rv + j];
                if ((int64_t)x == H) jH = j;
            }
            // start of the run before special j: after special j-1 (or `a` for the first)
            int64_t after = pos + (common ? 1 : 0);
            int64_t start = __shfl_up_sync(0xffffffffu, after, 1);
            if (lane == 0) start = a;
            const int nact = (dv - j0) < 32 ? (int)(dv - j0) : 32;
            // advance through the group, restarting after every exact step
            int g = 0;  // first lane of the group not yet added
            while (g < nact) {
                bool done_fast = false;
                if (s != PT(0)) {
                    const unsigned long long sb = FB<PT>::bits(s);
                    const int eb = (int)(sb >> FB<PT>::kMant);
                    const int e = eb - eblo;
                    if (eb != 0 && e >= 0 && e < nE) {
                        const unsigned long long* Pe = P + (int64_t)e * d1;
                        const int32_t* Te = T + (int64_t)e * d1;
                        const unsigned long long S =
                            (sb & ((1ull << FB<PT>::kMant) - 1ull)) | (1ull << FB<PT>::kMant);
                        const unsigned long long lim = (1ull << (FB<PT>::kMant + 1)) - S;
                        unsigned long long dr = 0, ds = 0;
                        bool tr = false, ts = false, sat = false;
                        if (lane >= g && lane < nact) {
                            const unsigned long long pb = Pe[start];
                            sat = pb >= kSat - (1ull << 55);
                            dr = Pe[pos] - pb;
                            tr = Te[pos] != Te[start];
                            ds = grid_units<PT>(t, eb, &ts);
                        }
                        // inclusive prefix of (dr + ds) over lanes g..nact-1
                        unsigned long long both = sat_add(dr, ds);
                        unsigned long long incl = both;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl = sat_add(incl, u);
                        }
                        unsigned long long excl = __shfl_up_sync(0xffffffffu, incl, 1);
                        if (lane == 0) excl = 0ull;
                        const bool bad_run = (lane >= g && lane < nact) &&
                                             (sat || tr || sat_add(excl, dr) > lim);
                        const bool bad_sp = (lane >= g && lane < nact) &&
                                            (ts || sat_add(sat_add(excl, dr), ds) > lim);
                        const unsigned bal = __ballot_sync(0xffffffffu, bad_run || bad_sp);
                        if (bal == 0) {
                            const unsigned long long tot =
                                __shfl_sync(0xffffffffu, incl, nact - 1);
                            s = from_units<PT>(S + tot, eb);
                            g = nact;
                            done_fast = true;
                        } else {
                            const int fl = __ffs(bal) - 1;
                            const unsigned long long ex = __shfl_sync(0xffffffffu, excl, fl);
                            const unsigned long long drf = __shfl_sync(0xffffffffu, dr, fl);
                            const bool run_bad = __shfl_sync(0xffffffffu, bad_run, fl);
                            const int64_t st_f = __shfl_sync(0xffffffffu, start, fl);
                            const int64_t pos_f = __shfl_sync(0xffffffffu, pos, fl);
                            const PT t_f = __shfl_sync(0xffffffffu, t, fl);
                            if (run_bad) {
                                s = from_units<PT>(S + ex, eb);
                                s = tab_run<PT>(s, st_f, pos_f, pH, P, T, eblo, nE, d1);
                            } else {
                                s = from_units<PT>(S + ex + drf, eb);
                            }
                            s = p_add(s, t_f);
                            g = fl + 1;
                            done_fast = true;
                        }
                    }
                }
                if (!done_fast) {  // running sum outside the tables: one pair exactly
                    const int64_t st_g = __shfl_sync(0xffffffffu, start, g);
                    const int64_t pos_g = __shfl_sync(0xffffffffu, pos, g);
                    const PT t_g = __shfl_sync(0xffffffffu, t, g);
                    s = tab_run<PT>(s, st_g, pos_g, pH, P, T, eblo, nE, d1);
                    s = p_add(s, t_g);
                    ++g;
                }
            }
            a = __shfl_sync(0xffffffffu, after, nact - 1);
            j0 += nact;
        }
        s = tab_run_warp<PT>(s, a, dH, pH, P, T, eblo, nE, d1);
        // jH: the lane that saw x == H
        const unsigned hb = __ballot_sync(0xffffffffu, jH >= 0);
        if (hb) jH = __shfl_sync(0xffffffffu, jH, __ffs(hb) - 1);
        if (lane == 0) {
            const int64_t e = (H < v) ? (int64_t)up_ptr[H] + (k - nlow[H])
                                      : (int64_t)up_ptr[v] + (jH - nlow[v]);
            score[e] = key_bits(s);
        }
    }
}

// edges walked together by a thread of k_score_edges (4 spilled and ran slower)
constexpr int kScoreChains = 2;

template <class P, class Key>
static spc_status launch_score_edges(spc_context* ctx, int64_t m, const GraphView& g, Work& W,
                                     void* score, int wsize, int vflag, uint32_t* status,
                                     bool count) {
    SPC_LAUNCH(ctx, (k_score_edges<P, Key, kScoreChains>),
               grid_for(m, kThreads, ctx->num_sms * 8), kThreads, 0, m, W.eu.as<int32_t>(), W.ev.as<int32_t>(), g.rowptr, g.col,
               W.p.as<P>(), static_cast<Key*>(score), g.w, W.w_und.p, wsize, vflag, status,
               count ? op_counter(ctx, "(k_score_edges<P, Key, kScoreChains>)", 0) : nullptr);
    return SPC_OK;
}

template <class P, class Key>
static spc_status launch_score_staged(spc_context* ctx, int64_t m, const GraphView& g, Work& W,
                                      void* score, int wsize, int vflag, uint32_t* status,
                                      bool count) {
    constexpr size_t smem = stage_smem_bytes<P>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices already set up
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(attr_devs.load() & bit)) {
        SPC_CUDA(cudaFuncSetAttribute(k_score_staged<P, Key>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_devs.fetch_or(bit);
    }
    const int64_t tiles = (m + 31) / 32;
    const int grid = grid_for(tiles, kStageWarps, ctx->num_sms * (sizeof(P) == 8 ? 3 : 5));
    SPC_LAUNCH(ctx, (k_score_staged<P, Key>), grid, kStageWarps * 32, smem, m,
               W.eu.as<int32_t>(), W.ev.as<int32_t>(), g.rowptr, g.col, W.p.as<P>(),
               static_cast<Key*>(score), g.w, W.w_und.p, wsize, vflag, status,
               count ? op_counter(ctx, "(k_score_staged<P, Key>)", 4) : nullptr);
    return SPC_OK;
}

template <class Key>
static spc_status launch_score_packed(spc_context* ctx, int64_t m, const GraphView& g, Work& W,
                                      void* score, int wsize, int vflag, uint32_t* status,
                                      bool count) {
    static std::atomic<unsigned long long> attr_devs{0};  // devices already set up
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(attr_devs.load() & bit)) {
        SPC_CUDA(cudaFuncSetAttribute(k_score_packed<Key>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPkSmem));
        attr_devs.fetch_or(bit);
    }
    const int64_t tiles = (m + 31) / 32;
    const int grid = grid_for(tiles, kPkWarps, ctx->num_sms * 4);
    // binary32 rows only: symmetry is checked by the fingerprint of the normalise kernel, and
    // the arithmetic count serves the binary64 roofline alone
    (void)wsize;
    (void)vflag;
    (void)count;
    SPC_LAUNCH(ctx, k_score_packed<Key>, grid, kPkWarps * 32, kPkSmem, m, W.eu.as<int32_t>(),
               W.ev.as<int32_t>(), g.rowptr, W.pk.as<uint2>(), static_cast<Key*>(score), status);
    return SPC_OK;
}

// schedule 3: rows staged in shared memory (binary32 rows as packed (column, p) pairs)
template <class P, class Key>
static spc_status launch_score_stage(spc_context* ctx, int64_t m, const GraphView& g, Work& W,
                                     void* score, int wsize, int vflag, uint32_t* status,
                                     bool count) {
    if constexpr (std::is_same<P, float>::value)
        return launch_score_packed<Key>(ctx, m, g, W, score, wsize, vflag, status, count);
    else
        return launch_score_staged<P, Key>(ctx, m, g, W, score, wsize, vflag, status, count);
}

static int pick_default_schedule(int64_t n, int64_t nnz) {
    return (n > 0 && nnz / n > 48) ? 2 : 3;  // long rows favour a warp per row
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
    const int persist = ctx->num_sms * 2;
    const bool fp = !std::is_same<WT, int32_t>::value;
    uint32_t* status = ctx->d_status;
    int32_t* long_count = W.counters.as<int32_t>() + 8;
    int32_t* heavy_count = W.counters.as<int32_t>() + 10;
    int32_t* long_rows = W.long_rows.as<int32_t>();
    const int gb = grid_for(n, kThreads, maxb);
    const double s_w = sizeof(WT), s_p = sizeof(P), s_acc = sizeof(Acc), s_key = sizeof(Key);
    SPC_CUDA(cudaMemsetAsync(long_count, 0, sizeof(int32_t), ctx->stream));
    // rowptr, columns and weights read once; degree and the two per-row counts written once
    note_bytes(ctx, 8.0 * (n + 1) + nnz * (4 + s_w) + n * (s_acc + 8));
    SPC_LAUNCH(ctx, k_rows_degree<WT>, gb, kThreads, 0, n, nnz, g.rowptr, g.col,
               static_cast<const WT*>(g.w), validate ? 1 : 0, W.deg.as<Acc>(),
               W.up_cnt.as<int32_t>(), W.first_up.as<int32_t>(), long_rows, long_count, status);
    SPC_LAUNCH(ctx, k_long_rows_meta<WT>, persist, kThreads, 0, g.rowptr, g.col, long_rows,
               long_count, W.deg.as<Acc>(), W.up_cnt.as<int32_t>(), W.first_up.as<int32_t>(),
               W.lr_base.as<int64_t>(), W.lr_len.as<int64_t>(), W.lr_idx.as<int64_t>(),
               heavy_count);
    SPC_TRY(scan_i32(ctx, W.up_cnt.as<int32_t>(), W.up_ptr.as<int32_t>(), n));
    // the edge count and the number of long rows
    int64_t sizes[2];
    {
        const void* ptrs[2] = {W.up_ptr.as<int32_t>() + n, long_count};
        const int bytes[2] = {4, 4};
        SPC_TRY(read_vals(ctx, 2, ptrs, bytes, sizes));
    }
    const int64_t m = sizes[0];
    const int64_t n_long = sizes[1];
    if (n_long > 0) {
        SPC_TRY(scan_i64_i64(ctx, W.lr_len.as<int64_t>(), W.lr_eoff.as<int64_t>(), n_long));
        SPC_LAUNCH(ctx, k_long_rows_flat<WT>, maxb, kThreads, 0, n, g.rowptr, g.col,
                   static_cast<const WT*>(g.w), validate ? 1 : 0, long_rows, long_count,
                   W.lr_eoff.as<int64_t>(), W.deg.as<Acc>(), status);
    }
    // every input check of every row so far
    SPC_TRY(check_status(ctx));
    if (2 * m + g.ndiag != nnz) return SPC_ERR_NOT_SYMMETRIC;
    g.m = m;
    // rowptr, columns, weights, degrees and row counts read once; p and the undirected edge
    // list written once (no model on levels with long rows: another kernel takes their part)
    if (n_long == 0)
        note_bytes(ctx, 8.0 * (n + 1) + nnz * (4 + s_w) + n * (s_acc + 8) + nnz * s_p +
                            m * (8 + s_w));
    // the symmetry of rows up to kLongRow is checked by the score kernels' walks when scores
    // are computed; without scores, here
    const int wsize = (int)sizeof(WT);
    const bool mirror_here = validate && (score == nullptr || m == 0);
    // binary32 levels that are scored check symmetry by the fingerprint of the flat normalise
    // kernel; the others by the score walks (or, without scores, by k_rows_edges' searches)
    const bool fingerprint = std::is_same<WT, float>::value && validate && !mirror_here && n > 0;
    const int vflag = validate && !fingerprint ? 1 : 0;
    // the score schedule: forced, or autotuned once per shape bucket (every schedule computes
    // the same bits)
    int lg_deg = 0, lg_m = 0;
    while ((1ll << (lg_deg + 1)) <= (n > 0 ? nnz / n : 0)) ++lg_deg;
    while ((1ll << (lg_m + 1)) <= m) ++lg_m;
    const int64_t tkey = ((int64_t)g.wtype << 16) | (lg_deg << 8) | lg_m;
    if (schedule != 1 && schedule != 2 && schedule != 3) {
        schedule = 0;
        for (const auto& tk : ctx->tuned)
            if (tk.first == tkey) schedule = tk.second;
        if (schedule == 0 && capturing(ctx)) schedule = pick_default_schedule(n, nnz);
    }
    // binary32 rows: the packed schedule reads only the (column, p) pairs; p alone serves the
    // other schedules (and the autotuner, which times them) and the hub kernels
    const bool need_p = score == nullptr || n_long > 0 || schedule != 3;
    {
        // long rows (exact degrees from per-binade tables, then p and their edges) on the
        // second stream while the short rows run here
        std::unique_ptr<SideBranch> side;
        if (n_long > 0) {
            side.reset(new SideBranch(ctx));
            SPC_TRY(side->status());
            if (fp) {
                SPC_TRY(seqtab_full(ctx, g.w, std::is_same<WT, float>::value, n_long,
                                    W.lr_base.as<int64_t>(), W.lr_len.as<int64_t>(),
                                    W.lr_idx.as<int64_t>(), W.deg.p, W.tab_w));
            }
            SPC_LAUNCH(ctx, k_long_rows_edges<WT>, maxb, kThreads, 0, g.rowptr, g.col,
                       static_cast<const WT*>(g.w), validate ? 1 : 0, W.deg.as<Acc>(),
                       W.first_up.as<int32_t>(), W.up_ptr.as<int32_t>(), long_rows, long_count,
                       W.lr_eoff.as<int64_t>(), W.p.as<P>(), W.eu.as<int32_t>(),
                       W.ev.as<int32_t>(), W.w_und.as<WT>(), status);
            side->leave();
        }
        if constexpr (std::is_same<WT, float>::value) {
            if (!mirror_here && n > 0) {
                unsigned long long* sym = nullptr;
                if (fingerprint) {
                    sym = W.sym.as<unsigned long long>();
                    SPC_CUDA(cudaMemsetAsync(sym, 0, 8, ctx->stream));
                }
                SPC_LAUNCH(ctx, k_rows_edges_flat, grid_for(nnz, (int)kFlatTile, maxb), kThreads,
                           0, n, nnz, g.rowptr, g.col, static_cast<const float*>(g.w),
                           W.deg.as<float>(), W.first_up.as<int32_t>(), W.up_ptr.as<int32_t>(),
                           need_p ? W.p.as<float>() : nullptr, W.pk.as<uint2>(),
                           W.eu.as<int32_t>(), W.ev.as<int32_t>(), W.w_und.as<float>(), sym,
                           ctx->sym_key[0], ctx->sym_key[1], status);
                if (fingerprint) SPC_LAUNCH(ctx, k_sym_check, 1, 32, 0, sym, status);
            } else {
                SPC_LAUNCH(ctx, k_rows_edges<WT>, gb, kThreads, 0, n, g.rowptr, g.col,
                           static_cast<const WT*>(g.w), mirror_here ? 1 : 0, W.deg.as<Acc>(),
                           W.first_up.as<int32_t>(), W.up_ptr.as<int32_t>(), W.p.as<P>(),
                           W.eu.as<int32_t>(), W.ev.as<int32_t>(), W.w_und.as<WT>(), status);
            }
        } else {
            SPC_LAUNCH(ctx, k_rows_edges<WT>, gb, kThreads, 0, n, g.rowptr, g.col,
                       static_cast<const WT*>(g.w), mirror_here ? 1 : 0, W.deg.as<Acc>(),
                       W.first_up.as<int32_t>(), W.up_ptr.as<int32_t>(), W.p.as<P>(),
                       W.eu.as<int32_t>(), W.ev.as<int32_t>(), W.w_und.as<WT>(), status);
        }
    }  // the main stream waits for the long rows here
    if (score == nullptr || m == 0) {
        if (validate) SPC_TRY(check_status(ctx));
        return SPC_OK;
    }
    if (schedule == 0) {  // not tuned yet for this shape: time each schedule once
        if (!ctx->tune_ev[0])
            for (auto& ev : ctx->tune_ev) SPC_CUDA(cudaEventCreate(&ev));
        const int gw = grid_for(n, kThreads / 32, maxb);
        SPC_CUDA(cudaEventRecord(ctx->tune_ev[0], ctx->stream));
        SPC_TRY((launch_score_edges<P, Key>(ctx, m, g, W, score, wsize, vflag, status, false)));
        SPC_CUDA(cudaEventRecord(ctx->tune_ev[1], ctx->stream));
        SPC_LAUNCH(ctx, (k_score_warp_row<P, Key>), gw, kThreads, 0, n, g.rowptr, g.col,
                   W.p.as<P>(), W.up_ptr.as<int32_t>(), W.first_up.as<int32_t>(),
                   static_cast<Key*>(score), g.w, W.w_und.p, wsize, vflag, status, nullptr);
        SPC_CUDA(cudaEventRecord(ctx->tune_ev[2], ctx->stream));
        SPC_TRY((launch_score_stage<P, Key>(ctx, m, g, W, score, wsize, vflag, status,
                                            false)));
        SPC_CUDA(cudaEventRecord(ctx->tune_ev[3], ctx->stream));
        SPC_CUDA(cudaEventSynchronize(ctx->tune_ev[3]));
        float t[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 3; ++k)
            SPC_CUDA(cudaEventElapsedTime(&t[k], ctx->tune_ev[k], ctx->tune_ev[k + 1]));
        schedule = 1;
        if (t[1] < t[schedule - 1]) schedule = 2;
        if (t[2] < t[schedule - 1]) schedule = 3;
        ctx->tuned.push_back({tkey, schedule});
    }
    // rowptr, every stored column and p read once, every score written once (no model on
    // levels with long rows: the hub kernels take their edges)
    const double score_bytes = n_long == 0 ? 8.0 * (n + 1) + nnz * (4 + s_p) + m * s_key : 0.0;
    // hub edges: per-binade tables of every hub row's normalised weights (on the second
    // stream, while the other edges are scored here), then one thread per hub entry (one warp
    // per entry whose other row is long)
    std::unique_ptr<SideBranch> side;
    HubMaps hm{nullptr, nullptr, n};
    if (n_long > 0) {
        side.reset(new SideBranch(ctx));
        SPC_TRY(side->status());
        SPC_TRY(seqtab_build(ctx, W.p.p, std::is_same<P, float>::value, n_long,
                             W.lr_base.as<int64_t>(), W.lr_len.as<int64_t>(), W.tab_p));
        // column maps of the largest hubs, within 64 M entries of memory
        const int64_t maps = std::min<int64_t>(kMaxHubMaps, (int64_t(64) << 20) / (n + 1));
        if (maps > 0) {
            SPC_TRY(ensure(ctx, W.hub_map, (size_t)(maps * n + 1) * 4));
            SPC_TRY(ensure(ctx, W.hub_slot, (size_t)(n_long + kMaxHubMaps) * 4));
            int32_t* slot_of = W.hub_slot.as<int32_t>();
            int32_t* slot_hub = slot_of + n_long;
            int32_t* nslots = W.counters.as<int32_t>() + 13;
            SPC_LAUNCH(ctx, k_hub_slots, 1, 1024, 0, long_count, W.lr_len.as<int64_t>(), n,
                       (int)maps, slot_of, slot_hub, nslots);
            SPC_LAUNCH(ctx, k_hub_posmap, grid_for(maps * n, kThreads, maxb), kThreads, 0,
                       g.rowptr, g.col, long_rows, slot_hub, nslots, n, W.hub_map.as<int32_t>());
            hm = HubMaps{W.hub_map.as<int32_t>(), slot_of, n};
        }
        side->leave();
    }
    if (schedule == 3) {
        note_bytes(ctx, score_bytes);
        SPC_TRY((launch_score_stage<P, Key>(ctx, m, g, W, score, wsize, vflag, status, true)));
    } else if (schedule == 2) {
        const int warps_per_block = kThreads / 32;
        note_bytes(ctx, score_bytes);
        const int gw = grid_for(n, warps_per_block, maxb);
        SPC_LAUNCH(ctx, (k_score_warp_row<P, Key>), gw, kThreads, 0, n, g.rowptr, g.col,
                   W.p.as<P>(), W.up_ptr.as<int32_t>(), W.first_up.as<int32_t>(),
                   static_cast<Key*>(score), g.w, W.w_und.p, wsize, vflag, status,
                   op_counter(ctx, "(k_score_warp_row<P, Key>)", 2));
    } else {
        note_bytes(ctx, score_bytes);
        SPC_TRY((launch_score_edges<P, Key>(ctx, m, g, W, score, wsize, vflag, status, true)));
    }
    if (n_long == 0) return validate ? check_status(ctx) : SPC_OK;
    side.reset();  // the main stream waits for the tables
    const SeqTabView tv = seqtab_view(W.tab_p, W.lr_base.as<int64_t>(), W.lr_len.as<int64_t>());
    SPC_LAUNCH(ctx, k_hub_leaf_score<P>, grid_for(n_long, kThreads / 32, maxb), kThreads, 0,
               g.rowptr, g.col, W.p.as<P>(), long_rows, long_count, tv, W.hub_leaf.as<P>());
    SPC_LAUNCH(ctx, (k_score_hub<P, Key>), maxb, kThreads, 0, g.rowptr, g.col, W.p.as<P>(),
               W.up_ptr.as<int32_t>(), W.first_up.as<int32_t>(), long_rows, long_count,
               W.lr_eoff.as<int64_t>(), tv, hm, W.hub_leaf.as<P>(), static_cast<Key*>(score),
               W.heavy.as<int32_t>(), heavy_count, status);
    SPC_LAUNCH(ctx, (k_score_hub_heavy<P, Key>), persist, kThreads, 0, g.rowptr, g.col,
               W.p.as<P>(), W.up_ptr.as<int32_t>(), W.first_up.as<int32_t>(), long_rows,
               long_count, W.lr_eoff.as<int64_t>(), tv, hm, W.heavy.as<int32_t>(), heavy_count,
               static_cast<Key*>(score), status);
    return validate ? check_status(ctx) : SPC_OK;  // every input check, symmetry included
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
