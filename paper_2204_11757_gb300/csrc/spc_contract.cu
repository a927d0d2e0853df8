// S7: contraction into super-nodes (Definition 1), S9: its backward, and the weights-only
// forward with the assignment held fixed.
//
// For every fine undirected edge e = (u, v): U = c(u), V = c(v).  U == V: the edge is inside a
// super-node; emap[e] = -1 and its weight goes to self_mass[U].  Otherwise key(e) =
// (min(U,V), max(U,V)).  A stable radix sort of (key, eid) -- input in eid order -- groups the
// fine edges of every coarse edge with ascending eids; segment heads numbered by a scan give
// the coarse edge ids in lexicographic (U, V) order, and each coarse weight is the sequential
// sum of its segment (ascending eid, IEEE round-to-nearest), so the result is reproducible.
// The coarse CSR: row U holds first the coarse edges (V', U) with V' < U (a stable sort by
// the second end point, the "transpose") and then the edges (U, V) with V > U (contiguous in
// coarse-edge order), which leaves every row sorted.
#include <type_traits>

#include <atomic>
#include <memory>

#include "spc_scan.cuh"
#include "spc_seqsum.cuh"

namespace spc {

namespace {

template <class WT> struct CT;
template <> struct CT<int32_t> {
    using Acc = long long;
    __device__ static Acc add(Acc a, int32_t w) { return a + w; }
};
template <> struct CT<float> {
    using Acc = float;
    __device__ static Acc add(Acc a, float w) { return __fadd_rn(a, w); }
};
template <> struct CT<double> {
    using Acc = double;
    __device__ static Acc add(Acc a, double w) { return __dadd_rn(a, w); }
};

// classify fine edges: inter flag and intra flag
__global__ void __launch_bounds__(kThreads)
k_classify(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
           const int32_t* __restrict__ lift, uint8_t* __restrict__ inter,
           uint8_t* __restrict__ intra, uint32_t* __restrict__ zero_a, int64_t words_a,
           uint32_t* __restrict__ zero_b, uint32_t* __restrict__ zero_c, int64_t words_bc,
           int32_t* __restrict__ counters) {
    spc::pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e = t0; e < m; e += stride) {
        const bool x = lift[eu[e]] != lift[ev[e]];
        inter[e] = x ? 1 : 0;
        intra[e] = x ? 0 : 1;
    }
    // the accumulators the contraction adds into start at zero: the self-mass, the coarse
    // degree counts, the long-segment list counts of both streams
    for (int64_t i = t0; i < words_a; i += stride) zero_a[i] = 0u;
    for (int64_t i = t0; i < words_bc; i += stride) {
        zero_b[i] = 0u;
        zero_c[i] = 0u;
    }
    if (t0 == 0) {
        counters[9] = 0;
        counters[11] = 0;
    }
}

__global__ void __launch_bounds__(kThreads)
k_scatter_keys(int64_t m, int nb, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
               const int32_t* __restrict__ lift, const int32_t* __restrict__ inter_pos,
               const int32_t* __restrict__ intra_pos, uint64_t* __restrict__ ckey,
               uint32_t* __restrict__ cval, uint32_t* __restrict__ ikey,
               uint32_t* __restrict__ ival, int32_t* __restrict__ emap) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t U = lift[eu[e]], V = lift[ev[e]];
        if (U != V) {
            const uint64_t lo = (uint64_t)(U < V ? U : V), hi = (uint64_t)(U < V ? V : U);
            const int32_t q = inter_pos[e];
            ckey[q] = (lo << nb) | hi;
            cval[q] = (uint32_t)e;
        } else {
            const int32_t q = intra_pos[e];
            ikey[q] = (uint32_t)U;
            ival[q] = (uint32_t)e;
            emap[e] = -1;
        }
    }
}

// atomicAdd(cnt + key, 1) by every active lane (all 32 lanes call it): lanes with the same
// key (the edges of a hub super-node) add their count with one atomic
__device__ __forceinline__ void warp_count(int32_t* cnt, int32_t key, bool act) {
    const unsigned peers = __match_any_sync(0xffffffffu, act ? key : -1);
    if (act && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + key, __popc(peers));
}

// Buckets of at most kSmallBucket items: each item is ranked by one thread (at most
// kSmallBucket comparisons per item).  Longer ones are listed by the scan of the bucket sizes:
// up to kWarpBucket items, one warp ranks the bucket's items by comparison in shared memory;
// up to kBlockBucket items, one CTA sorts the bucket in shared memory (bitonic network).
constexpr int kSmallBucket = 64;
constexpr int kWarpBucket = 256;
constexpr int kBlockBucket = 8192;
constexpr int kBlockSortThreads = 512;
static_assert((kBlockSortThreads / 32) * kWarpBucket <= kBlockBucket,
              "the warps' stages share the CTA's");

// scan storer of the two packed bucket sizes (spc_scan.cuh PairLd: inter, intra): both
// exclusive prefixes and totals, and per side the ranking statistics -- sum of squared sizes in
// stats[0] / stats[2], largest size in stats[1] / stats[3] -- and the list of buckets longer
// than kSmallBucket (counts in stats[6] / stats[7]).
struct BucketOffSt {
    int32_t* off_c;
    int32_t* off_i;
    int64_t n;
    unsigned long long* stats;
    int32_t* list_c;
    int32_t* list_i;
    struct Local {
        unsigned long long sq[2], mx[2];
    };
    __device__ Local begin() const { return Local{{0ull, 0ull}, {0ull, 0ull}}; }
    __device__ void operator()(Local& L, int64_t g, bool valid, unsigned long long excl,
                               unsigned long long val) const {
        if (!valid) return;
        off_c[g] = (int32_t)(excl >> 31);
        off_i[g] = (int32_t)(excl & 0x7fffffffull);
        const unsigned long long c[2] = {val >> 31, val & 0x7fffffffull};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            L.sq[side] += c[side] * c[side];
            L.mx[side] = c[side] > L.mx[side] ? c[side] : L.mx[side];
            if (c[side] > (unsigned long long)kSmallBucket)
                (side ? list_i : list_c)[atomicAdd(stats + 6 + side, 1ull)] = (int32_t)g;
        }
    }
    __device__ void finish(Local& L) const {
        __shared__ unsigned long long sh[4];
        if (threadIdx.x < 4) sh[threadIdx.x] = 0ull;
        __syncthreads();
        for (int side = 0; side < 2; ++side) {
            if (L.sq[side]) atomicAdd(&sh[2 * side], L.sq[side]);
            if (L.mx[side]) atomicMax(&sh[2 * side + 1], L.mx[side]);
        }
        __syncthreads();
        if (threadIdx.x < 4 && sh[threadIdx.x]) {
            if (threadIdx.x & 1) atomicMax(stats + threadIdx.x, sh[threadIdx.x]);
            else atomicAdd(stats + threadIdx.x, sh[threadIdx.x]);
        }
    }
    __device__ void total(unsigned long long tot) const {
        off_c[n] = (int32_t)(tot >> 31);
        off_i[n] = (int32_t)(tot & 0x7fffffffull);
    }
};

// the same for the coarse degrees (upper, lower), plus the coarse row pointers -- row U starts
// after every upper and lower entry of the rows before it -- and the lower rows' ranking
// statistics: sum of squared sizes in stats[0], largest size in stats[1]
struct RowPtrSt {
    int32_t* ufirst;
    int32_t* lstart;
    int64_t* rowptr;
    int64_t n;
    unsigned long long* stats;
    struct Local {
        unsigned long long sq, mx;
    };
    __device__ Local begin() const { return Local{0ull, 0ull}; }
    __device__ void operator()(Local& L, int64_t g, bool valid, unsigned long long excl,
                               unsigned long long val) const {
        if (!valid) return;
        const int32_t u = (int32_t)(excl >> 31), l = (int32_t)(excl & 0x7fffffffull);
        ufirst[g] = u;
        lstart[g] = l;
        rowptr[g] = (int64_t)u + l;
        const unsigned long long low = val & 0x7fffffffull;
        L.sq += low * low;
        L.mx = low > L.mx ? low : L.mx;
    }
    __device__ void finish(Local& L) const {
        __shared__ unsigned long long sh[2];
        if (threadIdx.x < 2) sh[threadIdx.x] = 0ull;
        __syncthreads();
        if (L.sq) atomicAdd(&sh[0], L.sq);
        if (L.mx) atomicMax(&sh[1], L.mx);
        __syncthreads();
        if (threadIdx.x == 0 && sh[0]) atomicAdd(stats, sh[0]);
        if (threadIdx.x == 1 && sh[1]) atomicMax(stats + 1, sh[1]);
    }
    __device__ void total(unsigned long long tot) const {
        const int32_t u = (int32_t)(tot >> 31), l = (int32_t)(tot & 0x7fffffffull);
        ufirst[n] = u;
        lstart[n] = l;
        rowptr[n] = (int64_t)u + l;
    }
};

// ---- grouping by buckets --------------------------------------------------------------
// The coarse edges need the inter edges in (lower super-node a, upper super-node b, eid)
// order, the self-masses the intra edges in (super-node, eid) order.  Both orders are
// reached without a global sort: the items are counted per bucket (a for an inter edge, the
// super-node for an intra edge), scattered into their bucket's range in any order, and each
// item then moves to its rank within its bucket.  The ranking costs the sum over buckets of
// the squared bucket size; the host takes this path only while that stays a small multiple
// of the item count (and every bucket is short), else it sorts by radix.

// bucket of fine edge e, one 32-bit tag per (array, bucket) for warp matching: an inter edge's
// lower super-node, an intra edge's super-node with the top bit set (ids are below 2^31);
// inactive lanes all-ones
__device__ __forceinline__ uint32_t bucket_tag(int32_t U, int32_t V, bool act) {
    if (!act) return 0xffffffffu;
    return U != V ? (uint32_t)(U < V ? U : V) : (0x80000000u | (uint32_t)U);
}

// Step 1: the bucket sizes, one atomic (without a result) per group of equal buckets in a
// warp.  Also zeroes what the contraction adds into later: the coarse degree counts and the
// long-segment list counts of both streams.
__global__ void __launch_bounds__(kThreads)
k_bucket_count(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
               const int32_t* __restrict__ lift, int32_t* cnt_c, int32_t* cnt_i,
               unsigned long long* stats, uint32_t* __restrict__ zero_b,
               uint32_t* __restrict__ zero_c, int64_t words_bc, int32_t* __restrict__ counters) {
    spc::pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x; e0 < m; e0 += stride) {  // warp-uniform
        const int64_t e = e0 + threadIdx.x;
        const bool act = e < m;
        int32_t U = 0, V = 0;
        if (act) {
            U = lift[eu[e]];
            V = lift[ev[e]];
        }
        const uint32_t tag = bucket_tag(U, V, act);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        if (act && lane == __ffs(peers) - 1)
            atomicAdd((U != V ? cnt_c : cnt_i) + (tag & 0x7fffffffu), __popc(peers));
    }
    for (int64_t i = t0; i < words_bc; i += stride) {
        zero_b[i] = 0u;
        zero_c[i] = 0u;
    }
    if (t0 == 0) {
        counters[9] = 0;
        counters[11] = 0;
        stats[4] = 0ull;  // the lower rows' statistics, added by the row-pointer scan
        stats[5] = 0ull;
    }
}

// Step 2 (after the exclusive scans off_c, off_i of the sizes): every edge takes a slot of
// its bucket by counting the bucket's size down, which leaves the counts zero for the next
// call; the statistics (already read by the host) are zeroed too.  An inter edge stores one
// 16-byte item (a, b, eid, 0), an intra edge one 8-byte item (super-node, eid) and emap -1:
// one store per item.
__global__ void __launch_bounds__(kThreads)
k_bucket_scatter(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                 const int32_t* __restrict__ lift, const int32_t* __restrict__ off_c,
                 const int32_t* __restrict__ off_i, int32_t* cnt_c, int32_t* cnt_i,
                 unsigned long long* __restrict__ stats, uint4* __restrict__ citem,
                 uint2* __restrict__ iitem, int32_t* __restrict__ emap) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x < 4) stats[threadIdx.x] = 0ull;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x; e0 < m; e0 += stride) {  // warp-uniform
        const int64_t e = e0 + threadIdx.x;
        const bool act = e < m;
        int32_t U = 0, V = 0;
        if (act) {
            U = lift[eu[e]];
            V = lift[ev[e]];
        }
        const uint32_t tag = bucket_tag(U, V, act);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        const int leader = __ffs(peers) - 1;
        const bool inter = U != V;
        const int32_t b = (int32_t)(tag & 0x7fffffffu);
        int32_t old = 0;
        if (act && lane == leader) old = atomicSub((inter ? cnt_c : cnt_i) + b, __popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        if (!act) continue;
        const int below = __popc(peers & ((1u << lane) - 1u));
        const int32_t q = (inter ? off_c : off_i)[b] + old - 1 - below;
        if (inter) {
            citem[q] = make_uint4((uint32_t)b, (uint32_t)(U < V ? V : U), (uint32_t)e, 0u);
        } else {
            iitem[q] = make_uint2((uint32_t)U, (uint32_t)e);
            emap[e] = -1;
        }
    }
}

// warp sort of the items of one bucket (at most kWarpBucket, in sk[0, s)) by ranking: every
// item's rank is the number of smaller keys of the bucket (all distinct: they hold the eid).
// Each lane keeps its items (lane, lane + 32, ...) in registers and every key is read once per
// warp (a broadcast) and compared with all of them; the items then move to their ranks in the
// stage and leave it in order, with the head flag of every coarse edge's first item.
template <bool kInter, int kPer>
__device__ __forceinline__ void warp_sort_bucket(unsigned long long* sk, int s, int lane,
                                                 int32_t bkt, int32_t lo, int nb,
                                                 uint64_t* __restrict__ key2,
                                                 uint32_t* __restrict__ val2,
                                                 uint8_t* __restrict__ head) {
    unsigned long long k[kPer];
    int r[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int i = lane + 32 * t;
        k[t] = i < s ? sk[i] : ~0ull;
        r[t] = 0;
    }
    for (int j = 0; j < s; ++j) {
        const unsigned long long x = sk[j];
#pragma unroll
        for (int t = 0; t < kPer; ++t) r[t] += x < k[t] ? 1 : 0;
    }
    __syncwarp();  // every key is read: the stage takes the sorted order
#pragma unroll
    for (int t = 0; t < kPer; ++t)
        if (lane + 32 * t < s) sk[r[t]] = k[t];
    __syncwarp();
    for (int i = lane; i < s; i += 32) {
        const unsigned long long x = sk[i];
        if constexpr (kInter) {
            key2[lo + i] = ((uint64_t)bkt << nb) | (x >> 32);
            val2[lo + i] = (uint32_t)x;
            head[lo + i] = (i == 0 || (sk[i - 1] >> 32) != (x >> 32)) ? 1 : 0;
        } else {
            val2[lo + i] = (uint32_t)x;
        }
    }
}

// Step 3, long buckets (listed by the scan of the sizes), sorted by one 64-bit key -- (b << 32)
// | eid for inter edges (a is the bucket), the eid for intra edges -- and written back in
// order: inter edges as (key, eid) with their head flags, intra edges as eids.  Buckets of more
// than kWarpBucket items: one CTA each, a bitonic network over the next power of two (padding
// keys all ones) in shared memory.  The others: one warp each (warp_sort_bucket).
template <bool kInter>
__global__ void __launch_bounds__(kBlockSortThreads, 3)
k_bucket_sort_long(const int32_t* __restrict__ list, const unsigned long long* __restrict__ list_cnt,
                   const int32_t* __restrict__ off, int nb, const uint4* __restrict__ citem,
                   const uint2* __restrict__ iitem, uint64_t* __restrict__ key2,
                   uint32_t* __restrict__ val2, uint8_t* __restrict__ head) {
    spc::pdl_wait();
    extern __shared__ unsigned long long sk[];  // kBlockBucket keys
    const int64_t cnt = (int64_t)*list_cnt;
    for (int64_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int32_t bkt = list[q];
        const int32_t lo = off[bkt];
        const int s = off[bkt + 1] - lo;  // kSmallBucket < s <= kBlockBucket (host checked)
        if (s <= kWarpBucket) continue;   // a warp's bucket (below)
        int P = 1;
        while (P < s) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            unsigned long long k = ~0ull;
            if (i < s) {
                if constexpr (kInter) {
                    const uint4 it = citem[lo + i];
                    k = ((uint64_t)it.y << 32) | it.z;
                } else {
                    k = iitem[lo + i].y;
                }
            }
            sk[i] = k;
        }
        __syncthreads();
        for (int len = 2; len <= P; len <<= 1) {
            for (int j = len >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                    const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // bit j of i is 0
                    const unsigned long long x = sk[i], y = sk[i + j];
                    const bool up = (i & len) == 0;
                    if ((x > y) == up) {
                        sk[i] = y;
                        sk[i + j] = x;
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < s; i += blockDim.x) {
            const unsigned long long k = sk[i];
            if constexpr (kInter) {
                const uint64_t b = k >> 32;
                key2[lo + i] = ((uint64_t)bkt << nb) | b;
                val2[lo + i] = (uint32_t)k;
                head[lo + i] = (i == 0 || (sk[i - 1] >> 32) != b) ? 1 : 0;
            } else {
                val2[lo + i] = (uint32_t)k;
            }
        }
        __syncthreads();
    }
    // buckets of at most kWarpBucket items, one warp each, in the warp's part of the stage
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long* wk = sk + (size_t)wib * kWarpBucket;
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; q < cnt; q += nwarps) {
        const int32_t bkt = list[q];
        const int32_t lo = off[bkt];
        const int s = off[bkt + 1] - lo;
        if (s > kWarpBucket) continue;  // a CTA's bucket (above)
        for (int i = lane; i < s; i += 32) {
            if constexpr (kInter) {
                const uint4 it = citem[lo + i];
                wk[i] = ((uint64_t)it.y << 32) | it.z;
            } else {
                wk[i] = iitem[lo + i].y;
            }
        }
        __syncwarp();
        if (s <= 128)
            warp_sort_bucket<kInter, 4>(wk, s, lane, bkt, lo, nb, key2, val2, head);
        else
            warp_sort_bucket<kInter, 8>(wk, s, lane, bkt, lo, nb, key2, val2, head);
        __syncwarp();  // the next bucket overwrites the stage
    }
}

// Step 3, inter edges in short buckets: the item at p goes to its rank by (key, eid) within
// its bucket [off_c[a], off_c[a + 1]); head marks the first item (smallest eid) of every
// coarse edge.  Runs after k_bucket_sort_long, whose list it then empties.
__global__ void __launch_bounds__(kThreads)
k_bucket_rank_inter(int64_t cnt, int nb, const int32_t* __restrict__ off_c,
                    const uint4* __restrict__ citem, uint64_t* __restrict__ key2,
                    uint32_t* __restrict__ val2, uint8_t* __restrict__ head,
                    unsigned long long* __restrict__ list_cnt) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *list_cnt = 0ull;  // long buckets are sorted
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < cnt;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint4 it = citem[p];
        const uint32_t b = it.y, v = it.z;
        const int32_t lo = off_c[it.x], hi = off_c[it.x + 1];
        if (hi - lo > kSmallBucket) continue;
        int32_t r = 0;
        bool first = true;
#pragma unroll 4
        for (int32_t j = lo; j < hi; ++j) {
            const uint4 jt = citem[j];
            const bool same_before = jt.y == b && jt.z < v;
            r += (jt.y < b || same_before) ? 1 : 0;
            first = first && !same_before;
        }
        key2[lo + r] = ((uint64_t)it.x << nb) | b;
        val2[lo + r] = v;
        head[lo + r] = first ? 1 : 0;
    }
}

// Step 3, intra edges in short buckets: the eid at p goes to its rank within its super-node's
// bucket.  Runs after k_bucket_sort_long, whose list it then empties.
__global__ void __launch_bounds__(kThreads)
k_bucket_rank_intra(int64_t cnt, const int32_t* __restrict__ off_i,
                    const uint2* __restrict__ iitem, uint32_t* __restrict__ ival2,
                    unsigned long long* __restrict__ list_cnt) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *list_cnt = 0ull;  // long buckets are sorted
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < cnt;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint2 it = iitem[p];
        const uint32_t v = it.y;
        const int32_t lo = off_i[it.x], hi = off_i[it.x + 1];
        if (hi - lo > kSmallBucket) continue;
        int32_t r = 0;
#pragma unroll 4
        for (int32_t j = lo; j < hi; ++j) r += iitem[j].y < v ? 1 : 0;
        ival2[lo + r] = v;
    }
}

__global__ void k_set_i32(int32_t* p, int32_t v) {
    spc::pdl_wait();
    if (threadIdx.x == 0) *p = v;
}

template <class K>
__global__ void __launch_bounds__(kThreads)
k_heads(int64_t cnt, const K* __restrict__ key, uint8_t* __restrict__ head) {
    spc::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// coarse edge id of every sorted item; emap, perm; segment starts and end points at heads.
// Every coarse edge (U, V) also counts into up_deg[U] and low_deg[V] (result-free atomics, one
// per group of equal rows in a warp).
__global__ void __launch_bounds__(kThreads)
k_emit_segments(int64_t cnt, int nb, const uint64_t* __restrict__ key,
                const uint32_t* __restrict__ val, const uint8_t* __restrict__ head,
                const int32_t* __restrict__ hpos, int32_t* __restrict__ emap,
                int32_t* __restrict__ perm, int32_t* __restrict__ seg, int32_t* __restrict__ cU,
                int32_t* __restrict__ cV, int32_t* up_deg, int32_t* low_deg) {
    spc::pdl_wait();
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt;
         i0 += (int64_t)gridDim.x * blockDim.x) {  // warp-uniform
        const int64_t i = i0 + threadIdx.x;
        const bool act = i < cnt;
        bool h = false;
        int32_t U = 0, V = 0;
        if (act) {
            const int32_t ce = hpos[i] + head[i] - 1;
            const uint32_t e = val[i];
            emap[e] = ce;
            perm[i] = (int32_t)e;
            h = head[i] != 0;
            if (h) {
                seg[ce] = (int32_t)i;
                const uint64_t k = key[i];
                U = (int32_t)(k >> nb);
                V = (int32_t)(k & ((1ull << nb) - 1ull));
                cU[ce] = U;
                cV[ce] = V;
            }
        }
        warp_count(up_deg, U, h);
        warp_count(low_deg, V, h);
    }
}

// run r of a sorted key array starts at start[r]; start[n_runs] = cnt
__global__ void __launch_bounds__(kThreads)
k_run_starts(int64_t cnt, const uint8_t* __restrict__ head, const int32_t* __restrict__ hpos,
             int32_t* __restrict__ start) {
    spc::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (head[i]) start[hpos[i]] = (int32_t)i;
        if (i == cnt - 1) start[hpos[i] + head[i]] = (int32_t)cnt;
    }
}

// Segment sums: out[slot(r)] = sum of w_und[idx[j]] for j in [start[r], start[r+1]), left to
// right.  slot(r) = r, or key[start[r]] when `key` is given (self-mass by super-node).  Short
// segments: one thread each; segments longer than kLongRow go to a list for k_segsum_long.
template <class WT, class Out>
__global__ void __launch_bounds__(kThreads)
k_segsum_short(int64_t nseg, const int32_t* __restrict__ start, const uint32_t* __restrict__ idx,
               const uint32_t* __restrict__ key, const WT* __restrict__ w_und, Out* __restrict__ out,
               int32_t* __restrict__ long_list, int32_t* __restrict__ long_count,
               uint32_t* status) {
    spc::pdl_wait();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nseg;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j0 = start[r], j1 = start[r + 1];
        if (j1 - j0 > kLongRow) {
            long_list[atomicAdd(long_count, 1)] = (int32_t)r;
            continue;
        }
        typename CT<WT>::Acc s = 0;
        if (j1 - j0 <= 4) {
            // short segment: every index and term in flight before the left-to-right sum
            uint32_t ix[4];
            WT t[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < j1) ix[q] = idx[j0 + q];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < j1) t[q] = w_und[ix[q]];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + q < j1) s = CT<WT>::add(s, t[q]);
        } else {
            for (int32_t j = j0; j < j1; ++j) s = CT<WT>::add(s, w_und[idx[j]]);
        }
        if constexpr (std::is_same<WT, int32_t>::value && sizeof(Out) == 4) {
            if (s > 2147483647ll) atomicOr(status, DEV_OVERFLOW);
        }
        out[key ? (int64_t)key[j0] : r] = (Out)s;
    }
}

template <class WT, class Out>
__global__ void __launch_bounds__(kThreads)
k_segsum_long(const int32_t* __restrict__ start, const uint32_t* __restrict__ idx,
              const uint32_t* __restrict__ key, const WT* __restrict__ w_und, Out* __restrict__ out,
              const int32_t* __restrict__ long_list, const int32_t* __restrict__ long_count,
              uint32_t* status) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    for (int32_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int64_t r = long_list[q];
        const int32_t j0 = start[r], j1 = start[r + 1];
        // integer weights only (exact in any order); floating-point long segments go through
        // the per-binade tables (long_segment_sums)
        static_assert(std::is_same<WT, int32_t>::value, "integer weights only");
        const long long s =
            cta_sum_i64(j1 - j0, [&](int64_t k) { return (long long)w_und[idx[j0 + k]]; });
        if (threadIdx.x == 0) {
            if constexpr (sizeof(Out) == 4) {
                if (s > 2147483647ll) atomicOr(status, DEV_OVERFLOW);
            }
            out[key ? (int64_t)key[j0] : r] = (Out)s;
        }
        __syncthreads();
    }
}

// long segment q (segment r = long_list[q]): its length, and the slot its sum goes to
__global__ void k_long_seg_prep(const int32_t* __restrict__ long_list,
                                const int32_t* __restrict__ long_count,
                                const int32_t* __restrict__ start, const uint32_t* __restrict__ key,
                                int64_t* __restrict__ len, int64_t* __restrict__ out_idx) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
        const int32_t r = long_list[q];
        len[q] = start[r + 1] - start[r];
        out_idx[q] = key ? (int64_t)key[start[r]] : (int64_t)r;
    }
}

// the terms of all long segments, gathered contiguously (segment q at base[q])
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_gather_long_terms(const int32_t* __restrict__ long_list, const int32_t* __restrict__ long_count,
                    const int32_t* __restrict__ start, const uint32_t* __restrict__ idx,
                    const WT* __restrict__ w_und, const int64_t* __restrict__ base,
                    WT* __restrict__ terms) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    const int64_t total = base[cnt];
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (base[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int32_t r = long_list[lo];
        terms[f] = w_und[idx[start[r] + (f - base[lo])]];
    }
}

// lower rows by radix sort: key V, value the coarse edge id
__global__ void __launch_bounds__(kThreads)
k_transpose_keys(int64_t m_c, const int32_t* __restrict__ cV, uint32_t* __restrict__ tkey,
                 uint32_t* __restrict__ tval) {
    spc::pdl_wait();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m_c;
         k += (int64_t)gridDim.x * blockDim.x) {
        tkey[k] = (uint32_t)cV[k];
        tval[k] = (uint32_t)k;
    }
}

// lower rows by buckets, step 1: coarse edge k takes a slot of row V's lower range by counting
// low_deg[V] down (zero afterwards)
__global__ void __launch_bounds__(kThreads)
k_lower_scatter(int64_t m_c, const int32_t* __restrict__ cV, const int32_t* __restrict__ lstart,
                int32_t* low_deg, uint32_t* __restrict__ slot) {
    spc::pdl_wait();
    const int lane = threadIdx.x & 31;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x; k0 < m_c;
         k0 += (int64_t)gridDim.x * blockDim.x) {  // warp-uniform
        const int64_t k = k0 + threadIdx.x;
        const bool act = k < m_c;
        const int32_t V = act ? cV[k] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, V);
        const int leader = __ffs(peers) - 1;
        int32_t old = 0;
        if (act && lane == leader) old = atomicSub(low_deg + V, __popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        if (act) slot[lstart[V] + old - 1 - __popc(peers & ((1u << lane) - 1u))] = (uint32_t)k;
    }
}

// lower rows by buckets, step 2 (rows of at most kLowerRowThread entries): one thread per row V
// ranks the row's coarse edges by id (the order of U) among the row's slots, which it reads
// contiguously, and writes the row's lower entries; longer rows are listed for
// k_fill_lower_long.
constexpr int32_t kLowerRowThread = 32;

template <class WT>
__global__ void __launch_bounds__(kThreads)
k_fill_lower_rows(int64_t n_c, const uint32_t* __restrict__ slot,
                  const int32_t* __restrict__ lstart, const int64_t* __restrict__ rowptr_c,
                  const int32_t* __restrict__ cU, const WT* __restrict__ a_und,
                  int32_t* __restrict__ col_c, WT* __restrict__ w_c,
                  int32_t* __restrict__ long_rows, int32_t* long_count) {
    spc::pdl_wait();
    for (int64_t V = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; V < n_c;
         V += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lo = lstart[V], hi = lstart[V + 1];
        if (hi - lo > kLowerRowThread) {
            long_rows[atomicAdd(long_count, 1)] = (int32_t)V;
            continue;
        }
        const int64_t base = rowptr_c[V];
        for (int32_t p = lo; p < hi; ++p) {
            const uint32_t k = slot[p];
            int32_t r = 0;
            for (int32_t j = lo; j < hi; ++j) r += slot[j] < k ? 1 : 0;
            col_c[base + r] = cU[k];
            w_c[base + r] = a_und[k];
        }
    }
}

// lower rows longer than kLowerRowThread entries: one warp per listed row, lanes over its slots
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_fill_lower_long(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ long_count,
                  const uint32_t* __restrict__ slot, const int32_t* __restrict__ lstart,
                  const int64_t* __restrict__ rowptr_c, const int32_t* __restrict__ cU,
                  const WT* __restrict__ a_und, int32_t* __restrict__ col_c,
                  WT* __restrict__ w_c) {
    spc::pdl_wait();
    const int32_t cnt = *long_count;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < cnt;
         q += nwarps) {
        const int32_t V = long_rows[q];
        const int32_t lo = lstart[V], hi = lstart[V + 1];
        const int64_t base = rowptr_c[V];
        for (int32_t p = lo + lane; p < hi; p += 32) {
            const uint32_t k = slot[p];
            int32_t r = 0;
            for (int32_t j = lo; j < hi; ++j) r += slot[j] < k ? 1 : 0;
            col_c[base + r] = cU[k];
            w_c[base + r] = a_und[k];
        }
    }
}

// row V, lower part: coarse edges (U, V), U < V, in transpose-sorted order
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_fill_lower(int64_t m_c, const uint32_t* __restrict__ tkey, const uint32_t* __restrict__ tval,
             const int32_t* __restrict__ lstart, const int64_t* __restrict__ rowptr_c,
             const int32_t* __restrict__ cU, const WT* __restrict__ a_und,
             int32_t* __restrict__ col_c, WT* __restrict__ w_c) {
    spc::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_c;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t V = tkey[i], k = tval[i];
        const int64_t pos = rowptr_c[V] + (i - lstart[V]);
        col_c[pos] = cU[k];
        w_c[pos] = a_und[k];
    }
}

// row U, upper part: coarse edges (U, V), V > U, contiguous in coarse-edge order
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_fill_upper(int64_t m_c, const int32_t* __restrict__ cU, const int32_t* __restrict__ cV,
             const int32_t* __restrict__ lstart, const WT* __restrict__ a_und,
             int32_t* __restrict__ col_c, WT* __restrict__ w_c) {
    spc::pdl_wait();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m_c;
         k += (int64_t)gridDim.x * blockDim.x) {
        // row U starts at ufirst[U] + lstart[U]; its lower part has lstart[U+1] - lstart[U]
        // entries, then its upper entries in coarse-edge order from k = ufirst[U]
        const int32_t U = cU[k];
        const int64_t pos = (int64_t)lstart[U + 1] + k;
        col_c[pos] = cV[k];
        w_c[pos] = a_und[k];
    }
}

template <class WT>
__global__ void __launch_bounds__(kThreads)
k_backward(int64_t m, const int32_t* __restrict__ emap, const WT* __restrict__ grad_a,
           WT* __restrict__ grad_w) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = emap[e];
        grad_w[e] = k >= 0 ? grad_a[k] : WT(0);
    }
}

// Sums of the segments that k_segsum_short left to the long list: integer weights by CTA
// reductions, floating point by per-binade tables (exact left-to-right sums).
template <class WT, class Out>
spc_status long_segment_sums(spc_context* ctx, const int32_t* start, const uint32_t* idx,
                             const uint32_t* key, const WT* w_und, Out* out) {
    Work& W = ctx->work;
    const bool side = on_side(ctx);
    int32_t* long_list = (side ? W.long_segs_side : W.long_segs).as<int32_t>();
    int32_t* long_cnt = W.counters.as<int32_t>() + (side ? 11 : 9);
    if constexpr (std::is_same<WT, int32_t>::value) {
        SPC_LAUNCH(ctx, (k_segsum_long<WT, Out>), ctx->num_sms * 2, kThreads, 0, start, idx, key,
                   w_und, out, long_list, long_cnt, ctx->d_status);
        return SPC_OK;
    } else {
        int64_t nlong = 0;
        SPC_TRY(read_i32(ctx, long_cnt, &nlong));
        if (nlong == 0) return SPC_OK;
        int64_t* len = (side ? W.seg_len_side : W.seg_len).as<int64_t>();
        int64_t* base = (side ? W.seg_base_side : W.seg_base).as<int64_t>();
        int64_t* oidx = (side ? W.seg_idx_side : W.seg_idx).as<int64_t>();
        SPC_LAUNCH(ctx, k_long_seg_prep, grid_for(nlong, kThreads, ctx->num_sms * 8), kThreads, 0,
                   long_list, long_cnt, start, key, len, oidx);
        SPC_TRY(scan_i64_i64(ctx, len, base, nlong));
        int64_t total = 0;
        SPC_TRY(read_i64(ctx, base + nlong, &total));
        Buf& tbuf = side ? W.seg_terms_side : W.seg_terms;
        SPC_TRY(ensure(ctx, tbuf, (size_t)(total + 1) * sizeof(WT)));
        WT* terms = tbuf.as<WT>();
        SPC_LAUNCH(ctx, k_gather_long_terms<WT>, grid_for(total, kThreads, ctx->num_sms * 8),
                   kThreads, 0, long_list, long_cnt, start, idx, w_und, base, terms);
        const bool f32 = std::is_same<WT, float>::value;
        SeqTabBufs& tab = side ? W.tab_s_side : W.tab_s;
        SPC_TRY(seqtab_full(ctx, terms, f32, nlong, base, len, oidx, out, tab));
        return SPC_OK;
    }
}

// The lower rows of the coarse CSR take the bucket path while every row holds at most
// kRankMax lower entries and the ranking work (the sum of squared row sizes) is at most
// kRankWork per coarse edge; the inter and intra buckets while none is longer than
// kBlockBucket.
constexpr int64_t kRankMax = 1024;
constexpr int64_t kRankWork = 48;

// one CTA per long bucket, each with kBlockBucket keys of shared memory
static spc_status sort_long_buckets(spc_context* ctx, bool inter, const int32_t* list,
                                    const unsigned long long* list_cnt, const int32_t* off,
                                    int nb, const uint4* citem, const uint2* iitem,
                                    uint64_t* key2, uint32_t* val2, uint8_t* head) {
    constexpr int smem = kBlockBucket * 8;
    static std::atomic<unsigned long long> attr_devs{0};  // devices already set up
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(attr_devs.load() & bit)) {
        SPC_CUDA(cudaFuncSetAttribute(k_bucket_sort_long<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        SPC_CUDA(cudaFuncSetAttribute(k_bucket_sort_long<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr_devs.fetch_or(bit);
    }
    const int grid = ctx->num_sms * 3;
    if (inter) {
        SPC_LAUNCH(ctx, k_bucket_sort_long<true>, grid, kBlockSortThreads, smem, list, list_cnt,
                   off, nb, citem, iitem, key2, val2, head);
    } else {
        SPC_LAUNCH(ctx, k_bucket_sort_long<false>, grid, kBlockSortThreads, smem, list, list_cnt,
                   off, nb, citem, iitem, key2, val2, head);
    }
    return SPC_OK;
}

template <class WT>
spc_status contract_typed(spc_context* ctx, const GraphView& g, const int32_t* lift,
                          int64_t n_c, LevelBufs& lv) {
    using Acc = typename CT<WT>::Acc;
    Work& W = ctx->work;
    const int64_t m = g.m;
    const int maxb = ctx->num_sms * 8;
    uint32_t* status = ctx->d_status;
    int nb = 1;
    while ((1ll << nb) < n_c) ++nb;
    const int gm = grid_for(m, kThreads, maxb);
    Acc* self_mass = lv.self_mass.as<Acc>();
    int32_t* up_deg = W.up_deg.as<int32_t>();
    int32_t* low_deg = W.low_deg.as<int32_t>();
    uint64_t* ckey = W.c_key.as<uint64_t>();
    uint32_t* cval = W.c_val.as<uint32_t>();
    uint32_t* ikey = W.i_key.as<uint32_t>();
    uint32_t* ival = W.i_val.as<uint32_t>();
    int32_t* emap = lv.emap.as<int32_t>();
    // the bucket path's scattered items, one store each
    SPC_TRY(ensure(ctx, W.c_item, (size_t)(m + 1) * 16));
    SPC_TRY(ensure(ctx, W.i_item, (size_t)(m + 1) * 8));
    uint4* citem = W.c_item.as<uint4>();
    uint2* iitem = W.i_item.as<uint2>();
    // ---- bucket sizes, offsets and ranking work ------------------------------------------
    // the counts are zero between calls (the scatter counts them down); a call that stopped
    // in between leaves them dirty
    int32_t* cnt_c = W.b_cnt.as<int32_t>();
    int32_t* cnt_i = cnt_c + (n_c + 1);
    int32_t* off_c = W.b_off.as<int32_t>();
    int32_t* off_i = off_c + (n_c + 1);
    unsigned long long* bstats = W.b_stats.as<unsigned long long>();
    int32_t* list_c = W.b_list.as<int32_t>();  // long buckets (at most m / kSmallBucket each)
    int32_t* list_i = list_c + (m / kSmallBucket + 1);
    if (W.b_dirty) {
        SPC_CUDA(cudaMemsetAsync(W.b_cnt.p, 0, W.b_cnt.bytes, ctx->stream));
        SPC_CUDA(cudaMemsetAsync(W.b_stats.p, 0, W.b_stats.bytes, ctx->stream));
    }
    W.b_dirty = true;
    SPC_LAUNCH(ctx, k_bucket_count, gm, kThreads, 0, m, W.eu.as<int32_t>(), W.ev.as<int32_t>(),
               lift, cnt_c, cnt_i, bstats, reinterpret_cast<uint32_t*>(up_deg),
               reinterpret_cast<uint32_t*>(low_deg), (int64_t)(n_c + 1),
               W.counters.as<int32_t>());
    SPC_TRY(scan_fused<unsigned long long>(
        ctx, n_c, PairLd{cnt_c, cnt_i}, BucketOffSt{off_c, off_i, n_c, bstats, list_c, list_i},
        (double)n_c * 16.0));
    int64_t bv[8];
    {
        const void* ptrs[8] = {off_c + n_c, off_i + n_c, bstats, bstats + 1, bstats + 2,
                               bstats + 3, bstats + 6, bstats + 7};
        const int bytes[8] = {4, 4, 8, 8, 8, 8, 8, 8};
        SPC_TRY(read_vals(ctx, 8, ptrs, bytes, bv));
    }
    const int64_t long_c = bv[6], long_i = bv[7];  // buckets longer than kSmallBucket
    const int64_t m_inter = bv[0];
    const int64_t m_intra = bv[1];
    const bool buckets = bv[3] <= kBlockBucket && bv[5] <= kBlockBucket;
    if (buckets) {
        if (m > 0) {
            SPC_LAUNCH(ctx, k_bucket_scatter, gm, kThreads, 0, m, W.eu.as<int32_t>(),
                       W.ev.as<int32_t>(), lift, off_c, off_i, cnt_c, cnt_i, bstats, citem,
                       iitem, emap);
        }
    } else {
        SPC_CUDA(cudaMemsetAsync(cnt_c, 0, (size_t)(n_c + 1) * 8, ctx->stream));
        SPC_CUDA(cudaMemsetAsync(W.b_stats.p, 0, W.b_stats.bytes, ctx->stream));
        // radix path: compaction by flag scans (self-mass zeroed here, all its sums add in)
        uint8_t* inter = W.c_flag.as<uint8_t>();
        uint8_t* intra = inter + (m + 1);
        int32_t* inter_pos = W.c_pos.as<int32_t>();
        int32_t* intra_pos = W.c_head.as<int32_t>();
        SPC_LAUNCH(ctx, k_classify, gm, kThreads, 0, m, W.eu.as<int32_t>(), W.ev.as<int32_t>(),
                   lift, inter, intra, reinterpret_cast<uint32_t*>(self_mass),
                   (int64_t)(n_c * sizeof(Acc) / 4), reinterpret_cast<uint32_t*>(up_deg),
                   reinterpret_cast<uint32_t*>(low_deg), (int64_t)(n_c + 1),
                   W.counters.as<int32_t>());
        SPC_TRY(scan_flags_u8(ctx, inter, inter_pos, m));
        SPC_TRY(scan_flags_u8(ctx, intra, intra_pos, m));
        if (m > 0) {
            SPC_LAUNCH(ctx, k_scatter_keys, gm, kThreads, 0, m, nb, W.eu.as<int32_t>(),
                       W.ev.as<int32_t>(), lift, inter_pos, intra_pos, ckey, cval, ikey, ival,
                       emap);
        }
    }
    W.b_dirty = false;
    // The self-mass (intra edges) and the coarse edges are independent from here: the
    // self-mass runs on the second stream with its own temporaries, the coarse edges here.
    SPC_TRY(ensure(ctx, W.long_segs_side, (size_t)(m + 1) * 4));
    SPC_TRY(ensure(ctx, W.seg_len_side, (size_t)(m + 1) * 8));
    SPC_TRY(ensure(ctx, W.seg_base_side, (size_t)(m + 2) * 8));
    SPC_TRY(ensure(ctx, W.seg_idx_side, (size_t)(m + 1) * 8));
    std::unique_ptr<SideBranch> side(new SideBranch(ctx));
    SPC_TRY(side->status());
    if (buckets) {
        // self-mass of super-node U: its bucket, in eid order (empty buckets give zero)
        uint32_t* ival2 = W.i_val2.as<uint32_t>();
        if (m_intra > 0) {
            if (long_i > 0)
                SPC_TRY(sort_long_buckets(ctx, false, list_i, bstats + 7, off_i, nb, nullptr,
                                          iitem, nullptr, ival2, nullptr));
            SPC_LAUNCH(ctx, k_bucket_rank_intra, grid_for(m_intra, kThreads, maxb), kThreads, 0,
                       m_intra, off_i, iitem, ival2, bstats + 7);
        }
        SPC_LAUNCH(ctx, (k_segsum_short<WT, Acc>), grid_for(n_c, kThreads, maxb), kThreads, 0,
                   n_c, off_i, ival2, nullptr, W.w_und.as<WT>(), self_mass,
                   W.long_segs_side.as<int32_t>(), W.counters.as<int32_t>() + 11, status);
        SPC_TRY((long_segment_sums<WT, Acc>(ctx, off_i, ival2, nullptr, W.w_und.as<WT>(),
                                             self_mass)));
    } else {
        // self-mass: runs of equal super-node ids after a stable sort, summed in eid order
        SPC_TRY(radix_sort_u32(ctx, ikey, ival, W.i_key2.as<uint32_t>(),
                               W.i_val2.as<uint32_t>(), m_intra, nb));
        if (m_intra > 0) {
            int32_t* long_list = W.long_segs_side.as<int32_t>();
            int32_t* long_cnt = W.counters.as<int32_t>() + 11;
            uint8_t* ihead = W.c_flag.as<uint8_t>() + (m + 1);  // intra flags are consumed
            int32_t* ihpos = W.c_head.as<int32_t>();
            int32_t* istart = W.i_key2.as<int32_t>();           // sort scratch is free again
            const int gi = grid_for(m_intra, kThreads, maxb);
            SPC_LAUNCH(ctx, k_heads<uint32_t>, gi, kThreads, 0, m_intra, ikey, ihead);
            SPC_TRY(scan_flags_u8(ctx, ihead, ihpos, m_intra));
            SPC_LAUNCH(ctx, k_run_starts, gi, kThreads, 0, m_intra, ihead, ihpos, istart);
            int64_t n_runs = 0;
            SPC_TRY(read_i32(ctx, ihpos + m_intra, &n_runs));
            SPC_LAUNCH(ctx, (k_segsum_short<WT, Acc>), grid_for(n_runs, kThreads, maxb),
                       kThreads, 0, n_runs, istart, ival, ikey, W.w_und.as<WT>(), self_mass,
                       long_list, long_cnt, status);
            SPC_TRY((long_segment_sums<WT, Acc>(ctx, istart, ival, ikey, W.w_und.as<WT>(),
                                                 self_mass)));
        }
    }
    side->leave();
    // coarse edges: the inter edges in (a, b, eid) order with a head flag per coarse edge
    int32_t* long_list = W.long_segs.as<int32_t>();
    int32_t* long_cnt = W.counters.as<int32_t>() + 9;
    uint8_t* head = W.c_flag.as<uint8_t>();  // flags are consumed; reuse as heads
    int32_t* hpos = W.c_pos.as<int32_t>();
    const uint64_t* skey = ckey;
    const uint32_t* sval = cval;
    if (buckets) {
        if (m_inter > 0) {
            if (long_c > 0)
                SPC_TRY(sort_long_buckets(ctx, true, list_c, bstats + 6, off_c, nb, citem,
                                          nullptr, W.c_key2.as<uint64_t>(),
                                          W.c_val2.as<uint32_t>(), head));
            SPC_LAUNCH(ctx, k_bucket_rank_inter, grid_for(m_inter, kThreads, maxb), kThreads, 0,
                       m_inter, nb, off_c, citem, W.c_key2.as<uint64_t>(),
                       W.c_val2.as<uint32_t>(), head, bstats + 6);
        }
        skey = W.c_key2.as<uint64_t>();
        sval = W.c_val2.as<uint32_t>();
    } else {
        SPC_TRY(radix_sort_u64(ctx, ckey, cval, W.c_key2.as<uint64_t>(), W.c_val2.as<uint32_t>(),
                               m_inter, 2 * nb));
        if (m_inter > 0) {
            SPC_LAUNCH(ctx, k_heads<uint64_t>, grid_for(m_inter, kThreads, maxb), kThreads, 0,
                       m_inter, ckey, head);
        }
    }
    int32_t* seg = lv.seg.as<int32_t>();
    int32_t* perm = lv.perm.as<int32_t>();
    int32_t* cU = W.cU.as<int32_t>();
    int32_t* cV = W.cV.as<int32_t>();
    int64_t m_c = 0;
    bool lower_buckets = true;
    if (m_inter > 0) {
        const int gi = grid_for(m_inter, kThreads, maxb);
        SPC_TRY(scan_flags_u8(ctx, head, hpos, m_inter));
        SPC_LAUNCH(ctx, k_emit_segments, gi, kThreads, 0, m_inter, nb, skey, sval, head, hpos,
                   emap, perm, seg, cU, cV, up_deg, low_deg);
    }
    // coarse CSR: row U holds its lower entries (coarse edges (U', U), ascending U') and then
    // its upper entries (coarse edges (U, V), contiguous in coarse-edge order)
    int32_t* ufirst = W.ufirst.as<int32_t>();
    int32_t* lstart = W.lstart.as<int32_t>();
    int64_t* rowptr_c = lv.rowptr_c.as<int64_t>();
    SPC_TRY(scan_fused<unsigned long long>(ctx, n_c, PairLd{up_deg, low_deg},
                                           RowPtrSt{ufirst, lstart, rowptr_c, n_c, bstats + 4},
                                           (double)n_c * 24.0));
    if (m_inter > 0) {
        int64_t ev[3];
        const void* ptrs[3] = {hpos + m_inter, bstats + 4, bstats + 5};
        const int bytes[3] = {4, 8, 8};
        SPC_TRY(read_vals(ctx, 3, ptrs, bytes, ev));
        m_c = ev[0];
        lower_buckets = ev[2] <= kRankMax && ev[1] <= kRankWork * m_c;
    }
    SPC_LAUNCH(ctx, k_set_i32, 1, 32, 0, seg + m_c, (int32_t)m_inter);
    WT* a_und = lv.a_und.as<WT>();
    if (m_c > 0) {
        SPC_LAUNCH(ctx, (k_segsum_short<WT, WT>), grid_for(m_c, kThreads, maxb), kThreads, 0,
                   m_c, seg, reinterpret_cast<const uint32_t*>(perm), nullptr, W.w_und.as<WT>(),
                   a_und, long_list, long_cnt, status);
        SPC_TRY((long_segment_sums<WT, WT>(ctx, seg, reinterpret_cast<const uint32_t*>(perm),
                                            nullptr, W.w_und.as<WT>(), a_und)));
    }
    if (m_c > 0) {
        const int gc = grid_for(m_c, kThreads, maxb);
        uint32_t* tkey = W.t_key.as<uint32_t>();
        uint32_t* tval = W.t_val.as<uint32_t>();
        if (lower_buckets) {
            SPC_LAUNCH(ctx, k_lower_scatter, gc, kThreads, 0, m_c, cV, lstart, low_deg, tval);
            int32_t* lrows = W.t_key.as<int32_t>();  // free on the bucket path
            int32_t* lcount = W.lower_long.as<int32_t>();
            SPC_CUDA(cudaMemsetAsync(lcount, 0, sizeof(int32_t), ctx->stream));
            SPC_LAUNCH(ctx, k_fill_lower_rows<WT>, grid_for(n_c, kThreads, maxb), kThreads, 0,
                       n_c, tval, lstart, rowptr_c, cU, a_und, lv.col_c.as<int32_t>(),
                       lv.w_c.as<WT>(), lrows, lcount);
            SPC_LAUNCH(ctx, k_fill_lower_long<WT>, ctx->num_sms * 2, kThreads, 0, lrows, lcount,
                       tval, lstart, rowptr_c, cU, a_und, lv.col_c.as<int32_t>(),
                       lv.w_c.as<WT>());
        } else {
            SPC_LAUNCH(ctx, k_transpose_keys, gc, kThreads, 0, m_c, cV, tkey, tval);
            SPC_TRY(radix_sort_u32(ctx, tkey, tval, W.t_key2.as<uint32_t>(),
                                   W.t_val2.as<uint32_t>(), m_c, nb));
            SPC_LAUNCH(ctx, k_fill_lower<WT>, gc, kThreads, 0, m_c, tkey, tval, lstart, rowptr_c,
                       cU, a_und, lv.col_c.as<int32_t>(), lv.w_c.as<WT>());
        }
        SPC_LAUNCH(ctx, k_fill_upper<WT>, gc, kThreads, 0, m_c, cU, cV, lstart, a_und,
                   lv.col_c.as<int32_t>(), lv.w_c.as<WT>());
    }
    lv.m_c = m_c;
    lv.m_inter = m_inter;
    lv.n_c = n_c;
    return SPC_OK;
}

template <class WT>
spc_status forward_typed(spc_context* ctx, const int32_t* perm, const int32_t* seg, int64_t m_c,
                         const WT* w_und, WT* a_und) {
    if (m_c <= 0) return SPC_OK;
    Work& W = ctx->work;
    const size_t M = (size_t)m_c + 1;
    SPC_TRY(ensure(ctx, W.long_segs, M * 4));
    SPC_TRY(ensure(ctx, W.counters, 64 * 4));
    SPC_TRY(ensure(ctx, W.seg_len, M * 8));
    SPC_TRY(ensure(ctx, W.seg_base, (M + 1) * 8));
    SPC_TRY(ensure(ctx, W.seg_idx, M * 8));
    int32_t* long_list = W.long_segs.as<int32_t>();
    int32_t* long_cnt = W.counters.as<int32_t>() + 9;
    SPC_CUDA(cudaMemsetAsync(long_cnt, 0, sizeof(int32_t), ctx->stream));
    SPC_LAUNCH(ctx, (k_segsum_short<WT, WT>), grid_for(m_c, kThreads, ctx->num_sms * 8), kThreads,
               0, m_c, seg, reinterpret_cast<const uint32_t*>(perm), nullptr, w_und, a_und,
               long_list, long_cnt, ctx->d_status);
    return long_segment_sums<WT, WT>(ctx, seg, reinterpret_cast<const uint32_t*>(perm), nullptr,
                                     w_und, a_und);
}

// ---- the self-mass reading of the multilevel driver ----------------------------------------
// Under this reading a super-node keeps the weight inside it.  The proof of Theorem 2 treats the
// merged node as (w_a + w_b) / (d_a + d_b): its own coordinate holds w_ab + w_ba and its degree
// keeps the internal weight.  The next level's input graph therefore holds, for every
// super-node U with mass(U) != 0, the diagonal entry 2 mass(U) in its ascending-column place,
// where mass(U) is U's accumulated internal weight: the masses of its members (ascending member
// id, summed left to right from 0) plus the weight of this level's edges inside U (the
// contraction's self-mass).  Degrees and scores of that graph follow with no other change.

// members of every super-node in ascending id: a stable sort of (lift[x], x) by lift
__global__ void __launch_bounds__(kThreads)
k_member_keys(int64_t n, const int32_t* __restrict__ lift, uint32_t* __restrict__ key,
              uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        key[x] = (uint32_t)lift[x];
        val[x] = (uint32_t)x;
    }
}

// start[U] = first sorted position of U's members; start[n_c] = n.  Every super-node of a
// relabelled lift has at least one member.
__global__ void __launch_bounds__(kThreads)
k_member_starts(int64_t n, int64_t n_c, const uint32_t* __restrict__ key,
                int32_t* __restrict__ start) {
    spc::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t U = key[i];
        if (i == 0 || key[i - 1] != U) start[U] = (int32_t)i;
        if (i == n - 1) start[n_c] = (int32_t)n;
    }
}

// mass[U] = (sum of the members' masses) + self_mass[U], one IEEE addition
template <class WT>
__global__ void __launch_bounds__(kThreads)
k_mass_add_self(int64_t n_c, const WT* __restrict__ self, WT* __restrict__ mass) {
    spc::pdl_wait();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        mass[u] = CT<WT>::add(mass[u], self[u]);
}

// integer weights (int64 masses): exact in any order, so the members' masses are added by
// atomics onto the self-mass
__global__ void __launch_bounds__(kThreads)
k_mass_int_init(int64_t n_c, const long long* __restrict__ self, long long* __restrict__ mass) {
    spc::pdl_wait();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_c;
         u += (int64_t)gridDim.x * blockDim.x)
        mass[u] = self[u];
}

__global__ void __launch_bounds__(kThreads)
k_mass_int_add(int64_t n, const int32_t* __restrict__ lift, const long long* __restrict__ prev,
               long long* mass) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const long long v = prev[x];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(mass + lift[x]),
                         (unsigned long long)v);
    }
}

// diagonal flags scanned in one pass: pos[x] = #{y < x : mass[y] != 0} (pos[n] = the count),
// and the new row pointers rowptr[x] + pos[x]
template <class AT>
struct DiagLd {
    const AT* mass;
    __device__ unsigned long long operator()(int64_t g) const {
        return mass[g] != AT(0) ? 1ull : 0ull;
    }
};

struct DiagSt {
    const int64_t* rowptr;
    int64_t* rowptr_d;
    int32_t* pos;
    int64_t n;
    struct Local {};
    __device__ Local begin() const { return Local{}; }
    __device__ void operator()(Local&, int64_t g, bool valid, unsigned long long excl,
                               unsigned long long) const {
        if (!valid) return;
        pos[g] = (int32_t)excl;
        rowptr_d[g] = rowptr[g] + (int64_t)excl;
    }
    __device__ void finish(Local&) const {}
    __device__ void total(unsigned long long tot) const {
        pos[n] = (int32_t)tot;
        rowptr_d[n] = rowptr[n] + (int64_t)tot;
    }
};

// every stored entry moves up by the diagonal entries before it: those of the rows above its
// row, and its own row's when the entry's column is above the diagonal.  Each block takes
// kDiagTile consecutive entries and marks their rows in shared memory (tile_rows).
constexpr int64_t kDiagTile = 2048;

template <class WT>
__global__ void __launch_bounds__(kThreads)
k_diag_entries(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
               const int32_t* __restrict__ col, const WT* __restrict__ w,
               const int32_t* __restrict__ pos, int32_t* __restrict__ col_d,
               WT* __restrict__ w_d) {
    spc::pdl_wait();
    __shared__ int64_t s_rows[2];
    __shared__ int32_t s_row[kDiagTile];
    for (int64_t base = (int64_t)blockIdx.x * kDiagTile; base < nnz;
         base += (int64_t)gridDim.x * kDiagTile) {
        const int64_t end = base + kDiagTile < nnz ? base + kDiagTile : nnz;
        const int64_t r_lo = tile_rows(rowptr, n, base, end, -1, s_row, s_rows);
        for (int64_t j = base + threadIdx.x; j < end; j += blockDim.x) {
            const int64_t x = r_lo + s_row[j - base];
            const int32_t y = col[j];
            const int32_t p0 = pos[x];
            const int64_t d = (int64_t)p0 + ((pos[x + 1] > p0 && (int64_t)y > x) ? 1 : 0);
            col_d[j + d] = y;
            w_d[j + d] = w[j];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int32_t diag_weight(long long m, uint32_t* status) {
    const long long v = 2 * m;
    if (v > 2147483647ll) atomicOr(status, DEV_OVERFLOW);
    return (int32_t)v;
}
__device__ __forceinline__ float diag_weight(float m, uint32_t*) { return __fmul_rn(m, 2.0f); }
__device__ __forceinline__ double diag_weight(double m, uint32_t*) { return __dmul_rn(m, 2.0); }

// the diagonal entry of every row with mass: after the row's entries below the diagonal
template <class WT, class AT>
__global__ void __launch_bounds__(kThreads)
k_diag_place(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
             const int32_t* __restrict__ pos, const AT* __restrict__ mass,
             int32_t* __restrict__ col_d, WT* __restrict__ w_d, uint32_t* status) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (pos[x + 1] == pos[x]) continue;
        int64_t lo = rowptr[x], hi = rowptr[x + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)col[mid] < x) lo = mid + 1; else hi = mid;
        }
        const int64_t at = lo + pos[x];
        col_d[at] = (int32_t)x;
        w_d[at] = (WT)diag_weight(mass[x], status);
    }
}

template <class WT>
spc_status carry_mass_typed(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                            const void* prev_mass, const void* self_mass, Buf& mass_out) {
    using Acc = typename CT<WT>::Acc;
    Work& W = ctx->work;
    const int maxb = ctx->num_sms * 8;
    SPC_TRY(ensure(ctx, mass_out, (size_t)(n_c + 1) * sizeof(Acc)));
    Acc* out = mass_out.as<Acc>();
    const Acc* self = static_cast<const Acc*>(self_mass);
    const Acc* prev = static_cast<const Acc*>(prev_mass);
    if (n_c <= 0) return SPC_OK;
    if constexpr (std::is_same<WT, int32_t>::value) {
        SPC_LAUNCH(ctx, k_mass_int_init, grid_for(n_c, kThreads, maxb), kThreads, 0, n_c, self,
                   out);
        SPC_LAUNCH(ctx, k_mass_int_add, grid_for(n, kThreads, maxb), kThreads, 0, n, lift, prev,
                   out);
        return SPC_OK;
    } else {
        int nb = 1;
        while ((1ll << nb) < n_c) ++nb;
        uint32_t* key = W.ms_key.as<uint32_t>();
        uint32_t* val = W.ms_val.as<uint32_t>();
        int32_t* start = W.ms_start.as<int32_t>();
        const int gn = grid_for(n, kThreads, maxb);
        SPC_LAUNCH(ctx, k_member_keys, gn, kThreads, 0, n, lift, key, val);
        SPC_TRY(radix_sort_u32(ctx, key, val, W.ms_key2.as<uint32_t>(), W.ms_val2.as<uint32_t>(),
                               n, nb));
        SPC_LAUNCH(ctx, k_member_starts, gn, kThreads, 0, n, n_c, key, start);
        int32_t* long_list = W.long_segs.as<int32_t>();
        int32_t* long_cnt = W.counters.as<int32_t>() + 9;
        SPC_LAUNCH(ctx, k_set_i32, 1, 32, 0, long_cnt, 0);
        SPC_LAUNCH(ctx, (k_segsum_short<WT, WT>), grid_for(n_c, kThreads, maxb), kThreads, 0,
                   n_c, start, val, nullptr, prev, out, long_list, long_cnt, ctx->d_status);
        SPC_TRY((long_segment_sums<WT, WT>(ctx, start, val, nullptr, prev, out)));
        SPC_LAUNCH(ctx, k_mass_add_self<WT>, grid_for(n_c, kThreads, maxb), kThreads, 0, n_c,
                   self, out);
        return SPC_OK;
    }
}

template <class WT>
spc_status diag_graph_typed(spc_context* ctx, const GraphView& g, const void* mass_v,
                            GraphView& out) {
    using Acc = typename CT<WT>::Acc;
    Work& W = ctx->work;
    const int64_t n = g.n;
    const int maxb = ctx->num_sms * 8;
    out = g;
    if (n <= 0) return SPC_OK;
    const Acc* mass = static_cast<const Acc*>(mass_v);
    SPC_TRY(ensure(ctx, W.dg_rowptr, (size_t)(n + 1) * 8));
    SPC_TRY(ensure(ctx, W.dg_pos, (size_t)(n + 1) * 4));
    SPC_TRY(ensure(ctx, W.dg_col, (size_t)(g.nnz + n + 1) * 4));
    SPC_TRY(ensure(ctx, W.dg_w, (size_t)(g.nnz + n + 1) * sizeof(WT)));
    int64_t* rowptr_d = W.dg_rowptr.as<int64_t>();
    int32_t* pos = W.dg_pos.as<int32_t>();
    int32_t* col_d = W.dg_col.as<int32_t>();
    WT* w_d = W.dg_w.as<WT>();
    SPC_TRY(scan_fused<unsigned long long>(ctx, n, DiagLd<Acc>{mass},
                                           DiagSt{g.rowptr, rowptr_d, pos, n},
                                           (double)n * (sizeof(Acc) + 8.0 + 8.0 + 4.0)));
    int64_t nd = 0;
    SPC_TRY(read_i32(ctx, pos + n, &nd));
    if (g.nnz > 0) {
        note_bytes(ctx, (double)g.nnz * 2.0 * (4.0 + sizeof(WT)) + (double)(n + 1) * 12.0);
        SPC_LAUNCH(ctx, k_diag_entries<WT>, grid_for(g.nnz, (int)kDiagTile, maxb), kThreads, 0,
                   n, g.nnz, g.rowptr, g.col, static_cast<const WT*>(g.w), pos, col_d, w_d);
    }
    if (nd > 0) {
        SPC_LAUNCH(ctx, (k_diag_place<WT, Acc>), grid_for(n, kThreads, maxb), kThreads, 0, n,
                   g.rowptr, g.col, pos, mass, col_d, w_d, ctx->d_status);
    }
    out.rowptr = rowptr_d;
    out.col = col_d;
    out.w = w_d;
    out.nnz = g.nnz + nd;
    out.ndiag = nd;
    return SPC_OK;
}

}  // namespace

spc_status run_contract(spc_context* ctx, const GraphView& g, const int32_t* lift, int64_t n_c,
                        LevelBufs& lv) {
    switch (g.wtype) {
        case SPC_I32: return contract_typed<int32_t>(ctx, g, lift, n_c, lv);
        case SPC_F32: return contract_typed<float>(ctx, g, lift, n_c, lv);
        case SPC_F64: return contract_typed<double>(ctx, g, lift, n_c, lv);
    }
    return SPC_ERR_INVALID_ARG;
}

spc_status run_contract_forward(spc_context* ctx, const int32_t* perm, const int32_t* seg,
                                int64_t m_c, const void* w_und, spc_dtype wt, void* a_und) {
    if (wt == SPC_F32)
        return forward_typed<float>(ctx, perm, seg, m_c, static_cast<const float*>(w_und),
                                    static_cast<float*>(a_und));
    if (wt == SPC_F64)
        return forward_typed<double>(ctx, perm, seg, m_c, static_cast<const double*>(w_und),
                                     static_cast<double*>(a_und));
    return SPC_ERR_INVALID_ARG;
}

spc_status run_contract_backward(spc_context* ctx, const int32_t* emap, int64_t m,
                                 const void* grad_a, void* grad_w, spc_dtype wt) {
    if (m <= 0) return SPC_OK;
    const int gb = grid_for(m, kThreads, ctx->num_sms * 8);
    if (wt == SPC_F32) {
        SPC_LAUNCH(ctx, k_backward<float>, gb, kThreads, 0, m, emap,
                   static_cast<const float*>(grad_a), static_cast<float*>(grad_w));
    } else if (wt == SPC_F64) {
        SPC_LAUNCH(ctx, k_backward<double>, gb, kThreads, 0, m, emap,
                   static_cast<const double*>(grad_a), static_cast<double*>(grad_w));
    } else {
        return SPC_ERR_INVALID_ARG;
    }
    return SPC_OK;
}

}  // namespace spc

namespace spc {

spc_status run_carry_mass(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                          const void* prev_mass, const void* self_mass, spc_dtype wt,
                          Buf& mass_out, const void** mass_ptr) {
    if (!prev_mass) {  // nothing carried in: (0 + 0 + ...) + self = self, bit for bit
        *mass_ptr = self_mass;
        return SPC_OK;
    }
    spc_status st = SPC_ERR_INVALID_ARG;
    switch (wt) {
        case SPC_I32: st = carry_mass_typed<int32_t>(ctx, n, lift, n_c, prev_mass, self_mass, mass_out); break;
        case SPC_F32: st = carry_mass_typed<float>(ctx, n, lift, n_c, prev_mass, self_mass, mass_out); break;
        case SPC_F64: st = carry_mass_typed<double>(ctx, n, lift, n_c, prev_mass, self_mass, mass_out); break;
    }
    *mass_ptr = st == SPC_OK ? mass_out.p : nullptr;
    return st;
}

spc_status run_diag_graph(spc_context* ctx, const GraphView& g, const void* mass,
                          GraphView& out) {
    switch (g.wtype) {
        case SPC_I32: return diag_graph_typed<int32_t>(ctx, g, mass, out);
        case SPC_F32: return diag_graph_typed<float>(ctx, g, mass, out);
        case SPC_F64: return diag_graph_typed<double>(ctx, g, mass, out);
    }
    return SPC_ERR_INVALID_ARG;
}

}  // namespace spc
