// S5-S6: the merge loop of Algorithm 1, done in parallel, and the relabelling.
//
// Algorithm 1 walks the edges in ascending (f, eid) order and merges the two super-nodes of
// an edge unless they are already one, until n_c super-nodes remain.  Because the keys
// (f, eid) are all distinct, that loop is Kruskal's algorithm stopped after n - n_c successful
// merges: the merging edges are exactly the n - n_c lightest edges of the (unique) minimum
// spanning forest, and the partition is the components of those edges.  So:
//   1. Boruvka rounds build the minimum spanning forest: every component picks its lightest
//      incident edge by atomicMin on the key (two phases for 64-bit scores: the score bits,
//      then the edge id among the edges that tie), picked edges are forest edges (cut
//      property) and are united in a lock-free union-find whose roots are always the smallest
//      node id of their set; edges inside one component drop out of the work list.  Only a
//      prefix of the score order takes part: Kruskal's first n - n_c merges all lie among the
//      lightest edges, so the rounds run on the edges up to a threshold chosen from a score
//      histogram to hold about 1.5 (n - n_c) edges (on very large graphs the slab's edges are
//      first compacted into the work list); if that prefix's forest has fewer than n - n_c
//      edges, the rounds resume on the next slab, the forest found so far kept.
//   2. The forest edges are compacted in eid order.  For one graph an exact radix select on
//      11-bit digits of (score, eid) finds the (n - n_c)-th lightest and every forest edge up to
//      it is united in a second union-find; for batches the forest edges are radix-sorted by
//      score and then by graph (stable, so ties stay in eid order) and the first
//      n_b - target_b of each graph are united.
//   3. Relabel: root = smallest member; flag roots, exclusive scan, id = scan[root] (Definition
//      1's super-nodes, numbered by smallest member).
// Every retry loop is bounded (spin_limit: kSpinLimit unless the context lowered it); giving up
// sets DEV_TIMEOUT in the status word.
#include <atomic>

#include "spc_scan.cuh"

namespace spc {

namespace {

__device__ __forceinline__ int32_t ld_parent(const int32_t* parent, int32_t x) {
    return __ldcg(parent + x);
}

// find with path halving; parent pointers only ever move to an ancestor, so racing writes are
// benign.  Bounded: the chain of a forest over n nodes is shorter than kSpinLimit.  Giving up
// returns a node of the set (an ancestor of x): every index stays in range.
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x, uint32_t* status) {
    const uint32_t lim = spin_limit(status);
    for (uint32_t it = 0; it < lim; ++it) {
        int32_t p = ld_parent(parent, x);
        if (p == x) return x;
        int32_t gp = ld_parent(parent, p);
        if (gp != p) parent[x] = gp;
        x = gp;
    }
    atomicOr(status, DEV_TIMEOUT);
    return x;
}

// atomicMin of v into a[idx] by every active lane of the warp (all 32 lanes call it).  When
// neighbouring lanes target the same slot -- the edges of a hub component -- the lanes of each
// slot first take their minimum together and one lane issues the atomic.
__device__ __forceinline__ void warp_atomic_min_u64(unsigned long long* a, int32_t idx,
                                                    unsigned long long v, bool act) {
    const int lane = threadIdx.x & 31;
    const int32_t key = act ? idx : -1;
    const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    if (!__any_sync(0xffffffffu, act && lane > 0 && prev == key)) {
        if (act) atomicMin(a + idx, v);
        return;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (!act) return;  // inactive lanes form their own group
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned hmin = __reduce_min_sync(peers, hi);
    const unsigned lmin = __reduce_min_sync(peers, hi == hmin ? lo : 0xffffffffu);
    if (lane == __ffs(peers) - 1) atomicMin(a + idx, ((unsigned long long)hmin << 32) | lmin);
}

__device__ __forceinline__ void warp_atomic_min_i32(int32_t* a, int32_t idx, int32_t v,
                                                    bool act) {
    const int lane = threadIdx.x & 31;
    const int32_t key = act ? idx : -1;
    const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    if (!__any_sync(0xffffffffu, act && lane > 0 && prev == key)) {
        if (act) atomicMin(a + idx, v);
        return;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (!act) return;
    const int32_t vmin = __reduce_min_sync(peers, v);
    if (lane == __ffs(peers) - 1) atomicMin(a + idx, vmin);
}

// unite the sets of a and b; the larger root is hooked below the smaller one with a CAS, so a
// root is always the smallest node id of its set.  Returns true if the sets were distinct.
__device__ __forceinline__ bool uf_unite(int32_t* parent, int32_t a, int32_t b,
                                         uint32_t* status) {
    const uint32_t lim = spin_limit(status);
    for (uint32_t it = 0; it < lim; ++it) {
        a = uf_find(parent, a, status);
        b = uf_find(parent, b, status);
        if (a == b) return false;
        if (a > b) { int32_t t = a; a = b; b = t; }
        int32_t old = atomicCAS(parent + b, b, a);
        if (old == b) return true;
    }
    atomicOr(status, DEV_TIMEOUT);
    return false;
}

__global__ void k_iota(int32_t* a, int64_t n) {
    spc::pdl_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// Start state of the spanning-forest rounds in one launch: parent[i] = i, both parities'
// best-key slots "none", best-edge slots "none" (64-bit scores), forest flags and merge marks
// cleared, the two work-list counts zero.
__global__ void k_bv_init(int64_t n, int64_t m, int32_t* __restrict__ parent,
                          unsigned long long* __restrict__ bk0, unsigned long long* __restrict__ bk1,
                          int32_t* __restrict__ be0, int32_t* __restrict__ be1,
                          uint8_t* __restrict__ msf, uint8_t* __restrict__ merged,
                          int32_t* __restrict__ counts) {
    spc::pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < n; i += stride) {
        parent[i] = (int32_t)i;
        bk0[i] = ~0ull;
        bk1[i] = ~0ull;
        if (be0) {
            be0[i] = INT32_MAX;
            be1[i] = INT32_MAX;
        }
    }
    for (int64_t e = t0; e <= m; e += stride) {
        msf[e] = 0;
        if (merged && e < m) merged[e] = 0;
    }
    if (t0 < 2) counts[t0] = 0;
}

template <class KT> struct MinKey;
// 64-bit scores: best_k holds the score bits, best_e the smallest edge id among the ties
template <> struct MinKey<unsigned long long> {
    static constexpr bool two_phase = true;
    __device__ static unsigned long long pack(unsigned long long k, int32_t) { return k; }
};
// 32-bit scores: one atomicMin on (score bits << 32 | edge id)
template <> struct MinKey<unsigned int> {
    static constexpr bool two_phase = false;
    __device__ static unsigned long long pack(unsigned int k, int32_t e) {
        return ((unsigned long long)k << 32) | (uint32_t)e;
    }
};

// Boruvka phase A: current roots of both ends; keep inter-component edges; lower the
// component minima.  The first Boruvka pass reads every edge directly and keeps only the
// score prefix (key >> tau_shift <= *tau_top).  Each thread takes kMkItems edges per pass
// (their loads overlap), and the survivors are appended with one global atomic per block
// and pass.
constexpr int kMkItems = 2;
constexpr uint32_t kNoSlab = 0xffffffffu;  // no lower bound on the score slab

// Per-graph score slabs of a batch: the first Boruvka pass keeps an edge of graph g when its
// key lies in (lo[g], tau[g]] (lo[g] all ones: no lower bound).  node_graph null: no slabs.
template <class KT>
struct GraphSlab {
    const int32_t* node_graph;
    const KT* tau;
    const KT* lo;
    __device__ __forceinline__ bool outside(int32_t u, KT k) const {
        const int32_t g = node_graph[u];
        const KT l = lo[g];
        return k > tau[g] || (l != ~KT(0) && k <= l);
    }
};

// The start of a further slab: the forest found so far (parent, forest flags) stays; the
// best-edge slots of both parities and the work-list counts are reset.
__global__ void k_bv_reinit(int64_t n, unsigned long long* __restrict__ bk0,
                            unsigned long long* __restrict__ bk1, int32_t* __restrict__ be0,
                            int32_t* __restrict__ be1, int32_t* __restrict__ counts) {
    spc::pdl_wait();
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        bk0[i] = ~0ull;
        bk1[i] = ~0ull;
        if (be0) {
            be0[i] = INT32_MAX;
            be1[i] = INT32_MAX;
        }
    }
    if (t0 < 2) counts[t0] = 0;
}

// the slab just done becomes the lower bound of the next
__global__ void k_bump_slab(const uint32_t* __restrict__ tau_top, uint32_t* __restrict__ tau_lo) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *tau_lo = *tau_top;
}

// The edges of the current score slab as the first Boruvka work list: every edge whose key
// lies in the slab is written as (e, eu[e], ev[e]).  A streaming pass: each thread takes
// kSlItems consecutive edges (their keys in 16-byte loads; key 16-byte aligned), the ends are
// read only for the slab's edges, and one global atomic per kThreads * kSlItems edges places
// a block's survivors, so the list is in edge order within each block's chunk (the next
// rounds' parent and flag accesses stay close together); the forest does not depend on the
// order (every component's lightest edge is unique).
constexpr int kSlItems = 16;
constexpr int64_t kSlabListMin = int64_t{1} << 25;

template <class KT>
__global__ void __launch_bounds__(kThreads)
k_slab_list(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
            const KT* __restrict__ key, int tau_shift, const uint32_t* __restrict__ tau_top,
            const uint32_t* __restrict__ tau_lo, int32_t* __restrict__ wo_e,
            int32_t* __restrict__ wo_u, int32_t* __restrict__ wo_v,
            int32_t* __restrict__ out_count) {
    static_assert(kSlItems * sizeof(KT) % 16 == 0, "whole 16-byte loads");
    constexpr int kVec = (int)(kSlItems * sizeof(KT) / 16);
    spc::pdl_wait();
    __shared__ int32_t sh_wsum[kThreads / 32];
    __shared__ int32_t sh_base;
    const uint32_t top = tau_top ? *tau_top : 0xffffffffu;
    const uint32_t lo = tau_lo ? *tau_lo : kNoSlab;
    const int64_t per = (int64_t)kThreads * kSlItems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = (int64_t)blockIdx.x * per; base < m; base += (int64_t)gridDim.x * per) {
        const int64_t i0 = base + (int64_t)threadIdx.x * kSlItems;
        KT k[kSlItems];
        if (i0 + kSlItems <= m) {
            const uint4* p = reinterpret_cast<const uint4*>(key + i0);
            uint4 q[kVec];
#pragma unroll
            for (int j = 0; j < kVec; ++j) q[j] = p[j];
            memcpy(k, q, sizeof(k));
        } else {
#pragma unroll
            for (int it = 0; it < kSlItems; ++it) k[it] = i0 + it < m ? key[i0 + it] : KT(0);
        }
        unsigned keep = 0;  // bit it: edge i0 + it lies in the slab
#pragma unroll
        for (int it = 0; it < kSlItems; ++it) {
            const uint32_t bin = (uint32_t)(k[it] >> tau_shift);
            const bool in = i0 + it < m && bin <= top && (lo == kNoSlab || bin > lo);
            keep |= in ? 1u << it : 0u;
        }
        const int32_t nkeep = __popc(keep);
        int32_t incl = nkeep;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) sh_wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const int32_t t = sh_wsum[w];
                sh_wsum[w] = tot;
                tot += t;
            }
            sh_base = tot ? atomicAdd(out_count, tot) : 0;
        }
        __syncthreads();
        int32_t slot = sh_base + sh_wsum[warp] + incl - nkeep;
        while (keep) {
            const int it = __ffs(keep) - 1;
            keep &= keep - 1;
            const int64_t i = i0 + it;
            wo_e[slot] = (int32_t)i;
            wo_u[slot] = eu[i];
            wo_v[slot] = ev[i];
            ++slot;
        }
        __syncthreads();
    }
}

template <class KT>
__global__ void __launch_bounds__(kThreads)
k_bv_minkey(int round0, int direct, int64_t m, const int32_t* __restrict__ in_count,
            const int32_t* __restrict__ wi_e, const int32_t* __restrict__ wi_u,
            const int32_t* __restrict__ wi_v, const int32_t* __restrict__ eu,
            const int32_t* __restrict__ ev, const KT* __restrict__ key, int tau_shift,
            const uint32_t* __restrict__ tau_top, const uint32_t* __restrict__ tau_lo,
            GraphSlab<KT> gs, int32_t* parent, unsigned long long* best_k, int32_t* wo_e,
            int32_t* wo_u, int32_t* wo_v, int32_t* out_count, uint32_t* status) {
    spc::pdl_wait();
    __shared__ int32_t sh_wsum[kThreads / 32];
    __shared__ int32_t sh_base;
    const int64_t cnt = round0 ? m : (int64_t)*in_count;
    const uint32_t top = tau_top ? *tau_top : 0xffffffffu;
    // a first round over the next slab of scores skips the slabs already done
    const uint32_t lo = tau_lo ? *tau_lo : kNoSlab;
    const int64_t per = (int64_t)blockDim.x * kMkItems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = (int64_t)blockIdx.x * per; base < cnt; base += (int64_t)gridDim.x * per) {
        int32_t e[kMkItems], u[kMkItems], v[kMkItems];
        bool in[kMkItems];
#pragma unroll
        for (int it = 0; it < kMkItems; ++it) {
            const int64_t i = base + (int64_t)it * blockDim.x + threadIdx.x;
            in[it] = i < cnt;
            e[it] = 0; u[it] = 0; v[it] = 0;
            if (in[it]) {
                if (round0) { e[it] = (int32_t)i; u[it] = eu[i]; v[it] = ev[i]; }
                else { e[it] = wi_e[i]; u[it] = wi_u[i]; v[it] = wi_v[i]; }
            }
        }
        KT k[kMkItems];
#pragma unroll
        for (int it = 0; it < kMkItems; ++it) {
            k[it] = in[it] ? key[e[it]] : KT(0);
            if (round0 && in[it]) {
                const uint32_t bin = (uint32_t)(k[it] >> tau_shift);
                if (bin > top || (lo != kNoSlab && bin <= lo)) in[it] = false;
                if (gs.node_graph && gs.outside(u[it], k[it])) in[it] = false;
            }
        }
        int32_t ru[kMkItems], rv[kMkItems];
        int32_t nkeep = 0;
#pragma unroll
        for (int it = 0; it < kMkItems; ++it) {
            // direct: the selection's first round, every node still its own component
            ru[it] = in[it] ? (direct ? u[it] : uf_find(parent, u[it], status)) : 0;
            rv[it] = in[it] ? (direct ? v[it] : uf_find(parent, v[it], status)) : 0;
            in[it] = in[it] && ru[it] != rv[it];
            const unsigned long long pk = MinKey<KT>::pack(k[it], e[it]);
            warp_atomic_min_u64(best_k, ru[it], pk, in[it]);
            warp_atomic_min_u64(best_k, rv[it], pk, in[it]);
            nkeep += in[it] ? 1 : 0;
        }
        // block-wide exclusive prefix of the survivors, one global atomic per block and pass
        int32_t incl = nkeep;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) sh_wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const int32_t t = sh_wsum[w];
                sh_wsum[w] = tot;
                tot += t;
            }
            sh_base = tot ? atomicAdd(out_count, tot) : 0;
        }
        __syncthreads();
        int32_t slot = sh_base + sh_wsum[warp] + incl - nkeep;
#pragma unroll
        for (int it = 0; it < kMkItems; ++it) {
            if (in[it]) {
                wo_e[slot] = e[it];
                wo_u[slot] = ru[it];
                wo_v[slot] = rv[it];
                ++slot;
            }
        }
        __syncthreads();
    }
}


// The last Boruvka rounds in one CTA.  Once the work list holds at most kFinishMax items (the
// last rounds of a large level; every round of a small one) a round is a few microseconds of
// work and three launches; here one CTA of kFinishThreads runs every remaining round, its
// phases separated by block barriers: the lowering of the component minima (as k_bv_minkey,
// the survivors compacted into the other list through a shared-memory counter), the tie-break
// by edge id for 64-bit scores (as k_bv_tiebreak), the hook (as k_bv_hook).  Each component's
// lightest edge is unique, so the forest does not depend on the order of the lists.
// round0: the first round reads the edges directly (e = i, u = eu[i], v = ev[i]) with the
// score-prefix filter, like k_bv_minkey's first round.
constexpr int kFinishMax = 16384;
constexpr int kFinishThreads = 1024;

template <class KT>
__global__ void __launch_bounds__(kFinishThreads, 1)
k_bv_finish(int round0, int par0, int64_t m, int32_t* count_in, int32_t* li_e, int32_t* li_u,
            int32_t* li_v, int32_t* lo_e, int32_t* lo_u, int32_t* lo_v,
            const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
            const KT* __restrict__ key, int tau_shift, const uint32_t* __restrict__ tau_top,
            const uint32_t* __restrict__ tau_lo, GraphSlab<KT> gs, int32_t* parent,
            unsigned long long* bk0, unsigned long long* bk1, int32_t* be0, int32_t* be1,
            uint8_t* msf, uint32_t* status) {
    spc::pdl_wait();
    __shared__ int32_t sh_cnt[2];
    const uint32_t top = tau_top ? *tau_top : 0xffffffffu;
    const uint32_t slab_lo = tau_lo ? *tau_lo : kNoSlab;
    int64_t cnt = round0 ? m : (int64_t)*count_in;
    int par = par0;
    int32_t *ie = li_e, *iu = li_u, *iv = li_v, *oe = lo_e, *ou = lo_u, *ov = lo_v;
    for (int r = 0; cnt > 0; ++r) {
        if (r >= 64) {  // every round at least halves the components that still have edges
            if (threadIdx.x == 0) atomicOr(status, DEV_TIMEOUT);
            break;
        }
        unsigned long long* bk = par ? bk1 : bk0;
        unsigned long long* bk_next = par ? bk0 : bk1;
        int32_t* be = par ? be1 : be0;
        int32_t* be_next = par ? be0 : be1;
        if (threadIdx.x == 0) sh_cnt[0] = 0;
        __syncthreads();
        // lower the component minima; keep the edges between two components
        for (int64_t i = threadIdx.x; i < cnt; i += kFinishThreads) {
            int32_t e, u, v;
            if (round0 && r == 0) { e = (int32_t)i; u = eu[i]; v = ev[i]; }
            else { e = ie[i]; u = iu[i]; v = iv[i]; }
            const KT k = key[e];
            if (round0 && r == 0) {
                const uint32_t bin = (uint32_t)(k >> tau_shift);
                if (bin > top || (slab_lo != kNoSlab && bin <= slab_lo)) continue;
                if (gs.node_graph && gs.outside(u, k)) continue;
            }
            const int32_t ru = uf_find(parent, u, status), rv = uf_find(parent, v, status);
            if (ru == rv) continue;
            const unsigned long long pk = MinKey<KT>::pack(k, e);
            atomicMin(bk + ru, pk);
            atomicMin(bk + rv, pk);
            const int32_t slot = atomicAdd(&sh_cnt[0], 1);
            oe[slot] = e;
            ou[slot] = ru;
            ov[slot] = rv;
        }
        __syncthreads();
        const int32_t kept = sh_cnt[0];
        if (MinKey<KT>::two_phase) {  // among equal scores, the smallest edge id
            for (int32_t i = threadIdx.x; i < kept; i += kFinishThreads) {
                const int32_t e = oe[i], ru = ou[i], rv = ov[i];
                const unsigned long long k = (unsigned long long)key[e];
                if (k == bk[ru]) atomicMin(be + ru, e);
                if (k == bk[rv]) atomicMin(be + rv, e);
            }
            __syncthreads();
        }
        // hook the picked edges; clear the next round's slots of these components
        for (int32_t i = threadIdx.x; i < kept; i += kFinishThreads) {
            const int32_t e = oe[i], ru = ou[i], rv = ov[i];
            bool picked;
            if (MinKey<KT>::two_phase) {
                picked = be[ru] == e || be[rv] == e;
                be_next[ru] = INT32_MAX;
                be_next[rv] = INT32_MAX;
            } else {
                picked = (int32_t)(uint32_t)bk[ru] == e || (int32_t)(uint32_t)bk[rv] == e;
            }
            bk_next[ru] = ~0ull;
            bk_next[rv] = ~0ull;
            if (picked) {
                msf[e] = 1;
                uf_unite(parent, ru, rv, status);
            }
        }
        __syncthreads();
        cnt = kept;
        par ^= 1;
        int32_t* t;
        t = ie; ie = oe; oe = t;
        t = iu; iu = ou; ou = t;
        t = iv; iv = ov; ov = t;
    }
}

// histogram of the top 15 bits of the scores (bits below the sign), per block in shared memory,
// over a sample of the keys: one chunk of kHistChunk consecutive keys in every 2^samp (samp 0:
// every key).  The threshold it gives only sizes the score prefix, never changes a result.
constexpr int kHistChunk = 256;

template <class KT>
__global__ void __launch_bounds__(1024)
k_key_hist(int64_t m, const KT* __restrict__ key, int shift, int samp,
           uint32_t* __restrict__ hist) {
    spc::pdl_wait();
    extern __shared__ uint32_t sh_hist[];
    for (int b = threadIdx.x; b < 32768; b += blockDim.x) sh_hist[b] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = ((v / kHistChunk) << samp) * kHistChunk + v % kHistChunk;
        if (i >= m) break;  // i grows with v
        const uint32_t b = (uint32_t)(key[i] >> shift) & 32767u;
        const unsigned peers = __match_any_sync(__activemask(), b);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&sh_hist[b], __popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 32768; b += blockDim.x)
        if (sh_hist[b]) atomicAdd(hist + b, sh_hist[b]);
}

// inclusive scan of x over the block (blockDim.x a multiple of 32, at most 1024), by warp
// shuffles and one pass over the warp totals; ws: 32 words of shared memory.  All threads call
// it; ws may be reused after it returns.
__device__ __forceinline__ unsigned long long block_incl_scan(unsigned long long x,
                                                               unsigned long long* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long y = lane < nw ? ws[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const unsigned long long r = x + (w ? ws[w - 1] : 0ull);
    __syncthreads();
    return r;
}

// smallest bin whose cumulative count reaches `need` (all bins when need >= m); the histogram
// stays for a later attempt of the same selection.  Each thread holds 32 consecutive bins in registers; the
// block scan of the thread totals is two rounds of warp shuffles.
__global__ void __launch_bounds__(1024)
k_pick_tau(uint32_t* __restrict__ hist, int64_t need, uint32_t* __restrict__ tau_top) {
    spc::pdl_wait();
    constexpr int kPer = 32768 / 1024;
    __shared__ unsigned long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint4* h4 = reinterpret_cast<uint4*>(hist) + (int64_t)t * (kPer / 4);
    uint32_t v[kPer];
    unsigned long long loc = 0;
#pragma unroll
    for (int j = 0; j < kPer / 4; ++j) {
        const uint4 q = h4[j];
        v[4 * j] = q.x;
        v[4 * j + 1] = q.y;
        v[4 * j + 2] = q.z;
        v[4 * j + 3] = q.w;
        loc += (unsigned long long)q.x + q.y + q.z + q.w;
    }
    unsigned long long x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    if (t == 0) *tau_top = 32767u;
    __syncthreads();
    if (w == 0) {
        unsigned long long y = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        wsum[lane] = y;
    }
    __syncthreads();
    const unsigned long long incl = x + (w ? wsum[w - 1] : 0ull);
    unsigned long long run = incl - loc;
    if (run < (unsigned long long)need && incl >= (unsigned long long)need) {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            run += v[j];
            if (run >= (unsigned long long)need) {
                *tau_top = (uint32_t)(t * kPer + j);
                break;
            }
        }
    }
}

// Boruvka phase B (64-bit scores only): among the edges whose score equals the component
// minimum, keep the smallest edge id.
__global__ void __launch_bounds__(kThreads)
k_bv_tiebreak(const int32_t* __restrict__ count, const int32_t* __restrict__ wl_e,
              const int32_t* __restrict__ wl_u, const int32_t* __restrict__ wl_v,
              const unsigned long long* __restrict__ key, const unsigned long long* best_k,
              int32_t* best_e) {
    spc::pdl_wait();
    const int64_t cnt = *count;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt;
         i0 += (int64_t)gridDim.x * blockDim.x) {  // uniform per warp: the helpers need it
        const int64_t i = i0 + threadIdx.x;
        const bool act = i < cnt;
        int32_t e = 0, ru = 0, rv = 0;
        unsigned long long k = 0;
        if (act) {
            e = wl_e[i]; ru = wl_u[i]; rv = wl_v[i];
            k = key[e];
        }
        warp_atomic_min_i32(best_e, ru, e, act && k == best_k[ru]);
        warp_atomic_min_i32(best_e, rv, e, act && k == best_k[rv]);
    }
}

// Boruvka phase C: an edge picked by either end is a forest edge; unite.  Also clears the
// other parity's minima at both ends, ready for the next round (the roots that next round
// touches are all ends of this round's work list).
template <class KT>
__global__ void __launch_bounds__(kThreads)
k_bv_hook(const int32_t* __restrict__ count, const int32_t* __restrict__ wl_e,
          const int32_t* __restrict__ wl_u, const int32_t* __restrict__ wl_v,
          const unsigned long long* __restrict__ best_k, const int32_t* __restrict__ best_e,
          unsigned long long* other_k, int32_t* other_e, int32_t* parent, uint8_t* msf,
          int32_t* spent_count, uint32_t* status) {
    spc::pdl_wait();
    // this round's input count is read by nobody after phase A: zero it here, it is the
    // next round's output count
    if (blockIdx.x == 0 && threadIdx.x == 0) *spent_count = 0;
    const int64_t cnt = *count;
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < cnt;
         i0 += (int64_t)gridDim.x * blockDim.x) {  // uniform per warp
        const int64_t i = i0 + threadIdx.x;
        const bool act = i < cnt;
        int32_t e = 0, ru = -1, rv = -1;
        if (act) { e = wl_e[i]; ru = wl_u[i]; rv = wl_v[i]; }
        // a slot shared with the previous lane (a hub component) is cleared by that lane
        const int32_t pu = __shfl_up_sync(0xffffffffu, ru, 1);
        const int32_t pv = __shfl_up_sync(0xffffffffu, rv, 1);
        if (!act) continue;
        const bool clr_u = lane == 0 || pu != ru, clr_v = lane == 0 || pv != rv;
        bool picked;
        if (MinKey<KT>::two_phase) {
            picked = best_e[ru] == e || best_e[rv] == e;
            if (clr_u) other_e[ru] = INT32_MAX;
            if (clr_v) other_e[rv] = INT32_MAX;
        } else {
            picked = (int32_t)(uint32_t)best_k[ru] == e || (int32_t)(uint32_t)best_k[rv] == e;
        }
        if (clr_u) other_k[ru] = ~0ull;
        if (clr_v) other_k[rv] = ~0ull;
        if (picked) {
            msf[e] = 1;
            uf_unite(parent, ru, rv, status);
        }
    }
}

// forest edges -> (score key, eid) list in eid order
template <class KT>
__global__ void __launch_bounds__(kThreads)
k_compact_msf(int64_t m, const uint8_t* __restrict__ msf, const int32_t* __restrict__ pos,
              const KT* __restrict__ key, KT* __restrict__ out_k, uint32_t* __restrict__ out_v) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (msf[e]) {
            const int32_t q = pos[e];
            out_k[q] = key[e];
            out_v[q] = (uint32_t)e;
        }
    }
}

// graph id of every node of a block-diagonal batch
__global__ void k_node_graph(int64_t n, int64_t B, const int64_t* __restrict__ graph_ptr,
                             int32_t* __restrict__ node_graph) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = B;  // largest b with graph_ptr[b] <= x
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (graph_ptr[mid] <= x) lo = mid; else hi = mid;
        }
        node_graph[x] = (int32_t)lo;
    }
}

// second sort key for batches: graph of the edge's smaller end point
__global__ void k_graph_keys(const int32_t* __restrict__ count, const uint32_t* __restrict__ eids,
                             const int32_t* __restrict__ eu, const int32_t* __restrict__ node_graph,
                             uint32_t* __restrict__ gkey) {
    spc::pdl_wait();
    const int64_t cnt = *count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        gkey[i] = (uint32_t)node_graph[eu[eids[i]]];
}

// ---- per-graph score prefixes of a batch ------------------------------------------------
// Graphs of a batch are disjoint, so each one's Kruskal merges are the lightest forest edges
// of any prefix of its own scores whose forest holds them (the argument of the single-graph
// prefix, graph by graph).  Each graph's first slab is its lightest 1.5 (n_b - n_c,b) keys;
// a graph whose forest falls short takes the next slab of twice as many keys.  One CTA per
// graph finds the threshold with two histogram passes over its keys (2048 bins each: the 11
// highest value bits, then the next 11 among the keys of the chosen bin), so the slab's top
// is exact up to its low bits (they are all included).
constexpr int kGpThreads = 256;
constexpr int kGpBins = 2048;
template <class KT> struct GpShift;
template <> struct GpShift<unsigned int> { static constexpr int s1 = 20, s2 = 9; };
template <> struct GpShift<unsigned long long> { static constexpr int s1 = 52, s2 = 41; };

// the first bin whose running count over hist reaches `need` (1 <= need <= total); also the
// count before it.  Every thread of the block calls it.
__device__ void cta_find_bin(const uint32_t* hist, int64_t need, int* bin_out,
                             int64_t* before_out) {
    __shared__ unsigned long long s_part[kGpThreads / 32];
    __shared__ int s_bin;
    __shared__ long long s_before;
    constexpr int kPer = kGpBins / kGpThreads;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned long long loc = 0;
    for (int j = 0; j < kPer; ++j) loc += hist[t * kPer + j];
    unsigned long long incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_part[w] = incl;
    if (t == 0) s_bin = kGpBins - 1;
    __syncthreads();
    unsigned long long base = 0;
    for (int i = 0; i < w; ++i) base += s_part[i];
    unsigned long long run = base + incl - loc;  // count before this thread's bins
    if (run < (unsigned long long)need && run + loc >= (unsigned long long)need) {
        for (int j = 0; j < kPer; ++j) {
            const uint32_t c = hist[t * kPer + j];
            if (run + c >= (unsigned long long)need) {
                s_bin = t * kPer + j;
                s_before = (long long)run;
                break;
            }
            run += c;
        }
    }
    __syncthreads();
    *bin_out = s_bin;
    *before_out = s_before;
    __syncthreads();
}

// the smallest threshold t (its low s2 bits all set) with at least `need` keys of key[e0, e1)
// at or below it; 1 <= need <= e1 - e0.  Every thread of the block calls it.
template <class KT>
__device__ KT cta_select_key(const KT* __restrict__ key, int64_t e0, int64_t e1, int64_t need,
                             uint32_t* hist) {
    constexpr int S1 = GpShift<KT>::s1, S2 = GpShift<KT>::s2;
    constexpr int kB = 8;  // keys per thread in flight (one CTA may walk a large graph)
    const int64_t step = (int64_t)blockDim.x * kB;
    for (int i = threadIdx.x; i < kGpBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int64_t b0 = e0 + threadIdx.x; b0 < e1; b0 += step) {
        KT k[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) {
            const int64_t e = b0 + (int64_t)q * blockDim.x;
            k[q] = e < e1 ? key[e] : KT(0);
        }
#pragma unroll
        for (int q = 0; q < kB; ++q)
            if (b0 + (int64_t)q * blockDim.x < e1)
                atomicAdd(&hist[(uint32_t)(k[q] >> S1) & (kGpBins - 1)], 1u);
    }
    __syncthreads();
    int c1;
    int64_t before;
    cta_find_bin(hist, need, &c1, &before);
    for (int i = threadIdx.x; i < kGpBins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int64_t b0 = e0 + threadIdx.x; b0 < e1; b0 += step) {
        KT k[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) {
            const int64_t e = b0 + (int64_t)q * blockDim.x;
            k[q] = e < e1 ? key[e] : KT(0);
        }
#pragma unroll
        for (int q = 0; q < kB; ++q)
            if (b0 + (int64_t)q * blockDim.x < e1 && (int)(k[q] >> S1) == c1)
                atomicAdd(&hist[(uint32_t)(k[q] >> S2) & (kGpBins - 1)], 1u);
    }
    __syncthreads();
    int c2;
    int64_t before2;
    cta_find_bin(hist, need - before, &c2, &before2);
    return ((KT)c1 << S1) | ((KT)c2 << S2) | (((KT)1 << S2) - 1);
}

// attempt 0: every graph's first slab [0, tau]; later attempts: a graph whose forest (the
// forest flags of its edge range) holds fewer than its n_b - n_c,b merges, and whose slab does
// not yet reach its last key, takes the next slab (old tau, new tau] of twice the keys (and
// counts into *n_short); every other graph an empty slab.
template <class KT>
__global__ void __launch_bounds__(kGpThreads)
k_graph_prefix(int64_t B, int attempt, const int64_t* __restrict__ graph_ptr,
               const int32_t* __restrict__ up_ptr, const int64_t* __restrict__ targets,
               const KT* __restrict__ key, const uint8_t* __restrict__ msf,
               int64_t* __restrict__ need, KT* __restrict__ tau, KT* __restrict__ lo,
               int32_t* n_short) {
    spc::pdl_wait();
    __shared__ uint32_t hist[kGpBins];
    __shared__ int s_short;
    __shared__ unsigned long long s_sum[kGpThreads / 32];
    constexpr KT kAll = ~KT(0);
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const int64_t n0 = graph_ptr[b], n1 = graph_ptr[b + 1];
        const int64_t e0 = up_ptr[n0], e1 = up_ptr[n1], mb = e1 - e0;
        const int64_t k_b = (n1 - n0) - targets[b] > 0 ? (n1 - n0) - targets[b] : 0;
        int64_t nd;
        if (attempt == 0) {
            nd = k_b + k_b / 2;
            if (threadIdx.x == 0) lo[b] = k_b == 0 ? KT(0) : kAll;
        } else {
            // the forest edges of this graph so far
            unsigned long long f = 0;
            for (int64_t b0 = e0 + threadIdx.x; b0 < e1; b0 += (int64_t)blockDim.x * 8) {
                uint8_t fl[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int64_t e = b0 + (int64_t)q * blockDim.x;
                    fl[q] = e < e1 ? msf[e] : 0;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) f += fl[q] ? 1 : 0;
            }
            for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
            if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = f;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long tot = 0;
                for (int i = 0; i < kGpThreads / 32; ++i) tot += s_sum[i];
                s_short = ((int64_t)tot < k_b && need[b] < mb) ? 1 : 0;
                lo[b] = tau[b];  // done up to the old top: the next slab starts above it
            }
            __syncthreads();
            if (!s_short) continue;  // empty slab (tau, tau]
            nd = 2 * need[b];
            if (threadIdx.x == 0) atomicAdd(n_short, 1);
        }
        if (k_b == 0) {
            if (threadIdx.x == 0) { tau[b] = KT(0); need[b] = 0; }  // empty slab (0, 0]
        } else if (nd >= mb) {
            if (threadIdx.x == 0) { tau[b] = kAll; need[b] = mb; }   // every key
        } else {
            const KT t = cta_select_key<KT>(key, e0, e1, nd, hist);
            if (threadIdx.x == 0) { tau[b] = t; need[b] = nd; }
        }
        __syncthreads();
    }
}


// per graph: first forest edge position and the number of merges k_b = n_b - target_b
__global__ void k_graph_segments(int64_t B, const int64_t* __restrict__ graph_ptr,
                                 const int64_t* __restrict__ targets,
                                 const int32_t* __restrict__ up_ptr,
                                 const int32_t* __restrict__ msf_pos, int32_t* __restrict__ seg_start,
                                 int32_t* __restrict__ k_graph) {
    spc::pdl_wait();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        seg_start[b] = msf_pos[up_ptr[graph_ptr[b]]];
        const int64_t nb = graph_ptr[b + 1] - graph_ptr[b];
        int64_t k = nb - targets[b];
        k_graph[b] = (int32_t)(k < 0 ? 0 : k);
    }
}

// unite the ends of the first k forest edges of every graph (sorted by score)
__global__ void __launch_bounds__(kThreads)
k_select_unite(const int32_t* __restrict__ count, const uint32_t* __restrict__ eids,
               const uint32_t* __restrict__ gkey, const int32_t* __restrict__ seg_start,
               const int32_t* __restrict__ k_graph, int64_t k_single,
               const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, int32_t* parent,
               uint8_t* merged, uint32_t* status) {
    spc::pdl_wait();
    const int64_t cnt = *count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rank = i, k = k_single;
        if (gkey) {
            const uint32_t b = gkey[i];
            rank = i - seg_start[b];
            k = k_graph[b];
        }
        if (rank < k) {
            const int32_t e = (int32_t)eids[i];
            uf_unite(parent, eu[e], ev[e], status);
            if (merged) merged[e] = 1;
        }
    }
}

// ---- exact selection of the k lightest forest edges (single graph) ------------------------------
// Composite key (score bits, eid) is unique.  Round r histograms an 11-bit digit (most
// significant first: the score's digits, then the eid's) over the items whose earlier digits
// match the ones picked so far.  The last block of a round to finish (ticket counter after a
// fence) picks that round's digit -- the bin holding the remaining rank -- and stores it with
// the rank left inside the bin, for the next round.
constexpr int kSelBits = 11;
constexpr int kSelBins = 1 << kSelBits;

template <class KT> struct SelBits {
    static constexpr int kKeyBits = sizeof(KT) == 8 ? 63 : 31;  // sign bit always clear
    static constexpr int kHiRounds = (kKeyBits + kSelBits - 1) / kSelBits;
    static constexpr int kRounds = kHiRounds + 3;                 // eid: 32 bits = 11 + 11 + 10
};

// digit r of (hi, lo) and its width
template <class KT>
__device__ __forceinline__ uint32_t sel_digit(KT hi, uint32_t lo, int r) {
    constexpr int H = SelBits<KT>::kHiRounds, KB = SelBits<KT>::kKeyBits;
    if (r < H) {
        const int top = KB - kSelBits * r;                 // exclusive upper bit of digit r
        const int lowb = top - kSelBits > 0 ? top - kSelBits : 0;
        return (uint32_t)(hi >> lowb) & ((1u << (top - lowb)) - 1u);
    }
    const int q = r - H;
    const int top = 32 - kSelBits * q;
    const int lowb = top - kSelBits > 0 ? top - kSelBits : 0;
    return (lo >> lowb) & ((1u << (top - lowb)) - 1u);
}

struct SelState {
    unsigned long long need;     // rank (1-based) still to find among the matching items
    uint32_t dig[16];
    uint32_t ticket[16];
};

// One select round: histogram of digit r over the items whose digits 0..r-1 are the ones
// picked so far; the last block to finish picks digit r.  n_dev, when given, holds the item
// count (a candidate list compacted on the device).
template <class KT>
__global__ void __launch_bounds__(kThreads)
k_rsel_round(int r, int64_t n_host, const int32_t* __restrict__ n_dev,
             const KT* __restrict__ keys, const uint32_t* __restrict__ vals,
             uint32_t* __restrict__ hist, SelState* st) {
    spc::pdl_wait();
    __shared__ uint32_t sh_h[kSelBins];
    __shared__ uint32_t sh_dig[16];
    __shared__ bool sh_last;
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) sh_h[b] = 0;
    if (threadIdx.x < 16) sh_dig[threadIdx.x] = st->dig[threadIdx.x];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const KT hi = keys[i];
        const uint32_t lo = vals[i];
        bool match = true;
        for (int q = 0; q < r; ++q) match = match && sel_digit<KT>(hi, lo, q) == sh_dig[q];
        if (match) atomicAdd(&sh_h[sel_digit<KT>(hi, lo, r)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBins; b += blockDim.x)
        if (sh_h[b]) atomicAdd(hist + r * kSelBins + b, sh_h[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&st->ticket[r], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    // the last block: pick the bin holding rank `need`
    __threadfence();
    constexpr int kPer = kSelBins / kThreads;
    const uint32_t* h = hist + r * kSelBins;
    unsigned long long loc = 0;
    uint32_t c[kPer];
    for (int j = 0; j < kPer; ++j) {
        c[j] = __ldcg(h + threadIdx.x * kPer + j);
        loc += c[j];
    }
    __shared__ unsigned long long sh_ws[32];
    const unsigned long long incl = block_incl_scan(loc, sh_ws);
    const unsigned long long need = st->need;
    unsigned long long run = incl - loc;
    if (run < need && incl >= need) {
        for (int j = 0; j < kPer; ++j) {
            if (run + c[j] >= need) {
                st->dig[r] = (uint32_t)(threadIdx.x * kPer + j);
                st->need = need - run;
                break;
            }
            run += c[j];
        }
    }
}

// Rounds r0 .. R-1 of the select in one CTA, over the candidates still matching after the
// full-width rounds (usually few): per round a shared-memory histogram of digit r over the
// items whose digits 0..r-1 are the picked ones, a block scan, the pick.
constexpr int kRestThreads = 1024;
constexpr int64_t kRestMax = 16384;  // candidates a single CTA takes

template <class KT>
__global__ void __launch_bounds__(kRestThreads)
k_rsel_rest(int r0, const int32_t* __restrict__ n_dev, const KT* __restrict__ keys,
            const uint32_t* __restrict__ vals, SelState* st) {
    spc::pdl_wait();
    constexpr int R = SelBits<KT>::kRounds;
    constexpr int kPer = kSelBins / kRestThreads;
    __shared__ uint32_t sh_h[kSelBins];
    __shared__ uint32_t sh_dig[16];
    __shared__ unsigned long long sh_ws[32];
    __shared__ unsigned long long sh_need;
    const int64_t n = *n_dev;
    if (threadIdx.x < 16) sh_dig[threadIdx.x] = st->dig[threadIdx.x];
    if (threadIdx.x == 0) sh_need = st->need;
    for (int r = r0; r < R; ++r) {
        for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) sh_h[b] = 0;
        __syncthreads();
        // candidates often share their digits (exactly equal scores): lanes holding the same
        // digit add with one shared-memory atomic
        for (int64_t i0 = 0; i0 < n; i0 += blockDim.x) {
            const int64_t i = i0 + threadIdx.x;
            bool match = i < n;
            uint32_t d = 0;
            if (match) {
                const KT hi = keys[i];
                const uint32_t lo = vals[i];
                for (int q = 0; q < r; ++q) match = match && sel_digit<KT>(hi, lo, q) == sh_dig[q];
                d = sel_digit<KT>(hi, lo, r);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, match ? d : 0xffffffffu);
            if (match && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&sh_h[d], (uint32_t)__popc(peers));
        }
        __syncthreads();
        unsigned long long loc = 0;
        uint32_t c[kPer];
        for (int j = 0; j < kPer; ++j) {
            c[j] = sh_h[threadIdx.x * kPer + j];
            loc += c[j];
        }
        const unsigned long long incl = block_incl_scan(loc, sh_ws);
        const unsigned long long need = sh_need;
        unsigned long long run = incl - loc;
        __syncthreads();  // every thread has read sh_need
        if (run < need && incl >= need) {
            for (int j = 0; j < kPer; ++j) {
                if (run + c[j] >= need) {
                    sh_dig[r] = (uint32_t)(threadIdx.x * kPer + j);
                    sh_need = need - run;
                    break;
                }
                run += c[j];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 16) st->dig[threadIdx.x] = sh_dig[threadIdx.x];
    if (threadIdx.x == 0) st->need = sh_need;
}

// keep the items whose digits 0..r are the ones picked so far (order is irrelevant to the
// select); one global atomic per block and pass
template <class KT>
__global__ void __launch_bounds__(kThreads)
k_rsel_compact(int r, int64_t n, const KT* __restrict__ keys, const uint32_t* __restrict__ vals,
               const SelState* __restrict__ st, KT* __restrict__ out_k,
               uint32_t* __restrict__ out_v, int32_t* __restrict__ out_n) {
    spc::pdl_wait();
    __shared__ uint32_t sh_dig[16];
    __shared__ int32_t sh_cnt, sh_base;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 16) sh_dig[threadIdx.x] = st->dig[threadIdx.x];
    __syncthreads();
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        bool keep = false;
        KT hi = 0;
        uint32_t lo = 0;
        if (i < n) {
            hi = keys[i];
            lo = vals[i];
            keep = true;
            for (int q = 0; q <= r; ++q) keep = keep && sel_digit<KT>(hi, lo, q) == sh_dig[q];
        }
        const unsigned b = __ballot_sync(0xffffffffu, keep);
        if (threadIdx.x == 0) sh_cnt = 0;
        __syncthreads();
        int wofs = 0;
        if (lane == 0 && b) wofs = atomicAdd(&sh_cnt, __popc(b));
        wofs = __shfl_sync(0xffffffffu, wofs, 0);
        __syncthreads();
        if (threadIdx.x == 0) sh_base = sh_cnt ? atomicAdd(out_n, sh_cnt) : 0;
        __syncthreads();
        if (keep) {
            const int pos = sh_base + wofs + __popc(b & ((1u << lane) - 1u));
            out_k[pos] = hi;
            out_v[pos] = lo;
        }
        __syncthreads();
    }
}

// unite the ends of every forest edge whose (score, eid) is at most the k-th smallest
template <class KT>
__global__ void __launch_bounds__(kThreads)
k_rsel_unite(int64_t n, const KT* __restrict__ keys, const uint32_t* __restrict__ vals,
             const SelState* __restrict__ st, const int32_t* __restrict__ eu,
             const int32_t* __restrict__ ev, int32_t* parent, uint8_t* merged, uint32_t* status) {
    spc::pdl_wait();
    constexpr int H = SelBits<KT>::kHiRounds, KB = SelBits<KT>::kKeyBits;
    KT thi = 0;
    for (int q = 0; q < H; ++q) {
        const int top = KB - kSelBits * q;
        const int lowb = top - kSelBits > 0 ? top - kSelBits : 0;
        thi |= (KT)st->dig[q] << lowb;
    }
    uint32_t tlo = 0;
    for (int q = 0; q < 3; ++q) {
        const int top = 32 - kSelBits * q;
        const int lowb = top - kSelBits > 0 ? top - kSelBits : 0;
        tlo |= st->dig[H + q] << lowb;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const KT hi = keys[i];
        const uint32_t lo = vals[i];
        if (hi < thi || (hi == thi && lo <= tlo)) {
            uf_unite(parent, eu[lo], ev[lo], status);
            if (merged) merged[lo] = 1;
        }
    }
}

// selection state, the per-round histograms (`words` of them) and the candidate count
__global__ void k_rsel_init(SelState* st, unsigned long long k, uint32_t* __restrict__ hist,
                            int words, int32_t* __restrict__ cand) {
    spc::pdl_wait();
    if (threadIdx.x == 0) { st->need = k; *cand = 0; }
    if (threadIdx.x < 16) { st->dig[threadIdx.x] = 0; st->ticket[threadIdx.x] = 0; }
    for (int i = threadIdx.x; i < words; i += blockDim.x) hist[i] = 0;
}

// root (= smallest member) of every node and the root flags
__global__ void __launch_bounds__(kThreads)
k_roots(int64_t n, int32_t* parent, int32_t* __restrict__ flag, int32_t* __restrict__ warn,
        uint32_t* status) {
    spc::pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *warn = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = uf_find(parent, (int32_t)x, status);
        flag[x] = (r == (int32_t)x) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kThreads)
k_lift(int64_t n, int32_t* parent, const int32_t* __restrict__ ids, int32_t* __restrict__ lift,
       uint32_t* status) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        lift[x] = ids[uf_find(parent, (int32_t)x, status)];
}

__global__ void k_graph_ptr_c(int64_t B, const int64_t* __restrict__ graph_ptr,
                              const int32_t* __restrict__ ids, const int64_t* __restrict__ targets,
                              int64_t* __restrict__ graph_ptr_c, int32_t* __restrict__ warn) {
    spc::pdl_wait();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= B;
         b += (int64_t)gridDim.x * blockDim.x) {
        graph_ptr_c[b] = ids[graph_ptr[b]];
        if (b < B) {
            const int64_t nc = (int64_t)ids[graph_ptr[b + 1]] - ids[graph_ptr[b]];
            if (nc > targets[b]) atomicOr(warn, 1);
        }
    }
}

// relabel (S6) from the second union-find in W.parent2, plus per-graph offsets and the status
spc_status finish_select(spc_context* ctx, const GraphView& g, const SelectArgs& sa, int32_t* lift,
                         int64_t* n_c_out, int64_t* graph_ptr_c, int32_t* status_out,
                         bool batched) {
    Work& W = ctx->work;
    const int64_t n = g.n;
    const int maxb = ctx->num_sms * 8;
    uint32_t* status = ctx->d_status;
    int32_t* counters = W.counters.as<int32_t>();
    int32_t* parent2 = W.parent2.as<int32_t>();
    // ---- 3. relabel ------------------------------------------------------------------
    int32_t* flag = W.flag.as<int32_t>();
    int32_t* ids = W.ids.as<int32_t>();
    int32_t* warn = counters + 2;
    SPC_LAUNCH(ctx, k_roots, grid_for(n, kThreads, maxb), kThreads, 0, n, parent2, flag, warn,
               status);
    SPC_TRY(scan_i32(ctx, flag, ids, n));
    SPC_LAUNCH(ctx, k_lift, grid_for(n, kThreads, maxb), kThreads, 0, n, parent2, ids, lift,
               status);
    if (batched) {
        SPC_LAUNCH(ctx, k_graph_ptr_c, grid_for(sa.B + 1, kThreads, maxb), kThreads, 0, sa.B,
                   sa.d_graph_ptr, ids, sa.d_targets, graph_ptr_c, warn);
    }
    int64_t vals[2];
    {
        const void* ptrs[2] = {ids + n, warn};
        const int bytes[2] = {4, 4};
        SPC_TRY(read_vals(ctx, 2, ptrs, bytes, vals));
    }
    const int64_t n_c = vals[0];
    const int32_t warn_b = (int32_t)vals[1];
    *n_c_out = n_c;
    *status_out = (batched ? warn_b != 0 : n_c > sa.target) ? SPC_WARN_TARGET_NOT_REACHED : SPC_OK;
    return SPC_OK;
}

// key_hist: the score-prefix histogram (kTauBins words, zeroed before each selection's first
// attempt and kept for its later ones), then the radix-select histograms of every round
// (zeroed by k_rsel_init); zeroed once on allocation
constexpr int kTauBins = 32768;
constexpr size_t kKeyHistBytes = (size_t)(kTauBins + SelBits<uint64_t>::kRounds * kSelBins) * 4;
static spc_status ensure_key_hist(spc_context* ctx) {
    return ensure_zeroed(ctx, ctx->work.key_hist, kKeyHistBytes);
}

template <class KT>
spc_status select_typed(spc_context* ctx, const GraphView& g, const KT* key,
                        const SelectArgs& sa, int32_t* lift, uint8_t* merged, int64_t* n_c_out,
                        int64_t* graph_ptr_c, int32_t* status_out) {
    Work& W = ctx->work;
    const int64_t n = g.n, m = g.m;
    const int maxb = ctx->num_sms * 8;
    uint32_t* status = ctx->d_status;
    int32_t* parent = W.parent.as<int32_t>();
    int32_t* counters = W.counters.as<int32_t>();  // [0..1] work-list counts, [2] warn flag
    const bool batched = sa.B > 1 || sa.d_graph_ptr != nullptr;

    // ---- 0. score prefix (single graph): the lightest ~1.5 (n - n_c) edges ------------------
    const int64_t k_need = batched ? 0 : (n - sa.target > 0 ? n - sa.target : 0);
    const int tau_shift = sizeof(KT) == 8 ? 48 : 16;
    uint32_t* tau_top = reinterpret_cast<uint32_t*>(counters + 12);
    // Kruskal's first n - n_c merges are the lightest n - n_c edges of the minimum spanning
    // forest of any score prefix whose forest has that many edges; the forest of a longer
    // prefix is the shorter prefix's forest plus Boruvka over the next slab of scores between
    // its components.  So the selection starts with about 1.5 (n - n_c) edges and, when their
    // forest falls short, extends it slab by slab (twice the edges each time) instead of
    // starting over.
    int64_t need = k_need + k_need / 2;
    bool use_prefix = !batched && m > 65536 && k_need > 0 && need < m;
    // the threshold's histogram samples one key chunk in eight on large selections
    const int hist_samp = m >= (int64_t{1} << 22) ? 3 : 0;
    uint32_t* tau_lo = reinterpret_cast<uint32_t*>(counters + 14);
    int32_t* pos = W.c_pos.as<int32_t>();
    int64_t n_msf = 0;
    // a batch: every graph its own prefix (k_graph_prefix), which needs the graph of every node
    int32_t* node_graph = W.node_graph.as<int32_t>();
    if (batched) {
        SPC_LAUNCH(ctx, k_node_graph, grid_for(n, kThreads, maxb), kThreads, 0, n, sa.B,
                   sa.d_graph_ptr, node_graph);
    }
    const bool use_gprefix = batched && m > 65536 && sa.d_graph_ptr && sa.d_targets;
    GraphSlab<KT> gs{nullptr, nullptr, nullptr};
    int64_t* g_need = nullptr;
    KT* g_tau = nullptr;
    KT* g_lo = nullptr;
    int32_t* g_short = nullptr;
    const int g_grid = (int)std::min<int64_t>(sa.B, (int64_t)ctx->num_sms * 8);
    if (use_gprefix) {
        SPC_TRY(ensure(ctx, W.g_need, (size_t)(sa.B + 1) * 8));
        SPC_TRY(ensure(ctx, W.g_tau, (size_t)(sa.B + 1) * sizeof(KT)));
        SPC_TRY(ensure(ctx, W.g_lo, (size_t)(sa.B + 1) * sizeof(KT)));
        SPC_TRY(ensure(ctx, W.g_short, 16));
        g_need = W.g_need.as<int64_t>();
        g_tau = W.g_tau.as<KT>();
        g_lo = W.g_lo.as<KT>();
        g_short = W.g_short.as<int32_t>();
        gs = GraphSlab<KT>{node_graph, g_tau, g_lo};
    }
    for (int attempt = 0;; ++attempt) {
        const bool two = MinKey<KT>::two_phase;
        if (use_gprefix) {
            if (attempt == 0)
                SPC_LAUNCH(ctx, k_graph_prefix<KT>, g_grid, kGpThreads, 0, sa.B, 0,
                           sa.d_graph_ptr, W.up_ptr.as<int32_t>(), sa.d_targets, key,
                           W.msf.as<uint8_t>(), g_need, g_tau, g_lo, g_short);
        } else if (use_prefix) {
            SPC_TRY(ensure_key_hist(ctx));
            static std::atomic<unsigned long long> attr_devs{0};  // devices already set up
            const unsigned long long bit = 1ull << (ctx->device & 63);
            if (!(attr_devs.load() & bit)) {
                SPC_CUDA(cudaFuncSetAttribute(k_key_hist<KT>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              32768 * 4));
                attr_devs.fetch_or(bit);
            }
            if (attempt > 0) {
                // the histogram is still there: only the threshold moves up
                SPC_LAUNCH(ctx, k_bump_slab, 1, 32, 0, tau_top, tau_lo);
            } else {
                SPC_CUDA(cudaMemsetAsync(W.key_hist.p, 0, (size_t)kTauBins * 4, ctx->stream));
                note_bytes(ctx, (double)m * sizeof(KT) / (double)(1 << hist_samp));
                SPC_LAUNCH(ctx, k_key_hist<KT>, ctx->num_sms, 1024, 32768 * 4, m, key,
                           tau_shift, hist_samp, W.key_hist.as<uint32_t>());
            }
            // the histogram counts one key in 2^hist_samp
            const int64_t need_s = (need + (int64_t{1} << hist_samp) - 1) >> hist_samp;
            SPC_LAUNCH(ctx, k_pick_tau, 1, 1024, 0, W.key_hist.as<uint32_t>(), need_s, tau_top);
        } else if (attempt > 0) {
            SPC_LAUNCH(ctx, k_bump_slab, 1, 32, 0, tau_top, tau_lo);
        }
        const uint32_t* slab_lo = (attempt > 0 && !use_gprefix) ? tau_lo : nullptr;
        // the slab of a very large single-graph selection: its edges become the first work
        // list, so the first round does not sweep every edge.  Below kSlabListMin edges, and
        // for a batch's per-graph slabs, the extra pass costs more than the sweep it replaces.
        const bool slab_list = !batched && m >= kSlabListMin && (use_prefix || slab_lo) &&
                               (reinterpret_cast<uintptr_t>(key) & 15) == 0;
        if (attempt == 0) {
            SPC_LAUNCH(ctx, k_bv_init, grid_for(n > m ? n : m + 1, kThreads, maxb), kThreads, 0,
                       n, m, parent, W.best_k[0].as<unsigned long long>(),
                       W.best_k[1].as<unsigned long long>(),
                       two ? W.best_e[0].as<int32_t>() : nullptr,
                       two ? W.best_e[1].as<int32_t>() : nullptr, W.msf.as<uint8_t>(), merged,
                       counters);
        } else {
            SPC_LAUNCH(ctx, k_bv_reinit, grid_for(n, kThreads, maxb), kThreads, 0, n,
                       W.best_k[0].as<unsigned long long>(),
                       W.best_k[1].as<unsigned long long>(),
                       two ? W.best_e[0].as<int32_t>() : nullptr,
                       two ? W.best_e[1].as<int32_t>() : nullptr, counters);
        }
        if (slab_list) {
            note_bytes(ctx, (double)m * sizeof(KT) + (double)std::min<int64_t>(need, m) * 20);
            SPC_LAUNCH(ctx, k_slab_list<KT>, grid_for(m, kThreads * kSlItems, maxb), kThreads,
                       0, m, W.eu.as<int32_t>(), W.ev.as<int32_t>(), key, tau_shift,
                       use_prefix ? tau_top : nullptr, slab_lo, W.wl_e[0].as<int32_t>(),
                       W.wl_u[0].as<int32_t>(), W.wl_v[0].as<int32_t>(), counters);
        }
        // ---- 1. Boruvka minimum spanning forest (of the prefix) ---------------------------
        // the first round reads the edges themselves (filtered by the slab) unless the slab
        // list holds them; its count is then known on the device only
        const bool scan0 = !slab_list;
        int64_t cur = m;
        for (int round = 0; cur > 0; ++round) {
            const int in = round & 1, out = in ^ 1;
            const int par = round & 1;
            const int first = (round == 0 && scan0) ? 1 : 0;
            const int direct = (round == 0 && attempt == 0) ? 1 : 0;
            if (cur <= kFinishMax && (round > 0 || scan0)) {  // the remaining rounds in one CTA
                note_bytes(ctx, first ? (double)m * (8 + sizeof(KT))
                                      : (double)cur * (12 + sizeof(KT) + 8 + 32 + 12));
                SPC_LAUNCH(ctx, k_bv_finish<KT>, 1, kFinishThreads, 0, first, par,
                           m, counters + in, W.wl_e[in].as<int32_t>(), W.wl_u[in].as<int32_t>(),
                           W.wl_v[in].as<int32_t>(), W.wl_e[out].as<int32_t>(),
                           W.wl_u[out].as<int32_t>(), W.wl_v[out].as<int32_t>(),
                           W.eu.as<int32_t>(), W.ev.as<int32_t>(), key, tau_shift,
                           use_prefix ? tau_top : nullptr, slab_lo, gs, parent,
                           W.best_k[0].as<unsigned long long>(),
                           W.best_k[1].as<unsigned long long>(),
                           MinKey<KT>::two_phase ? W.best_e[0].as<int32_t>() : nullptr,
                           MinKey<KT>::two_phase ? W.best_e[1].as<int32_t>() : nullptr,
                           W.msf.as<uint8_t>(), status);
                break;
            }
            // algorithmic bytes: the first round reads every edge's ends and key; a later one
            // reads each work-list item (e, u, v) and key, walks two parents, lowers two best
            // slots (read and write) and writes the item back
            // (a first round over the slab list: about `need` items)
            const double items = round > 0 ? (double)cur : (double)std::min<int64_t>(need, m);
            note_bytes(ctx, first ? (double)m * (8 + sizeof(KT))
                                  : items * (12 + sizeof(KT) + 8 + 32 + 12));
            SPC_LAUNCH(ctx, k_bv_minkey<KT>,
                       grid_for(cur, kThreads * kMkItems, maxb), kThreads, 0,
                       first, direct, m, counters + in,
                       W.wl_e[in].as<int32_t>(), W.wl_u[in].as<int32_t>(),
                       W.wl_v[in].as<int32_t>(), W.eu.as<int32_t>(), W.ev.as<int32_t>(), key,
                       tau_shift, use_prefix ? tau_top : nullptr, slab_lo, gs, parent,
                       W.best_k[par].as<unsigned long long>(), W.wl_e[out].as<int32_t>(),
                       W.wl_u[out].as<int32_t>(), W.wl_v[out].as<int32_t>(), counters + out,
                       status);
            if (MinKey<KT>::two_phase) {
                note_bytes(ctx, (double)cur * (12 + 8 + 16 + 8));
                SPC_LAUNCH(ctx, k_bv_tiebreak, grid_for(cur, kThreads, maxb), kThreads, 0,
                           counters + out, W.wl_e[out].as<int32_t>(), W.wl_u[out].as<int32_t>(),
                           W.wl_v[out].as<int32_t>(),
                           reinterpret_cast<const unsigned long long*>(key),
                           W.best_k[par].as<unsigned long long>(), W.best_e[par].as<int32_t>());
            }
            // each item and the two best slots read, the forest flag written, one parent swap
            note_bytes(ctx, (double)cur * (12 + 24 + 1 + 8));
            SPC_LAUNCH(ctx, k_bv_hook<KT>, grid_for(cur, kThreads, maxb), kThreads, 0,
                       counters + out, W.wl_e[out].as<int32_t>(), W.wl_u[out].as<int32_t>(),
                       W.wl_v[out].as<int32_t>(), W.best_k[par].as<unsigned long long>(),
                       W.best_e[par].as<int32_t>(), W.best_k[par ^ 1].as<unsigned long long>(),
                       W.best_e[par ^ 1].as<int32_t>(), parent, W.msf.as<uint8_t>(),
                       counters + in, status);
            // next work-list size (a capture replays the recorded round count)
            SPC_TRY(read_loop_count(ctx, counters + out, &cur));
            // every round at least halves the components that still have edges
            if (round > 64) return SPC_ERR_TIMEOUT;
            // slot `out` (list and count) is the next round's input
        }
        SPC_TRY(scan_flags_u8(ctx, W.msf.as<uint8_t>(), pos, m));
        SPC_TRY(read_i32(ctx, pos + m, &n_msf));
        if (use_gprefix) {
            // graphs whose forest falls short take their next slab; done when none does
            SPC_CUDA(cudaMemsetAsync(g_short, 0, sizeof(int32_t), ctx->stream));
            SPC_LAUNCH(ctx, k_graph_prefix<KT>, g_grid, kGpThreads, 0, sa.B, attempt + 1,
                       sa.d_graph_ptr, W.up_ptr.as<int32_t>(), sa.d_targets, key,
                       W.msf.as<uint8_t>(), g_need, g_tau, g_lo, g_short);
            int64_t n_short = 0;
            SPC_TRY(read_i32(ctx, g_short, &n_short));
            if (n_short == 0) break;
            if (attempt > 64) return SPC_ERR_TIMEOUT;  // each slab doubles: never reached
            continue;
        }
        // the prefix's forest holds Kruskal's first n_msf merges; enough when >= n - n_c
        if (!use_prefix || n_msf >= k_need) break;
        // the next slab: twice the edges, or, when the forest came within 15 % of n - n_c,
        // the prefix its yield so far extrapolates to, and a quarter more
        int64_t next = need * 2;
        if (n_msf * 20 >= k_need * 17) {
            const int64_t est = (int64_t)((double)need * (double)k_need / (double)n_msf * 1.25);
            next = std::min(next, std::max(est, need + need / 8));
        }
        need = next;
        if (need >= m) use_prefix = false;  // the last slab: every remaining score
    }
    // ---- 2. lightest forest edges per graph ---------------------------------------------
    KT* sk = W.sel_key.as<KT>();
    uint32_t* sv = W.sel_val.as<uint32_t>();
    SPC_LAUNCH(ctx, k_compact_msf<KT>, grid_for(m, kThreads, maxb), kThreads, 0, m,
               W.msf.as<uint8_t>(), pos, key, sk, sv);
    const int key_bits = sizeof(KT) == 8 ? 63 : 31;  // scores are >= +0: sign bit clear
    const int64_t k_single_sel = batched ? 0 : (n - sa.target > 0 ? n - sa.target : 0);
    if (!batched && k_single_sel > 0 && k_single_sel < n_msf) {
        // single graph, proper subset: exact radix select of the k lightest, no sort
        constexpr int R = SelBits<KT>::kRounds;
        SPC_TRY(ensure_key_hist(ctx));
        uint32_t* hist = W.key_hist.as<uint32_t>() + kTauBins;
        SelState* sst = reinterpret_cast<SelState*>(counters + 16);
        int32_t* cn = counters + 52;
        SPC_LAUNCH(ctx, k_rsel_init, 1, 1024, 0, sst, (unsigned long long)k_single_sel, hist,
                   R * kSelBins, cn);
        const int gsel = grid_for(n_msf, kThreads, ctx->num_sms * 2);
        // two rounds over the whole forest, then the rest over the items still matching
        constexpr int kFull = 2;
        KT* ck = W.sel_key2.as<KT>();
        uint32_t* cv = W.sel_val2.as<uint32_t>();
        for (int r = 0; r < kFull; ++r) {
            SPC_LAUNCH(ctx, k_rsel_round<KT>, gsel, kThreads, 0, r, n_msf, nullptr, sk, sv,
                       hist, sst);
        }
        SPC_LAUNCH(ctx, k_rsel_compact<KT>, grid_for(n_msf, kThreads, maxb), kThreads, 0,
                   kFull - 1, n_msf, sk, sv, sst, ck, cv, cn);
        // few candidates (the usual case): the remaining rounds in one CTA; many (a level
        // where a large share of the forest has exactly equal scores): a launch per round
        int64_t ncand = 0;
        SPC_TRY(read_i32(ctx, cn, &ncand));
        if (ncand <= kRestMax) {
            SPC_LAUNCH(ctx, k_rsel_rest<KT>, 1, kRestThreads, 0, kFull, cn, ck, cv, sst);
        } else {
            for (int r = kFull; r < R; ++r)
                SPC_LAUNCH(ctx, k_rsel_round<KT>, grid_for(ncand, kThreads, ctx->num_sms * 2),
                           kThreads, 0, r, 0, cn, ck, cv, hist, sst);
        }
        int32_t* parent2 = W.parent2.as<int32_t>();
        SPC_LAUNCH(ctx, k_iota, grid_for(n, kThreads, maxb), kThreads, 0, parent2, n);
        SPC_LAUNCH(ctx, k_rsel_unite<KT>, grid_for(n_msf, kThreads, maxb), kThreads, 0, n_msf, sk,
                   sv, sst, W.eu.as<int32_t>(), W.ev.as<int32_t>(), parent2, merged, status);
        return finish_select(ctx, g, sa, lift, n_c_out, graph_ptr_c, status_out, batched);
    }
    if (sizeof(KT) == 8) {
        SPC_TRY(radix_sort_u64(ctx, reinterpret_cast<uint64_t*>(sk), sv,
                               W.sel_key2.as<uint64_t>(), W.sel_val2.as<uint32_t>(), n_msf,
                               key_bits));
    } else {
        SPC_TRY(radix_sort_u32(ctx, reinterpret_cast<uint32_t*>(sk), sv,
                               W.sel_key2.as<uint32_t>(), W.sel_val2.as<uint32_t>(), n_msf,
                               key_bits));
    }
    uint32_t* gkey = nullptr;
    int32_t* seg_start = nullptr;
    int32_t* k_graph = nullptr;
    int32_t* cnt_dev = counters + 3;
    SPC_CUDA(cudaMemcpyAsync(cnt_dev, pos + m, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                             ctx->stream));
    if (batched) {
        gkey = W.sel_key2.as<uint32_t>();  // reuse: free after the score sort
        uint32_t* gval = sv;
        SPC_LAUNCH(ctx, k_graph_keys, grid_for(n_msf, kThreads, maxb), kThreads, 0, cnt_dev,
                   gval, W.eu.as<int32_t>(), node_graph, gkey);
        int gbits = 1;
        while ((1ll << gbits) < sa.B) ++gbits;
        // stable sort by graph id keeps the score order inside every graph
        SPC_TRY(radix_sort_u32(ctx, gkey, gval, W.t_key.as<uint32_t>(), W.t_val.as<uint32_t>(),
                               n_msf, gbits));
        seg_start = W.seg_start.as<int32_t>();
        k_graph = W.k_graph.as<int32_t>();
        SPC_LAUNCH(ctx, k_graph_segments, grid_for(sa.B, kThreads, maxb), kThreads, 0, sa.B,
                   sa.d_graph_ptr, sa.d_targets, W.up_ptr.as<int32_t>(), pos, seg_start,
                   k_graph);
    }
    int32_t* parent2 = W.parent2.as<int32_t>();
    SPC_LAUNCH(ctx, k_iota, grid_for(n, kThreads, maxb), kThreads, 0, parent2, n);
    const int64_t k_single = batched ? 0 : (n - sa.target > 0 ? n - sa.target : 0);
    if (n_msf > 0) {
        SPC_LAUNCH(ctx, k_select_unite, grid_for(n_msf, kThreads, maxb), kThreads, 0, cnt_dev,
                   sv, gkey, seg_start, k_graph, k_single, W.eu.as<int32_t>(),
                   W.ev.as<int32_t>(), parent2, merged, status);
    }
    return finish_select(ctx, g, sa, lift, n_c_out, graph_ptr_c, status_out, batched);
}

}  // namespace

spc_status run_select(spc_context* ctx, const GraphView& g, const void* score,
                      const SelectArgs& sa, int32_t* lift, uint8_t* merged, int64_t* n_c,
                      int64_t* graph_ptr_c, int32_t* status) {
    if (score_is_f32(g.wtype))
        return select_typed<unsigned int>(ctx, g, static_cast<const unsigned int*>(score), sa,
                                          lift, merged, n_c, graph_ptr_c, status);
    return select_typed<unsigned long long>(ctx, g, static_cast<const unsigned long long*>(score),
                                            sa, lift, merged, n_c, graph_ptr_c, status);
}

}  // namespace spc
