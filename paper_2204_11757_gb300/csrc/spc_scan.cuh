// Device-wide exclusive scan fused with its producer and consumer.
//
// One pass with decoupled look-back (Merrill and Garland, "Single-pass parallel prefix scan
// with decoupled look-back", 2016): each tile of 4096 items publishes its sum, reads its
// predecessors' published sums (a warp looks at 32 at a time) and publishes its inclusive
// prefix.  Items come from a loader functor and go to a storer functor, so the kernel that
// computes the scanned values and the kernel that consumes the prefixes need not exist: no
// value or prefix array makes a round trip through memory, and there is one launch.
//
//   T   Ld::operator()(int64_t g) const           the value of item g (g < n), >= 0
//   St::Local St::begin() const                   per-thread state
//   void St::operator()(Local&, int64_t g, bool valid, T excl, T val) const
//                                                 called by every thread for every item slot
//                                                 of its tile (warp-uniform; valid: g < n)
//   void St::finish(Local&) const                 once per block, by every thread, at the end
//   void St::total(T tot) const                   the grand total, once
//
// Every wait on a predecessor is bounded (DEV_TIMEOUT in *err).  The tile statuses live in
// the context's scan temporaries and are zero between scans: the tile that finishes last
// resets them.
#pragma once
#include "spc_internal.cuh"

namespace spc {
namespace scanf {

constexpr int ST = 256;            // threads
constexpr int SI = 16;             // items per thread
constexpr int STILE = ST * SI;     // 4096 items per tile
constexpr int kSmallThreads = 1024;
constexpr int64_t kSmallMax = 16384;

// Tile status words: 2 flag bits over a 62-bit sum (every scanned value is >= 0).
constexpr unsigned long long kScanAgg = 1ull << 62;   // the tile's own sum is published
constexpr unsigned long long kScanInc = 2ull << 62;   // the sum of all tiles up to it
constexpr unsigned long long kScanVal = (1ull << 62) - 1ull;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive block scan of one value per thread (blockDim.x == ST); *total = the block's sum
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T wsum[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T s = (lane < ST / 32) ? wsum[lane] : T(0);
        s = warp_incl_scan(s);
        if (lane < ST / 32) wsum[lane] = s;
    }
    __syncthreads();
    T before = (warp > 0) ? wsum[warp - 1] : T(0);
    *total = wsum[ST / 32 - 1];
    __syncthreads();
    return before + incl - v;
}

// One pass over nt tiles.  Tiles take ids in launch order from *tile_ctr, so every tile a
// tile waits for has already started.  A tile reads all of its items before it stores any.
template <class T, class Ld, class St>
__global__ void __launch_bounds__(ST) k_scan_fused(Ld ld, St st, int64_t n,
                                                   unsigned long long* status,
                                                   uint32_t* tile_ctr, int64_t nt,
                                                   uint32_t* err) {
    spc::pdl_wait();
    __shared__ T buf[STILE + STILE / 32];
    __shared__ uint32_t sh_tile;
    __shared__ T sh_prefix;
    __shared__ bool sh_last;
    uint32_t* done_ctr = tile_ctr + 1;
    if (threadIdx.x == 0) sh_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = sh_tile;
    const int64_t base = tile * STILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T v[SI];
#pragma unroll
    for (int k = 0; k < SI; ++k) {  // all loads in flight before the first use
        const int64_t g = base + (int64_t)k * ST + threadIdx.x;
        v[k] = (g < n) ? ld(g) : T(0);
    }
#pragma unroll
    for (int k = 0; k < SI; ++k) {
        const int i = k * ST + threadIdx.x;
        buf[i + (i >> 5)] = v[k];
    }
    __syncthreads();
    T loc[SI];
    T run = 0;
#pragma unroll
    for (int j = 0; j < SI; ++j) {
        const int i = threadIdx.x * SI + j;
        loc[j] = run;
        run += buf[i + (i >> 5)];
    }
    T tot;
    const T pre = block_excl_scan<T>(run, &tot);
    if (warp == 0) {
        unsigned long long prefix = 0;
        if (tile > 0) {
            if (lane == 0) atomicExch(status + tile, kScanAgg | (unsigned long long)tot);
            int64_t top = tile - 1;
            bool done = false;
            while (!done) {
                const int64_t idx = top - lane;
                unsigned long long w = kScanInc;  // before tile 0: an inclusive zero
                if (idx >= 0) w = *reinterpret_cast<volatile unsigned long long*>(status + idx);
                uint32_t spins = 0;
                while (__any_sync(0xffffffffu, (w >> 62) == 0ull)) {
                    if ((w >> 62) == 0ull)
                        w = *reinterpret_cast<volatile unsigned long long*>(status + idx);
                    if (++spins > spin_limit(err)) {
                        if (lane == 0) atomicOr(err, DEV_TIMEOUT);
                        w = kScanInc;  // give up; the call reports the timeout
                    }
                }
                const unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2ull);
                const int stop = inc ? __ffs(inc) - 1 : 31;
                unsigned long long part = (lane <= stop) ? (w & kScanVal) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                prefix += part;
                done = inc != 0u;
                top -= 32;
            }
        }
        if (lane == 0) {
            atomicExch(status + tile, kScanInc | (prefix + (unsigned long long)tot));
            sh_prefix = (T)prefix;
        }
    }
    __syncthreads();
    const T off = sh_prefix + pre;
#pragma unroll
    for (int j = 0; j < SI; ++j) {
        const int i = threadIdx.x * SI + j;
        buf[i + (i >> 5)] = off + loc[j];
    }
    __syncthreads();
    typename St::Local sl = st.begin();
#pragma unroll
    for (int k = 0; k < SI; ++k) {
        const int i = k * ST + threadIdx.x;
        const int64_t g = base + i;
        st(sl, g, g < n, buf[i + (i >> 5)], v[k]);
    }
    st.finish(sl);
    if (tile == nt - 1 && threadIdx.x == 0) st.total(sh_prefix + tot);
    // The tile that finishes last resets the statuses and counters for the next scan: every
    // other tile has counted itself done after its look-back, so none reads them again.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        sh_last = atomicAdd(done_ctr, 1u) == (uint32_t)(nt - 1);
    }
    __syncthreads();
    if (sh_last) {
        __threadfence();
        for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) status[t] = 0ull;
        if (threadIdx.x == 0) {
            *tile_ctr = 0u;
            *done_ctr = 0u;
        }
    }
}

// small inputs: one CTA scans everything in chunks of 4 items per thread with a carry
template <class T, class Ld, class St>
__global__ void __launch_bounds__(kSmallThreads) k_scan_small_fused(Ld ld, St st, int64_t n) {
    spc::pdl_wait();
    __shared__ T wsum[kSmallThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename St::Local sl = st.begin();
    T carry = 0;
    for (int64_t base = 0; base < n; base += (int64_t)kSmallThreads * 4) {
        T v[4];
        T run = 0;
        const int64_t i0 = base + (int64_t)threadIdx.x * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (i0 + j < n) ? ld(i0 + j) : T(0);
            run += v[j];
        }
        T incl = warp_incl_scan(run);
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) wsum[lane] = warp_incl_scan(wsum[lane]);
        __syncthreads();
        T pre = carry + (warp > 0 ? wsum[warp - 1] : T(0)) + incl - run;
        const T tot = wsum[kSmallThreads / 32 - 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            st(sl, i0 + j, i0 + j < n, pre, v[j]);
            pre += v[j];
        }
        carry += tot;
        __syncthreads();
    }
    st.finish(sl);
    if (threadIdx.x == 0) st.total(carry);
}

}  // namespace scanf

// Scan of n items from `ld` into `st` on the context's current stream; `bytes`: the
// operation's algorithmic DRAM bytes for the kernel profile (0: no model).
template <class T, class Ld, class St>
spc_status scan_fused(spc_context* ctx, int64_t n, const Ld& ld, const St& st, double bytes) {
    using namespace scanf;
    if (n <= kSmallMax) {
        SPC_LAUNCH(ctx, (k_scan_small_fused<T, Ld, St>), 1, kSmallThreads, 0, ld, st, n);
        return SPC_OK;
    }
    const int64_t nt = (n + STILE - 1) / STILE;
    // statuses [nt] | tile counter, done counter: zero between scans, zeroed when allocated
    Buf& tmp = on_side(ctx) ? ctx->work.scan_tmp_side : ctx->work.scan_tmp;
    SPC_TRY(ensure_zeroed(ctx, tmp, (size_t)(nt + 1) * 8));
    unsigned long long* status = tmp.as<unsigned long long>();
    uint32_t* tile_ctr = reinterpret_cast<uint32_t*>(status + nt);
    if (bytes > 0) note_bytes(ctx, bytes);
    SPC_LAUNCH(ctx, (k_scan_fused<T, Ld, St>), (unsigned)nt, ST, 0, ld, st, n, status, tile_ctr,
               nt, ctx->d_status);
    return SPC_OK;
}

// ---- plain array loader and storer ----------------------------------------------------------
template <class In, class T>
struct ArrayLd {
    const In* in;
    __device__ T operator()(int64_t g) const { return (T)in[g]; }
};

// out[g] = exclusive prefix, out[n] = total
template <class T, class Out>
struct ArraySt {
    Out* out;
    int64_t n;
    struct Local {};
    __device__ Local begin() const { return Local{}; }
    __device__ void operator()(Local&, int64_t g, bool valid, T excl, T) const {
        if (valid) out[g] = (Out)excl;
    }
    __device__ void finish(Local&) const {}
    __device__ void total(T tot) const { out[n] = (Out)tot; }
};

// Two counts scanned at once: item g is (a[g] << 31) | b[g] (both sums below 2^31, so the
// packed sums never carry between the halves).  Writes both exclusive prefixes and totals.
struct PairLd {
    const int32_t* a;
    const int32_t* b;
    __device__ unsigned long long operator()(int64_t g) const {
        return ((unsigned long long)(uint32_t)a[g] << 31) | (uint32_t)b[g];
    }
};

}  // namespace spc
