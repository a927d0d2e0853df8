// Device-wide exclusive scan.  With a context: one pass with decoupled look-back (Merrill and
// Garland, "Single-pass parallel prefix scan with decoupled look-back", 2016): each tile of
// 4096 items publishes its sum, reads its predecessors' published sums (a warp looks at 32
// at a time) and publishes its inclusive prefix, so the input is read once and the output
// written once.  Every wait on a predecessor is bounded.  Without a context (the
// allocation-free entry point): three launches (reduce, scan of tile sums, downsweep) with no
// inter-block waits.
#include "spc_internal.cuh"

namespace spc {

namespace {

constexpr int ST = 256;            // threads
constexpr int SI = 16;             // items per thread
constexpr int STILE = ST * SI;     // 4096 items per tile

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

// exclusive block scan of one value per thread; returns the exclusive prefix, *total = sum
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

template <class In, class T>
__global__ void __launch_bounds__(ST) k_scan_reduce(const In* in, int64_t n, T* tile_sums) {
    spc::pdl_wait();
    const int64_t base = (int64_t)blockIdx.x * STILE;
    T s = 0;
#pragma unroll 4
    for (int k = 0; k < SI; ++k) {
        int64_t i = base + (int64_t)k * ST + threadIdx.x;
        if (i < n) s += (T)in[i];
    }
    T total;
    block_excl_scan<T>(s, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of nt tile sums in place, writes the grand total to *total_out
template <class T>
__global__ void __launch_bounds__(ST) k_scan_tiles(T* tile_sums, int64_t nt, T* total_out) {
    spc::pdl_wait();
    T carry = 0;
    for (int64_t base = 0; base < nt; base += ST) {
        int64_t i = base + threadIdx.x;
        T v = (i < nt) ? tile_sums[i] : T(0);
        T tot;
        T ex = block_excl_scan<T>(v, &tot);
        if (i < nt) tile_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <class In, class T, class Out>
__global__ void __launch_bounds__(ST) k_scan_down(const In* in, int64_t n, const T* tile_offs,
                                                  Out* out) {
    spc::pdl_wait();
    // padded shared tile: index i -> i + i/32 avoids bank conflicts on the blocked reads
    __shared__ T buf[STILE + STILE / 32];
    const int64_t base = (int64_t)blockIdx.x * STILE;
#pragma unroll 4
    for (int k = 0; k < SI; ++k) {
        int i = k * ST + threadIdx.x;
        int64_t g = base + i;
        buf[i + (i >> 5)] = (g < n) ? (T)in[g] : T(0);
    }
    __syncthreads();
    T loc[SI];
    T run = 0;
#pragma unroll
    for (int j = 0; j < SI; ++j) {
        int i = threadIdx.x * SI + j;
        loc[j] = run;
        run += buf[i + (i >> 5)];
    }
    T tot;
    T pre = block_excl_scan<T>(run, &tot);
    const T off = tile_offs[blockIdx.x] + pre;
#pragma unroll
    for (int j = 0; j < SI; ++j) {
        int i = threadIdx.x * SI + j;
        buf[i + (i >> 5)] = off + loc[j];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < SI; ++k) {
        int i = k * ST + threadIdx.x;
        int64_t g = base + i;
        if (g < n) out[g] = (Out)buf[i + (i >> 5)];
    }
}

template <class T, class Out>
__global__ void k_copy_total(const T* total, Out* dst) {
    spc::pdl_wait();
    if (threadIdx.x == 0) *dst = (Out)*total;
}

// small inputs: one CTA scans everything in chunks of 4 items per thread with a carry, and
// writes the total at out[n] (one launch instead of three plus a copy)
constexpr int kSmallThreads = 1024;
constexpr int64_t kSmallMax = 16384;

template <class In, class T, class Out>
__global__ void __launch_bounds__(kSmallThreads) k_scan_small(const In* in, int64_t n, Out* out) {
    spc::pdl_wait();
    __shared__ T wsum[kSmallThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T carry = 0;
    for (int64_t base = 0; base < n; base += (int64_t)kSmallThreads * 4) {
        T v[4];
        T run = 0;
        const int64_t i0 = base + (int64_t)threadIdx.x * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = (i0 + j < n) ? (T)in[i0 + j] : T(0);
            run += v[j];
        }
        T incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            T s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                T t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        T pre = carry + (warp > 0 ? wsum[warp - 1] : T(0)) + incl - run;
        const T tot = wsum[kSmallThreads / 32 - 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (i0 + j < n) out[i0 + j] = (Out)pre;
            pre += v[j];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = (Out)carry;
}

// Tile status words: 2 flag bits over a 62-bit sum (every scanned value is >= 0).
constexpr unsigned long long kScanAgg = 1ull << 62;   // the tile's own sum is published
constexpr unsigned long long kScanInc = 2ull << 62;   // the sum of all tiles up to it
constexpr unsigned long long kScanVal = (1ull << 62) - 1ull;

// One pass: tiles take ids in launch order from *tile_ctr, so every tile a tile waits for has
// already started.  status[0..nt) and *tile_ctr start at zero.  Works in place (in == out):
// a tile reads all of its items before it writes any, and reads no other tile's items.
template <class In, class T, class Out>
__global__ void __launch_bounds__(ST) k_scan_onepass(const In* in, int64_t n, Out* out,
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
    In v[SI];
#pragma unroll
    for (int k = 0; k < SI; ++k) {  // all loads in flight before the first use
        const int64_t g = base + (int64_t)k * ST + threadIdx.x;
        v[k] = (g < n) ? in[g] : In(0);
    }
#pragma unroll
    for (int k = 0; k < SI; ++k) {
        const int i = k * ST + threadIdx.x;
        buf[i + (i >> 5)] = (T)v[k];
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
                    if (++spins > kSpinLimit) {
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
#pragma unroll
    for (int k = 0; k < SI; ++k) {
        const int i = k * ST + threadIdx.x;
        const int64_t g = base + i;
        if (g < n) out[g] = (Out)buf[i + (i >> 5)];
    }
    if (tile == nt - 1 && threadIdx.x == 0) out[n] = (Out)(sh_prefix + tot);
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

template <class In, class T, class Out>
spc_status scan_impl(spc_context* ctx, const In* in, Out* out, int64_t n) {
    if (n <= kSmallMax) {
        SPC_LAUNCH(ctx, (k_scan_small<In, T, Out>), 1, kSmallThreads, 0, in, n, out);
        return SPC_OK;
    }
    const int64_t nt = (n + STILE - 1) / STILE;
    // statuses [nt] | tile counter, done counter: all zero between scans (each scan resets
    // them at its end); zeroed here only when the block is new
    const size_t need = (size_t)(nt + 1) * 8;
    Buf& tmp = on_side(ctx) ? ctx->work.scan_tmp_side : ctx->work.scan_tmp;
    SPC_TRY(ensure_zeroed(ctx, tmp, need));
    unsigned long long* status = tmp.as<unsigned long long>();
    uint32_t* tile_ctr = reinterpret_cast<uint32_t*>(status + nt);
    note_bytes(ctx, (double)n * (sizeof(In) + sizeof(Out)));  // input read, output written
    SPC_LAUNCH(ctx, (k_scan_onepass<In, T, Out>), (unsigned)nt, ST, 0, in, n, out, status,
               tile_ctr, nt, ctx->d_status);
    return SPC_OK;
}

}  // namespace

spc_status scan_i32(spc_context* ctx, const int32_t* in, int32_t* out, int64_t n) {
    return scan_impl<int32_t, int32_t, int32_t>(ctx, in, out, n);
}

spc_status scan_i64(spc_context* ctx, const int32_t* in, int64_t* out, int64_t n) {
    return scan_impl<int32_t, int64_t, int64_t>(ctx, in, out, n);
}

spc_status scan_i64_i64(spc_context* ctx, const int64_t* in, int64_t* out, int64_t n) {
    return scan_impl<int64_t, int64_t, int64_t>(ctx, in, out, n);
}

spc_status scan_flags_u8(spc_context* ctx, const uint8_t* in, int32_t* out, int64_t n) {
    return scan_impl<uint8_t, int32_t, int32_t>(ctx, in, out, n);
}

}  // namespace spc

namespace spc {

// Context-free exclusive scan of n int32 values (out[n] = total) on `stream`, with caller-owned
// temporaries: tmp must hold scan_raw_tmp_elems(n) int32 values.
int64_t scan_raw_tmp_elems(int64_t n) { return (n + STILE - 1) / STILE + 1; }

cudaError_t scan_i32_raw(cudaStream_t stream, const int32_t* in, int32_t* out, int64_t n,
                         int32_t* tmp) {
    const int64_t nt = (n + STILE - 1) / STILE;
    int32_t* tiles = tmp;
    int32_t* total = tmp + nt;
    if (nt > 0) k_scan_reduce<int32_t, int32_t><<<(unsigned)nt, ST, 0, stream>>>(in, n, tiles);
    k_scan_tiles<int32_t><<<1, ST, 0, stream>>>(tiles, nt, total);
    if (nt > 0) k_scan_down<int32_t, int32_t, int32_t><<<(unsigned)nt, ST, 0, stream>>>(in, n, tiles, out);
    k_copy_total<int32_t, int32_t><<<1, 32, 0, stream>>>(total, out + n);
    return cudaGetLastError();
}

}  // namespace spc
