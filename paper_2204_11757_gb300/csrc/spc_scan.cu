// Device-wide exclusive scan (reduce -> scan of tile sums -> downsweep).  No inter-block waits:
// the three phases are separate launches, so nothing here can spin.
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
    if (threadIdx.x == 0) *dst = (Out)*total;
}

// small inputs: one CTA scans everything in chunks of 4 items per thread with a carry, and
// writes the total at out[n] (one launch instead of three plus a copy)
constexpr int kSmallThreads = 1024;
constexpr int64_t kSmallMax = 16384;

template <class In, class T, class Out>
__global__ void __launch_bounds__(kSmallThreads) k_scan_small(const In* in, int64_t n, Out* out) {
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

template <class In, class T, class Out>
spc_status scan_impl(spc_context* ctx, const In* in, Out* out, int64_t n) {
    if (n <= kSmallMax) {
        SPC_LAUNCH(ctx, (k_scan_small<In, T, Out>), 1, kSmallThreads, 0, in, n, out);
        return SPC_OK;
    }
    const int64_t nt = (n + STILE - 1) / STILE;
    const size_t need = (size_t)(nt + 1) * sizeof(T) + 256;
    SPC_TRY(ensure(ctx, ctx->work.scan_tmp, need));
    T* tiles = ctx->work.scan_tmp.as<T>();
    T* total = tiles + nt;
    if (nt > 0) {
        SPC_LAUNCH(ctx, (k_scan_reduce<In, T>), (unsigned)nt, ST, 0, in, n, tiles);
    }
    SPC_LAUNCH(ctx, (k_scan_tiles<T>), 1, ST, 0, tiles, nt, total);
    if (nt > 0) {
        SPC_LAUNCH(ctx, (k_scan_down<In, T, Out>), (unsigned)nt, ST, 0, in, n, tiles, out);
    }
    // out[n] = total (device to device copy keeps everything on the stream)
    if (sizeof(T) == sizeof(Out)) {
        SPC_CUDA(cudaMemcpyAsync(out + n, total, sizeof(Out), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    } else {
        SPC_LAUNCH(ctx, (k_copy_total<T, Out>), 1, 32, 0, total, out + n);
    }
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
