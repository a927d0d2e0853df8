// Device-wide exclusive scan.  With a context: one pass with decoupled look-back
// (spc_scan.cuh).  Without a context (the allocation-free entry point): three launches
// (reduce, scan of tile sums, downsweep) with no inter-block waits.
#include "spc_scan.cuh"

namespace spc {

namespace {

using scanf::ST;
using scanf::SI;
using scanf::STILE;
using scanf::block_excl_scan;

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

template <class In, class T, class Out>
spc_status scan_impl(spc_context* ctx, const In* in, Out* out, int64_t n) {
    return scan_fused<T>(ctx, n, ArrayLd<In, T>{in}, ArraySt<T, Out>{out, n},
                         (double)n * (sizeof(In) + sizeof(Out)));  // input read, output written
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
