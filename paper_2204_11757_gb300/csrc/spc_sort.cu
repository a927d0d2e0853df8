// Stable LSD radix sort of (key, uint32 value) pairs, 8-bit digits.
//
// Per digit: an upsweep builds one 256-bin histogram per 4096-item tile (digit-major), a
// device-wide exclusive scan turns the histograms into output offsets, and a downsweep ranks
// every item inside its tile (warp __match_any_sync ranks, per-warp counters, cross-warp
// prefix), stages the tile in shared memory in digit order and writes it out so that items of
// one digit leave the tile as one contiguous run.  Tiles keep input order and ranks are stable,
// so equal keys keep their input order.  No inter-block waits.
#include <atomic>

#include "spc_internal.cuh"

namespace spc {

namespace {

constexpr int RT = 256;              // threads per block
constexpr int RW = RT / 32;          // warps
constexpr int RI = 16;               // items per lane
constexpr int RTILE = RT * RI;       // 4096 items per tile
constexpr int RADIX = 256;

template <class K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
    return (uint32_t)(key >> shift) & mask;
}

template <class K>
__global__ void __launch_bounds__(RT) k_rs_upsweep(const K* __restrict__ keys, int64_t count,
                                                   int shift, uint32_t mask,
                                                   int32_t* __restrict__ hist, int64_t tiles) {
    spc::pdl_wait();
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RTILE;
    const unsigned lane = threadIdx.x & 31;
#pragma unroll 4
    for (int k = 0; k < RI; ++k) {
        int64_t i = base + (int64_t)k * RT + threadIdx.x;
        bool valid = i < count;
        uint32_t d = valid ? digit_of(keys[i], shift, mask) : (RADIX + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = (int32_t)h[threadIdx.x];
}

template <class K>
struct SortSmem {
    K keys[RTILE];
    uint32_t vals[RTILE];
    uint32_t wcnt[RW][RADIX];
    uint32_t tile_base[RADIX];
    int32_t gofs[RADIX];
};

template <class K>
__global__ void __launch_bounds__(RT) k_rs_downsweep(const K* __restrict__ kin,
                                                     const uint32_t* __restrict__ vin,
                                                     K* __restrict__ kout,
                                                     uint32_t* __restrict__ vout, int64_t count,
                                                     int shift, uint32_t mask,
                                                     const int32_t* __restrict__ offs,
                                                     int64_t tiles) {
    spc::pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<K>& s = *reinterpret_cast<SortSmem<K>*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int d = lane; d < RADIX; d += 32) s.wcnt[warp][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * RTILE + (int64_t)warp * (32 * RI);
    K key[RI];
    uint32_t val[RI];
    uint32_t dig[RI];
    uint32_t rnk[RI];
#pragma unroll
    for (int k = 0; k < RI; ++k) {
        int64_t i = base + k * 32 + lane;
        bool valid = i < count;
        key[k] = valid ? kin[i] : K(0);
        val[k] = valid ? vin[i] : 0u;
        uint32_t d = valid ? digit_of(key[k], shift, mask) : (RADIX + lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? s.wcnt[warp][d] : 0u;
        rnk[k] = before + (uint32_t)__popc(peers & lt_mask);
        dig[k] = d;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) s.wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // cross-warp exclusive prefix per digit, then exclusive scan over digits
    {
        const int d = threadIdx.x;  // RT == RADIX
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            uint32_t t = s.wcnt[w][d];
            s.wcnt[w][d] = run;
            run += t;
        }
        // block-wide exclusive scan of `run` over the 256 digits
        uint32_t v = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        __shared__ uint32_t wsum[RW];
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            uint32_t x = (lane < RW) ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            if (lane < RW) wsum[lane] = x;
        }
        __syncthreads();
        uint32_t excl = v - run + (warp > 0 ? wsum[warp - 1] : 0u);
        s.tile_base[d] = excl;
        s.gofs[d] = offs[(int64_t)d * tiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RI; ++k) {
        if (dig[k] < RADIX) {
            uint32_t pos = s.tile_base[dig[k]] + s.wcnt[warp][dig[k]] + rnk[k];
            s.keys[pos] = key[k];
            s.vals[pos] = val[k];
        }
    }
    __syncthreads();
    const int64_t tb = (int64_t)blockIdx.x * RTILE;
    const int64_t rem = count - tb;
    const int valid_n = rem < RTILE ? (int)rem : RTILE;
    for (int i = threadIdx.x; i < valid_n; i += RT) {
        K k = s.keys[i];
        uint32_t d = digit_of(k, shift, mask);
        int64_t o = (int64_t)s.gofs[d] + (i - (int64_t)s.tile_base[d]);
        kout[o] = k;
        vout[o] = s.vals[i];
    }
}

// ---- one-sweep passes ---------------------------------------------------------------------------
// All digit histograms in one read of the keys; then one kernel per digit in which every tile
// ranks its items, publishes its per-digit counts and finds its output offsets by looking back
// over the tiles before it (decoupled look-back).  Tiles take ids in launch order from a
// counter, so every tile a tile waits for is already running; each wait is bounded.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 8;

template <class K>
__global__ void __launch_bounds__(RT) k_os_hist(const K* __restrict__ keys, int64_t count,
                                                int npass, int end_bit,
                                                uint32_t* __restrict__ hist) {
    spc::pdl_wait();
    constexpr int kCopies = 2;  // two copies (warps 0-3, 4-7) halve the contention on a bin
    __shared__ uint32_t h[kCopies][kMaxPasses][RADIX];
    const int warp = (threadIdx.x >> 5) * kCopies / RW;
    for (int i = threadIdx.x; i < kCopies * kMaxPasses * RADIX; i += RT) (&h[0][0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * RT) {
        const K k = keys[i];
        for (int p = 0; p < npass; ++p) {
            const int shift = 8 * p;
            const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
            atomicAdd(&h[warp][p][(uint32_t)(k >> shift) & ((1u << bits) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RADIX; i += RT) {
        uint32_t s = 0;
        for (int w = 0; w < kCopies; ++w) s += h[w][i / RADIX][i % RADIX];
        if (s) atomicAdd(hist + i, s);
    }
}

// exclusive scan of every pass's 256 bins (one block, one thread per bin)
__global__ void k_os_bases(int npass, const uint32_t* __restrict__ hist, uint32_t* __restrict__ base) {
    spc::pdl_wait();
    __shared__ uint32_t sh[RADIX];
    for (int p = 0; p < npass; ++p) {
        sh[threadIdx.x] = hist[p * RADIX + threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = 0;
            for (int d = 0; d < RADIX; ++d) {
                const uint32_t c = sh[d];
                sh[d] = run;
                run += c;
            }
        }
        __syncthreads();
        base[p * RADIX + threadIdx.x] = sh[threadIdx.x];
        __syncthreads();
    }
}

// One-sweep scatter pass: OT threads (OW warps) per tile of RTILE items, OI items per lane.
constexpr int OT = 512;
constexpr int OW = OT / 32;
constexpr int OI = RTILE / OT;

template <class K>
struct OsSmem {
    K keys[RTILE];
    uint32_t vals[RTILE];
    uint32_t wcnt[OW][RADIX];
    uint32_t tile_base[RADIX];
    int32_t gofs[RADIX];
};

template <class K>
__global__ void __launch_bounds__(OT, 2) k_os_pass(const K* __restrict__ kin,
                                                const uint32_t* __restrict__ vin,
                                                K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                int64_t count, int shift, uint32_t mask,
                                                const uint32_t* __restrict__ base,
                                                uint32_t* status, uint32_t* tile_counter,
                                                uint32_t* err) {
    spc::pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OsSmem<K>& s = *reinterpret_cast<OsSmem<K>*>(smem_raw);
    __shared__ uint32_t sh_tile;
    __shared__ uint32_t wsum[RADIX / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (threadIdx.x == 0) sh_tile = atomicAdd(tile_counter, 1u);
    for (int d = lane; d < RADIX; d += 32) s.wcnt[warp][d] = 0;
    __syncthreads();
    const int64_t tile = sh_tile;
    const int64_t wbase = tile * RTILE + (int64_t)warp * (32 * OI);
    K key[OI];
    uint32_t val[OI];
    uint32_t dr[OI];  // digit (low 16 bits; RADIX + lane when invalid) | rank in warp << 16
    // every load of the tile is issued before the first is used (all in flight at once)
#pragma unroll
    for (int k = 0; k < OI; ++k) {
        const int64_t i = wbase + k * 32 + lane;
        const bool valid = i < count;
        key[k] = valid ? __ldcs(kin + i) : K(0);
        val[k] = valid ? __ldcs(vin + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < OI; ++k) {
        const int64_t i = wbase + k * 32 + lane;
        const bool valid = i < count;
        const uint32_t d = valid ? digit_of(key[k], shift, mask) : (RADIX + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? s.wcnt[warp][d] : 0u;
        dr[k] = d | ((before + (uint32_t)__popc(peers & lt_mask)) << 16);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) s.wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // from here the first RADIX threads own one digit each
    const bool digit_thread = threadIdx.x < RADIX;
    const int d = digit_thread ? threadIdx.x : 0;
    uint32_t tcount = 0, prefix = 0;
    if (digit_thread) {
#pragma unroll
        for (int w = 0; w < OW; ++w) {
            const uint32_t t = s.wcnt[w][d];
            s.wcnt[w][d] = tcount;
            tcount += t;
        }
        // publish this tile's count, then look back for the items of digit d in earlier tiles
        uint32_t* my = status + tile * RADIX + d;
        atomicExch(my, kFlagAgg | tcount);
        for (int64_t t = tile - 1; t >= 0;) {
            const uint32_t v = *reinterpret_cast<volatile uint32_t*>(status + t * RADIX + d);
            if (v & kFlagInc) { prefix += v & kValMask; break; }
            if (v & kFlagAgg) { prefix += v & kValMask; --t; continue; }
            uint32_t spins = 0;  // predecessor not published yet: wait, bounded
            while ((*reinterpret_cast<volatile uint32_t*>(status + t * RADIX + d) &
                    (kFlagAgg | kFlagInc)) == 0u) {
                if (++spins > spin_limit(err)) { atomicOr(err, DEV_TIMEOUT); t = -1; break; }
            }
        }
        atomicExch(my, kFlagInc | (prefix + tcount));
    }
    // exclusive scan over digits of the tile counts: positions in the staged tile
    uint32_t v = tcount;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (digit_thread && lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = (lane < RADIX / 32) ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane < RADIX / 32) wsum[lane] = x;
    }
    __syncthreads();
    if (digit_thread) {
        s.tile_base[d] = v - tcount + (warp > 0 ? wsum[warp - 1] : 0u);
        s.gofs[d] = (int32_t)(base[d] + prefix);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < OI; ++k) {
        const uint32_t dk = dr[k] & 0xffffu;
        if (dk < RADIX) {
            const uint32_t pos = s.tile_base[dk] + s.wcnt[warp][dk] + (dr[k] >> 16);
            s.keys[pos] = key[k];
            s.vals[pos] = val[k];
        }
    }
    __syncthreads();
    const int64_t rem = count - tile * RTILE;
    const int valid_n = rem < RTILE ? (int)rem : RTILE;
    for (int i = threadIdx.x; i < valid_n; i += OT) {
        const K k = s.keys[i];
        const uint32_t dd = digit_of(k, shift, mask);
        const int64_t o = (int64_t)s.gofs[dd] + (i - (int64_t)s.tile_base[dd]);
        if (o >= 0 && o < count) {
            kout[o] = k;
            vout[o] = s.vals[i];
        } else {
            atomicOr(err, DEV_TIMEOUT);
        }
    }
}

template <class K>
spc_status radix_sort_impl(spc_context* ctx, K* keys, uint32_t* vals, K* keys_alt,
                           uint32_t* vals_alt, int64_t count, int end_bit) {
    if (count <= 1 || end_bit <= 0) return SPC_OK;
    const int64_t tiles = (count + RTILE - 1) / RTILE;
    const int npass = (end_bit + 7) / 8;
    if (npass > kMaxPasses || count >= (int64_t)kValMask) return SPC_ERR_TOO_LARGE;
    // hist [npass][256] | base [npass][256] | tile counters [npass] | status [npass][tiles][256]
    const size_t words = (size_t)npass * RADIX * 2 + 32 + (size_t)npass * tiles * RADIX;
    Buf& hbuf = on_side(ctx) ? ctx->work.sort_hist_side : ctx->work.sort_hist;
    SPC_TRY(ensure(ctx, hbuf, words * 4));
    uint32_t* hist = hbuf.as<uint32_t>();
    uint32_t* base = hist + (size_t)npass * RADIX;
    uint32_t* tctr = base + (size_t)npass * RADIX;
    uint32_t* stat = tctr + 32;
    SPC_CUDA(cudaMemsetAsync(hist, 0, words * 4, ctx->stream));
    const size_t smem = sizeof(OsSmem<K>);
    static std::atomic<unsigned long long> attr_devs{0};  // devices already set up
    const unsigned long long bit = 1ull << (ctx->device & 63);
    if (!(attr_devs.load() & bit)) {
        SPC_CUDA(cudaFuncSetAttribute(k_os_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        attr_devs.fetch_or(bit);
    }
    note_bytes(ctx, (double)count * sizeof(K));  // every key read once
    SPC_LAUNCH(ctx, k_os_hist<K>, grid_for(count, RT, ctx->num_sms * 4), RT, 0, keys, count,
               npass, end_bit, hist);
    SPC_LAUNCH(ctx, k_os_bases, 1, RADIX, 0, npass, hist, base);
    K* ka = keys;
    uint32_t* va = vals;
    K* kb = keys_alt;
    uint32_t* vb = vals_alt;
    for (int p = 0; p < npass; ++p) {
        const int shift = 8 * p;
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        const uint32_t mask = (1u << bits) - 1u;
        note_bytes(ctx, 2.0 * (double)count * (sizeof(K) + 4));  // pairs read once, written once
        SPC_LAUNCH(ctx, k_os_pass<K>, (unsigned)tiles, OT, smem, ka, va, kb, vb, count, shift,
                   mask, base + (size_t)p * RADIX, stat + (size_t)p * tiles * RADIX, tctr + p,
                   ctx->d_status);
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    if (npass & 1) {
        SPC_CUDA(cudaMemcpyAsync(keys, ka, (size_t)count * sizeof(K), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
        SPC_CUDA(cudaMemcpyAsync(vals, va, (size_t)count * sizeof(uint32_t),
                                 cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return SPC_OK;
}

}  // namespace

spc_status radix_sort_u64(spc_context* ctx, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                          uint32_t* vals_alt, int64_t count, int end_bit) {
    return radix_sort_impl<uint64_t>(ctx, keys, vals, keys_alt, vals_alt, count, end_bit);
}

spc_status radix_sort_u32(spc_context* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                          uint32_t* vals_alt, int64_t count, int end_bit) {
    return radix_sort_impl<uint32_t>(ctx, keys, vals, keys_alt, vals_alt, count, end_bit);
}

}  // namespace spc

namespace spc {

// Context-free stable LSD radix sort of (uint64 key, uint32 value) pairs on key bits
// [0, end_bit), launched on `stream` with caller-owned scratch: keys_alt/vals_alt of `count`
// items, hist of radix_raw_hist_elems(count) int32 and scan_tmp of
// scan_raw_tmp_elems(256 * tiles) int32.  The result ends in (keys, vals).
int64_t radix_raw_hist_elems(int64_t count) {
    return (int64_t)RADIX * ((count + RTILE - 1) / RTILE) + 1;
}

cudaError_t radix_sort_u64_raw(cudaStream_t stream, uint64_t* keys, uint32_t* vals,
                               uint64_t* keys_alt, uint32_t* vals_alt, int64_t count,
                               int end_bit, int32_t* hist, int32_t* scan_tmp) {
    if (count <= 1 || end_bit <= 0) return cudaSuccess;
    const int64_t tiles = (count + RTILE - 1) / RTILE;
    const size_t smem = sizeof(SortSmem<uint64_t>);
    cudaError_t e = cudaFuncSetAttribute(k_rs_downsweep<uint64_t>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    uint64_t* ka = keys;
    uint32_t* va = vals;
    uint64_t* kb = keys_alt;
    uint32_t* vb = vals_alt;
    int passes = 0;
    for (int shift = 0; shift < end_bit; shift += 8) {
        const int bits = (end_bit - shift) < 8 ? (end_bit - shift) : 8;
        const uint32_t mask = (1u << bits) - 1u;
        k_rs_upsweep<uint64_t><<<(unsigned)tiles, RT, 0, stream>>>(ka, count, shift, mask, hist,
                                                                  tiles);
        e = scan_i32_raw(stream, hist, hist, (int64_t)RADIX * tiles, scan_tmp);
        if (e != cudaSuccess) return e;
        k_rs_downsweep<uint64_t><<<(unsigned)tiles, RT, smem, stream>>>(ka, va, kb, vb, count,
                                                                       shift, mask, hist, tiles);
        uint64_t* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
        ++passes;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (passes & 1) {
        e = cudaMemcpyAsync(keys, ka, (size_t)count * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                            stream);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(vals, va, (size_t)count * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            stream);
    }
    return e;
}

}  // namespace spc
