// Per-binade prefix tables over long sequences, built by the whole GPU, and the exact
// evaluation of long left-to-right sums from them (see spc_seqsum.cuh).
//
// Build, for a batch of sequences: (1) one CTA per sequence finds the binade range its running
// sum can visit; (2) one CTA per (sequence, binade, 4096-term chunk) reduces the chunk's
// grid-rounded terms; (3) one thread per (sequence, binade) scans its chunk sums; (4) one CTA
// per (sequence, binade, chunk) scans the chunk again and writes the tables.
#include "spc_seqsum.cuh"

namespace spc {

namespace {

constexpr int kChunk = 4096;
constexpr int kCT = 256;  // threads of the chunk kernels (kChunk / kCT = 16 terms each)

// min and max term bits of every sequence: flat over all terms (loff = exclusive prefix of the
// lengths), reduced per warp when the warp's lanes share a sequence
template <class F>
__global__ void __launch_bounds__(kCT)
k_seq_minmax(int64_t nseq, const F* __restrict__ terms, const int64_t* __restrict__ base,
             const int64_t* __restrict__ loff, unsigned long long* __restrict__ mn,
             unsigned long long* __restrict__ mx) {
    spc::pdl_wait();
    const int64_t total = loff[nseq];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t wbase = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31;
    const int lane = threadIdx.x & 31;
    for (int64_t b0 = wbase; b0 < total; b0 += stride) {
        const int64_t f = b0 + lane;
        int64_t q = -1;
        unsigned long long v = 0;
        if (f < total) {
            int64_t lo = 0, hi = nseq - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (loff[mid] <= f) lo = mid; else hi = mid - 1;
            }
            q = lo;
            v = FB<F>::bits(terms[base[q] + (f - loff[q])]);
        }
        const int64_t q0 = __shfl_sync(0xffffffffu, q, 0);
        const bool same = __all_sync(0xffffffffu, q == q0);
        if (same) {
            unsigned long long a = v, b = v;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o);
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
                a = x < a ? x : a;
                b = y > b ? y : b;
            }
            if (lane == 0) { atomicMin(mn + q0, a); atomicMax(mx + q0, b); }
        } else if (q >= 0) {
            atomicMin(mn + q, v);
            atomicMax(mx + q, v);
        }
    }
}

// binade range and table sizes of every sequence
template <class F>
__global__ void k_seq_meta(int64_t nseq, const int64_t* __restrict__ len,
                           const unsigned long long* __restrict__ mn,
                           const unsigned long long* __restrict__ mx, int full,
                           int32_t* __restrict__ eblo, int32_t* __restrict__ nE,
                           int64_t* __restrict__ tsize, int64_t* __restrict__ tcnt) {
    spc::pdl_wait();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = len[q];
        int lo = (int)(mn[q] >> FB<F>::kMant);
        int hi;
        if (full) {
            // the sum is below L * max term: its binade is at most that of the bound
            const double bound = (double)L * (double)FB<F>::from_bits(mx[q]) * 1.0000001;
            const int top = (1 << (sizeof(F) == 8 ? 11 : 8)) - 2;
            if (isfinite(bound)) {
                int ex = 0;
                frexp(bound, &ex);  // bound = f * 2^ex, f in [0.5, 1)
                hi = ex - 1 + (FB<F>::kBiasM - FB<F>::kMant) + 1;
                if (hi > top) hi = top;
            } else {
                hi = top;
            }
        } else {
            hi = FB<F>::kEbHi;
        }
        if (lo < 1) lo = 1;
        if (lo < hi - 63) lo = hi - 63;
        if (lo > hi) lo = hi;
        const int n = hi - lo + 1;
        eblo[q] = lo;
        nE[q] = n;
        tsize[q] = (int64_t)n * (L + 1);
        tcnt[q] = (int64_t)n * ((L + kChunk - 1) / kChunk);
    }
}

struct Trip {
    int64_t q;
    int e;
    int64_t c;
    int64_t nch;
};

__device__ __forceinline__ Trip trip_of(int64_t t, int64_t nseq, const int64_t* trip_off,
                                        const int64_t* len) {
    int64_t lo = 0, hi = nseq - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (trip_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    Trip r;
    r.q = lo;
    r.nch = (len[lo] + kChunk - 1) / kChunk;
    const int64_t rem = t - trip_off[lo];
    r.e = (int)(rem / r.nch);
    r.c = rem - (int64_t)r.e * r.nch;
    return r;
}

template <class F>
__global__ void __launch_bounds__(kCT)
k_seq_chunk_sums(int64_t nseq, int64_t ntrip, const F* __restrict__ terms,
                 const int64_t* __restrict__ base, const int64_t* __restrict__ len,
                 const int32_t* __restrict__ eblo, const int64_t* __restrict__ trip_off,
                 unsigned long long* __restrict__ csum, int32_t* __restrict__ ctie) {
    spc::pdl_wait();
    __shared__ unsigned long long sh_s[kCT / 32];
    __shared__ int32_t sh_t[kCT / 32];
    for (int64_t t = blockIdx.x; t < ntrip; t += gridDim.x) {
        const Trip tr = trip_of(t, nseq, trip_off, len);
        const int eb = eblo[tr.q] + tr.e;
        const int64_t b = base[tr.q], L = len[tr.q];
        const int64_t k0 = tr.c * kChunk;
        const int64_t k1 = (k0 + kChunk < L) ? k0 + kChunk : L;
        unsigned long long s = 0;
        int32_t ties = 0;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            bool tie;
            s = sat_add(s, grid_units<F>(terms[b + k], eb, &tie));
            ties += tie ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s = sat_add(s, __shfl_xor_sync(0xffffffffu, s, o));
            ties += __shfl_xor_sync(0xffffffffu, ties, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { sh_s[warp] = s; sh_t[warp] = ties; }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long a = 0;
            int32_t tt = 0;
            for (int w = 0; w < kCT / 32; ++w) { a = sat_add(a, sh_s[w]); tt += sh_t[w]; }
            csum[t] = a;
            ctie[t] = tt;
        }
        __syncthreads();
    }
}

// exclusive scan of the chunk sums of every (sequence, binade) pair, in place
__global__ void k_seq_chunk_scan(int64_t nseq, const int64_t* __restrict__ len,
                                 const int32_t* __restrict__ nE,
                                 const int64_t* __restrict__ trip_off,
                                 unsigned long long* __restrict__ csum, int32_t* __restrict__ ctie) {
    spc::pdl_wait();
    for (int64_t q = blockIdx.x; q < nseq; q += gridDim.x) {
        const int64_t nch = (len[q] + kChunk - 1) / kChunk;
        for (int e = threadIdx.x; e < nE[q]; e += blockDim.x) {
            const int64_t t0 = trip_off[q] + (int64_t)e * nch;
            unsigned long long run = 0;
            int32_t tr = 0;
            for (int64_t c = 0; c < nch; ++c) {
                const unsigned long long v = csum[t0 + c];
                const int32_t tv = ctie[t0 + c];
                csum[t0 + c] = run;
                ctie[t0 + c] = tr;
                run = sat_add(run, v);
                tr += tv;
            }
        }
    }
}

template <class F>
__global__ void __launch_bounds__(kCT)
k_seq_chunk_write(int64_t nseq, int64_t ntrip, const F* __restrict__ terms,
                  const int64_t* __restrict__ base, const int64_t* __restrict__ len,
                  const int32_t* __restrict__ eblo, const int64_t* __restrict__ trip_off,
                  const int64_t* __restrict__ tab_off, const unsigned long long* __restrict__ csum,
                  const int32_t* __restrict__ ctie, unsigned long long* __restrict__ P,
                  int32_t* __restrict__ T) {
    spc::pdl_wait();
    constexpr int kItems = kChunk / kCT;
    __shared__ unsigned long long sh_s[kCT / 32];
    __shared__ int32_t sh_t[kCT / 32];
    for (int64_t t = blockIdx.x; t < ntrip; t += gridDim.x) {
        const Trip tr = trip_of(t, nseq, trip_off, len);
        const int eb = eblo[tr.q] + tr.e;
        const int64_t b = base[tr.q], L = len[tr.q];
        unsigned long long* Pq = P + tab_off[tr.q] + (int64_t)tr.e * (L + 1);
        int32_t* Tq = T + tab_off[tr.q] + (int64_t)tr.e * (L + 1);
        const int64_t k0 = tr.c * kChunk + (int64_t)threadIdx.x * kItems;
        unsigned long long r[kItems];
        int32_t ti[kItems];
        unsigned long long run = 0;
        int32_t trun = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = k0 + j;
            bool tie = false;
            r[j] = (k < L) ? grid_units<F>(terms[b + k], eb, &tie) : 0ull;
            ti[j] = tie ? 1 : 0;
            run = sat_add(run, r[j]);
            trun += ti[j];
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned long long v = run;
        int32_t tv = trun;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long a = __shfl_up_sync(0xffffffffu, v, o);
            const int32_t c = __shfl_up_sync(0xffffffffu, tv, o);
            if (lane >= o) { v = sat_add(v, a); tv += c; }
        }
        if (lane == 31) { sh_s[warp] = v; sh_t[warp] = tv; }
        __syncthreads();
        unsigned long long pre = csum[t];
        int32_t tpre = ctie[t];
        for (int w = 0; w < warp; ++w) { pre = sat_add(pre, sh_s[w]); tpre += sh_t[w]; }
        unsigned long long wex = __shfl_up_sync(0xffffffffu, v, 1);
        int32_t tex = __shfl_up_sync(0xffffffffu, tv, 1);
        if (lane == 0) { wex = 0; tex = 0; }
        pre = sat_add(pre, wex);
        tpre += tex;
        if (tr.c == 0 && threadIdx.x == 0) { Pq[0] = 0; Tq[0] = 0; }
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = k0 + j;
            pre = sat_add(pre, r[j]);
            tpre += ti[j];
            if (k < L) { Pq[k + 1] = pre; Tq[k + 1] = tpre; }
        }
        __syncthreads();
    }
}

// one full sum per sequence, by a warp: out[out_idx[q]] = left-to-right sum of its terms
template <class F, class Out>
__global__ void k_seq_full_sums(int64_t nseq, const F* __restrict__ terms,
                                const int64_t* __restrict__ base, const int64_t* __restrict__ len,
                                const int32_t* __restrict__ eblo, const int32_t* __restrict__ nE,
                                const int64_t* __restrict__ tab_off,
                                const unsigned long long* __restrict__ P,
                                const int32_t* __restrict__ T, const int64_t* __restrict__ out_idx,
                                Out* __restrict__ out) {
    spc::pdl_wait();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nseq;
         q += warps) {
        const int64_t L = len[q];
        const F s = tab_run_warp<F>(F(0), 0, L, terms + base[q], P + tab_off[q], T + tab_off[q],
                                    eblo[q], nE[q], L + 1);
        if ((threadIdx.x & 31) == 0) out[out_idx ? out_idx[q] : q] = (Out)s;
    }
}

template <class F>
spc_status build_typed(spc_context* ctx, const F* terms, int64_t nseq, const int64_t* base,
                       const int64_t* len, bool full, SeqTabBufs& tb) {
    if (nseq <= 0) return SPC_OK;
    const int maxb = ctx->num_sms * 8;
    SPC_TRY(ensure(ctx, tb.eblo, (size_t)nseq * 4));
    SPC_TRY(ensure(ctx, tb.nE, (size_t)nseq * 4));
    SPC_TRY(ensure(ctx, tb.tsize, (size_t)nseq * 8));
    SPC_TRY(ensure(ctx, tb.tcnt, (size_t)nseq * 8));
    SPC_TRY(ensure(ctx, tb.tab_off, (size_t)(nseq + 1) * 8));
    SPC_TRY(ensure(ctx, tb.trip_off, (size_t)(nseq + 1) * 8));
    SPC_TRY(ensure(ctx, tb.loff, (size_t)(nseq + 1) * 8));
    SPC_TRY(ensure(ctx, tb.mn, (size_t)nseq * 8));
    SPC_TRY(ensure(ctx, tb.mx, (size_t)nseq * 8));
    SPC_TRY(scan_i64_i64(ctx, len, tb.loff.as<int64_t>(), nseq));
    SPC_CUDA(cudaMemsetAsync(tb.mn.p, 0xff, (size_t)nseq * 8, ctx->stream));
    SPC_CUDA(cudaMemsetAsync(tb.mx.p, 0, (size_t)nseq * 8, ctx->stream));
    SPC_LAUNCH(ctx, k_seq_minmax<F>, maxb, kCT, 0, nseq, terms, base, tb.loff.as<int64_t>(),
               tb.mn.as<unsigned long long>(), tb.mx.as<unsigned long long>());
    SPC_LAUNCH(ctx, k_seq_meta<F>, grid_for(nseq, kThreads, maxb), kThreads, 0, nseq, len,
               tb.mn.as<unsigned long long>(), tb.mx.as<unsigned long long>(), full ? 1 : 0,
               tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(), tb.tsize.as<int64_t>(),
               tb.tcnt.as<int64_t>());
    SPC_TRY(scan_i64_i64(ctx, tb.tsize.as<int64_t>(), tb.tab_off.as<int64_t>(), nseq));
    SPC_TRY(scan_i64_i64(ctx, tb.tcnt.as<int64_t>(), tb.trip_off.as<int64_t>(), nseq));
    int64_t vals[2];
    {
        const void* ptrs[2] = {tb.tab_off.as<int64_t>() + nseq, tb.trip_off.as<int64_t>() + nseq};
        const int bytes[2] = {8, 8};
        SPC_TRY(read_vals(ctx, 2, ptrs, bytes, vals));
    }
    const int64_t elems = vals[0];
    const int64_t ntrip = vals[1];
    SPC_TRY(ensure(ctx, tb.P, (size_t)elems * 8 + 256));
    SPC_TRY(ensure(ctx, tb.T, (size_t)elems * 4 + 256));
    SPC_TRY(ensure(ctx, tb.csum, (size_t)ntrip * 8 + 256));
    SPC_TRY(ensure(ctx, tb.ctie, (size_t)ntrip * 4 + 256));
    tb.nseq = nseq;
    SPC_LAUNCH(ctx, k_seq_chunk_sums<F>, grid_for(ntrip, 1, maxb), kCT, 0, nseq, ntrip, terms,
               base, len, tb.eblo.as<int32_t>(), tb.trip_off.as<int64_t>(),
               tb.csum.as<unsigned long long>(), tb.ctie.as<int32_t>());
    SPC_LAUNCH(ctx, k_seq_chunk_scan, grid_for(nseq, 1, maxb), 64, 0, nseq, len,
               tb.nE.as<int32_t>(), tb.trip_off.as<int64_t>(), tb.csum.as<unsigned long long>(),
               tb.ctie.as<int32_t>());
    SPC_LAUNCH(ctx, k_seq_chunk_write<F>, grid_for(ntrip, 1, maxb), kCT, 0, nseq, ntrip, terms,
               base, len, tb.eblo.as<int32_t>(), tb.trip_off.as<int64_t>(),
               tb.tab_off.as<int64_t>(), tb.csum.as<unsigned long long>(), tb.ctie.as<int32_t>(),
               tb.P.as<unsigned long long>(), tb.T.as<int32_t>());
    return SPC_OK;
}

template <class F, class Out>
spc_status full_typed(spc_context* ctx, const F* terms, const int64_t* base, const int64_t* len,
                      const SeqTabBufs& tb, const int64_t* out_idx, Out* out) {
    if (tb.nseq <= 0) return SPC_OK;
    const int warps_per_block = kThreads / 32;
    SPC_LAUNCH(ctx, (k_seq_full_sums<F, Out>), grid_for(tb.nseq, warps_per_block, ctx->num_sms * 8),
               kThreads, 0, tb.nseq, terms, base, len, tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(),
               tb.tab_off.as<int64_t>(), tb.P.as<unsigned long long>(), tb.T.as<int32_t>(), out_idx,
               out);
    return SPC_OK;
}

}  // namespace

spc_status seqtab_build(spc_context* ctx, const void* terms, bool f32, int64_t nseq,
                        const int64_t* base, const int64_t* len, bool full, SeqTabBufs& tb) {
    if (f32) return build_typed<float>(ctx, static_cast<const float*>(terms), nseq, base, len, full, tb);
    return build_typed<double>(ctx, static_cast<const double*>(terms), nseq, base, len, full, tb);
}

spc_status seqtab_full_sums(spc_context* ctx, const void* terms, bool f32, const int64_t* base,
                            const int64_t* len, const SeqTabBufs& tb, const int64_t* out_idx,
                            void* out) {
    if (f32)
        return full_typed<float, float>(ctx, static_cast<const float*>(terms), base, len, tb,
                                        out_idx, static_cast<float*>(out));
    return full_typed<double, double>(ctx, static_cast<const double*>(terms), base, len, tb,
                                      out_idx, static_cast<double*>(out));
}

SeqTabView seqtab_view(const SeqTabBufs& tb, const int64_t* base, const int64_t* len) {
    SeqTabView v;
    v.base = base;
    v.len = len;
    v.eblo = tb.eblo.as<int32_t>();
    v.nE = tb.nE.as<int32_t>();
    v.tab_off = tb.tab_off.as<int64_t>();
    v.P = tb.P.as<unsigned long long>();
    v.T = tb.T.as<int32_t>();
    return v;
}

}  // namespace spc
