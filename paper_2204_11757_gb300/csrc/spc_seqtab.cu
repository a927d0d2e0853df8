// Per-binade prefix tables over long sequences, built by the whole GPU, and the exact
// evaluation of long left-to-right sums from them (see spc_seqsum.cuh).
//
// Build, for a batch of sequences: (1) the binade range each running sum can visit; (2) one CTA
// per (sequence, binade, 4096-term chunk) reduces the chunk's grid-rounded terms; (3) one
// thread per (sequence, binade) scans its chunk sums; (4) one CTA per (sequence, binade, chunk)
// scans the chunk again and writes the tables.
//
// Hub rows (the score walks) need every position of every binade, since the walks start from
// many running values.  A full sum from zero does not: its running sum s_k after k terms is
// within gamma_k A_k of the exact prefix sum A_k (recursive summation of non-negative terms,
// N. J. Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., Section 4.2,
// gamma_k = k u / (1 - k u)), so binade E can hold s_k only where that interval meets
// [2^E, 2^(E+1)).  Integer bounds of A_k (terms truncated to a per-sequence grid, prefix-summed
// exactly) give each binade a window of positions; the windows together hold about one entry
// per term instead of one per term and binade.  The walk adds natively at any position outside
// a window, so the windows only decide speed, never the result.
#include "spc_seqsum.cuh"

namespace spc {

namespace {

constexpr int kChunk = 4096;
constexpr int kCT = 256;  // threads of the chunk kernels (kChunk / kCT = 16 terms each)

// min and max term bits of every sequence, flat over all terms (loff = exclusive prefix of the
// lengths).  Each block takes one contiguous range of terms and each thread a strided part of
// it, keeping a running min/max while its terms stay in one sequence; the threads' results are
// combined per warp and per block, so a sequence of millions of terms costs one pair of
// atomics per block instead of one per warp (the atomics of one address serialise).
template <class F>
__global__ void __launch_bounds__(kCT)
k_seq_minmax(int64_t nseq, const F* __restrict__ terms, const int64_t* __restrict__ base,
             const int64_t* __restrict__ loff, unsigned long long* __restrict__ mn,
             unsigned long long* __restrict__ mx) {
    spc::pdl_wait();
    __shared__ int64_t sh_q[kCT / 32];
    __shared__ unsigned long long sh_mn[kCT / 32], sh_mx[kCT / 32];
    const int64_t total = loff[nseq];
    const int64_t per = ((total + gridDim.x - 1) / gridDim.x + kCT - 1) / kCT * kCT;
    const int64_t r0 = (int64_t)blockIdx.x * per;
    const int64_t r1 = r0 + per < total ? r0 + per : total;
    int64_t q = -1;
    unsigned long long a = ~0ull, b = 0ull;
    for (int64_t f = r0 + threadIdx.x; f < r1; f += kCT) {
        if (q < 0 || f >= loff[q + 1]) {  // entering another sequence
            if (q >= 0) { atomicMin(mn + q, a); atomicMax(mx + q, b); }
            int64_t lo = q < 0 ? 0 : q + 1, hi = nseq - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (loff[mid] <= f) lo = mid; else hi = mid - 1;
            }
            q = lo;
            a = ~0ull;
            b = 0ull;
        }
        const unsigned long long v = FB<F>::bits(terms[base[q] + (f - loff[q])]);
        a = v < a ? v : a;
        b = v > b ? v : b;
    }
    // combine the warp when its lanes end in one sequence, then the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q0 = __shfl_sync(0xffffffffu, q, 0);
    const bool same = __all_sync(0xffffffffu, q == q0 || q < 0);
    if (same) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, a, o);
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
            a = x < a ? x : a;
            b = y > b ? y : b;
        }
    } else if (q >= 0) {
        atomicMin(mn + q, a);
        atomicMax(mx + q, b);
    }
    if (lane == 0) {
        sh_q[warp] = same ? q0 : -1;
        sh_mn[warp] = a;
        sh_mx[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t cq = -1;
        unsigned long long ca = ~0ull, cb = 0ull;
        for (int w = 0; w < kCT / 32; ++w) {
            const int64_t wq = sh_q[w];
            if (wq < 0) continue;
            if (wq != cq) {
                if (cq >= 0) { atomicMin(mn + cq, ca); atomicMax(mx + cq, cb); }
                cq = wq;
                ca = ~0ull;
                cb = 0ull;
            }
            ca = sh_mn[w] < ca ? sh_mn[w] : ca;
            cb = sh_mx[w] > cb ? sh_mx[w] : cb;
        }
        if (cq >= 0) { atomicMin(mn + cq, ca); atomicMax(mx + cq, cb); }
    }
}

// binade range and table sizes of every sequence (running sums below 8)
template <class F>
__global__ void k_seq_meta(int64_t nseq, const int64_t* __restrict__ len,
                           const unsigned long long* __restrict__ mn,
                           int32_t* __restrict__ eblo, int32_t* __restrict__ nE,
                           int64_t* __restrict__ tsize, int64_t* __restrict__ tcnt) {
    spc::pdl_wait();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = len[q];
        int lo = (int)(mn[q] >> FB<F>::kMant);
        const int hi = FB<F>::kEbHi;
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

template <class F>
spc_status build_typed(spc_context* ctx, const F* terms, int64_t nseq, const int64_t* base,
                       const int64_t* len, SeqTabBufs& tb) {
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
               tb.mn.as<unsigned long long>(), tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(),
               tb.tsize.as<int64_t>(), tb.tcnt.as<int64_t>());
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

// ---- full sums through windowed tables -----------------------------------------------------

// binade range, grid exponent and pair count of every sequence.  The sum (and every term) is
// at most L * max term < 2^ex; the grid G = 2^gexp makes that at most 2^(61 - lg_nseq) units, so
// the exact prefix of all sequences' units stays below 2^61.  All terms zero: no binades.
template <class F>
__global__ void k_fs_meta(int64_t nseq, const int64_t* __restrict__ len,
                          const unsigned long long* __restrict__ mn,
                          const unsigned long long* __restrict__ mx, int lg_nseq,
                          int32_t* __restrict__ eblo, int32_t* __restrict__ nE,
                          int64_t* __restrict__ npe, int32_t* __restrict__ gexp) {
    spc::pdl_wait();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nseq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = len[q];
        const double mxv = (double)FB<F>::from_bits(mx[q]);
        if (!(mxv > 0.0)) {
            eblo[q] = 1;
            nE[q] = 0;
            npe[q] = 0;
            gexp[q] = 0;
            continue;
        }
        const double bound = (double)L * mxv * (1.0 + 0x1p-40);
        constexpr int kBias = FB<F>::kBiasM - FB<F>::kMant;
        constexpr int kTop = (1 << (sizeof(F) == 8 ? 11 : 8)) - 2;  // largest finite binade
        int ex = kTop - kBias + 2;  // bound beyond the finite range: 2^ex above every term
        if (isfinite(bound)) frexp(bound, &ex);  // bound < 2^ex
        int hi = ex + kBias;  // s_k <= A_L (1 + gamma) < 2^(ex + 1)
        if (hi > kTop) hi = kTop;
        int lo = (int)(mn[q] >> FB<F>::kMant);
        if (lo < 1) lo = 1;
        if (lo < hi - 63) lo = hi - 63;
        if (lo > hi) lo = hi;
        eblo[q] = lo;
        nE[q] = hi - lo + 1;
        npe[q] = hi - lo + 1;
        gexp[q] = ex - (61 - lg_nseq);
    }
}

// units of every term: floor(x / 2^gexp), exact integer arithmetic on the bits
template <class F>
__global__ void __launch_bounds__(kThreads)
k_fs_units(int64_t nseq, int64_t total, const F* __restrict__ terms,
           const int64_t* __restrict__ base, const int64_t* __restrict__ loff,
           const int32_t* __restrict__ gexp, long long* __restrict__ units) {
    spc::pdl_wait();
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nseq - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (loff[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const unsigned long long b = FB<F>::bits(terms[base[lo] + (f - loff[lo])]);
        int et = (int)(b >> FB<F>::kMant);
        unsigned long long mant = b & ((1ull << FB<F>::kMant) - 1ull);
        if (et == 0) et = 1; else mant |= 1ull << FB<F>::kMant;
        const int sh = et - FB<F>::kBiasM - gexp[lo];  // x = mant 2^(et - kBiasM)
        unsigned long long u;
        if (sh >= 0) u = mant << sh;  // < 2^61 by the choice of gexp
        else u = sh > -64 ? mant >> -sh : 0ull;
        units[f] = (long long)u;
    }
}

// the window of pair (q, e): the steps k at which the running sum can lie in binade
// eblo[q] + e, from monotone integer bounds C_k <= A_k / G < C_k + k + 1
template <class F>
__global__ void __launch_bounds__(kThreads)
k_fs_windows(int64_t nseq, const int64_t* __restrict__ len, const int64_t* __restrict__ loff,
             const long long* __restrict__ cu, const int32_t* __restrict__ eblo,
             const int32_t* __restrict__ nE, const int64_t* __restrict__ poff,
             const int32_t* __restrict__ gexp, int64_t* __restrict__ pw0,
             int64_t* __restrict__ plen, int64_t* __restrict__ pnch, int32_t* __restrict__ pq,
             int32_t* __restrict__ pe) {
    spc::pdl_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nseq * 64;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t >> 6;
        const int e = (int)(t & 63);
        if (e >= nE[q]) continue;
        const int64_t r = poff[q] + e;
        const int64_t L = len[q];
        const long long* C = cu + loff[q];
        const long long c0 = C[0];
        int64_t kmin = 0, kmax = L;  // steps k in [kmin, kmax]; empty when kmin > kmax
        // Every prefix of a left-to-right sum of non-negative terms with round-to-nearest
        // satisfies (1 - u)^k A_k <= s_k <= (1 + u)^k A_k (each step multiplies by 1 + delta,
        // |delta| <= u; by induction on k).  With the uniform factors of k = L the windows stay
        // finite for any length (a binary32 sum of tens of millions of terms still gets narrow
        // windows in its low binades).
        const double lu = (double)L * log1p(sizeof(F) == 8 ? 0x1p-53 : 0x1p-24);
        const double f_hi = exp(lu) * (1.0 + 0x1p-40);           // >= (1 + u)^L
        const double f_lo = exp(-lu * (1.0 + 0x1p-20)) * (1.0 - 0x1p-40);  // <= (1 - u)^L
        {
            constexpr int kBias = FB<F>::kBiasM - FB<F>::kMant;
            const int E2 = eblo[q] + e - kBias - gexp[q];  // binade [2^E2, 2^(E2+1)) in units
            constexpr double kCap = 0x1p62;
            double lo_t = ldexp(1.0, E2) / f_hi * (1.0 - 0x1p-40);
            double hi_t = ldexp(1.0, E2 + 1) / f_lo * (1.0 + 0x1p-40);
            lo_t = lo_t > kCap ? kCap : floor(lo_t);
            hi_t = hi_t > kCap ? kCap : ceil(hi_t);
            const long long thr_lo = (long long)lo_t, thr_hi = (long long)hi_t;
            // kmin: first k in [0, L] with C_k + k >= thr_lo (none: L + 1)
            int64_t a = 0, b = L + 1;
            while (a < b) {
                const int64_t mid = (a + b) >> 1;
                if ((C[mid] - c0) + mid >= thr_lo) b = mid; else a = mid + 1;
            }
            kmin = a;
            // kmax: last k in [0, L] with C_k < thr_hi (none: -1)
            a = -1;
            b = L;
            while (a < b) {
                const int64_t mid = (a + b + 1) >> 1;
                if (C[mid] - c0 < thr_hi) a = mid; else b = mid - 1;
            }
            kmax = a;
        }
        if (kmax > L - 1) kmax = L - 1;
        const int64_t nst = kmax >= kmin ? kmax - kmin + 1 : 0;
        pw0[r] = kmin;
        plen[r] = nst ? nst + 1 : 0;  // table entries: prefix positions kmin .. kmax + 1
        pnch[r] = (nst + kChunk - 1) / kChunk;
        pq[r] = (int32_t)q;
        pe[r] = e;
    }
}

// pair r of trip t (pcoff: exclusive prefix of the pairs' chunk counts)
__device__ __forceinline__ int64_t pair_of(int64_t t, int64_t npair, const int64_t* pcoff) {
    int64_t lo = 0, hi = npair - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (pcoff[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// grid-rounded sums (and half-grid ties) of the 4096-step chunks of every window
template <class F>
__global__ void __launch_bounds__(kCT)
k_fs_chunk_sums(int64_t ntrip, int64_t npair, const int64_t* __restrict__ pcoff,
                const int32_t* __restrict__ pq, const int32_t* __restrict__ pe,
                const int64_t* __restrict__ pw0, const int64_t* __restrict__ plen,
                const F* __restrict__ terms, const int64_t* __restrict__ base,
                const int32_t* __restrict__ eblo, unsigned long long* __restrict__ csum,
                int32_t* __restrict__ ctie) {
    spc::pdl_wait();
    __shared__ unsigned long long sh_s[kCT / 32];
    __shared__ int32_t sh_t[kCT / 32];
    for (int64_t t = blockIdx.x; t < ntrip; t += gridDim.x) {
        const int64_t r = pair_of(t, npair, pcoff);
        const int64_t q = pq[r];
        const int eb = eblo[q] + pe[r];
        const F* x = terms + base[q];
        const int64_t k0 = pw0[r] + (t - pcoff[r]) * kChunk;
        const int64_t kend = pw0[r] + plen[r] - 1;
        const int64_t k1 = k0 + kChunk < kend ? k0 + kChunk : kend;
        unsigned long long s = 0;
        int32_t ties = 0;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            bool tie;
            s = sat_add(s, grid_units<F>(x[k], eb, &tie));
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

// exclusive scan of every window's chunk sums, in place (one thread per pair)
// one block per pair: each thread takes a contiguous run of the pair's chunks, sums it, a
// block scan (saturating for the unit sums) gives every run its start, and each thread writes
// its chunks' exclusive prefixes.  (One thread per pair walked a 50M-term sum's 12,000 chunks
// per binade one dependent step at a time.)
constexpr int kChunkScanThreads = 256;

__global__ void __launch_bounds__(kChunkScanThreads)
k_fs_chunk_scan(int64_t npair, const int64_t* __restrict__ pcoff,
                unsigned long long* __restrict__ csum, int32_t* __restrict__ ctie) {
    spc::pdl_wait();
    __shared__ unsigned long long sh_v[kChunkScanThreads / 32];
    __shared__ int32_t sh_t[kChunkScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r = blockIdx.x; r < npair; r += gridDim.x) {
        const int64_t c0 = pcoff[r], len = pcoff[r + 1] - c0;
        const int64_t K = (len + kChunkScanThreads - 1) / kChunkScanThreads;
        const int64_t a = c0 + (int64_t)threadIdx.x * K;
        const int64_t b = a + K < c0 + len ? a + K : c0 + len;
        unsigned long long v = 0;
        int32_t tv = 0;
        for (int64_t c = a; c < b; ++c) {
            v = sat_add(v, csum[c]);
            tv += ctie[c];
        }
        // inclusive warp scan, then the warp totals
        unsigned long long iv = v;
        int32_t it = tv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, iv, o);
            const int32_t t = __shfl_up_sync(0xffffffffu, it, o);
            if (lane >= o) { iv = sat_add(iv, u); it += t; }
        }
        if (lane == 31) { sh_v[warp] = iv; sh_t[warp] = it; }
        __syncthreads();
        unsigned long long wv = 0;
        int32_t wt = 0;
        for (int w = 0; w < warp; ++w) { wv = sat_add(wv, sh_v[w]); wt += sh_t[w]; }
        unsigned long long ev = __shfl_up_sync(0xffffffffu, iv, 1);
        int32_t et = __shfl_up_sync(0xffffffffu, it, 1);
        if (lane == 0) { ev = 0ull; et = 0; }
        unsigned long long run = sat_add(wv, ev);
        int32_t tr = wt + et;
        for (int64_t c = a; c < b; ++c) {
            const unsigned long long x = csum[c];
            const int32_t tx = ctie[c];
            csum[c] = run;
            ctie[c] = tr;
            run = sat_add(run, x);
            tr += tx;
        }
        __syncthreads();  // sh_v / sh_t are rewritten for the next pair
    }
}

// table entries of every window: entry i of pair r (at ptoff[r] + i) is the prefix over the
// window's steps pw0 .. pw0 + i - 1
template <class F>
__global__ void __launch_bounds__(kCT)
k_fs_chunk_write(int64_t ntrip, int64_t npair, const int64_t* __restrict__ pcoff,
                 const int32_t* __restrict__ pq, const int32_t* __restrict__ pe,
                 const int64_t* __restrict__ pw0, const int64_t* __restrict__ plen,
                 const int64_t* __restrict__ ptoff, const F* __restrict__ terms,
                 const int64_t* __restrict__ base, const int32_t* __restrict__ eblo,
                 const unsigned long long* __restrict__ csum, const int32_t* __restrict__ ctie,
                 unsigned long long* __restrict__ P, int32_t* __restrict__ T) {
    spc::pdl_wait();
    constexpr int kItems = kChunk / kCT;
    __shared__ unsigned long long sh_s[kCT / 32];
    __shared__ int32_t sh_t[kCT / 32];
    for (int64_t t = blockIdx.x; t < ntrip; t += gridDim.x) {
        const int64_t r = pair_of(t, npair, pcoff);
        const int64_t q = pq[r];
        const int eb = eblo[q] + pe[r];
        const F* x = terms + base[q];
        const int64_t w0 = pw0[r];
        const int64_t kend = w0 + plen[r] - 1;
        unsigned long long* Pr = P + ptoff[r];
        int32_t* Tr = T + ptoff[r];
        const int64_t c = t - pcoff[r];
        const int64_t k0 = w0 + c * kChunk + (int64_t)threadIdx.x * kItems;
        unsigned long long rr[kItems];
        int32_t ti[kItems];
        unsigned long long run = 0;
        int32_t trun = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = k0 + j;
            bool tie = false;
            rr[j] = (k < kend) ? grid_units<F>(x[k], eb, &tie) : 0ull;
            ti[j] = tie ? 1 : 0;
            run = sat_add(run, rr[j]);
            trun += ti[j];
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned long long v = run;
        int32_t tv = trun;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long a = __shfl_up_sync(0xffffffffu, v, o);
            const int32_t cc = __shfl_up_sync(0xffffffffu, tv, o);
            if (lane >= o) { v = sat_add(v, a); tv += cc; }
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
        if (c == 0 && threadIdx.x == 0) { Pr[0] = 0; Tr[0] = 0; }
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t k = k0 + j;
            pre = sat_add(pre, rr[j]);
            tpre += ti[j];
            if (k < kend) { Pr[k - w0 + 1] = pre; Tr[k - w0 + 1] = tpre; }
        }
        __syncthreads();
    }
}

// one full sum per sequence, by a warp: binade by binade through the windows (32 probes per
// search round), one native addition at every binade crossing, tie, or position outside the
// current binade's window
template <class F>
__global__ void k_fs_walk(int64_t nseq, const F* __restrict__ terms,
                          const int64_t* __restrict__ base, const int64_t* __restrict__ len,
                          const int32_t* __restrict__ eblo, const int32_t* __restrict__ nE,
                          const int64_t* __restrict__ poff, const int64_t* __restrict__ pw0,
                          const int64_t* __restrict__ plen, const int64_t* __restrict__ ptoff,
                          const unsigned long long* __restrict__ P,
                          const int32_t* __restrict__ T, const int64_t* __restrict__ out_idx,
                          F* __restrict__ out) {
    spc::pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nseq;
         q += warps) {
        const int64_t L = len[q];
        const F* x = terms + base[q];
        const int lo_eb = eblo[q], ne = nE[q];
        // every binade's window (start, entries, table offset): lane l holds binades l and
        // l + 32 (at most 64), fetched by shuffles instead of dependent loads in the walk
        int64_t mw0[2] = {0, 0}, mlen[2] = {0, 0}, mtoff[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * h;
            if (e < ne) {
                const int64_t r = poff[q] + e;
                mw0[h] = pw0[r];
                mlen[h] = plen[r];
                mtoff[h] = ptoff[r];
            }
        }
        F s = F(0);
        int64_t a = 0;
        while (ne > 0 && a < L) {
            if (s == F(0)) { s = x[a++]; continue; }
            const unsigned long long sb = FB<F>::bits(s);
            const int eb = (int)(sb >> FB<F>::kMant);
            const int e = eb - lo_eb;  // the same in every lane
            if (eb == 0 || e < 0 || e >= ne) { s = FB<F>::add(s, x[a++]); continue; }
            const int eh = e >> 5, el = e & 31;
            const int64_t w0 = __shfl_sync(0xffffffffu, eh ? mw0[1] : mw0[0], el);
            const int64_t nent = __shfl_sync(0xffffffffu, eh ? mlen[1] : mlen[0], el);
            const int64_t toff = __shfl_sync(0xffffffffu, eh ? mtoff[1] : mtoff[0], el);
            // the next binade's window start (hint below)
            const int e1 = e + 1 < ne ? e + 1 : e;
            const int64_t nw0 = __shfl_sync(0xffffffffu, (e1 >> 5) ? mw0[1] : mw0[0], e1 & 31);
            const int64_t nlen = __shfl_sync(0xffffffffu, (e1 >> 5) ? mlen[1] : mlen[0], e1 & 31);
            if (nent == 0 || a < w0 || a > w0 + nent - 2) { s = FB<F>::add(s, x[a++]); continue; }
            const unsigned long long* Pr = P + toff;
            const int32_t* Tr = T + toff;
            const unsigned long long pa = Pr[a - w0];
            if (pa >= kSat - (1ull << 55)) { s = FB<F>::add(s, x[a++]); continue; }
            const unsigned long long S =
                (sb & ((1ull << FB<F>::kMant) - 1ull)) | (1ull << FB<F>::kMant);
            const unsigned long long lim = (1ull << (FB<F>::kMant + 1)) - S;
            const int32_t ta = Tr[a - w0];
            // largest k in [a, w0 + nent - 1] with P_k - P_a <= lim and no tie in [a, k)
            int64_t lo = a, hi = w0 + nent - 1;
            // The sum cannot reach the next binade before that binade's window starts, so the
            // answer is usually at or after the step before it (the last binade: the end).
            // One probe there, if it is good, leaves only the windows' overlap to search.
            int64_t hint = hi;
            if (e + 1 < ne && nlen > 0) hint = nw0 - 1;
            if (hint > lo && hint <= hi && Pr[hint - w0] - pa <= lim && Tr[hint - w0] == ta)
                lo = hint;
            while (hi > lo) {
                const int64_t step = (hi - lo + 31) / 32;
                const int64_t probe = lo + (int64_t)(lane + 1) * step;
                bool good = false;
                if (probe <= hi) good = (Pr[probe - w0] - pa <= lim) && (Tr[probe - w0] == ta);
                const int ngood = __popc(__ballot_sync(0xffffffffu, good));
                // good positions form a prefix of the probes (both conditions are monotone)
                const int64_t new_lo = lo + (int64_t)ngood * step;
                int64_t new_hi = lo + (int64_t)(ngood + 1) * step - 1;
                if (new_hi > hi) new_hi = hi;
                lo = new_lo > hi ? hi : new_lo;
                hi = new_hi;
                if (step == 1) break;
            }
            s = from_units<F>(S + (Pr[lo - w0] - pa), eb);
            a = lo;
            if (a < L) s = FB<F>::add(s, x[a++]);  // crossing, tie or window end: native step
        }
        if (lane == 0) out[out_idx ? out_idx[q] : q] = s;
    }
}

template <class F>
spc_status full_windowed(spc_context* ctx, const F* terms, int64_t nseq, const int64_t* base,
                         const int64_t* len, const int64_t* out_idx, F* out, SeqTabBufs& tb) {
    if (nseq <= 0) return SPC_OK;
    const int maxb = ctx->num_sms * 8;
    int lg = 0;
    while ((1ll << lg) < nseq) ++lg;
    SPC_TRY(ensure(ctx, tb.eblo, (size_t)nseq * 4));
    SPC_TRY(ensure(ctx, tb.nE, (size_t)nseq * 4));
    SPC_TRY(ensure(ctx, tb.gexp, (size_t)nseq * 4));
    SPC_TRY(ensure(ctx, tb.npe, (size_t)nseq * 8));
    SPC_TRY(ensure(ctx, tb.poff, (size_t)(nseq + 1) * 8));
    SPC_TRY(ensure(ctx, tb.loff, (size_t)(nseq + 1) * 8));
    SPC_TRY(ensure(ctx, tb.mn, (size_t)nseq * 8));
    SPC_TRY(ensure(ctx, tb.mx, (size_t)nseq * 8));
    SPC_TRY(scan_i64_i64(ctx, len, tb.loff.as<int64_t>(), nseq));
    SPC_CUDA(cudaMemsetAsync(tb.mn.p, 0xff, (size_t)nseq * 8, ctx->stream));
    SPC_CUDA(cudaMemsetAsync(tb.mx.p, 0, (size_t)nseq * 8, ctx->stream));
    SPC_LAUNCH(ctx, k_seq_minmax<F>, maxb, kCT, 0, nseq, terms, base, tb.loff.as<int64_t>(),
               tb.mn.as<unsigned long long>(), tb.mx.as<unsigned long long>());
    SPC_LAUNCH(ctx, k_fs_meta<F>, grid_for(nseq, kThreads, maxb), kThreads, 0, nseq, len,
               tb.mn.as<unsigned long long>(), tb.mx.as<unsigned long long>(), lg,
               tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(), tb.npe.as<int64_t>(),
               tb.gexp.as<int32_t>());
    SPC_TRY(scan_i64_i64(ctx, tb.npe.as<int64_t>(), tb.poff.as<int64_t>(), nseq));
    int64_t v1[2];
    {
        const void* ptrs[2] = {tb.loff.as<int64_t>() + nseq, tb.poff.as<int64_t>() + nseq};
        const int bytes[2] = {8, 8};
        SPC_TRY(read_vals(ctx, 2, ptrs, bytes, v1));
    }
    const int64_t total = v1[0], npair = v1[1];
    const long long* cu = nullptr;
    if (npair > 0) {
        SPC_TRY(ensure(ctx, tb.units, (size_t)(total + 1) * 8));
        SPC_TRY(ensure(ctx, tb.cunits, (size_t)(total + 1) * 8));
        SPC_TRY(ensure(ctx, tb.pw0, (size_t)npair * 8));
        SPC_TRY(ensure(ctx, tb.plen, (size_t)npair * 8));
        SPC_TRY(ensure(ctx, tb.pnch, (size_t)npair * 8));
        SPC_TRY(ensure(ctx, tb.pq, (size_t)npair * 4));
        SPC_TRY(ensure(ctx, tb.pe, (size_t)npair * 4));
        SPC_TRY(ensure(ctx, tb.ptoff, (size_t)(npair + 1) * 8));
        SPC_TRY(ensure(ctx, tb.pcoff, (size_t)(npair + 1) * 8));
        SPC_LAUNCH(ctx, k_fs_units<F>, grid_for(total, kThreads, maxb), kThreads, 0, nseq, total,
                   terms, base, tb.loff.as<int64_t>(), tb.gexp.as<int32_t>(),
                   tb.units.as<long long>());
        SPC_TRY(scan_i64_i64(ctx, tb.units.as<int64_t>(), tb.cunits.as<int64_t>(), total));
        cu = tb.cunits.as<long long>();
        SPC_LAUNCH(ctx, k_fs_windows<F>, grid_for(nseq * 64, kThreads, maxb), kThreads, 0, nseq,
                   len, tb.loff.as<int64_t>(), cu, tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(),
                   tb.poff.as<int64_t>(), tb.gexp.as<int32_t>(), tb.pw0.as<int64_t>(),
                   tb.plen.as<int64_t>(), tb.pnch.as<int64_t>(), tb.pq.as<int32_t>(),
                   tb.pe.as<int32_t>());
        SPC_TRY(scan_i64_i64(ctx, tb.plen.as<int64_t>(), tb.ptoff.as<int64_t>(), npair));
        SPC_TRY(scan_i64_i64(ctx, tb.pnch.as<int64_t>(), tb.pcoff.as<int64_t>(), npair));
        int64_t v2[2];
        {
            const void* ptrs[2] = {tb.ptoff.as<int64_t>() + npair, tb.pcoff.as<int64_t>() + npair};
            const int bytes[2] = {8, 8};
            SPC_TRY(read_vals(ctx, 2, ptrs, bytes, v2));
        }
        const int64_t elems = v2[0], ntrip = v2[1];
        SPC_TRY(ensure(ctx, tb.P, (size_t)elems * 8 + 256));
        SPC_TRY(ensure(ctx, tb.T, (size_t)elems * 4 + 256));
        SPC_TRY(ensure(ctx, tb.csum, (size_t)ntrip * 8 + 256));
        SPC_TRY(ensure(ctx, tb.ctie, (size_t)ntrip * 4 + 256));
        if (ntrip > 0) {
            // every window position's term read once
            note_bytes(ctx, (double)elems * sizeof(F));
            SPC_LAUNCH(ctx, k_fs_chunk_sums<F>, grid_for(ntrip, 1, maxb), kCT, 0, ntrip, npair,
                       tb.pcoff.as<int64_t>(), tb.pq.as<int32_t>(), tb.pe.as<int32_t>(),
                       tb.pw0.as<int64_t>(), tb.plen.as<int64_t>(), terms, base,
                       tb.eblo.as<int32_t>(), tb.csum.as<unsigned long long>(),
                       tb.ctie.as<int32_t>());
            SPC_LAUNCH(ctx, k_fs_chunk_scan, grid_for(npair, 1, maxb), kChunkScanThreads, 0, npair,
                       tb.pcoff.as<int64_t>(), tb.csum.as<unsigned long long>(),
                       tb.ctie.as<int32_t>());
            // every window position's term read once, its prefix (8 B) and tie count (4 B)
            // written once
            note_bytes(ctx, (double)elems * (sizeof(F) + 12));
            SPC_LAUNCH(ctx, k_fs_chunk_write<F>, grid_for(ntrip, 1, maxb), kCT, 0, ntrip, npair,
                       tb.pcoff.as<int64_t>(), tb.pq.as<int32_t>(), tb.pe.as<int32_t>(),
                       tb.pw0.as<int64_t>(), tb.plen.as<int64_t>(), tb.ptoff.as<int64_t>(), terms,
                       base, tb.eblo.as<int32_t>(), tb.csum.as<unsigned long long>(),
                       tb.ctie.as<int32_t>(), tb.P.as<unsigned long long>(), tb.T.as<int32_t>());
        }
    }
    tb.nseq = nseq;
    SPC_LAUNCH(ctx, k_fs_walk<F>, grid_for(nseq, kThreads / 32, maxb), kThreads, 0, nseq, terms,
               base, len, tb.eblo.as<int32_t>(), tb.nE.as<int32_t>(), tb.poff.as<int64_t>(),
               tb.pw0.as<int64_t>(), tb.plen.as<int64_t>(), tb.ptoff.as<int64_t>(),
               tb.P.as<unsigned long long>(), tb.T.as<int32_t>(), out_idx, out);
    return SPC_OK;
}

}  // namespace

spc_status seqtab_build(spc_context* ctx, const void* terms, bool f32, int64_t nseq,
                        const int64_t* base, const int64_t* len, SeqTabBufs& tb) {
    if (f32) return build_typed<float>(ctx, static_cast<const float*>(terms), nseq, base, len, tb);
    return build_typed<double>(ctx, static_cast<const double*>(terms), nseq, base, len, tb);
}

spc_status seqtab_full(spc_context* ctx, const void* terms, bool f32, int64_t nseq,
                       const int64_t* base, const int64_t* len, const int64_t* out_idx, void* out,
                       SeqTabBufs& tb) {
    if (f32)
        return full_windowed<float>(ctx, static_cast<const float*>(terms), nseq, base, len,
                                    out_idx, static_cast<float*>(out), tb);
    return full_windowed<double>(ctx, static_cast<const double*>(terms), nseq, base, len, out_idx,
                                 static_cast<double*>(out), tb);
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
