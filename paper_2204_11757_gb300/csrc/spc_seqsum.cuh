// Exact, parallel evaluation of IEEE sequential summation of nonnegative terms.
//
// Every sum on the path (degrees, scores, coarse weights, self-mass) is defined as the
// left-to-right IEEE round-to-nearest sum s_{k+1} = RN(s_k + t_k) in a fixed order.  A single
// thread walking a long sequence serialises a whole launch (hub rows, giant super-nodes), so
// long sums are evaluated in parallel without changing a single bit:
//
//   For s in the binade [2^E, 2^(E+1)) the representable numbers are the multiples of the grid
//   g = 2^(E - p + 1) (p = 53 or 24 significand bits), and 2^(E+1) is one of them.  With
//   s = S g, S integer, RN(s + t) = (S + round(t / g)) g as long as S + round(t / g) <= 2^p:
//   the sum stays on the same grid and the step is an integer addition of the term rounded to
//   the grid.  Only two kinds of steps fall outside that rule: a step whose result would pass
//   2^(E+1) (it is rounded on the coarser grid above), and an exact half-grid tie (decided by
//   the parity of S).  Both are done with one native IEEE addition.
//
//   So a run of terms is: integer prefix sums of the grid-rounded terms, a search for the
//   first step that crosses the binade or is a tie, one native addition there, repeat.  The
//   running sum only grows (terms >= 0), so a sum crosses at most ~60 binades.
//
// The evaluator built on it: per-binade prefix tables over a long sequence (spc_seqtab.cu),
// which let every edge of a hub row evaluate its runs of that row with a few searches
// (spc_score.cu) and a full sum jump from binade to binade.
#pragma once

#include "spc_internal.cuh"

namespace spc {

constexpr int kLongRow = 256;  // rows / segments longer than this are summed by a whole CTA
constexpr unsigned long long kSat = 1ull << 62;

template <class F> struct FB;
template <> struct FB<double> {
    static constexpr int kMant = 52;          // stored significand bits
    static constexpr int kBiasM = 1075;       // exponent bias + kMant
    static constexpr int kEbHi = 1025;        // biased exponent of the largest binade needed (s < 8)
    __device__ static unsigned long long bits(double x) {
        return (unsigned long long)__double_as_longlong(x);
    }
    __device__ static double from_bits(unsigned long long b) { return __longlong_as_double((long long)b); }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
};
template <> struct FB<float> {
    static constexpr int kMant = 23;
    static constexpr int kBiasM = 150;
    static constexpr int kEbHi = 129;
    __device__ static unsigned long long bits(float x) { return __float_as_uint(x); }
    __device__ static float from_bits(unsigned long long b) { return __uint_as_float((unsigned)b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
};

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
    unsigned long long c = a + b;
    return c > kSat ? kSat : c;
}

// round(t / g) for the grid of binade `eb` (biased exponent of the running sum), t >= 0 finite;
// an exact half-grid value rounds down and sets *tie.  Saturates at kSat.
template <class F>
__device__ __forceinline__ unsigned long long grid_units(F t, int eb, bool* tie) {
    const unsigned long long b = FB<F>::bits(t);
    int et = (int)(b >> FB<F>::kMant);
    unsigned long long mt = b & ((1ull << FB<F>::kMant) - 1ull);
    if (et == 0) et = 1; else mt |= (1ull << FB<F>::kMant);
    const int d = eb - et;
    *tie = false;
    if (d <= 0) {
        const int sh = -d;
        if (sh >= 62 - FB<F>::kMant - 1) return mt ? kSat : 0ull;
        return mt << sh;
    }
    if (d > FB<F>::kMant + 2) return 0ull;
    const unsigned long long q = mt >> d;
    const unsigned long long rem = mt & ((1ull << d) - 1ull);
    const unsigned long long half = 1ull << (d - 1);
    *tie = rem == half;
    return q + (rem > half ? 1ull : 0ull);
}

// s = S * grid(eb), S in [2^kMant, 2^(kMant+1)]
template <class F>
__device__ __forceinline__ F from_units(unsigned long long S, int eb) {
    return FB<F>::from_bits(((unsigned long long)eb << FB<F>::kMant) + (S - (1ull << FB<F>::kMant)));
}

// Sum of int64 terms by a whole CTA (exact in any order).
template <class Term>
__device__ long long cta_sum_i64(int64_t L, const Term& term) {
    __shared__ long long sh[32];
    long long s = 0;
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) s += term(i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < nw; ++w) t += sh[w];
    __syncthreads();
    return t;
}

}  // namespace spc

namespace spc {

// ---- per-binade prefix tables over long sequences (built by spc_seqtab.cu) ---------------------
// Sequence q has terms[base[q] .. base[q] + len[q]).  For every binade eb in [eblo[q],
// eblo[q] + nE[q]) the tables hold, at tab_off[q] + (eb - eblo[q]) * (len[q] + 1) + k,
//   P = sum of grid_units(term_t, eb) over t < k  (saturating at kSat)
//   T = number of half-grid ties among t < k.
struct SeqTabView {
    const int64_t* base;
    const int64_t* len;
    const int32_t* eblo;
    const int32_t* nE;
    const int64_t* tab_off;
    const unsigned long long* P;
    const int32_t* T;
};

SeqTabView seqtab_view(const SeqTabBufs& tb, const int64_t* base, const int64_t* len);

// The left-to-right sum continued over terms x[a, b) of one tabled sequence from running value
// s (x = the sequence's first term).  Identical to adding the terms one by one.
template <class F>
__device__ F tab_run(F s, int64_t a, int64_t b, const F* __restrict__ x,
                     const unsigned long long* __restrict__ P, const int32_t* __restrict__ T,
                     int eblo, int nE, int64_t d1) {
    while (a < b) {
        if (s == F(0)) { s = x[a++]; continue; }
        const unsigned long long sb = FB<F>::bits(s);
        const int eb = (int)(sb >> FB<F>::kMant);
        const int e = eb - eblo;
        if (eb == 0 || e < 0 || e >= nE) { s = FB<F>::add(s, x[a++]); continue; }
        const unsigned long long* Pe = P + (int64_t)e * d1;
        const int32_t* Te = T + (int64_t)e * d1;
        const unsigned long long base = Pe[a];
        if (base >= kSat - (1ull << 55)) { s = FB<F>::add(s, x[a++]); continue; }
        const unsigned long long S = (sb & ((1ull << FB<F>::kMant) - 1ull)) | (1ull << FB<F>::kMant);
        const unsigned long long lim = (1ull << (FB<F>::kMant + 1)) - S;
        int64_t lo = a, hi = b;  // largest k in [a, b] whose prefix stays on this grid
        if (Pe[b] - base <= lim) {
            lo = b;  // the whole run stays on this grid: no search
        } else {
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (Pe[mid] - base <= lim) lo = mid; else hi = mid - 1;
            }
        }
        int64_t k = lo;
        const int32_t ta = Te[a];
        if (Te[k] > ta) {  // a half-grid tie inside: stop at the first one
            int64_t l2 = a, h2 = k - 1;
            while (l2 < h2) {
                const int64_t mid = (l2 + h2) >> 1;
                if (Te[mid + 1] > ta) h2 = mid; else l2 = mid + 1;
            }
            k = l2;
        }
        s = from_units<F>(S + (Pe[k] - base), eb);
        a = k;
        if (a < b) s = FB<F>::add(s, x[a++]);  // binade crossing or tie: one native step
    }
    return s;
}

// Warp-cooperative version of tab_run (all 32 lanes call it with the same arguments and get
// the same result): each search probes 32 positions at once.
template <class F>
__device__ F tab_run_warp(F s, int64_t a, int64_t b, const F* __restrict__ x,
                          const unsigned long long* __restrict__ P, const int32_t* __restrict__ T,
                          int eblo, int nE, int64_t d1) {
    const int lane = threadIdx.x & 31;
    while (a < b) {
        if (s == F(0)) { s = x[a++]; continue; }
        const unsigned long long sb = FB<F>::bits(s);
        const int eb = (int)(sb >> FB<F>::kMant);
        const int e = eb - eblo;
        if (eb == 0 || e < 0 || e >= nE) { s = FB<F>::add(s, x[a++]); continue; }
        const unsigned long long* Pe = P + (int64_t)e * d1;
        const int32_t* Te = T + (int64_t)e * d1;
        const unsigned long long base = Pe[a];
        if (base >= kSat - (1ull << 55)) { s = FB<F>::add(s, x[a++]); continue; }
        const unsigned long long S = (sb & ((1ull << FB<F>::kMant) - 1ull)) | (1ull << FB<F>::kMant);
        const unsigned long long lim = (1ull << (FB<F>::kMant + 1)) - S;
        const int32_t ta = Te[a];
        // largest k in [a, b] with Pe[k] - base <= lim and no tie among [a, k)
        int64_t lo = a, hi = b;  // invariant: lo is good; answer in [lo, hi]
        if (Pe[b] - base <= lim && Te[b] == ta) lo = b;  // the whole run: no search
        while (hi - lo > 0) {
            const int64_t span = hi - lo;
            const int64_t step = (span + 31) / 32;
            const int64_t probe = lo + (int64_t)(lane + 1) * step;
            bool good = false;
            if (probe <= hi) good = (Pe[probe] - base <= lim) && (Te[probe] == ta);
            const unsigned bal = __ballot_sync(0xffffffffu, good && probe <= hi);
            // good positions form a prefix of the probes (both conditions are monotone)
            const int ngood = __popc(bal);
            const int64_t new_lo = lo + (int64_t)ngood * step;
            int64_t new_hi = lo + (int64_t)(ngood + 1) * step - 1;
            if (new_hi > hi) new_hi = hi;
            lo = new_lo > hi ? hi : new_lo;
            hi = new_hi;
            if (step == 1) break;
        }
        const int64_t k = lo;
        s = from_units<F>(S + (Pe[k] - base), eb);
        a = k;
        if (a < b) s = FB<F>::add(s, x[a++]);
    }
    return s;
}

}  // namespace spc
