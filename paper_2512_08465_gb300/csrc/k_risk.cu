// Risk Index reduction (Section II-C, Eq. 1-3), exact.
//
// R_i = lambda_i S_i + m * sum_{j != i} fl(lambda_i lambda_j) S_ij with m = 1
// (Eq. 3 as written, each unordered pair once) or 2 (both orderings of the
// ordered N-2 enumeration).  Every double term is converted exactly to a
// 192-bit fixed-point integer with least significant bit 2^-128, the terms are
// added with integer carries (associative, so any thread or warp order gives
// the same sum) and the total is rounded once to the nearest double, ties to
// even.  Exact for lambda in [2^-30, 2^10]: every product then lies in
// [2^-60, 2^20], whose least significant bit is at least 2^-112, and the sum of
// up to 2^20 elements times 2 stays below 2^64.
//
// One warp per element i; lanes stride over partners j.  With F (E x E, row i for
// element i) the pair terms are explicit pair frequencies F_ij instead of the
// products fl(lambda_i lambda_j) (common-cause extension).
#include "cs_internal.h"

namespace {

struct U192 {
    unsigned long long w0, w1, w2;
};

__device__ __forceinline__ void add192(U192& a, const U192& b) {
    unsigned long long s0 = a.w0 + b.w0;
    unsigned long long c0 = s0 < a.w0;
    unsigned long long s1 = a.w1 + b.w1;
    unsigned long long c1 = s1 < a.w1;
    unsigned long long s1c = s1 + c0;
    c1 += s1c < s1;
    a.w0 = s0;
    a.w1 = s1c;
    a.w2 = a.w2 + b.w2 + c1;
}

// exact conversion of a positive finite double >= 2^-76 to fixed point
__device__ __forceinline__ U192 to_fixed(double d) {
    U192 r{0ull, 0ull, 0ull};
    if (!(d > 0.0)) return r;
    unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    int e = (int)((bits >> 52) & 0x7ff);
    unsigned long long m = bits & ((1ull << 52) - 1);
    if (e == 0) return r;                // subnormal: outside the supported range
    m |= (1ull << 52);
    int s = e - 947;                     // value * 2^128 = m * 2^(e - 1075 + 128)
    if (s < 0) {
        m >>= (-s < 64 ? -s : 63);       // outside the supported range (not exact)
        s = 0;
    }
    if (s < 64) {
        r.w0 = m << s;
        r.w1 = s ? (m >> (64 - s)) : 0ull;
    } else if (s < 128) {
        int t = s - 64;
        r.w1 = m << t;
        r.w2 = t ? (m >> (64 - t)) : 0ull;
    } else {
        r.w2 = m << (s - 128);
    }
    return r;
}

__device__ __forceinline__ int msb64(unsigned long long x) { return 63 - __clzll(x); }

// round-to-nearest-even of X * 2^-128
__device__ double round_fixed(const U192& x) {
    int p;
    if (x.w2) p = 128 + msb64(x.w2);
    else if (x.w1) p = 64 + msb64(x.w1);
    else if (x.w0) p = msb64(x.w0);
    else return 0.0;
    if (p <= 52) return ldexp((double)x.w0, -128);
    const int s = p - 52;   // drop s low bits
    // mant = X >> s (fits in 53 bits)
    unsigned long long mant;
    auto shr = [&](int k) -> unsigned long long {   // (X >> k) & (2^64 - 1)
        if (k >= 128) return x.w2 >> (k - 128);
        if (k >= 64) {
            int t = k - 64;
            return t ? ((x.w1 >> t) | (x.w2 << (64 - t))) : x.w1;
        }
        return k ? ((x.w0 >> k) | (x.w1 << (64 - k))) : x.w0;
    };
    mant = shr(s) & ((1ull << 53) - 1);
    // round bit s-1, sticky = any bit below s-1
    const int rb = s - 1;
    const unsigned long long round_bit = (shr(rb) & 1ull);
    bool sticky = false;
    {
        // bits [0, rb): check limbs fully below, then the partial limb
        int full = rb / 64, part = rb % 64;
        unsigned long long limbs[3] = {x.w0, x.w1, x.w2};
        for (int q = 0; q < full; ++q) sticky |= limbs[q] != 0ull;
        if (part) sticky |= (limbs[full] & ((1ull << part) - 1)) != 0ull;
    }
    int ex = s - 128;
    if (round_bit && (sticky || (mant & 1ull))) {
        mant += 1ull;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            ex += 1;
        }
    }
    return ldexp((double)mant, ex);
}

__device__ __forceinline__ long long pair_index(long long i, long long j, long long E) {
    return i * E - (i * (i + 1)) / 2 + (j - i - 1);
}

__global__ void risk_kernel(int E, const uint8_t* S1, const uint8_t* S2, const double* lam, const double* F,
                            int mode, double* R, unsigned long long* missing) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < E; i += nwarps) {
        const double li = lam[i];
        U192 acc{0ull, 0ull, 0ull};
        unsigned long long miss = 0;
        for (int j = lane; j < E; j += 32) {
            if (j == i) continue;
            const long long k = (i < j) ? pair_index(i, j, E) : pair_index(j, i, E);
            const uint8_t s = S2[k];
            if (s == 255) { if (i < j) ++miss; continue; }   // each missing pair once
            if (s) add192(acc, to_fixed(F ? F[(long long)i * E + j] : li * lam[j]));   // F: explicit pair frequencies
        }
        for (int off = 16; off; off >>= 1) {
            U192 o;
            o.w0 = __shfl_xor_sync(0xffffffffu, acc.w0, off);
            o.w1 = __shfl_xor_sync(0xffffffffu, acc.w1, off);
            o.w2 = __shfl_xor_sync(0xffffffffu, acc.w2, off);
            add192(acc, o);
            miss += __shfl_xor_sync(0xffffffffu, miss, off);
        }
        if (lane == 0) {
            if (mode == CS_RISK_ORDERED) {   // exact doubling of the pair sum
                acc.w2 = (acc.w2 << 1) | (acc.w1 >> 63);
                acc.w1 = (acc.w1 << 1) | (acc.w0 >> 63);
                acc.w0 = acc.w0 << 1;
            }
            const uint8_t s1 = S1[i];
            if (s1 == 255) ++miss;
            else if (s1) add192(acc, to_fixed(li));
            R[i] = round_fixed(acc);
            if (missing && miss) atomicAdd(missing, miss);
        }
    }
}

// Monte-Carlo form: R for n_samples rate vectors (sample-major lam[s * E + i]) against
// the same severity tables.  One CTA per element i keeps its partner severities in
// shared memory (not-evaluated pairs count 0); its warps take the samples.  Each
// sample's R_i is the same exact fixed-point sum, rounded once, as risk_kernel's.  A
// rate outside [2^-30, 2^10] gives NaN for that entry and sets bit `bad_bit` of *err.
__global__ void risk_batch_kernel(int E, const uint8_t* __restrict__ S1, const uint8_t* __restrict__ S2,
                                  const double* __restrict__ lam, long long ns, int mode, double* __restrict__ R,
                                  int* err, int bad_bit) {
    extern __shared__ uint8_t srow[];                 // [E] severities of the pairs (i, j)
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = threadIdx.x; j < E; j += blockDim.x) {
        uint8_t v = 0;
        if (j != i) {
            const long long k = (i < j) ? pair_index(i, j, E) : pair_index(j, i, E);
            v = (S2[k] == 1) ? 1 : 0;
        }
        srow[j] = v;
    }
    __syncthreads();
    const uint8_t s1 = (S1[i] == 1) ? 1 : 0;
    const double lo = 0x1p-30, hi = 0x1p10;
    for (long long sm = warp; sm < ns; sm += nw) {
        const double* ls = lam + sm * E;
        const double li = ls[i];
        U192 acc{0ull, 0ull, 0ull};
        bool bad = !(li >= lo && li <= hi);
        for (int j = lane; j < E; j += 32) {
            const double lj = ls[j];
            if (!(lj >= lo && lj <= hi)) bad = true;
            if (srow[j]) add192(acc, to_fixed(li * lj));
        }
        for (int off = 16; off; off >>= 1) {
            U192 o;
            o.w0 = __shfl_xor_sync(0xffffffffu, acc.w0, off);
            o.w1 = __shfl_xor_sync(0xffffffffu, acc.w1, off);
            o.w2 = __shfl_xor_sync(0xffffffffu, acc.w2, off);
            add192(acc, o);
        }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            if (bad) {
                R[sm * E + i] = __longlong_as_double(0x7ff8000000000000ll);
                atomicOr(err, 1 << bad_bit);
                continue;
            }
            if (mode == CS_RISK_ORDERED) {   // exact doubling of the pair sum
                acc.w2 = (acc.w2 << 1) | (acc.w1 >> 63);
                acc.w1 = (acc.w1 << 1) | (acc.w0 >> 63);
                acc.w0 = acc.w0 << 1;
            }
            if (s1) add192(acc, to_fixed(li));
            R[sm * E + i] = round_fixed(acc);
        }
    }
}

}  // namespace

cudaError_t launch_risk_batch(int nE, const uint8_t* S1, const uint8_t* S2, const double* lam, long long ns,
                              int mode, double* R, int* err, int bad_bit, cudaStream_t s) {
    if (nE <= 0 || ns <= 0) return cudaSuccess;
    risk_batch_kernel<<<nE, 256, (size_t)nE, s>>>(nE, S1, S2, lam, ns, mode, R, err, bad_bit);
    return cudaGetLastError();
}

cudaError_t launch_risk(int nE, const uint8_t* S1, const uint8_t* S2, const double* lam, int mode,
                        double* R, int64_t* missing, cudaStream_t s, const double* F) {
    if (nE <= 0) return cudaSuccess;
    int blocks = (nE * 32 + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    risk_kernel<<<blocks, 256, 0, s>>>(nE, S1, S2, lam, F, mode, R, (unsigned long long*)missing);
    return cudaGetLastError();
}
