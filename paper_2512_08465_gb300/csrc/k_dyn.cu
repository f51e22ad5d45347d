// Small-signal screen of converged OPF points, one scenario per CTA
// (Section II-B-2: the system model is linearised at the OPF operating point
// and a scenario is unstable when an eigenvalue has a non-negative real part;
// the configuration adds a minimum damping ratio).
//
// Model (per in-service generator, machine data converted to the system base):
// states delta, omega, e'q, e'd, Efd (index 5k + s); E' = (e'q - j e'd) e^{j delta}
// behind j x' (x'd = x'q, Ra = 0); I = Y_red E' with Y_red the Kron reduction of
// the network (loads as constant admittances at the OPF voltage, machines as
// 1/(j x') to their internal nodes); i_d + j i_q = j I e^{-j delta};
//   d delta/dt = ws (omega - 1)
//   2H d omega/dt = Pm - (e'd i_d + e'q i_q) - D (omega - 1)
//   T'd0 d e'q/dt = -e'q - (x_d - x') i_d + Efd
//   T'q0 d e'd/dt = -e'd + (x_q - x') i_q
//   T_A d Efd/dt = -Efd + K_A (V_ref - |E' - j x' I|)
// The state matrix is written from hand-derived partial derivatives of these
// equations (the CPU oracle differentiates them automatically instead).
//
// Steps inside one CTA:
//  1. Y_bb = Ybus(outages masked) + loads + machine admittances, factorised as
//     a complex symmetric LDL^T on the network's shared symbolic analysis
//     (scalar complex blocks, same elimination-tree levels as the OPF kernel);
//  2. one thread per in-service machine solves Y_bb x = e_{bus} to get the
//     machine-bus entries of Y_bb^{-1}, hence Y_red;
//  3. equilibrium from the OPF point; one thread per machine pair writes the
//     5x5 block of A;
//  4. balancing by powers of two, Householder Hessenberg reduction, Francis
//     double-shift QR (eigenvalues only), with the same steps and thresholds
//     as the textbook algorithm; A lives in the CTA's global scratch (the
//     resident CTAs' matrices together fit in the 129 MB L2);
//  5. max Re and min damping ratio over all eigenvalues, classify.
// Angle reference: every rotor angle is referred to the first in-service
// machine (delta'_k = delta_k - delta_0, d delta'_k/dt = ws (omega_k - omega_0),
// delta_0 dropped).  The absolute-angle matrix has an exact zero eigenvalue
// (common rotation) to which the slow common-frequency mode is nearly parallel;
// the referred matrix (5m - 1 states) has the same eigenvalues less that zero
// and a well-conditioned slow mode.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "cs_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr double kEps = 2.220446049250313e-16;
// FP32 QR deflates a subdiagonal entry below kDeflTol times its two diagonal neighbours
// (not the FP32 unit roundoff): the screen's eigenvalues need only be within kEigDelta of
// the exact ones where the decisive ones are refined in FP64 (within the 5e-3 guard band
// where a network's screen has no refinement), and the sweeps that take a converged entry
// from ~1e-6 relative down to rounding level are most of the QR's work.
// On 118-bus state matrices (order 264-269, FP32 emulation) it cuts the sweeps per matrix
// from 785 to 322 on average, the largest eigenvalue error staying at 8e-5 either way.
constexpr float kDeflTol = 3e-6f;
// FP32 screen in global memory (no refinement): a decision this close to a threshold is
// taken by the FP64 screen instead
constexpr double kGuardRe = 5e-3;      // |max Re| within this of 0
constexpr double kGuardZeta = 5e-3;    // |min zeta - threshold| within this

struct DLay {
    int Yu, Yl, Yd, Ydi;      // complex arrays (2 doubles per entry)
    int Z;                    // [ng*ng] complex
    int rhs;                  // [ng*nb] complex
    int gen;                  // [ng * kGen]
    int A;                    // [(5ng)^2]
    int A32;                  // [(5ng)^2] floats (mixed precision screen)
    int wr, wi, v;            // [5ng]
    int total;
};
constexpr int kGen = 16;      // per-generator doubles: E(2) I(2) e^{jd}(2) Vt(2) |Vt| id iq eq ed ym(2)
enum { G_E = 0, G_I = 2, G_ED = 4, G_VT = 6, G_VTM = 8, G_ID = 9, G_IQ = 10, G_EQ = 11, G_EDD = 12, G_YM = 13 };

DLay make_dlayout(const DevNet& n) {
    DLay L{};
    int o = 0;
    auto take = [&](long cnt) { int r = o; o += (int)cnt; return r; };
    L.Yu = take(2L * n.nL); L.Yl = take(2L * n.nL); L.Yd = take(2L * n.nb); L.Ydi = take(2L * n.nb);
    L.Z = take(2L * n.ng * n.ng);
    L.rhs = take(2L * n.ng * n.nb);
    L.gen = take((long)kGen * n.ng);
    o = (o + 31) & ~31;
    L.A = take(25L * n.ng * n.ng);
    L.A32 = take((25L * n.ng * n.ng + 1) / 2);
    o = (o + 31) & ~31;
    L.wr = take(5L * n.ng); L.wi = take(5L * n.ng); L.v = take(5L * n.ng);
    L.total = (o + 31) & ~31;
    return L;
}

__device__ __forceinline__ cplx ld(const double* p) { return cplx{p[0], p[1]}; }
__device__ __forceinline__ void st(double* p, cplx v) { p[0] = v.re; p[1] = v.im; }

struct DShared {
    double red[2][kThreads];
    int ired[kThreads];
    double x[3];                     // next bulge column
    double u[4];                     // reflector of the current step: u0, u1, u2, beta
    double part[2][kThreads / 32];   // per-warp partial sums, double-buffered
    int lo, hi, its, fail, scen, m, nn;
    double hmax;
    double bal_f;
    int bal_i;
};

// block reductions ---------------------------------------------------------
__device__ int bmax_int(DShared& sh, int v) {
    const int tid = threadIdx.x;
    for (int off = 16; off; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((tid & 31) == 0) sh.ired[tid >> 5] = v;
    __syncthreads();
    int r = sh.ired[0];
    for (int w = 1; w < kThreads / 32; ++w) r = max(r, sh.ired[w]);
    __syncthreads();
    return r;
}
__device__ double bmax(DShared& sh, double v) {
    const int tid = threadIdx.x;
    for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((tid & 31) == 0) sh.red[0][tid >> 5] = v;
    __syncthreads();
    double r = sh.red[0][0];
    for (int w = 1; w < kThreads / 32; ++w) r = fmax(r, sh.red[0][w]);
    __syncthreads();
    return r;
}

// eigenvalues of [[p, q], [r, s]] (same formulas as the textbook closed form)
__device__ void eig2(double p, double q, double r, double s, double* re, double* im) {
    const double hm = 0.5 * (p - s);
    const double disc = hm * hm + q * r;
    const double mean = 0.5 * (p + s);
    if (disc >= 0.0) {
        const double root = sqrt(disc);
        const double big = mean + (hm >= 0.0 ? root : -root);
        const double det = p * s - q * r;
        const double other = (big != 0.0) ? det / big : mean - (hm >= 0.0 ? root : -root);
        re[0] = big; im[0] = 0.0;
        re[1] = other; im[1] = 0.0;
    } else {
        const double root = sqrt(-disc);
        re[0] = mean; im[0] = root;
        re[1] = mean; im[1] = -root;
    }
}


// ---------------------------------------------------------------------------
// Eigenvalues of a real matrix: balancing by powers of two, Householder
// reduction to upper Hessenberg form, Francis double-shift QR with deflation
// (eigenvalues only), as in the textbook algorithm.  A is row-major n x n in
// global memory; cs, rs, v are n-entry shared arrays of T.

// Balancing (radix 2).  Each sweep starts from exact off-diagonal column and
// row 1-norms; within the sweep the norms are updated as rows and columns are
// scaled (a scaling by a power of two changes the other norms by a known
// amount), so the sequential scan over the indices needs no reduction.  One
// thread takes each index's decision; only indices that are scaled cost a
// pass over the matrix.  The scale search stops at 2^+-kBalExp (T = float) or
// 2^+-(4 kBalExp) (T = double), so a row or column norm that is tiny next to
// the other cannot drive the factor to overflow or zero; an index whose best
// factor lies beyond that is scaled by the bound.  When dsc is given, dsc[i]
// receives the product of the factors of index i: the balanced matrix is
// diag(dsc)^-1 A diag(dsc), exactly (every factor is a power of two).
constexpr int kBalExp = 30;
template <typename T>
__device__ void balance(T* A, const int n, T* cs, T* rs, DShared& sh, T* dsc = nullptr) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const T fmaxb = (T)ldexp(1.0, sizeof(T) == 8 ? 4 * kBalExp : kBalExp), fminb = (T)1 / fmaxb;
    if (dsc)
        for (int j = tid; j < n; j += kThreads) dsc[j] = (T)1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        for (int j = tid; j < n; j += kThreads) {
            T c = 0;
            for (int i = 0; i < n; ++i)
                if (i != j) c += fabs(A[(size_t)i * n + j]);
            cs[j] = c;
        }
        for (int i = warp; i < n; i += kThreads / 32) {
            T r = 0;
            for (int j = lane; j < n; j += 32)
                if (j != i) r += fabs(A[(size_t)i * n + j]);
            for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
            if (lane == 0) rs[i] = r;
        }
        __syncthreads();
        bool changed = false;
        int i0 = 0;
        for (;;) {
            if (tid == 0) {
                int pick = -1;
                double fpick = 1.0;
                for (int i = i0; i < n && pick < 0; ++i) {
                    T c = cs[i];
                    const T r = rs[i];
                    if (c == 0 || r == 0 || !isfinite(c) || !isfinite(r)) continue;
                    T g = r / 2, f = 1;
                    const T ssum = c + r;
                    while (c < g && f < fmaxb) { f *= 2; c *= 4; }
                    g = r * 2;
                    while (c > g && f > fminb) { f /= 2; c /= 4; }
                    if ((c + r) / f < (T)0.95 * ssum) { pick = i; fpick = (double)f; }
                }
                sh.bal_i = pick;
                sh.bal_f = fpick;
            }
            __syncthreads();
            const int i = sh.bal_i;
            if (i < 0) break;
            const T f = (T)sh.bal_f, finv = (T)(1.0 / sh.bal_f);
            for (int j = tid; j < n; j += kThreads) {
                if (j == i) {
                    cs[i] *= f;
                    rs[i] *= finv;
                    if (dsc) dsc[i] *= f;
                    continue;
                }
                const T a = A[(size_t)i * n + j], b = A[(size_t)j * n + i];
                A[(size_t)i * n + j] = a * finv;
                A[(size_t)j * n + i] = b * f;
                cs[j] += fabs(a) * (finv - 1);
                rs[j] += fabs(b) * (f - 1);
            }
            changed = true;
            i0 = i + 1;
            __syncthreads();
        }
        if (!changed) break;
    }
}

// Householder reduction to upper Hessenberg form (column k: reflector from
// rows k+1.., applied from the left to columns k+1.. and from the right to all
// rows).  The reflector lives in shared memory.
template <typename T>
__device__ void hessenberg(T* A, const int n, T* v, DShared& sh) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = 0; k + 2 < n; ++k) {
        T t = 0;
        for (int i = k + 2 + tid; i < n; i += kThreads) {
            const T q = A[(size_t)i * n + k];
            t += q * q;
        }
        for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) sh.part[k & 1][warp] = (double)t;
        __syncthreads();
        T tail = 0;
        for (int w = 0; w < kThreads / 32; ++w) tail += (T)sh.part[k & 1][w];
        if (tail == 0) continue;               // column already reduced (uniform)
        const T x0 = A[(size_t)(k + 1) * n + k];
        const T nrm = sqrt(x0 * x0 + tail);
        const T alpha = (x0 >= 0) ? -nrm : nrm;
        const T v0 = x0 - alpha;
        const T beta = (T)2 / (v0 * v0 + tail);
        const int mm = n - k - 1;
        for (int i = tid; i < mm; i += kThreads) v[i] = (i == 0) ? v0 : A[(size_t)(k + 1 + i) * n + k];
        __syncthreads();
        for (int j = k + 1 + tid; j < n; j += kThreads) {          // left, columns k+1..n-1
            T* col = A + (size_t)(k + 1) * n + j;
            T s = 0;
#pragma unroll 8
            for (int i = 0; i < mm; ++i) s += v[i] * col[(size_t)i * n];
            s *= beta;
#pragma unroll 8
            for (int i = 0; i < mm; ++i) col[(size_t)i * n] -= s * v[i];
        }
        for (int i = k + 1 + tid; i < n; i += kThreads)            // column k itself
            A[(size_t)i * n + k] = (i == k + 1) ? alpha : (T)0;
        __syncthreads();
        for (int i = warp; i < n; i += kThreads / 32) {            // right, all rows
            T* row = A + (size_t)i * n + k + 1;
            T s = 0;
            for (int j = lane; j < mm; j += 32) s += row[j] * v[j];
            for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            s *= beta;
            for (int j = lane; j < mm; j += 32) row[j] -= s * v[j];
        }
        __syncthreads();
    }
}

// Francis double-shift QR on the Hessenberg matrix in global memory,
// eigenvalues only (updates restricted to the active block lo..hi).
// sh.fail = 2 if it does not converge in 30 n sweeps.
template <typename T>
__device__ void hqr_global(T* A, const int n, double* wr, double* wi, DShared& sh) {
    const int tid = threadIdx.x;
    const double eps = (sizeof(T) == 8) ? kEps : (double)kDeflTol;       // deflation tolerance
    {
        double hm = 0.0;
        for (int w = tid; w < n * n; w += kThreads) {
            const int i = w / n, j = w % n;
            if (j >= i - 1) hm = fmax(hm, fabs((double)A[w]));
        }
        hm = bmax(sh, hm);
        if (tid == 0) {
            sh.hmax = hm;
            sh.hi = n - 1;
            sh.its = 0;
        }
        __syncthreads();
    }
    while (sh.hi >= 0) {
        const int hi = sh.hi;
        // top of the unreduced block ending at hi: largest l <= hi with a negligible A[l][l-1]
        int cand = 0;
        for (int l = 1 + tid; l <= hi; l += kThreads) {
            double sd = fabs((double)A[(size_t)(l - 1) * n + l - 1]) + fabs((double)A[(size_t)l * n + l]);
            if (sd == 0.0) sd = sh.hmax;
            if (fabs((double)A[(size_t)l * n + l - 1]) <= eps * sd) cand = max(cand, l);
        }
        const int lo = bmax_int(sh, cand);
        if (lo == hi) {
            if (tid == 0) {
                wr[hi] = A[(size_t)hi * n + hi];
                wi[hi] = 0.0;
                sh.hi = hi - 1;
                sh.its = 0;
            }
            __syncthreads();
            continue;
        }
        if (lo == hi - 1) {
            if (tid == 0) {
                double re[2], im[2];
                eig2(A[(size_t)(hi - 1) * n + hi - 1], A[(size_t)(hi - 1) * n + hi], A[(size_t)hi * n + hi - 1],
                     A[(size_t)hi * n + hi], re, im);
                wr[hi - 1] = re[0]; wi[hi - 1] = im[0];
                wr[hi] = re[1]; wi[hi] = im[1];
                sh.hi = hi - 2;
                sh.its = 0;
            }
            __syncthreads();
            continue;
        }
        if (sh.its >= 30 * n) {
            if (tid == 0) sh.fail = 2;
            __syncthreads();
            break;
        }
        __syncthreads();
        if (tid == 0) {
            const int its = ++sh.its;
            double sft, tft;
            const double a11 = A[(size_t)(hi - 1) * n + hi - 1], a12 = A[(size_t)(hi - 1) * n + hi];
            const double a21 = A[(size_t)hi * n + hi - 1], a22 = A[(size_t)hi * n + hi];
            if (its == 10 || its == 20) {              // exceptional shift
                const double ww = fabs(a21) + fabs(A[(size_t)(hi - 1) * n + hi - 2]);
                sft = 1.5 * ww;
                tft = ww * ww;
            } else {
                sft = a11 + a22;
                tft = a11 * a22 - a12 * a21;
            }
            const double h00 = A[(size_t)lo * n + lo], h01 = A[(size_t)lo * n + lo + 1];
            const double h10 = A[(size_t)(lo + 1) * n + lo], h11 = A[(size_t)(lo + 1) * n + lo + 1];
            const double h21 = A[(size_t)(lo + 2) * n + lo + 1];
            sh.x[0] = h00 * h00 + h01 * h10 - sft * h00 + tft;
            sh.x[1] = h10 * (h00 + h11 - sft);
            sh.x[2] = h10 * h21;
        }
        __syncthreads();
        // The reflector of each step is computed once, by thread 0, and broadcast: on this
        // GPU a warp-wide FP64 instruction costs the FP64 pipe the same whatever its active
        // lanes, so every warp computing it would multiply that cost by the warp count.
        for (int k = lo; k <= hi - 1; ++k) {
            const int len = (k + 2 <= hi) ? 3 : 2;
            const bool more = (k + 1 <= hi - 1);
            if (tid == 0) {
                const double x0 = sh.x[0], x1 = sh.x[1], x2 = (len == 3) ? sh.x[2] : 0.0;
                const double t2 = x1 * x1 + x2 * x2;
                if (t2 != 0.0) {
                    const double nrm = sqrt(x0 * x0 + t2);
                    const double al = (x0 >= 0.0) ? -nrm : nrm;
                    sh.u[0] = x0 - al;
                    sh.u[1] = x1;
                    sh.u[2] = x2;
                    sh.u[3] = 2.0 / ((x0 - al) * (x0 - al) + t2);
                } else {
                    sh.u[3] = 0.0;                 // no reflector this step
                }
            }
            __syncthreads();
            const T bt = (T)sh.u[3];
            if (bt != (T)0) {
                const T u0 = (T)sh.u[0], u1 = (T)sh.u[1], u2 = (len == 3) ? (T)sh.u[2] : (T)0;
                const int c0 = (k > lo) ? k - 1 : lo;
                for (int j = c0 + tid; j <= hi; j += kThreads) {   // rows k..k+len-1
                    T* p0 = A + (size_t)k * n + j;
                    T d = u0 * p0[0] + u1 * p0[n];
                    if (len == 3) d += u2 * p0[2 * n];
                    d *= bt;
                    p0[0] -= d * u0;
                    p0[n] -= d * u1;
                    if (len == 3) p0[2 * n] -= d * u2;
                }
                __syncthreads();
                const int r1 = (k + 3 < hi) ? k + 3 : hi;
                for (int i = lo + tid; i <= r1; i += kThreads) {   // columns k..k+len-1
                    T* p0 = A + (size_t)i * n + k;
                    T d = p0[0] * u0 + p0[1] * u1;
                    if (len == 3) d += p0[2] * u2;
                    d *= bt;
                    p0[0] -= d * u0;
                    p0[1] -= d * u1;
                    if (len == 3) p0[2] -= d * u2;
                    if (i > k && i <= k + 3) sh.x[i - k - 1] = (double)p0[0];   // next bulge column
                }
                __syncthreads();
            } else if (more) {
                if (tid == 0) {
                    sh.x[0] = A[(size_t)(k + 1) * n + k];
                    sh.x[1] = A[(size_t)(k + 2) * n + k];
                    sh.x[2] = (k + 3 <= hi) ? (double)A[(size_t)(k + 3) * n + k] : 0.0;
                }
                __syncthreads();
            }
        }
        for (int i = lo + 2 + tid; i <= hi; i += kThreads) {
            A[(size_t)i * n + i - 2] = (T)0;
            if (i >= lo + 3) A[(size_t)i * n + i - 3] = (T)0;
        }
        __syncthreads();
    }
}

template <typename T>
__device__ void eigen_screen(T* A, const int n, T* cs, T* rs, T* v, double* wr, double* wi, DShared& sh) {
    balance<T>(A, n, cs, rs, sh);
    hessenberg<T>(A, n, v, sh);
    hqr_global<T>(A, n, wr, wi, sh);
}

// ---------------------------------------------------------------------------
// Packed Hessenberg storage for the shared-memory QR: row i keeps columns
// max(i-3, 0)..n-1 (the Hessenberg part plus the two sub-diagonals the bulge
// passes through).  hq_off(n, i) is the offset of row i; hq_off(n, n) the size.
__host__ __device__ inline int hq_start(int i) { return i > 3 ? i - 3 : 0; }
__host__ __device__ inline int hq_off(int n, int i) {
    if (i <= 3) return n * i;
    return 3 * n + (i - 3) * (n + 3) - (i * (i - 1) / 2 - 3);
}
constexpr int kHqHead = 4;          // floats before the packed matrix: the order n (int bits), padding

// Slot of one scenario in the balanced-matrix buffer (front kernel -> cluster
// Hessenberg kernel -> refinement kernel), floats: the head, the balanced
// matrix (row-major n x n), then the balancing factors D (the balanced matrix is
// D^-1 A D) and the Householder factors beta_k.  The cluster kernel overwrites
// the matrix area with the Householder vectors once it has loaded the matrix:
// vector k (entries for rows k+1..n-1, the first one the reflector's head) at
// refl_off(n, k).
__host__ __device__ inline size_t ab_mat_floats(int nmax) { return ((size_t)nmax * nmax + 3) & ~(size_t)3; }
__host__ __device__ inline size_t ab_d_off(int nmax) { return kHqHead + ab_mat_floats(nmax); }
__host__ __device__ inline size_t ab_beta_off(int nmax) { return ab_d_off(nmax) + (((size_t)nmax + 3) & ~(size_t)3); }
__host__ __device__ inline size_t ab_stride(int nmax) { return ab_beta_off(nmax) + (((size_t)nmax + 3) & ~(size_t)3); }
__host__ __device__ inline int refl_off(int n, int k) { return k * (n - 1) - (k * (k - 1)) / 2; }

// Candidates of the FP64 refinement per scenario (shared-memory QR -> refinement
// kernel), floats: [0] count (int bits), [1] flags (int bits; bit 2c: candidate c
// may carry the largest real part, bit 2c+1: the smallest damping ratio), then
// the FP32 eigenvalue (re, im >= 0) of each candidate.
constexpr int kRefK = 4;                     // candidates per scenario at most (more: FP64 re-run)
constexpr int kCandStride = 4 + 2 * kRefK;
// Bound on the distance of an FP32 eigenvalue of the 118-bus state matrix from the
// exact one (measured differences are below 3e-5): an eigenvalue can decide max Re
// or min zeta only if its FP32 value is within this bound of deciding it.
constexpr float kEigDelta = 1e-3f;
// Refined statistics within this distance of a threshold (max Re = 0, min zeta =
// damping_min) are decided by the FP64 screen instead (the refined values are within
// ~1e-9 of the FP64 screen's).
constexpr double kRefinedGuard = 1e-7;

// max Re and min damping ratio over the n eigenvalues (block-wide, result on all threads)
__device__ void eig_stats(DShared& sh, int n, const double* wr, const double* wi, double& maxre, double& minz) {
    const int tid = threadIdx.x;
    double mr = -INFINITY, mz = INFINITY;
    if (!sh.fail) {
        for (int i = tid; i < n; i += kThreads) {
            mr = fmax(mr, wr[i]);
            const double mg = sqrt(wr[i] * wr[i] + wi[i] * wi[i]);
            mz = fmin(mz, mg > 0.0 ? -wr[i] / mg : 1.0);
        }
    }
    maxre = bmax(sh, mr);
    minz = -bmax(sh, -mz);
}

// Kernel modes.  FULL64: FP64 screen of every converged OPF point (the FP64
// form).  MIXED_INLINE: FP32 screen in global memory with the FP64 re-run
// inline (mixed form, kept for networks the tensor-core path does not take).
// FRONT: model and FP32 balancing; the balanced matrix goes to a per-scenario
// buffer for hess_cluster_kernel.  RERUN: FP64 screen of the scenarios that
// the FP32 screen could not decide (status 6).  FRONT_LARGE / QR_LARGE: the
// mixed form of networks whose Hessenberg matrix exceeds shared memory: the
// balanced FP32 matrix, padded to the network's largest state order with a
// decoupled -1 diagonal (so one batch has one order), goes to the tensor-core
// blocked Hessenberg reduction (k_tc.cu), then FP32 QR in global memory over the
// padded order with statistics over the first n eigenvalues (the padding's -1
// eigenvalues deflate first, into the last positions), guard band to RERUN.
enum { DYN_FULL64 = 0, DYN_MIXED_INLINE = 1, DYN_FRONT = 2, DYN_RERUN = 3, DYN_FRONT_LARGE = 4, DYN_QR_LARGE = 5 };

template <int kMode>
__global__ void __launch_bounds__(kThreads)
dyn_kernel(DevNet net, EvalArgs a, OpfOut o, double damping_min, double* scratch, size_t per_cta, DLay L,
           float* hbuf, size_t hstride, double* a64, size_t a64stride, int* counter) {
    __shared__ DShared sh;
    extern __shared__ double dsm[];   // [ng] ints (compact -> generator id), then cs, rs, v [5 ng] each
    int* gidx = reinterpret_cast<int*>(dsm);
    double* cs_d = dsm + ((net.ng + 1) >> 1);
    double* rs_d = cs_d + 5 * net.ng;
    double* v_d = rs_d + 5 * net.ng;
    const int tid = threadIdx.x;
    double* W = scratch + per_cta * blockIdx.x;
    const int nb = net.nb, ng = net.ng, nbr = net.nbr;
    const int nx = 2 * nb + 2 * ng;
    const double* Pd = net.Pd + (size_t)a.level * nb;
    const double* Qd = net.Qd + (size_t)a.level * nb;

    for (;;) {
        if (tid == 0) sh.scen = atomicAdd(counter, 1);
        __syncthreads();
        const int s = sh.scen;
        if (s >= a.n) break;
        if (o.status[s] != (kMode == DYN_RERUN ? 6 : 1)) {
            __syncthreads();
            continue;
        }
        if (kMode == DYN_QR_LARGE) {                  // QR of the padded Hessenberg matrix (tensor-core reduction)
            float* slot = hbuf + (size_t)s * hstride;
            const int n = __float_as_int(slot[0]), nmax = 5 * ng - 1;
            double* wr = W + L.wr;
            double* wi = W + L.wi;
            if (tid == 0) sh.fail = 0;
            __syncthreads();
            hqr_global<float>(slot + kHqHead, nmax, wr, wi, sh);
            double maxre = 0.0, minz = 0.0;
            eig_stats(sh, n, wr, wi, maxre, minz);
            if (tid == 0) {
                const bool near = sh.fail || !(fabs(maxre) > kGuardRe) || !(fabs(minz - damping_min) > kGuardZeta);
                if (near) {                           // decision too close to call in FP32: FP64 screen
                    o.status[s] = 6;
                    atomicAdd(a.reruns, 1);
                } else {
                    uint8_t k;
                    if (maxre >= 0.0) k = CS_SS_UNSTABLE;
                    else if (minz < damping_min) k = CS_SS_POORLY_DAMPED;
                    else k = CS_SECURE;
                    if (a.out.n_islands[s] > 1) {     // main island: the scenario's class stays ISLANDED
                        if (a.out.main_klass) a.out.main_klass[s] = k;
                    } else {
                        a.out.klass[s] = k;
                        a.out.severe[s] = (k != CS_SECURE);
                    }
                    a.out.max_re[s] = maxre;
                    a.out.min_zeta[s] = minz;
                }
            }
            __syncthreads();
            continue;
        }
        const Outage out = decode_outage(nbr, ng, a.ei[s], a.ej[s], a.ek ? a.ek[s] : -1);
        const double* xs = o.x + (size_t)s * nx;
        // main island of an islanded scenario: the OPF point has Vm = 0 at the buses
        // outside it; those buses, their branches and their machines are out of the model
        const bool isl = a.out.n_islands[s] > 1;
        auto live = [&](int i) { return !isl || xs[nb + i] != 0.0; };
        if (tid == 0) {
            int m = 0;
            for (int k = 0; k < ng; ++k)
                if (!gen_out(out, k) && live(net.gbus[k])) gidx[m++] = k;
            sh.m = m;
            sh.nn = 5 * m - 1;           // angles referred to the first in-service machine
            sh.fail = 0;
        }
        __syncthreads();
        const int m = sh.m, n = sh.nn;

        // ---- 1. assemble Y_bb on the symbolic pattern ----
        for (int tg = tid; tg < nb + net.nL; tg += kThreads) {
            if (tg < nb) {
                const int j = tg, i = net.perm[j];
                if (!live(i)) {                       // de-energised bus: identity row
                    st(W + L.Yd + 2 * j, cm(1.0, 0.0));
                    continue;
                }
                const double Vm = xs[nb + i];
                cplx y = cm(net.gsh[i], net.bsh[i]);
                y = y + (1.0 / (Vm * Vm)) * cm(Pd[i], -Qd[i]);
                for (int e = net.bus_br_ptr[i]; e < net.bus_br_ptr[i + 1]; ++e) {
                    const int code = net.bus_br[e];
                    const int b = code >> 1, side = code & 1;
                    if (br_out(out, b)) continue;
                    y = y + (side ? net.ytt[b] : net.yff[b]);
                }
                for (int e = net.bus_gen_ptr[i]; e < net.bus_gen_ptr[i + 1]; ++e) {
                    const int k = net.bus_gen[e];
                    if (gen_out(out, k)) continue;
                    y = y + cm(0.0, -1.0 / net.xp[k]);
                }
                st(W + L.Yd + 2 * j, y);
            } else {
                const int q = tg - nb;
                const int Rb = net.perm[net.Lrow[q]];
                cplx y = cm(0.0, 0.0);
                for (int e = net.blk_br_ptr[q]; e < net.blk_br_ptr[q + 1]; ++e) {
                    const int b = net.blk_br[e];
                    if (br_out(out, b) || !live(net.f[b])) continue;
                    y = y + ((net.f[b] == Rb) ? net.yft[b] : net.ytf[b]);
                }
                st(W + L.Yu + 2 * q, y);
            }
        }
        __syncthreads();
        // ---- complex LDL^T, level by level ----
        for (int lev = 0; lev < net.nlevels; ++lev) {
            const int t0 = net.tgt_ptr[lev], t1 = net.tgt_ptr[lev + 1];
            for (int w = tid; w < t1 - t0; w += kThreads) {
                const int tg = net.tgt[t0 + w];
                double* A = (tg < nb) ? (W + L.Yd + 2 * tg) : (W + L.Yu + 2 * (tg - nb));
                cplx acc = ld(A);
                for (int u = net.upd_ptr[tg]; u < net.upd_ptr[tg + 1]; ++u)
                    acc = acc - ld(W + L.Yl + 2 * net.upd_a[u]) * ld(W + L.Yu + 2 * net.upd_b[u]);
                st(A, acc);
            }
            __syncthreads();
            for (int w = net.lev_ptr[lev] + tid; w < net.lev_ptr[lev + 1]; w += kThreads) {
                const int j = net.lev_col[w];
                const cplx d = ld(W + L.Yd + 2 * j);
                if (!(abs2(d) > 0.0) || !isfinite(abs2(d))) sh.fail = 1;
                st(W + L.Ydi + 2 * j, cdiv(cm(1.0, 0.0), d));
            }
            __syncthreads();
            for (int w = tid; w < t1 - t0; w += kThreads) {
                const int tg = net.tgt[t0 + w];
                if (tg < nb) continue;
                const int q = tg - nb;
                st(W + L.Yl + 2 * q, ld(W + L.Yu + 2 * q) * ld(W + L.Ydi + 2 * net.Lcol[q]));
            }
            __syncthreads();
        }
        // ---- 2. machine-bus entries of Y_bb^{-1}: one sparse solve per machine ----
        for (int kk = tid; kk < m; kk += kThreads) {
            double* y = W + L.rhs + (size_t)2 * nb * kk;
            for (int j = 0; j < nb; ++j) { y[2 * j] = 0.0; y[2 * j + 1] = 0.0; }
            const int jb = net.iperm[net.gbus[gidx[kk]]];
            y[2 * jb] = 1.0;
            for (int j = 0; j < nb; ++j) {           // forward, elimination order
                cplx acc = ld(y + 2 * j);
                for (int e = net.Lrowptr[j]; e < net.Lrowptr[j + 1]; ++e)
                    acc = acc - ld(W + L.Yl + 2 * net.Lrowblk[e]) * ld(y + 2 * net.Lrowcol[e]);
                st(y + 2 * j, acc);
            }
            for (int j = 0; j < nb; ++j) st(y + 2 * j, ld(y + 2 * j) * ld(W + L.Ydi + 2 * j));
            for (int j = nb - 1; j >= 0; --j) {       // backward
                cplx acc = ld(y + 2 * j);
                for (int e = net.Lcolptr[j]; e < net.Lcolptr[j + 1]; ++e)
                    acc = acc - ld(W + L.Yl + 2 * e) * ld(y + 2 * net.Lrow[e]);
                st(y + 2 * j, acc);
            }
        }
        __syncthreads();
        // Y_red[k][l] = ym_k delta_kl - ym_k ym_l (Ybb^-1)[b_k][b_l]
        for (int w = tid; w < m * m; w += kThreads) {
            const int k = w / m, l = w % m;
            const cplx ymk = cm(0.0, -1.0 / net.xp[gidx[k]]), yml = cm(0.0, -1.0 / net.xp[gidx[l]]);
            const int jl = net.iperm[net.gbus[gidx[l]]];
            cplx z = ld(W + L.rhs + (size_t)2 * nb * k + 2 * jl);
            cplx v = cm(0.0, 0.0) - ymk * yml * z;
            if (k == l) v = v + ymk;
            st(W + L.Z + 2 * (size_t)(k * m + l), v);
        }
        // ---- 3. equilibrium per machine ----
        for (int kk = tid; kk < m; kk += kThreads) {
            const int k = gidx[kk], i = net.gbus[k];
            double sa, ca;
            sincos(xs[i], &sa, &ca);
            const cplx V = xs[nb + i] * cm(ca, sa);
            const cplx S = cm(xs[2 * nb + k], xs[2 * nb + ng + k]);
            const cplx I = conj(cdiv(S, V));
            const cplx EQ = V + mulj(net.xq[k] * I);
            const double delta = atan2(EQ.im, EQ.re);
            double sd, cd;
            sincos(delta, &sd, &cd);
            const cplx ejd = cm(cd, sd);
            const cplx rot = mulj(conj(ejd));            // j e^{-j delta}
            const cplx Idq = I * rot, Vdq = V * rot;   // OPF current, used for the equilibrium only
            const double xp = net.xp[k];
            const double eq = Vdq.im + xp * Idq.re;
            const double ed = Vdq.re - xp * Idq.im;
            const cplx E = cm(eq, -ed) * ejd;
            double* g = W + L.gen + kGen * kk;
            st(g + G_E, E);
            st(g + G_ED, ejd);
            g[G_EQ] = eq;
            g[G_EDD] = ed;
        }
        __syncthreads();
        // network currents at the equilibrium state: I = Y_red E' (the OPF injection up
        // to the OPF residual), and the dq currents and terminal voltage from them
        for (int kk = tid; kk < m; kk += kThreads) {
            double* g = W + L.gen + kGen * kk;
            cplx I = cm(0.0, 0.0);
            for (int ll = 0; ll < m; ++ll)
                I = I + ld(W + L.Z + 2 * (size_t)(kk * m + ll)) * ld(W + L.gen + kGen * ll + G_E);
            const cplx rot = mulj(conj(ld(g + G_ED)));
            const cplx Idq = I * rot;
            const cplx Vt = ld(g + G_E) - mulj(net.xp[gidx[kk]] * I);
            st(g + G_I, I);
            st(g + G_VT, Vt);
            g[G_VTM] = sqrt(abs2(Vt));
            g[G_ID] = Idq.re;
            g[G_IQ] = Idq.im;
        }
        __syncthreads();
        // ---- state matrix: one thread per 5x5 block (k, l) ----
        // (the front kernel keeps it per scenario for the FP64 refinement)
        double* A = (kMode == DYN_FRONT && a64) ? a64 + (size_t)s * a64stride : W + L.A;
        for (int w = tid; w < m * m; w += kThreads) {
            const int kk = w / m, ll = w % m;
            const int k = gidx[kk];
            const double* gk = W + L.gen + kGen * kk;
            const double* gl = W + L.gen + kGen * ll;
            const cplx Y = ld(W + L.Z + 2 * (size_t)(kk * m + ll));
            const cplx El = ld(gl + G_E), ejl = ld(gl + G_ED);
            const cplx dE[3] = {mulj(El), ejl, cm(0.0, -1.0) * ejl};   // d E'_l / d(delta, e'q, e'd)
            const cplx rotk = mulj(conj(ld(gk + G_ED)));
            const cplx Ik = ld(gk + G_I), Vt = ld(gk + G_VT);
            const double idk = gk[G_ID], iqk = gk[G_IQ], eqk = gk[G_EQ], edk = gk[G_EDD], Vtm = gk[G_VTM];
            const double xp = net.xp[k];
            double blk[5][5];
            for (int r = 0; r < 5; ++r)
                for (int c = 0; c < 5; ++c) blk[r][c] = 0.0;
            const int colmap[3] = {0, 2, 3};
            for (int th = 0; th < 3; ++th) {
                const cplx dI = Y * dE[th];
                cplx didq = rotk * dI;
                if (kk == ll && th == 0) didq = didq + cm(0.0, -1.0) * cplx{idk, iqk};
                double dPe = edk * didq.re + eqk * didq.im;
                if (kk == ll && th == 1) dPe += iqk;
                if (kk == ll && th == 2) dPe += idk;
                cplx dVt = cm(0.0, -xp) * dI;
                if (kk == ll) dVt = dVt + dE[th];
                const double dVm = (Vt.re * dVt.re + Vt.im * dVt.im) / Vtm;
                const int c = colmap[th];
                blk[1][c] = -dPe / net.H2[k];
                blk[2][c] = -(net.xd[k] - xp) * didq.re / net.Td0[k];
                blk[3][c] = (net.xq[k] - xp) * didq.im / net.Tq0[k];
                blk[4][c] = -net.KA[k] * dVm / net.TA[k];
            }
            // angle rows: d delta'_k/dt = ws (omega_k - omega_0) for k != 0 (row of delta_0 dropped)
            if (kk == ll && kk != 0) blk[0][1] = net.ws;
            if (ll == 0 && kk != 0) blk[0][1] = -net.ws;
            if (kk == ll) {
                blk[1][1] = -net.Dm[k] / net.H2[k];
                blk[2][2] += -1.0 / net.Td0[k];
                blk[2][4] = 1.0 / net.Td0[k];
                blk[3][3] += -1.0 / net.Tq0[k];
                blk[4][4] = -1.0 / net.TA[k];
            }
            // reduced indexing: full index 5k + s -> 5k + s - 1, the angle of machine 0 dropped
            for (int r = 0; r < 5; ++r) {
                if (kk == 0 && r == 0) continue;
                for (int c = 0; c < 5; ++c) {
                    if (ll == 0 && c == 0) continue;
                    A[(size_t)(5 * kk + r - 1) * n + 5 * ll + c - 1] = blk[r][c];
                }
            }
        }
        __syncthreads();
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (sh.fail) {                                // Y_bb singular: no model at this point
            if (tid == 0) {
                if (isl) {                            // the main island's class; the scenario's stays ISLANDED
                    if (a.out.main_klass) a.out.main_klass[s] = CS_EIG_FAIL;
                } else {
                    a.out.klass[s] = CS_EIG_FAIL;
                    a.out.severe[s] = 1;
                }
                a.out.max_re[s] = nan;
                a.out.min_zeta[s] = nan;
                if (kMode == DYN_FRONT || kMode == DYN_FRONT_LARGE) o.status[s] = 7;
            }
            __syncthreads();
            continue;
        }
        // ---- 4. eigenvalues: FP64, or an FP32 screen with an FP64 re-run in the guard band ----
        double* wr = W + L.wr;
        double* wi = W + L.wi;
        double maxre = 0.0, minz = 0.0;
        if (kMode == DYN_FRONT) {                     // balanced FP32 matrix for the cluster kernel
            float* dst = hbuf + (size_t)s * hstride;
            float* A32 = dst + kHqHead;
            for (int w = tid; w < n * n; w += kThreads) A32[w] = (float)A[w];
            if (tid == 0) dst[0] = __int_as_float(n);
            __syncthreads();
            balance<float>(A32, n, reinterpret_cast<float*>(cs_d), reinterpret_cast<float*>(rs_d), sh,
                           dst + ab_d_off(5 * ng - 1));
            __syncthreads();
            continue;
        }
        if (kMode == DYN_FRONT_LARGE) {               // balanced FP32 matrix, padded, for the tensor-core reduction
            float* A32 = reinterpret_cast<float*>(W + L.A32);
            for (int w = tid; w < n * n; w += kThreads) A32[w] = (float)A[w];
            __syncthreads();
            balance<float>(A32, n, reinterpret_cast<float*>(cs_d), reinterpret_cast<float*>(rs_d), sh);
            __syncthreads();
            float* slot = hbuf + (size_t)s * hstride;
            const int nmax = 5 * ng - 1;
            float* M = slot + kHqHead;
            for (int w = tid; w < nmax * nmax; w += kThreads) {
                const int i = w / nmax, j = w % nmax;
                M[w] = (i < n && j < n) ? A32[i * n + j] : (i == j ? -1.0f : 0.0f);
            }
            if (tid == 0) slot[0] = __int_as_float(n);
            __syncthreads();
            continue;
        }
        if (kMode == DYN_MIXED_INLINE) {
            float* A32 = reinterpret_cast<float*>(W + L.A32);
            for (int w = tid; w < n * n; w += kThreads) A32[w] = (float)A[w];
            __syncthreads();
            eigen_screen<float>(A32, n, reinterpret_cast<float*>(cs_d), reinterpret_cast<float*>(rs_d),
                                reinterpret_cast<float*>(v_d), wr, wi, sh);
            eig_stats(sh, n, wr, wi, maxre, minz);
            const bool near = sh.fail || !(fabs(maxre) > kGuardRe) || !(fabs(minz - damping_min) > kGuardZeta);
            if (near) {                               // decision too close to call in FP32
                if (tid == 0) {
                    sh.fail = 0;
                    atomicAdd(a.reruns, 1);
                }
                __syncthreads();
                eigen_screen<double>(A, n, cs_d, rs_d, v_d, wr, wi, sh);
                eig_stats(sh, n, wr, wi, maxre, minz);
            }
        } else {
            eigen_screen<double>(A, n, cs_d, rs_d, v_d, wr, wi, sh);
            eig_stats(sh, n, wr, wi, maxre, minz);
        }
        // ---- 5. class ----
        {
            if (tid == 0) {
                uint8_t k;
                if (sh.fail) k = CS_EIG_FAIL;
                else if (maxre >= 0.0) k = CS_SS_UNSTABLE;
                else if (minz < damping_min) k = CS_SS_POORLY_DAMPED;
                else k = CS_SECURE;
                if (isl) {
                    if (a.out.main_klass) a.out.main_klass[s] = k;
                } else {
                    a.out.klass[s] = k;
                    a.out.severe[s] = (k != CS_SECURE);
                }
                a.out.max_re[s] = sh.fail ? nan : maxre;
                a.out.min_zeta[s] = sh.fail ? nan : minz;
            }
            __syncthreads();
        }
    }
}

__global__ void record_kernel(int nbr, int nE, EvalArgs a) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += gridDim.x * blockDim.x) {
        const int ei = a.ei[s], ej = a.ej[s];
        if (ei < 0 || ei >= nE || ej >= nE || ej < -1) continue;
        if (a.ek && a.ek[s] >= 0 && a.ek[s] != ei && a.ek[s] != ej) continue;   // N-3: not in the N-2 tables
        const uint8_t S = a.out.severe[s] ? 1 : 0;
        if (ej < 0 || ej == ei) {
            a.sev_n1[ei] = S;
        } else {
            const long long i = min(ei, ej), j = max(ei, ej);
            const long long k = i * nE - (i * (i + 1)) / 2 + (j - i - 1);
            a.sev_pairs[k] = S;
        }
    }
}



// ---------------------------------------------------------------------------
// FP32 screen, middle part: Householder reduction to Hessenberg form of the
// balanced matrix, held on chip by a cluster of two CTAs (each keeps half of
// the rows in its shared memory; the 269 x 269 matrix of the 118-bus network
// is 289 KB, more than one CTA may hold).  Per column, each CTA writes its
// rows' part of the reflector and of the squared norm into both CTAs' shared
// memory (distributed shared memory), then the partial sums v^T A of the left
// update; two cluster barriers per column.  Exchange buffers alternate with the
// column parity, so a CTA that runs ahead never overwrites what its peer still
// reads.  The packed Hessenberg matrix goes to hbuf for hqr_smem_kernel.
constexpr int kHsThreads = 256;
constexpr int kHsWarps = kHsThreads / 32;
constexpr int kHsCols = 12;         // columns per lane in the row pass: orders up to 32 * 12 + 1

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kHsThreads, 1)
hess_cluster_kernel(EvalArgs a, OpfOut o, float* __restrict__ abuf, size_t astride, float* __restrict__ hbuf,
                    size_t hstride, int nmax, int* counter) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ float csm[];
    const int hmax = (nmax + 1) / 2;
    float* As = csm;                                  // own rows, row stride n
    float* vb = As + (size_t)hmax * nmax;             // [2 parity][nmax] raw column k (vb[.][0] = x0)
    float* wb = vb + 2 * nmax;                        // [2 parity][2 rank][nmax] partial v^T A
    float* np = wb + 4 * nmax;                        // [2 parity][2 rank] partial squared norms
    __shared__ float red[kHsWarps];
    __shared__ int scen;
    float* peer_vb = cl.map_shared_rank(vb, rank ^ 1);
    float* peer_wb = cl.map_shared_rank(wb, rank ^ 1);
    float* peer_np = cl.map_shared_rank(np, rank ^ 1);
    int* peer_scen = cl.map_shared_rank(&scen, rank ^ 1);

    for (;;) {
        if (rank == 0 && tid == 0) {
            const int s0 = atomicAdd(counter, 1);
            scen = s0;
            *peer_scen = s0;
        }
        cl.sync();
        const int s = scen;
        cl.sync();                                    // both have read scen
        if (s >= a.n) break;
        if (o.status[s] != 1) continue;
        float* src = abuf + (size_t)s * astride;
        const int n = __float_as_int(src[0]);
        const float* Ag = src + kHqHead;
        // Householder vectors and factors for the refinement kernel: rank 0 writes them
        // over the slot's matrix, after both CTAs have loaded their rows (the first
        // cluster barrier of column 0)
        float* refl = src + kHqHead;
        float* betas = src + ab_beta_off(nmax);
        const int h = (n + 1) / 2, r0 = rank * h, r1 = min(n, r0 + h), nr = max(0, r1 - r0);
        for (int w = tid; w < nr * n; w += kHsThreads) As[w] = Ag[(size_t)r0 * n + w];
        __syncthreads();
        for (int k = 0; k + 2 < n; ++k) {
            const int par = k & 1;
            float* v = vb + par * nmax;
            float* pv = peer_vb + par * nmax;
            const int i0 = max(r0, k + 1);
            float t = 0.0f;
            for (int i = i0 + tid; i < r1; i += kHsThreads) {
                const float q = As[(i - r0) * n + k];
                v[i - k - 1] = q;
                pv[i - k - 1] = q;
                if (i >= k + 2) t += q * q;
            }
            for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) red[warp] = t;
            __syncthreads();
            if (tid == 0) {
                float tt = 0.0f;
                for (int q = 0; q < kHsWarps; ++q) tt += red[q];
                np[par * 2 + rank] = tt;
                peer_np[par * 2 + rank] = tt;
            }
            cl.sync();                                // reflector and norm partials in place
            const float tail = np[par * 2] + np[par * 2 + 1];
            if (tail == 0.0f) {                       // column already reduced (same in both CTAs)
                if (rank == 0 && tid == 0) betas[k] = 0.0f;
                continue;
            }
            const float x0 = v[0];
            const float nrm = sqrtf(x0 * x0 + tail);
            const float alpha = (x0 >= 0.0f) ? -nrm : nrm;
            const float v0 = x0 - alpha;
            const float beta = 2.0f / (v0 * v0 + tail);
            // this CTA's copy of the reflector takes v0 in place of x0 (the peer writes only the
            // other parity's copy during this column)
            __syncthreads();
            if (tid == 0) v[0] = v0;
            __syncthreads();
            if (rank == 0) {
                float* rk = refl + refl_off(n, k);
                for (int i = tid; i < n - k - 1; i += kHsThreads) rk[i] = v[i];
                if (tid == 0) betas[k] = beta;
            }
            float* w_own = wb + (par * 2 + rank) * nmax;
            float* w_peer = peer_wb + (par * 2 + rank) * nmax;
            for (int j = k + 1 + tid; j < n; j += kHsThreads) {   // partial v^T A over own rows
                float acc = 0.0f;
                const float* col = As + (i0 - r0) * n + j;
                const float* vv = v + (i0 - k - 1);
                for (int i = 0; i < r1 - i0; ++i) acc += vv[i] * col[i * n];
                w_own[j] = acc;
                w_peer[j] = acc;
            }
            cl.sync();                                // partial sums exchanged
            // One pass per own row, a warp per row: the left update (rows k+1..),
            // column k, then the right update, with the row held in registers.  Each
            // lane keeps w and v for its columns k+1+lane+32t in registers.
            const float* w0 = wb + (par * 2) * nmax;
            const float* w1 = wb + (par * 2 + 1) * nmax;
            const int mm = n - k - 1;
            float wr_[kHsCols], vr_[kHsCols];
#pragma unroll
            for (int t = 0; t < kHsCols; ++t) {
                const int jj = lane + 32 * t;             // offset from column k+1
                wr_[t] = (jj < mm) ? beta * (w0[k + 1 + jj] + w1[k + 1 + jj]) : 0.0f;
                vr_[t] = (jj < mm) ? v[jj] : 0.0f;
            }
            for (int i = warp; i < nr; i += kHsWarps) {
                float* row = As + i * n + k + 1;
                const int gi = r0 + i;
                const float vi = (gi >= k + 1) ? v[gi - k - 1] : 0.0f;
                float x[kHsCols];
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < kHsCols; ++t) {
                    const int jj = lane + 32 * t;
                    x[t] = (jj < mm) ? row[jj] - vi * wr_[t] : 0.0f;
                    acc += x[t] * vr_[t];
                }
                for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                acc *= beta;
#pragma unroll
                for (int t = 0; t < kHsCols; ++t) {
                    const int jj = lane + 32 * t;
                    if (jj < mm) row[jj] = x[t] - acc * vr_[t];
                }
                if (lane == 0 && gi >= k + 1) row[-1] = (gi == k + 1) ? alpha : 0.0f;
            }
            __syncthreads();
        }
        float* dst = hbuf + (size_t)s * hstride;      // packed rows for the shared-memory QR
        if (rank == 0 && tid == 0) dst[0] = __int_as_float(n);
        for (int i = r0 + warp; i < r1; i += kHsWarps) {
            const int j0 = hq_start(i);
            float* drow = dst + kHqHead + hq_off(n, i) - j0;
            for (int j = j0 + lane; j < n; j += 32) drow[j] = As[(i - r0) * n + j];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP32 screen, last part: Francis double-shift QR of the packed Hessenberg
// matrix held in shared memory (one scenario per CTA, one CTA per SM).  Every
// thread carries the same loop state (lo, hi, shifts, reflector), computed
// redundantly from shared memory in FP32, so a bulge step costs two barriers.
// Exceptional shifts come every tenth sweep without a deflation, and a stalled
// window also deflates at the normwise FP32 level (kStallIts).  A scenario whose
// QR does not converge is marked for the FP64 re-run; the others get their
// refinement candidates and go on to eig_refine_kernel, which classifies them.
#ifndef CS_QR_THREADS
#define CS_QR_THREADS 256
#endif
constexpr int kQrThreads = CS_QR_THREADS;
// FP32 QR without a deflation for this many sweeps (the double-shift iteration can
// stall at FP32 rounding level): from then on a subdiagonal entry below eps_32 times
// the largest entry of the matrix counts as negligible too.  The screen's eigenvalues
// only need to be within kEigDelta of the exact ones (the decisive ones are refined in
// FP64), which that normwise perturbation respects.
constexpr int kStallIts = 40;
// the column phase of a bulge step covers at most 2 kQrThreads rows (orders up to 32 kHsCols + 1)
static_assert(2 * kQrThreads > 32 * kHsCols + 1, "QR column phase: at most two rows per thread");

__device__ __forceinline__ void eig2f(float p, float q, float r, float s, float* re, float* im) {
    const float hm = 0.5f * (p - s);
    const float disc = hm * hm + q * r;
    const float mean = 0.5f * (p + s);
    if (disc >= 0.0f) {
        const float root = sqrtf(disc);
        const float big = mean + (hm >= 0.0f ? root : -root);
        const float det = p * s - q * r;
        const float other = (big != 0.0f) ? det / big : mean - (hm >= 0.0f ? root : -root);
        re[0] = big; im[0] = 0.0f;
        re[1] = other; im[1] = 0.0f;
    } else {
        const float root = sqrtf(-disc);
        re[0] = mean; im[0] = root;
        re[1] = mean; im[1] = -root;
    }
}

__global__ void __launch_bounds__(kQrThreads, 1)
hqr_smem_kernel(EvalArgs a, OpfOut o, const float* __restrict__ hbuf, size_t hstride, int nmax,
                double damping_min, float* __restrict__ cand, int* counter) {
    extern __shared__ float qsm[];
    __shared__ float red[2][kQrThreads / 32];
    __shared__ float xs[2][3];
    __shared__ int scen;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* H = qsm;                                           // hq_off(nmax, nmax) floats
    int* rb = reinterpret_cast<int*>(qsm + ((hq_off(nmax, nmax) + 3) & ~3));   // row i at H[rb[i] + j]
    float* wr = reinterpret_cast<float*>(rb + nmax);
    float* wi = wr + nmax;
    const float eps = 1.1920928955078125e-07f;

    for (;;) {
        if (tid == 0) scen = atomicAdd(counter, 1);
        __syncthreads();
        const int s = scen;
        if (s >= a.n) break;
        if (o.status[s] != 1) {
            __syncthreads();
            continue;
        }
        const float* src = hbuf + (size_t)s * hstride;
        const int n = __float_as_int(src[0]);
        const int hs = hq_off(n, n);
        {
            const float4* s4 = reinterpret_cast<const float4*>(src + kHqHead);
            float4* d4 = reinterpret_cast<float4*>(H);
            for (int w = tid; w < (hs >> 2); w += kQrThreads) d4[w] = s4[w];
            for (int w = (hs & ~3) + tid; w < hs; w += kQrThreads) H[w] = src[kHqHead + w];
        }
        for (int i = tid; i < n; i += kQrThreads) rb[i] = hq_off(n, i) - hq_start(i);
        __syncthreads();
        float hmax;
        {
            float hm = 0.0f;
            for (int w = tid; w < hs; w += kQrThreads) hm = fmaxf(hm, fabsf(H[w]));
            for (int off = 16; off; off >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, off));
            if (lane == 0) red[0][warp] = hm;
            __syncthreads();
            hmax = red[0][0];
            for (int w = 1; w < kQrThreads / 32; ++w) hmax = fmaxf(hmax, red[0][w]);
        }
        int hi = n - 1, its = 0;
        bool fail = false;
        while (hi >= 0) {
            // top of the unreduced block ending at hi (every warp scans; all agree)
            int lo = 0;
            for (int base = hi; base >= 1; base -= 32) {
                const int l = base - lane;
                bool neg = false;
                if (l >= 1) {
                    float sd = fabsf(H[rb[l - 1] + l - 1]) + fabsf(H[rb[l] + l]);
                    if (sd == 0.0f) sd = hmax;
                    const float h = fabsf(H[rb[l] + l - 1]);
                    // after kStallIts sweeps without a deflation, a subdiagonal entry at FP32
                    // rounding level of the whole matrix also counts as negligible
                    neg = h <= kDeflTol * sd || (its >= kStallIts && h <= eps * hmax);
                }
                const unsigned m = __ballot_sync(0xffffffffu, neg);
                if (m) {
                    lo = base - (__ffs(m) - 1);
                    break;
                }
            }
            if (lo == hi) {
                if (tid == 0) {
                    wr[hi] = H[rb[hi] + hi];
                    wi[hi] = 0.0f;
                }
                hi -= 1;
                its = 0;
                continue;
            }
            if (lo == hi - 1) {
                if (tid == 0) {
                    float re[2], im[2];
                    eig2f(H[rb[hi - 1] + hi - 1], H[rb[hi - 1] + hi], H[rb[hi] + hi - 1], H[rb[hi] + hi], re, im);
                    wr[hi - 1] = re[0]; wi[hi - 1] = im[0];
                    wr[hi] = re[1]; wi[hi] = im[1];
                }
                hi -= 2;
                its = 0;
                continue;
            }
            if (its >= 30 * n) {
                fail = true;
                break;
            }
            ++its;
            float sft, tft;
            {
                const float a11 = H[rb[hi - 1] + hi - 1], a12 = H[rb[hi - 1] + hi];
                const float a21 = H[rb[hi] + hi - 1], a22 = H[rb[hi] + hi];
                if (its % 10 == 0) {                       // exceptional shift, every tenth sweep
                    const float ww = fabsf(a21) + fabsf(H[rb[hi - 1] + hi - 2]);
                    sft = 1.5f * ww;
                    tft = ww * ww;
                } else {
                    sft = a11 + a22;
                    tft = a11 * a22 - a12 * a21;
                }
            }
            float x0, x1, x2;
            {
                const float h00 = H[rb[lo] + lo], h01 = H[rb[lo] + lo + 1];
                const float h10 = H[rb[lo + 1] + lo], h11 = H[rb[lo + 1] + lo + 1];
                const float h21 = H[rb[lo + 2] + lo + 1];
                x0 = h00 * h00 + h01 * h10 - sft * h00 + tft;
                x1 = h10 * (h00 + h11 - sft);
                x2 = h10 * h21;
            }
            __syncthreads();              // every warp has read the block and the shifts before the sweep writes
            // rows this thread updates in the column phase (fixed for the sweep; the order is
            // at most 2 * kQrThreads on this path), and their packed offsets
            const int rbi0 = (lo + tid <= hi) ? rb[lo + tid] : 0;
            const int rbi1 = (lo + tid + kQrThreads <= hi) ? rb[lo + tid + kQrThreads] : 0;
            for (int k = lo; k <= hi - 1; ++k) {
                const int len = (k + 2 <= hi) ? 3 : 2;
                const float t2 = x1 * x1 + (len == 3 ? x2 * x2 : 0.0f);
                const bool more = (k + 1 <= hi - 1);
                if (t2 != 0.0f) {
                    const float nrm = sqrtf(x0 * x0 + t2);
                    const float al = (x0 >= 0.0f) ? -nrm : nrm;
                    const float u0 = x0 - al, u1 = x1, u2 = (len == 3) ? x2 : 0.0f;
                    const float bt = 2.0f / (u0 * u0 + t2);
                    const int c0 = (k > lo) ? k - 1 : lo;
                    const int b0 = rb[k], b1 = rb[k + 1], b2 = (len == 3) ? rb[k + 2] : 0;
                    for (int j = c0 + tid; j <= hi; j += kQrThreads) {     // rows k..k+len-1
                        const float p0 = H[b0 + j], p1 = H[b1 + j];
                        const float p2 = (len == 3) ? H[b2 + j] : 0.0f;
                        const float d = (u0 * p0 + u1 * p1 + u2 * p2) * bt;
                        H[b0 + j] = p0 - d * u0;
                        H[b1 + j] = p1 - d * u1;
                        if (len == 3) H[b2 + j] = p2 - d * u2;
                    }
                    __syncthreads();
                    const int r1 = (k + 3 < hi) ? k + 3 : hi;
                    for (int i = lo + tid, m = 0; i <= r1; i += kQrThreads, ++m) {   // columns k..k+len-1
                        float* p = H + (m == 0 ? rbi0 : rbi1) + k;
                        const float q0 = p[0], q1 = p[1];
                        const float q2 = (len == 3) ? p[2] : 0.0f;
                        const float d = (q0 * u0 + q1 * u1 + q2 * u2) * bt;
                        const float n0 = q0 - d * u0;
                        p[0] = n0;
                        p[1] = q1 - d * u1;
                        if (len == 3) p[2] = q2 - d * u2;
                        if (i > k && i <= k + 3) xs[k & 1][i - k - 1] = n0;     // next bulge column
                    }
                    __syncthreads();
                    if (more) {
                        x0 = xs[k & 1][0];
                        x1 = xs[k & 1][1];
                        x2 = (k + 3 <= hi) ? xs[k & 1][2] : 0.0f;
                    }
                } else if (more) {
                    x0 = H[rb[k + 1] + k];
                    x1 = H[rb[k + 2] + k];
                    x2 = (k + 3 <= hi) ? H[rb[k + 3] + k] : 0.0f;
                    __syncthreads();                       // all read before the next step writes column k
                }
            }
            for (int i = lo + 2 + tid; i <= hi; i += kQrThreads) {
                H[rb[i] + i - 2] = 0.0f;
                if (i >= lo + 3) H[rb[i] + i - 3] = 0.0f;
            }
            __syncthreads();
        }
        __syncthreads();                                   // wr, wi written by thread 0
        // statistics over all eigenvalues: max Re, min damping ratio
        float mr = -INFINITY, mz = INFINITY;
        if (!fail) {
            for (int i = tid; i < n; i += kQrThreads) {
                mr = fmaxf(mr, wr[i]);
                const float mg = sqrtf(wr[i] * wr[i] + wi[i] * wi[i]);
                mz = fminf(mz, mg > 0.0f ? -wr[i] / mg : 1.0f);
            }
        }
        for (int off = 16; off; off >>= 1) {
            mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, off));
            mz = fminf(mz, __shfl_xor_sync(0xffffffffu, mz, off));
        }
        if (lane == 0) {
            red[0][warp] = mr;
            red[1][warp] = mz;
        }
        __syncthreads();
        if (tid == 0) {
            float maxre = red[0][0], minz = red[1][0];
            for (int w = 1; w < kQrThreads / 32; ++w) {
                maxre = fmaxf(maxre, red[0][w]);
                minz = fminf(minz, red[1][w]);
            }
            // The class is decided after the FP64 refinement (eig_refine_kernel), from
            // values within ~1e-9 of the FP64 screen's, so no FP32 guard band applies here;
            // a QR that did not converge goes to the FP64 screen.
            if (fail) {
                o.status[s] = 6;
                atomicAdd(a.reruns, 1);
            } else {
                // Candidates of the FP64 refinement, in index order: every eigenvalue
                // (im >= 0 of a pair) whose exact value may carry the largest real part
                // or the smallest damping ratio, given |FP32 - exact| <= kEigDelta.
                // Damping ratio of lambda with |delta lambda| <= d moves by at most 2 d / |lambda|.
                float zu = INFINITY;
                for (int i = 0; i < n; ++i) {
                    if (wi[i] < 0.0f) continue;
                    const float mg = sqrtf(wr[i] * wr[i] + wi[i] * wi[i]);
                    const float z = mg > 0.0f ? -wr[i] / mg : 1.0f;
                    zu = fminf(zu, mg > 0.0f ? z + 2.0f * kEigDelta / mg : INFINITY);
                }
                float* cs = cand + (size_t)s * kCandStride;
                int cnt = 0, flags = 0;
                for (int i = 0; i < n; ++i) {
                    if (wi[i] < 0.0f) continue;
                    const float mg = sqrtf(wr[i] * wr[i] + wi[i] * wi[i]);
                    const float z = mg > 0.0f ? -wr[i] / mg : 1.0f;
                    const bool cre = wr[i] >= maxre - 2.0f * kEigDelta;
                    const bool cz = !(mg > 0.0f) || z - 2.0f * kEigDelta / mg <= zu;
                    if (!cre && !cz) continue;
                    if (cnt < kRefK) {
                        cs[4 + 2 * cnt] = wr[i];
                        cs[5 + 2 * cnt] = wi[i];
                        flags |= (cre ? 1 : 0) << (2 * cnt);
                        flags |= (cz ? 2 : 0) << (2 * cnt);
                    }
                    ++cnt;
                }
                if (cnt > kRefK) {                         // too many to refine: FP64 screen
                    o.status[s] = 6;
                    atomicAdd(a.reruns, 1);
                } else {
                    cs[0] = __int_as_float(cnt);
                    cs[1] = __int_as_float(flags);
                    o.status[s] = 8;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64 refinement of the FP32 screen's decisive eigenvalues.  For each candidate
// (an FP32 eigenvalue sigma that may carry max Re or min zeta), one warp computes
// the right and another the left eigenvector of the packed FP32 Hessenberg matrix
// H by two passes of inverse iteration with shift sigma, and takes each back to
// the balanced matrix through the Householder vectors of the cluster kernel.  The
// eigenvalue is then the two-sided Rayleigh quotient w^H A v / w^H v with the
// scenario's FP64 state matrix A (v, w scaled by the balancing factors), whose
// error is second order in the vectors' FP32 error.  The statistics over the
// refined candidates decide the class.  A candidate whose quotient is
// ill-conditioned or lands away from sigma sends the scenario to the FP64 screen.
//
// Inverse iteration on an upper Hessenberg G - sigma I, one warp: Gaussian
// elimination with partial pivoting between each carried row and the next row of
// G (the only one with an entry below the diagonal), U^{-X} b (X = H or T) formed
// row by row as U's rows appear, so U is never stored; the row operations E_k
// (swap flag and multiplier) are kept and applied as E_0^X ... E_{n-2}^X at the
// end.  The left vector solves (H - sigma I)^H z = b with G = H; the right one
// solves (H - sigma I) x = b as (G - sigma I)^T (J x) = J b with G = J H^T J
// (J reverses the order), which is upper Hessenberg again.
constexpr int kRfThreads = 256;
constexpr int kRfWarps = kRfThreads / 32;
static_assert(2 * kRefK <= kRfWarps, "one warp per eigenvector");

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cconj2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cdiv2(float2 a, float2 b) {
    const float sc = fmaxf(fabsf(b.x), fabsf(b.y));
    const float bx = b.x / sc, by = b.y / sc;
    const float d = (bx * bx + by * by) * sc;
    return make_float2((a.x * bx + a.y * by) / d, (a.y * bx - a.x * by) / d);
}

template <bool kRight>
__device__ __forceinline__ float hess_g(const float* Hs, const int* rb, int n, int i, int j) {
    return kRight ? Hs[rb[n - 1 - j] + n - 1 - i] : Hs[rb[i] + j];
}

// y <- (G - sig I)^{-X} y (X = H for the left vector, T for the right one), one warp.
template <bool kRight>
__device__ void hess_inverse_pass(const float* Hs, const int* rb, int n, float2 sig, float tiny, float2* y, float2* c,
                                  float2* mul, unsigned* swp, int lane) {
    const bool cj = !kRight;
    for (int j = lane; j < n; j += 32)
        c[j] = make_float2(hess_g<kRight>(Hs, rb, n, 0, j) - (j == 0 ? sig.x : 0.0f), j == 0 ? -sig.y : 0.0f);
    for (int w = lane; w < (n + 31) / 32; w += 32) swp[w] = 0u;
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const bool last = (k == n - 1);
        const float2 ck = c[k];
        const float2 bk = y[k];
        const float rk = last ? 0.0f : hess_g<kRight>(Hs, rb, n, k + 1, k);
        const bool sw = !last && fabsf(rk) > fabsf(ck.x) + fabsf(ck.y);
        float2 pk = sw ? make_float2(rk, 0.0f) : ck;
        if (pk.x == 0.0f && pk.y == 0.0f) pk.x = tiny;             // exactly singular: perturb the pivot
        const float2 ok = sw ? ck : make_float2(rk, 0.0f);
        const float2 mk = last ? make_float2(0.0f, 0.0f) : cdiv2(ok, pk);
        const float2 yk = cdiv2(bk, cj ? cconj2(pk) : pk);
        __syncwarp();                                               // every lane has read c[k], y[k]
        for (int j = k + 1 + lane; j < n; j += 32) {
            float2 rj = make_float2(hess_g<kRight>(Hs, rb, n, k + 1, j), 0.0f);
            if (j == k + 1) {
                rj.x -= sig.x;
                rj.y -= sig.y;
            }
            const float2 cv = c[j];
            const float2 pj = sw ? rj : cv, oj = sw ? cv : rj;
            const float2 t = cmul2(cj ? cconj2(pj) : pj, yk);
            y[j] = make_float2(y[j].x - t.x, y[j].y - t.y);
            const float2 u = cmul2(mk, pj);
            c[j] = make_float2(oj.x - u.x, oj.y - u.y);
        }
        if (lane == 0) {
            y[k] = yk;
            mul[k] = mk;
            if (sw) swp[k >> 5] |= 1u << (k & 31);
        }
        __syncwarp();
    }
    if (lane == 0) {
        for (int k = n - 2; k >= 0; --k) {
            const float2 t = cmul2(cj ? cconj2(mul[k]) : mul[k], y[k + 1]);
            y[k] = make_float2(y[k].x - t.x, y[k].y - t.y);
            if ((swp[k >> 5] >> (k & 31)) & 1u) {
                const float2 q = y[k];
                y[k] = y[k + 1];
                y[k + 1] = q;
            }
        }
    }
    __syncwarp();
}

// scale y to a largest component of modulus 1; false if it has none (zero or not finite)
__device__ bool warp_normalise(float2* y, int n, int lane) {
    float mx = 0.0f;
    for (int j = lane; j < n; j += 32) mx = fmaxf(mx, fmaxf(fabsf(y[j].x), fabsf(y[j].y)));
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (!(mx > 0.0f) || !isfinite(mx)) return false;
    const float inv = 1.0f / mx;
    for (int j = lane; j < n; j += 32) y[j] = make_float2(y[j].x * inv, y[j].y * inv);
    __syncwarp();
    return true;
}

struct RfShared {
    int scen, cnt, flags;
    float tiny;
    int bad[2 * kRefK];
    float hred[kRfWarps];
    double acc[kRfWarps][kRefK][6];   // per warp: num (re, im), den (re, im), |v|^2, |w|^2
};

__global__ void __launch_bounds__(kRfThreads, 1)
eig_refine_kernel(EvalArgs a, OpfOut o, const float* __restrict__ hbuf, size_t hstride, const float* __restrict__ abuf,
                  size_t astride, const double* __restrict__ a64, size_t a64stride, const float* __restrict__ cand,
                  int nmax, double damping_min, int* counter) {
    extern __shared__ float4 rsm4[];
    float* rsm = reinterpret_cast<float*>(rsm4);
    __shared__ RfShared sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t hsz = ((size_t)hq_off(nmax, nmax) + 3) & ~(size_t)3;
    const size_t vsz = (size_t)4 * kRefK * nmax * 2;                 // FP64 vectors (doubles as float pairs)
    float* Hs = rsm;                                                  // packed H, later the FP64 vectors
    double2* vA = reinterpret_cast<double2*>(rsm);                    // [kRefK][nmax]
    double2* wA = vA + (size_t)kRefK * nmax;                          // [kRefK][nmax]
    int* rb = reinterpret_cast<int*>(rsm + (hsz > vsz ? hsz : vsz));
    float2* wk = reinterpret_cast<float2*>(rb + ((nmax + 3) & ~3));   // per warp: c, mul [nmax] each
    float2* vec = wk + (size_t)kRfWarps * 2 * nmax;                   // [2 kRefK][nmax] vectors
    unsigned* swp = reinterpret_cast<unsigned*>(vec + (size_t)2 * kRefK * nmax);   // per warp: bits
    const int swords = (nmax + 31) / 32;

    for (;;) {
        if (tid == 0) sh.scen = atomicAdd(counter, 1);
        __syncthreads();
        const int s = sh.scen;
        if (s >= a.n) break;
        if (o.status[s] != 8) {
            __syncthreads();
            continue;
        }
        const float* src = hbuf + (size_t)s * hstride;
        const int n = __float_as_int(src[0]);
        const int hs = hq_off(n, n);
        const float* slot = abuf + (size_t)s * astride;
        const float* cs = cand + (size_t)s * kCandStride;
        {
            const float4* s4 = reinterpret_cast<const float4*>(src + kHqHead);
            float4* d4 = reinterpret_cast<float4*>(Hs);
            for (int w = tid; w < (hs >> 2); w += kRfThreads) d4[w] = s4[w];
            for (int w = (hs & ~3) + tid; w < hs; w += kRfThreads) Hs[w] = src[kHqHead + w];
        }
        for (int i = tid; i < n; i += kRfThreads) rb[i] = hq_off(n, i) - hq_start(i);
        if (tid == 0) {
            sh.cnt = __float_as_int(cs[0]);
            sh.flags = __float_as_int(cs[1]);
        }
        if (tid < 2 * kRefK) sh.bad[tid] = 0;
        __syncthreads();
        {
            float hm = 0.0f;
            for (int w = tid; w < hs; w += kRfThreads) hm = fmaxf(hm, fabsf(Hs[w]));
            for (int off = 16; off; off >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, off));
            if (lane == 0) sh.hred[warp] = hm;
            __syncthreads();
            if (tid == 0) {
                float m = sh.hred[0];
                for (int w = 1; w < kRfWarps; ++w) m = fmaxf(m, sh.hred[w]);
                sh.tiny = 1.1920928955078125e-07f * (m > 0.0f ? m : 1.0f);
            }
            __syncthreads();
        }
        const int cnt = sh.cnt;
        // ---- eigenvectors of H, one warp each: task 2c = right vector of candidate c, 2c+1 = left ----
        if (warp < 2 * cnt) {
            const int c = warp >> 1;
            const bool right = (warp & 1) == 0;
            const float2 sig = make_float2(cs[4 + 2 * c], cs[5 + 2 * c]);
            float2* y = vec + (size_t)warp * nmax;
            float2* cw = wk + (size_t)warp * 2 * nmax;
            float2* mw = cw + nmax;
            unsigned* sb = swp + warp * swords;
            for (int j = lane; j < n; j += 32) y[j] = make_float2(1.0f, 0.0f);
            __syncwarp();
            bool ok = true;
            for (int pass = 0; pass < 2 && ok; ++pass) {
                if (right) hess_inverse_pass<true>(Hs, rb, n, sig, sh.tiny, y, cw, mw, sb, lane);
                else hess_inverse_pass<false>(Hs, rb, n, sig, sh.tiny, y, cw, mw, sb, lane);
                ok = warp_normalise(y, n, lane);
            }
            if (ok && right) {                                   // J x -> x
                for (int j = lane; j < n / 2; j += 32) {
                    const float2 q = y[j];
                    y[j] = y[n - 1 - j];
                    y[n - 1 - j] = q;
                }
                __syncwarp();
            }
            if (ok) {                                            // Q x: reflectors n-3 .. 0
                const float* betas = slot + ab_beta_off(nmax);
                for (int k = n - 3; k >= 0; --k) {
                    const float bt = betas[k];
                    if (bt == 0.0f) continue;
                    const float* u = slot + kHqHead + refl_off(n, k);
                    const int mm = n - k - 1;
                    float sr = 0.0f, si = 0.0f;
                    for (int i = lane; i < mm; i += 32) {
                        const float2 q = y[k + 1 + i];
                        sr += u[i] * q.x;
                        si += u[i] * q.y;
                    }
                    for (int off = 16; off; off >>= 1) {
                        sr += __shfl_xor_sync(0xffffffffu, sr, off);
                        si += __shfl_xor_sync(0xffffffffu, si, off);
                    }
                    sr *= bt;
                    si *= bt;
                    for (int i = lane; i < mm; i += 32) {
                        const float2 q = y[k + 1 + i];
                        y[k + 1 + i] = make_float2(q.x - sr * u[i], q.y - si * u[i]);
                    }
                    __syncwarp();
                }
                ok = warp_normalise(y, n, lane);
            }
            if (lane == 0 && !ok) sh.bad[warp] = 1;
        }
        __syncthreads();
        // ---- FP64: v_A = D v_B, w_A = D^-1 w_B; two-sided Rayleigh quotient with A ----
        const float* D = slot + ab_d_off(nmax);
        for (int w = tid; w < cnt * n; w += kRfThreads) {
            const int c = w / n, j = w % n;
            const double d = (double)D[j];
            const float2 v = vec[(size_t)(2 * c) * nmax + j], u = vec[(size_t)(2 * c + 1) * nmax + j];
            vA[(size_t)c * nmax + j] = make_double2(d * v.x, d * v.y);
            wA[(size_t)c * nmax + j] = make_double2(u.x / d, u.y / d);
        }
        __syncthreads();
        {
            double acc[kRefK][6];
#pragma unroll
            for (int c = 0; c < kRefK; ++c)
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[c][q] = 0.0;
            const double* A = a64 + (size_t)s * a64stride;
            for (int i = warp; i < n; i += kRfWarps) {
                const double* Ar = A + (size_t)i * n;
                double pr[kRefK], pi[kRefK];
#pragma unroll
                for (int c = 0; c < kRefK; ++c) pr[c] = pi[c] = 0.0;
                for (int j = lane; j < n; j += 32) {
                    const double aij = Ar[j];
#pragma unroll
                    for (int c = 0; c < kRefK; ++c) {
                        if (c < cnt) {
                            const double2 v = vA[(size_t)c * nmax + j];
                            pr[c] = fma(aij, v.x, pr[c]);
                            pi[c] = fma(aij, v.y, pi[c]);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < kRefK; ++c) {
                    if (c >= cnt) continue;
                    for (int off = 16; off; off >>= 1) {
                        pr[c] += __shfl_xor_sync(0xffffffffu, pr[c], off);
                        pi[c] += __shfl_xor_sync(0xffffffffu, pi[c], off);
                    }
                    const double2 w = wA[(size_t)c * nmax + i], v = vA[(size_t)c * nmax + i];
                    // conj(w_i) (A v)_i and conj(w_i) v_i
                    acc[c][0] += w.x * pr[c] + w.y * pi[c];
                    acc[c][1] += w.x * pi[c] - w.y * pr[c];
                    acc[c][2] += w.x * v.x + w.y * v.y;
                    acc[c][3] += w.x * v.y - w.y * v.x;
                    acc[c][4] += v.x * v.x + v.y * v.y;
                    acc[c][5] += w.x * w.x + w.y * w.y;
                }
            }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < kRefK; ++c)
#pragma unroll
                    for (int q = 0; q < 6; ++q) sh.acc[warp][c][q] = acc[c][q];
        }
        __syncthreads();
        if (tid == 0) {
            bool good = true;
            double maxre = -INFINITY, minz = INFINITY;
            for (int c = 0; c < cnt; ++c) {
                double t[6] = {0, 0, 0, 0, 0, 0};
                for (int w = 0; w < kRfWarps; ++w)
                    for (int q = 0; q < 6; ++q) t[q] += sh.acc[w][c][q];
                const cplx lam = cdiv(cm(t[0], t[1]), cm(t[2], t[3]));
                const double sx = cs[4 + 2 * c], sy = cs[5 + 2 * c];
                const bool ok = !sh.bad[2 * c] && !sh.bad[2 * c + 1] && isfinite(lam.re) && isfinite(lam.im) &&
                                t[2] * t[2] + t[3] * t[3] >= 1e-10 * t[4] * t[5] &&
                                fabs(lam.re - sx) <= 2.0 * kEigDelta && fabs(fabs(lam.im) - sy) <= 2.0 * kEigDelta;
                if (!ok) {
                    good = false;
                    break;
                }
                const double mg = sqrt(lam.re * lam.re + lam.im * lam.im);
                if ((sh.flags >> (2 * c)) & 1) maxre = fmax(maxre, lam.re);
                if ((sh.flags >> (2 * c)) & 2) minz = fmin(minz, mg > 0.0 ? -lam.re / mg : 1.0);
            }
            if (!good || !(maxre > -INFINITY) || !(minz < INFINITY) || !(fabs(maxre) > kRefinedGuard) ||
                !(fabs(minz - damping_min) > kRefinedGuard)) {
                o.status[s] = 6;                                // FP64 screen instead
                atomicAdd(a.reruns, 1);
            } else {
                uint8_t k;
                if (maxre >= 0.0) k = CS_SS_UNSTABLE;
                else if (minz < damping_min) k = CS_SS_POORLY_DAMPED;
                else k = CS_SECURE;
                if (a.out.n_islands[s] > 1) {                   // main island: the scenario's class stays ISLANDED
                    if (a.out.main_klass) a.out.main_klass[s] = k;
                } else {
                    a.out.klass[s] = k;
                    a.out.severe[s] = (k != CS_SECURE);
                }
                a.out.max_re[s] = maxre;
                a.out.min_zeta[s] = minz;
                o.status[s] = 1;
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t dyn_scratch_doubles(const DevNet& net) { return (size_t)make_dlayout(net).total; }

size_t dyn_hbuf_stride(const DevNet& net) {
    const int nmax = 5 * net.ng - 1;
    return (size_t)kHqHead + (size_t)((hq_off(nmax, nmax) + 3) & ~3);
}

size_t dyn_abuf_stride(const DevNet& net) { return ab_stride(5 * net.ng - 1); }

size_t dyn_a64_stride(const DevNet& net) {
    const size_t nmax = 5 * (size_t)net.ng - 1;
    return nmax * nmax;
}

size_t dyn_cand_stride() { return kCandStride; }

static size_t qr_smem_bytes(int nmax) {
    return sizeof(float) * ((size_t)((hq_off(nmax, nmax) + 3) & ~3) + 3 * (size_t)nmax);
}

static size_t refine_smem_bytes(int nmax) {
    const size_t hsz = ((size_t)hq_off(nmax, nmax) + 3) & ~(size_t)3;
    const size_t vsz = (size_t)8 * kRefK * nmax;
    return sizeof(float) * (std::max(hsz, vsz) + (((size_t)nmax + 3) & ~(size_t)3) + (size_t)kRfWarps * 4 * nmax +
                            (size_t)4 * kRefK * nmax + (size_t)kRfWarps * ((nmax + 31) / 32));
}

static size_t hess_smem_bytes(int nmax) {
    return sizeof(float) * ((size_t)((nmax + 1) / 2) * nmax + 6 * (size_t)nmax + 4);
}

bool dyn_split_fits(const DevNet& net, int device) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return false;
    const int nmax = 5 * net.ng - 1;
    if (nmax - 1 > 32 * kHsCols) return false;
    return qr_smem_bytes(nmax) + 1024 <= (size_t)optin && hess_smem_bytes(nmax) + 1024 <= (size_t)optin &&
           refine_smem_bytes(nmax) + sizeof(RfShared) + 1024 <= (size_t)optin;
}

template <int kMode>
static cudaError_t launch_mode(const DevNet& net, const EvalArgs& a, OpfOut o, double damping_min, double* scratch,
                               size_t per_cta, const DLay& L, float* hbuf, size_t hstride, double* a64, int grid,
                               int* counter, cudaStream_t s) {
    const size_t smem = sizeof(double) * ((size_t)((net.ng + 1) >> 1) + 15 * (size_t)net.ng);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(dyn_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dyn_kernel<kMode><<<grid, kThreads, smem, s>>>(net, a, o, damping_min, scratch, per_cta, L, hbuf, hstride, a64,
                                                   dyn_a64_stride(net), counter);
    return cudaGetLastError();
}

cudaError_t launch_dyn(const DevNet& net, const EvalArgs& a, OpfOut o, double damping_min, int precision,
                       double* scratch, size_t scratch_per_cta, int grid, float* abuf, float* hbuf, double* a64,
                       float* cand, float* hws, int sms, int* counters, int* launches, cudaStream_t s) {
    *launches = 0;
    if (a.n <= 0) return cudaSuccess;
    const DLay L = make_dlayout(net);
    if ((size_t)L.total > scratch_per_cta) return cudaErrorInvalidValue;
    cudaError_t e;
    if (precision == CS_PREC_MIXED && hbuf && abuf && a64 && cand) {
        // FP32 screen in five kernels: front (model, balancing) at several CTAs per SM,
        // Hessenberg reduction on a two-CTA cluster, QR from shared memory at one CTA per
        // SM, FP64 refinement of the decisive eigenvalues, and the FP64 re-run of the
        // scenarios the FP32 screen cannot decide.
        const size_t hstride = dyn_hbuf_stride(net), astride = dyn_abuf_stride(net);
        e = launch_mode<DYN_FRONT>(net, a, o, damping_min, scratch, scratch_per_cta, L, abuf, astride, a64, grid,
                                   counters, s);
        if (e != cudaSuccess) return e;
        const int nmax = 5 * net.ng - 1;
        const size_t hsm = hess_smem_bytes(nmax);
        e = cudaFuncSetAttribute(hess_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
        if (e != cudaSuccess) return e;
        const int gh = 2 * (int)std::min<int64_t>((int64_t)std::max(1, sms / 2), a.n);
        hess_cluster_kernel<<<gh, kHsThreads, hsm, s>>>(a, o, abuf, astride, hbuf, hstride, nmax, counters + 3);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t qsm = qr_smem_bytes(nmax);
        e = cudaFuncSetAttribute(hqr_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
        if (e != cudaSuccess) return e;
        const int gq = (int)std::min<int64_t>((int64_t)sms, a.n);
        hqr_smem_kernel<<<gq, kQrThreads, qsm, s>>>(a, o, hbuf, hstride, nmax, damping_min, cand, counters + 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t rsm = refine_smem_bytes(nmax);
        e = cudaFuncSetAttribute(eig_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
        if (e != cudaSuccess) return e;
        eig_refine_kernel<<<gq, kRfThreads, rsm, s>>>(a, o, hbuf, hstride, abuf, astride, a64, dyn_a64_stride(net),
                                                       cand, nmax, damping_min, counters + 4);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_mode<DYN_RERUN>(net, a, o, damping_min, scratch, scratch_per_cta, L, nullptr, 0, nullptr, grid,
                                   counters + 2, s);
        if (e != cudaSuccess) return e;
        *launches = 5;
    } else if (precision == CS_PREC_MIXED && abuf && hws) {
        // networks whose Hessenberg matrix exceeds one block's shared memory: model and
        // balancing, the blocked Hessenberg reduction of the whole chunk on the tensor
        // cores, FP32 QR per scenario, FP64 re-run of the undecided ones
        const int nmax = 5 * net.ng - 1;
        const size_t astride = dyn_abuf_stride(net);
        e = launch_mode<DYN_FRONT_LARGE>(net, a, o, damping_min, scratch, scratch_per_cta, L, abuf, astride, nullptr,
                                         grid, counters, s);
        if (e != cudaSuccess) return e;
        e = launch_hess_tc(a.n, nmax, abuf + kHqHead, (long long)astride, hws, a.err, s);
        if (e != cudaSuccess) return e;
        e = launch_mode<DYN_QR_LARGE>(net, a, o, damping_min, scratch, scratch_per_cta, L, abuf, astride, nullptr, grid,
                                      counters + 1, s);
        if (e != cudaSuccess) return e;
        e = launch_mode<DYN_RERUN>(net, a, o, damping_min, scratch, scratch_per_cta, L, nullptr, 0, nullptr, grid,
                                   counters + 2, s);
        if (e != cudaSuccess) return e;
        *launches = 4;
    } else if (precision == CS_PREC_MIXED) {
        e = launch_mode<DYN_MIXED_INLINE>(net, a, o, damping_min, scratch, scratch_per_cta, L, nullptr, 0, nullptr,
                                          grid, counters, s);
        if (e != cudaSuccess) return e;
        *launches = 1;
    } else {
        e = launch_mode<DYN_FULL64>(net, a, o, damping_min, scratch, scratch_per_cta, L, nullptr, 0, nullptr, grid,
                                    counters, s);
        if (e != cudaSuccess) return e;
        *launches = 1;
    }
    if (a.sev_n1 && a.sev_pairs) {
        int blocks = (a.n + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        record_kernel<<<blocks, 256, 0, s>>>(net.nbr, net.nE, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 1;
    }
    return cudaSuccess;
}
