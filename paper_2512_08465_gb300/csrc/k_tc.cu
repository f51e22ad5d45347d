// Tensor-core (tcgen05) building blocks for the eigen screen of large networks.
//
// The Householder reduction of a state matrix to Hessenberg form is, in its
// blocked form, a sequence of panel factorisations and trailing-matrix updates
// C <- C + alpha A B with a short inner dimension (the panel width).  At the
// state orders of large networks (2,499 for 500 generators) the updates carry
// about 70 % of the reduction's flops, so they run on the 5th-generation tensor
// cores: operands staged in shared memory in the canonical K-major layout,
// tcgen05.mma issued by one thread, the FP32 accumulator in tensor memory, read
// back with tcgen05.ld for the epilogue.  The eigen screen needs FP32 accuracy,
// which one TF32 product does not give, so every operand is split into two TF32
// terms (x = x_hi + x_lo, x_hi = tf32(x), x_lo = tf32(x - x_hi)) and the product
// is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below FP32
// rounding): three MMAs per K-step, all into the same FP32 accumulator.
//
// Every wait on an mbarrier is bounded: after kSpinLimit polls the block sets
// the error word, stops issuing work and still releases its tensor memory.
#include <algorithm>
#include <cstdint>

#include "cs_internal.h"

namespace {

constexpr int kTcThreads = 128;          // 4 warps: one per 32-lane quarter of the accumulator
constexpr int kBM = 128;                 // rows of a tile (MMA M)
constexpr int kBN = 64;                  // columns of a tile (MMA N)
constexpr int kBK = 32;                  // inner dimension staged per round (4 MMA K-steps of 8)
constexpr int kKStep = 8;                // K of one kind::tf32 MMA
constexpr uint32_t kTmemCols = 64;       // accumulator columns (FP32), a power of two >= 32
constexpr long long kSpinLimit = 1ll << 22;

// Shared-memory tile in the canonical no-swizzle K-major layout: core matrices of
// 8 rows x 4 TF32 (16 bytes per row, 128 contiguous bytes each); along K the core
// matrices of one 8-row group are adjacent (leading byte offset 128), the 8-row
// groups follow one another (stride byte offset (kBK / 4) * 128 = 1024).
__device__ __forceinline__ int tile_index(int r, int k) {
    return ((r >> 3) * (kBK / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}
constexpr uint32_t kLbo = 128;
constexpr uint32_t kSbo = (kBK / 4) * 128;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading and stride
// byte offsets (all in 16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D in FP32, A and B in TF32, both K-major, M = kBM, N = kBN.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long spin = 0; spin < kSpinLimit; ++spin) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// C_b += alpha A_b B_b for every b of the batch (FP32; A is M x K with element (m, k)
// at A_b[m * am + k * ak], B is K x N with (k, n) at B_b[k * bk + n * bn], C is M x N
// row-major with row stride ldc), in three TF32 products per term.  Grid:
// (ceil(M / kBM), ceil(N / kBN), batch).
__global__ void __launch_bounds__(kTcThreads, 1)
tc_gemm_kernel(int M, int N, int K, const float* __restrict__ A, long long am, long long ak, long long sA,
               const float* __restrict__ B, long long bk, long long bn, long long sB, float* __restrict__ C,
               long long ldc, long long sC, float alpha, int accumulate, int* err) {
    extern __shared__ __align__(1024) float tc_smem[];
    float* a_hi = tc_smem;                            // kBM x kBK each, canonical layout
    float* a_lo = a_hi + kBM * kBK;
    float* b_hi = a_lo + kBM * kBK;                   // kBN x kBK each
    float* b_lo = b_hi + kBN * kBK;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int timed_out;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const float* Ab = A + (long long)blockIdx.z * sA;
    const float* Bb = B + (long long)blockIdx.z * sB;
    float* Cb = C + (long long)blockIdx.z * sC;
    const uint32_t mb = smem_addr(&mbar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        timed_out = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mb), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    uint32_t phase = 0;
    const int rounds = (K + kBK - 1) / kBK;
    for (int rd = 0; rd < rounds && !timed_out; ++rd) {
        const int k0 = rd * kBK;
        // stage A (kBM x kBK) and B^T (kBN x kBK) as TF32 pairs; zeros outside the matrices
        // consecutive threads walk the operand's contiguous dimension (coalesced loads)
        for (int w = tid; w < kBM * kBK; w += kTcThreads) {
            const int r = (am == 1) ? w % kBM : w / kBK, k = (am == 1) ? w / kBM : w % kBK;
            const int gr = m0 + r, gk = k0 + k;
            const float x = (gr < M && gk < K) ? Ab[(long long)gr * am + (long long)gk * ak] : 0.0f;
            const float hi = tf32_round(x);
            a_hi[tile_index(r, k)] = hi;
            a_lo[tile_index(r, k)] = tf32_round(x - hi);
        }
        for (int w = tid; w < kBN * kBK; w += kTcThreads) {
            const int k = (bk == 1) ? w % kBK : w / kBN, n = (bk == 1) ? w / kBK : w % kBN;
            const int gn = n0 + n, gk = k0 + k;
            const float x = (gn < N && gk < K) ? alpha * Bb[(long long)gk * bk + (long long)gn * bn] : 0.0f;
            const float hi = tf32_round(x);
            b_hi[tile_index(n, k)] = hi;
            b_lo[tile_index(n, k)] = tf32_round(x - hi);
        }
        // the generic-proxy stores must be visible to the tensor cores' async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < kBK / kKStep; ++ks) {
                // one K-step is two core matrices along K: 256 bytes further
                const uint32_t off = (uint32_t)ks * 2u * 128u;
                const uint64_t dah = smem_desc(smem_addr(a_hi) + off), dal = smem_desc(smem_addr(a_lo) + off);
                const uint64_t dbh = smem_desc(smem_addr(b_hi) + off), dbl = smem_desc(smem_addr(b_lo) + off);
                const uint32_t acc0 = (rd > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                    :: "r"(tmem), "l"(dah), "l"(dbh), "r"(kIdesc), "r"(acc0) : "memory");
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                    :: "r"(tmem), "l"(dah), "l"(dbl), "r"(kIdesc), "r"(1u) : "memory");
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                    :: "r"(tmem), "l"(dal), "l"(dbh), "r"(kIdesc), "r"(1u) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mb) : "memory");
        }
        // the MMAs read the staged tiles: wait for them before the next round overwrites
        if (!mbar_wait(mb, phase)) {
            if (lane == 0) timed_out = 1;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!timed_out && rounds > 0) {
        // epilogue: warp w holds rows 32 w .. 32 w + 31 (TMEM lanes), 8 columns per load
        const int row = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < kBN; c0 += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float* crow = Cb + (long long)row * ldc;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = n0 + c0 + q;
                    if (col < N) crow[col] = accumulate ? crow[col] + __uint_as_float(v[q]) : __uint_as_float(v[q]);
                }
            }
        }
    }
    if (timed_out && tid == 0 && err) atomicOr(err, ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

static cudaError_t tc_gemm_any(int batch, int M, int N, int K, const float* A, long long am, long long ak,
                               long long sA, const float* B, long long bk, long long bn, long long sB, float* C,
                               long long ldc, long long sC, float alpha, int accumulate, int* err, cudaStream_t s) {
    if (batch <= 0 || M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN), (unsigned)batch);
    const size_t smem = sizeof(float) * 2 * (size_t)(kBM + kBN) * kBK;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<<<grid, kTcThreads, smem, s>>>(M, N, K, A, am, ak, sA, B, bk, bn, sB, C, ldc, sC, alpha, accumulate,
                                                   err);
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm_strided(int batch, int M, int N, int K, const float* A, long long am, long long ak,
                                   long long sA, const float* B, long long bk, long long bn, long long sB, float* C,
                                   long long ldc, long long sC, float alpha, int* err, cudaStream_t s) {
    return tc_gemm_any(batch, M, N, K, A, am, ak, sA, B, bk, bn, sB, C, ldc, sC, alpha, 1, err, s);
}

cudaError_t launch_tc_gemm(int batch, int M, int N, int K, const float* A, long long lda, long long sA,
                           const float* B, long long ldb, long long sB, float* C, long long ldc, long long sC,
                           float alpha, int* err, cudaStream_t s) {
    return launch_tc_gemm_strided(batch, M, N, K, A, lda, 1, sA, B, ldb, 1, sB, C, ldc, sC, alpha, err, s);
}

namespace {

// ---------------------------------------------------------------------------
// Blocked Householder reduction to upper Hessenberg form (the first step of the
// eigenvalue screen of Section II-B-2), for state matrices too large for one
// block's shared memory.  Panels of kNB columns; within a panel, column j is
// brought up to date with the panel's earlier reflectors from both sides
// (right: A P, through Y = A V T; left: P^T = I - V T^T V^T), its reflector is
// formed, and Y's column j = tau_j (A v_j - Y V^T v_j) is accumulated with one
// matrix-vector product over the panel-start matrix; T grows by one column.
// After the panel the trailing columns get A <- P^T (A P): A -= Y V^T (right,
// all rows), W = V^T A, W <- T^T W, A -= V W (left, rows below the panel's first
// reflector) -- the three products on the tensor cores; then the panel's
// finished columns are written back.  Per matrix the workspace holds V^T (kNB x
// n), Y (n x kNB), W and T^T W (kNB x n each), the panel's finished columns (kNB x
// n), the product y (n), tau (kNB) and T (kNB x kNB).
constexpr int kNB = 32;
constexpr int kHsT = 256;

struct HessWs {
    float *Vt, *Y, *W, *W2, *P, *y, *tau, *T;
};
__host__ __device__ inline size_t hess_ws_floats(int n) {
    return (size_t)5 * kNB * n + (size_t)n + kNB + (size_t)kNB * kNB + 64;
}
__device__ inline HessWs hess_ws(float* base, int n) {
    HessWs w;
    w.Vt = base;
    w.Y = w.Vt + (size_t)kNB * n;
    w.W = w.Y + (size_t)kNB * n;
    w.W2 = w.W + (size_t)kNB * n;
    w.P = w.W2 + (size_t)kNB * n;
    w.y = w.P + (size_t)kNB * n;
    w.tau = w.y + n;
    w.T = w.tau + kNB;
    return w;
}

template <int K>
__device__ void block_sum(float (&v)[K], float* red, int cnt) {
    // red: [kHsT / 32][K] floats of shared memory; result broadcast in v
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = 0; i < cnt; ++i)
        for (int off = 16; off; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    if (lane == 0)
        for (int i = 0; i < cnt; ++i) red[warp * K + i] = v[i];
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
        float t = 0.0f;
        for (int w = 0; w < kHsT / 32; ++w) t += red[w * K + i];
        v[i] = t;
    }
    __syncthreads();
}

// Column j of panel (k, jj = j - k): bring it up to date, form its reflector.
__global__ void __launch_bounds__(kHsT) hess_col_kernel(int n, int k, int j, float* A, long long sA, float* wsb,
                                                       size_t wss) {
    extern __shared__ float cbuf[];                    // n floats: the column
    __shared__ float red[(kHsT / 32) * kNB];
    __shared__ float u[kNB];
    const int tid = threadIdx.x, jj = j - k;
    const float* Ab = A + (long long)blockIdx.x * sA;
    const HessWs w = hess_ws(wsb + (size_t)blockIdx.x * wss, n);
    // right update: c = A(:, j) - Y(:, 0:jj) V(j, 0:jj)^T
    for (int r = tid; r < n; r += kHsT) {
        float c = Ab[(long long)r * n + j];
        for (int i = 0; i < jj; ++i) c -= w.Y[(size_t)r * kNB + i] * w.Vt[(size_t)i * n + j];
        cbuf[r] = c;
    }
    __syncthreads();
    if (jj > 0) {                                      // left update: c -= V T^T V^T c (rows k+1..)
        float acc[kNB];
#pragma unroll
        for (int i = 0; i < kNB; ++i) acc[i] = 0.0f;
        for (int r = k + 1 + tid; r < n; r += kHsT) {
            const float c = cbuf[r];
#pragma unroll
            for (int i = 0; i < kNB; ++i)
                if (i < jj) acc[i] += w.Vt[(size_t)i * n + r] * c;
        }
        block_sum<kNB>(acc, red, jj);
        if (tid < jj) {                                // u = T^T acc (T upper triangular)
            float t = 0.0f;
            for (int l = 0; l <= tid; ++l) t += w.T[l * kNB + tid] * acc[l];
            u[tid] = t;
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < n; r += kHsT) {
            float c = cbuf[r];
            for (int i = 0; i < jj; ++i) c -= w.Vt[(size_t)i * n + r] * u[i];
            cbuf[r] = c;
        }
        __syncthreads();
    }
    // reflector of c(j+1 .. n-1): beta e1 = (I - tau v v^T) c, v(j+1) = 1
    float ss[1] = {0.0f};
    for (int r = j + 2 + tid; r < n; r += kHsT) ss[0] += cbuf[r] * cbuf[r];
    block_sum<1>(ss, red, 1);
    const float a0 = cbuf[j + 1];
    float beta = a0, tau = 0.0f, scale = 0.0f;
    if (ss[0] > 0.0f) {
        beta = -copysignf(sqrtf(a0 * a0 + ss[0]), a0);
        tau = (beta - a0) / beta;
        scale = 1.0f / (a0 - beta);
    }
    for (int r = tid; r < n; r += kHsT) {
        w.P[(size_t)jj * n + r] = (r <= j) ? cbuf[r] : (r == j + 1 ? beta : 0.0f);
        w.Vt[(size_t)jj * n + r] = (r <= j) ? 0.0f : (r == j + 1 ? 1.0f : cbuf[r] * scale);
    }
    if (tid == 0) w.tau[jj] = tau;
}

// y = A(:, j+1:n) v_j over the panel-start matrix: a warp per row.
__global__ void __launch_bounds__(kHsT) hess_mv_kernel(int n, int k, int j, const float* A, long long sA, float* wsb,
                                                      size_t wss) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jj = j - k;
    const int r = blockIdx.x * (kHsT / 32) + warp;
    const float* Ab = A + (long long)blockIdx.y * sA;
    const HessWs w = hess_ws(wsb + (size_t)blockIdx.y * wss, n);
    if (r >= n) return;
    const float* row = Ab + (long long)r * n;
    const float* v = w.Vt + (size_t)jj * n;
    float acc = 0.0f;
    for (int c = j + 1 + lane; c < n; c += 32) acc += row[c] * v[c];
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) w.y[r] = acc;
}

// Y(:, jj) = tau (y - Y(:, 0:jj) V(:, 0:jj)^T v_j); T(0:jj, jj) = -tau T s; T(jj, jj) = tau.
__global__ void __launch_bounds__(kHsT) hess_yt_kernel(int n, int k, int j, float* wsb, size_t wss) {
    __shared__ float red[(kHsT / 32) * kNB];
    __shared__ float sv[kNB];
    const int tid = threadIdx.x, jj = j - k;
    const HessWs w = hess_ws(wsb + (size_t)blockIdx.x * wss, n);
    const float tau = w.tau[jj];
    float acc[kNB];
#pragma unroll
    for (int i = 0; i < kNB; ++i) acc[i] = 0.0f;
    if (jj > 0) {
        for (int r = j + 1 + tid; r < n; r += kHsT) {
            const float v = w.Vt[(size_t)jj * n + r];
#pragma unroll
            for (int i = 0; i < kNB; ++i)
                if (i < jj) acc[i] += w.Vt[(size_t)i * n + r] * v;
        }
        block_sum<kNB>(acc, red, jj);
        if (tid < jj) sv[tid] = acc[tid];
        __syncthreads();
    }
    for (int r = tid; r < n; r += kHsT) {
        float t = w.y[r];
        for (int i = 0; i < jj; ++i) t -= w.Y[(size_t)r * kNB + i] * sv[i];
        w.Y[(size_t)r * kNB + jj] = tau * t;
    }
    if (tid < jj) {
        float t = 0.0f;
        for (int l = tid; l < jj; ++l) t += w.T[tid * kNB + l] * sv[l];
        w.T[tid * kNB + jj] = -tau * t;
    }
    if (tid == 0) w.T[jj * kNB + jj] = tau;
}

// W2 = T^T W (nbp x m, row stride m): W2(i, c) = sum_{l <= i} T(l, i) W(l, c).
__global__ void hess_tw_kernel(int n, int nbp, int m, float* wsb, size_t wss) {
    const HessWs w = hess_ws(wsb + (size_t)blockIdx.y * wss, n);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nbp * m; q += gridDim.x * blockDim.x) {
        const int i = q / m, c = q % m;
        float t = 0.0f;
        for (int l = 0; l <= i; ++l) t += w.T[l * kNB + i] * w.W[(size_t)l * m + c];
        w.W2[(size_t)i * m + c] = t;
    }
}

// the panel's finished columns k .. k + nbp - 1 back into A
__global__ void hess_put_kernel(int n, int k, int nbp, float* A, long long sA, float* wsb, size_t wss) {
    float* Ab = A + (long long)blockIdx.y * sA;
    const HessWs w = hess_ws(wsb + (size_t)blockIdx.y * wss, n);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nbp * n; q += gridDim.x * blockDim.x) {
        const int jj = q / n, r = q % n;
        Ab[(long long)r * n + k + jj] = w.P[(size_t)jj * n + r];
    }
}

}  // namespace

size_t hess_tc_workspace_floats(int n) { return hess_ws_floats(n); }

cudaError_t launch_hess_tc(int batch, int n, float* A, long long sA, float* ws, int* err, cudaStream_t s) {
    if (batch <= 0 || n < 3) return cudaSuccess;
    const size_t wss = hess_ws_floats(n);
    const size_t csm = sizeof(float) * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(hess_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
    if (e != cudaSuccess) return e;
    // workspace views of the first matrix for the tensor-core products (layout of hess_ws)
    const long long sW = (long long)wss;
    float* Vt0 = ws;
    float* Y0 = Vt0 + (size_t)kNB * n;
    float* W0 = Y0 + (size_t)kNB * n;
    float* W20 = W0 + (size_t)kNB * n;
    for (int k = 0; k < n - 2; k += kNB) {
        const int nbp = std::min(kNB, n - 2 - k);
        for (int j = k; j < k + nbp; ++j) {
            hess_col_kernel<<<batch, kHsT, csm, s>>>(n, k, j, A, sA, ws, wss);
            hess_mv_kernel<<<dim3((unsigned)((n + kHsT / 32 - 1) / (kHsT / 32)), (unsigned)batch), kHsT, 0, s>>>(
                n, k, j, A, sA, ws, wss);
            hess_yt_kernel<<<batch, kHsT, 0, s>>>(n, k, j, ws, wss);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int c0 = k + nbp, m = n - c0;           // trailing columns
        if (m > 0) {
            // right: A(:, c0:) -= Y V(c0:, :)^T   (V(r, i) = Vt[i n + r])
            e = tc_gemm_any(batch, n, m, nbp, Y0, kNB, 1, sW, Vt0 + c0, n, 1, sW, A + c0, n, sA, -1.0f, 1, err, s);
            if (e != cudaSuccess) return e;
            // left: W = V(k+1:, :)^T A(k+1:, c0:), W2 = T^T W, A(k+1:, c0:) -= V(k+1:, :) W2
            e = tc_gemm_any(batch, nbp, m, n - k - 1, Vt0 + k + 1, n, 1, sW, A + (long long)(k + 1) * n + c0, n, 1,
                            sA, W0, m, sW, 1.0f, 0, err, s);
            if (e != cudaSuccess) return e;
            hess_tw_kernel<<<dim3((unsigned)std::min(1024, (nbp * m + 255) / 256), (unsigned)batch), 256, 0, s>>>(
                n, nbp, m, ws, wss);
            e = tc_gemm_any(batch, n - k - 1, m, nbp, Vt0 + k + 1, 1, n, sW, W20, m, 1, sW,
                            A + (long long)(k + 1) * n + c0, n, sA, -1.0f, 1, err, s);
            if (e != cudaSuccess) return e;
        }
        hess_put_kernel<<<dim3((unsigned)std::min(1024, (nbp * n + 255) / 256), (unsigned)batch), 256, 0, s>>>(
            n, k, nbp, A, sA, ws, wss);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
