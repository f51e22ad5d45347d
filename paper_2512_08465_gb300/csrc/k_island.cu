// Scenario decode (Section II-A) and islanding (Section II-B-3).
//
// Islanding: one warp per scenario.  The lanes initialise a parent array of
// the bus graph in shared memory; lane 0 unions the end buses of every
// in-service branch (union by smaller index, path halving); the lanes then
// count the roots.  Generator outages do not change the topology.  Every bus
// counts, so an isolated bus is an island of its own.
#include "cs_internal.h"

namespace {

constexpr int kWarpsPerBlock = 8;   // per CTA, fewer when n_bus ints per warp exceed the shared memory

__device__ int uf_find(int* p, int u) {
    while (p[u] != u) {
        p[u] = p[p[u]];
        u = p[u];
    }
    return u;
}

__global__ void islands_kernel(DevNet net, EvalArgs a, int* islanded) {
    extern __shared__ int sh_parent[];
    const int wpb = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* parent = sh_parent + warp * net.nb;
    const int nwarps_total = gridDim.x * wpb;
    for (int s = blockIdx.x * wpb + warp; s < a.n; s += nwarps_total) {
        const int ei = a.ei[s], ej = a.ej[s], ek = a.ek ? a.ek[s] : -1;
        const bool bad = ei < -1 || ej < -1 || ek < -1 || ei >= net.nE || ej >= net.nE || ek >= net.nE ||
                         (ei < 0 && ej >= 0) || (ej < 0 && ek >= 0);
        if (bad) {
            if (lane == 0) {
                atomicOr(a.err, ERR_BAD_ELEMENT);
                islanded[s] = 2;
                a.out.klass[s] = 255;
                a.out.severe[s] = 1;
                a.out.n_islands[s] = 0;
                a.out.opf_iters[s] = 0;
                a.out.cost[s] = __longlong_as_double(0x7ff8000000000000ll);
                if (a.out.v_margin) a.out.v_margin[s] = __longlong_as_double(0x7ff8000000000000ll);
                if (a.out.max_loading) a.out.max_loading[s] = __longlong_as_double(0x7ff8000000000000ll);
                if (a.out.shed_mw) a.out.shed_mw[s] = __longlong_as_double(0x7ff8000000000000ll);
                if (a.out.main_klass) a.out.main_klass[s] = 255;
                a.out.max_re[s] = __longlong_as_double(0x7ff8000000000000ll);
                a.out.min_zeta[s] = __longlong_as_double(0x7ff8000000000000ll);
            }
            continue;
        }
        const Outage o = decode_outage(net.nbr, net.ng, ei, ej, ek);
        for (int u = lane; u < net.nb; u += 32) parent[u] = u;
        __syncwarp();
        if (lane == 0) {
            for (int b = 0; b < net.nbr; ++b) {
                if (br_out(o, b)) continue;
                int x = uf_find(parent, net.f[b]);
                int y = uf_find(parent, net.t[b]);
                if (x != y) {
                    if (x < y) parent[y] = x; else parent[x] = y;
                }
            }
        }
        __syncwarp();
        int cnt = 0;
        for (int u = lane; u < net.nb; u += 32) cnt += (parent[u] == u);
        for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) {
            islanded[s] = cnt > 1 ? 1 : 0;
            a.out.n_islands[s] = (int16_t)(cnt > 32767 ? 32767 : cnt);
            // main-island fields: the OPF kernel fills them for islanded scenarios
            // when the main-island form is on
            if (a.out.shed_mw) a.out.shed_mw[s] = cnt > 1 ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
            if (a.out.main_klass) a.out.main_klass[s] = 255;
            if (cnt > 1) {
                a.out.klass[s] = CS_ISLANDED;
                a.out.severe[s] = 1;
                a.out.opf_iters[s] = 0;
                const double nan = __longlong_as_double(0x7ff8000000000000ll);
                a.out.cost[s] = nan;
                if (a.out.v_margin) a.out.v_margin[s] = nan;
                if (a.out.max_loading) a.out.max_loading[s] = nan;
                a.out.max_re[s] = nan;
                a.out.min_zeta[s] = nan;
            }
        }
        __syncwarp();
    }
}

// k -> (i, j), i < j, lexicographic: start(i) = i*E - i*(i+1)/2.
__device__ __forceinline__ long long pair_start(long long i, long long E) {
    return i * E - (i * (i + 1)) / 2;
}

__global__ void enumerate_kernel(int E, long long first, long long count, int* ei, int* ej) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        const long long k = first + q;
        long long lo = 0, hi = E - 2;          // largest i with start(i) <= k
        while (lo < hi) {
            long long mid = (lo + hi + 1) >> 1;
            if (pair_start(mid, E) <= k) lo = mid; else hi = mid - 1;
        }
        ei[q] = (int)lo;
        ej[q] = (int)(k - pair_start(lo, E) + lo + 1);
    }
}

}  // namespace

cudaError_t launch_islands(const DevNet& net, const EvalArgs& a, int* islanded, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    // one parent array of n_bus ints per warp; above the default 48 KB the kernel opts in
    // to the device's per-CTA maximum, and fewer warps share a CTA if even that is short
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t per_warp = sizeof(int) * (size_t)net.nb;
    int wpb = kWarpsPerBlock;
    while (wpb > 1 && per_warp * wpb > (size_t)optin) --wpb;
    const size_t smem = per_warp * wpb;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;     // one bus array alone does not fit
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(islands_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int blocks = (a.n + wpb - 1) / wpb;
    if (blocks > 4096) blocks = 4096;
    islands_kernel<<<blocks, 32 * wpb, smem, s>>>(net, a, islanded);
    return cudaGetLastError();
}

// Triples i < j < k in lexicographic order (the N-3 extension): the triples before
// those starting with i number C(E,3) - C(E-i,3); within i, (j, k) is the pair of
// rank r among the E-1-i elements after i.
__device__ __forceinline__ long long choose3(long long x) { return x < 3 ? 0 : x * (x - 1) * (x - 2) / 6; }

__global__ void enumerate3_kernel(int E, long long first, long long count, int* ei, int* ej, int* ek) {
    const long long total = choose3(E);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        const long long t = first + q;
        long long lo = 0, hi = E - 3;           // largest i with total - C(E-i,3) <= t
        while (lo < hi) {
            long long mid = (lo + hi + 1) >> 1;
            if (total - choose3(E - mid) <= t) lo = mid; else hi = mid - 1;
        }
        const long long r = t - (total - choose3(E - lo));
        const long long m = E - 1 - lo;         // elements after i
        long long a = 0, b = m - 2;             // largest p with pair_start(p, m) <= r
        while (a < b) {
            long long mid = (a + b + 1) >> 1;
            if (pair_start(mid, m) <= r) a = mid; else b = mid - 1;
        }
        ei[q] = (int)lo;
        ej[q] = (int)(lo + 1 + a);
        ek[q] = (int)(lo + 1 + (r - pair_start(a, m) + a + 1));
    }
}

cudaError_t launch_enumerate3(int nE, int64_t first, int64_t count, int* ei, int* ej, int* ek, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    enumerate3_kernel<<<(int)blocks, 256, 0, s>>>(nE, (long long)first, (long long)count, ei, ej, ek);
    return cudaGetLastError();
}

cudaError_t launch_enumerate(int nE, int64_t first, int64_t count, int* ei, int* ej, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    enumerate_kernel<<<(int)blocks, 256, 0, s>>>(nE, (long long)first, (long long)count, ei, ej);
    return cudaGetLastError();
}
