// Internal declarations shared by the libcs translation units (host + device).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cs.h"

#define CS_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------- complex ----
struct cplx {
    double re, im;
};
CS_HD cplx cm(double r, double i) { return cplx{r, i}; }
CS_HD cplx operator+(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
CS_HD cplx operator-(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
CS_HD cplx operator-(cplx a) { return cplx{-a.re, -a.im}; }
CS_HD cplx operator*(cplx a, cplx b) { return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
CS_HD cplx operator*(double s, cplx a) { return cplx{s * a.re, s * a.im}; }
CS_HD cplx conj(cplx a) { return cplx{a.re, -a.im}; }
CS_HD cplx mulj(cplx a) { return cplx{-a.im, a.re}; }          // j * a
CS_HD double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
CS_HD cplx cdiv(cplx a, cplx b) {
    double d = b.re * b.re + b.im * b.im;
    return cplx{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// ----------------------------------------------------- device network data ----
// All arrays are device pointers owned by the library (one allocation per net).
struct DevNet {
    int nb, nbr, ng, nlev, ref;     // ref: reference bus (original index)
    double base;                    // MVA
    double ws;                      // synchronous speed, rad/s
    int nE;                         // outage elements = nbr + ng

    // branches (original order)
    const int* f;
    const int* t;
    const cplx* yff;
    const cplx* yft;
    const cplx* ytf;
    const cplx* ytt;
    const double* smax2;            // (rate / base)^2

    // buses (original order)
    const double* vmin;
    const double* vmax;
    const double* gsh;              // p.u.
    const double* bsh;
    const double* Pd;               // [nlev * nb] p.u.
    const double* Qd;

    // generators (original order), p.u. on base
    const int* gbus;
    const double* pmin;
    const double* pmax;
    const double* qmin;
    const double* qmax;
    const double* c2;               // $/MW^2h
    const double* c1;               // $/MWh
    const double* c0;
    // machine data converted to the system base
    const double* xd;
    const double* xq;
    const double* xp;               // x'd = x'q
    const double* Td0;
    const double* Tq0;
    const double* KA;
    const double* TA;
    const double* H2;               // 2 H (system base)
    const double* Dm;               // D (system base)

    // incidence (original bus order)
    const int* bus_br_ptr;          // [nb + 1]
    const int* bus_br;              // entries 2*branch + side (0 = from end, 1 = to end)
    const int* bus_gen_ptr;         // [nb + 1]
    const int* bus_gen;

    // symbolic analysis of the bus graph (new = elimination order)
    int nL;                         // off-diagonal blocks of L
    const int* perm;                // new -> old bus
    const int* iperm;               // old -> new
    const int* Lcolptr;             // [nb + 1] CSC over new columns
    const int* Lrow;                // [nL] new row index of each block
    const int* Lcol;                // [nL] new column index of each block
    const int* Lrowptr;             // [nb + 1] CSR over new rows
    const int* Lrowcol;             // [nL] column k of each row entry
    const int* Lrowblk;             // [nL] block id of each row entry
    int nlevels;
    const int* lev_ptr;             // [nlevels + 1] into lev_col
    const int* lev_col;             // new column ids, grouped by elimination-tree height
    const int* tgt_ptr;             // [nlevels + 1] into tgt (factor targets per level)
    const int* tgt;                 // target ids: j (diagonal of column j) or nb + block id
    const int* upd_ptr;             // [nb + nL + 1] per target id
    const int* upd_a;               // block (i,k)
    const int* upd_b;               // block (j,k)
    const int* blk_br_ptr;          // [nL + 1] branches whose off-diagonal pair is block q
    const int* blk_br;
};

// scenario masks: up to two outaged elements
struct Outage {
    int br0, br1, br2;   // outaged branches (-1 none)
    int g0, g1, g2;      // outaged generators (-1 none)
};

// Outage set of a scenario from up to three element ids (-1 = none; a repeated id
// counts once; the third id is the N-3 extension).
CS_HD Outage decode_outage(int nbr, int ng, int ei, int ej, int ek = -1) {
    Outage o{-1, -1, -1, -1, -1, -1};
    int e[3] = {ei, ej, ek};
    for (int q = 0; q < 3; ++q) {
        int v = e[q];
        if (v < 0) continue;
        if (v < nbr) {
            if (o.br0 < 0) o.br0 = v;
            else if (v != o.br0 && o.br1 < 0) o.br1 = v;
            else if (v != o.br0 && v != o.br1) o.br2 = v;
        } else if (v < nbr + ng) {
            int g = v - nbr;
            if (o.g0 < 0) o.g0 = g;
            else if (g != o.g0 && o.g1 < 0) o.g1 = g;
            else if (g != o.g0 && g != o.g1) o.g2 = g;
        }
    }
    return o;
}
CS_HD bool br_out(const Outage& o, int b) { return b == o.br0 || b == o.br1 || b == o.br2; }
CS_HD bool gen_out(const Outage& o, int g) { return g == o.g0 || g == o.g1 || g == o.g2; }
CS_HD int n_br_out(const Outage& o) { return (o.br0 >= 0) + (o.br1 >= 0) + (o.br2 >= 0); }
CS_HD int n_gen_out(const Outage& o) { return (o.g0 >= 0) + (o.g1 >= 0) + (o.g2 >= 0); }

// ------------------------------------------------------------ kernel API ----
// Per-scenario intermediate state written by the OPF kernel, read by the
// dynamics kernel (device, chunk-sized).
struct OpfOut {
    double* x;          // [chunk * (2 nb + 2 ng)]  Va, Vm, Pg, Qg
    int* status;        // [chunk] 0 not run, 1 converged, 2 failed, 3 islanded;
                        // small-signal screen: 6 = FP64 re-run pending, 7 = done early
};

struct EvalArgs {
    const int* ei;
    const int* ej;
    int n;
    int level;
    cs_result out;          // device pointers
    uint8_t* sev_n1;        // severity table of the level: [nE] (255 = missing)
    uint8_t* sev_pairs;     // [nE*(nE-1)/2]
    int* err;               // device error word
    int* reruns;            // device counter: FP64 eigen re-runs of the mixed-precision screen
    const int* ek;          // [n] third outage element (N-3), or nullptr
    bool main_island;       // islanded scenarios also get the OPF of their main island
};

// launch wrappers (return cudaError_t)
cudaError_t launch_islands(const DevNet& net, const EvalArgs& a, int* islanded, cudaStream_t s);
cudaError_t launch_opf(const DevNet& net, const EvalArgs& a, const int* islanded, OpfOut o,
                       double tol, int max_it, double* scratch, size_t scratch_per_cta, int grid,
                       int* counter, cudaStream_t s);
size_t opf_scratch_doubles(const DevNet& net);
int opf_ctas_per_sm();       // resident OPF CTAs per SM the kernel is built for
// Small-signal screen.  counters: 5 work counters (zeroed by the caller).
// abuf, hbuf, a64, cand (mixed form, NULL otherwise): a.n * dyn_abuf_stride(net)
// and a.n * dyn_hbuf_stride(net) floats for the balanced matrices with their
// balancing and Householder factors (front kernel -> cluster Hessenberg kernel ->
// refinement) and the packed Hessenberg matrices (-> shared-memory QR), a.n *
// dyn_a64_stride(net) doubles for the FP64 state matrices and a.n *
// dyn_cand_stride() floats for the refinement candidates; only usable when
// dyn_split_fits(net, device).  Otherwise, mixed form with abuf and hws (a.n *
// hess_tc_workspace_floats(5 ng - 1) floats): the tensor-core Hessenberg path.
// *launches: kernels issued (the reduction's own launches not counted).
cudaError_t launch_dyn(const DevNet& net, const EvalArgs& a, OpfOut o, double damping_min, int precision,
                       double* scratch, size_t scratch_per_cta, int grid, float* abuf, float* hbuf, double* a64,
                       float* cand, float* hws, int sms, int* counters, int* launches, cudaStream_t s);
size_t dyn_scratch_doubles(const DevNet& net);
size_t dyn_hbuf_stride(const DevNet& net);
size_t dyn_abuf_stride(const DevNet& net);
size_t dyn_a64_stride(const DevNet& net);     // doubles per scenario: the FP64 state matrix (mixed form)
size_t dyn_cand_stride();                     // floats per scenario: refinement candidates (mixed form)
bool dyn_split_fits(const DevNet& net, int device);
cudaError_t launch_risk(int nE, const uint8_t* S1, const uint8_t* S2, const double* lam, int mode,
                        double* R, int64_t* missing, cudaStream_t s, const double* F = nullptr);
cudaError_t launch_risk_batch(int nE, const uint8_t* S1, const uint8_t* S2, const double* lam, long long ns,
                              int mode, double* R, int* err, int bad_bit, cudaStream_t s);
// C_b += alpha A_b B_b on the tensor cores (TF32 x 3 terms, FP32 accumulation), row-major
// FP32, batch strides sA / sB / sC in elements; a bounded wait that gives up sets ERR_TIMEOUT
cudaError_t launch_tc_gemm(int batch, int M, int N, int K, const float* A, long long lda, long long sA,
                           const float* B, long long ldb, long long sB, float* C, long long ldc, long long sC,
                           float alpha, int* err, cudaStream_t s);
// the same with general element strides: A(m, k) = A[m * am + k * ak], B(k, n) = B[k * bk + n * bn]
cudaError_t launch_tc_gemm_strided(int batch, int M, int N, int K, const float* A, long long am, long long ak,
                                   long long sA, const float* B, long long bk, long long bn, long long sB, float* C,
                                   long long ldc, long long sC, float alpha, int* err, cudaStream_t s);
// Blocked Householder reduction of `batch` row-major n x n FP32 matrices (stride sA apart)
// to upper Hessenberg form, in place (entries below the subdiagonal set to zero); the
// trailing updates on the tensor cores.  ws: hess_tc_workspace_floats(n) floats per matrix.
size_t hess_tc_workspace_floats(int n);
cudaError_t launch_hess_tc(int batch, int n, float* A, long long sA, float* ws, int* err, cudaStream_t s);
cudaError_t launch_enumerate(int nE, int64_t first, int64_t count, int* ei, int* ej,
                             cudaStream_t s);
cudaError_t launch_enumerate3(int nE, int64_t first, int64_t count, int* ei, int* ej, int* ek,
                              cudaStream_t s);

// error bits of the device error word
enum { ERR_BAD_ELEMENT = 1, ERR_SCRATCH = 2, ERR_BAD_RATE = 4, ERR_TIMEOUT = 8 };
