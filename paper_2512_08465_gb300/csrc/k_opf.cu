// Primal-dual interior-point AC optimal power flow, one scenario per CTA
// (Section II-B-1: a contingency is severe when the OPF does not converge or
// its solution violates an operational limit).
//
// Algorithm: the MIPS primal-dual interior-point method (Wang, Murillo-Sanchez,
// Zimmerman, Thomas 2007) in polar coordinates, x = [Va, Vm, Pg, Qg], cost
// sum c2 (B Pg)^2 + c1 B Pg + c0, equalities = bus power balance and the
// reference angle, inequalities = |S|^2 flow limits at both branch ends and
// box bounds on Vm, Pg, Qg.  Start Va = 0, Vm = 1, Pg = (Pmin + Pmax)/2,
// Qg = 0, z = max(-h, 1), mu = 1/z, lam = 0; step factor 0.99995, centring
// sigma = 0.1; stop when the feasibility, gradient, complementarity and cost
// conditions are all below tol, at most max_it iterations.
//
// GB300 design:
//  * persistent grid: each CTA pulls scenarios from an atomic counter, so
//    scenarios with uneven iteration counts never idle a CTA;
//  * outaged elements are masked, the network pattern is kept: an outaged
//    branch contributes numeric zeros and its flow rows are inactive, an
//    outaged generator's variables are decoupled and its bound rows inactive;
//  * the Newton system is reduced exactly before factorisation: the generator
//    variables (diagonal in the Hessian) are eliminated into the multiplier
//    diagonal, and the reference-angle row is replaced by dVa_ref = 0 (its
//    multiplier step is recovered from its own Newton row afterwards).  What
//    remains has one 4x4 block [dVa, dVm, dlamP, dlamQ] per bus and the bus
//    graph as block pattern;
//  * that matrix is factorised as a block LDL^T on ONE symbolic analysis per
//    network (minimum-degree order, elimination tree, fill pattern and
//    left-looking update lists, built on the host at load time), with the
//    4x4 pivot blocks inverted by Gauss-Jordan with partial pivoting.  Columns
//    of one elimination-tree level are independent, so a level is one
//    parallel step of the CTA (16 threads per target block).  The narrow
//    upper levels leave most threads at barriers, so CTAs are small (128
//    threads) and three are resident per SM to overlap one another's waits;
//  * every branch quantity (flows, first and second derivatives of both end
//    powers, the weighted 4x4 Hessian) is computed once per iteration by one
//    thread from the branch's own four voltage variables and gathered by
//    buses and blocks, deterministically (no atomics);
//  * main-island form (an extension after Sections II-A, V-A and VI): an
//    islanded scenario gets the OPF of the component whose in-service
//    generators have the largest total Pmax.  Buses outside it are masked like
//    outaged elements (identity blocks, no rows, no constraints, their load
//    shed), so the pattern and the symbolic analysis stay those of the
//    network; the reference moves to the island's largest unit when the
//    original one lies outside.  A generator bus carries the generator's
//    multiplier diagonal, so its reference block stays a regular pivot
//    wherever it falls in the elimination order.
#include <cmath>

#include "cs_internal.h"

namespace {

#ifndef CS_OPF_THREADS
#define CS_OPF_THREADS 128
#endif
#ifndef CS_OPF_CTAS
#define CS_OPF_CTAS 4
#endif
constexpr int kThreads = CS_OPF_THREADS;   // threads per scenario CTA
constexpr int kCtasPerSm = CS_OPF_CTAS;    // resident CTAs per SM the register budget is sized for
constexpr int kWarps = kThreads / 32;
constexpr int kRec = 46;     // doubles per branch record
constexpr double kXi = 0.99995;
constexpr double kSigma = 0.1;
constexpr double kLimitTol = 1e-6;
constexpr int kRefineSteps = 3;              // FP64 iterative refinement steps per Newton solve (at most)
constexpr double kRefineTol = 4.0 * 2.220446049250313e-16;   // refinement done: backward error at rounding level
constexpr double kBackwardTol = 1e-15;       // componentwise backward error accepted from the block solve + GMRES
constexpr int kDenseMax = 1024;              // dense fallback for reduced systems up to this order
constexpr int kPanel = 8;                    // panel width of the dense fallback's blocked LU
constexpr int kGmresM = 8;                   // GMRES iterations per Newton solve (at most)
constexpr int kRedMax = kGmresM + 1 > 10 ? kGmresM + 1 : 10;   // values per block reduction (at most)

// record layout
constexpr int R_DSF = 0, R_DST = 8, R_GF = 16, R_GT = 20, R_H = 24, R_LG = 34, R_NG = 38, R_SF = 42, R_ST = 44;

__device__ __forceinline__ int hidx(int p, int q) {
    if (p > q) { int t = p; p = q; q = t; }
    // (0,0)0 (0,1)1 (0,2)2 (0,3)3 (1,1)4 (1,2)5 (1,3)6 (2,2)7 (2,3)8 (3,3)9
    const int base[4] = {0, 4, 7, 9};
    return base[p] + (q - p);
}

struct Lay {
    // bus
    int Va, Vm, lP, lQ, zu, zl, muu, mul, gP, gQ, LxVa, LxVm, NVa, NVm, DP, DQ, rP, rQ, dzu, dzl, dmuu, dmul;
    // gen
    int Pg, Qg, gz, gmu, gdz, gdmu, MP, MQ, NP, NQ, LxP, LxQ, dPg, dQg;
    // branch
    int zf, zt, muf, mut, hf, ht, dzf, dzt, dmuf, dmut, rec;
    // KKT: assembled blocks (Kb, Kd) kept for refinement, factor (Ub, Lb, Db, Di), vectors
    int Kb, Kd, Ub, Lb, Db, Di, x, bv, rv, cs, drs, dpiv;   // drs, dpiv: dense backstop's row scales, pivots
    int kv, kz, gx0, gxb, gr;   // GMRES: Krylov basis, preconditioned basis, start, best iterate, work
    int uf, cap, dead;          // main island: union-find parents (int), capacity per root, bus flags (bytes)
    long dense;                 // dense fallback matrix (4nb)^2, -1 if the network is too large
    long total;
};

Lay make_layout(const DevNet& n) {
    Lay L{};
    int o = 0;
    auto take = [&](int cnt) { int r = o; o += cnt; return r; };
    int nb = n.nb, ng = n.ng, nbr = n.nbr;
    L.Va = take(nb); L.Vm = take(nb); L.lP = take(nb); L.lQ = take(nb); L.zu = take(nb); L.zl = take(nb);
    L.muu = take(nb); L.mul = take(nb); L.gP = take(nb); L.gQ = take(nb); L.LxVa = take(nb); L.LxVm = take(nb);
    L.NVa = take(nb); L.NVm = take(nb); L.DP = take(nb); L.DQ = take(nb); L.rP = take(nb); L.rQ = take(nb);
    L.dzu = take(nb); L.dzl = take(nb); L.dmuu = take(nb); L.dmul = take(nb);
    L.Pg = take(ng); L.Qg = take(ng); L.gz = take(4 * ng); L.gmu = take(4 * ng); L.gdz = take(4 * ng);
    L.gdmu = take(4 * ng); L.MP = take(ng); L.MQ = take(ng); L.NP = take(ng); L.NQ = take(ng);
    L.LxP = take(ng); L.LxQ = take(ng); L.dPg = take(ng); L.dQg = take(ng);
    L.zf = take(nbr); L.zt = take(nbr); L.muf = take(nbr); L.mut = take(nbr); L.hf = take(nbr); L.ht = take(nbr);
    L.dzf = take(nbr); L.dzt = take(nbr); L.dmuf = take(nbr); L.dmut = take(nbr);
    L.rec = take(kRec * nbr);
    o = (o + 15) & ~15;
    L.Kb = take(16 * n.nL); L.Kd = take(16 * nb);
    L.Ub = take(16 * n.nL); L.Lb = take(16 * n.nL); L.Db = take(16 * nb); L.Di = take(16 * nb);
    L.x = take(4 * nb); L.bv = take(4 * nb); L.rv = take(4 * nb); L.cs = take(4 * nb);
    L.drs = take(4 * nb); L.dpiv = take(2 * nb);
    L.kv = take(4 * nb * (kGmresM + 1)); L.kz = take(4 * nb * kGmresM);
    L.gx0 = take(4 * nb); L.gxb = take(4 * nb); L.gr = take(4 * nb);
    L.uf = take((nb + 1) / 2); L.cap = take(nb); L.dead = take((nb + 7) / 8);
    o = (o + 31) & ~31;
    if (4 * nb <= kDenseMax) {
        L.dense = o;
        L.total = (long)o + (long)16 * nb * nb;
    } else {
        L.dense = -1;
        L.total = o;
    }
    L.total = (L.total + 31) & ~31L;
    return L;
}

// ------------------------------------------------------------------ helpers --
struct RedBuf {
    double v[kRedMax][kWarps];
};

__device__ __forceinline__ double red_op(int op, double a, double b) {
    return op == 1 ? a + b : (op == 0 ? fmax(a, b) : fmin(a, b));
}

// reduce K values per thread: ops[k] = 0 max, 1 sum, 2 min.  Result broadcast in out[]
// (shared).  Warp shuffles, then one pass over the per-warp results.
template <int K>
__device__ void block_reduce(RedBuf& rb, double (&val)[K], const int (&ops)[K], double* out) {
    static_assert(K <= kRedMax, "block_reduce: more values than RedBuf and Scal::red hold");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < K; ++k) {
        double v = val[k];
        for (int off = 16; off; off >>= 1) v = red_op(ops[k], v, __shfl_xor_sync(0xffffffffu, v, off));
        val[k] = v;
    }
    if (kWarps == 1) {
        if (tid == 0)
            for (int k = 0; k < K; ++k) out[k] = val[k];
        __syncthreads();
        return;
    }
    if (lane == 0)
        for (int k = 0; k < K; ++k) rb.v[k][warp] = val[k];
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < K; ++k) {
            double v = rb.v[k][0];
            for (int w = 1; w < kWarps; ++w) v = red_op(ops[k], v, rb.v[k][w]);
            out[k] = v;
        }
    }
    __syncthreads();
}

// Inverse of the symmetric part of a 4x4 pivot block: LU factorisation with
// partial pivoting, forward/back substitution for each column of the identity,
// then symmetrisation of the result.  (Near the end of the interior-point
// iteration some pivot blocks are nearly singular; the LU-based inverse keeps
// the error low-rank, which the iterative refinement removes, where a
// Gauss-Jordan inverse did not.)  Four lanes of one warp (q = 0..3, aligned
// to a multiple of 4) take one pivot: each repeats the factorisation (one
// instruction stream, so the FP64 pipe pays for it once) and solves for column
// q.  Returns false, on all four lanes, if a pivot is exactly zero or not
// finite.
__device__ bool inv4(const double* A, double* Ainv, int q) {
    const unsigned grp = 0xFu << (threadIdx.x & 28);
    double a[4][4], dinv[4];
    int piv[4] = {0, 1, 2, 3};
    for (int r = 0; r < 4; ++r)                  // symmetric part of the updated pivot
        for (int c = 0; c < 4; ++c) a[r][c] = 0.5 * (A[4 * r + c] + A[4 * c + r]);
    bool ok = true;
    for (int c = 0; c < 4 && ok; ++c) {
        int p = c;
        double best = fabs(a[c][c]);
        for (int r = c + 1; r < 4; ++r)
            if (fabs(a[r][c]) > best) { best = fabs(a[r][c]); p = r; }
        if (!(best > 0.0) || !isfinite(best)) { ok = false; break; }
        if (p != c) {
            for (int k = 0; k < 4; ++k) { double t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
            int t = piv[c]; piv[c] = piv[p]; piv[p] = t;
        }
        dinv[c] = 1.0 / a[c][c];                  // one division per pivot
        for (int r = c + 1; r < 4; ++r) {
            a[r][c] *= dinv[c];
            const double m = a[r][c];
            for (int k = c + 1; k < 4; ++k) a[r][k] -= m * a[c][k];
        }
    }
    // the group reads A above before any lane of it writes the inverse (A and Ainv
    // are different arrays, but the symmetrisation below reads what others wrote)
    double y[4];
    if (ok) {
        for (int i = 0; i < 4; ++i) {
            double v = (piv[i] == q) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= a[i][k] * y[k];
            y[i] = v;
        }
        for (int i = 3; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < 4; ++k) v -= a[i][k] * y[k];
            y[i] = v * dinv[i];
        }
        for (int i = 0; i < 4; ++i) Ainv[4 * i + q] = y[i];
    }
    __syncwarp(grp);
    // Symmetrise.  Only the lower blocks are stored and updated with L(i,k) U(j,k)^T,
    // which assumes a symmetric pivot inverse; an LU-based inverse of a nearly singular
    // symmetric block is far from symmetric in rounding, and the factorisation would
    // then not be a consistent L D L^T (refinement stalls).
    double t[4];
    if (ok)
        for (int i = 0; i < 4; ++i) t[i] = Ainv[4 * q + i];   // row q, written by lane i
    __syncwarp(grp);
    if (ok)
        for (int i = 0; i < 4; ++i) Ainv[4 * i + q] = 0.5 * (y[i] + t[i]);
    __syncwarp(grp);
    return ok;
}

// One branch at the current iterate: flows, derivatives, weighted Hessian,
// Lagrangian-gradient and N contributions.  If init, also sets z, mu of the
// two flow rows from h (z = max(-h, 1), mu = gamma / z).
__device__ void eval_branch(const DevNet& net, int b, double* W, const Lay& L, double gamma,
                            bool init) {
    const int f = net.f[b], t = net.t[b];
    double* rec = W + L.rec + (size_t)kRec * b;
    const double vf = W[L.Vm + f], vt = W[L.Vm + t];
    double sf, cf, st, ct;
    sincos(W[L.Va + f], &sf, &cf);
    sincos(W[L.Va + t], &st, &ct);
    const cplx ef = cm(cf, sf), et = cm(ct, st);
    const cplx Vf = vf * ef, Vt = vt * et;
    const cplx yff = net.yff[b], yft = net.yft[b], ytf = net.ytf[b], ytt = net.ytt[b];
    const cplx zero = cm(0.0, 0.0);
    const cplx dVf[4] = {mulj(Vf), ef, zero, zero};
    const cplx dVt[4] = {zero, zero, mulj(Vt), et};
    const cplx If = yff * Vf + yft * Vt;
    const cplx It = ytf * Vf + ytt * Vt;
    cplx dIf[4], dIt[4], dSf[4], dSt[4];
    for (int p = 0; p < 4; ++p) {
        dIf[p] = yff * dVf[p] + yft * dVt[p];
        dIt[p] = ytf * dVf[p] + ytt * dVt[p];
    }
    const cplx Sf = Vf * conj(If), St = Vt * conj(It);
    for (int p = 0; p < 4; ++p) {
        dSf[p] = dVf[p] * conj(If) + Vf * conj(dIf[p]);
        dSt[p] = dVt[p] * conj(It) + Vt * conj(dIt[p]);
    }
    const double smax2 = net.smax2[b];
    const double hf = abs2(Sf) - smax2, ht = abs2(St) - smax2;
    double zf, zt, muf, mut;
    if (init) {
        zf = fmax(-hf, 1.0);
        zt = fmax(-ht, 1.0);
        muf = gamma / zf;
        mut = gamma / zt;
        W[L.zf + b] = zf; W[L.zt + b] = zt; W[L.muf + b] = muf; W[L.mut + b] = mut;
    } else {
        zf = W[L.zf + b]; zt = W[L.zt + b]; muf = W[L.muf + b]; mut = W[L.mut + b];
    }
    W[L.hf + b] = hf;
    W[L.ht + b] = ht;
    double gf[4], gt[4];
    for (int p = 0; p < 4; ++p) {
        gf[p] = 2.0 * (Sf.re * dSf[p].re + Sf.im * dSf[p].im);
        gt[p] = 2.0 * (St.re * dSt[p].re + St.im * dSt[p].im);
    }
    const double lPf = W[L.lP + f], lQf = W[L.lQ + f], lPt = W[L.lP + t], lQt = W[L.lQ + t];
    // weights: Re(c * d2S) = lamP Re d2S + lamQ Im d2S + 2 mu Re(conj(S) d2S)
    const cplx wf = cm(lPf, -lQf) + (2.0 * muf) * conj(Sf);
    const cplx wt = cm(lPt, -lQt) + (2.0 * mut) * conj(St);
    const double bf = muf / zf, bt = mut / zt;
    // second derivatives of V: f end (0,0) -V_f, (0,1) j e_f ; t end (2,2) -V_t, (2,3) j e_t
    for (int p = 0; p < 4; ++p) {
        for (int q = p; q < 4; ++q) {
            cplx d2Vf = zero, d2Vt = zero;
            if (p == 0 && q == 0) d2Vf = -Vf;
            if (p == 0 && q == 1) d2Vf = mulj(ef);
            if (p == 2 && q == 2) d2Vt = -Vt;
            if (p == 2 && q == 3) d2Vt = mulj(et);
            const cplx d2If = yff * d2Vf + yft * d2Vt;
            const cplx d2It = ytf * d2Vf + ytt * d2Vt;
            const cplx d2Sf = d2Vf * conj(If) + dVf[p] * conj(dIf[q]) + dVf[q] * conj(dIf[p]) + Vf * conj(d2If);
            const cplx d2St = d2Vt * conj(It) + dVt[p] * conj(dIt[q]) + dVt[q] * conj(dIt[p]) + Vt * conj(d2It);
            double h = (wf * d2Sf).re + (wt * d2St).re;
            h += 2.0 * muf * (dSf[q].re * dSf[p].re + dSf[q].im * dSf[p].im);
            h += 2.0 * mut * (dSt[q].re * dSt[p].re + dSt[q].im * dSt[p].im);
            h += bf * gf[p] * gf[q] + bt * gt[p] * gt[q];
            rec[R_H + hidx(p, q)] = h;
        }
    }
    const double nf = (muf * hf + gamma) / zf, nt = (mut * ht + gamma) / zt;
    for (int p = 0; p < 4; ++p) {
        rec[R_DSF + 2 * p] = dSf[p].re;
        rec[R_DSF + 2 * p + 1] = dSf[p].im;
        rec[R_DST + 2 * p] = dSt[p].re;
        rec[R_DST + 2 * p + 1] = dSt[p].im;
        rec[R_GF + p] = gf[p];
        rec[R_GT + p] = gt[p];
        rec[R_LG + p] = lPf * dSf[p].re + lQf * dSf[p].im + lPt * dSt[p].re + lQt * dSt[p].im +
                        muf * gf[p] + mut * gt[p];
        rec[R_NG + p] = nf * gf[p] + nt * gt[p];
    }
    rec[R_SF] = Sf.re;
    rec[R_SF + 1] = Sf.im;
    rec[R_ST] = St.re;
    rec[R_ST + 1] = St.im;
}

// Solve (L D L^T) v = v in place for the 4-vector-per-bus array v (new order):
// forward by elimination-tree levels, block diagonal, backward by levels.
__device__ void ldl_solve(const DevNet& net, const double* W, const Lay& L, double* v) {
    const int tid = threadIdx.x, nb = net.nb, lane = tid & 31, warp = tid >> 5;
    for (int lev = 0; lev < net.nlevels; ++lev) {
        const int c0 = net.lev_ptr[lev], c1 = net.lev_ptr[lev + 1];
        if (c1 - c0 <= kWarps) {
            // narrow level (the top of the elimination tree): a warp per column, its
            // lanes over the blocks of the row, partial sums reduced by shuffles
            if (warp < c1 - c0) {
                const int j = net.lev_col[c0 + warp];
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                for (int e = net.Lrowptr[j] + lane; e < net.Lrowptr[j + 1]; e += 32) {
                    const double* Lq = W + L.Lb + 16 * net.Lrowblk[e];
                    const double* y = v + 4 * net.Lrowcol[e];
                    const double y0 = y[0], y1 = y[1], y2 = y[2], y3 = y[3];
                    a0 += Lq[0] * y0 + Lq[1] * y1 + Lq[2] * y2 + Lq[3] * y3;
                    a1 += Lq[4] * y0 + Lq[5] * y1 + Lq[6] * y2 + Lq[7] * y3;
                    a2 += Lq[8] * y0 + Lq[9] * y1 + Lq[10] * y2 + Lq[11] * y3;
                    a3 += Lq[12] * y0 + Lq[13] * y1 + Lq[14] * y2 + Lq[15] * y3;
                }
                for (int off = 16; off; off >>= 1) {
                    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
                    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
                    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
                    a3 += __shfl_xor_sync(0xffffffffu, a3, off);
                }
                if (lane < 4) v[4 * j + lane] -= (lane == 0 ? a0 : lane == 1 ? a1 : lane == 2 ? a2 : a3);
            }
        } else {
            for (int w = tid; w < 4 * (c1 - c0); w += kThreads) {
                const int j = net.lev_col[c0 + (w >> 2)], r = w & 3;
                double acc = v[4 * j + r];
                for (int e = net.Lrowptr[j]; e < net.Lrowptr[j + 1]; ++e) {
                    const double* Lq = W + L.Lb + 16 * net.Lrowblk[e] + 4 * r;
                    const double* y = v + 4 * net.Lrowcol[e];
                    acc -= Lq[0] * y[0] + Lq[1] * y[1] + Lq[2] * y[2] + Lq[3] * y[3];
                }
                v[4 * j + r] = acc;
            }
        }
        __syncthreads();
    }
    for (int j = tid; j < nb; j += kThreads) {
        const double* Di = W + L.Di + 16 * j;
        double* y = v + 4 * j;
        const double y0 = y[0], y1 = y[1], y2 = y[2], y3 = y[3];
        for (int r = 0; r < 4; ++r)
            y[r] = Di[4 * r] * y0 + Di[4 * r + 1] * y1 + Di[4 * r + 2] * y2 + Di[4 * r + 3] * y3;
    }
    __syncthreads();
    for (int lev = net.nlevels - 1; lev >= 0; --lev) {
        const int c0 = net.lev_ptr[lev], c1 = net.lev_ptr[lev + 1];
        if (c1 - c0 <= kWarps) {
            if (warp < c1 - c0) {
                const int j = net.lev_col[c0 + warp];
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                for (int e = net.Lcolptr[j] + lane; e < net.Lcolptr[j + 1]; e += 32) {
                    const double* Lq = W + L.Lb + 16 * e;
                    const double* xi = v + 4 * net.Lrow[e];
                    const double x0 = xi[0], x1 = xi[1], x2 = xi[2], x3 = xi[3];
                    a0 += Lq[0] * x0 + Lq[4] * x1 + Lq[8] * x2 + Lq[12] * x3;
                    a1 += Lq[1] * x0 + Lq[5] * x1 + Lq[9] * x2 + Lq[13] * x3;
                    a2 += Lq[2] * x0 + Lq[6] * x1 + Lq[10] * x2 + Lq[14] * x3;
                    a3 += Lq[3] * x0 + Lq[7] * x1 + Lq[11] * x2 + Lq[15] * x3;
                }
                for (int off = 16; off; off >>= 1) {
                    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
                    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
                    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
                    a3 += __shfl_xor_sync(0xffffffffu, a3, off);
                }
                if (lane < 4) v[4 * j + lane] -= (lane == 0 ? a0 : lane == 1 ? a1 : lane == 2 ? a2 : a3);
            }
        } else {
            for (int w = tid; w < 4 * (c1 - c0); w += kThreads) {
                const int j = net.lev_col[c0 + (w >> 2)], r = w & 3;
                double acc = v[4 * j + r];
                for (int e = net.Lcolptr[j]; e < net.Lcolptr[j + 1]; ++e) {
                    const double* Lq = W + L.Lb + 16 * e + r;
                    const double* xi = v + 4 * net.Lrow[e];
                    acc -= Lq[0] * xi[0] + Lq[4] * xi[1] + Lq[8] * xi[2] + Lq[12] * xi[3];
                }
                v[4 * j + r] = acc;
            }
        }
        __syncthreads();
    }
}

// r = b - K x with the assembled (unfactored) blocks, one thread per (bus, row),
// and the componentwise backward error of x, max_i |r_i| / (|K| |x| + |b|)_i
// (returned per thread, to be max-reduced by the caller).
__device__ double kkt_residual(const DevNet& net, const double* W, const Lay& L, const double* x, double* r) {
    const int tid = threadIdx.x, nb = net.nb;
    double worst = 0.0;
    for (int w = tid; w < 4 * nb; w += kThreads) {
        const int i = w >> 2, rr = w & 3;
        const double* Kd = W + L.Kd + 16 * i + 4 * rr;
        const double* xi = x + 4 * i;
        const double bw = W[L.bv + w];
        double acc = bw, sc = fabs(bw);
        for (int c = 0; c < 4; ++c) {
            const double t = Kd[c] * xi[c];
            acc -= t;
            sc += fabs(t);
        }
        for (int e = net.Lrowptr[i]; e < net.Lrowptr[i + 1]; ++e) {        // blocks (i, k), k < i
            const double* Kq = W + L.Kb + 16 * net.Lrowblk[e] + 4 * rr;
            const double* xk = x + 4 * net.Lrowcol[e];
            for (int c = 0; c < 4; ++c) {
                const double t = Kq[c] * xk[c];
                acc -= t;
                sc += fabs(t);
            }
        }
        for (int e = net.Lcolptr[i]; e < net.Lcolptr[i + 1]; ++e) {        // blocks (j, i)^T, j > i
            const double* Kq = W + L.Kb + 16 * e + rr;
            const double* xj = x + 4 * net.Lrow[e];
            for (int c = 0; c < 4; ++c) {
                const double t = Kq[4 * c] * xj[c];
                acc -= t;
                sc += fabs(t);
            }
        }
        r[w] = acc;
        const double be = (sc > 0.0) ? fabs(acc) / sc : (acc == 0.0 ? 0.0 : INFINITY);
        worst = fmax(worst, isfinite(be) ? be : INFINITY);
    }
    __syncthreads();
    return worst;
}

// y = K x with the assembled blocks (x, y: 4-vectors per bus, new order).
__device__ void kkt_matvec(const DevNet& net, const double* W, const Lay& L, const double* x, double* y) {
    const int tid = threadIdx.x, nb = net.nb;
    for (int w = tid; w < 4 * nb; w += kThreads) {
        const int i = w >> 2, rr = w & 3;
        const double* Kd = W + L.Kd + 16 * i + 4 * rr;
        const double* xi = x + 4 * i;
        double acc = Kd[0] * xi[0] + Kd[1] * xi[1] + Kd[2] * xi[2] + Kd[3] * xi[3];
        for (int e = net.Lrowptr[i]; e < net.Lrowptr[i + 1]; ++e) {
            const double* Kq = W + L.Kb + 16 * net.Lrowblk[e] + 4 * rr;
            const double* xk = x + 4 * net.Lrowcol[e];
            acc += Kq[0] * xk[0] + Kq[1] * xk[1] + Kq[2] * xk[2] + Kq[3] * xk[3];
        }
        for (int e = net.Lcolptr[i]; e < net.Lcolptr[i + 1]; ++e) {
            const double* Kq = W + L.Kb + 16 * e + rr;
            const double* xj = x + 4 * net.Lrow[e];
            acc += Kq[0] * xj[0] + Kq[4] * xj[1] + Kq[8] * xj[2] + Kq[12] * xj[3];
        }
        y[w] = acc;
    }
    __syncthreads();
}

struct GmresShared {
    double H[kGmresM + 1][kGmresM];
    double g[kGmresM + 1], c[kGmresM], s[kGmresM], y[kGmresM];
};

// GMRES on K d = r, right-preconditioned by the block LDL^T factors, starting
// from the current solution x (r = b - K x in rv, omega0 its backward error).
// When the pivot blocks are nearly singular, the factors are exact except in
// a subspace of small dimension, so a few Krylov steps remove what plain
// refinement cannot.  Arnoldi with classical Gram-Schmidt applied twice; the
// candidate solution is formed and its componentwise backward error checked
// after every step; x ends as the best candidate.  Returns its backward error.
__device__ double kkt_gmres(const DevNet& net, double* W, const Lay& L, RedBuf& rb, double* red, GmresShared& gs,
                            double omega0) {
    const int tid = threadIdx.x, N = 4 * net.nb;
    double* x = W + L.x;
    double* x0 = W + L.gx0;
    double* xb = W + L.gxb;
    double* V = W + L.kv;
    double* Z = W + L.kz;
    double* t = W + L.gr;
    const int ops_sum[1] = {1}, ops_max[1] = {0};
    int ops_h[kGmresM + 1];
    for (int i = 0; i <= kGmresM; ++i) ops_h[i] = 1;
    {
        double ss = 0.0;
        for (int w = tid; w < N; w += kThreads) {
            x0[w] = x[w];
            xb[w] = x[w];
            const double rw = W[L.rv + w];
            ss += rw * rw;
        }
        double v1[1] = {ss};
        block_reduce<1>(rb, v1, ops_sum, red);
    }
    const double beta = sqrt(red[0]);
    if (!(beta > 0.0) || !isfinite(beta)) return omega0;
    for (int w = tid; w < N; w += kThreads) V[w] = W[L.rv + w] / beta;
    if (tid == 0) {
        for (int i = 0; i <= kGmresM; ++i) gs.g[i] = 0.0;
        gs.g[0] = beta;
    }
    __syncthreads();
    double best = omega0;
    for (int j = 0; j < kGmresM; ++j) {
        double* zj = Z + (size_t)j * N;
        for (int w = tid; w < N; w += kThreads) zj[w] = V[(size_t)j * N + w];
        __syncthreads();
        ldl_solve(net, W, L, zj);
        kkt_matvec(net, W, L, zj, t);
        for (int pass = 0; pass < 2; ++pass) {              // classical Gram-Schmidt, twice
            double h[kGmresM + 1];
            for (int i = 0; i <= kGmresM; ++i) h[i] = 0.0;
            for (int w = tid; w < N; w += kThreads) {
                const double tw = t[w];
#pragma unroll
                for (int i = 0; i <= kGmresM; ++i)
                    if (i <= j) h[i] += V[(size_t)i * N + w] * tw;
            }
            block_reduce<kGmresM + 1>(rb, h, ops_h, red);
            for (int w = tid; w < N; w += kThreads) {
                double tw = t[w];
#pragma unroll
                for (int i = 0; i <= kGmresM; ++i)
                    if (i <= j) tw -= red[i] * V[(size_t)i * N + w];
                t[w] = tw;
            }
            if (tid == 0)
                for (int i = 0; i <= j; ++i) gs.H[i][j] = (pass == 0 ? 0.0 : gs.H[i][j]) + red[i];
            __syncthreads();
        }
        double hn;
        {
            double ss = 0.0;
            for (int w = tid; w < N; w += kThreads) ss += t[w] * t[w];
            double v1[1] = {ss};
            block_reduce<1>(rb, v1, ops_sum, red);
            hn = sqrt(red[0]);
        }
        if (tid == 0) {                                     // Givens rotations, least-squares solve
            gs.H[j + 1][j] = hn;
            for (int i = 0; i < j; ++i) {
                const double a0 = gs.H[i][j], a1 = gs.H[i + 1][j];
                gs.H[i][j] = gs.c[i] * a0 + gs.s[i] * a1;
                gs.H[i + 1][j] = -gs.s[i] * a0 + gs.c[i] * a1;
            }
            const double d = hypot(gs.H[j][j], gs.H[j + 1][j]);
            gs.c[j] = (d > 0.0) ? gs.H[j][j] / d : 1.0;
            gs.s[j] = (d > 0.0) ? gs.H[j + 1][j] / d : 0.0;
            gs.H[j][j] = d;
            gs.H[j + 1][j] = 0.0;
            gs.g[j + 1] = -gs.s[j] * gs.g[j];
            gs.g[j] = gs.c[j] * gs.g[j];
            for (int i = j; i >= 0; --i) {
                double acc = gs.g[i];
                for (int k = i + 1; k <= j; ++k) acc -= gs.H[i][k] * gs.y[k];
                gs.y[i] = (gs.H[i][i] != 0.0) ? acc / gs.H[i][i] : 0.0;
            }
        }
        __syncthreads();
        if (hn > 0.0)
            for (int w = tid; w < N; w += kThreads) V[(size_t)(j + 1) * N + w] = t[w] / hn;
        for (int w = tid; w < N; w += kThreads) {
            double xw = x0[w];
            for (int i = 0; i <= j; ++i) xw += gs.y[i] * Z[(size_t)i * N + w];
            x[w] = xw;
        }
        __syncthreads();
        double v1[1] = {kkt_residual(net, W, L, x, t)};
        block_reduce<1>(rb, v1, ops_max, red);
        const double om = red[0];
        if (om < best) {
            best = om;
            for (int w = tid; w < N; w += kThreads) xb[w] = x[w];
        }
        if (om <= kBackwardTol || !(hn > 0.0)) break;
        __syncthreads();
    }
    __syncthreads();
    for (int w = tid; w < N; w += kThreads) x[w] = xb[w];
    __syncthreads();
    return best;
}

struct DenseShared {
    double val[kWarps];
    int idx[kWarps];
    int piv;
    double pv;
};

// Dense LU with partial pivoting of the equilibrated assembled reduced system
// (order 4 nb, row-major in scratch), solving for b into x.  Backstop for the Newton steps
// whose block solve did not reach the backward-error target.  The factors, the
// scales and the pivot sequence stay in the scratch for dense_resolve (the
// refinement of the backstop's solution).  Returns false when a pivot column is
// exactly zero.
__device__ bool dense_solve(const DevNet& net, double* W, const Lay& L, DenseShared& ds) {
    const int tid = threadIdx.x, nb = net.nb, N = 4 * nb;
    const int warp = tid >> 5, lane = tid & 31;
    double* A = W + L.dense;
    double* x = W + L.x;
    for (long w = tid; w < (long)N * N; w += kThreads) A[w] = 0.0;
    __syncthreads();
    for (int w = tid; w < 16 * nb; w += kThreads) {
        const int i = w >> 4, r = (w >> 2) & 3, c = w & 3;
        A[(long)(4 * i + r) * N + 4 * i + c] = W[L.Kd + 16 * i + 4 * r + c];
    }
    for (int w = tid; w < 16 * net.nL; w += kThreads) {
        const int q = w >> 4, r = (w >> 2) & 3, c = w & 3;
        const int i = net.Lrow[q], j = net.Lcol[q];
        const double v = W[L.Kb + 16 * q + 4 * r + c];
        A[(long)(4 * i + r) * N + 4 * j + c] = v;
        A[(long)(4 * j + c) * N + 4 * i + r] = v;
    }
    // Equilibrate rows then columns by powers of two (exact): the reduced system's
    // rows span ~1e-5..1e12 near convergence, and partial pivoting is only normwise
    // stable, so without scaling the balance rows lose all accuracy.
    double* rs = W + L.drs;         // row scales
    double* cs = W + L.cs;          // column scales
    int* piv = reinterpret_cast<int*>(W + L.dpiv);   // row exchanged with row k at step k
    for (int i = tid; i < N; i += kThreads) {
        double m = 0.0;
        for (int j = 0; j < N; ++j) m = fmax(m, fabs(A[(long)i * N + j]));
        int e;
        frexp(m, &e);
        rs[i] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
    }
    __syncthreads();
    for (int i = warp; i < N; i += kWarps) {
        const double ri = rs[i];
        for (int j = lane; j < N; j += 32) A[(long)i * N + j] *= ri;
    }
    for (int w = tid; w < N; w += kThreads) x[w] = W[L.bv + w] * rs[w];
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) {
        double m = 0.0;
        for (int i = 0; i < N; ++i) m = fmax(m, fabs(A[(long)i * N + j]));
        int e;
        frexp(m, &e);
        cs[j] = (m > 0.0) ? ldexp(1.0, -e) : 1.0;
    }
    __syncthreads();
    for (int i = warp; i < N; i += kWarps)
        for (int j = lane; j < N; j += 32) A[(long)i * N + j] *= cs[j];
    __syncthreads();
    // Right-looking LU with partial pivoting in panels of kPanel columns: the panel is
    // factorised column by column (whole rows are swapped), then the block row of U
    // is solved with the panel's unit lower triangle and the trailing matrix takes
    // one rank-kPanel update, so it is read and written once per panel.  The right-
    // hand side is eliminated along the way.
    for (int k0 = 0; k0 < N; k0 += kPanel) {
        const int ke = min(k0 + kPanel, N);
        for (int k = k0; k < ke; ++k) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < N; i += kThreads) {
                const double a = fabs(A[(long)i * N + k]);
                if (a > best) { best = a; bi = i; }
            }
            for (int off = 16; off; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) { ds.val[warp] = best; ds.idx[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double b0 = ds.val[0];
                int i0 = ds.idx[0];
                for (int q = 1; q < kWarps; ++q)
                    if (ds.val[q] > b0 || (ds.val[q] == b0 && ds.idx[q] < i0)) { b0 = ds.val[q]; i0 = ds.idx[q]; }
                ds.piv = i0;
                ds.pv = b0;
                piv[k] = i0;
            }
            __syncthreads();
            if (!(ds.pv > 0.0) || !isfinite(ds.pv)) return false;
            const int p = ds.piv;
            if (p != k) {
                for (int c = tid; c < N; c += kThreads) {
                    const double t = A[(long)k * N + c];
                    A[(long)k * N + c] = A[(long)p * N + c];
                    A[(long)p * N + c] = t;
                }
                if (tid == 0) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
                __syncthreads();
            }
            const double* pk = A + (long)k * N;
            const double inv = 1.0 / pk[k];
            const double xk = x[k];
            for (int i = k + 1 + tid; i < N; i += kThreads) {       // column k and the rest of the panel
                double* ri = A + (long)i * N;
                const double l = ri[k] * inv;
                ri[k] = l;
                for (int j = k + 1; j < ke; ++j) ri[j] -= l * pk[j];
                x[i] -= l * xk;
            }
            __syncthreads();
        }
        if (ke == N) break;
        for (int j = ke + tid; j < N; j += kThreads) {               // U block row: unit lower solve
            for (int r = k0 + 1; r < ke; ++r) {
                double acc = A[(long)r * N + j];
                for (int t = k0; t < r; ++t) acc -= A[(long)r * N + t] * A[(long)t * N + j];
                A[(long)r * N + j] = acc;
            }
        }
        __syncthreads();
        const int kb = ke - k0;
        for (int i = ke + warp; i < N; i += kWarps) {                // trailing rank-kb update
            double* ri = A + (long)i * N;
            double l[kPanel];
#pragma unroll
            for (int t = 0; t < kPanel; ++t) l[t] = (t < kb) ? ri[k0 + t] : 0.0;
            for (int j = ke + lane; j < N; j += 32) {
                double acc = ri[j];
#pragma unroll
                for (int t = 0; t < kPanel; ++t)
                    if (t < kb) acc -= l[t] * A[(long)(k0 + t) * N + j];
                ri[j] = acc;
            }
        }
        __syncthreads();
    }
    for (int k = N - 1; k >= 0; --k) {
        if (tid == 0) x[k] /= A[(long)k * N + k];
        __syncthreads();
        const double xk = x[k];
        for (int i = tid; i < k; i += kThreads) x[i] -= A[(long)i * N + k] * xk;
        __syncthreads();
    }
    for (int w = tid; w < N; w += kThreads) x[w] *= cs[w];     // undo the column scaling
    __syncthreads();
    return true;
}

// v <- K^{-1} v with the factors dense_solve left (row scaling, the recorded row
// exchanges, unit lower and upper triangular solves, column scaling).
__device__ void dense_resolve(const DevNet& net, double* W, const Lay& L, double* v) {
    const int tid = threadIdx.x, N = 4 * net.nb;
    const double* A = W + L.dense;
    const double* rs = W + L.drs;
    const double* cs = W + L.cs;
    const int* piv = reinterpret_cast<const int*>(W + L.dpiv);
    for (int w = tid; w < N; w += kThreads) v[w] *= rs[w];
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < N; ++k) {
            const int p = piv[k];
            if (p != k) { const double t = v[k]; v[k] = v[p]; v[p] = t; }
        }
    __syncthreads();
    for (int k = 0; k < N - 1; ++k) {
        const double vk = v[k];
        for (int i = k + 1 + tid; i < N; i += kThreads) v[i] -= A[(long)i * N + k] * vk;
        __syncthreads();
    }
    for (int k = N - 1; k >= 0; --k) {
        if (tid == 0) v[k] /= A[(long)k * N + k];
        __syncthreads();
        const double vk = v[k];
        for (int i = tid; i < k; i += kThreads) v[i] -= A[(long)i * N + k] * vk;
        __syncthreads();
    }
    for (int w = tid; w < N; w += kThreads) v[w] *= cs[w];
    __syncthreads();
}

struct Scal {          // per-scenario scalars in shared memory
    double gamma, f, f_prev, lref, dlref, ap, ad;
    double red[kRedMax];
    double niq, shed;  // number of inequality rows; load outside the main island (p.u.)
    int fail;
    int conv;
    int scen;
    int ref;           // reference bus of this scenario (-1: no main island)
    int isl;           // 1: main-island form of an islanded scenario
};

// In service in this scenario: not outaged and, in the main-island form of an
// islanded scenario (isl), inside the main island (per-bus flags in the scratch).
struct Live {
    const DevNet& net;
    const Outage& out;
    const double* W;
    const Lay& L;
    const int& isl;        // shared per-scenario flag: the main-island form is on
    __device__ bool bus(int i) const {
        return !isl || reinterpret_cast<const unsigned char*>(W + L.dead)[i] == 0;
    }
    __device__ bool br(int b) const { return !br_out(out, b) && bus(net.f[b]); }
    __device__ bool gen(int k) const { return !gen_out(out, k) && bus(net.gbus[k]); }
};

__device__ int uf_root(int* p, int u) {
    while (p[u] != u) {
        p[u] = p[p[u]];
        u = p[u];
    }
    return u;
}

// Main island of an islanded scenario (one thread; the components are the
// islanding kernel's, rebuilt here).  Union by the smaller index makes every
// root its component's lowest bus, so scanning roots in bus order with a
// strict comparison gives equal totals to the component of the lowest bus.
// Capacities are summed in per unit in generator order.  Sets the bus flags,
// sc.ref (-1 if no component has generation), sc.shed and sc.niq.
__device__ __noinline__ void main_island_setup(const DevNet& net, const Outage& out, const double* Pd, double* W,
                                  const Lay& L, Scal& sc) {
    const int nb = net.nb;
    int* par = reinterpret_cast<int*>(W + L.uf);
    double* cap = W + L.cap;
    unsigned char* dead = reinterpret_cast<unsigned char*>(W + L.dead);
    for (int i = 0; i < nb; ++i) { par[i] = i; cap[i] = 0.0; }
    for (int b = 0; b < net.nbr; ++b) {
        if (br_out(out, b)) continue;
        const int x = uf_root(par, net.f[b]), y = uf_root(par, net.t[b]);
        if (x != y) {
            if (x < y) par[y] = x; else par[x] = y;
        }
    }
    for (int k = 0; k < net.ng; ++k)
        if (!gen_out(out, k)) cap[uf_root(par, net.gbus[k])] += net.pmax[k];
    int main = -1;
    double best = 0.0;
    for (int i = 0; i < nb; ++i)
        if (par[i] == i && cap[i] > best) { main = i; best = cap[i]; }
    double shed = 0.0;
    int nb_live = 0;
    for (int i = 0; i < nb; ++i) {
        const bool d = (main < 0) || uf_root(par, i) != main;
        dead[i] = d ? 1 : 0;
        if (d) shed += Pd[i]; else ++nb_live;
    }
    int ref = -1;
    if (main >= 0) {
        if (!dead[net.ref]) {
            ref = net.ref;
        } else {
            double pb = -INFINITY;
            for (int k = 0; k < net.ng; ++k)
                if (!gen_out(out, k) && !dead[net.gbus[k]] && net.pmax[k] > pb) { pb = net.pmax[k]; ref = net.gbus[k]; }
        }
    }
    int nbr_live = 0, ng_live = 0;
    for (int b = 0; b < net.nbr; ++b) nbr_live += (!br_out(out, b) && !dead[net.f[b]]) ? 1 : 0;
    for (int k = 0; k < net.ng; ++k) ng_live += (!gen_out(out, k) && !dead[net.gbus[k]]) ? 1 : 0;
    sc.ref = ref;
    sc.shed = shed;
    sc.niq = 2.0 * nbr_live + 2.0 * nb_live + 4.0 * ng_live;
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
opf_kernel(DevNet net, EvalArgs a, const int* islanded, OpfOut o, double tol, int max_it,
           double* scratch, size_t per_cta, Lay L, int* counter) {
    __shared__ RedBuf rb;
    __shared__ double fsum[kThreads];      // partial update sums of the narrow factorisation levels
    __shared__ Scal sc;
    const int tid = threadIdx.x;
    double* W = scratch + per_cta * blockIdx.x;
    const int nb = net.nb, ng = net.ng, nbr = net.nbr;
    const double B = net.base;
    const double* Pd = net.Pd + (size_t)a.level * nb;
    const double* Qd = net.Qd + (size_t)a.level * nb;
    const int nx = 2 * nb + 2 * ng;

    for (;;) {
        if (tid == 0) sc.scen = atomicAdd(counter, 1);
        __syncthreads();
        const int s = sc.scen;
        if (s >= a.n) break;
        const bool isl = islanded[s] == 1 && a.main_island;
        if (islanded[s] != 0 && !isl) {        // islanded or invalid: nothing to do here
            if (tid == 0) o.status[s] = 3;
            __syncthreads();
            continue;
        }
        const Outage out = decode_outage(nbr, ng, a.ei[s], a.ej[s], a.ek ? a.ek[s] : -1);
        if (tid == 0) {
            sc.isl = isl ? 1 : 0;
            if (isl) {
                main_island_setup(net, out, Pd, W, L, sc);
            } else {
                sc.ref = net.ref;
                sc.niq = 2.0 * (nbr - n_br_out(out)) + 2.0 * nb + 4.0 * (ng - n_gen_out(out));
            }
        }
        __syncthreads();
        if (sc.ref < 0) {                      // no component has generation: nothing to run
            if (tid == 0) {
                const double nan = __longlong_as_double(0x7ff8000000000000ll);
                o.status[s] = 3;
                a.out.opf_iters[s] = 0;
                if (a.out.shed_mw) a.out.shed_mw[s] = B * sc.shed;
                if (a.out.main_klass) a.out.main_klass[s] = CS_OPF_NONCONV;
                if (a.out.max_loading) a.out.max_loading[s] = nan;
                if (a.out.v_margin) a.out.v_margin[s] = nan;
            }
            for (int i = tid; i < nb; i += kThreads) {
                if (a.out.Va) a.out.Va[(size_t)s * nb + i] = 0.0;
                if (a.out.Vm) a.out.Vm[(size_t)s * nb + i] = 0.0;
            }
            __syncthreads();
            continue;
        }
        const Live lv{net, out, W, L, sc.isl};
        const double niq = sc.niq;

        // ---------------- initial point ----------------
        if (tid == 0) {
            sc.gamma = 1.0;
            sc.lref = 0.0;
            sc.fail = 0;
            sc.conv = 0;
        }
        for (int i = tid; i < nb; i += kThreads) {
            W[L.Va + i] = 0.0;
            W[L.Vm + i] = 1.0;
            W[L.lP + i] = 0.0;
            W[L.lQ + i] = 0.0;
        }
        for (int k = tid; k < ng; k += kThreads) {
            const bool off = !lv.gen(k);
            W[L.Pg + k] = off ? 0.0 : 0.5 * (net.pmin[k] + net.pmax[k]);
            W[L.Qg + k] = 0.0;
        }
        __syncthreads();
        const int ops10[10] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 0};
        int it = 0;
        // evaluate(x) then the convergence quantities; init = first call
        auto evaluate = [&](bool init) {
            const double gamma = init ? 1.0 : sc.gamma;
            for (int b = tid; b < nbr; b += kThreads) {
                if (!lv.br(b)) {
                    double* rec = W + L.rec + (size_t)kRec * b;
                    for (int q = 0; q < kRec; ++q) rec[q] = 0.0;
                    W[L.zf + b] = 1.0; W[L.zt + b] = 1.0; W[L.muf + b] = 0.0; W[L.mut + b] = 0.0;
                    W[L.hf + b] = -1.0; W[L.ht + b] = -1.0;
                    continue;
                }
                eval_branch(net, b, W, L, gamma, init);
            }
            __syncthreads();
            // per-thread partial reductions: maxg, maxh, maxx, maxz, maxmu, maxLx, maxlam, sumzmu, cost, nonfinite
            double v[10] = {0.0, -INFINITY, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int b = tid; b < nbr; b += kThreads) {
                if (!lv.br(b)) continue;
                const double zf = W[L.zf + b], zt = W[L.zt + b], mf = W[L.muf + b], mt = W[L.mut + b];
                v[1] = fmax(v[1], fmax(W[L.hf + b], W[L.ht + b]));
                v[3] = fmax(v[3], fmax(zf, zt));
                v[4] = fmax(v[4], fmax(mf, mt));
                v[7] += zf * mf + zt * mt;
            }
            for (int i = tid; i < nb; i += kThreads) {
                if (!lv.bus(i)) {              // outside the main island: no rows, no bounds, load shed
                    if (init) { W[L.zu + i] = 1.0; W[L.zl + i] = 1.0; W[L.muu + i] = 0.0; W[L.mul + i] = 0.0; }
                    W[L.gP + i] = 0.0; W[L.gQ + i] = 0.0; W[L.LxVa + i] = 0.0; W[L.LxVm + i] = 0.0;
                    W[L.NVa + i] = 0.0; W[L.NVm + i] = 0.0; W[L.DP + i] = 0.0; W[L.DQ + i] = 0.0;
                    W[L.rP + i] = 0.0; W[L.rQ + i] = 0.0;
                    continue;
                }
                const double Vm = W[L.Vm + i], Va = W[L.Va + i];
                const double hu = Vm - net.vmax[i], hl = net.vmin[i] - Vm;
                double zu, zl, muu, mul;
                if (init) {
                    zu = fmax(-hu, 1.0); zl = fmax(-hl, 1.0);
                    muu = gamma / zu; mul = gamma / zl;
                    W[L.zu + i] = zu; W[L.zl + i] = zl; W[L.muu + i] = muu; W[L.mul + i] = mul;
                } else {
                    zu = W[L.zu + i]; zl = W[L.zl + i]; muu = W[L.muu + i]; mul = W[L.mul + i];
                }
                const double lP = W[L.lP + i], lQ = W[L.lQ + i];
                double Sre = Vm * Vm * net.gsh[i], Sim = -Vm * Vm * net.bsh[i];
                double LxVa = 0.0, LxVm = 2.0 * Vm * (lP * net.gsh[i] - lQ * net.bsh[i]) + muu - mul;
                double NVa = 0.0, NVm = (muu * hu + gamma) / zu - (mul * hl + gamma) / zl;
                for (int e = net.bus_br_ptr[i]; e < net.bus_br_ptr[i + 1]; ++e) {
                    const int code = net.bus_br[e];
                    const int b = code >> 1, side = code & 1;
                    if (!lv.br(b)) continue;
                    const double* rec = W + L.rec + (size_t)kRec * b;
                    Sre += rec[side ? R_ST : R_SF];
                    Sim += rec[(side ? R_ST : R_SF) + 1];
                    const int p0 = 2 * side;
                    LxVa += rec[R_LG + p0];
                    LxVm += rec[R_LG + p0 + 1];
                    NVa += rec[R_NG + p0];
                    NVm += rec[R_NG + p0 + 1];
                }
                if (i == sc.ref) LxVa += sc.lref;
                double Pgen = 0.0, Qgen = 0.0, DP = 0.0, DQ = 0.0, rP = 0.0, rQ = 0.0;
                for (int e = net.bus_gen_ptr[i]; e < net.bus_gen_ptr[i + 1]; ++e) {
                    const int k = net.bus_gen[e];
                    if (!lv.gen(k)) continue;
                    const double Pg = W[L.Pg + k], Qg = W[L.Qg + k];
                    const double h4[4] = {Pg - net.pmax[k], net.pmin[k] - Pg, Qg - net.qmax[k], net.qmin[k] - Qg};
                    double z4[4], m4[4];
                    for (int q = 0; q < 4; ++q) {
                        if (init) {
                            z4[q] = fmax(-h4[q], 1.0);
                            m4[q] = gamma / z4[q];
                            W[L.gz + 4 * k + q] = z4[q];
                            W[L.gmu + 4 * k + q] = m4[q];
                        } else {
                            z4[q] = W[L.gz + 4 * k + q];
                            m4[q] = W[L.gmu + 4 * k + q];
                        }
                        v[1] = fmax(v[1], h4[q]);
                        v[3] = fmax(v[3], z4[q]);
                        v[4] = fmax(v[4], m4[q]);
                        v[7] += z4[q] * m4[q];
                    }
                    const double PgMW = B * Pg;
                    const double LxP = B * (2.0 * net.c2[k] * PgMW + net.c1[k]) - lP + m4[0] - m4[1];
                    const double LxQ = -lQ + m4[2] - m4[3];
                    const double NP = LxP + (m4[0] * h4[0] + gamma) / z4[0] - (m4[1] * h4[1] + gamma) / z4[1];
                    const double NQ = LxQ + (m4[2] * h4[2] + gamma) / z4[2] - (m4[3] * h4[3] + gamma) / z4[3];
                    const double MP = 2.0 * net.c2[k] * B * B + m4[0] / z4[0] + m4[1] / z4[1];
                    const double MQ = m4[2] / z4[2] + m4[3] / z4[3];
                    W[L.LxP + k] = LxP; W[L.LxQ + k] = LxQ; W[L.NP + k] = NP; W[L.NQ + k] = NQ;
                    W[L.MP + k] = MP; W[L.MQ + k] = MQ;
                    DP += 1.0 / MP;
                    DQ += 1.0 / MQ;
                    rP += NP / MP;
                    rQ += NQ / MQ;
                    Pgen += Pg;
                    Qgen += Qg;
                    v[2] = fmax(v[2], fmax(fabs(Pg), fabs(Qg)));
                    v[5] = fmax(v[5], fmax(fabs(LxP), fabs(LxQ)));
                    v[8] += net.c2[k] * PgMW * PgMW + net.c1[k] * PgMW + net.c0[k];
                }
                NVa += LxVa;
                NVm += LxVm;
                const double gP = Sre - Pgen + Pd[i], gQ = Sim - Qgen + Qd[i];
                W[L.gP + i] = gP; W[L.gQ + i] = gQ;
                W[L.LxVa + i] = LxVa; W[L.LxVm + i] = LxVm; W[L.NVa + i] = NVa; W[L.NVm + i] = NVm;
                W[L.DP + i] = DP; W[L.DQ + i] = DQ; W[L.rP + i] = rP; W[L.rQ + i] = rQ;
                v[0] = fmax(v[0], fmax(fabs(gP), fabs(gQ)));
                v[1] = fmax(v[1], fmax(hu, hl));
                v[2] = fmax(v[2], fmax(fabs(Va), fabs(Vm)));
                v[3] = fmax(v[3], fmax(zu, zl));
                v[4] = fmax(v[4], fmax(muu, mul));
                v[5] = fmax(v[5], fmax(fabs(LxVa), fabs(LxVm)));
                v[6] = fmax(v[6], fmax(fabs(lP), fabs(lQ)));
                v[7] += zu * muu + zl * mul;
                if (!isfinite(gP) || !isfinite(gQ) || !isfinite(NVa) || !isfinite(NVm)) v[9] = 1.0;
            }
            if (tid == 0) v[6] = fmax(v[6], fabs(sc.lref));
            block_reduce<10>(rb, v, ops10, sc.red);
            if (tid == 0) {
                const double maxg = sc.red[0], maxh = sc.red[1], maxx = sc.red[2], maxz = sc.red[3];
                const double maxmu = sc.red[4], maxLx = sc.red[5], maxlam = sc.red[6], zmu = sc.red[7];
                sc.f = sc.red[8];
                if (init) sc.f_prev = sc.f;
                const double feas = fmax(maxg, maxh) / (1.0 + fmax(maxx, maxz));
                const double grad = maxLx / (1.0 + fmax(maxlam, maxmu));
                const double comp = zmu / (1.0 + maxx);
                const double cost = fabs(sc.f - sc.f_prev) / (1.0 + fabs(sc.f_prev));
                if (sc.red[9] != 0.0 || !isfinite(sc.f) || !isfinite(feas) || !isfinite(grad) || !isfinite(comp))
                    sc.fail = 1;
                sc.conv = (feas < tol && grad < tol && comp < tol && cost < tol) ? 1 : 0;
            }
            __syncthreads();
        };

        evaluate(true);

        while (!sc.conv && !sc.fail && it < max_it) {
            ++it;
            const double gamma = sc.gamma;
            // ---------------- assemble the reduced KKT blocks ----------------
            for (int tg = tid; tg < nb + net.nL; tg += kThreads) {
                double blk[16];
                for (int q = 0; q < 16; ++q) blk[q] = 0.0;
                if (tg < nb) {
                    const int j = tg, i = net.perm[j];
                    const double Vm = W[L.Vm + i];
                    double J[2][2] = {{0.0, 2.0 * net.gsh[i] * Vm}, {0.0, -2.0 * net.bsh[i] * Vm}};
                    blk[5] = 2.0 * (W[L.lP + i] * net.gsh[i] - W[L.lQ + i] * net.bsh[i]) +
                             W[L.muu + i] / W[L.zu + i] + W[L.mul + i] / W[L.zl + i];
                    for (int e = net.bus_br_ptr[i]; e < net.bus_br_ptr[i + 1]; ++e) {
                        const int code = net.bus_br[e];
                        const int b = code >> 1, side = code & 1;
                        if (!lv.br(b)) continue;
                        const double* rec = W + L.rec + (size_t)kRec * b;
                        const int p0 = 2 * side;
                        const double* dS = rec + (side ? R_DST : R_DSF);
                        for (int r = 0; r < 2; ++r)
                            for (int c = 0; c < 2; ++c) blk[4 * r + c] += rec[R_H + hidx(p0 + r, p0 + c)];
                        for (int c = 0; c < 2; ++c) {
                            J[0][c] += dS[2 * (p0 + c)];
                            J[1][c] += dS[2 * (p0 + c) + 1];
                        }
                    }
                    for (int q = 0; q < 2; ++q)
                        for (int r = 0; r < 2; ++r) {
                            blk[4 * r + 2 + q] = J[q][r];
                            blk[4 * (2 + q) + r] = J[q][r];
                        }
                    blk[10] = -W[L.DP + i];
                    blk[15] = -W[L.DQ + i];
                    if (i == sc.ref) {
                        for (int q = 0; q < 4; ++q) { blk[q] = 0.0; blk[4 * q] = 0.0; }
                        blk[0] = 1.0;
                    }
                    const bool on = lv.bus(i);
                    if (!on)                   // outside the main island: identity block, zero step
                        for (int q = 0; q < 16; ++q) blk[q] = (q % 5 == 0) ? 1.0 : 0.0;
                    double* D = W + L.Kd + 16 * j;
                    double* Dc = W + L.Db + 16 * j;
                    for (int q = 0; q < 16; ++q) { D[q] = blk[q]; Dc[q] = blk[q]; }
                    double bq[4] = {0.0, 0.0, 0.0, 0.0};
                    if (on) {
                        bq[0] = (i == sc.ref) ? 0.0 : -W[L.NVa + i];
                        bq[1] = -W[L.NVm + i];
                        bq[2] = -W[L.gP + i] - W[L.rP + i];
                        bq[3] = -W[L.gQ + i] - W[L.rQ + i];
                    }
                    for (int q = 0; q < 4; ++q) { W[L.bv + 4 * j + q] = bq[q]; W[L.x + 4 * j + q] = bq[q]; }
                } else {
                    const int q = tg - nb;
                    const int Rn = net.Lrow[q], Cn = net.Lcol[q];
                    const int Rb = net.perm[Rn], Cb = net.perm[Cn];
                    for (int e = net.blk_br_ptr[q]; e < net.blk_br_ptr[q + 1]; ++e) {
                        const int b = net.blk_br[e];
                        if (!lv.br(b)) continue;
                        const double* rec = W + L.rec + (size_t)kRec * b;
                        const bool flip = (net.f[b] != Rb);     // stored block is (t row, f col)
                        double K[16];
                        for (int r = 0; r < 4; ++r)
                            for (int c = 0; c < 4; ++c) {
                                double v;
                                if (r < 2 && c < 2) v = rec[R_H + hidx(r, 2 + c)];
                                else if (r < 2) v = rec[R_DST + 2 * r + (c - 2)];          // J(t,f)^T
                                else if (c < 2) v = rec[R_DSF + 2 * (2 + c) + (r - 2)];    // J(f,t)
                                else v = 0.0;
                                K[4 * r + c] = v;
                            }
                        for (int r = 0; r < 4; ++r)
                            for (int c = 0; c < 4; ++c) blk[4 * r + c] += flip ? K[4 * c + r] : K[4 * r + c];
                    }
                    if (Rb == sc.ref) for (int c = 0; c < 4; ++c) blk[c] = 0.0;
                    if (Cb == sc.ref) for (int r = 0; r < 4; ++r) blk[4 * r] = 0.0;
                    double* U = W + L.Ub + 16 * q;
                    double* Kq = W + L.Kb + 16 * q;
                    for (int c = 0; c < 16; ++c) { U[c] = blk[c]; Kq[c] = blk[c]; }
                }
            }
            __syncthreads();
            // ---------------- block LDL^T, level by level ----------------
            for (int lev = 0; lev < net.nlevels; ++lev) {
                const int t0 = net.tgt_ptr[lev], t1 = net.tgt_ptr[lev + 1], nt = t1 - t0;
                if (nt > 0 && 32 * nt <= kThreads) {
                    // few targets (the top of the elimination tree, where each target has the
                    // longest update lists): S groups of 16 threads per target each sum every
                    // S-th update, then one thread per entry subtracts the S partial sums
                    const int S = kThreads / (16 * nt);
                    if (tid < 16 * nt * S) {
                        const int ti = tid / (16 * S), g = (tid / 16) % S, e = tid & 15;
                        const int tg = net.tgt[t0 + ti];
                        const int r = e >> 2, c = e & 3;
                        double acc = 0.0;
                        for (int u = net.upd_ptr[tg] + g; u < net.upd_ptr[tg + 1]; u += S) {
                            const double* La = W + L.Lb + 16 * net.upd_a[u] + 4 * r;
                            const double* Ubb = W + L.Ub + 16 * net.upd_b[u] + 4 * c;
                            acc += La[0] * Ubb[0] + La[1] * Ubb[1] + La[2] * Ubb[2] + La[3] * Ubb[3];
                        }
                        fsum[tid] = acc;
                    }
                    __syncthreads();
                    if (tid < 16 * nt) {
                        const int ti = tid >> 4, e = tid & 15;
                        const int tg = net.tgt[t0 + ti];
                        double* A = (tg < nb) ? (W + L.Db + 16 * tg) : (W + L.Ub + 16 * (tg - nb));
                        double part = 0.0;
                        for (int g = 0; g < S; ++g) part += fsum[ti * 16 * S + g * 16 + e];
                        A[e] -= part;
                    }
                } else {
                    for (int w = tid; w < 16 * nt; w += kThreads) {
                        const int tg = net.tgt[t0 + (w >> 4)];
                        const int r = (w & 15) >> 2, c = w & 3;
                        double* A = (tg < nb) ? (W + L.Db + 16 * tg) : (W + L.Ub + 16 * (tg - nb));
                        double acc = A[4 * r + c];
                        for (int u = net.upd_ptr[tg]; u < net.upd_ptr[tg + 1]; ++u) {
                            const double* La = W + L.Lb + 16 * net.upd_a[u] + 4 * r;
                            const double* Ubb = W + L.Ub + 16 * net.upd_b[u] + 4 * c;
                            acc -= La[0] * Ubb[0] + La[1] * Ubb[1] + La[2] * Ubb[2] + La[3] * Ubb[3];
                        }
                        A[4 * r + c] = acc;
                    }
                }
                __syncthreads();
                {
                    const int c0 = net.lev_ptr[lev], nc = net.lev_ptr[lev + 1] - c0;
                    for (int w = tid; w < 4 * nc; w += kThreads) {     // four lanes per pivot
                        const int j = net.lev_col[c0 + (w >> 2)];
                        if (!inv4(W + L.Db + 16 * j, W + L.Di + 16 * j, w & 3)) sc.fail = 1;
                    }
                }
                __syncthreads();
                for (int w = tid; w < 16 * (t1 - t0); w += kThreads) {
                    const int tg = net.tgt[t0 + (w >> 4)];
                    if (tg < nb) continue;
                    const int q = tg - nb;
                    const int r = (w & 15) >> 2, c = w & 3;
                    const double* U = W + L.Ub + 16 * q + 4 * r;
                    const double* Di = W + L.Di + 16 * net.Lcol[q] + c;
                    W[L.Lb + 16 * q + 4 * r + c] = U[0] * Di[0] + U[1] * Di[4] + U[2] * Di[8] + U[3] * Di[12];
                }
                __syncthreads();
            }
            if (sc.fail) break;
            // ---------------- solve, then FP64 iterative refinement against the assembled K ----------------
            // The blocks are eliminated in a fixed order without pivoting between blocks;
            // near convergence some pivot blocks become nearly singular (a load bus whose
            // voltage sits at a bound has one free local variable for two balance rows),
            // which leaves a low-rank error in the first solve that refinement removes.
            // Refinement stops once the componentwise backward error is at rounding level.
            ldl_solve(net, W, L, W + L.x);
            for (int ref_step = 0;; ++ref_step) {
                double v1[1] = {kkt_residual(net, W, L, W + L.x, W + L.rv)};
                const int ops1[1] = {0};
                block_reduce<1>(rb, v1, ops1, sc.red);
                if (sc.red[0] <= kRefineTol || ref_step == kRefineSteps) break;   // NaN: refine, then caught below
                ldl_solve(net, W, L, W + L.rv);
                for (int w = tid; w < 4 * nb; w += kThreads) W[L.x + w] += W[L.rv + w];
                __syncthreads();
            }
            if (!(sc.red[0] <= kBackwardTol)) {
                // Krylov steps on the factors, then, if those stall, the dense backstop
                __shared__ GmresShared gs;
                const double om = kkt_gmres(net, W, L, rb, sc.red, gs, sc.red[0]);
                if (L.dense >= 0 && !(om <= kBackwardTol)) {
                    __shared__ DenseShared ds;
                    if (!dense_solve(net, W, L, ds)) sc.fail = 1;
                    __syncthreads();
                    if (sc.fail) break;
                    // FP64 refinement of the backstop's solution with its own factors; the
                    // best iterate is kept (refinement diverges on a system too ill-conditioned
                    // for FP64, and then the backstop's first solution is the best there is)
                    double best = INFINITY;
                    for (int ref_step = 0;; ++ref_step) {
                        double v1[1] = {kkt_residual(net, W, L, W + L.x, W + L.rv)};
                        const int ops1[1] = {0};
                        block_reduce<1>(rb, v1, ops1, sc.red);
                        const double om_now = sc.red[0];
                        if (ref_step > 0 && !(om_now < best)) {          // no progress: back to the best
                            for (int w = tid; w < 4 * nb; w += kThreads) W[L.x + w] = W[L.gxb + w];
                            __syncthreads();
                            break;
                        }
                        best = om_now;
                        if (om_now <= kRefineTol || ref_step == kRefineSteps) break;
                        for (int w = tid; w < 4 * nb; w += kThreads) W[L.gxb + w] = W[L.x + w];
                        dense_resolve(net, W, L, W + L.rv);
                        for (int w = tid; w < 4 * nb; w += kThreads) W[L.x + w] += W[L.rv + w];
                        __syncthreads();
                    }
                }
            }
            // ---------------- recover the eliminated steps, dz, dmu, ratios ----------------
            double rp = INFINITY, rd = INFINITY, bad = 0.0;
            for (int k = tid; k < ng; k += kThreads) {
                if (!lv.gen(k)) continue;
                const int jn = net.iperm[net.gbus[k]];
                const double dlP = W[L.x + 4 * jn + 2], dlQ = W[L.x + 4 * jn + 3];
                const double dPg = (-W[L.NP + k] + dlP) / W[L.MP + k];
                const double dQg = (-W[L.NQ + k] + dlQ) / W[L.MQ + k];
                W[L.dPg + k] = dPg;
                W[L.dQg + k] = dQg;
                const double Pg = W[L.Pg + k], Qg = W[L.Qg + k];
                const double h4[4] = {Pg - net.pmax[k], net.pmin[k] - Pg, Qg - net.qmax[k], net.qmin[k] - Qg};
                const double dh4[4] = {dPg, -dPg, dQg, -dQg};
                for (int q = 0; q < 4; ++q) {
                    const double z = W[L.gz + 4 * k + q], m = W[L.gmu + 4 * k + q];
                    const double dz = -h4[q] - z - dh4[q];
                    const double dm = -m + (gamma - m * dz) / z;
                    W[L.gdz + 4 * k + q] = dz;
                    W[L.gdmu + 4 * k + q] = dm;
                    if (dz < 0.0) rp = fmin(rp, -z / dz);
                    if (dm < 0.0) rd = fmin(rd, -m / dm);
                    if (!isfinite(dz) || !isfinite(dm)) bad = 1.0;
                }
            }
            for (int b = tid; b < nbr; b += kThreads) {
                if (!lv.br(b)) continue;
                const double* rec = W + L.rec + (size_t)kRec * b;
                const int fn = net.iperm[net.f[b]], tn = net.iperm[net.t[b]];
                const double dx[4] = {W[L.x + 4 * fn], W[L.x + 4 * fn + 1], W[L.x + 4 * tn], W[L.x + 4 * tn + 1]};
                double gdf = 0.0, gdt = 0.0;
                for (int p = 0; p < 4; ++p) {
                    gdf += rec[R_GF + p] * dx[p];
                    gdt += rec[R_GT + p] * dx[p];
                }
                const double zf = W[L.zf + b], zt = W[L.zt + b], mf = W[L.muf + b], mt = W[L.mut + b];
                const double dzf = -W[L.hf + b] - zf - gdf, dzt = -W[L.ht + b] - zt - gdt;
                const double dmf = -mf + (gamma - mf * dzf) / zf, dmt = -mt + (gamma - mt * dzt) / zt;
                W[L.dzf + b] = dzf; W[L.dzt + b] = dzt; W[L.dmuf + b] = dmf; W[L.dmut + b] = dmt;
                if (dzf < 0.0) rp = fmin(rp, -zf / dzf);
                if (dzt < 0.0) rp = fmin(rp, -zt / dzt);
                if (dmf < 0.0) rd = fmin(rd, -mf / dmf);
                if (dmt < 0.0) rd = fmin(rd, -mt / dmt);
                if (!isfinite(dzf) || !isfinite(dzt) || !isfinite(dmf) || !isfinite(dmt)) bad = 1.0;
            }
            for (int i = tid; i < nb; i += kThreads) {
                if (!lv.bus(i)) continue;
                const int jn = net.iperm[i];
                const double dVm = W[L.x + 4 * jn + 1];
                const double Vm = W[L.Vm + i];
                const double hu = Vm - net.vmax[i], hl = net.vmin[i] - Vm;
                const double zu = W[L.zu + i], zl = W[L.zl + i], mu_ = W[L.muu + i], ml = W[L.mul + i];
                const double dzu = -hu - zu - dVm, dzl = -hl - zl + dVm;
                const double dmu = -mu_ + (gamma - mu_ * dzu) / zu, dml = -ml + (gamma - ml * dzl) / zl;
                W[L.dzu + i] = dzu; W[L.dzl + i] = dzl; W[L.dmuu + i] = dmu; W[L.dmul + i] = dml;
                if (dzu < 0.0) rp = fmin(rp, -zu / dzu);
                if (dzl < 0.0) rp = fmin(rp, -zl / dzl);
                if (dmu < 0.0) rd = fmin(rd, -mu_ / dmu);
                if (dml < 0.0) rd = fmin(rd, -ml / dml);
                for (int r = 0; r < 4; ++r)
                    if (!isfinite(W[L.x + 4 * jn + r])) bad = 1.0;
            }
            if (tid == 0) {
                // multiplier step of the reference-angle row from its Newton row
                const int i = sc.ref;
                double row = 0.0;
                for (int e = net.bus_br_ptr[i]; e < net.bus_br_ptr[i + 1]; ++e) {
                    const int code = net.bus_br[e];
                    const int b = code >> 1, side = code & 1;
                    if (!lv.br(b)) continue;
                    const double* rec = W + L.rec + (size_t)kRec * b;
                    const int fn = net.iperm[net.f[b]], tn = net.iperm[net.t[b]];
                    const double dx[4] = {W[L.x + 4 * fn], W[L.x + 4 * fn + 1], W[L.x + 4 * tn], W[L.x + 4 * tn + 1]};
                    const int p = 2 * side;
                    for (int q = 0; q < 4; ++q) row += rec[R_H + hidx(p, q)] * dx[q];
                    row += rec[R_DSF + 2 * p] * W[L.x + 4 * fn + 2] + rec[R_DSF + 2 * p + 1] * W[L.x + 4 * fn + 3];
                    row += rec[R_DST + 2 * p] * W[L.x + 4 * tn + 2] + rec[R_DST + 2 * p + 1] * W[L.x + 4 * tn + 3];
                }
                sc.dlref = -W[L.NVa + i] - row;
            }
            {
                double v3[3] = {rp, rd, bad};
                const int ops3[3] = {2, 2, 0};
                block_reduce<3>(rb, v3, ops3, sc.red);
            }
            if (tid == 0) {
                sc.ap = fmin(kXi * sc.red[0], 1.0);
                sc.ad = fmin(kXi * sc.red[1], 1.0);
                if (sc.red[2] != 0.0 || !isfinite(sc.dlref)) sc.fail = 1;
            }
            __syncthreads();
            if (sc.fail) break;
            // ---------------- update ----------------
            const double ap = sc.ap, ad = sc.ad;
            double zmu = 0.0;
            for (int i = tid; i < nb; i += kThreads) {
                if (!lv.bus(i)) continue;
                const int jn = net.iperm[i];
                W[L.Va + i] += ap * W[L.x + 4 * jn];
                W[L.Vm + i] += ap * W[L.x + 4 * jn + 1];
                W[L.lP + i] += ad * W[L.x + 4 * jn + 2];
                W[L.lQ + i] += ad * W[L.x + 4 * jn + 3];
                const double zu = W[L.zu + i] + ap * W[L.dzu + i], zl = W[L.zl + i] + ap * W[L.dzl + i];
                const double mu_ = W[L.muu + i] + ad * W[L.dmuu + i], ml = W[L.mul + i] + ad * W[L.dmul + i];
                W[L.zu + i] = zu; W[L.zl + i] = zl; W[L.muu + i] = mu_; W[L.mul + i] = ml;
                zmu += zu * mu_ + zl * ml;
            }
            for (int k = tid; k < ng; k += kThreads) {
                if (!lv.gen(k)) continue;
                W[L.Pg + k] += ap * W[L.dPg + k];
                W[L.Qg + k] += ap * W[L.dQg + k];
                for (int q = 0; q < 4; ++q) {
                    const double z = W[L.gz + 4 * k + q] + ap * W[L.gdz + 4 * k + q];
                    const double m = W[L.gmu + 4 * k + q] + ad * W[L.gdmu + 4 * k + q];
                    W[L.gz + 4 * k + q] = z;
                    W[L.gmu + 4 * k + q] = m;
                    zmu += z * m;
                }
            }
            for (int b = tid; b < nbr; b += kThreads) {
                if (!lv.br(b)) continue;
                const double zf = W[L.zf + b] + ap * W[L.dzf + b], zt = W[L.zt + b] + ap * W[L.dzt + b];
                const double mf = W[L.muf + b] + ad * W[L.dmuf + b], mt = W[L.mut + b] + ad * W[L.dmut + b];
                W[L.zf + b] = zf; W[L.zt + b] = zt; W[L.muf + b] = mf; W[L.mut + b] = mt;
                zmu += zf * mf + zt * mt;
            }
            {
                double v1[1] = {zmu};
                const int ops1[1] = {1};
                block_reduce<1>(rb, v1, ops1, sc.red);
            }
            if (tid == 0) {
                sc.lref += ad * sc.dlref;
                sc.gamma = kSigma * sc.red[0] / niq;
                sc.f_prev = sc.f;
            }
            __syncthreads();
            evaluate(false);
        }
        // ---------------- outputs ----------------
        double viol = 0.0, load_max = 0.0, vmarg = INFINITY;
        const bool converged = sc.conv && !sc.fail;
        if (converged) {
            for (int b = tid; b < nbr; b += kThreads) {
                if (!lv.br(b)) continue;
                const double sm = sqrt(net.smax2[b]);
                const double sf = sqrt(fmax(W[L.hf + b] + net.smax2[b], 0.0));
                const double st = sqrt(fmax(W[L.ht + b] + net.smax2[b], 0.0));
                if (sf - sm > kLimitTol || st - sm > kLimitTol) viol = 1.0;
                load_max = fmax(load_max, fmax(sf, st) / sm);
            }
            for (int i = tid; i < nb; i += kThreads) {
                if (!lv.bus(i)) continue;
                const double Vm = W[L.Vm + i];
                if (Vm - net.vmax[i] > kLimitTol || net.vmin[i] - Vm > kLimitTol) viol = 1.0;
                vmarg = fmin(vmarg, fmin(Vm - net.vmin[i], net.vmax[i] - Vm));
            }
            for (int k = tid; k < ng; k += kThreads) {
                if (!lv.gen(k)) continue;
                const double Pg = W[L.Pg + k], Qg = W[L.Qg + k];
                if (Pg - net.pmax[k] > kLimitTol || net.pmin[k] - Pg > kLimitTol ||
                    Qg - net.qmax[k] > kLimitTol || net.qmin[k] - Qg > kLimitTol) viol = 1.0;
            }
        }
        {
            double v3[3] = {viol, load_max, vmarg};   // non-binary severity: loading, voltage margin
            const int ops3[3] = {0, 0, 2};
            block_reduce<3>(rb, v3, ops3, sc.red);
        }
        double* xs = o.x + (size_t)s * nx;
        for (int i = tid; i < nb; i += kThreads) {
            // a bus outside the main island is de-energised: Vm = 0 also tells the
            // small-signal kernels which buses are out
            const bool on = lv.bus(i);
            xs[i] = on ? W[L.Va + i] : 0.0;
            xs[nb + i] = on ? W[L.Vm + i] : 0.0;
            if (a.out.Va) a.out.Va[(size_t)s * nb + i] = xs[i];
            if (a.out.Vm) a.out.Vm[(size_t)s * nb + i] = xs[nb + i];
        }
        for (int k = tid; k < ng; k += kThreads) {
            xs[2 * nb + k] = W[L.Pg + k];
            xs[2 * nb + ng + k] = W[L.Qg + k];
        }
        if (tid == 0) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            a.out.opf_iters[s] = (int16_t)it;
            a.out.cost[s] = converged ? sc.f : nan;
            if (a.out.max_loading) a.out.max_loading[s] = converged ? sc.red[1] : nan;
            if (a.out.v_margin) a.out.v_margin[s] = converged ? sc.red[2] : nan;
            if (isl) {                         // main island of an islanded scenario: class unchanged
                const bool ok = converged && sc.red[0] == 0.0;
                o.status[s] = ok ? 1 : 3;      // within limits: on to the small-signal screen, which sets main_klass
                if (a.out.shed_mw) a.out.shed_mw[s] = B * sc.shed;
                if (a.out.main_klass && !ok) a.out.main_klass[s] = converged ? CS_LIMIT : CS_OPF_NONCONV;
            } else if (!converged || sc.red[0] != 0.0) {
                o.status[s] = 2;
                a.out.klass[s] = converged ? CS_LIMIT : CS_OPF_NONCONV;
                a.out.severe[s] = 1;
                a.out.max_re[s] = nan;
                a.out.min_zeta[s] = nan;
            } else {
                o.status[s] = 1;
            }
        }
        __syncthreads();
    }
}

}  // namespace

int opf_ctas_per_sm() { return kCtasPerSm; }

size_t opf_scratch_doubles(const DevNet& net) { return (size_t)make_layout(net).total; }

cudaError_t launch_opf(const DevNet& net, const EvalArgs& a, const int* islanded, OpfOut o, double tol,
                       int max_it, double* scratch, size_t scratch_per_cta, int grid, int* counter,
                       cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const Lay L = make_layout(net);
    if ((size_t)L.total > scratch_per_cta) return cudaErrorInvalidValue;
    opf_kernel<<<grid, kThreads, 0, s>>>(net, a, islanded, o, tol, max_it, scratch, scratch_per_cta, L, counter);
    return cudaGetLastError();
}
