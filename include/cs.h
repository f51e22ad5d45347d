/* cs.h -- C ABI of libcs: GB300-native N-2 contingency screening with a
 * probabilistic Risk Index.
 *
 * Method (arXiv 2512.08465): every contingency scenario -- one or two failed
 * lines, transformers or generators -- is screened by three checks (Section
 * II-B): islanding (II-B-3), AC optimal power flow feasibility and operational
 * limits (II-B-1), and small-signal stability of the linearised state matrix
 * (II-B-2).  The binary severities are reduced into each component's Risk Index
 * R_i = F_i S_i + sum_{j != i} F_ij S_ij (Section II-C, Eq. 1-3).
 *
 * Conventions for every entry point:
 *  - No exceptions cross the ABI; every call returns a cs_status.
 *  - The library never keeps a caller pointer after the call returns.  Host
 *    buffers are read or written before return; device buffers passed to the
 *    *_device entry points are used asynchronously on the given CUDA stream and
 *    must stay valid until that stream reaches the point of the call.
 *  - Element ids: [0, n_branch) are branches, [n_branch, n_branch + n_gen) are
 *    generators (Section II-A: lines, transformers, generators).
 *  - One cs_ctx is used by one host thread at a time (calls on one ctx are
 *    serialised by an internal mutex; distinct ctx objects are independent).
 *  - On error the message of the last failing call on that ctx is available
 *    from cs_last_error().
 */
#ifndef CS_H
#define CS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cs_status;
enum {
    CS_OK = 0,
    CS_PENDING = 1,            /* cs_poll: the request has not finished yet */
    CS_E_ARG = -1,             /* invalid argument (sizes, ids, ranges, NULL) */
    CS_E_NOMEM = -2,           /* allocation failed, or opt.hbm_budget would be exceeded */
    CS_E_BASE_INSECURE = -3,   /* base case not secure and the options require it */
    CS_E_TIMEOUT = -4,         /* a bounded device wait gave up */
    CS_E_CUDA = -5,            /* a CUDA runtime call failed */
    CS_E_UNKNOWN_ID = -6,      /* unknown network or request id */
    CS_E_NUMERIC = -7          /* a kernel reported an internal inconsistency */
};

/* Severity classes (Section II-B).  S = 1 for every class except CS_SECURE. */
enum {
    CS_SECURE = 0,
    CS_ISLANDED = 1,           /* more than one island (Section II-B-3) */
    CS_OPF_NONCONV = 2,        /* OPF did not converge or hit a non-finite value (II-B-1) */
    CS_LIMIT = 3,              /* converged OPF violates an operational limit (II-B-1) */
    CS_SS_UNSTABLE = 4,        /* an eigenvalue with non-negative real part (II-B-2) */
    CS_SS_POORLY_DAMPED = 5,   /* minimum damping ratio below damping_min */
    CS_EIG_FAIL = 6            /* the eigenvalue iteration did not converge */
};

/* Risk Index pair readings (Section II-C).  EQ3 counts every unordered pair
 * once, as Eq. 3 is written; ORDERED counts both orderings of the ordered N-2
 * enumeration of Section II-A, which reproduces the values printed in
 * Section V (1.472 for a line with every scenario severe under Table I). */
enum { CS_RISK_EQ3 = 0, CS_RISK_ORDERED = 1 };

/* Precision forms.  FP64: every step in FP64.  MIXED: the eigenvalue screen
 * (balancing, Hessenberg reduction, QR) runs in FP32; the eigenvalues that can
 * carry max Re or min zeta are then refined in FP64 (two-sided Rayleigh quotient
 * with the FP64 state matrix) and decide the class.  The whole screen is re-run
 * in FP64 when the FP32 iteration fails, a refinement is ill-conditioned, or a
 * refined statistic lies within 1e-7 of its threshold (|max Re| or |min zeta -
 * damping_min|).  Classes are those of the FP64 form and max_re / min_zeta
 * agree with it to about 1e-9.  (Networks whose Hessenberg matrix exceeds one
 * block's shared memory, state order above ~300, run the FP32 screen in global
 * memory without the refinement, re-run in FP64 within 5e-3 of a threshold:
 * FP32 error outside that band.)  The OPF stays in FP64 in both forms: FP32
 * factors of its Newton systems do not reach the backward-error target. */
enum { CS_PREC_FP64 = 0, CS_PREC_MIXED = 1 };

typedef struct cs_ctx cs_ctx;

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    double damping_min;        /* damping-ratio threshold; 0 = Re >= 0 rule only (II-B-2) */
    double opf_tol;            /* interior-point stopping tolerance (all four conditions) */
    int32_t opf_max_it;        /* interior-point iteration cap */
    int32_t require_secure_base; /* 1: cs_load_network fails with CS_E_BASE_INSECURE */
    int32_t ctas_per_sm;       /* resident scenario blocks per SM; 0 = automatic */
    int32_t chunk;             /* scenarios per internal batch; 0 = automatic (8192, fewer where a
                                  network's workspaces would pass ~6 GB) */
    int32_t precision;         /* CS_PREC_FP64 (default) or CS_PREC_MIXED */
    int64_t hbm_budget;        /* device bytes the context may hold (networks, workspaces,
                                  request buffers); 0 = no limit */
    int32_t serve_slots;       /* batches in flight on the serving path (1..8, default 3) */
    int32_t batch_cap;         /* scenarios per serving batch (default 4096; larger requests are
                                  split over batches) */
    int32_t main_island;       /* 1: an islanded scenario also gets the OPF of its main island
                                  (see cs_result.main_klass); 0 (default): not run, as in the paper */
    int32_t autotune;          /* 1: cs_load_network times the launch shapes of the persistent
                                  kernels (resident OPF blocks per SM, resident small-signal blocks
                                  per SM) on a sample of the network's N-2 pairs and keeps the
                                  fastest for that network (cs_network_stats reports it); results
                                  do not depend on the shape.  0 (default): fixed shapes.  Ignored
                                  when ctas_per_sm is set. */
} cs_options;

/* Fills *opt with the defaults (damping_min 0.05, opf_tol 1e-8, opf_max_it 50,
 * FP64 form, no device-memory budget, 3 serving slots, batches of 4096, no
 * main-island OPF, no autotuning). */
void cs_default_options(cs_options* opt);

/* Raw network data in structure-of-arrays form, host memory, copied by
 * cs_load_network (the caller keeps ownership).  Units: MW / MVAr / MVA for
 * powers, per unit on base_mva for impedances and voltages, $/MW^2h and $/MWh
 * for costs, machine base (MVA = Pmax) for machine reactances, H and D. */
typedef struct {
    int32_t n_bus, n_branch, n_gen, n_levels, ref_bus;
    double base_mva, f_hz;
    const double *Vmin, *Vmax, *Gs, *Bs;          /* [n_bus] */
    const double *Pd, *Qd;                        /* [n_levels * n_bus], level-major */
    const int32_t *f, *t;                         /* [n_branch] bus indices */
    const double *r, *x, *b, *rate, *tap;         /* [n_branch] */
    const int32_t* gbus;                          /* [n_gen] */
    const double *Pmin, *Pmax, *Qmin, *Qmax;      /* [n_gen] MW / MVAr */
    const double *c2, *c1, *c0;                   /* [n_gen] */
    const double *H, *D, *xd, *xq, *xdp;          /* [n_gen] machine base */
    const double *Td0p, *Tq0p, *KA, *TA;          /* [n_gen] seconds / gain */
    int32_t opf_max_it;                           /* this network's interior-point iteration cap
                                                     (0..10000); 0 = the context's opf_max_it */
} cs_network_desc;

/* Per-scenario results, structure of arrays with n records.  Which memory
 * (device or host) each entry point expects is stated at the entry point.
 * Vm / Va, v_margin / max_loading, shed_mw / main_klass are optional (NULL = not
 * written; the request path cs_poll returns every field but Vm / Va). */
typedef struct {
    uint8_t* klass;            /* CS_SECURE .. CS_EIG_FAIL */
    uint8_t* severe;           /* S_c in {0, 1} */
    int16_t* n_islands;        /* number of islands of the post-contingency network */
    int16_t* opf_iters;        /* interior-point iterations taken (0 if not run) */
    double* cost;              /* OPF cost, $/h (NaN if not converged) */
    double* max_re;            /* largest real part, structural zero mode removed (NaN if not run) */
    double* min_zeta;          /* smallest damping ratio (NaN if not run) */
    double* Vm;                /* optional [n * n_bus] */
    double* Va;                /* optional [n * n_bus] */
    /* optional non-binary severity of the converged OPF point (an extension named in
     * the paper's outlook, Section VI; NULL = not written, NaN when the OPF did not
     * converge or was not run): */
    double* v_margin;          /* min over buses of min(Vm - Vmin, Vmax - Vm), p.u. */
    double* max_loading;       /* max over in-service branch ends of |S| / Smax */
    /* optional main-island result of an islanded scenario (NULL = not written).  Section II-A
     * takes the island tied to the largest generation as the reference once a network
     * splits, Section V-A ties most failed cases to an isolated slack bus and Section VI
     * names load shed as a severity; with cs_options.main_island = 1 an islanded scenario
     * (klass and severe stay CS_ISLANDED and 1) gets the OPF of its main island: the
     * component whose in-service generators have the largest total Pmax (equal totals:
     * the component of the lowest-numbered bus), with the reference bus moved to the
     * island's largest in-service unit (lowest index among equals) when the original one
     * lies outside.  opf_iters, cost, v_margin, max_loading, Vm and Va then describe that
     * OPF (Vm = Va = 0 at buses outside the main island), and max_re / min_zeta the
     * small-signal screen of the main island (its in-service units, angles referred to the
     * first of them) when its OPF converged within every limit. */
    double* shed_mw;           /* active load outside the main island, MW (0 if not islanded,
                                  NaN if islanded and main_island = 0) */
    uint8_t* main_klass;       /* class of the main island with the precedence of Section II-B:
                                  CS_OPF_NONCONV (also: no component has generation), CS_LIMIT,
                                  CS_EIG_FAIL, CS_SS_UNSTABLE, CS_SS_POORLY_DAMPED or CS_SECURE;
                                  255 if not islanded or main_island = 0 */
} cs_result;

/* Create / destroy a context on opt->device (NULL = defaults).  cs_create
 * fails with CS_E_CUDA when no usable CUDA device is present. */
cs_status cs_create(const cs_options* opt, cs_ctx** out);
cs_status cs_destroy(cs_ctx* ctx);

/* Copy a network to the device and prepare it (Section II-A step 1): the
 * symbolic analysis of the bus-level KKT and admittance patterns (one
 * minimum-degree ordering and elimination tree reused by every scenario of the
 * network), the static device data, and the base case of every load level.
 * The network stays resident until cs_unload_network.  Fails with CS_E_ARG on
 * inconsistent sizes or indices, CS_E_BASE_INSECURE when a base case is not
 * secure and opt.require_secure_base is set. */
cs_status cs_load_network(cs_ctx* ctx, const cs_network_desc* net, int32_t* net_id);

/* The descriptor checks cs_load_network applies, on their own: HOST only, no
 * context and no device.  CS_OK, or CS_E_ARG with a message naming the first
 * offending entry (NULL array, sizes, an index out of range or a self loop, a
 * non-finite load, shunt, impedance, tap, limit, cost or machine constant, a zero
 * series impedance, a non-positive rating, tap, Pmax or time constant, Vmin <= 0
 * or Vmin > Vmax, Pmin > Pmax, Qmin > Qmax, c2 < 0, D < 0) written to msg (at most
 * msg_len bytes with its terminating zero; msg may be NULL). */
cs_status cs_check_network(const cs_network_desc* net, char* msg, int32_t msg_len);
cs_status cs_unload_network(cs_ctx* ctx, int32_t net_id);

/* Sizes of a loaded network and of its symbolic analysis (Section II-A step 1),
 * for work accounting: stats[0..7] = n_bus, n_branch, n_gen, off-diagonal
 * 4x4 blocks of L (and of the bus-level KKT pattern below the diagonal),
 * block updates of one numeric factorisation, elimination-tree levels,
 * largest state-matrix order (5 n_gen - 1), load levels, then the launch shape
 * the network's evaluations use: resident OPF blocks per SM, resident
 * small-signal blocks per SM, 1 if the autotuner chose them (0 if they are
 * the defaults or ctas_per_sm), and the network's interior-point iteration
 * cap (stats[11]).  The first n_stats
 * entries are written (HOST array). */
cs_status cs_network_stats(cs_ctx* ctx, int32_t net_id, int64_t* stats, int32_t n_stats);

/* The symbolic analysis a loaded network gets (cs_load_network), on its own:
 * HOST only, no context and no device.  Every scenario's Newton system (4x4
 * blocks per bus, Section II-B-1) and the small-signal model's network matrix
 * (Section II-B-2) have the bus graph with every branch in service as block
 * pattern, an outage only zeroing values, so one ordering and one fill pattern
 * serve all contingencies.  The paper has no counterpart (it calls external
 * solvers); this entry point exposes the analysis for inspection and testing.
 *   n_bus, n_branch, f[k], t[k]: the bus graph (HOST arrays; parallel branches
 *     allowed, self loops rejected); ref_bus: eliminated last (-1: none);
 *   perm[n_bus]: elimination order, perm[new] = old bus (exact minimum degree on
 *     the elimination graph, ties to the smaller bus index);
 *   col_ptr[n_bus + 1], row[cap]: rows (new indices, ascending, all below the
 *     diagonal) of each column's off-diagonal blocks of L, CSC;
 *   level[n_bus]: elimination-tree height of each column (new index); the
 *     columns of one height are independent and form one parallel step;
 *   stats[0..3]: off-diagonal blocks of L, levels, block updates of one numeric
 *     factorisation, the capacity row needs.
 * Every output pointer may be NULL (skipped).  CS_E_ARG: sizes or ends out of
 * range, a self loop, a NULL edge array, or cap below stats[3] (the other
 * outputs are then written). */
cs_status cs_symbolic_pattern(int32_t n_bus, int32_t n_branch, const int32_t* f, const int32_t* t,
                              int32_t ref_bus, int32_t* perm, int32_t* col_ptr, int32_t* row, int64_t cap,
                              int32_t* level, int64_t* stats);

/* Base-case result of a level (host out, one record). */
cs_status cs_base_result(cs_ctx* ctx, int32_t net_id, int32_t level, const cs_result* out);

/* Evaluate n scenarios of (net_id, level) with DEVICE buffers: elem_i, elem_j
 * [n] int32 (elem_j = -1 gives an N-1 scenario, elem_i = elem_j = -1 the base
 * case), out fields device pointers of n records.  Asynchronous on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  Every severity is also
 * recorded in the context's severity table of (net_id, level) that
 * cs_risk_index reads.  Sizes and ids are validated: n, net_id and level on
 * the host (CS_E_ARG); element ids on the device.  A record whose ids are out
 * of range (below -1, at or above n_branch + n_gen, or elem_i = -1 with
 * elem_j >= 0) gets class 255, severe = 1, NaN cost and eigen statistics, is
 * not written to the severity table, and sets a device error bit that the
 * next cs_sync reports as CS_E_ARG.  The other records are unaffected.  Every
 * step runs in the library's kernels: islanding, the interior-point OPF, the
 * dynamic model + eigenvalues and the classification (Section II-B). */
cs_status cs_evaluate_device(cs_ctx* ctx, int32_t net_id, int32_t level,
                             const int32_t* elem_i, const int32_t* elem_j, int64_t n,
                             const cs_result* out, void* stream);

/* Wait for all work of the context on `stream` and report device-side errors
 * (invalid element ids, bounded-wait time-outs). */
cs_status cs_sync(cs_ctx* ctx, void* stream);

/* Non-blocking submission with HOST buffers (copied before return); the
 * serving path.  A scheduler thread of the context batches queued requests
 * continuously: whenever one of opt.serve_slots streams (each with its own
 * workspace) is free, it fills a batch of at most opt.batch_cap scenarios with
 * the oldest request's next scenarios and those of every later queued request
 * for the same (net_id, level), in arrival order; a request that does not fit
 * what is left of the batch is split, the rest waiting for the next free slot.
 * Batches of different networks run side by side, and a request arriving while
 * others run starts within about one batch time.  A request completes when its
 * last slice is back.  A batch starts only when
 * its device footprint fits opt.hbm_budget next to everything the context
 * holds (its chunk shrinks first, then it waits for a running batch).
 * Severities are recorded in the context's severity tables as for
 * cs_evaluate_device.  cs_poll retrieves the results. */
cs_status cs_submit_contingencies(cs_ctx* ctx, int32_t net_id, int32_t level,
                                  const int32_t* elem_i, const int32_t* elem_j, int64_t n,
                                  uint64_t* request_id);

/* Copy the results of a finished request into the HOST record `out` (n
 * records of the request; NULL fields are skipped, Vm/Va are not returned on
 * this path).  Waits at most timeout_us microseconds (0 = just test); returns
 * CS_PENDING if the request is still queued or running.  A finished request
 * is released by the successful poll; a failed one returns its error
 * (CS_E_NOMEM when its batch cannot fit opt.hbm_budget) and is released. */
cs_status cs_poll(cs_ctx* ctx, uint64_t request_id, int32_t timeout_us, const cs_result* out);

/* Counters of the serving path (no counterpart in the paper): stats[0..8] =
 * batches launched, requests completed, requests that joined another
 * request's batch, batch starts deferred by the memory budget, requests failed
 * for memory, peak device bytes held, device bytes held now, requests queued,
 * batches in flight.  The first n_stats entries are written (HOST array). */
cs_status cs_serving_stats(cs_ctx* ctx, int64_t* stats, int32_t n_stats);

/* Risk Index (Section II-C, Eq. 3) of every element from the context's
 * severity table of (net_id, level): R_i = lambda_i S_i + m * sum_j
 * fl(lambda_i lambda_j) S_ij with m = 1 (CS_RISK_EQ3) or 2 (CS_RISK_ORDERED).
 * The sum is accumulated exactly in 192-bit fixed point and rounded once to
 * the nearest double, so the result is independent of evaluation order.
 * lambda, R_out: HOST arrays of n_branch + n_gen doubles.  lambda must lie in
 * [2^-30, 2^10] (CS_E_ARG otherwise).  N-1 scenarios and pairs never evaluated
 * contribute 0 and are counted in *n_missing (may be NULL). */
cs_status cs_risk_index(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda,
                        int32_t mode, double* R_out, int64_t* n_missing);

/* Stateless device form of the same reduction: S1 [E] uint8 N-1 severities,
 * S2 [E*(E-1)/2] uint8 severities of the unordered pairs i < j in
 * lexicographic order, lambda and R [E] doubles; all DEVICE pointers,
 * asynchronous on `stream`.  Range of lambda as above (checked on the host
 * copy by cs_risk_index only; here out-of-range values give NaN). */
cs_status cs_risk_reduce_device(int32_t n_elem, const uint8_t* S1, const uint8_t* S2,
                                const double* lambda, int32_t mode, double* R, void* stream);

/* Scenario decode (Section II-A): write pairs k = first .. first+count-1 of
 * the lexicographic enumeration of unordered pairs i < j over n_elem elements
 * into DEVICE arrays elem_i, elem_j, in integer arithmetic. */
cs_status cs_enumerate_pairs_device(int32_t n_elem, int64_t first, int64_t count,
                                    int32_t* elem_i, int32_t* elem_j, void* stream);

/* N-3 extension of the enumeration (the paper's outlook, Section VI): as
 * cs_evaluate_device with a third DEVICE id array elem_k ([n] int32; -1 = none,
 * repeated ids count once).  Each id is -1 (none) or in [0, n_branch + n_gen),
 * and a -1 may only be followed by -1s (an invalid record is marked as in
 * cs_evaluate_device).  Records of scenarios with
 * three distinct elements are not written to the N-2 severity tables; N-1 and
 * N-2 records are, as in cs_evaluate_device. */
cs_status cs_evaluate_device_n3(cs_ctx* ctx, int32_t net_id, int32_t level,
                                const int32_t* elem_i, const int32_t* elem_j, const int32_t* elem_k,
                                int64_t n, const cs_result* out, void* stream);

/* Unordered triples i < j < k of n_elem >= 3 elements in lexicographic order:
 * writes `count` triples starting at rank `first` into DEVICE arrays (int32).
 * CS_E_ARG if the range exceeds C(n_elem, 3). */
cs_status cs_enumerate_triples_device(int32_t n_elem, int64_t first, int64_t count,
                                      int32_t* elem_i, int32_t* elem_j, int32_t* elem_k, void* stream);

/* Risk Index with explicit pair frequencies (common-cause extension of Eq. 2,
 * the paper's outlook): R_i = lambda_i S_i + m * sum_j F_ij S_ij, F a HOST
 * array [E * E], row i used for element i, every entry 0 or in [2^-60, 2^20]
 * (else CS_E_ARG); exact and rounded once like cs_risk_index, which it equals
 * bit for bit when F_ij = fl(lambda_i lambda_j).  lambda, R_out: HOST [E]. */
cs_status cs_risk_index_pair_freq(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda,
                                  const double* F, int32_t mode, double* R_out, int64_t* n_missing);

/* Monte-Carlo form of the Risk Index over uncertain failure rates (the
 * paper's outlook, Section VI): R for n_samples rate vectors against the
 * context's severity tables of (net_id, level), each sample exactly as
 * cs_risk_index computes it (bit-identical), pairs never evaluated counting 0.
 * lambda: DEVICE array [n_samples * (n_branch + n_gen)], sample-major; R:
 * DEVICE array of the same shape.  Asynchronous on `stream` after a device
 * synchronisation (the tables may have been written on any stream).  A rate
 * outside [2^-30, 2^10] makes that entry NaN and the next cs_sync return
 * CS_E_ARG. */
cs_status cs_risk_index_batch(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda,
                              int64_t n_samples, int32_t mode, double* R, void* stream);

/* Tensor-core matrix update, the building block of the blocked Hessenberg
 * reduction that the eigen screen of large networks uses (Section II-B-2: the
 * eigenvalues of the state matrix, whose reduction to Hessenberg form is, in
 * blocked form, mostly such updates): C_b += alpha A_b B_b for b = 0..batch-1,
 * on the tcgen05 tensor cores with every operand split into two TF32 terms and
 * three products accumulated in FP32 (about FP32 accuracy).  DEVICE arrays,
 * row-major FP32: A_b = A + b * stride_a (M x K, row stride lda), B_b (K x N,
 * ldb), C_b (M x N, ldc), read and written in place.  Asynchronous on `stream`.
 * CS_E_ARG for negative sizes or strides shorter than a row.  A tensor-core wait
 * that runs out (it never should) leaves C_b unchanged and makes the next cs_sync
 * of the context return CS_E_TIMEOUT (ctx may be NULL: then the wait is not
 * reported). */
cs_status cs_tc_gemm_update(cs_ctx* ctx, int32_t batch, int32_t M, int32_t N, int32_t K, const float* A,
                            int64_t lda, int64_t stride_a, const float* B, int64_t ldb, int64_t stride_b,
                            float* C, int64_t ldc, int64_t stride_c, float alpha, void* stream);

/* Reduction of `batch` FP32 matrices to upper Hessenberg form by Householder
 * similarities (the first step of the eigenvalue screen, Section II-B-2), in the
 * blocked form for large state matrices: panels of 32 columns reduced with their
 * reflectors accumulated as V, T and Y = A V T, and the trailing updates
 * A <- (I - V T V^T)^T (A - Y V^T) on the tensor cores (cs_tc_gemm_update's
 * TF32 x 3 products).  A: DEVICE, row-major n x n matrices `stride` floats apart,
 * overwritten by their Hessenberg forms (entries below the subdiagonal set to 0);
 * the eigenvalues are those of the inputs up to FP32 rounding.  The context keeps
 * a workspace of about 160 n floats per matrix.  Asynchronous on `stream`;
 * CS_E_ARG for a bad order, stride or pointer; a tensor-core wait that runs out
 * makes the next cs_sync return CS_E_TIMEOUT. */
cs_status cs_hessenberg_tc(cs_ctx* ctx, int32_t batch, int32_t n, float* A, int64_t stride, void* stream);

/* cs_risk_index without any device allocation (the paper has no counterpart:
 * this is a deployment variant of the Eq. 3 reduction).  Same arguments,
 * result and errors as cs_risk_index, bit for bit.  For callers that must not
 * call cudaMalloc/cudaFree (a serving loop whose other streams would stall on
 * the synchronisation cudaFree implies, or a process whose device memory is
 * reserved in full by another allocator).  Its scratch is one static device
 * array per device sized for at most 4096 outage elements (n_branch + n_gen);
 * larger networks are rejected with CS_E_ARG and a message naming the limit.
 * The array's address is looked up on the first call for a device, which
 * should come before any stream capture on that device.  All calls in the
 * process share the array, so they are serialised by a process-wide lock;
 * each returns after its stream has drained.  It is ordered after the
 * evaluations issued before it by device-side waits on their workspaces'
 * completion events (no device-wide synchronisation) and holds the context lock
 * only to enqueue, so the serving scheduler keeps running while it waits; the
 * network cannot be unloaded during the call.  Blocking; HOST lambda, R_out. */
cs_status cs_risk_index_static(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda,
                               int32_t mode, double* R_out, int64_t* n_missing);

/* Measured ALU peaks of `device` for roofline reporting: independent fused
 * multiply-add chains in FP64 and FP32 timed with CUDA events, in TFLOP/s
 * (2 flops per FMA).  Host outputs.  Runs ~10 ms of GPU work. */
cs_status cs_alu_peak(int32_t device, double* fp64_tflops, double* fp32_tflops);

/* Message of the last failing call on ctx (never NULL; "" if none). */
const char* cs_last_error(cs_ctx* ctx);

/* Kernel launches issued by the last cs_evaluate_device / cs_submit call. */
int64_t cs_last_launch_count(cs_ctx* ctx);

/* Number of scenarios whose FP32 eigen screen was re-run in FP64 (MIXED form),
 * accumulated since the context was created; waits for the device. */
cs_status cs_eigen_reruns(cs_ctx* ctx, int64_t* count);

/* Per-kernel device timing (off by default).  When enabled, every evaluation
 * records CUDA events on its stream around the islanding, OPF and small-signal
 * launches.  cs_kernel_times waits for those events and returns the summed
 * milliseconds per kernel (ms[3]: islanding, OPF, small-signal + recording) and
 * the launch counts (launches[3], may be NULL) since cs_set_timing was called. */
cs_status cs_set_timing(cs_ctx* ctx, int32_t enable);
cs_status cs_kernel_times(cs_ctx* ctx, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* CS_H */
