/*
 * pf.h -- C ABI of the GB300 power-flow residual / Jacobian library (libpf.so).
 *
 * Tasks (1) and (2) of Newton power flow (Sec. I): evaluate the bus power
 * mismatches F(theta, V) and the nonzero values of their Jacobian J in a
 * fixed sparsity pattern, for the models of Sec. II-A (Bus, PQ load, PV
 * generator, Slack, Line / two-winding transformer, Shunt) in either the
 * extended formulation of Eqs. (1)-(3) or the classic reduced one.
 *
 * Conventions shared by every entry point
 *   - Floating point is IEEE binary64 throughout; indices are int32 unless
 *     noted; offsets into batched vectors are int64.
 *   - Per-unit quantities, angles in radians.
 *   - Residual sign: F = power flowing out of the bus into its branches
 *     + shunt consumption + load - generation (the sign of Eq. 4, where
 *     P_h leaves bus h).
 *   - Branch model (Eq. 4 extended with reactive power, tap and shift):
 *     g + jb = 1/(r + jx), charging b_c split b_c/2 per end, end
 *     conductances g_fr, g_to, tap tau and shift phi on the from side,
 *     delta = theta_f - theta_t - phi:
 *       P_f =  V_f^2 (g+g_fr)/tau^2     - (V_f V_t/tau)(g cos d + b sin d)
 *       Q_f = -V_f^2 (b+b_c/2)/tau^2    - (V_f V_t/tau)(g sin d - b cos d)
 *       P_t =  V_t^2 (g+g_to)           - (V_f V_t/tau)(g cos d - b sin d)
 *       Q_t = -V_t^2 (b+b_c/2)          + (V_f V_t/tau)(g sin d + b cos d)
 *   - State vector x of one instance: [theta(N), V(N)] and, in the extended
 *     formulation, [Q_g (PV units in input order, then the slack), P_s]
 *     (Eq. 3).  In the reduced formulation x still carries every theta and
 *     V; the slack angle and the PV / slack magnitudes are read as fixed.
 *   - Reduced rows / columns: P / theta of the non-slack buses in ascending
 *     bus order, then Q / V of the PQ-type buses in ascending bus order.
 *     Extended rows: [g_p(N), g_q(N), g_V(gens), g_theta] (Eq. 2); columns
 *     [theta(N), V(N), Q_g(gens), P_s] (Eq. 3); g_V = V - Vset and
 *     g_theta = theta_s - theta_set.
 *   - The J pattern is the structural union of every model's entries: CSR,
 *     ascending columns, parallel branches merged, the four diagonal
 *     entries of a bus always present when their row and column exist,
 *     out-of-service / masked branches kept as explicit zeros.
 *   - Results are deterministic (no floating-point atomics): a bus's sums
 *     over its branch ends are exact integer sums rounded once (or, for a
 *     bus with more than 32 neighbours or an out-of-range term, FP64 sums in
 *     a fixed order), every other sum runs in a fixed order, so F and J are
 *     identical run to run, for every tuning choice, and between a batch and
 *     the single-instance evaluation of each of its instances.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Evaluation calls are asynchronous on that stream, allocate
 *     nothing and may be captured in a CUDA graph; device buffers passed to
 *     them must stay valid until the stream reaches the call.
 *   - A context belongs to the device that was current when it was built.
 *     Every call on it makes that device current for its duration and
 *     restores the caller's device afterwards; `stream` must belong to it.
 *   - Every function returns PF_OK (0) or an error code; pf_last_error()
 *     returns a message for the calling thread's last failure.
 */
#ifndef PF_H
#define PF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PF_API __attribute__((visibility("default")))
#else
#define PF_API
#endif

/* ---- status codes ------------------------------------------------------ */
#define PF_OK 0
#define PF_ERR_INVALID 1      /* malformed system, bad argument or size    */
#define PF_ERR_OOM 2          /* device or host allocation failed          */
#define PF_ERR_CUDA 3         /* a CUDA runtime call or launch failed      */
#define PF_ERR_TIMEOUT 4      /* a bounded device wait gave up             */
#define PF_ERR_UNSUPPORTED 5  /* valid input outside the library's limits  */
#define PF_ERR_DEVICE 6       /* a kernel raised the context's error flag  */
#define PF_ERR_NUMERIC 7      /* Newton: J numerically singular            */

/* ---- formulations (Sec. II-A) ------------------------------------------- */
#define PF_REDUCED 0          /* classic: P/theta non-slack, Q/V PQ buses  */
#define PF_EXTENDED 1         /* Eqs. (1)-(3): g_p, g_q, g_V, g_theta      */

typedef struct pf_ctx pf_ctx;

/* One network, as host arrays (the library copies them; the caller may
 * free them when pf_build returns).  Optional arrays may be NULL. */
typedef struct pf_system {
  int32_t n_bus;                 /* N >= 2                                    */
  int32_t n_branch;              /* M >= 0 (lines and transformers)           */
  const int32_t *br_from;        /* [M] from bus, 0 <= . < N                  */
  const int32_t *br_to;          /* [M] to bus, != from                       */
  const double *br_r;            /* [M] series resistance                     */
  const double *br_x;            /* [M] series reactance, r^2 + x^2 > 0       */
  const double *br_b;            /* [M] total line charging b_c (NULL: 0)      */
  const double *br_tap;          /* [M] off-nominal tap tau > 0 (NULL: 1)     */
  const double *br_shift;        /* [M] phase shift phi, radians (NULL: 0)    */
  const double *br_g_fr;         /* [M] from-end conductance g_{L,h} (NULL: 0)*/
  const double *br_g_to;         /* [M] to-end conductance g_{L,k} (NULL: 0)  */
  const uint8_t *br_status;      /* [M] 0 = out of service (NULL: all in)     */
  int32_t n_load;
  const int32_t *load_bus;       /* [n_load] PQ loads: bus, P, Q (constant)   */
  const double *load_p;
  const double *load_q;
  int32_t n_pv;
  const int32_t *pv_bus;         /* [n_pv] PV units: bus (!= slack), P, Vset  */
  const double *pv_p;
  const double *pv_vset;
  int32_t slack_bus;             /* exactly one slack generator              */
  double slack_vset;
  double slack_theta;
  int32_t n_shunt;
  const int32_t *sh_bus;         /* [n_shunt] shunts: consumption g V^2, -b V^2 */
  const double *sh_g;
  const double *sh_b;
} pf_system;

/* One evaluation instance of a batch (many contingency / scenario instances in one launch). */
typedef struct pf_instance {
  int32_t grid;                  /* index into the grids array of pf_build_batch */
  int32_t outage;                /* branch of that grid taken out for this instance, -1: none */
} pf_instance;

typedef struct pf_dims {
  int32_t formulation;
  int32_t n_grids;
  int32_t n_instances;
  int32_t max_degree;            /* largest bus degree over all grids         */
  int64_t n_bus;                 /* sum over grids                            */
  int64_t n_branch;              /* sum over grids                            */
  int64_t n_inc;                 /* branch ends = 2 * n_branch               */
  int64_t n_x;                   /* sum over instances: length of x          */
  int64_t n_f;                   /* sum over instances: length of F          */
  int64_t nnz;                   /* sum over instances: length of J values   */
  int64_t n_bus_inst;            /* sum over instances of N (p_inj / q_inj length) */
  int64_t n_branch_inst;         /* sum over instances of M (status override length) */
  int64_t n_gen_inst;            /* extended: sum over instances of the generators (PV units,
                                    then the slack) -- the length of gen_mode / gen_qlim */
} pf_dims;

/* Per-call overrides (device pointers; every field may be NULL). */
typedef struct pf_overrides {
  const double *p_inj;           /* [n_bus_inst] net P injection per bus (P_g - P_load),
                                    replaces the system's (Sec. II-A PQ / PV models) */
  const double *q_inj;           /* [n_bus_inst] net Q injection per bus (-Q_load) */
  const uint8_t *status;         /* [n_branch_inst] per-instance branch mask, 0 = out;
                                    combined with the instance's outage           */
  const double *br_r;            /* [n_branch] per-grid parameter overrides of the */
  const double *br_x;            /*   branch model (adjoint / sensitivity use);   */
  const double *br_b;            /*   each NULL keeps the built value             */
  const double *br_tap;
  const uint8_t *gen_mode;       /* extended, [n_gen_inst]: 0 = voltage control (g_V = V - Vset);
                                    otherwise the generator is held at a reactive limit and
                                    g_V = Q_g - gen_qlim (Sec. II-A: PV -> PQ switching in the
                                    same formulation; the J pattern carries both entries of
                                    every g_V row, so switching never changes it) */
  const double *gen_qlim;        /* [n_gen_inst] the held reactive output (read where mode != 0) */
} pf_overrides;

/* Gradients of a vector-Jacobian product (device pointers; NULL skips).
 * Layout: [n_cot][...] with the per-instance blocks concatenated. */
typedef struct pf_grads {
  double *x;                     /* [n_cot][n_x]      v^T dF/dx                  */
  double *p_inj;                 /* [n_cot][n_bus_inst] v^T dF/dP_inj            */
  double *q_inj;                 /* [n_cot][n_bus_inst] v^T dF/dQ_inj            */
  double *br_r;                  /* [n_cot][n_branch_inst] v^T dF/dr             */
  double *br_x;                  /* [n_cot][n_branch_inst] v^T dF/dx (reactance) */
  double *br_b;                  /* [n_cot][n_branch_inst] v^T dF/db_c           */
  double *br_tap;                /* [n_cot][n_branch_inst] v^T dF/dtau           */
} pf_grads;

typedef struct pf_tuning {
  int32_t tile_inc;              /* 32, 64, 96 or 128: each lane of the fused kernel has tile_inc / 32
                                    pairs of connected buses (and their voltage records) in flight
                                    at once (the chunk of a bus with > 32 neighbours) */
  int32_t ctas_per_sm;           /* persistent CTAs per SM of the fused kernels and the adjoint
                                    state kernel (the fused kernel's warps then claim their work
                                    from a counter); 0 = one CTA for every unit of work */
  int32_t split_rounds;          /* size of the fused kernel's tiles (one warp per tile and
                                    instance): 0 = up to 32 consecutive buses and 96 pairs of
                                    connected buses, 1 = 16 and 48, 2 = 8 and 24 -- more warps with
                                    shorter work, for contexts that fill less than a wave (the
                                    smaller tilings are built on first use).  Results are
                                    bit-identical. */
  int32_t fuse_phasor;           /* 1: the fused kernel forms the voltage records of each tile's
                                    buses and of their neighbours outside the tile itself (one
                                    launch per evaluation, no record gathers; neighbours' records
                                    are formed again by every tile that reaches them); 0: a phasor
                                    kernel forms every record once before it.  Bit-identical. */
} pf_tuning;

/* ---- build (once) -------------------------------------------------------- */

/* Builds the device index maps of one network (Sec. III: the Jacobian pattern
 * that the paper assembles from triplets on every call is built once here):
 * the per-bus incidence list, the CSR pattern of J and the per-nonzero
 * contribution list, all on the device with integer-only, deterministic
 * kernels.  Validates the system on the host first.  Synchronises `stream`
 * before returning.  On success *out owns all device memory of the context.
 * Errors: PF_ERR_INVALID (index out of range, from == to, r = x = 0,
 * tau <= 0, non-finite value, PV unit on the slack bus, two PV units on one
 * bus in the extended formulation, bad formulation), PF_ERR_UNSUPPORTED
 * (sizes beyond int32 index range), PF_ERR_OOM, PF_ERR_CUDA. */
PF_API int pf_build(const pf_system *sys, int32_t formulation, void *stream, pf_ctx **out);

/* Batched form: n_grids networks and n_inst instances over them, evaluated
 * together by one launch of each kernel.  Instance k owns the k-th block of x, F
 * and J values (offsets from pf_offsets).  Same errors as pf_build, plus
 * PF_ERR_INVALID for a bad grid index or outage branch. */
PF_API int pf_build_batch(const pf_system *grids, int32_t n_grids, const pf_instance *inst,
                   int32_t n_inst, int32_t formulation, void *stream, pf_ctx **out);

/* Frees every device and host resource of the context.  NULL is ignored. */
PF_API void pf_destroy(pf_ctx *ctx);

/* ---- sizes and maps (host-side copies) ------------------------------------ */

PF_API int pf_get_dims(const pf_ctx *ctx, pf_dims *dims);

/* Per-instance offsets into x, F and J values: three host arrays of
 * n_instances + 1 entries each (any may be NULL). */
PF_API int pf_offsets(const pf_ctx *ctx, int64_t *x_off, int64_t *f_off, int64_t *nnz_off);

/* CSR pattern of J of grid `grid`: rowptr [n_f(grid)+1], colind [nnz(grid)],
 * host buffers.  Identical for every instance of that grid. */
PF_API int pf_pattern(const pf_ctx *ctx, int32_t grid, int32_t *rowptr, int32_t *colind);
PF_API int pf_grid_sizes(const pf_ctx *ctx, int32_t grid, int32_t *n_f, int32_t *nnz, int32_t *n_x);

/* Per-bus incidence list of grid `grid` (host buffers): ptr [N+1]; for each
 * branch end at a bus, code = 2*branch + end (end 0 = from, 1 = to) and the
 * other bus, ordered by (other bus, branch).  Local numbering. */
PF_API int pf_incidence(const pf_ctx *ctx, int32_t grid, int32_t *ptr, int32_t *code, int32_t *other);

/* Per-nonzero contribution list of J of grid `grid`, in CSR order: sources
 * of each nonzero in summation order -- branch ends as incidence-list
 * positions, shunts as 2*M + shunt index, -1 for the constant +-1 entries of
 * the extended formulation.  ptr [nnz+1] (int64), src [ptr[nnz]] (host).
 * Call with src == NULL to obtain ptr (and so the length) only. */
PF_API int pf_contributions(const pf_ctx *ctx, int32_t grid, int64_t *ptr, int32_t *src);

/* ---- evaluation (hot path) ------------------------------------------------ */

/* Task (1): F(x) for every instance.  x: [n_x], F: [n_f] device buffers. */
PF_API int pf_residual(pf_ctx *ctx, const double *x, double *F, void *stream);

/* Task (2): J values in CSR order of pf_pattern.  vals: [nnz] device. */
PF_API int pf_jacobian(pf_ctx *ctx, const double *x, double *vals, void *stream);

/* Tasks (1) and (2) in one fused pass.  F or vals may be NULL to skip. */
PF_API int pf_residual_jacobian(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream);

/* Same, with per-call overrides (ov may be NULL). */
PF_API int pf_eval(pf_ctx *ctx, const double *x, const pf_overrides *ov, double *F, double *vals,
            void *stream);

/* The two kernels of an evaluation, one at a time: PF_STAGE_PHASOR computes
 * the per-bus records (the unit phasor (cos theta, sin theta) and V in fixed
 * point, and 1/V) into the context's scratch; PF_STAGE_FUSED runs the fused
 * F / J kernel, reading that scratch (a PF_STAGE_PHASOR call at the same x
 * must precede it on the stream).  Under the tuning fuse_phasor = 1 the fused
 * kernel forms the records it needs itself, and PF_STAGE_PHASOR computes only
 * those of buses with more than 32 neighbours.  pf_eval runs both.  For
 * timing each kernel and for overlapping the stages with other work.  ov may
 * be NULL; F or vals may be NULL. */
#define PF_STAGE_PHASOR 1
#define PF_STAGE_FUSED 2
PF_API int pf_eval_stage(pf_ctx *ctx, int32_t stage, const double *x, const pf_overrides *ov, double *F,
                         double *vals, void *stream);

/* Allocation-free variant of pf_residual_jacobian (the paper has no
 * counterpart; it serves callers that cannot allocate device memory at call
 * time -- code that must not synchronise the device, hosts with a fixed
 * device-memory budget, plug-ins that may use only memory handed to them).
 * Same inputs, outputs and results as pf_residual_jacobian; F or vals may be
 * NULL.  It calls no cudaMalloc / cudaFree: the per-bus scratch of the
 * evaluation is a static device array of 2^18 instance-buses (8 MiB), held by
 * every GPU that loads the library until the process exits.
 *   - Contexts with more than 2^18 buses summed over their instances are
 *     rejected with PF_ERR_UNSUPPORTED (use pf_residual_jacobian).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call, from any context, shares the one array: calls whose GPU
 *     work overlaps (other streams, other threads) race and give wrong
 *     results.  The array keeps the last call's contents; nothing in it needs
 *     to start at zero. */
PF_API int pf_residual_jacobian_static(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream);

/* End-to-end form for callers holding host memory: copies x (host) in,
 * evaluates, copies F and vals (host; either may be NULL) out and
 * synchronises `stream`.  With several instances the work is pipelined over
 * up to 8 chunks of instances on internal streams (copy in, evaluate, copy
 * out overlap; the calls wait for `stream`'s earlier work first).
 * Page-locked host buffers give the full copy rate and the overlap.  Device
 * staging buffers, streams and events are created on the first call and
 * kept. */
PF_API int pf_residual_jacobian_host(pf_ctx *ctx, const double *x_host, double *F_host,
                              double *vals_host, void *stream);

/* Adjoint (differentiation of F): for n_cot cotangents v
 * ([n_cot][n_f], device), the vector-Jacobian products v^T dF/d(x, P_inj,
 * Q_inj, r, x, b_c, tau) into the non-NULL arrays of g.  Trigonometric terms
 * are recomputed, nothing from a forward call is stored.  ov may be NULL.
 * Sums run in a fixed order: every cotangent of a batch gives the bits of a
 * single-cotangent call.  With 16 or more cotangents they are first copied
 * to a transposed device buffer owned by the context, allocated by the first
 * call with that many (or more) cotangents: make that call outside stream
 * capture.  Errors: PF_ERR_INVALID (NULL x / v / g, n_cot <= 0), PF_ERR_OOM,
 * PF_ERR_CUDA. */
PF_API int pf_vjp(pf_ctx *ctx, const double *x, const pf_overrides *ov, const double *v,
           int32_t n_cot, const pf_grads *g, void *stream);

/* ---- Newton iterations around the hot path (tasks 3 and 4 of Sec. I) ---------- */

typedef struct pf_newton_info {
  int32_t iterations;            /* Newton updates applied                              */
  int32_t converged;             /* 1 when every instance reached max |F| <= tol        */
  double max_mismatch;           /* max over instances of max |F| at the last evaluation */
  double eval_ms;                /* host wall time in F + J evaluation and the norm     */
  double solve_ms;               /* ... in the sparse solves (task 3)                   */
  double update_ms;              /* ... in the updates (task 4)                         */
} pf_newton_info;

/* Linear solver of the Newton loop (a library solve, outside the hot path). */
#define PF_SOLVER_LU 0        /* default: LU refactorization -- a host LU of the first J (METIS
                                 ordering, partial pivoting) fixes the ordering, pivots and
                                 factor patterns; cuSOLVER-Rf refactors every later J and solves
                                 on the device */
#define PF_SOLVER_QR 1        /* cuSOLVER's device sparse QR, from scratch every iteration */
PF_API int pf_set_newton_solver(pf_ctx *ctx, int32_t solver);

/* Newton power flow on every instance: repeat { F, J at x (this library's
 * kernels); stop when max |F| <= tol for every instance; per instance that
 * has not converged, solve J dx = F with the chosen solver;
 * x <- x - dx on the unknowns (task 4, on the device) } for at most max_iter
 * updates.  x: the
 * instances' states ([n_x], device), updated in place.  Synchronises `stream`
 * every iteration (the convergence test is read on the host).  Device
 * scratch (F, J values, dx) is allocated on the first call.  Errors:
 * PF_ERR_INVALID (NULL x, max_iter < 0, tol < 0 or NaN), PF_ERR_NUMERIC (a
 * singular J), PF_ERR_CUDA.  info may be NULL. */
PF_API int pf_newton(pf_ctx *ctx, double *x, double tol, int32_t max_iter, void *stream, pf_newton_info *info);

/* Newton power flow with reactive limits (extended formulation; Sec. II-A):
 * pf_newton's iterations with the generators' modes of gen_mode; after each
 * converged solve, every generator in voltage control whose Q_g lies above
 * q_max or below q_min is switched to that limit (gen_mode 1 or 2, gen_qlim
 * set) and the solve is repeated, until no switch happens (at most
 * max_rounds solves).  q_min, q_max: [n_gen_inst] device; gen_mode
 * (uint8) and gen_qlim: [n_gen_inst] device, read as the starting modes and
 * updated in place (all zero = every generator in voltage control).
 * info->iterations counts the Newton updates of all solves; *rounds (may be
 * NULL) the solves.  PF_ERR_INVALID for the reduced formulation. */
PF_API int pf_newton_qlim(pf_ctx *ctx, double *x, const double *q_min, const double *q_max, uint8_t *gen_mode,
                          double *gen_qlim, double tol, int32_t max_iter, int32_t max_rounds, void *stream,
                          pf_newton_info *info, int32_t *rounds);

/* Fast decoupled power flow (the method Sec. V names as future work; XB
 * variant of Stott and Alsac, reduced formulation): B' from 1/x of the
 * branches (non-slack rows), B'' = -Im(Y_bus) without phase shifts (PQ
 * rows), each built on the host from the context and factored once
 * (host LU, cuSOLVER-Rf); every iteration solves B' dtheta = -F_P / V with
 * F from this library's kernels, updates theta, re-evaluates F and solves
 * B'' dV = -F_Q / V.  An instance's outage branch is left out of its
 * matrices (one factored pair per distinct grid and outage; per-call status
 * masks are not applied to them).  Stops when max |F| <= tol for every
 * instance or after max_iter iterations; x updated in place.  PF_ERR_INVALID
 * for the extended formulation. */
PF_API int pf_fdlf(pf_ctx *ctx, double *x, double tol, int32_t max_iter, void *stream, pf_newton_info *info);

/* Convergence test of task (4): norms[i] = max |F| over the rows of instance
 * i (device, [n_inst] doubles), exact in any order (a maximum). */
PF_API int pf_mismatch_norm(pf_ctx *ctx, const double *F, double *norms, void *stream);

/* Task (4): x <- x - dx on the unknowns of every instance (dx in the row /
 * column order of J, [n_f] device; x [n_x] device, in place). */
PF_API int pf_newton_update(pf_ctx *ctx, double *x, const double *dx, void *stream);

/* ---- tuning ------------------------------------------------------------------ */

PF_API int pf_get_tuning(const pf_ctx *ctx, pf_tuning *t);
/* Sets the launch parameters of the evaluation kernels (synchronises
 * `stream` first; allocates the schedule counters of ctas_per_sm > 0 on
 * first use).  Never changes results.  PF_ERR_INVALID for values outside
 * the documented range (tile_inc 32/64/96/128, ctas_per_sm 0..32,
 * split_rounds 0/1/2). */
PF_API int pf_set_tuning(pf_ctx *ctx, const pf_tuning *t, void *stream);
/* Times the fused evaluation at x for each candidate tuning (a batch of
 * about 2 ms of back-to-back evaluations, 5 to 200, the faster of two
 * batches), keeps the fastest and returns it in *chosen.  x, F, vals: device
 * buffers used as scratch for the timing runs. */
PF_API int pf_autotune(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream,
                pf_tuning *chosen);
/* pf_autotune with a tuning cache, so that a process does not time again
 * what an earlier one chose.  `path` names a text file of tunings, one per
 * line, keyed by the GPU (name, SM count) and the context (formulation,
 * numbers of grids, instances, buses, branches, rounds and J nonzeros, and a
 * hash of the per-grid round counts and of the instance list).  A valid
 * entry for this context is applied without any timing (*from_cache = 1);
 * otherwise pf_autotune runs and its choice is appended to the file
 * (*from_cache = 0).  A file that is missing or unreadable, or holds lines
 * that do not parse or values outside pf_set_tuning's ranges, is treated as
 * holding no entry; a file that cannot be written leaves the chosen tuning
 * set and still returns PF_OK.  Never changes results.  from_cache may be
 * NULL.  Errors: those of pf_autotune; PF_ERR_INVALID for a NULL path. */
PF_API int pf_autotune_cache(pf_ctx *ctx, const char *path, const double *x, double *F, double *vals,
                             void *stream, pf_tuning *chosen, int32_t *from_cache);

/* The per-bus trigonometric routine of the evaluation (table-driven reduction
 * by multiples of pi/16384 and short Taylor polynomials), exposed so it can be
 * checked against a reference sin / cos: cos_out[i], sin_out[i] of theta[i],
 * n device entries each, asynchronous on `stream`. */
PF_API int pf_sincos(pf_ctx *ctx, const double *theta, int64_t n, double *cos_out, double *sin_out,
                     void *stream);

/* The per-bus records of the evaluation's first stage, exposed so they can be
 * checked: for every bus of every instance (instance-bus order, as p_inj),
 * four doubles (V cos theta, V sin theta, V, 1/V) -- the bus voltage in
 * rectangular form (the sin / cos of pf_sincos times V) and the reciprocal
 * of V by one cubically convergent correction of the hardware approximation.
 * A bus with |V| < 2^-500 gets 2^-600 in place of V in the first, second and
 * fourth entries.  x: device, length n_x; rec: device, 4 n_bus_inst doubles,
 * caller-owned.  Asynchronous on `stream`. */
PF_API int pf_voltage_records(pf_ctx *ctx, const double *x, double *rec, void *stream);

/* Measurement helper (not part of the method): the FP64 fused multiply-add
 * rate of `device`, in G operations/s (one FMA counts one operation), from
 * three timed launches of a kernel that keeps 2,048 threads per SM on eight
 * independent FMA chains each (the fastest of the three is reported; *ms, if
 * not NULL, receives its duration).  The denominator of the FP64 fractions
 * the benchmark reports beside the evaluation's roofline.  Allocates and
 * frees a small device buffer; synchronises `stream`.  Errors: PF_ERR_INVALID
 * for a NULL gops, PF_ERR_CUDA. */
PF_API int pf_fp64_peak(int32_t device, double *gops, double *ms, void *stream);

/* ---- errors --------------------------------------------------------------------- */
/* Test hook: with the environment variable PF_FAIL_ALLOC=<n> set when
 * pf_build / pf_build_batch starts, the n-th device allocation of that build
 * (counted from 0) fails without allocating: the build returns PF_ERR_OOM and
 * frees everything it had allocated.  For exercising the error path without a
 * GPU fault; unset in normal use. */

PF_API const char *pf_error_string(int32_t code);
PF_API const char *pf_last_error(void);
/* Reads and clears the context's device error flag (a kernel found an
 * inconsistent map or a bounded wait ran out), and checks that the schedule
 * counters of persistent fused grids (ctas_per_sm > 0) are back at zero.
 * Synchronises `stream`.  Returns PF_OK or PF_ERR_DEVICE / PF_ERR_TIMEOUT. */
PF_API int pf_check_device(pf_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
