// Internal layout of a pf_ctx.  `View` is the plain set of device pointers
// and sizes that kernels receive by value; `Ctx` adds the host-side
// bookkeeping.  All arrays are structure-of-arrays in HBM.
//
// Numbering: the grids of a context are concatenated, so every bus, branch
// and branch end ("incidence") has one global index; F rows, J columns and
// CSR positions are local to a grid (identical for all of its instances)
// and are offset per instance into the caller's x / F / vals vectors.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <cstdlib>
#include <vector>

#include "../../include/pf.h"

namespace pf {

constexpr int kNumSMsDefault = 152;
// `tile_inc` (32, 64, 96 or 128) sets how many slots each lane of the fused
// kernel fetches ahead (tile_inc / 32) and the chunk of a large bus.
constexpr int kMaxTileInc = 128;
constexpr int kMinTileInc = 32;
constexpr int kMaxGroup = 32;      // parallel branches between one pair of buses
// The evaluation kernels work on rounds of 32 buses with equal (or adjacent)
// numbers of neighbours, one bus per lane; a bus with more than
// kLaneMaxDegree neighbours is evaluated by a whole warp.
constexpr int kLaneMaxDegree = 32;
// Tiles of the fused F / J kernel: up to kTileBuses consecutive buses of a
// grid (no large bus among them) with at most kTilePairs pairs of connected
// buses, so that the tile's rows of J and F are contiguous ranges that one
// warp stages in shared memory and writes out whole.  The tuning choice
// split_rounds = s cuts smaller tiles, of up to kTileBuses >> s buses and
// kTilePairs >> s pairs (more warps with shorter work, for contexts that fill
// less than a wave).
constexpr int kTileBuses = 32;
constexpr int kTilePairs = 96;

constexpr int kSinCosTable = 32768;  // table of (cos, sin)(i pi / 16384)
// Instance-buses are grouped in chunks of 2^kChunkLog2 for the per-bus kernels'
// instance lookup (View::chunk_inst).
constexpr int kChunkLog2 = 8;

// Fixed-point form of the evaluation kernels (pf_eval.cu).  The merged branch
// coefficients (G, B) of a slot are stored as round((G, B) 2^(59 - coef_log2)),
// where 2^coef_log2 bounds |G| and |B| (over the sums of |G|, |B| of a group
// of parallel branches, so that any subset under a mask stays in range), as
// 30-bit limbs (value = h 2^30 + l, 0 <= l < 2^30).  kMaxCoefLog2 caps that
// bound: a slot with a larger coefficient holds kBadLimb in h and its buses
// are evaluated in FP64 instead.  kBadLimb also marks a per-bus record whose
// voltage is outside (-2, 2) or whose angle is not finite.
constexpr int kMaxCoefLog2 = 12;
constexpr long long kBadFix = (long long)0x8000000000000000ULL;
constexpr int kBadLimb = (int)0x80000000;

// round(g * scale) for a power-of-two scale, or kBadFix when the result would
// not be below 2^59 in magnitude (or g is not finite).  The build and the
// masked evaluation path both convert with this function, so a group
// re-summed under a mask with every branch in service gives the built bits.
__device__ __forceinline__ long long to_fix(double g, double scale) {
  const double s = __dmul_rn(g, scale);                // exact: scale is a power of two
  if (!(fabs(s) < 0x1p59)) return kBadFix;
  return __double2ll_rn(s);
}

// (G, B) fixed-point values as limbs {G h, G l, B h, B l}; kBadLimb marks a
// value out of range.
__device__ __forceinline__ int4 coef_limbs(long long g, long long b) {
  if (g == kBadFix || b == kBadFix) return make_int4(kBadLimb, 0, kBadLimb, 0);
  return make_int4((int)(g >> 30), (int)(g & 0x3fffffff), (int)(b >> 30), (int)(b & 0x3fffffff));
}

// Grid of a kernel whose CTAs walk `work` units with a grid-stride loop,
// capped at ctas_per_sm CTAs per SM when that is set.  The units of a grid
// alternate between heavy and light rounds, so a capped grid is made odd:
// with an even stride every CTA would take only heavy or only light rounds.
inline int64_t capped_grid(int64_t work, int ctas_per_sm, int num_sms) {
  const int64_t cap = (int64_t)ctas_per_sm * num_sms;
  if (ctas_per_sm <= 0 || work <= cap) return work;
  return (cap & 1) ? cap : cap - 1;
}

// Thread-local error message behind pf_last_error().
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define PF_CUDA_TRY(expr)                                                            \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess)                                                           \
      return ::pf::fail(_e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA,  \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));         \
  } while (0)

#define PF_TRY(expr)         \
  do {                       \
    int _rc = (expr);        \
    if (_rc) return _rc;     \
  } while (0)

// Device error flag bits (set with integer atomics).
constexpr int kErrMap = 1;      // an index-map entry failed a consistency check
constexpr int kErrTimeout = 2;  // a bounded wait gave up

struct View {
  int formulation;
  int n_grids, n_inst;
  int64_t n_bus, n_branch, n_inc, n_bus_inst;
  int64_t bus_inst_begin;   // first instance bus of k_phasor (0; later for an instance range)
  int64_t n_lane_units;     // sum over instances of the rounds of 32 buses of its grid
  int64_t n_large_units;    // sum over instances of the buses with more than 32 ends
  int64_t grid1_nx;         // a context of one grid: the length of an instance's x (0 otherwise)
  int32_t grid1_nbus;       // a context of one grid: its number of buses (0 otherwise)

  // per bus
  const int32_t *inc_ptr;   // [n_bus+1] first incidence of each bus
  const int32_t *row_p;     // [n_bus] local F row of the P mismatch, -1 absent
  const int32_t *row_q;     // [n_bus] local F row of the Q mismatch, -1 absent
  const int32_t *base_p;    // [n_bus] rowptr[row_p]: first CSR position of the P row
  const int32_t *base_q;    // [n_bus] rowptr[row_q]
  const int2 *diag;         // [n_bus] in-row offsets of columns (theta_o, V_o), -1 absent
  const int32_t *len_tv;    // [n_bus] theta + V columns of the bus's rows
  const int32_t *gen;       // [n_bus] extended: local generator index, -1 none
  const double2 *bus_hat;   // [n_bus] (A^, C^): sums over ends of A_e, C_e plus shunt g, b
  const double2 *bus_sh;    // [n_bus] (g, b) shunt totals
  const double2 *bus_inj;   // [n_bus] (P_inj, Q_inj): net injections (P_g - P_load, -Q_load)
  const int4 *bus_meta;     // [n_bus] {row_p, row_q, base_p, base_q}
  const int4 *bus_meta2;    // [n_bus] {diag theta, diag V, len_tv, gen}
  const int32_t *bus_grid;  // [n_bus]

  // per branch
  const int32_t *br_from, *br_to;   // global bus ids
  const double *br_r, *br_x, *br_b, *br_tap, *br_shift, *br_gfr, *br_gto;
  // per branch, for the adjoint: (g, b_s) = 1/(r + jx), (alpha, beta) = d(g, b_s)/dr,
  // (1/tau, b_c), (cos phi, sin phi)
  const double2 *br_k_gb, *br_k_ab, *br_k_tc, *br_k_ph;
  const uint8_t *br_status;

  // per incidence, sorted by (own bus, other bus, branch)
  const int32_t *inc_own, *inc_other, *inc_code;  // code = 2*branch + end
  const double2 *inc_gb;    // (G, B) of this end (rotated series admittance / tau)
  const double2 *inc_ac;    // (A, C) of this end: V_o^2 coefficients of P and -Q
  const int2 *inc_rt;       // in-row offsets of (theta_k, V_k) columns, -1 absent
  const int32_t *inc_grp;   // at a group head: parallel ends to the same bus; else 0
  const int32_t *inc_mirror;// position of the other end of the same branch
  const int32_t *inc_of_code;// [2 n_branch] position of branch end `code` (= 2 branch + end)
  const int4 *inc_meta;     // {own, other, parallel-group length at a head else 0, code}
  const int4 *inc_pos;      // local CSR positions of this end's (P,theta_k), (P,V_k), (Q,theta_k), (Q,V_k); -1 absent

  // per grid
  const int64_t *grid_bus_off, *grid_br_off;  // [n_grids+1]
  const int32_t *grid_nbus, *grid_slack, *grid_ngen;
  const int64_t *grid_gen_off;                // [n_grids+1]
  const double *grid_theta_set;
  const int32_t *grid_row_gth;                // extended: g_theta row, else -1
  const int32_t *grid_pos_gth;                // CSR position of the g_theta entry
  const double *gen_vset;                     // [sum ngen]
  const int32_t *gen_pos;                     // [sum ngen] CSR position of the g_V entry
  const int32_t *gen_bus;                     // [sum ngen] global bus of each generator

  // rounds of the fused kernel (per grid, buses sorted by degree)
  const int64_t *grid_round_off;              // [n_grids+1]
  const int4 *unit_rec;                       // per round of 32 buses of every instance:
                                              //   {instance, round, first slot, items per lane | buses << 8}
  const int4 *unit_info;                      // per unit: {grid, buses of the grid, first bus of the grid, 0}
  const longlong2 *unit_ptr;                  // per unit, two entries: {x offset, F offset},
                                              //   {J offset, record base} of its instance
  const int2 *large_rec;                      // per large bus of every instance: {instance, bus}
  const int64_t *inst_rec_base;               // per instance: inst_bus_off - grid_bus_off of its grid
  const int4 *round_desc;                     // {first slot, items per lane, buses, flags (1 = one large bus)}
  const int32_t *rbus;                        // [32 per round] global bus id, -1 padding
  const int4 *rbus_meta, *rbus_meta2;         // bus records in round order
  const double2 *rbus_hat, *rbus_inj;
  const int32_t *bus_npair;                   // per bus: groups of parallel branches (distinct neighbours)
  const int4 *slot_meta;                      // group j of lane l at slot first + 32 j + l:
                                              //   {other bus, group length (-1 padding), code and index of its first end}
  const int4 *slot_pos;                       // the group's four CSR positions
  const double2 *slot_gb, *slot_ac;           // the group's coefficients summed in incidence order
  const double2 *slot_gbm;                    // the same for the group's mirror ends (at the other bus)
  const int4 *slot_gbx;                       // slot_gb in fixed point (see to_fix, coef_limbs)
  const int4 *slot_idx;                       // {other bus, in-row offsets of (theta_k, V_k) as two int16
                                              //  (-1 absent), group length (-1 padding), code of a
                                              //  single branch or first end of a group}
  // tiles of the fused F / J kernel: consecutive buses, their pairs of
  // connected buses listed bus by bus (the groups of parallel branches in
  // incidence order), in the formats of the slot arrays
  const int32_t *pair_ptr;                    // [n_bus+1] first pair of each bus (none for a large bus)
  const int4 *pair_meta;                      // as slot_meta
  const int4 *pair_idx;                       // as slot_idx, with the bus's index in its tile in
                                              //   bits 16..23 of the group length field and the index of
                                              //   the other bus's record among the tile's records (the
                                              //   tile's buses, then its external neighbours) in bits 24..31
  const double2 *pair_gb, *pair_ac;           // as slot_gb, slot_ac
  const int4 *pair_gbx;                       // as slot_gbx
  const int4 *tunit;                          // per tile of every instance, eight int4: {first bus, buses,
                                              //   first pair, pairs}, {J position of the first P row and
                                              //   length of the tile's P rows, the same for Q}, {first P
                                              //   row, P rows, first Q row, Q rows}, {instance, grid, first
                                              //   bus of the grid, buses of the grid}, {x offset, F offset}
                                              //   and {J offset, record base} as int64, {first external
                                              //   neighbour in tile_ext, external neighbours, 0, 0}, padding
  const int32_t *tile_ext;                    // per tile: the buses outside it that its pairs reach, ascending
  int64_t n_tile_units;                       // tiles over all instances
  int32_t tile_stage;                         // doubles of J a tile stages (its P and Q rows, two pads)

  int coef_log2;                              // 2^coef_log2 bounds the coefficients of slot_gbx
  double coef_scale;                          // 2^(59 - coef_log2)

  // per instance
  const int32_t *inst_grid, *inst_outage;     // outage: global branch id or -1
  const int64_t *inst_x_off, *inst_f_off, *inst_v_off, *inst_bus_off, *inst_br_off;
  const int64_t *inst_gen_off;                // extended: generators of earlier instances
  const int32_t *chunk_inst;                  // per chunk of 2^kChunkLog2 instance-buses (and one past the
                                              //   last): the instance of its first bus (of the last bus)

  // scratch: one 32-byte record per instance bus.  The F / J kernels use the
  // fixed-point form {cos theta 2^60, sin theta 2^60, V 2^60 as 30-bit limbs
  // (V h = kBadLimb when |V| >= 2 or theta is not finite), bits of V}; the
  // adjoint kernels the FP64 form {V cos theta, V sin theta, V, 1/V}
  // (launch_phasor chooses).
  double2 *phasor;
  int32_t *dev_error;
  const longlong2 *sincos_fix;                // [kSinCosTable] (cos, sin)(i pi / 16384) times 2^62, rounded
};

struct Ctx {
  View v{};
  int device = 0;                  // the device current at pf_build: every call runs on it
  int num_sms = kNumSMsDefault;
  pf_tuning tuning{64, 0, 0, 0};
  int max_degree = 0, max_group = 0;
  int64_t n_x = 0, n_f = 0, nnz = 0, n_branch_inst = 0;

  // host copies of per-grid / per-instance layout
  std::vector<int64_t> grid_bus_off, grid_br_off, grid_row_off, grid_nnz_off, grid_cptr_off,
      grid_csrc_off, grid_sh_off;
  std::vector<int32_t> grid_nf, grid_nnz, grid_nx, grid_nshunt;
  std::vector<int32_t> inst_grid, inst_outage;
  std::vector<int64_t> x_off, f_off, v_off, bus_off, br_off, gen_off;
  int64_t n_gen_inst = 0;
  bool any_outage = false;

  // device arrays not in View
  int32_t *rowptr = nullptr;       // per grid n_f+1 local entries, at grid_row_off
  int32_t *colind = nullptr;       // per grid nnz entries, at grid_nnz_off
  int64_t *contrib_ptr = nullptr;  // per grid nnz+1 local entries, at grid_cptr_off
  int32_t *contrib_src = nullptr;  // at grid_csrc_off

  // override scratch (coefficients recomputed from per-call parameters), in
  // incidence order and permuted to slot / round order
  double2 *ov_gb = nullptr, *ov_ac = nullptr, *ov_hat = nullptr;
  double2 *ov_slot_gb = nullptr, *ov_slot_ac = nullptr, *ov_slot_gbm = nullptr, *ov_rbus_hat = nullptr;
  int4 *ov_slot_gbx = nullptr;
  double2 *ov_pair_gb = nullptr, *ov_pair_ac = nullptr;
  int4 *ov_pair_gbx = nullptr;
  int64_t n_pairs = 0;
  // the tiles of each split_rounds value (built on first use): the pair list's
  // index records with each pair's bus index in its tile, the unit records,
  // the staged J doubles per tile, and per instance its first unit
  struct TileSet {
    int4 *pair_idx = nullptr;
    int4 *tunit = nullptr;
    int32_t *ext = nullptr;
    int64_t n_units = 0;
    int32_t stage = 0;
    std::vector<int64_t> tile_off;
  };
  TileSet tiles[3];
  int64_t n_slots = 0, n_rounds = 0;
  std::vector<int64_t> grid_round_off;
  std::vector<int64_t> lane_off, large_off;   // per instance: first unit of k_fused / k_fused_large

  // host-call staging, allocated on first use
  double *stage_x = nullptr, *stage_f = nullptr, *stage_v = nullptr;
  // transposed cotangents of pf_vjp, allocated on first use and grown
  double *vt_scratch = nullptr;
  int64_t vt_cap = 0;
  // pipelined host-buffer evaluation: internal streams and events, created on first use
  cudaStream_t pipe_stream[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> pipe_events;
  // dynamic schedule of a persistent k_fused grid (tuning.ctas_per_sm > 0):
  // {next unit, CTAs done}, zero between launches; allocated by pf_set_tuning
  unsigned long long *work_ctr = nullptr;
  // Newton-iteration state (pf_newton.cu), created on first use
  int newton_solver = PF_SOLVER_LU;
  void *newton = nullptr;
  void (*newton_free)(void *) = nullptr;

  std::vector<void *> allocations;
};

// Makes a context's device current for the span of a call and restores the
// caller's device afterwards (nothing is switched when it is current already).
struct DeviceGuard {
  int prev = -1;
  int status = 0;                  // the cudaError_t of the switch
  explicit DeviceGuard(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev) {
      status = (int)cudaSetDevice(dev);
      if (status == 0) prev = cur;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;
};

#define PF_ON_DEVICE(ctxref)                                                       \
  const ::pf::DeviceGuard pf_device_guard_((ctxref).device);                       \
  if (pf_device_guard_.status) return ::pf::fail(PF_ERR_CUDA, "cannot make the context's device current")

// Host-side fault injection for tests: with PF_FAIL_ALLOC=<n> in the
// environment when a build starts, the n-th device allocation of that build
// (counted from 0) reports failure without allocating, so that the error path
// (PF_ERR_OOM, everything allocated so far freed) can be exercised without any
// GPU fault.  BuildAllocScope reads the variable for the span of one build;
// alloc_fault() counts.
inline thread_local long long g_alloc_count = 0, g_alloc_fail_at = -1;

inline void begin_build_allocs() {
  const char *e = std::getenv("PF_FAIL_ALLOC");
  g_alloc_count = 0;
  g_alloc_fail_at = (e && *e) ? std::atoll(e) : -1;
}

inline bool alloc_fault() { return g_alloc_fail_at >= 0 && g_alloc_count++ == g_alloc_fail_at; }

// Arms the hook for one build and disarms it when the build returns.
struct BuildAllocScope {
  BuildAllocScope() { begin_build_allocs(); }
  ~BuildAllocScope() { g_alloc_fail_at = -1; }
};

template <class T>
int dev_alloc(Ctx &c, T **p, size_t n, std::vector<void *> *list = nullptr) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (alloc_fault()) return fail(PF_ERR_OOM, "device allocation failed (PF_FAIL_ALLOC)");
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess)
    return fail(PF_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) +
                                " bytes: " + cudaGetErrorString(e));
  (list ? *list : c.allocations).push_back(q);
  *p = static_cast<T *>(q);
  return PF_OK;
}

template <class T>
int upload(Ctx &c, T **p, const std::vector<T> &h, cudaStream_t s) {
  PF_TRY(dev_alloc(c, p, h.size()));
  if (!h.empty())
    PF_CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return PF_OK;
}

// ---- build (pf_build.cu) ----
int build_context(Ctx &c, const pf_system *grids, int n_grids, const pf_instance *inst,
                  int n_inst, int formulation, cudaStream_t s);
// Copies per-call coefficients (incidence / bus order) into slot / round order.
int permute_overrides(Ctx &c, cudaStream_t s);
// The tiles of split_rounds = split (built once) become the fused kernel's.
int use_tile_set(Ctx &c, int split, cudaStream_t s);
// Newton iterations (pf_newton.cu).
int newton(Ctx &c, double *x, double tol, int max_iter, cudaStream_t s, pf_newton_info *info,
           const pf_overrides *ov = nullptr);
int newton_qlim(Ctx &c, double *x, const double *q_min, const double *q_max, uint8_t *mode, double *qlim, double tol,
                int max_iter, int max_rounds, cudaStream_t s, pf_newton_info *info, int *rounds);
int newton_norms(Ctx &c, const double *F, double *norms, cudaStream_t s);
int fdlf(Ctx &c, double *x, double tol, int max_iter, cudaStream_t s, pf_newton_info *info);
int newton_update(Ctx &c, double *x, const double *dx, cudaStream_t s);
// F and J of the instances [i0, i1) only (pf_eval.cu; built coefficients, no overrides).
int launch_eval_range(Ctx &c, int i0, int i1, const double *x, double *F, double *vals, cudaStream_t s);
// The per-bus records of every instance bus into v.phasor (pf_eval.cu): the
// fixed-point form of the F / J kernels (fixed = true) or the FP64 form of the
// adjoint kernels.
int launch_phasor(const View &v, int num_sms, const double *x, cudaStream_t s, bool fixed);
// Per-end coefficients (G, B, A, C) and per-bus sums (A^, C^) from the branch
// parameters; any of r, x, b, tap may be overridden by device arrays.
int compute_coefficients(Ctx &c, const double *r, const double *x, const double *b,
                         const double *tap, double2 *gb, double2 *ac, double2 *hat, cudaStream_t s);

// ---- evaluation (pf_eval.cu) ----
int launch_eval(Ctx &c, const double *x, const pf_overrides *ov, double *F, double *vals,
                cudaStream_t s);
// stage mask: 1 = phasors, 2 = fused kernel, 3 = both
int launch_eval_stages(Ctx &c, int stages, const double *x, const pf_overrides *ov, double *F, double *vals,
                       cudaStream_t s);
int launch_vjp(Ctx &c, const double *x, const pf_overrides *ov, const double *v, int n_cot,
               const pf_grads *g, cudaStream_t s);
// F / J evaluation whose per-bus phasor scratch is `scratch` instead of the context's.
int launch_eval_scratch(Ctx &c, const double *x, double *F, double *vals, double2 *scratch, cudaStream_t s);
// The phasor routine alone (verification).
int launch_sincos(Ctx &c, const double *t, int64_t n, double *cs, double *sn, cudaStream_t s);
// The context behind a C-ABI handle.
Ctx *ctx_of(pf_ctx *h);

// Largest i in [0, n) with off[i] <= key (off ascending, off[0] = 0).
__device__ __forceinline__ int find_segment(const int64_t *__restrict__ off, int n, int64_t key) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace pf
