// C ABI of libpf.so (declarations and contracts in include/pf.h).
#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "pf_internal.cuh"

struct pf_ctx {
  pf::Ctx c;
};

namespace pf {

thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

}  // namespace pf

using pf::fail;

pf::Ctx *pf::ctx_of(pf_ctx *h) { return h ? &h->c : nullptr; }

namespace {

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// Tuning cache: a line is "<tag> <key> <tile_inc> <ctas_per_sm> <split_rounds> <fuse_phasor>".
constexpr const char *kTuningTag = "pf-tuning-v2";

bool tuning_valid(const pf_tuning &t) {
  return t.tile_inc >= pf::kMinTileInc && t.tile_inc <= pf::kMaxTileInc && t.tile_inc % 32 == 0 &&
         t.ctas_per_sm >= 0 && t.ctas_per_sm <= 32 && t.split_rounds >= 0 && t.split_rounds <= 2 &&
         (t.fuse_phasor == 0 || t.fuse_phasor == 1);
}

// 64-bit FNV-1a over the bytes of v.
template <class T>
uint64_t fnv1a(uint64_t h, const std::vector<T> &v) {
  const unsigned char *p = reinterpret_cast<const unsigned char *>(v.data());
  for (size_t i = 0; i < v.size() * sizeof(T); ++i) h = (h ^ p[i]) * 0x100000001b3ULL;
  return h;
}

// The GPU and the shape of the context, without blanks; empty if the device
// cannot be queried.
std::string tuning_key(const pf::Ctx &c) {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "";
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  uint64_t h = 0xcbf29ce484222325ULL;
  h = fnv1a(h, c.grid_round_off);
  h = fnv1a(h, c.inst_grid);
  h = fnv1a(h, c.inst_outage);
  std::ostringstream k;
  k << name << ":sm" << prop.multiProcessorCount << ":f" << c.v.formulation << ":g" << c.v.n_grids << ":i"
    << c.v.n_inst << ":b" << c.v.n_bus << ":br" << c.v.n_branch << ":r" << c.n_rounds << ":nnz" << c.nnz << ":h"
    << std::hex << h;
  return k.str();
}

// Chunks of instances of the pipelined host-buffer evaluation.  The copy out
// of F and J is the slowest stage, so the chunks grow: chunk k ends at
// instance max(k + 1, I (k+1)^2 / C^2), and the first copy out starts after a
// small chunk's copy in and evaluation.
constexpr int kHostChunks = 8;
constexpr bool kHostGrowingChunks = true;

int host_chunk_end(int I, int C, int k) {
  const int64_t n = (int64_t)(k + 1);
  if (!kHostGrowingChunks) return (int)((int64_t)I * n / C);
  return (int)std::max<int64_t>(n, (int64_t)I * n * n / ((int64_t)C * C));
}

void free_ctx(pf_ctx *ctx) {
  if (!ctx) return;
  for (auto &q : ctx->c.pipe_stream)
    if (q) cudaStreamDestroy(q);
  for (auto &e : ctx->c.pipe_events) cudaEventDestroy(e);
  for (void *p : ctx->c.allocations) cudaFree(p);
  if (ctx->c.stage_x) cudaFree(ctx->c.stage_x);
  if (ctx->c.vt_scratch) cudaFree(ctx->c.vt_scratch);
  if (ctx->c.newton && ctx->c.newton_free) ctx->c.newton_free(ctx->c.newton);
  if (ctx->c.stage_f) cudaFree(ctx->c.stage_f);
  if (ctx->c.stage_v) cudaFree(ctx->c.stage_v);
  delete ctx;
}

int check_grid(const pf_ctx *ctx, int32_t grid) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  if (grid < 0 || grid >= ctx->c.v.n_grids) return fail(PF_ERR_INVALID, "grid index out of range");
  return PF_OK;
}

template <class T>
int copy_out(T *dst, const T *src, size_t n) {
  if (n == 0) return PF_OK;
  PF_CUDA_TRY(cudaMemcpy(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost));
  return PF_OK;
}

}  // namespace

extern "C" {

int pf_build_batch(const pf_system *grids, int32_t n_grids, const pf_instance *inst, int32_t n_inst,
                   int32_t formulation, void *stream, pf_ctx **out) {
  if (!out) return fail(PF_ERR_INVALID, "out is NULL");
  *out = nullptr;
  pf_ctx *ctx = new (std::nothrow) pf_ctx();
  if (!ctx) return fail(PF_ERR_OOM, "host allocation failed");
  int rc = pf::build_context(ctx->c, grids, n_grids, inst, n_inst, formulation, as_stream(stream));
  if (rc) {
    std::string msg = pf_last_error();
    free_ctx(ctx);
    pf::set_error(msg);
    return rc;
  }
  *out = ctx;
  return PF_OK;
}

int pf_build(const pf_system *sys, int32_t formulation, void *stream, pf_ctx **out) {
  if (!sys) return fail(PF_ERR_INVALID, "sys is NULL");
  pf_instance one{0, -1};
  return pf_build_batch(sys, 1, &one, 1, formulation, stream, out);
}

void pf_destroy(pf_ctx *ctx) {
  if (!ctx) return;
  const pf::DeviceGuard on_device(ctx->c.device);
  cudaDeviceSynchronize();
  free_ctx(ctx);
}

int pf_get_dims(const pf_ctx *ctx, pf_dims *d) {
  if (!ctx || !d) return fail(PF_ERR_INVALID, "NULL argument");
  const pf::Ctx &c = ctx->c;
  d->formulation = c.v.formulation;
  d->n_grids = c.v.n_grids;
  d->n_instances = c.v.n_inst;
  d->max_degree = c.max_degree;
  d->n_gen_inst = c.n_gen_inst;
  d->n_bus = c.v.n_bus;
  d->n_branch = c.v.n_branch;
  d->n_inc = c.v.n_inc;
  d->n_x = c.n_x;
  d->n_f = c.n_f;
  d->nnz = c.nnz;
  d->n_bus_inst = c.v.n_bus_inst;
  d->n_branch_inst = c.n_branch_inst;
  return PF_OK;
}

int pf_offsets(const pf_ctx *ctx, int64_t *x_off, int64_t *f_off, int64_t *nnz_off) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  const pf::Ctx &c = ctx->c;
  const size_t n = c.x_off.size();
  if (x_off) std::memcpy(x_off, c.x_off.data(), n * sizeof(int64_t));
  if (f_off) std::memcpy(f_off, c.f_off.data(), n * sizeof(int64_t));
  if (nnz_off) std::memcpy(nnz_off, c.v_off.data(), n * sizeof(int64_t));
  return PF_OK;
}

int pf_grid_sizes(const pf_ctx *ctx, int32_t grid, int32_t *n_f, int32_t *nnz, int32_t *n_x) {
  PF_TRY(check_grid(ctx, grid));
  if (n_f) *n_f = ctx->c.grid_nf[grid];
  if (nnz) *nnz = ctx->c.grid_nnz[grid];
  if (n_x) *n_x = ctx->c.grid_nx[grid];
  return PF_OK;
}

int pf_pattern(const pf_ctx *ctx, int32_t grid, int32_t *rowptr, int32_t *colind) {
  PF_TRY(check_grid(ctx, grid));
  PF_ON_DEVICE(ctx->c);
  const pf::Ctx &c = ctx->c;
  if (rowptr) PF_TRY(copy_out(rowptr, c.rowptr + c.grid_row_off[grid], (size_t)c.grid_nf[grid] + 1));
  if (colind) PF_TRY(copy_out(colind, c.colind + c.grid_nnz_off[grid], (size_t)c.grid_nnz[grid]));
  return PF_OK;
}

int pf_incidence(const pf_ctx *ctx, int32_t grid, int32_t *ptr, int32_t *code, int32_t *other) {
  PF_TRY(check_grid(ctx, grid));
  PF_ON_DEVICE(ctx->c);
  const pf::Ctx &c = ctx->c;
  const int64_t b0 = c.grid_bus_off[grid], b1 = c.grid_bus_off[grid + 1];
  const int64_t l0 = c.grid_br_off[grid], l1 = c.grid_br_off[grid + 1];
  const int64_t e0 = 2 * l0, ne = 2 * (l1 - l0);
  if (ptr) {
    std::vector<int32_t> h(b1 - b0 + 1);
    PF_TRY(copy_out(h.data(), c.v.inc_ptr + b0, h.size()));
    for (auto &q : h) q -= (int32_t)e0;
    std::memcpy(ptr, h.data(), h.size() * sizeof(int32_t));
  }
  if (code) {
    std::vector<int32_t> h(ne);
    PF_TRY(copy_out(h.data(), c.v.inc_code + e0, h.size()));
    for (auto &q : h) q -= (int32_t)(2 * l0);
    std::memcpy(code, h.data(), h.size() * sizeof(int32_t));
  }
  if (other) {
    std::vector<int32_t> h(ne);
    PF_TRY(copy_out(h.data(), c.v.inc_other + e0, h.size()));
    for (auto &q : h) q -= (int32_t)b0;
    std::memcpy(other, h.data(), h.size() * sizeof(int32_t));
  }
  return PF_OK;
}

int pf_contributions(const pf_ctx *ctx, int32_t grid, int64_t *ptr, int32_t *src) {
  PF_TRY(check_grid(ctx, grid));
  PF_ON_DEVICE(ctx->c);
  const pf::Ctx &c = ctx->c;
  if (ptr) PF_TRY(copy_out(ptr, c.contrib_ptr + c.grid_cptr_off[grid], (size_t)c.grid_nnz[grid] + 1));
  if (src)
    PF_TRY(copy_out(src, c.contrib_src + c.grid_csrc_off[grid],
                    (size_t)(c.grid_csrc_off[grid + 1] - c.grid_csrc_off[grid])));
  return PF_OK;
}

int pf_eval(pf_ctx *ctx, const double *x, const pf_overrides *ov, double *F, double *vals, void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  return pf::launch_eval(ctx->c, x, ov, F, vals, as_stream(stream));
}

int pf_eval_stage(pf_ctx *ctx, int32_t stage, const double *x, const pf_overrides *ov, double *F, double *vals,
                  void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  if (stage != PF_STAGE_PHASOR && stage != PF_STAGE_FUSED)
    return fail(PF_ERR_INVALID, "stage must be PF_STAGE_PHASOR or PF_STAGE_FUSED");
  return pf::launch_eval_stages(ctx->c, stage, x, ov, F, vals, as_stream(stream));
}

int pf_residual(pf_ctx *ctx, const double *x, double *F, void *stream) {
  if (!F) return fail(PF_ERR_INVALID, "F is NULL");
  return pf_eval(ctx, x, nullptr, F, nullptr, stream);
}

int pf_jacobian(pf_ctx *ctx, const double *x, double *vals, void *stream) {
  if (!vals) return fail(PF_ERR_INVALID, "vals is NULL");
  return pf_eval(ctx, x, nullptr, nullptr, vals, stream);
}

int pf_residual_jacobian(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream) {
  return pf_eval(ctx, x, nullptr, F, vals, stream);
}

int pf_residual_jacobian_host(pf_ctx *ctx, const double *x_host, double *F_host, double *vals_host,
                              void *stream) {
  if (!ctx || !x_host) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  pf::Ctx &c = ctx->c;
  cudaStream_t s = as_stream(stream);
  if (!c.stage_x) {
    PF_CUDA_TRY(cudaMalloc(&c.stage_x, std::max<int64_t>(c.n_x, 1) * sizeof(double)));
    PF_CUDA_TRY(cudaMalloc(&c.stage_f, std::max<int64_t>(c.n_f, 1) * sizeof(double)));
    PF_CUDA_TRY(cudaMalloc(&c.stage_v, std::max<int64_t>(c.nnz, 1) * sizeof(double)));
  }
  double *F_dev = F_host ? c.stage_f : nullptr, *v_dev = vals_host ? c.stage_v : nullptr;
  const int I = c.v.n_inst;
  const int C = std::min(I, kHostChunks);
  if (C <= 1) {
    PF_CUDA_TRY(cudaMemcpyAsync(c.stage_x, x_host, c.n_x * sizeof(double), cudaMemcpyHostToDevice, s));
    PF_TRY(pf::launch_eval(c, c.stage_x, nullptr, F_dev, v_dev, s));
    if (F_host) PF_CUDA_TRY(cudaMemcpyAsync(F_host, c.stage_f, c.n_f * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (vals_host)
      PF_CUDA_TRY(cudaMemcpyAsync(vals_host, c.stage_v, c.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    return PF_OK;
  }
  // Pipeline over chunks of instances: copy in (stream 0), evaluate (stream 1) and copy
  // out (stream 2) overlap, so the time approaches that of the largest of the three.
  if (!c.pipe_stream[0]) {
    for (auto &q : c.pipe_stream) PF_CUDA_TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    c.pipe_events.resize(2 * kHostChunks + 2);
    for (auto &e : c.pipe_events) PF_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaStream_t s_in = c.pipe_stream[0], s_ev = c.pipe_stream[1], s_out = c.pipe_stream[2];
  cudaEvent_t ev_start = c.pipe_events[2 * kHostChunks], ev_end = c.pipe_events[2 * kHostChunks + 1];
  PF_CUDA_TRY(cudaEventRecord(ev_start, s));                  // after the caller's earlier work
  PF_CUDA_TRY(cudaStreamWaitEvent(s_in, ev_start, 0));
  PF_CUDA_TRY(cudaStreamWaitEvent(s_ev, ev_start, 0));
  PF_CUDA_TRY(cudaStreamWaitEvent(s_out, ev_start, 0));
  for (int k = 0; k < C; ++k) {
    const int i0 = k ? host_chunk_end(I, C, k - 1) : 0, i1 = host_chunk_end(I, C, k);
    if (i0 == i1) continue;                                   // an empty leading chunk
    cudaEvent_t ev_in = c.pipe_events[2 * k], ev_done = c.pipe_events[2 * k + 1];
    const int64_t x0 = c.x_off[i0], nx = c.x_off[i1] - x0;
    PF_CUDA_TRY(cudaMemcpyAsync(c.stage_x + x0, x_host + x0, nx * sizeof(double), cudaMemcpyHostToDevice, s_in));
    PF_CUDA_TRY(cudaEventRecord(ev_in, s_in));
    PF_CUDA_TRY(cudaStreamWaitEvent(s_ev, ev_in, 0));
    PF_TRY(pf::launch_eval_range(c, i0, i1, c.stage_x, F_dev, v_dev, s_ev));
    PF_CUDA_TRY(cudaEventRecord(ev_done, s_ev));
    PF_CUDA_TRY(cudaStreamWaitEvent(s_out, ev_done, 0));
    if (F_host) {
      const int64_t f0 = c.f_off[i0], nf = c.f_off[i1] - f0;
      PF_CUDA_TRY(cudaMemcpyAsync(F_host + f0, c.stage_f + f0, nf * sizeof(double), cudaMemcpyDeviceToHost, s_out));
    }
    if (vals_host) {
      const int64_t v0 = c.v_off[i0], nv = c.v_off[i1] - v0;
      PF_CUDA_TRY(cudaMemcpyAsync(vals_host + v0, c.stage_v + v0, nv * sizeof(double), cudaMemcpyDeviceToHost, s_out));
    }
  }
  PF_CUDA_TRY(cudaEventRecord(ev_end, s_out));
  PF_CUDA_TRY(cudaStreamWaitEvent(s, ev_end, 0));
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  return PF_OK;
}

int pf_vjp(pf_ctx *ctx, const double *x, const pf_overrides *ov, const double *v, int32_t n_cot,
           const pf_grads *g, void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  return pf::launch_vjp(ctx->c, x, ov, v, n_cot, g, as_stream(stream));
}

int pf_newton(pf_ctx *ctx, double *x, double tol, int32_t max_iter, void *stream, pf_newton_info *info) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  return pf::newton(ctx->c, x, tol, max_iter, as_stream(stream), info);
}

int pf_newton_qlim(pf_ctx *ctx, double *x, const double *q_min, const double *q_max, uint8_t *gen_mode,
                   double *gen_qlim, double tol, int32_t max_iter, int32_t max_rounds, void *stream,
                   pf_newton_info *info, int32_t *rounds) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  int r = 0;
  PF_TRY(pf::newton_qlim(ctx->c, x, q_min, q_max, gen_mode, gen_qlim, tol, max_iter, max_rounds,
                         as_stream(stream), info, &r));
  if (rounds) *rounds = r;
  return PF_OK;
}

int pf_fdlf(pf_ctx *ctx, double *x, double tol, int32_t max_iter, void *stream, pf_newton_info *info) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  return pf::fdlf(ctx->c, x, tol, max_iter, as_stream(stream), info);
}

int pf_set_newton_solver(pf_ctx *ctx, int32_t solver) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  if (solver != PF_SOLVER_LU && solver != PF_SOLVER_QR)
    return fail(PF_ERR_INVALID, "solver must be PF_SOLVER_LU or PF_SOLVER_QR");
  ctx->c.newton_solver = solver;
  return PF_OK;
}

int pf_mismatch_norm(pf_ctx *ctx, const double *F, double *norms, void *stream) {
  if (!ctx || !F || !norms) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  return pf::newton_norms(ctx->c, F, norms, as_stream(stream));
}

int pf_newton_update(pf_ctx *ctx, double *x, const double *dx, void *stream) {
  if (!ctx || !x || !dx) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  return pf::newton_update(ctx->c, x, dx, as_stream(stream));
}

int pf_get_tuning(const pf_ctx *ctx, pf_tuning *t) {
  if (!ctx || !t) return fail(PF_ERR_INVALID, "NULL argument");
  *t = ctx->c.tuning;
  return PF_OK;
}

int pf_set_tuning(pf_ctx *ctx, const pf_tuning *t, void *stream) {
  if (!ctx || !t) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  if (t->tile_inc < pf::kMinTileInc || t->tile_inc > pf::kMaxTileInc || t->tile_inc % 32 != 0)
    return fail(PF_ERR_INVALID, "tile_inc must be 32, 64, 96 or 128");
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return fail(PF_ERR_INVALID, "ctas_per_sm must be in [0, 32]");
  if (t->split_rounds < 0 || t->split_rounds > 2) return fail(PF_ERR_INVALID, "split_rounds must be 0, 1 or 2");
  if (t->fuse_phasor != 0 && t->fuse_phasor != 1) return fail(PF_ERR_INVALID, "fuse_phasor must be 0 or 1");
  cudaStream_t s = as_stream(stream);
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  pf::Ctx &c = ctx->c;
  if (t->ctas_per_sm > 0 && !c.work_ctr) {
    void *p = nullptr;
    const size_t bytes = 2 * sizeof(unsigned long long);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return fail(PF_ERR_OOM, "cudaMalloc of the schedule counters");
    c.allocations.push_back(p);
    PF_CUDA_TRY(cudaMemset(p, 0, bytes));
    c.work_ctr = static_cast<unsigned long long *>(p);
  }
  PF_TRY(pf::use_tile_set(c, t->split_rounds, s));
  c.tuning.tile_inc = t->tile_inc;
  c.tuning.ctas_per_sm = t->ctas_per_sm;
  c.tuning.split_rounds = t->split_rounds;
  c.tuning.fuse_phasor = t->fuse_phasor;
  return PF_OK;
}

int pf_autotune(pf_ctx *ctx, const double *x, double *F, double *vals, void *stream, pf_tuning *chosen) {
  if (!ctx || !x) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  cudaStream_t s = as_stream(stream);
  const int tiles[] = {32, 64, 96, 128};
  const int ctas[] = {0, 8, 16};
  pf_tuning best = ctx->c.tuning;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  PF_CUDA_TRY(cudaEventCreate(&e0));
  PF_CUDA_TRY(cudaEventCreate(&e1));
  // milliseconds per evaluation over `reps` evaluations back to back
  auto time_evals = [&](int reps, float *per_eval) -> int {
    PF_CUDA_TRY(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) PF_TRY(pf::launch_eval(ctx->c, x, nullptr, F, vals, s));
    PF_CUDA_TRY(cudaEventRecord(e1, s));
    PF_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    PF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *per_eval = ms / reps;
    return PF_OK;
  };
  int rc = PF_OK;
  for (int k = 0; k < 2 * 3 * 4 * 3 && !rc; ++k) {   // phasor form x tile sizes x fetch widths x CTAs per SM
    const pf_tuning t{tiles[(k / 3) % 4], ctas[k % 3], (k / 12) % 3, k / 36};
    rc = pf_set_tuning(ctx, &t, stream);
    if (rc) break;
    for (int w = 0; w < 2 && !rc; ++w) rc = pf::launch_eval(ctx->c, x, nullptr, F, vals, s);
    // a batch of about 2 ms (5 to 200 evaluations), timed twice, the faster kept: short
    // evaluations are otherwise compared on the noise of a few microseconds
    float probe = 0.f, t1 = 0.f, t2 = 0.f;
    if (!rc) rc = time_evals(3, &probe);
    const int reps = std::max(5, std::min(200, (int)std::ceil(2.0f / std::max(probe, 1e-4f))));
    if (!rc) rc = time_evals(reps, &t1);
    if (!rc) rc = time_evals(reps, &t2);
    if (rc) break;
    const float ms = std::min(t1, t2);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  PF_TRY(pf_set_tuning(ctx, &best, stream));
  if (chosen) *chosen = best;
  return PF_OK;
}

int pf_autotune_cache(pf_ctx *ctx, const char *path, const double *x, double *F, double *vals, void *stream,
                      pf_tuning *chosen, int32_t *from_cache) {
  if (!ctx || !path) return fail(PF_ERR_INVALID, "NULL argument");
  PF_ON_DEVICE(ctx->c);
  if (from_cache) *from_cache = 0;
  const std::string key = tuning_key(ctx->c);
  if (key.empty()) return fail(PF_ERR_CUDA, "cannot query the device for the tuning key");
  {
    std::ifstream in(path);
    std::string line;
    pf_tuning found{};
    bool have = false;
    while (in && std::getline(in, line)) {             // the last valid entry for the key wins
      std::istringstream ls(line);
      std::string tag, k;
      pf_tuning t{};
      if (ls >> tag >> k >> t.tile_inc >> t.ctas_per_sm >> t.split_rounds >> t.fuse_phasor && tag == kTuningTag &&
          k == key &&
          tuning_valid(t)) {
        found = t;
        have = true;
      }
    }
    if (have) {
      PF_TRY(pf_set_tuning(ctx, &found, stream));
      if (chosen) *chosen = found;
      if (from_cache) *from_cache = 1;
      return PF_OK;
    }
  }
  pf_tuning t{};
  PF_TRY(pf_autotune(ctx, x, F, vals, stream, &t));
  std::ofstream out(path, std::ios::app);
  if (out)
    out << kTuningTag << ' ' << key << ' ' << t.tile_inc << ' ' << t.ctas_per_sm << ' ' << t.split_rounds << ' '
        << t.fuse_phasor << '\n';
  if (chosen) *chosen = t;
  return PF_OK;
}

int pf_sincos(pf_ctx *ctx, const double *theta, int64_t n, double *cos_out, double *sin_out, void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  return pf::launch_sincos(ctx->c, theta, n, cos_out, sin_out, as_stream(stream));
}

int pf_voltage_records(pf_ctx *ctx, const double *x, double *rec, void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  if (!x || !rec) return fail(PF_ERR_INVALID, "x or rec is NULL");
  const cudaStream_t s = as_stream(stream);
  PF_TRY(pf::launch_phasor(ctx->c.v, ctx->c.num_sms, x, s, false));
  PF_CUDA_TRY(cudaMemcpyAsync(rec, ctx->c.v.phasor, sizeof(double) * 4 * (size_t)ctx->c.v.n_bus_inst,
                              cudaMemcpyDeviceToDevice, s));
  return PF_OK;
}

const char *pf_error_string(int32_t code) {
  switch (code) {
    case PF_OK: return "ok";
    case PF_ERR_INVALID: return "invalid argument or system";
    case PF_ERR_OOM: return "out of memory";
    case PF_ERR_CUDA: return "CUDA error";
    case PF_ERR_TIMEOUT: return "bounded device wait timed out";
    case PF_ERR_UNSUPPORTED: return "outside the library's limits";
    case PF_ERR_DEVICE: return "device-side consistency check failed";
    case PF_ERR_NUMERIC: return "numerically singular Jacobian";
    default: return "unknown error code";
  }
}

const char *pf_last_error(void) { return pf::g_last_error.c_str(); }

int pf_check_device(pf_ctx *ctx, void *stream) {
  if (!ctx) return fail(PF_ERR_INVALID, "ctx is NULL");
  PF_ON_DEVICE(ctx->c);
  int32_t h = 0;
  cudaStream_t s = as_stream(stream);
  PF_CUDA_TRY(cudaMemcpyAsync(&h, ctx->c.v.dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  PF_CUDA_TRY(cudaMemsetAsync(ctx->c.v.dev_error, 0, sizeof(int32_t), s));
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  if (h & pf::kErrTimeout) return fail(PF_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h) return fail(PF_ERR_DEVICE, "device error flag " + std::to_string(h));
  if (ctx->c.work_ctr) {
    // the schedule counters of persistent k_fused grids are zero between launches
    unsigned long long w[2];
    PF_CUDA_TRY(cudaMemcpyAsync(w, ctx->c.work_ctr, sizeof(w), cudaMemcpyDeviceToHost, s));
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    for (unsigned long long x : w)
      if (x) return fail(PF_ERR_DEVICE, "schedule counter not reset");
  }
  return PF_OK;
}

}  // extern "C"
