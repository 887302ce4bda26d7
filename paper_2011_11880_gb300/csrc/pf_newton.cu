// Newton iterations around the hot path: tasks (3) and (4) of Newton power
// flow (Sec. I).  Every iteration evaluates F and J with the library's
// kernels, checks convergence (max |F| per instance, on the device), solves
// J dx = F per instance with cuSOLVER's sparse QR (a library call: the linear
// solve is outside the hot path) and updates the unknowns, x <- x - dx, on
// the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#define DISABLE_CUSOLVER_DEPRECATED
#include <cusolverRf.h>
#include <cusolverSp.h>
#include <cusolverSp_LOWLEVEL_PREVIEW.h>
#include <cusparse.h>

#include "pf_internal.cuh"

namespace pf {
namespace {

// max |F| over the rows of each instance.  |F| is non-negative, so its bit
// pattern orders like the value and an integer atomicMax gives the exact
// maximum in any order (a NaN, positive after fabs, wins over every number).
__global__ void k_mismatch_norm(View v, const int64_t *__restrict__ f_off, int64_t n_f, const double *__restrict__ F,
                                unsigned long long *__restrict__ norm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_f; r += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(f_off, v.n_inst, r);
    atomicMax(norm + inst, (unsigned long long)__double_as_longlong(fabs(F[r])));
  }
}

// Task (4): x <- x - dx on the unknowns of every instance.  Reduced
// formulation: theta of a bus with a P row (the slack has none) and V of a
// bus with a Q row (PQ-type buses), at the bus's row index; extended: the
// columns are numbered like x itself.
__global__ void k_newton_update(View v, double *__restrict__ x, const double *__restrict__ dx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t lb = q - v.inst_bus_off[inst];
    const int64_t b = v.grid_bus_off[g] + lb;
    const int32_t nb = v.grid_nbus[g];
    double *__restrict__ xi = x + v.inst_x_off[inst];
    const double *__restrict__ di = dx + v.inst_f_off[inst];
    const int4 m = v.bus_meta[b];                       // {row_p, row_q, ...}
    if (m.x >= 0) xi[lb] = __dsub_rn(xi[lb], di[m.x]);
    if (m.y >= 0) xi[nb + lb] = __dsub_rn(xi[nb + lb], di[m.y]);
    if (v.formulation == PF_EXTENDED && lb == 0) {     // generator Q_g and slack P_s columns
      const int32_t extra = v.grid_ngen[g] + 1;
      for (int32_t j = 0; j < extra; ++j) xi[2 * nb + j] = __dsub_rn(xi[2 * nb + j], di[2 * nb + j]);
    }
  }
}

// Reactive limits (Sec. II-A): a generator in voltage control whose Q_g lies
// above q_max or below q_min is switched to that limit.  One thread per
// instance-generator; counts the switches.
__global__ void k_qlim_check(View v, const double *__restrict__ x, const double *__restrict__ q_min,
                             const double *__restrict__ q_max, uint8_t *__restrict__ mode, double *__restrict__ qlim,
                             int64_t n_gen_inst, unsigned int *__restrict__ switched) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_gen_inst; q += stride) {
    if (mode[q] != 0) continue;
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_gen_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t gi = q - v.inst_gen_off[inst];
    const double qg = x[v.inst_x_off[inst] + 2 * (int64_t)v.grid_nbus[g] + gi];
    if (qg > q_max[q]) {
      mode[q] = 1;
      qlim[q] = q_max[q];
      atomicAdd(switched, 1u);
    } else if (qg < q_min[q]) {
      mode[q] = 2;
      qlim[q] = q_min[q];
      atomicAdd(switched, 1u);
    }
  }
}

// LU refactorization of one instance's J (the pattern is fixed, so the
// ordering and pivoting of a first LU are reused): a host LU of the first J
// with a METIS fill-reducing ordering and partial pivoting gives P, Q, L, U
// (P A Q^T = L U); cuSOLVER-Rf then refactors every later J on the device and
// solves with the factors.
struct RfInst {
  cusolverRfHandle_t rf = nullptr;
  int *dP = nullptr, *dQ = nullptr;
  double *dT = nullptr;
};

struct Solver {
  cusolverSpHandle_t sp = nullptr;
  cusparseMatDescr_t descr = nullptr;
  std::vector<RfInst> rf;                 // per instance, created on first use
  std::vector<std::vector<int>> h_rowptr, h_colind;   // per grid, host copies of the pattern
  double *F = nullptr, *vals = nullptr, *dx = nullptr;
  unsigned long long *norm = nullptr;
  int64_t *f_off = nullptr;
  unsigned int *switched = nullptr;
};

int make_solver(Ctx &c, Solver **out) {
  if (c.newton) {
    *out = static_cast<Solver *>(c.newton);
    return PF_OK;
  }
  Solver *S = new Solver();
  c.newton = S;
  c.newton_free = [](void *p) {
    Solver *s = static_cast<Solver *>(p);
    for (RfInst &r : s->rf) {
      if (r.rf) cusolverRfDestroy(r.rf);
      if (r.dP) cudaFree(r.dP);
      if (r.dQ) cudaFree(r.dQ);
      if (r.dT) cudaFree(r.dT);
    }
    if (s->sp) cusolverSpDestroy(s->sp);
    if (s->descr) cusparseDestroyMatDescr(s->descr);
    delete s;
  };
  if (cusolverSpCreate(&S->sp) != CUSOLVER_STATUS_SUCCESS) return fail(PF_ERR_CUDA, "cusolverSpCreate failed");
  if (cusparseCreateMatDescr(&S->descr) != CUSPARSE_STATUS_SUCCESS)
    return fail(PF_ERR_CUDA, "cusparseCreateMatDescr failed");
  cusparseSetMatType(S->descr, CUSPARSE_MATRIX_TYPE_GENERAL);
  cusparseSetMatIndexBase(S->descr, CUSPARSE_INDEX_BASE_ZERO);
  PF_TRY(dev_alloc(c, &S->F, c.n_f));
  PF_TRY(dev_alloc(c, &S->vals, c.nnz));
  PF_TRY(dev_alloc(c, &S->dx, c.n_f));
  PF_TRY(dev_alloc(c, &S->norm, c.v.n_inst));
  PF_TRY(dev_alloc(c, &S->switched, 1));
  PF_TRY(upload(c, &S->f_off, c.f_off, nullptr));
  *out = S;
  return PF_OK;
}

int launch_norm(Ctx &c, const int64_t *f_off, const double *F, unsigned long long *norm, cudaStream_t s) {
  PF_CUDA_TRY(cudaMemsetAsync(norm, 0, c.v.n_inst * sizeof(unsigned long long), s));
  if (c.n_f > 0) {
    const int64_t blocks = std::min<int64_t>((c.n_f + 255) / 256, (int64_t)c.num_sms * 16);
    k_mismatch_norm<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(c.v, f_off, c.n_f, F, norm);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

int launch_update(Ctx &c, double *x, const double *dx, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((c.v.n_bus_inst + 255) / 256, (int64_t)c.num_sms * 16);
  k_newton_update<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(c.v, x, dx);
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

#define PF_SOLVER_TRY(expr, what)                                                             \
  do {                                                                                        \
    const cusolverStatus_t _st = (expr);                                                     \
    if (_st != CUSOLVER_STATUS_SUCCESS)                                                      \
      return fail(PF_ERR_CUDA, std::string(what) + " failed with status " + std::to_string((int)_st)); \
  } while (0)

// First factorization of instance i: host LU of its current J, then the
// device refactorization object.
int rf_setup(Ctx &c, Solver *S, int i, cudaStream_t s) {
  const int g = c.inst_grid[i];
  const int n = c.grid_nf[g], nnz = c.grid_nnz[g];
  if (S->h_rowptr.empty()) {
    S->h_rowptr.resize(c.v.n_grids);
    S->h_colind.resize(c.v.n_grids);
  }
  std::vector<int> &rp = S->h_rowptr[g], &ci = S->h_colind[g];
  if (rp.empty()) {
    rp.resize(n + 1);
    ci.resize(nnz);
    PF_CUDA_TRY(cudaMemcpy(rp.data(), c.rowptr + c.grid_row_off[g], (n + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    PF_CUDA_TRY(cudaMemcpy(ci.data(), c.colind + c.grid_nnz_off[g], nnz * sizeof(int), cudaMemcpyDeviceToHost));
  }
  std::vector<double> va(nnz);
  PF_CUDA_TRY(cudaMemcpyAsync(va.data(), S->vals + c.v_off[i], nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  // fill-reducing symmetric ordering r, B = A(r, r)
  std::vector<int> r(n), rpB(rp), ciB(ci), map(nnz);
  PF_SOLVER_TRY(cusolverSpXcsrmetisndHost(S->sp, n, nnz, S->descr, rp.data(), ci.data(), nullptr, r.data()),
                "cusolverSpXcsrmetisndHost");
  size_t bytes = 0;
  PF_SOLVER_TRY(cusolverSpXcsrperm_bufferSizeHost(S->sp, n, n, nnz, S->descr, rpB.data(), ciB.data(), r.data(),
                                                  r.data(), &bytes), "cusolverSpXcsrperm_bufferSizeHost");
  std::vector<char> buf(bytes + 1);
  for (int k = 0; k < nnz; ++k) map[k] = k;
  PF_SOLVER_TRY(cusolverSpXcsrpermHost(S->sp, n, n, nnz, S->descr, rpB.data(), ciB.data(), r.data(), r.data(),
                                       map.data(), buf.data()), "cusolverSpXcsrpermHost");
  std::vector<double> vb(nnz);
  for (int k = 0; k < nnz; ++k) vb[k] = va[map[k]];
  // host LU with partial pivoting
  csrluInfoHost_t info = nullptr;
  PF_SOLVER_TRY(cusolverSpCreateCsrluInfoHost(&info), "cusolverSpCreateCsrluInfoHost");
  struct InfoGuard {
    csrluInfoHost_t p;
    ~InfoGuard() { cusolverSpDestroyCsrluInfoHost(p); }
  } guard{info};
  PF_SOLVER_TRY(cusolverSpXcsrluAnalysisHost(S->sp, n, nnz, S->descr, rpB.data(), ciB.data(), info),
                "cusolverSpXcsrluAnalysisHost");
  size_t internal = 0, work = 0;
  PF_SOLVER_TRY(cusolverSpDcsrluBufferInfoHost(S->sp, n, nnz, S->descr, vb.data(), rpB.data(), ciB.data(), info,
                                               &internal, &work), "cusolverSpDcsrluBufferInfoHost");
  std::vector<char> wbuf(work + 1);
  PF_SOLVER_TRY(cusolverSpDcsrluFactorHost(S->sp, n, nnz, S->descr, vb.data(), rpB.data(), ciB.data(), info, 1.0,
                                           wbuf.data()), "cusolverSpDcsrluFactorHost");
  int singular = -1;
  PF_SOLVER_TRY(cusolverSpDcsrluZeroPivotHost(S->sp, info, 1e-14, &singular), "cusolverSpDcsrluZeroPivotHost");
  if (singular >= 0)
    return fail(PF_ERR_NUMERIC, "J is singular (instance " + std::to_string(i) + ", pivot " +
                                    std::to_string(singular) + ")");
  int nnzL = 0, nnzU = 0;
  PF_SOLVER_TRY(cusolverSpXcsrluNnzHost(S->sp, &nnzL, &nnzU, info), "cusolverSpXcsrluNnzHost");
  std::vector<int> Plu(n), Qlu(n), rpL(n + 1), ciL(nnzL), rpU(n + 1), ciU(nnzU);
  std::vector<double> vL(nnzL), vU(nnzU);
  PF_SOLVER_TRY(cusolverSpDcsrluExtractHost(S->sp, Plu.data(), Qlu.data(), S->descr, vL.data(), rpL.data(),
                                            ciL.data(), S->descr, vU.data(), rpU.data(), ciU.data(), info,
                                            wbuf.data()), "cusolverSpDcsrluExtractHost");
  // permutations relative to A: the ordering composed with the pivoting
  std::vector<int> P(n), Q(n);
  for (int j = 0; j < n; ++j) {
    P[j] = r[Plu[j]];
    Q[j] = r[Qlu[j]];
  }
  RfInst &R = S->rf[i];
  PF_SOLVER_TRY(cusolverRfCreate(&R.rf), "cusolverRfCreate");
  PF_SOLVER_TRY(cusolverRfSetResetValuesFastMode(R.rf, CUSOLVERRF_RESET_VALUES_FAST_MODE_ON),
                "cusolverRfSetResetValuesFastMode");
  PF_SOLVER_TRY(cusolverRfSetMatrixFormat(R.rf, CUSOLVERRF_MATRIX_FORMAT_CSR, CUSOLVERRF_UNIT_DIAGONAL_ASSUMED_L),
                "cusolverRfSetMatrixFormat");
  PF_SOLVER_TRY(cusolverRfSetAlgs(R.rf, CUSOLVERRF_FACTORIZATION_ALG0, CUSOLVERRF_TRIANGULAR_SOLVE_ALG1),
                "cusolverRfSetAlgs");
  PF_SOLVER_TRY(cusolverRfSetupHost(n, nnz, rp.data(), ci.data(), va.data(), nnzL, rpL.data(), ciL.data(),
                                    vL.data(), nnzU, rpU.data(), ciU.data(), vU.data(), P.data(), Q.data(), R.rf),
                "cusolverRfSetupHost");
  PF_SOLVER_TRY(cusolverRfAnalyze(R.rf), "cusolverRfAnalyze");
  PF_CUDA_TRY(cudaMalloc(&R.dP, n * sizeof(int)));
  PF_CUDA_TRY(cudaMalloc(&R.dQ, n * sizeof(int)));
  PF_CUDA_TRY(cudaMalloc(&R.dT, n * sizeof(double)));
  PF_CUDA_TRY(cudaMemcpy(R.dP, P.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  PF_CUDA_TRY(cudaMemcpy(R.dQ, Q.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  return PF_OK;
}

// J dx = F for instance i by LU refactorization (S->dx[i] = S->F[i] on entry).
int rf_solve(Ctx &c, Solver *S, int i, cudaStream_t s) {
  const int g = c.inst_grid[i];
  const int n = c.grid_nf[g], nnz = c.grid_nnz[g];
  if (S->rf.empty()) S->rf.resize(c.v.n_inst);
  RfInst &R = S->rf[i];
  if (!R.rf) PF_TRY(rf_setup(c, S, i, s));
  {
    // the factors are computed by the refactorization (after the setup, too)
    PF_SOLVER_TRY(cusolverRfResetValues(n, nnz, c.rowptr + c.grid_row_off[g], c.colind + c.grid_nnz_off[g],
                                        S->vals + c.v_off[i], R.dP, R.dQ, R.rf), "cusolverRfResetValues");
    PF_SOLVER_TRY(cusolverRfRefactor(R.rf), "cusolverRfRefactor");
  }
  PF_SOLVER_TRY(cusolverRfSolve(R.rf, R.dP, R.dQ, 1, R.dT, n, S->dx + c.f_off[i], n), "cusolverRfSolve");
  return PF_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

int newton_norms(Ctx &c, const double *F, double *norms, cudaStream_t s) {
  Solver *S;
  PF_TRY(make_solver(c, &S));
  PF_TRY(launch_norm(c, S->f_off, F, reinterpret_cast<unsigned long long *>(norms), s));
  return PF_OK;
}

int newton_update(Ctx &c, double *x, const double *dx, cudaStream_t s) { return launch_update(c, x, dx, s); }

int newton(Ctx &c, double *x, double tol, int max_iter, cudaStream_t s, pf_newton_info *info,
           const pf_overrides *ov) {
  if (!x) return fail(PF_ERR_INVALID, "x is NULL");
  if (max_iter < 0 || !(tol >= 0.0)) return fail(PF_ERR_INVALID, "max_iter must be >= 0 and tol >= 0");
  Solver *S;
  PF_TRY(make_solver(c, &S));
  if (cusolverSpSetStream(S->sp, s) != CUSOLVER_STATUS_SUCCESS) return fail(PF_ERR_CUDA, "cusolverSpSetStream failed");
  pf_newton_info r{};
  const int I = c.v.n_inst;
  std::vector<unsigned long long> h_norm(I);
  for (int it = 0;; ++it) {
    auto t0 = std::chrono::steady_clock::now();
    PF_TRY(launch_eval(c, x, ov, S->F, S->vals, s));
    PF_TRY(launch_norm(c, S->f_off, S->F, S->norm, s));
    PF_CUDA_TRY(cudaMemcpyAsync(h_norm.data(), S->norm, I * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    r.eval_ms += ms_since(t0);
    double worst = 0.0;
    bool done = true;
    std::vector<char> active(I, 0);
    for (int i = 0; i < I; ++i) {
      double n;
      std::memcpy(&n, &h_norm[i], sizeof(double));
      if (!(n <= worst)) worst = n;            // NaN propagates
      active[i] = !(n <= tol);
      done = done && !active[i];
    }
    r.max_mismatch = worst;
    if (done) {
      r.converged = 1;
      break;
    }
    if (it >= max_iter || worst != worst) break;
    // task (3): J dx = F per instance that has not converged (dx = 0 for the others)
    t0 = std::chrono::steady_clock::now();
    PF_CUDA_TRY(cudaMemsetAsync(S->dx, 0, c.n_f * sizeof(double), s));
    for (int i = 0; i < I; ++i) {
      if (!active[i]) continue;
      const int g = c.inst_grid[i];
      const int n = c.grid_nf[g], nnz = c.grid_nnz[g];
      if (n == 0) continue;
      if (c.newton_solver == PF_SOLVER_LU) {
        PF_CUDA_TRY(cudaMemcpyAsync(S->dx + c.f_off[i], S->F + c.f_off[i], n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        PF_CUDA_TRY(cudaStreamSynchronize(s));
        PF_TRY(rf_solve(c, S, i, s));
        continue;
      }
      int singular = -1;
      const cusolverStatus_t st = cusolverSpDcsrlsvqr(
          S->sp, n, nnz, S->descr, S->vals + c.v_off[i], c.rowptr + c.grid_row_off[g], c.colind + c.grid_nnz_off[g],
          S->F + c.f_off[i], 1e-14, /*reorder: METIS nested dissection*/ 3, S->dx + c.f_off[i], &singular);
      if (st != CUSOLVER_STATUS_SUCCESS)
        return fail(PF_ERR_CUDA, "cusolverSpDcsrlsvqr failed with status " + std::to_string((int)st));
      if (singular >= 0)
        return fail(PF_ERR_NUMERIC, "J is singular (instance " + std::to_string(i) + ", iteration " +
                                        std::to_string(it) + ", pivot " + std::to_string(singular) + ")");
    }
    // cuSOLVER-Rf works on the legacy default stream: wait for all of it
    if (c.newton_solver == PF_SOLVER_LU) PF_CUDA_TRY(cudaDeviceSynchronize());
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    r.solve_ms += ms_since(t0);
    // task (4)
    t0 = std::chrono::steady_clock::now();
    PF_TRY(launch_update(c, x, S->dx, s));
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    r.update_ms += ms_since(t0);
    r.iterations = it + 1;
  }
  if (info) *info = r;
  return PF_OK;
}

int newton_qlim(Ctx &c, double *x, const double *q_min, const double *q_max, uint8_t *mode, double *qlim, double tol,
                int max_iter, int max_rounds, cudaStream_t s, pf_newton_info *info, int *rounds) {
  if (c.v.formulation != PF_EXTENDED) return fail(PF_ERR_INVALID, "reactive limits need the extended formulation");
  if (!x || !mode || !qlim || ((!q_min || !q_max) && c.n_gen_inst > 0))
    return fail(PF_ERR_INVALID, "x, q_min, q_max, gen_mode and gen_qlim must not be NULL");
  if (max_rounds < 1) return fail(PF_ERR_INVALID, "max_rounds must be >= 1");
  Solver *S;
  PF_TRY(make_solver(c, &S));
  pf_overrides ov{};
  ov.gen_mode = mode;
  ov.gen_qlim = qlim;
  pf_newton_info total{};
  int r = 0;
  for (r = 1; r <= max_rounds; ++r) {
    pf_newton_info one{};
    PF_TRY(newton(c, x, tol, max_iter, s, &one, &ov));
    total.iterations += one.iterations;
    total.eval_ms += one.eval_ms;
    total.solve_ms += one.solve_ms;
    total.update_ms += one.update_ms;
    total.max_mismatch = one.max_mismatch;
    total.converged = 0;
    if (!one.converged) break;
    unsigned int h_switched = 0;
    if (c.n_gen_inst > 0) {
      PF_CUDA_TRY(cudaMemsetAsync(S->switched, 0, sizeof(unsigned int), s));
      const int64_t blocks = std::min<int64_t>((c.n_gen_inst + 255) / 256, (int64_t)c.num_sms * 16);
      k_qlim_check<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(c.v, x, q_min, q_max, mode, qlim,
                                                                         c.n_gen_inst, S->switched);
      PF_CUDA_TRY(cudaGetLastError());
      PF_CUDA_TRY(cudaMemcpyAsync(&h_switched, S->switched, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
      PF_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (h_switched == 0) {
      total.converged = 1;
      break;
    }
  }
  if (info) *info = total;
  if (rounds) *rounds = std::min(r, max_rounds);
  return PF_OK;
}

}  // namespace pf
