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

// Fast decoupled half-iteration, per instance bus with a row of the half
// (P for half 0, Q for half 1): rhs = -F / V at the bus's row.
__global__ void k_fdlf_rhs(View v, const double *__restrict__ F, const double *__restrict__ x,
                           double *__restrict__ rhs, int half) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t lb = q - v.inst_bus_off[inst];
    const int4 m = v.bus_meta[v.grid_bus_off[g] + lb];
    const int32_t row = half == 0 ? m.x : m.y;
    if (row < 0) continue;
    const int64_t f0 = v.inst_f_off[inst];
    const double V = x[v.inst_x_off[inst] + v.grid_nbus[g] + lb];
    rhs[f0 + row] = -F[f0 + row] / V;
  }
}

// ... then theta (half 0) or V (half 1) += the solution at the bus's row.
__global__ void k_fdlf_update(View v, double *__restrict__ x, const double *__restrict__ d, int half) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t lb = q - v.inst_bus_off[inst];
    const int4 m = v.bus_meta[v.grid_bus_off[g] + lb];
    const int32_t row = half == 0 ? m.x : m.y;
    if (row < 0) continue;
    const int64_t xi = v.inst_x_off[inst] + (half == 0 ? 0 : v.grid_nbus[g]) + lb;
    x[xi] = __dadd_rn(x[xi], d[v.inst_f_off[inst] + row]);
  }
}

struct Solver {
  cusolverSpHandle_t sp = nullptr;
  cusparseMatDescr_t descr = nullptr;
  std::vector<RfInst> rf;                 // per instance, created on first use
  std::vector<RfInst> fd1, fd2;           // fast decoupled: B' and B'' per (grid, outage) pair
  std::vector<int> fd_n1;                 // per pair: rows of B' (the rows of B'' follow)
  std::vector<int> fd_of_inst;            // per instance: its pair
  double *rhs = nullptr;                  // fast decoupled right-hand sides, [n_f]
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
    for (auto *list : {&s->rf, &s->fd1, &s->fd2})
      for (RfInst &r : *list) {
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

// Host LU of a CSR matrix (rp, ci, va; n rows) with a METIS fill-reducing
// ordering and partial pivoting, handed to a cuSOLVER-Rf object that
// refactors later values of the same pattern on the device.
int rf_factor_host(Solver *S, int n, const std::vector<int> &rp, const std::vector<int> &ci,
                   const std::vector<double> &va, RfInst &R, const std::string &what) {
  const int nnz = rp[n];
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
    return fail(PF_ERR_NUMERIC, what + " is singular (pivot " + std::to_string(singular) + ")");
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
  PF_SOLVER_TRY(cusolverRfCreate(&R.rf), "cusolverRfCreate");
  PF_SOLVER_TRY(cusolverRfSetResetValuesFastMode(R.rf, CUSOLVERRF_RESET_VALUES_FAST_MODE_ON),
                "cusolverRfSetResetValuesFastMode");
  PF_SOLVER_TRY(cusolverRfSetMatrixFormat(R.rf, CUSOLVERRF_MATRIX_FORMAT_CSR, CUSOLVERRF_UNIT_DIAGONAL_ASSUMED_L),
                "cusolverRfSetMatrixFormat");
  PF_SOLVER_TRY(cusolverRfSetAlgs(R.rf, CUSOLVERRF_FACTORIZATION_ALG0, CUSOLVERRF_TRIANGULAR_SOLVE_ALG1),
                "cusolverRfSetAlgs");
  PF_SOLVER_TRY(cusolverRfSetupHost(n, nnz, const_cast<int *>(rp.data()), const_cast<int *>(ci.data()),
                                    const_cast<double *>(va.data()), nnzL, rpL.data(), ciL.data(),
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

// First factorization of instance i: host LU of its current J.
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
  return rf_factor_host(S, n, rp, ci, va, S->rf[i], "J of instance " + std::to_string(i));
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

namespace {

// CSR (sorted columns, duplicates summed in insertion order) of triplets.
void triplets_to_csr(int n, std::vector<std::pair<int64_t, double>> &t, std::vector<int> &rp, std::vector<int> &ci,
                     std::vector<double> &va) {
  std::stable_sort(t.begin(), t.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
  rp.assign(n + 1, 0);
  ci.clear();
  va.clear();
  for (size_t k = 0; k < t.size();) {
    const int64_t key = t[k].first;
    double sum = t[k].second;
    size_t j = k + 1;
    for (; j < t.size() && t[j].first == key; ++j) sum += t[j].second;
    const int row = (int)(key / n), col = (int)(key % n);
    ci.push_back(col);
    va.push_back(sum);
    rp[row + 1]++;
    k = j;
  }
  for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
}

// B' and B'' of grid g with global branch `outage` out of service (-1:
// none), XB variant, built on the host from the device copies of the grid's
// data and factored once into slot k.
int fdlf_setup(Ctx &c, Solver *S, int g, int32_t outage, int k) {
  const View &v = c.v;
  const int64_t b0 = c.grid_bus_off[g], nb = c.grid_bus_off[g + 1] - b0;
  const int64_t l0 = c.grid_br_off[g], nl = c.grid_br_off[g + 1] - l0;
  std::vector<int32_t> from(nl), to(nl);
  std::vector<double> r(nl), x(nl), bc(nl), tap(nl);
  std::vector<uint8_t> st(nl);
  std::vector<double2> sh(nb);
  std::vector<int4> meta(nb);
  PF_CUDA_TRY(cudaMemcpy(from.data(), v.br_from + l0, nl * sizeof(int32_t), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(to.data(), v.br_to + l0, nl * sizeof(int32_t), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(r.data(), v.br_r + l0, nl * sizeof(double), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(x.data(), v.br_x + l0, nl * sizeof(double), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(bc.data(), v.br_b + l0, nl * sizeof(double), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(tap.data(), v.br_tap + l0, nl * sizeof(double), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(st.data(), v.br_status + l0, nl * sizeof(uint8_t), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(sh.data(), v.bus_sh + b0, nb * sizeof(double2), cudaMemcpyDeviceToHost));
  PF_CUDA_TRY(cudaMemcpy(meta.data(), v.bus_meta + b0, nb * sizeof(int4), cudaMemcpyDeviceToHost));
  int n1 = 0, n2 = 0;
  for (const int4 &m : meta) {
    n1 += m.x >= 0;
    n2 += m.y >= 0;
  }
  // rows: P row of a bus (0..n1), Q row minus n1 (0..n2)
  std::vector<std::pair<int64_t, double>> t1, t2;
  auto put = [](std::vector<std::pair<int64_t, double>> &t, int n, int i, int j, double val) {
    if (i >= 0 && j >= 0) t.push_back({(int64_t)i * n + j, val});
  };
  for (int64_t b = 0; b < nb; ++b) {               // keep every diagonal in the pattern
    put(t1, n1, meta[b].x, meta[b].x, 0.0);
    if (meta[b].y >= 0) put(t2, n2, meta[b].y - n1, meta[b].y - n1, 0.0);
  }
  for (int64_t l = 0; l < nl; ++l) {
    if (!st[l] || l0 + l == outage) continue;
    const int64_t f = from[l] - b0, t = to[l] - b0;
    const int pf = meta[f].x, pt = meta[t].x;
    const int qf = meta[f].y >= 0 ? meta[f].y - n1 : -1, qt = meta[t].y >= 0 ? meta[t].y - n1 : -1;
    const double y1 = 1.0 / x[l];
    put(t1, n1, pf, pf, y1);
    put(t1, n1, pt, pt, y1);
    put(t1, n1, pf, pt, -y1);
    put(t1, n1, pt, pf, -y1);
    const double bs = -x[l] / (r[l] * r[l] + x[l] * x[l]);
    put(t2, n2, qf, qf, -(bs + 0.5 * bc[l]) / (tap[l] * tap[l]));
    put(t2, n2, qt, qt, -(bs + 0.5 * bc[l]));
    put(t2, n2, qf, qt, bs / tap[l]);
    put(t2, n2, qt, qf, bs / tap[l]);
  }
  for (int64_t b = 0; b < nb; ++b)
    if (meta[b].y >= 0) put(t2, n2, meta[b].y - n1, meta[b].y - n1, -sh[b].y);
  S->fd_n1[k] = n1;
  for (int which = 0; which < 2; ++which) {
    const int n = which == 0 ? n1 : n2;
    if (n == 0) continue;
    std::vector<int> rp, ci;
    std::vector<double> va;
    triplets_to_csr(n, which == 0 ? t1 : t2, rp, ci, va);
    RfInst &R = which == 0 ? S->fd1[k] : S->fd2[k];
    PF_TRY(rf_factor_host(S, n, rp, ci, va, R, which == 0 ? "B'" : "B''"));
    // the factors come from a refactorization of the same values
    int *drp, *dci;
    double *dva;
    PF_CUDA_TRY(cudaMalloc(&drp, (n + 1) * sizeof(int)));
    PF_CUDA_TRY(cudaMalloc(&dci, rp[n] * sizeof(int)));
    PF_CUDA_TRY(cudaMalloc(&dva, rp[n] * sizeof(double)));
    PF_CUDA_TRY(cudaMemcpy(drp, rp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice));
    PF_CUDA_TRY(cudaMemcpy(dci, ci.data(), rp[n] * sizeof(int), cudaMemcpyHostToDevice));
    PF_CUDA_TRY(cudaMemcpy(dva, va.data(), rp[n] * sizeof(double), cudaMemcpyHostToDevice));
    const cusolverStatus_t s1 = cusolverRfResetValues(n, rp[n], drp, dci, dva, R.dP, R.dQ, R.rf);
    const cusolverStatus_t s2 = s1 == CUSOLVER_STATUS_SUCCESS ? cusolverRfRefactor(R.rf) : s1;
    cudaDeviceSynchronize();
    cudaFree(drp);
    cudaFree(dci);
    cudaFree(dva);
    if (s2 != CUSOLVER_STATUS_SUCCESS)
      return fail(PF_ERR_CUDA, "cuSOLVER-Rf refactorization of the fast decoupled matrices failed");
  }
  return PF_OK;
}

}  // namespace

int fdlf(Ctx &c, double *x, double tol, int max_iter, cudaStream_t s, pf_newton_info *info) {
  if (c.v.formulation != PF_REDUCED) return fail(PF_ERR_INVALID, "the fast decoupled method uses the reduced formulation");
  if (!x) return fail(PF_ERR_INVALID, "x is NULL");
  if (max_iter < 0 || !(tol >= 0.0)) return fail(PF_ERR_INVALID, "max_iter must be >= 0 and tol >= 0");
  Solver *S;
  PF_TRY(make_solver(c, &S));
  const int I = c.v.n_inst;
  if (S->fd_of_inst.empty()) {
    // one pair of factored matrices per distinct (grid, outage) of the instances
    std::vector<std::pair<int, int32_t>> keys;
    S->fd_of_inst.assign(I, -1);
    for (int i = 0; i < I; ++i) {
      const std::pair<int, int32_t> key{c.inst_grid[i], c.inst_outage[i]};
      int k = -1;
      for (size_t j = 0; j < keys.size(); ++j)
        if (keys[j] == key) k = (int)j;
      if (k < 0) {
        k = (int)keys.size();
        keys.push_back(key);
      }
      S->fd_of_inst[i] = k;
    }
    S->fd1.resize(keys.size());
    S->fd2.resize(keys.size());
    S->fd_n1.assign(keys.size(), 0);
    PF_TRY(dev_alloc(c, &S->rhs, c.n_f));
    for (size_t k = 0; k < keys.size(); ++k) PF_TRY(fdlf_setup(c, S, keys[k].first, keys[k].second, (int)k));
  }
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((c.v.n_bus_inst + 255) / 256, (int64_t)c.num_sms * 16));
  pf_newton_info r{};
  std::vector<unsigned long long> h_norm(I);
  for (int it = 0;; ++it) {
    auto t0 = std::chrono::steady_clock::now();
    PF_TRY(launch_eval(c, x, nullptr, S->F, nullptr, s));
    PF_TRY(launch_norm(c, S->f_off, S->F, S->norm, s));
    PF_CUDA_TRY(cudaMemcpyAsync(h_norm.data(), S->norm, I * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PF_CUDA_TRY(cudaStreamSynchronize(s));
    r.eval_ms += ms_since(t0);
    double worst = 0.0;
    for (int i = 0; i < I; ++i) {
      double nrm;
      std::memcpy(&nrm, &h_norm[i], sizeof(double));
      if (!(nrm <= worst)) worst = nrm;
    }
    r.max_mismatch = worst;
    if (worst <= tol) {
      r.converged = 1;
      break;
    }
    if (it >= max_iter || worst != worst) break;
    for (int half = 0; half < 2; ++half) {
      if (half == 1) {                                   // F at the updated angles
        t0 = std::chrono::steady_clock::now();
        PF_TRY(launch_eval(c, x, nullptr, S->F, nullptr, s));
        PF_CUDA_TRY(cudaStreamSynchronize(s));
        r.eval_ms += ms_since(t0);
      }
      t0 = std::chrono::steady_clock::now();
      PF_CUDA_TRY(cudaMemsetAsync(S->rhs, 0, c.n_f * sizeof(double), s));
      k_fdlf_rhs<<<(unsigned)blocks, 256, 0, s>>>(c.v, S->F, x, S->rhs, half);
      PF_CUDA_TRY(cudaGetLastError());
      PF_CUDA_TRY(cudaStreamSynchronize(s));
      for (int i = 0; i < I; ++i) {
        const int g = c.inst_grid[i], k = S->fd_of_inst[i];
        const int n1 = S->fd_n1[k], n = half == 0 ? n1 : c.grid_nf[g] - n1;
        if (n == 0) continue;
        RfInst &R = half == 0 ? S->fd1[k] : S->fd2[k];
        double *b = S->rhs + c.f_off[i] + (half == 0 ? 0 : n1);
        PF_SOLVER_TRY(cusolverRfSolve(R.rf, R.dP, R.dQ, 1, R.dT, n, b, n), "cusolverRfSolve");
      }
      PF_CUDA_TRY(cudaDeviceSynchronize());            // cuSOLVER-Rf works on the legacy default stream
      r.solve_ms += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      k_fdlf_update<<<(unsigned)blocks, 256, 0, s>>>(c.v, x, S->rhs, half);
      PF_CUDA_TRY(cudaGetLastError());
      PF_CUDA_TRY(cudaStreamSynchronize(s));
      r.update_ms += ms_since(t0);
    }
    r.iterations = it + 1;
  }
  if (info) *info = r;
  return PF_OK;
}

}  // namespace pf
