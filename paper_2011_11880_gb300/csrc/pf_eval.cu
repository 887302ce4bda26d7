// Evaluation kernels: tasks (1) and (2) of Newton power flow (Sec. I) for
// every instance of a context, in one persistent pass over (instance, tile)
// units.
//
// Arithmetic form.  For a branch end at bus o whose other end is bus k, with
// per-end coefficients (G, B, A, C) built once from the branch model (see
// k_coeff in pf_build.cu), the terminal powers of Eq. (4) extended with Q,
// tap and shift are
//     P_o =  A V_o^2 - X,   Q_o = -C V_o^2 - Y,
//     X = V_o V_k xh,       Y = V_o V_k yh,
//     xh = cos(t_o) u + sin(t_o) w,   yh = sin(t_o) u - cos(t_o) w,
//     u  = G cos(t_k) - B sin(t_k),   w  = G sin(t_k) + B cos(t_k),
// which is the polar form with the angle difference expanded, so that the
// only trigonometry is one sincos per bus (kernel k_phasor).  The partials
// follow from the same expansion:
//     dP_o/dt_k = -Y,  dQ_o/dt_k = X,  dP_o/dV_k = -V_o xh,  dQ_o/dV_k = -V_o yh,
// and, summed over the ends of bus o with a = V_k xh, b = V_k yh,
//     F_P = V_o (V_o A^ - sum a) - P_inj,    F_Q = -V_o (V_o C^ + sum b) - Q_inj,
//     dF_P/dt_o = V_o sum b,   dF_Q/dt_o = -V_o sum a,
//     dF_P/dV_o = 2 V_o A^ - sum a,   dF_Q/dV_o = -2 V_o C^ - sum b,
// where A^ = sum A + shunt g and C^ = sum C + shunt b.  No division, 16
// FP64 operations per branch end for F and J.
//
// Determinism: every sum runs in the order of the incidence list (one
// thread per bus, one thread per parallel-branch group), so results are
// bit-identical run to run and for every tile size.
#include <algorithm>

#include "pf_internal.cuh"

namespace pf {

namespace {

__global__ void k_phasor(View v, const double *__restrict__ x) {
  // Let the fused kernel start launching; it waits for this grid's results.
  cudaTriggerProgrammaticLaunchCompletion();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int64_t lb = q - v.inst_bus_off[inst];
    double s, c;
    sincos(__ldg(x + v.inst_x_off[inst] + lb), &s, &c);
    v.phasor[q] = make_double2(c, s);
  }
}

struct EvalArgs {
  const double *x;
  double *F;
  double *vals;
  const double2 *gb;
  const double2 *ac;
  const double *ahat;
  const double *chat;
  const double *p_inj;     // per-instance-bus override or nullptr
  const double *q_inj;
  const uint8_t *status;   // per-instance-branch mask or nullptr
  int cap;                 // branch ends staged per chunk (= blockDim.x)
};

template <bool WF, bool WJ, bool MASKED>
__global__ void __launch_bounds__(1024) k_fused(View v, EvalArgs a) {
  extern __shared__ double sm[];
  const int cap = a.cap;
  double *s_a = sm;             // V_k xh
  double *s_b = sm + cap;       // V_k yh
  double *s_pt = sm + 2 * cap;  // dP/dt_k
  double *s_qt = sm + 3 * cap;  // dQ/dt_k
  double *s_pv = sm + 4 * cap;  // dP/dV_k
  double *s_qv = sm + 5 * cap;  // dQ/dV_k
  double *s_ma = sm + (WJ ? 6 : 2) * cap;  // masked: A of the end, 0 when out
  double *s_mc = s_ma + cap;
  __shared__ int s_cut;

  // Wait for k_phasor (programmatic dependent launch).
  cudaGridDependencySynchronize();

  for (int64_t u = blockIdx.x; u < v.n_units; u += gridDim.x) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_unit_off, v.n_inst, u);
    const int g = v.inst_grid[inst];
    const int64_t t = v.grid_tile_off[g] + (u - v.inst_unit_off[inst]);
    const int32_t b0 = v.tile_bus0[t], b1 = v.tile_bus1[t];
    const int32_t e0 = v.inc_ptr[b0], e1 = v.inc_ptr[b1];
    const int64_t gb0 = v.grid_bus_off[g];
    const int32_t nb = v.grid_nbus[g];
    const double *__restrict__ xi = a.x + v.inst_x_off[inst];
    const double *__restrict__ Vi = xi + nb - gb0;                 // V by global bus id
    const double2 *__restrict__ ph = v.phasor + v.inst_bus_off[inst] - gb0;
    double *__restrict__ vi = WJ ? a.vals + v.inst_v_off[inst] : nullptr;
    const int32_t outage = MASKED ? v.inst_outage[inst] : -1;
    const int64_t st_base = MASKED ? v.inst_br_off[inst] - v.grid_br_off[g] : 0;

    const int32_t ob = b0 + (int32_t)threadIdx.x;
    const bool owner = ob < b1;
    double acc_a = 0.0, acc_b = 0.0, acc_ma = 0.0, acc_mc = 0.0;
    int32_t op0 = 0, op1 = 0;
    if (owner) {
      op0 = v.inc_ptr[ob];
      op1 = v.inc_ptr[ob + 1];
    }

    for (int32_t cs = e0; cs < e1;) {
      int32_t ce = min(cs + cap, e1);
      if (ce < e1) {
        // A bus with more ends than `cap`: cut the chunk at the last group
        // head in (cs, ce] so no group of parallel branches is split.
        if (threadIdx.x == 0) s_cut = cs;
        __syncthreads();
        for (int j = threadIdx.x; j < cap; j += blockDim.x) {
          const int32_t p = cs + 1 + j;
          if (p <= ce && v.inc_grp[p] > 0) atomicMax(&s_cut, p);
        }
        __syncthreads();
        const int32_t cut = s_cut;
        __syncthreads();
        if (cut == cs) {
          if (threadIdx.x == 0) atomicOr(v.dev_error, kErrChunk);
          break;
        }
        ce = cut;
      }
      const int n = ce - cs;

      // ---- phase A: one thread per branch end ----
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int32_t e = cs + j;
        const int32_t o = v.inc_own[e], k = v.inc_other[e];
        double2 G = a.gb[e];
        bool in = true;
        if (MASKED) {
          const int32_t l = v.inc_code[e] >> 1;
          in = (l != outage) && (a.status == nullptr || a.status[st_base + l] != 0);
          if (!in) G = make_double2(0.0, 0.0);
        }
        const double2 pk = ph[k], po = ph[o];
        const double vk = Vi[k];
        const double uu = G.x * pk.x - G.y * pk.y;
        const double ww = G.x * pk.y + G.y * pk.x;
        const double xh = po.x * uu + po.y * ww;
        const double yh = po.y * uu - po.x * ww;
        const double ea = vk * xh, eb = vk * yh;
        s_a[j] = ea;
        s_b[j] = eb;
        if (WJ) {
          const double vo = Vi[o];
          s_pt[j] = -(vo * eb);
          s_qt[j] = vo * ea;
          s_pv[j] = -(vo * xh);
          s_qv[j] = -(vo * yh);
        }
        if (MASKED) {
          const double2 ac = a.ac[e];
          s_ma[j] = in ? ac.x : 0.0;
          s_mc[j] = in ? ac.y : 0.0;
        }
      }
      __syncthreads();

      // ---- off-diagonal entries: one thread per group of parallel ends ----
      if (WJ) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          const int32_t e = cs + j;
          const int32_t len = v.inc_grp[e];
          if (len == 0) continue;
          double pt = s_pt[j], qt = s_qt[j], pv = s_pv[j], qv = s_qv[j];
          for (int q = 1; q < len; ++q) {
            pt += s_pt[j + q];
            qt += s_qt[j + q];
            pv += s_pv[j + q];
            qv += s_qv[j + q];
          }
          const int32_t o = v.inc_own[e];
          const int2 rt = v.inc_rt[e];
          const int32_t bp = v.base_p[o], bq = v.base_q[o];
          if (bp >= 0) {
            if (rt.x >= 0) vi[bp + rt.x] = pt;
            if (rt.y >= 0) vi[bp + rt.y] = pv;
          }
          if (bq >= 0) {
            if (rt.x >= 0) vi[bq + rt.x] = qt;
            if (rt.y >= 0) vi[bq + rt.y] = qv;
          }
        }
      }

      // ---- bus sums, in list order ----
      if (owner) {
        const int32_t lo = max(op0, cs), hi = min(op1, ce);
        for (int32_t e = lo; e < hi; ++e) {
          acc_a += s_a[e - cs];
          acc_b += s_b[e - cs];
          if (MASKED) {
            acc_ma += s_ma[e - cs];
            acc_mc += s_mc[e - cs];
          }
        }
      }
      __syncthreads();
      cs = ce;
    }

    // ---- per-bus results: F rows and the diagonal of J ----
    if (owner) {
      const int32_t o = ob;
      const int64_t lb = o - gb0;
      const double vo = Vi[o];
      double ah, ch;
      if (MASKED) {
        ah = acc_ma + v.g_sh[o];
        ch = acc_mc + v.b_sh[o];
      } else {
        ah = a.ahat[o];
        ch = a.chat[o];
      }
      const int32_t rp = v.row_p[o], rq = v.row_q[o];
      const bool ext = v.formulation == PF_EXTENDED;
      const int32_t gi = ext ? v.gen[o] : -1;
      const bool is_slack = ext && (lb == v.grid_slack[g]);
      if (WF) {
        double *__restrict__ Fi = a.F + v.inst_f_off[inst];
        const double pin = a.p_inj ? a.p_inj[v.inst_bus_off[inst] + lb] : v.p_inj[o];
        const double qin = a.q_inj ? a.q_inj[v.inst_bus_off[inst] + lb] : v.q_inj[o];
        double fp = vo * (vo * ah - acc_a) - pin;
        double fq = -(vo * (vo * ch + acc_b)) - qin;
        if (is_slack) {
          fp -= xi[2 * nb + v.grid_ngen[g]];
          Fi[v.grid_row_gth[g]] = xi[lb] - v.grid_theta_set[g];
        }
        if (gi >= 0) {
          fq -= xi[2 * nb + gi];
          Fi[2 * nb + gi] = vo - v.gen_vset[v.grid_gen_off[g] + gi];
        }
        if (rp >= 0) Fi[rp] = fp;
        if (rq >= 0) Fi[rq] = fq;
      }
      if (WJ) {
        const int2 d = v.diag[o];
        const int32_t bp = v.base_p[o], bq = v.base_q[o];
        if (bp >= 0) {
          if (d.x >= 0) vi[bp + d.x] = vo * acc_b;
          if (d.y >= 0) vi[bp + d.y] = 2.0 * vo * ah - acc_a;
        }
        if (bq >= 0) {
          if (d.x >= 0) vi[bq + d.x] = -(vo * acc_a);
          if (d.y >= 0) vi[bq + d.y] = -2.0 * vo * ch - acc_b;
        }
        if (is_slack) {
          vi[bp + v.len_tv[o]] = -1.0;          // d g_p / d P_s
          vi[v.grid_pos_gth[g]] = 1.0;         // d g_theta / d theta_s
        }
        if (gi >= 0) {
          vi[bq + v.len_tv[o]] = -1.0;          // d g_q / d Q_g
          vi[v.gen_pos[v.grid_gen_off[g] + gi]] = 1.0;  // d g_V / d V
        }
      }
    }
  }
}

template <bool WF, bool WJ, bool MASKED>
int launch_fused(Ctx &c, const EvalArgs &a, cudaStream_t s) {
  const int cap = a.cap;
  const size_t smem = (size_t)cap * sizeof(double) * ((WJ ? 6 : 2) + (MASKED ? 2 : 0));
  auto kern = k_fused<WF, WJ, MASKED>;
  // the kernel also holds a few bytes of static shared memory: opt in above 46 KB
  if (smem > 46 * 1024)
    PF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t grid = c.v.n_units;
  if (c.tuning.ctas_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)c.tuning.ctas_per_sm * c.num_sms);
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)cap);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PF_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, c.v, a));
  return PF_OK;
}

}  // namespace

int launch_eval(Ctx &c, const double *x, const pf_overrides *ov, double *F, double *vals, cudaStream_t s) {
  return launch_eval_stages(c, 3, x, ov, F, vals, s);
}

int launch_eval_stages(Ctx &c, int stages, const double *x, const pf_overrides *ov, double *F, double *vals,
                       cudaStream_t s) {
  if (!x) return fail(PF_ERR_INVALID, "x is NULL");
  if (stages < 1 || stages > 3) return fail(PF_ERR_INVALID, "stage must be PF_STAGE_PHASOR or PF_STAGE_FUSED");
  if (!F && !vals) return PF_OK;
  EvalArgs a{};
  a.x = x;
  a.F = F;
  a.vals = vals;
  a.gb = c.v.inc_gb;
  a.ac = c.v.inc_ac;
  a.ahat = c.v.a_hat;
  a.chat = c.v.c_hat;
  a.cap = c.tuning.tile_inc;
  if (ov) {
    a.p_inj = ov->p_inj;
    a.q_inj = ov->q_inj;
    a.status = ov->status;
    if (ov->br_r || ov->br_x || ov->br_b || ov->br_tap) {
      if (stages & 2)
        PF_TRY(compute_coefficients(c, ov->br_r, ov->br_x, ov->br_b, ov->br_tap, c.ov_gb, c.ov_ac, c.ov_ahat,
                                    c.ov_chat, s));
      a.gb = c.ov_gb;
      a.ac = c.ov_ac;
      a.ahat = c.ov_ahat;
      a.chat = c.ov_chat;
    }
  }
  const bool masked = c.any_outage || a.status != nullptr;
  if (stages & 1) {
    const int tb = 256;
    int64_t blocks = (c.v.n_bus_inst + tb - 1) / tb;
    blocks = std::min<int64_t>(blocks, (int64_t)c.num_sms * 16);
    k_phasor<<<(unsigned)std::max<int64_t>(blocks, 1), tb, 0, s>>>(c.v, x);
    PF_CUDA_TRY(cudaGetLastError());
  }
  if (!(stages & 2)) return PF_OK;
  const bool wf = F != nullptr, wj = vals != nullptr;
  if (wf && wj) return masked ? launch_fused<true, true, true>(c, a, s) : launch_fused<true, true, false>(c, a, s);
  if (wf) return masked ? launch_fused<true, false, true>(c, a, s) : launch_fused<true, false, false>(c, a, s);
  return masked ? launch_fused<false, true, true>(c, a, s) : launch_fused<false, true, false>(c, a, s);
}

}  // namespace pf

// ---------------------------------------------------------------------------
// Evaluation with caller-provided phasor scratch (used by the allocation-free
// entry point, whose scratch is a static device array).
// ---------------------------------------------------------------------------

namespace pf {

namespace {

template <bool WF, bool WJ, bool MASKED>
int launch_fused_view(const View &v, int num_sms, const pf_tuning &t, const EvalArgs &a, cudaStream_t s) {
  const size_t smem = (size_t)a.cap * sizeof(double) * ((WJ ? 6 : 2) + (MASKED ? 2 : 0));
  auto kern = k_fused<WF, WJ, MASKED>;
  if (smem > 46 * 1024)
    PF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t grid = v.n_units;
  if (t.ctas_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)t.ctas_per_sm * num_sms);
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)a.cap);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PF_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, v, a));
  return PF_OK;
}

}  // namespace

int launch_eval_scratch(Ctx &c, const double *x, double *F, double *vals, double2 *scratch, cudaStream_t s) {
  if (!x) return fail(PF_ERR_INVALID, "x is NULL");
  if (!scratch) return fail(PF_ERR_INVALID, "scratch is NULL");
  if (!F && !vals) return PF_OK;
  View v = c.v;
  v.phasor = scratch;
  EvalArgs a{};
  a.x = x;
  a.F = F;
  a.vals = vals;
  a.gb = c.v.inc_gb;
  a.ac = c.v.inc_ac;
  a.ahat = c.v.a_hat;
  a.chat = c.v.c_hat;
  a.cap = c.tuning.tile_inc;
  const int tb = 256;
  int64_t blocks = (v.n_bus_inst + tb - 1) / tb;
  blocks = std::min<int64_t>(blocks, (int64_t)c.num_sms * 16);
  k_phasor<<<(unsigned)std::max<int64_t>(blocks, 1), tb, 0, s>>>(v, x);
  PF_CUDA_TRY(cudaGetLastError());
  const bool masked = c.any_outage;
  const bool wf = F != nullptr, wj = vals != nullptr;
  if (wf && wj)
    return masked ? launch_fused_view<true, true, true>(v, c.num_sms, c.tuning, a, s)
                  : launch_fused_view<true, true, false>(v, c.num_sms, c.tuning, a, s);
  if (wf)
    return masked ? launch_fused_view<true, false, true>(v, c.num_sms, c.tuning, a, s)
                  : launch_fused_view<true, false, false>(v, c.num_sms, c.tuning, a, s);
  return masked ? launch_fused_view<false, true, true>(v, c.num_sms, c.tuning, a, s)
                : launch_fused_view<false, true, false>(v, c.num_sms, c.tuning, a, s);
}

}  // namespace pf
