// Adjoint: vector-Jacobian products v^T dF/d(x, P_inj, Q_inj, r, x, b_c, tau)
// for a batch of cotangents.  Trigonometric terms are recomputed (one sincos
// per bus in k_phasor, shared with the forward kernel), nothing from a
// forward call is kept.
//
// State part.  For bus o with branch ends e (other bus k) and mirror ends e'
// (the same branch seen from k), using the rotated form of pf_eval.cu:
//   dL/dtheta_o = v_P(o) V_o sum_e b_e - v_Q(o) V_o sum_e a_e
//               + sum_e [ -v_P(k) Y_e' + v_Q(k) X_e' ]
//   dL/dV_o     = v_P(o) (2 V_o A^ - sum a) - v_Q(o) (2 V_o C^ + sum b)
//               + sum_e [ -v_P(k) V_k xh_e' - v_Q(k) V_k yh_e' ]
// plus the +-1 terms of the extended rows.  Sums run in incidence-list order
// (deterministic).  The terms of one end are computed once per tile and
// reused for every cotangent.
//
// Parameter part.  One thread per (instance, branch): the partials of the
// four terminal powers with respect to g, b, b_c and tau, chained to r and x
// through g = r/D, b = -x/D, D = r^2 + x^2, dotted with the four cotangent
// entries of the branch's rows.
#include <algorithm>

#include "pf_internal.cuh"

namespace pf {

namespace {

struct VjpArgs {
  const double *x;
  const double *v;        // [n_cot][n_f]
  int n_cot;
  int64_t n_f;
  const double2 *gb;
  const double2 *ac;
  const double2 *hat;
  const uint8_t *status;
  double *gx;             // [n_cot][n_x]
  int64_t n_x;
  int cap;
};

__global__ void k_phasor_adj(View v, const double *__restrict__ x) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int64_t lb = q - v.inst_bus_off[inst];
    double s, c;
    sincos(x[v.inst_x_off[inst] + lb], &s, &c);
    v.phasor[2 * q] = make_double2(c, s);
    v.phasor[2 * q + 1] = make_double2(x[v.inst_x_off[inst] + v.grid_nbus[v.inst_grid[inst]] + lb], 0.0);
  }
}

__device__ __forceinline__ bool end_in(const View &v, int32_t e, int32_t outage, const uint8_t *status,
                                       int64_t st_base) {
  const int32_t l = v.inc_code[e] >> 1;
  return (l != outage) && (status == nullptr || status[st_base + l] != 0);
}

// Rotated terms of end e (own bus o, other bus k): xh, yh.
__device__ __forceinline__ void rotated(double2 G, double2 po, double2 pk, double &xh, double &yh) {
  const double uu = G.x * pk.x - G.y * pk.y;
  const double ww = G.x * pk.y + G.y * pk.x;
  xh = po.x * uu + po.y * ww;
  yh = po.y * uu - po.x * ww;
}

__global__ void __launch_bounds__(1024) k_vjp_state(View v, VjpArgs a) {
  extern __shared__ double sm[];
  const int cap = a.cap;
  double *s_a = sm, *s_b = sm + cap, *s_g = sm + 2 * cap, *s_h = sm + 3 * cap;
  double *s_ma = sm + 4 * cap, *s_mc = sm + 5 * cap;
  __shared__ int s_cut;
  const bool masked = a.status != nullptr || v.inst_outage != nullptr;

  for (int64_t u = blockIdx.x; u < v.n_units; u += gridDim.x) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_unit_off, v.n_inst, u);
    const int g = v.inst_grid[inst];
    const int64_t t = v.grid_tile_off[g] + (u - v.inst_unit_off[inst]);
    const int32_t b0 = v.tile_bus0[t], b1 = v.tile_bus1[t];
    const int32_t e0 = v.inc_ptr[b0], e1 = v.inc_ptr[b1];
    const int64_t gb0 = v.grid_bus_off[g];
    const int32_t nb = v.grid_nbus[g];
    const double *__restrict__ xi = a.x + v.inst_x_off[inst];
    const double *__restrict__ Vi = xi + nb - gb0;
    const double2 *__restrict__ phb = v.phasor + 2 * (v.inst_bus_off[inst] - gb0);
    const int32_t outage = masked ? v.inst_outage[inst] : -1;
    const int64_t st_base = v.inst_br_off[inst] - v.grid_br_off[g];
    const int64_t f0 = v.inst_f_off[inst];
    const int32_t ob = b0 + (int32_t)threadIdx.x;
    const bool owner = ob < b1;
    const bool single = (e1 - e0) <= cap;

    if (single) {
      // own and mirror terms of this thread's end, kept for every cotangent
      const int j = threadIdx.x;
      const int n = e1 - e0;
      double mx = 0.0, my = 0.0, vk = 0.0;
      int32_t rpk = -1, rqk = -1;
      if (j < n) {
        const int32_t e = e0 + j;
        const int32_t o = v.inc_own[e], k = v.inc_other[e], em = v.inc_mirror[e];
        const bool in = !masked || end_in(v, e, outage, a.status, st_base);
        const double2 po = phb[2 * o], pk = phb[2 * k];
        double2 G = a.gb[e], Gm = a.gb[em];
        if (!in) G = Gm = make_double2(0.0, 0.0);
        double xh, yh;
        rotated(G, po, pk, xh, yh);
        vk = Vi[k];
        s_a[j] = vk * xh;
        s_b[j] = vk * yh;
        rotated(Gm, pk, po, mx, my);
        rpk = v.row_p[k];
        rqk = v.row_q[k];
        if (masked) {
          const double2 ac = a.ac[e];
          s_ma[j] = in ? ac.x : 0.0;
          s_mc[j] = in ? ac.y : 0.0;
        }
      }
      __syncthreads();
      double sa = 0.0, sb = 0.0, ma = 0.0, mc = 0.0;
      int32_t op0 = 0, op1 = 0;
      if (owner) {
        op0 = v.inc_ptr[ob];
        op1 = v.inc_ptr[ob + 1];
        for (int32_t e = op0; e < op1; ++e) {
          sa += s_a[e - e0];
          sb += s_b[e - e0];
          if (masked) {
            ma += s_ma[e - e0];
            mc += s_mc[e - e0];
          }
        }
      }
      for (int c = 0; c < a.n_cot; ++c) {
        const double *__restrict__ vc = a.v + (int64_t)c * a.n_f + f0;
        if (j < n) {
          const int32_t o = v.inc_own[e0 + j];
          const double vo = Vi[o];
          const double vpk = rpk >= 0 ? vc[rpk] : 0.0;
          const double vqk = rqk >= 0 ? vc[rqk] : 0.0;
          // X' = V_k V_o mx, Y' = V_k V_o my
          const double vv = vk * vo;
          s_g[j] = -vpk * (vv * my) + vqk * (vv * mx);
          s_h[j] = -vpk * (vk * mx) - vqk * (vk * my);
        }
        __syncthreads();
        if (owner) {
          double gt = 0.0, gv = 0.0;
          for (int32_t e = op0; e < op1; ++e) {
            gt += s_g[e - e0];
            gv += s_h[e - e0];
          }
          const int32_t o = ob;
          const int64_t lb = o - gb0;
          const double vo = Vi[o];
          const double ah = masked ? ma + v.bus_sh[o].x : a.hat[o].x;
          const double ch = masked ? mc + v.bus_sh[o].y : a.hat[o].y;
          const int32_t rp = v.row_p[o], rq = v.row_q[o];
          const double vp = rp >= 0 ? vc[rp] : 0.0;
          const double vq = rq >= 0 ? vc[rq] : 0.0;
          double dth = vp * (vo * sb) - vq * (vo * sa) + gt;
          double dv = vp * (2.0 * vo * ah - sa) - vq * (2.0 * vo * ch + sb) + gv;
          double *__restrict__ gx = a.gx + (int64_t)c * a.n_x + v.inst_x_off[inst];
          if (v.formulation == PF_EXTENDED) {
            const int32_t gi = v.gen[o];
            if (lb == v.grid_slack[g]) {
              dth += vc[v.grid_row_gth[g]];
              gx[2 * nb + v.grid_ngen[g]] = -vp;        // P_s
            }
            if (gi >= 0) {
              dv += vc[2 * nb + gi];
              gx[2 * nb + gi] = -vq;                    // Q_g
            }
          }
          gx[lb] = dth;
          gx[nb + lb] = dv;
        }
        __syncthreads();
      }
    } else {
      // A bus with more ends than `cap`: chunk over its ends for every
      // cotangent, recomputing the rotated terms.
      for (int c = 0; c < a.n_cot; ++c) {
        const double *__restrict__ vc = a.v + (int64_t)c * a.n_f + f0;
        double sa = 0.0, sb = 0.0, ma = 0.0, mc = 0.0, gt = 0.0, gv = 0.0;
        for (int32_t cs = e0; cs < e1;) {
          int32_t ce = min(cs + cap, e1);
          if (ce < e1) {
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
          for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const int32_t e = cs + j;
            const int32_t o = v.inc_own[e], k = v.inc_other[e], em = v.inc_mirror[e];
            const bool in = !masked || end_in(v, e, outage, a.status, st_base);
            const double2 po = phb[2 * o], pk = phb[2 * k];
            double2 G = a.gb[e], Gm = a.gb[em];
            if (!in) G = Gm = make_double2(0.0, 0.0);
            double xh, yh, mx, my;
            rotated(G, po, pk, xh, yh);
            rotated(Gm, pk, po, mx, my);
            const double vk = Vi[k], vo = Vi[o];
            s_a[j] = vk * xh;
            s_b[j] = vk * yh;
            const int32_t rpk = v.row_p[k], rqk = v.row_q[k];
            const double vpk = rpk >= 0 ? vc[rpk] : 0.0;
            const double vqk = rqk >= 0 ? vc[rqk] : 0.0;
            const double vv = vk * vo;
            s_g[j] = -vpk * (vv * my) + vqk * (vv * mx);
            s_h[j] = -vpk * (vk * mx) - vqk * (vk * my);
            if (masked) {
              const double2 ac = a.ac[e];
              s_ma[j] = in ? ac.x : 0.0;
              s_mc[j] = in ? ac.y : 0.0;
            }
          }
          __syncthreads();
          if (owner) {
            const int32_t lo = max(v.inc_ptr[ob], cs), hi = min(v.inc_ptr[ob + 1], ce);
            for (int32_t e = lo; e < hi; ++e) {
              sa += s_a[e - cs];
              sb += s_b[e - cs];
              gt += s_g[e - cs];
              gv += s_h[e - cs];
              if (masked) {
                ma += s_ma[e - cs];
                mc += s_mc[e - cs];
              }
            }
          }
          __syncthreads();
          cs = ce;
        }
        if (owner) {
          const int32_t o = ob;
          const int64_t lb = o - gb0;
          const double vo = Vi[o];
          const double ah = masked ? ma + v.bus_sh[o].x : a.hat[o].x;
          const double ch = masked ? mc + v.bus_sh[o].y : a.hat[o].y;
          const int32_t rp = v.row_p[o], rq = v.row_q[o];
          const double vp = rp >= 0 ? vc[rp] : 0.0;
          const double vq = rq >= 0 ? vc[rq] : 0.0;
          double dth = vp * (vo * sb) - vq * (vo * sa) + gt;
          double dv = vp * (2.0 * vo * ah - sa) - vq * (2.0 * vo * ch + sb) + gv;
          double *__restrict__ gx = a.gx + (int64_t)c * a.n_x + v.inst_x_off[inst];
          if (v.formulation == PF_EXTENDED) {
            const int32_t gi = v.gen[o];
            if (lb == v.grid_slack[g]) {
              dth += vc[v.grid_row_gth[g]];
              gx[2 * nb + v.grid_ngen[g]] = -vp;
            }
            if (gi >= 0) {
              dv += vc[2 * nb + gi];
              gx[2 * nb + gi] = -vq;
            }
          }
          gx[lb] = dth;
          gx[nb + lb] = dv;
        }
      }
    }
  }
}

struct ParamArgs {
  const double *x;
  const double *v;
  int n_cot;
  int64_t n_f, n_bi;          // n_bi: branches summed over instances
  const double *r, *xr, *b, *tap;   // overrides or nullptr
  const uint8_t *status;
  double *gr, *gxr, *gb, *gtap;
  double *gp, *gq;            // injection grads
  int64_t n_busi;
};

// one thread per (instance, branch)
__global__ void k_vjp_params(View v, ParamArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.n_bi; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_br_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t l = v.grid_br_off[g] + (q - v.inst_br_off[inst]);   // global branch
    const int64_t gb0 = v.grid_bus_off[g];
    const int32_t nb = v.grid_nbus[g];
    const double *__restrict__ xi = a.x + v.inst_x_off[inst];
    const double2 *__restrict__ phb = v.phasor + 2 * (v.inst_bus_off[inst] - gb0);
    const int32_t f = v.br_from[l], t = v.br_to[l];
    bool in = v.br_status[l] != 0 && l != v.inst_outage[inst];
    if (a.status) in = in && a.status[q] != 0;
    double d_r[4], d_x[4], d_b[4], d_t[4];   // order: P_f, Q_f, P_t, Q_t
    if (in) {
      const double r = a.r ? a.r[l] : v.br_r[l];
      const double x = a.xr ? a.xr[l] : v.br_x[l];
      const double bc = a.b ? a.b[l] : v.br_b[l];
      const double tau = a.tap ? a.tap[l] : v.br_tap[l];
      const double dd = r * r + x * x;
      const double g_ = r / dd, b_ = -x / dd;
      const double id2 = 1.0 / (dd * dd);
      const double dg_dr = (x * x - r * r) * id2, dg_dx = -2.0 * r * x * id2;
      const double db_dr = 2.0 * r * x * id2, db_dx = (x * x - r * r) * id2;
      const double2 pf = phb[2 * f], pt = phb[2 * t];
      // delta = theta_f - theta_t - phi
      const double cD = pf.x * pt.x + pf.y * pt.y, sD = pf.y * pt.x - pf.x * pt.y;
      double sp, cp;
      sincos(v.br_shift[l], &sp, &cp);
      const double cd = cD * cp + sD * sp, sd = sD * cp - cD * sp;
      const double vf = xi[nb + (f - gb0)], vt = xi[nb + (t - gb0)];
      const double it = 1.0 / tau;
      const double vv = vf * vt * it;
      const double vf2t = vf * vf * it * it, vt2 = vt * vt;
      const double Pf_g = vf2t - vv * cd, Pf_b = -vv * sd;
      const double Qf_g = -vv * sd, Qf_b = -vf2t + vv * cd;
      const double Pt_g = vt2 - vv * cd, Pt_b = vv * sd;
      const double Qt_g = vv * sd, Qt_b = -vt2 + vv * cd;
      d_r[0] = Pf_g * dg_dr + Pf_b * db_dr; d_x[0] = Pf_g * dg_dx + Pf_b * db_dx;
      d_r[1] = Qf_g * dg_dr + Qf_b * db_dr; d_x[1] = Qf_g * dg_dx + Qf_b * db_dx;
      d_r[2] = Pt_g * dg_dr + Pt_b * db_dr; d_x[2] = Pt_g * dg_dx + Pt_b * db_dx;
      d_r[3] = Qt_g * dg_dr + Qt_b * db_dr; d_x[3] = Qt_g * dg_dx + Qt_b * db_dx;
      d_b[0] = 0.0; d_b[1] = -0.5 * vf2t; d_b[2] = 0.0; d_b[3] = -0.5 * vt2;
      const double vv2 = vv * it;
      d_t[0] = -2.0 * vf2t * it * (g_ + v.br_gfr[l]) + vv2 * (g_ * cd + b_ * sd);
      d_t[1] = 2.0 * vf2t * it * (b_ + 0.5 * bc) + vv2 * (g_ * sd - b_ * cd);
      d_t[2] = vv2 * (g_ * cd - b_ * sd);
      d_t[3] = -vv2 * (g_ * sd + b_ * cd);
    } else {
      for (int i = 0; i < 4; ++i) d_r[i] = d_x[i] = d_b[i] = d_t[i] = 0.0;
    }
    const int32_t rows[4] = {v.row_p[f], v.row_q[f], v.row_p[t], v.row_q[t]};
    const int64_t f0 = v.inst_f_off[inst];
    for (int c = 0; c < a.n_cot; ++c) {
      const double *__restrict__ vc = a.v + (int64_t)c * a.n_f + f0;
      double w[4];
      for (int i = 0; i < 4; ++i) w[i] = rows[i] >= 0 ? vc[rows[i]] : 0.0;
      const int64_t o = (int64_t)c * a.n_bi + q;
      if (a.gr) a.gr[o] = w[0] * d_r[0] + w[1] * d_r[1] + w[2] * d_r[2] + w[3] * d_r[3];
      if (a.gxr) a.gxr[o] = w[0] * d_x[0] + w[1] * d_x[1] + w[2] * d_x[2] + w[3] * d_x[3];
      if (a.gb) a.gb[o] = w[0] * d_b[0] + w[1] * d_b[1] + w[2] * d_b[2] + w[3] * d_b[3];
      if (a.gtap) a.gtap[o] = w[0] * d_t[0] + w[1] * d_t[1] + w[2] * d_t[2] + w[3] * d_t[3];
    }
  }
}

// one thread per (instance, bus): dF_P/dP_inj = -1, dF_Q/dQ_inj = -1
__global__ void k_vjp_inj(View v, const double *__restrict__ vv, int n_cot, int64_t n_f, double *gp, double *gq) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t b = v.grid_bus_off[g] + (q - v.inst_bus_off[inst]);
    const int32_t rp = v.row_p[b], rq = v.row_q[b];
    const int64_t f0 = v.inst_f_off[inst];
    for (int c = 0; c < n_cot; ++c) {
      const double *__restrict__ vc = vv + (int64_t)c * n_f + f0;
      const int64_t o = (int64_t)c * v.n_bus_inst + q;
      if (gp) gp[o] = rp >= 0 ? -vc[rp] : 0.0;
      if (gq) gq[o] = rq >= 0 ? -vc[rq] : 0.0;
    }
  }
}

}  // namespace

int launch_vjp(Ctx &c, const double *x, const pf_overrides *ov, const double *v, int n_cot, const pf_grads *g,
               cudaStream_t s) {
  if (!x || !v || !g) return fail(PF_ERR_INVALID, "x, v and g must not be NULL");
  if (n_cot <= 0) return fail(PF_ERR_INVALID, "n_cot must be positive");
  const int tb = 256;
  const int64_t cap_blocks = (int64_t)c.num_sms * 16;
  k_phasor_adj<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((c.v.n_bus_inst + tb - 1) / tb, cap_blocks)),
                 tb, 0, s>>>(c.v, x);
  PF_CUDA_TRY(cudaGetLastError());
  const double2 *gb = c.v.inc_gb, *ac = c.v.inc_ac, *hat = c.v.bus_hat;
  const uint8_t *status = ov ? ov->status : nullptr;
  const double *r = nullptr, *xr = nullptr, *b = nullptr, *tap = nullptr;
  if (ov && (ov->br_r || ov->br_x || ov->br_b || ov->br_tap)) {
    r = ov->br_r; xr = ov->br_x; b = ov->br_b; tap = ov->br_tap;
    PF_TRY(compute_coefficients(c, r, xr, b, tap, c.ov_gb, c.ov_ac, c.ov_hat, s));
    gb = c.ov_gb;
    ac = c.ov_ac;
    hat = c.ov_hat;
  }
  if (g->x) {
    VjpArgs a{};
    a.x = x; a.v = v; a.n_cot = n_cot; a.n_f = c.n_f; a.gb = gb; a.ac = ac; a.hat = hat;
    a.status = status; a.gx = g->x; a.n_x = c.n_x; a.cap = c.tuning.tile_inc;
    View vv = c.v;
    if (!c.any_outage) vv.inst_outage = nullptr;   // unmasked fast path unless outages exist
    const size_t smem = (size_t)a.cap * sizeof(double) * 6;
    if (smem > 46 * 1024)
      PF_CUDA_TRY(cudaFuncSetAttribute(k_vjp_state, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t grid = c.v.n_units;
    if (c.tuning.ctas_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)c.tuning.ctas_per_sm * c.num_sms);
    k_vjp_state<<<(unsigned)std::max<int64_t>(grid, 1), a.cap, smem, s>>>(vv, a);
    PF_CUDA_TRY(cudaGetLastError());
  }
  if (g->br_r || g->br_x || g->br_b || g->br_tap) {
    ParamArgs p{};
    p.x = x; p.v = v; p.n_cot = n_cot; p.n_f = c.n_f; p.n_bi = c.n_branch_inst;
    p.r = r; p.xr = xr; p.b = b; p.tap = tap; p.status = status;
    p.gr = g->br_r; p.gxr = g->br_x; p.gb = g->br_b; p.gtap = g->br_tap;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((c.n_branch_inst + tb - 1) / tb, cap_blocks));
    k_vjp_params<<<(unsigned)blocks, tb, 0, s>>>(c.v, p);
    PF_CUDA_TRY(cudaGetLastError());
  }
  if (g->p_inj || g->q_inj) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((c.v.n_bus_inst + tb - 1) / tb, cap_blocks));
    k_vjp_inj<<<(unsigned)blocks, tb, 0, s>>>(c.v, v, n_cot, c.n_f, g->p_inj, g->q_inj);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

}  // namespace pf
