// Adjoint: vector-Jacobian products v^T dF/d(x, P_inj, Q_inj, r, x, b_c, tau)
// for a batch of cotangents.  Trigonometric terms are recomputed (the forward
// kernels' phasor records, one sincos per bus), nothing from a forward call
// is kept.
//
// State part.  For bus o with pairs (o, k) (parallel branches merged) the
// gradient gathers the column of J^T at theta_o and V_o:
//   dL/dtheta_o = v_P(o) S_Y - v_Q(o) S_X
//               + sum_k [ v_P(k) dP_k/dtheta_o + v_Q(k) dQ_k/dtheta_o ]
//   dL/dV_o     = v_P(o) (2 V_o^2 A^ - S_X) / V_o - v_Q(o) (2 V_o^2 C^ + S_Y) / V_o
//               + sum_k [ v_P(k) dP_k/dV_o + v_Q(k) dQ_k/dV_o ]
// (S_X, S_Y as in the forward kernels, from the rectangular voltages; the
// mirror partials from the merged coefficients of the ends at k towards o),
// plus the +-1 terms of the extended rows.  One lane per bus on the forward
// kernel's rounds; the cotangents run in chunks whose sums stay in
// registers; per chunk, one pass over the bus's pairs forms W = conj(E_o) E_k
// once for the own terms and the mirror partials (12 FP64 operations per pair
// instead of 16).
//
// Parameter part.  One thread per (instance, branch): the partials of the
// four terminal powers with respect to g, b, b_c and tau, chained to r and x
// through g = r/D, b = -x/D, D = r^2 + x^2, dotted with the four cotangent
// entries of the branch's rows.
#include <algorithm>

#include "pf_internal.cuh"

namespace pf {

namespace {

// From this many cotangents on, they are read from a transposed copy.
constexpr int kVjpTransposeMin = 16;

struct VjpArgs {
  const double *x;
  const double *v;        // [n_cot][n_f]
  const double *vt;       // [n_f][n_cot] transposed copy, or nullptr
  int n_cot;
  int64_t n_f, n_x;
  const double2 *gb, *ac, *hat;       // per end (incidence order) / per bus
  const double2 *sgb, *sgbm, *sac;    // per slot: merged own and mirror coefficients, own A, C
  const double2 *rhat;                // per bus in round order
  const uint8_t *status;
  const uint8_t *gen_mode;  // extended, per instance-generator: != 0 held at a reactive limit
  double *gx;             // [n_cot][n_x]
};

// Cotangent c at row `row` (instance-offset) in either layout.
__device__ __forceinline__ double cot_at(const double *v, const double *vt, int n_cot, int64_t n_f, int c,
                                         int64_t row) {
  return vt ? __ldg(vt + row * n_cot + c) : __ldg(v + (int64_t)c * n_f + row);
}

__device__ __forceinline__ double cot_row(const VjpArgs &a, int c, int64_t f0, int32_t row) {
  return row >= 0 ? cot_at(a.v, a.vt, a.n_cot, a.n_f, c, f0 + row) : 0.0;
}

// X and Y of one branch end (own voltage Eo, other voltage Ek, rectangular),
// as in the forward kernels.
struct Terms {
  double X, Y;
};

__device__ __forceinline__ Terms rotated(double2 G, double2 Eo, double2 Ek) {
  const double uu = __fma_rn(G.x, Ek.x, __dmul_rn(-G.y, Ek.y));
  const double ww = __fma_rn(G.x, Ek.y, __dmul_rn(G.y, Ek.x));
  Terms r;
  r.X = __fma_rn(Eo.x, uu, __dmul_rn(Eo.y, ww));
  r.Y = __fma_rn(Eo.y, uu, __dmul_rn(-Eo.x, ww));
  return r;
}

// -x, by flipping the sign bit on the integer pipe (exact, no FP64 issue).
__device__ __forceinline__ double neg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// Diagonal partials of bus o from its sums S_X, S_Y, V_o, 1/V_o, A^ and C^.
struct Diag {
  double pt, qt, pv, qv;
};

__device__ __forceinline__ Diag diag_partials(double sx, double sy, double vo, double rvo, double ah, double ch) {
  const double v2 = __dmul_rn(vo, vo);
  Diag d;
  d.pt = sy;
  d.qt = neg(sx);
  d.pv = __dmul_rn(__fma_rn(v2, ah, __fma_rn(v2, ah, -sx)), rvo);
  d.qv = __dmul_rn(__fma_rn(v2, ch, __fma_rn(v2, ch, sy)), -rvo);
  return d;
}

__device__ __forceinline__ bool end_in(const View &v, int32_t e, int32_t outage, const uint8_t *status,
                                       int64_t st_base) {
  const int32_t l = v.inc_code[e] >> 1;
  return (l != outage) && (status == nullptr || status[st_base + l] != 0);
}

// Under an outage mask: own coefficients, own A, C and mirror coefficients of
// the branches in service of a group of `len` parallel ends e, e+1, ...,
// each summed in incidence order (zero when none is in service).
struct PairCoeff {
  double2 gb, ac, gbm;
  bool any_out;
};

__device__ __forceinline__ PairCoeff masked_pair(const View &v, const VjpArgs &a, int32_t e, int32_t len,
                                                 int32_t outage, int64_t st_base) {
  PairCoeff r{make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0), false};
  bool first = true;
  for (int32_t i = 0; i < len; ++i) {
    if (!end_in(v, e + i, outage, a.status, st_base)) {
      r.any_out = true;
      continue;
    }
    const double2 g = __ldg(a.gb + e + i), c = __ldg(a.ac + e + i), m = __ldg(a.gb + v.inc_mirror[e + i]);
    if (first) {
      r.gb = g; r.ac = c; r.gbm = m;
      first = false;
    } else {
      r.gb = make_double2(__dadd_rn(r.gb.x, g.x), __dadd_rn(r.gb.y, g.y));
      r.ac = make_double2(__dadd_rn(r.ac.x, c.x), __dadd_rn(r.ac.y, c.y));
      r.gbm = make_double2(__dadd_rn(r.gbm.x, m.x), __dadd_rn(r.gbm.y, m.y));
    }
  }
  return r;
}

// The partials of bus k's P and Q rows with respect to theta_o and V_o, for
// the (merged) branch end at k towards o with coefficients Gm:
//   dP_k/dt_o = -Y',  dQ_k/dt_o = X',  dP_k/dV_o = -X' / V_o,  dQ_k/dV_o = -Y' / V_o,
// with X', Y' the terms of that end (own voltage E_k, other voltage E_o).
struct Mirror {
  double pt, qt, pv, qv;
};

__device__ __forceinline__ Mirror mirror_partials(double2 Gm, double2 Eo, double rvo, double2 Ek) {
  const Terms t = rotated(Gm, Ek, Eo);
  Mirror m;
  m.pt = neg(t.Y);
  m.qt = t.X;
  m.pv = __dmul_rn(-t.X, rvo);
  m.qv = __dmul_rn(-t.Y, rvo);
  return m;
}


// Writes dL/dtheta_o, dL/dV_o (and, in the extended formulation, the
// gradients of the generator / slack unknowns) of cotangent c.
__device__ __forceinline__ void write_state_grad(const View &v, const VjpArgs &a, int inst, int g, int64_t lb,
                                                 int32_t nb, int32_t gi, int32_t rp, int32_t rq, int c, double gt,
                                                 double gvv) {
  const int64_t f0 = v.inst_f_off[inst];
  double *__restrict__ gx = a.gx + (int64_t)c * a.n_x + v.inst_x_off[inst];
  if (v.formulation == PF_EXTENDED) {
    if (lb == v.grid_slack[g]) {
      gt = __dadd_rn(gt, cot_row(a, c, f0, v.grid_row_gth[g]));   // d g_theta / d theta_s = 1
      gx[2 * nb + v.grid_ngen[g]] = -cot_row(a, c, f0, rp);        // d g_p / d P_s = -1
    }
    if (gi >= 0) {
      const double vgv = cot_row(a, c, f0, 2 * nb + gi);
      if (a.gen_mode && a.gen_mode[v.inst_gen_off[inst] + gi]) {
        gx[2 * nb + gi] = __dsub_rn(vgv, cot_row(a, c, f0, rq));   // d g_V / d Q_g = 1, d g_q / d Q_g = -1
      } else {
        gvv = __dadd_rn(gvv, vgv);                                // d g_V / d V = 1
        gx[2 * nb + gi] = -cot_row(a, c, f0, rq);                  // d g_q / d Q_g = -1
      }
    }
  }
  gx[lb] = gt;
  gx[nb + lb] = gvv;
}

// State part, one warp per round of 32 buses, one bus per lane (the forward
// kernel's rounds and slots).  For the lane's bus o:
//   dL/dtheta_o = v_P(o) dP_o/dt_o + v_Q(o) dQ_o/dt_o + sum over pairs (o,k) [v_P(k) dP_k/dt_o + v_Q(k) dQ_k/dt_o]
//   dL/dV_o     = the same with V_o,
// the diagonal partials from the bus sums (as in the forward kernel) and the
// mirror partials recomputed per chunk of CH cotangents, whose sums are kept
// in registers.  Sums in a fixed order: pairs in list order, then own rows.
// A chunk of 16 cotangents is held in 128 registers (16 one-warp CTAs per SM,
// a few bytes spilled): 15 % faster on the 70k grid with 64 cotangents than
// the 186 registers the kernel takes unbounded (12 CTAs per SM).
template <int CH, bool MASKED>
__global__ void __launch_bounds__(32, (CH == 16 ? 16 : 1)) k_vjp_lane(View v, VjpArgs a) {
  const int lane = threadIdx.x & 31;
  const int n_chunks = (a.n_cot + CH - 1) / CH;
  const int64_t n_work = v.n_lane_units * n_chunks;
  for (int64_t w = blockIdx.x; w < n_work; w += gridDim.x) {
    // unit of work: one round and one chunk of CH cotangents
    const int64_t u = w % v.n_lane_units;
    const int c0 = (int)(w / v.n_lane_units) * CH;
    const int4 ur = __ldg(v.unit_rec + u);
    const int inst = ur.x;
    const int64_t r = ur.y;
    const int g = __ldg(v.inst_grid + inst);
    const double2 *__restrict__ rec = v.phasor + 2 * __ldg(v.inst_rec_base + inst);
    const int32_t outage = MASKED ? v.inst_outage[inst] : -1;
    const int64_t st_base = MASKED ? v.inst_br_off[inst] - v.grid_br_off[g] : 0;
    const int64_t f0 = v.inst_f_off[inst];
    const int64_t rb = 32 * r + lane;
    if (lane >= (ur.w >> 8)) continue;           // no bus on this lane (no warp-wide operation follows)
    const int32_t o = __ldg(v.rbus + rb);
    const int4 bm = __ldg(v.rbus_meta + rb);
    const int32_t gi = __ldg(v.rbus_meta2 + rb).w;
    const int64_t gb0 = v.grid_bus_off[g];
    const int32_t nb = v.grid_nbus[g];
    const int32_t D = ur.w & 0xff;
    const int64_t q0 = (int64_t)ur.z + lane;
    const double2 Eo = rec[2 * o];
    const double2 vr = rec[2 * o + 1];             // (V_o, 1/V_o)

    // One pass over the pairs: W = conj(E_o) E_k gives both the own terms
    // (X - jY = y W, summed into S_X, S_Y for the diagonal partials) and the
    // mirror partials of bus k's rows at theta_o, V_o (X' - jY' = y_m conj(W)),
    // which meet the cotangents of k's rows at once.  The own rows'
    // contributions are added after the pairs.
    double sx = 0.0, sy = 0.0;
    bool any_out = false;                        // masked: an end of this bus is out of service
    double gt[CH], gvv[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) gt[i] = gvv[i] = 0.0;
    for (int32_t j = 0; j < D; ++j) {
      const int64_t q = q0 + 32 * j;
      const int4 meta = __ldg(v.slot_meta + q);
      if (meta.y < 0) continue;
      double2 G = __ldg(a.sgb + q), Gm = __ldg(a.sgbm + q);
      if (MASKED) {
        if (meta.y == 1) {
          if (!end_in(v, meta.w, outage, a.status, st_base)) {
            G = Gm = make_double2(0.0, 0.0);
            any_out = true;
          }
        } else {
          const PairCoeff pc = masked_pair(v, a, meta.w, meta.y, outage, st_base);
          G = pc.gb;
          Gm = pc.gbm;
          any_out |= pc.any_out;
        }
      }
      const int32_t k = meta.x;
      const double2 Ek = rec[2 * k];
      const double wr = __fma_rn(Eo.x, Ek.x, __dmul_rn(Eo.y, Ek.y));       // W = conj(E_o) E_k
      const double wi = __fma_rn(Eo.x, Ek.y, __dmul_rn(-Eo.y, Ek.x));
      sx = __dadd_rn(sx, __fma_rn(G.x, wr, __dmul_rn(-G.y, wi)));          // X
      sy = __dadd_rn(sy, __fma_rn(-G.x, wi, __dmul_rn(-G.y, wr)));         // Y = -(G wi + B wr)
      const double xm = __fma_rn(Gm.x, wr, __dmul_rn(Gm.y, wi));           // X'
      const double ym = __fma_rn(Gm.x, wi, __dmul_rn(-Gm.y, wr));          // Y'
      Mirror m;
      m.pt = neg(ym);
      m.qt = xm;
      m.pv = __dmul_rn(-xm, vr.y);
      m.qv = __dmul_rn(-ym, vr.y);
      const int4 bk = __ldg(v.bus_meta + k);
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        if (c0 + i < a.n_cot) {
          const double vp = cot_row(a, c0 + i, f0, bk.x), vq = cot_row(a, c0 + i, f0, bk.y);
          gt[i] = __fma_rn(m.qt, vq, __fma_rn(m.pt, vp, gt[i]));
          gvv[i] = __fma_rn(m.qv, vq, __fma_rn(m.pv, vp, gvv[i]));
        }
      }
    }
    // A^, C^: built, or re-summed over the ends in service in the built order
    double2 hat = __ldg(a.rhat + rb);
    if (MASKED && any_out) {
      double ma = 0.0, mc = 0.0;
      for (int32_t j = 0; j < D; ++j) {
        const int64_t q = q0 + 32 * j;
        const int4 meta = __ldg(v.slot_meta + q);
        if (meta.y < 0) continue;
        double2 AC;
        if (meta.y == 1)
          AC = end_in(v, meta.w, outage, a.status, st_base) ? __ldg(a.sac + q) : make_double2(0.0, 0.0);
        else
          AC = masked_pair(v, a, meta.w, meta.y, outage, st_base).ac;
        ma = __dadd_rn(ma, AC.x);
        mc = __dadd_rn(mc, AC.y);
      }
      const double2 sh = __ldg(v.bus_sh + o);
      hat = make_double2(__dadd_rn(ma, sh.x), __dadd_rn(mc, sh.y));
    }
    const Diag d = diag_partials(sx, sy, vr.x, vr.y, hat.x, hat.y);
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      if (c0 + i < a.n_cot) {
        const double vp = cot_row(a, c0 + i, f0, bm.x), vq = cot_row(a, c0 + i, f0, bm.y);
        const double t = __fma_rn(d.qt, vq, __fma_rn(d.pt, vp, gt[i]));
        const double w = __fma_rn(d.qv, vq, __fma_rn(d.pv, vp, gvv[i]));
        write_state_grad(v, a, inst, g, o - gb0, nb, gi, bm.x, bm.y, c0 + i, t, w);
      }
    }
  }
}

template <int CH, bool MASKED>
__global__ void __launch_bounds__(32) k_vjp_large(View v, VjpArgs a) {
  const int lane = threadIdx.x & 31;
  for (int64_t u = blockIdx.x; u < v.n_large_units; u += gridDim.x) {
    const int2 lr = __ldg(v.large_rec + u);
    const int inst = lr.x;
    const int32_t o = lr.y;
    const int g = __ldg(v.inst_grid + inst);
    const double2 *__restrict__ rec = v.phasor + 2 * __ldg(v.inst_rec_base + inst);
    const int32_t outage = MASKED ? v.inst_outage[inst] : -1;
    const int64_t st_base = MASKED ? v.inst_br_off[inst] - v.grid_br_off[g] : 0;
    const int64_t f0 = v.inst_f_off[inst];
    const int32_t e0 = __ldg(v.inc_ptr + o), e1 = __ldg(v.inc_ptr + o + 1);
    const int4 bm = __ldg(v.bus_meta + o);
    const int32_t gi = __ldg(v.bus_meta2 + o).w;
    const double2 Eo = rec[2 * o];
    const double2 vr = rec[2 * o + 1];             // (V_o, 1/V_o)
    double sx = 0.0, sy = 0.0, sma = 0.0, smc = 0.0;
    for (int32_t e = e0 + lane; e < e1; e += 32) {
      double2 G = __ldg(a.gb + e), AC = __ldg(a.ac + e);
      if (MASKED && !end_in(v, e, outage, a.status, st_base)) G = AC = make_double2(0.0, 0.0);
      const int32_t k = __ldg(v.inc_other + e);
      const Terms t = rotated(G, Eo, rec[2 * k]);
      sx = __dadd_rn(sx, t.X);
      sy = __dadd_rn(sy, t.Y);
      if (MASKED) {
        sma = __dadd_rn(sma, AC.x);
        smc = __dadd_rn(smc, AC.y);
      }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      sx = __dadd_rn(sx, __shfl_xor_sync(0xffffffffu, sx, m));
      sy = __dadd_rn(sy, __shfl_xor_sync(0xffffffffu, sy, m));
      if (MASKED) {
        sma = __dadd_rn(sma, __shfl_xor_sync(0xffffffffu, sma, m));
        smc = __dadd_rn(smc, __shfl_xor_sync(0xffffffffu, smc, m));
      }
    }
    double ah, ch;
    if (MASKED) {
      const double2 sh = __ldg(v.bus_sh + o);
      ah = __dadd_rn(sma, sh.x);
      ch = __dadd_rn(smc, sh.y);
    } else {
      const double2 h = __ldg(a.hat + o);
      ah = h.x;
      ch = h.y;
    }
    const Diag d = diag_partials(sx, sy, vr.x, vr.y, ah, ch);
    for (int c0 = 0; c0 < a.n_cot; c0 += CH) {
      double gt[CH], gvv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) gt[i] = gvv[i] = 0.0;
      for (int32_t e = e0 + lane; e < e1; e += 32) {
        double2 Gm = __ldg(a.gb + __ldg(v.inc_mirror + e));
        if (MASKED && !end_in(v, e, outage, a.status, st_base)) Gm = make_double2(0.0, 0.0);
        const int32_t k = __ldg(v.inc_other + e);
        const Mirror m = mirror_partials(Gm, Eo, vr.y, rec[2 * k]);
        const int4 bk = __ldg(v.bus_meta + k);
#pragma unroll
        for (int i = 0; i < CH; ++i) {
          if (c0 + i < a.n_cot) {
            const double vp = cot_row(a, c0 + i, f0, bk.x), vq = cot_row(a, c0 + i, f0, bk.y);
            gt[i] = __fma_rn(m.qt, vq, __fma_rn(m.pt, vp, gt[i]));
            gvv[i] = __fma_rn(m.qv, vq, __fma_rn(m.pv, vp, gvv[i]));
          }
        }
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
          gt[i] = __dadd_rn(gt[i], __shfl_xor_sync(0xffffffffu, gt[i], m));
          gvv[i] = __dadd_rn(gvv[i], __shfl_xor_sync(0xffffffffu, gvv[i], m));
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
          if (c0 + i < a.n_cot) {
            const double vp = cot_row(a, c0 + i, f0, bm.x), vq = cot_row(a, c0 + i, f0, bm.y);
            const double t = __fma_rn(d.qt, vq, __fma_rn(d.pt, vp, gt[i]));
            const double w = __fma_rn(d.qv, vq, __fma_rn(d.pv, vp, gvv[i]));
            write_state_grad(v, a, inst, g, o - v.grid_bus_off[g], v.grid_nbus[g], gi, bm.x, bm.y, c0 + i, t, w);
          }
        }
      }
    }
  }
}

struct ParamArgs {
  const double *v;            // [n_cot][n_f], or
  const double *vt;           // [n_f][n_cot] (transposed copy) when not nullptr
  int n_cot;
  int64_t n_f, n_bi;          // n_bi: branches summed over instances
  const double *r, *xr, *b, *tap;   // overrides or nullptr
  const uint8_t *status;
  double *gr, *gxr, *gb, *gtap;
};

// One thread per (instance, branch).  With the branch's constants
//   g + j b_s = 1 / (r + j x),  alpha = (x^2 - r^2)/D^2,  beta = 2 r x / D^2  (D = r^2 + x^2),
// so that dg/dr = db_s/dx = alpha and db_s/dr = -dg/dx = beta, and the state's
//   (V_f V_t / tau) cos / sin of delta = theta_f - theta_t - phi (from E_f conj(E_t)),
// the derivatives of the four terminal powers (P_f, Q_f, P_t, Q_t) with
// respect to g, b_s, b_c and tau are formed once and dotted with the
// cotangent entries of the four rows for every cotangent.  OVR: the
// constants come from per-call parameters instead of the build.
constexpr int kParamChunk = 32;   // cotangents per thread of k_vjp_params

template <bool OVR>
__global__ void __launch_bounds__(128) k_vjp_params(View v, ParamArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int n_chunks = (a.n_cot + kParamChunk - 1) / kParamChunk;
  const int64_t n_work = a.n_bi * n_chunks;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += stride) {
    const int64_t q = w % a.n_bi;
    const int c0 = (int)(w / a.n_bi) * kParamChunk;
    const int c1 = min(a.n_cot, c0 + kParamChunk);
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_br_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t l = v.grid_br_off[g] + (q - v.inst_br_off[inst]);   // global branch
    const double2 *__restrict__ rec = v.phasor + 2 * __ldg(v.inst_rec_base + inst);
    const int32_t f = v.br_from[l], t = v.br_to[l];
    bool in = v.br_status[l] != 0 && l != v.inst_outage[inst];
    if (a.status) in = in && a.status[q] != 0;
    double d_r[4], d_x[4], d_t[4], db1 = 0.0, db3 = 0.0;   // rows: P_f, Q_f, P_t, Q_t
    if (in) {
      double gs, bs, al, be, it, bc;
      const double2 ph = __ldg(v.br_k_ph + l);             // (cos phi, sin phi)
      if (OVR) {
        const double r = a.r ? a.r[l] : v.br_r[l];
        const double x = a.xr ? a.xr[l] : v.br_x[l];
        const double dd = r * r + x * x;
        const double inv = 1.0 / dd;
        gs = r * inv;
        bs = -x * inv;
        al = (x * x - r * r) * (inv * inv);
        be = 2.0 * r * x * (inv * inv);
        it = 1.0 / (a.tap ? a.tap[l] : v.br_tap[l]);
        bc = a.b ? a.b[l] : v.br_b[l];
      } else {
        const double2 k1 = __ldg(v.br_k_gb + l), k2 = __ldg(v.br_k_ab + l), k3 = __ldg(v.br_k_tc + l);
        gs = k1.x; bs = k1.y; al = k2.x; be = k2.y; it = k3.x; bc = k3.y;
      }
      const double2 Ef = rec[2 * f], Et = rec[2 * t];
      const double vf = rec[2 * f + 1].x, vt = rec[2 * t + 1].x;
      // V_f V_t (cos, sin)(theta_f - theta_t), then rotated by -phi and divided by tau
      const double cD = Ef.x * Et.x + Ef.y * Et.y, sD = Ef.y * Et.x - Ef.x * Et.y;
      const double pgc = (cD * ph.x + sD * ph.y) * it, pgs = (sD * ph.x - cD * ph.y) * it;
      const double vfi = vf * it;
      const double vf2t = vfi * vfi, vt2 = vt * vt;
      // d/dg and d/db_s of each row
      const double Fg[4] = {vf2t - pgc, -pgs, vt2 - pgc, pgs};
      const double Fb[4] = {-pgs, pgc - vf2t, pgs, pgc - vt2};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        d_r[i] = Fg[i] * al + Fb[i] * be;
        d_x[i] = Fb[i] * al - Fg[i] * be;
      }
      db1 = -0.5 * vf2t;
      db3 = -0.5 * vt2;
      // tau-derivatives: the V_f V_t terms scale with 1/tau, the V_f^2 terms with 1/tau^2
      const double gc = gs * pgc, bsd = bs * pgs, gsd = gs * pgs, bcd = bs * pgc;
      const double tf = 2.0 * it * vf2t;
      d_t[0] = it * (gc + bsd) - tf * (gs + v.br_gfr[l]);
      d_t[1] = tf * (bs + 0.5 * bc) + it * (gsd - bcd);
      d_t[2] = it * (gc - bsd);
      d_t[3] = -it * (gsd + bcd);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) d_r[i] = d_x[i] = d_t[i] = 0.0;
    }
    const int4 mf = __ldg(v.bus_meta + f), mt = __ldg(v.bus_meta + t);
    const int32_t rows[4] = {mf.x, mf.y, mt.x, mt.y};
    const int64_t f0 = v.inst_f_off[inst];
#pragma unroll 4
    for (int c = c0; c < c1; ++c) {
      double w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) w[i] = rows[i] >= 0 ? cot_at(a.v, a.vt, a.n_cot, a.n_f, c, f0 + rows[i]) : 0.0;
      const int64_t o = (int64_t)c * a.n_bi + q;
      if (a.gr) a.gr[o] = w[0] * d_r[0] + w[1] * d_r[1] + w[2] * d_r[2] + w[3] * d_r[3];
      if (a.gxr) a.gxr[o] = w[0] * d_x[0] + w[1] * d_x[1] + w[2] * d_x[2] + w[3] * d_x[3];
      if (a.gb) a.gb[o] = w[1] * db1 + w[3] * db3;
      if (a.gtap) a.gtap[o] = w[0] * d_t[0] + w[1] * d_t[1] + w[2] * d_t[2] + w[3] * d_t[3];
    }
  }
}

// v [n_cot][n_f] -> vt [n_f][n_cot], 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) k_transpose(const double *__restrict__ v, int n_cot, int64_t n_f,
                                                   double *__restrict__ vt) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;    // rows of F
  const int c0 = blockIdx.y * 32;                  // cotangents
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int c = c0 + j;
    const int64_t r = r0 + threadIdx.x;
    if (c < n_cot && r < n_f) tile[j][threadIdx.x] = v[(int64_t)c * n_f + r];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + j;
    const int c = c0 + threadIdx.x;
    if (c < n_cot && r < n_f) vt[r * n_cot + c] = tile[threadIdx.x][j];
  }
}

// one thread per (cotangent, instance bus): dF_P/dP_inj = -1, dF_Q/dQ_inj = -1
__global__ void k_vjp_inj(View v, const double *__restrict__ vv, int n_cot, int64_t n_f, double *gp, double *gq) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c = blockIdx.y; c < n_cot; c += gridDim.y)
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < v.n_bus_inst; q += stride) {
    const int64_t t = (int64_t)c * v.n_bus_inst + q;
    const int inst = v.n_inst == 1 ? 0 : find_segment(v.inst_bus_off, v.n_inst, q);
    const int g = v.inst_grid[inst];
    const int64_t b = v.grid_bus_off[g] + (q - v.inst_bus_off[inst]);
    const int4 bm = __ldg(v.bus_meta + b);
    const double *__restrict__ vc = vv + c * n_f + v.inst_f_off[inst];
    if (gp) gp[t] = bm.x >= 0 ? -vc[bm.x] : 0.0;
    if (gq) gq[t] = bm.y >= 0 ? -vc[bm.y] : 0.0;
  }
}

template <int CH, bool MASKED>
int launch_state(const Ctx &c, const VjpArgs &a, cudaStream_t s) {
  const int cps = c.tuning.ctas_per_sm;
  if (c.v.n_lane_units > 0) {
    const int64_t work = c.v.n_lane_units * ((a.n_cot + CH - 1) / CH);
    k_vjp_lane<CH, MASKED><<<(unsigned)capped_grid(work, cps, c.num_sms), 32, 0, s>>>(c.v, a);
    PF_CUDA_TRY(cudaGetLastError());
  }
  if (c.v.n_large_units > 0) {
    k_vjp_large<CH, MASKED><<<(unsigned)capped_grid(c.v.n_large_units, cps, c.num_sms), 32, 0, s>>>(c.v, a);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

template <int CH>
int launch_state_ch(const Ctx &c, const VjpArgs &a, bool masked, cudaStream_t s) {
  return masked ? launch_state<CH, true>(c, a, s) : launch_state<CH, false>(c, a, s);
}

}  // namespace

int launch_vjp(Ctx &c, const double *x, const pf_overrides *ov, const double *v, int n_cot, const pf_grads *g,
               cudaStream_t s) {
  if (!x || !v || !g) return fail(PF_ERR_INVALID, "x, v and g must not be NULL");
  if (n_cot <= 0) return fail(PF_ERR_INVALID, "n_cot must be positive");
  const int tb = 256;
  const int64_t cap_blocks = (int64_t)c.num_sms * 16;
  // E = V (cos, sin), V and 1/V of every bus: the forward kernels' per-bus records
  PF_TRY(launch_phasor(c.v, c.num_sms, x, s, false));
  VjpArgs a{};
  a.x = x; a.v = v; a.n_cot = n_cot; a.n_f = c.n_f; a.n_x = c.n_x;
  a.gb = c.v.inc_gb; a.ac = c.v.inc_ac; a.hat = c.v.bus_hat;
  a.sgb = c.v.slot_gb; a.sgbm = c.v.slot_gbm; a.sac = c.v.slot_ac; a.rhat = c.v.rbus_hat;
  a.status = ov ? ov->status : nullptr;
  a.gen_mode = ov ? ov->gen_mode : nullptr;
  const double *r = nullptr, *xr = nullptr, *b = nullptr, *tap = nullptr;
  if (ov && (ov->br_r || ov->br_x || ov->br_b || ov->br_tap)) {
    r = ov->br_r; xr = ov->br_x; b = ov->br_b; tap = ov->br_tap;
    PF_TRY(compute_coefficients(c, r, xr, b, tap, c.ov_gb, c.ov_ac, c.ov_hat, s));
    PF_TRY(permute_overrides(c, s));
    a.gb = c.ov_gb; a.ac = c.ov_ac; a.hat = c.ov_hat;
    a.sgb = c.ov_slot_gb; a.sgbm = c.ov_slot_gbm; a.sac = c.ov_slot_ac; a.rhat = c.ov_rbus_hat;
  }
  // many cotangents: read them from a transposed copy, so that one row's
  // cotangents are contiguous for the per-bus and per-branch loops
  if (n_cot >= kVjpTransposeMin && (g->x || g->br_r || g->br_x || g->br_b || g->br_tap)) {
    const int64_t need = c.n_f * (int64_t)n_cot;
    if (c.vt_cap < need) {
      if (c.vt_scratch) cudaFree(c.vt_scratch);
      c.vt_scratch = nullptr;
      c.vt_cap = 0;
      cudaError_t e = cudaMalloc(&c.vt_scratch, need * sizeof(double));
      if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA,
                    std::string("pf_vjp: allocating the transposed cotangents (make the first call with this "
                                "many cotangents outside stream capture): ") + cudaGetErrorString(e));
      c.vt_cap = need;
    }
    const dim3 grid((unsigned)((c.n_f + 31) / 32), (unsigned)((n_cot + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(v, n_cot, c.n_f, c.vt_scratch);
    PF_CUDA_TRY(cudaGetLastError());
    a.vt = c.vt_scratch;
  }
  if (g->x) {
    a.gx = g->x;
    const bool masked = c.any_outage || a.status != nullptr;
    if (n_cot >= 32) PF_TRY(launch_state_ch<16>(c, a, masked, s));
    else if (n_cot >= 16) PF_TRY(launch_state_ch<8>(c, a, masked, s));
    else if (n_cot >= 4) PF_TRY(launch_state_ch<4>(c, a, masked, s));
    else PF_TRY(launch_state_ch<1>(c, a, masked, s));
  }
  if (g->br_r || g->br_x || g->br_b || g->br_tap) {
    ParamArgs p{};
    p.v = v; p.vt = a.vt; p.n_cot = n_cot; p.n_f = c.n_f; p.n_bi = c.n_branch_inst;
    p.r = r; p.xr = xr; p.b = b; p.tap = tap; p.status = a.status;
    p.gr = g->br_r; p.gxr = g->br_x; p.gb = g->br_b; p.gtap = g->br_tap;
    const int64_t work = c.n_branch_inst * ((n_cot + kParamChunk - 1) / kParamChunk);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + 127) / 128, cap_blocks * 2));
    if (r || xr || b || tap) k_vjp_params<true><<<(unsigned)blocks, 128, 0, s>>>(c.v, p);
    else k_vjp_params<false><<<(unsigned)blocks, 128, 0, s>>>(c.v, p);
    PF_CUDA_TRY(cudaGetLastError());
  }
  if (g->p_inj || g->q_inj) {
    const int64_t bx = std::max<int64_t>(1, std::min<int64_t>((c.v.n_bus_inst + tb - 1) / tb, cap_blocks));
    const int by = (int)std::min<int64_t>(n_cot, std::max<int64_t>(1, cap_blocks / bx));
    k_vjp_inj<<<dim3((unsigned)bx, (unsigned)by), tb, 0, s>>>(c.v, v, n_cot, c.n_f, g->p_inj, g->q_inj);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

}  // namespace pf
