// pf_build: validates the systems on the host, then builds every index map on
// the device with integer-only, deterministic kernels:
//   * the per-bus incidence list (branch ends sorted by (own bus, other bus,
//     branch)), with parallel-branch groups and mirror positions;
//   * the formulation row / column maps (Sec. II-A, Eqs. 1-3 and the classic
//     reduced form) and the CSR pattern of J (Sec. III: the pattern the paper
//     assembles from triplets on every call is built once here);
//   * the per-nonzero contribution list;
//   * per-end branch coefficients and per-bus sums of the constant terms.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pf_internal.cuh"
#include "pf_sort_scan.cuh"

namespace pf {

namespace {

constexpr int TB = 256;

inline unsigned nblk(int64_t n, int tb = TB) { return (unsigned)((n + tb - 1) / tb); }

struct TempList {
  std::vector<void *> p;
  ~TempList() {
    for (void *q : p) cudaFree(q);
  }
  template <class T>
  int alloc(T **out, size_t n) {
    if (n == 0) n = 1;
    if (alloc_fault()) return fail(PF_ERR_OOM, "device allocation failed (PF_FAIL_ALLOC, build scratch)");
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess)
      return fail(PF_ERR_OOM, "cudaMalloc (build scratch): " + std::string(cudaGetErrorString(e)));
    p.push_back(q);
    *out = static_cast<T *>(q);
    return PF_OK;
  }
};

// --------------------------------------------------------------------------
// host validation
// --------------------------------------------------------------------------

bool finite(double v) { return std::isfinite(v); }

int validate(const pf_system &g, int gi, int formulation, int *n_pv_distinct) {
  auto bad = [&](const std::string &m) {
    return fail(PF_ERR_INVALID, "grid " + std::to_string(gi) + ": " + m);
  };
  if (g.n_bus < 2) return bad("n_bus must be >= 2");
  if (g.n_branch < 0 || g.n_load < 0 || g.n_pv < 0 || g.n_shunt < 0) return bad("negative count");
  const int64_t n = g.n_bus;
  if (g.n_branch > 0 && (!g.br_from || !g.br_to || !g.br_r || !g.br_x))
    return bad("br_from, br_to, br_r and br_x are required");
  for (int64_t k = 0; k < g.n_branch; ++k) {
    const int f = g.br_from[k], t = g.br_to[k];
    if (f < 0 || f >= n || t < 0 || t >= n) return bad("branch " + std::to_string(k) + ": bus index out of range");
    if (f == t) return bad("branch " + std::to_string(k) + ": from == to");
    const double r = g.br_r[k], x = g.br_x[k];
    if (!finite(r) || !finite(x) || !(r * r + x * x > 0.0))
      return bad("branch " + std::to_string(k) + ": r, x must be finite with r^2 + x^2 > 0");
    if (g.br_b && !finite(g.br_b[k])) return bad("branch " + std::to_string(k) + ": b not finite");
    if (g.br_tap && !(finite(g.br_tap[k]) && g.br_tap[k] > 0.0))
      return bad("branch " + std::to_string(k) + ": tap must be finite and > 0");
    if (g.br_shift && !finite(g.br_shift[k])) return bad("branch " + std::to_string(k) + ": shift not finite");
    if (g.br_g_fr && !finite(g.br_g_fr[k])) return bad("branch " + std::to_string(k) + ": g_fr not finite");
    if (g.br_g_to && !finite(g.br_g_to[k])) return bad("branch " + std::to_string(k) + ": g_to not finite");
  }
  if (g.slack_bus < 0 || g.slack_bus >= n) return bad("slack bus out of range");
  if (!finite(g.slack_vset) || !finite(g.slack_theta)) return bad("slack set-points not finite");
  if (g.n_load > 0 && (!g.load_bus || !g.load_p || !g.load_q)) return bad("load arrays missing");
  for (int64_t k = 0; k < g.n_load; ++k) {
    if (g.load_bus[k] < 0 || g.load_bus[k] >= n) return bad("load " + std::to_string(k) + ": bus out of range");
    if (!finite(g.load_p[k]) || !finite(g.load_q[k])) return bad("load " + std::to_string(k) + ": not finite");
  }
  if (g.n_pv > 0 && (!g.pv_bus || !g.pv_p || !g.pv_vset)) return bad("PV arrays missing");
  std::vector<char> seen(n, 0);
  int distinct = 0;
  for (int64_t k = 0; k < g.n_pv; ++k) {
    const int b = g.pv_bus[k];
    if (b < 0 || b >= n) return bad("PV " + std::to_string(k) + ": bus out of range");
    if (b == g.slack_bus) return bad("PV " + std::to_string(k) + ": unit on the slack bus");
    if (!finite(g.pv_p[k]) || !finite(g.pv_vset[k])) return bad("PV " + std::to_string(k) + ": not finite");
    if (seen[b]) {
      if (formulation == PF_EXTENDED)
        return bad("PV " + std::to_string(k) + ": two PV units on one bus (extended formulation)");
    } else {
      ++distinct;
    }
    seen[b] = 1;
  }
  if (g.n_shunt > 0 && (!g.sh_bus || !g.sh_g || !g.sh_b)) return bad("shunt arrays missing");
  for (int64_t k = 0; k < g.n_shunt; ++k) {
    if (g.sh_bus[k] < 0 || g.sh_bus[k] >= n) return bad("shunt " + std::to_string(k) + ": bus out of range");
    if (!finite(g.sh_g[k]) || !finite(g.sh_b[k])) return bad("shunt " + std::to_string(k) + ": not finite");
  }
  *n_pv_distinct = distinct;
  return PF_OK;
}

// --------------------------------------------------------------------------
// device kernels
// --------------------------------------------------------------------------

__global__ void k_bus_type(int8_t *type, const int32_t *pv_bus, int64_t n_pv, const int64_t *slack_glob,
                           int n_grids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pv) type[pv_bus[i]] = 1;
  if (i < n_grids) type[slack_glob[i]] = 2;  // a PV unit never sits on the slack bus
}

__global__ void k_flags(const int8_t *type, int64_t n, uint8_t *ns, uint8_t *pq) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  ns[b] = type[b] != 2;
  pq[b] = type[b] == 0;
}

__global__ void k_row_maps(View v, const int8_t *type, const int64_t *ex_ns, const int64_t *ex_pq,
                           int32_t *row_p, int32_t *row_q, int32_t *gen) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.n_bus) return;
  const int g = v.bus_grid[b];
  const int64_t b0 = v.grid_bus_off[g];
  const int nb = v.grid_nbus[g];
  gen[b] = -1;
  if (v.formulation == PF_REDUCED) {
    row_p[b] = type[b] != 2 ? (int32_t)(ex_ns[b] - ex_ns[b0]) : -1;
    row_q[b] = type[b] == 0 ? (int32_t)(nb - 1 + ex_pq[b] - ex_pq[b0]) : -1;
  } else {
    row_p[b] = (int32_t)(b - b0);
    row_q[b] = (int32_t)(nb + b - b0);
  }
}

// extended: generator index of each generator bus; gen_bus of each generator
__global__ void k_gen_map(View v, const int32_t *pv_bus, const int32_t *pv_grid, const int64_t *grid_pv_off,
                          int64_t n_pv, int32_t *gen, int32_t *gen_bus) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pv) {
    const int g = pv_grid[i];
    const int32_t gi = (int32_t)(i - grid_pv_off[g]);
    gen[pv_bus[i]] = gi;
    gen_bus[v.grid_gen_off[g] + gi] = pv_bus[i];
  }
  if (i < v.n_grids) {
    const int g = (int)i;
    const int32_t gi = v.grid_ngen[g] - 1;
    const int32_t s = (int32_t)(v.grid_bus_off[g] + v.grid_slack[g]);
    gen[s] = gi;
    gen_bus[v.grid_gen_off[g] + gi] = s;
  }
}

__global__ void k_make_keys(const int32_t *from, const int32_t *to, int64_t m, uint64_t *keys, uint32_t *vals) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * m) return;
  const int64_t l = e >> 1;
  const uint32_t own = (uint32_t)((e & 1) ? to[l] : from[l]);
  const uint32_t oth = (uint32_t)((e & 1) ? from[l] : to[l]);
  keys[e] = ((uint64_t)own << 32) | oth;
  vals[e] = (uint32_t)e;
}

__global__ void k_unpack(const uint64_t *keys, const uint32_t *vals, int64_t n, int32_t *own, int32_t *oth,
                         int32_t *code, int32_t *pos_of, int32_t *deg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  own[i] = (int32_t)(k >> 32);
  oth[i] = (int32_t)(k & 0xffffffffu);
  code[i] = (int32_t)vals[i];
  pos_of[vals[i]] = (int32_t)i;
  atomicAdd(deg + (int32_t)(k >> 32), 1);
}

__global__ void k_i64_to_i32(const int64_t *in, int32_t *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

__global__ void k_mirror_groups(View v, const int32_t *pos_of, int32_t *mirror, int32_t *grp, int32_t *stats) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n_inc) return;
  mirror[i] = pos_of[v.inc_code[i] ^ 1];
  const int32_t o = v.inc_own[i];
  const int32_t lo = v.inc_ptr[o], hi = v.inc_ptr[o + 1];
  const bool head = (i == lo) || (v.inc_other[i - 1] != v.inc_other[i]);
  int32_t len = 0;
  if (head) {
    len = 1;
    while (i + len < hi && v.inc_other[i + len] == v.inc_other[i]) ++len;
    atomicMax(stats + 0, len);
  }
  grp[i] = len;
  if (i == lo) atomicMax(stats + 1, hi - lo);
}

__device__ __forceinline__ bool has_col(const View &v, int32_t j, bool theta) {
  return theta ? (v.row_p[j] >= 0) : (v.row_q[j] >= 0);
}

// Visits, in ascending bus order, the buses of {o} U {other ends of o's
// branches} whose theta (or V) column exists: f(bus, head incidence or -1, group length).
template <class F>
__device__ __forceinline__ void walk_block(const View &v, int32_t o, bool theta, F &&f) {
  const int32_t p0 = v.inc_ptr[o], p1 = v.inc_ptr[o + 1];
  bool o_done = false;
  for (int32_t i = p0; i < p1;) {
    const int32_t len = v.inc_grp[i];
    const int32_t k = v.inc_other[i];
    if (!o_done && o < k) {
      if (has_col(v, o, theta)) f(o, -1, 0);
      o_done = true;
    }
    if (has_col(v, k, theta)) f(k, i, len);
    i += (len > 0 ? len : 1);
  }
  if (!o_done && has_col(v, o, theta)) f(o, -1, 0);
}

// Row structure of every bus: in-row offsets of each neighbour's columns,
// diagonal offsets, row lengths.
__global__ void k_row_struct(View v, const int64_t *grid_f_off, int2 *inc_rt, int2 *diag, int32_t *len_tv,
                             int32_t *rowlen) {
  const int64_t ob = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ob >= v.n_bus) return;
  const int32_t o = (int32_t)ob;
  int32_t nth = 0, nv = 0;
  int2 d = make_int2(-1, -1);
  walk_block(v, o, true, [&](int32_t j, int32_t i, int32_t len) {
    if (i < 0) d.x = nth;
    else for (int32_t q = 0; q < len; ++q) inc_rt[i + q].x = nth;
    ++nth;
  });
  // ends whose other bus has no theta column
  for (int32_t i = v.inc_ptr[o]; i < v.inc_ptr[o + 1]; ++i)
    if (!has_col(v, v.inc_other[i], true)) inc_rt[i].x = -1;
  walk_block(v, o, false, [&](int32_t j, int32_t i, int32_t len) {
    if (i < 0) d.y = nth + nv;
    else for (int32_t q = 0; q < len; ++q) inc_rt[i + q].y = nth + nv;
    ++nv;
  });
  for (int32_t i = v.inc_ptr[o]; i < v.inc_ptr[o + 1]; ++i)
    if (!has_col(v, v.inc_other[i], false)) inc_rt[i].y = -1;
  diag[o] = d;
  len_tv[o] = nth + nv;
  const int g = v.bus_grid[o];
  const bool ext = v.formulation == PF_EXTENDED;
  const bool is_slack = (o == v.grid_bus_off[g] + v.grid_slack[g]);
  if (v.row_p[o] >= 0) rowlen[grid_f_off[g] + v.row_p[o]] = nth + nv + ((ext && is_slack) ? 1 : 0);
  if (v.row_q[o] >= 0) rowlen[grid_f_off[g] + v.row_q[o]] = nth + nv + ((ext && v.gen[o] >= 0) ? 1 : 0);
}

// extended: rows g_V (per generator: entries at V_b and at Q_g, so that the
// row serves voltage control and a held reactive limit alike) and g_theta
// (per grid, one entry)
__global__ void k_gen_rowlen(View v, const int64_t *grid_f_off, int32_t *rowlen, int64_t n_gen_tot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_gen_tot) {
    const int32_t b = v.gen_bus[i];
    const int g = v.bus_grid[b];
    const int64_t gi = i - v.grid_gen_off[g];
    rowlen[grid_f_off[g] + 2 * (int64_t)v.grid_nbus[g] + gi] = 2;
  }
  if (i < v.n_grids) {
    const int g = (int)i;
    rowlen[grid_f_off[g] + 2 * (int64_t)v.grid_nbus[g] + v.grid_ngen[g]] = 1;
  }
}

// rowptr of grid g, entry r in [0, n_f(g)]: S[f_off + r] - S[f_off]
__global__ void k_rowptr(const int64_t *S, const int64_t *grid_f_off, const int64_t *grid_row_off, int n_grids,
                         int64_t total, int32_t *rowptr, int32_t *nnz_out, int32_t *err) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int g = find_segment(grid_row_off, n_grids, q);
  const int64_t r = q - grid_row_off[g];
  const int64_t val = S[grid_f_off[g] + r] - S[grid_f_off[g]];
  if (val > 0x7fffffffLL) atomicOr(err, kErrMap);
  rowptr[q] = (int32_t)val;
  if (q + 1 == grid_row_off[g + 1]) nnz_out[g] = (int32_t)val;
}

__global__ void k_colind(View v, const int32_t *rowptr, const int64_t *grid_row_off, const int64_t *grid_nnz_off,
                         int32_t *base_p, int32_t *base_q, int32_t *colind) {
  const int64_t ob = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ob >= v.n_bus) return;
  const int32_t o = (int32_t)ob;
  const int g = v.bus_grid[o];
  const int32_t *rp = rowptr + grid_row_off[g];
  int32_t *ci = colind + grid_nnz_off[g];
  const int64_t b0 = v.grid_bus_off[g];
  const int32_t nb = v.grid_nbus[g];
  const bool ext = v.formulation == PF_EXTENDED;
  const bool is_slack = (o == b0 + v.grid_slack[g]);
  for (int which = 0; which < 2; ++which) {
    const int32_t row = which == 0 ? v.row_p[o] : v.row_q[o];
    if (row < 0) {
      (which == 0 ? base_p : base_q)[o] = -1;
      continue;
    }
    const int32_t base = rp[row];
    (which == 0 ? base_p : base_q)[o] = base;
    int32_t pos = base;
    walk_block(v, o, true, [&](int32_t j, int32_t, int32_t) { ci[pos++] = v.row_p[j]; });
    walk_block(v, o, false, [&](int32_t j, int32_t, int32_t) { ci[pos++] = v.row_q[j]; });
    if (ext && which == 0 && is_slack) ci[pos++] = 2 * nb + v.grid_ngen[g];       // P_s column
    if (ext && which == 1 && v.gen[o] >= 0) ci[pos++] = 2 * nb + v.gen[o];         // Q_g column
  }
}

// extended: the g_V and g_theta entries
__global__ void k_gen_cols(View v, const int32_t *rowptr, const int64_t *grid_row_off, const int64_t *grid_nnz_off,
                           int32_t *colind, int32_t *gen_pos, int32_t *grid_pos_gth, int32_t *grid_row_gth,
                           int64_t n_gen_tot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_gen_tot) {
    const int32_t b = v.gen_bus[i];
    const int g = v.bus_grid[b];
    const int64_t gi = i - v.grid_gen_off[g];
    const int32_t row = 2 * v.grid_nbus[g] + (int32_t)gi;
    const int32_t pos = rowptr[grid_row_off[g] + row];
    colind[grid_nnz_off[g] + pos] = v.row_q[b];                    // V_b column (< 2 N)
    colind[grid_nnz_off[g] + pos + 1] = 2 * v.grid_nbus[g] + (int32_t)gi;   // Q_g column
    gen_pos[i] = pos;                                              // the Q_g entry is at pos + 1
  }
  if (i < v.n_grids) {
    const int g = (int)i;
    const int32_t row = 2 * v.grid_nbus[g] + v.grid_ngen[g];
    const int32_t pos = rowptr[grid_row_off[g] + row];
    colind[grid_nnz_off[g] + pos] = v.grid_slack[g];
    grid_pos_gth[g] = pos;
    grid_row_gth[g] = row;
  }
}

__global__ void k_item_keys(const int32_t *bus, int64_t n, uint64_t *keys, uint32_t *vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = ((uint64_t)(uint32_t)bus[i] << 32) | (uint32_t)i;
  vals[i] = (uint32_t)i;
  (void)0;
}

__global__ void k_count_bus(const uint64_t *keys, int64_t n, int32_t *cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + (int32_t)(keys[i] >> 32), 1);
}

// per-bus sums of item values in item order (items sorted by (bus, index))
__global__ void k_bus_sums(const int64_t *ptr, const uint32_t *order, const double *v0, const double *v1,
                           int64_t n_bus, double *o0, double *o1, double s0, double s1) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bus) return;
  double a = 0.0, c = 0.0;
  for (int64_t j = ptr[b]; j < ptr[b + 1]; ++j) {
    a += v0[order[j]];
    if (v1) c += v1[order[j]];
  }
  o0[b] = s0 * a;
  if (o1) o1[b] = s1 * c;
}

__global__ void k_net_injection(const double *pg, const double *pl, const double *ql, int64_t n, double *p,
                                double *q) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  p[b] = pg[b] - pl[b];
  q[b] = -ql[b];
}

// per-end coefficients of the rotated branch form (see the evaluation kernel)
// Per branch, for the adjoint: the series admittance g + j b_s = 1/(r + jx),
// its derivative with respect to r (dg/dr = (x^2 - r^2)/D^2, db_s/dr = 2 r x/D^2,
// D = r^2 + x^2; the x-derivatives follow from the Cauchy-Riemann relations),
// 1/tau, b_c and (cos phi, sin phi).
__global__ void k_branch_consts(View v, double2 *kgb, double2 *kab, double2 *ktc, double2 *kph) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= v.n_branch) return;
  const double r = v.br_r[l], x = v.br_x[l];
  const double d = r * r + x * x;
  const double inv = 1.0 / d;
  kgb[l] = make_double2(r * inv, -x * inv);
  kab[l] = make_double2((x * x - r * r) * (inv * inv), 2.0 * r * x * (inv * inv));
  ktc[l] = make_double2(1.0 / v.br_tap[l], v.br_b[l]);
  double sp, cp;
  sincos(v.br_shift[l], &sp, &cp);
  kph[l] = make_double2(cp, sp);
}

__global__ void k_coeff(View v, const double *r_ov, const double *x_ov, const double *b_ov, const double *tap_ov,
                        double2 *gb, double2 *ac) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n_inc) return;
  const int32_t code = v.inc_code[i];
  const int32_t l = code >> 1;
  if (!v.br_status[l]) {
    gb[i] = make_double2(0.0, 0.0);
    ac[i] = make_double2(0.0, 0.0);
    return;
  }
  const double r = r_ov ? r_ov[l] : v.br_r[l];
  const double x = x_ov ? x_ov[l] : v.br_x[l];
  const double bc = b_ov ? b_ov[l] : v.br_b[l];
  const double tau = tap_ov ? tap_ov[l] : v.br_tap[l];
  const double d = r * r + x * x;
  const double g = r / d, b = -x / d;
  double sp, cp;
  sincos(v.br_shift[l], &sp, &cp);
  const double it = 1.0 / tau;
  if ((code & 1) == 0) {  // from end: transformer side
    gb[i] = make_double2((g * cp - b * sp) * it, (g * sp + b * cp) * it);
    ac[i] = make_double2((g + v.br_gfr[l]) * it * it, (b + 0.5 * bc) * it * it);
  } else {                // to end
    gb[i] = make_double2((g * cp + b * sp) * it, (b * cp - g * sp) * it);
    ac[i] = make_double2(g + v.br_gto[l], b + 0.5 * bc);
  }
}

// A^ = (sum of A_e over the bus's ends, in list order) + shunt g; same for C^.
// The evaluation's masked path accumulates in the same order, so a mask of
// all ones gives the same bits.
// A^ and C^ of every bus: the sum of its ends' A, C plus the shunt, in the
// order the evaluation kernels use when they sum under a mask, so that a
// masked evaluation with every branch in service gives the same bits:
// groups of parallel branches merged in incidence order and summed in list
// order for a bus with up to 32 groups; for a larger bus, 32 lane-strided
// partial sums over its ends combined by the butterfly of k_fused_large.
__global__ void k_hat(View v, const double2 *ac, double2 *hat) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= v.n_bus) return;
  const int32_t e0 = v.inc_ptr[o], e1 = v.inc_ptr[o + 1];
  double sa = 0.0, sc = 0.0;
  if (v.bus_npair[o] <= kLaneMaxDegree) {
    for (int32_t e = e0; e < e1;) {
      const int32_t len = v.inc_grp[e];
      double2 t = ac[e];
      for (int32_t i = 1; i < len; ++i)
        t = make_double2(__dadd_rn(t.x, ac[e + i].x), __dadd_rn(t.y, ac[e + i].y));
      sa = __dadd_rn(sa, t.x);
      sc = __dadd_rn(sc, t.y);
      e += len;
    }
  } else {
    double pa[32], pc[32];
    for (int l = 0; l < 32; ++l) {
      pa[l] = 0.0;
      pc[l] = 0.0;
      for (int32_t e = e0 + l; e < e1; e += 32) {
        pa[l] = __dadd_rn(pa[l], ac[e].x);
        pc[l] = __dadd_rn(pc[l], ac[e].y);
      }
    }
    for (int m = 16; m >= 1; m >>= 1) {
      double qa[32], qc[32];
      for (int l = 0; l < 32; ++l) {
        qa[l] = __dadd_rn(pa[l], pa[l ^ m]);
        qc[l] = __dadd_rn(pc[l], pc[l ^ m]);
      }
      for (int l = 0; l < 32; ++l) {
        pa[l] = qa[l];
        pc[l] = qc[l];
      }
    }
    sa = pa[0];
    sc = pc[0];
  }
  const double2 sh = v.bus_sh[o];
  hat[o] = make_double2(__dadd_rn(sa, sh.x), __dadd_rn(sc, sh.y));
}

// per bus: the number of groups of parallel branches (distinct neighbours)
__global__ void k_npair(View v, int32_t *npair) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= v.n_bus) return;
  int32_t n = 0;
  for (int32_t e = v.inc_ptr[o]; e < v.inc_ptr[o + 1]; ++e) n += v.inc_grp[e] > 0;
  npair[o] = n;
}

__global__ void k_pack_bus(View v, const int32_t *base_p, const int32_t *base_q, const int2 *diag,
                           const int32_t *len_tv, int4 *m1, int4 *m2) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= v.n_bus) return;
  m1[o] = make_int4(v.row_p[o], v.row_q[o], base_p[o], base_q[o]);
  const int2 d = diag[o];
  m2[o] = make_int4(d.x, d.y, len_tv[o], v.gen[o]);
}

__global__ void k_pack_inc(View v, const int2 *rt, const int32_t *base_p, const int32_t *base_q, int4 *meta,
                           int4 *pos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n_inc) return;
  const int2 r = rt[i];
  const int32_t o = v.inc_own[i];
  meta[i] = make_int4(o, v.inc_other[i], v.inc_grp[i], v.inc_code[i]);
  const int32_t bp = base_p[o], bq = base_q[o];
  pos[i] = make_int4(bp >= 0 && r.x >= 0 ? bp + r.x : -1, bp >= 0 && r.y >= 0 ? bp + r.y : -1,
                     bq >= 0 && r.x >= 0 ? bq + r.x : -1, bq >= 0 && r.y >= 0 ? bq + r.y : -1);
}

__global__ void k_pack2(const double *a, const double *b, int64_t n, double2 *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(a[i], b[i]);
}

// per-nonzero contribution list: pass 0 counts, pass 1 writes
__global__ void k_contrib(View v, int pass, const int64_t *grid_nnz_off, const int64_t *grid_cptr_off,
                          const int64_t *grid_csrc_off, const int64_t *sh_ptr, const uint32_t *sh_order,
                          const int64_t *grid_sh_off, const int64_t *grid_inc_off, const int32_t *grid_nbr,
                          int32_t *count, const int64_t *cptr, int32_t *src) {
  const int64_t ob = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ob >= v.n_bus) return;
  const int32_t o = (int32_t)ob;
  const int g = v.bus_grid[o];
  const bool ext = v.formulation == PF_EXTENDED;
  const bool is_slack = (o == v.grid_bus_off[g] + v.grid_slack[g]);
  const int64_t ioff = grid_inc_off[g];
  const int32_t p0 = v.inc_ptr[o], p1 = v.inc_ptr[o + 1];
  for (int which = 0; which < 2; ++which) {
    const int32_t base = which == 0 ? v.base_p[o] : v.base_q[o];
    if (base < 0) continue;
    int32_t pos = base;
    auto emit = [&](int32_t j, int32_t i, int32_t len, bool vcol) {
      const int64_t k = grid_nnz_off[g] + pos;
      if (pass == 0) {
        int32_t n = (i < 0) ? (p1 - p0) : len;
        if (i < 0 && vcol) n += (int32_t)(sh_ptr[o + 1] - sh_ptr[o]);
        count[k] = n;
      } else {
        int64_t w = grid_csrc_off[g] + cptr[grid_cptr_off[g] + pos];
        if (i < 0) {
          for (int32_t e = p0; e < p1; ++e) src[w++] = (int32_t)(e - ioff);
          if (vcol)
            for (int64_t s = sh_ptr[o]; s < sh_ptr[o + 1]; ++s)
              src[w++] = 2 * grid_nbr[g] + (int32_t)(sh_order[s] - grid_sh_off[g]);
        } else {
          for (int32_t e = i; e < i + len; ++e) src[w++] = (int32_t)(e - ioff);
        }
      }
      ++pos;
    };
    walk_block(v, o, true, [&](int32_t j, int32_t i, int32_t len) { emit(j, i, len, false); });
    walk_block(v, o, false, [&](int32_t j, int32_t i, int32_t len) { emit(j, i, len, true); });
    const bool extra = ext && ((which == 0 && is_slack) || (which == 1 && v.gen[o] >= 0));
    if (extra) {
      const int64_t k = grid_nnz_off[g] + pos;
      if (pass == 0) count[k] = 1;
      else src[grid_csrc_off[g] + cptr[grid_cptr_off[g] + pos]] = -1;
    }
  }
}

__global__ void k_contrib_const(View v, int pass, const int64_t *grid_nnz_off, const int64_t *grid_cptr_off,
                                const int64_t *grid_csrc_off, const int32_t *gen_pos, const int32_t *grid_pos_gth,
                                int64_t n_gen_tot, int32_t *count, const int64_t *cptr, int32_t *src) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto put = [&](int g, int32_t pos) {
    if (pass == 0) count[grid_nnz_off[g] + pos] = 1;
    else src[grid_csrc_off[g] + cptr[grid_cptr_off[g] + pos]] = -1;
  };
  if (i < n_gen_tot) {
    put(v.bus_grid[v.gen_bus[i]], gen_pos[i]);
    put(v.bus_grid[v.gen_bus[i]], gen_pos[i] + 1);
  }
  if (i < v.n_grids) put((int)i, grid_pos_gth[i]);
}

// local contribution pointer of grid g: S[nnz_off + k] - S[nnz_off], k in [0, nnz(g)]
__global__ void k_cptr(const int64_t *S, const int64_t *grid_nnz_off, const int64_t *grid_cptr_off, int n_grids,
                       int64_t total, int64_t *cptr, int64_t *src_len) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int g = find_segment(grid_cptr_off, n_grids, q);
  const int64_t k = q - grid_cptr_off[g];
  cptr[q] = S[grid_nnz_off[g] + k] - S[grid_nnz_off[g]];
  if (q + 1 == grid_cptr_off[g + 1]) src_len[g] = cptr[q];
}

// ---- rounds of the evaluation kernels ----------------------------------------------------

// sort key: grid, then class (number of neighbours, or kLaneMaxDegree + 1
// for a bus with more), then bus id
__global__ void k_round_keys(View v, uint64_t *keys, uint32_t *vals) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.n_bus) return;
  const int32_t d = v.bus_npair[b];
  const uint64_t cls = d > kLaneMaxDegree ? kLaneMaxDegree + 1 : d;
  keys[b] = ((uint64_t)v.bus_grid[b] << 37) | (cls << 31) | (uint64_t)b;
  vals[b] = (uint32_t)b;
}

__global__ void k_count_large(View v, int32_t *n_large) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.n_bus) return;
  if (v.bus_npair[b] > kLaneMaxDegree) atomicAdd(n_large + v.bus_grid[b], 1);
}

// one thread per round: its buses and items per lane
__global__ void k_round_fill(View v, const uint32_t *sorted, const int64_t *grid_round_off, const int32_t *n_large,
                             int64_t n_rounds, int32_t *rbus, int4 *desc, int32_t *slots) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rounds) return;
  const int g = find_segment(grid_round_off, v.n_grids, r);
  const int64_t rl = r - grid_round_off[g];
  const int64_t gb0 = v.grid_bus_off[g];
  const int64_t n_norm = v.grid_nbus[g] - n_large[g];
  const int64_t n_norm_rounds = (n_norm + 31) / 32;
  if (rl < n_norm_rounds) {
    int32_t nb = 0, dmax = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t i = 32 * rl + l;
      int32_t b = -1;
      if (i < n_norm) {
        b = (int32_t)sorted[gb0 + i];
        dmax = max(dmax, v.bus_npair[b]);
        ++nb;
      }
      rbus[32 * r + l] = b;
    }
    desc[r] = make_int4(0, dmax, nb, 0);
    slots[r] = 32 * dmax;
  } else {
    const int32_t b = (int32_t)sorted[gb0 + n_norm + (rl - n_norm_rounds)];
    for (int l = 0; l < 32; ++l) rbus[32 * r + l] = l == 0 ? b : -1;
    desc[r] = make_int4(0, v.bus_npair[b], 1, 1);
    slots[r] = 0;
  }
}

__global__ void k_round_base(const int64_t *S, int64_t n_rounds, int4 *desc, int32_t *err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rounds) return;
  if (S[r] > 0x7fffffffLL) atomicOr(err, kErrMap);
  desc[r].x = (int32_t)S[r];
}

// one thread per (round, lane): the slots of the lane's bus, one per group of
// parallel branches (pair of buses) in incidence order, then padding
__global__ void k_slot_fill(View v, int64_t n_rounds, const int4 *desc, const int32_t *rbus, int4 *smeta,
                            int4 *spos, int4 *sidx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 32 * n_rounds) return;
  const int64_t r = t >> 5;
  const int l = (int)(t & 31);
  const int4 d = desc[r];
  if (d.w) return;                               // a large bus: no slots
  const int32_t b = rbus[t];
  int j = 0;
  if (b >= 0) {
    for (int32_t e = v.inc_ptr[b]; e < v.inc_ptr[b + 1]; ++e) {
      const int32_t len = v.inc_grp[e];
      if (len == 0) continue;
      const int64_t q = (int64_t)d.x + 32 * j + l;
      smeta[q] = make_int4(v.inc_other[e], len, v.inc_code[e], e);
      const int4 p = v.inc_pos[e];
      spos[q] = p;
      // the P and Q rows of a bus have the same columns: one in-row offset each for theta_k, V_k
      const int32_t bp = v.base_p[b], bq = v.base_q[b];
      const int32_t ot = p.x >= 0 ? p.x - bp : (p.z >= 0 ? p.z - bq : -1);
      const int32_t ov = p.y >= 0 ? p.y - bp : (p.w >= 0 ? p.w - bq : -1);
      sidx[q] = make_int4(v.inc_other[e], (ot & 0xffff) | (ov << 16), len, len == 1 ? v.inc_code[e] : e);
      ++j;
    }
  }
  for (; j < d.y; ++j) {
    const int64_t q = (int64_t)d.x + 32 * j + l;
    smeta[q] = make_int4(0, -1, 0, 0);
    spos[q] = make_int4(-1, -1, -1, -1);
    sidx[q] = make_int4(0, -1, -1, 0);
  }
}

// bus records in round order (and, for per-call overrides, the coefficients)
__global__ void k_rbus_fill(View v, int64_t n, const int32_t *rbus, const double2 *hat, int4 *m1, int4 *m2,
                            double2 *rh, double2 *ri) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t b = rbus[i];
  if (b >= 0) {
    if (m1) m1[i] = v.bus_meta[b];
    if (m2) m2[i] = v.bus_meta2[b];
    rh[i] = hat[b];
    if (ri) ri[i] = v.bus_inj[b];
  } else {
    if (m1) m1[i] = make_int4(-1, -1, -1, -1);
    if (m2) m2[i] = make_int4(-1, -1, 0, -1);
    rh[i] = make_double2(0.0, 0.0);
    if (ri) ri[i] = make_double2(0.0, 0.0);
  }
}

// per round of 32 buses of every instance: its instance, round and
// descriptor.  The rounds of a grid ascend in neighbour count; an instance's
// units take them heaviest and lightest alternately (n-1, 0, n-2, 1, ...), so
// the CTAs that run side by side -- all of them, when one instance fills less
// than a wave -- carry a mix of long and short rounds.
// Each unit also carries its grid and instance offsets, so that the
// evaluation kernel has every pointer of a unit after one round of loads.
__global__ void k_unit_fill(View v, const int64_t *lane_off, int4 *unit, int4 *info, longlong2 *ptr) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= v.n_lane_units) return;
  const int inst = find_segment(lane_off, v.n_inst, u);
  const int g = v.inst_grid[inst];
  const int64_t j = u - lane_off[inst], n = lane_off[inst + 1] - lane_off[inst];
  const int64_t r = v.grid_round_off[g] + ((j & 1) ? (j >> 1) : n - 1 - (j >> 1));
  const int4 d = v.round_desc[r];
  unit[u] = make_int4(inst, (int32_t)r, d.x, d.y | (d.z << 8));
  info[u] = make_int4(g, v.grid_nbus[g], (int32_t)v.grid_bus_off[g], 0);
  ptr[2 * u] = make_longlong2(v.inst_x_off[inst], v.inst_f_off[inst]);
  ptr[2 * u + 1] = make_longlong2(v.inst_v_off[inst], v.inst_bus_off[inst] - v.grid_bus_off[g]);
}

// per large bus of every instance: its instance and bus (the rounds after
// the grid's rounds of 32 buses hold one large bus each)
__global__ void k_large_fill(View v, const int64_t *large_off, const int64_t *lane_rounds, int2 *out) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= v.n_large_units) return;
  const int inst = find_segment(large_off, v.n_inst, u);
  const int g = v.inst_grid[inst];
  const int64_t r = v.grid_round_off[g] + lane_rounds[g] + (u - large_off[inst]);
  out[u] = make_int2(inst, v.rbus[32 * r]);
}

// per chunk of instance-buses: the instance of its first bus; one more entry
// for the last bus
__global__ void k_chunk_inst(View v, int64_t n_chunks, int32_t *out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_chunks) return;
  const int64_t q = c < n_chunks ? (c << kChunkLog2) : v.n_bus_inst - 1;
  out[c] = find_segment(v.inst_bus_off, v.n_inst, q);
}

__global__ void k_rec_base(View v, int64_t *base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n_inst) return;
  base[i] = v.inst_bus_off[i] - v.grid_bus_off[v.inst_grid[i]];
}

// per slot: the coefficients of its group of parallel branches, summed in
// incidence order (the merged branch end of the pair of buses)
__global__ void k_slot_coeff(View v, int64_t n_slots, const int4 *smeta, const double2 *gb, const double2 *ac,
                             double2 *sgb, double2 *sac, double2 *sgbm) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_slots) return;
  const int4 m = smeta[q];
  if (m.y > 0) {
    double2 g = gb[m.w], a = ac[m.w], gm = gb[v.inc_mirror[m.w]];
    for (int32_t i = 1; i < m.y; ++i) {
      const double2 gi = gb[m.w + i], ai = ac[m.w + i], mi = gb[v.inc_mirror[m.w + i]];
      g = make_double2(__dadd_rn(g.x, gi.x), __dadd_rn(g.y, gi.y));
      a = make_double2(__dadd_rn(a.x, ai.x), __dadd_rn(a.y, ai.y));
      gm = make_double2(__dadd_rn(gm.x, mi.x), __dadd_rn(gm.y, mi.y));
    }
    sgb[q] = g;
    sac[q] = a;
    if (sgbm) sgbm[q] = gm;
  } else {
    sgb[q] = make_double2(0.0, 0.0);
    sac[q] = make_double2(0.0, 0.0);
    if (sgbm) sgbm[q] = make_double2(0.0, 0.0);
  }
}

// per slot: the larger of sum |G_i| and sum |B_i| over its group's ends (any
// subset of the group under a mask stays below it), maximised over all slots
// into *mx (the bit pattern of a non-negative double orders as an integer)
__global__ void k_slot_absmax(int64_t n_slots, const int4 *smeta, const double2 *gb, unsigned long long *mx) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_slots) return;
  const int4 m = smeta[q];
  if (m.y <= 0) return;
  double sg = 0.0, sb = 0.0;
  for (int32_t i = 0; i < m.y; ++i) {
    const double2 gi = gb[m.w + i];
    sg += fabs(gi.x);
    sb += fabs(gi.y);
  }
  const double a = fmax(sg, sb);
  if (a > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(isfinite(a) ? a : 0x1p1000));
}

// per slot: its merged (G, B) in the fixed point of the evaluation kernels
__global__ void k_slot_fix(int64_t n_slots, const int4 *smeta, const double2 *sgb, double scale, int4 *sgbx) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_slots) return;
  const double2 g = sgb[q];
  sgbx[q] = smeta[q].y > 0 ? coef_limbs(to_fix(g.x, scale), to_fix(g.y, scale)) : make_int4(0, 0, 0, 0);
}

template <class T>
std::vector<T> to_host(const T *d, size_t n, cudaStream_t s, int *rc) {
  std::vector<T> h(n);
  if (n) {
    cudaError_t e = cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) *rc = fail(PF_ERR_CUDA, std::string("copy to host: ") + cudaGetErrorString(e));
  }
  return h;
}

// Sums per bus of item values, in item order.
int bus_sums(Ctx &c, TempList &tmp, const int32_t *d_item_bus, int64_t n_items, const double *d_v0,
             const double *d_v1, double s0, double s1, double *out0, double *out1, int64_t **ptr_out,
             uint32_t **order_out, cudaStream_t s) {
  const int64_t n_bus = c.v.n_bus;
  const int64_t np = sort_padded(n_items);
  uint64_t *keys;
  uint32_t *vals;
  int32_t *cnt;
  int64_t *ptr, *stmp;
  PF_TRY(tmp.alloc(&keys, np));
  PF_TRY(tmp.alloc(&vals, np));
  PF_TRY(tmp.alloc(&cnt, n_bus));
  PF_TRY(tmp.alloc(&ptr, n_bus + 1));
  PF_TRY(tmp.alloc(&stmp, scan_tmp_elems(n_bus)));
  PF_CUDA_TRY(cudaMemsetAsync(cnt, 0, n_bus * sizeof(int32_t), s));
  if (n_items > 0) {
    k_item_keys<<<nblk(n_items), TB, 0, s>>>(d_item_bus, n_items, keys, vals);
    PF_TRY(bitonic_sort_pairs(keys, vals, n_items, s));
    k_count_bus<<<nblk(n_items), TB, 0, s>>>(keys, n_items, cnt);
  }
  PF_TRY(exclusive_scan<int32_t>(cnt, ptr, n_bus, stmp, s));
  k_bus_sums<<<nblk(n_bus), TB, 0, s>>>(ptr, vals, d_v0, d_v1, n_bus, out0, out1, s0, s1);
  PF_CUDA_TRY(cudaGetLastError());
  if (ptr_out) *ptr_out = ptr;
  if (order_out) *order_out = vals;
  return PF_OK;
}

}  // namespace

// --------------------------------------------------------------------------
// coefficients (also used per call when branch parameters are overridden)
// --------------------------------------------------------------------------

int compute_coefficients(Ctx &c, const double *r, const double *x, const double *b, const double *tap,
                         double2 *gb, double2 *ac, double2 *hat, cudaStream_t s) {
  if (c.v.n_inc > 0) {
    k_coeff<<<nblk(c.v.n_inc), TB, 0, s>>>(c.v, r, x, b, tap, gb, ac);
    PF_CUDA_TRY(cudaGetLastError());
  }
  k_hat<<<nblk(c.v.n_bus), TB, 0, s>>>(c.v, ac, hat);
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

// ---- rounds of the fused kernel: buses sorted by degree, 32 per round ---------------

int build_rounds(Ctx &c, cudaStream_t s) {
  View &v = c.v;
  const int G = v.n_grids;
  const int64_t N = v.n_bus;
  TempList tmp;
  const int64_t np = sort_padded(N);
  uint64_t *keys;
  uint32_t *vals;
  int32_t *n_large;
  PF_TRY(tmp.alloc(&keys, np));
  PF_TRY(tmp.alloc(&vals, np));
  PF_TRY(tmp.alloc(&n_large, G));
  PF_CUDA_TRY(cudaMemsetAsync(n_large, 0, G * sizeof(int32_t), s));
  k_round_keys<<<nblk(N), TB, 0, s>>>(v, keys, vals);
  k_count_large<<<nblk(N), TB, 0, s>>>(v, n_large);
  PF_CUDA_TRY(cudaGetLastError());
  PF_TRY(bitonic_sort_pairs(keys, vals, N, s));
  int rc = PF_OK;
  std::vector<int32_t> h_large = to_host(n_large, G, s, &rc);
  if (rc) return rc;
  c.grid_round_off.assign(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    const int64_t n_norm = c.grid_bus_off[g + 1] - c.grid_bus_off[g] - h_large[g];
    c.grid_round_off[g + 1] = c.grid_round_off[g] + (n_norm + 31) / 32 + h_large[g];
  }
  const int64_t R = c.grid_round_off[G];
  c.n_rounds = R;
  int64_t *d_round_off, *S, *stmp;
  int32_t *rbus, *slots, *err;
  int4 *desc;
  PF_TRY(upload(c, &d_round_off, c.grid_round_off, s));
  PF_TRY(dev_alloc(c, &rbus, 32 * R));
  PF_TRY(dev_alloc(c, &desc, R));
  PF_TRY(tmp.alloc(&slots, R));
  PF_TRY(tmp.alloc(&S, R + 1));
  PF_TRY(tmp.alloc(&stmp, scan_tmp_elems(R) + 1));
  PF_TRY(tmp.alloc(&err, 1));
  PF_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  k_round_fill<<<nblk(R), TB, 0, s>>>(v, vals, d_round_off, n_large, R, rbus, desc, slots);
  PF_CUDA_TRY(cudaGetLastError());
  PF_TRY(exclusive_scan<int32_t>(slots, S, R, stmp, s));
  k_round_base<<<nblk(R), TB, 0, s>>>(S, R, desc, err);
  PF_CUDA_TRY(cudaGetLastError());
  std::vector<int64_t> total = to_host(S + R, 1, s, &rc);
  if (rc) return rc;
  std::vector<int32_t> herr = to_host(err, 1, s, &rc);
  if (rc) return rc;
  if (herr[0]) return fail(PF_ERR_UNSUPPORTED, "more than 2^31 evaluation slots");
  const int64_t NS = total[0];
  c.n_slots = NS;
  int4 *smeta, *spos, *sidx, *m1, *m2;
  double2 *sgb, *sac, *sgbm, *rh, *ri;
  PF_TRY(dev_alloc(c, &smeta, NS));
  PF_TRY(dev_alloc(c, &spos, NS));
  PF_TRY(dev_alloc(c, &sidx, NS));
  PF_TRY(dev_alloc(c, &sgb, NS));
  PF_TRY(dev_alloc(c, &sac, NS));
  PF_TRY(dev_alloc(c, &sgbm, NS));
  PF_TRY(dev_alloc(c, &c.ov_slot_gbm, NS));
  PF_TRY(dev_alloc(c, &m1, 32 * R));
  PF_TRY(dev_alloc(c, &m2, 32 * R));
  PF_TRY(dev_alloc(c, &rh, 32 * R));
  PF_TRY(dev_alloc(c, &ri, 32 * R));
  PF_TRY(dev_alloc(c, &c.ov_slot_gb, NS));
  PF_TRY(dev_alloc(c, &c.ov_slot_ac, NS));
  PF_TRY(dev_alloc(c, &c.ov_rbus_hat, 32 * R));
  if (NS > 0) {
    k_slot_fill<<<nblk(32 * R), TB, 0, s>>>(v, R, desc, rbus, smeta, spos, sidx);
    k_slot_coeff<<<nblk(NS), TB, 0, s>>>(v, NS, smeta, v.inc_gb, v.inc_ac, sgb, sac, sgbm);
    PF_CUDA_TRY(cudaGetLastError());
  }
  k_rbus_fill<<<nblk(32 * R), TB, 0, s>>>(v, 32 * R, rbus, v.bus_hat, m1, m2, rh, ri);
  PF_CUDA_TRY(cudaGetLastError());
  // fixed-point coefficients: 2^coef_log2 bounds |G|, |B| over every group
  // (capped at kMaxCoefLog2; larger coefficients are marked kBadFix)
  {
    unsigned long long *mx;
    PF_TRY(tmp.alloc(&mx, 1));
    PF_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    if (NS > 0) {
      k_slot_absmax<<<nblk(NS), TB, 0, s>>>(NS, smeta, v.inc_gb, mx);
      PF_CUDA_TRY(cudaGetLastError());
    }
    std::vector<unsigned long long> hm = to_host(mx, 1, s, &rc);
    if (rc) return rc;
    double m = 0.0;
    std::memcpy(&m, &hm[0], sizeof(double));
    int lg = 1;
    while (lg < kMaxCoefLog2 && !(m < std::ldexp(1.0, lg))) ++lg;
    v.coef_log2 = lg;
    v.coef_scale = std::ldexp(1.0, 59 - lg);
    int4 *sgbx;
    PF_TRY(dev_alloc(c, &sgbx, NS));
    PF_TRY(dev_alloc(c, &c.ov_slot_gbx, NS));
    if (NS > 0) {
      k_slot_fix<<<nblk(NS), TB, 0, s>>>(NS, smeta, sgb, v.coef_scale, sgbx);
      PF_CUDA_TRY(cudaGetLastError());
    }
    v.slot_gbx = sgbx;
  }
  v.grid_round_off = d_round_off;
  v.round_desc = desc;
  v.rbus = rbus;
  v.rbus_meta = m1;
  v.rbus_meta2 = m2;
  v.rbus_hat = rh;
  v.rbus_inj = ri;
  v.slot_meta = smeta;
  v.slot_pos = spos;
  v.slot_idx = sidx;
  v.slot_gb = sgb;
  v.slot_ac = sac;
  v.slot_gbm = sgbm;
  if (c.n_rounds >= 0x7fffffffLL / 32) return fail(PF_ERR_UNSUPPORTED, "too many evaluation rounds");
  // units of work: the rounds of 32 buses and the large buses of every instance
  const int I = v.n_inst;
  std::vector<int64_t> lane_rounds(G), lane_off(I + 1, 0), large_off(I + 1, 0);
  for (int g = 0; g < G; ++g) lane_rounds[g] = c.grid_round_off[g + 1] - c.grid_round_off[g] - h_large[g];
  for (int i = 0; i < I; ++i) {
    const int g = c.inst_grid[i];
    lane_off[i + 1] = lane_off[i] + lane_rounds[g];
    large_off[i + 1] = large_off[i] + h_large[g];
  }
  v.n_lane_units = lane_off[I];
  v.n_large_units = large_off[I];
  c.lane_off = lane_off;
  c.large_off = large_off;
  int64_t *d_lane_off, *d_large_off, *d_lane_rounds, *rec_base;
  int4 *unit, *uinfo;
  longlong2 *uptr;
  int2 *large;
  PF_TRY(upload(c, &d_lane_off, lane_off, s));
  PF_TRY(upload(c, &d_large_off, large_off, s));
  PF_TRY(upload(c, &d_lane_rounds, lane_rounds, s));
  PF_TRY(dev_alloc(c, &unit, v.n_lane_units));
  PF_TRY(dev_alloc(c, &uinfo, v.n_lane_units));
  PF_TRY(dev_alloc(c, &uptr, 2 * v.n_lane_units));
  if (c.v.n_bus >= 0x7fffffffLL) return fail(PF_ERR_UNSUPPORTED, "more than 2^31 buses");
  PF_TRY(dev_alloc(c, &large, v.n_large_units));
  PF_TRY(dev_alloc(c, &rec_base, I));
  if (v.n_lane_units > 0) k_unit_fill<<<nblk(v.n_lane_units), TB, 0, s>>>(v, d_lane_off, unit, uinfo, uptr);
  if (v.n_large_units > 0) k_large_fill<<<nblk(v.n_large_units), TB, 0, s>>>(v, d_large_off, d_lane_rounds, large);
  k_rec_base<<<nblk(I), TB, 0, s>>>(v, rec_base);
  {
    const int64_t n_chunks = (v.n_bus_inst + (1 << kChunkLog2) - 1) >> kChunkLog2;
    int32_t *ci;
    PF_TRY(dev_alloc(c, &ci, n_chunks + 1));
    k_chunk_inst<<<nblk(n_chunks + 1), TB, 0, s>>>(v, n_chunks, ci);
    v.chunk_inst = ci;
  }
  PF_CUDA_TRY(cudaGetLastError());
  v.unit_rec = unit;
  v.unit_info = uinfo;
  v.unit_ptr = uptr;
  v.large_rec = large;
  v.inst_rec_base = rec_base;
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  return PF_OK;
}

// ---- tiles of the fused kernel: consecutive buses, pairs listed bus by bus ---------------

// per bus: its pairs in the tile kernel's list (none for a large bus)
__global__ void k_pair_count(View v, int32_t *cnt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.n_bus) return;
  const int32_t d = v.bus_npair[b];
  cnt[b] = d > kLaneMaxDegree ? 0 : d;
}

__global__ void k_pair_ptr(const int64_t *S, int64_t n_bus, int32_t *ptr, int32_t *err) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b > n_bus) return;
  if (S[b] > 0x7fffffffLL) atomicOr(err, kErrMap);
  ptr[b] = (int32_t)S[b];
}

// The tiles of grid g, formed greedily along the bus order: a tile takes the
// next bus while it holds fewer than kTileBuses buses and the bus's pairs keep
// it within kTilePairs; a large bus ends the tile and belongs to none.
// (split_rounds = s: at most cap_bus = kTileBuses >> s buses and cap_pairs =
// kTilePairs >> s pairs, a bus with more pairs alone in its tile.)
// Pass 0 counts them (cnt[g]); pass 1 writes, per tile t (global index from
// off[g]), {first bus, buses, first pair, pairs}, the J segments of its P and Q
// rows {P start, P length, Q start, Q length}, its F rows {first P row, P
// rows, first Q row, Q rows}, and each bus's index in its tile.  The rows of a
// tile's buses must be consecutive (they are in both formulations); a tile
// where they are not sets kErrMap.
__global__ void k_tiles(View v, int pass, int cap_bus, int cap_pairs, int64_t *cnt, const int64_t *off, int4 *desc,
                        int4 *seg, int4 *frow, int32_t *bus_local, int32_t *max_stage, int32_t *err) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= v.n_grids) return;
  const int64_t gb0 = v.grid_bus_off[g], nb = v.grid_nbus[g];
  const bool ext = v.formulation == PF_EXTENDED;
  const int32_t slack = v.grid_slack[g];
  int64_t t = pass ? off[g] : 0;
  int64_t b = 0;
  while (b < nb) {
    if (v.bus_npair[gb0 + b] > kLaneMaxDegree) {       // large: in no tile
      ++b;
      continue;
    }
    const int64_t b0 = b;
    int32_t pairs = 0;
    while (b < nb && b - b0 < cap_bus) {
      const int32_t d = v.bus_npair[gb0 + b];
      if (d > kLaneMaxDegree || (b > b0 && pairs + d > cap_pairs)) break;
      pairs += d;
      ++b;
    }
    if (pass) {
      int32_t rp0 = -1, rp1 = -1, rq0 = -1, rq1 = -1, np_ = 0, nq_ = 0;
      int32_t sp0 = 0, sp1 = 0, sq0 = 0, sq1 = 0;
      for (int64_t i = b0; i < b; ++i) {
        const int64_t o = gb0 + i;
        bus_local[o] = (int32_t)(i - b0);
        const int4 bm = v.bus_meta[o], bm2 = v.bus_meta2[o];
        const int32_t lp = bm2.z + (ext && i == slack ? 1 : 0);
        const int32_t lq = bm2.z + (ext && bm2.w >= 0 ? 1 : 0);
        if (bm.x >= 0) {
          if (rp0 < 0) { rp0 = bm.x; sp0 = bm.z; }
          rp1 = bm.x;
          sp1 = bm.z + lp;
          ++np_;
        }
        if (bm.y >= 0) {
          if (rq0 < 0) { rq0 = bm.y; sq0 = bm.w; }
          rq1 = bm.y;
          sq1 = bm.w + lq;
          ++nq_;
        }
      }
      if ((np_ && rp1 - rp0 + 1 != np_) || (nq_ && rq1 - rq0 + 1 != nq_)) atomicOr(err, kErrMap);
      desc[t] = make_int4((int32_t)(gb0 + b0), (int32_t)(b - b0), v.pair_ptr[gb0 + b0], pairs);
      seg[t] = make_int4(sp0, sp1 - sp0, sq0, sq1 - sq0);
      frow[t] = make_int4(rp0, np_, rq0, nq_);
      atomicMax(max_stage, (sp1 - sp0) + (sq1 - sq0) + 3);
    }
    ++t;
  }
  if (!pass) cnt[g] = t;
}

// per bus of a tile: its pairs (groups of parallel branches in incidence
// order) in the formats of the slot arrays (pmeta: nullptr to leave it)
__global__ void k_pair_fill(View v, const int32_t *bus_local, int4 *pmeta, int4 *pidx) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.n_bus) return;
  if (v.bus_npair[b] > kLaneMaxDegree) return;
  int64_t q = v.pair_ptr[b];
  const int32_t bp = v.base_p[b], bq = v.base_q[b];
  for (int32_t e = v.inc_ptr[b]; e < v.inc_ptr[b + 1]; ++e) {
    const int32_t len = v.inc_grp[e];
    if (len == 0) continue;
    if (pmeta) pmeta[q] = make_int4(v.inc_other[e], len, v.inc_code[e], e);
    const int4 p = v.inc_pos[e];
    const int32_t ot = p.x >= 0 ? p.x - bp : (p.z >= 0 ? p.z - bq : -1);
    const int32_t ov = p.y >= 0 ? p.y - bp : (p.w >= 0 ? p.w - bq : -1);
    pidx[q] = make_int4(v.inc_other[e], (ot & 0xffff) | (ov << 16), len | (bus_local[b] << 16),
                        len == 1 ? v.inc_code[e] : e);
    ++q;
  }
}

// Per tile: its external neighbours -- the buses outside the tile that its
// pairs reach -- in ascending order (pass 0 counts them, pass 1 writes them at
// ext_off[t]), and in bits 24..31 of each pair's group-length field the
// index of the neighbour's voltage record among the tile's records (buses of
// the tile first, in order, then the external neighbours), for the form of
// the fused kernel that computes the records itself.
__global__ void k_tile_ext(int64_t n_tiles, const int4 *desc, int pass, const int64_t *ext_off, int32_t *ext_cnt,
                           int32_t *ext, int4 *pidx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const int4 d = desc[t];                            // {first bus, buses, first pair, pairs}
  int32_t list[kTilePairs];
  int n = 0;
  for (int32_t p = 0; p < d.w; ++p) {
    const int32_t k = pidx[d.z + p].x;
    if (k >= d.x && k < d.x + d.y) continue;
    int i = n;                                       // insertion into the sorted list, no duplicates
    while (i > 0 && list[i - 1] > k) --i;
    if (i > 0 && list[i - 1] == k) continue;
    for (int j = n; j > i; --j) list[j] = list[j - 1];
    list[i] = k;
    ++n;
  }
  if (pass == 0) {
    ext_cnt[t] = n;
    return;
  }
  for (int i = 0; i < n; ++i) ext[ext_off[t] + i] = list[i];
  for (int32_t p = 0; p < d.w; ++p) {
    int4 q = pidx[d.z + p];
    int32_t loc;
    if (q.x >= d.x && q.x < d.x + d.y) {
      loc = q.x - d.x;
    } else {
      int lo = 0, hi = n - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (list[mid] < q.x) lo = mid + 1; else hi = mid;
      }
      loc = kTileBuses + lo;
    }
    q.z = (q.z & 0x00ffffff) | (loc << 24);
    pidx[d.z + p] = q;
  }
}

// per tile of every instance: its eight-int4 unit record
__global__ void k_tunit_fill(View v, const int64_t *tile_off, const int64_t *grid_tile_off, const int4 *desc,
                             const int4 *seg, const int4 *frow, const int64_t *ext_off, int4 *unit) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= v.n_tile_units) return;
  const int inst = find_segment(tile_off, v.n_inst, u);
  const int g = v.inst_grid[inst];
  const int64_t t = grid_tile_off[g] + (u - tile_off[inst]);
  int4 *r = unit + 8 * u;
  r[0] = desc[t];
  r[1] = seg[t];
  r[2] = frow[t];
  r[3] = make_int4(inst, g, (int32_t)v.grid_bus_off[g], v.grid_nbus[g]);
  const int64_t xo = v.inst_x_off[inst], fo = v.inst_f_off[inst], vo = v.inst_v_off[inst],
                rb = v.inst_bus_off[inst] - v.grid_bus_off[g];
  r[4] = make_int4((int32_t)(xo & 0xffffffff), (int32_t)(xo >> 32), (int32_t)(fo & 0xffffffff), (int32_t)(fo >> 32));
  r[5] = make_int4((int32_t)(vo & 0xffffffff), (int32_t)(vo >> 32), (int32_t)(rb & 0xffffffff), (int32_t)(rb >> 32));
  r[6] = make_int4((int32_t)ext_off[t], (int32_t)(ext_off[t + 1] - ext_off[t]), 0, 0);
  r[7] = make_int4(0, 0, 0, 0);
}

// The tiles of split_rounds = split: the partition, each pair's bus index in
// its tile (the pair index records of this partition) and the unit records.
int build_tile_set(Ctx &c, int split, cudaStream_t s) {
  View &v = c.v;
  Ctx::TileSet &ts = c.tiles[split];
  const int G = v.n_grids;
  const int64_t N = v.n_bus, NP = c.n_pairs;
  const int cap_bus = kTileBuses >> split, cap_pairs = kTilePairs >> split;
  TempList tmp;
  int rc = PF_OK;
  int32_t *err, *bus_local, *max_stage;
  int64_t *gcnt;
  PF_TRY(tmp.alloc(&err, 1));
  PF_TRY(tmp.alloc(&max_stage, 1));
  PF_TRY(tmp.alloc(&gcnt, G));
  PF_TRY(tmp.alloc(&bus_local, N));
  PF_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  PF_CUDA_TRY(cudaMemsetAsync(max_stage, 0, sizeof(int32_t), s));
  k_tiles<<<nblk(G, 64), 64, 0, s>>>(v, 0, cap_bus, cap_pairs, gcnt, nullptr, nullptr, nullptr, nullptr, nullptr,
                                      nullptr, err);
  PF_CUDA_TRY(cudaGetLastError());
  std::vector<int64_t> h_cnt = to_host(gcnt, G, s, &rc);
  if (rc) return rc;
  std::vector<int64_t> grid_tile_off(G + 1, 0);
  for (int g = 0; g < G; ++g) grid_tile_off[g + 1] = grid_tile_off[g] + h_cnt[g];
  const int64_t T = grid_tile_off[G];
  int64_t *d_gto;
  int4 *desc, *seg, *frow, *pidx;
  PF_TRY(tmp.alloc(&d_gto, G + 1));
  PF_CUDA_TRY(cudaMemcpyAsync(d_gto, grid_tile_off.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PF_TRY(tmp.alloc(&desc, T));
  PF_TRY(tmp.alloc(&seg, T));
  PF_TRY(tmp.alloc(&frow, T));
  k_tiles<<<nblk(G, 64), 64, 0, s>>>(v, 1, cap_bus, cap_pairs, nullptr, d_gto, desc, seg, frow, bus_local,
                                      max_stage, err);
  PF_CUDA_TRY(cudaGetLastError());
  PF_TRY(dev_alloc(c, &pidx, NP));
  k_pair_fill<<<nblk(N), TB, 0, s>>>(v, bus_local, nullptr, pidx);
  PF_CUDA_TRY(cudaGetLastError());
  // external neighbours of every tile and the pairs' record indices
  int32_t *ext_cnt, *ext;
  int64_t *ext_S, *ext_tmp;
  PF_TRY(tmp.alloc(&ext_cnt, T));
  PF_TRY(tmp.alloc(&ext_S, T + 1));
  PF_TRY(tmp.alloc(&ext_tmp, scan_tmp_elems(T) + 1));
  if (T > 0) {
    k_tile_ext<<<nblk(T, 64), 64, 0, s>>>(T, desc, 0, nullptr, ext_cnt, nullptr, pidx);
    PF_CUDA_TRY(cudaGetLastError());
  }
  PF_TRY(exclusive_scan<int32_t>(ext_cnt, ext_S, T, ext_tmp, s));
  std::vector<int64_t> n_ext = to_host(ext_S + T, 1, s, &rc);
  if (rc) return rc;
  if (n_ext[0] > 0x7fffffffLL) return fail(PF_ERR_UNSUPPORTED, "more than 2^31 external neighbours of tiles");
  PF_TRY(dev_alloc(c, &ext, n_ext[0]));
  if (T > 0) {
    k_tile_ext<<<nblk(T, 64), 64, 0, s>>>(T, desc, 1, ext_S, nullptr, ext, pidx);
    PF_CUDA_TRY(cudaGetLastError());
  }
  // units: the tiles of every instance, instance by instance
  const int I = v.n_inst;
  ts.tile_off.assign(I + 1, 0);
  for (int i = 0; i < I; ++i) ts.tile_off[i + 1] = ts.tile_off[i] + h_cnt[c.inst_grid[i]];
  ts.n_units = ts.tile_off[I];
  int64_t *d_tile_off;
  int4 *unit;
  PF_TRY(tmp.alloc(&d_tile_off, I + 1));
  PF_CUDA_TRY(cudaMemcpyAsync(d_tile_off, ts.tile_off.data(), (I + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PF_TRY(dev_alloc(c, &unit, 8 * ts.n_units));
  if (ts.n_units > 0) {
    View vu = v;
    vu.n_tile_units = ts.n_units;
    k_tunit_fill<<<nblk(ts.n_units), TB, 0, s>>>(vu, d_tile_off, d_gto, desc, seg, frow, ext_S, unit);
    PF_CUDA_TRY(cudaGetLastError());
  }
  std::vector<int32_t> herr = to_host(err, 1, s, &rc);
  if (rc) return rc;
  std::vector<int32_t> hstage = to_host(max_stage, 1, s, &rc);
  if (rc) return rc;
  if (herr[0]) return fail(PF_ERR_UNSUPPORTED, "tile layout: rows of consecutive buses are not consecutive");
  ts.pair_idx = pidx;
  ts.tunit = unit;
  ts.ext = ext;
  ts.stage = (hstage[0] + 1) & ~1;
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  return PF_OK;
}

int use_tile_set(Ctx &c, int split, cudaStream_t s) {
  if (!c.tiles[split].tunit) PF_TRY(build_tile_set(c, split, s));
  const Ctx::TileSet &ts = c.tiles[split];
  c.v.pair_idx = ts.pair_idx;
  c.v.tunit = ts.tunit;
  c.v.tile_ext = ts.ext;
  c.v.n_tile_units = ts.n_units;
  c.v.tile_stage = ts.stage;
  return PF_OK;
}

// The list of pairs of connected buses bus by bus (shared by every tiling),
// their coefficients, and the tiles of split_rounds = 0.
int build_tiles(Ctx &c, cudaStream_t s) {
  View &v = c.v;
  const int64_t N = v.n_bus;
  TempList tmp;
  int rc = PF_OK;
  int32_t *cnt, *err, *ptr;
  int64_t *S, *stmp;
  PF_TRY(tmp.alloc(&cnt, N));
  PF_TRY(tmp.alloc(&S, N + 1));
  PF_TRY(tmp.alloc(&stmp, scan_tmp_elems(N) + 1));
  PF_TRY(tmp.alloc(&err, 1));
  PF_TRY(dev_alloc(c, &ptr, N + 1));
  PF_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  k_pair_count<<<nblk(N), TB, 0, s>>>(v, cnt);
  PF_CUDA_TRY(cudaGetLastError());
  PF_TRY(exclusive_scan<int32_t>(cnt, S, N, stmp, s));
  k_pair_ptr<<<nblk(N + 1), TB, 0, s>>>(S, N, ptr, err);
  PF_CUDA_TRY(cudaGetLastError());
  v.pair_ptr = ptr;
  std::vector<int64_t> total = to_host(S + N, 1, s, &rc);
  if (rc) return rc;
  std::vector<int32_t> herr = to_host(err, 1, s, &rc);
  if (rc) return rc;
  if (herr[0]) return fail(PF_ERR_UNSUPPORTED, "more than 2^31 pairs of connected buses");
  const int64_t NP = total[0];
  c.n_pairs = NP;
  int4 *pmeta, *pgbx;
  double2 *pgb, *pac;
  PF_TRY(dev_alloc(c, &pmeta, NP));
  PF_TRY(dev_alloc(c, &pgb, NP));
  PF_TRY(dev_alloc(c, &pac, NP));
  PF_TRY(dev_alloc(c, &pgbx, NP));
  PF_TRY(dev_alloc(c, &c.ov_pair_gb, NP));
  PF_TRY(dev_alloc(c, &c.ov_pair_ac, NP));
  PF_TRY(dev_alloc(c, &c.ov_pair_gbx, NP));
  {
    // the pair metadata (any tiling's bus indices would do; these are rewritten per tiling)
    int4 *scratch;
    int32_t *zero_local;
    PF_TRY(tmp.alloc(&scratch, NP));
    PF_TRY(tmp.alloc(&zero_local, N));
    PF_CUDA_TRY(cudaMemsetAsync(zero_local, 0, N * sizeof(int32_t), s));
    k_pair_fill<<<nblk(N), TB, 0, s>>>(v, zero_local, pmeta, scratch);
    PF_CUDA_TRY(cudaGetLastError());
    if (NP > 0) {
      k_slot_coeff<<<nblk(NP), TB, 0, s>>>(v, NP, pmeta, v.inc_gb, v.inc_ac, pgb, pac, nullptr);
      k_slot_fix<<<nblk(NP), TB, 0, s>>>(NP, pmeta, pgb, v.coef_scale, pgbx);
      PF_CUDA_TRY(cudaGetLastError());
    }
    PF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  v.pair_meta = pmeta;
  v.pair_gb = pgb;
  v.pair_ac = pac;
  v.pair_gbx = pgbx;
  return use_tile_set(c, 0, s);
}

int permute_overrides(Ctx &c, cudaStream_t s) {
  if (c.n_slots > 0) {
    k_slot_coeff<<<nblk(c.n_slots), TB, 0, s>>>(c.v, c.n_slots, c.v.slot_meta, c.ov_gb, c.ov_ac, c.ov_slot_gb,
                                                c.ov_slot_ac, c.ov_slot_gbm);
    k_slot_fix<<<nblk(c.n_slots), TB, 0, s>>>(c.n_slots, c.v.slot_meta, c.ov_slot_gb, c.v.coef_scale,
                                              c.ov_slot_gbx);
    PF_CUDA_TRY(cudaGetLastError());
  }
  k_rbus_fill<<<nblk(32 * c.n_rounds), TB, 0, s>>>(c.v, 32 * c.n_rounds, c.v.rbus, c.ov_hat, nullptr, nullptr,
                                                   c.ov_rbus_hat, nullptr);
  if (c.n_pairs > 0) {
    k_slot_coeff<<<nblk(c.n_pairs), TB, 0, s>>>(c.v, c.n_pairs, c.v.pair_meta, c.ov_gb, c.ov_ac, c.ov_pair_gb,
                                                c.ov_pair_ac, nullptr);
    k_slot_fix<<<nblk(c.n_pairs), TB, 0, s>>>(c.n_pairs, c.v.pair_meta, c.ov_pair_gb, c.v.coef_scale,
                                              c.ov_pair_gbx);
  }
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

// --------------------------------------------------------------------------
// the build
// --------------------------------------------------------------------------

int build_context(Ctx &c, const pf_system *grids, int n_grids, const pf_instance *inst, int n_inst,
                  int formulation, cudaStream_t s) {
  const BuildAllocScope fault_scope;
  if (formulation != PF_REDUCED && formulation != PF_EXTENDED)
    return fail(PF_ERR_INVALID, "formulation must be PF_REDUCED or PF_EXTENDED");
  if (n_grids <= 0 || !grids) return fail(PF_ERR_INVALID, "no grids");
  if (n_inst <= 0 || !inst) return fail(PF_ERR_INVALID, "no instances");
  const bool ext = formulation == PF_EXTENDED;
  View &v = c.v;
  v.formulation = formulation;
  v.n_grids = n_grids;
  v.n_inst = n_inst;

  // ---- host: validate, concatenate, sizes ----
  std::vector<int> npv_distinct(n_grids);
  int64_t N = 0, M = 0, NL = 0, NPV = 0, NSH = 0, NGEN = 0;
  for (int g = 0; g < n_grids; ++g) {
    PF_TRY(validate(grids[g], g, formulation, &npv_distinct[g]));
    N += grids[g].n_bus;
    M += grids[g].n_branch;
    NL += grids[g].n_load;
    NPV += grids[g].n_pv;
    NSH += grids[g].n_shunt;
    NGEN += ext ? grids[g].n_pv + 1 : 0;
  }
  if (N >= 0x7fffffffLL - 1 || 2 * M >= 0x7fffffffLL - 1 || NSH + 2 * M >= 0x7fffffffLL)
    return fail(PF_ERR_UNSUPPORTED, "more buses or branch ends than int32 indices allow");
  for (int i = 0; i < n_inst; ++i) {
    if (inst[i].grid < 0 || inst[i].grid >= n_grids)
      return fail(PF_ERR_INVALID, "instance " + std::to_string(i) + ": grid index out of range");
    if (inst[i].outage < -1 || inst[i].outage >= grids[inst[i].grid].n_branch)
      return fail(PF_ERR_INVALID, "instance " + std::to_string(i) + ": outage branch out of range");
  }
  v.n_bus = N;
  v.n_branch = M;
  v.n_inc = 2 * M;

  std::vector<int32_t> h_from(M), h_to(M), h_bus_grid(N);
  std::vector<double> h_r(M), h_x(M), h_b(M), h_tap(M), h_shift(M), h_gfr(M), h_gto(M);
  std::vector<uint8_t> h_status(M);
  std::vector<int32_t> h_load_bus(NL), h_pv_bus(NPV), h_pv_grid(NPV), h_sh_bus(NSH);
  std::vector<double> h_load_p(NL), h_load_q(NL), h_pv_p(NPV), h_sh_g(NSH), h_sh_b(NSH), h_vset(NGEN);
  std::vector<int64_t> h_grid_bus_off(n_grids + 1), h_grid_br_off(n_grids + 1), h_grid_pv_off(n_grids + 1),
      h_grid_gen_off(n_grids + 1), h_slack_glob(n_grids), h_grid_sh_off(n_grids + 1);
  std::vector<int32_t> h_grid_nbus(n_grids), h_grid_slack(n_grids), h_grid_ngen(n_grids), h_grid_nbr(n_grids);
  std::vector<double> h_theta_set(n_grids);
  c.grid_nf.resize(n_grids);
  c.grid_nx.resize(n_grids);
  c.grid_nshunt.resize(n_grids);
  {
    int64_t bo = 0, mo = 0, lo = 0, po = 0, so = 0, go = 0;
    for (int g = 0; g < n_grids; ++g) {
      const pf_system &G = grids[g];
      h_grid_bus_off[g] = bo;
      h_grid_br_off[g] = mo;
      h_grid_pv_off[g] = po;
      h_grid_gen_off[g] = go;
      h_grid_sh_off[g] = so;
      h_grid_nbus[g] = G.n_bus;
      h_grid_nbr[g] = G.n_branch;
      h_grid_slack[g] = G.slack_bus;
      h_slack_glob[g] = bo + G.slack_bus;
      h_theta_set[g] = G.slack_theta;
      h_grid_ngen[g] = ext ? G.n_pv + 1 : 0;
      c.grid_nshunt[g] = G.n_shunt;
      for (int64_t b = 0; b < G.n_bus; ++b) h_bus_grid[bo + b] = g;
      for (int64_t k = 0; k < G.n_branch; ++k) {
        h_from[mo + k] = (int32_t)(bo + G.br_from[k]);
        h_to[mo + k] = (int32_t)(bo + G.br_to[k]);
        h_r[mo + k] = G.br_r[k];
        h_x[mo + k] = G.br_x[k];
        h_b[mo + k] = G.br_b ? G.br_b[k] : 0.0;
        h_tap[mo + k] = G.br_tap ? G.br_tap[k] : 1.0;
        h_shift[mo + k] = G.br_shift ? G.br_shift[k] : 0.0;
        h_gfr[mo + k] = G.br_g_fr ? G.br_g_fr[k] : 0.0;
        h_gto[mo + k] = G.br_g_to ? G.br_g_to[k] : 0.0;
        h_status[mo + k] = G.br_status ? (G.br_status[k] ? 1 : 0) : 1;
      }
      for (int64_t k = 0; k < G.n_load; ++k) {
        h_load_bus[lo + k] = (int32_t)(bo + G.load_bus[k]);
        h_load_p[lo + k] = G.load_p[k];
        h_load_q[lo + k] = G.load_q[k];
      }
      for (int64_t k = 0; k < G.n_pv; ++k) {
        h_pv_bus[po + k] = (int32_t)(bo + G.pv_bus[k]);
        h_pv_grid[po + k] = g;
        h_pv_p[po + k] = G.pv_p[k];
        if (ext) h_vset[go + k] = G.pv_vset[k];
      }
      if (ext) h_vset[go + G.n_pv] = G.slack_vset;
      for (int64_t k = 0; k < G.n_shunt; ++k) {
        h_sh_bus[so + k] = (int32_t)(bo + G.sh_bus[k]);
        h_sh_g[so + k] = G.sh_g[k];
        h_sh_b[so + k] = G.sh_b[k];
      }
      const int64_t n = G.n_bus;
      c.grid_nf[g] = (int32_t)(ext ? 2 * n + G.n_pv + 2 : (n - 1) + (n - 1 - npv_distinct[g]));
      c.grid_nx[g] = (int32_t)(ext ? 2 * n + G.n_pv + 2 : 2 * n);
      bo += n;
      mo += G.n_branch;
      lo += G.n_load;
      po += G.n_pv;
      so += G.n_shunt;
      go += ext ? G.n_pv + 1 : 0;
    }
    h_grid_bus_off[n_grids] = bo;
    h_grid_br_off[n_grids] = mo;
    h_grid_pv_off[n_grids] = po;
    h_grid_gen_off[n_grids] = go;
    h_grid_sh_off[n_grids] = so;
  }
  c.grid_bus_off = h_grid_bus_off;
  c.grid_br_off = h_grid_br_off;
  c.grid_sh_off = h_grid_sh_off;

  // ---- upload ----
  int32_t *d_from, *d_to, *d_bus_grid, *d_load_bus, *d_pv_bus, *d_pv_grid, *d_sh_bus;
  double *d_r, *d_x, *d_b, *d_tap, *d_shift, *d_gfr, *d_gto, *d_vset;
  uint8_t *d_status;
  int64_t *d_grid_bus_off, *d_grid_br_off, *d_grid_gen_off;
  int32_t *d_grid_nbus, *d_grid_slack, *d_grid_ngen;
  double *d_theta_set;
  PF_TRY(upload(c, &d_from, h_from, s));
  PF_TRY(upload(c, &d_to, h_to, s));
  PF_TRY(upload(c, &d_r, h_r, s));
  PF_TRY(upload(c, &d_x, h_x, s));
  PF_TRY(upload(c, &d_b, h_b, s));
  PF_TRY(upload(c, &d_tap, h_tap, s));
  PF_TRY(upload(c, &d_shift, h_shift, s));
  PF_TRY(upload(c, &d_gfr, h_gfr, s));
  PF_TRY(upload(c, &d_gto, h_gto, s));
  PF_TRY(upload(c, &d_status, h_status, s));
  PF_TRY(upload(c, &d_bus_grid, h_bus_grid, s));
  PF_TRY(upload(c, &d_grid_bus_off, h_grid_bus_off, s));
  PF_TRY(upload(c, &d_grid_br_off, h_grid_br_off, s));
  PF_TRY(upload(c, &d_grid_gen_off, h_grid_gen_off, s));
  PF_TRY(upload(c, &d_grid_nbus, h_grid_nbus, s));
  PF_TRY(upload(c, &d_grid_slack, h_grid_slack, s));
  PF_TRY(upload(c, &d_grid_ngen, h_grid_ngen, s));
  PF_TRY(upload(c, &d_theta_set, h_theta_set, s));
  PF_TRY(upload(c, &d_vset, h_vset, s));
  TempList tmp;
  int64_t *d_slack_glob, *d_grid_pv_off, *d_grid_sh_off;
  {
    auto up_tmp = [&](auto **p, const auto &h) -> int {
      PF_TRY(tmp.alloc(p, h.size()));
      if (!h.empty())
        PF_CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, s));
      return PF_OK;
    };
    PF_TRY(up_tmp(&d_load_bus, h_load_bus));
    PF_TRY(up_tmp(&d_pv_bus, h_pv_bus));
    PF_TRY(up_tmp(&d_pv_grid, h_pv_grid));
    PF_TRY(up_tmp(&d_sh_bus, h_sh_bus));
    PF_TRY(up_tmp(&d_slack_glob, h_slack_glob));
    PF_TRY(up_tmp(&d_grid_pv_off, h_grid_pv_off));
    PF_TRY(up_tmp(&d_grid_sh_off, h_grid_sh_off));
    double *d_load_p, *d_load_q, *d_pv_p, *d_sh_g, *d_sh_b;
    PF_TRY(up_tmp(&d_load_p, h_load_p));
    PF_TRY(up_tmp(&d_load_q, h_load_q));
    PF_TRY(up_tmp(&d_pv_p, h_pv_p));
    PF_TRY(up_tmp(&d_sh_g, h_sh_g));
    PF_TRY(up_tmp(&d_sh_b, h_sh_b));

    v.br_from = d_from; v.br_to = d_to; v.br_r = d_r; v.br_x = d_x; v.br_b = d_b; v.br_tap = d_tap;
    v.br_shift = d_shift; v.br_gfr = d_gfr; v.br_gto = d_gto; v.br_status = d_status;
    v.bus_grid = d_bus_grid;
    v.grid_bus_off = d_grid_bus_off; v.grid_br_off = d_grid_br_off; v.grid_gen_off = d_grid_gen_off;
    v.grid_nbus = d_grid_nbus; v.grid_slack = d_grid_slack; v.grid_ngen = d_grid_ngen;
    v.grid_theta_set = d_theta_set; v.gen_vset = d_vset;

    // ---- injections and shunt totals per bus (sums in item order) ----
    double *g_sh, *b_sh, *p_inj, *q_inj, *pl, *ql, *pg;
    PF_TRY(tmp.alloc(&g_sh, N));
    PF_TRY(tmp.alloc(&b_sh, N));
    PF_TRY(tmp.alloc(&p_inj, N));
    PF_TRY(tmp.alloc(&q_inj, N));
    PF_TRY(tmp.alloc(&pl, N));
    PF_TRY(tmp.alloc(&ql, N));
    PF_TRY(tmp.alloc(&pg, N));
    int64_t *sh_ptr;
    uint32_t *sh_order;
    PF_TRY(bus_sums(c, tmp, d_sh_bus, NSH, d_sh_g, d_sh_b, 1.0, 1.0, g_sh, b_sh, &sh_ptr, &sh_order, s));
    PF_TRY(bus_sums(c, tmp, d_load_bus, NL, d_load_p, d_load_q, 1.0, 1.0, pl, ql, nullptr, nullptr, s));
    PF_TRY(bus_sums(c, tmp, d_pv_bus, NPV, d_pv_p, nullptr, 1.0, 1.0, pg, nullptr, nullptr, nullptr, s));
    k_net_injection<<<nblk(N), TB, 0, s>>>(pg, pl, ql, N, p_inj, q_inj);
    PF_CUDA_TRY(cudaGetLastError());
    double2 *bus_sh, *bus_inj;
    PF_TRY(dev_alloc(c, &bus_sh, N));
    PF_TRY(dev_alloc(c, &bus_inj, N));
    k_pack2<<<nblk(N), TB, 0, s>>>(g_sh, b_sh, N, bus_sh);
    k_pack2<<<nblk(N), TB, 0, s>>>(p_inj, q_inj, N, bus_inj);
    PF_CUDA_TRY(cudaGetLastError());
    v.bus_sh = bus_sh; v.bus_inj = bus_inj;

    // ---- bus types and row maps ----
    int8_t *type;
    uint8_t *ns, *pq;
    int64_t *ex_ns, *ex_pq, *stmp;
    PF_TRY(tmp.alloc(&type, N));
    PF_TRY(tmp.alloc(&ns, N));
    PF_TRY(tmp.alloc(&pq, N));
    PF_TRY(tmp.alloc(&ex_ns, N + 1));
    PF_TRY(tmp.alloc(&ex_pq, N + 1));
    PF_TRY(tmp.alloc(&stmp, scan_tmp_elems(std::max<int64_t>(N, 2 * M) + 1)));
    PF_CUDA_TRY(cudaMemsetAsync(type, 0, N, s));
    k_bus_type<<<nblk(std::max<int64_t>(NPV, n_grids)), TB, 0, s>>>(type, d_pv_bus, NPV, d_slack_glob, n_grids);
    k_flags<<<nblk(N), TB, 0, s>>>(type, N, ns, pq);
    PF_TRY(exclusive_scan<uint8_t>(ns, ex_ns, N, stmp, s));
    PF_TRY(exclusive_scan<uint8_t>(pq, ex_pq, N, stmp, s));
    int32_t *row_p, *row_q, *gen, *gen_bus;
    PF_TRY(dev_alloc(c, &row_p, N));
    PF_TRY(dev_alloc(c, &row_q, N));
    PF_TRY(dev_alloc(c, &gen, N));
    PF_TRY(dev_alloc(c, &gen_bus, NGEN));
    k_row_maps<<<nblk(N), TB, 0, s>>>(v, type, ex_ns, ex_pq, row_p, row_q, gen);
    PF_CUDA_TRY(cudaGetLastError());
    if (ext) {
      k_gen_map<<<nblk(std::max<int64_t>(NPV, n_grids)), TB, 0, s>>>(v, d_pv_bus, d_pv_grid, d_grid_pv_off, NPV,
                                                                    gen, gen_bus);
      PF_CUDA_TRY(cudaGetLastError());
    }
    v.row_p = row_p; v.row_q = row_q; v.gen = gen; v.gen_bus = gen_bus;

    // ---- incidence list ----
    const int64_t NI = 2 * M;
    const int64_t np = sort_padded(NI);
    uint64_t *keys;
    uint32_t *vals;
    int32_t *pos_of, *deg, *inc_own, *inc_other, *inc_code, *inc_ptr, *mirror, *grp, *stats;
    int64_t *ptr64;
    PF_TRY(tmp.alloc(&keys, np));
    PF_TRY(tmp.alloc(&vals, np));
    PF_TRY(dev_alloc(c, &pos_of, NI));
    PF_TRY(tmp.alloc(&deg, N));
    PF_TRY(tmp.alloc(&ptr64, N + 1));
    PF_TRY(tmp.alloc(&stats, 4));
    PF_TRY(dev_alloc(c, &inc_own, NI));
    PF_TRY(dev_alloc(c, &inc_other, NI));
    PF_TRY(dev_alloc(c, &inc_code, NI));
    PF_TRY(dev_alloc(c, &inc_ptr, N + 1));
    PF_TRY(dev_alloc(c, &mirror, NI));
    PF_TRY(dev_alloc(c, &grp, NI));
    PF_CUDA_TRY(cudaMemsetAsync(deg, 0, N * sizeof(int32_t), s));
    PF_CUDA_TRY(cudaMemsetAsync(stats, 0, 4 * sizeof(int32_t), s));
    if (NI > 0) {
      k_make_keys<<<nblk(NI), TB, 0, s>>>(d_from, d_to, M, keys, vals);
      PF_TRY(bitonic_sort_pairs(keys, vals, NI, s));
      k_unpack<<<nblk(NI), TB, 0, s>>>(keys, vals, NI, inc_own, inc_other, inc_code, pos_of, deg);
      PF_CUDA_TRY(cudaGetLastError());
    }
    PF_TRY(exclusive_scan<int32_t>(deg, ptr64, N, stmp, s));
    k_i64_to_i32<<<nblk(N + 1), TB, 0, s>>>(ptr64, inc_ptr, N + 1);
    v.inc_own = inc_own; v.inc_other = inc_other; v.inc_code = inc_code; v.inc_ptr = inc_ptr;
    if (NI > 0) {
      k_mirror_groups<<<nblk(NI), TB, 0, s>>>(v, pos_of, mirror, grp, stats);
      PF_CUDA_TRY(cudaGetLastError());
    }
    v.inc_mirror = mirror; v.inc_grp = grp; v.inc_of_code = pos_of;
    {
      int32_t *npair;
      PF_TRY(dev_alloc(c, &npair, N));
      k_npair<<<nblk(N), TB, 0, s>>>(v, npair);
      PF_CUDA_TRY(cudaGetLastError());
      v.bus_npair = npair;
    }
    int rc = PF_OK;
    std::vector<int32_t> hstats = to_host(stats, 4, s, &rc);
    if (rc) return rc;
    c.max_group = hstats[0];
    c.max_degree = hstats[1];
    if (c.max_group > kMaxGroup)
      return fail(PF_ERR_UNSUPPORTED, "more than " + std::to_string(kMaxGroup) +
                                          " parallel branches between one pair of buses");

    // ---- row structure, rowptr, colind ----
    int64_t FT = 0;
    std::vector<int64_t> h_grid_f_off(n_grids + 1), h_grid_row_off(n_grids + 1);
    for (int g = 0; g < n_grids; ++g) {
      h_grid_f_off[g] = FT;
      h_grid_row_off[g] = FT + g;
      FT += c.grid_nf[g];
    }
    h_grid_f_off[n_grids] = FT;
    h_grid_row_off[n_grids] = FT + n_grids;
    c.grid_row_off = h_grid_row_off;
    int64_t *d_grid_f_off, *d_grid_row_off;
    PF_TRY(up_tmp(&d_grid_f_off, h_grid_f_off));
    PF_TRY(upload(c, &d_grid_row_off, h_grid_row_off, s));
    int2 *inc_rt, *diag;
    int32_t *len_tv, *rowlen, *rowptr, *nnz_g, *err;
    int64_t *S, *stmp2;
    PF_TRY(dev_alloc(c, &inc_rt, NI));
    PF_TRY(dev_alloc(c, &diag, N));
    PF_TRY(dev_alloc(c, &len_tv, N));
    PF_TRY(tmp.alloc(&rowlen, FT));
    PF_TRY(tmp.alloc(&S, FT + 1));
    PF_TRY(tmp.alloc(&stmp2, scan_tmp_elems(FT) + 1));
    PF_TRY(dev_alloc(c, &rowptr, FT + n_grids));
    PF_TRY(tmp.alloc(&nnz_g, n_grids));
    PF_TRY(dev_alloc(c, &err, 1));
    PF_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    v.dev_error = err;
    k_row_struct<<<nblk(N), TB, 0, s>>>(v, d_grid_f_off, inc_rt, diag, len_tv, rowlen);
    if (ext) k_gen_rowlen<<<nblk(std::max<int64_t>(NGEN, n_grids)), TB, 0, s>>>(v, d_grid_f_off, rowlen, NGEN);
    PF_CUDA_TRY(cudaGetLastError());
    PF_TRY(exclusive_scan<int32_t>(rowlen, S, FT, stmp2, s));
    k_rowptr<<<nblk(FT + n_grids), TB, 0, s>>>(S, d_grid_f_off, d_grid_row_off, n_grids, FT + n_grids, rowptr,
                                               nnz_g, err);
    PF_CUDA_TRY(cudaGetLastError());
    v.inc_rt = inc_rt; v.diag = diag; v.len_tv = len_tv;
    c.rowptr = rowptr;
    c.grid_nnz = to_host(nnz_g, n_grids, s, &rc);
    if (rc) return rc;
    {
      std::vector<int32_t> herr = to_host(err, 1, s, &rc);
      if (rc) return rc;
      if (herr[0]) return fail(PF_ERR_UNSUPPORTED, "a grid has more than 2^31 Jacobian nonzeros");
    }
    c.grid_nnz_off.assign(n_grids + 1, 0);
    for (int g = 0; g < n_grids; ++g) c.grid_nnz_off[g + 1] = c.grid_nnz_off[g] + c.grid_nnz[g];
    const int64_t NNZ = c.grid_nnz_off[n_grids];
    int64_t *d_grid_nnz_off;
    PF_TRY(upload(c, &d_grid_nnz_off, c.grid_nnz_off, s));
    int32_t *base_p, *base_q, *colind, *gen_pos, *pos_gth, *row_gth;
    PF_TRY(dev_alloc(c, &base_p, N));
    PF_TRY(dev_alloc(c, &base_q, N));
    PF_TRY(dev_alloc(c, &colind, NNZ));
    PF_TRY(dev_alloc(c, &gen_pos, NGEN));
    PF_TRY(dev_alloc(c, &pos_gth, n_grids));
    PF_TRY(dev_alloc(c, &row_gth, n_grids));
    PF_CUDA_TRY(cudaMemsetAsync(pos_gth, 0xff, n_grids * sizeof(int32_t), s));
    PF_CUDA_TRY(cudaMemsetAsync(row_gth, 0xff, n_grids * sizeof(int32_t), s));
    k_colind<<<nblk(N), TB, 0, s>>>(v, rowptr, d_grid_row_off, d_grid_nnz_off, base_p, base_q, colind);
    if (ext)
      k_gen_cols<<<nblk(std::max<int64_t>(NGEN, n_grids)), TB, 0, s>>>(v, rowptr, d_grid_row_off, d_grid_nnz_off,
                                                                      colind, gen_pos, pos_gth, row_gth, NGEN);
    PF_CUDA_TRY(cudaGetLastError());
    v.base_p = base_p; v.base_q = base_q; v.gen_pos = gen_pos;
    v.grid_pos_gth = pos_gth; v.grid_row_gth = row_gth;
    c.colind = colind;

    // ---- coefficients ----
    double2 *gb, *ac, *hat;
    PF_TRY(dev_alloc(c, &gb, NI));
    PF_TRY(dev_alloc(c, &ac, NI));
    PF_TRY(dev_alloc(c, &hat, N));
    PF_TRY(compute_coefficients(c, nullptr, nullptr, nullptr, nullptr, gb, ac, hat, s));
    v.inc_gb = gb; v.inc_ac = ac; v.bus_hat = hat;
    PF_TRY(dev_alloc(c, &c.ov_gb, NI));
    PF_TRY(dev_alloc(c, &c.ov_ac, NI));
    PF_TRY(dev_alloc(c, &c.ov_hat, N));

    // ---- packed records for the evaluation kernels ----
    int4 *bus_meta, *bus_meta2, *inc_meta, *inc_pos;
    PF_TRY(dev_alloc(c, &bus_meta, N));
    PF_TRY(dev_alloc(c, &bus_meta2, N));
    PF_TRY(dev_alloc(c, &inc_meta, NI));
    PF_TRY(dev_alloc(c, &inc_pos, NI));
    k_pack_bus<<<nblk(N), TB, 0, s>>>(v, base_p, base_q, diag, len_tv, bus_meta, bus_meta2);
    if (NI > 0) k_pack_inc<<<nblk(NI), TB, 0, s>>>(v, inc_rt, base_p, base_q, inc_meta, inc_pos);
    PF_CUDA_TRY(cudaGetLastError());
    v.bus_meta = bus_meta; v.bus_meta2 = bus_meta2; v.inc_meta = inc_meta; v.inc_pos = inc_pos;

    // ---- contribution list ----
    int32_t *count;
    int64_t *S2, *stmp3, *src_len;
    PF_TRY(tmp.alloc(&count, NNZ));
    PF_TRY(tmp.alloc(&S2, NNZ + 1));
    PF_TRY(tmp.alloc(&stmp3, scan_tmp_elems(NNZ) + 1));
    PF_TRY(tmp.alloc(&src_len, n_grids));
    std::vector<int64_t> h_grid_inc_off(n_grids + 1);
    for (int g = 0; g <= n_grids; ++g) h_grid_inc_off[g] = 2 * h_grid_br_off[g];
    int64_t *d_grid_inc_off;
    int32_t *d_grid_nbr;
    PF_TRY(up_tmp(&d_grid_inc_off, h_grid_inc_off));
    PF_TRY(up_tmp(&d_grid_nbr, h_grid_nbr));
    c.grid_cptr_off.assign(n_grids + 1, 0);
    for (int g = 0; g < n_grids; ++g) c.grid_cptr_off[g + 1] = c.grid_cptr_off[g] + c.grid_nnz[g] + 1;
    int64_t *d_grid_cptr_off;
    PF_TRY(up_tmp(&d_grid_cptr_off, c.grid_cptr_off));
    k_contrib<<<nblk(N), TB, 0, s>>>(v, 0, d_grid_nnz_off, d_grid_cptr_off, nullptr, sh_ptr, sh_order,
                                     d_grid_sh_off, d_grid_inc_off, d_grid_nbr, count, nullptr, nullptr);
    if (ext)
      k_contrib_const<<<nblk(std::max<int64_t>(NGEN, n_grids)), TB, 0, s>>>(
          v, 0, d_grid_nnz_off, d_grid_cptr_off, nullptr, gen_pos, pos_gth, NGEN, count, nullptr, nullptr);
    PF_CUDA_TRY(cudaGetLastError());
    PF_TRY(exclusive_scan<int32_t>(count, S2, NNZ, stmp3, s));
    int64_t *cptr;
    const int64_t CPT = c.grid_cptr_off[n_grids];
    PF_TRY(dev_alloc(c, &cptr, CPT));
    k_cptr<<<nblk(CPT), TB, 0, s>>>(S2, d_grid_nnz_off, d_grid_cptr_off, n_grids, CPT, cptr, src_len);
    PF_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> h_src_len = to_host(src_len, n_grids, s, &rc);
    if (rc) return rc;
    c.grid_csrc_off.assign(n_grids + 1, 0);
    for (int g = 0; g < n_grids; ++g) c.grid_csrc_off[g + 1] = c.grid_csrc_off[g] + h_src_len[g];
    int64_t *d_grid_csrc_off;
    PF_TRY(up_tmp(&d_grid_csrc_off, c.grid_csrc_off));
    int32_t *src;
    PF_TRY(dev_alloc(c, &src, c.grid_csrc_off[n_grids]));
    k_contrib<<<nblk(N), TB, 0, s>>>(v, 1, d_grid_nnz_off, d_grid_cptr_off, d_grid_csrc_off, sh_ptr, sh_order,
                                     d_grid_sh_off, d_grid_inc_off, d_grid_nbr, nullptr, cptr, src);
    if (ext)
      k_contrib_const<<<nblk(std::max<int64_t>(NGEN, n_grids)), TB, 0, s>>>(
          v, 1, d_grid_nnz_off, d_grid_cptr_off, d_grid_csrc_off, gen_pos, pos_gth, NGEN, nullptr, cptr, src);
    PF_CUDA_TRY(cudaGetLastError());
    c.contrib_ptr = cptr;
    c.contrib_src = src;
  }

  // ---- instances ----
  c.inst_grid.resize(n_inst);
  c.inst_outage.resize(n_inst);
  c.x_off.assign(n_inst + 1, 0);
  c.f_off.assign(n_inst + 1, 0);
  c.v_off.assign(n_inst + 1, 0);
  c.bus_off.assign(n_inst + 1, 0);
  c.br_off.assign(n_inst + 1, 0);
  c.gen_off.assign(n_inst + 1, 0);
  c.any_outage = false;
  for (int i = 0; i < n_inst; ++i) {
    const int g = inst[i].grid;
    c.inst_grid[i] = g;
    c.inst_outage[i] = inst[i].outage >= 0 ? (int32_t)(h_grid_br_off[g] + inst[i].outage) : -1;
    c.any_outage |= inst[i].outage >= 0;
    c.x_off[i + 1] = c.x_off[i] + c.grid_nx[g];
    c.f_off[i + 1] = c.f_off[i] + c.grid_nf[g];
    c.v_off[i + 1] = c.v_off[i] + c.grid_nnz[g];
    c.bus_off[i + 1] = c.bus_off[i] + h_grid_nbus[g];
    c.br_off[i + 1] = c.br_off[i] + h_grid_nbr[g];
    c.gen_off[i + 1] = c.gen_off[i] + h_grid_ngen[g];
  }
  c.n_gen_inst = c.gen_off[n_inst];
  v.grid1_nx = n_grids == 1 ? c.grid_nx[0] : 0;
  v.grid1_nbus = n_grids == 1 ? h_grid_nbus[0] : 0;
  c.n_x = c.x_off[n_inst];
  c.n_f = c.f_off[n_inst];
  c.nnz = c.v_off[n_inst];
  v.n_bus_inst = c.bus_off[n_inst];
  c.n_branch_inst = c.br_off[n_inst];
  int32_t *d_inst_grid, *d_inst_outage;
  int64_t *d_x_off, *d_f_off, *d_v_off, *d_bus_off, *d_br_off, *d_gen_off;
  PF_TRY(upload(c, &d_inst_grid, c.inst_grid, s));
  PF_TRY(upload(c, &d_inst_outage, c.inst_outage, s));
  PF_TRY(upload(c, &d_x_off, c.x_off, s));
  PF_TRY(upload(c, &d_f_off, c.f_off, s));
  PF_TRY(upload(c, &d_v_off, c.v_off, s));
  PF_TRY(upload(c, &d_bus_off, c.bus_off, s));
  PF_TRY(upload(c, &d_br_off, c.br_off, s));
  PF_TRY(upload(c, &d_gen_off, c.gen_off, s));
  v.inst_grid = d_inst_grid; v.inst_outage = d_inst_outage;
  v.inst_x_off = d_x_off; v.inst_f_off = d_f_off; v.inst_v_off = d_v_off;
  v.inst_bus_off = d_bus_off; v.inst_br_off = d_br_off; v.inst_gen_off = d_gen_off;
  PF_TRY(dev_alloc(c, &v.phasor, 2 * v.n_bus_inst));

  int dev = 0;
  PF_CUDA_TRY(cudaGetDevice(&dev));
  c.device = dev;
  PF_CUDA_TRY(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev));

  // (cos, sin) of i pi / 16384 for the table-driven phasor routine, evaluated in
  // long double on the host and rounded once to 2^-62.
  {
    std::vector<longlong2> tabf(kSinCosTable);
    const long double pi = 3.14159265358979323846264338327950288419716939937510L;
    const long double two62 = 4611686018427387904.0L;
    for (int i = 0; i < kSinCosTable; ++i) {
      const long double a = pi * (long double)i / (long double)(kSinCosTable / 2);
      tabf[i] = make_longlong2(llroundl(cosl(a) * two62), llroundl(sinl(a) * two62));
    }
    longlong2 *d_tabf;
    PF_TRY(upload(c, &d_tabf, tabf, s));
    v.sincos_fix = d_tabf;
  }
  {
    const int64_t M = v.n_branch;
    double2 *kgb, *kab, *ktc, *kph;
    PF_TRY(dev_alloc(c, &kgb, M));
    PF_TRY(dev_alloc(c, &kab, M));
    PF_TRY(dev_alloc(c, &ktc, M));
    PF_TRY(dev_alloc(c, &kph, M));
    if (M > 0) {
      k_branch_consts<<<nblk(M), TB, 0, s>>>(v, kgb, kab, ktc, kph);
      PF_CUDA_TRY(cudaGetLastError());
    }
    v.br_k_gb = kgb; v.br_k_ab = kab; v.br_k_tc = ktc; v.br_k_ph = kph;
  }
  PF_TRY(build_rounds(c, s));
  PF_TRY(build_tiles(c, s));
  PF_CUDA_TRY(cudaStreamSynchronize(s));
  return PF_OK;
}

}  // namespace pf
