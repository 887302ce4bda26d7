// Evaluation kernels: tasks (1) and (2) of Newton power flow (Sec. I) for
// every instance of a context.
//
// Arithmetic form.  For a branch end at bus o whose other end is bus k, with
// per-end coefficients (G, B, A, C) built once from the branch model (see
// k_coeff in pf_build.cu), the terminal powers of Eq. (4) extended with Q,
// tap and shift are, with the bus voltages in rectangular form
// E = V (cos t, sin t) = (e, f),
//     P_o =  A V_o^2 - X,   Q_o = -C V_o^2 - Y,
//     X = e_o u + f_o w,    Y = f_o u - e_o w,
//     u = G e_k - B f_k,    w = G f_k + B e_k,
// which is the polar form with the angle difference expanded (X = V_o V_k
// times the rotated cosine term), so that the only trigonometry is one
// sin/cos pair per bus (k_phasor).  The partials follow from the same
// expansion:
//     dP_o/dt_k = -Y,  dQ_o/dt_k = X,  dP_o/dV_k = -X / V_k,  dQ_o/dV_k = -Y / V_k,
// and, with S_X = sum X and S_Y = sum Y over the ends of bus o,
//     F_P = V_o^2 A^ - S_X - P_inj,    F_Q = -(V_o^2 C^ + S_Y) - Q_inj,
//     dF_P/dt_o = S_Y,   dF_Q/dt_o = -S_X,
//     dF_P/dV_o = (2 V_o^2 A^ - S_X) / V_o,   dF_Q/dV_o = -(2 V_o^2 C^ + S_Y) / V_o,
// where A^ = sum A + shunt g and C^ = sum C + shunt b.  1/V is formed once
// per bus by k_phasor_fx.  GB300 issues FP64 arithmetic at 2 operations per
// clock per SM, so the pair terms are formed in fixed point on the integer
// pipe instead (see "Fixed-point arithmetic of the pair terms" below): the
// unit phasors (cos t, sin t), V and the merged coefficients (G, B) of a pair
// of connected buses (parallel branches merged) as 30-bit limbs, products from
// 32 x 32 -> 64-bit multiplies, the bus sums S_X, S_Y exact in 96 bits; each
// J value and each sum is rounded once to double, to nearest even, by the
// FP64 pipe's conversion (a bus whose sum does not fit in 64 bits takes the
// FP64 form below).  The per-bus rows (F, the diagonal
// values) stay in FP64: 8 operations per bus.  A bus whose inputs fall outside
// the fixed-point ranges is evaluated in FP64 from x (the form above).
//
// Work decomposition (k_tile).  The buses of each grid are cut, in bus order,
// into tiles of up to 32 consecutive buses with at most kTilePairs pairs of
// connected buses, so that a tile's rows of J and of F are contiguous ranges.
// One warp evaluates one tile of one instance: the lanes share the tile's
// pairs evenly (pair p on lane p mod 32), each pair's four off-diagonal J
// entries go to the tile's rows staged in shared memory and its terms X, Y to
// shared memory; then lane l sums the terms of bus l exactly and writes the
// bus's diagonal entries and F rows to the staging, and the warp writes the
// staged rows out whole, every store of the warp to consecutive addresses.  A
// bus with more than 32 neighbours is evaluated by a whole warp in a second
// kernel.  The launch has one one-warp CTA per tile and instance, or
// (ctas_per_sm > 0) a persistent grid whose warps claim units from a counter.
//
// Determinism: every operation is an explicitly rounded intrinsic or exact
// integer arithmetic, the bus sums of a bus with up to 32 neighbours are exact
// (so independent of the order of the terms), and every other sum runs in a
// fixed order -- a group's
// coefficients in incidence-list order, the FP64 fallback of the bus sums in
// list order, lane-strided partial sums over the ends combined by a fixed
// butterfly for a larger bus -- so results are bit-identical run to run,
// across code paths and for every tuning.
#include <algorithm>

#include "pf_internal.cuh"

namespace pf {

namespace {

// -x, by flipping the sign bit on the integer pipe (exact, no FP64 issue).
__device__ __forceinline__ double neg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// ---------------------------------------------------------------------------
// Per-bus voltage records, split between the integer and the FP64 pipes.
// GB300 issues FP64 arithmetic at 2 operations per clock per SM and 64-bit
// integer work many times faster, on separate pipes; the trigonometric
// routine runs in 64-bit fixed point, the products with V and the
// reciprocal 1/V on the FP64 pipe.
//
// (cos t, sin t) for |t| < 32, by table-driven argument reduction (after
// P. T. P. Tang's table-driven elementary functions):
//   |t| = U 2^-57 (exact for |t| >= 2^-5, truncated at 2^-57 below);
//   y = |t| 16384/pi from the 128-bit product U * round(2^65/pi), k = nearest
//   integer to y, r = (y - k) pi/16384 from (y - k) 2^64 * round(pi 2^61),
//   so |r| <= pi/32768 with an error below 2^-58;
//   h = 1 - cos r = r^2/2 and sin r = r - r^3/6 in fixed point (the first
//   omitted terms, r^4/24 and r^5/120, are below 3.6e-18 and 7e-23; r^3/6,
//   C_k h and S_k h from 32-bit factors, to 2^-57);
//   cos t = C_k - (C_k h + S_k sin r),  sin t = S_k + (C_k sin r - S_k h)
//   with the table (C_k, S_k) = (cos, sin)(k pi/16384) as 2^62-scaled
//   integers (32768 entries, from long double on the host); the sums are
//   formed in 2^-62 fixed point and rounded once to double.
// Then E = V (cos t, sin t) by two FP64 multiplies, and 1/V by the hardware's
// approximate reciprocal r0 and one Householder step of order 2: with
// e = 1 - V r0, 1/V = r0 (1 + e + e^2 + ...), so r1 = r0 + r0 (e + e^2) has
// relative error e^3 (3 FP64 operations).  Arguments |t| >= 32, and V
// non-finite or of magnitude >= 2^977, use sincos() and FP64 arithmetic.
// ---------------------------------------------------------------------------
constexpr unsigned long long kInvStepFix = 0xa2f9836e4e44152aULL;   // round(2^65 / pi)
constexpr long long kStepFix = 0x6487ed5110b4611aLL;                // round(pi 2^61)
constexpr int kSixth32 = 0x2aaaaaab;                                 // round(2^32 / 6)

// z 2^-62 as a double, rounded to nearest (ties away from zero).
__device__ __forceinline__ double fix62_to_double(long long z) {
  if (z == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)z & 0x8000000000000000ULL;
  const unsigned long long a = sign ? 0ULL - (unsigned long long)z : (unsigned long long)z;
  const int lz = __clzll((long long)a);
  const unsigned long long n = a << lz;                                              // top bit 63
  const unsigned long long mag =
      ((unsigned long long)(1024 - lz) << 52) + ((n >> 11) & 0xfffffffffffffULL) + ((n >> 10) & 1ULL);
  return __longlong_as_double((long long)(sign | mag));
}

// 1/s for a finite normal s with 2^-600 <= |s| < 2^977 (see above).
__device__ __forceinline__ double recip(double s) {
  double r0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(s));
  const double e = __fma_rn(-s, r0, 1.0);
  return __fma_rn(r0, __fma_rn(e, e, e), r0);
}

// (V cos t, V sin t) and 1/V of a per-bus record; sv is V after the dead-bus
// substitution.
struct RectV {
  double2 E;
  double rv;
};

// (cos t, sin |t|) 2^62 for |t| < 32 by the table-driven routine above (the
// fixed-point values before any rounding to double; the caller applies the
// sign of t to the sine).
__device__ __forceinline__ longlong2 unit_fix_small(double t, const longlong2 *__restrict__ tabf) {
  const unsigned long long tb = (unsigned long long)__double_as_longlong(t);
  const int et = (int)((tb >> 52) & 0x7ff);
  const unsigned long long mt = (tb & 0xfffffffffffffULL) | (et ? (1ULL << 52) : 0ULL);
  const int sh = et - 1018;                                   // |t| 2^57 = mt 2^(et - 1018)
  const unsigned long long U = sh >= 0 ? mt << sh : (sh > -64 ? mt >> -sh : 0ULL);
  // y 2^108 = U * kInvStepFix; k = round(y), f = y - k
  const unsigned long long wh = __umul64hi(U, kInvStepFix), wl = U * kInvStepFix;
  const unsigned long long tr = wh + (1ULL << 43);
  const unsigned k = (unsigned)(tr >> 44);
  const long long fk = (long long)(tr & ((1ULL << 44) - 1)) - (1LL << 43);          // f 2^44
  const long long F = (long long)(((unsigned long long)fk << 20) | (wl >> 44));      // f 2^64
  const long long R = __mul64hi(F, kStepFix);                                        // r 2^75
  const long long R2 = __mul64hi(R, R);                                              // r^2 2^86
  // r^3/6 (< 2^-42.6) needs only 32-bit factors: r 2^43 and r^2 2^54
  const int r3 = __mulhi(__mulhi((int)(R2 >> 32), (int)(R >> 32)), kSixth32);       // r^3/6 2^65
  const long long SR = R - ((long long)r3 << 10);                                    // sin r 2^75
  const long long H = R2 >> 12;                                                      // r^2/2 2^75
  const int idx = (int)(k & (kSinCosTable - 1));
  const longlong2 Tf = __ldg(tabf + idx);                                            // (C, S) 2^62
  // h < 2^-27.7: C h and S h from 32-bit factors (C 2^30, h 2^58) to 2^-57
  const int h32 = (int)(H >> 17), c32 = (int)(Tf.x >> 32), s32 = (int)(Tf.y >> 32);
  const long long dc = -(((long long)c32 * h32) >> 15) - __mul64hi(Tf.y, SR);          // 2^73
  const long long ds = __mul64hi(Tf.x, SR) - (((long long)s32 * h32) >> 15);
  return make_longlong2(Tf.x + (dc >> 11), Tf.y + (ds >> 11));                      // (cos t, sin |t|)
}

// Arguments the fixed-point routine does not take: |t| >= 32 or t not finite
// (or a voltage too large for the routine's FP64 products).
__device__ __forceinline__ bool phasor_slow(double t, double sv) {
  return (__double2hiint(t) & 0x7fffffff) >= 0x40400000 || (__double2hiint(sv) & 0x7ff00000) >= 0x7d000000;
}

__device__ __forceinline__ RectV rect_voltage(double t, double sv, const longlong2 *__restrict__ tabf) {
  RectV o;
  if (phasor_slow(t, sv)) {
    double sn, cs;
    sincos(t, &sn, &cs);
    o.E = make_double2(__dmul_rn(sv, cs), __dmul_rn(sv, sn));
    o.rv = __drcp_rn(sv);
    return o;
  }
  const longlong2 u = unit_fix_small(t, tabf);
  const double ey = __dmul_rn(sv, fix62_to_double(u.y));
  o.E = make_double2(__dmul_rn(sv, fix62_to_double(u.x)), __double2hiint(t) < 0 ? neg(ey) : ey);   // sin is odd
  o.rv = recip(sv);
  return o;
}

// The voltage in rectangular form E = V (cos theta, sin theta), then V and
// 1/V.  A voltage below 2^-500 in magnitude (a dead bus) is replaced by
// 2^-600 in E and 1/V: every term then carries a factor of at most 2^-600
// where it should carry V (terms that are zero to far below any tolerance),
// and the dF/dV values, which divide that factor out again, stay exact.
constexpr double kDeadV = 0x1p-600;

__device__ __forceinline__ double dead_sub(double vm) {
  return (__double2hiint(vm) & 0x7ff00000) < 0x20b00000 ? kDeadV : vm;   // |V| < 2^-500
}

// The instance of instance-bus q: chunk_inst holds the instance of the first
// bus of every chunk of 2^kChunkLog2 instance-buses, so a thread searches only
// between its chunk's first instance and the next chunk's (no search at all
// when one instance spans the chunk, as it mostly does for grids larger than
// a chunk), and no thread waits for another.
__device__ __forceinline__ int bus_instance(const View &v, int64_t q) {
  if (v.n_inst <= 1) return 0;
  const int64_t c = q >> kChunkLog2;
  const int i0 = __ldg(v.chunk_inst + c), i1 = __ldg(v.chunk_inst + c + 1);
  return i0 == i1 ? i0 : i0 + find_segment(v.inst_bus_off + i0, i1 - i0 + 1, q);
}

// FP64 records for the adjoint kernels, one thread per instance-bus:
// (V cos theta, V sin theta) and (V, 1/V) side by side in 32 bytes, so that a
// gather of a neighbour's data hits one sector.
__global__ void __launch_bounds__(256) k_phasor(View v, const double *__restrict__ x) {
  // Let the dependent kernel start launching; it waits for this grid's results.
  cudaTriggerProgrammaticLaunchCompletion();
  const int64_t q = v.bus_inst_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < v.n_bus_inst) {
    const int inst = bus_instance(v, q);
    const int64_t lb = q - v.inst_bus_off[inst];
    const double *xi = x + v.inst_x_off[inst];
    const double th = __ldg(xi + lb);
    const double vm = __ldg(xi + v.grid_nbus[v.inst_grid[inst]] + lb);
    const RectV r = rect_voltage(th, dead_sub(vm), v.sincos_fix);
    v.phasor[2 * q] = r.E;
    v.phasor[2 * q + 1] = make_double2(vm, r.rv);
  }
}

// x 2^60 as a signed integer for |x| < 2 (exact for |x| >= 2^-8, truncated
// toward zero below), from the bits of x on the integer pipe.
__device__ __forceinline__ long long fix60_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffULL) | (e ? (1ULL << 52) : 0ULL);
  const int sh = e - 1015;                                    // x 2^60 = m 2^(e - 1015)
  const long long a = (long long)(sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ULL));
  return (long long)b < 0 ? -a : a;
}

// 30-bit limbs {h, l} of a fixed-point value below 2^61 in magnitude:
// value = h 2^30 + l with 0 <= l < 2^30.
__device__ __forceinline__ int2 limbs(long long z) { return make_int2((int)(z >> 30), (int)(z & 0x3fffffff)); }

// The fixed-point record of a bus for the F / J kernels, as two int4:
// {cos theta 2^60, sin theta 2^60} as 30-bit limbs, then {V 2^60} as limbs
// and 1/V (a double), 32 bytes.  The trigonometric routine runs on the
// integer pipe and its fixed-point result is kept (rounded from 2^62 to 2^60,
// no rounding to double); V 2^60 is exact for 2^-8 <= |V| < 2.  A voltage
// outside (-2, 2), or an angle that is not finite, gets kBadLimb in place of
// V's high limb: the buses that see it evaluate in FP64 from x.  1/V is
// formed (on the FP64 pipe, otherwise idle here) only for the buses the
// fixed-point form takes, V in [1/4, 2), and only where asked (want_rv: a
// tile's own buses need it, the neighbours' records it forms do not).
__device__ __forceinline__ void make_record(double th, double vm, const longlong2 *__restrict__ tabf, int4 &r0,
                                          int4 &r1, bool want_rv = true) {
  long long c60, s60;
  bool finite = true;
  if ((__double2hiint(th) & 0x7fffffff) < 0x40400000) {       // |t| < 32
    const longlong2 u = unit_fix_small(th, tabf);
    c60 = (u.x + 2) >> 2;
    s60 = (u.y + 2) >> 2;
    if (__double2hiint(th) < 0) s60 = -s60;                    // sin is odd
  } else {
    double sn, cs;
    sincos(th, &sn, &cs);
    c60 = __double2ll_rn(__dmul_rn(cs, 0x1p60));
    s60 = __double2ll_rn(__dmul_rn(sn, 0x1p60));
    finite = (__double2hiint(th) & 0x7ff00000) != 0x7ff00000;
  }
  int2 vl = limbs(fix60_of(vm));
  if (!finite || (__double2hiint(vm) & 0x7fffffff) >= 0x40000000) vl = make_int2(kBadLimb, 0);   // |V| >= 2, NaN
  const int2 cl = limbs(c60), sl = limbs(s60);
  r0 = make_int4(cl.x, cl.y, sl.x, sl.y);
  const double rv = (want_rv && vl.x >= (1 << 28)) ? recip(vm) : 0.0;
  r1 = make_int4(vl.x, vl.y, __double2loint(rv), __double2hiint(rv));
}

// The records of every instance-bus, one thread each (the F / J kernel then
// gathers its buses' and their neighbours' records; 1/V is formed here, off
// that kernel's dependence chain).  GRID1: every instance is of the one grid
// of the context, so instance blockIdx.y + i0 holds buses blockIdx.x * 256 +
// threadIdx.x at the same offsets (no instance lookup); otherwise a 1-D grid
// over the instance-buses and a lookup of each one's instance.
template <bool GRID1>
__global__ void __launch_bounds__(256) k_phasor_fx(View v, const double *__restrict__ x, int i0) {
  cudaTriggerProgrammaticLaunchCompletion();
  int inst;
  int64_t q, lb;
  int32_t nb;
  if (GRID1) {
    nb = v.grid1_nbus;
    inst = i0 + (int)blockIdx.y;
    lb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (lb >= nb) return;
    q = (int64_t)inst * nb + lb;
  } else {
    q = v.bus_inst_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= v.n_bus_inst) return;
    inst = bus_instance(v, q);
    lb = q - v.inst_bus_off[inst];
    nb = v.grid_nbus[v.inst_grid[inst]];
  }
  {
    const double *xi = x + (GRID1 ? (int64_t)inst * v.grid1_nx : v.inst_x_off[inst]);
    const double th = __ldg(xi + lb);
    const double vm = __ldg(xi + nb + lb);
    int4 r0, r1;
    make_record(th, vm, v.sincos_fix, r0, r1);
    int4 *rec = reinterpret_cast<int4 *>(v.phasor);
    rec[2 * q] = r0;
    rec[2 * q + 1] = r1;
  }
}

// The same for a context of one grid with an even number of buses and x on a
// 16-byte boundary: two consecutive buses per thread, their angles and
// magnitudes in one 16-byte load each and their records in 64 contiguous
// bytes (fewer instructions per bus for the index arithmetic and the loads),
// in 32 registers so that 2,048 threads fit on an SM.
__global__ void __launch_bounds__(256, 8) k_phasor_fx2(View v, const double *__restrict__ x, int i0) {
  cudaTriggerProgrammaticLaunchCompletion();
  const int32_t nb = v.grid1_nbus;
  const int inst = i0 + (int)blockIdx.y;
  const int64_t lb = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (lb >= nb) return;
  const double *xi = x + (int64_t)inst * v.grid1_nx;
  const double2 th = __ldg(reinterpret_cast<const double2 *>(xi + lb));
  const double2 vm = __ldg(reinterpret_cast<const double2 *>(xi + nb + lb));
  int4 a0, a1, b0, b1;
  make_record(th.x, vm.x, v.sincos_fix, a0, a1);
  make_record(th.y, vm.y, v.sincos_fix, b0, b1);
  int4 *rec = reinterpret_cast<int4 *>(v.phasor) + 2 * ((int64_t)inst * nb + lb);
  rec[0] = a0;
  rec[1] = a1;
  rec[2] = b0;
  rec[3] = b1;
}

// ---------------------------------------------------------------------------
// Fixed-point arithmetic of the pair terms (integer pipe).
//
// With the unit phasors U = (cos theta, sin theta) of k_phasor_fx, the own
// voltage E_o = V_o U_o and the merged coefficients (G, B) of a pair,
//     T = (G + jB) conj(E_o) U_k = (X - jY) / V_k,
// so that the pair's values are
//     X = V_k Re T,  -Y = V_k Im T          (the theta-column values and the bus sums)
//     -X / V_k = -Re T,  -Y / V_k = Im T    (the V-column values).
// Every fixed-point factor is held as 30-bit limbs (value = h 2^30 + l,
// 0 <= l < 2^30) and a product a b 2^-60 is formed from three 32 x 32 -> 64
// multiplies, h_a h_b + ((h_a l_b + l_a h_b) >> 30), the l_a l_b term dropped:
// low by less than 2 units (3 for a sum of two products).  Scales: U, V and
// E_o at 2^60 (|U| <= 1, |V|, |E_o| < 2), conj(E_o) U_k at 2^60, (G, B) at
// 2^(59 - c) with |G|, |B| < 2^c, T and X, Y at 2^(59 - c); every partial
// sum stays below 2^63.  With the 2^-57 error of the phasor routine the
// absolute error of T is below 2^(c - 55) (about 3e-17 max(|G|, |B|)), of X,
// Y below 2^(c - 54); X and Y are summed exactly in 96 bits and every value is
// rounded once to double (to nearest).
// ---------------------------------------------------------------------------

// a b, exact, from 32-bit factors (one 32 x 32 -> 64 multiply).
__device__ __forceinline__ long long wmul(int a, int b) { return (long long)a * (long long)b; }

// (a1 b1 + a2 b2) 2^-60 from limbs.
__device__ __forceinline__ long long dot60(int2 a1, int2 b1, int2 a2, int2 b2) {
  const long long m = wmul(a1.x, b1.y) + wmul(a1.y, b1.x) + wmul(a2.x, b2.y) + wmul(a2.y, b2.x);
  return wmul(a1.x, b1.x) + wmul(a2.x, b2.x) + (m >> 30);
}

// a b 2^-60 from limbs.
__device__ __forceinline__ long long mul60(int2 a, int2 b) {
  const long long m = wmul(a.x, b.y) + wmul(a.y, b.x);
  return wmul(a.x, b.x) + (m >> 30);
}

// z 2^-s as a double, rounded to nearest (ties away from zero); 2^-s |z| must
// be a normal double.
__device__ __forceinline__ double fix_to_double(long long z, int s) {
  // branch-free: for z = 0 the bits formed below are discarded by the final select
  const unsigned long long sign = (unsigned long long)z & 0x8000000000000000ULL;
  const unsigned long long a = sign ? 0ULL - (unsigned long long)z : (unsigned long long)z;
  const int lz = __clzll((long long)a);
  const unsigned long long n = a << (lz & 63);                                       // top bit 63
  const unsigned long long mag =
      ((unsigned long long)(1086 - s - lz) << 52) + ((n >> 11) & 0xfffffffffffffULL) + ((n >> 10) & 1ULL);
  return __longlong_as_double(z == 0 ? 0LL : (long long)(sign | mag));
}

// z 2^-s as a double on the integer pipe, for z > 0 with at most 53
// significant bits (so the value is exact: no rounding step), such as V 2^60
// formed from the double V; other z give meaningless bits.
__device__ __forceinline__ double exact_fix_to_double(long long z, int s) {
  const int lz = __clzll(z);
  const unsigned long long n = (unsigned long long)z << (lz & 63);                  // top bit 63
  return __longlong_as_double(
      (long long)(((unsigned long long)(1086 - s - lz) << 52) + ((n >> 11) & 0xfffffffffffffULL)));
}

// Exact sums on the integer pipe: a 96-bit two's-complement accumulator of
// fixed-point terms (|term| < 2^63; 2^31 terms cannot overflow it).  The sum
// does not depend on the order of the terms, so every schedule and tuning
// gives the same bits.  An add is one carry chain of three 32-bit adds.
struct Acc96 {
  unsigned l0, l1;
  int h;
};

// Adds a signed 64-bit term.
__device__ __forceinline__ void acc_add64(Acc96 &a, long long x) {
  const unsigned x0 = (unsigned)x, x1 = (unsigned)((unsigned long long)x >> 32);
  const int sx = (int)x1 >> 31;
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.s32 %2, %2, %5;"
      : "+r"(a.l0), "+r"(a.l1), "+r"(a.h)
      : "r"(x0), "r"(x1), "r"(sx));
}

// Whether the accumulator's value fits in 64 bits (the usual case: it is then
// rounded to double once by the FP64 pipe's conversion; a bus whose sums do
// not fit takes the FP64 form, a choice that depends only on the inputs).
__device__ __forceinline__ bool fits64(const Acc96 &a) { return a.h == ((int)a.l1 >> 31); }

// The low 64 bits (the value, when fits64).
__device__ __forceinline__ long long low64(const Acc96 &a) {
  return (long long)(((unsigned long long)a.l1 << 32) | a.l0);
}

struct EvalArgs {
  const double *x;
  double *F;
  double *vals;
  const double2 *gb;        // per end, incidence order
  const double2 *ac;
  const double2 *hat;       // per bus
  const double2 *pgb, *pac; // per pair of the tile kernel's list
  const int4 *pgbx;
  const double *p_inj;     // per-instance-bus override or nullptr
  const double *q_inj;
  const uint8_t *status;   // per-instance-branch mask or nullptr
  const uint8_t *gen_mode; // extended, per instance-generator: != 0 holds Q_g at gen_qlim, or nullptr
  const double *gen_qlim;
  // a persistent (capped) k_tile grid: {next unit, CTAs done} counters of
  // its dynamic schedule, zero at launch and reset by the grid's last CTA;
  // nullptr: CTA b takes units b, b + grid, ...
  unsigned long long *work;
};

// X and Y of one branch end (own voltage Eo, other voltage Ek, rectangular),
// in FP64.
struct EndTerms {
  double X, Y;
};

__device__ __forceinline__ EndTerms end_terms(double2 G, double2 Eo, double2 Ek) {
  // negations are applied to inputs (exact), so they fold into operand modifiers
  const double uu = __fma_rn(G.x, Ek.x, __dmul_rn(-G.y, Ek.y));
  const double ww = __fma_rn(G.x, Ek.y, __dmul_rn(G.y, Ek.x));
  EndTerms r;
  r.X = __fma_rn(Eo.x, uu, __dmul_rn(Eo.y, ww));
  r.Y = __fma_rn(Eo.y, uu, __dmul_rn(-Eo.x, ww));
  return r;
}

// The four off-diagonal values of a pair (CSR positions p, -1 where the
// formulation has no such entry) from its X, Y and 1/V_k (FP64 path).
__device__ __forceinline__ void write_pair(double *vi, int4 p, double X, double Y, double rvk) {
  if (p.x >= 0) vi[p.x] = neg(Y);                    // dP_o / dtheta_k
  if (p.y >= 0) vi[p.y] = __dmul_rn(-X, rvk);        // dP_o / dV_k
  if (p.z >= 0) vi[p.z] = X;                         // dQ_o / dtheta_k
  if (p.w >= 0) vi[p.w] = __dmul_rn(-Y, rvk);        // dQ_o / dV_k
}

// FP64 voltage of a bus for the FP64 path: E = V (cos, sin) (V after the
// dead-bus substitution) from the record's unit phasor and x's V, and 1/V --
// the values of the adjoint's FP64 records.  An angle that is not finite
// gives E = NaN, as the FP64 form would.
struct VoltD {
  double2 E;
  double v, rv;
};

__device__ __forceinline__ VoltD volt_fp64(int4 u, const double *__restrict__ xi, int32_t nb, int64_t lb) {
  const double th = xi[lb], vm = xi[nb + lb];
  const double sv = dead_sub(vm);
  VoltD r;
  if ((__double2hiint(th) & 0x7ff00000) == 0x7ff00000) {
    const double nan = __dsub_rn(th, th);
    r.E = make_double2(nan, nan);
  } else {
    const long long c = ((long long)u.x << 30) + u.y, s = ((long long)u.z << 30) + u.w;
    r.E = make_double2(__dmul_rn(sv, fix_to_double(c, 60)), __dmul_rn(sv, fix_to_double(s, 60)));
  }
  r.v = vm;
  r.rv = (__double2hiint(sv) & 0x7ff00000) >= 0x7d000000 ? __drcp_rn(sv) : recip(sv);
  return r;
}

__device__ __forceinline__ bool end_in_service(const View &v, int32_t e, int32_t outage, const uint8_t *status,
                                               int64_t st_base) {
  const int32_t l = __ldg(v.inc_code + e) >> 1;
  return (l != outage) && (status == nullptr || status[st_base + l] != 0);
}

__device__ __forceinline__ int64_t gb0_of(const View &v, int g) { return __ldg(v.grid_bus_off + g); }

// Off-diagonal entries of a group of `len` parallel branch ends e, e+1, ...
// (same own bus o, same other bus k, so the same four CSR positions), from
// X and Y summed over the group in list order (FP64).  For a group of one
// branch these are the single end's terms.
__device__ __forceinline__ void write_group(const View &v, const EvalArgs &a, int32_t e, int32_t len, double2 Eo,
                                            const VoltD &Ek, int4 p, double *vi, bool masked, int32_t outage,
                                            int64_t st_base) {
  double X = 0.0, Y = 0.0;
  for (int32_t q = 0; q < len; ++q) {
    double2 G = __ldg(a.gb + e + q);
    if (masked && !end_in_service(v, e + q, outage, a.status, st_base)) G = make_double2(0.0, 0.0);
    const EndTerms tq = end_terms(G, Eo, Ek.E);
    if (q == 0) {
      X = tq.X; Y = tq.Y;
    } else {
      X = __dadd_rn(X, tq.X); Y = __dadd_rn(Y, tq.Y);
    }
  }
  write_pair(vi, p, X, Y, Ek.rv);
}

// Under an outage mask: the coefficients of the branches in service of the
// group of `len` parallel branch ends e, e+1, ..., summed in incidence order
// (zero when none is in service).
struct GroupCoeff {
  double2 gb, ac;
  bool any_out;
};

__device__ __forceinline__ GroupCoeff masked_group(const View &v, const EvalArgs &a, int32_t e, int32_t len,
                                                   int32_t outage, int64_t st_base) {
  GroupCoeff r{make_double2(0.0, 0.0), make_double2(0.0, 0.0), false};
  bool first = true;
  for (int32_t i = 0; i < len; ++i) {
    if (!end_in_service(v, e + i, outage, a.status, st_base)) {
      r.any_out = true;
      continue;
    }
    const double2 gi = __ldg(a.gb + e + i), ci = __ldg(a.ac + e + i);
    if (first) {
      r.gb = gi;
      r.ac = ci;
      first = false;
    } else {
      r.gb = make_double2(__dadd_rn(r.gb.x, gi.x), __dadd_rn(r.gb.y, gi.y));
      r.ac = make_double2(__dadd_rn(r.ac.x, ci.x), __dadd_rn(r.ac.y, ci.y));
    }
  }
  return r;
}

// The groups of a bus as laid out for a kernel: group j at q0 + stride j,
// j < n (slots of a round: stride 32, padding marked by a negative group
// length; the tile kernel's pair list: stride 1), with the arrays of that
// layout (meta, idx, coefficients).
struct Walk {
  const int4 *meta, *idx;
  const double2 *gb, *ac;
  int64_t q0;
  int stride;
  int32_t n;
};

// Under an outage mask, for a bus with an end out of service: A^ and C^
// summed over its groups' ends in service (groups merged in incidence order,
// then summed in list order, as k_hat builds them), plus the shunt.
__device__ __forceinline__ double2 masked_hat(const View &v, const EvalArgs &a, const Walk &wk,
                                           int32_t outage, int64_t st_base, int32_t o) {
  double sa = 0.0, sc = 0.0;
  for (int32_t j = 0; j < wk.n; ++j) {
    const int64_t q = wk.q0 + (int64_t)wk.stride * j;
    const int4 m = __ldg(wk.meta + q);
    if (m.y < 0) continue;
    double2 ac;
    if (m.y == 1) {
      ac = end_in_service(v, m.w, outage, a.status, st_base) ? __ldg(wk.ac + q) : make_double2(0.0, 0.0);
    } else {
      ac = masked_group(v, a, m.w, m.y, outage, st_base).ac;
    }
    sa = __dadd_rn(sa, ac.x);
    sc = __dadd_rn(sc, ac.y);
  }
  const double2 sh = __ldg(v.bus_sh + o);
  return make_double2(__dadd_rn(sa, sh.x), __dadd_rn(sc, sh.y));
}

// z 2^-s as a double by the hardware conversion on the FP64 pipe (rounded to
// nearest even), the scale applied to the exponent; 2^-s |z| must be a normal
// double.  The pair loop converts its four values this way: one FP64-pipe
// instruction each, where the integer routine (fix_to_double) takes some
// twenty instructions of the issue slots the kernel is bound by.
__device__ __forceinline__ double fix_to_double_cvt(long long z, int s) {
  const double d = __ll2double_rn(z);
  return __hiloint2double(z == 0 ? 0 : __double2hiint(d) - (s << 20), __double2loint(d));
}

// Where a bus's in-row J values go: the first entry of its P row and of its
// Q row, either staged in shared memory or in J itself (nullptr: the row
// does not exist, or J is not wanted).
struct RowSink {
  double *prow, *qrow;
  __device__ __forceinline__ void p(int32_t off, double x) const {
    if (prow) prow[off] = x;
  }
  __device__ __forceinline__ void q(int32_t off, double x) const {
    if (qrow) qrow[off] = x;
  }
};

// F rows, the extended formulation's extra rows and the diagonal of J for
// bus o (global id) of one instance, from the sums over its ends; in-row
// values through the sink, the bus's F_P and F_Q to fpr and fqr (nullptr:
// no such row), the extended formulation's g_V and g_theta rows straight to
// F and J.
template <bool WF, bool WJ>
__device__ __forceinline__ void finalize_bus(const View &v, const EvalArgs &a, int inst, int g, int32_t o,
                                             int64_t gb0, int32_t nb, const double *xi, double *Fi, double *vi,
                                             const RowSink &rs, double *fpr, double *fqr,
                                             double vo, double rvo, double sx, double sy, double ah, double ch,
                                             int4 bm, int4 bm2, double2 inj) {
  const int64_t lb = o - gb0;
  // the extended formulation's rows behind one branch on a launch-wide value,
  // so that the reduced formulation's buses jump over them
  const bool ext = v.formulation == PF_EXTENDED;
  const double v2 = __dmul_rn(vo, vo);
  const double tp = __fma_rn(v2, ah, -sx);          // V_o^2 A^ - S_X
  const double tq = __fma_rn(v2, ch, sy);           // V_o^2 C^ + S_Y
  if (WF) {
    double pin = inj.x, qin = inj.y;
    if (a.p_inj || a.q_inj) {                      // per-call injections (a launch-wide choice)
      const int64_t q = v.inst_bus_off[inst] + lb;
      if (a.p_inj) pin = a.p_inj[q];
      if (a.q_inj) qin = a.q_inj[q];
    }
    double fp = __dsub_rn(tp, pin);
    double fq = __dadd_rn(-tq, -qin);
    if (ext) {
      const int32_t gi = bm2.w;
      if (lb == v.grid_slack[g]) {
        fp = __dsub_rn(fp, xi[2 * nb + v.grid_ngen[g]]);
        Fi[v.grid_row_gth[g]] = __dsub_rn(xi[lb], v.grid_theta_set[g]);
      }
      if (gi >= 0) {
        const double qg = xi[2 * nb + gi];
        fq = __dsub_rn(fq, qg);
        const int64_t gq = v.inst_gen_off[inst] + gi;
        Fi[2 * nb + gi] = (a.gen_mode && a.gen_mode[gq]) ? __dsub_rn(qg, a.gen_qlim[gq])       // held at a limit
                                                         : __dsub_rn(vo, v.gen_vset[v.grid_gen_off[g] + gi]);
      }
    }
    if (fpr) *fpr = fp;
    if (fqr) *fqr = fq;
  }
  if (WJ) {
    if (bm2.x >= 0) {
      rs.p(bm2.x, sy);                                   // dF_P / dtheta_o
      rs.q(bm2.x, neg(sx));                              // dF_Q / dtheta_o
    }
    if (bm2.y >= 0) {
      rs.p(bm2.y, __dmul_rn(__fma_rn(v2, ah, tp), rvo));  // dF_P / dV_o
      rs.q(bm2.y, __dmul_rn(__fma_rn(v2, ch, tq), -rvo)); // dF_Q / dV_o
    }
    if (ext) {
      const int32_t gi = bm2.w;
      if (lb == v.grid_slack[g]) {
        rs.p(bm2.z, -1.0);                    // d g_p / d P_s
        vi[v.grid_pos_gth[g]] = 1.0;         // d g_theta / d theta_s
      }
      if (gi >= 0) {
        rs.q(bm2.z, -1.0);                    // d g_q / d Q_g
        const bool held = a.gen_mode && a.gen_mode[v.inst_gen_off[inst] + gi];
        const int32_t p = v.gen_pos[v.grid_gen_off[g] + gi];
        vi[p] = held ? 0.0 : 1.0;             // d g_V / d V
        vi[p + 1] = held ? 1.0 : 0.0;         // d g_V / d Q_g
      }
    }
  }
}

// Without a per-call status mask the only branch out of service is the
// instance's outage, whose two ends sit at incidence positions oute (-1: no
// outage): a group of parallel ends [e, e + len) holding neither keeps its
// built coefficients, so only the groups that hold it are summed again.
__device__ __forceinline__ bool outside_group(const EvalArgs &a, int32_t e, int32_t len, int2 oute) {
  return a.status == nullptr && (unsigned)(oute.x - e) >= (unsigned)len && (unsigned)(oute.y - e) >= (unsigned)len;
}

// The incidence positions of the two ends of branch `outage` (-1 none).
__device__ __forceinline__ int2 outage_ends(const View &v, int32_t outage) {
  return outage >= 0 ? make_int2(__ldg(v.inc_of_code + 2 * outage), __ldg(v.inc_of_code + 2 * outage + 1))
                     : make_int2(-1, -1);
}

// The merged coefficients (G, B) of a slot (len: its group length, cw: the
// code of a single branch or the first end of a group) as the mask leaves
// them: the built value, zero for a single branch out of service, or the
// re-summed branches in service of a group.
template <bool MASKED>
__device__ __forceinline__ double2 slot_gb(const View &v, const EvalArgs &a, int32_t len, int32_t cw, double2 G,
                                           int32_t outage, int64_t st_base, bool &any_out, int2 oute) {
  if (!MASKED) return G;
  if (len > 1 && outside_group(a, cw, len, oute)) return G;
  if (len == 1) {
    const int32_t l = cw >> 1;
    if (l == outage || (a.status != nullptr && a.status[st_base + l] == 0)) {
      any_out = true;
      return make_double2(0.0, 0.0);
    }
    return G;
  }
  const GroupCoeff mg = masked_group(v, a, cw, len, outage, st_base);
  any_out |= mg.any_out;
  return mg.gb;
}

// The same in fixed point (GX: the slot's sgbx entry); a re-summed group is
// converted as the build converts it.
template <bool MASKED>
__device__ __forceinline__ int4 slot_gbx(const View &v, const EvalArgs &a, int32_t len, int32_t cw, int4 GX,
                                         int32_t outage, int64_t st_base, bool &any_out, int2 oute) {
  if (!MASKED) return GX;
  if (len > 1 && outside_group(a, cw, len, oute)) return GX;
  if (len == 1) {
    const int32_t l = cw >> 1;
    if (l == outage || (a.status != nullptr && a.status[st_base + l] == 0)) {
      any_out = true;
      return make_int4(0, 0, 0, 0);
    }
    return GX;
  }
  const GroupCoeff mg = masked_group(v, a, cw, len, outage, st_base);
  any_out |= mg.any_out;
  return coef_limbs(to_fix(mg.gb.x, v.coef_scale), to_fix(mg.gb.y, v.coef_scale));
}

// The 32-byte record of a bus in one load: {cos h, cos l, sin h, sin l} and
// {V h, V l, 1/V lo, 1/V hi} (fixed-point form) -- the record starts on a
// 32-byte boundary.
struct Rec {
  int4 u, w;
};

__device__ __forceinline__ Rec load_rec(const int4 *p) {
  Rec r;
  asm("ld.global.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r.u.x), "=r"(r.u.y), "=r"(r.u.z), "=r"(r.u.w), "=r"(r.w.x), "=r"(r.w.y), "=r"(r.w.z),
                 "=r"(r.w.w)
               : "l"(p));
  return r;
}

// The own bus's voltage for the fixed-point pair terms, from its record:
// E_o = V_o U_o at 2^60 as limbs (and -f_o), V_o at 2^60 and as a double;
// `fast` when V_o lies in [1/4, 2) (kBadLimb is negative).
struct OwnV {
  int2 eo, fo, nfo;
  double rvo;
  double vo;                                      // V_o
  bool fast;
};

__device__ __forceinline__ OwnV own_voltage(const Rec &ro) {
  OwnV w;
  const int2 vl = make_int2(ro.w.x, ro.w.y);
  w.rvo = __hiloint2double(ro.w.w, ro.w.z);
  // exact for 2^-8 <= V < 2 (the only V used, `fast`), on the integer pipe
  w.vo = exact_fix_to_double(((long long)ro.w.x << 30) + ro.w.y, 60);
  w.fast = ro.w.x >= (1 << 28);
  w.eo = limbs(mul60(vl, make_int2(ro.u.x, ro.u.y)));
  const long long f = mul60(vl, make_int2(ro.u.z, ro.u.w));
  w.fo = limbs(f);
  w.nfo = limbs(-f);
  return w;
}

// One pair's fixed-point terms from the neighbour's record rk and the merged
// coefficients gx: T = (G + jB) conj(E_o) U_k and X = V_k Re T, -Y = V_k Im T,
// all at 2^(59 - c).  `ok` is false when the record or a coefficient is
// marked out of range.
struct PairT {
  long long xx, my, tr, ti;
  bool ok;
};

__device__ __forceinline__ PairT pair_terms(const OwnV &w, const Rec &rk, int4 gx) {
  PairT t;
  t.ok = rk.w.x != kBadLimb && gx.x != kBadLimb && gx.z != kBadLimb;
  const int2 ck = make_int2(rk.u.x, rk.u.y), sk = make_int2(rk.u.z, rk.u.w), vk = make_int2(rk.w.x, rk.w.y);
  // conj(E_o) U_k 2^60
  const long long pr = dot60(w.eo, ck, w.fo, sk);
  const long long pi = dot60(w.eo, sk, w.nfo, ck);
  const int2 prl = limbs(pr), pil = limbs(pi), npil = limbs(-pi);
  // T = (G + jB) conj(E_o) U_k 2^(59 - c)
  const int2 gl = make_int2(gx.x, gx.y), bl = make_int2(gx.z, gx.w);
  t.tr = dot60(gl, prl, bl, npil);
  t.ti = dot60(gl, pil, bl, prl);
  // X = V_k Re T, -Y = V_k Im T, 2^(59 - c)
  t.xx = mul60(vk, limbs(t.tr));
  t.my = mul60(vk, limbs(t.ti));
  return t;
}

// A unit's instance: its grid and where its state, outputs and records live.
struct UnitCtx {
  int inst, g;
  int64_t gb0;
  int32_t nb;
  const double *xi;
  double *Fi, *vi;
  const int4 *rec4;
  int32_t outage;
  int64_t st_base;
  const int4 *srec;          // the tile's records in shared memory (the kernel forms them), or nullptr
  int own_loc;               // the bus's record index among them
};

// The rest of bus o after its pairs, on its lead lane: the sums rounded to
// double (or, when the fixed-point form does not hold for the bus, every value
// of the bus again in FP64 from x and the records, pairs in list order), A^
// and C^ re-summed under a mask, the F rows and diagonal values
// (finalize_bus).  bm2, hat, inj: the bus's row data; wk: its groups.
template <bool WF, bool WJ, bool MASKED>
__device__ __forceinline__ void finish_bus(const View &v, const EvalArgs &a, const UnitCtx &uc, int32_t o,
                                           int4 bm, int4 bm2, double2 hat, double2 inj, const RowSink &rs,
                                           double *fpr, double *fqr, bool fast, bool any_out, const Acc96 &ax,
                                           const Acc96 &ay, const OwnV &w, const Walk &wk, int sT) {
  double sx, sy, vo, rvo;
  if (fast) {
    sx = fix_to_double_cvt(low64(ax), sT);   // (fast: both sums fit in 64 bits)
    sy = neg(fix_to_double_cvt(low64(ay), sT));
    vo = w.vo;
    rvo = w.rvo;                                 // V_o in [1/4, 2): from k_phasor_fx
  } else {
    // FP64 form of the whole bus, pairs in list order
    const VoltD Vo = volt_fp64(uc.srec ? uc.srec[2 * uc.own_loc] : uc.rec4[2 * o], uc.xi, uc.nb, o - uc.gb0);
    vo = Vo.v;
    rvo = Vo.rv;
    sx = 0.0;
    sy = 0.0;
    bool unused = false;
    for (int32_t j = 0; j < wk.n; ++j) {
      const int64_t q = wk.q0 + (int64_t)wk.stride * j;
      const int4 m = __ldg(wk.idx + q);
      const int32_t len = (short)(m.z & 0xffff);
      if (len < 0) continue;
      const double2 Gi = slot_gb<MASKED>(v, a, len, m.w, __ldg(wk.gb + q), uc.outage, uc.st_base, unused,
                                         MASKED ? outage_ends(v, uc.outage) : make_int2(-1, -1));
      const VoltD Vk = volt_fp64(uc.srec ? uc.srec[2 * ((m.z >> 24) & 0xff)] : uc.rec4[2 * m.x], uc.xi, uc.nb,
                                 m.x - uc.gb0);
      const EndTerms tm = end_terms(Gi, Vo.E, Vk.E);
      sx = __dadd_rn(sx, tm.X);
      sy = __dadd_rn(sy, tm.Y);
      if (WJ) {
        const int32_t ot = (short)(m.y & 0xffff), ov = m.y >> 16;
        if (ot >= 0) {
          rs.p(ot, neg(tm.Y));
          rs.q(ot, tm.X);
        }
        if (ov >= 0) {
          rs.p(ov, __dmul_rn(-tm.X, Vk.rv));
          rs.q(ov, __dmul_rn(-tm.Y, Vk.rv));
        }
      }
    }
  }
  // A^, C^: built (every end in service), else re-summed over the ends in
  // service in the same order as the built value
  if (MASKED && any_out) hat = masked_hat(v, a, wk, uc.outage, uc.st_base, o);
  finalize_bus<WF, WJ>(v, a, uc.inst, uc.g, o, uc.gb0, uc.nb, uc.xi, uc.Fi, uc.vi, rs, fpr, fqr, vo, rvo, sx, sy,
                       hat.x, hat.y, bm, bm2, inj);
}

// n values from shared memory (src) to global memory (dst) by one thread: the
// 16-byte aligned middle as one bulk copy of the tensor memory accelerator
// (cp.async.bulk, asynchronous: the caller commits the group and waits for its
// reads of shared memory before the buffer is written again), a value at
// either end outside it by a plain store; src and dst lie at the same offset
// modulo 16 bytes.  The warp's writes to src must be made visible to the
// async proxy first (fence.proxy.async.shared::cta and a warp barrier).
__device__ __forceinline__ void bulk_out(double *dst, const double *src, int32_t n) {
  if (n <= 0) return;
  const int32_t i0 = (int32_t)((reinterpret_cast<uintptr_t>(dst) >> 3) & 1);
  if (i0) dst[0] = src[0];
  const int32_t n2 = (n - i0) >> 1;
  if (n2 > 0) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(src + i0);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(dst + i0), "r"(sa), "r"(16 * n2));
  }
  if ((n - i0) & 1) dst[n - 1] = src[n - 1];
}

// Shared memory of a k_tile warp (byte offsets, 16-byte aligned): E_o limbs
// of each bus ({e, f} and {-f, -}: 32 x 2 int4), staging index of each bus's P and Q row (32 int2,
// -1 none), per-bus flags (32 int: 1 FP64 form, 2 an end out of service), X
// and -Y of each pair (kTilePairs longlong2), the tile's F values (P rows,
// then Q rows: 64 doubles), then the staged J rows (v.tile_stage doubles).
constexpr int kTsOwn = 0;
constexpr int kTsBase = kTsOwn + 32 * 32;
constexpr int kTsFlag = kTsBase + 32 * 8;
constexpr int kTsXY = kTsFlag + 32 * 4;
constexpr int kTsF = kTsXY + kTilePairs * 16;
constexpr int kTileSmemFixed = kTsF + 64 * 8;
// With the records formed in the kernel (PHX), they follow: the tile's buses
// at 0..31, its external neighbours from kTileBuses on (32 bytes each), and
// the staged J rows after them.
constexpr int kTileRecBytes = (kTileBuses + kTilePairs) * 32;
static_assert(kTileSmemFixed % 16 == 0, "shared-memory layout of k_tile");

// One-warp CTAs resident per SM (the register budget of k_tile): 28 for the
// F + J evaluation (72 registers), 24 under a mask, 20 for a persistent
// schedule, 16 where the kernel forms its records (the form for one instance,
// which fills only about 14 warps per SM).
template <int ITEMS, bool WF, bool WJ, bool MASKED, bool DYN, bool PHX>
struct TileMinCtas {
  static constexpr int value = DYN ? 20 : PHX ? 16 : MASKED ? 24 : 28;
};

// One warp per tile of one instance: up to 32 consecutive buses of a grid and
// their pairs of connected buses (at most kTilePairs), so that the tile's J
// values form two contiguous ranges of J (its P rows and its Q rows) and its
// F values two contiguous ranges of F.
//   phase 0: lane l takes bus l of the tile: its record gives E_o, kept in
//            shared memory for every lane;
//   phase 1: lane l takes pairs l, l + 32, l + 64 of the tile's list (so the
//            lanes share the pairs evenly whatever the buses' numbers of
//            neighbours), ITEMS of them with their records in flight at once:
//            the pair's fixed-point terms, its four J values into the staged
//            rows and X, -Y into shared memory;
//   phase 2: lane l sums its bus's X, -Y exactly (96-bit integers, so the
//            order does not matter) and finishes the bus (finish_bus: the FP64
//            form where the fixed-point one does not hold, F rows, diagonal
//            values);
//   phase 3: the staged rows of J leave whole, each by one bulk copy of the
//            tensor memory accelerator (lane 0 issues it and waits for it
//            to have read the staging before the next unit), F's rows by
//            the lanes.
// With a persistent grid (DYN) the warps claim their units from a counter;
// the last CTA resets it.  With PHX the warp first forms the records of its
// tile's buses and of their external neighbours itself (from x, into shared
// memory): no phasor kernel before it and no record gathers from L2, at the
// price of forming a neighbour's record in every tile that reaches it.
template <int ITEMS, bool WF, bool WJ, bool MASKED, bool DYN, bool PHX>
__global__ void __launch_bounds__(32, (TileMinCtas<ITEMS, WF, WJ, MASKED, DYN, PHX>::value))
    k_tile(View v, EvalArgs a) {
  // Let a dependent launch start (the next evaluation's k_tile with
  // fuse_phasor: it waits for this grid before it reads x or writes).
  cudaTriggerProgrammaticLaunchCompletion();
  extern __shared__ __align__(16) unsigned char s_raw[];
  int4 *const s_own = reinterpret_cast<int4 *>(s_raw + kTsOwn);
  int2 *const s_base = reinterpret_cast<int2 *>(s_raw + kTsBase);
  int *const s_flag = reinterpret_cast<int *>(s_raw + kTsFlag);
  longlong2 *const s_xy = reinterpret_cast<longlong2 *>(s_raw + kTsXY);
  double *const s_f = reinterpret_cast<double *>(s_raw + kTsF);
  int4 *const s_rec = reinterpret_cast<int4 *>(s_raw + kTileSmemFixed);
  double *const s_j = reinterpret_cast<double *>(s_raw + kTileSmemFixed + (PHX ? kTileRecBytes : 0));
  const int lane = threadIdx.x & 31;
  const int sT = 59 - v.coef_log2;
  unsigned long long *const work = DYN ? a.work : nullptr;
  int64_t u = blockIdx.x;
  unsigned long long claim = 0;
  if (work) {
    // The counters were reset by the previous launch's last CTA; as a
    // programmatic dependent this grid may start before that write is
    // visible, so it waits for its prerequisite grids before the first claim.
    cudaGridDependencySynchronize();
    if (lane == 0) claim = atomicAdd(work, 1ULL);
    u = (int64_t)__shfl_sync(0xffffffffu, claim, 0);
  }
  for (; u < v.n_tile_units; u = work ? (int64_t)__shfl_sync(0xffffffffu, claim, 0) : u + gridDim.x) {
    if (work && lane == 0) claim = atomicAdd(work, 1ULL);
    const int4 *ur = v.tunit + 8 * u;
    const int4 td = __ldg(ur), ts = __ldg(ur + 1), tf = __ldg(ur + 2), ti = __ldg(ur + 3);
    const longlong2 up0 = __ldg(reinterpret_cast<const longlong2 *>(ur + 4));
    const longlong2 up1 = __ldg(reinterpret_cast<const longlong2 *>(ur + 5));
    const int inst = ti.x, g = ti.y;
    const int32_t fp = td.z, np = td.w;
    const double *__restrict__ xi = a.x + up0.x;
    double *__restrict__ Fi = WF ? a.F + up0.y : nullptr;
    double *__restrict__ vi = WJ ? a.vals + up1.x : nullptr;
    const int4 *__restrict__ rec4 = reinterpret_cast<const int4 *>(v.phasor) + 2 * up1.y;
    const int32_t outage = MASKED ? v.inst_outage[inst] : -1;
    const int64_t st_base = MASKED ? v.inst_br_off[inst] - v.grid_br_off[g] : 0;
    const int2 oute = MASKED ? outage_ends(v, outage) : make_int2(-1, -1);
    // staged J: the P rows at s_j[padP ..), the Q rows at s_j[offQ + padQ ..),
    // each at the offset modulo 16 bytes of its destination
    const int32_t padP = WJ ? (int32_t)((reinterpret_cast<uintptr_t>(vi + ts.x) >> 3) & 1) : 0;
    const int32_t offQ = (padP + ts.y + 1) & ~1;
    const int32_t padQ = WJ ? (int32_t)((reinterpret_cast<uintptr_t>(vi + ts.z) >> 3) & 1) : 0;

    // Under a mask, only a tile holding an end of its instance's outaged branch
    // (or any tile, with a per-call status mask) needs the masked coefficients:
    // a pair's group holds the outaged branch only if its own bus is an end of
    // it, and the tile's buses' ends are one contiguous range of incidence
    // positions.  The other tiles take the built coefficients, the same bits.
    bool um = false;
    if (MASKED) {
      if (a.status != nullptr) {
        um = true;
      } else if (outage >= 0) {
        const int32_t e0 = __ldg(v.inc_ptr + td.x), e1 = __ldg(v.inc_ptr + td.x + td.y);
        um = (oute.x >= e0 && oute.x < e1) || (oute.y >= e0 && oute.y < e1);
      }
    }

    const bool owner = lane < td.y;
    const int32_t o = td.x + lane;
    int4 bm = make_int4(-1, -1, -1, -1);
    if (owner) bm = __ldg(v.bus_meta + o);
    OwnV w{make_int2(0, 0), make_int2(0, 0), make_int2(0, 0), 0.0, 1.0, true};
    // the first pass's pairs (static data: loaded before any wait for the
    // previous grid)
    int4 idx[ITEMS], GX[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const int32_t p = 32 * it + lane;
      idx[it] = make_int4(0, -1, -1, 0);
      if (p < np) {
        idx[it] = __ldg(v.pair_idx + fp + p);
        GX[it] = __ldg(a.pgbx + fp + p);
      }
    }
    // the bus's row data for phase 2, also static: early where the kernel
    // forms its records (registers to spare), after the pairs otherwise
    int32_t pr0 = 0, pr1 = 0;
    int4 bm2 = make_int4(-1, -1, -1, -1);
    double2 hat = make_double2(0.0, 0.0), inj = make_double2(0.0, 0.0);
    if (PHX && owner) {
      pr0 = __ldg(v.pair_ptr + o) - fp;
      pr1 = __ldg(v.pair_ptr + o + 1) - fp;
      bm2 = __ldg(v.bus_meta2 + o);
      hat = __ldg(a.hat + o);
      if (WF) inj = __ldg(v.bus_inj + o);
    }
    if (PHX) {
      // the records of the tile's buses and of its external neighbours, records
      // lane, lane + 32, ...: every bus and every value of x first, then the
      // arithmetic
      constexpr int kRecPerLane = (kTileBuses + kTilePairs) / 32;
      const int4 te = __ldg(ur + 6);             // {first external neighbour, external neighbours}
      const int32_t n_rec = td.y + te.y;
      int32_t bl[kRecPerLane];
#pragma unroll
      for (int i = 0; i < kRecPerLane; ++i) {
        const int32_t r = lane + 32 * i;
        bl[i] = r < td.y ? td.x + r : (r < n_rec ? __ldg(v.tile_ext + te.x + (r - td.y)) : -1);
      }
      // x may come from the stream's previous kernel (a programmatic dependent launch)
      cudaGridDependencySynchronize();
      double th[kRecPerLane], vm[kRecPerLane];
#pragma unroll
      for (int i = 0; i < kRecPerLane; ++i) {
        if (bl[i] >= 0) {
          const int64_t lb = bl[i] - ti.z;
          th[i] = __ldg(xi + lb);
          vm[i] = __ldg(xi + ti.w + lb);
        }
      }
#pragma unroll
      for (int i = 0; i < kRecPerLane; ++i) {
        if (bl[i] >= 0) {
          const int32_t r = lane + 32 * i;
          int4 r0, r1;
          make_record(th[i], vm[i], v.sincos_fix, r0, r1, r < td.y);   // 1/V: the tile's own buses only
          const int32_t slot = r < td.y ? r : kTileBuses + (r - td.y);
          s_rec[2 * slot] = r0;
          s_rec[2 * slot + 1] = r1;
        }
      }
      __syncwarp();
    }

    // (the first pass always runs: it waits for the records and sets up the buses)
    for (int32_t p0 = 0; p0 == 0 || p0 < np; p0 += 32 * ITEMS) {
      if (p0 > 0) {
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
          const int32_t p = p0 + 32 * it + lane;
          idx[it] = make_int4(0, -1, -1, 0);
          if (p < np) {
            idx[it] = __ldg(v.pair_idx + fp + p);
            GX[it] = __ldg(a.pgbx + fp + p);
          }
        }
      }
      if (p0 == 0) {
        // phase 0 (the records come from k_phasor_fx, a programmatic dependent launch)
        if (!PHX) cudaGridDependencySynchronize();
        if (owner) {
          w = own_voltage(PHX ? Rec{s_rec[2 * lane], s_rec[2 * lane + 1]} : load_rec(rec4 + 2 * o));
          s_own[2 * lane] = make_int4(w.eo.x, w.eo.y, w.fo.x, w.fo.y);
          s_own[2 * lane + 1] = make_int4(w.nfo.x, w.nfo.y, 0, 0);
          s_base[lane] = make_int2((WJ && bm.z >= 0) ? padP + bm.z - ts.x : -1,
                                   (WJ && bm.w >= 0) ? offQ + padQ + bm.w - ts.z : -1);
          s_flag[lane] = 0;
        }
        __syncwarp();
      }
      // phase 1
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int32_t p = p0 + 32 * it + lane;
        if (idx[it].z < 0) continue;
        const int32_t len = idx[it].z & 0xffff, ol = (idx[it].z >> 16) & 0xff;
        bool anyo = false;
        const int4 gx = (MASKED && um) ? slot_gbx<true>(v, a, len, idx[it].w, GX[it], outage, st_base, anyo, oute)
                                       : GX[it];
        const int4 e = s_own[2 * ol], e2 = s_own[2 * ol + 1];
        OwnV wo;
        wo.eo = make_int2(e.x, e.y);
        wo.fo = make_int2(e.z, e.w);
        wo.nfo = make_int2(e2.x, e2.y);
        const int loc = (idx[it].z >> 24) & 0xff;
        const PairT t = pair_terms(wo, PHX ? Rec{s_rec[2 * loc], s_rec[2 * loc + 1]} : load_rec(rec4 + 2 * idx[it].x),
                                   gx);
        s_xy[p] = make_longlong2(t.xx, t.my);
        if (!t.ok || anyo) atomicOr(s_flag + ol, (t.ok ? 0 : 1) | (anyo ? 2 : 0));
        if (WJ) {
          // the pair's four values into the staged rows (staging indices, -1: no such row)
          const int2 bs = s_base[ol];
          const int32_t ot = (short)(idx[it].y & 0xffff), ov = idx[it].y >> 16;
          if (ot >= 0) {
            if (bs.x >= 0) s_j[bs.x + ot] = fix_to_double_cvt(t.my, sT);       // dP_o / dtheta_k = -Y
            if (bs.y >= 0) s_j[bs.y + ot] = fix_to_double_cvt(t.xx, sT);       // dQ_o / dtheta_k = X
          }
          if (ov >= 0) {
            if (bs.x >= 0) s_j[bs.x + ov] = neg(fix_to_double_cvt(t.tr, sT));  // dP_o / dV_k = -X / V_k
            if (bs.y >= 0) s_j[bs.y + ov] = fix_to_double_cvt(t.ti, sT);       // dQ_o / dV_k = -Y / V_k
          }
        }
      }
    }
    __syncwarp();
    // phase 2
    if (owner) {
      if (!PHX) {
        pr0 = __ldg(v.pair_ptr + o) - fp;
        pr1 = __ldg(v.pair_ptr + o + 1) - fp;
      }
      Acc96 ax{0u, 0u, 0}, ay{0u, 0u, 0};
      for (int32_t q = pr0; q < pr1; ++q) {
        const longlong2 xy = s_xy[q];
        acc_add64(ax, xy.x);
        acc_add64(ay, xy.y);
      }
      const int fl = s_flag[lane];
      const bool fast = w.fast && !(fl & 1) && fits64(ax) && fits64(ay);
      if (!PHX) {
        bm2 = __ldg(v.bus_meta2 + o);
        hat = __ldg(a.hat + o);
        if (WF) inj = __ldg(v.bus_inj + o);
      }
      const int2 bs = s_base[lane];
      const RowSink rs{bs.x >= 0 ? s_j + bs.x : nullptr, bs.y >= 0 ? s_j + bs.y : nullptr};
      const UnitCtx uc{inst, g, ti.z, ti.w, xi, Fi, vi, rec4, outage, st_base, PHX ? s_rec : nullptr, lane};
      const Walk wk{v.pair_meta, v.pair_idx, a.pgb, a.pac, (int64_t)fp + pr0, 1, pr1 - pr0};
      finish_bus<WF, WJ, MASKED>(v, a, uc, o, bm, bm2, hat, inj, rs, (WF && bm.x >= 0) ? s_f + (bm.x - tf.x) : nullptr,
                                 (WF && bm.y >= 0) ? s_f + 32 + (bm.y - tf.z) : nullptr, fast, (fl & 2) != 0, ax, ay,
                                 w, wk, sT);
    }
    __syncwarp();
    // phase 3: the staged rows of J leave by bulk copies issued by lane 0, the
    // F rows by the lanes
    if (WJ) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        bulk_out(vi + ts.x, s_j + padP, ts.y);
        bulk_out(vi + ts.z, s_j + offQ + padQ, ts.w);
        asm volatile("cp.async.bulk.commit_group;");
      }
    }
    if (WF) {
      if (lane < tf.y) Fi[tf.x + lane] = s_f[lane];
      if (lane < tf.w) Fi[tf.z + lane] = s_f[32 + lane];
    }
    if (WJ && lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();                                // the next unit reuses the staging
  }
  // Every CTA leaves the loop once, after a claim past the last unit; the last
  // one to leave resets both counters for the next launch.
  if (work && lane == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1ULL) == gridDim.x - 1) {
      work[0] = 0ULL;
      work[1] = 0ULL;
    }
  }
}

// Buses with more than 32 ends, one warp each (launched after k_tile, so the
// records are complete), in FP64.  Lane l takes ends l, l + 32, l + 64, ... of
// the bus's list and sums them in that order; the 32 partial sums are then
// combined by a fixed butterfly, so the result depends on neither the
// tuning nor the schedule.  Off-diagonal entries as in k_tile's FP64 form.
template <int ITEMS, bool WF, bool WJ, bool MASKED>
__global__ void __launch_bounds__(32) k_fused_large(View v, EvalArgs a) {
  const int lane = threadIdx.x & 31;
  for (int64_t u = blockIdx.x; u < v.n_large_units; u += gridDim.x) {
    const int2 lr = __ldg(v.large_rec + u);       // {instance, bus}
    const int inst = lr.x;
    const int32_t o = lr.y;
    const int g = __ldg(v.inst_grid + inst);
    const double *__restrict__ xi = a.x + __ldg(v.inst_x_off + inst);
    const int4 *__restrict__ rec4 = reinterpret_cast<const int4 *>(v.phasor) + 2 * __ldg(v.inst_rec_base + inst);
    double *__restrict__ vi = WJ ? a.vals + __ldg(v.inst_v_off + inst) : nullptr;
    const int32_t outage = MASKED ? v.inst_outage[inst] : -1;
    const int64_t st_base = MASKED ? v.inst_br_off[inst] - v.grid_br_off[g] : 0;
    const int32_t e0 = __ldg(v.inc_ptr + o), e1 = __ldg(v.inc_ptr + o + 1);
    const int64_t gb0 = gb0_of(v, g);
    const int32_t nb = v.grid_nbus[g];
    const VoltD Vo = volt_fp64(rec4[2 * o], xi, nb, o - gb0);
    double sx = 0.0, sy = 0.0, acc_ma = 0.0, acc_mc = 0.0;
    for (int32_t cs = e0; cs < e1; cs += 32 * ITEMS) {
      int4 meta[ITEMS];
      double2 G[ITEMS];
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int32_t e = cs + it * 32 + lane;
        if (e < e1) {
          meta[it] = __ldg(v.inc_meta + e);
          G[it] = __ldg(a.gb + e);
        }
      }
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int32_t e = cs + it * 32 + lane;
        if (e >= e1) continue;
        double2 Gi = G[it];
        bool in = true;
        if (MASKED) {
          const int32_t l = meta[it].w >> 1;
          in = (l != outage) && (a.status == nullptr || a.status[st_base + l] != 0);
          if (!in) Gi = make_double2(0.0, 0.0);
        }
        const int32_t k = meta[it].y;
        const VoltD Vk = volt_fp64(rec4[2 * k], xi, nb, k - gb0);
        const EndTerms tm = end_terms(Gi, Vo.E, Vk.E);
        sx = __dadd_rn(sx, tm.X);
        sy = __dadd_rn(sy, tm.Y);
        if (MASKED) {
          const double2 ac = __ldg(a.ac + e);
          acc_ma = __dadd_rn(acc_ma, in ? ac.x : 0.0);
          acc_mc = __dadd_rn(acc_mc, in ? ac.y : 0.0);
        }
        if (WJ) {
          const int4 p = __ldg(v.inc_pos + e);
          if (meta[it].z == 1) {
            write_pair(vi, p, tm.X, tm.Y, Vk.rv);
          } else if (meta[it].z > 1) {
            write_group(v, a, e, meta[it].z, Vo.E, Vk, p, vi, MASKED, outage, st_base);
          }
        }
      }
    }
    // fixed butterfly: every lane ends with the same sums
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      sx = __dadd_rn(sx, __shfl_xor_sync(0xffffffffu, sx, m));
      sy = __dadd_rn(sy, __shfl_xor_sync(0xffffffffu, sy, m));
      if (MASKED) {
        acc_ma = __dadd_rn(acc_ma, __shfl_xor_sync(0xffffffffu, acc_ma, m));
        acc_mc = __dadd_rn(acc_mc, __shfl_xor_sync(0xffffffffu, acc_mc, m));
      }
    }
    if (lane == 0) {
      double ah, ch;
      if (MASKED) {
        const double2 sh = __ldg(v.bus_sh + o);
        ah = __dadd_rn(acc_ma, sh.x);
        ch = __dadd_rn(acc_mc, sh.y);
      } else {
        const double2 hat = __ldg(a.hat + o);
        ah = hat.x;
        ch = hat.y;
      }
      const double2 inj = WF ? __ldg(v.bus_inj + o) : make_double2(0.0, 0.0);
      const int4 bm = __ldg(v.bus_meta + o);
      const RowSink rs{(WJ && bm.z >= 0) ? vi + bm.z : nullptr, (WJ && bm.w >= 0) ? vi + bm.w : nullptr};
      double *Fi = WF ? a.F + v.inst_f_off[inst] : nullptr;
      finalize_bus<WF, WJ>(v, a, inst, g, o, gb0, nb, xi, Fi, vi, rs, (WF && bm.x >= 0) ? Fi + bm.x : nullptr,
                           (WF && bm.y >= 0) ? Fi + bm.y : nullptr, Vo.v, Vo.rv, sx, sy, ah, ch, bm,
                           __ldg(v.bus_meta2 + o), inj);
    }
  }
}

// pdl: k_tile is launched as a programmatic dependent of the stream's
// previous kernel (k_phasor_fx), so its CTAs start before that grid ends and
// load the static maps and the branch coefficients ahead of their wait for
// it; set only where no kernel that wrote those coefficients comes directly
// before it.  With t.fuse_phasor k_tile forms the records itself: it waits for
// the stream's previous kernel before it reads x, so that an evaluation's
// k_tile starts while the previous one's last tiles run (a persistent grid
// then takes its units by a static stride).
template <int ITEMS, bool WF, bool WJ, bool MASKED>
int launch_fused_t(const View &v, int num_sms, const pf_tuning &t, const EvalArgs &a, bool pdl, cudaStream_t s) {
  if (v.n_tile_units > 0) {
    const bool phx = t.fuse_phasor != 0;
    const int64_t grid = capped_grid(v.n_tile_units, t.ctas_per_sm, num_sms);
    EvalArgs ak = a;
    if (grid == v.n_tile_units || phx) ak.work = nullptr;   // one CTA per unit: the hardware schedules them
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = kTileSmemFixed + (phx ? kTileRecBytes : 0) + (WJ ? 8 * v.tile_stage : 0);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (phx) PF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tile<ITEMS, WF, WJ, MASKED, false, true>, v, ak));
    else if (ak.work) PF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tile<ITEMS, WF, WJ, MASKED, true, false>, v, ak));
    else PF_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tile<ITEMS, WF, WJ, MASKED, false, false>, v, ak));
  }
  if (v.n_large_units > 0) {
    const int64_t grid = capped_grid(v.n_large_units, t.ctas_per_sm, num_sms);
    k_fused_large<ITEMS, WF, WJ, MASKED><<<(unsigned)grid, 32, 0, s>>>(v, a);
    PF_CUDA_TRY(cudaGetLastError());
  }
  return PF_OK;
}

template <int ITEMS>
int launch_fused_items(const View &v, int num_sms, const pf_tuning &t, const EvalArgs &a, bool masked, bool pdl,
                       cudaStream_t s) {
  const bool wf = a.F != nullptr, wj = a.vals != nullptr;
  if (wf && wj)
    return masked ? launch_fused_t<ITEMS, true, true, true>(v, num_sms, t, a, pdl, s)
                  : launch_fused_t<ITEMS, true, true, false>(v, num_sms, t, a, pdl, s);
  if (wf)
    return masked ? launch_fused_t<ITEMS, true, false, true>(v, num_sms, t, a, pdl, s)
                  : launch_fused_t<ITEMS, true, false, false>(v, num_sms, t, a, pdl, s);
  return masked ? launch_fused_t<ITEMS, false, true, true>(v, num_sms, t, a, pdl, s)
                : launch_fused_t<ITEMS, false, true, false>(v, num_sms, t, a, pdl, s);
}

int launch_fused(const View &v, int num_sms, const pf_tuning &t, const EvalArgs &a, bool masked, cudaStream_t s,
                 bool pdl = true) {
  switch (t.tile_inc) {
    case 32: return launch_fused_items<1>(v, num_sms, t, a, masked, pdl, s);
    case 64: return launch_fused_items<2>(v, num_sms, t, a, masked, pdl, s);
    case 96: return launch_fused_items<3>(v, num_sms, t, a, masked, pdl, s);
    case 128: return launch_fused_items<4>(v, num_sms, t, a, masked, pdl, s);
    default: return fail(PF_ERR_INVALID, "tile_inc must be 32, 64, 96 or 128");
  }
}

// The view of the instances [i0, i1): their units are contiguous in the unit
// lists and their buses in the phasor scratch; every other index stays global.
View range_view(const Ctx &c, int i0, int i1) {
  View v = c.v;
  v.unit_rec = c.v.unit_rec + c.lane_off[i0];
  v.unit_info = c.v.unit_info + c.lane_off[i0];
  v.unit_ptr = c.v.unit_ptr + 2 * c.lane_off[i0];
  v.n_lane_units = c.lane_off[i1] - c.lane_off[i0];
  v.large_rec = c.v.large_rec + c.large_off[i0];
  v.n_large_units = c.large_off[i1] - c.large_off[i0];
  v.bus_inst_begin = c.bus_off[i0];
  v.n_bus_inst = c.bus_off[i1];
  const std::vector<int64_t> &toff = c.tiles[c.tuning.split_rounds].tile_off;
  v.tunit = c.v.tunit + 8 * toff[i0];
  v.n_tile_units = toff[i1] - toff[i0];
  return v;
}

void built_coefficients(const View &v, EvalArgs &a) {
  a.gb = v.inc_gb;
  a.ac = v.inc_ac;
  a.hat = v.bus_hat;
  a.pgb = v.pair_gb;
  a.pac = v.pair_ac;
  a.pgbx = v.pair_gbx;
}

__global__ void k_sincos(const double *__restrict__ t, int64_t n, const longlong2 *__restrict__ tabf,
                         double *__restrict__ c, double *__restrict__ sn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RectV r = rect_voltage(t[i], 1.0, tabf);
  c[i] = r.E.x;
  sn[i] = r.E.y;
}

}  // namespace

int launch_phasor(const View &v, int num_sms, const double *x, cudaStream_t s, bool fixed) {
  (void)num_sms;
  const int tb = 256;
  const int64_t blocks = (v.n_bus_inst - v.bus_inst_begin + tb - 1) / tb;
  if (blocks <= 0) return PF_OK;
  if (fixed && v.n_grids == 1) {
    // one grid: instances [i0, i1) of the range, a 2-D launch without instance lookup
    const int64_t nb = v.n_bus;
    const int64_t i0 = v.bus_inst_begin / nb, i1 = v.n_bus_inst / nb;
    const bool two = (nb % 2 == 0) && (v.grid1_nx % 2 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0);
    for (int64_t c0 = i0; c0 < i1; c0 += 65535) {
      const unsigned ni = (unsigned)std::min<int64_t>(65535, i1 - c0);
      if (two) k_phasor_fx2<<<dim3((unsigned)((nb / 2 + tb - 1) / tb), ni), tb, 0, s>>>(v, x, (int)c0);
      else k_phasor_fx<true><<<dim3((unsigned)((nb + tb - 1) / tb), ni), tb, 0, s>>>(v, x, (int)c0);
    }
  } else if (fixed) {
    k_phasor_fx<false><<<(unsigned)blocks, tb, 0, s>>>(v, x, 0);
  } else {
    k_phasor<<<(unsigned)blocks, tb, 0, s>>>(v, x);
  }
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

// Whether an evaluation launches the phasor kernel before the fused one.
bool needs_phasor_kernel(const Ctx &c) { return !c.tuning.fuse_phasor || c.v.n_large_units > 0; }

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
  a.work = c.work_ctr;
  built_coefficients(c.v, a);
  bool params = false;                           // per-call branch parameters
  if (ov) {
    a.p_inj = ov->p_inj;
    a.q_inj = ov->q_inj;
    a.status = ov->status;
    a.gen_mode = ov->gen_mode;
    a.gen_qlim = ov->gen_qlim;
    if (ov->gen_mode && !ov->gen_qlim) return fail(PF_ERR_INVALID, "gen_mode needs gen_qlim");
    if (ov->br_r || ov->br_x || ov->br_b || ov->br_tap) {
      params = true;
      if (stages & 2) {
        PF_TRY(compute_coefficients(c, ov->br_r, ov->br_x, ov->br_b, ov->br_tap, c.ov_gb, c.ov_ac, c.ov_hat, s));
        PF_TRY(permute_overrides(c, s));
      }
      a.gb = c.ov_gb;
      a.ac = c.ov_ac;
      a.hat = c.ov_hat;
      a.pgb = c.ov_pair_gb;
      a.pac = c.ov_pair_ac;
      a.pgbx = c.ov_pair_gbx;
    }
  }
  const bool masked = c.any_outage || a.status != nullptr;
  // (with the records formed in the fused kernel, the phasor kernel runs only
  // for the buses of more than 32 neighbours, whose kernel reads records)
  if ((stages & 1) && needs_phasor_kernel(c)) PF_TRY(launch_phasor(c.v, c.num_sms, x, s, true));
  if (!(stages & 2)) return PF_OK;
  // the fused stage alone with per-call branch parameters: the kernel that
  // wrote its coefficients comes directly before it
  return launch_fused(c.v, c.num_sms, c.tuning, a, masked, s, !(params && stages == 2));
}

// F and J of the instances [i0, i1): the units of those instances are
// contiguous in the unit lists, their buses contiguous in the phasor scratch.
int launch_eval_range(Ctx &c, int i0, int i1, const double *x, double *F, double *vals, cudaStream_t s) {
  if (!x) return fail(PF_ERR_INVALID, "x is NULL");
  if (i0 < 0 || i1 > c.v.n_inst || i0 >= i1) return fail(PF_ERR_INVALID, "bad instance range");
  if (!F && !vals) return PF_OK;
  const View v = range_view(c, i0, i1);
  EvalArgs a{};
  a.x = x;
  a.F = F;
  a.vals = vals;
  a.work = c.work_ctr;
  built_coefficients(c.v, a);
  if (needs_phasor_kernel(c)) PF_TRY(launch_phasor(v, c.num_sms, x, s, true));
  return launch_fused(v, c.num_sms, c.tuning, a, c.any_outage, s);
}

// Evaluation with caller-provided phasor scratch (used by the allocation-free
// entry point, whose scratch is a static device array).
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
  a.work = c.work_ctr;
  built_coefficients(c.v, a);
  if (needs_phasor_kernel(c)) PF_TRY(launch_phasor(v, c.num_sms, x, s, true));
  return launch_fused(v, c.num_sms, c.tuning, a, c.any_outage, s);
}

// The phasor routine alone, for verification against a reference sin / cos.
int launch_sincos(Ctx &c, const double *t, int64_t n, double *cs, double *sn, cudaStream_t s) {
  if (n <= 0) return PF_OK;
  if (!t || !cs || !sn) return fail(PF_ERR_INVALID, "NULL argument");
  k_sincos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, n, c.v.sincos_fix, cs, sn);
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

}  // namespace pf
