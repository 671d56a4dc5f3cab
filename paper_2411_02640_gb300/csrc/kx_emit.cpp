// CUDA source emitter: turns one mechanism into per-point kernels for
// sm_103a, specialised to that mechanism.
//
// On GB300 the float64 pipe is the scarce unit (about 2 DFMA per clock per
// SM, against 128 float32 lanes), so float64 ACCURACY is produced off the
// float64 pipe wherever the error bars allow:
//
//  * Production rates, default (emit_rates_class_df): double-float (float32
//    pair) arithmetic in log space.  Reactions are grouped into classes of
//    one code shape (kind, reversibility, blend, reactant and product entry
//    counts); each class is one loop over per-class constant tables
//    (Arrhenius triples, packed species/coefficient entries, efficiencies,
//    blend parameters) with a straight-line body.  Per state: one ln T and
//    1/T, ln |C_k| and mu_k = G_k/RT + ln |C_k| (Eq. (Ck)); per reaction
//    ln k_f (Eq. (k_f)), the falloff blend, ln |R_f| and the log ratio
//    ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T)) (Eq. (K_p)); the net
//    rate from the larger rate and that ratio; wdot accumulated in float
//    pairs under a per-state power-of-two scale.  A reaction whose rates
//    are below 2^-40 of the scale's anchor for every state of a warp (a
//    warp vote on float32 estimates) is evaluated in float32 instead: its
//    error, bounded by its size, stays orders of magnitude under the
//    float-pair path's own.  The tables make the compile time independent
//    of the mechanism's size.
//  * Production rates, warp-cooperative (emit_wdot_wc; small batches): the
//    lanes of a warp share a state, species vectors and per-reaction rates
//    in shared memory, wdot gathered species-major; the same float32 path
//    per round of reactions.
//  * Adjoint (emit_vjp_df one thread per state, emit_vjp_wc one warp per
//    state): v^T d wdot/d(T, Y) in double-float arithmetic, each term a
//    float-pair mantissa times a power of two under its own running scale.
//  * Production rates, native float64 (rates_arith = 1, emit_rates64): one
//    thread per point, fully unrolled, constants as immediates (the paper's
//    per-thread model, Sec. 2.4): one ln T and 1/T shared by every
//    Arrhenius term, the special cases of Eq. (k_f) and one shared
//    exponential for reactions with equal (beta, E) emitted next to each
//    other; k_r = exp(ln k_f - ln K_c), or the paper's per-species
//    exp(-G/RT) products with one division (kc_mode = 1); float64 exp/log
//    of our own (table-driven, Tang's method).  Table-driven above 64
//    species or 400 reactions.
//  * Transport (emit_transport): loops over per-species and per-pair
//    coefficient tables, double-float by default; Wilke's sum over
//    unordered pairs (phi_jk from phi_kj), symmetric D_kj evaluated once per
//    pair and added to both rows.
//  * Thermo (emit_thermo): two float-pair Horner evaluations per species.
//
// The mixed-precision production rates (KX_MIXED) run the same class loops
// with a float32 body for the Arrhenius, third-body and falloff arithmetic;
// the Gibbs sums of ln K_c stay in float pairs (through the species
// chemical potentials G_k/RT + ln C_k), the forward/reverse cancellation is
// resolved from that ratio and wdot is accumulated in float64
// (emit_class_mixed_body; the fully unrolled form is emit_rates_mixed).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <sstream>
#include <tuple>

#include "kx_internal.h"

namespace kx {

const char* kTables =
#include "kx_tables.inc"
    ;

const char* kDevicePrelude = R"KXPRE(
#define KX_INF __longlong_as_double(0x7ff0000000000000LL)
#define KX_NAN __longlong_as_double(0x7ff8000000000000LL)
#define KX_INV_LN10 0.43429448190325182765
#define KX_LN10 2.30258509299404568402
#define KX_LOG2E_F 1.44269504f
#define KX_RND_F 12582912.0f          /* 1.5 * 2^23: adding it rounds a float to an integer */

// Conversions between float64 and float32 by integer operations: on this
// GPU the F2F/I2F conversions issue on the float64 pipe, which is the
// bottleneck, while integer ops go to the ALU pipe.
// Round-to-nearest float of a double within float's normal range; |x| below
// it gives 0, above it (and nan) gives +-inf.
__device__ __forceinline__ float kx_d2f(double x) {
  const long long b = __double_as_longlong(x) + (1LL << 28);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  const unsigned sgn = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sgn);
  if (e >= 255) return __uint_as_float(sgn | 0x7f800000u);
  return __uint_as_float(sgn | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | ((unsigned)b >> 29));
}
// Exact double of a normal float (zero and subnormals give 0).
__device__ __forceinline__ double kx_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}
// Nearest integer of a float with |t| < 2^22, without the XU pipe.
__device__ __forceinline__ int kx_rint(float t) { return __float_as_int(t + KX_RND_F) - 0x4b400000; }
// Float of an integer with |n| < 2^22, without the conversion unit.
__device__ __forceinline__ float kx_i2f(int n) { return __int_as_float(0x4b400000 + n) - KX_RND_F; }

#if KX_T64
__shared__ double kx_s_exp[256];
__shared__ double kx_s_log[1024];
// float64 exp: x = k ln2/256 + r with k = rint(x 256/ln2) found in float32
// and r by a two-constant Cody-Waite reduction in float64; e^r - 1 =
// r + r^2 q(r) with the short tail q in float32 (|r^2 q| < 1.1e-6, so its
// float32 rounding is below 1e-13 relative); 2^(j/256) from a shared table
// and 2^(k>>8) by an exponent-field add.  |x| >= 700, inf and nan take the
// library path.
__device__ __forceinline__ double kx_exp(double x) {
#ifdef KX_LIBMATH
  return exp(x);
#else
  if (!(fabs(x) < 700.0)) return exp(x);
  const int k = kx_rint(kx_d2f(x) * KX_256_OVER_LN2F);
  const double kd = (double)k;
  double r = fma(kd, -KX_LN2_256_HI, x);
  r = fma(kd, -KX_LN2_256_LO, r);
  const float rf = kx_d2f(r);
  const float qf = fmaf(fmaf(fmaf(rf, 8.33333333e-3f, 4.16666667e-2f), rf, 0.166666667f), rf, 0.5f);
  const double s = fma(r * r, kx_f2d(qf), r);
  const double tj = kx_s_exp[k & 255];
  const double v = fma(tj, s, tj);
  return __hiloint2double(__double2hiint(v) + (int)((unsigned)(k >> 8) << 20), __double2loint(v));
#endif
}

// float64 natural log: x = 2^e m, m in [1,2); c = 1 + (2j+1)/512 is the
// centre of m's cell, r = (m - c)/c with 1/c from the table, and
// log1p(r) = r - r^2 q(r) with the tail q in float32 (|r^2 q| < 2e-6).
// Zero, negative, subnormal, inf and nan inputs take the library path.
__device__ __forceinline__ double kx_log(double x) {
#ifdef KX_LIBMATH
  return log(x);
#else
  if (!(x >= 2.2250738585072014e-308 && x < KX_INF)) return log(x);
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) - 1023;
  const int j = (hi >> 12) & 0xff;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(x));
  const double r = (m - kx_s_log[4 * j]) * kx_s_log[4 * j + 1];
  const float rf = kx_d2f(r);
  const float qf = fmaf(fmaf(fmaf(rf, -0.2f, 0.25f), rf, -0.333333333f), rf, 0.5f);
  const double t = fma(-(r * r), kx_f2d(qf), r);
  const double ed = (double)e;
  return fma(ed, KX_LN2_HI, kx_s_log[4 * j + 2]) + (fma(ed, KX_LN2_LO, kx_s_log[4 * j + 3]) + t);
#endif
}

#endif  // KX_T64

// fac * 2^t as a float64 for |t| up to ~1100 and fac in [0, 1]: the
// mantissa comes from float32 exp2 of t minus its nearest integer n, the
// power 2^n is added to the float64 exponent field (no float64 arithmetic).
__device__ __forceinline__ double kx_pow2_scaled(float t, float fac) {
  if (!(t > -4000.0f && t < 4000.0f)) {
    if (t != t || fac != fac) return KX_NAN;
    return (t > 0.0f && fac > 0.0f) ? KX_INF : 0.0;
  }
  const float tr = t + KX_RND_F;
  const int n = __float_as_int(tr) - 0x4b400000;
  const float m = exp2f(t - (tr - KX_RND_F)) * fac;
  if (!(m >= 0.0f)) return KX_NAN;
  const double dm = kx_f2d(m);
  const int hi = __double2hiint(dm);
  const int E = ((hi >> 20) & 0x7ff) + n;
  if (m == 0.0f || E <= 0) return 0.0;
  if (E >= 0x7ff) return KX_INF;
  return __hiloint2double(hi + (int)((unsigned)n << 20), __double2loint(dm));
}

// Net rate of progress R_f - R_r from ln R_f (float32) and the float64
// log-ratio ln(R_r/R_f): the larger of the two rates times
// (1 - smaller/larger) = -expm1(-|ln ratio|), so the cancellation near
// equilibrium is resolved from the float64 ratio, not by subtracting two
// rounded rates.
__device__ __forceinline__ double kx_net_rate(float lnRf, double lnrho) {
  const float a = kx_d2f(lnrho);
  const float e = lnRf + fmaxf(a, 0.0f);
  const float fac = -expm1f(-fabsf(a));
  const double mag = kx_pow2_scaled(e * KX_LOG2E_F, fac);
  return a > 0.0f ? -mag : mag;
}

// Net rate of progress from ln |R_f| and a = ln(|R_r|/|R_f|) (float32, a
// rounded once from its float-pair sum), with the signs sf, sr (1: negative)
// of the two rates: the larger magnitude times 1 - e^-|a| for equal signs
// (the cancellation near equilibrium resolved from a) or 1 + e^-|a| for
// opposite signs.
__device__ __forceinline__ double kx_net_rate_s(float lnRf, float a, int sf, int sr) {
  const float e = lnRf + fmaxf(a, 0.0f);
  const float fac = sf == sr ? -expm1f(-fabsf(a)) : 1.0f + __expf(-fabsf(a));
  const double mag = kx_pow2_scaled(e * KX_LOG2E_F, fac);
  const int neg = sf == sr ? ((a > 0.0f) != (sf != 0)) : sf;
  return neg ? -mag : mag;
}

// ln(Pr/(1+Pr)) and ln(1/(1+Pr)) from ln Pr without overflow (float32).
__device__ __forceinline__ float kx_ln_pr_ratio(float lnPr) {
  return lnPr < 0.0f ? lnPr - log1pf(__expf(lnPr)) : -log1pf(__expf(-lnPr));
}
__device__ __forceinline__ float kx_ln_inv_1p(float lnPr) {
  return lnPr < 0.0f ? -log1pf(__expf(lnPr)) : -(lnPr + log1pf(__expf(-lnPr)));
}

#if KX_TDF
__shared__ float2 kx_s_dexp[256];
#endif
#if KX_TDFR
__shared__ float4 kx_s_dlog[256];
#endif
__device__ __forceinline__ void kx_load_tables() {
#if KX_T64 && !defined(KX_LIBMATH)
  for (int t = threadIdx.x; t < 256; t += blockDim.x) kx_s_exp[t] = kx_exp2_tab[t];
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) kx_s_log[t] = kx_log_tab[t];
#endif
#if KX_TDF
  for (int t = threadIdx.x; t < 256; t += blockDim.x) kx_s_dexp[t] = kx_dexp2_tab[t];
#endif
#if KX_TDFR
  for (int t = threadIdx.x; t < 256; t += blockDim.x) kx_s_dlog[t] = kx_dlog_tab[t];
#endif
  __syncthreads();
}

// ---- double-float (float32 pair) arithmetic for float64-accurate work on
// the float32 pipe.  Error-free transformations after Knuth (two-sum),
// Dekker (fast two-sum) and the FMA two-product; the __f*_rn intrinsics keep
// the compiler from contracting or reassociating them.
struct kx_df { float hi, lo; };
__device__ __forceinline__ kx_df kx_mk(float h, float l) { kx_df r; r.hi = h; r.lo = l; return r; }
__device__ __forceinline__ kx_df kx_qts(float a, float b) {      // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return kx_mk(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ kx_df kx_ts(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return kx_mk(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// a*b + c
__device__ __forceinline__ kx_df kx_df_fma(kx_df a, kx_df b, kx_df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const kx_df s = kx_ts(p, c.hi);
  return kx_qts(s.hi, __fadd_rn(s.lo, __fadd_rn(pe, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, c.lo)))));
}
// a*b + c without the final renormalisation (inner Horner steps and running
// sums: the next step only needs hi + lo, not |lo| <= ulp(hi)/2)
__device__ __forceinline__ kx_df kx_df_fma_u(kx_df a, kx_df b, kx_df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const kx_df s = kx_ts(p, c.hi);
  return kx_mk(s.hi, __fadd_rn(s.lo, __fadd_rn(pe, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, c.lo)))));
}
__device__ __forceinline__ kx_df kx_df_mul(kx_df a, kx_df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return kx_qts(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p))));
}
// a*b without the final renormalisation (an operand of a further product or running sum)
__device__ __forceinline__ kx_df kx_df_mul_u(kx_df a, kx_df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return kx_mk(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p))));
}
__device__ __forceinline__ double kx_df2d(kx_df a) { return kx_f2d(a.hi) + kx_f2d(a.lo); }
// a / b: a reciprocal estimate refined by one Newton step, then one
// correction of the quotient from the exact remainder a - q1 b
__device__ __forceinline__ kx_df kx_df_div(kx_df a, kx_df b) {
  float rb = __fdividef(1.0f, b.hi);
  rb = __fmaf_rn(rb, __fmaf_rn(-b.hi, rb, 1.0f), rb);
  const float q1 = __fmul_rn(a.hi, rb);
  const float p = __fmul_rn(q1, b.hi);
  const float pe = __fmaf_rn(q1, b.hi, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), __fmaf_rn(-q1, b.lo, a.lo));
  return kx_qts(q1, __fmul_rn(r, rb));
}
// 1/sqrt(x) of a positive float pair: the float32 estimate y, r = 1 - x y^2 in
// float pairs (y^2 as an exact product pair), y (1 + r/2 + 3r^2/8)
__device__ __forceinline__ kx_df kx_df_rsqrt(kx_df x) {
  const float y = rsqrtf(x.hi);
  const float p = __fmul_rn(y, y);
  const kx_df xy2 = kx_df_mul(x, kx_mk(p, __fmaf_rn(y, y, -p)));
  const float r = __fadd_rn(__fsub_rn(1.0f, xy2.hi), -xy2.lo);
  return kx_qts(y, __fmul_rn(y, __fmaf_rn(__fmul_rn(0.375f, r), r, __fmul_rn(0.5f, r))));
}
__device__ __forceinline__ kx_df kx_d2df(double x) {
  const float h = kx_d2f(x);
  return kx_mk(h, kx_d2f(x - kx_f2d(h)));
}
#if KX_TDF
// e^x of a double-float x: x = k ln2/256 + r (k from the high part in
// float32, ln2/256 split in three floats, the first short enough that k C1
// is exact), e^r = 1 + r + r^2 q(r) with the tail in float32, times
// 2^(j/256) from a float-pair table and 2^(k>>8) as an exact float scale.
// Relative error about 1e-13; |x| >= 80 (and nan) go through float64.
__device__ __forceinline__ kx_df kx_df_exp(kx_df x) {
  if (!(fabsf(x.hi) < 80.0f)) return kx_d2df(exp(kx_df2d(x)));
  const float tk = __fmaf_rn(x.hi, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_C1F, x.hi);
  const float p = __fmul_rn(kf, KX_C2F);
  const float pe = __fmaf_rn(kf, KX_C2F, -p);
  kx_df r = kx_ts(t1, -p);
  r = kx_qts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, KX_C3F))));
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df s = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  s = kx_qts(s.hi, __fadd_rn(s.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  const kx_df v = kx_df_fma_u(kx_mk(tj.x, tj.y), s, kx_mk(tj.x, tj.y));   // unnormalised: feeds products and sums
  const float sc = __int_as_float(((k >> 8) + 127) << 23);
  return kx_mk(__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc));
}

// e^x of a float64 x with two float64 operations: x is split into a float
// pair (one subtraction), the reduction x = k ln2/256 + r and e^r 2^(j/256)
// run in double-float arithmetic on the float32 pipe (ln2/256 split in three
// floats, the first of 5 significant bits so that k E1 is exact for
// |k| < 2^19), the float-pair mantissa returns to float64 (one addition) and
// 2^(k>>8) is an exponent-field add.  Relative error about 2e-12 (the
// 48-bit float pair that holds x), used where the error bar allows it.
__device__ __forceinline__ double kx_exp_r(double x) {
#ifdef KX_LIBMATH
  return exp(x);
#else
  if (!(fabs(x) < 700.0)) return exp(x);
  const float xh = kx_d2f(x);
  const float xl = kx_d2f(x - kx_f2d(xh));
  const float tk = __fmaf_rn(xh, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_E1F, xh);
  const float p = __fmul_rn(kf, KX_E2F);
  const float pe = __fmaf_rn(kf, KX_E2F, -p);
  kx_df r = kx_ts(t1, -p);
  r = kx_qts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(xl, pe), __fmul_rn(kf, KX_E3F))));
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df sv = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  sv = kx_qts(sv.hi, __fadd_rn(sv.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  const kx_df v = kx_df_fma(kx_mk(tj.x, tj.y), sv, kx_mk(tj.x, tj.y));
  const double vd = kx_f2d(v.hi) + kx_f2d(v.lo);
  return __hiloint2double(__double2hiint(vd) + (int)((unsigned)(k >> 8) << 20), __double2loint(vd));
#endif
}
#endif  // KX_TDF

#if KX_TDFR
// ---- double-float arithmetic for the float64-accurate production rates
// (log-space rates on the float32 pipe; the few float64 operations left are
// the final conversion of each production rate).
#define KX_INF_F __int_as_float(0x7f800000)
// a + b (error about 2^-47 (|a| + |b|))
__device__ __forceinline__ kx_df kx_df_add(kx_df a, kx_df b) {
  const kx_df s = kx_ts(a.hi, b.hi);
  return kx_qts(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// a + b without the final renormalisation: the high parts summed exactly
// (two-sum), the low parts and the rounding error added once.  For running
// sums that are renormalised (kx_ts) or converted (hi + lo) once at the end.
__device__ __forceinline__ kx_df kx_df_add_u(kx_df a, kx_df b) {
  const kx_df s = kx_ts(a.hi, b.hi);
  return kx_mk(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ kx_df kx_df_norm(kx_df a) { return kx_ts(a.hi, a.lo); }
__device__ __forceinline__ kx_df kx_df_neg(kx_df a) { return kx_mk(-a.hi, -a.lo); }
__device__ __forceinline__ kx_df kx_df_sub(kx_df a, kx_df b) { return kx_df_add(a, kx_df_neg(b)); }
// a b with b a float
__device__ __forceinline__ kx_df kx_df_mulf(kx_df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return kx_qts(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
// Float pair of a double: the high part keeps 24 significant bits
// (truncation), the low part the remaining 29 bits rounded once.  Values
// below float's normal range give 0; above it, +-inf (nan stays nan).
__device__ __forceinline__ kx_df kx_d2df_i(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -126) return kx_mk(0.0f, 0.0f);
  if (e > 127) return kx_mk(__double2float_rn(x), 0.0f);
  const unsigned sgn = (unsigned)hi & 0x80000000u;
  const float h = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29));
  const unsigned r29 = lo & 0x1fffffffu;
  const float l = __fmaf_rn(__fsub_rn(__int_as_float(0x4b000000 | (int)(r29 >> 6)), 8388608.0f), 0x1p-46f,
                            __fmul_rn(__fsub_rn(__int_as_float(0x4b000000 | (int)(r29 & 63u)), 8388608.0f), 0x1p-52f));
  return kx_mk(h, __uint_as_float(sgn | __float_as_uint(__fmul_rn(l, __int_as_float((e + 127) << 23)))));
}
// e ln2 + log(c_j) + log1p((m - c_j)/c_j) for a positive value 2^e m, m =
// mh + ml in [1, 2) with its top 8 fraction bits j (Tang's table-driven log
// with a float-pair table of 1/c_j and log c_j; |r| <= 1/512, the r^2/2 term
// exact as a product pair, the rest of the series in float32, below 3e-9).
__device__ __forceinline__ kx_df kx_df_log_core(int e, int j, float mh, float ml) {
  const float c = __int_as_float(0x3f800000 | ((2 * j + 1) << 14));
  const float4 t = kx_s_dlog[j];
  const kx_df d = kx_qts(__fsub_rn(mh, c), ml);
  const float rh = __fmul_rn(d.hi, t.x);
  const float rl = __fmaf_rn(d.hi, t.y, __fmaf_rn(d.lo, t.x, __fmaf_rn(d.hi, t.x, -rh)));
  const float hr = __fmul_rn(-0.5f, rh);
  const float h2 = __fmul_rn(hr, rh);
  const float h2e = __fmaf_rn(hr, rh, -h2);
  const float p = __fmaf_rn(__fmaf_rn(__fmaf_rn(rh, -0.166666672f, 0.2f), rh, -0.25f), rh, 0.333333343f);
  const float tail = __fmul_rn(__fmul_rn(__fmul_rn(rh, rh), rh), p);
  const kx_df l1 = kx_qts(rh, h2);
  const float l1lo = __fadd_rn(l1.lo, __fadd_rn(__fadd_rn(rl, h2e), __fmaf_rn(-rh, rl, tail)));
  const float ef = __fsub_rn(__int_as_float(0x4b400000 + e), KX_RND_F);
  const float a1 = __fmul_rn(ef, KX_LN2_1F);
  const float p2 = __fmul_rn(ef, KX_LN2_2F);
  const float p2e = __fmaf_rn(ef, KX_LN2_2F, -p2);
  const kx_df s = kx_ts(a1, t.z);
  const kx_df u = kx_ts(s.hi, p2);
  const kx_df v = kx_ts(u.hi, l1.hi);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s.lo, u.lo), __fadd_rn(v.lo, p2e)),
                             __fadd_rn(__fmaf_rn(ef, KX_LN2_3F, t.w), l1lo));
  return kx_qts(v.hi, lo);
}
// ln x of a positive normal double
__device__ __forceinline__ kx_df kx_df_log_d(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned r29 = lo & 0x1fffffffu;
  const float mh = __int_as_float(0x3f800000 | ((hi & 0xfffff) << 3) | (int)(lo >> 29));
  const float ml = __fmaf_rn(__fsub_rn(__int_as_float(0x4b000000 | (int)(r29 >> 6)), 8388608.0f), 0x1p-46f,
                             __fmul_rn(__fsub_rn(__int_as_float(0x4b000000 | (int)(r29 & 63u)), 8388608.0f), 0x1p-52f));
  return kx_df_log_core((hi >> 20) - 1023, (hi >> 12) & 0xff, mh, ml);
}
// ln x of a float pair; x.hi must be positive and normal, else -1e4 is
// returned, a stand-in for ln 0 that every caller clamps
__device__ __forceinline__ kx_df kx_df_log(kx_df x) {
  if (!(x.hi >= 1.17549435e-38f && x.hi < KX_INF_F)) return kx_mk(-1.0e4f, 0.0f);
  const int b = __float_as_int(x.hi);
  const int e = (b >> 23) - 127;
  const float mh = __int_as_float((b & 0x7fffff) | 0x3f800000);
  const float ml = __fmul_rn(x.lo, __int_as_float((127 - e) << 23));
  return kx_df_log_core(e, (b >> 15) & 0xff, mh, ml);
}
// e^x of a float pair as a float pair: 0 for x <= -87, inf for x >= 88.7
// (reduction and tail as in kx_df_exp)
__device__ __forceinline__ kx_df kx_df_exp_s(kx_df x) {
  if (!(x.hi > -87.0f)) return kx_mk(0.0f, 0.0f);
  if (!(x.hi < 88.7f)) return kx_mk(KX_INF_F, 0.0f);
  const float tk = __fmaf_rn(x.hi, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_C1F, x.hi);
  const float p = __fmul_rn(kf, KX_C2F);
  const float pe = __fmaf_rn(kf, KX_C2F, -p);
  kx_df r = kx_ts(t1, -p);
  r = kx_qts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, KX_C3F))));
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df s = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  s = kx_qts(s.hi, __fadd_rn(s.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  const kx_df v = kx_df_fma(kx_mk(tj.x, tj.y), s, kx_mk(tj.x, tj.y));
  const float sc = __int_as_float(((k >> 8) + 127) << 23);
  return kx_mk(__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc));
}
// e^x of a non-positive float pair (the upper range test of kx_df_exp_s drops out); x may be
// unnormalised (|x.lo| a few ulp of x.hi)
__device__ __forceinline__ kx_df kx_df_exp_n(kx_df x) {
  if (!(x.hi > -87.0f)) return kx_mk(0.0f, 0.0f);
  const float tk = __fmaf_rn(x.hi, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_C1F, x.hi);
  const float p = __fmul_rn(kf, KX_C2F);
  const float pe = __fmaf_rn(kf, KX_C2F, -p);
  kx_df r = kx_ts(t1, -p);
  r = kx_ts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, KX_C3F))));   // x.lo may exceed r.hi: two-sum
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df s = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  s = kx_qts(s.hi, __fadd_rn(s.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  const kx_df v = kx_df_fma(kx_mk(tj.x, tj.y), s, kx_mk(tj.x, tj.y));
  const float sc = __int_as_float(((k >> 8) + 127) << 23);
  return kx_mk(__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc));
}
// e^x 2^-S of a float pair as a float pair, S an integer with |S| <= 1100 and
// Sl = S ln2 in float32 (for the range test only): 0 where x - S ln2 <= -87,
// inf where it is >= 88.7.  The reduction x = k ln2/256 + r takes x itself
// (|x| < 830 there, so |k| < 2^19 and the 5-bit first part of ln2/256 keeps
// k E1 exact); S is subtracted from the power of two.
__device__ __forceinline__ kx_df kx_df_exp_sc(kx_df x, int S, float Sl) {
  const float xs = __fsub_rn(x.hi, Sl);
  if (!(xs > -87.0f)) return kx_mk(0.0f, 0.0f);
  if (!(xs < 88.7f)) return kx_mk(KX_INF_F, 0.0f);
  const float tk = __fmaf_rn(x.hi, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_E1F, x.hi);
  const float p = __fmul_rn(kf, KX_E2F);
  const float pe = __fmaf_rn(kf, KX_E2F, -p);
  kx_df r = kx_ts(t1, -p);
  r = kx_ts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, KX_E3F))));   // x.lo may exceed r.hi: two-sum
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df s = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  s = kx_qts(s.hi, __fadd_rn(s.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  const kx_df v = kx_df_fma_u(kx_mk(tj.x, tj.y), s, kx_mk(tj.x, tj.y));   // unnormalised: feeds products and sums
  const float sc = __int_as_float(((k >> 8) - S + 127) << 23);
  return kx_mk(__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc));
}
// e^x of a float pair as v 2^p: v a float pair in [1, 2) (unnormalised), p the
// integer power of two of the reduction x = k ln2/256 + r (p = k >> 8).
// x <= -760 gives v = 0 and p = -2000 (below every float64); x >= 720 gives
// v = inf and p = 1100 (above every float64); nan gives 0.  |x| < 760 keeps
// |k| < 2^19, so the 5-bit first part of ln2/256 keeps k E1 exact.
__device__ __forceinline__ kx_df kx_df_exp_m(kx_df x, int& p) {
  if (!(x.hi > -760.0f)) { p = -2000; return kx_mk(0.0f, 0.0f); }
  if (!(x.hi < 720.0f)) { p = 1100; return kx_mk(KX_INF_F, 0.0f); }
  const float tk = __fmaf_rn(x.hi, KX_256_OVER_LN2F, KX_RND_F);
  const int k = __float_as_int(tk) - 0x4b400000;
  const float kf = __fsub_rn(tk, KX_RND_F);
  const float t1 = __fmaf_rn(-kf, KX_E1F, x.hi);
  const float pp = __fmul_rn(kf, KX_E2F);
  const float pe = __fmaf_rn(kf, KX_E2F, -pp);
  kx_df r = kx_ts(t1, -pp);
  r = kx_ts(r.hi, __fadd_rn(r.lo, __fsub_rn(__fsub_rn(x.lo, pe), __fmul_rn(kf, KX_E3F))));   // x.lo may exceed r.hi: two-sum
  const float q = __fmaf_rn(__fmaf_rn(__fmaf_rn(r.hi, 8.33333333e-3f, 4.16666667e-2f), r.hi, 0.166666667f), r.hi, 0.5f);
  kx_df s = kx_qts(r.hi, __fmul_rn(__fmul_rn(r.hi, r.hi), q));
  s = kx_qts(s.hi, __fadd_rn(s.lo, r.lo));
  const float2 tj = kx_s_dexp[k & 255];
  p = k >> 8;
  return kx_df_fma_u(kx_mk(tj.x, tj.y), s, kx_mk(tj.x, tj.y));   // unnormalised: feeds products and sums
}
// Element k of a per-thread vector kept in global scratch at stride s.
template <typename V> struct kx_strided {
  V* p;
  long long s;
  __device__ __forceinline__ V& operator[](int k) const { return p[(long long)k * s]; }
};
// nu q for a coefficient nu in {-2, -1, 1, 2}: an exact scaling of both parts
// (larger coefficients take the float-pair product kx_df_mulf)
__device__ __forceinline__ kx_df kx_df_scale2(kx_df q, float nu) { return kx_mk(__fmul_rn(q.hi, nu), __fmul_rn(q.lo, nu)); }
// (a.hi + a.lo) 2^S as a double: one float64 addition, the power of two
// added to the exponent field (ldexp only when the result leaves the normal
// range)
__device__ __forceinline__ double kx_df2d_s(kx_df a, int S) {
  if (a.hi == 0.0f && a.lo == 0.0f) return 0.0;   // (an unnormalised sum may hold its value in lo alone)
  if (!(fabsf(a.hi) < KX_INF_F)) return (double)a.hi;
  const double d = kx_f2d(a.hi) + kx_f2d(a.lo);
  if (d == 0.0) return 0.0;
  const int hi = __double2hiint(d);
  const int E = ((hi >> 20) & 0x7ff) + S;
  if (E > 0 && E < 0x7ff) return __hiloint2double(hi + (int)((unsigned)S << 20), __double2loint(d));
  return ldexp(d, S);
}
// ln(1 + y) for 0 <= y <= 1 (absolute error about 1e-15)
__device__ __forceinline__ kx_df kx_df_log1p(kx_df y) {
  const kx_df s = kx_qts(1.0f, y.hi);
  return kx_df_log(kx_qts(s.hi, __fadd_rn(s.lo, y.lo)));
}
#endif  // KX_TDFR
)KXPRE";

// Device helpers of the adjoint kernels only (emitted after the common prelude in those kernels,
// so that the other kernels' sources, and their source hashes, do not carry them).
const char* kAdjointPrelude = R"KXADJ(
// m1 2^e1 - m2 2^e2 as a float pair times 2^e, e = max(e1, e2): the term with the smaller power of
// two is brought to the larger's (dropped below 2^-126 of it), then one float-pair subtraction.  In
// double-float arithmetic this is as accurate as forming the difference from the log-ratio of the two
// terms: both lose relative precision as 1/|ln(m1 2^e1 / m2 2^e2)| near cancellation, from the
// absolute error of the logarithms the terms come from.
__device__ __forceinline__ kx_df kx_df_sub_m(kx_df m1, int e1, kx_df m2, int e2, int& e) {
  e = max(e1, e2);
  const int d1 = e1 - e, d2 = e2 - e;
  const float s1 = d1 >= -126 ? __int_as_float((d1 + 127) << 23) : 0.0f;
  const float s2 = d2 >= -126 ? __int_as_float((d2 + 127) << 23) : 0.0f;
  return kx_df_sub(kx_mk(__fmul_rn(m1.hi, s1), __fmul_rn(m1.lo, s1)), kx_mk(__fmul_rn(m2.hi, s2), __fmul_rn(m2.lo, s2)));
}
// A running sum as a float pair under its own scale 2^-s, 16 bytes (one load and one store).
struct __align__(16) kx_acc { float hi, lo; int s, pad; };
__device__ __forceinline__ void kx_acc_add(kx_df& acc, int& s, kx_df m, int e);
__device__ __forceinline__ void kx_acc_add(kx_acc& a, kx_df m, int e) {
  kx_acc t = a;
  kx_df v = kx_mk(t.hi, t.lo);
  int s = t.s;
  kx_acc_add(v, s, m, e);
  t.hi = v.hi; t.lo = v.lo; t.s = s;
  a = t;
}
// acc 2^s += m 2^e for a running sum kept as a float pair under its own
// scale 2^-s (s = -100000: empty).  m is first brought to [1, 2) (its power
// of two moved into e); a term that would land above 2^96 raises the scale
// so that it sits at 2^62 (the sum rescaled by the exact power of two); a
// term under 2^-126 of the scale drops out; inf and nan propagate.
__device__ __forceinline__ void kx_acc_add(kx_df& acc, int& s, kx_df m, int e) {
  const float ah = fabsf(m.hi);
  if (!(ah < KX_INF_F)) { acc = kx_mk(m.hi, 0.0f); if (s < e) s = e; return; }
  if (ah == 0.0f) return;
  const int eh = max((int)((__float_as_uint(ah) >> 23) & 0xffu) - 127, -126);
  const int h1 = eh >> 1, h2 = eh - h1;   // 2^-eh in two exact steps (|h1|, |h2| <= 64)
  const float n1 = __int_as_float((127 - h1) << 23), n2 = __int_as_float((127 - h2) << 23);
  m = kx_mk(__fmul_rn(__fmul_rn(m.hi, n1), n2), __fmul_rn(__fmul_rn(m.lo, n1), n2));
  e += eh;
  if (e > s + 96) {
    const int d = s - (e - 62);
    const float f = d >= -126 ? __int_as_float((d + 127) << 23) : 0.0f;
    acc = kx_mk(__fmul_rn(acc.hi, f), __fmul_rn(acc.lo, f));
    s = e - 62;
  }
  const int d = e - s;
  if (d >= -126) {
    const float sc = __int_as_float((d + 127) << 23);
    acc = kx_df_add_u(acc, kx_mk(__fmul_rn(m.hi, sc), __fmul_rn(m.lo, sc)));
  }
}
)KXADJ";

namespace {

// ------------------------------------------------------------------ text helpers
std::string fmt(const char* f, ...) {
  va_list ap, ap2;
  va_start(ap, f);
  va_copy(ap2, ap);
  const int n = vsnprintf(nullptr, 0, f, ap);
  va_end(ap);
  std::string out(n > 0 ? n : 0, '\0');
  if (n > 0) vsnprintf(&out[0], n + 1, f, ap2);
  va_end(ap2);
  return out;
}

// float64 literal that reads back bit-exactly
std::string D(double v) {
  if (std::isnan(v)) return "KX_NAN";
  if (std::isinf(v)) return v > 0 ? "KX_INF" : "(-KX_INF)";
  std::string s = fmt("%.17g", v);
  if (s.find_first_of(".en") == std::string::npos) s += ".0";
  return s[0] == '-' ? "(" + s + ")" : s;
}

// float32 literal (value rounded to float first)
std::string F(double v) {
  float f = (float)v;
  if (std::isinf(f)) return v > 0 ? "__int_as_float(0x7f800000)" : "(-__int_as_float(0x7f800000))";
  std::string s = fmt("%.9g", (double)f);
  if (s.find_first_of(".en") == std::string::npos) s += ".0";
  s += "f";
  return s[0] == '-' ? "(" + s + ")" : s;
}

std::string fpair(double v) {
  const float h = (float)v;
  const float l = (float)(v - (double)h);
  return F(h) + "," + F(l);
}

std::string DFc(double v) { return "kx_mk(" + fpair(v) + ")"; }

// float32-pipe instruction estimates of the double-float primitives (for the
// operation counts)
constexpr double kDfAdd = 11, kDfMul = 7, kDfFma = 15, kDfMulf = 5, kDfDiv = 16, kDfExp = 30, kDfLog = 40;

struct Out {
  std::ostringstream o;
  int ind = 1;
  void operator()(const std::string& s) { o << std::string(2 * ind, ' ') << s << "\n"; }
};

bool is_small_int(double b) { return b == std::floor(b) && std::fabs(b) <= 4.0; }

// ln k expression (float64) of an Arrhenius triple, or "" when k is A alone.
std::string ln_arrh64(const Arrh& a, OpCounts& c) {
  std::string s = D(std::log(a.A));
  if (a.E != 0.0) { s = fmt("fma(%s, iT, %s)", D(-a.E).c_str(), s.c_str()); c.fp64 += 1; }
  if (a.beta != 0.0) { s = fmt("fma(%s, lnT, %s)", D(a.beta).c_str(), s.c_str()); c.fp64 += 1; }
  return s;
}

std::string ln_arrh32(const Arrh& a, OpCounts& c) {
  std::string s = F(std::log(a.A));
  if (a.E != 0.0) { s = fmt("fmaf(%s, iTf, %s)", F(-a.E).c_str(), s.c_str()); c.fp32 += 1; }
  if (a.beta != 0.0) { s = fmt("fmaf(%s, lnTf, %s)", F(a.beta).c_str(), s.c_str()); c.fp32 += 1; }
  return s;
}

// Species that need G/RT: those of reversible reactions.
std::vector<char> gibbs_needed(const Mechanism& m) {
  std::vector<char> need(m.ns, 0);
  for (auto& r : m.rx)
    if (r.reversible) {
      for (auto& e : r.reac) need[e.first] = 1;
      for (auto& e : r.prod) need[e.first] = 1;
    }
  return need;
}

std::vector<char> species_used(const Mechanism& m) {
  std::vector<char> used(m.ns, 0);
  for (auto& r : m.rx) {
    for (auto& e : r.reac) used[e.first] = 1;
    for (auto& e : r.prod) used[e.first] = 1;
    if (r.collider >= 0) used[r.collider] = 1;
    for (auto& e : r.eff) used[e.first] = 1;
  }
  return used;
}

// Distinct NASA mid temperatures get one range flag each.
std::map<double, int> tmid_flags(const Mechanism& m) {
  std::map<double, int> f;
  for (int k = 0; k < m.ns; ++k)
    if (!f.count(m.Tmid[k])) { int id = (int)f.size(); f[m.Tmid[k]] = id; }
  return f;
}

std::string sel(const std::string& flag, double lo, double hi) {
  if (lo == hi) return D(lo);
  return fmt("(%s ? %s : %s)", flag.c_str(), D(lo).c_str(), D(hi).c_str());
}

// G/RT of species k as float64 (Eq. (Ck)): a polynomial in T, a5/T, -a0 ln T.
void emit_gibbs64(Out& o, const Mechanism& m, int k, const std::string& flag, OpCounts& c) {
  const double* lo = &m.a_lo[7 * k];
  const double* hi = &m.a_hi[7 * k];
  auto co = [&](const double* a, int n) {
    switch (n) {
      case 0: return a[0] - a[6];
      case 1: return -a[1] / 2.0;
      case 2: return -a[2] / 6.0;
      case 3: return -a[3] / 12.0;
      default: return -a[4] / 20.0;
    }
  };
  std::string h = sel(flag, co(lo, 4), co(hi, 4));
  for (int n = 3; n >= 0; --n) h = fmt("fma(%s, T, %s)", h.c_str(), sel(flag, co(lo, n), co(hi, n)).c_str());
  o(fmt("const double g_%d = fma(%s, lnT, fma(%s, iT, %s));", k, sel(flag, -lo[0], -hi[0]).c_str(),
        sel(flag, lo[5], hi[5]).c_str(), h.c_str()));
  c.fp64 += 6;
}

// G/RT of species k as a float pair: the same polynomial with float-pair
// immediates (range selected by the flag) and float-pair T, ln T, 1/T.
void emit_gibbs_df(Out& o, const Mechanism& m, int k, const std::string& flag, OpCounts& c) {
  const double* lo = &m.a_lo[7 * k];
  const double* hi = &m.a_hi[7 * k];
  auto co = [&](const double* a, int n) {
    switch (n) {
      case 0: return a[0] - a[6];
      case 1: return -a[1] / 2.0;
      case 2: return -a[2] / 6.0;
      case 3: return -a[3] / 12.0;
      case 4: return -a[4] / 20.0;
      case 5: return a[5];
      default: return -a[0];
    }
  };
  auto dsel = [&](int n) {
    const double a = co(lo, n), b = co(hi, n);
    if (a == b) return DFc(a);
    const float ah = (float)a, bh = (float)b;
    return fmt("kx_mk(%s ? %s : %s, %s ? %s : %s)", flag.c_str(), F(ah).c_str(), F(bh).c_str(), flag.c_str(),
               F((float)(a - (double)ah)).c_str(), F((float)(b - (double)bh)).c_str());
  };
  std::string h = dsel(4);
  for (int n = 3; n >= 0; --n) h = fmt("kx_df_fma(%s, Td, %s)", h.c_str(), dsel(n).c_str());
  o(fmt("const kx_df g_%d = kx_df_fma(%s, lnT, kx_df_fma(%s, iT, %s));", k, dsel(6).c_str(), dsel(5).c_str(), h.c_str()));
  c.fp32 += 6 * kDfFma + 14;
}

std::string nasa_flag(const Mechanism& m, int k, const std::map<double, int>& flags) {
  return fmt("lo%d", flags.at(m.Tmid[k]));
}

// Concentrations C_k (float64) and [M]; y_k = Y_k/W_k.
void emit_concentrations64(Out& o, const Mechanism& m, const std::vector<char>& used, OpCounts& c) {
  o(fmt("const double cM = P * iT * %s;", D(1.0 / R_U).c_str()));
  std::string sum;
  for (int k = 0; k < m.ns; ++k) {
    o(fmt("const double y_%d = Y_[(long long)%d * ld + i] * %s;", k, k, D(1.0 / m.W[k]).c_str()));
    sum += (k ? " + y_" : "y_") + std::to_string(k);
  }
  o("const double sig = " + sum + ";");
  o("if (!(sig > 0.0 && sig < KX_INF)) KX_BAD_POINT");
  o("const double fC = cM / sig;");
  for (int k = 0; k < m.ns; ++k)
    if (used[k]) o(fmt("const double C_%d = y_%d * fC;", k, k));
  c.fp64 += 2 * m.ns + 3;
  c.div64 += 1;
}

// Third-body concentration [X]_i (float64).
std::string third_body64(const Reaction& r, OpCounts& c) {
  if (r.collider >= 0) return fmt("C_%d", r.collider);
  std::string s = r.default_eff == 1.0 ? std::string("cM") : fmt("%s * cM", D(r.default_eff).c_str());
  for (auto& e : r.eff) {
    double a = e.second - r.default_eff;
    if (a == 0.0) continue;
    s = fmt("fma(%s, C_%d, %s)", D(a).c_str(), e.first, s.c_str());
    c.fp64 += 1;
  }
  return s;
}

std::string third_body32(const Reaction& r, OpCounts& c) {
  if (r.collider >= 0) return fmt("Cf_%d", r.collider);
  std::string s = r.default_eff == 1.0 ? std::string("cMf") : fmt("%s * cMf", F(r.default_eff).c_str());
  for (auto& e : r.eff) {
    double a = e.second - r.default_eff;
    if (a == 0.0) continue;
    s = fmt("fmaf(%s, Cf_%d, %s)", F(a).c_str(), e.first, s.c_str());
    c.fp32 += 1;
  }
  return s;
}

std::string conc_product(const std::vector<std::pair<int, int>>& side, const std::string& pre) {
  std::string s;
  for (auto& e : side)
    for (int n = 0; n < e.second; ++n) s += " * " + pre + std::to_string(e.first);
  return s;
}

int sum_nu(const Reaction& r) {
  int dn = 0;
  for (auto& e : r.prod) dn += e.second;
  for (auto& e : r.reac) dn -= e.second;
  return dn;
}

// sum_k nu_k v_k over products minus reactants, as an fma chain on `var`.
std::string nu_sum(const Reaction& r, const char* var, OpCounts& c) {
  std::map<int, int> nu;
  for (auto& e : r.prod) nu[e.first] += e.second;
  for (auto& e : r.reac) nu[e.first] -= e.second;
  std::string s;
  for (auto& kv : nu) {
    if (kv.second == 0) continue;
    std::string term = fmt("%s_%d", var, kv.first);
    if (s.empty()) {
      s = kv.second == 1 ? term : kv.second == -1 ? "-" + term : fmt("%s * %s", D(kv.second).c_str(), term.c_str());
    } else {
      s = kv.second == 1 ? s + " + " + term : kv.second == -1 ? s + " - " + term
                                                               : fmt("fma(%s, %s, %s)", D(kv.second).c_str(), term.c_str(), s.c_str());
    }
    c.fp64 += 1;
  }
  return s.empty() ? "0.0" : s;
}

// ------------------------------------------------------------------ rates, float64
// Order of emission: reactions sharing a (beta, E) pair (and neither being
// a special case) are emitted next to each other so that their common
// exp(beta ln T - E/T) is computed once and dies at once (Sec. 2.3.1).
std::vector<int> emission_order(const Mechanism& m, std::map<int, int>& share_group) {
  std::map<std::pair<double, double>, std::vector<int>> groups;
  for (int i = 0; i < m.nr(); ++i) {
    const Reaction& r = m.rx[i];
    if ((r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) && !(r.k.beta == 0.0 && r.k.E == 0.0) &&
        !(r.k.E == 0.0 && is_small_int(r.k.beta)))
      groups[{r.k.beta, r.k.E}].push_back(i);
  }
  std::vector<int> order;
  std::vector<char> done(m.nr(), 0);
  int gid = 0;
  for (int i = 0; i < m.nr(); ++i) {
    if (done[i]) continue;
    const Reaction& r = m.rx[i];
    auto it = groups.find({r.k.beta, r.k.E});
    if ((r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) && it != groups.end() && it->second.size() > 1 &&
        it->second[0] == i) {
      for (int j : it->second) { order.push_back(j); done[j] = 1; share_group[j] = gid; }
      ++gid;
    } else if (!done[i]) {
      order.push_back(i);
      done[i] = 1;
    }
  }
  return order;
}

void emit_rates64(Out& o, const Mechanism& m, const EmitOptions& opt, bool rop, OpCounts& c) {
  const auto used = species_used(m);
  const auto need_g = gibbs_needed(m);
  const auto flags = tmid_flags(m);
  o("const double lnT = log(T);");
  o("const double iT = 1.0 / T;");
  c.log64 += 1; c.div64 += 1;
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  if (any_plog) { o("const double lnP = kx_log(P);"); c.log64 += 1; }
  emit_concentrations64(o, m, used, c);
  for (auto& f : flags) o(fmt("const bool lo%d = T < %s;", f.second, D(f.first).c_str()));
  for (int k = 0; k < m.ns; ++k)
    if (need_g[k]) emit_gibbs64(o, m, k, nasa_flag(m, k, flags), c);
  o(fmt("const double lnPRT = %s - lnT;", D(std::log(P_ATM / R_U)).c_str()));
  c.fp64 += 1;
  if (opt.kc_mode == 1) {
    o("const double PRT = P_ATM_R * iT;");
    for (int k = 0; k < m.ns; ++k)
      if (need_g[k]) { o(fmt("const double eg_%d = kx_exp(-g_%d);", k, k)); c.exp64 += 1; }
  }
  if (!rop)
    for (int k = 0; k < m.ns; ++k) o(fmt("double w_%d = 0.0;", k));

  std::map<int, int> share;
  std::vector<int> order = emission_order(m, share);
  int open_group = -1;
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const int i = order[oi];
    const Reaction& r = m.rx[i];
    if (share.count(i) && share[i] != open_group) {
      o(fmt("{  // shared exp(beta lnT - E/T), beta = %s, E/R = %s", D(r.k.beta).c_str(), D(r.k.E).c_str()));
      ++o.ind;
      Arrh a = r.k;
      a.A = 1.0;
      o(fmt("const double ex = kx_exp(%s);", ln_arrh64(a, c).c_str()));
      c.exp64 += 1;
      open_group = share[i];
    }
    o(fmt("{  // reaction %d", i));
    ++o.ind;
    bool kf_is_exp = false;   // kf = exp(lkf) with lkf available
    if (r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) {
      if (share.count(i)) {
        o(fmt("const double kf = %s * ex;", D(r.k.A).c_str()));
        c.fp64 += 1;
      } else if (r.k.beta == 0.0 && r.k.E == 0.0) {
        o(fmt("const double kf = %s;", D(r.k.A).c_str()));
        o(fmt("const double lkf = %s;", D(std::log(r.k.A)).c_str()));
        kf_is_exp = true;
      } else if (r.k.E == 0.0 && is_small_int(r.k.beta)) {
        int b = (int)r.k.beta;
        std::string s = D(r.k.A);
        for (int n = 0; n < std::abs(b); ++n) s += b > 0 ? " * T" : " * iT";
        o("const double kf = " + s + ";");
        c.fp64 += std::abs(b);
      } else {
        o(fmt("const double lkf = %s;", ln_arrh64(r.k, c).c_str()));
        o("const double kf = kx_exp(lkf);");
        c.exp64 += 1;
        kf_is_exp = true;
      }
    } else if (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) {
      o(fmt("const double lk0 = %s;", ln_arrh64(r.k0, c).c_str()));
      o(fmt("const double lki = %s;", ln_arrh64(r.k, c).c_str()));
      o(fmt("const double X = %s;", third_body64(r, c).c_str()));
      o("const double lnPr = fmax(lk0 - lki + kx_log(X), -690.77552789821368);");
      o("const double Pr = kx_exp(lnPr);");
      c.fp64 += 2; c.log64 += 1; c.exp64 += 1;
      if (r.blend == Blend::Troe) {
        const double al = r.troe[0];
        std::string Fc;
        if (1.0 - al != 0.0) { Fc = fmt("%s * kx_exp(T * %s)", D(1.0 - al).c_str(), D(-1.0 / r.troe[1]).c_str()); c.exp64 += 1; c.fp64 += 2; }
        if (al != 0.0) { Fc += (Fc.empty() ? "" : " + ") + fmt("%s * kx_exp(T * %s)", D(al).c_str(), D(-1.0 / r.troe[2]).c_str()); c.exp64 += 1; c.fp64 += 2; }
        Fc += (Fc.empty() ? "" : " + ") + fmt("kx_exp(%s * iT)", D(-r.troe[3]).c_str());
        c.exp64 += 1; c.fp64 += 1;
        o("const double lFc = kx_log(" + Fc + ") * KX_INV_LN10;");
        o("const double xx = fma(lnPr, KX_INV_LN10, fma(-0.67, lFc, -0.4));");
        o("const double ff = xx / (fma(-1.27, lFc, 0.75) - 0.14 * xx);");
        o("const double F = kx_exp(KX_LN10 * lFc / fma(ff, ff, 1.0));");
        c.log64 += 1; c.exp64 += 1; c.div64 += 2; c.fp64 += 8;
      } else if (r.blend == Blend::Sri) {
        o("const double lPr = lnPr * KX_INV_LN10;");
        o(fmt("const double base = %s * kx_exp(%s * iT) + kx_exp(T * %s);", D(r.sri[0]).c_str(), D(-r.sri[1]).c_str(),
              D(-1.0 / r.sri[2]).c_str()));
        o(fmt("const double F = %s * kx_exp(fma(%s, lnT, kx_log(base) / fma(lPr, lPr, 1.0)));", D(r.sri[3]).c_str(),
              D(r.sri[4]).c_str()));
        c.exp64 += 3; c.log64 += 1; c.div64 += 1; c.fp64 += 8;
      } else {
        o("const double F = 1.0;");
      }
      if (r.kind == Kind::Falloff) {
        o("const double kf = kx_exp(lki) * (Pr / (1.0 + Pr)) * F;");
      } else {
        o("const double kf = kx_exp(lk0) * (1.0 / (1.0 + Pr)) * F;");
      }
      c.exp64 += 1; c.div64 += 1; c.fp64 += 3;
    } else {  // PLOG
      const auto& t = r.plog;
      auto lk = [&](size_t j) {
        Arrh a{t[j][1], t[j][2], t[j][3]};
        return ln_arrh64(a, c);
      };
      o("double lkf;");
      o(fmt("if (P <= %s) lkf = %s;", D(t[0][0]).c_str(), lk(0).c_str()));
      for (size_t j = 0; j + 1 < t.size(); ++j) {
        double l1 = std::log(t[j][0]), l2 = std::log(t[j + 1][0]);
        o(fmt("else if (P < %s) { const double l1 = %s; lkf = fma(%s - l1, (lnP - %s) * %s, l1); }", D(t[j + 1][0]).c_str(),
              lk(j).c_str(), lk(j + 1).c_str(), D(l1).c_str(), D(1.0 / (l2 - l1)).c_str()));
      }
      o(fmt("else lkf = %s;", lk(t.size() - 1).c_str()));
      o("const double kf = kx_exp(lkf);");
      c.exp64 += 1; c.fp64 += 3;
      kf_is_exp = true;
    }
    std::string q;
    if (r.reversible) {
      const int dn = sum_nu(r);
      if (opt.kc_mode == 1) {
        std::string num = "kf" + conc_product(r.reac, "eg_");
        std::string den = conc_product(r.prod, "eg_").substr(3);
        for (int n = 0; n < -dn; ++n) num += " * PRT";
        for (int n = 0; n < dn; ++n) den += " * PRT";
        o("const double kr = (" + num + ") / (" + den + ");");
        c.div64 += 1; c.fp64 += 4;
      } else {
        std::string lnkc = nu_sum(r, "g", c);
        // ln K_c = -sum nu g + dn lnPRT
        std::string lk = dn == 0 ? "-(" + lnkc + ")" : fmt("fma(%s, lnPRT, -(%s))", D(dn).c_str(), lnkc.c_str());
        if (dn != 0) c.fp64 += 1;
        o("const double lnKc = " + lk + ";");
        if (kf_is_exp) o("const double kr = kx_exp(lkf - lnKc);");
        else o("const double kr = kf * kx_exp(-lnKc);");
        c.exp64 += 1; c.fp64 += 1;
      }
      o("const double q = kf" + conc_product(r.reac, "C_") + " - kr" + conc_product(r.prod, "C_") + ";");
    } else {
      o("const double q = kf" + conc_product(r.reac, "C_") + ";");
    }
    for (auto& e : r.reac) c.fp64 += e.second;
    for (auto& e : r.prod) c.fp64 += e.second;
    c.fp64 += 1;
    std::string qq = "q";
    if (r.kind == Kind::ThreeBody) {
      o(fmt("const double qX = q * (%s);", third_body64(r, c).c_str()));
      qq = "qX";
      c.fp64 += 1;
    }
    if (rop) {
      o(fmt("out_[(long long)%d * ld + i] = %s;", i, qq.c_str()));
    } else {
      std::map<int, int> nu;
      for (auto& e : r.prod) nu[e.first] += e.second;
      for (auto& e : r.reac) nu[e.first] -= e.second;
      for (auto& kv : nu) {
        if (kv.second == 1) o(fmt("w_%d += %s;", kv.first, qq.c_str()));
        else if (kv.second == -1) o(fmt("w_%d -= %s;", kv.first, qq.c_str()));
        else if (kv.second != 0) o(fmt("w_%d = fma(%s, %s, w_%d);", kv.first, D(kv.second).c_str(), qq.c_str(), kv.first));
        if (kv.second != 0) c.fp64 += 1;
      }
    }
    --o.ind;
    o("}");
    const bool last_of_group = share.count(i) && (oi + 1 == order.size() || !share.count(order[oi + 1]) ||
                                                  share[order[oi + 1]] != share[i]);
    if (last_of_group) {
      --o.ind;
      o("}");
      open_group = -1;
    }
  }
  if (!rop)
    for (int k = 0; k < m.ns; ++k) o(fmt("out_[(long long)%d * ld + i] = w_%d;", k, k));
}

// ------------------------------------------------------------------ rates, mixed
// float32: ln k_f, third-body [X], falloff blending, ln R_f = ln(c_i k_f
// prod C^nu').  float64: ln C_k, G_k/RT, mu_k = G_k/RT + ln C_k and
// ln(R_r/R_f) = sum_k nu_k mu_k - (sum nu) ln(p_atm/(R T)), which is
// -ln K_c + sum nu ln C (Eq. K_p); q = R_f - R_r from kx_net_rate; wdot
// accumulated in float64.
void emit_rates_mixed(Out& o, const Mechanism& m, bool rop, OpCounts& c) {
  const auto used = species_used(m);
  const auto need_g = gibbs_needed(m);
  const auto flags = tmid_flags(m);
  o("const kx_df Td = kx_d2df_i(T);");
  o("const kx_df lnT = kx_df_log_d(T);");
  o("const kx_df iT = kx_df_div(kx_mk(1.0f, 0.0f), Td);");
  o("const float lnTf = lnT.hi, iTf = iT.hi, Tf = Td.hi;");
  c.fp32 += 45 + 12 + kDfDiv;
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  if (any_plog) { o("const float lnPf = __logf(kx_d2f(P));"); c.log32 += 1; }
  o(fmt("const kx_df cM = kx_df_mul(kx_df_mul(kx_d2df_i(P), iT), %s);", DFc(1.0 / R_U).c_str()));
  // y_k = Y_k/W_k and sigma = sum y_k as float pairs; C_k = y_k C_M/sigma
  std::string s0;
  for (int k = 0; k < m.ns; ++k) {
    o(fmt("const double Yk_%d = Y_[(long long)%d * ld + i];", k, k));
    o(fmt("const kx_df y_%d = kx_df_mul(kx_d2df_i(Yk_%d), %s);", k, k, DFc(1.0 / m.W[k]).c_str()));
  }
  // pairwise sum of the y_k (short dependence chains)
  std::vector<std::string> terms;
  for (int k = 0; k < m.ns; ++k) terms.push_back(fmt("y_%d", k));
  int tmp = 0;
  while (terms.size() > 1) {
    std::vector<std::string> next;
    for (size_t j = 0; j + 1 < terms.size(); j += 2) {
      o(fmt("const kx_df sg%d = kx_df_add(%s, %s);", tmp, terms[j].c_str(), terms[j + 1].c_str()));
      next.push_back(fmt("sg%d", tmp++));
    }
    if (terms.size() % 2) next.push_back(terms.back());
    terms = next;
  }
  o("const kx_df sig = " + terms[0] + ";");
  o("if (!(sig.hi > 0.0f && sig.hi < KX_INF_F)) KX_BAD_POINT");
  o("const kx_df fC = kx_df_div(cM, sig);");
  o("const kx_df lnfC = kx_df_log(fC);");
  o("const float cMf = cM.hi, fCf = fC.hi;");
  c.fp32 += m.ns * (12 + kDfMul + kDfAdd) + kDfDiv + kDfLog;
  bool any_tb = false;
  for (auto& r : m.rx) any_tb |= r.third_body();
  for (int k = 0; k < m.ns; ++k) {
    if (!used[k]) continue;
    // ln |C_k| = ln |Y_k| - ln W_k + ln(C_M/sigma) as a float pair, floored at -700 (absent species:
    // zero rates, not nan); the sign of C_k is kept apart
    o(fmt("const long long yb_%d = __double_as_longlong(Yk_%d) & 0x7fffffffffffffffLL;", k, k));
    o(fmt("kx_df lnC_%d = kx_mk(-700.0f, 0.0f);", k));
    o(fmt("if (yb_%d >= 0x0010000000000000LL && yb_%d < 0x7ff0000000000000LL) {", k, k));
    o(fmt("  lnC_%d = kx_df_add(kx_df_log_d(__longlong_as_double(yb_%d)), kx_df_sub(lnfC, %s));", k, k, DFc(std::log(m.W[k])).c_str()));
    o(fmt("  if (!(lnC_%d.hi > -700.0f)) lnC_%d = kx_mk(-700.0f, 0.0f);", k, k));
    o("}");
    o(fmt("const float lnCf_%d = lnC_%d.hi;", k, k));
    o(fmt("const int ng_%d = __double_as_longlong(Yk_%d) < 0LL;", k, k));
    if (any_tb) o(fmt("const float Cf_%d = y_%d.hi * fCf;", k, k));
    c.fp32 += kDfLog + 12 + 2 * kDfAdd + 4;
  }
  for (auto& f : flags) {
    long long b;
    std::memcpy(&b, &f.first, 8);
    o(fmt("const bool lo%d = __double_as_longlong(T) < %lldLL;", f.second, b));
  }
  for (int k = 0; k < m.ns; ++k)
    if (need_g[k]) {
      emit_gibbs_df(o, m, k, nasa_flag(m, k, flags), c);
      o(fmt("const kx_df mu_%d = kx_df_add(g_%d, lnC_%d);", k, k, k));
      c.fp32 += kDfAdd;
    }
  o(fmt("const kx_df lnPRT = kx_df_sub(%s, lnT);", DFc(std::log(P_ATM / R_U)).c_str()));
  c.fp32 += kDfAdd;
  if (!rop)
    for (int k = 0; k < m.ns; ++k) o(fmt("double w_%d = 0.0;", k));
  for (int i = 0; i < m.nr(); ++i) {
    const Reaction& r = m.rx[i];
    o(fmt("{  // reaction %d", i));
    ++o.ind;
    std::string lnRf;
    if (r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) {
      lnRf = ln_arrh32(r.k, c);
      if (r.kind == Kind::ThreeBody) {
        o(fmt("const float lX = __logf(%s);", third_body32(r, c).c_str()));
        c.log32 += 1;
        lnRf += " + lX";
      }
    } else if (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) {
      o(fmt("const float lk0 = %s;", ln_arrh32(r.k0, c).c_str()));
      o(fmt("const float lki = %s;", ln_arrh32(r.k, c).c_str()));
      o(fmt("const float lnPr = fmaxf(lk0 - lki + __logf(%s), -690.0f);", third_body32(r, c).c_str()));
      c.log32 += 1; c.fp32 += 2;
      std::string lnF = "0.0f";
      if (r.blend == Blend::Troe) {
        const double al = r.troe[0];
        std::string Fc;
        if (1.0 - al != 0.0) Fc = fmt("%s * __expf(Tf * %s)", F(1.0 - al).c_str(), F(-1.0 / r.troe[1]).c_str());
        if (al != 0.0) Fc += (Fc.empty() ? "" : " + ") + fmt("%s * __expf(Tf * %s)", F(al).c_str(), F(-1.0 / r.troe[2]).c_str());
        Fc += (Fc.empty() ? "" : " + ") + fmt("__expf(%s * iTf)", F(-r.troe[3]).c_str());
        o("const float lFc = __log10f(" + Fc + ");");
        o("const float xx = fmaf(lnPr, 0.434294482f, fmaf(-0.67f, lFc, -0.4f));");
        o("const float ff = __fdividef(xx, fmaf(-1.27f, lFc, 0.75f) - 0.14f * xx);");
        o("const float lnF = __fdividef(2.30258509f * lFc, fmaf(ff, ff, 1.0f));");
        c.exp32 += 3; c.log32 += 1; c.div32 += 2; c.fp32 += 14;
        lnF = "lnF";
      } else if (r.blend == Blend::Sri) {
        o("const float lPr = lnPr * 0.434294482f;");
        o(fmt("const float base = %s * __expf(%s * iTf) + __expf(Tf * %s);", F(r.sri[0]).c_str(), F(-r.sri[1]).c_str(),
              F(-1.0 / r.sri[2]).c_str()));
        o(fmt("const float lnF = %s + %s * lnTf + __fdividef(__logf(base), fmaf(lPr, lPr, 1.0f));", F(std::log(r.sri[3])).c_str(),
              F(r.sri[4]).c_str()));
        c.exp32 += 2; c.log32 += 1; c.div32 += 1; c.fp32 += 8;
        lnF = "lnF";
      }
      if (r.kind == Kind::Falloff) lnRf = "lki + kx_ln_pr_ratio(lnPr) + " + lnF;
      else lnRf = "lk0 + kx_ln_inv_1p(lnPr) + " + lnF;
      c.exp32 += 1; c.log32 += 1; c.fp32 += 4;
    } else {  // PLOG
      const auto& t = r.plog;
      auto lk = [&](size_t j) { return ln_arrh32(Arrh{t[j][1], t[j][2], t[j][3]}, c); };
      o("float lkf;");
      o(fmt("if (P <= %s) lkf = %s;", D(t[0][0]).c_str(), lk(0).c_str()));
      for (size_t j = 0; j + 1 < t.size(); ++j) {
        double l1 = std::log(t[j][0]), l2 = std::log(t[j + 1][0]);
        o(fmt("else if (P < %s) { const float l1 = %s; lkf = fmaf(%s - l1, (lnPf - %s) * %s, l1); }", D(t[j + 1][0]).c_str(),
              lk(j).c_str(), lk(j + 1).c_str(), F(l1).c_str(), F(1.0 / (l2 - l1)).c_str()));
      }
      o(fmt("else lkf = %s;", lk(t.size() - 1).c_str()));
      lnRf = "lkf";
      c.fp32 += 3;
    }
    for (auto& e : r.reac) {
      lnRf += e.second == 1 ? fmt(" + lnCf_%d", e.first) : fmt(" + %d.0f * lnCf_%d", e.second, e.first);
      c.fp32 += 1;
    }
    o("const float lnRf = " + lnRf + ";");
    // signs of prod C^nu' and prod C^nu'' (negative mass fractions)
    std::string sf = "0", sr = "0";
    for (auto& e : r.reac) if (e.second % 2) sf += fmt(" ^ ng_%d", e.first);
    for (auto& e : r.prod) if (e.second % 2) sr += fmt(" ^ ng_%d", e.first);
    if (r.reversible) {
      // ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T)) in float pairs, rounded to float32 once
      const int dn = sum_nu(r);
      std::map<int, int> nu;
      for (auto& e : r.prod) nu[e.first] += e.second;
      for (auto& e : r.reac) nu[e.first] -= e.second;
      std::string acc;
      for (auto& kv : nu) {
        if (kv.second == 0) continue;
        const std::string term = kv.second == 1 || kv.second == -1 ? fmt("mu_%d", kv.first)
                                                                 : fmt("kx_df_mulf(mu_%d, %s)", kv.first, F(std::abs(kv.second)).c_str());
        if (acc.empty()) acc = kv.second > 0 ? term : "kx_df_neg(" + term + ")";
        else acc = fmt("kx_df_%s(%s, %s)", kv.second > 0 ? "add" : "sub", acc.c_str(), term.c_str());
        c.fp32 += kDfAdd;
      }
      if (acc.empty()) acc = "kx_mk(0.0f, 0.0f)";
      if (dn != 0) { acc = fmt("kx_df_add(%s, kx_df_mulf(lnPRT, %s))", acc.c_str(), F(-dn).c_str()); c.fp32 += kDfAdd + kDfMulf; }
      o("const float lnra = (" + acc + ").hi;");
      o("const double q = kx_net_rate_s(lnRf, lnra, " + sf + ", " + sr + ");");
      c.exp32 += 2; c.fp32 += 10;
    } else {
      o("const double q0 = kx_pow2_scaled(lnRf * KX_LOG2E_F, 1.0f);");
      o("const double q = (" + sf + ") ? -q0 : q0;");
      c.exp32 += 1; c.fp32 += 2;
    }
    if (rop) {
      o(fmt("out_[(long long)%d * ld + i] = q;", i));
    } else {
      std::map<int, int> nu;
      for (auto& e : r.prod) nu[e.first] += e.second;
      for (auto& e : r.reac) nu[e.first] -= e.second;
      for (auto& kv : nu) {
        if (kv.second == 1) o(fmt("w_%d += q;", kv.first));
        else if (kv.second == -1) o(fmt("w_%d -= q;", kv.first));
        else if (kv.second != 0) o(fmt("w_%d = fma(%s, q, w_%d);", kv.first, D(kv.second).c_str(), kv.first));
        if (kv.second != 0) c.fp64 += 1;
      }
    }
    --o.ind;
    o("}");
  }
  if (!rop)
    for (int k = 0; k < m.ns; ++k) o(fmt("out_[(long long)%d * ld + i] = w_%d;", k, k));
}

// ------------------------------------------------------------------ rates, table driven
// For large mechanisms the fully unrolled kernels spill heavily and take
// minutes to compile.  This variant keeps thread-per-point but walks a
// reaction table in a loop: every thread of a warp handles the same
// reaction at the same time, so the control flow and the table loads are
// uniform (broadcasts), and the species state (C_k, G_k/RT, wdot_k) lives
// in per-thread local-memory arrays indexed by the table's species numbers
// (interleaved across threads, so each access is one coalesced line).
// Same arithmetic, in the same order per reaction, as the unrolled kernels.
//
// Reaction record: ints  {kind, reversible, n_reac, n_prod, dn, eff_offset,
//                         n_eff, blend, plog_offset, n_plog, const_kf, pad,
//                         species[6], nu[6]}
//                  doubles {ln A, beta, -E, ln A0, beta0, -E0, default_eff,
//                           blend parameters[5], pad...}
constexpr int RI = 24, RD = 16;

void emit_rate_tables(Out& g, const Mechanism& m, bool mixed) {
  std::string ri, rd, eff, plog, nasa, tm;
  int eo = 0, po = 0;
  for (const Reaction& r : m.rx) {
    int kind = r.kind == Kind::Elementary ? 0 : r.kind == Kind::ThreeBody ? 1 : r.kind == Kind::Falloff ? 2
             : r.kind == Kind::ChemAct ? 3 : 4;
    int blend = r.blend == Blend::Lindemann ? 0 : r.blend == Blend::Troe ? 1 : 2;
    int ne = 0;
    std::string e;
    if (r.third_body()) {
      if (r.collider >= 0) { e += fmt("%d,", r.collider); ne = -1; }   // collider marker
      else for (auto& x : r.eff) if (x.second != r.default_eff) { e += fmt("%d,", x.first); ++ne; }
    }
    const bool constk = (r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) && r.k.beta == 0.0 && r.k.E == 0.0;
    int v[RI] = {kind, r.reversible ? 1 : 0, (int)r.reac.size(), (int)r.prod.size(), sum_nu(r), eo, ne, blend, po,
                 (int)r.plog.size(), constk ? 1 : 0, 0};
    for (size_t j = 0; j < r.reac.size(); ++j) { v[12 + j] = r.reac[j].first; v[18 + j] = r.reac[j].second; }
    for (size_t j = 0; j < r.prod.size(); ++j) { v[12 + r.reac.size() + j] = r.prod[j].first; v[18 + r.reac.size() + j] = r.prod[j].second; }
    for (int j = 0; j < RI; ++j) ri += std::to_string(v[j]) + ",";
    double d[RD] = {std::log(r.k.A > 0 ? r.k.A : 1e-300), r.k.beta, -r.k.E, 0, 0, 0, r.default_eff, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (r.has_k0) { d[3] = std::log(r.k0.A); d[4] = r.k0.beta; d[5] = -r.k0.E; }
    if (r.blend == Blend::Troe) { d[7] = 1.0 - r.troe[0]; d[8] = r.troe[0]; d[9] = -1.0 / r.troe[1]; d[10] = -1.0 / r.troe[2]; d[11] = -r.troe[3]; }
    if (r.blend == Blend::Sri) { d[7] = r.sri[0]; d[8] = -r.sri[1]; d[9] = -1.0 / r.sri[2]; d[10] = std::log(r.sri[3]); d[11] = r.sri[4]; }
    for (int j = 0; j < RD; ++j) rd += (mixed ? F(d[j]) : D(d[j])) + ",";
    // efficiency table entries: (species, alpha - default) ; collider: (species, 0)
    if (r.third_body()) {
      if (r.collider >= 0) { eff += fmt("{%d, %s},", r.collider, D(0.0).c_str()); eo += 1; }
      else for (auto& x : r.eff) if (x.second != r.default_eff) { eff += fmt("{%d, %s},", x.first, D(x.second - r.default_eff).c_str()); ++eo; }
    }
    for (auto& t : r.plog) { plog += fmt("%s,%s,%s,%s,", D(std::log(t[0])).c_str(), D(std::log(t[1])).c_str(), D(t[2]).c_str(), D(-t[3]).c_str()); ++po; }
    (void)e;
  }
  g(fmt("__device__ const int kx_ri[%d] = {%s0};", RI * m.nr() + 1, ri.c_str()));
  g(fmt("__device__ const %s kx_rd[%d] = {%s0};", mixed ? "float" : "double", RD * m.nr() + 1, rd.c_str()));
  g("struct kx_eff_t { int k; double a; };");
  g(fmt("__device__ const kx_eff_t kx_eff[%d] = {%s{0, 0.0}};", eo + 1, eff.c_str()));
  g(fmt("__device__ const double kx_plog[%d] = {%s0.0};", 4 * po + 1, plog.c_str()));
  // NASA-7 Gibbs coefficients as a polynomial in T plus a5/T - a0 ln T, both ranges, and Tmid
  for (int k = 0; k < m.ns; ++k) {
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = rg == 0 ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
      const double cfs[7] = {a[0] - a[6], -a[1] / 2.0, -a[2] / 6.0, -a[3] / 12.0, -a[4] / 20.0, a[5], -a[0]};
      for (int j = 0; j < 7; ++j) nasa += D(cfs[j]) + ",";
      nasa += D(0.0) + ",";
    }
    tm += D(m.Tmid[k]) + ",";
  }
  g(fmt("__device__ const double kx_gc[%d] = {%s0.0};", 16 * m.ns + 1, nasa.c_str()));
  g(fmt("__device__ const double kx_tmid[%d] = {%s0.0};", m.ns + 1, tm.c_str()));
  std::string iw, lw;
  for (int k = 0; k < m.ns; ++k) { iw += D(1.0 / m.W[k]) + ","; lw += D(std::log(m.W[k])) + ","; }
  g(fmt("__device__ const double kx_riw[%d] = {%s0.0};", m.ns + 1, iw.c_str()));
  g(fmt("__device__ const double kx_rlw[%d] = {%s0.0};", m.ns + 1, lw.c_str()));
}

void emit_rates_table64(Out& o, Out& g, const Mechanism& m, bool rop, OpCounts& c) {
  emit_rate_tables(g, m, false);
  const int ns = m.ns;
  o("const double lnT = log(T);");
  o("const double iT = 1.0 / T;");
  o("const double lnP = kx_log(P);");
  o(fmt("const double cM = P * iT * %s;", D(1.0 / R_U).c_str()));
  o(fmt("double C[%d], g[%d]%s;", ns, ns, rop ? "" : fmt(", w[%d]", ns).c_str()));
  o("double sig = 0.0;");
  o(fmt("for (int k = 0; k < %d; ++k) { const double y = Y_[(long long)k * ld + i] * kx_riw[k]; C[k] = y; sig += y; }", ns));
  o("if (!(sig > 0.0 && sig < KX_INF)) KX_BAD_POINT");
  o("const double fC = cM / sig;");
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o("  C[k] *= fC;");
  o("  const double* a = kx_gc + 16 * k + (T < kx_tmid[k] ? 0 : 8);");
  o("  g[k] = fma(a[6], lnT, fma(a[5], iT, fma(fma(fma(fma(a[4], T, a[3]), T, a[2]), T, a[1]), T, a[0])));");
  if (!rop) o("  w[k] = 0.0;");
  o("}");
  o(fmt("const double lnPRT = %s - lnT;", D(std::log(P_ATM / R_U)).c_str()));
  c.fp64 += ns * 9.0 + 6; c.div64 += 2; c.log64 += 2;
  o("#pragma unroll 1");
  o(fmt("for (int r = 0; r < %d; ++r) {", m.nr()));
  o(fmt("  const int* h = kx_ri + %d * r; const double* d = kx_rd + %d * r;", RI, RD));
  o("  const int kind = h[0];");
  o("  double lkf = fma(d[1], lnT, fma(d[2], iT, d[0]));");
  o("  double kf, X = 0.0;");
  o("  if (kind >= 1 && kind <= 3) {");
  o("    if (h[6] < 0) X = C[kx_eff[h[5]].k];");
  o("    else { X = d[6] * cM; for (int e = 0; e < h[6]; ++e) X = fma(kx_eff[h[5] + e].a, C[kx_eff[h[5] + e].k], X); }");
  o("  }");
  o("  if (kind == 2 || kind == 3) {");
  o("    const double lk0 = fma(d[4], lnT, fma(d[5], iT, d[3]));");
  o("    const double lnPr = fmax(lk0 - lkf + kx_log(X), -690.77552789821368);");
  o("    const double Pr = kx_exp(lnPr);");
  o("    double F = 1.0;");
  o("    if (h[7] == 1) {");
  o("      const double lFc = kx_log(d[7] * kx_exp(T * d[9]) + d[8] * kx_exp(T * d[10]) + kx_exp(d[11] * iT)) * KX_INV_LN10;");
  o("      const double xx = fma(lnPr, KX_INV_LN10, fma(-0.67, lFc, -0.4));");
  o("      const double ff = xx / (fma(-1.27, lFc, 0.75) - 0.14 * xx);");
  o("      F = kx_exp(KX_LN10 * lFc / fma(ff, ff, 1.0));");
  o("    } else if (h[7] == 2) {");
  o("      const double lPr = lnPr * KX_INV_LN10;");
  o("      const double base = d[7] * kx_exp(d[8] * iT) + kx_exp(T * d[9]);");
  o("      F = kx_exp(d[10] + fma(d[11], lnT, kx_log(base) / fma(lPr, lPr, 1.0)));");
  o("    }");
  o("    if (kind == 2) kf = kx_exp(lkf) * (Pr / (1.0 + Pr)) * F;");
  o("    else { kf = kx_exp(lk0) * (1.0 / (1.0 + Pr)) * F; }");
  o("    lkf = kx_log(kf);");
  o("  } else if (kind == 4) {");
  o("    const double* t = kx_plog + 4 * h[8]; const int np = h[9];");
  o("    if (lnP <= t[0]) lkf = fma(t[2], lnT, fma(t[3], iT, t[1]));");
  o("    else if (lnP >= t[4 * (np - 1)]) { const double* u = t + 4 * (np - 1); lkf = fma(u[2], lnT, fma(u[3], iT, u[1])); }");
  o("    else { int j = 0; while (!(lnP < t[4 * (j + 1)])) ++j; const double* u = t + 4 * j;");
  o("      const double l1 = fma(u[2], lnT, fma(u[3], iT, u[1])), l2 = fma(u[6], lnT, fma(u[7], iT, u[5]));");
  o("      lkf = fma(l2 - l1, (lnP - u[0]) / (u[4] - u[0]), l1); }");
  o("    kf = kx_exp(lkf);");
  o("  } else {");
  o("    kf = h[10] ? exp(d[0]) : kx_exp(lkf);");
  o("  }");
  o("  double Rf = kf, Rr = 0.0;");
  o("  const int nre = h[2], npr = h[3];");
  o("  for (int j = 0; j < nre; ++j) { const double cj = C[h[12 + j]]; Rf *= cj; if (h[18 + j] == 2) Rf *= cj; }");
  o("  if (h[1]) {");
  o("    double sg = 0.0;");
  o("    for (int j = 0; j < nre + npr; ++j) { const double nu = (j < nre ? -1.0 : 1.0) * h[18 + j]; sg = fma(nu, g[h[12 + j]], sg); }");
  o("    const double lnKc = fma((double)h[4], lnPRT, -sg);");
  o("    Rr = kx_exp(lkf - lnKc);");
  o("    for (int j = nre; j < nre + npr; ++j) { const double cj = C[h[12 + j]]; Rr *= cj; if (h[18 + j] == 2) Rr *= cj; }");
  o("  }");
  o("  double q = Rf - Rr;");
  o("  if (kind == 1) q *= X;");
  if (rop) o("  out_[(long long)r * ld + i] = q;");
  else {
    o("  for (int j = 0; j < nre + npr; ++j) { const double nu = (j < nre ? -1.0 : 1.0) * h[18 + j]; w[h[12 + j]] = fma(nu, q, w[h[12 + j]]); }");
  }
  o("}");
  if (!rop) o(fmt("for (int k = 0; k < %d; ++k) out_[(long long)k * ld + i] = w[k];", ns));
  // counts: per reaction ~ 2 (lkf) + exps + products + lnKc + scatter
  for (const Reaction& r : m.rx) {
    c.fp64 += 2 + 2 * (r.reac.size() + r.prod.size()) + 3 + (r.reac.size() + r.prod.size());
    c.exp64 += r.reversible ? 2 : 1;
    if (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) { c.exp64 += 6; c.log64 += 3; c.div64 += 3; c.fp64 += 12; }
  }
}

// mixed precision, table driven (see emit_rates_mixed for the split)
void emit_rates_table_mixed(Out& o, Out& g, const Mechanism& m, bool rop, OpCounts& c) {
  emit_rate_tables(g, m, true);
  const int ns = m.ns;
  o("const double lnT = log(T);");
  o("const double iT = 1.0 / T;");
  o("const float lnTf = kx_d2f(lnT), iTf = kx_d2f(iT), Tf = kx_d2f(T);");
  o("const float lnPf = __logf(kx_d2f(P));");
  o(fmt("const double cM = P * iT * %s;", D(1.0 / R_U).c_str()));
  o(fmt("double mu[%d]; float lC[%d], Cf[%d];%s", ns, ns, ns, rop ? "" : fmt(" double w[%d];", ns).c_str()));
  o("double sig = 0.0;");
  o(fmt("for (int k = 0; k < %d; ++k) sig = fma(Y_[(long long)k * ld + i], kx_riw[k], sig);", ns));
  o("if (!(sig > 0.0 && sig < KX_INF)) KX_BAD_POINT");
  o("const double fC = cM / sig;");
  o("const double lnfC = kx_log(fC);");
  o("const float cMf = kx_d2f(cM), fCf = kx_d2f(fC);");
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o("  const double Yk = Y_[(long long)k * ld + i];");
  o("  const double lnC = fmax(kx_log(Yk) + (lnfC - kx_rlw[k]), -700.0);");
  o("  lC[k] = kx_d2f(lnC);");
  o("  Cf[k] = kx_d2f(Yk * kx_riw[k]) * fCf;");
  o("  const double* a = kx_gc + 16 * k + (T < kx_tmid[k] ? 0 : 8);");
  o("  mu[k] = lnC + fma(a[6], lnT, fma(a[5], iT, fma(fma(fma(fma(a[4], T, a[3]), T, a[2]), T, a[1]), T, a[0])));");
  if (!rop) o("  w[k] = 0.0;");
  o("}");
  o(fmt("const double lnPRT = %s - lnT;", D(std::log(P_ATM / R_U)).c_str()));
  c.fp64 += ns * 12.0 + 6; c.log64 += ns + 2; c.div64 += 2;
  o("#pragma unroll 1");
  o(fmt("for (int r = 0; r < %d; ++r) {", m.nr()));
  o(fmt("  const int* h = kx_ri + %d * r; const float* d = kx_rd + %d * r;", RI, RD));
  o("  const int kind = h[0];");
  o("  float lkf = fmaf(d[1], lnTf, fmaf(d[2], iTf, d[0]));");
  o("  float lX = 0.0f;");
  o("  if (kind >= 1 && kind <= 3) {");
  o("    float X;");
  o("    if (h[6] < 0) X = Cf[kx_eff[h[5]].k];");
  o("    else { X = d[6] * cMf; for (int e = 0; e < h[6]; ++e) X = fmaf((float)kx_eff[h[5] + e].a, Cf[kx_eff[h[5] + e].k], X); }");
  o("    lX = __logf(X);");
  o("  }");
  o("  if (kind == 2 || kind == 3) {");
  o("    const float lk0 = fmaf(d[4], lnTf, fmaf(d[5], iTf, d[3]));");
  o("    const float lnPr = fmaxf(lk0 - lkf + lX, -690.0f);");
  o("    float lnF = 0.0f;");
  o("    if (h[7] == 1) {");
  o("      const float lFc = __log10f(d[7] * __expf(Tf * d[9]) + d[8] * __expf(Tf * d[10]) + __expf(d[11] * iTf));");
  o("      const float xx = fmaf(lnPr, 0.434294482f, fmaf(-0.67f, lFc, -0.4f));");
  o("      const float ff = __fdividef(xx, fmaf(-1.27f, lFc, 0.75f) - 0.14f * xx);");
  o("      lnF = __fdividef(2.30258509f * lFc, fmaf(ff, ff, 1.0f));");
  o("    } else if (h[7] == 2) {");
  o("      const float lPr = lnPr * 0.434294482f;");
  o("      const float base = d[7] * __expf(d[8] * iTf) + __expf(Tf * d[9]);");
  o("      lnF = d[10] + d[11] * lnTf + __fdividef(__logf(base), fmaf(lPr, lPr, 1.0f));");
  o("    }");
  o("    lkf = (kind == 2 ? lkf + kx_ln_pr_ratio(lnPr) : lk0 + kx_ln_inv_1p(lnPr)) + lnF;");
  o("    lX = 0.0f;");
  o("  } else if (kind == 4) {");
  o("    const double* t = kx_plog + 4 * h[8]; const int np = h[9]; const double lnP = (double)lnPf;");
  o("    double l;");
  o("    if (lnP <= t[0]) l = fma(t[2], lnT, fma(t[3], iT, t[1]));");
  o("    else if (lnP >= t[4 * (np - 1)]) { const double* u = t + 4 * (np - 1); l = fma(u[2], lnT, fma(u[3], iT, u[1])); }");
  o("    else { int j = 0; while (!(lnP < t[4 * (j + 1)])) ++j; const double* u = t + 4 * j;");
  o("      const double l1 = fma(u[2], lnT, fma(u[3], iT, u[1])), l2 = fma(u[6], lnT, fma(u[7], iT, u[5]));");
  o("      l = fma(l2 - l1, (lnP - u[0]) / (u[4] - u[0]), l1); }");
  o("    lkf = kx_d2f(l);");
  o("  }");
  o("  const int nre = h[2], npr = h[3];");
  o("  float lnRf = lkf + lX;");
  o("  for (int j = 0; j < nre; ++j) lnRf = fmaf((float)h[18 + j], lC[h[12 + j]], lnRf);");
  o("  double q;");
  o("  if (h[1]) {");
  o("    double s = (double)(-h[4]) * lnPRT;");
  o("    for (int j = 0; j < nre + npr; ++j) { const double nu = (j < nre ? -1.0 : 1.0) * h[18 + j]; s = fma(nu, mu[h[12 + j]], s); }");
  o("    q = kx_net_rate(lnRf, s);");
  o("  } else {");
  o("    q = kx_pow2_scaled(lnRf * KX_LOG2E_F, 1.0f);");
  o("  }");
  if (rop) o("  out_[(long long)r * ld + i] = q;");
  else o("  for (int j = 0; j < nre + npr; ++j) { const double nu = (j < nre ? -1.0 : 1.0) * h[18 + j]; w[h[12 + j]] = fma(nu, q, w[h[12 + j]]); }");
  o("}");
  if (!rop) o(fmt("for (int k = 0; k < %d; ++k) out_[(long long)k * ld + i] = w[k];", ns));
  for (const Reaction& r : m.rx) {
    c.fp64 += 1 + 2 * (r.reac.size() + r.prod.size());
    c.fp32 += 4 + r.reac.size();
    c.exp32 += 2;
    if (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) { c.exp32 += 5; c.log32 += 3; c.fp32 += 14; }
  }
}

// ------------------------------------------------------------------ rates, float64 accuracy on the float32 pipe
// Every quantity of the log-space rate evaluation is a float pair
// (double-float, about 2^-47 per operation): ln T, 1/T, ln |C_k|, G_k/RT,
// mu_k = G_k/RT + ln |C_k|, ln k_f, the falloff blending, ln |R_f| and
// ln(|R_r|/|R_f|) = sum nu mu - (sum nu) ln(p_atm/(R T)).  The net rate is
// the larger rate times 1 -+ e^-|ln ratio| (minus when R_f and R_r have the
// same sign; a negative mass fraction makes a concentration, and the
// products it enters, negative), and wdot is accumulated in float pairs
// scaled by 2^-S, where S is chosen per state from a float32 upper bound of
// every reaction's larger rate (a pre-pass over the reactions), so that the
// largest scaled rate is near 2^64 and nothing can overflow; terms more than
// 2^190 below the largest rate underflow to zero.  wdot_k = w_k 2^S leaves
// through one float64 addition per species.
//
// Reactions are grouped into classes of one code shape (kind, reversibility,
// blending, numbers of reactant and product entries, a coefficient nu
// counting as nu entries of the species); each class is one loop over its
// table with straight-line code, warp-uniform loads and no inner loops over
// species.  Each state's species vectors ({ln |C|, mu} as a float4 and the
// float-pair accumulators) live in per-thread local arrays, so the kernel
// compiles in seconds for any mechanism size.
struct DfClass {
  Kind kind;
  bool rev;
  Blend blend;
  int nre, npr;
  bool kconst;          // k = A (beta = E = 0; elementary and three-body reactions): ln k needs no arithmetic
  std::vector<int> rx;
  int maxnu = 0;        // largest |net coefficient| of an entry (set with the tables)
};

std::vector<int> entries(const std::vector<std::pair<int, int>>& side) {
  std::vector<int> e;
  for (auto& s : side)
    for (int n = 0; n < s.second; ++n) e.push_back(s.first);
  return e;
}

// Mixed-precision body of one reaction class (see emit_rates_mixed for the
// split): float32 ln k_f, [X], falloff blend and ln |R_f|; the float-pair
// Gibbs sum ln(|R_r|/|R_f|) rounded once to float32; q as a float64 from
// kx_net_rate_s.  Species vectors {ln |C|, C (float32), mu (pair)} in v_j.
void emit_class_mixed_body(Out& o, const DfClass& d, int ci, int E, OpCounts& c) {
  const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
  const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
  o(d.kconst ? "  float lk = f0.x;   // k = A" : "  float lk = fmaf(f0.z, lnTf, fmaf(f1.x, iTf, f0.x));");
  if (tb) {
    o(fmt("  const int2 e = kx_e%d[r];", ci));
    o("  const float4 f2 = f[2];");
    o("  float X;   // [X] = eff_default C_M + sum_e (eff_e - eff_default) C_e, float32");
    o("  if (e.y < 0) X = sv[kx_effd[e.x].k].y;");
    o("  else { X = f2.x * cMf; for (int j = 0; j < e.y; ++j) { const kx_effd_t q = kx_effd[e.x + j]; X = fmaf(q.ahi, sv[q.k].y, X); } }");
    c.fp32 += d.rx.size() * 8;
  }
  if (d.kind == Kind::ThreeBody) { o("  lk += __logf(X);"); c.log32 += d.rx.size(); }
  if (fo) {
    o("  const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
    o("  const float lk0 = fmaf(f3.x, lnTf, fmaf(f3.z, iTf, f2.z));");
    o("  const float lnPr = fmaxf(lk0 - lk + __logf(X), -690.0f);");
    o("  float lnF = 0.0f;");
    if (d.blend == Blend::Troe) {
      o("  const float lFc = __log10f(f4.x * __expf(Tf * f5.x) + f4.z * __expf(Tf * f5.z) + __expf(f6.x * iTf));");
      o("  const float xx = fmaf(lnPr, 0.434294482f, fmaf(-0.67f, lFc, -0.4f));");
      o("  const float ff = __fdividef(xx, fmaf(-1.27f, lFc, 0.75f) - 0.14f * xx);");
      o("  lnF = __fdividef(2.30258509f * lFc, fmaf(ff, ff, 1.0f));");
      c.exp32 += d.rx.size() * 3; c.log32 += d.rx.size(); c.div32 += d.rx.size() * 2; c.fp32 += d.rx.size() * 14;
    } else if (d.blend == Blend::Sri) {
      o("  const float lPr = lnPr * 0.434294482f;");
      o("  const float base = f4.x * __expf(f4.z * iTf) + __expf(Tf * f5.x);");
      o("  lnF = f5.z + f6.x * lnTf + __fdividef(__logf(base), fmaf(lPr, lPr, 1.0f));");
      c.exp32 += d.rx.size() * 2; c.log32 += d.rx.size(); c.div32 += d.rx.size(); c.fp32 += d.rx.size() * 8;
    }
    if (d.kind == Kind::Falloff) o("  lk = lk + kx_ln_pr_ratio(lnPr) + lnF;");
    else o("  lk = lk0 + kx_ln_inv_1p(lnPr) + lnF;");
    c.exp32 += d.rx.size(); c.log32 += d.rx.size() * 2; c.fp32 += d.rx.size() * 6;
  } else if (d.kind == Kind::Plog) {
    o(fmt("  const int2 e = kx_e%d[r];", ci));
    o("  const float* t = kx_plogf + 8 * e.x; const long long* tp = kx_plogp + e.x; const int np = e.y;");
    o("  const long long Pb = __double_as_longlong(P);");
    o("  if (Pb <= tp[0]) lk = fmaf(t[4], lnTf, fmaf(t[6], iTf, t[2]));");
    o("  else if (Pb >= tp[np - 1]) { const float* u = t + 8 * (np - 1); lk = fmaf(u[4], lnTf, fmaf(u[6], iTf, u[2])); }");
    o("  else {");
    o("    int j = 0; while (!(Pb < tp[j + 1])) ++j;");
    o("    const float* u = t + 8 * j;");
    o("    const float l1 = fmaf(u[4], lnTf, fmaf(u[6], iTf, u[2])), l2 = fmaf(u[12], lnTf, fmaf(u[14], iTf, u[10]));");
    o("    lk = fmaf(l2 - l1, __fdividef(lnPf - u[0], u[8] - u[0]), l1);");
    o("  }");
    c.fp32 += d.rx.size() * 8;
  }
  std::string lnRf = "lk";
  for (int j = 0; j < d.nre; ++j) lnRf += fmt(" + v%d.x", j);
  o("  const float lnRf = " + lnRf + ";");
  std::string sfx = "0", srx = "0";
  for (int j = 0; j < d.nre; ++j) sfx += fmt(" ^ KX_NEG(k%d)", j);
  for (int j = d.nre; j < E; ++j) srx += fmt(" ^ KX_NEG(k%d)", j);
  o("  const int sf = anyneg ? (" + sfx + ") : 0;");
  c.fp32 += d.rx.size() * (2 + d.nre);
  if (d.rev) {
    const int dn = d.npr - d.nre;
    o("  // ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T)) in float pairs, rounded to float32 once");
    std::string first = d.nre > 0 ? "kx_df_neg(kx_mk(v0.z, v0.w))" : "kx_mk(v0.z, v0.w)";
    o("  kx_df dl = " + first + ";");
    // the high parts summed exactly (two-sum), the errors and low parts beside them, one rounding at the end
    for (int j = 1; j < E; ++j)
      o(fmt("  dl = kx_df_add_u(dl, kx_mk(%sv%d.z, %sv%d.w));", j < d.nre ? "-" : "", j, j < d.nre ? "-" : "", j));
    if (dn == 1 || dn == -1) o(fmt("  dl = kx_df_add_u(dl, %s);", dn == 1 ? "kx_df_neg(lnPRT)" : "lnPRT"));
    else if (dn != 0) o(fmt("  dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, %s));", F(-dn).c_str()));
    o("  const double q = kx_net_rate_s(lnRf, __fadd_rn(dl.hi, dl.lo), sf, anyneg ? (" + srx + ") : 0);");
    c.fp32 += d.rx.size() * ((E - 1) * kDfAdd + (dn ? kDfAdd + kDfMulf : 0) + 10); c.exp32 += d.rx.size() * 2;
  } else {
    o("  const double q0 = kx_pow2_scaled(lnRf * KX_LOG2E_F, 1.0f);");
    o("  const double q = sf ? -q0 : q0;");
    c.exp32 += d.rx.size(); c.fp32 += d.rx.size() * 2;
  }
}

// Reaction classes of one code shape and their constant tables: per class the
// packed species entries (kx_s<c>), the Arrhenius / blend records (kx_f<c>) and
// the efficiency / PLOG index pairs (kx_e<c>); the efficiencies, PLOG tables
// and per-species G/RT coefficients, T_mid, 1/W and ln W shared by all classes.
// merged: one class per (kind, reversibility, blend), entry counts the class's largest, shorter
// reactions padded with entries of species ns (a zero vector the warp-cooperative kernel keeps) and
// each record's f1.w holding -dn, the negated change in mole count (the padding hides it)
std::vector<DfClass> emit_class_tables(Out& g, const Mechanism& m, bool merged = false) {
  const int ns = m.ns;
  std::vector<DfClass> cls;
  for (int i = 0; i < m.nr(); ++i) {
    const Reaction& r = m.rx[i];
    const int nre = (int)entries(r.reac).size(), npr = (int)entries(r.prod).size();
    const Blend bl = (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) ? r.blend : Blend::Lindemann;
    const bool kc = !merged && (r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) && r.k.beta == 0.0 && r.k.E == 0.0;
    auto it = std::find_if(cls.begin(), cls.end(), [&](const DfClass& d) {
      return d.kind == r.kind && d.rev == r.reversible && d.blend == bl &&
             (merged || (d.nre == nre && d.npr == npr && d.kconst == kc));
    });
    if (it == cls.end()) { cls.push_back(DfClass{r.kind, r.reversible, bl, nre, npr, kc, {}, 0}); it = cls.end() - 1; }
    it->nre = std::max(it->nre, nre);
    it->npr = std::max(it->npr, npr);
    it->rx.push_back(i);
  }
  std::string eff, plog, plogp;
  int eo = 0, po = 0;
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    DfClass& d = cls[ci];
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const int NF = fo ? 7 : tb ? 3 : 2;
    std::string si, sf, se;
    for (int i : d.rx) {
      const Reaction& r = m.rx[i];
      auto er = entries(r.reac), ep = entries(r.prod);
      const int dn_i = (int)ep.size() - (int)er.size();
      if (merged) {
        while ((int)er.size() < d.nre) er.push_back(ns);
        while ((int)ep.size() < d.npr) ep.push_back(ns);
      }
      {
        // entry j: species k in the low 16 bits, and in the high 16 bits the upper half of the float32
        // of c, the species' net coefficient on its first entry and 0 on repeats (so that the
        // accumulators are updated once per species); integers up to 256 in magnitude are exact there
        std::vector<int> ek(er);
        ek.insert(ek.end(), ep.begin(), ep.end());
        std::map<int, int> net;
        for (int k : er) net[k] -= 1;
        for (int k : ep) net[k] += 1;
        std::set<int> seen;
        for (int k : ek) {
          const int cc = seen.count(k) ? 0 : net[k];
          seen.insert(k);
          d.maxnu = std::max(d.maxnu, std::abs(cc));
          const float fc = (float)cc;
          uint32_t fb;
          std::memcpy(&fb, &fc, 4);
          si += std::to_string((int32_t)((fb & 0xffff0000u) | (uint32_t)k)) + ",";
        }
      }
      si += std::to_string(i) + ",";
      for (int j = E + 1; j < P; ++j) si += "0,";
      double maxeff = r.default_eff;
      for (auto& x : r.eff) maxeff = std::max(maxeff, x.second);
      sf += "{" + fpair(std::log(r.k.A > 0 ? r.k.A : 1e-300)) + "," + fpair(r.k.beta) + "},";
      sf += "{" + fpair(-r.k.E) + "," + F(std::log(std::max(maxeff, 1e-30))) + "," + (merged ? F(-dn_i) : std::string("0.0f")) + "},";
      if (tb) {
        double p[5] = {0, 0, 0, 0, 0};
        if (r.blend == Blend::Troe) { p[0] = 1.0 - r.troe[0]; p[1] = r.troe[0]; p[2] = -1.0 / r.troe[1]; p[3] = -1.0 / r.troe[2]; p[4] = -r.troe[3]; }
        if (r.blend == Blend::Sri) { p[0] = r.sri[0]; p[1] = -r.sri[1]; p[2] = -1.0 / r.sri[2]; p[3] = std::log(r.sri[3]); p[4] = r.sri[4]; }
        const double la0 = r.has_k0 ? std::log(r.k0.A > 0 ? r.k0.A : 1e-300) : 0.0;
        sf += "{" + fpair(r.default_eff) + "," + fpair(la0) + "},";
        if (fo) {
          sf += "{" + fpair(r.k0.beta) + "," + fpair(-r.k0.E) + "},";
          sf += "{" + fpair(p[0]) + "," + fpair(p[1]) + "},";
          sf += "{" + fpair(p[2]) + "," + fpair(p[3]) + "},";
          sf += "{" + fpair(p[4]) + ",0.0f,0.0f},";
        }
        int n = 0;
        if (r.collider >= 0) { eff += fmt("{%d, 0.0f, 0.0f, 0},", r.collider); n = -1; ++eo; }
        else for (auto& x : r.eff) if (x.second != r.default_eff) { eff += fmt("{%d, %s, 0},", x.first, fpair(x.second - r.default_eff).c_str()); ++n; ++eo; }
        se += fmt("{%d,%d},", n < 0 ? eo - 1 : eo - n, n);
      } else if (d.kind == Kind::Plog) {
        se += fmt("{%d,%d},", po, (int)r.plog.size());
        for (auto& t : r.plog) {
          plog += fpair(std::log(t[0])) + "," + fpair(std::log(t[1])) + "," + fpair(t[2]) + "," + fpair(-t[3]) + ",";
          long long b;
          std::memcpy(&b, &t[0], 8);
          plogp += std::to_string(b) + "LL,";
          ++po;
        }
      }
    }
    for (int j = 0; j < P; ++j) si += "0,";   // one record past the last: the loops prefetch it
    g(fmt("__device__ const __align__(16) int kx_s%d[%d] = {%s};", (int)ci, P * ((int)d.rx.size() + 1), si.c_str()));
    g(fmt("__device__ const float4 kx_f%d[%d] = {%s};", (int)ci, NF * (int)d.rx.size(), sf.c_str()));
    if (tb || d.kind == Kind::Plog) g(fmt("__device__ const int2 kx_e%d[%d] = {%s};", (int)ci, (int)d.rx.size(), se.c_str()));
  }
  g("struct __align__(16) kx_effd_t { int k; float ahi, alo; int pad; };");
  g(fmt("__device__ const kx_effd_t kx_effd[%d] = {%s{0, 0.0f, 0.0f, 0}};", eo + 1, eff.c_str()));
  g(fmt("__device__ const float kx_plogf[%d] = {%s0.0f};", 8 * po + 1, plog.c_str()));
  g(fmt("__device__ const long long kx_plogp[%d] = {%s0LL};", po + 1, plogp.c_str()));
  // G/RT coefficients per species and range: T-polynomial c0..c4, a5 (1/T), -a0 (ln T), as float pairs
  std::string nasa, tmb, iw, lw;
  for (int k = 0; k < ns; ++k) {
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = rg == 0 ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
      const double cfs[7] = {a[0] - a[6], -a[1] / 2.0, -a[2] / 6.0, -a[3] / 12.0, -a[4] / 20.0, a[5], -a[0]};
      for (int j = 0; j < 7; ++j) nasa += fpair(cfs[j]) + ",";
      nasa += "0.0f,0.0f,";
    }
    long long b;
    std::memcpy(&b, &m.Tmid[k], 8);
    tmb += std::to_string(b) + "LL,";
    iw += fpair(1.0 / m.W[k]) + ",";
    lw += fpair(std::log(m.W[k])) + ",";
  }
  g(fmt("__device__ const __align__(16) float kx_gcf[%d] = {%s0.0f};", 32 * ns + 4, nasa.c_str()));
  g(fmt("__device__ const long long kx_tmidb[%d] = {%s0LL};", ns + 1, tmb.c_str()));
  g(fmt("__device__ const float kx_iwf[%d] = {%s0.0f};", 2 * ns + 1, iw.c_str()));
  g(fmt("__device__ const float kx_lwf[%d] = {%s0.0f};", 2 * ns + 1, lw.c_str()));

  return cls;
}

void emit_rates_class_df(Out& o, Out& g, const Mechanism& m, const EmitOptions& opt, bool rop, OpCounts& c) {
  const int ns = m.ns;
  // The per-state scale 2^-S of the accumulation: up to 64 species it is set by the first rate and
  // raised when a later rate outgrows it (no extra pass over the reactions; 53/325: 8.4 -> 7.8 ms per
  // 2^20 states); larger mechanisms, whose rates span more decades and whose every rescale touches
  // more accumulators, bound all rates first in float32 (160/900: 142-150 against 158-160 ms per 2^22
  // states with the running scale)
  const bool bounded = ns > 64;
  // mixed precision: float32 rates, float-pair chemical potentials and Gibbs sums, float64 accumulation
  const bool mx = opt.mixed;
  std::vector<DfClass> cls = emit_class_tables(g, m);

  // ---- per state: T, ln T, 1/T, C_M, sigma, and the species vectors
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  o("#define KX_PF(p) kx_mk((p)[0], (p)[1])");
  o("const kx_df Td = kx_d2df_i(T);");
  o("const kx_df lnT = kx_df_log_d(T);");
  o("const kx_df iT = kx_df_div(kx_mk(1.0f, 0.0f), Td);");
  if (any_plog) o("const kx_df lnP = kx_df_log_d(P);");
  o(fmt("const kx_df cM = kx_df_mul(kx_df_mul(kx_d2df_i(P), iT), %s);", DFc(1.0 / R_U).c_str()));
  o(fmt("const kx_df lnPRT = kx_df_sub(%s, lnT);", DFc(std::log(P_ATM / R_U)).c_str()));
  if (opt.scratch && !rop) {
    // species vectors in the caller's global scratch, element k of this thread at k * nthr + gtid
    o("const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;");
    o("const kx_strided<float4> sv{(float4*)kx_scr + gtid, nthr};   // {ln |C_k| (pair), mu_k (pair)}");
    o(fmt("const kx_strided<kx_df> w{(kx_df*)(kx_scr + (long long)%d * 16 * nthr) + gtid, nthr};", ns));
  } else if (mx) {
    o(fmt("float4 sv[%d];   // {ln |C_k|, C_k (float32), mu_k (pair)}", ns));
    if (!rop) o(fmt("double w[%d];", ns));
  } else {
    o(fmt("float4 sv[%d];   // {ln |C_k| (pair), mu_k (pair)}", ns));
    if (!rop) o(fmt("kx_df w[%d];", ns));
  }
  o("kx_df sig = kx_mk(0.0f, 0.0f);");
  o(fmt("for (int k = 0; k < %d; ++k) sig = kx_df_fma(kx_d2df_i(Y_[(long long)k * ld + i]), KX_PF(kx_iwf + 2 * k), sig);", ns));
  o("if (!(sig.hi > 0.0f && sig.hi < KX_INF_F)) KX_BAD_POINT");
  o("const kx_df fC = kx_df_div(cM, sig);");
  o("const kx_df lnfC = kx_df_log(fC);");
  o("const long long Tb = __double_as_longlong(T);");
  // signs of the concentrations: bit k of the mask words set for Y_k < 0
  const int nw = (ns + 63) / 64;
  for (int q = 0; q < nw; ++q) o(fmt("unsigned long long nm%d = 0ull;", q));
  {
    std::string sel = fmt("nm%d", nw - 1);
    for (int q = nw - 2; q >= 0; --q) sel = fmt("((k) < %d ? nm%d : %s)", 64 * (q + 1), q, sel.c_str());
    o("#define KX_NEG(k) ((int)((" + sel + " >> ((k) & 63)) & 1ull))");
  }
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o("  const double Yk = Y_[(long long)k * ld + i];");
  o("  const long long yb = __double_as_longlong(Yk) & 0x7fffffffffffffffLL;");
  o("  // ln |C_k| = ln |Y_k| - ln W_k + ln(C_M/sigma), floored at -700 (Y_k = 0 or |Y_k| below 1e-304: absent)");
  o("  kx_df l = kx_mk(-700.0f, 0.0f);");
  o("  if (yb >= 0x0010000000000000LL && yb < 0x7ff0000000000000LL) {");
  o("    l = kx_df_add(kx_df_log_d(__longlong_as_double(yb)), kx_df_sub(lnfC, KX_PF(kx_lwf + 2 * k)));");
  o("    if (!(l.hi > -700.0f)) l = kx_mk(-700.0f, 0.0f);");
  o("  }");
  {
    std::string s = "  if (Yk < 0.0) {";
    for (int q = 0; q < nw; ++q) s += fmt(" %sif ((k >> 6) == %d) nm%d |= 1ull << (k & 63);", q ? "else " : "", q, q);
    o(s + " }");
  }
  o("  const float* a = kx_gcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("  kx_df gk = kx_df_fma(KX_PF(a + 8), Td, KX_PF(a + 6));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 4));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 2));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 0));");
  o("  gk = kx_df_fma(KX_PF(a + 10), iT, gk);");
  o("  gk = kx_df_fma(KX_PF(a + 12), lnT, gk);");
  o("  const kx_df mk_ = kx_df_add(gk, l);");
  if (mx) {
    o("  sv[k] = make_float4(l.hi, kx_df_mul(kx_d2df_i(Yk), KX_PF(kx_iwf + 2 * k)).hi * fC.hi, mk_.hi, mk_.lo);");
    if (!rop) o("  w[k] = 0.0;");
  } else {
    o("  sv[k] = make_float4(l.hi, l.lo, mk_.hi, mk_.lo);");
    if (!rop) o("  w[k] = kx_mk(0.0f, 0.0f);");
  }
  o("}");
  {   // no negative mass fraction in this state (the usual case): the sign parities are all 0
    std::string any = "nm0";
    for (int q = 1; q < nw; ++q) any += fmt(" | nm%d", q);
    o("const bool anyneg = (" + any + ") != 0ull;");
  }
  c.fp32 += 40 + 45 + kDfDiv + 2 * kDfMul + kDfAdd + kDfDiv + kDfLog;
  c.fp32 += ns * (12 + kDfFma) + ns * (45 + 2 * kDfAdd + 6 * kDfFma + kDfAdd);

  // Class loops are software-pipelined: each iteration loads the next
  // reaction's record and species vectors, and the accumulators of the
  // previous reaction, before computing its own rate; the previous rate is
  // added to its accumulators at the end.  Local-memory latency thus hides
  // behind one reaction's arithmetic.
  static const char* xyzw[4] = {"x", "y", "z", "w"};
  auto comp = [&](const char* base, int j) { return fmt("%s%d.%s", base, j / 4, xyzw[j % 4]); };
  auto spc = [&](const char* base, int j) { return fmt("(%s & 0xffff)", comp(base, j).c_str()); };
  auto prologue = [&](const DfClass& d, int ci) {
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    o(fmt("const int4* sp4 = (const int4*)kx_s%d;", ci));
    for (int q = 0; q < P / 4; ++q) o(fmt("int4 c%d = sp4[%d];", q, q));
    for (int j = 0; j < E; ++j) o(fmt("float4 v%d = sv[%s];", j, spc("c", j).c_str()));
  };
  auto prefetch = [&](const DfClass& d) {
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    for (int q = 0; q < P / 4; ++q) o(fmt("  const int4 n%d = sp4[%d * (r + 1) + %d];", q, P / 4, q));
    for (int j = 0; j < E; ++j) o(fmt("  const float4 u%d = sv[%s];", j, spc("n", j).c_str()));
  };
  auto advance = [&](const DfClass& d) {
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    for (int q = 0; q < P / 4; ++q) o(fmt("  c%d = n%d;", q, q));
    for (int j = 0; j < E; ++j) o(fmt("  v%d = u%d;", j, j));
  };

  if (mx) o("const float lnTf = lnT.hi, iTf = iT.hi, Tf = Td.hi, cMf = cM.hi;");
  if (mx && any_plog) o("const float lnPf = lnP.hi;");
  if (!rop && !mx && bounded) {
    o("const float lnTf = lnT.hi, iTf = iT.hi, Tf = Td.hi, lnPRTf = lnPRT.hi, lncMf = __logf(cM.hi);");
    o("float U = -1.0e30f;");
    for (size_t ci = 0; ci < cls.size(); ++ci) {
      const DfClass& d = cls[ci];
      const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const int NF = fo ? 7 : tb ? 3 : 2;
      o("{");
      ++o.ind;
      prologue(d, (int)ci);
      o("#pragma unroll 1");
      o(fmt("for (int r = 0; r < %d; ++r) {", (int)d.rx.size()));
      prefetch(d);
      o(fmt("  const float4* f = kx_f%d + %d * r;", (int)ci, NF));
      o("  const float4 f0 = f[0], f1 = f[1];");
      o(d.kconst ? "  float b = f0.x;" : "  float b = fmaf(f0.z, lnTf, fmaf(f1.x, iTf, f0.x));");
      if (d.kind == Kind::ThreeBody) {
        o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
        o("  b += e.y < 0 ? sv[kx_effd[e.x].k].x : lncMf + f1.z;");
      } else if (fo) {
        o("  const float4 f2 = f[2], f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
        o("  // ln F <= max(0, ln F_cent) (Troe); ln d + e ln T + max(0, ln base) (SRI)");
        if (d.blend == Blend::Troe)
          o("  const float lf = fmaxf(0.0f, __logf(f4.x * __expf(Tf * f5.x) + f4.z * __expf(Tf * f5.z) + __expf(f6.x * iTf)));");
        else if (d.blend == Blend::Sri)
          o("  const float lf = f5.z + f6.x * lnTf + fmaxf(0.0f, __logf(f4.x * __expf(f4.z * iTf) + __expf(Tf * f5.x)));");
        else
          o("  const float lf = 0.0f;");
        if (d.kind == Kind::ChemAct) o("  b = fmaf(f3.x, lnTf, fmaf(f3.z, iTf, f2.z)) + lf;");
        else o("  b += lf;");
      } else if (d.kind == Kind::Plog) {
        o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
        o("  const float* t = kx_plogf + 8 * e.x;");
        o("  b = -1.0e30f;");
        o("  for (int j = 0; j < e.y; ++j) b = fmaxf(b, fmaf(t[8 * j + 4], lnTf, fmaf(t[8 * j + 6], iTf, t[8 * j + 2])));");
      }
      for (int j = 0; j < d.nre; ++j) o(fmt("  b += v%d.x;", j));
      if (d.rev) {
        const int dn = d.npr - d.nre;
        std::string s = dn == 0 ? std::string("0.0f") : fmt("%s * lnPRTf", F(-dn).c_str());
        for (int j = 0; j < d.nre; ++j) s += fmt(" - v%d.z", j);
        for (int j = d.nre; j < d.nre + d.npr; ++j) s += fmt(" + v%d.z", j);
        o("  b += fmaxf(" + s + ", 0.0f);");
      }
      o("  U = fmaxf(U, b);");
      advance(d);
      o("}");
      --o.ind;
      o("}");
      c.fp32 += d.rx.size() * (8.0 + 2 * (d.nre + d.npr));
    }
    o("// largest scaled rate near 2^63.5; |S| < 2^11 keeps S ln2 exact to the float-pair precision");
    o("const int S = kx_rint(fminf(fmaxf(U * KX_LOG2E_F, -1000.0f), 1000.0f)) - 63;");
    o("const float lnSf = __fmul_rn(kx_i2f(S), 0.693147182f);   // S ln2 for the range tests of the scaled exponential");
  }

  if (!rop && !mx && !bounded) {
    // the state's scale 2^-S: set by its first rate (scaled to 2^62) and raised to a later rate (to
    // 2^62 again), with every accumulator rescaled, when that rate would land above 2^96.  The largest
    // scaled rate thus sits between 2^62 and 2^97, a running sum stays below ~2^116, and float pairs keep
    // their full precision for terms down to 2^-164 of the largest (anchoring the largest rate lower,
    // near 2^0, measured 5e-10 errors: rescaled partial sums fell into the subnormal range)
    o("int S = -100000;   // no rate yet");
  }

  // ---- main pass, one loop per class.  Emitted twice: for warps in which some state has a
  // negative mass fraction (signed concentration products), and for the usual warps without,
  // where a shadowing constant anyneg = false folds every sign parity away.
  auto main_pass = [&](OpCounts& c) {
    for (size_t ci = 0; ci < cls.size(); ++ci) {
      const DfClass& d = cls[ci];
      const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const int NF = fo ? 7 : tb ? 3 : 2;
      const int E = d.nre + d.npr;
      o(fmt("{   // class %d: %d reactions, %d reactant and %d product entries", (int)ci, (int)d.rx.size(), d.nre, d.npr));
      ++o.ind;
      prologue(d, (int)ci);
      if (!rop) {
        std::string pdecl = "int";
        for (int j = 0; j < E; ++j) pdecl += fmt("%s p%d = 0", j ? "," : "", j);
        o(pdecl + ";   // entries of the previous reaction (coefficient 0: nothing to add)");
        o(mx ? "double qp = 0.0;" : "kx_df qp = kx_mk(0.0f, 0.0f);");
      }
      o("#pragma unroll 1");
      o(fmt("for (int r = 0; r < %d; ++r) {", (int)d.rx.size()));
      if (!rop)
        for (int j = 0; j < E; ++j) o(fmt("  %s wl%d = w[p%d & 0xffff];", mx ? "const double" : "kx_df", j, j));
      prefetch(d);
      for (int j = 0; j < E; ++j) o(fmt("  const int k%d = %s;", j, spc("c", j).c_str()));
      if (rop) o(fmt("  const int ri = %s;", comp("c", E).c_str()));
      o(fmt("  const float4* f = kx_f%d + %d * r;", (int)ci, NF));
      o("  const float4 f0 = f[0], f1 = f[1];");
      if (mx) {
        emit_class_mixed_body(o, d, (int)ci, E, c);
      } else {
        if (tb) {
          o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
          o("  const float4 f2 = f[2];");
          o("  kx_df X;   // [X] = eff_default C_M + (C_M/sigma) sum_e (eff_e - eff_default) Y_e/W_e");
          o("  if (e.y < 0) {");
          o("    const int kc = kx_effd[e.x].k;");
          o("    X = kx_df_mul(kx_df_mul(kx_d2df_i(Y_[(long long)kc * ld + i]), KX_PF(kx_iwf + 2 * kc)), fC);");
          o("  } else {");
          o("    kx_df t = kx_mk(0.0f, 0.0f);");
          o("    for (int j = 0; j < e.y; ++j) {");
          o("      const kx_effd_t q = kx_effd[e.x + j];");
          o("      t = kx_df_fma(kx_mk(q.ahi, q.alo), kx_df_mul(kx_d2df_i(Y_[(long long)q.k * ld + i]), KX_PF(kx_iwf + 2 * q.k)), t);");
          o("    }");
          o("    X = kx_df_fma(kx_mk(f2.x, f2.y), cM, kx_df_mul(fC, t));");
          o("  }");
          c.fp32 += d.rx.size() * (kDfFma + kDfMul + 3 * (kDfFma + kDfMul + 12));
        }
        // Elementary and three-body reactions of a warp whose states all have this reaction's rate
        // below 2^-40 of their scale's anchor (2^(S+62), the largest rate so far; with the bounding
        // pass, the state's largest rate) take float32: their contribution is bounded by that rate,
        // and float32's relative error (~1e-4 with the logarithms' absolute error) leaves an error
        // below 1e-16 of the largest rate per reaction, three orders under the float-pair path's own
        // error on the largest rates.  The estimates take the float pairs' high parts.
        // Falloff and chemically activated reactions estimate their blended ln k in float32 (the
        // same formulas as the float-pair path below, with the fast exponential and logarithm).
        const bool fastp = !rop && opt.rates_negligible == 0 && (d.kind == Kind::Elementary || d.kind == Kind::ThreeBody || fo);
        if (fastp) {
          if (fo) {
            o("  const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
            o("  float lfe = fmaf(f0.z, lnT.hi, fmaf(f1.x, iT.hi, f0.x));   // ln k_inf (float32)");
            o("  const float lk0e = fmaf(f3.x, lnT.hi, fmaf(f3.z, iT.hi, f2.z));   // ln k_0");
            o("  const float lpe = lk0e - lfe + __logf(X.hi);   // ln Pr (nan for [X] < 0: no float32 path)");
            if (d.blend == Blend::Troe) {
              o("  const float lFc = __logf(f4.x * __expf(Td.hi * f5.x) + f4.z * __expf(Td.hi * f5.z) + __expf(f6.x * iT.hi)) * 0.434294482f;");
              o("  const float xe = fmaf(lpe, 0.434294482f, fmaf(-0.67f, lFc, -0.4f));");
              o("  const float fe = __fdividef(xe, fmaf(-0.14f, xe, fmaf(-1.27f, lFc, 0.75f)));");
              o("  const float lFe = __fdividef(2.30258509f * lFc, fmaf(fe, fe, 1.0f));   // ln F (Troe)");
            } else if (d.blend == Blend::Sri) {
              o("  const float lPe = lpe * 0.434294482f;");
              o("  const float lFe = f5.z + f6.x * lnT.hi + __fdividef(__logf(f4.x * __expf(f4.z * iT.hi) + __expf(Td.hi * f5.x)), "
                "fmaf(lPe, lPe, 1.0f));   // ln F (SRI)");
            } else {
              o("  const float lFe = 0.0f;");
            }
            o("  const float l1e = __logf(1.0f + __expf(-fabsf(lpe)));   // ln(1 + e^-|ln Pr|)");
            o(d.kind == Kind::Falloff ? "  lfe += (lpe < 0.0f ? lpe - l1e : -l1e) + lFe;   // k_inf Pr/(1+Pr) F"
                                      : "  lfe = lk0e + lFe - (lpe < 0.0f ? l1e : lpe + l1e);   // k_0 F/(1+Pr)");
            c.fp32 += d.rx.size() * 40.0;
          } else {
            o(d.kconst ? "  float lfe = f0.x;" : "  float lfe = fmaf(f0.z, lnT.hi, fmaf(f1.x, iT.hi, f0.x));   // ln |R_f| (float32)");
          }
          for (int j = 0; j < d.nre; ++j) o(fmt("  lfe += v%d.x;", j));
          o(d.kind == Kind::ThreeBody ? "  const float lxe = __logf(X.hi);   // ln [X] (nan for [X] <= 0: no float32 path)"
                                      : "  const float lxe = 0.0f;");
          o("  float lme = lfe + lxe;");
          if (d.rev) {
            const int dn = d.npr - d.nre;
            std::string t = dn == 0 ? std::string("0.0f") : fmt("%s * lnPRT.hi", F(-dn).c_str());
            for (int j = 0; j < d.nre; ++j) t += fmt(" - v%d.z", j);
            for (int j = d.nre; j < E; ++j) t += fmt(" + v%d.z", j);
            o("  const float lre = lfe + (" + t + ");   // ln |R_r| (float32)");
            o("  lme = fmaxf(lme, lre + lxe);");
          }
          std::string sfx = "0", srx = "0";
          for (int j = 0; j < d.nre; ++j) sfx += fmt(" ^ KX_NEG(k%d)", j);
          for (int j = d.nre; j < E; ++j) srx += fmt(" ^ KX_NEG(k%d)", j);
          o("  kx_df q;");
          o("  if (__all_sync(__activemask(), lme < __fmul_rn(kx_i2f(S + 22), 0.693147182f))) {");
          o("    const float sl = __fmul_rn(kx_i2f(S), 0.693147182f);   // the rate scaled by 2^-S");
          o("    float qf = __expf(lfe - sl);");
          o("    if (anyneg && (" + sfx + ")) qf = -qf;");
          if (d.rev) {
            o("    float qr = __expf(lre - sl);");
            o("    if (anyneg && (" + srx + ")) qr = -qr;");
            o("    qf -= qr;");
          }
          o("    q = kx_mk(qf, 0.0f);");
          o("  } else {");
          c.fp32 += d.rx.size() * (6.0 + d.nre + (d.rev ? E + 3 : 0));
        }
        o(d.kconst ? "  kx_df lk = kx_mk(f0.x, f0.y);   // k = A"
                   : "  kx_df lk = kx_df_fma_u(kx_mk(f0.z, f0.w), lnT, kx_df_fma_u(kx_mk(f1.x, f1.y), iT, kx_mk(f0.x, f0.y)));");
        if (fo) {
          if (!fastp) o("  const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
          o("  const kx_df lk0 = kx_df_fma(kx_mk(f3.x, f3.y), lnT, kx_df_fma(kx_mk(f3.z, f3.w), iT, kx_mk(f2.z, f2.w)));");
          o("  kx_df lnPr = kx_df_add(kx_df_sub(lk0, lk), kx_df_log(X));");
          o("  if (!(lnPr.hi > -690.775528f)) lnPr = kx_mk(-690.775528f, 0.0f);");
          o("  kx_df lnF = kx_mk(0.0f, 0.0f);");
          const std::string il10 = DFc(1.0 / std::log(10.0));
          if (d.blend == Blend::Troe) {
            o("  kx_df Fc = kx_df_exp_s(kx_df_mul(kx_mk(f6.x, f6.y), iT));");
            o("  Fc = kx_df_fma(kx_mk(f4.x, f4.y), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.x, f5.y))), Fc);");
            o("  Fc = kx_df_fma(kx_mk(f4.z, f4.w), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.z, f5.w))), Fc);");
            o(fmt("  const kx_df lFc = kx_df_mul(kx_df_log(Fc), %s);", il10.c_str()));
            o(fmt("  const kx_df xx = kx_df_fma(lnPr, %s, kx_df_fma(%s, lFc, %s));", il10.c_str(), DFc(-0.67).c_str(), DFc(-0.4).c_str()));
            o(fmt("  const kx_df ff = kx_df_div(xx, kx_df_fma(%s, xx, kx_df_fma(%s, lFc, %s)));", DFc(-0.14).c_str(), DFc(-1.27).c_str(),
                  DFc(0.75).c_str()));
            o(fmt("  lnF = kx_df_div(kx_df_mul(%s, lFc), kx_df_fma(ff, ff, kx_mk(1.0f, 0.0f)));", DFc(std::log(10.0)).c_str()));
            c.fp32 += d.rx.size() * (3 * (kDfMul + kDfExp) + 2 * kDfFma + kDfLog + kDfMul + 4 * kDfFma + 2 * kDfDiv + kDfMul);
          } else if (d.blend == Blend::Sri) {
            o(fmt("  const kx_df lPr = kx_df_mul(lnPr, %s);", il10.c_str()));
            o("  const kx_df base = kx_df_fma(kx_mk(f4.x, f4.y), kx_df_exp_s(kx_df_mul(kx_mk(f4.z, f4.w), iT)), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.x, f5.y))));");
            o("  lnF = kx_df_add(kx_mk(f5.z, f5.w), kx_df_fma(kx_mk(f6.x, f6.y), lnT, kx_df_div(kx_df_log(base), kx_df_fma(lPr, lPr, kx_mk(1.0f, 0.0f)))));");
            c.fp32 += d.rx.size() * (2 * (kDfMul + kDfExp) + kDfFma + kDfMul + kDfLog + 2 * kDfFma + kDfDiv + kDfAdd);
          }
          o("  // ln(Pr/(1+Pr)) (falloff) or ln(1/(1+Pr)) (chemically activated) from l1p = ln(1 + e^-|ln Pr|)");
          o("  const bool small = lnPr.hi < 0.0f;");
          o("  const kx_df l1p = kx_df_log1p(kx_df_exp_n(small ? lnPr : kx_df_neg(lnPr)));");
          if (d.kind == Kind::Falloff) o("  lk = kx_df_add(lk, kx_df_add(small ? kx_df_sub(lnPr, l1p) : kx_df_neg(l1p), lnF));");
          else o("  lk = kx_df_add(lk0, kx_df_sub(lnF, small ? l1p : kx_df_add(lnPr, l1p)));");
          c.fp32 += d.rx.size() * (2 * kDfFma + 2 * kDfAdd + kDfLog + kDfExp + kDfLog + 3 * kDfAdd);
        } else if (d.kind == Kind::Plog) {
          o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
          o("  const float* t = kx_plogf + 8 * e.x; const long long* tp = kx_plogp + e.x; const int np = e.y;");
          o("  const long long Pb = __double_as_longlong(P);");
          o("  if (Pb <= tp[0]) lk = kx_df_fma(KX_PF(t + 4), lnT, kx_df_fma(KX_PF(t + 6), iT, KX_PF(t + 2)));");
          o("  else if (Pb >= tp[np - 1]) { const float* u = t + 8 * (np - 1); lk = kx_df_fma(KX_PF(u + 4), lnT, kx_df_fma(KX_PF(u + 6), iT, KX_PF(u + 2))); }");
          o("  else {");
          o("    int j = 0; while (!(Pb < tp[j + 1])) ++j;");
          o("    const float* u = t + 8 * j;");
          o("    const kx_df l1 = kx_df_fma(KX_PF(u + 4), lnT, kx_df_fma(KX_PF(u + 6), iT, KX_PF(u + 2)));");
          o("    const kx_df l2 = kx_df_fma(KX_PF(u + 12), lnT, kx_df_fma(KX_PF(u + 14), iT, KX_PF(u + 10)));");
          o("    lk = kx_df_fma(kx_df_sub(l2, l1), kx_df_div(kx_df_sub(lnP, KX_PF(u)), kx_df_sub(KX_PF(u + 8), KX_PF(u))), l1);");
          o("  }");
          c.fp32 += d.rx.size() * (4 * kDfFma + 3 * kDfAdd + kDfDiv);
        }
        // ln |R_f| (scaled by 2^-S) and the sign of prod C^nu'
        o("  kx_df lf = lk;");
        for (int j = 0; j < d.nre; ++j) o(fmt("  lf = kx_df_add_u(lf, kx_mk(v%d.x, v%d.y));", j, j));
        std::string sfx = "0", srx = "0";
        for (int j = 0; j < d.nre; ++j) sfx += fmt(" ^ KX_NEG(k%d)", j);
        for (int j = d.nre; j < E; ++j) srx += fmt(" ^ KX_NEG(k%d)", j);
        o("  int sf = anyneg ? (" + sfx + ") : 0;");
        o("  kx_df L = lf, fac = kx_mk(1.0f, 0.0f);");
        o("  bool rev = false;");
        c.fp32 += d.rx.size() * ((d.kconst ? 0 : 2 * kDfFma) + d.nre * kDfAdd + kDfExp + kDfMul);
        if (d.rev) {
          const int dn = d.npr - d.nre;
          o("  {   // ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T))");
          std::string first = d.nre > 0 ? "kx_df_neg(kx_mk(v0.z, v0.w))" : "kx_mk(v0.z, v0.w)";
          o("    kx_df dl = " + first + ";");
          for (int j = 1; j < E; ++j)
            o(fmt("    dl = kx_df_add_u(dl, kx_mk(%sv%d.z, %sv%d.w));", j < d.nre ? "-" : "", j, j < d.nre ? "-" : "", j));
          if (dn == 1 || dn == -1) o(fmt("    dl = kx_df_add_u(dl, %s);", dn == 1 ? "kx_df_neg(lnPRT)" : "lnPRT"));
          else if (dn != 0) o(fmt("    dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, %s));", F(-dn).c_str()));
          o("    const int sr = anyneg ? (" + srx + ") : 0;");
          o("    rev = dl.hi > 0.0f;");
          o("    if (rev) L = kx_df_add_u(lf, dl);");
          o("    const kx_df e = kx_df_exp_n(rev ? kx_df_neg(dl) : dl);");
          o("    // |R_f| -+ |R_r| = larger (1 -+ e^-|ln ratio|): minus for equal signs, plus for opposite signs");
          o("    const float pm = sf == sr ? -1.0f : 1.0f;");
          o("    const kx_df s1 = kx_qts(1.0f, pm * e.hi);");
          o("    fac = kx_mk(s1.hi, __fmaf_rn(pm, e.lo, s1.lo));");
          o("    if (sf == sr) sf ^= (int)rev;");
          o("  }");
          c.fp32 += d.rx.size() * ((E - 1) * kDfAdd + (dn ? kDfAdd + kDfMulf : 0) + kDfAdd + kDfExp + 10);
        }
        if (rop) {
          o("  const int Sr = kx_rint(fminf(fmaxf(L.hi * KX_LOG2E_F, -1000.0f), 1000.0f));");
          o("  kx_df q = kx_df_mul_u(kx_df_exp_sc(L, Sr, __fmul_rn(kx_i2f(Sr), 0.693147182f)), fac);");
          c.fp32 += d.rx.size() * 4;
        } else {
          const std::string qd = fastp ? "q" : "kx_df q";
          if (bounded) {
            o("  " + qd + " = kx_df_mul_u(kx_df_exp_sc(L, S, lnSf), fac);   // |R| 2^-S (the products and sums after it take hi + lo as is)");
          } else {
          o("  int ex;");
          o("  " + qd + " = kx_df_mul_u(kx_df_exp_m(L, ex), fac);   // |R| = q 2^ex (products and sums after it take hi + lo as is)");
          o("  if (ex > S + 96) {   // the state's first rate, or one 2^34 above its scale's anchor: raise the scale");
          o("    // 2^d in two exact steps (each at least 2^-126): sums still representable after a jump of more");
          o("    // than 2^126 keep their value");
          o("    const int d = S - (ex - 62), d1 = max(d, -126), d2 = d - d1;");
          o("    const float f1 = __int_as_float((d1 + 127) << 23), f2 = d2 >= -126 ? __int_as_float((d2 + 127) << 23) : 0.0f;");
          o(fmt("    for (int k = 0; k < %d; ++k) w[k] = kx_mk(__fmul_rn(__fmul_rn(w[k].hi, f1), f2), __fmul_rn(__fmul_rn(w[k].lo, f1), f2));", ns));
          for (int j = 0; j < E; ++j)
            o(fmt("    wl%d = kx_mk(__fmul_rn(__fmul_rn(wl%d.hi, f1), f2), __fmul_rn(__fmul_rn(wl%d.lo, f1), f2));", j, j, j));
          o("    qp = kx_mk(__fmul_rn(__fmul_rn(qp.hi, f1), f2), __fmul_rn(__fmul_rn(qp.lo, f1), f2));");
          o("    S = ex - 62;");
          o("  }");
          o("  { const int d = ex - S; const float sc = d >= -126 ? __int_as_float((d + 127) << 23) : 0.0f; "
            "q = kx_mk(__fmul_rn(q.hi, sc), __fmul_rn(q.lo, sc)); }   // q 2^(ex - S)");
          }
        }
        o("  if (sf) q = kx_df_neg(q);");
        if (fastp) o("  }");
        if (d.kind == Kind::ThreeBody) { o("  q = kx_df_mul_u(q, X);"); c.fp32 += d.rx.size() * kDfMul; }
      }
      if (rop) {
        o(mx ? "  out_[(long long)ri * ld + i] = q;" : "  out_[(long long)ri * ld + i] = kx_df2d_s(q, Sr);");
        c.fp64 += d.rx.size();
      } else if (mx) {
        for (int j = 0; j < E; ++j)
          o(fmt("  { const unsigned cj = (unsigned)p%d & 0xffff0000u; if (cj != 0u) w[p%d & 0xffff] = fma(kx_f2d(__uint_as_float(cj)), qp, wl%d); }", j, j, j));
        o("  qp = q;");
        for (int j = 0; j < E; ++j) o(fmt("  p%d = %s;", j, comp("c", j).c_str()));
        c.fp64 += d.rx.size() * E;
      } else {
        // the previous reaction's rate into its accumulators (loaded at the top of this iteration)
        for (int j = 0; j < E; ++j)
          o(fmt("  { const unsigned cj = (unsigned)p%d & 0xffff0000u; if (cj != 0u) w[p%d & 0xffff] = kx_df_add_u(wl%d, %s(qp, __uint_as_float(cj))); }",
                j, j, j, d.maxnu <= 2 ? "kx_df_scale2" : "kx_df_mulf"));
        o("  qp = q;");
        for (int j = 0; j < E; ++j) o(fmt("  p%d = %s;", j, comp("c", j).c_str()));
        c.fp32 += d.rx.size() * E * (kDfAdd + kDfMulf) / 2.0;
      }
      advance(d);
      o("}");
      if (!rop && mx)
        for (int j = 0; j < E; ++j)
          o(fmt("{ const unsigned cj = (unsigned)p%d & 0xffff0000u; if (cj != 0u) { const int kk = p%d & 0xffff; w[kk] = fma(kx_f2d(__uint_as_float(cj)), qp, w[kk]); } }",
                j, j));
      else if (!rop)
        for (int j = 0; j < E; ++j)
          o(fmt("{ const unsigned cj = (unsigned)p%d & 0xffff0000u; if (cj != 0u) { const int kk = p%d & 0xffff; w[kk] = kx_df_add_u(w[kk], %s(qp, __uint_as_float(cj))); } }",
                j, j, d.maxnu <= 2 ? "kx_df_scale2" : "kx_df_mulf"));
      --o.ind;
      o("}");
    }
  };
  o("if (__any_sync(__activemask(), anyneg)) {");
  ++o.ind;
  main_pass(c);
  --o.ind;
  o("} else {");
  ++o.ind;
  o("const bool anyneg = false;   // no state of this warp has a negative mass fraction");
  {
    OpCounts once;   // the operations are counted for one of the two copies
    main_pass(once);
  }
  --o.ind;
  o("}");
  if (!rop) {
    o(fmt(mx ? "for (int k = 0; k < %d; ++k) out_[(long long)k * ld + i] = w[k];"
             : "for (int k = 0; k < %d; ++k) out_[(long long)k * ld + i] = kx_df2d_s(w[k], S);", ns));
    c.fp64 += mx ? 0 : ns;
  }
}

// ------------------------------------------------------------------ adjoint
// Vector-Jacobian product of the production rates at fixed p.  With
// a_i = sum_k nu_ki v_k, v^T wdot = sum_i a_i q_i, so each reaction adds
// a_i dq_i to the adjoints of its own inputs (T, C_k, G_k/RT, [M]) in one
// forward sweep; nothing is stored per reaction.  The chain to (T, Y) is
// closed per point at the end: dG_k/RT/dT = -H_k/(R T^2) (Gibbs-Helmholtz),
// C_k = [M] y_k / sigma with [M] = p/(R T), y_k = Y_k/W_k, sigma = sum y.
// For q = c (R_f - R_r), R_f = k_f prod C^nu', R_r = k_r prod C^nu'',
// ln k_r = ln k_f + sum nu G/RT - dn ln(p_atm/(R T)):
//   dq/dT|_C,G = c ((R_f - R_r) dln k_f/dT - R_r dn/T),
//   dq/dG_k = -c R_r nu_k,  dq/dC_k = c (nu'_k R_f - nu''_k R_r)/C_k.
std::string dln_arrh(const Arrh& a) {
  if (a.E == 0.0) return a.beta == 0.0 ? std::string("0.0") : fmt("%s * iT", D(a.beta).c_str());
  return fmt("fma(%s, iT, %s) * iT", D(a.E).c_str(), D(a.beta).c_str());
}

// product of the concentrations of `side` with one factor of species k removed
std::string conc_product_without(const std::vector<std::pair<int, int>>& side, int k) {
  std::string s;
  bool removed = false;
  for (auto& e : side)
    for (int n = 0; n < e.second; ++n) {
      if (e.first == k && !removed) { removed = true; continue; }
      s += " * C_" + std::to_string(e.first);
    }
  return s;
}

void emit_vjp64(Out& o, const Mechanism& m, OpCounts& c) {
  const auto used = species_used(m);
  const auto need_g = gibbs_needed(m);
  const auto flags = tmid_flags(m);
  o("const double lnT = log(T);");
  o("const double iT = 1.0 / T;");
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  if (any_plog) o("const double lnP = kx_log(P);");
  emit_concentrations64(o, m, used, c);
  for (auto& f : flags) o(fmt("const bool lo%d = T < %s;", f.second, D(f.first).c_str()));
  for (int k = 0; k < m.ns; ++k)
    if (need_g[k]) emit_gibbs64(o, m, k, nasa_flag(m, k, flags), c);
  o(fmt("const double lnPRT = %s - lnT;", D(std::log(P_ATM / R_U)).c_str()));
  for (int k = 0; k < m.ns; ++k) o(fmt("const double v_%d = V_[(long long)%d * ld + i];", k, k));
  for (int k = 0; k < m.ns; ++k) o(fmt("double gC_%d = 0.0;", k));
  for (int k = 0; k < m.ns; ++k)
    if (need_g[k]) o(fmt("double gg_%d = 0.0;", k));
  o("double gT = 0.0, gM = 0.0;");
  for (int i = 0; i < m.nr(); ++i) {
    const Reaction& r = m.rx[i];
    o(fmt("{  // reaction %d", i));
    ++o.ind;
    std::map<int, int> nu;
    for (auto& e : r.prod) nu[e.first] += e.second;
    for (auto& e : r.reac) nu[e.first] -= e.second;
    std::string a;
    for (auto& kv : nu) {
      if (kv.second == 0) continue;
      std::string t = fmt("v_%d", kv.first);
      if (a.empty()) a = kv.second == 1 ? t : kv.second == -1 ? "-" + t : fmt("%s * %s", D(kv.second).c_str(), t.c_str());
      else a = kv.second == 1 ? a + " + " + t : kv.second == -1 ? a + " - " + t : fmt("fma(%s, %s, %s)", D(kv.second).c_str(), t.c_str(), a.c_str());
    }
    o("const double a = " + (a.empty() ? std::string("0.0") : a) + ";");
    bool has_dX = false;
    if (r.kind == Kind::Elementary || r.kind == Kind::ThreeBody) {
      o(fmt("const double lkf = %s;", ln_arrh64(r.k, c).c_str()));
      o("const double kf = kx_exp(lkf);");
      o("const double dT = " + dln_arrh(r.k) + ";");
    } else if (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) {
      o(fmt("const double lk0 = %s, dk0 = %s;", ln_arrh64(r.k0, c).c_str(), dln_arrh(r.k0).c_str()));
      o(fmt("const double lki = %s, dki = %s;", ln_arrh64(r.k, c).c_str(), dln_arrh(r.k).c_str()));
      o(fmt("const double X = %s;", third_body64(r, c).c_str()));
      o("const double lnPr = fmax(lk0 - lki + kx_log(X), -690.77552789821368);");
      o("const double Pr = kx_exp(lnPr);");
      o("const double ipr = 1.0 / (1.0 + Pr);");
      if (r.blend == Blend::Troe) {
        const double al = r.troe[0];
        o(fmt("const double e3 = %s * kx_exp(T * %s), e1 = %s * kx_exp(T * %s), e2 = kx_exp(%s * iT);", D(1.0 - al).c_str(),
              D(-1.0 / r.troe[1]).c_str(), D(al).c_str(), D(-1.0 / r.troe[2]).c_str(), D(-r.troe[3]).c_str()));
        o(fmt("const double Fc = e3 + e1 + e2, dFc = e3 * %s + e1 * %s + e2 * %s * iT * iT;", D(-1.0 / r.troe[1]).c_str(),
              D(-1.0 / r.troe[2]).c_str(), D(r.troe[3]).c_str()));
        o("const double lFc = kx_log(Fc) * KX_INV_LN10;");
        o("const double xx = fma(lnPr, KX_INV_LN10, fma(-0.67, lFc, -0.4));");
        o("const double nn = fma(-1.27, lFc, 0.75);");
        o("const double den = nn - 0.14 * xx, iden = 1.0 / den;");
        o("const double ff = xx * iden, g1 = 1.0 / fma(ff, ff, 1.0);");
        o("const double F = kx_exp(KX_LN10 * lFc * g1);");
        o("const double h2 = -2.0 * ff * g1 * g1 * lFc;");
        o("const double dF_lnPr = h2 * nn * iden * iden;");
        o("const double dF_T = fma(h2, fma(-0.67, den, 1.1762 * xx) * iden * iden, g1) * dFc / Fc;");
      } else if (r.blend == Blend::Sri) {
        o("const double lPr = lnPr * KX_INV_LN10, Xs = 1.0 / fma(lPr, lPr, 1.0);");
        o(fmt("const double ea = %s * kx_exp(%s * iT), eb = kx_exp(T * %s);", D(r.sri[0]).c_str(), D(-r.sri[1]).c_str(),
              D(-1.0 / r.sri[2]).c_str()));
        o("const double base = ea + eb, lnb = kx_log(base);");
        o(fmt("const double F = %s * kx_exp(fma(%s, lnT, Xs * lnb));", D(r.sri[3]).c_str(), D(r.sri[4]).c_str()));
        o("const double dF_lnPr = -2.0 * lPr * Xs * Xs * lnb * KX_INV_LN10;");
        o(fmt("const double dF_T = %s * iT + Xs * (ea * %s * iT * iT + eb * %s) / base;", D(r.sri[4]).c_str(),
              D(r.sri[1]).c_str(), D(-1.0 / r.sri[2]).c_str()));
      } else {
        o("const double F = 1.0, dF_lnPr = 0.0, dF_T = 0.0;");
      }
      if (r.kind == Kind::Falloff) {
        o("const double kf = kx_exp(lki) * (Pr * ipr) * F;");
        o("const double dP = ipr + dF_lnPr;");
        o("const double dT = fma(dk0 - dki, dP, dki) + dF_T;");
      } else {
        o("const double kf = kx_exp(lk0) * ipr * F;");
        o("const double dP = dF_lnPr - Pr * ipr;");
        o("const double dT = fma(dk0 - dki, dP, dk0) + dF_T;");
      }
      o("const double dX = dP / X;");
      has_dX = true;
    } else {  // PLOG
      const auto& t = r.plog;
      auto lk = [&](size_t j) { return ln_arrh64(Arrh{t[j][1], t[j][2], t[j][3]}, c); };
      auto dk = [&](size_t j) { return dln_arrh(Arrh{t[j][1], t[j][2], t[j][3]}); };
      o("double lkf, dT;");
      o(fmt("if (P <= %s) { lkf = %s; dT = %s; }", D(t[0][0]).c_str(), lk(0).c_str(), dk(0).c_str()));
      for (size_t j = 0; j + 1 < t.size(); ++j) {
        double l1 = std::log(t[j][0]), l2 = std::log(t[j + 1][0]);
        o(fmt("else if (P < %s) { const double w = (lnP - %s) * %s; const double l1 = %s, d1 = %s; lkf = fma(%s - l1, w, l1); dT = fma(%s - d1, w, d1); }",
              D(t[j + 1][0]).c_str(), D(l1).c_str(), D(1.0 / (l2 - l1)).c_str(), lk(j).c_str(), dk(j).c_str(), lk(j + 1).c_str(),
              dk(j + 1).c_str()));
      }
      o(fmt("else { lkf = %s; dT = %s; }", lk(t.size() - 1).c_str(), dk(t.size() - 1).c_str()));
      o("const double kf = kx_exp(lkf);");
    }
    const int dn = sum_nu(r);
    o("const double Rf = kf" + conc_product(r.reac, "C_") + ";");
    if (r.reversible) {
      std::string lnkc = nu_sum(r, "g", c);
      std::string lk = dn == 0 ? "-(" + lnkc + ")" : fmt("fma(%s, lnPRT, -(%s))", D(dn).c_str(), lnkc.c_str());
      o("const double kr = kf * kx_exp(-(" + lk + "));");
      o("const double Rr = kr" + conc_product(r.prod, "C_") + ";");
    } else {
      o("const double kr = 0.0, Rr = 0.0;");
    }
    std::string cm = "1.0";
    if (r.kind == Kind::ThreeBody) {
      o(fmt("const double X = %s;", third_body64(r, c).c_str()));
      cm = "X";
    }
    o("const double aq = a * " + cm + ";");
    o(dn != 0 ? fmt("gT = fma(aq, fma(Rf - Rr, dT, %s * Rr * iT), gT);", D(-dn).c_str())
              : std::string("gT = fma(aq, (Rf - Rr) * dT, gT);"));
    if (r.reversible)
      for (auto& kv : nu)
        if (kv.second != 0) o(fmt("gg_%d = fma(%s, aq * Rr, gg_%d);", kv.first, D(-kv.second).c_str(), kv.first));
    // concentration adjoints from the mass-action products
    std::map<int, int> f_nu, r_nu;
    for (auto& e : r.reac) f_nu[e.first] += e.second;
    for (auto& e : r.prod) r_nu[e.first] += e.second;
    for (auto& kv : f_nu)
      o(fmt("gC_%d = fma(aq, %s * kf%s, gC_%d);", kv.first, D(kv.second).c_str(), conc_product_without(r.reac, kv.first).c_str(),
            kv.first));
    if (r.reversible)
      for (auto& kv : r_nu)
        o(fmt("gC_%d = fma(aq, %s * kr%s, gC_%d);", kv.first, D(-kv.second).c_str(), conc_product_without(r.prod, kv.first).c_str(),
              kv.first));
    // third-body adjoint gX, distributed over [M] and the listed species
    std::string gX;
    if (r.kind == Kind::ThreeBody) gX = "a * (Rf - Rr)";
    else if (has_dX) gX = "a * (Rf - Rr) * dX";
    if (!gX.empty()) {
      o("const double gX = " + gX + ";");
      if (r.collider >= 0) {
        o(fmt("gC_%d += gX;", r.collider));
      } else {
        o(r.default_eff == 1.0 ? std::string("gM += gX;") : fmt("gM = fma(%s, gX, gM);", D(r.default_eff).c_str()));
        for (auto& e : r.eff) {
          const double d = e.second - r.default_eff;
          if (d != 0.0) o(fmt("gC_%d = fma(%s, gX, gC_%d);", e.first, D(d).c_str(), e.first));
        }
      }
    }
    --o.ind;
    o("}");
  }
  // close the chain: G_k/RT(T), C_k([M], y), [M](T)
  for (int k = 0; k < m.ns; ++k) {
    if (!need_g[k]) continue;
    const std::string fl = nasa_flag(m, k, flags);
    const double* lo = &m.a_lo[7 * k];
    const double* hi = &m.a_hi[7 * k];
    std::string h = sel(fl, lo[4] / 5.0, hi[4] / 5.0);
    for (int n = 3; n >= 0; --n) h = fmt("fma(%s, T, %s)", h.c_str(), sel(fl, lo[n] / (n + 1), hi[n] / (n + 1)).c_str());
    h = fmt("fma(%s, iT, %s)", sel(fl, lo[5], hi[5]).c_str(), h.c_str());
    o(fmt("gT = fma(-gg_%d * iT, %s, gT);", k, h.c_str()));
  }
  std::string sx = "0.0";
  for (int k = 0; k < m.ns; ++k)
    if (used[k]) sx = fmt("fma(gC_%d, C_%d, %s)", k, k, sx.c_str());
  o("const double gCX = " + sx + ";");            // sum_k gC_k C_k
  o("gM += gCX / cM;");
  o("gT_[i] = fma(-gM * cM, iT, gT);");
  // dC_k/dy_j = fC (delta_kj - X_k), X_k = C_k/[M]
  o("const double gavg = gCX / cM;");
  for (int k = 0; k < m.ns; ++k)
    o(fmt("gY_[(long long)%d * ld + i] = fC * (%s - gavg) * %s;", k, used[k] ? fmt("gC_%d", k).c_str() : "0.0", D(1.0 / m.W[k]).c_str()));
}

// Vector-Jacobian product of the production rates in double-float
// arithmetic on the float32 pipe (float64 accuracy), thread per state, one
// loop per reaction class over the forward kernel's tables.  With
// a_i = sum_k nu_ki v_k, v^T wdot = sum_i a_i q_i, so each reaction adds a_i
// dq_i to the adjoints of its own inputs; every term is formed from the
// log-space rates as a float-pair mantissa times a power of two:
//   d/dT (at fixed C, G/RT):  a_i c_i ((R_f - R_r) dln k_f/dT - dn R_r / T),
//   d/d(G_k/RT):             -a_i c_i nu_k R_r,
//   d/dC_k:                  a_i c_i (nu'_k R_f - nu''_k R_r) / C_k, one term
//                            exp(ln |R| - ln |C_k|) per entry (so absent
//                            species, C_k = 0, keep their exact derivative),
//   d/d[X] (third body):     a_i (R_f - R_r) (times dln k_f/d[X] for falloff).
// The rates span hundreds of decades and R/C_k more, so every accumulator
// carries its own running power-of-two scale (kx_acc_add).  The chain to
// (T, Y) is closed per state in float64: Gibbs-Helmholtz for G_k/RT(T),
// C_k = [M] y_k / sigma with [M] = p/(R T).
void emit_vjp_df(Out& o, Out& g, const Mechanism& m, OpCounts& c, bool recip) {
  const int ns = m.ns;
  // a rate below float64 (ln |R| <= -740, where an absent species meets other small factors) keeps
  // its exact mantissa and power of two: e^x = 2^-2016 e^(x + 2016 ln2), the shift a float pair
  // (1.7e-12 relative off 2016 ln2, so such a rate is off by at most that much)
  const std::string shift = DFc(2016.0 * std::log(2.0));
  std::vector<DfClass> cls = emit_class_tables(g, m);
  // H/RT coefficients per species and NASA range: a0, a1/2, a2/3, a3/4, a4/5 (in T) and a5 (over T)
  {
    std::string hc, iwd;
    for (int k = 0; k < ns; ++k) {
      for (int rg = 0; rg < 2; ++rg) {
        const double* a = rg == 0 ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
        const double h[6] = {a[0], a[1] / 2.0, a[2] / 3.0, a[3] / 4.0, a[4] / 5.0, a[5]};
        for (int j = 0; j < 6; ++j) hc += D(h[j]) + ",";
      }
      iwd += D(1.0 / m.W[k]) + ",";
    }
    g(fmt("__device__ const double kx_hrt[%d] = {%s0.0};", 12 * ns + 1, hc.c_str()));
    std::string hf;
    for (int k = 0; k < ns; ++k)
      for (int rg = 0; rg < 2; ++rg) {
        const double* a = rg == 0 ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
        const double h[8] = {a[0], a[1] / 2.0, a[2] / 3.0, a[3] / 4.0, a[4] / 5.0, a[5], 0.0, 0.0};
        for (int j = 0; j < 8; ++j) hf += fpair(h[j]) + ",";
      }
    g(fmt("__device__ const __align__(16) float kx_hcf[%d] = {%s0.0f};", 32 * ns + 4, hf.c_str()));
    g(fmt("__device__ const double kx_iwd[%d] = {%s0.0};", ns + 1, iwd.c_str()));
  }
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  o("#define KX_PF(p) kx_mk((p)[0], (p)[1])");
  o("const kx_df Td = kx_d2df_i(T);");
  o("const kx_df lnT = kx_df_log_d(T);");
  o("const kx_df iT = kx_df_div(kx_mk(1.0f, 0.0f), Td);");
  o("const kx_df iT2 = kx_df_mul(iT, iT);");
  if (any_plog) o("const kx_df lnP = kx_df_log_d(P);");
  o(fmt("const kx_df cM = kx_df_mul(kx_df_mul(kx_d2df_i(P), iT), %s);", DFc(1.0 / R_U).c_str()));
  o(fmt("const kx_df lnPRT = kx_df_sub(%s, lnT);", DFc(std::log(P_ATM / R_U)).c_str()));
  o(fmt("float4 sv[%d];   // {ln |C_k| (pair), mu_k = G_k/RT + ln |C_k| (pair)}", ns));
  o(fmt("float2 yv[%d];   // Y_k/W_k (pair)", ns));
  o(fmt("float4 vh[%d];   // {cotangent v_k (pair), H_k/RT (pair)}", ns));
  if (recip) o(fmt("float4 ic[%d];   // 1/|C_k| = {mantissa (pair), power of two (int bits), 0}", ns));
  o(fmt("kx_acc gc[%d];   // adjoints of C_k, each a float pair under its own scale 2^-s", ns));
  o("kx_df gTa = kx_mk(0.0f, 0.0f), gMa = kx_mk(0.0f, 0.0f);   // adjoints of T (fixed C) and of [M]");
  o("int sT = -100000, sM = -100000;");
  o("kx_df sig = kx_mk(0.0f, 0.0f);");
  o(fmt("for (int k = 0; k < %d; ++k) sig = kx_df_fma(kx_d2df_i(Y_[(long long)k * ld + i]), KX_PF(kx_iwf + 2 * k), sig);", ns));
  o("if (!(sig.hi > 0.0f && sig.hi < KX_INF_F)) KX_BAD_POINT");
  o("const kx_df fC = kx_df_div(cM, sig);");
  o("const kx_df lnfC = kx_df_log(fC);");
  o("const long long Tb = __double_as_longlong(T);");
  const int nw = (ns + 63) / 64;
  for (int q = 0; q < nw; ++q) o(fmt("unsigned long long nm%d = 0ull;", q));
  {
    std::string sel = fmt("nm%d", nw - 1);
    for (int q = nw - 2; q >= 0; --q) sel = fmt("((k) < %d ? nm%d : %s)", 64 * (q + 1), q, sel.c_str());
    o("#define KX_NEG(k) ((int)((" + sel + " >> ((k) & 63)) & 1ull))");
  }
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o("  const double Yk = Y_[(long long)k * ld + i];");
  o("  const long long yb = __double_as_longlong(Yk) & 0x7fffffffffffffffLL;");
  o("  kx_df l = kx_mk(-700.0f, 0.0f);   // ln |C_k|, floored at -700 (absent species)");
  o("  if (yb >= 0x0010000000000000LL && yb < 0x7ff0000000000000LL) {");
  o("    l = kx_df_add(kx_df_log_d(__longlong_as_double(yb)), kx_df_sub(lnfC, KX_PF(kx_lwf + 2 * k)));");
  o("    if (!(l.hi > -700.0f)) l = kx_mk(-700.0f, 0.0f);");
  o("  }");
  {
    std::string s = "  if (Yk < 0.0) {";
    for (int q = 0; q < nw; ++q) s += fmt(" %sif ((k >> 6) == %d) nm%d |= 1ull << (k & 63);", q ? "else " : "", q, q);
    o(s + " }");
  }
  o("  const float* a = kx_gcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("  kx_df gk = kx_df_fma(KX_PF(a + 8), Td, KX_PF(a + 6));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 4));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 2));");
  o("  gk = kx_df_fma(gk, Td, KX_PF(a + 0));");
  o("  gk = kx_df_fma(KX_PF(a + 10), iT, gk);");
  o("  gk = kx_df_fma(KX_PF(a + 12), lnT, gk);");
  o("  const kx_df mk_ = kx_df_add(gk, l);");
  o("  sv[k] = make_float4(l.hi, l.lo, mk_.hi, mk_.lo);");
  o("  const kx_df yk = kx_df_mul(kx_d2df_i(Yk), KX_PF(kx_iwf + 2 * k));");
  o("  yv[k] = make_float2(yk.hi, yk.lo);");
  o("  const kx_df vk = kx_d2df_i(V_[(long long)k * ld + i]);");
  o("  const float* hc = kx_hcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("  kx_df hk = kx_df_fma(KX_PF(hc + 8), Td, KX_PF(hc + 6));");
  o("  hk = kx_df_fma(hk, Td, KX_PF(hc + 4));");
  o("  hk = kx_df_fma(hk, Td, KX_PF(hc + 2));");
  o("  hk = kx_df_fma(hk, Td, KX_PF(hc + 0));");
  o("  hk = kx_df_fma(KX_PF(hc + 10), iT, hk);   // H_k/RT");
  o("  vh[k] = make_float4(vk.hi, vk.lo, hk.hi, hk.lo);");
  if (recip) o("  { int e; const kx_df mi = kx_df_exp_m(kx_df_neg(l), e); ic[k] = make_float4(mi.hi, mi.lo, __int_as_float(e), 0.0f); }");
  o("  gc[k] = kx_acc{0.0f, 0.0f, -100000, 0};");
  o("}");
  c.fp32 += 40 + 45 + kDfDiv + 3 * kDfMul + kDfAdd + kDfDiv + kDfLog;
  c.fp32 += ns * (12 + kDfFma) + ns * (45 + 2 * kDfAdd + 6 * kDfFma + kDfAdd + kDfMul);

  static const char* xyzw[4] = {"x", "y", "z", "w"};
  auto comp = [&](const char* base, int j) { return fmt("%s%d.%s", base, j / 4, xyzw[j % 4]); };
  const std::string il10 = DFc(1.0 / std::log(10.0));
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    const DfClass& d = cls[ci];
    const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const int NF = fo ? 7 : tb ? 3 : 2;
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    const double NC = (double)d.rx.size();
    o(fmt("{   // class %d: %d reactions, %d reactant and %d product entries", (int)ci, (int)d.rx.size(), d.nre, d.npr));
    ++o.ind;
    o("#pragma unroll 1");
    o(fmt("for (int r = 0; r < %d; ++r) {", (int)d.rx.size()));
    o(fmt("  const int4* sp4 = (const int4*)kx_s%d + %d * r;", (int)ci, P / 4));
    for (int q = 0; q < P / 4; ++q) o(fmt("  const int4 c%d = sp4[%d];", q, q));
    for (int j = 0; j < E; ++j) o(fmt("  const int k%d = %s & 0xffff;", j, comp("c", j).c_str()));
    for (int j = 0; j < E; ++j) o(fmt("  const float4 v%d = sv[k%d];", j, j));
    o(fmt("  const float4* f = kx_f%d + %d * r;", (int)ci, NF));
    o("  const float4 f0 = f[0], f1 = f[1];");
    o("  // a = sum_k nu_k v_k over the reaction's species (net coefficients on first entries)");
    o("  // and, for the chemical potentials' temperature dependence, dh = sum_k nu_k H_k/RT");
    o("  kx_df av = kx_mk(0.0f, 0.0f), dh = kx_mk(0.0f, 0.0f);");
    for (int j = 0; j < E; ++j)
      o(fmt("  { const unsigned cj = (unsigned)%s & 0xffff0000u; if (cj != 0u) { const float4 w = vh[k%d]; const float cf = __uint_as_float(cj); "
            "av = kx_df_add_u(av, kx_df_mulf(kx_mk(w.x, w.y), cf)); dh = kx_df_add_u(dh, kx_df_mulf(kx_mk(w.z, w.w), cf)); } }",
            comp("c", j).c_str(), j));
    o("  const kx_df lA = kx_mk(f0.x, f0.y), bA = kx_mk(f0.z, f0.w), nEA = kx_mk(f1.x, f1.y);");
    o("  kx_df lk = kx_df_fma(bA, lnT, kx_df_fma(nEA, iT, lA));");
    o("  kx_df dT = kx_df_mul(iT, kx_df_fma(kx_df_neg(nEA), iT, bA));   // dln k/dT = beta/T + E/T^2");
    c.fp32 += NC * (E * (kDfAdd + kDfMulf) + 2 * kDfFma + kDfMul + kDfFma);
    std::string aq = "av";
    if (tb) {
      o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
      o("  const float4 f2 = f[2];");
      o("  kx_df X;   // [X] = eff_default C_M + (C_M/sigma) sum_e (eff_e - eff_default) Y_e/W_e");
      o("  if (e.y < 0) {");
      o("    const int kc = kx_effd[e.x].k;");
      o("    X = kx_df_mul(kx_mk(yv[kc].x, yv[kc].y), fC);");
      o("  } else {");
      o("    kx_df t = kx_mk(0.0f, 0.0f);");
      o("    for (int j = 0; j < e.y; ++j) {");
      o("      const kx_effd_t q = kx_effd[e.x + j];");
      o("      t = kx_df_fma(kx_mk(q.ahi, q.alo), kx_mk(yv[q.k].x, yv[q.k].y), t);");
      o("    }");
      o("    X = kx_df_fma(kx_mk(f2.x, f2.y), cM, kx_df_mul(fC, t));");
      o("  }");
      c.fp32 += NC * (kDfFma + kDfMul + 3 * kDfFma);
    }
    if (d.kind == Kind::ThreeBody) {
      o("  const kx_df aq = kx_df_mul(av, X);");
      aq = "aq";
      c.fp32 += NC * kDfMul;
    }
    if (fo) {
      o("  const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
      o("  const kx_df b0 = kx_mk(f3.x, f3.y), nE0 = kx_mk(f3.z, f3.w);");
      o("  const kx_df lk0 = kx_df_fma(b0, lnT, kx_df_fma(nE0, iT, kx_mk(f2.z, f2.w)));");
      o("  const kx_df dk0 = kx_df_mul(iT, kx_df_fma(kx_df_neg(nE0), iT, b0));");
      o("  kx_df lnPr = kx_df_add(kx_df_sub(lk0, lk), kx_df_log(X));");
      o("  if (!(lnPr.hi > -690.775528f)) lnPr = kx_mk(-690.775528f, 0.0f);");
      o("  // with e = e^-|ln Pr|: Pr/(1+Pr) and 1/(1+Pr) as e/(1+e) and 1/(1+e) (Pr < 1) or the other way round");
      o("  const bool small = lnPr.hi < 0.0f;");
      o("  const kx_df ee = kx_df_exp_n(small ? lnPr : kx_df_neg(lnPr));");
      o("  const kx_df i1e = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_add(kx_mk(1.0f, 0.0f), ee));");
      o("  const kx_df e1e = kx_df_mul(ee, i1e);");
      o("  const kx_df P1 = small ? e1e : i1e, P0 = small ? i1e : e1e;   // Pr/(1+Pr), 1/(1+Pr)");
      o("  const kx_df l1p = kx_df_log1p(ee);");
      o("  kx_df lnF = kx_mk(0.0f, 0.0f), dFl = kx_mk(0.0f, 0.0f), dFT = kx_mk(0.0f, 0.0f);   // ln F, dln F/dln Pr, dln F/dT");
      if (d.blend == Blend::Troe) {
        o("  {   // Troe: F_cent = (1-alpha) e^(-T/T***) + alpha e^(-T/T*) + e^(-T**/T)");
        o("    const kx_df p0 = kx_mk(f4.x, f4.y), p1 = kx_mk(f4.z, f4.w), p2 = kx_mk(f5.x, f5.y), p3 = kx_mk(f5.z, f5.w), p4 = kx_mk(f6.x, f6.y);");
        o("    const kx_df e3 = kx_df_mul(p0, kx_df_exp_s(kx_df_mul(Td, p2)));");
        o("    const kx_df e1 = kx_df_mul(p1, kx_df_exp_s(kx_df_mul(Td, p3)));");
        o("    const kx_df e2 = kx_df_exp_s(kx_df_mul(p4, iT));");
        o("    const kx_df Fc = kx_df_add(kx_df_add(e3, e1), e2);");
        o("    const kx_df dFc = kx_df_fma(e3, p2, kx_df_fma(e1, p3, kx_df_neg(kx_df_mul(kx_df_mul(e2, p4), iT2))));");
        o(fmt("    const kx_df lFc = kx_df_mul(kx_df_log(Fc), %s);", il10.c_str()));
        o(fmt("    const kx_df xx = kx_df_fma(lnPr, %s, kx_df_fma(%s, lFc, %s));", il10.c_str(), DFc(-0.67).c_str(), DFc(-0.4).c_str()));
        o(fmt("    const kx_df nn = kx_df_fma(%s, lFc, %s);", DFc(-1.27).c_str(), DFc(0.75).c_str()));
        o(fmt("    const kx_df den = kx_df_fma(%s, xx, nn);", DFc(-0.14).c_str()));
        o("    const kx_df iden = kx_df_div(kx_mk(1.0f, 0.0f), den);");
        o("    const kx_df ff = kx_df_mul(xx, iden);");
        o("    const kx_df g1 = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_fma(ff, ff, kx_mk(1.0f, 0.0f)));");
        o(fmt("    lnF = kx_df_mul(kx_df_mul(%s, lFc), g1);", DFc(std::log(10.0)).c_str()));
        o("    const kx_df h2 = kx_df_mul(kx_df_mul(kx_df_mul(kx_mk(-2.0f, 0.0f), ff), kx_df_mul(g1, g1)), lFc);");
        o("    const kx_df id2 = kx_df_mul(iden, iden);");
        o("    dFl = kx_df_mul(kx_df_mul(h2, nn), id2);");
        o(fmt("    dFT = kx_df_mul(kx_df_fma(kx_df_mul(h2, kx_df_fma(%s, den, kx_df_mul(%s, xx))), id2, g1), kx_df_div(dFc, Fc));",
              DFc(-0.67).c_str(), DFc(1.27 - 0.14 * 0.67).c_str()));
        o("  }");
        c.fp32 += NC * (3 * (kDfMul + kDfExp) + 2 * kDfMul + 2 * kDfAdd + 3 * kDfFma + kDfLog + kDfMul + 4 * kDfFma + 3 * kDfDiv + 12 * kDfMul);
      } else if (d.blend == Blend::Sri) {
        o("  {   // SRI: F = d T^e (a e^(-b/T) + e^(-T/c))^X, X = 1/(1 + log10^2 Pr)");
        o("    const kx_df pa = kx_mk(f4.x, f4.y), pnb = kx_mk(f4.z, f4.w), pnc = kx_mk(f5.x, f5.y), pld = kx_mk(f5.z, f5.w), pe = kx_mk(f6.x, f6.y);");
        o(fmt("    const kx_df lPr = kx_df_mul(lnPr, %s);", il10.c_str()));
        o("    const kx_df Xs = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_fma(lPr, lPr, kx_mk(1.0f, 0.0f)));");
        o("    const kx_df ea = kx_df_mul(pa, kx_df_exp_s(kx_df_mul(pnb, iT)));");
        o("    const kx_df eb = kx_df_exp_s(kx_df_mul(Td, pnc));");
        o("    const kx_df base = kx_df_add(ea, eb);");
        o("    const kx_df lnb = kx_df_log(base);");
        o("    lnF = kx_df_add(pld, kx_df_fma(pe, lnT, kx_df_mul(Xs, lnb)));");
        o(fmt("    dFl = kx_df_mul(kx_df_mul(kx_df_mul(kx_mk(-2.0f, 0.0f), lPr), kx_df_mul(Xs, Xs)), kx_df_mul(lnb, %s));", il10.c_str()));
        o("    // dln F/dT = e/T + X (a b e^(-b/T)/T^2 - e^(-T/c)/c)/base, with pnb = -b and pnc = -1/c");
        o("    dFT = kx_df_fma(pe, iT, kx_df_mul(Xs, kx_df_div(kx_df_fma(kx_df_neg(kx_df_mul(ea, pnb)), iT2, kx_df_mul(eb, pnc)), base)));");
        o("  }");
        c.fp32 += NC * (2 * (kDfMul + kDfExp) + 14 * kDfMul + 3 * kDfDiv + kDfLog + 4 * kDfFma + 2 * kDfAdd);
      }
      if (d.kind == Kind::Falloff) {
        o("  lk = kx_df_add(lk, kx_df_add(small ? kx_df_sub(lnPr, l1p) : kx_df_neg(l1p), lnF));   // k_inf Pr/(1+Pr) F");
        o("  const kx_df dP = kx_df_add(P0, dFl);   // dln k_f/dln Pr");
        o("  dT = kx_df_add(kx_df_fma(kx_df_sub(dk0, dT), dP, dT), dFT);");
      } else {
        o("  lk = kx_df_add(lk0, kx_df_sub(lnF, small ? l1p : kx_df_add(lnPr, l1p)));   // k_0 F/(1+Pr)");
        o("  const kx_df dP = kx_df_sub(dFl, P1);");
        o("  dT = kx_df_add(kx_df_fma(kx_df_sub(dk0, dT), dP, dk0), dFT);");
      }
      o("  const kx_df dX = kx_df_div(dP, X);   // dln k_f/d[X]");
      c.fp32 += NC * (2 * kDfFma + kDfMul + kDfAdd + kDfLog + kDfExp + 2 * kDfDiv + kDfMul + kDfLog + 6 * kDfAdd + kDfFma);
    } else if (d.kind == Kind::Plog) {
      o(fmt("  const int2 e = kx_e%d[r];", (int)ci));
      o("  const float* t = kx_plogf + 8 * e.x; const long long* tp = kx_plogp + e.x; const int np = e.y;");
      o("  const long long Pb = __double_as_longlong(P);");
      o("  // ln k and dln k/dT of table entry u: ln A + beta ln T - E/T, beta/T + E/T^2");
      o("#define KX_PLK(u) kx_df_fma(KX_PF((u) + 4), lnT, kx_df_fma(KX_PF((u) + 6), iT, KX_PF((u) + 2)))");
      o("#define KX_PLD(u) kx_df_mul(iT, kx_df_fma(kx_df_neg(KX_PF((u) + 6)), iT, KX_PF((u) + 4)))");
      o("  if (Pb <= tp[0]) { lk = KX_PLK(t); dT = KX_PLD(t); }");
      o("  else if (Pb >= tp[np - 1]) { const float* u = t + 8 * (np - 1); lk = KX_PLK(u); dT = KX_PLD(u); }");
      o("  else {");
      o("    int j = 0; while (!(Pb < tp[j + 1])) ++j;");
      o("    const float* u = t + 8 * j;");
      o("    const kx_df w = kx_df_div(kx_df_sub(lnP, KX_PF(u)), kx_df_sub(KX_PF(u + 8), KX_PF(u)));");
      o("    const kx_df l1 = KX_PLK(u), l2 = KX_PLK(u + 8), d1 = KX_PLD(u), d2 = KX_PLD(u + 8);");
      o("    lk = kx_df_fma(kx_df_sub(l2, l1), w, l1);");
      o("    dT = kx_df_fma(kx_df_sub(d2, d1), w, d1);");
      o("  }");
      o("#undef KX_PLK");
      o("#undef KX_PLD");
      c.fp32 += NC * (8 * kDfFma + 4 * kDfMul + 5 * kDfAdd + kDfDiv);
    }
    // log-space rates and the net rate
    o("  kx_df lf = lk;");
    for (int j = 0; j < d.nre; ++j) o(fmt("  lf = kx_df_add_u(lf, kx_mk(v%d.x, v%d.y));", j, j));
    std::string sfx = "0", srx = "0";
    for (int j = 0; j < d.nre; ++j) sfx += fmt(" ^ KX_NEG(k%d)", j);
    for (int j = d.nre; j < E; ++j) srx += fmt(" ^ KX_NEG(k%d)", j);
    o("  const int sf = " + sfx + ";");
    o("  kx_df lr = kx_mk(0.0f, 0.0f);");
    c.fp32 += NC * (d.nre * kDfAdd);
    // R_f = mfs 2^ef (signed); for reversible reactions R_r = mr 2^er (signed), and R_f - R_r and the
    // temperature term from the two by aligned subtraction (two exponentials per reaction)
    o("  int ef;");
    o(fmt("  kx_df mf = kx_df_exp_m(lf.hi <= -740.0f ? kx_df_add(lf, %s) : lf, ef);   // |R_f| = mf 2^ef", shift.c_str()));
    o("  if (lf.hi <= -740.0f) ef -= 2016;");
    o("  const kx_df mfs = sf ? kx_df_neg(mf) : mf;");
    c.fp32 += NC * kDfExp;
    const bool need_q = tb;
    if (d.rev) {
      const int dn = d.npr - d.nre;
      o("  const int sr = " + srx + ";");
      std::string first = d.nre > 0 ? "kx_df_neg(kx_mk(v0.z, v0.w))" : "kx_mk(v0.z, v0.w)";
      o("  kx_df dl = " + first + ";   // ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T))");
      for (int j = 1; j < E; ++j)
        o(fmt("  dl = kx_df_add_u(dl, kx_mk(%sv%d.z, %sv%d.w));", j < d.nre ? "-" : "", j, j < d.nre ? "-" : "", j));
      if (dn == 1 || dn == -1) o(fmt("  dl = kx_df_add_u(dl, %s);", dn == 1 ? "kx_df_neg(lnPRT)" : "lnPRT"));
      else if (dn != 0) o(fmt("  dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, %s));", F(-dn).c_str()));
      o("  lr = kx_df_add_u(lf, dl);");
      o("  int er;");
      o(fmt("  kx_df mr = kx_df_exp_m(lr.hi <= -740.0f ? kx_df_add(lr, %s) : lr, er);", shift.c_str()));
      o("  if (lr.hi <= -740.0f) er -= 2016;");
      o("  if (sr) mr = kx_df_neg(mr);   // R_r = mr 2^er");
      o("  // d/dT at fixed C: a c (dln k_f/dT (R_f - R_r) + R_r/T (sum_k nu_k H_k/RT - dn)), the second part");
      o("  // the chemical potentials' -dG_k/RT/dT = H_k/(R T^2) (Gibbs-Helmholtz) times d q/d(G_k/RT) =");
      o("  // -c nu_k R_r; as one term: a c (R_f dT - R_r (dT - (dh - dn)/T))");
      o(fmt("  { int et; const kx_df t = kx_df_sub_m(kx_df_mul_u(mfs, dT), ef, kx_df_mul_u(mr, kx_df_sub(dT, kx_df_mul(iT, %s))), er, et);",
            dn != 0 ? fmt("kx_df_add(dh, kx_mk(%s, 0.0f))", F(-dn).c_str()).c_str() : "dh"));
      o(fmt("    kx_acc_add(gTa, sT, kx_df_mul_u(%s, t), et); }", aq.c_str()));
      if (need_q) o("  int eq; const kx_df mq = kx_df_sub_m(mfs, ef, mr, er, eq);   // R_f - R_r = mq 2^eq");
      c.fp32 += NC * ((E - 1) * kDfAdd + (dn ? kDfAdd + kDfMulf : 0) + kDfAdd + kDfExp + 4 * kDfMul + 2 * kDfAdd + 8 + 20);
      if (need_q) c.fp32 += NC * (kDfAdd + 8);
    } else {
      o(fmt("  kx_acc_add(gTa, sT, kx_df_mul_u(kx_df_mul_u(%s, dT), mfs), ef);   // d/dT at fixed C: a c dln k_f/dT R_f", aq.c_str()));
      if (need_q) o("  const int eq = ef; const kx_df mq = mfs;");
      c.fp32 += NC * (2 * kDfMul + 20);
    }
    // d/dC_k: one term per entry, R/C_k with the sign of R/C_k: as |R| = m 2^e and 1/|C_k| = m' 2^e'
    // (per state), a product of mantissas (recip), or one log-space exponential exp(ln |R| - ln |C_k|)
    // per entry
    if (!recip) {
      for (int j = 0; j < E; ++j) {
        const bool reac = j < d.nre;
        if (!reac && !d.rev) continue;
        o(fmt("  { int et; kx_df mt = kx_df_exp_m(kx_df_sub(%s, kx_mk(v%d.x, v%d.y)), et);", reac ? "lf" : "lr", j, j));
        o(fmt("    if (%s ^ KX_NEG(k%d)) mt = kx_df_neg(mt);", reac ? "sf" : "sr", j));
        o(fmt("    kx_acc_add(gc[k%d], kx_df_mul_u(%s, mt), et); }", j, reac ? aq.c_str() : ("kx_df_neg(" + aq + ")").c_str()));
      }
    } else {
      o(fmt("  { const kx_df af = kx_df_mul_u(%s, mfs);", aq.c_str()));
      if (d.rev) o(fmt("    const kx_df ar = kx_df_mul_u(%s, mr);   // mr carries the sign of R_r", ("kx_df_neg(" + aq + ")").c_str()));
      for (int j = 0; j < E; ++j) {
        const bool reac = j < d.nre;
        if (!reac && !d.rev) continue;
        o(fmt("    { const float4 q = ic[k%d]; kx_df mt = kx_df_mul_u(%s, kx_mk(q.x, q.y)); if (KX_NEG(k%d)) mt = kx_df_neg(mt);", j,
              reac ? "af" : "ar", j));
        o(fmt("      kx_acc_add(gc[k%d], mt, %s + __float_as_int(q.z)); }", j, reac ? "ef" : "er"));
      }
      o("  }");
    }
    if (recip) c.fp32 += NC * (2 * kDfMul + E * (kDfMul + 20));
    else c.fp32 += NC * E * (kDfAdd + kDfExp + kDfMul + 20);
    // third-body adjoint a (R_f - R_r) (times dln k_f/d[X] in a falloff), spread over [M] and the listed species
    if (tb) {
      o(d.kind == Kind::ThreeBody ? "  const kx_df gX = kx_df_mul_u(av, mq);" : "  const kx_df gX = kx_df_mul_u(kx_df_mul_u(av, mq), dX);");
      o("  if (e.y < 0) {");
      o("    const int kc = kx_effd[e.x].k;");
      o("    kx_acc_add(gc[kc], gX, eq);");
      o("  } else {");
      o("    kx_acc_add(gMa, sM, kx_df_mul_u(kx_mk(f2.x, f2.y), gX), eq);");
      o("    for (int j = 0; j < e.y; ++j) {");
      o("      const kx_effd_t q = kx_effd[e.x + j];");
      o("      kx_acc_add(gc[q.k], kx_df_mul_u(kx_mk(q.ahi, q.alo), gX), eq);");
      o("    }");
      o("  }");
      c.fp32 += NC * (2 * kDfMul + 4 * (kDfMul + 20));
    }
    o("}");
    --o.ind;
    o("}");
  }
  // ---- close the chain in float64
  o("const double iTd = 1.0 / T;");
  o("const double cMd = kx_df2d(cM), fCd = kx_df2d(fC);");
  o("const double gT = kx_df2d_s(gTa, sT);");
  o("double gCX = 0.0;   // sum_k gC_k C_k");
  o(fmt("for (int k = 0; k < %d; ++k) gCX = fma(kx_df2d_s(kx_mk(gc[k].hi, gc[k].lo), gc[k].s), fCd * Y_[(long long)k * ld + i] * kx_iwd[k], gCX);", ns));
  o("const double gM = kx_df2d_s(gMa, sM) + gCX / cMd;");
  o("gT_[i] = fma(-gM * cMd, iTd, gT);   // [M] = p/(R T)");
  o("const double gavg = gCX / cMd;");
  o(fmt("for (int k = 0; k < %d; ++k) gY_[(long long)k * ld + i] = fCd * (kx_df2d_s(kx_mk(gc[k].hi, gc[k].lo), gc[k].s) - gavg) * kx_iwd[k];", ns));
  c.fp64 += ns * 6 + 12;
  c.fp32 += ns * 5 * kDfFma;
}

// ------------------------------------------------------------------ thermo
// Mixture cp and h in float-pair arithmetic on the float32 pipe (float64
// accuracy; the NASA polynomials need no float64 pipe): per species two
// Horner evaluations in T with float-pair coefficients of the range given by
// T < T_mid, weighted by Y_k R/W_k.
void emit_thermo(Out& o, const Mechanism& m, OpCounts& c) {
  const auto flags = tmid_flags(m);
  for (auto& f : flags) {
    long long b;
    std::memcpy(&b, &f.first, 8);
    o(fmt("const bool lo%d = __double_as_longlong(T) < %lldLL;", f.second, b));
  }
  o("const kx_df Td = kx_d2df_i(T);");
  o("const kx_df iT = kx_df_div(kx_mk(1.0f, 0.0f), Td);");
  o("kx_df cp = kx_mk(0.0f, 0.0f), hs = kx_mk(0.0f, 0.0f);");
  c.fp32 += 12 + kDfDiv;
  auto dsel = [&](const std::string& fl, double a, double b) {
    if (a == b) return DFc(a);
    const float ah = (float)a, bh = (float)b;
    return fmt("kx_mk(%s ? %s : %s, %s ? %s : %s)", fl.c_str(), F(ah).c_str(), F(bh).c_str(), fl.c_str(),
               F((float)(a - (double)ah)).c_str(), F((float)(b - (double)bh)).c_str());
  };
  for (int k = 0; k < m.ns; ++k) {
    const std::string fl = nasa_flag(m, k, flags);
    const double* lo = &m.a_lo[7 * k];
    const double* hi = &m.a_hi[7 * k];
    // cp/R = a0 + a1 T + a2 T^2 + a3 T^3 + a4 T^4
    std::string cpk = dsel(fl, lo[4], hi[4]);
    for (int n = 3; n >= 0; --n) cpk = fmt("kx_df_fma(%s, Td, %s)", cpk.c_str(), dsel(fl, lo[n], hi[n]).c_str());
    // H/RT = a0 + a1/2 T + a2/3 T^2 + a3/4 T^3 + a4/5 T^4 + a5/T
    std::string h = dsel(fl, lo[4] / 5.0, hi[4] / 5.0);
    for (int n = 3; n >= 0; --n) h = fmt("kx_df_fma(%s, Td, %s)", h.c_str(), dsel(fl, lo[n] / (n + 1), hi[n] / (n + 1)).c_str());
    h = fmt("kx_df_fma(%s, iT, %s)", dsel(fl, lo[5], hi[5]).c_str(), h.c_str());
    o(fmt("{ const kx_df yr = kx_df_mul(kx_d2df_i(Y_[(long long)%d * ld + i]), %s);", k, DFc(R_U / m.W[k]).c_str()));
    o(fmt("  cp = kx_df_fma(yr, %s, cp);", cpk.c_str()));
    o(fmt("  hs = kx_df_fma(yr, %s, hs); }", h.c_str()));
    c.fp32 += 12 + kDfMul + 11 * kDfFma + 28;
  }
  o("out0_[i] = kx_df2d(cp);");
  o("out1_[i] = kx_df2d(kx_df_mul(hs, Td));");
  c.fp64 += 2;
}

// ------------------------------------------------------------------ transport
// The O(N_s) and O(N_s^2) sums of the mixing rules run as loops over
// coefficient tables in global memory (the addresses are the same for every
// thread of a warp, so each load is a broadcast), with each thread's species
// vectors staged in its own column of shared memory, [species][thread].
// Compile time and instruction-cache footprint stay O(1) in the mechanism
// size, where fully unrolled pair sums grow as N_s^2.
//
// Wilke (the eta formula with phi_kj): with u_k = sqrt(eta_k) W_k^(-1/4) and
// a_kj = (1 + W_k/W_j)^(-1/2)/sqrt(8),
//   sum_j X_j phi_kj = S0_k + 2 u_k S1_k + u_k^2 S2_k,
//   S0_k = sum_j a_kj X_j, S1_k = sum_j a_kj X_j/u_j, S2_k = sum_j a_kj X_j/u_j^2,
// three products with a constant matrix; every term is positive.
// Diffusion: S_k = sum_{j != k} X_j / D_kj(1 atm), each symmetric pair
// evaluated once and added to both rows (Sec. 2.3.2), or the full matrix.
//
// Three arithmetics share the loop structure:
//   f64: native float64, polynomials in ln T as fitted;
//   df:  double-float (float32 pairs, ~2^-47 relative per operation) on the
//        float32 pipe, polynomials re-expanded about L0 = ln sqrt(300*3000)
//        so every Horner step is well conditioned -- float64 accuracy
//        without the float64 pipe, which is the scarce unit on this GPU;
//   f32: float32 (the mixed precision), polynomials re-expanded about L0 and
//        scaled by log2(e) so each property is one exp2.
double wilke_a(const Mechanism& m, int k, int j) { return 1.0 / std::sqrt(8.0 * (1.0 + m.W[k] / m.W[j])); }

// Double-double host arithmetic from error-free transformations (std::fma is exact IEEE arithmetic
// on every host), so that the emitted constants are the same bits on every platform: long double is
// 80-bit on x86-64 and 128-bit on aarch64.
struct HostDD { double hi, lo; };
HostDD hdd_norm(double a, double b) { const double s = a + b; return {s, b - (s - a)}; }
HostDD hdd_add(HostDD a, HostDD b) {
  const double s = a.hi + b.hi, bb = s - a.hi;
  const double e = (a.hi - (s - bb)) + (b.hi - bb);
  return hdd_norm(s, e + a.lo + b.lo);
}
HostDD hdd_mul(HostDD a, HostDD b) {
  const double p = a.hi * b.hi;
  return hdd_norm(p, std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi));
}

// p(L) = sum c_n L^n re-expanded about L0: d_m = sum_{n>=m} C(n,m) c_n L0^(n-m), in double-double
void shift_poly(const double* cf, double L0, double scale, double out[5]) {
  static const double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  HostDD pw[5] = {{1.0, 0.0}};
  for (int k = 1; k < 5; ++k) pw[k] = hdd_mul(pw[k - 1], {L0, 0.0});
  for (int mm = 0; mm < 5; ++mm) {
    HostDD d = {0.0, 0.0};
    for (int n = mm; n < 5; ++n) d = hdd_add(d, hdd_mul(hdd_mul({binom[n][mm], 0.0}, {cf[n], 0.0}), pw[n - mm]));
    d = hdd_mul(d, {scale, 0.0});
    out[mm] = d.hi + d.lo;
  }
}

struct TrMode {
  enum { F64, DF, F32 } kind;
  const char* ty;     // arithmetic type
  const char* st;     // shared / table element type
};

void emit_transport(Out& o, Out& g, const Mechanism& m, const EmitOptions& opt, OpCounts& c) {
  const int ns = m.ns;
  TrMode md;
  if (opt.mixed) md = {TrMode::F32, "float", "float"};
  else if (opt.tr_mode == 0) md = {TrMode::DF, "kx_df", "float2"};
  else md = {TrMode::F64, "double", "double"};
  // direct fits (of eta, lambda, 1/D themselves) are evaluated without exponentials and, in every
  // arithmetic, in L = ln T - L0: their monomial form in ln T is badly conditioned (condition numbers
  // up to ~1e6 for 1/D_kj); the re-expansion is computed in double-double.  L0 = ln sqrt(300 * 3000),
  // correctly rounded, as a literal (no host libm in the emitted constants)
  const bool direct = m.fit_direct;
  const double L0 = (md.kind == TrMode::F64 && !direct) ? 0.0 : 6.855075021153224;
  const double SC = (md.kind == TrMode::F32 && !direct) ? 1.4426950408889634 : 1.0;   // exp2 form for float32
  const int B = opt.block;
  // float64-accurate viscosity keeps two vectors per species (X, v = 1/u) in shared memory
  // and forms z1, z2 in the loop: two multiplies per pair buy twice the resident warps
  const bool two_arrays = md.kind != TrMode::F32 && opt.part != 2;
  // X_k of this thread: a column of shared memory, or a per-thread local array (tr_layout 2: halves
  // the shared memory per thread, so twice the warps are resident)
  const bool xlocal = opt.tr_layout >= 2;
  auto XS = [&](const std::string& idx) { return xlocal ? fmt("xl[%s]", idx.c_str()) : fmt("sX[%s * %d + t]", idx.c_str(), B); };
  // the other vectors (z1 = v or X v, z2, and the diffusion sums S in the z1 slot): shared-memory
  // columns, or per-thread local arrays (tr_layout 3: no shared memory at all)
  const bool vlocal = opt.tr_layout == 3;
  auto VS = [&](const char* arr, const std::string& idx) {
    const std::string a = std::string(arr) == "sS" ? "sZ1" : arr;
    return vlocal ? fmt("l%s[%s]", a.c_str() + 1, idx.c_str()) : fmt("%s[%s * %d + t]", a.c_str(), idx.c_str(), B);
  };
  // ---- element literal, load, store and arithmetic spelled per mode
  auto lit = [&](double v) -> std::string {
    if (md.kind == TrMode::F64) return D(v);
    if (md.kind == TrMode::F32) return F(v);
    const float h = (float)v;
    return fmt("{%s, %s}", F(h).c_str(), F((float)(v - (double)h)).c_str());
  };
  auto ld = [&](const std::string& e) { return md.kind == TrMode::DF ? fmt("kx_mk((%s).x, (%s).y)", e.c_str(), e.c_str()) : e; };
  auto st = [&](const std::string& dst, const std::string& v) {
    return md.kind == TrMode::DF ? fmt("%s = make_float2((%s).hi, (%s).lo);", dst.c_str(), v.c_str(), v.c_str())
                                 : fmt("%s = %s;", dst.c_str(), v.c_str());
  };
  auto FMA = [&](const std::string& a, const std::string& b, const std::string& cc) {
    return fmt("%s(%s, %s, %s)", md.kind == TrMode::DF ? "kx_df_fma" : md.kind == TrMode::F32 ? "fmaf" : "fma", a.c_str(), b.c_str(),
               cc.c_str());
  };
  // a*b + c into a running sum that is renormalised once at the end (float pairs: no final renormalisation)
  auto ACC = [&](const std::string& a, const std::string& b, const std::string& cc) {
    return md.kind == TrMode::DF ? fmt("kx_df_fma_u(%s, %s, %s)", a.c_str(), b.c_str(), cc.c_str()) : FMA(a, b, cc);
  };
  auto MUL = [&](const std::string& a, const std::string& b) {
    return md.kind == TrMode::DF ? fmt("kx_df_mul(%s, %s)", a.c_str(), b.c_str()) : fmt("(%s) * (%s)", a.c_str(), b.c_str());
  };
  // a*b feeding a further product or running sum (float pairs: no final renormalisation)
  auto MULU = [&](const std::string& a, const std::string& b) {
    return md.kind == TrMode::DF ? fmt("kx_df_mul_u(%s, %s)", a.c_str(), b.c_str()) : MUL(a, b);
  };
  auto EXP = [&](const std::string& a) {
    return fmt("%s(%s)", md.kind == TrMode::DF ? "kx_df_exp" : md.kind == TrMode::F32 ? "exp2f" : "kx_exp", a.c_str());
  };
  auto NEG = [&](const std::string& a) {
    return md.kind == TrMode::DF ? fmt("kx_mk(-(%s).hi, -(%s).lo)", a.c_str(), a.c_str()) : fmt("(-(%s))", a.c_str());
  };
  auto TOD = [&](const std::string& a) {
    return md.kind == TrMode::DF ? fmt("kx_df2d(%s)", a.c_str()) : md.kind == TrMode::F32 ? fmt("kx_f2d(%s)", a.c_str()) : a;
  };
  auto FROMD = [&](const std::string& a) {
    return md.kind == TrMode::DF ? fmt("kx_d2df(%s)", a.c_str()) : md.kind == TrMode::F32 ? fmt("kx_d2f(%s)", a.c_str()) : a;
  };
  const std::string ZERO = md.kind == TrMode::DF ? "kx_mk(0.f, 0.f)" : md.kind == TrMode::F32 ? "0.0f" : "0.0";
  auto horner = [&](const std::string& tab) {   // polynomial with coefficients tab[0..4]
    std::string r = ld(tab + "[4]");
    for (int n = 3; n >= 0; --n) r = FMA(r, "L", ld(fmt("%s[%d]", tab.c_str(), n)));
    return r;
  };
  auto coefs = [&](const double* cf, double s, double add, double out[5]) {
    if (L0 == 0.0) for (int n = 0; n < 5; ++n) out[n] = cf[n] * s;
    else shift_poly(cf, L0, s * SC, out);
    out[0] += add * SC;
  };
  // 1/sqrt and sqrt of a positive value in the kernel's arithmetic
  auto RSQRT = [&](const std::string& a) {
    return md.kind == TrMode::DF ? fmt("kx_df_rsqrt(%s)", a.c_str()) : md.kind == TrMode::F32 ? fmt("rsqrtf(%s)", a.c_str())
                                                                                                 : fmt("(1.0 / sqrt(%s))", a.c_str());
  };
  auto DIV = [&](const std::string& a, const std::string& b) {
    return md.kind == TrMode::DF ? fmt("kx_df_div(%s, %s)", a.c_str(), b.c_str())
                                 : md.kind == TrMode::F32 ? fmt("__fdividef(%s, %s)", a.c_str(), b.c_str())
                                                          : fmt("((%s) / (%s))", a.c_str(), b.c_str());
  };
  // per-op costs, for the manifest
  const double cf_fma = md.kind == TrMode::DF ? 14 : 1, cf_exp = md.kind == TrMode::DF ? 45 : 1;
  auto count_fma = [&](double n) {
    if (md.kind == TrMode::F64) c.fp64 += n; else c.fp32 += n * cf_fma;
  };
  auto count_exp = [&](double n) {
    if (md.kind == TrMode::F64) c.exp64 += n; else if (md.kind == TrMode::F32) c.exp32 += n; else c.fp32 += n * cf_exp;
  };
  // ---- module-scope tables
  {
    std::string pv, pl, wa, dself, w, iw, sqw, w4, iw4, sqwp, isqwp;
    for (int k = 0; k < ns; ++k) {
      double d[5];
      if (direct) coefs(&m.eta[5 * k], 1.0, 0.0, d);                  // eta_k
      else coefs(&m.eta[5 * k], -0.5, 0.25 * std::log(m.W[k]), d);   // ln v_k = -(ln eta_k / 2 - ln W_k / 4)
      for (int n = 0; n < 5; ++n) pv += lit(d[n]) + ",";
      coefs(&m.lam[5 * k], 1.0, 0.0, d);
      for (int n = 0; n < 5; ++n) pl += lit(d[n]) + ",";
      if (direct) {   // 1/D_kk in L = ln T - L0
        double e[5];
        shift_poly(&m.dif[5 * ((size_t)k * ns + k)], L0, 1.0, e);
        for (int n = 0; n < 5; ++n) dself += D(e[n]) + ",";
      } else {
        for (int n = 0; n < 5; ++n) dself += D(m.dif[5 * ((size_t)k * ns + k) + n]) + ",";
      }
      sqwp += lit(std::sqrt(m.W[k])) + ",";
      isqwp += lit(1.0 / std::sqrt(m.W[k])) + ",";
      w4 += lit(std::sqrt(std::sqrt(m.W[k]))) + ",";   // correctly rounded square roots: the same bits on every host
      iw4 += lit(1.0 / std::sqrt(std::sqrt(m.W[k]))) + ",";
      w += D(m.W[k]) + ",";
      iw += D(1.0 / m.W[k]) + ",";
      sqw += D(std::sqrt(m.W[k])) + ",";
      for (int j = 0; j < ns; ++j) wa += lit(wilke_a(m, k, j)) + ",";
    }
    std::string dc;
    int np = 0;
    for (int k = 0; k < ns; ++k)
      for (int j = (opt.diff_mode == 2 ? 0 : k + 1); j < ns; ++j) {
        if (j == k) continue;
        double d[5];
        coefs(&m.dif[5 * ((size_t)k * ns + j)], direct ? 1.0 : -1.0, 0.0, d);   // 1/D_kj, or -ln D_kj
        for (int n = 0; n < 5; ++n) dc += lit(d[n]) + ",";
        dc += lit(0.0) + ",";                 // each pair padded to 6 entries for vector loads
        ++np;
      }
    const char* T = md.st;
    g(fmt("__device__ const %s kx_pv[%d] = {%s};", T, 5 * ns, pv.c_str()));
    g(fmt("__device__ const %s kx_pl[%d] = {%s};", T, 5 * ns, pl.c_str()));
    g(fmt("__device__ const %s kx_wa[%d] = {%s};", T, ns * ns, wa.c_str()));
    std::string pad;
    for (int n = 0; n < 6; ++n) pad += lit(0.0) + (n < 5 ? "," : "");
    g(fmt("__device__ const %s kx_dc[%d] __attribute__((aligned(16))) = {%s%s};", T, 6 * np + 6, dc.c_str(), pad.c_str()));
    g(fmt("__device__ const double kx_dself[%d] = {%s};", 5 * ns, dself.c_str()));
    g(fmt("__device__ const double kx_w[%d] = {%s};", ns, w.c_str()));
    g(fmt("__device__ const double kx_iw[%d] = {%s};", ns, iw.c_str()));
    g(fmt("__device__ const double kx_sqw[%d] = {%s};", ns, sqw.c_str()));
    g(fmt("__device__ const %s kx_w4[%d] = {%s};", T, ns, w4.c_str()));
    g(fmt("__device__ const %s kx_sqwp[%d] = {%s};", T, ns, sqwp.c_str()));
    g(fmt("__device__ const %s kx_isqwp[%d] = {%s};", T, ns, isqwp.c_str()));
    g(fmt("__device__ const %s kx_iw4[%d] = {%s};", T, ns, iw4.c_str()));
  }
  o("const double lnT = log(T);");
  c.log64 += 1;
  if (L0 == 0.0) o("const double L = lnT;");
  else o(fmt("const %s L = %s;", md.ty, FROMD(fmt("lnT - %s", D(L0).c_str())).c_str()));
  if (vlocal) {   // every species vector in per-thread local arrays
    o(fmt("%s xl[%d], lZ1[%d], lZ2[%d];", md.st, ns, ns, ns));
  } else if (xlocal) {   // X in a per-thread local array, the other vectors in shared memory
    o(fmt("%s xl[%d];", md.st, ns));
    o(fmt("%s* const sZ1 = (%s*)kx_dyn;", md.st, md.st));
    o(fmt("%s* const sZ2 = sZ1 + %d;", md.st, ns * B));
  } else {
    o(fmt("%s* const sX = (%s*)kx_dyn;", md.st, md.st));
    o(fmt("%s* const sZ1 = sX + %d;", md.st, ns * B));
    o(fmt("%s* const sZ2 = sZ1 + %d;", md.st, ns * B));
  }
  o("const int t = threadIdx.x;");
  o("double sy = 0.0, sY = 0.0;");
  o(fmt("for (int k = 0; k < %d; ++k) { const double Yk = Y_[(long long)k * ld + i]; sY += Yk; sy = fma(Yk, kx_iw[k], sy); }", ns));
  o("const double isig = 1.0 / sy;");
  o("if (!(isig > 0 && isig < KX_INF)) KX_BAD_POINT");
  o("const double iWbar = 1.0 / (sY * isig);");
  c.fp64 += 2 * ns + 1; c.div64 += 2;
  const bool p1 = opt.part != 2, p2 = opt.part != 1;
  // float64 accuracy, all vectors local: Wilke's phi_kj evaluated once per unordered pair (j > k),
  // the other direction from phi_jk = phi_kj rho_j/rho_k with rho = eta/W (exact identity), added to
  // a column accumulator C_j (the z2 slot)
  const bool wsym = two_arrays && vlocal && opt.diff_mode != 2;
  if (!p1) {
    o(fmt("for (int k = 0; k < %d; ++k) %s", ns, st(XS("k"),
                                                    FROMD("Y_[(long long)k * ld + i] * kx_iw[k] * isig")).c_str()));
    c.fp64 += ns;
  }
  if (p1) {
  // per species: X, v = 1/u, z1 = X v, z2 = X v^2, Mathur sums
  o(fmt("%s sl = %s, sil = %s;", md.ty, ZERO.c_str(), ZERO.c_str()));
  o("#pragma unroll 1");
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o(fmt("  const %s X = %s;", md.ty, FROMD("Y_[(long long)k * ld + i] * kx_iw[k] * isig").c_str()));
  o("  " + st(XS("k"), "X"));
  o(fmt("  const %s* pv = kx_pv + 5 * k; const %s* pl = kx_pl + 5 * k;", md.st, md.st));
  if (direct) {   // v = W^(1/4)/sqrt(eta)
    o(fmt("  const %s eta = %s;", md.ty, horner("pv").c_str()));
    o(fmt("  const %s v = %s;", md.ty, MUL(RSQRT("eta"), ld("kx_w4[k]")).c_str()));
  } else {
    o(fmt("  const %s v = %s;", md.ty, EXP(horner("pv")).c_str()));
  }
  if (two_arrays) {
    o("  " + st(VS("sZ1", "k"), "v"));          // z1 = X v and z2 = z1 v are formed in the Wilke loop
    if (wsym) o("  " + st(VS("sZ2", "k"), ZERO));
  } else {
    o(fmt("  const %s z1 = %s;", md.ty, MUL("X", "v").c_str()));
    o("  " + st(VS("sZ1", "k"), "z1"));
    o("  " + st(VS("sZ2", "k"), MUL("z1", "v")));
  }
  if (direct) {
    o(fmt("  const %s lam = %s;", md.ty, horner("pl").c_str()));
    o("  sl = " + FMA("X", "lam", "sl") + ";");
    o("  sil = " + FMA("X", DIV(md.kind == TrMode::DF ? "kx_mk(1.f, 0.f)" : md.kind == TrMode::F32 ? "1.0f" : "1.0", "lam"), "sil") + ";");
  } else {
    o(fmt("  const %s ll = %s;", md.ty, horner("pl").c_str()));
    o("  sl = " + FMA("X", EXP("ll"), "sl") + ";");
    o("  sil = " + FMA("X", EXP(NEG("ll")), "sil") + ";");
  }
  o("}");
  count_fma(ns * 14.0); count_exp(ns * 3.0);
  c.fp64 += 2 * ns;
  // Wilke rows
  o("double mu = 0.0;");
  if (wsym) {
    // den_k = sum_j X_j phi_kj = X_k + sum_{j>k} X_j phi_kj + rho_k sum_{j<k} (X_j/rho_j) phi_jk, with
    // phi_kk = 1, phi_kj = a_kj (1 + u_k v_j)^2, rho_k = eta_k/W_k = u_k^2/sqrt(W_k).  Row k adds its
    // pairs to its own sum and X_k/rho_k phi_kj to C_j; C_k is complete when row k starts.
    const std::string ONE1 = md.kind == TrMode::DF ? "kx_mk(1.f, 0.f)" : "1.0";
    o("#pragma unroll 1");
    o(fmt("for (int k = 0; k < %d; ++k) {", ns));
    o(fmt("  const %s* pv = kx_pv + 5 * k;", md.st));
    if (direct) {
      o(fmt("  const %s eta = %s;", md.ty, horner("pv").c_str()));
      o(fmt("  const %s u = %s;", md.ty, MUL(MUL("eta", RSQRT("eta")), ld("kx_iw4[k]")).c_str()));
    } else {
      o(fmt("  const %s u = %s;", md.ty, EXP(NEG(horner("pv"))).c_str()));
    }
    o(fmt("  const %s Xk = %s, vk = %s;", md.ty, ld(XS("k")).c_str(), ld(VS("sZ1", "k")).c_str()));
    o(fmt("  const %s xr = %s;   // X_k / rho_k = X_k v_k^2 sqrt(W_k)", md.ty,
          MUL(MUL("Xk", MUL("vk", "vk")), ld("kx_sqwp[k]")).c_str()));
    o(fmt("  %s r0 = %s, r1 = %s;", md.ty, ZERO.c_str(), ZERO.c_str()));
    o(fmt("  const %s* a = kx_wa + %d * k;", md.st, ns));
    o("  int j = k + 1;");
    o("  #pragma unroll 2");
    o(fmt("  for (; j + 1 < %d; j += 2) {", ns));
    o(fmt("    const %s A = %s, Ab = %s;", md.ty, ld("a[j]").c_str(), ld("a[j + 1]").c_str()));
    o(fmt("    const %s xa = %s, va = %s, xb = %s, vb = %s;", md.ty, ld(XS("j")).c_str(), ld(VS("sZ1", "j")).c_str(),
          ld(XS("(j + 1)")).c_str(), ld(VS("sZ1", "(j + 1)")).c_str()));
    o(fmt("    const %s wa = %s, wb = %s;", md.ty, ACC("u", "va", ONE1).c_str(), ACC("u", "vb", ONE1).c_str()));
    o(fmt("    const %s pa = %s, pb = %s;", md.ty, MULU("A", MULU("wa", "wa")).c_str(), MULU("Ab", MULU("wb", "wb")).c_str()));
    o(fmt("    r0 = %s; r1 = %s;", ACC("xa", "pa", "r0").c_str(), ACC("xb", "pb", "r1").c_str()));
    o(fmt("    const %s ca = %s, cb = %s;", md.ty, ACC("xr", "pa", ld(VS("sZ2", "j"))).c_str(),
          ACC("xr", "pb", ld(VS("sZ2", "(j + 1)"))).c_str()));
    o("    " + st(VS("sZ2", "j"), "ca"));
    o("    " + st(VS("sZ2", "(j + 1)"), "cb"));
    o("  }");
    o(fmt("  if (j < %d) {", ns));
    o(fmt("    const %s A = %s, xa = %s, va = %s;", md.ty, ld("a[j]").c_str(), ld(XS("j")).c_str(), ld(VS("sZ1", "j")).c_str()));
    o(fmt("    const %s wa = %s;", md.ty, ACC("u", "va", ONE1).c_str()));
    o(fmt("    const %s pa = %s;", md.ty, MULU("A", MULU("wa", "wa")).c_str()));
    o(fmt("    r0 = %s;", ACC("xa", "pa", "r0").c_str()));
    o(fmt("    const %s ca = %s;", md.ty, ACC("xr", "pa", ld(VS("sZ2", "j"))).c_str()));
    o("    " + st(VS("sZ2", "j"), "ca"));
    o("  }");
    o(fmt("  const %s rho = %s;", md.ty, MUL(MUL("u", "u"), ld("kx_isqwp[k]")).c_str()));
    o(fmt("  const %s den = %s;", md.ty, FMA("rho", ld(VS("sZ2", "k")), FMA("r1", ONE1, FMA("r0", ONE1, "Xk"))).c_str()));
    o(fmt("  mu = fma(%s * %s, kx_sqw[k] / %s, mu);", TOD("Xk").c_str(), TOD(MUL("u", "u")).c_str(), TOD("den").c_str()));
    o("}");
    // per unordered pair three accumulating multiply-adds and two products; in float pairs these are the
    // unnormalised forms (12 and 4 float32 instructions), not the renormalised ones of count_fma
    if (md.kind == TrMode::DF) c.fp32 += ns * (ns - 1) / 2.0 * (3 * 12 + 2 * 4);
    else count_fma(ns * (ns - 1) / 2.0 * 5);
    count_fma(ns * 10.0); count_exp(ns);
    c.fp64 += 4 * ns; c.div64 += ns;
  } else {
  o("#pragma unroll 1");
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o(fmt("  const %s* pv = kx_pv + 5 * k;", md.st));
  if (direct) {   // u = sqrt(eta)/W^(1/4) = eta / sqrt(eta) / W^(1/4)
    o(fmt("  const %s eta = %s;", md.ty, horner("pv").c_str()));
    o(fmt("  const %s u = %s;", md.ty, MUL(MUL("eta", RSQRT("eta")), ld("kx_iw4[k]")).c_str()));
  } else {
    o(fmt("  const %s u = %s;", md.ty, EXP(NEG(horner("pv"))).c_str()));
  }
  if (two_arrays) {
    // float64 accuracy: den_k = sum_j a_kj X_j (1 + u_k v_j)^2 with w = 1 + u_k v_j formed per pair
    // (three products and one accumulation per pair; even and odd j in two chains)
    const std::string ONE1 = md.kind == TrMode::DF ? "kx_mk(1.f, 0.f)" : "1.0";
    o(fmt("  %s s0 = %s, t0 = %s;", md.ty, ZERO.c_str(), ZERO.c_str()));
    o(fmt("  const %s* a = kx_wa + %d * k;", md.st, ns));
    o("  #pragma unroll 2");
    o(fmt("  for (int j = 0; j + 1 < %d; j += 2) {", ns));
    o(fmt("    const %s A = %s, Ab = %s;", md.ty, ld("a[j]").c_str(), ld("a[j + 1]").c_str()));
    o(fmt("    const %s xa = %s, va = %s, xb = %s, vb = %s;", md.ty, ld(XS("j")).c_str(),
          ld(VS("sZ1", "j")).c_str(), ld(XS("(j + 1)")).c_str(), ld(VS("sZ1", "(j + 1)")).c_str()));
    o(fmt("    const %s wa = %s, wb = %s;", md.ty, FMA("u", "va", ONE1).c_str(), FMA("u", "vb", ONE1).c_str()));
    o(fmt("    s0 = %s;", FMA(MUL("A", "xa"), MUL("wa", "wa"), "s0").c_str()));
    o(fmt("    t0 = %s;", FMA(MUL("Ab", "xb"), MUL("wb", "wb"), "t0").c_str()));
    o("  }");
    if (ns % 2) {
      o(fmt("  { const %s A = %s, xa = %s, va = %s;", md.ty, ld(fmt("a[%d]", ns - 1)).c_str(), ld(XS(std::to_string(ns - 1))).c_str(),
            ld(VS("sZ1", std::to_string(ns - 1))).c_str()));
      o(fmt("    const %s wa = %s;", md.ty, FMA("u", "va", ONE1).c_str()));
      o(fmt("    s0 = %s; }", FMA(MUL("A", "xa"), MUL("wa", "wa"), "s0").c_str()));
    }
    o(fmt("  const %s den = %s;", md.ty, FMA("t0", ONE1, "s0").c_str()));
  } else {
  // two partial sums per product (even and odd j): six independent accumulation chains
  o(fmt("  %s s0 = %s, s1 = %s, s2 = %s, t0 = %s, t1 = %s, t2 = %s;", md.ty, ZERO.c_str(), ZERO.c_str(), ZERO.c_str(),
        ZERO.c_str(), ZERO.c_str(), ZERO.c_str()));
  o(fmt("  const %s* a = kx_wa + %d * k;", md.st, ns));
  o("  #pragma unroll 2");
  o(fmt("  for (int j = 0; j + 1 < %d; j += 2) {", ns));
  o(fmt("    const %s A = %s, Ab = %s;", md.ty, ld("a[j]").c_str(), ld("a[j + 1]").c_str()));
  // the three vectors of species j: X_j, z1_j = X_j v_j, z2_j = z1_j v_j
  auto vecs = [&](const std::string& jj, const char* sfx) {
    if (!two_arrays)
      return fmt("const %s x%s = %s, y%s = %s, z%s = %s;", md.ty, sfx, ld(XS(jj)).c_str(), sfx,
                 ld(VS("sZ1", jj)).c_str(), sfx, ld(VS("sZ2", jj)).c_str());
    return fmt("const %s x%s = %s, v%s = %s; const %s y%s = %s; const %s z%s = %s;", md.ty, sfx,
               ld(XS(jj)).c_str(), sfx, ld(VS("sZ1", jj)).c_str(), md.ty,
               sfx, MUL(fmt("x%s", sfx), fmt("v%s", sfx)).c_str(), md.ty, sfx, MUL(fmt("y%s", sfx), fmt("v%s", sfx)).c_str());
  };
  o("    " + vecs("j", "a") + " " + vecs("(j + 1)", "b"));
  o(fmt("    s0 = %s; s1 = %s; s2 = %s;", FMA("A", "xa", "s0").c_str(), FMA("A", "ya", "s1").c_str(), FMA("A", "za", "s2").c_str()));
  o(fmt("    t0 = %s; t1 = %s; t2 = %s;", FMA("Ab", "xb", "t0").c_str(), FMA("Ab", "yb", "t1").c_str(), FMA("Ab", "zb", "t2").c_str()));
  o("  }");
  if (ns % 2) {
    o(fmt("  { const %s A = %s; %s", md.ty, ld(fmt("a[%d]", ns - 1)).c_str(), vecs(std::to_string(ns - 1), "a").c_str()));
    o(fmt("    s0 = %s; s1 = %s; s2 = %s; }", FMA("A", "xa", "s0").c_str(), FMA("A", "ya", "s1").c_str(), FMA("A", "za", "s2").c_str()));
  }
  const std::string ONE = md.kind == TrMode::DF ? "kx_mk(1.f, 0.f)" : md.kind == TrMode::F32 ? "1.0f" : "1.0";
  o(fmt("  s0 = %s; s1 = %s; s2 = %s;", FMA("t0", ONE, "s0").c_str(), FMA("t1", ONE, "s1").c_str(), FMA("t2", ONE, "s2").c_str()));
  const std::string two_s1 = md.kind == TrMode::DF ? "kx_mk(2.f * s1.hi, 2.f * s1.lo)" : md.kind == TrMode::F32 ? "2.0f * s1" : "2.0 * s1";
  o(fmt("  const %s den = %s;", md.ty, FMA("u", FMA("u", "s2", two_s1), "s0").c_str()));
  }
  o(fmt("  mu = fma(%s * %s, kx_sqw[k] / %s, mu);", TOD(ld(XS("k"))).c_str(), TOD(MUL("u", "u")).c_str(),
        TOD("den").c_str()));
  o("}");
  count_fma(ns * (3.0 * ns + 8)); count_exp(ns);
  c.fp64 += 4 * ns; c.div64 += ns;
  }
  o("out0_[i] = mu;");
  o(fmt("out1_[i] = 0.5 * (%s + 1.0 / %s);", TOD("sl").c_str(), TOD("sil").c_str()));
  c.fp64 += 4; c.div64 += 1;
  }  // part 1
  if (!p2) return;
  // mixture-averaged diffusion, S in the sZ1 columns
  if (!vlocal) o(fmt("%s* const sS = sZ1;", md.st));
  o(fmt("for (int k = 0; k < %d; ++k) %s", ns, st(VS("sS", "k"), ZERO).c_str()));
  o(fmt("const %s* cf = kx_dc;", md.st));
  // the next pair's coefficients are loaded one iteration ahead (the table
  // carries one zero pair of padding), so their latency hides behind the
  // current pair's arithmetic
  std::string vec;
  // exponential of one pair's polynomial, coefficients in the float4/double2/float2 triple (x, y, z);
  // float pairs: no renormalisation inside (the exponential and the running sums take hi + lo as is)
  auto pexp = [&](const char* e, const char* x, const char* y, const char* z) {
    if (direct && md.kind == TrMode::DF)   // 1/D_kj itself
      return fmt("const kx_df %s = kx_df_fma_u(kx_df_fma_u(kx_df_fma_u(kx_df_fma_u(kx_mk(%s.x, %s.y), L, kx_mk(%s.z, %s.w)), L, "
                 "kx_mk(%s.x, %s.y)), L, kx_mk(%s.z, %s.w)), L, kx_mk(%s.x, %s.y));",
                 e, z, z, y, y, y, y, x, x, x, x);
    if (direct && md.kind == TrMode::F64)
      return fmt("const double %s = fma(fma(fma(fma(%s.x, L, %s.y), L, %s.x), L, %s.y), L, %s.x);", e, z, y, y, x, x);
    if (direct)
      return fmt("const float %s = fmaf(fmaf(fmaf(fmaf(%s.x, L, %s.y), L, %s.x), L, %s.y), L, %s.x);", e, z, y, y, x, x);
    if (md.kind == TrMode::DF)
      return fmt("const kx_df %s = kx_df_exp(kx_df_fma_u(kx_df_fma_u(kx_df_fma_u(kx_df_fma_u(kx_mk(%s.x, %s.y), L, kx_mk(%s.z, %s.w)), L, "
                 "kx_mk(%s.x, %s.y)), L, kx_mk(%s.z, %s.w)), L, kx_mk(%s.x, %s.y)));",
                 e, z, z, y, y, y, y, x, x, x, x);
    if (md.kind == TrMode::F64)
      return fmt("const double %s = kx_exp(fma(fma(fma(fma(%s.x, L, %s.y), L, %s.x), L, %s.y), L, %s.x));", e, z, y, y, x, x);
    return fmt("const float %s = exp2f(fmaf(fmaf(fmaf(fmaf(%s.x, L, %s.y), L, %s.x), L, %s.y), L, %s.x));", e, z, y, y, x, x);
  };
  vec = md.kind == TrMode::DF ? "float4" : md.kind == TrMode::F64 ? "double2" : "float2";
  o(fmt("const %s* cq = (const %s*)kx_dc;", vec.c_str(), vec.c_str()));
  o(fmt("%s n0 = cq[0], n1 = cq[1], n2 = cq[2];", vec.c_str()));
  const std::string take = fmt("const %s c0 = n0, c1 = n1, c2 = n2; cq += 3; n0 = cq[0]; n1 = cq[1]; n2 = cq[2];", vec.c_str());
  if (opt.diff_mode == 2) {
    o("#pragma unroll 1");
    o(fmt("for (int k = 0; k < %d; ++k) {", ns));
    o(fmt("  %s Sk = %s;", md.ty, ZERO.c_str()));
    o("  #pragma unroll 2");
    o(fmt("  for (int j = 0; j < %d; ++j) {", ns));
    o("    if (j == k) continue;");
    o("    " + take);
    o("    " + pexp("e", "c0", "c1", "c2"));
    o("    Sk = " + FMA(ld(XS("j")), "e", "Sk") + ";");
    o("  }");
    o("  " + st(VS("sS", "k"), "Sk"));
    o("}");
    count_fma(ns * (ns - 1) * 5.0); count_exp(ns * (ns - 1.0));
  } else {
    // two pairs per iteration with their own row accumulators (four pairs in flight with the
    // unroll); the coefficient stream is read one pair ahead
    o("#pragma unroll 1");
    o(fmt("for (int k = 0; k < %d; ++k) {", ns - 1));
    o(fmt("  %s Sk = %s, Sk1 = %s;", md.ty, ld(VS("sS", "k")).c_str(), ZERO.c_str()));
    o(fmt("  const %s Xk = %s;", md.ty, ld(XS("k")).c_str()));
    o("  int j = k + 1;");
    o("  #pragma unroll 2");
    o(fmt("  for (; j + 1 < %d; j += 2) {", ns));
    o(fmt("    const %s a0 = n0, a1 = n1, a2 = n2, b0 = cq[3], b1 = cq[4], b2 = cq[5];", vec.c_str()));
    o("    cq += 6; n0 = cq[0]; n1 = cq[1]; n2 = cq[2];");
    o("    " + pexp("ea", "a0", "a1", "a2"));
    o("    " + pexp("eb", "b0", "b1", "b2"));
    o("    Sk = " + ACC(ld(XS("j")), "ea", "Sk") + ";");
    o("    Sk1 = " + ACC(ld(XS("(j + 1)")), "eb", "Sk1") + ";");
    o(fmt("    const %s Sa = %s;", md.ty, ACC("Xk", "ea", ld(VS("sS", "j"))).c_str()));
    o(fmt("    const %s Sb = %s;", md.ty, ACC("Xk", "eb", ld(VS("sS", "(j + 1)"))).c_str()));
    o("    " + st(VS("sS", "j"), "Sa"));
    o("    " + st(VS("sS", "(j + 1)"), "Sb"));
    o("  }");
    o(fmt("  if (j < %d) {", ns));
    o("    " + take);
    o("    " + pexp("e", "c0", "c1", "c2"));
    o("    Sk = " + ACC(ld(XS("j")), "e", "Sk") + ";");
    o(fmt("    const %s Sj = %s;", md.ty, ACC("Xk", "e", ld(VS("sS", "j"))).c_str()));
    o("    " + st(VS("sS", "j"), "Sj"));
    o("  }");
    const std::string ONE2 = md.kind == TrMode::DF ? "kx_mk(1.f, 0.f)" : md.kind == TrMode::F32 ? "1.0f" : "1.0";
    o("  " + st(VS("sS", "k"), FMA("Sk1", ONE2, "Sk")));
    o("}");
    count_fma(ns * (ns - 1) / 2.0 * 6); count_exp(ns * (ns - 1) / 2.0);
  }
  o(fmt("const double pr = %s / P;", D(P_ATM).c_str()));
  o(fmt("for (int k = 0; k < %d; ++k) {", ns));
  o(fmt("  const double Sk = %s, Xk = %s;", TOD(ld(VS("sS", "k"))).c_str(), TOD(ld(XS("k"))).c_str()));
  o("  const double* ds = kx_dself + 5 * k;");
  // D_k = (Wbar - X_k W_k)/Wbar / (S_k p/p_atm); a species with no partner present gets D_kk
  if (direct)
    o(fmt("  out2_[(long long)k * ld + i] = Sk > 0.0 ? fma(-Xk, kx_w[k] * iWbar, 1.0) * pr / Sk"
          " : pr / fma(fma(fma(fma(ds[4], lnT - %s, ds[3]), lnT - %s, ds[2]), lnT - %s, ds[1]), lnT - %s, ds[0]);",
          D(L0).c_str(), D(L0).c_str(), D(L0).c_str(), D(L0).c_str()));
  else
    o("  out2_[(long long)k * ld + i] = Sk > 0.0 ? fma(-Xk, kx_w[k] * iWbar, 1.0) * pr / Sk"
      " : exp(fma(fma(fma(fma(ds[4], lnT, ds[3]), lnT, ds[2]), lnT, ds[1]), lnT, ds[0])) * pr;");
  o("}");
  c.fp64 += 5 * ns + 4; c.div64 += ns + 2;
}

// ------------------------------------------------------------------ warp-cooperative rates
// Float64-accurate production rates with G states per warp (G a power of two
// up to 32) and the reactions of each class spread over the lanes.  Each
// warp keeps its states' species vectors {ln |C_k|, mu_k} and one entry per
// reaction (the signed rate as a float-pair mantissa and a power of two) in
// its own slice of shared memory, so no per-state vector lives in local
// memory; the work of a class is dealt out as (state, reaction) pairs,
// lane + 32 t, so partial rounds are shared by the group's states.  Phases
// per group of G states (warp-synchronous, no block barrier):
//   1. per-state scalars (lane g < G): T, ln T, 1/T, C_M, ln(p_atm/RT);
//   2. species (lane l serves state l mod G): sigma = sum Y_k/W_k reduced
//      over the state's lanes in a fixed tree order, then ln |C_k|, G_k/RT
//      (Eq. (Ck)) and mu_k = G_k/RT + ln |C_k| into shared memory;
//   3. reaction classes: ln k_f (Eq. (k_f)), third body and falloff blend,
//      ln |R_f| and ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/RT) (Eq. (K_p)),
//      the net rate from the larger rate and that ratio, kept unscaled as
//      m 2^e (m a float pair, e an integer);
//   4. the state's scale 2^-S from the largest e (the largest scaled rate
//      near 2^62), each rate scaled in place;
//   5. production rates gathered species-major (wdot_k = sum_i nu_ki q_i,
//      a fixed order) from per-lane chunks of a balanced entry list, partial
//      sums of species that straddle chunks combined in chunk order;
//   6. wdot_k 2^S written out as float64.
struct WcLayout {
  int G = 1, warps = 4, nw32 = 1, svs = 1;
  int off_sv = 0, off_yv = 0, off_qm = 0, off_sci = 0, off_nm = 0, off_qe = 0, warp_bytes = 0;
};

WcLayout wc_layout_of(const Mechanism& m, int group, int block) {
  WcLayout L;
  L.warps = block / 32;
  L.nw32 = (m.ns + 32) / 32;   // species 0..ns (ns: the zero entry that pads shorter reactions)
  // species region per state: the {ln |C|, mu} float4s of species 0..ns, later reused for up to
  // ns + 31 float-pair slots
  L.svs = std::max(m.ns + 1, (m.ns + 32) / 2 + 1);
  const int per_state = 80 + 16 * L.svs + 8 * L.svs + 8 * m.nr() + 8 + 4 * L.nw32 + 2 * m.nr();
  // one state per warp unless asked otherwise: the kernel serves small batches, where the
  // parallelism of many warps per state matters most
  L.G = group > 0 ? group : 1;
  (void)per_state;
  const int G = L.G;
  auto up16 = [](int b) { return (b + 15) / 16 * 16; };
  L.off_sv = up16(80 * G);
  L.off_yv = up16(L.off_sv + 16 * G * L.svs);
  L.off_qm = up16(L.off_yv + 8 * G * L.svs);
  L.off_sci = up16(L.off_qm + 8 * G * m.nr());
  L.off_nm = up16(L.off_sci + 8 * G);
  L.off_qe = up16(L.off_nm + 4 * G * L.nw32);
  L.warp_bytes = up16(L.off_qe + 2 * G * m.nr());
  return L;
}

std::string emit_wdot_wc(const Mechanism& m, const EmitOptions& opt, const std::string& entry, OpCounts& c,
                         Out& globals) {
  const int ns = m.ns, nr = m.nr();
  const WcLayout L = wc_layout_of(m, opt.rates_group, opt.block);
  const int G = L.G, NW32 = L.nw32, SVS = L.svs;
  const int LG = __builtin_ctz(G);
  const bool merged = true;
  std::vector<DfClass> cls = emit_class_tables(globals, m, merged);
  Out& g = globals;

  // ---- gather table: species-major entries (reaction, net coefficient), cut into 32/G chunks of
  // nearly equal length, stored entry-major ([j][chunk]) so that the lanes' loads of one step are
  // contiguous; each entry: reaction index in bits 0-14, "last entry of its slot" in bit 15 and the
  // upper half of the float32 coefficient in bits 16-31.  A slot is one chunk's partial sum of one
  // species; species k sums its slots kx_wslot[k] .. + count in chunk order.
  struct GE { int r; int k; int nu; };
  std::vector<GE> ent;
  int maxnu = 0;
  for (int k = 0; k < ns; ++k)
    for (int i = 0; i < nr; ++i) {
      int nu = 0;
      for (auto& s : m.rx[i].reac) if (s.first == k) nu -= s.second;
      for (auto& s : m.rx[i].prod) if (s.first == k) nu += s.second;
      if (nu != 0) { ent.push_back({i, k, nu}); maxnu = std::max(maxnu, std::abs(nu)); }
    }
  const int NCH = 32 / G, NE = (int)ent.size();
  const int CL = std::max(1, (NE + NCH - 1) / NCH);
  std::vector<int> tab((size_t)CL * NCH, 0);   // padding entries: reaction 0, coefficient 0
  std::vector<int> chslot(NCH, 0), sfirst(ns, 0), scount(ns, 0);
  int nslot = 0;
  for (int ch = 0; ch < NCH; ++ch) {
    const int b = ch * NE / NCH, e = (ch + 1) * NE / NCH;
    chslot[ch] = nslot;
    for (int j = b; j < e; ++j) {
      const bool last = j + 1 == e || ent[j + 1].k != ent[j].k;
      const float fc = (float)ent[j].nu;
      uint32_t fb;
      std::memcpy(&fb, &fc, 4);
      tab[(size_t)(j - b) * NCH + ch] = (int32_t)((fb & 0xffff0000u) | (last ? 0x8000u : 0u) | (uint32_t)ent[j].r);
      if (j == b || ent[j - 1].k != ent[j].k) { if (scount[ent[j].k] == 0) sfirst[ent[j].k] = nslot; }
      if (last) { ++scount[ent[j].k]; ++nslot; }
    }
  }
  if (nr > 0x7fff) return "";
  {
    std::string t;
    for (int v : tab) t += std::to_string(v) + ",";
    g(fmt("__device__ const int kx_wtab[%d] = {%s0};", (int)tab.size() + 1, t.c_str()));
    std::string cs, ss;
    for (int ch = 0; ch < NCH; ++ch) cs += std::to_string(chslot[ch]) + ",";
    for (int k = 0; k < ns; ++k) ss += fmt("{%d,%d},", sfirst[k], scount[k]);
    g(fmt("__device__ const int kx_wchs[%d] = {%s0};", NCH + 1, cs.c_str()));
    g(fmt("__device__ const int2 kx_wslot[%d] = {%s{0,0}};", ns + 1, ss.c_str()));
  }

  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  Out o;
  o.ind = 1;
  o(fmt("const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;"));
  o(fmt("unsigned char* const wsm = kx_dyn + wib * %d;", L.warp_bytes));
  o("#define KX_PF(p) kx_mk((p)[0], (p)[1])");
  o("float4* const sc4 = (float4*)wsm;   // [G][5]: {Td, ln T}, {1/T, ln(p_atm/RT)}, {C_M, C_M/sigma}, {ln p}, {T, p bits}");
  o(fmt("float4* const sv = (float4*)(wsm + %d);   // [G][%d]: {ln |C_k|, mu_k} float pairs; later the gather slots", L.off_sv, SVS));
  o(fmt("float2* const yv = (float2*)(wsm + %d);   // [G][%d]: Y_k/W_k float pairs (third-body sums)", L.off_yv, SVS));
  o(fmt("float2* const qm = (float2*)(wsm + %d);   // [G][nr]: rate mantissas, then scaled rates", L.off_qm));
  o(fmt("int2* const sci = (int2*)(wsm + %d);      // [G]: {largest rate exponent, flag: 0 ok, 1 outside the domain, 2 past n}", L.off_sci));
  o(fmt("unsigned* const nmk = (unsigned*)(wsm + %d);   // [G][%d]: bit k set for Y_k < 0", L.off_nm, NW32));
  o(fmt("short* const qe = (short*)(wsm + %d);     // [G][nr]: rate exponents", L.off_qe));
  o(fmt("const long long nwarp = (long long)gridDim.x * %d;", L.warps));
  o(fmt("for (long long i0 = ((long long)blockIdx.x * %d + wib) * %d; i0 < n; i0 += nwarp * %d) {", L.warps, G, G));
  ++o.ind;
  // ---- 1. per-state scalars
  o(fmt("if (lane < %d) {", G));
  ++o.ind;
  o("const long long i = i0 + lane;");
  o("double T = 1000.0, P = 101325.0;");
  o("int flag = 2;");
  o("if (i < n) {");
  o("  T = T_[i]; P = P_[i]; flag = 0;");
  o("  if (!(T > 0.0 && P > 0.0 && T < KX_INF && P < KX_INF)) { flag = 1; T = 1000.0; P = 101325.0; }");
  o("}");
  o("const kx_df Td = kx_d2df_i(T);");
  o("const kx_df lnT = kx_df_log_d(T);");
  o("const kx_df iT = kx_df_div(kx_mk(1.0f, 0.0f), Td);");
  o(fmt("const kx_df cM = kx_df_mul(kx_df_mul(kx_d2df_i(P), iT), %s);", DFc(1.0 / R_U).c_str()));
  o(fmt("const kx_df lnPRT = kx_df_sub(%s, lnT);", DFc(std::log(P_ATM / R_U)).c_str()));
  o("sc4[5 * lane + 0] = make_float4(Td.hi, Td.lo, lnT.hi, lnT.lo);");
  o("sc4[5 * lane + 1] = make_float4(iT.hi, iT.lo, lnPRT.hi, lnPRT.lo);");
  o("sc4[5 * lane + 2] = make_float4(cM.hi, cM.lo, 0.0f, 0.0f);");
  if (any_plog) {
    o("const kx_df lnP = kx_df_log_d(P);");
    o("sc4[5 * lane + 3] = make_float4(lnP.hi, lnP.lo, 0.0f, 0.0f);");
  }
  o("sc4[5 * lane + 4] = make_float4(__int_as_float(__double2loint(T)), __int_as_float(__double2hiint(T)), "
    "__int_as_float(__double2loint(P)), __int_as_float(__double2hiint(P)));");
  o("sci[lane] = make_int2(-32768, flag);");
  o(fmt("for (int w = 0; w < %d; ++w) nmk[%d * lane + w] = 0u;", NW32, NW32));
  o(fmt("sv[%d * lane + %d] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // the padding species: ln |C| = mu = 0", SVS, ns));
  --o.ind;
  o("}");
  o("__syncwarp();");
  c.fp32 += 40 + 45 + kDfDiv + 2 * kDfMul + kDfAdd;
  // ---- 2. species: lane serves state gs = lane mod G, species lane/G + (32/G) t
  const int NT = (ns * G + 31) / 32;
  o(fmt("const int gs = lane & %d;", G - 1));
  o("const long long is = i0 + gs;");
  o("const bool inb = is < n;");
  o(fmt("double Yv[%d];", NT));
  o("kx_df sg = kx_mk(0.0f, 0.0f);");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o(fmt("  const int k = (lane >> %d) + %d * t;", LG, 32 / G));
  o(fmt("  Yv[t] = (k < %d && inb) ? Y_[(long long)k * ld + is] : 0.0;", ns));
  o(fmt("  if (k < %d) {", ns));
  o("    const kx_df yk = kx_df_mul(kx_d2df_i(Yv[t]), KX_PF(kx_iwf + 2 * k));");
  o(fmt("    yv[%d * gs + k] = make_float2(yk.hi, yk.lo);", SVS));
  o("    sg = kx_df_add(sg, yk);");
  o("  }");
  o("}");
  o("// sigma of state gs: a butterfly over the lanes that serve it, then lane gs's sum for all");
  for (int off = G; off < 32; off *= 2)
    o(fmt("{ const float h = __shfl_xor_sync(0xffffffffu, sg.hi, %d), l = __shfl_xor_sync(0xffffffffu, sg.lo, %d); "
          "sg = kx_df_add(sg, kx_mk(h, l)); }", off, off));
  o("sg = kx_mk(__shfl_sync(0xffffffffu, sg.hi, gs), __shfl_sync(0xffffffffu, sg.lo, gs));");
  o(fmt("const float4 s0 = sc4[5 * gs + 0], s1 = sc4[5 * gs + 1], s2 = sc4[5 * gs + 2], s4 = sc4[5 * gs + 4];"));
  o("const kx_df Tg = kx_mk(s0.x, s0.y), lnTg = kx_mk(s0.z, s0.w), iTg = kx_mk(s1.x, s1.y);");
  o("const long long Tb = ((long long)__float_as_int(s4.y) << 32) | (unsigned)__float_as_int(s4.x);   // T's float64 bits");
  o("const kx_df fC = kx_df_div(kx_mk(s2.x, s2.y), sg);");
  o("const kx_df lnfC = kx_df_log(fC);");
  o("__syncwarp();");
  o(fmt("if (lane < %d) {", G));
  o("  sc4[5 * lane + 2] = make_float4(s2.x, s2.y, fC.hi, fC.lo);");
  o("  if (!(sg.hi > 0.0f && sg.hi < KX_INF_F) && sci[lane].y == 0) sci[lane].y = 1;");
  o("}");
  o("bool neg = false;");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o(fmt("  const int k = (lane >> %d) + %d * t;", LG, 32 / G));
  o(fmt("  if (k < %d) {", ns));
  o("    const double Yk = Yv[t];");
  o("    const long long yb = __double_as_longlong(Yk) & 0x7fffffffffffffffLL;");
  o("    kx_df l = kx_mk(-700.0f, 0.0f);   // ln |C_k|, floored at -700 (absent species)");
  o("    if (yb >= 0x0010000000000000LL && yb < 0x7ff0000000000000LL) {");
  o("      l = kx_df_add(kx_df_log_d(__longlong_as_double(yb)), kx_df_sub(lnfC, KX_PF(kx_lwf + 2 * k)));");
  o("      if (!(l.hi > -700.0f)) l = kx_mk(-700.0f, 0.0f);");
  o("    }");
  o(fmt("    if (Yk < 0.0) { neg = true; atomicOr(&nmk[%d * gs + (k >> 5)], 1u << (k & 31)); }", NW32));
  o("    const float* a = kx_gcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("    kx_df gk = kx_df_fma(KX_PF(a + 8), Tg, KX_PF(a + 6));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 4));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 2));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 0));");
  o("    gk = kx_df_fma(KX_PF(a + 10), iTg, gk);");
  o("    gk = kx_df_fma(KX_PF(a + 12), lnTg, gk);");
  o("    const kx_df mk_ = kx_df_add(gk, l);");
  o(fmt("    sv[%d * gs + k] = make_float4(l.hi, l.lo, mk_.hi, mk_.lo);", SVS));
  o("  }");
  o("}");
  o("const bool grpneg = __any_sync(0xffffffffu, neg);");
  if (G == 1) o("int emax = -32768;   // the largest power of two of the rates this lane has formed");
  o("__syncwarp();");
  c.fp32 += ns * (12 + kDfFma) + kDfDiv + kDfLog + ns * (45 + 2 * kDfAdd + 6 * kDfFma + kDfAdd);

  // ---- 3. reaction classes
  static const char* xyzw[4] = {"x", "y", "z", "w"};
  auto comp = [&](const char* base, int j) { return fmt("%s%d.%s", base, j / 4, xyzw[j % 4]); };
  auto main_pass = [&](OpCounts& c, bool sgn) {
    for (size_t ci = 0; ci < cls.size(); ++ci) {
      const DfClass& d = cls[ci];
      const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
      const int NF = fo ? 7 : tb ? 3 : 2;
      const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
      const int NC = (int)d.rx.size();
      o(fmt("#pragma unroll 1"));
      o(fmt("for (int p = lane; p < %d; p += 32) {   // class %d: %d reactions, %d reactant and %d product entries", G * NC,
            (int)ci, NC, d.nre, d.npr));
      ++o.ind;
      o(fmt("const int g = p & %d, r = p >> %d;   // lanes of one reaction side by side (its record loaded once)", G - 1, LG));
      o("const float4 A0 = sc4[5 * g + 0], A1 = sc4[5 * g + 1];");
      o("const kx_df Td = kx_mk(A0.x, A0.y), lnT = kx_mk(A0.z, A0.w), iT = kx_mk(A1.x, A1.y), lnPRT = kx_mk(A1.z, A1.w);");
      if (tb) {
        o("const float4 A2 = sc4[5 * g + 2];");
        o("const kx_df cM = kx_mk(A2.x, A2.y), fC = kx_mk(A2.z, A2.w);");
        o(fmt("const float2* yg = yv + %d * g;", SVS));
      }
      if (d.kind == Kind::Plog) {
        o("const float4 A3 = sc4[5 * g + 3], A4 = sc4[5 * g + 4];");
        o("const kx_df lnP = kx_mk(A3.x, A3.y);");
        o("const double P = __hiloint2double(__float_as_int(A4.w), __float_as_int(A4.z));");
      }
      o(fmt("const int4* sp4 = (const int4*)kx_s%d + %d * r;", (int)ci, P / 4));
      for (int q = 0; q < P / 4; ++q) o(fmt("const int4 c%d = sp4[%d];", q, q));
      o(fmt("const float4* svg = sv + %d * g;", SVS));
      for (int j = 0; j < E; ++j) o(fmt("const float4 v%d = svg[%s & 0xffff];", j, comp("c", j).c_str()));
      if (sgn) {
        o(fmt("const unsigned* nmg = nmk + %d * g;", NW32));
        for (int j = 0; j < E; ++j) o(fmt("const int k%d = %s & 0xffff;", j, comp("c", j).c_str()));
      }
      o(fmt("const int ri = %s;", comp("c", E).c_str()));
      o(fmt("const float4* f = kx_f%d + %d * r;", (int)ci, NF));
      o("const float4 f0 = f[0], f1 = f[1];");
      if (tb) {
        o(fmt("const int2 e = kx_e%d[r];", (int)ci));
        o("const float4 f2 = f[2];");
        o("kx_df X;   // [X] = eff_default C_M + (C_M/sigma) sum_e (eff_e - eff_default) Y_e/W_e");
        o("if (e.y < 0) {");
        o("  const int kc = kx_effd[e.x].k;");
        o("  X = kx_df_mul(kx_mk(yg[kc].x, yg[kc].y), fC);");
        o("} else {");
        o("  kx_df t = kx_mk(0.0f, 0.0f);");
        o("  for (int j = 0; j < e.y; ++j) {");
        o("    const kx_effd_t q = kx_effd[e.x + j];");
        o("    t = kx_df_fma(kx_mk(q.ahi, q.alo), kx_mk(yg[q.k].x, yg[q.k].y), t);");
        o("  }");
        o("  X = kx_df_fma(kx_mk(f2.x, f2.y), cM, kx_df_mul(fC, t));");
        o("}");
        c.fp32 += NC * (kDfFma + kDfMul + 3 * (kDfFma + kDfMul + 12));
      }
      // The float32 path of the thread-per-state kernel, per round: one state per warp (G = 1), so
      // the state's running largest power of two is a warp max of the lanes' own; a round whose
      // reactions all have both rates below 2^-40 of it takes float32 (the rate scaled by 2^-emx,
      // stored with the power of two emx)
      const bool fastp = G == 1 && opt.rates_negligible == 0 && (d.kind == Kind::Elementary || d.kind == Kind::ThreeBody || fo);
      const int dnf = d.npr - d.nre;
      auto negbit0 = [&](int j) { return fmt("((nmg[k%d >> 5] >> (k%d & 31)) & 1)", j, j); };
      if (fastp) {
        if (fo) {
          o("const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
          o("float lfe = fmaf(f0.z, lnT.hi, fmaf(f1.x, iT.hi, f0.x));   // ln k_inf (float32)");
          o("const float lk0e = fmaf(f3.x, lnT.hi, fmaf(f3.z, iT.hi, f2.z));");
          o("const float lpe = lk0e - lfe + __logf(X.hi);");
          if (d.blend == Blend::Troe) {
            o("const float lFc = __logf(f4.x * __expf(Td.hi * f5.x) + f4.z * __expf(Td.hi * f5.z) + __expf(f6.x * iT.hi)) * 0.434294482f;");
            o("const float xe = fmaf(lpe, 0.434294482f, fmaf(-0.67f, lFc, -0.4f));");
            o("const float fe = __fdividef(xe, fmaf(-0.14f, xe, fmaf(-1.27f, lFc, 0.75f)));");
            o("const float lFe = __fdividef(2.30258509f * lFc, fmaf(fe, fe, 1.0f));");
          } else if (d.blend == Blend::Sri) {
            o("const float lPe = lpe * 0.434294482f;");
            o("const float lFe = f5.z + f6.x * lnT.hi + __fdividef(__logf(f4.x * __expf(f4.z * iT.hi) + __expf(Td.hi * f5.x)), "
              "fmaf(lPe, lPe, 1.0f));");
          } else {
            o("const float lFe = 0.0f;");
          }
          o("const float l1e = __logf(1.0f + __expf(-fabsf(lpe)));");
          o(d.kind == Kind::Falloff ? "lfe += (lpe < 0.0f ? lpe - l1e : -l1e) + lFe;"
                                    : "lfe = lk0e + lFe - (lpe < 0.0f ? l1e : lpe + l1e);");
        } else {
          o(d.kconst ? "float lfe = f0.x;" : "float lfe = fmaf(f0.z, lnT.hi, fmaf(f1.x, iT.hi, f0.x));");
        }
        for (int j = 0; j < d.nre; ++j) o(fmt("lfe += v%d.x;", j));
        o(d.kind == Kind::ThreeBody ? "const float lxe = __logf(X.hi);" : "const float lxe = 0.0f;");
        o("float lme = lfe + lxe;");
        std::string t = merged ? std::string("f1.w * lnPRT.hi") : (dnf == 0 ? std::string("0.0f") : fmt("%s * lnPRT.hi", F(-dnf).c_str()));
        for (int j = 0; j < d.nre; ++j) t += fmt(" - v%d.z", j);
        for (int j = d.nre; j < E; ++j) t += fmt(" + v%d.z", j);
        if (d.rev) {
          o("const float lre = lfe + (" + t + ");");
          o("lme = fmaxf(lme, lre + lxe);");
        }
        std::string sfe = "0", sre = "0";
        if (sgn) {
          for (int j = 0; j < d.nre; ++j) sfe += " ^ " + negbit0(j);
          for (int j = d.nre; j < E; ++j) sre += " ^ " + negbit0(j);
        }
        o("const int emx = __reduce_max_sync(__activemask(), emax);");
        o("kx_df q;");
        o("int ex;");
        o("if (__all_sync(__activemask(), lme < __fmul_rn(kx_i2f(emx - 40), 0.693147182f))) {");
        o("  const float sl = __fmul_rn(kx_i2f(emx), 0.693147182f);");
        o("  float qf = __expf(lfe - sl);");
        o("  if (" + sfe + ") qf = -qf;");
        if (d.rev) {
          o("  float qr = __expf(lre - sl);");
          o("  if (" + sre + ") qr = -qr;");
          o("  qf -= qr;");
        }
        o("  q = kx_mk(qf, 0.0f);");
        o("  ex = emx;");
        o("} else {");
        c.fp32 += NC * (8.0 + d.nre + (d.rev ? E : 0) + (fo ? 40 : 0));
      }
      o(d.kconst ? "kx_df lk = kx_mk(f0.x, f0.y);   // k = A"
                 : "kx_df lk = kx_df_fma_u(kx_mk(f0.z, f0.w), lnT, kx_df_fma_u(kx_mk(f1.x, f1.y), iT, kx_mk(f0.x, f0.y)));");
      if (fo) {
        if (!fastp) o("const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
        o("const kx_df lk0 = kx_df_fma(kx_mk(f3.x, f3.y), lnT, kx_df_fma(kx_mk(f3.z, f3.w), iT, kx_mk(f2.z, f2.w)));");
        o("kx_df lnPr = kx_df_add(kx_df_sub(lk0, lk), kx_df_log(X));");
        o("if (!(lnPr.hi > -690.775528f)) lnPr = kx_mk(-690.775528f, 0.0f);");
        o("kx_df lnF = kx_mk(0.0f, 0.0f);");
        const std::string il10 = DFc(1.0 / std::log(10.0));
        if (d.blend == Blend::Troe) {
          o("kx_df Fc = kx_df_exp_s(kx_df_mul(kx_mk(f6.x, f6.y), iT));");
          o("Fc = kx_df_fma(kx_mk(f4.x, f4.y), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.x, f5.y))), Fc);");
          o("Fc = kx_df_fma(kx_mk(f4.z, f4.w), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.z, f5.w))), Fc);");
          o(fmt("const kx_df lFc = kx_df_mul(kx_df_log(Fc), %s);", il10.c_str()));
          o(fmt("const kx_df xx = kx_df_fma(lnPr, %s, kx_df_fma(%s, lFc, %s));", il10.c_str(), DFc(-0.67).c_str(), DFc(-0.4).c_str()));
          o(fmt("const kx_df ff = kx_df_div(xx, kx_df_fma(%s, xx, kx_df_fma(%s, lFc, %s)));", DFc(-0.14).c_str(), DFc(-1.27).c_str(),
                DFc(0.75).c_str()));
          o(fmt("lnF = kx_df_div(kx_df_mul(%s, lFc), kx_df_fma(ff, ff, kx_mk(1.0f, 0.0f)));", DFc(std::log(10.0)).c_str()));
          c.fp32 += NC * (3 * (kDfMul + kDfExp) + 2 * kDfFma + kDfLog + kDfMul + 4 * kDfFma + 2 * kDfDiv + kDfMul);
        } else if (d.blend == Blend::Sri) {
          o(fmt("const kx_df lPr = kx_df_mul(lnPr, %s);", il10.c_str()));
          o("const kx_df base = kx_df_fma(kx_mk(f4.x, f4.y), kx_df_exp_s(kx_df_mul(kx_mk(f4.z, f4.w), iT)), kx_df_exp_s(kx_df_mul(Td, kx_mk(f5.x, f5.y))));");
          o("lnF = kx_df_add(kx_mk(f5.z, f5.w), kx_df_fma(kx_mk(f6.x, f6.y), lnT, kx_df_div(kx_df_log(base), kx_df_fma(lPr, lPr, kx_mk(1.0f, 0.0f)))));");
          c.fp32 += NC * (2 * (kDfMul + kDfExp) + kDfFma + kDfMul + kDfLog + 2 * kDfFma + kDfDiv + kDfAdd);
        }
        o("const bool small = lnPr.hi < 0.0f;");
        o("const kx_df l1p = kx_df_log1p(kx_df_exp_n(small ? lnPr : kx_df_neg(lnPr)));");
        if (d.kind == Kind::Falloff) o("lk = kx_df_add(lk, kx_df_add(small ? kx_df_sub(lnPr, l1p) : kx_df_neg(l1p), lnF));");
        else o("lk = kx_df_add(lk0, kx_df_sub(lnF, small ? l1p : kx_df_add(lnPr, l1p)));");
        c.fp32 += NC * (2 * kDfFma + 2 * kDfAdd + kDfLog + kDfExp + kDfLog + 3 * kDfAdd);
      } else if (d.kind == Kind::Plog) {
        o(fmt("const int2 e = kx_e%d[r];", (int)ci));
        o("const float* t = kx_plogf + 8 * e.x; const long long* tp = kx_plogp + e.x; const int np = e.y;");
        o("const long long Pb = __double_as_longlong(P);");
        o("if (Pb <= tp[0]) lk = kx_df_fma(KX_PF(t + 4), lnT, kx_df_fma(KX_PF(t + 6), iT, KX_PF(t + 2)));");
        o("else if (Pb >= tp[np - 1]) { const float* u = t + 8 * (np - 1); lk = kx_df_fma(KX_PF(u + 4), lnT, kx_df_fma(KX_PF(u + 6), iT, KX_PF(u + 2))); }");
        o("else {");
        o("  int j = 0; while (!(Pb < tp[j + 1])) ++j;");
        o("  const float* u = t + 8 * j;");
        o("  const kx_df l1 = kx_df_fma(KX_PF(u + 4), lnT, kx_df_fma(KX_PF(u + 6), iT, KX_PF(u + 2)));");
        o("  const kx_df l2 = kx_df_fma(KX_PF(u + 12), lnT, kx_df_fma(KX_PF(u + 14), iT, KX_PF(u + 10)));");
        o("  lk = kx_df_fma(kx_df_sub(l2, l1), kx_df_div(kx_df_sub(lnP, KX_PF(u)), kx_df_sub(KX_PF(u + 8), KX_PF(u))), l1);");
        o("}");
        c.fp32 += NC * (4 * kDfFma + 3 * kDfAdd + kDfDiv);
      }
      int real_re = 0, real_e = 0;   // entries without the padding, for the operation counts
      for (int i : d.rx) {
        real_re += (int)entries(m.rx[i].reac).size();
        real_e += (int)entries(m.rx[i].reac).size() + (int)entries(m.rx[i].prod).size();
      }
      o("kx_df lf = lk;");
      for (int j = 0; j < d.nre; ++j) o(fmt("lf = kx_df_add_u(lf, kx_mk(v%d.x, v%d.y));", j, j));
      auto negbit = [&](int j) { return fmt("((nmg[k%d >> 5] >> (k%d & 31)) & 1)", j, j); };
      std::string sfx = "0", srx = "0";
      if (sgn) {
        for (int j = 0; j < d.nre; ++j) sfx += " ^ " + negbit(j);
        for (int j = d.nre; j < E; ++j) srx += " ^ " + negbit(j);
      }
      o("int sf = " + sfx + ";");
      o("kx_df L = lf, fac = kx_mk(1.0f, 0.0f);");
      c.fp32 += NC * (2 * kDfFma + kDfExp + kDfMul) + real_re * kDfAdd;
      if (d.rev) {
        const int dn = d.npr - d.nre;
        o("{   // ln(|R_r|/|R_f|) = sum nu mu - dn ln(p_atm/(R T))");
        std::string first = d.nre > 0 ? "kx_df_neg(kx_mk(v0.z, v0.w))" : "kx_mk(v0.z, v0.w)";
        o("  kx_df dl = " + first + ";");
        for (int j = 1; j < E; ++j)
          o(fmt("  dl = kx_df_add_u(dl, kx_mk(%sv%d.z, %sv%d.w));", j < d.nre ? "-" : "", j, j < d.nre ? "-" : "", j));
        if (merged) o("  dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, f1.w));   // -dn ln(p_atm/RT), dn of this reaction");
        else if (dn == 1 || dn == -1) o(fmt("  dl = kx_df_add_u(dl, %s);", dn == 1 ? "kx_df_neg(lnPRT)" : "lnPRT"));
        else if (dn != 0) o(fmt("  dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, %s));", F(-dn).c_str()));
        o("  const int sr = " + srx + ";");
        o("  const bool rev = dl.hi > 0.0f;");
        o("  if (rev) L = kx_df_add_u(lf, dl);");
        o("  const kx_df e = kx_df_exp_n(rev ? kx_df_neg(dl) : dl);");
        o("  const float pm = sf == sr ? -1.0f : 1.0f;   // |R_f| -+ |R_r| = larger (1 -+ e^-|ln ratio|)");
        o("  const kx_df s1 = kx_qts(1.0f, pm * e.hi);");
        o("  fac = kx_mk(s1.hi, __fmaf_rn(pm, e.lo, s1.lo));");
        o("  if (sf == sr) sf ^= (int)rev;");
        o("}");
        c.fp32 += (real_e - NC) * kDfAdd + NC * (kDfAdd + kDfMulf + kDfAdd + kDfExp + 10);
        (void)dn;
      }
      if (fastp) {
        o("q = kx_df_mul_u(kx_df_exp_m(L, ex), fac);   // |R| = q 2^ex");
        o("if (sf) q = kx_df_neg(q);");
        o("emax = max(emax, ex);");
        o("}");
      } else {
        o("int ex;");
        o("kx_df q = kx_df_mul_u(kx_df_exp_m(L, ex), fac);   // |R| = q 2^ex");
        o("if (sf) q = kx_df_neg(q);");
      }
      if (d.kind == Kind::ThreeBody) { o("q = kx_df_mul_u(q, X);"); c.fp32 += NC * kDfMul; }
      o(fmt("qm[%d * g + ri] = make_float2(q.hi, q.lo);", nr));
      o(fmt("qe[%d * g + ri] = (short)ex;", nr));
      --o.ind;
      o("}");
    }
  };
  o("if (grpneg) {");
  ++o.ind;
  main_pass(c, true);
  --o.ind;
  o("} else {");
  ++o.ind;
  {
    OpCounts once;
    main_pass(once, false);
  }
  --o.ind;
  o("}");
  // ---- 4. the largest exponent of each state (a warp max over its rates); rates scaled in place
  o("__syncwarp();");
  o(fmt("for (int g = 0; g < %d; ++g) {", G));
  o("  int e = -32768;");
  o(fmt("  for (int r = lane; r < %d; r += 32) e = max(e, (int)qe[%d * g + r]);", nr, nr));
  o("  e = __reduce_max_sync(0xffffffffu, e);");
  o("  if (lane == 0) sci[g].x = e;");
  o("}");
  o("__syncwarp();");
  o("#pragma unroll 1");
  o(fmt("for (int p = lane; p < %d; p += 32) {", G * nr));
  o(fmt("  const int g = p / %d;", nr));
  o("  const int d = (int)qe[p] - (sci[g].x - 62);   // S = e_max - 62; 2^d normal for d >= -126 (below: under 2^-188 of the largest)");
  o("  const float2 v = qm[p];");
  o("  const float sc = d >= -126 ? __int_as_float((d + 127) << 23) : 0.0f;");
  o("  qm[p] = make_float2(__fmul_rn(v.x, sc), __fmul_rn(v.y, sc));");
  o("}");
  o("__syncwarp();");
  c.fp32 += nr * 4;
  // ---- 5. gather: lane serves state gs and chunk lane / G
  o(fmt("{   // species-major sums from chunk %s of the entry list", "lane / G"));
  ++o.ind;
  o(fmt("const int ch = lane >> %d;", LG));
  o(fmt("const float2* qg = qm + %d * gs;", nr));
  o(fmt("float2* const slot = (float2*)(sv + %d * gs);", SVS));
  o("int sl = kx_wchs[ch];");
  o("kx_df acc = kx_mk(0.0f, 0.0f);");
  o("#pragma unroll 4");
  o(fmt("for (int j = 0; j < %d; ++j) {", CL));
  o(fmt("  const unsigned w = (unsigned)kx_wtab[%d * j + ch];", NCH));
  o("  const float2 q = qg[w & 0x7fffu];");
  o(fmt("  acc = kx_df_add_u(acc, %s(kx_mk(q.x, q.y), __uint_as_float(w & 0xffff0000u)));",
        maxnu <= 2 ? "kx_df_scale2" : "kx_df_mulf"));
  o("  if (w & 0x8000u) { slot[sl++] = make_float2(acc.hi, acc.lo); acc = kx_mk(0.0f, 0.0f); }");
  o("}");
  --o.ind;
  o("}");
  o("__syncwarp();");
  c.fp32 += (double)NE * (kDfAdd + (maxnu <= 2 ? 2 : kDfMulf));
  if (nslot > 2 * SVS) return "";
  // ---- 6. output: pairs (state, species), consecutive lanes on consecutive states
  o("#pragma unroll 1");
  o(fmt("for (int p = lane; p < %d; p += 32) {", G * ns));
  o(fmt("  const int g = p & %d, k = p >> %d;", G - 1, LG));
  o("  const long long i = i0 + g;");
  o("  const int2 st = sci[g];");
  o("  if (st.y == 2) continue;");
  o("  if (st.y == 1) { out_[(long long)k * ld + i] = KX_NAN; continue; }");
  o("  const int2 sl = kx_wslot[k];");
  o(fmt("  const float2* slot = (const float2*)(sv + %d * g);", SVS));
  o("  kx_df w = kx_mk(0.0f, 0.0f);");
  o("  for (int j = 0; j < sl.y; ++j) w = kx_df_add_u(w, kx_mk(slot[sl.x + j].x, slot[sl.x + j].y));");
  o("  out_[(long long)k * ld + i] = kx_df2d_s(w, st.x - 62);");
  o("}");
  o(fmt("if (lane < %d && sci[lane].y == 1) atomicMin(&kx_bad_first, (unsigned long long)(i0 + lane));", G));
  o("__syncwarp();");
  --o.ind;
  o("}");
  c.fp64 += ns;
  c.fp32 += ns * kDfAdd;
  return o.o.str();
}

// ------------------------------------------------------------------ warp-cooperative adjoint
// The double-float adjoint with one state per warp and everything per state in shared memory:
//   1. per-state scalars (lane 0);
//   2. species over the lanes: ln |C_k|, mu_k, the cotangent v_k, H_k/RT, the signed reciprocal
//      1/C_k as mantissa and power of two, Y_k/W_k;
//   3. reactions over the lanes (classes merged by kind, as in the warp-cooperative rates): per
//      reaction the temperature terms into the lane's running d/dT and d/d[M] sums, and the
//      reaction's a c R_f, -a c R_r and third-body a (R_f - R_r) [dln k_f/d[X]] terms, each a
//      mantissa and a power of two, into shared memory;
//   4. d/dC_k gathered species-major from a balanced entry list (one chunk per lane; each term a
//      reaction's mantissa times 1/C_k, or a third-body term times an efficiency), partial sums
//      under their own scales, combined in chunk order;
//   5. the chain to (T, Y) in float64 (lane sums reduced in a fixed butterfly order).
struct VwLayout {
  int svs = 1, nw32 = 1;
  int off_sv = 0, off_vh = 0, off_ic = 0, off_yv = 0, off_rf = 0, off_re = 0, off_tb = 0, off_nm = 0, warp_bytes = 0;
};

VwLayout vjp_wc_layout(const Mechanism& m) {
  VwLayout L;
  L.nw32 = (m.ns + 32) / 32;
  L.svs = std::max(m.ns + 1, (m.ns + 33) / 2);   // species 0..ns; sv and vh later hold ns + 32 gather slots
  auto up16 = [](int b) { return (b + 15) / 16 * 16; };
  const int nr = m.nr();
  L.off_sv = 96;
  L.off_vh = L.off_sv + 16 * L.svs;
  L.off_ic = L.off_vh + 16 * L.svs;
  L.off_yv = L.off_ic + 16 * L.svs;
  int ntb = 0;
  for (auto& r : m.rx) ntb += r.third_body() ? 1 : 0;
  L.off_rf = up16(L.off_yv + 8 * L.svs);
  L.off_re = L.off_rf + 16 * nr;
  L.off_tb = up16(L.off_re + 8 * nr);
  L.off_nm = L.off_tb + 16 * std::max(ntb, 1);
  L.warp_bytes = up16(L.off_nm + 4 * L.nw32);
  return L;
}

std::string emit_vjp_wc(const Mechanism& m, const EmitOptions& opt, OpCounts& c, Out& g) {
  (void)opt;
  const int ns = m.ns, nr = m.nr();
  const VwLayout L = vjp_wc_layout(m);
  const int SVS = L.svs, NW32 = L.nw32;
  std::vector<DfClass> cls = emit_class_tables(g, m, true);
  const std::string shift = DFc(2016.0 * std::log(2.0));
  // third-body reactions' slots in the per-warp third-body array: consecutive in class order
  std::vector<int> tbslot(nr, -1), tbbase(cls.size(), 0), tbreac;
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    tbbase[ci] = (int)tbreac.size();
    if (m.rx[cls[ci].rx[0]].third_body())
      for (int i : cls[ci].rx) { tbslot[i] = (int)tbreac.size(); tbreac.push_back(i); }
  }
  // H/RT coefficients as float pairs per species and range
  {
    std::string hf, iwd;
    for (int k = 0; k < ns; ++k) {
      for (int rg = 0; rg < 2; ++rg) {
        const double* a = rg == 0 ? &m.a_lo[7 * k] : &m.a_hi[7 * k];
        const double h[8] = {a[0], a[1] / 2.0, a[2] / 3.0, a[3] / 4.0, a[4] / 5.0, a[5], 0.0, 0.0};
        for (int j = 0; j < 8; ++j) hf += fpair(h[j]) + ",";
      }
      iwd += D(1.0 / m.W[k]) + ",";
    }
    g(fmt("__device__ const __align__(16) float kx_hcf[%d] = {%s0.0f};", 32 * ns + 4, hf.c_str()));
    g(fmt("__device__ const double kx_iwd[%d] = {%s0.0};", ns + 1, iwd.c_str()));
  }
  // ---- gather table: per species k, its reactant entries (kind 0: nu'_k a c R_f / C_k), product entries
  // of reversible reactions (kind 1: -nu''_k a c R_r / C_k) and third-body efficiencies (kind 2:
  // (eff_k - eff_default) a (R_f - R_r) [dln k_f/d[X]], or 1 for a named collider); entry bits:
  // reaction (kind 2: its third-body slot) 0-13, kind 14-15, species 16-30, "last of its slot" 31; the
  // coefficient as a float pair
  // (stoichiometric coefficients are exact in its high part, efficiency differences such as 0.7 - 1
  // are not)
  struct GE { int r, kind, k; double coef; };
  std::vector<GE> ent;
  for (int k = 0; k < ns; ++k)
    for (int i = 0; i < nr; ++i) {
      const Reaction& r = m.rx[i];
      int a = 0, b = 0;
      for (auto& s : r.reac) if (s.first == k) a += s.second;
      for (auto& s : r.prod) if (s.first == k) b += s.second;
      if (a) ent.push_back({i, 0, k, (double)a});
      if (b && r.reversible) ent.push_back({i, 1, k, (double)b});
      if (r.third_body()) {
        if (r.collider >= 0) { if (r.collider == k) ent.push_back({tbslot[i], 2, k, 1.0}); }
        else for (auto& e : r.eff) if (e.first == k && e.second != r.default_eff) ent.push_back({tbslot[i], 2, k, e.second - r.default_eff});
      }
    }
  if (nr >= (1 << 14) || ns >= (1 << 15)) return "";
  const int NCH = 32, NE = (int)ent.size();
  const int CL = std::max(1, (NE + NCH - 1) / NCH);
  std::vector<std::pair<int32_t, double>> tab((size_t)CL * NCH, {0, 0.0});
  std::vector<int> chslot(NCH, 0), sfirst(ns, 0), scount(ns, 0);
  int nslot = 0;
  for (int ch = 0; ch < NCH; ++ch) {
    const int b = ch * NE / NCH, e = (ch + 1) * NE / NCH;
    chslot[ch] = nslot;
    for (int j = b; j < e; ++j) {
      const bool last = j + 1 == e || ent[j + 1].k != ent[j].k;
      tab[(size_t)(j - b) * NCH + ch] = {(int32_t)((uint32_t)ent[j].r | ((uint32_t)ent[j].kind << 14) | ((uint32_t)ent[j].k << 16) |
                                                   (last ? 0x80000000u : 0u)), ent[j].coef};
      if ((j == b || ent[j - 1].k != ent[j].k) && scount[ent[j].k] == 0) sfirst[ent[j].k] = nslot;
      if (last) { ++scount[ent[j].k]; ++nslot; }
    }
  }
  if (nslot > 2 * SVS) return "";
  {
    std::string t;
    for (auto& v : tab) t += fmt("{%d,%s,0},", v.first, fpair(v.second).c_str());
    g(fmt("__device__ const __align__(16) struct { int w; float c, cl; int pad; } kx_vtab[%d] = {%s{0,0.0f,0.0f,0}};",
          (int)tab.size() + 1, t.c_str()));
    std::string cs, ss;
    for (int ch = 0; ch < NCH; ++ch) cs += std::to_string(chslot[ch]) + ",";
    for (int k = 0; k < ns; ++k) ss += fmt("{%d,%d},", sfirst[k], scount[k]);
    g(fmt("__device__ const int kx_vchs[%d] = {%s0};", NCH + 1, cs.c_str()));
    std::string tr;
    for (int i : tbreac) tr += std::to_string(i) + ",";
    g("// third-body slot -> reaction: {" + tr + "}");
    g(fmt("__device__ const int2 kx_vslot[%d] = {%s{0,0}};", ns + 1, ss.c_str()));
  }
  bool any_plog = false;
  for (auto& r : m.rx) any_plog |= r.kind == Kind::Plog;
  const int NT = (ns + 31) / 32;
  Out o;
  o.ind = 1;
  o("#define KX_PF(p) kx_mk((p)[0], (p)[1])");
  o("const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;");
  o(fmt("unsigned char* const wsm = kx_dyn + wib * %d;", L.warp_bytes));
  o("float4* const sc4 = (float4*)wsm;   // {Td, ln T}, {1/T, ln(p_atm/RT)}, {C_M, C_M/sigma}, {ln p, 1/T^2}, {T, p bits}");
  o("int* const scf = (int*)(wsm + 80);   // state flag: 0 ok, 1 outside the domain");
  o(fmt("float4* const sv = (float4*)(wsm + %d);   // {ln |C_k|, mu_k}; later the gather slots", L.off_sv));
  o(fmt("float4* const vh = (float4*)(wsm + %d);   // {v_k, H_k/RT}", L.off_vh));
  o(fmt("float4* const ic = (float4*)(wsm + %d);   // 1/C_k: {signed mantissa, power of two}", L.off_ic));
  o(fmt("float2* const yv = (float2*)(wsm + %d);   // Y_k/W_k", L.off_yv));
  o(fmt("float4* const rf = (float4*)(wsm + %d);   // per reaction {a c R_f, -a c R_r} mantissas", L.off_rf));
  o(fmt("int2* const re = (int2*)(wsm + %d);       // per reaction their powers of two", L.off_re));
  o(fmt("float4* const rt = (float4*)(wsm + %d);   // per third-body reaction {its term's mantissa, power of two}", L.off_tb));
  o(fmt("unsigned* const nmk = (unsigned*)(wsm + %d);", L.off_nm));
  o(fmt("const long long nwarp = (long long)gridDim.x * %d;", opt.block / 32));
  o(fmt("for (long long i = (long long)blockIdx.x * %d + wib; i < n; i += nwarp) {", opt.block / 32));
  ++o.ind;
  // ---- 1. scalars
  o("if (lane == 0) {");
  o("  double T = T_[i], P = P_[i];");
  o("  int flag = 0;");
  o("  if (!(T > 0.0 && P > 0.0 && T < KX_INF && P < KX_INF)) { flag = 1; T = 1000.0; P = 101325.0; }");
  o("  const kx_df Td = kx_d2df_i(T), lnT = kx_df_log_d(T), iT = kx_df_div(kx_mk(1.0f, 0.0f), Td), iT2 = kx_df_mul(iT, iT);");
  o(fmt("  const kx_df cM = kx_df_mul(kx_df_mul(kx_d2df_i(P), iT), %s);", DFc(1.0 / R_U).c_str()));
  o(fmt("  const kx_df lnPRT = kx_df_sub(%s, lnT);", DFc(std::log(P_ATM / R_U)).c_str()));
  o("  sc4[0] = make_float4(Td.hi, Td.lo, lnT.hi, lnT.lo);");
  o("  sc4[1] = make_float4(iT.hi, iT.lo, lnPRT.hi, lnPRT.lo);");
  o("  sc4[2] = make_float4(cM.hi, cM.lo, 0.0f, 0.0f);");
  o(any_plog ? "  const kx_df lnP = kx_df_log_d(P);" : "  const kx_df lnP = kx_mk(0.0f, 0.0f);");
  o("  sc4[3] = make_float4(lnP.hi, lnP.lo, iT2.hi, iT2.lo);");
  o("  sc4[4] = make_float4(__int_as_float(__double2loint(T)), __int_as_float(__double2hiint(T)), "
    "__int_as_float(__double2loint(P)), __int_as_float(__double2hiint(P)));");
  o("  *scf = flag;");
  o(fmt("  for (int w = 0; w < %d; ++w) nmk[w] = 0u;", NW32));
  o(fmt("  sv[%d] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); vh[%d] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // padding species", ns, ns));
  o(fmt("  ic[%d] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); yv[%d] = make_float2(0.0f, 0.0f);", ns, ns));
  o("}");
  o("__syncwarp();");
  // ---- 2. species
  o("const float4 s0 = sc4[0], s1 = sc4[1], s2 = sc4[2], s4 = sc4[4];");
  o("const kx_df Tg = kx_mk(s0.x, s0.y), lnTg = kx_mk(s0.z, s0.w), iTg = kx_mk(s1.x, s1.y);");
  o("const long long Tb = ((long long)__float_as_int(s4.y) << 32) | (unsigned)__float_as_int(s4.x);");
  o(fmt("double Yv[%d];", NT));
  o("kx_df sg = kx_mk(0.0f, 0.0f);");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o("  const int k = lane + 32 * t;");
  o(fmt("  Yv[t] = k < %d ? Y_[(long long)k * ld + i] : 0.0;", ns));
  o(fmt("  if (k < %d) {", ns));
  o("    const kx_df yk = kx_df_mul(kx_d2df_i(Yv[t]), KX_PF(kx_iwf + 2 * k));");
  o("    yv[k] = make_float2(yk.hi, yk.lo);");
  o("    sg = kx_df_add(sg, yk);");
  o("  }");
  o("}");
  for (int off = 1; off < 32; off *= 2)
    o(fmt("{ const float h = __shfl_xor_sync(0xffffffffu, sg.hi, %d), l = __shfl_xor_sync(0xffffffffu, sg.lo, %d); sg = kx_df_add(sg, kx_mk(h, l)); }", off, off));
  o("sg = kx_mk(__shfl_sync(0xffffffffu, sg.hi, 0), __shfl_sync(0xffffffffu, sg.lo, 0));");
  o("const kx_df fC = kx_df_div(kx_mk(s2.x, s2.y), sg);");
  o("const kx_df lnfC = kx_df_log(fC);");
  o("__syncwarp();");
  o("if (lane == 0) {");
  o("  sc4[2] = make_float4(s2.x, s2.y, fC.hi, fC.lo);");
  o("  if (!(sg.hi > 0.0f && sg.hi < KX_INF_F)) *scf = 1;");
  o("}");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o("  const int k = lane + 32 * t;");
  o(fmt("  if (k < %d) {", ns));
  o("    const double Yk = Yv[t];");
  o("    const long long yb = __double_as_longlong(Yk) & 0x7fffffffffffffffLL;");
  o("    kx_df l = kx_mk(-700.0f, 0.0f);");
  o("    if (yb >= 0x0010000000000000LL && yb < 0x7ff0000000000000LL) {");
  o("      l = kx_df_add(kx_df_log_d(__longlong_as_double(yb)), kx_df_sub(lnfC, KX_PF(kx_lwf + 2 * k)));");
  o("      if (!(l.hi > -700.0f)) l = kx_mk(-700.0f, 0.0f);");
  o("    }");
  o("    if (Yk < 0.0) atomicOr(&nmk[k >> 5], 1u << (k & 31));");
  o("    const float* a = kx_gcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("    kx_df gk = kx_df_fma(KX_PF(a + 8), Tg, KX_PF(a + 6));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 4));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 2));");
  o("    gk = kx_df_fma(gk, Tg, KX_PF(a + 0));");
  o("    gk = kx_df_fma(KX_PF(a + 10), iTg, gk);");
  o("    gk = kx_df_fma(KX_PF(a + 12), lnTg, gk);");
  o("    const kx_df mk_ = kx_df_add(gk, l);");
  o("    sv[k] = make_float4(l.hi, l.lo, mk_.hi, mk_.lo);");
  o("    const float* hc = kx_hcf + 32 * k + (Tb < kx_tmidb[k] ? 0 : 16);");
  o("    kx_df hk = kx_df_fma(KX_PF(hc + 8), Tg, KX_PF(hc + 6));");
  o("    hk = kx_df_fma(hk, Tg, KX_PF(hc + 4));");
  o("    hk = kx_df_fma(hk, Tg, KX_PF(hc + 2));");
  o("    hk = kx_df_fma(hk, Tg, KX_PF(hc + 0));");
  o("    hk = kx_df_fma(KX_PF(hc + 10), iTg, hk);");
  o("    const kx_df vk = kx_d2df_i(V_[(long long)k * ld + i]);");
  o("    vh[k] = make_float4(vk.hi, vk.lo, hk.hi, hk.lo);");
  o("    int e; kx_df mi = kx_df_exp_m(kx_df_neg(l), e);");
  o("    if (Yk < 0.0) mi = kx_df_neg(mi);   // the reciprocal carries the concentration's sign");
  o("    ic[k] = make_float4(mi.hi, mi.lo, __int_as_float(e), 0.0f);");
  o("  }");
  o("}");
  o("__syncwarp();");
  c.fp32 += 40 + 45 + kDfDiv + 3 * kDfMul + kDfAdd + kDfDiv + kDfLog;
  c.fp32 += ns * (12 + kDfMul + kDfAdd) + ns * (45 + 2 * kDfAdd + 11 * kDfFma + kDfAdd + kDfExp);
  // ---- 3. reactions
  static const char* xyzw[4] = {"x", "y", "z", "w"};
  auto comp = [&](const char* base, int j) { return fmt("%s%d.%s", base, j / 4, xyzw[j % 4]); };
  const std::string il10 = DFc(1.0 / std::log(10.0));
  o("kx_df gTa = kx_mk(0.0f, 0.0f), gMa = kx_mk(0.0f, 0.0f);   // this lane's d/dT (fixed C) and d/d[M] sums");
  o("int sT = -100000, sM = -100000;");
  o("{");
  ++o.ind;
  o("const float4 A0 = sc4[0], A1 = sc4[1], A2 = sc4[2], A3 = sc4[3], A4 = sc4[4];");
  o("const kx_df Td = kx_mk(A0.x, A0.y), lnT = kx_mk(A0.z, A0.w), iT = kx_mk(A1.x, A1.y), lnPRT = kx_mk(A1.z, A1.w);");
  o("const kx_df cM = kx_mk(A2.x, A2.y), fC = kx_mk(A2.z, A2.w), lnP = kx_mk(A3.x, A3.y), iT2 = kx_mk(A3.z, A3.w);");
  o("const double P = __hiloint2double(__float_as_int(A4.w), __float_as_int(A4.z));");
  o("(void)lnP; (void)P; (void)cM; (void)fC;");
  o("#define KX_NEG(k) ((int)((nmk[(k) >> 5] >> ((k) & 31)) & 1u))");
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    const DfClass& d = cls[ci];
    const bool tb = d.kind == Kind::ThreeBody || d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const bool fo = d.kind == Kind::Falloff || d.kind == Kind::ChemAct;
    const int NF = fo ? 7 : tb ? 3 : 2;
    const int E = d.nre + d.npr, P = (E + 1 + 3) / 4 * 4;
    const double NC = (double)d.rx.size();
    o("#pragma unroll 1");
    o(fmt("for (int r = lane; r < %d; r += 32) {   // class %d: %d reactions, %d reactant and %d product entries (padded)",
          (int)d.rx.size(), (int)ci, (int)d.rx.size(), d.nre, d.npr));
    ++o.ind;
    o(fmt("const int4* sp4 = (const int4*)kx_s%d + %d * r;", (int)ci, P / 4));
    for (int q = 0; q < P / 4; ++q) o(fmt("const int4 c%d = sp4[%d];", q, q));
    for (int j = 0; j < E; ++j) o(fmt("const int k%d = %s & 0xffff;", j, comp("c", j).c_str()));
    for (int j = 0; j < E; ++j) o(fmt("const float4 v%d = sv[k%d];", j, j));
    o(fmt("const int ri = %s;", comp("c", E).c_str()));
    o(fmt("const float4* f = kx_f%d + %d * r;", (int)ci, NF));
    o("const float4 f0 = f[0], f1 = f[1];");
    o("kx_df av = kx_mk(0.0f, 0.0f), dh = kx_mk(0.0f, 0.0f);   // sum_k nu_k v_k, sum_k nu_k H_k/RT");
    for (int j = 0; j < E; ++j)
      o(fmt("{ const unsigned cj = (unsigned)%s & 0xffff0000u; if (cj != 0u) { const float4 w = vh[k%d]; const float cf = __uint_as_float(cj); "
            "av = kx_df_add_u(av, kx_df_mulf(kx_mk(w.x, w.y), cf)); dh = kx_df_add_u(dh, kx_df_mulf(kx_mk(w.z, w.w), cf)); } }",
            comp("c", j).c_str(), j));
    o("const kx_df lA = kx_mk(f0.x, f0.y), bA = kx_mk(f0.z, f0.w), nEA = kx_mk(f1.x, f1.y);");
    o("kx_df lk = kx_df_fma(bA, lnT, kx_df_fma(nEA, iT, lA));");
    o("kx_df dT = kx_df_mul(iT, kx_df_fma(kx_df_neg(nEA), iT, bA));");
    c.fp32 += NC * (2 * kDfFma + kDfMul + kDfFma) + NC * E * (kDfAdd + kDfMulf);
    std::string aq = "av";
    if (tb) {
      o(fmt("const int2 e = kx_e%d[r];", (int)ci));
      o("const float4 f2 = f[2];");
      o("kx_df X;");
      o("if (e.y < 0) {");
      o("  const int kc = kx_effd[e.x].k;");
      o("  X = kx_df_mul(kx_mk(yv[kc].x, yv[kc].y), fC);");
      o("} else {");
      o("  kx_df t = kx_mk(0.0f, 0.0f);");
      o("  for (int j = 0; j < e.y; ++j) {");
      o("    const kx_effd_t q = kx_effd[e.x + j];");
      o("    t = kx_df_fma(kx_mk(q.ahi, q.alo), kx_mk(yv[q.k].x, yv[q.k].y), t);");
      o("  }");
      o("  X = kx_df_fma(kx_mk(f2.x, f2.y), cM, kx_df_mul(fC, t));");
      o("}");
      c.fp32 += NC * (kDfFma + kDfMul + 3 * kDfFma);
    }
    if (d.kind == Kind::ThreeBody) { o("const kx_df aq = kx_df_mul(av, X);"); aq = "aq"; c.fp32 += NC * kDfMul; }
    if (fo) {
      o("const float4 f3 = f[3], f4 = f[4], f5 = f[5], f6 = f[6];");
      o("const kx_df b0 = kx_mk(f3.x, f3.y), nE0 = kx_mk(f3.z, f3.w);");
      o("const kx_df lk0 = kx_df_fma(b0, lnT, kx_df_fma(nE0, iT, kx_mk(f2.z, f2.w)));");
      o("const kx_df dk0 = kx_df_mul(iT, kx_df_fma(kx_df_neg(nE0), iT, b0));");
      o("kx_df lnPr = kx_df_add(kx_df_sub(lk0, lk), kx_df_log(X));");
      o("if (!(lnPr.hi > -690.775528f)) lnPr = kx_mk(-690.775528f, 0.0f);");
      o("const bool small = lnPr.hi < 0.0f;");
      o("const kx_df ee = kx_df_exp_n(small ? lnPr : kx_df_neg(lnPr));");
      o("const kx_df i1e = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_add(kx_mk(1.0f, 0.0f), ee));");
      o("const kx_df e1e = kx_df_mul(ee, i1e);");
      o("const kx_df P1 = small ? e1e : i1e, P0 = small ? i1e : e1e;");
      o("const kx_df l1p = kx_df_log1p(ee);");
      o("kx_df lnF = kx_mk(0.0f, 0.0f), dFl = kx_mk(0.0f, 0.0f), dFT = kx_mk(0.0f, 0.0f);");
      if (d.blend == Blend::Troe) {
        o("{");
        o("  const kx_df p0 = kx_mk(f4.x, f4.y), p1 = kx_mk(f4.z, f4.w), p2 = kx_mk(f5.x, f5.y), p3 = kx_mk(f5.z, f5.w), p4 = kx_mk(f6.x, f6.y);");
        o("  const kx_df e3 = kx_df_mul(p0, kx_df_exp_s(kx_df_mul(Td, p2)));");
        o("  const kx_df e1 = kx_df_mul(p1, kx_df_exp_s(kx_df_mul(Td, p3)));");
        o("  const kx_df e2 = kx_df_exp_s(kx_df_mul(p4, iT));");
        o("  const kx_df Fc = kx_df_add(kx_df_add(e3, e1), e2);");
        o("  const kx_df dFc = kx_df_fma(e3, p2, kx_df_fma(e1, p3, kx_df_neg(kx_df_mul(kx_df_mul(e2, p4), iT2))));");
        o(fmt("  const kx_df lFc = kx_df_mul(kx_df_log(Fc), %s);", il10.c_str()));
        o(fmt("  const kx_df xx = kx_df_fma(lnPr, %s, kx_df_fma(%s, lFc, %s));", il10.c_str(), DFc(-0.67).c_str(), DFc(-0.4).c_str()));
        o(fmt("  const kx_df nn = kx_df_fma(%s, lFc, %s);", DFc(-1.27).c_str(), DFc(0.75).c_str()));
        o(fmt("  const kx_df den = kx_df_fma(%s, xx, nn);", DFc(-0.14).c_str()));
        o("  const kx_df iden = kx_df_div(kx_mk(1.0f, 0.0f), den);");
        o("  const kx_df ff = kx_df_mul(xx, iden);");
        o("  const kx_df g1 = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_fma(ff, ff, kx_mk(1.0f, 0.0f)));");
        o(fmt("  lnF = kx_df_mul(kx_df_mul(%s, lFc), g1);", DFc(std::log(10.0)).c_str()));
        o("  const kx_df h2 = kx_df_mul(kx_df_mul(kx_df_mul(kx_mk(-2.0f, 0.0f), ff), kx_df_mul(g1, g1)), lFc);");
        o("  const kx_df id2 = kx_df_mul(iden, iden);");
        o("  dFl = kx_df_mul(kx_df_mul(h2, nn), id2);");
        o(fmt("  dFT = kx_df_mul(kx_df_fma(kx_df_mul(h2, kx_df_fma(%s, den, kx_df_mul(%s, xx))), id2, g1), kx_df_div(dFc, Fc));",
              DFc(-0.67).c_str(), DFc(1.27 - 0.14 * 0.67).c_str()));
        o("}");
        c.fp32 += NC * (3 * (kDfMul + kDfExp) + 2 * kDfMul + 2 * kDfAdd + 3 * kDfFma + kDfLog + kDfMul + 4 * kDfFma + 3 * kDfDiv + 12 * kDfMul);
      } else if (d.blend == Blend::Sri) {
        o("{");
        o("  const kx_df pa = kx_mk(f4.x, f4.y), pnb = kx_mk(f4.z, f4.w), pnc = kx_mk(f5.x, f5.y), pld = kx_mk(f5.z, f5.w), pe = kx_mk(f6.x, f6.y);");
        o(fmt("  const kx_df lPr = kx_df_mul(lnPr, %s);", il10.c_str()));
        o("  const kx_df Xs = kx_df_div(kx_mk(1.0f, 0.0f), kx_df_fma(lPr, lPr, kx_mk(1.0f, 0.0f)));");
        o("  const kx_df ea = kx_df_mul(pa, kx_df_exp_s(kx_df_mul(pnb, iT)));");
        o("  const kx_df eb = kx_df_exp_s(kx_df_mul(Td, pnc));");
        o("  const kx_df base = kx_df_add(ea, eb);");
        o("  const kx_df lnb = kx_df_log(base);");
        o("  lnF = kx_df_add(pld, kx_df_fma(pe, lnT, kx_df_mul(Xs, lnb)));");
        o(fmt("  dFl = kx_df_mul(kx_df_mul(kx_df_mul(kx_mk(-2.0f, 0.0f), lPr), kx_df_mul(Xs, Xs)), kx_df_mul(lnb, %s));", il10.c_str()));
        o("  dFT = kx_df_fma(pe, iT, kx_df_mul(Xs, kx_df_div(kx_df_fma(kx_df_neg(kx_df_mul(ea, pnb)), iT2, kx_df_mul(eb, pnc)), base)));");
        o("}");
        c.fp32 += NC * (2 * (kDfMul + kDfExp) + 14 * kDfMul + 3 * kDfDiv + kDfLog + 4 * kDfFma + 2 * kDfAdd);
      }
      if (d.kind == Kind::Falloff) {
        o("lk = kx_df_add(lk, kx_df_add(small ? kx_df_sub(lnPr, l1p) : kx_df_neg(l1p), lnF));");
        o("const kx_df dP = kx_df_add(P0, dFl);");
        o("dT = kx_df_add(kx_df_fma(kx_df_sub(dk0, dT), dP, dT), dFT);");
      } else {
        o("lk = kx_df_add(lk0, kx_df_sub(lnF, small ? l1p : kx_df_add(lnPr, l1p)));");
        o("const kx_df dP = kx_df_sub(dFl, P1);");
        o("dT = kx_df_add(kx_df_fma(kx_df_sub(dk0, dT), dP, dk0), dFT);");
      }
      o("const kx_df dX = kx_df_div(dP, X);");
      c.fp32 += NC * (2 * kDfFma + kDfMul + kDfAdd + kDfLog + kDfExp + 2 * kDfDiv + kDfMul + kDfLog + 6 * kDfAdd + kDfFma);
    } else if (d.kind == Kind::Plog) {
      o(fmt("const int2 e = kx_e%d[r];", (int)ci));
      o("const float* t = kx_plogf + 8 * e.x; const long long* tp = kx_plogp + e.x; const int np = e.y;");
      o("const long long Pb = __double_as_longlong(P);");
      o("#define KX_PLK(u) kx_df_fma(KX_PF((u) + 4), lnT, kx_df_fma(KX_PF((u) + 6), iT, KX_PF((u) + 2)))");
      o("#define KX_PLD(u) kx_df_mul(iT, kx_df_fma(kx_df_neg(KX_PF((u) + 6)), iT, KX_PF((u) + 4)))");
      o("if (Pb <= tp[0]) { lk = KX_PLK(t); dT = KX_PLD(t); }");
      o("else if (Pb >= tp[np - 1]) { const float* u = t + 8 * (np - 1); lk = KX_PLK(u); dT = KX_PLD(u); }");
      o("else {");
      o("  int j = 0; while (!(Pb < tp[j + 1])) ++j;");
      o("  const float* u = t + 8 * j;");
      o("  const kx_df w = kx_df_div(kx_df_sub(lnP, KX_PF(u)), kx_df_sub(KX_PF(u + 8), KX_PF(u)));");
      o("  const kx_df l1 = KX_PLK(u), l2 = KX_PLK(u + 8), d1 = KX_PLD(u), d2 = KX_PLD(u + 8);");
      o("  lk = kx_df_fma(kx_df_sub(l2, l1), w, l1);");
      o("  dT = kx_df_fma(kx_df_sub(d2, d1), w, d1);");
      o("}");
      o("#undef KX_PLK");
      o("#undef KX_PLD");
      c.fp32 += NC * (8 * kDfFma + 4 * kDfMul + 5 * kDfAdd + kDfDiv);
    }
    o("kx_df lf = lk;");
    for (int j = 0; j < d.nre; ++j) o(fmt("lf = kx_df_add_u(lf, kx_mk(v%d.x, v%d.y));", j, j));
    std::string sfx = "0", srx = "0";
    for (int j = 0; j < d.nre; ++j) sfx += fmt(" ^ KX_NEG(k%d)", j);
    for (int j = d.nre; j < E; ++j) srx += fmt(" ^ KX_NEG(k%d)", j);
    o("const int sf = " + sfx + ";");
    // R_f = mfs 2^ef (signed); for reversible reactions R_r = mr 2^er (signed), and R_f - R_r and the
    // temperature term from the two by aligned subtraction (two exponentials per reaction)
    o("int ef;");
    o(fmt("kx_df mf = kx_df_exp_m(lf.hi <= -740.0f ? kx_df_add(lf, %s) : lf, ef);", shift.c_str()));
    o("if (lf.hi <= -740.0f) ef -= 2016;");
    o("const kx_df mfs = sf ? kx_df_neg(mf) : mf;");
    o(fmt("const kx_df af = kx_df_mul_u(%s, mfs);", aq.c_str()));
    o("kx_df ar = kx_mk(0.0f, 0.0f);");
    o("int er = -100000;");
    o("int eq = ef;");
    o("kx_df mq = mfs;   // R_f - R_r = mq 2^eq");
    c.fp32 += NC * (kDfExp + kDfMul + 10);
    if (d.rev) {
      o("const int sr = " + srx + ";");
      std::string first = d.nre > 0 ? "kx_df_neg(kx_mk(v0.z, v0.w))" : "kx_mk(v0.z, v0.w)";
      o("kx_df dl = " + first + ";");
      for (int j = 1; j < E; ++j)
        o(fmt("dl = kx_df_add_u(dl, kx_mk(%sv%d.z, %sv%d.w));", j < d.nre ? "-" : "", j, j < d.nre ? "-" : "", j));
      o("dl = kx_df_add_u(dl, kx_df_mulf(lnPRT, f1.w));   // -dn ln(p_atm/RT), dn of this reaction");
      o("const kx_df lr = kx_df_add_u(lf, dl);");
      o(fmt("kx_df mr = kx_df_exp_m(lr.hi <= -740.0f ? kx_df_add(lr, %s) : lr, er);", shift.c_str()));
      o("if (lr.hi <= -740.0f) er -= 2016;");
      o("if (sr) mr = kx_df_neg(mr);");
      o("// d/dT at fixed C: a c (R_f dT - R_r (dT - (sum_k nu_k H_k/RT - dn)/T)) (Gibbs-Helmholtz for the second part)");
      o("{ int et; const kx_df t = kx_df_sub_m(kx_df_mul_u(mfs, dT), ef, "
        "kx_df_mul_u(mr, kx_df_sub(dT, kx_df_mul(iT, kx_df_add(dh, kx_mk(f1.w, 0.0f))))), er, et);");
      o(fmt("  kx_acc_add(gTa, sT, kx_df_mul_u(%s, t), et); }", aq.c_str()));
      if (tb) o("mq = kx_df_sub_m(mfs, ef, mr, er, eq);");
      o(fmt("ar = kx_df_mul_u(kx_df_neg(%s), mr);", aq.c_str()));
      c.fp32 += NC * ((E - 1) * kDfAdd + kDfAdd + kDfMulf + kDfExp + 10 + 5 * kDfMul + 3 * kDfAdd + 8 + 20);
      if (tb) c.fp32 += NC * (kDfAdd + 8);
    } else {
      o(fmt("kx_acc_add(gTa, sT, kx_df_mul_u(kx_df_mul_u(%s, dT), mfs), ef);", aq.c_str()));
      c.fp32 += NC * (2 * kDfMul + 20);
    }
    if (tb) {
      o(d.kind == Kind::ThreeBody ? "const kx_df gX = kx_df_mul_u(av, mq);" : "const kx_df gX = kx_df_mul_u(kx_df_mul_u(av, mq), dX);");
      o("if (e.y >= 0) kx_acc_add(gMa, sM, kx_df_mul_u(kx_mk(f2.x, f2.y), gX), eq);");
      o(fmt("rt[%d + r] = make_float4(gX.hi, gX.lo, __int_as_float(eq), 0.0f);", tbbase[ci]));
      c.fp32 += NC * (3 * kDfMul + 20);
    }
    o("rf[ri] = make_float4(af.hi, af.lo, ar.hi, ar.lo);");
    o("re[ri] = make_int2(ef, er);");
    --o.ind;
    o("}");
  }
  o("#undef KX_NEG");
  --o.ind;
  o("}");
  o("__syncwarp();");
  // ---- 4. gather of d/dC_k
  o("{");
  ++o.ind;
  o("float4* const slot = sv;   // sv and vh are free now");
  o("int sl = kx_vchs[lane];");
  o("kx_df acc = kx_mk(0.0f, 0.0f);");
  o("int as = -100000;");
  o("#pragma unroll 2");
  o(fmt("for (int j = 0; j < %d; ++j) {", CL));
  o(fmt("  const int wv = kx_vtab[%d * j + lane].w;", NCH));
  o(fmt("  const float cf = kx_vtab[%d * j + lane].c, cl = kx_vtab[%d * j + lane].cl;", NCH, NCH));
  o("  if (cf != 0.0f) {");
  o("    const int r = wv & 0x3fff, kind = (wv >> 14) & 3, k = (wv >> 16) & 0x7fff;");
  o("    kx_df mt;");
  o("    int et;");
  o("    if (kind == 2) { const float4 gx = rt[r]; mt = kx_df_mul_u(kx_mk(gx.x, gx.y), kx_mk(cf, cl)); et = __float_as_int(gx.z); }");
  o("    else {");
  o("      const float4 q = rf[r], iq = ic[k];");
  o("      mt = kx_df_mul_u(kind == 0 ? kx_mk(q.x, q.y) : kx_mk(q.z, q.w), kx_mk(iq.x, iq.y));");
  o("      et = (kind == 0 ? re[r].x : re[r].y) + __float_as_int(iq.z);");
  o("      mt = kx_df_mulf(mt, cf);   // an integer stoichiometric coefficient");
  o("    }");
  o("    kx_acc_add(acc, as, mt, et);");
  o("  }");
  o("  if (wv < 0) { slot[sl++] = make_float4(acc.hi, acc.lo, __int_as_float(as), 0.0f); acc = kx_mk(0.0f, 0.0f); as = -100000; }");
  o("}");
  --o.ind;
  o("}");
  o("__syncwarp();");
  c.fp32 += (double)NE * (kDfMul + kDfMulf + 20);
  // ---- 5. the chain to (T, Y) in float64
  o("const int flag = *scf;");
  o("const float4 F2 = sc4[2], F1 = sc4[1];");
  o("const double cMd = kx_df2d(kx_mk(F2.x, F2.y)), fCd = kx_df2d(kx_mk(F2.z, F2.w));");
  o("const double iTd = 1.0 / __hiloint2double(__float_as_int(sc4[4].y), __float_as_int(sc4[4].x));");
  o(fmt("double gck[%d];", NT));
  o("double gCX = 0.0;");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o("  const int k = lane + 32 * t;");
  o("  gck[t] = 0.0;");
  o(fmt("  if (k < %d) {", ns));
  o("    const int2 s = kx_vslot[k];");
  o("    kx_df a = kx_mk(0.0f, 0.0f);");
  o("    int sa = -100000;");
  o("    for (int j = 0; j < s.y; ++j) { const float4 q = sv[s.x + j]; kx_acc_add(a, sa, kx_mk(q.x, q.y), __float_as_int(q.z)); }");
  o("    gck[t] = kx_df2d_s(a, sa);");
  o("    gCX = fma(gck[t], fCd * kx_df2d(kx_mk(yv[k].x, yv[k].y)), gCX);");
  o("  }");
  o("}");
  o("double gT = kx_df2d_s(gTa, sT), gM = kx_df2d_s(gMa, sM);");
  for (int off = 1; off < 32; off *= 2) {
    o(fmt("gCX += __shfl_xor_sync(0xffffffffu, gCX, %d);", off));
    o(fmt("gT += __shfl_xor_sync(0xffffffffu, gT, %d);", off));
    o(fmt("gM += __shfl_xor_sync(0xffffffffu, gM, %d);", off));
  }
  o("gCX = __shfl_sync(0xffffffffu, gCX, 0); gT = __shfl_sync(0xffffffffu, gT, 0); gM = __shfl_sync(0xffffffffu, gM, 0);");
  o("gM += gCX / cMd;");
  o("const double gavg = gCX / cMd;");
  o("if (lane == 0) gT_[i] = flag ? KX_NAN : fma(-gM * cMd, iTd, gT);");
  o("#pragma unroll");
  o(fmt("for (int t = 0; t < %d; ++t) {", NT));
  o("  const int k = lane + 32 * t;");
  o(fmt("  if (k < %d) gY_[(long long)k * ld + i] = flag ? KX_NAN : fCd * (gck[t] - gavg) * kx_iwd[k];", ns));
  o("}");
  o("if (lane == 0 && flag) atomicMin(&kx_bad_first, (unsigned long long)i);");
  o("__syncwarp();");
  --o.ind;
  o("}");
  c.fp64 += ns * 6 + 12;
  return o.o.str();
}

}  // namespace

// Shared memory per thread of the transport kernels, in bytes.
int transport_smem_per_thread(const Mechanism& m, bool mixed, int part, int layout) {
  // diffusion: X and S; viscosity: X, X/u, X/u^2 (float32) or X and 1/u (float64 accuracy);
  // layout 2 keeps X in local memory
  if (layout == 3) return 0;
  return (((part == 2 || !mixed) ? 2 : 3) - (layout == 2 ? 1 : 0)) * m.ns * (mixed ? 4 : 8);
}

// ------------------------------------------------------------------ kernels
bool wdot_is_wc(const Mechanism& m, KernelKind kind, const EmitOptions& opt) {
  (void)m;
  return kind == KernelKind::Wdot && !opt.mixed && !opt.scratch && opt.rates_arith != 1 && opt.rates_layout == 2;
}

WcShape wdot_wc_shape(const Mechanism& m, const EmitOptions& opt) {
  const WcLayout L = wc_layout_of(m, opt.rates_group, opt.block);
  WcShape w;
  w.states_per_warp = L.G;
  w.states_per_block = L.G * L.warps;
  w.smem_per_block = L.warp_bytes * L.warps;
  // lane use of the merged classes: one class per (kind, reversibility, blend)
  std::map<std::tuple<int, bool, int>, int> count;
  for (auto& r : m.rx)
    ++count[std::make_tuple((int)r.kind, r.reversible,
                            (r.kind == Kind::Falloff || r.kind == Kind::ChemAct) ? (int)r.blend : (int)Blend::Lindemann)];
  double pairs = 0, slots = 0;
  for (auto& kv : count) {
    pairs += (double)L.G * kv.second;
    slots += 32.0 * std::ceil(L.G * kv.second / 32.0);
  }
  w.lane_use = slots > 0 ? pairs / slots : 1.0;
  return w;
}

// The warp-cooperative production-rate kernel (emit_wdot_wc) with its own
// grid-stride loop over groups of states.
std::string emit_wc_kernel(const Mechanism& m, const EmitOptions& opt, const std::string& entry, OpCounts* counts) {
  OpCounts c;
  Out globals;
  globals.ind = 0;
  const std::string body = emit_wdot_wc(m, opt, entry, c, globals);
  if (body.empty()) return "";
  std::ostringstream s;
  s << "// mechanism " << m.name << ": " << m.ns << " species, " << m.nr() << " reactions\n";
  s << "#define P_ATM_R " << D(P_ATM / R_U) << "\n";
  s << "#define KX_T64 0\n#define KX_TDF 1\n#define KX_TDFR 1\n";
  s << kTables << "\n" << kDevicePrelude << "\n";
  s << "extern __shared__ __align__(16) unsigned char kx_dyn[];\n";
  s << globals.o.str();
  s << "__device__ unsigned long long kx_bad_first = 0xffffffffffffffffull;\n";
  // 80 registers by default: six blocks of 128 threads per SM (measured on 53/325 with one state per
  // warp: 64 / 80 / 96 registers -> 8.97 / 8.74 / 8.93 ms per 2^20 states)
  const int rreg = opt.maxrreg > 0 ? opt.maxrreg : 80;
  const int min_blocks = std::max(1, 65536 / (rreg * opt.block));
  s << "extern \"C\" __global__ void __launch_bounds__(" << opt.block << ", " << min_blocks << ") " << entry
    << "(const double* __restrict__ T_, const double* __restrict__ P_, const double* __restrict__ Y_, long long ld, "
    << "double* __restrict__ out_, long long n)\n{\n";
  s << "  kx_load_tables();\n";
  s << body;
  s << "}\n";
  if (counts) *counts = c;
  return s.str();
}

bool vjp_is_wc(const Mechanism& m, KernelKind kind, const EmitOptions& opt) {
  (void)m;
  return kind == KernelKind::Vjp && opt.rates_arith != 1 && opt.vjp_layout == 2;
}

int vjp_wc_smem(const Mechanism& m, const EmitOptions& opt) { return vjp_wc_layout(m).warp_bytes * (opt.block / 32); }

// The warp-cooperative adjoint (emit_vjp_wc) with its own grid-stride loop over states.
std::string emit_vjp_wc_kernel(const Mechanism& m, const EmitOptions& opt, const std::string& entry, OpCounts* counts) {
  OpCounts c;
  Out globals;
  globals.ind = 0;
  const std::string body = emit_vjp_wc(m, opt, c, globals);
  if (body.empty()) return "";
  std::ostringstream s;
  s << "// mechanism " << m.name << ": " << m.ns << " species, " << m.nr() << " reactions\n";
  s << "#define P_ATM_R " << D(P_ATM / R_U) << "\n";
  s << "#define KX_T64 0\n#define KX_TDF 1\n#define KX_TDFR 1\n";
  s << kTables << "\n" << kDevicePrelude << "\n" << kAdjointPrelude << "\n";
  s << "extern __shared__ __align__(16) unsigned char kx_dyn[];\n";
  s << globals.o.str();
  s << "__device__ unsigned long long kx_bad_first = 0xffffffffffffffffull;\n";
  const int rreg = opt.maxrreg > 0 ? opt.maxrreg : 128;
  const int min_blocks = std::max(1, 65536 / (rreg * opt.block));
  s << "extern \"C\" __global__ void __launch_bounds__(" << opt.block << ", " << min_blocks << ") " << entry
    << "(const double* __restrict__ T_, const double* __restrict__ P_, const double* __restrict__ Y_, long long ld, "
    << "const double* __restrict__ V_, double* __restrict__ gT_, double* __restrict__ gY_, long long n)\n{\n";
  s << "  kx_load_tables();\n";
  s << body;
  s << "}\n";
  if (counts) *counts = c;
  return s.str();
}

std::string emit_kernel(const Mechanism& m, KernelKind kind, const EmitOptions& opt, const std::string& entry,
                        OpCounts* counts) {
  if (vjp_is_wc(m, kind, opt)) return emit_vjp_wc_kernel(m, opt, entry, counts);
  OpCounts c;
  Out body, globals;
  body.ind = 2;
  globals.ind = 0;
  std::string outs, nan_fill;
  switch (kind) {
    case KernelKind::Wdot:
    case KernelKind::Rop: {
      const bool rop = kind == KernelKind::Rop;
      if (wdot_is_wc(m, kind, opt)) return emit_wc_kernel(m, opt, entry, counts);
      outs = "double* __restrict__ out_";
      if (opt.scratch && !rop) outs += ", unsigned char* __restrict__ kx_scr, long long nthr";
      nan_fill = fmt("for (int k = 0; k < %d; ++k) out_[(long long)k * ld + i] = KX_NAN;", rop ? m.nr() : m.ns);
      const bool table = opt.rates_mode == 2 || (opt.rates_mode == 0 && (m.ns > 64 || m.nr() > 400));
      if ((!opt.mixed && (opt.rates_arith != 1 || opt.scratch)) || (opt.mixed && opt.rates_mode == 0))
        emit_rates_class_df(body, globals, m, opt, rop, c);
      else if (table && opt.mixed) emit_rates_table_mixed(body, globals, m, rop, c);
      else if (table) emit_rates_table64(body, globals, m, rop, c);
      else if (opt.mixed) emit_rates_mixed(body, m, rop, c);
      else emit_rates64(body, m, opt, rop, c);
      break;
    }
    case KernelKind::Thermo:
      outs = "double* __restrict__ out0_, double* __restrict__ out1_";
      nan_fill = "out0_[i] = KX_NAN; out1_[i] = KX_NAN;";
      emit_thermo(body, m, c);
      break;
    case KernelKind::Transport:
      outs = "double* __restrict__ out0_, double* __restrict__ out1_, double* __restrict__ out2_";
      // each half writes only its own outputs (the other pointers are null)
      if (opt.part == 1) nan_fill = "out0_[i] = KX_NAN; out1_[i] = KX_NAN;";
      else if (opt.part == 2) nan_fill = fmt("for (int k = 0; k < %d; ++k) out2_[(long long)k * ld + i] = KX_NAN;", m.ns);
      else nan_fill = fmt("out0_[i] = KX_NAN; out1_[i] = KX_NAN; for (int k = 0; k < %d; ++k) out2_[(long long)k * ld + i] = KX_NAN;", m.ns);
      emit_transport(body, globals, m, opt, c);
      break;
    case KernelKind::Vjp:
      outs = "const double* __restrict__ V_, double* __restrict__ gT_, double* __restrict__ gY_";
      nan_fill = fmt("gT_[i] = KX_NAN; for (int k = 0; k < %d; ++k) gY_[(long long)k * ld + i] = KX_NAN;", m.ns);
      if (opt.rates_arith == 1) emit_vjp64(body, m, c);
      else emit_vjp_df(body, globals, m, c, opt.vjp_form == 0);
      break;
  }
  std::ostringstream s;
  s << "// mechanism " << m.name << ": " << m.ns << " species, " << m.nr() << " reactions\n";
  s << "#define P_ATM_R " << D(P_ATM / R_U) << "\n";
  const bool df_rates = (kind == KernelKind::Wdot || kind == KernelKind::Rop) &&
                        ((!opt.mixed && (opt.rates_arith != 1 || opt.scratch)) || (opt.mixed && opt.rates_mode == 0));
  const bool table_sel = opt.rates_mode == 2 || (opt.rates_mode == 0 && (m.ns > 64 || m.nr() > 400));
  const bool mixed_unrolled = (kind == KernelKind::Wdot || kind == KernelKind::Rop) && opt.mixed && !table_sel && !df_rates;
  const bool vjp_df = kind == KernelKind::Vjp && opt.rates_arith != 1;
  const bool t64 = kind != KernelKind::Thermo && kind != KernelKind::Transport && !df_rates && !mixed_unrolled && !vjp_df;
  // table-driven float64 rate kernels take their exponentials from kx_exp_r (error ~2e-12 against
  // a 1e-10 bar); the unrolled ones keep kx_exp, whose short inline sequence keeps compile time
  // of the straight-line code in check
  const bool table_rates = opt.rates_mode == 2 || (opt.rates_mode == 0 && (m.ns > 64 || m.nr() > 400));
  const bool rates64 = (kind == KernelKind::Wdot || kind == KernelKind::Rop) && !opt.mixed && table_rates && !df_rates;
  const bool tdf = (kind == KernelKind::Transport && !opt.mixed && opt.tr_mode == 0) || rates64 || df_rates || mixed_unrolled || vjp_df ||
                   kind == KernelKind::Thermo;
  s << "#define KX_T64 " << (t64 || (kind == KernelKind::Transport && !opt.mixed && opt.tr_mode == 1)) << "\n";
  s << "#define KX_TDF " << tdf << "\n";
  s << "#define KX_TDFR " << (df_rates || mixed_unrolled || vjp_df || kind == KernelKind::Thermo) << "\n";
  s << kTables << "\n" << kDevicePrelude << "\n";
  if (vjp_df) s << kAdjointPrelude << "\n";
  s << "extern __shared__ __align__(16) unsigned char kx_dyn[];\n";
  s << globals.o.str();
  // the smallest index of a point outside the domain since the host last read and reset it
  s << "__device__ unsigned long long kx_bad_first = 0xffffffffffffffffull;\n";
  nan_fill = "atomicMin(&kx_bad_first, (unsigned long long)i); " + nan_fill;
  s << "#define KX_BAD_POINT { " << nan_fill << " continue; }\n";
  // a register cap is expressed as a minimum number of resident blocks (ptxas
  // ignores --maxrregcount for kernels that carry launch bounds).  Defaults,
  // measured on the 53/325 mechanism (2^20 states): the unrolled native
  // float64 rate kernel runs best at 128 registers and the mixed ones at 96
  // (more resident warps hide instruction fetch, table and dependence
  // latency better than the spills they cost); the float-pair rate kernel at
  // 128 (four blocks: its pipelined loops keep two reactions' operands live);
  // the transport kernels with their vectors in local memory at 64 (eight
  // blocks of 128: residency is what hides the local-memory latency), except
  // the float-pair viscosity kernel with Wilke's pairs evaluated once per
  // unordered pair at 80 (six blocks: its row and column sums hold more live
  // values; 4.49 against 5.10 ms at 64 on 2^20 states); with shared-memory
  // columns at 128; thermo at 48.
  int rreg = opt.maxrreg;
  const bool unrolled_rates = (kind == KernelKind::Wdot || kind == KernelKind::Rop) && !df_rates &&
                              !(opt.rates_mode == 2 || (opt.rates_mode == 0 && (m.ns > 64 || m.nr() > 400)));
  if (rreg == 0 && unrolled_rates) rreg = opt.mixed ? 96 : 128;
  if (rreg == 0 && df_rates) rreg = opt.mixed ? 72 : 128;
  if (rreg == 0 && kind == KernelKind::Transport)
    rreg = opt.tr_layout != 3 ? 128 : (!opt.mixed && opt.tr_mode == 0 && opt.part == 1 && opt.diff_mode != 2) ? 80 : 64;
  if (rreg == 0 && kind == KernelKind::Thermo) rreg = 48;
  // the double-float adjoint is bound by the latency of its local-memory vectors: residency wins
  // (53/325, 2^18 states: 64 / 80 / 96 / 123 registers -> 6.26 / 7.16 / 7.33 / 8.58 ms)
  if (rreg == 0 && vjp_df) rreg = 64;
  const int min_blocks = rreg > 0 ? std::max(1, 65536 / (rreg * opt.block)) : 0;
  s << "extern \"C\" __global__ void __launch_bounds__(" << opt.block;
  if (min_blocks > 0) s << ", " << min_blocks;
  s << ") " << entry
    << "(const double* __restrict__ T_, const double* __restrict__ P_, const double* __restrict__ Y_, long long ld, "
    << outs << ", long long n)\n{\n";
  std::string text = body.o.str();
  if (rates64) {
    for (size_t at = text.find("kx_exp("); at != std::string::npos; at = text.find("kx_exp(", at + 8)) text.replace(at, 7, "kx_exp_r(");
  }
  s << "  kx_load_tables();\n";
  s << "  for (long long i = (long long)blockIdx.x * " << opt.block << " + threadIdx.x; i < n; i += (long long)gridDim.x * "
    << opt.block << ") {\n";
  s << "    const double T = T_[i], P = P_[i];\n";
  s << "    if (!(T > 0.0 && P > 0.0 && T < KX_INF && P < KX_INF)) { " << nan_fill << " continue; }\n";
  s << text;
  s << "  }\n}\n";
  if (counts) *counts = c;
  return s.str();
}

}  // namespace kx
