// Helix propagation and Kalman update of the 5-parameter track state
// (y, z, sin phi, dz/ds_T, q/pT) in a uniform Bz field (Sec. 2, Fig. 1c).
//
// The state is binary32 with z kept relative to a per-track reference (the
// seed cluster's z) so that drift-time coordinates of ~2.5e4 cm keep their
// resolution.  The covariance is a packed lower triangle; it is held in FP64
// for the first `fp64_updates` updates after every (re)seed (a few more while
// it is still converging in the passes whose covariance is an output,
// zone_update), where the seed covariance is large and the subtraction
// C -= G C[0:2,:] cancels, and in FP32 afterwards.  chi2 is accumulated in
// FP64.
#pragma once
#include "common.cuh"

namespace tpc {

// packed index of (i, j), i >= j
#define TPC_CI(i, j) ((i) * ((i) + 1) / 2 + (j))

enum : uint32_t {
  TF_TIE = TPC_TF_TAINT_TIE,
  TF_GATE = TPC_TF_TAINT_GATE,
  TF_EDGE = TPC_TF_TAINT_EDGE,
  TF_SLIM = TPC_TF_TAINT_SLIM,
  TF_SEED_FAIL = TPC_TF_SEED_FAIL,
  TF_BACK_FAIL = TPC_TF_BACK_FAIL,
  TF_REFIT_FAIL = TPC_TF_REFIT_FAIL
};

// y, z and sin phi are accumulated over up to ~300 row steps; each is kept as
// an unevaluated sum hi + lo of two binary32 numbers (TwoSum, Knuth, TAOCP
// vol. 2, 4.2.2) so that the position does not drift by ulp(y) per step.
struct TrkState {
  float x;   // row radius
  int row;
  float y, z, s, t, q;  // z relative to zref
  float yl, zl, sl;     // low parts of y, z, s
  float zref;
};

// hi + lo += d, the rounding error of the new sum kept in lo.
__device__ __forceinline__ void acc2(float& hi, float& lo, float d) {
  const float b = __fadd_rn(lo, d);
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
}

// Square root and reciprocal of the binary32 Kalman arithmetic: the hardware
// approximations (relative error about 1e-7, three orders below the parity
// tolerances, and shorter dependency chains than the IEEE-rounded forms that
// the grid and link stages keep).  ksqrt needs v > 0.
__device__ __forceinline__ float ksqrt(float v) { return v * rsqrtf(v); }
__device__ __forceinline__ float kinv(float v) { return __fdividef(1.0f, v); }

// Conversions between binary32 and binary64 done with integer operations on
// the IEEE 754 encodings (sign, biased exponent, fraction; binary32 bias 127,
// binary64 bias 1023).  The FP64 zone is bound by the FP64 pipe (1/64 of the
// FP32 rate on this part), which also executes the hardware conversions;
// these sequences run on the integer pipes instead and give the same results
// for zero, normal numbers, infinities and NaNs (binary32 subnormals, which the
// zone's values never are, become zero).
// Widening is exact: the 23 fraction bits move to the top of the 52.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = u & 0x7F800000u;
  const uint32_t mag = (u & 0x7FFFFFFFu) >> 3;  // exponent and the top 20 fraction bits, one word lower
  const uint32_t hi_e = e == 0x7F800000u ? (mag | 0x7FF00000u) : mag + (896u << 20);  // rebias by 1023 - 127
  const uint32_t hi = (u & 0x80000000u) | (e == 0u ? 0u : hi_e);
  const uint32_t lo = e == 0u ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}
// Narrowing rounds to nearest, ties to even: the top 23 of the 52 fraction
// bits are kept and the 29 discarded ones decide the increment, which may
// carry into the exponent (up to infinity, as IEEE 754 overflow does).
__device__ __forceinline__ float narrow(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  uint32_t r = ((uint32_t)(e - 896) << 23) + (((hi & 0x000FFFFFu) << 3) | (lo >> 29));
  const uint32_t rest = lo & 0x1FFFFFFFu;
  r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;
  if (e == 0x7FF) r = ((hi & 0x000FFFFFu) | lo) ? 0x7FC00000u : 0x7F800000u;  // NaN, infinity
  else if (e - 896 > 254) r = 0x7F800000u;                                        // overflow
  else if (e - 896 < 1) r = 0u;                                                   // below the normal range
  return __uint_as_float(sign | r);
}

// C <- J C J^T for the sparse first-order Jacobian of one propagation step:
// J = I except J[y,s] = j02, J[y,q] = kap j02, J[z,s] = j12, J[z,t] = j13,
// J[z,q] = kap j12 and J[s,q] = 2 kap, with kap = -K dx / 2 (prop_state).
// Every row of J takes columns s and q of C in the combination
// u = C[s,:] + kap C[q,:], so forming u once brings the transport from 51
// multiply-adds to 42.
template <typename T>
__device__ __forceinline__ void cov_transport(T* C, T j02, T j12, T j13, T kap) {
  const T c00 = C[0], c10 = C[1], c11 = C[2], c20 = C[3], c21 = C[4], c22 = C[5], c30 = C[6], c31 = C[7],
          c32 = C[8], c33 = C[9], c40 = C[10], c41 = C[11], c42 = C[12], c43 = C[13], c44 = C[14];
  const T u0 = c20 + kap * c40, u1 = c21 + kap * c41, u2 = c22 + kap * c42, u3 = c32 + kap * c43,
          u4 = c42 + kap * c44;
  // A = J C, rows 0..2 (the columns that C' needs)
  const T a00 = c00 + j02 * u0, a02 = c20 + j02 * u2, a04 = c40 + j02 * u4;
  const T a10 = c10 + j12 * u0 + j13 * c30;
  const T a11 = c11 + j12 * u1 + j13 * c31;
  const T a12 = c21 + j12 * u2 + j13 * c32;
  const T a13 = c31 + j12 * u3 + j13 * c33;
  const T a14 = c41 + j12 * u4 + j13 * c43;
  const T a20 = u0 + kap * c40, a21 = u1 + kap * c41, a22 = u2 + kap * c42, a23 = u3 + kap * c43,
          a24 = u4 + kap * c44;
  // C' = A J^T, lower triangle; v_i = A[i,s] + kap A[i,q]
  const T v0 = a02 + kap * a04, v1 = a12 + kap * a14, v2 = a22 + kap * a24;
  C[0] = a00 + j02 * v0;
  C[1] = a10 + j02 * v1;
  C[2] = a11 + j12 * v1 + j13 * a13;
  C[3] = a20 + j02 * v2;
  C[4] = a21 + j12 * v2 + j13 * a23;
  C[5] = v2 + kap * a24;
  C[6] = c30 + j02 * u3;
  C[7] = c31 + j12 * u3 + j13 * c33;
  C[8] = u3 + kap * c43;
  // C[9] = c33 unchanged
  C[10] = c40 + j02 * u4;
  C[11] = c41 + j12 * u4 + j13 * c43;
  C[12] = u4 + kap * c44;
  // C[13], C[14] unchanged
}

// Residual of a measurement against the compensated state: (m - hi) is exact
// when m and hi are close (Sterbenz), the low parts are then subtracted.
__device__ __forceinline__ float residual_y(const TrkState& p, float my) {
  return __fsub_rn(__fsub_rn(my, p.y), p.yl);
}
// z measurement mz (absolute); mz - zref is split exactly into hi + lo first.
__device__ __forceinline__ float residual_z(const TrkState& p, float mz) {
  const float dh = __fsub_rn(mz, p.zref);
  const float bb = __fsub_rn(dh, mz);
  const float dl = __fsub_rn(__fsub_rn(mz, __fsub_rn(dh, bb)), __fadd_rn(p.zref, bb));
  return __fadd_rn(__fsub_rn(dh, p.z), __fsub_rn(dl, p.zl));
}

// Kalman update with the measurement (my, mz) (mz absolute); returns the
// chi2 increment.
template <typename T>
__device__ __forceinline__ float kalman_update(TrkState& p, T* C, float my, float mz, T V) {
  const float r0 = residual_y(p, my), r1 = residual_z(p, mz);
  const T S00 = C[0] + V, S01 = C[1], S11 = C[2] + V;
  const T idet = kinv(S00 * S11 - S01 * S01);
  const T I00 = S11 * idet, I01 = -S01 * idet, I11 = S00 * idet;
  const T k0[5] = {C[0], C[1], C[3], C[6], C[10]};  // column 0
  const T k1[5] = {C[1], C[2], C[4], C[7], C[11]};  // column 1
  T g0[5], g1[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    g0[i] = k0[i] * I00 + k1[i] * I01;
    g1[i] = k0[i] * I01 + k1[i] * I11;
  }
  // state increments G r in binary32 (the state is binary32; the gain is
  // rounded once), covariance in T
  float f0[5], f1[5];
#pragma unroll
  for (int i = 0; i < 5; i++) {
    f0[i] = (float)g0[i];
    f1[i] = (float)g1[i];
  }
  acc2(p.y, p.yl, f0[0] * r0 + f1[0] * r1);
  acc2(p.z, p.zl, f0[1] * r0 + f1[1] * r1);
  acc2(p.s, p.sl, f0[2] * r0 + f1[2] * r1);
  p.t += f0[3] * r0 + f1[3] * r1;
  p.q += f0[4] * r0 + f1[4] * r1;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) C[TPC_CI(i, j)] -= g0[i] * k0[j] + g1[i] * k1[j];
  // chi2 increment r^T S^-1 r (binary32), accumulated by the caller in FP64
  const float i00 = (float)I00, i01 = (float)I01, i11 = (float)I11;
  return r0 * (i00 * r0 + i01 * r1) + r1 * (i01 * r0 + i11 * r1);
}

// Propagation of the state to row2 at radius x2.  Returns false when
// |sin phi| reaches s_max; otherwise fills the first-order Jacobian:
// J[y,s] = dx / cm^3, J[z,s] = t dx sm / cm^3, J[z,t] = dS and kap = -K dx / 2,
// which gives J[y,q] = kap J[y,s], J[z,q] = kap J[z,s] and J[s,q] = 2 kap
// (sm, cm: sine and cosine of the mean direction).
struct Jac {
  float j02, j12, j13, kap;
};

__device__ __forceinline__ bool prop_state(TrkState& p, int row2, float x2, const KConst& kc, uint32_t& flags,
                                           Jac* J) {
  const float dx = x2 - p.x;  // exact for neighbouring rows (Sterbenz)
  const float kap = -kc.K * p.q;
  const float s1 = p.s, s2 = s1 + kap * dx;
  if (fabsf(fabsf(s1) - kc.s_max) <= 1e-5f || fabsf(fabsf(s2) - kc.s_max) <= 1e-5f) flags |= TF_SLIM;
  if (!(fabsf(s1) < kc.s_max && fabsf(s2) < kc.s_max)) return false;
  const float c1 = ksqrt(1.0f - s1 * s1), c2 = ksqrt(1.0f - s2 * s2);
  const float icc = kinv(c1 + c2);
  const float ss = s1 + s2;
  const float dy = dx * ss * icc;
  // arc length: sin(phi2 - phi1) = kap*dx*g with g = c1 + s1 (s1+s2)/(c1+c2),
  // so dS = dx*g*asin(a)/a, a = kap*dx*g, free of the cancellation of
  // asin(s2) - asin(s1) in binary32; asin(a)/a from its Taylor series
  // 1 + a^2/6 + 3a^4/40 + 5a^6/112 + 35a^8/1152 (+ O(a^10)) for |a| < 0.1
  const float g = c1 + s1 * ss * icc;
  const float a = kap * dx * g;
  float h;
  if (fabsf(a) < 0.1f) {
    const float a2 = a * a;
    h = 1.0f + a2 * (1.0f / 6.0f + a2 * (3.0f / 40.0f + a2 * (5.0f / 112.0f + a2 * (35.0f / 1152.0f))));
  } else {
    h = asinf(a) / a;
  }
  const float dS = dx * g * h;
  if (J) {
    const float sm = 0.5f * ss, cm = ksqrt(1.0f - sm * sm), icm3 = kinv(cm * cm * cm);
    J->j02 = dx * icm3;
    J->j12 = p.t * dx * sm * icm3;
    J->j13 = dS;
    J->kap = -kc.K * dx * 0.5f;
  }
  acc2(p.y, p.yl, dy);
  acc2(p.z, p.zl, p.t * dS);
  acc2(p.s, p.sl, kap * dx);
  p.x = x2;
  p.row = row2;
  return true;
}

// The FP64-zone covariance operations.  Inline: in the zone kernels the
// covariance stays in registers (out of line it went through local memory,
// 5-13% slower); the binary32 kernels instantiate the row steps without the
// zone path, so they do not carry this code.
// The transport of cov_transport written with explicit fused multiply-adds
// (an expression a + b c + d e is fma(d, e, fma(b, c, a))), so that
// cov_transport_d_diag below can be derived from it operation by operation.
__device__ __forceinline__ void cov_transport_d(double* D, const Jac& J) {
  const double j02 = widen(J.j02), j12 = widen(J.j12), j13 = widen(J.j13), kap = widen(J.kap);
  const double c00 = D[0], c10 = D[1], c11 = D[2], c20 = D[3], c21 = D[4], c22 = D[5], c30 = D[6], c31 = D[7],
               c32 = D[8], c33 = D[9], c40 = D[10], c41 = D[11], c42 = D[12], c43 = D[13], c44 = D[14];
  const double u0 = fma(kap, c40, c20), u1 = fma(kap, c41, c21), u2 = fma(kap, c42, c22), u3 = fma(kap, c43, c32),
               u4 = fma(kap, c44, c42);
  const double a00 = fma(j02, u0, c00), a02 = fma(j02, u2, c20), a04 = fma(j02, u4, c40);
  const double a10 = fma(j13, c30, fma(j12, u0, c10));
  const double a11 = fma(j13, c31, fma(j12, u1, c11));
  const double a12 = fma(j13, c32, fma(j12, u2, c21));
  const double a13 = fma(j13, c33, fma(j12, u3, c31));
  const double a14 = fma(j13, c43, fma(j12, u4, c41));
  const double a20 = fma(kap, c40, u0), a21 = fma(kap, c41, u1), a22 = fma(kap, c42, u2), a23 = fma(kap, c43, u3),
               a24 = fma(kap, c44, u4);
  const double v0 = fma(kap, a04, a02), v1 = fma(kap, a14, a12), v2 = fma(kap, a24, a22);
  D[0] = fma(j02, v0, a00);
  D[1] = fma(j02, v1, a10);
  D[2] = fma(j13, a13, fma(j12, v1, a11));
  D[3] = fma(j02, v2, a20);
  D[4] = fma(j13, a23, fma(j12, v2, a21));
  D[5] = fma(kap, a24, v2);
  D[6] = fma(j02, u3, c30);
  D[7] = fma(j13, c33, fma(j12, u3, c31));
  D[8] = fma(kap, c43, u3);
  D[10] = fma(j02, u4, c40);
  D[11] = fma(j13, c43, fma(j12, u4, c41));
  D[12] = fma(kap, c44, u4);
}

// cov_transport_d of a diagonal D (off-diagonal entries +0, diagonal ones
// positive): the first transport after a (re)seed, whose first update leaves
// the seed covariance diagonal.  Every operation of cov_transport_d whose
// result is fixed by the zeros is left out -- b (+0) + x is x for x positive
// or an fma result, and fma(b, +0, +0) is +0 in round to nearest -- and the
// others are the same operations on the same operands, so the result is the
// same to the bit: 17 fused multiply-adds instead of 42.
__device__ __forceinline__ void cov_transport_d_diag(double* D, const Jac& J) {
  const double j02 = widen(J.j02), j12 = widen(J.j12), j13 = widen(J.j13), kap = widen(J.kap);
  const double c00 = D[0], c11 = D[2], c22 = D[5], c33 = D[9], c44 = D[14];
  const double u4 = fma(kap, c44, 0.0);
  const double a02 = fma(j02, c22, 0.0), a04 = fma(j02, u4, 0.0);
  const double a12 = fma(j12, c22, 0.0), a13 = fma(j13, c33, 0.0), a14 = fma(j12, u4, 0.0);
  const double a24 = fma(kap, c44, u4);
  const double v0 = fma(kap, a04, a02), v1 = fma(kap, a14, a12), v2 = fma(kap, a24, c22);
  D[0] = fma(j02, v0, c00);
  D[1] = fma(j02, v1, 0.0);
  D[2] = fma(j13, a13, fma(j12, v1, c11));
  D[3] = fma(j02, v2, 0.0);
  D[4] = fma(j12, v2, 0.0);
  D[5] = fma(kap, a24, v2);
  D[6] = 0.0;
  D[7] = a13;
  D[8] = 0.0;
  D[10] = a04;
  D[11] = a14;
  D[12] = a24;
}

struct UpdOut {
  float d0, d1, d2, d3, d4;  // state increments G r
  float chi2;                // r^T S^-1 r
};

// 1/v in binary64 for positive v in the binary32 normal range: the
// hardware's approximate binary32 reciprocal r of v truncated to binary32
// (relative error a few 2^-23) refined by one third-order step
// r (1 + e + e^2) with e = 1 - v r,
// the first terms of r / (1 - e) = 1/v, which cubes the relative error (to
// about 2^-63), so that the result is within rounding of 1/v: three
// dependent binary64 operations, where two Newton-Raphson steps take four.
__device__ __forceinline__ double krcp(double v) {
  // the seed needs neither rounding nor special cases (v is a positive
  // binary32 normal): v's top 32 significant bits as a binary32 (truncated,
  // exponent rebiased by 1023 - 127 = 896), its approximate reciprocal, and
  // that binary32 widened exactly (fraction to the top of the 52 bits)
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t f = ((hi - (896u << 20)) << 3) | (lo >> 29);
  const uint32_t u = __float_as_uint(kinv(__uint_as_float(f)));
  const double r = __hiloint2double((int)((u >> 3) + (896u << 20)), (int)(u << 29));
  const double e = fma(-v, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Kalman update of the FP64 covariance D for residual (r0, r1).  The
// measurement covariance is V I, so the update with (y, z) equals an update
// with y followed by one with z on the updated covariance (sequential
// processing of uncorrelated measurement components): two rank-one
// downdates with scalar gains, 48 binary64 operations with no 2x2 inverse.
// The binary32 outputs are the state increment w0 r0 + w1 e1, where e1 is
// the z residual after the y step, and the chi2 increment r0^2/s0 + e1^2/s1
// (= r^T S^-1 r).
__device__ __forceinline__ UpdOut kalman_update_d(double* D, float r0, float r1, double V) {
  // y: gain w0 = C[:,y] / s0
  const double s0 = D[0] + V, i0 = krcp(s0);
  const double k0[5] = {D[0], D[1], D[3], D[6], D[10]};
  double w0[5];
#pragma unroll
  for (int i = 0; i < 5; i++) w0[i] = k0[i] * i0;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) D[TPC_CI(i, j)] = fma(-w0[i], k0[j], D[TPC_CI(i, j)]);
  // z on the updated covariance: gain w1 = C'[:,z] / s1
  const double s1 = D[2] + V, i1 = krcp(s1);
  const double k1[5] = {D[1], D[2], D[4], D[7], D[11]};
  double w1[5];
#pragma unroll
  for (int i = 0; i < 5; i++) w1[i] = k1[i] * i1;
#pragma unroll
  for (int i = 0; i < 5; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) D[TPC_CI(i, j)] = fma(-w1[i], k1[j], D[TPC_CI(i, j)]);
  const float e1 = r1 - narrow(w0[1]) * r0;
  UpdOut o;
  o.d0 = narrow(w0[0]) * r0 + narrow(w1[0]) * e1;
  o.d1 = narrow(w0[1]) * r0 + narrow(w1[1]) * e1;
  o.d2 = narrow(w0[2]) * r0 + narrow(w1[2]) * e1;
  o.d3 = narrow(w0[3]) * r0 + narrow(w1[3]) * e1;
  o.d4 = narrow(w0[4]) * r0 + narrow(w1[4]) * e1;
  o.chi2 = r0 * r0 * narrow(i0) + e1 * e1 * narrow(i1);
  return o;
}

// kalman_update_d of a diagonal D (the first update after a (re)seed): the
// y step then changes only C_yy and the z step only C_zz, every other gain
// entry is +0 and every other downdate adds -0 to its entry, which leaves it
// unchanged; the binary32 outputs are the same expressions of the same gains.
// 12 binary64 operations instead of 48, the same result to the bit.
__device__ __forceinline__ UpdOut kalman_update_d_diag(double* D, float r0, float r1, double V) {
  const double s0 = D[0] + V, i0 = krcp(s0);
  const double w00 = D[0] * i0;
  D[0] = fma(-w00, D[0], D[0]);
  const double s1 = D[2] + V, i1 = krcp(s1);
  const double w11 = D[2] * i1;
  D[2] = fma(-w11, D[2], D[2]);
  const double w0[5] = {w00, 0.0, 0.0, 0.0, 0.0}, w1[5] = {0.0, w11, 0.0, 0.0, 0.0};
  const float e1 = r1 - narrow(w0[1]) * r0;
  UpdOut o;
  o.d0 = narrow(w0[0]) * r0 + narrow(w1[0]) * e1;
  o.d1 = narrow(w0[1]) * r0 + narrow(w1[1]) * e1;
  o.d2 = narrow(w0[2]) * r0 + narrow(w1[2]) * e1;
  o.d3 = narrow(w0[3]) * r0 + narrow(w1[3]) * e1;
  o.d4 = narrow(w0[4]) * r0 + narrow(w1[4]) * e1;
  o.chi2 = r0 * r0 * narrow(i0) + e1 * e1 * narrow(i1);
  return o;
}

// One Kalman update of the state with covariance in FP64 (zone) or FP32;
// diag: the zone's covariance is known to be diagonal (the first update
// after a (re)seed).
__device__ __forceinline__ float update_any(TrkState& p, bool zone, double* D, float* C, float my, float mz,
                                             const KConst& kc, bool diag = false) {
  if (zone) {
    const float r0 = residual_y(p, my), r1 = residual_z(p, mz);
    const UpdOut o = diag ? kalman_update_d_diag(D, r0, r1, kc.Vd) : kalman_update_d(D, r0, r1, kc.Vd);
    acc2(p.y, p.yl, o.d0);
    acc2(p.z, p.zl, o.d1);
    acc2(p.s, p.sl, o.d2);
    p.t += o.d3;
    p.q += o.d4;
    return o.chi2;
  }
  return kalman_update<float>(p, C, my, mz, kc.V);
}

// The FP64 zone after a (re)seed holds the first kc.fp64_updates Kalman
// updates.  In the passes whose covariance is an output (the backward pass,
// the refits, the codec's fit) it holds, up to twice as many, further ones
// while the last update still more than halved the variance of sin phi,
// dz/ds_T or q/pT: the covariance is then still converging, and the next
// update's subtraction C -= G C[0:2,:] would cancel leading digits of those
// entries in binary32.  The forward pass, whose covariance only gates the
// pick-up, keeps the fixed count.
// zone_update makes one update (covariance in D inside the zone, else in C),
// counts it in nupd and moves the covariance into C when the zone ends with
// it; zend, kc.fp64_updates at the (re)seed, is the count that ends the zone,
// zmax the largest it may become.
__device__ __forceinline__ float zone_update(TrkState& p, bool zone, double* D, float* C, float my, float mz,
                                             const KConst& kc, int& nupd, int& zend, int zmax, bool diag = false) {
  const double b5 = D[5], b9 = D[9], b14 = D[14];
  const float x = update_any(p, zone, D, C, my, mz, kc, diag);
  nupd++;
  if (zone && nupd == zend) {
    if (zend < zmax && (b5 > 2.0 * D[5] || b9 > 2.0 * D[9] || b14 > 2.0 * D[14])) {
      zend++;
    } else {
#pragma unroll
      for (int i = 0; i < 15; i++) C[i] = narrow(D[i]);
    }
  }
  return x;
}

// Propagation with the covariance in FP64 (zone) or FP32; diag: the zone's
// covariance is known to be diagonal (the first propagation after a
// (re)seed, which follows the first update).
__device__ __forceinline__ bool propagate_any(TrkState& p, bool zone, double* D, float* C, int row2, float x2,
                                              const KConst& kc, uint32_t& flags, bool diag = false) {
  Jac J;
  if (!prop_state(p, row2, x2, kc, flags, &J)) return false;
  if (zone && diag) cov_transport_d_diag(D, J);
  else if (zone) cov_transport_d(D, J);
  else cov_transport<float>(C, J.j02, J.j12, J.j13, J.kap);
  return true;
}

template <typename T>
__device__ __forceinline__ void cov_seed(T* C, const KConst& kc) {
#pragma unroll
  for (int i = 0; i < 15; i++) C[i] = T(0);
#pragma unroll
  for (int i = 0; i < 5; i++) C[TPC_CI(i, i)] = (T)kc.c0[i];
}

// Start a state at (y, z) with direction (s, t) and curvature q, z kept
// relative to zref = z.
__device__ __forceinline__ void seed_state(TrkState& p, int row, float x, float y, float z, float s, float t,
                                           float q) {
  p.x = x;
  p.row = row;
  p.y = y;
  p.z = 0.0f;
  p.zref = z;
  p.s = s;
  p.t = t;
  p.q = q;
  p.yl = p.zl = p.sl = 0.0f;
}

// chi2 accumulated in FP64 from binary32 increments: the increments of up to
// 16 updates are summed in binary32 and then added to the FP64 total, so the
// FP64 pipe (1/64 of the FP32 rate on this part) sees one add per 16 updates.
struct Chi2Acc {
  double total;
  float part;
  int n;
  __device__ __forceinline__ void reset() {
    total = 0.0;
    part = 0.0f;
    n = 0;
  }
  __device__ __forceinline__ void add(float x) {
    part += x;
    if (++n == 16) {
      total += (double)part;
      part = 0.0f;
      n = 0;
    }
  }
  __device__ __forceinline__ double value() const { return total + (double)part; }
};

// Work tallies kept in registers by one thread.
struct LocalTally {
  unsigned prop = 0, prop64 = 0, upd32 = 0, upd64 = 0, cand = 0;
  __device__ __forceinline__ void flush(Counts* cn, int phase) {
    Tally t;
    t.prop = prop;
    t.prop64 = prop64;
    t.upd32 = upd32;
    t.upd64 = upd64;
    t.cand = cand;
    t.flush(cn, phase);
  }
};

}  // namespace tpc
