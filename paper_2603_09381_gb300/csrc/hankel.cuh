// Bessel functions J0, J1, Y0, Y1 of a positive real argument in FP64, for the
// Hankel functions H_nu = J_nu + i Y_nu of the Helmholtz kernels.
//
// z >= 8: Hankel's modulus-phase form (DLMF 10.17.3-10.17.4; Abramowitz &
//   Stegun 9.2.5-9.2.10)
//     H_nu(z) = sqrt(2/(pi z)) e^{i w} (P_nu(z) + i Q_nu(z)),  w = z - nu pi/2 - pi/4,
//   with P_nu and Q_nu from
//   - z >= 60: the asymptotic expansion in 1/z^2,
//       P = sum_k (-1)^k a_{2k}(nu) z^{-2k},  Q = sum_k (-1)^k a_{2k+1}(nu) z^{-2k-1},
//       a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (k! 8^k),
//     12 terms (remainder below 1e-17: for real z it is bounded by the first
//     omitted term, DLMF 10.17(iii));
//   - 8 <= z < 60: polynomial fits of P_nu - 1 and z Q_nu in 1/z^2 on
//     [8, 12), [12, 20), [20, 30), [30, 60) (hankel_fit.h, written by
//     gen_hankel_fit.py from 40-digit values; within 2e-17 of P_nu and Q_nu).
//   One sincos of w_0 = z - pi/4 serves both orders (w_1 = w_0 - pi/2); the
//   subtraction adds at most half an ulp of z to the phase.
// The interval of z is chosen on z rounded to FP32 (comparisons on the FP32
// pipes): next to a boundary either neighbouring form is within its bound.
// z < 8: CUDA's j0 / y0 / j1 / y1.
// Complex z (lossy interiors, self blocks): Miller's backward recurrence
//   J_{n-1} = (2n/z) J_n - J_{n+1} from an even start M > |z| + 25 + 3 sqrt|z|,
//   normalised by 1 = J0 + 2 sum J_2k (A&S 9.1.27, 9.1.46), and Neumann's
//   series (A&S 9.1.88)
//     (pi/2) Y0 = (ln(z/2) + gamma) J0 - 2 sum_{k>=1} (-1)^k J_2k / k,
//   with its derivative for Y1 = -Y0':
//     (pi/2) Y1 = -J0/z + (ln(z/2) + gamma) J1 + sum_{k>=1} (-1)^k (J_{2k-1} - J_{2k+1})/k.
#pragma once
#include <cuda_runtime.h>
#include "hankel_fit.h"

constexpr double HK_ZA = 8.0;    // modulus-phase form from here up
constexpr double HK_ZS = 60.0;   // asymptotic series from here up
constexpr int HK_TERMS = 12;     // a_0 .. a_11

// a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j-1)^2) / (8 j), with the (-1)^floor(k/2)
// sign of the series folded in (evaluated at compile time).
constexpr double hk_coef(int nu, int k) {
  double a = 1.0;
  for (int j = 1; j <= k; ++j) a *= (4.0 * nu * nu - (2.0 * j - 1) * (2.0 * j - 1)) / (8.0 * j);
  return ((k / 2) & 1) ? -a : a;
}
#define HK_ROW(nu) \
  {hk_coef(nu, 0), hk_coef(nu, 1), hk_coef(nu, 2), hk_coef(nu, 3), hk_coef(nu, 4), hk_coef(nu, 5), hk_coef(nu, 6), \
   hk_coef(nu, 7), hk_coef(nu, 8), hk_coef(nu, 9), hk_coef(nu, 10), hk_coef(nu, 11)}
static __constant__ double c_hk_a0[HK_TERMS] = HK_ROW(0);
static __constant__ double c_hk_a1[HK_TERMS] = HK_ROW(1);
#undef HK_ROW

// J and Y of orders 0 and 1 from P_nu, Q_nu (iz = 1/z).
__device__ __forceinline__ void hankel_combine(double z, double iz, double P0, double Q0, double P1, double Q1,
                                               double& J0, double& Y0, double& J1, double& Y1) {
  double c, d;
  sincos(z - 0.78539816339744830962, &d, &c);                  // sin, cos of z - pi/4
  const double s = sqrt(0.63661977236758134308 * iz);          // sqrt(2/(pi z))
  J0 = s * (P0 * c - Q0 * d);
  Y0 = s * (P0 * d + Q0 * c);
  J1 = s * (P1 * d + Q1 * c);
  Y1 = s * (Q1 * d - P1 * c);
}

// z >= 60: the expansion's 12 terms (P from the even, Q from the odd indices).
__device__ __forceinline__ void hankel_series(double z, double iz, double& J0, double& Y0, double& J1, double& Y1) {
  constexpr int PE = 10, QO = 11;
  const double u = iz * iz;
  double P0 = c_hk_a0[PE], P1 = c_hk_a1[PE];
  double Q0 = c_hk_a0[QO], Q1 = c_hk_a1[QO];
#pragma unroll
  for (int k = PE - 2; k >= 0; k -= 2) {
    P0 = fma(P0, u, c_hk_a0[k]);
    P1 = fma(P1, u, c_hk_a1[k]);
  }
#pragma unroll
  for (int k = QO - 2; k >= 1; k -= 2) {
    Q0 = fma(Q0, u, c_hk_a0[k]);
    Q1 = fma(Q1, u, c_hk_a1[k]);
  }
  hankel_combine(z, iz, P0, Q0 * iz, P1, Q1 * iz, J0, Y0, J1, Y1);
}

// z >= 8 (iz = 1/z)
__device__ __forceinline__ void hankel_asym(double z, double iz, double& J0, double& Y0, double& J1, double& Y1) {
  const float zf = (float)z;
  if (zf >= (float)HK_ZS) {
    hankel_series(z, iz, J0, Y0, J1, Y1);
    return;
  }
  const double v = iz * iz;
  double P0, zQ0, P1, zQ1;
  if (zf >= 30.f) hankel_fit3(v, P0, zQ0, P1, zQ1);
  else if (zf >= 20.f) hankel_fit2(v, P0, zQ0, P1, zQ1);
  else if (zf >= 12.f) hankel_fit1(v, P0, zQ0, P1, zQ1);
  else hankel_fit0(v, P0, zQ0, P1, zQ1);
  hankel_combine(z, iz, P0, zQ0 * iz, P1, zQ1 * iz, J0, Y0, J1, Y1);
}

// Below z = 8 CUDA's j0/y0/j1/y1 (~1e-15 absolute, measured against scipy
// on GB300).
__device__ __forceinline__ void hankel01(double z, double& J0, double& Y0, double& J1, double& Y1) {
  if ((float)z >= (float)HK_ZA) hankel_asym(z, 1.0 / z, J0, Y0, J1, Y1);
  else { J0 = j0(z); Y0 = y0(z); J1 = j1(z); Y1 = y1(z); }
}

// Same, with 1/z supplied by the caller.
__device__ __forceinline__ void hankel01_inv(double z, double iz, double& J0, double& Y0, double& J1, double& Y1) {
  if ((float)z >= (float)HK_ZA) hankel_asym(z, iz, J0, Y0, J1, Y1);
  else { J0 = j0(z); Y0 = y0(z); J1 = j1(z); Y1 = y1(z); }
}

// ---- complex argument (lossy interior wavenumbers, self blocks only) ---------------
// Miller / Neumann in complex arithmetic (principal branch of the logarithm);
// valid for moderate |z| and Im z >= 0 (the self blocks need |z| <= k- diam(Gamma)).
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zlog(double2 a) { return make_double2(log(hypot(a.x, a.y)), atan2(a.y, a.x)); }

__device__ __forceinline__ void bessel_complex(double2 z, double2& J0, double2& Y0, double2& J1, double2& Y1) {
  const double az = hypot(z.x, z.y);
  int M = (int)(az + 25.0 + 3.0 * sqrt(az));
  M += (M & 1);
  const double2 t2z = zdiv(make_double2(2.0, 0.0), z);
  double2 jp1 = make_double2(0, 0), jn = make_double2(1e-30, 0);
  double2 norm = make_double2(0, 0), s0 = make_double2(0, 0), s1 = make_double2(0, 0);
  for (int n = M; n >= 1; --n) {
    if ((n & 1) == 0) {
      const int k = n >> 1;
      norm.x += 2.0 * jn.x; norm.y += 2.0 * jn.y;
      const double c = ((k & 1) ? -1.0 : 1.0) / k;
      s0.x += c * jn.x; s0.y += c * jn.y;
    } else {
      const int m = (n + 1) >> 1;
      const double c = (m == 1) ? -1.0 : ((m & 1) ? -1.0 : 1.0) * (1.0 / m + 1.0 / (m - 1));
      s1.x += c * jn.x; s1.y += c * jn.y;
    }
    const double2 a = zmul(make_double2(n * t2z.x, n * t2z.y), jn);
    const double2 jm1 = make_double2(a.x - jp1.x, a.y - jp1.y);
    jp1 = jn;
    jn = jm1;
  }
  norm.x += jn.x; norm.y += jn.y;
  const double2 inv = zdiv(make_double2(1, 0), norm);
  J0 = zmul(jn, inv);
  J1 = zmul(jp1, inv);
  s0 = zmul(s0, inv);
  s1 = zmul(s1, inv);
  double2 lg = zlog(make_double2(0.5 * z.x, 0.5 * z.y));
  lg.x += 0.57721566490153286061;
  const double tp = 0.63661977236758134308;
  const double2 a0 = zmul(lg, J0);
  Y0 = make_double2(tp * (a0.x - 2.0 * s0.x), tp * (a0.y - 2.0 * s0.y));
  const double2 q = zdiv(J0, z), a1 = zmul(lg, J1);
  Y1 = make_double2(tp * (-q.x + a1.x + s1.x), tp * (-q.y + a1.y + s1.y));
}
