// weno_frac.cuh -- the finite-volume kernels' WENO5-JS face value (2D:
// kernels_fv.cu, 3D: fv3d.cu): each reconstruction as a fraction, the two
// of a face over one reciprocal.
#pragma once

#include "sif_internal.cuh"

// WENO5-JS reconstruction as a fraction num / den, up to a factor common
// to both (the face flux adds two of them over one division).  With
// t_r = (eps + b_r)^2 the nonlinear weights d_r / t_r, scaled by t0 t1 t2,
// are d_r u_r with u_0 = t1 t2, u_1 = t0 t2, u_2 = t0 t1; the linear
// weights d_r = (0.1, 0.6, 0.3) and the candidates' 1/6 are folded into
// the candidates' coefficients.  The smoothness indicators
// b_r = 13/12 D_r^2 + 1/4 E_r^2 enter only through t_r, so they are taken
// as 12/13 b_r = D_r^2 + 3/13 E_r^2 with eps scaled by 12/13 (eps12_13):
// every t_r scales by (13/12)^2, which cancels in num / den.
__device__ __forceinline__ void weno5_frac(double v1, double v2, double v3, double v4, double v5,
                                          double eps12_13, double &num, double &den) {
  const double k3_13 = 3.0 / 13.0;
  double d0 = (v1 + v3) - 2.0 * v2;
  double e0 = (v1 + 3.0 * v3) - 4.0 * v2;
  double d1 = (v2 + v4) - 2.0 * v3;
  double e1 = v2 - v4;
  double d2 = (v3 + v5) - 2.0 * v4;
  double e2 = (3.0 * v3 + v5) - 4.0 * v4;
  // eps' + b_r' = eps' + D_r^2 + 3/13 E_r^2
  double t0 = (k3_13 * e0) * e0 + (d0 * d0 + eps12_13);
  double t1 = (k3_13 * e1) * e1 + (d1 * d1 + eps12_13);
  double t2 = (k3_13 * e2) * e2 + (d2 * d2 + eps12_13);
  // d_r q_r: 0.1 (2 v1 - 7 v2 + 11 v3) / 6, 0.6 (-v2 + 5 v3 + 2 v4) / 6,
  // 0.3 (2 v3 + 5 v4 - v5) / 6
  double q0 = (1.0 / 30.0) * v1 - (7.0 / 60.0) * v2 + (11.0 / 60.0) * v3;
  double q1 = 0.5 * v3 - 0.1 * v2 + 0.2 * v4;
  double q2 = 0.1 * v3 + 0.25 * v4 - 0.05 * v5;
  t0 *= t0;
  t1 *= t1;
  t2 *= t2;
  double u0 = t1 * t2, u1 = t0 * t2, u2 = t0 * t1;
  num = u0 * q0 + u1 * q1 + u2 * q2;
  den = 0.1 * u0 + 0.6 * u1 + 0.3 * u2;
}

// A (num_l / den_l + num_r / den_r) over one reciprocal of den_l den_r
// (positive: the denominators are sums of products of squares plus
// epsilon); two divisions if the products leave the reciprocal's range
__device__ __forceinline__ double face_value(double A, double nl, double dl, double nr, double dr) {
  double n = nl * dr + nr * dl, d = dl * dr;
  if (d < 0x1p1000 && isfinite(n)) return A * n * recip_newton3(d);
  return A * (nl / dl + nr / dr);
}

