// Dormand-Prince 5(4) embedded Runge-Kutta pair (Dormand and Prince, 1980),
// the adaptive integrator of the forward pass: nodes c_s, coupling a_sj,
// fifth-order weights b_s (equal to the last row of a: first same as last)
// and the difference e_s = b_s - b*_s to the fourth-order weights, whose
// combination h sum e_s k_s is the local error estimate.  Stages are
// numbered 1..7 as in the usual tables; index 0 is unused.
#pragma once

namespace llg {
namespace dp {

__host__ __device__ constexpr double c(int s) {
  return s == 2 ? 1.0 / 5 : s == 3 ? 3.0 / 10 : s == 4 ? 4.0 / 5 : s == 5 ? 8.0 / 9 : (s >= 6 ? 1.0 : 0.0);
}

// a(s, j), j < s
__host__ __device__ constexpr double a(int s, int j) {
  return s == 2 ? (j == 1 ? 1.0 / 5 : 0.0)
       : s == 3 ? (j == 1 ? 3.0 / 40 : j == 2 ? 9.0 / 40 : 0.0)
       : s == 4 ? (j == 1 ? 44.0 / 45 : j == 2 ? -56.0 / 15 : j == 3 ? 32.0 / 9 : 0.0)
       : s == 5 ? (j == 1 ? 19372.0 / 6561 : j == 2 ? -25360.0 / 2187 : j == 3 ? 64448.0 / 6561
                 : j == 4 ? -212.0 / 729 : 0.0)
       : s == 6 ? (j == 1 ? 9017.0 / 3168 : j == 2 ? -355.0 / 33 : j == 3 ? 46732.0 / 5247
                 : j == 4 ? 49.0 / 176 : j == 5 ? -5103.0 / 18656 : 0.0)
       : s == 7 ? (j == 1 ? 35.0 / 384 : j == 3 ? 500.0 / 1113 : j == 4 ? 125.0 / 192
                 : j == 5 ? -2187.0 / 6784 : j == 6 ? 11.0 / 84 : 0.0)
       : 0.0;
}

// fifth-order weights (b_7 = 0)
__host__ __device__ constexpr double b(int s) { return s <= 6 ? a(7, s) : 0.0; }

// b_s - b*_s with b* the fourth-order weights
__host__ __device__ constexpr double e(int s) {
  return s == 1 ? 35.0 / 384 - 5179.0 / 57600
       : s == 3 ? 500.0 / 1113 - 7571.0 / 16695
       : s == 4 ? 125.0 / 192 - 393.0 / 640
       : s == 5 ? -2187.0 / 6784 + 92097.0 / 339200
       : s == 6 ? 11.0 / 84 - 187.0 / 2100
       : s == 7 ? -1.0 / 40
       : 0.0;
}

}  // namespace dp
}  // namespace llg
