// LGF generation math (Sec. 2, Eq. GL_B and the far-field expansions).
//
// G(n) = - int_0^inf e^{-6t} I_{n1}(2t) I_{n2}(2t) I_{n3}(2t) dt is evaluated with
// the double-exponential (exp-sinh) substitution t = exp((pi/2) sinh u) and the
// trapezoidal rule in u.  The integrand is a product of exponentially scaled
// modified Bessel functions ive(k, 2t) = e^{-2t} I_k(2t).  ive(k, z) for
// k = 0..K at one argument z is produced by Miller's backward recurrence
// I_{k-1} = (2k/z) I_k + I_{k+1}, normalised with the generating-function
// identity e^{-z} (I_0 + 2 sum_{k>=1} I_k) = 1; for large z the Hankel
// expansion ive(k,z) ~ (2 pi z)^{-1/2} sum_m (-1)^m a_m(k) z^{-m} is used.
// Functions are __host__ __device__ so the same code can be unit-checked on
// the host.
#pragma once
#include <cmath>

#ifndef FLGF_HD
#ifdef __CUDACC__
#define FLGF_HD __host__ __device__
#else
#define FLGF_HD
#endif
#endif

namespace flgf {

constexpr double kPi = 3.14159265358979323846264338327950288;
// exp-sinh rule: u in [kUmin, kUmax] with step kHu.
constexpr double kUmin = -4.5;
constexpr double kUmax = 5.75;
constexpr double kHu = 1.0 / 64.0;
constexpr int kQuadNodes = int((kUmax - kUmin) / kHu) + 1;
constexpr double kZAsym = 2.0e4;  // Hankel expansion above this argument

FLGF_HD inline double de_node_u(int j) { return kUmin + kHu * j; }
FLGF_HD inline double de_node_t(int j) { return exp(0.5 * kPi * sinh(de_node_u(j))); }
FLGF_HD inline double de_node_w(int j) {
  const double u = de_node_u(j);
  return kHu * de_node_t(j) * 0.5 * kPi * cosh(u);
}

// ive(k, z) for k = 0..K into out[0..K] (stride `stride` between orders).
FLGF_HD inline void ive_orders(double z, int K, double* out, int stride) {
  if (z >= kZAsym) {
    const double pre = 1.0 / sqrt(2.0 * kPi * z);
    for (int k = 0; k <= K; ++k) {
      const double mu = 4.0 * k * (double)k;
      double term = 1.0, sum = 1.0;
      for (int m = 1; m < 60; ++m) {
        const double r = (mu - (2.0 * m - 1.0) * (2.0 * m - 1.0)) / (8.0 * m * z);
        term *= -r;
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      out[k * stride] = pre * sum;
    }
    return;
  }
  if (z <= 0.0) {
    for (int k = 0; k <= K; ++k) out[k * stride] = (k == 0) ? 1.0 : 0.0;
    return;
  }
  // Start order: far enough above both K and the bulk (~sqrt(z)) of the sequence.
  const int M = K + 40 + (int)(12.0 * sqrt(z) + 2.0 * cbrt(z));
  double ip1 = 0.0, ik = 1e-300, sum = 0.0;
  for (int k = M; k >= 1; --k) {
    // ik = I_k, ip1 = I_{k+1}; produce I_{k-1}
    if (k <= K) out[k * stride] = ik;
    sum += 2.0 * ik;
    const double im1 = (2.0 * k / z) * ik + ip1;
    ip1 = ik;
    ik = im1;
    if (ik > 1e250) {  // rescale everything computed so far
      const double s = 1e-250;
      ik *= s; ip1 *= s; sum *= s;
      for (int q = k; q <= K; ++q) out[q * stride] *= s;
    }
  }
  out[0] = ik;
  sum += ik;
  const double inv = 1.0 / sum;
  for (int k = 0; k <= K; ++k) out[k * stride] *= inv;
}

// Far-field expansions; A3 carries the sign-corrected (subtracted) term.
FLGF_HD inline double lgf_asym2(double x1, double x2, double x3) {
  const double a = x1 * x1, b = x2 * x2, c = x3 * x3;
  const double r2 = a + b + c, r = sqrt(r2);
  const double r7 = r2 * r2 * r2 * r;
  const double q = a * a + b * b + c * c - 3.0 * (a * b + a * c + b * c);
  return -1.0 / (4.0 * kPi * r) - q / (16.0 * kPi * r7);
}
FLGF_HD inline double lgf_asym3(double x1, double x2, double x3) {
  const double a = x1 * x1, b = x2 * x2, c = x3 * x3;
  const double r2 = a + b + c, r = sqrt(r2);
  const double r4 = r2 * r2, r12 = r4 * r4 * r4;
  const double p = -228.0 * (b * c * a * a + b * c * c * a + b * b * c * a)
                   + 621.0 * (a * a * b * b + c * c * b * b + a * a * c * c)
                   - 244.0 * (b * a * a * a + c * a * a * a + b * b * b * a + c * c * c * a
                              + b * c * c * c + b * b * b * c)
                   + 23.0 * (a * a * a * a + b * b * b * b + c * c * c * c);
  return lgf_asym2(x1, x2, x3) - p / (128.0 * kPi * r12 * r);
}

}  // namespace flgf
