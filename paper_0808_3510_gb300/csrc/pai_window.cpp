// pai_window.cpp -- FP64 host math of the Kaiser-Bessel window (paper Sec. 3.2)
// used at plan time: I0, the window transform, the tap polynomials, the
// prescale table and the truncation error of Fourmont's identity (Lemma in
// Sec. 3.1).
//
// Parametrisation.  With oversampling c (= M / nt), interpolation length K and
// shape alpha, write H = c K (half the tap count, in grid units) and
// beta = alpha / c.  In the grid variable y = c (omega - j/c) the window
// transform of Sec. 3.2 becomes
//   psi_hat(y / c) = (2c / I0(beta H)) * phi(y),
//   phi(y) = sinh(beta sqrt(H^2 - y^2)) / sqrt(H^2 - y^2),
// and the window at theta is psi(theta) = I0(H sqrt(beta^2 - (theta/c)^2)) / I0(beta H).
// Fourmont's identity e^{-i omega theta} = 1/(2 pi c psi(theta)) sum_j
// psi_hat(omega - j/c) e^{-i j theta / c} (constant 1/(2 pi c): the Fourier
// coefficient of a 2 pi c periodic function) therefore reads
//   e^{-i omega theta} = s(theta) sum_j phi(c omega - j) e^{-i j theta / c},
//   s(theta) = 1 / (pi I0(H sqrt(beta^2 - (theta/c)^2))),
// so the shape depends on (beta, H) only and c enters through s(theta).
#include <cmath>
#include <cstring>

#include "pai_internal.h"

namespace pai {

// Modified Bessel function of the first kind, order 0, by its power series
// sum_k ((x/2)^k / k!)^2.  All terms are positive, so there is no
// cancellation; the series is summed until the terms no longer change the sum.
double bessel_i0(double x) {
  double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / ((double)k * (double)k);
    double next = sum + term;
    if (next == sum) break;
    sum = next;
  }
  return sum;
}

double kb_phi(double y, double H, double beta) {
  double s2 = H * H - y * y;
  if (s2 > 0) {
    double s = std::sqrt(s2);
    double a = beta * s;
    if (a < 1e-4) return beta * (1.0 + a * a / 6.0);
    return std::sinh(a) / s;
  }
  double s = std::sqrt(-s2);
  double a = beta * s;
  if (a < 1e-4) return beta * (1.0 - a * a / 6.0);
  return std::sin(a) / s;
}

// The window transform of the requested kind in grid units, and the factor
// s(theta) of the identity e^{-i omega theta} = s(theta) sum_j phi(c omega - j) e^{-i j theta / c}:
//   Kaiser-Bessel: phi as above, s = 1 / (pi I0(H sqrt(beta^2 - (theta/c)^2)));
//   indicator of [-c pi, c pi] (truncated sinc): psi_hat(u) = 2 sin(c pi u) / u,
//     so with 1/(2 pi c) and psi = 1 on [-pi, pi]: phi(y) = sin(pi y) / (pi y), s = 1.
double window_phi(int kind, double y, double H, double beta) {
  if (kind == 1) {
    const double pi = 3.14159265358979323846;
    if (std::fabs(y) < 1e-8) return 1.0 - (pi * y) * (pi * y) / 6.0;
    return std::sin(pi * y) / (pi * y);
  }
  return kb_phi(y, H, beta);
}

double window_s(int kind, double theta, double c, int H, double beta) {
  const double pi = 3.14159265358979323846;
  if (kind == 1) return 1.0;
  double arg = beta * beta - (theta / c) * (theta / c);
  if (arg <= 0) return 0.0;
  return 1.0 / (pi * bessel_i0(H * std::sqrt(arg)));
}

// Solve the (n x n) system A x = b in place (Gaussian elimination, partial pivoting).
static bool solve(int n, double* A, double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return true;
}

// Tap it = t + H - 1 at fraction f = z + 1/2 sits at distance y = f - t.
// Pair p (0 <= p < H) is tap it = p; its mirror it' = 2H-1-p satisfies
// w_{it'}(z) = w_p(-z) because phi is even.
double fit_window(int kind, int H, double beta, WindowPoly* out) {
  std::memset(out, 0, sizeof(*out));
  const int n = kDeg + 1;
  const double peak = window_phi(kind, 0.0, H, beta);
  const double pi = 3.14159265358979323846;
  double worst = 0.0;
  for (int p = 0; p < H; ++p) {
    const double t = p - H + 1;
    double A[n * n], b[n];
    for (int i = 0; i < n; ++i) {
      double z = 0.5 * std::cos(pi * (i + 0.5) / n);
      double zp = 1.0;
      for (int d = 0; d < n; ++d) { A[i * n + d] = zp; zp *= z; }
      b[i] = window_phi(kind, z + 0.5 - t, H, beta) / peak;
    }
    if (!solve(n, A, b)) return 1e30;
    for (int e = 0; e < kHalfCoef; ++e) {
      out->ce[p][e] = (float)b[2 * e];
      out->co[p][e] = (float)b[2 * e + 1];
    }
    // verify both taps of the pair on a fine grid, in FP64 with the FP32 coefficients
    for (int i = 0; i <= 256; ++i) {
      double z = -0.5 + i / 256.0;
      double z2 = z * z, E = 0, O = 0;
      for (int e = kHalfCoef - 1; e >= 0; --e) {
        E = E * z2 + out->ce[p][e];
        O = O * z2 + out->co[p][e];
      }
      double wp = E + z * O, wm = E - z * O;
      double ep = std::fabs(wp - window_phi(kind, z + 0.5 - t, H, beta) / peak);
      double em = std::fabs(wm - window_phi(kind, -z + 0.5 - t, H, beta) / peak);
      if (ep > worst) worst = ep;
      if (em > worst) worst = em;
    }
  }
  return worst;
}

double predicted_error(int kind, double c, int H, double beta) {
  const double pi = 3.14159265358979323846;
  double worst = 0.0;
  for (int it = 0; it <= 64; ++it) {
    double theta = -pi + 2.0 * pi * it / 64.0;
    double s = window_s(kind, theta, c, H, beta);
    if (!(s > 0)) return 1.0;
    for (int fi = 0; fi < 32; ++fi) {
      double f = fi / 32.0;
      double re = 0, im = 0;
      for (int t = -H + 1; t <= H; ++t) {
        double w = window_phi(kind, f - t, H, beta);
        re += w * std::cos(t * theta / c);
        im -= w * std::sin(t * theta / c);
      }
      re = std::cos(f * theta / c) - s * re;
      im = -std::sin(f * theta / c) - s * im;
      double e = std::sqrt(re * re + im * im);
      if (e > worst) worst = e;
    }
  }
  return worst;
}

double prescale_range(double c, int H, double beta) {
  const double pi = 3.14159265358979323846;
  const double edge = beta * beta - (pi / c) * (pi / c);
  if (!(edge > 0)) return 1e300;
  return bessel_i0(H * beta) / bessel_i0(H * std::sqrt(edge));
}

void prescale_table(int kind, int nt, double c, int H, double beta, double extra, float* out) {
  const double pi = 3.14159265358979323846;
  const double peak = window_phi(kind, 0.0, H, beta);
  for (int n = 0; n < nt; ++n) {
    double theta = 2.0 * pi * n / nt - pi;
    out[n] = (float)(extra * peak * window_s(kind, theta, c, H, beta));
  }
}

}  // namespace pai
