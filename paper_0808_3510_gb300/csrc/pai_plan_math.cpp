// pai_plan_math.cpp -- per-problem parameter choice and FP64 plan-time tables
// shared by every entry point that launches the row kernels.
#include <algorithm>
#include <cmath>

#include "../../include/pai.h"
#include "pai_internal.h"

namespace pai {

namespace {
constexpr double kPi = 3.14159265358979323846;

bool is_even_pos(int v) { return v >= 2 && (v % 2) == 0; }

int next_pow2(long long v) {
  int m = 1;
  while (m < v) m <<= 1;
  return m;
}

int ilog2(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}
}  // namespace

void split_ff(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

int validate_geometry(const pai_geometry& g) {
  if (g.dim != 2 && g.dim != 3) return PAI_ERR_INVALID_ARG;
  if (!is_even_pos(g.nx) || !is_even_pos(g.nt) || !is_even_pos(g.nz)) return PAI_ERR_INVALID_ARG;
  if (g.dim == 3 && !is_even_pos(g.ny)) return PAI_ERR_INVALID_ARG;
  if (!(g.dx > 0) || !(g.dt > 0) || !(g.c > 0) || !(g.dz > 0)) return PAI_ERR_INVALID_ARG;
  if (g.dim == 3 && !(g.dy > 0)) return PAI_ERR_INVALID_ARG;
  if (g.method < PAI_METHOD_KB || g.method > PAI_METHOD_NEAREST) return PAI_ERR_INVALID_ARG;
  if (!(g.oversampling == 0 || g.oversampling > 1.0 || (g.oversampling == 1.0 && method_interp(g.method))))
    return PAI_ERR_INVALID_ARG;
  if (!(g.K >= 0) || !(g.alpha >= 0)) return PAI_ERR_INVALID_ARG;
  if (!std::isfinite(g.dx + g.dt + g.c + g.dz + g.oversampling + g.K + g.alpha)) return PAI_ERR_INVALID_ARG;
  if (g.dim == 3 && !std::isfinite(g.dy)) return PAI_ERR_INVALID_ARG;
  if (g.nt > (1 << 14)) return PAI_ERR_UNSUPPORTED;  // padded length M <= 16384 * 2
  return PAI_OK;
}

// Padded length M = smallest power of two >= c_os nt (at least 32); window
// shape beta = alpha / c_os (default: pi (2 - 1/c) (1 - 1e-3), the paper's
// "alpha slightly smaller than pi (2c - 1)"); half tap count H = ceil(c_os K)
// or, with K = 0, the smallest H whose truncation error is <= 1e-8.
int choose_problem_params(const pai_geometry& g, ProblemParams& p) {
  p.method = g.method;
  const double c_req = g.oversampling > 0 ? g.oversampling : 2.0;
  long long want = (long long)std::ceil(c_req * g.nt - 1e-9);
  p.M = std::max(32, next_pow2(want));
  if (p.M > 16 * 1024) return PAI_ERR_UNSUPPORTED;
  p.mshift = ilog2(p.M);
  p.c_eff = (double)p.M / g.nt;
  if (method_interp(g.method)) {
    // no window: H only sizes the ghost cells the interpolation reads
    p.beta = 0.0;
    p.H = 2;
    return PAI_OK;
  }
  if (g.method == PAI_METHOD_TSINC) {
    p.beta = 0.0;
    const double K = g.K > 0 ? g.K : 3.0;
    p.H = (int)std::ceil(c_req * K - 1e-9);
    if (p.H < 2) p.H = 2;
    if (p.H > kMaxH) return PAI_ERR_UNSUPPORTED;
    return PAI_OK;
  }
  if (g.alpha > 0) {
    p.beta = g.alpha / c_req;
    if (!(g.alpha < kPi * (2 * c_req - 1))) return PAI_ERR_INVALID_ARG;
  } else {
    p.beta = kPi * (2.0 - 1.0 / p.c_eff) * (1.0 - 1e-3);
  }
  if (g.K > 0) {
    p.H = (int)std::ceil(c_req * g.K - 1e-9);
    if (p.H < 2) p.H = 2;
    if (p.H > kMaxH) return PAI_ERR_UNSUPPORTED;
  } else {
    p.H = 0;
    for (int h = 2; h <= kMaxH; ++h)
      if (predicted_error(0, p.c_eff, h, p.beta) <= 1e-8) {
        p.H = h;
        break;
      }
    if (!p.H) p.H = kMaxH;
  }
  return PAI_OK;
}

int window_shape_ok(double c_eff, double beta) {
  // the Lemma's condition on the shape alpha = beta c: pi < alpha < pi (2c - 1)
  const double a = beta * c_eff;
  return a > kPi && a < kPi * (2 * c_eff - 1);
}

double default_beta(double c_eff) { return kPi * (2.0 - 1.0 / c_eff) * (1.0 - 1e-3); }

int smallest_padded_length(const pai_geometry& g, int H, double tol) {
  for (long long M = std::max<long long>(32, next_pow2((long long)g.nt + 1)); M <= 16 * 1024; M <<= 1) {
    const double c = (double)M / g.nt;
    const double beta = default_beta(c);
    if (predicted_error(0, c, H, beta) <= tol && prescale_range(c, H, beta) <= kMaxPrescaleRange) return (int)M;
  }
  return 0;
}

void lateral_axes(const pai_geometry& g, int& n1, int& n2, double& d1, double& d2) {
  if (g.dim == 2) {
    n1 = 1; n2 = g.nx; d1 = 1.0; d2 = g.dx;
  } else {
    n1 = g.nx; n2 = g.ny; d1 = g.dx; d2 = g.dy;
  }
}

void fill_row_tables(const pai_geometry& g, double c_eff, int H, double beta, float* prescale, float* rowS,
                     float* zt) {
  if (method_interp(g.method)) {
    for (int n = 0; n < g.nt; ++n) prescale[n] = 1.0f;  // the plain oversampled DFT
  } else {
    prescale_table(method_window(g.method), g.nt, c_eff, H, beta, 1.0, prescale);
  }
  int n1, n2;
  double d1, d2;
  lateral_axes(g, n1, n2, d1, d2);
  const int half = n2 / 2;
  const int rows = n1 * (half + 1);
  for (int r = 0; r < rows; ++r) {
    int i1 = r / (half + 1), i2 = r % (half + 1);
    int k1 = (n1 == 1) ? 0 : (i1 < n1 / 2 ? i1 : i1 - n1);
    double a1 = k1 / (n1 * d1), a2 = i2 / (n2 * d2);
    split_ff(a1 * a1 + a2 * a2, rowS[2 * r], rowS[2 * r + 1]);
  }
  const int lz = g.nz / 2 + 1;
  for (int l = 0; l < lz; ++l) {
    double kz = l / (g.nz * g.dz);
    split_ff(kz * kz, zt[4 * l], zt[4 * l + 1]);
    zt[4 * l + 2] = (float)kz;
    zt[4 * l + 3] = 0.0f;
  }
}

void fill_row_scalars(const pai_geometry& g, int M, RowProblem& r) {
  int n1, n2;
  double d1, d2;
  lateral_axes(g, n1, n2, d1, d2);
  r.nt = g.nt;
  r.M = M;
  r.nz = g.nz;
  r.lz = g.nz / 2 + 1;
  r.n1 = n1;
  r.n2 = n2;
  r.rows = n1 * (n2 / 2 + 1);
  r.tpr = M / kElemsPerThread;
  r.slot = row_slot_stride(M);
  r.mshift = 0;
  while ((1 << r.mshift) < M) ++r.mshift;
  r.nzshift = 0;
  if ((g.nz & (g.nz - 1)) == 0)
    while ((1 << r.nzshift) < g.nz) ++r.nzshift;
  const double B = (double)M * g.c * g.dt;
  split_ff(B * B, r.B2hi, r.B2lo);
  r.wscale = (float)(2.0 * g.c * g.dt / g.dz * B / ((double)n1 * n2 * g.nz));
  r.nt_over_M = (float)((double)g.nt / M);
  r.method = g.method;
}

void twiddle_table(int TW, float2* tw) {
  auto w = [&](long long k) {
    const double a = -2.0 * kPi * (double)(k % TW) / TW;
    return make_float2((float)std::cos(a), (float)std::sin(a));
  };
  for (int j = 0; j < kTwLo; ++j) tw[j] = w(j);
  const int nhi = twiddle_entries(TW) - kTwLo;
  for (int i = 0; i < nhi; ++i) tw[kTwLo + i] = w((long long)kTwLo * i);
}

}  // namespace pai
