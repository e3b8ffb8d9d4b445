// Smooth cutoff of the data, g = w_cut * p (Eq. data-part of Sec. 2; w_cut
// built as in Sec. 5 by convolving a mollifier with the indicator of the
// measured box).
//
// Host: the weight table.  Positions are in sampling steps on every data
// axis and the data box is [0, n_a] on axis a.  A sample at distance s_a =
// min(u_a, n_a - u_a) from the faces of axis a gets
//   w = integral over {v : v_a <= s_a for all a} of phi(v) dv,
// phi(v) = C exp(-1 / (1 - |v|^2/eps)^4) on |v|^2 < eps (the bump is even in
// every coordinate, so a distance to the upper face counts like one to the
// lower face).  Distances are integers and only those below
// R = ceil(sqrt(eps)) constrain the integral, so (R+1)^d numbers describe
// every sample.  Each is a tensor Gauss-Legendre sum over the box
// [-sqrt(eps), min(s_a, sqrt(eps))] per axis, divided by the same sum over the
// full cube; the bump is smooth on R^d, and 64 points per axis keep the
// quadrature error below 1e-9 at every eps.  The table is symmetric under
// permutations of the axes, so 3-D entries are computed for sorted distance
// triples only, over a few host threads.
//
// Device: one streaming pass with 16- or 8-byte vectors.  Out of place, a
// flat grid-stride walk over the output; in place, one group of threads per
// data row, and rows far from every lateral face touch only their first R
// and last R - 1 samples (the others keep weight one).  A row's lateral
// distances pick a slice of the table; only samples within R of a time face
// look it up per sample.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "pai_internal.h"

namespace pai {

int cutoff_radius(double eps) { return (int)std::ceil(std::sqrt(eps) - 1e-12); }

namespace {

constexpr int kCutQuad = 64;

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's iteration on the
// three-term recurrence of the Legendre polynomials, started from the
// asymptotic estimate of each root.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct AxisRule {
  std::vector<double> v2, w;  // squared nodes and weights on [-r, min(s, r)]
};

double bump(double r2, double eps) {
  const double q = 1.0 - r2 / eps;
  if (q <= 0.0) return 0.0;
  const double q2 = q * q;
  return std::exp(-1.0 / (q2 * q2));
}

double cube_sum(const AxisRule* ax, int dim, double eps) {
  double acc = 0.0;
  if (dim == 2) {
    for (size_t i = 0; i < ax[0].w.size(); ++i) {
      double row = 0.0;
      for (size_t k = 0; k < ax[1].w.size(); ++k) row += ax[1].w[k] * bump(ax[0].v2[i] + ax[1].v2[k], eps);
      acc += ax[0].w[i] * row;
    }
    return acc;
  }
  for (size_t i = 0; i < ax[0].w.size(); ++i) {
    double plane = 0.0;
    for (size_t j = 0; j < ax[1].w.size(); ++j) {
      const double a = ax[0].v2[i] + ax[1].v2[j];
      if (a >= eps) continue;
      double row = 0.0;
      for (size_t k = 0; k < ax[2].w.size(); ++k) row += ax[2].w[k] * bump(a + ax[2].v2[k], eps);
      plane += ax[1].w[j] * row;
    }
    acc += ax[0].w[i] * plane;
  }
  return acc;
}

}  // namespace

void cutoff_table(int dim, double eps, std::vector<double>& out) {
  const int R = cutoff_radius(eps), R1 = R + 1;
  const double r = std::sqrt(eps);
  std::vector<double> gx, gw;
  gauss_legendre(kCutQuad, gx, gw);
  // one rule per clipped distance s = 0..R (s = R: the whole diameter)
  std::vector<AxisRule> rules(R1);
  for (int s = 0; s <= R; ++s) {
    const double lo = -r, hi = std::min((double)s, r), h = 0.5 * (hi - lo), m = 0.5 * (hi + lo);
    rules[s].v2.resize(kCutQuad);
    rules[s].w.resize(kCutQuad);
    for (int i = 0; i < kCutQuad; ++i) {
      const double v = m + h * gx[i];
      rules[s].v2[i] = v * v;
      rules[s].w[i] = h * gw[i];
    }
  }
  size_t n = 1;
  for (int a = 0; a < dim; ++a) n *= R1;
  out.assign(n, 1.0);
  // sorted distance tuples s_0 <= s_1 (<= s_2) with at least one below R
  std::vector<std::vector<int>> tuples;
  if (dim == 2) {
    for (int a = 0; a < R; ++a)
      for (int b = a; b <= R; ++b) tuples.push_back({a, b});
  } else {
    for (int a = 0; a < R; ++a)
      for (int b = a; b <= R; ++b)
        for (int c = b; c <= R; ++c) tuples.push_back({a, b, c});
  }
  std::vector<double> val(tuples.size());
  AxisRule full[3] = {rules[R], rules[R], rules[R]};
  const double norm = cube_sum(full, dim, eps);
  auto work = [&](size_t begin, size_t step) {
    for (size_t t = begin; t < tuples.size(); t += step) {
      AxisRule ax[3];
      for (int a = 0; a < dim; ++a) ax[a] = rules[tuples[t][a]];
      val[t] = cube_sum(ax, dim, eps) / norm;
    }
  };
  const size_t nthr = dim == 3 ? std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
  std::vector<std::thread> pool;
  for (size_t k = 1; k < nthr; ++k) pool.emplace_back(work, k, nthr);
  work(0, nthr);
  for (auto& th : pool) th.join();
  // scatter to every permutation of each tuple
  for (size_t t = 0; t < tuples.size(); ++t) {
    std::vector<int> p = tuples[t];
    do {
      size_t idx = 0;
      for (int a = 0; a < dim; ++a) idx = idx * R1 + p[a];
      out[idx] = val[t];
    } while (std::next_permutation(p.begin(), p.end()));
  }
}

// ---------------------------------------------------------------------------
// device pass
// ---------------------------------------------------------------------------

template <int V>
struct VecOf;
template <>
struct VecOf<1> {
  using T = float;
};
template <>
struct VecOf<2> {
  using T = float2;
};
template <>
struct VecOf<4> {
  using T = float4;
};

template <int V>
__device__ __forceinline__ void scale_vec(typename VecOf<V>::T& v, const float* w) {
  if constexpr (V == 1) {
    v *= w[0];
  } else if constexpr (V == 2) {
    v.x *= w[0];
    v.y *= w[1];
  } else {
    v.x *= w[0];
    v.y *= w[1];
    v.z *= w[2];
    v.w *= w[3];
  }
}

// One group of tpr threads per data row (rpb = blockDim.x / tpr rows per CTA),
// grid-stride over the rows.
template <int V>
__global__ void __launch_bounds__(256) cutoff_kernel(CutoffLaunch a, int tpr, int band_only) {
  using Vec = typename VecOf<V>::T;
  const int rpb = blockDim.x / tpr;
  const int lr = threadIdx.x / tpr, lane = threadIdx.x - lr * tpr;
  const long long rows = (long long)a.nx * a.ny;
  const int R = a.R, R1 = a.R + 1, nt = a.nt;
  for (long long r = (long long)blockIdx.x * rpb + lr; r < rows; r += (long long)gridDim.x * rpb) {
    const int x = (int)(r / a.ny), y = (int)(r - (long long)x * a.ny);
    const int sx = min(min(x, a.nx - x), R);
    const int sy = a.dim == 3 ? min(min(y, a.ny - y), R) : R;
    const float* T = a.table + (a.dim == 3 ? (sx * R1 + sy) * R1 : sx * R1);
    const float wi = __ldg(T + R);  // the row's weight away from the time faces
    const float* src = a.in + ((long long)x * a.in_ny + y) * nt;
    float* dst = a.out + r * nt;
    if (band_only && sx == R && sy == R) {
      // in place, far from the lateral faces: samples t < R and t > nt - R only
      for (int k = lane; k < 2 * R - 1; k += tpr) {
        const int t = k < R ? k : nt - 2 * R + 1 + k;
        dst[t] = src[t] * __ldg(T + min(t, nt - t));
      }
      continue;
    }
    const Vec* s4 = reinterpret_cast<const Vec*>(src);
    Vec* d4 = reinterpret_cast<Vec*>(dst);
    const int nv = nt / V;
    for (int j = lane; j < nv; j += tpr) {
      Vec v = s4[j];
      float w[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int t = j * V + e;
        const int s = min(t, nt - t);
        w[e] = s < R ? __ldg(T + s) : wi;
      }
      scale_vec<V>(v, w);
      d4[j] = v;
    }
  }
}

// Out of place: a flat grid-stride walk over every vector of the output with
// U vectors per thread in flight (loads first, then weights and stores); the
// (row, j) position advances by the constant stride q nv + rem without
// divisions, so the work splits evenly over the resident threads whatever
// the row length.
template <int V, int U>
__global__ void __launch_bounds__(256) cutoff_stream_kernel(CutoffLaunch a, int nv, long long total, int q, int rem) {
  using Vec = typename VecOf<V>::T;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  unsigned row = (unsigned)(i / nv);
  int j = (int)(i - (long long)row * nv);
  const int R = a.R, R1 = a.R + 1, nt = a.nt;
  const unsigned ny = (unsigned)a.ny;
  for (; i < total; i += U * stride) {
    Vec v[U];
    unsigned rw[U];
    int jj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      rw[u] = row;
      jj[u] = j;
      j += rem;
      row += q;
      if (j >= nv) {
        j -= nv;
        ++row;
      }
    }
    unsigned xs[U], ys[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xs[u] = ny == 1 ? rw[u] : rw[u] / ny;
      ys[u] = rw[u] - xs[u] * ny;
      if (i + u * stride < total)
        v[u] = reinterpret_cast<const Vec*>(a.in + ((long long)xs[u] * a.in_ny + ys[u]) * nt)[jj[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i + u * stride >= total) continue;
      const int x = (int)xs[u], y = (int)ys[u];
      const int sx = min(min(x, a.nx - x), R);
      const int sy = a.dim == 3 ? min(min(y, a.ny - y), R) : R;
      const float* T = a.table + (a.dim == 3 ? (sx * R1 + sy) * R1 : sx * R1);
      const float wi = __ldg(T + R);
      float w[V];
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int tt = jj[u] * V + e;
        const int s = min(tt, nt - tt);
        w[e] = s < R ? __ldg(T + s) : wi;
      }
      scale_vec<V>(v[u], w);
      reinterpret_cast<Vec*>(a.out + (long long)rw[u] * nt)[jj[u]] = v[u];
    }
  }
}

template <int V>
cudaError_t launch_stream(const CutoffLaunch& a, cudaStream_t stream, int sms) {
  constexpr int U = 4;
  const int nv = a.nt / V;
  const long long total = (long long)a.nx * a.ny * nv;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cutoff_stream_kernel<V, U>, 256, 0);
  if (e != cudaSuccess) return e;
  const long long want = (total + 255) / 256;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(want, (long long)std::max(sms, 1) * std::max(occ, 1)));
  const long long stride = (long long)blocks * 256;
  const int q = (int)(stride / nv), rem = (int)(stride % nv);
  cutoff_stream_kernel<V, U><<<blocks, 256, 0, stream>>>(a, nv, total, q, rem);
  return cudaGetLastError();
}

cudaError_t launch_cutoff(const CutoffLaunch& a, cudaStream_t stream, int sms) {
  const long long rows = (long long)a.nx * a.ny;
  if (rows == 0 || a.nt == 0) return cudaSuccess;
  const bool in_place = a.in == a.out;
  const uintptr_t ai = reinterpret_cast<uintptr_t>(a.in), ao = reinterpret_cast<uintptr_t>(a.out);
  int V = 1;
  if (a.nt % 4 == 0 && ai % 16 == 0 && ao % 16 == 0)
    V = 4;
  else if (a.nt % 2 == 0 && ai % 8 == 0 && ao % 8 == 0)
    V = 2;
  if (!in_place) {
    if (V == 4) return launch_stream<4>(a, stream, sms);
    if (V == 2) return launch_stream<2>(a, stream, sms);
    return launch_stream<1>(a, stream, sms);
  }
  const int nv = a.nt / V;
  int tpr = 32;
  while (tpr < 256 && tpr < nv) tpr *= 2;
  const int rpb = 256 / tpr;
  const long long want = (rows + rpb - 1) / rpb;
  const int blocks = (int)std::min<long long>(want, (long long)std::max(sms, 1) * 8);
  const int band = in_place ? 1 : 0;
  if (V == 4)
    cutoff_kernel<4><<<blocks, 256, 0, stream>>>(a, tpr, band);
  else if (V == 2)
    cutoff_kernel<2><<<blocks, 256, 0, stream>>>(a, tpr, band);
  else
    cutoff_kernel<1><<<blocks, 256, 0, stream>>>(a, tpr, band);
  return cudaGetLastError();
}

}  // namespace pai
