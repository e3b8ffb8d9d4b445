// pai_internal.h -- descriptors shared by the host planner and the sm_103a
// kernels of libpai.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/pai.h"

namespace pai {

// Largest half tap count supported by the row kernels: taps per node = 2H <= 24.
constexpr int kMaxH = 12;
// Truncation-error bound of the window the tuner picks when the request leaves
// it open (K, oversampling and alpha 0).  The bound is on the error of
// Fourmont's identity, i.e. relative to the sum of the row's magnitudes; a
// row's relative L2 error can exceed it by up to about sqrt(nt) when its
// samples cancel, so 1e-7 keeps every spectrum row within the 1e-5 agreement
// required with the direct reconstruction for nt up to 16384 (measured: a
// 1e-6 bound let one row of the 64-problem batch reach 2e-5).
constexpr double kAutoWindowTol = 1e-7;
// Largest prescale dynamic range (prescale_range) the tuner accepts: FP32
// errors grow about as 1e-8 times the range (measured: 3e-7 at range 8 with
// c = 2, 16 taps; 4e-5 at range 5600 with c = 1.2, 16 taps), so 32 keeps them
// near 1e-6, a tenth of the required agreement.
constexpr double kMaxPrescaleRange = 32.0;
// Polynomial degree of each tap's window polynomial in z = frac - 1/2.
// Even part: z^0, z^2, ..., z^6 (4 coefficients); odd part: z^1, ..., z^7.
// Degree 7 fits the Kaiser-Bessel taps as closely as degree 9 does once the
// FP32 coefficients are rounded (about 3e-8 of the peak for H >= 5 at c = 2).
constexpr int kDeg = 7;
constexpr int kHalfCoef = (kDeg + 1) / 2;  // 4
// Complex values each thread holds during an in-shared-memory FFT pass.
constexpr int kElemsPerThread = 16;

// Window polynomials, identical for every problem of a plan (the window shape
// depends only on beta = alpha / c_os and H = c_os * K, both shared by the
// batch).  Tap it = t + H - 1 (t = -H+1 .. H) and its mirror 2H-1-it share
// one pair p = min(it, 2H-1-it):
//   w_it(z)        = E_p(z^2) + z O_p(z^2)
//   w_{2H-1-it}(z) = E_p(z^2) - z O_p(z^2)
// Passed by value as a kernel parameter, so the coefficients are
// constant-bank operands of the FMAs.
struct WindowPoly {
  float ce[kMaxH][kHalfCoef];  // even coefficients, lowest degree first
  float co[kMaxH][kHalfCoef];  // odd coefficients (of z^1, z^3, ...)
};

// One reconstruction problem as the row kernels see it.  Lateral axes are
// (n1, n2) with n2 the axis halved by the real-to-complex lateral FFT:
// 2-D: (1, nx); 3-D: (nx, ny).  Row r = i1 * (n2/2 + 1) + i2.
struct RowProblem {
  const float2* pt;        // lateral spectrum rows [rows][nt] (fwd in / adj out)
  float2* fh;              // image half spectrum [n1*n2][lz] (fwd out / adj in)
  const float* prescale;   // [nt] window prescale incl. all constant factors
  const float2* rowS;      // [rows] float-float |K_lat / 2 pi|^2
  const float4* zt;        // [lz] (az_hi, az_lo, kz, 0): az = kz^2, kz = l/(nz dz)
  int nt, M, nz, lz;
  int n1, n2, rows;
  int tpr;                 // threads per row in the FFT = M / kElemsPerThread
  int rpc;                 // rows per CTA work item
  int slot;                // complex values per row slot in shared memory (row_slot_stride(M))
  float B2hi, B2lo;        // (M c dt)^2 as float-float: node x = B sqrt(S + az)
  float wscale;            // 2 c dt/dz * B / (n1 n2 nz): W = wscale * kz / x
  float nt_over_M;         // for the node phase
  int mshift;              // log2(M)
  int nzshift;             // log2(nz) when nz is a power of two, else 0
  int method;              // PAI_METHOD_*
  int qmode;               // adjoint kernel evaluates the discrete forward model (depth-row layout only)
  int paired;              // 2-D, forward: pt holds Z[k][m] (k < nx = n2, m < nt/2, row stride nt/2), the
                           // lateral DFT of the sample pairs p[x][2m] + i p[x][2m+1]; the forward row kernel
                           // separates row k's samples from Z[k] and Z[nx - k]
};

struct WorkItem {
  int problem;  // index into the RowProblem array
  int row0;     // first row; rows row0 .. min(row0 + rpc, rows) - 1
};

struct RowLaunch {
  const RowProblem* problems;  // device array
  const WorkItem* items;       // device array, ordered by decreasing cost
  int nitems;
  int* counter;                // device work counter, zeroed before each launch
  const float2* tw;            // e^{-2 pi i k / Mmax}, k < Mmax
  int Mmax;
  int H;                       // half tap count (taps = 2H)
  int fft_region;              // complex values of shared memory used by the row slots (adjoint: nodes follow)
  // adjoint only: sorted-bin spread buffers
  int chunk;                   // nodes per bin chunk
  int bin_offset;              // bytes from the start of dynamic shared memory to the bins
  int bin_slot;                // bytes of bins per row slot: chunk * (2H+1) complex, 16-aligned
  int spread_mode;             // adjoint spread: 0 tap phases (deterministic), 1 shared-memory atomics per
                               // node, 2 shared-memory atomics per run of nodes with equal j0, 3 node pairs
                               // spread by one warp per row (deterministic; windowed methods, 32 or 64
                               // threads per row), 4 node pairs spread by every warp of the row with
                               // shared-memory atomics (windowed methods, a multiple of 32 threads per row)
  int paired;                  // forward: some problem is in the paired layout (RowProblem::paired)
};

// Complex values one row slot needs: the padded FFT layout (one pad per 32)
// and the flat layout with 2*kMaxH ghost cells must both fit.
__host__ __device__ inline int row_slot_stride(int M) { return M + ((M >> 5) > 2 * kMaxH ? (M >> 5) : 2 * kMaxH); }

// Host-side window math (FP64), pai_window.cpp
double bessel_i0(double x);
// Normalised window transform in grid units: phi(y) = sinh(beta sqrt(H^2 - y^2)) / sqrt(H^2 - y^2)
// (analytic continuation sin(...) / ... for |y| > H).
double kb_phi(double y, double H, double beta);
// Window kinds: 0 Kaiser-Bessel, 1 indicator of [-c pi, c pi] (truncated sinc).
double window_phi(int kind, double y, double H, double beta);
double window_s(int kind, double theta, double c, int H, double beta);
// Fit the tap polynomials; returns the max abs fit error relative to phi(0).
double fit_window(int kind, int H, double beta, WindowPoly* out);
// Truncation error of Fourmont's identity for (c, H, beta), max over theta and offsets.
double predicted_error(int kind, double c, int H, double beta);
// Dynamic range of the Kaiser-Bessel prescale over theta in [-pi, pi]:
// s(pi) / s(0) = I0(H beta) / I0(H sqrt(beta^2 - (pi/c)^2)).  The FP32 FFT of
// the prescaled samples carries rounding errors relative to its largest
// values, so the reconstruction's FP32 error grows about in proportion.
double prescale_range(double c, int H, double beta);
// Prescale for sample n: s(theta_n) * phi(0) * extra, theta_n = 2 pi n/nt - pi.
void prescale_table(int kind, int nt, double c, int H, double beta, double extra, float* out);

// Plan-time parameters and tables shared by all entry points, pai_plan_math.cpp.
// Functions returning int return pai_status values.
struct ProblemParams {
  int M = 0, mshift = 0, H = 0;
  double c_eff = 0, beta = 0;
  int method = 0;  // PAI_METHOD_*
};
void split_ff(double v, float& hi, float& lo);
int validate_geometry(const pai_geometry& g);
int choose_problem_params(const pai_geometry& g, ProblemParams& p);
// Kaiser-Bessel shape for oversampling c: beta = pi (2 - 1/c) (1 - 1e-3) (alpha = beta c
// slightly below pi (2c - 1)), and the Lemma's condition pi < beta c < pi (2c - 1).
double default_beta(double c_eff);
int window_shape_ok(double c_eff, double beta);
// Smallest power-of-two padded length M > nt (at least 32, at most 16384) whose
// oversampling c = M / nt and default shape give a truncation error <= tol with
// half tap count H; 0 if there is none.
int smallest_padded_length(const pai_geometry& g, int H, double tol);
// Lateral axes (n1, n2) with n2 halved by the R2C transform, and their spacings.
void lateral_axes(const pai_geometry& g, int& n1, int& n2, double& d1, double& d2);
// prescale [nt], rowS [2 * rows] (float-float), zt [4 * (nz/2 + 1)].
void fill_row_tables(const pai_geometry& g, double c_eff, int H, double beta, float* prescale, float* rowS,
                     float* zt);
// Window kind used by a method (0 KB, 1 sinc) and whether the method gathers with a window at all.
inline int method_window(int method) { return method == PAI_METHOD_TSINC ? 1 : 0; }
inline bool method_interp(int method) { return method == PAI_METHOD_LINEAR || method == PAI_METHOD_NEAREST; }
// Scalar fields of RowProblem (everything except pointers and rpc).
void fill_row_scalars(const pai_geometry& g, int M, RowProblem& r);
// Two-level twiddle table for transforms of every length dividing TW (a power
// of two): tw[j] = w^j for j < kTwLo, tw[kTwLo + i] = w^(kTwLo i) for
// i < TW / kTwLo, w = e^{-2 pi i / TW}; w^k = tw[kTwLo + (k >> 6)] tw[k & 63].
constexpr int kTwLoShift = 6;
constexpr int kTwLo = 1 << kTwLoShift;
inline int twiddle_entries(int TW) { return kTwLo + (TW > kTwLo ? TW / kTwLo : 1); }
void twiddle_table(int TW, float2* tw);

// zf selects the depth-fused kernels (see pai_row_kernels.cuh).
cudaError_t launch_row_forward(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                               cudaStream_t s, bool zf = false);
cudaError_t launch_row_adjoint(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                               cudaStream_t s, bool zf = false);
// Shared memory (bytes) of the row slots of one CTA of `threads` threads for padded length M.
size_t row_fft_region_bytes(int threads, int M);

// FFTs along a strided axis of A[outer][L][C] for power-of-two L, pai_lateral.cu.
bool lateral_supported(int L, int C);
cudaError_t launch_lateral_r2c(const float* in, float2* out, int L, int C, int outer, const float2* tw, int twstride,
                               cudaStream_t s);
cudaError_t launch_lateral_c2r(const float2* in, float* out, int L, int C, int outer, const float2* tw, int twstride,
                               cudaStream_t s);
cudaError_t launch_lateral_c2c(const float2* in, float2* out, int L, int C, int outer, bool inverse, const float2* tw,
                               int twstride, cudaStream_t s);
// In-place FFT of `rows` contiguous complex lines of power-of-two length L (32 <= L <= 16384).
cudaError_t launch_rows_c2c(float2* data, int L, int rows, bool inverse, const float2* tw, int twstride,
                            cudaStream_t s);
// kind: 0 forward row kernel, 1 adjoint row kernel, 2 adjoint row kernel with the pair spread, 3 forward row
// kernel for launches with problems in the paired layout, 4 adjoint with the atomic pair spread
int row_kernel_max_ctas_per_sm(int kind, int threads, size_t smem, int H, bool zf = false);

// Data cutoff w_cut (pai_cutoff.cu).  R = ceil(sqrt(eps)); the table holds
// (R+1)^dim weights indexed by the clipped distances to the faces, time last.
int cutoff_radius(double eps);
void cutoff_table(int dim, double eps, std::vector<double>& out);
struct CutoffLaunch {
  const float* in;     // input row (x, y) at (x * in_ny + y) * nt
  float* out;          // output row (x, y) at (x * ny + y) * nt
  const float* table;  // device, (R+1)^dim weights
  int nx, ny, nt, in_ny;
  int R, dim;
};
cudaError_t launch_cutoff(const CutoffLaunch& a, cudaStream_t stream, int sms);

}  // namespace pai
