// pai_api.cu -- plans and entry points of libpai (C ABI declared in include/pai.h).
//
// A call of pai_reconstruct runs Algorithm 2 as three stream-ordered stages:
//   (a) cuFFT real-to-complex lateral transform of every problem (Eq. fft-1a),
//       layout [row][n] with the halved lateral axis last;
//   (b) ONE persistent launch of the fused row kernel over every lateral
//       frequency row of every problem (prescale, oversampled FFT, window
//       gather, weight: Algorithm 1 + Eq. fft-0), writing the half image
//       spectrum;
//   (c) cuFFT complex-to-real inverse transform of every problem (Eq. fft-1).
// The sequence is captured once per (input, output) pointer pair into a CUDA
// graph and replayed.  pai_adjoint runs the transposed stages in reverse.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pai.h"
#include "pai_internal.h"

using namespace pai;

namespace {

constexpr double kPi = 3.14159265358979323846;

struct ProblemHost {
  pai_geometry g;
  int M = 0, mshift = 0, H = 0;
  double c_eff = 0, K_eff = 0, alpha_eff = 0, beta = 0, pred_err = 0;
  int n1 = 0, n2 = 0, rows = 0, lz = 0, tpr = 0, rpc = 0;
  size_t data_off = 0, img_off = 0;   // floats into the concatenated data / image
  size_t pt_off = 0, fh_off = 0;      // complex values into the workspaces
  size_t pre_off = 0, rowS_off = 0, zt_off = 0;
  cufftHandle lat_r2c = 0, lat_c2r = 0, img_c2r = 0, img_r2c = 0;
  bool made[4] = {false, false, false, false};  // which of the four handles cufftCreate made
  bool have_plans = false;
  bool own_lateral = false;  // lateral R2C by the library's own kernel (2-D, power-of-two nx)
  bool paired = false;       // 2-D otherwise: cuFFT C2C of the sample pairs (RowProblem::paired)
  size_t data_len() const { return (size_t)g.nx * (g.dim == 3 ? g.ny : 1) * g.nt; }
  size_t img_len() const { return (size_t)g.nx * (g.dim == 3 ? g.ny : 1) * g.nz; }
};

struct GraphEntry {
  const void* in = nullptr;
  void* out = nullptr;
  bool adjoint = false;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct pai_plan_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  std::vector<ProblemHost> probs;
  int H = 0, Mmax = 0, threads = 512, ctas = 0, ctas_adj = 0, fft_region = 0;
  int threads_adj = 512, fft_region_adj = 0;  // the adjoint row kernel's own CTA shape
  int TW = 0;  // twiddle table length (power of two >= every FFT length the plan runs)
  int chunk = 128, bin_offset = 0, bin_slot = 0;  // adjoint sorted-bin spread
  int method = PAI_METHOD_KB;                       // PAI_METHOD_*, shared by the batch
  int spread_mode = 1;                              // adjoint spread (RowLaunch::spread_mode): atomics
  int spread_tuned = 1;                             // the faster spread found when the plan was built
  int spread_det = 0;                               // the faster deterministic spread (0 or 3)
  bool pairs_ok = false;                            // spread mode 3 applies to every problem of the plan
  size_t smem_adj3 = 0;                             // mode 3: shared memory of the adjoint row kernel
  int ctas_adj3 = 0;                                //         and its CTA count
  bool pairs_atom_ok = false;                       // spread mode 4 applies to every problem of the plan
  int ctas_adj4 = 0;                                // mode 4: CTA count (shared memory as mode 3)
  bool any_paired = false;  // some problem's lateral spectrum is in the paired layout (RowProblem::paired)
  bool zf = false;      // forward: every stage by the library's kernels (depth-row layout)
  bool zf_adj = false;  // adjoint: the same choice, tuned separately
  size_t smem_fwd = 0, smem_adj = 0;
  WindowPoly poly{};
  double beta = 0, pred_err = 0, fit_err = 0;
  size_t data_total = 0, img_total = 0;
  long long nodes = 0;
  int rows_total = 0;
  // device memory
  float2* d_pt = nullptr;        // lateral spectra
  float2* d_fh = nullptr;        // half image spectra
  float* d_tables = nullptr;     // prescale / rowS / zt, packed (16-byte aligned sections)
  float2* d_tw = nullptr;
  RowProblem* d_problems = nullptr;
  WorkItem* d_items_fwd = nullptr;
  int nitems_fwd = 0;
  WorkItem* d_items_adj = nullptr;
  int nitems_adj = 0;
  int* d_counter = nullptr;
  void* d_cufft_work = nullptr;
  // batched plans: per-problem stages fork over branch streams (problem i on
  // branch i % nbranch), each branch with its own cuFFT work area
  int nbranch = 1;
  std::vector<cudaStream_t> branch;
  std::vector<void*> branch_work;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  size_t cufft_work = 0;
  size_t ws_bytes = 0;
  // host staging for pai_reconstruct_host
  float* d_stage_in = nullptr;
  float* d_stage_out = nullptr;
  // pipelined host calls: two staging pairs, upload / download streams
  float* d_pipe_in[2] = {nullptr, nullptr};
  float* d_pipe_out[2] = {nullptr, nullptr};
  cudaStream_t s_up = nullptr, s_down = nullptr;
  cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_down[2] = {nullptr, nullptr};
  long long host_calls = 0;
  bool pipe_ready = false;  // streams, staging pairs and events of the pipelined host calls exist
  // discrete forward model plans (pai_forward_plan): this plan's geometry is
  // the padded box; the image / detector geometry and the box buffers
  bool qmode = false;
  pai_geometry qimg{};
  float* d_qin = nullptr;   // box image
  float* d_qout = nullptr;  // box data
  // data cutoff w_cut (pai_set_cutoff): weight table on the device
  float* d_cut = nullptr;
  int cut_R = 0;
  double cut_eps = 0.0;
  bool use_graph = true;
  std::string tune_log;  // what the plan's tuner timed and kept, one line per measurement
  // host-side failure injection for the tests of the error paths (set from
  // the environment when the plan is built; see plan_malloc / plan_fft)
  long long alloc_budget = -1;  // PAI_FAULT_ALLOC_BYTES: device bytes this plan may allocate (-1: no cap)
  long long alloc_used = 0;
  int fft_fail_at = -1;         // PAI_FAULT_CUFFT_PLAN: the n-th cuFFT plan creation (from 0) fails
  int fft_made = 0;
  size_t items_fwd_bytes = 0, items_adj_bytes = 0;
  std::vector<GraphEntry> graphs;
  long long own_kernels = 0, fft_execs = 0;
  int own_kernels_per_call = 0, fft_per_call = 0;
  int own_kernels_per_adj = 0, fft_per_adj = 0;
};

namespace {

pai_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PAI_OK;
  if (e == cudaErrorMemoryAllocation) return PAI_ERR_OOM;
  return PAI_ERR_CUDA;
}

pai_status fft_status(cufftResult r) {
  if (r == CUFFT_SUCCESS) return PAI_OK;
  if (r == CUFFT_ALLOC_FAILED) return PAI_ERR_OOM;
  return PAI_ERR_CUFFT;
}

// Device allocation of a plan.  With an allocation cap set (failure
// injection) a request beyond it fails like an exhausted device, before any
// CUDA call, so the unwinding of a partly built plan can be tested without
// exhausting a GPU.
pai_status plan_malloc(pai_plan_s* P, void** ptr, size_t bytes) {
  if (P->alloc_budget >= 0 && P->alloc_used + (long long)bytes > P->alloc_budget) return PAI_ERR_OOM;
  const cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) return cuda_status(e);
  P->alloc_used += (long long)bytes;
  return PAI_OK;
}

// cuFFT plan creation of a plan; with PAI_FAULT_CUFFT_PLAN = n the n-th
// creation (counted from 0 over the plan's build) reports a cuFFT failure
// without calling cuFFT.
cufftResult plan_fft(pai_plan_s* P, cufftHandle h, int rank, int* n, int* inem, int istride, int idist, int* onem,
                     int ostride, int odist, cufftType type, int batch, size_t* ws) {
  if (P->fft_made++ == P->fft_fail_at) return CUFFT_INTERNAL_ERROR;
  return cufftMakePlanMany(h, rank, n, inem, istride, idist, onem, ostride, odist, type, batch, ws);
}

long long env_ll(const char* name, long long dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  const long long x = std::strtoll(v, &end, 10);
  return (end && *end == 0) ? x : dflt;
}

#define PAI_TRY(x)                      \
  do {                                  \
    pai_status _s = (x);                \
    if (_s != PAI_OK) return _s;        \
  } while (0)
#define PAI_CUDA(x) PAI_TRY(cuda_status(x))
#define PAI_FFT(x) PAI_TRY(fft_status(x))

pai_status validate(const pai_geometry& g) { return (pai_status)validate_geometry(g); }

pai_status choose_params(ProblemHost& p) {
  ProblemParams pp;
  pai_status st = (pai_status)choose_problem_params(p.g, pp);
  if (st != PAI_OK) return st;
  p.M = pp.M;
  p.mshift = pp.mshift;
  p.H = pp.H;
  p.c_eff = pp.c_eff;
  p.beta = pp.beta;
  return PAI_OK;
}

pai_status make_cufft_plans(pai_plan_s* P, ProblemHost& p, size_t& work) {
  const pai_geometry& g = p.g;
  size_t ws = 0;
  // lateral R2C / C2R: batch over time samples, element stride nt
  {
    int rank = g.dim - 1;
    int n[2], inem[2], onem[2];
    if (g.dim == 2) {
      n[0] = g.nx; inem[0] = g.nx; onem[0] = g.nx / 2 + 1;
    } else {
      n[0] = g.nx; n[1] = g.ny; inem[0] = g.nx; inem[1] = g.ny; onem[0] = g.nx; onem[1] = g.ny / 2 + 1;
    }
    PAI_FFT(cufftCreate(&p.lat_r2c));
    p.made[0] = true;
    PAI_FFT(cufftSetAutoAllocation(p.lat_r2c, 0));
    if (p.paired) {
      // C2C of the nt/2 complex columns p[x][2m] + i p[x][2m+1] -> Z[k][m]
      int pn[1] = {g.nx}, pe[1] = {g.nx};
      PAI_FFT(plan_fft(P, p.lat_r2c, 1, pn, pe, g.nt / 2, 1, pe, g.nt / 2, 1, CUFFT_C2C, g.nt / 2, &ws));
    } else {
      PAI_FFT(plan_fft(P, p.lat_r2c, rank, n, inem, g.nt, 1, onem, g.nt, 1, CUFFT_R2C, g.nt, &ws));
    }
    work = std::max(work, ws);
    PAI_FFT(cufftCreate(&p.lat_c2r));
    p.made[1] = true;
    PAI_FFT(cufftSetAutoAllocation(p.lat_c2r, 0));
    PAI_FFT(plan_fft(P, p.lat_c2r, rank, n, onem, g.nt, 1, inem, g.nt, 1, CUFFT_C2R, g.nt, &ws));
    work = std::max(work, ws);
  }
  // image C2R / R2C over all axes, natural layout, depth halved
  {
    int rank = g.dim;
    int n[3];
    if (g.dim == 2) {
      n[0] = g.nx; n[1] = g.nz;
    } else {
      n[0] = g.nx; n[1] = g.ny; n[2] = g.nz;
    }
    PAI_FFT(cufftCreate(&p.img_c2r));
    p.made[2] = true;
    PAI_FFT(cufftSetAutoAllocation(p.img_c2r, 0));
    PAI_FFT(plan_fft(P, p.img_c2r, rank, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1, &ws));
    work = std::max(work, ws);
    PAI_FFT(cufftCreate(&p.img_r2c));
    p.made[3] = true;
    PAI_FFT(cufftSetAutoAllocation(p.img_r2c, 0));
    PAI_FFT(plan_fft(P, p.img_r2c, rank, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1, &ws));
    work = std::max(work, ws);
  }
  p.have_plans = true;
  return PAI_OK;
}

// Destroys every handle cufftCreate made, also those of a plan whose
// construction failed half way.
void destroy_fft(ProblemHost& p) {
  if (p.made[0]) cufftDestroy(p.lat_r2c);
  if (p.made[1]) cufftDestroy(p.lat_c2r);
  if (p.made[2]) cufftDestroy(p.img_c2r);
  if (p.made[3]) cufftDestroy(p.img_r2c);
  for (bool& m : p.made) m = false;
  p.have_plans = false;
}

void release(pai_plan_s* P) {
  if (!P) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  if (P->s_up) cudaStreamSynchronize(P->s_up);
  if (P->s_down) cudaStreamSynchronize(P->s_down);
  cudaFree(P->d_qin);
  cudaFree(P->d_qout);
  cudaFree(P->d_cut);
  for (int k = 0; k < 2; ++k) {
    cudaFree(P->d_pipe_in[k]);
    cudaFree(P->d_pipe_out[k]);
    if (P->ev_up[k]) cudaEventDestroy(P->ev_up[k]);
    if (P->ev_comp[k]) cudaEventDestroy(P->ev_comp[k]);
    if (P->ev_down[k]) cudaEventDestroy(P->ev_down[k]);
  }
  if (P->s_up) cudaStreamDestroy(P->s_up);
  if (P->s_down) cudaStreamDestroy(P->s_down);
  for (auto& ge : P->graphs)
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
  for (auto& p : P->probs) destroy_fft(p);
  cudaFree(P->d_pt);
  cudaFree(P->d_fh);
  cudaFree(P->d_tables);
  cudaFree(P->d_tw);
  cudaFree(P->d_problems);
  if (P->d_items_adj == P->d_items_fwd) P->d_items_adj = nullptr;
  cudaFree(P->d_items_fwd);
  cudaFree(P->d_items_adj);
  cudaFree(P->d_counter);
  cudaFree(P->d_cufft_work);
  for (void* w : P->branch_work) cudaFree(w);
  for (cudaStream_t s : P->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : P->ev_join) cudaEventDestroy(e);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  cudaFree(P->d_stage_in);
  cudaFree(P->d_stage_out);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  cudaSetDevice(prev);
  delete P;
}

pai_status set_fft_streams(pai_plan_s* P, cudaStream_t s) {
  if (P->nbranch > 1) return PAI_OK;  // batched plans keep their plans on the branch streams
  for (auto& p : P->probs) {
    PAI_FFT(cufftSetStream(p.lat_r2c, s));
    PAI_FFT(cufftSetStream(p.lat_c2r, s));
    PAI_FFT(cufftSetStream(p.img_c2r, s));
    PAI_FFT(cufftSetStream(p.img_r2c, s));
  }
  return PAI_OK;
}

RowLaunch make_launch(pai_plan_s* P, bool adjoint) {
  RowLaunch L{};
  L.problems = P->d_problems;
  L.items = adjoint ? P->d_items_adj : P->d_items_fwd;
  L.nitems = adjoint ? P->nitems_adj : P->nitems_fwd;
  L.counter = P->d_counter + (adjoint ? 1 : 0);
  L.tw = P->d_tw;
  L.Mmax = P->TW;
  L.H = P->H;
  L.fft_region = adjoint ? P->fft_region_adj : P->fft_region;
  L.chunk = P->chunk;
  L.bin_offset = P->bin_offset;
  L.bin_slot = P->bin_slot;
  L.spread_mode = P->spread_mode;
  L.paired = !adjoint && P->any_paired ? 1 : 0;
  return L;
}

pai_status enqueue_row(pai_plan_s* P, bool adjoint, cudaStream_t s, int threads, int ctas, size_t smem,
                       bool zf = false) {
  RowLaunch L = make_launch(P, adjoint);
  if (adjoint && (P->spread_mode == 3 || P->spread_mode == 4)) {
    // the pair-spread kernels' own occupancy gives their CTA counts
    smem = P->smem_adj3;
    ctas = P->spread_mode == 3 ? P->ctas_adj3 : P->ctas_adj4;
  }
  PAI_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(int), s));
  cudaError_t e = adjoint ? launch_row_adjoint(L, P->poly, threads, ctas, smem, s, zf)
                          : launch_row_forward(L, P->poly, threads, ctas, smem, s, zf);
  return cuda_status(e);
}

// Lateral forward transform (Eq. fft-1a) of a real array x[x][(y)][c], c < C,
// into complex rows out[row][c] (row = i1 (n2/2+1) + i2), by the library's
// kernels: 2-D one R2C along x; 3-D an R2C along y then an in-place C2C
// along x.  The adjoint uses the same transform on the image (C = nz).
pai_status own_lateral_fwd(pai_plan_s* P, const ProblemHost& p, const float* in, float2* out, int C, cudaStream_t s) {
  const pai_geometry& g = p.g;
  if (g.dim == 2) return cuda_status(launch_lateral_r2c(in, out, g.nx, C, 1, P->d_tw, P->TW / g.nx, s));
  PAI_CUDA(launch_lateral_r2c(in, out, g.ny, C, g.nx, P->d_tw, P->TW / g.ny, s));
  return cuda_status(launch_lateral_c2c(out, out, g.nx, (g.ny / 2 + 1) * C, 1, false, P->d_tw, P->TW / g.nx, s));
}

// Lateral inverse (Hermitian C2R) of complex rows in[row][c] into the real
// array out[x][(y)][c]; 3-D runs the C2C along x in place on `in` first.
pai_status own_lateral_inv(pai_plan_s* P, const ProblemHost& p, float2* in, float* out, int C, cudaStream_t s) {
  const pai_geometry& g = p.g;
  if (g.dim == 2) return cuda_status(launch_lateral_c2r(in, out, g.nx, C, 1, P->d_tw, P->TW / g.nx, s));
  PAI_CUDA(launch_lateral_c2c(in, in, g.nx, (g.ny / 2 + 1) * C, 1, true, P->d_tw, P->TW / g.nx, s));
  return cuda_status(launch_lateral_c2r(in, out, g.ny, C, g.nx, P->d_tw, P->TW / g.ny, s));
}

// Stage (a) of the forward operator for problem p.
pai_status enqueue_lateral(pai_plan_s* P, const ProblemHost& p, const float* d_p, cudaStream_t s) {
  if (P->zf || p.own_lateral) return own_lateral_fwd(P, p, d_p + p.data_off, P->d_pt + p.pt_off, p.g.nt, s);
  if (p.paired)
    return fft_status(cufftExecC2C(p.lat_r2c, reinterpret_cast<cufftComplex*>(const_cast<float*>(d_p) + p.data_off),
                                   (cufftComplex*)(P->d_pt + p.pt_off), CUFFT_FORWARD));
  return fft_status(cufftExecR2C(p.lat_r2c, const_cast<float*>(d_p) + p.data_off, (cufftComplex*)(P->d_pt + p.pt_off)));
}

// Stage (c) of the forward operator for problem p: depth-row layout -> inverse
// depth FFT of every row, then the lateral C2R.
pai_status enqueue_inverse(pai_plan_s* P, const ProblemHost& p, float* d_f, cudaStream_t s) {
  if (P->zf) {
    PAI_CUDA(launch_rows_c2c(P->d_fh + p.fh_off, p.g.nz, p.rows, true, P->d_tw, P->TW / p.g.nz, s));
    return own_lateral_inv(P, p, P->d_fh + p.fh_off, d_f + p.img_off, p.g.nz, s);
  }
  return fft_status(cufftExecC2R(p.img_c2r, (cufftComplex*)(P->d_fh + p.fh_off), d_f + p.img_off));
}

// First and last stages of the adjoint for problem p.
pai_status enqueue_adj_first(pai_plan_s* P, const ProblemHost& p, const float* d_h, cudaStream_t s) {
  if (P->zf_adj) {
    PAI_TRY(own_lateral_fwd(P, p, d_h + p.img_off, P->d_fh + p.fh_off, p.g.nz, s));
    return cuda_status(launch_rows_c2c(P->d_fh + p.fh_off, p.g.nz, p.rows, false, P->d_tw, P->TW / p.g.nz, s));
  }
  return fft_status(cufftExecR2C(p.img_r2c, const_cast<float*>(d_h) + p.img_off, (cufftComplex*)(P->d_fh + p.fh_off)));
}

pai_status enqueue_adj_last(pai_plan_s* P, const ProblemHost& p, float* d_pbar, cudaStream_t s) {
  if (P->zf_adj) return own_lateral_inv(P, p, P->d_pt + p.pt_off, d_pbar + p.data_off, p.g.nt, s);
  return fft_status(cufftExecC2R(p.lat_c2r, (cufftComplex*)(P->d_pt + p.pt_off), d_pbar + p.data_off));
}

// Per-problem stages of a batched plan run on the branch streams: fork from s,
// enqueue problem i on branch i % nbranch, join back into s.
pai_status fork(pai_plan_s* P, cudaStream_t s) {
  if (P->nbranch <= 1) return PAI_OK;
  PAI_CUDA(cudaEventRecord(P->ev_fork, s));
  for (auto b : P->branch) PAI_CUDA(cudaStreamWaitEvent(b, P->ev_fork, 0));
  return PAI_OK;
}

pai_status join(pai_plan_s* P, cudaStream_t s) {
  if (P->nbranch <= 1) return PAI_OK;
  for (int b = 0; b < P->nbranch; ++b) {
    PAI_CUDA(cudaEventRecord(P->ev_join[b], P->branch[b]));
    PAI_CUDA(cudaStreamWaitEvent(s, P->ev_join[b], 0));
  }
  return PAI_OK;
}

cudaStream_t stream_of(pai_plan_s* P, size_t i, cudaStream_t s) {
  return P->nbranch > 1 ? P->branch[i % P->nbranch] : s;
}

// The per-problem first stage (forward: lateral R2C of the data; adjoint:
// image-side transforms) and last stage (forward: inverse; adjoint: lateral
// C2R), forked over the branch streams of a batched plan.
pai_status enqueue_first(pai_plan_s* P, const float* in, cudaStream_t s, bool adjoint) {
  PAI_TRY(fork(P, s));
  for (size_t i = 0; i < P->probs.size(); ++i) {
    const cudaStream_t si = stream_of(P, i, s);
    PAI_TRY(adjoint ? enqueue_adj_first(P, P->probs[i], in, si) : enqueue_lateral(P, P->probs[i], in, si));
  }
  return join(P, s);
}

pai_status enqueue_last(pai_plan_s* P, float* out, cudaStream_t s, bool adjoint) {
  PAI_TRY(fork(P, s));
  for (size_t i = 0; i < P->probs.size(); ++i) {
    const cudaStream_t si = stream_of(P, i, s);
    PAI_TRY(adjoint ? enqueue_adj_last(P, P->probs[i], out, si) : enqueue_inverse(P, P->probs[i], out, si));
  }
  return join(P, s);
}

// Stages (a)-(c) for the forward operator, enqueued on s.  spectrum_only
// stops after the row stage with the half image spectrum in d_fh (always the
// non-fused row kernel).
pai_status enqueue_forward(pai_plan_s* P, const float* d_p, float* d_f, cudaStream_t s, bool spectrum_only) {
  PAI_TRY(enqueue_first(P, d_p, s, false));
  const bool zf = P->zf && !spectrum_only;
  PAI_TRY(enqueue_row(P, false, s, P->threads, P->ctas, P->smem_fwd, zf));
  if (!spectrum_only) PAI_TRY(enqueue_last(P, d_f, s, false));
  return PAI_OK;
}

pai_status enqueue_adjoint(pai_plan_s* P, const float* d_h, float* d_pbar, cudaStream_t s) {
  PAI_TRY(enqueue_first(P, d_h, s, true));
  PAI_TRY(enqueue_row(P, true, s, P->threads_adj, P->ctas_adj, P->smem_adj, P->zf_adj));
  return enqueue_last(P, d_pbar, s, true);
}

pai_status run(pai_plan_s* P, const void* in, void* out, bool adjoint) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != P->device) cudaSetDevice(P->device);
  pai_status st = PAI_OK;
  if (!P->use_graph) {
    st = adjoint ? enqueue_adjoint(P, (const float*)in, (float*)out, P->stream)
                 : enqueue_forward(P, (const float*)in, (float*)out, P->stream, false);
  } else {
    GraphEntry* hit = nullptr;
    for (auto& ge : P->graphs)
      if (ge.in == in && ge.out == out && ge.adjoint == adjoint) hit = &ge;
    if (!hit) {
      // capture on the private stream (the caller's stream may be the legacy default stream)
      st = set_fft_streams(P, P->cap_stream);
      cudaGraph_t graph = nullptr;
      if (st == PAI_OK) st = cuda_status(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
      if (st == PAI_OK) {
        pai_status st2 = adjoint ? enqueue_adjoint(P, (const float*)in, (float*)out, P->cap_stream)
                                 : enqueue_forward(P, (const float*)in, (float*)out, P->cap_stream, false);
        cudaError_t e = cudaStreamEndCapture(P->cap_stream, &graph);
        st = (st2 != PAI_OK) ? st2 : cuda_status(e);
      }
      cudaGraphExec_t exec = nullptr;
      if (st == PAI_OK) st = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
      if (graph) cudaGraphDestroy(graph);
      pai_status st3 = set_fft_streams(P, P->stream);
      if (st == PAI_OK) st = st3;
      if (st == PAI_OK) {
        if (P->graphs.size() >= 8) {
          cudaGraphExecDestroy(P->graphs.front().exec);
          P->graphs.erase(P->graphs.begin());
        }
        GraphEntry ge;
        ge.in = in; ge.out = out; ge.adjoint = adjoint; ge.exec = exec;
        P->graphs.push_back(ge);
        hit = &P->graphs.back();
      } else if (exec) {
        cudaGraphExecDestroy(exec);
      }
    }
    if (st == PAI_OK) st = cuda_status(cudaGraphLaunch(hit->exec, P->stream));
  }
  if (st == PAI_OK) {
    P->own_kernels += adjoint ? P->own_kernels_per_adj : P->own_kernels_per_call;
    P->fft_execs += adjoint ? P->fft_per_adj : P->fft_per_call;
  }
  if (prev != P->device) cudaSetDevice(prev);
  return st;
}

// What the tuner decided for a set of geometries on a device, kept for the
// process so that later plans of the same geometries make the same choices
// (same results bit for bit, no tuning time): the window (half tap count and
// padded lengths), the CTA sizes, the adjoint's spread and the pipelines.
struct Wisdom {
  int H = 0;
  std::vector<int> M;  // empty: the window was not tuned
  int threads = 0, threads_adj = 0, spread_tuned = 1, spread_det = 0;
  bool zf = false, zf_adj = false;
  std::string log;
};
std::mutex g_wisdom_mutex;
std::map<std::string, Wisdom> g_wisdom;

std::string wisdom_key(int device, const pai_geometry* gs, int count) {
  std::string k = std::to_string(device) + ":" + std::to_string(count);
  char buf[512];
  for (int i = 0; i < count; ++i) {
    const pai_geometry& g = gs[i];
    std::snprintf(buf, sizeof buf, "|%d %d %d %a %a %d %a %a %d %a %a %a %a %d", g.dim, g.nx, g.ny, g.dx, g.dy, g.nt,
                  g.dt, g.c, g.nz, g.dz, g.oversampling, g.K, g.alpha, g.method);
    k += buf;
  }
  return k;
}

// Plan construction shared by pai_plan and pai_plan_batched.
pai_status build_plan(const pai_geometry* gs, int count, void* stream, pai_plan_s** out, bool qmode = false) {
  if (!gs || !out || count < 1) return PAI_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) PAI_TRY(validate(gs[i]));
  for (int i = 1; i < count; ++i)
    if (gs[i].method != gs[0].method) return PAI_ERR_INVALID_ARG;  // one evaluation method per plan
  pai_plan_s* P = new (std::nothrow) pai_plan_s();
  if (!P) return PAI_ERR_OOM;
  struct Guard {
    pai_plan_s* p;
    ~Guard() { if (p) release(p); }
  } guard{P};
  PAI_CUDA(cudaGetDevice(&P->device));
  P->stream = (cudaStream_t)stream;
  PAI_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  const char* env_graph = std::getenv("PAI_USE_GRAPH");
  P->use_graph = !(env_graph && env_graph[0] == '0');
  P->alloc_budget = env_ll("PAI_FAULT_ALLOC_BYTES", -1);
  P->fft_fail_at = (int)env_ll("PAI_FAULT_CUFFT_PLAN", -1);

  // ---- parameters -------------------------------------------------------
  P->probs.resize(count);
  for (int i = 0; i < count; ++i) {
    ProblemHost& p = P->probs[i];
    p.g = gs[i];
    if (p.g.dim == 2) { p.g.ny = 1; p.g.dy = 1.0; }
    PAI_TRY(choose_params(p));
  }
  P->method = gs[0].method;
  // The window of the whole plan from every problem's padded length M (set
  // in p.M): a common half tap count (H > 0: that one; 0: the largest the
  // problems chose) and, for Kaiser-Bessel, a common shape beta from the
  // smallest oversampling, so one set of tap polynomials serves the launch.
  auto set_window = [&](int Hc) -> pai_status {
    P->H = 0;
    P->Mmax = 0;
    P->pred_err = 0.0;
    double c_min = 1e30;
    for (auto& p : P->probs) {
      p.mshift = 0;
      while ((1 << p.mshift) < p.M) ++p.mshift;
      p.c_eff = (double)p.M / p.g.nt;
      P->H = std::max(P->H, Hc > 0 ? Hc : p.H);
      P->Mmax = std::max(P->Mmax, p.M);
      c_min = std::min(c_min, p.c_eff);
    }
    if (P->method == PAI_METHOD_KB) {
      bool user_alpha = count == 1 && gs[0].alpha > 0;
      P->beta = user_alpha ? P->probs[0].beta : default_beta(c_min);
      for (auto& p : P->probs) {
        p.H = P->H;
        p.beta = P->beta;
        p.K_eff = p.H / p.c_eff;
        p.alpha_eff = p.beta * p.c_eff;
        if (!window_shape_ok(p.c_eff, p.beta)) return PAI_ERR_INVALID_ARG;
        p.pred_err = predicted_error(0, p.c_eff, p.H, p.beta);
        P->pred_err = std::max(P->pred_err, p.pred_err);
      }
      P->fit_err = fit_window(0, P->H, P->beta, &P->poly);
      if (!(P->fit_err < 1e-6)) return PAI_ERR_UNSUPPORTED;
    } else if (P->method == PAI_METHOD_TSINC) {
      // the indicator window: a fixed shape, only the common tap count
      P->beta = 0.0;
      for (auto& p : P->probs) {
        p.H = P->H;
        p.beta = 0.0;
        p.K_eff = p.H / p.c_eff;
        p.alpha_eff = 0.0;
        p.pred_err = predicted_error(1, p.c_eff, p.H, 0.0);
        P->pred_err = std::max(P->pred_err, p.pred_err);
      }
      P->fit_err = fit_window(1, P->H, 0.0, &P->poly);
      if (!(P->fit_err < 1e-6)) return PAI_ERR_UNSUPPORTED;
    } else {
      // interpolation of the plain oversampled DFT: no window, no a-priori bound
      P->beta = 0.0;
      std::memset(&P->poly, 0, sizeof(P->poly));
      P->fit_err = 0.0;
      P->pred_err = -1.0;
      for (auto& p : P->probs) {
        p.H = P->H;
        p.beta = 0.0;
        p.K_eff = 0.0;
        p.alpha_eff = 0.0;
        p.pred_err = -1.0;
      }
    }
    return PAI_OK;
  };
  PAI_TRY(set_window(0));
  std::vector<int> rule_M(count);
  for (int i = 0; i < count; ++i) rule_M[i] = P->probs[i].M;
  const int rule_H = P->H;

  // Window candidates for the tuner when the request leaves the window to the
  // plan (Kaiser-Bessel, K, oversampling and alpha all 0): for each half tap
  // count H, every problem takes the smallest power-of-two M whose
  // oversampling keeps the truncation error within kAutoWindowTol under the
  // common shape; the plan times the candidates and keeps the fastest.
  struct WindowCandidate {
    int H;
    std::vector<int> M;
  };
  std::vector<WindowCandidate> cands;
  bool auto_window = !qmode && P->method == PAI_METHOD_KB;
  for (int i = 0; i < count; ++i)
    if (gs[i].K != 0 || gs[i].oversampling != 0 || gs[i].alpha != 0) auto_window = false;
  if (auto_window) {
    for (int H = 3; H <= 8; ++H) {
      std::vector<int> Ms(count);
      bool ok = true;
      for (int i = 0; i < count && ok; ++i) {
        Ms[i] = smallest_padded_length(P->probs[i].g, H, kAutoWindowTol);
        ok = Ms[i] > 0;
      }
      // the common shape comes from the smallest oversampling; raise any M
      // whose problem then misses the bound (a few rounds at most)
      for (int round = 0; ok && round < 8; ++round) {
        double c_min = 1e30;
        for (int i = 0; i < count; ++i) c_min = std::min(c_min, (double)Ms[i] / P->probs[i].g.nt);
        const double beta = default_beta(c_min);
        bool changed = false;
        for (int i = 0; i < count && ok; ++i) {
          const double c = (double)Ms[i] / P->probs[i].g.nt;
          if (!window_shape_ok(c, beta) || predicted_error(0, c, H, beta) > kAutoWindowTol ||
              prescale_range(c, H, beta) > kMaxPrescaleRange) {
            Ms[i] *= 2;
            ok = Ms[i] <= 16 * 1024;
            changed = true;
          }
        }
        if (!changed) break;
        if (round == 7) ok = false;
      }
      if (!ok) continue;
      bool dup = false;
      for (auto& c : cands) dup = dup || c.M == Ms;
      if (!dup) cands.push_back({H, Ms});
    }
  }
  int tw_need = P->Mmax;
  for (auto& c : cands)
    for (int m : c.M) tw_need = std::max(tw_need, m);

  // ---- CTA shape ----------------------------------------------------------
  int sms = 0;
  PAI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
  int smem_optin = 0;
  PAI_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
  int tpr_max = P->Mmax / kElemsPerThread;
  const char* env_t = std::getenv("PAI_THREADS");
  int threads = env_t ? std::atoi(env_t) : 512;
  // forward-model plans (no tuner): the spread's barriers favour small CTAs
  if (qmode && !env_t) threads = 128;
  threads = std::max(threads, tpr_max);
  threads = std::max(threads, 64);
  // row slots of a CTA must tile it exactly: the CTA size is a power of two
  if (threads > 1024 || (threads & (threads - 1)) != 0) return PAI_ERR_UNSUPPORTED;

  // ---- pipeline: all stages by the library's kernels when every size allows -----
  {
    const char* env_zf = std::getenv("PAI_FUSED_DEPTH");
    bool zf = !(env_zf && env_zf[0] == '0');
    for (auto& p : P->probs) {
      const pai_geometry& g = p.g;
      const bool nz_ok = (g.nz & (g.nz - 1)) == 0 && g.nz >= 32 && g.nz <= 16384;
      bool lat_ok;
      if (g.dim == 2) {
        lat_ok = lateral_supported(g.nx, g.nt) && lateral_supported(g.nx, g.nz);
      } else {
        const int h = g.ny / 2 + 1;
        lat_ok = lateral_supported(g.ny, g.nt) && lateral_supported(g.ny, g.nz) &&
                 lateral_supported(g.nx, h * g.nt) && lateral_supported(g.nx, h * g.nz);
      }
      zf = zf && nz_ok && lat_ok;
    }
    if (qmode) {
      // the forward model runs on the depth-row adjoint pipeline only
      zf = true;
      for (auto& p : P->probs) {
        const pai_geometry& g = p.g;
        const bool nz_ok = (g.nz & (g.nz - 1)) == 0 && g.nz >= 32 && g.nz <= 16384;
        bool lat_ok;
        if (g.dim == 2) {
          lat_ok = lateral_supported(g.nx, g.nt) && lateral_supported(g.nx, g.nz);
        } else {
          const int h = g.ny / 2 + 1;
          lat_ok = lateral_supported(g.ny, g.nt) && lateral_supported(g.ny, g.nz) &&
                   lateral_supported(g.nx, h * g.nt) && lateral_supported(g.nx, h * g.nz);
        }
        if (!(nz_ok && lat_ok)) return PAI_ERR_UNSUPPORTED;
      }
    }
    P->zf = zf;
    P->zf_adj = zf;
    P->qmode = qmode;
  }

  // ---- layout -------------------------------------------------------------
  size_t data_off = 0, img_off = 0, pt_off = 0, fh_off = 0, tab_off = 0;
  auto align4 = [](size_t v) { return (v + 3) & ~(size_t)3; };
  for (auto& p : P->probs) {
    double d1, d2;
    lateral_axes(p.g, p.n1, p.n2, d1, d2);
    p.rows = p.n1 * (p.n2 / 2 + 1);
    p.lz = p.g.nz / 2 + 1;
    p.tpr = p.M / kElemsPerThread;
    p.data_off = data_off;
    p.img_off = img_off;
    p.pt_off = pt_off;
    p.fh_off = fh_off;
    data_off += p.data_len();
    img_off += p.img_len();
    pt_off += (size_t)p.rows * p.g.nt;
    // half image spectrum [n1 n2][lz] (non-fused row kernel) or depth rows [rows][nz] (fused)
    fh_off += std::max((size_t)p.n1 * p.n2 * p.lz, (size_t)p.rows * p.g.nz);
    p.pre_off = tab_off;
    tab_off = align4(tab_off + p.g.nt);
    p.rowS_off = tab_off;
    tab_off = align4(tab_off + 2 * (size_t)p.rows);
    p.zt_off = tab_off;
    tab_off = align4(tab_off + 4 * (size_t)p.lz);
    P->rows_total += p.rows;
    const int half = p.n2 / 2;
    long long mirror_rows = (long long)p.n1 * std::max(0, half - 1);
    long long plain_rows = (long long)p.rows - mirror_rows;
    P->nodes += mirror_rows * (long long)p.g.nz + plain_rows * (long long)(p.g.nz / 2 + 1);
  }
  P->data_total = data_off;
  P->img_total = img_off;

  // ---- tables (FP64 on the host) ------------------------------------------
  std::vector<float> tables(tab_off, 0.0f);
  for (auto& p : P->probs)
    fill_row_tables(p.g, p.c_eff, p.H, p.beta, &tables[p.pre_off], &tables[p.rowS_off], &tables[p.zt_off]);
  P->TW = tw_need;  // covers every window candidate's padded length
  for (auto& p : P->probs) {
    p.own_lateral = p.g.dim == 2 && lateral_supported(p.g.nx, p.g.nt);
    // 2-D sizes the library's lateral kernel does not take: cuFFT C2C of the
    // sample pairs instead of cuFFT's strided R2C (which packs and
    // post-processes in passes of their own); the row kernel separates
    p.paired = p.g.dim == 2 && !p.own_lateral && !P->zf;
    if (p.paired) P->any_paired = true;
    if (p.own_lateral || P->zf) P->TW = std::max(P->TW, p.g.nx);
    if (P->zf) {
      P->TW = std::max(P->TW, p.g.nz);
      if (p.g.dim == 3) P->TW = std::max(P->TW, p.g.ny);
    }
  }
  std::vector<float2> tw(twiddle_entries(P->TW));
  twiddle_table(P->TW, tw.data());

  // ---- device memory ------------------------------------------------------
  PAI_TRY(plan_malloc(P, (void**)&P->d_pt, std::max<size_t>(pt_off, 1) * sizeof(float2)));
  PAI_TRY(plan_malloc(P, (void**)&P->d_fh, std::max<size_t>(fh_off, 1) * sizeof(float2)));
  PAI_TRY(plan_malloc(P, (void**)&P->d_tables, std::max<size_t>(tab_off, 4) * sizeof(float)));
  PAI_TRY(plan_malloc(P, (void**)&P->d_tw, tw.size() * sizeof(float2)));
  PAI_TRY(plan_malloc(P, (void**)&P->d_problems, count * sizeof(RowProblem)));
  PAI_TRY(plan_malloc(P, (void**)&P->d_counter, 4 * sizeof(int)));
  PAI_CUDA(cudaMemcpy(P->d_tables, tables.data(), tab_off * sizeof(float), cudaMemcpyHostToDevice));
  PAI_CUDA(cudaMemcpy(P->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));

  std::vector<RowProblem> rp(count);
  for (int i = 0; i < count; ++i) {
    ProblemHost& p = P->probs[i];
    RowProblem& r = rp[i];
    r.pt = P->d_pt + p.pt_off;
    r.fh = P->d_fh + p.fh_off;
    r.prescale = P->d_tables + p.pre_off;
    r.rowS = reinterpret_cast<const float2*>(P->d_tables + p.rowS_off);
    r.zt = reinterpret_cast<const float4*>(P->d_tables + p.zt_off);
    fill_row_scalars(p.g, p.M, r);
    r.paired = p.paired ? 1 : 0;
    if (qmode) {
      r.qmode = 1;
      r.wscale = (float)(0.5 / ((double)r.n1 * r.n2 * p.g.nz));
    }
  }

  // ---- cuFFT ----------------------------------------------------------------
  size_t work = 0;
  for (auto& p : P->probs) PAI_TRY(make_cufft_plans(P, p, work));
  P->cufft_work = work;
  P->nbranch = std::min(count, 4);  // measured on the 64-problem batch: 4 beat 2, 6, 8, 16, 32
  if (P->nbranch > 1) {
    P->branch.resize(P->nbranch, nullptr);
    P->branch_work.resize(P->nbranch, nullptr);
    P->ev_join.resize(P->nbranch, nullptr);
    PAI_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    for (int b = 0; b < P->nbranch; ++b) {
      PAI_CUDA(cudaStreamCreateWithFlags(&P->branch[b], cudaStreamNonBlocking));
      PAI_CUDA(cudaEventCreateWithFlags(&P->ev_join[b], cudaEventDisableTiming));
      if (work) PAI_TRY(plan_malloc(P, &P->branch_work[b], work));
    }
    for (size_t i = 0; i < P->probs.size(); ++i) {
      auto& p = P->probs[i];
      const int b = (int)(i % P->nbranch);
      for (cufftHandle h : {p.lat_r2c, p.lat_c2r, p.img_c2r, p.img_r2c}) {
        if (work) PAI_FFT(cufftSetWorkArea(h, P->branch_work[b]));
        PAI_FFT(cufftSetStream(h, P->branch[b]));
      }
    }
  } else {
    if (work) {
      PAI_TRY(plan_malloc(P, &P->d_cufft_work, work));
      for (auto& p : P->probs) {
        PAI_FFT(cufftSetWorkArea(p.lat_r2c, P->d_cufft_work));
        PAI_FFT(cufftSetWorkArea(p.lat_c2r, P->d_cufft_work));
        PAI_FFT(cufftSetWorkArea(p.img_c2r, P->d_cufft_work));
        PAI_FFT(cufftSetWorkArea(p.img_r2c, P->d_cufft_work));
      }
    }
  }
  PAI_TRY(set_fft_streams(P, P->stream));

  // ---- work items and launch shape ------------------------------------------
  auto build_items = [&](int T, std::vector<WorkItem>& items) {
    items.clear();
    std::vector<std::pair<double, WorkItem>> tmp;
    for (int i = 0; i < count; ++i) {
      ProblemHost& p = P->probs[i];
      const int rpc = T / p.tpr;
      const double cost = (double)p.M * p.mshift + 2.0 * P->H * p.g.nz;  // per row, rough
      for (int r0 = 0; r0 < p.rows; r0 += rpc) {
        WorkItem w;
        w.problem = i;
        w.row0 = r0;
        tmp.push_back({cost * std::min(rpc, p.rows - r0), w});
      }
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const std::pair<double, WorkItem>& a,
                                                 const std::pair<double, WorkItem>& b) { return a.first > b.first; });
    for (auto& t : tmp) items.push_back(t.second);
  };
  // CTA shape of the forward row kernel: rows per CTA, shared memory, work items
  auto finish_shape = [&](int T) -> pai_status {
    for (int i = 0; i < count; ++i) rp[i].rpc = T / P->probs[i].tpr;
    P->threads = T;
    size_t region = 0;
    for (int i = 0; i < count; ++i)
      region = std::max(region, (size_t)rp[i].rpc * (size_t)rp[i].slot * sizeof(float2));
    P->fft_region = (int)(region / sizeof(float2));
    P->smem_fwd = region;
    if (P->smem_fwd > (size_t)smem_optin) return PAI_ERR_UNSUPPORTED;
    const int occ_f = row_kernel_max_ctas_per_sm(P->any_paired ? 3 : 0, T, P->smem_fwd, P->H, P->zf);
    if (occ_f < 1) return PAI_ERR_UNSUPPORTED;
    std::vector<WorkItem> items;
    build_items(T, items);
    P->nitems_fwd = (int)items.size();
    P->ctas = std::min(P->nitems_fwd, occ_f * sms);
    if (P->d_items_fwd) P->alloc_used -= (long long)P->items_fwd_bytes;
    cudaFree(P->d_items_fwd);
    P->d_items_fwd = nullptr;
    P->items_fwd_bytes = items.size() * sizeof(WorkItem);
    PAI_TRY(plan_malloc(P, (void**)&P->d_items_fwd, P->items_fwd_bytes));
    PAI_CUDA(cudaMemcpy(P->d_items_fwd, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    PAI_CUDA(cudaMemcpy(P->d_problems, rp.data(), count * sizeof(RowProblem), cudaMemcpyHostToDevice));
    return PAI_OK;
  };
  // CTA shape of the adjoint row kernel (row slots, then the node lists)
  auto finish_shape_adj = [&](int T) -> pai_status {
    int node_cap = 0;
    size_t region = 0;
    for (int i = 0; i < count; ++i) {
      const int rpc = T / P->probs[i].tpr;
      node_cap = std::max(node_cap, rpc * (P->probs[i].g.nz + 2));
      region = std::max(region, (size_t)rpc * (size_t)rp[i].slot * sizeof(float2));
    }
    P->threads_adj = T;
    P->fft_region_adj = (int)(region / sizeof(float2));
    // Chunk of the adjoint spread: at most the threads of a row slot (one node
    // per thread) and spanning fewer than M - 2H cells (same-sign nodes are at
    // most M c dt / (nz dz) cells apart).
    double gap = 1.0;
    int tpr_min = 1 << 30, m_min = 1 << 30;
    for (auto& p : P->probs) {
      gap = std::max(gap, (double)p.M * p.g.c * p.g.dt / (p.g.nz * p.g.dz));
      tpr_min = std::min(tpr_min, p.tpr);
      m_min = std::min(m_min, p.M);
    }
    const int span_cap = std::max(1, (int)((m_min - 2 * P->H - 1) / (std::ceil(gap) + 1)));
    P->chunk = std::max(1, std::min(tpr_min, span_cap));
    P->bin_slot = 0;
    P->bin_offset = (int)(region + (size_t)node_cap * sizeof(float4));
    P->smem_adj = (size_t)P->bin_offset;
    if (P->smem_adj > (size_t)smem_optin) return PAI_ERR_UNSUPPORTED;
    const int occ_a = row_kernel_max_ctas_per_sm(1, T, P->smem_adj, P->H, P->zf);
    if (occ_a < 1) return PAI_ERR_UNSUPPORTED;
    // spread mode 3 (node pairs spread by one warp per row): windowed
    // methods, rows of one or two warps, and 32 consecutive pairs spanning
    // fewer than M - 2H cells (consecutive nodes of one sign are at most
    // M c dt / (nz dz) cells apart)
    // spread mode 4 (every warp of the row, atomics): windowed methods and
    // rows of whole warps
    P->pairs_ok = !method_interp(P->method) && std::getenv("PAI_NO_PAIRS") == nullptr;
    P->pairs_atom_ok = P->pairs_ok;
    for (auto& p : P->probs) {
      const double g1 = std::ceil((double)p.M * p.g.c * p.g.dt / (p.g.nz * p.g.dz)) + 1.0;
      if (p.tpr != 32 && p.tpr != 64) P->pairs_ok = false;
      if (!(32.0 * g1 + 2.0 * P->H + 2.0 < (double)p.M)) P->pairs_ok = false;
      if (p.tpr % 32 != 0) P->pairs_atom_ok = false;
    }
    P->smem_adj3 = P->smem_adj;
    P->ctas_adj3 = 0;
    P->ctas_adj4 = 0;
    if (P->pairs_ok) {
      const int occ3 = row_kernel_max_ctas_per_sm(2, T, P->smem_adj3, P->H, P->zf);
      if (occ3 < 1) P->pairs_ok = false;
      P->ctas_adj3 = occ3 * sms;
    }
    if (P->pairs_atom_ok) {
      const int occ4 = row_kernel_max_ctas_per_sm(4, T, P->smem_adj3, P->H, P->zf);
      if (occ4 < 1) P->pairs_atom_ok = false;
      P->ctas_adj4 = occ4 * sms;
    }
    std::vector<WorkItem> items;
    build_items(T, items);
    P->nitems_adj = (int)items.size();
    P->ctas_adj = std::min(P->nitems_adj, occ_a * sms);
    P->ctas_adj3 = std::min(P->nitems_adj, P->ctas_adj3);
    P->ctas_adj4 = std::min(P->nitems_adj, P->ctas_adj4);
    if (P->d_items_adj == P->d_items_fwd) P->d_items_adj = nullptr;
    if (P->d_items_adj) P->alloc_used -= (long long)P->items_adj_bytes;
    cudaFree(P->d_items_adj);
    P->d_items_adj = nullptr;
    P->items_adj_bytes = items.size() * sizeof(WorkItem);
    PAI_TRY(plan_malloc(P, (void**)&P->d_items_adj, P->items_adj_bytes));
    PAI_CUDA(cudaMemcpy(P->d_items_adj, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    return PAI_OK;
  };
  const char* env_tune = std::getenv("PAI_AUTOTUNE");
  bool tune = !(env_tune && env_tune[0] == '0') && !env_t && !qmode;
  char logline[512];
  // an earlier plan of the same geometries on this device: reuse its choices
  const char* env_wis = std::getenv("PAI_WISDOM");
  const bool use_wisdom = tune && !(env_wis && env_wis[0] == '0');
  const std::string wkey = use_wisdom ? wisdom_key(P->device, gs, count) : std::string();
  Wisdom wis;
  bool have_wis = false;
  if (use_wisdom) {
    std::lock_guard<std::mutex> lock(g_wisdom_mutex);
    auto it = g_wisdom.find(wkey);
    if (it != g_wisdom.end()) {
      wis = it->second;
      have_wis = true;
    }
  }
  if (have_wis) P->tune_log = "reused the choices of an earlier plan of the same geometries on this device:\n" + wis.log;
  // ---- tuner: the window (half tap count and every problem's padded length) ---
  // (the candidates above and the fixed rule's choice, each timed as one
  // forward row-kernel launch over the whole plan)
  std::vector<float> tables_c(tab_off, 0.0f);
  auto apply = [&](const WindowCandidate& c) -> pai_status {
      for (int i = 0; i < count; ++i) P->probs[i].M = c.M[i];
      PAI_TRY(set_window(c.H));
      for (int i = 0; i < count; ++i) {
        ProblemHost& p = P->probs[i];
        p.tpr = p.M / kElemsPerThread;
        fill_row_tables(p.g, p.c_eff, p.H, p.beta, &tables_c[p.pre_off], &tables_c[p.rowS_off], &tables_c[p.zt_off]);
        fill_row_scalars(p.g, p.M, rp[i]);
      }
      PAI_CUDA(cudaMemcpy(P->d_tables, tables_c.data(), tab_off * sizeof(float), cudaMemcpyHostToDevice));
      tpr_max = P->Mmax / kElemsPerThread;
      return PAI_OK;
  };
  if (tune && !cands.empty() && have_wis && (int)wis.M.size() == count) {
    PAI_TRY(apply(WindowCandidate{wis.H, wis.M}));
    threads = std::max(threads, tpr_max);
    if (threads > 1024) return PAI_ERR_UNSUPPORTED;
  } else if (tune && !cands.empty()) {
    bool have_rule = false;
    for (auto& c : cands) have_rule = have_rule || (c.H == rule_H && c.M == rule_M);
    if (!have_rule) cands.insert(cands.begin(), WindowCandidate{rule_H, rule_M});
    cudaEvent_t e0, e1;
    PAI_CUDA(cudaEventCreate(&e0));
    PAI_CUDA(cudaEventCreate(&e1));
    PAI_CUDA(cudaMemset(P->d_pt, 0, pt_off * sizeof(float2)));
    int best_i = -1;
    float best_ms = 1e30f;
    for (size_t k = 0; k < cands.size(); ++k) {
      if (apply(cands[k]) != PAI_OK) continue;
      const int T = std::min(1024, std::max(512, tpr_max));
      if (finish_shape(T) != PAI_OK) continue;
      float best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, P->cap_stream);
        if (enqueue_row(P, false, P->cap_stream, T, P->ctas, P->smem_fwd, P->zf) != PAI_OK) break;
        cudaEventRecord(e1, P->cap_stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
      }
      long long msum = 0;
      int mmin = 1 << 30, mmax = 0;
      for (int m : cands[k].M) {
        msum += m;
        mmin = std::min(mmin, m);
        mmax = std::max(mmax, m);
      }
      std::snprintf(logline, sizeof logline,
                    "window: H=%d (taps %d), padded lengths %d..%d (sum %lld), max predicted error %.2e%s: "
                    "forward row kernel %.4f ms\n",
                    cands[k].H, 2 * cands[k].H, mmin, mmax, msum, P->pred_err,
                    (cands[k].H == rule_H && cands[k].M == rule_M) ? " [fixed rule]" : "", best);
      P->tune_log += logline;
      if (best < best_ms) {
        best_ms = best;
        best_i = (int)k;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    PAI_TRY(apply(cands[best_i >= 0 ? best_i : 0]));
    threads = std::max(threads, tpr_max);
    if (threads > 1024) return PAI_ERR_UNSUPPORTED;
    std::snprintf(logline, sizeof logline, "window: kept H=%d\n", P->H);
    P->tune_log += logline;
  }
  // ---- tuner: pick the CTA size by timing the forward row kernel -------------
  if (tune && have_wis) {
    threads = std::max(wis.threads, tpr_max);
  } else if (tune) {
    int best_T = 0;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    PAI_CUDA(cudaEventCreate(&e0));
    PAI_CUDA(cudaEventCreate(&e1));
    PAI_CUDA(cudaMemset(P->d_pt, 0, pt_off * sizeof(float2)));
    for (int T : {32, 64, 128, 256, 512, 1024}) {
      if (T < tpr_max) continue;
      if (finish_shape(T) != PAI_OK) continue;
      float best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, P->cap_stream);
        if (enqueue_row(P, false, P->cap_stream, T, P->ctas, P->smem_fwd, P->zf) != PAI_OK) break;
        cudaEventRecord(e1, P->cap_stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
      }
      std::snprintf(logline, sizeof logline, "forward CTA: %d threads: forward row kernel %.4f ms\n", T, best);
      P->tune_log += logline;
      if (best < best_ms) { best_ms = best; best_T = T; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    if (best_T) threads = best_T;
  }
  {
    // prefer the requested size; fall back to smaller CTAs if shared memory does not fit
    pai_status st = PAI_ERR_UNSUPPORTED;
    for (int T = threads; T >= std::max(tpr_max, 32) && st != PAI_OK; T /= 2) st = finish_shape(T);
    if (st != PAI_OK) return st;
  }
  // ---- tuner: the adjoint row kernel's CTA size, timed the same way ----------
  // (the spread's barriers and the forward's FFT passes favour different sizes)
  int threads_adj = threads;
  if (tune && have_wis) {
    threads_adj = std::max(wis.threads_adj, tpr_max);
  } else if (tune) {
    int best_T = 0;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    PAI_CUDA(cudaEventCreate(&e0));
    PAI_CUDA(cudaEventCreate(&e1));
    PAI_CUDA(cudaMemset(P->d_fh, 0, fh_off * sizeof(float2)));
    for (int T : {32, 64, 128, 256, 512, 1024}) {
      if (T < tpr_max) continue;
      if (finish_shape_adj(T) != PAI_OK) continue;
      float best = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, P->cap_stream);
        if (enqueue_row(P, true, P->cap_stream, T, P->ctas_adj, P->smem_adj, P->zf_adj) != PAI_OK) break;
        cudaEventRecord(e1, P->cap_stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
      }
      std::snprintf(logline, sizeof logline, "adjoint CTA: %d threads: adjoint row kernel %.4f ms\n", T, best);
      P->tune_log += logline;
      if (best < best_ms) { best_ms = best; best_T = T; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    if (best_T) threads_adj = best_T;
  }
  {
    pai_status st = PAI_ERR_UNSUPPORTED;
    for (int T = threads_adj; T >= std::max(tpr_max, 32) && st != PAI_OK; T /= 2) st = finish_shape_adj(T);
    if (st != PAI_OK) return st;
  }
  // ---- tuner: the adjoint's spread, shared-memory atomics or tap phases ------
  // (atomics skip the barriers but serialise where many nodes share a cell)
  const char* env_spread = std::getenv("PAI_SPREAD");
  int env_mode = !env_spread ? -1
                 : std::strcmp(env_spread, "tap") == 0 ? 0
                 : std::strcmp(env_spread, "atomic") == 0 ? 1
                 : std::strcmp(env_spread, "runs") == 0 ? 2
                 : std::strcmp(env_spread, "pairs") == 0 ? 3
                 : std::strcmp(env_spread, "pairs_atomic") == 0 ? 4 : -1;
  if (env_mode == 3 && !P->pairs_ok) env_mode = 0;
  if (env_mode == 4 && !P->pairs_atom_ok) env_mode = 1;
  P->spread_det = P->pairs_ok ? 3 : 0;
  if (env_mode >= 0) {
    P->spread_tuned = env_mode;
  } else if (have_wis) {
    P->spread_tuned = wis.spread_tuned == 3 && !P->pairs_ok         ? 0
                      : wis.spread_tuned == 4 && !P->pairs_atom_ok ? 1
                                                                   : wis.spread_tuned;
    P->spread_det = wis.spread_det == 3 && !P->pairs_ok ? 0 : wis.spread_det;
  } else if (tune || qmode) {
    cudaEvent_t e0, e1;
    PAI_CUDA(cudaEventCreate(&e0));
    PAI_CUDA(cudaEventCreate(&e1));
    PAI_CUDA(cudaMemset(P->d_fh, 0, fh_off * sizeof(float2)));
    float best_ms[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    for (int mode = 0; mode < 5; ++mode) {
      if (mode == 3 && !P->pairs_ok) continue;
      if (mode == 4 && !P->pairs_atom_ok) continue;
      P->spread_mode = mode;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, P->cap_stream);
        if (enqueue_row(P, true, P->cap_stream, P->threads_adj, P->ctas_adj, P->smem_adj, P->zf_adj) != PAI_OK) break;
        cudaEventRecord(e1, P->cap_stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best_ms[mode] = std::min(best_ms[mode], ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    static const char* kSpreadName[5] = {"tap phases", "atomics per node", "atomics per run", "node pairs",
                                         "node pairs, atomics"};
    for (int mode = 0; mode < 5; ++mode)
      if (best_ms[mode] < 1e29f) {
        std::snprintf(logline, sizeof logline, "adjoint spread: %s: adjoint row kernel %.4f ms\n", kSpreadName[mode],
                      best_ms[mode]);
        P->tune_log += logline;
      }
    P->spread_tuned = 0;
    for (int mode = 1; mode < 5; ++mode)
      if (best_ms[mode] < best_ms[P->spread_tuned]) P->spread_tuned = mode;
    P->spread_det = (P->pairs_ok && best_ms[3] < best_ms[0]) ? 3 : 0;
  }
  P->spread_mode = P->spread_tuned;
  // ---- tuner: when both pipelines apply, keep the faster one ----------------
  // (library kernels for every stage vs cuFFT for the inverse and the adjoint's
  // image-side and data-side transforms), timed on one eager forward pass each
  if (P->zf && tune && have_wis) {
    P->zf = wis.zf;
    P->zf_adj = wis.zf_adj;
  } else if (P->zf && tune) {
    float* d_in = nullptr;
    float* d_out = nullptr;
    float ms_zf = 1e30f, ms_cufft = 1e30f;
    if (cudaMalloc(&d_in, P->data_total * sizeof(float)) == cudaSuccess &&
        cudaMalloc(&d_out, P->img_total * sizeof(float)) == cudaSuccess &&
        cudaMemset(d_in, 0, P->data_total * sizeof(float)) == cudaSuccess &&
        cudaMemset(d_out, 0, P->img_total * sizeof(float)) == cudaSuccess) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float adj_zf = 1e30f, adj_cufft = 1e30f;
      for (int variant = 0; variant < 4; ++variant) {
        const bool adjoint = variant >= 2;
        P->zf = P->zf_adj = (variant % 2) == 0;
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
          cudaEventRecord(e0, P->cap_stream);
          set_fft_streams(P, P->cap_stream);
          pai_status st = adjoint ? enqueue_adjoint(P, d_out, d_in, P->cap_stream)
                                  : enqueue_forward(P, d_in, d_out, P->cap_stream, false);
          if (st != PAI_OK) break;
          cudaEventRecord(e1, P->cap_stream);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) best = std::min(best, ms);
        }
        if (adjoint) (variant == 2 ? adj_zf : adj_cufft) = best;
        else (variant == 0 ? ms_zf : ms_cufft) = best;
      }
      P->zf_adj = adj_zf <= adj_cufft;
      std::snprintf(logline, sizeof logline,
                    "pipeline: forward pass %.4f ms with the library's transforms, %.4f ms with cuFFT; adjoint "
                    "%.4f / %.4f ms\n", ms_zf, ms_cufft, adj_zf, adj_cufft);
      P->tune_log += logline;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      set_fft_streams(P, P->stream);
    }
    cudaFree(d_in);
    cudaFree(d_out);
    cudaGetLastError();
    P->zf = ms_zf <= ms_cufft;
    if (ms_zf >= 1e29f && ms_cufft >= 1e29f) P->zf = P->zf_adj = true;
    if (!P->zf) {
      int own_lat = 0;
      for (auto& p : P->probs) own_lat += p.own_lateral ? 1 : 0;
      P->own_kernels_per_call = 1 + own_lat;
      P->fft_per_call = 2 * count - own_lat;
    }
  }
  if (P->zf) {
    int k = 1;  // the row kernel
    for (auto& p : P->probs) k += (p.g.dim == 2) ? 3 : 5;  // lateral forward + depth FFT + lateral inverse
    P->own_kernels_per_call = k;
    P->fft_per_call = 0;
  } else {
    int own_lat = 0;
    for (auto& p : P->probs) own_lat += p.own_lateral ? 1 : 0;
    P->own_kernels_per_call = 1 + own_lat;  // the row kernel and the library's lateral kernels
    P->fft_per_call = 2 * count - own_lat;
  }
  if (P->zf_adj) {
    int k = 1;
    for (auto& p : P->probs) k += (p.g.dim == 2) ? 3 : 5;
    P->own_kernels_per_adj = k;
    P->fft_per_adj = 0;
  } else {
    P->own_kernels_per_adj = 1;
    P->fft_per_adj = 2 * count;
  }
  PAI_CUDA(cudaDeviceSynchronize());
  P->ws_bytes = (size_t)P->alloc_used;  // every device buffer the plan holds
  if (use_wisdom && !have_wis) {
    Wisdom w;
    if (!cands.empty()) {
      w.H = P->H;
      for (auto& p : P->probs) w.M.push_back(p.M);
    }
    w.threads = P->threads;
    w.threads_adj = P->threads_adj;
    w.spread_tuned = P->spread_tuned;
    w.spread_det = P->spread_det;
    w.zf = P->zf;
    w.zf_adj = P->zf_adj;
    w.log = P->tune_log;
    std::lock_guard<std::mutex> lock(g_wisdom_mutex);
    g_wisdom.emplace(wkey, std::move(w));
  }
  guard.p = nullptr;
  *out = P;
  return PAI_OK;
}

// Zero-padded copy of an image [nx][ny][nz] into the box [bx][by][bz]
// (the image at the box origin, zeros elsewhere); z fastest, coalesced.
__global__ void pad_box_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz,
                               int by, int bz, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i % bz);
    const long long xy = i / bz;
    const int y = (int)(xy % by);
    const int x = (int)(xy / by);
    out[i] = (x < nx && y < ny && z < nz) ? in[((size_t)x * ny + y) * nz + z] : 0.0f;
  }
}

// Box of the discrete forward model along one axis: room for the image and for
// the distance sound travels in the recorded time, so that no periodic image of
// the object reaches the detectors within it (next power of two).
int forward_box_extent(int n, double d, const pai_geometry& g) {
  const double travel = g.c * g.nt * g.dt / d;
  const long long need = (long long)n + (long long)std::ceil(travel - 1e-9) + 2;
  long long b = 32;
  while (b < need) b <<= 1;
  return b > (1 << 30) ? (1 << 30) : (int)b;
}

// Device buffers are read and written two floats at a time.
bool aligned8(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 7) == 0;
}

}  // namespace

// the detector data grid of a single-problem plan: [nx][ny][nt]
static const pai_geometry& data_geometry(pai_plan_t plan) { return plan->qmode ? plan->qimg : plan->probs[0].g; }

extern "C" {

pai_status pai_plan(const pai_geometry* g, void* cuda_stream, pai_plan_t* out) {
  if (!g || !out) return PAI_ERR_INVALID_ARG;
  return build_plan(g, 1, cuda_stream, out);
}

pai_status pai_plan_batched(const pai_geometry* g, int count, void* cuda_stream, pai_plan_t* out) {
  if (!g || !out || count < 1) return PAI_ERR_INVALID_ARG;
  return build_plan(g, count, cuda_stream, out);
}

pai_status pai_reconstruct(pai_plan_t plan, const float* d_p, float* d_f) {
  if (!plan || !d_p || !d_f || !aligned8(d_p, d_f)) return PAI_ERR_INVALID_ARG;
  if (plan->qmode) return PAI_ERR_INVALID_ARG;  // a forward-model plan
  return run(plan, d_p, d_f, false);
}

pai_status pai_adjoint(pai_plan_t plan, const float* d_h, float* d_pbar) {
  if (!plan || !d_h || !d_pbar || !aligned8(d_h, d_pbar)) return PAI_ERR_INVALID_ARG;
  if (plan->qmode) return PAI_ERR_INVALID_ARG;  // a forward-model plan
  return run(plan, d_h, d_pbar, true);
}

pai_status pai_spectrum(pai_plan_t plan, const float* d_p, float* d_fhat) {
  if (!plan || !d_p || !d_fhat || !aligned8(d_p, d_fhat)) return PAI_ERR_INVALID_ARG;
  if (plan->qmode) return PAI_ERR_INVALID_ARG;  // a forward-model plan
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = enqueue_forward(plan, d_p, nullptr, plan->stream, true);
  if (st == PAI_OK) {
    size_t out = 0;
    for (auto& p : plan->probs) {
      const size_t n = (size_t)p.n1 * p.n2 * p.lz;
      if (st == PAI_OK)
        st = cuda_status(cudaMemcpyAsync(reinterpret_cast<float2*>(d_fhat) + out, plan->d_fh + p.fh_off,
                                         n * sizeof(float2), cudaMemcpyDeviceToDevice, plan->stream));
      out += n;
    }
    plan->own_kernels += 1;
    for (auto& p : plan->probs) {
      if (plan->zf || p.own_lateral) plan->own_kernels += (p.g.dim == 2) ? 1 : 2;
      else plan->fft_execs += 1;
    }
  }
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_reconstruct_host(pai_plan_t plan, const float* h_p, float* h_f) {
  if (!plan || !h_p || !h_f) return PAI_ERR_INVALID_ARG;
  if (plan->qmode) return PAI_ERR_INVALID_ARG;  // a forward-model plan
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = PAI_OK;
  if (!plan->d_stage_in || !plan->d_stage_out) {
    st = plan_malloc(plan, (void**)&plan->d_stage_in, plan->data_total * sizeof(float));
    if (st == PAI_OK) st = plan_malloc(plan, (void**)&plan->d_stage_out, plan->img_total * sizeof(float));
    if (st != PAI_OK) {
      // leave no half-made staging pair behind: the next call starts over
      if (plan->d_stage_in) plan->alloc_used -= (long long)(plan->data_total * sizeof(float));
      cudaFree(plan->d_stage_in);
      plan->d_stage_in = nullptr;
      plan->d_stage_out = nullptr;
    }
  }
  if (st == PAI_OK)
    st = cuda_status(cudaMemcpyAsync(plan->d_stage_in, h_p, plan->data_total * sizeof(float),
                                     cudaMemcpyHostToDevice, plan->stream));
  if (st == PAI_OK) st = run(plan, plan->d_stage_in, plan->d_stage_out, false);
  if (st == PAI_OK)
    st = cuda_status(cudaMemcpyAsync(h_f, plan->d_stage_out, plan->img_total * sizeof(float),
                                     cudaMemcpyDeviceToHost, plan->stream));
  if (st == PAI_OK) st = cuda_status(cudaStreamSynchronize(plan->stream));
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

// Call k uses staging pair k mod 2.  Upload stream: wait until call k-2's
// transforms have read d_pipe_in (ev_comp), copy in, record ev_up.  Plan
// stream: wait for the upload and for call k-2's download of d_pipe_out
// (ev_down), run the graph, record ev_comp.  Download stream: wait for the
// transforms, copy out, record ev_down.
pai_status pai_reconstruct_host_async(pai_plan_t plan, const float* h_p, float* h_f) {
  if (!plan || !h_p || !h_f) return PAI_ERR_INVALID_ARG;
  if (plan->qmode) return PAI_ERR_INVALID_ARG;  // a forward-model plan
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = PAI_OK;
  if (!plan->pipe_ready) {
    if (!plan->s_up) st = cuda_status(cudaStreamCreateWithFlags(&plan->s_up, cudaStreamNonBlocking));
    if (st == PAI_OK && !plan->s_down) st = cuda_status(cudaStreamCreateWithFlags(&plan->s_down, cudaStreamNonBlocking));
    for (int k = 0; k < 2 && st == PAI_OK; ++k) {
      if (!plan->d_pipe_in[k]) st = plan_malloc(plan, (void**)&plan->d_pipe_in[k], plan->data_total * sizeof(float));
      if (st == PAI_OK && !plan->d_pipe_out[k])
        st = plan_malloc(plan, (void**)&plan->d_pipe_out[k], plan->img_total * sizeof(float));
      if (st == PAI_OK && !plan->ev_up[k])
        st = cuda_status(cudaEventCreateWithFlags(&plan->ev_up[k], cudaEventDisableTiming));
      if (st == PAI_OK && !plan->ev_comp[k])
        st = cuda_status(cudaEventCreateWithFlags(&plan->ev_comp[k], cudaEventDisableTiming));
      if (st == PAI_OK && !plan->ev_down[k])
        st = cuda_status(cudaEventCreateWithFlags(&plan->ev_down[k], cudaEventDisableTiming));
    }
    // a failed set-up keeps what it made (released with the plan) and is
    // completed by the next call
    plan->pipe_ready = st == PAI_OK;
  }
  const int k = (int)(plan->host_calls & 1);
  const bool reuse = plan->host_calls >= 2;  // events of call k-2 exist
  if (st == PAI_OK && reuse) st = cuda_status(cudaStreamWaitEvent(plan->s_up, plan->ev_comp[k], 0));
  if (st == PAI_OK)
    st = cuda_status(cudaMemcpyAsync(plan->d_pipe_in[k], h_p, plan->data_total * sizeof(float),
                                     cudaMemcpyHostToDevice, plan->s_up));
  if (st == PAI_OK) st = cuda_status(cudaEventRecord(plan->ev_up[k], plan->s_up));
  if (st == PAI_OK) st = cuda_status(cudaStreamWaitEvent(plan->stream, plan->ev_up[k], 0));
  if (st == PAI_OK && reuse) st = cuda_status(cudaStreamWaitEvent(plan->stream, plan->ev_down[k], 0));
  if (st == PAI_OK) st = run(plan, plan->d_pipe_in[k], plan->d_pipe_out[k], false);
  if (st == PAI_OK) st = cuda_status(cudaEventRecord(plan->ev_comp[k], plan->stream));
  if (st == PAI_OK) st = cuda_status(cudaStreamWaitEvent(plan->s_down, plan->ev_comp[k], 0));
  if (st == PAI_OK)
    st = cuda_status(cudaMemcpyAsync(h_f, plan->d_pipe_out[k], plan->img_total * sizeof(float),
                                     cudaMemcpyDeviceToHost, plan->s_down));
  if (st == PAI_OK) st = cuda_status(cudaEventRecord(plan->ev_down[k], plan->s_down));
  if (st == PAI_OK) ++plan->host_calls;
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_host_wait(pai_plan_t plan) {
  if (!plan) return PAI_ERR_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = PAI_OK;
  if (plan->s_down) st = cuda_status(cudaStreamSynchronize(plan->s_down));
  if (st == PAI_OK && plan->s_up) st = cuda_status(cudaStreamSynchronize(plan->s_up));
  if (st == PAI_OK) st = cuda_status(cudaStreamSynchronize(plan->stream));
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_profile_stages(pai_plan_t plan, const float* d_in, float* d_out, int reps, int adjoint, double* ms) {
  if (!plan || !d_in || !d_out || !ms || reps < 1) return PAI_ERR_INVALID_ARG;
  if (plan->qmode && !adjoint) return PAI_ERR_INVALID_ARG;  // a forward-model plan runs its adjoint pipeline
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  cudaEvent_t ev[4];
  pai_status st = PAI_OK;
  int made = 0;
  for (; made < 4 && st == PAI_OK; ++made) st = cuda_status(cudaEventCreate(&ev[made]));
  double acc[3] = {0, 0, 0};
  cudaStream_t s = plan->stream;
  for (int r = 0; r < reps && st == PAI_OK; ++r) {
    st = cuda_status(cudaEventRecord(ev[0], s));
    if (st == PAI_OK) st = enqueue_first(plan, d_in, s, adjoint != 0);
    if (st == PAI_OK) st = cuda_status(cudaEventRecord(ev[1], s));
    if (st == PAI_OK)
      st = enqueue_row(plan, adjoint != 0, s, adjoint ? plan->threads_adj : plan->threads,
                       adjoint ? plan->ctas_adj : plan->ctas,
                       adjoint ? plan->smem_adj : plan->smem_fwd, adjoint ? plan->zf_adj : plan->zf);
    if (st == PAI_OK) st = cuda_status(cudaEventRecord(ev[2], s));
    if (st == PAI_OK) st = enqueue_last(plan, d_out, s, adjoint != 0);
    if (st == PAI_OK) st = cuda_status(cudaEventRecord(ev[3], s));
    if (st == PAI_OK) st = cuda_status(cudaEventSynchronize(ev[3]));
    for (int k = 0; k < 3 && st == PAI_OK; ++k) {
      float t = 0;
      st = cuda_status(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      acc[k] += t;
    }
    if (st == PAI_OK) {
      plan->own_kernels += adjoint ? plan->own_kernels_per_adj : plan->own_kernels_per_call;
      plan->fft_execs += adjoint ? plan->fft_per_adj : plan->fft_per_call;
    }
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  if (st == PAI_OK)
    for (int k = 0; k < 3; ++k) ms[k] = acc[k] / reps;
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_set_deterministic(pai_plan_t plan, int deterministic) {
  if (!plan || (deterministic != 0 && deterministic != 1)) return PAI_ERR_INVALID_ARG;
  const int mode = deterministic ? (plan->spread_tuned == 3 ? 3 : plan->spread_det) : plan->spread_tuned;
  if (mode == plan->spread_mode) return PAI_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = cuda_status(cudaStreamSynchronize(plan->stream));
  if (st == PAI_OK) {
    // captured graphs hold the launch parameters: capture again on next use
    for (auto& ge : plan->graphs)
      if (ge.exec) cudaGraphExecDestroy(ge.exec);
    plan->graphs.clear();
    plan->spread_mode = mode;
  }
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_set_stream(pai_plan_t plan, void* cuda_stream) {
  if (!plan) return PAI_ERR_INVALID_ARG;
  plan->stream = (cudaStream_t)cuda_stream;
  return set_fft_streams(plan, plan->stream);
}

pai_status pai_get_info(pai_plan_t plan, pai_plan_info* info) {
  if (!plan || !info) return PAI_ERR_INVALID_ARG;
  const ProblemHost& p = plan->probs[0];
  info->count = (int)plan->probs.size();
  info->M = p.M;
  info->taps = plan->method == PAI_METHOD_LINEAR ? 2 : plan->method == PAI_METHOD_NEAREST ? 1 : 2 * plan->H;
  info->oversampling = p.c_eff;
  info->K = p.K_eff;
  info->alpha = p.alpha_eff;
  info->predicted_error = plan->pred_err;
  info->threads_per_cta = plan->threads;
  info->ctas = plan->ctas;
  info->rows = plan->rows_total;
  info->nodes = plan->nodes;
  info->workspace_bytes = plan->ws_bytes;
  info->uses_graph = plan->use_graph ? 1 : 0;
  info->library_ffts = (plan->zf ? 1 : 0) | (plan->zf_adj ? 2 : 0);
  return PAI_OK;
}

pai_status pai_get_problem_info(pai_plan_t plan, int index, pai_problem_info* info) {
  if (!plan || !info || index < 0 || index >= (int)plan->probs.size()) return PAI_ERR_INVALID_ARG;
  const ProblemHost& p = plan->probs[index];
  info->M = p.M;
  info->taps = plan->method == PAI_METHOD_LINEAR ? 2 : plan->method == PAI_METHOD_NEAREST ? 1 : 2 * plan->H;
  info->oversampling = p.c_eff;
  info->K = p.K_eff;
  info->alpha = p.alpha_eff;
  info->predicted_error = p.pred_err;
  return PAI_OK;
}

pai_status pai_tuning_log(pai_plan_t plan, char* buf, size_t cap, size_t* len) {
  if (!plan || (cap > 0 && !buf)) return PAI_ERR_INVALID_ARG;
  const std::string& t = plan->tune_log;
  if (len) *len = t.size();
  if (cap > 0) {
    const size_t n = std::min(cap - 1, t.size());
    std::memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return PAI_OK;
}

pai_status pai_launch_count(pai_plan_t plan, long long* kernels) {
  if (!plan || !kernels) return PAI_ERR_INVALID_ARG;
  *kernels = plan->own_kernels;
  return PAI_OK;
}

pai_status pai_destroy(pai_plan_t plan) {
  if (!plan) return PAI_OK;
  release(plan);
  return PAI_OK;
}

pai_status pai_window_probe(int H, double beta, double c, int n, const double* y, double* phi_out,
                            double* pred_err, double* fit_err) {
  if (H < 2 || H > kMaxH || !(c > 1.0) || !(beta * c > kPi) || !(beta * c <= kPi * (2 * c - 1) * (1 + 1e-12)) || n < 0)
    return PAI_ERR_INVALID_ARG;
  if (n > 0 && (!y || !phi_out)) return PAI_ERR_INVALID_ARG;
  const double peak = kb_phi(0.0, H, beta);
  for (int i = 0; i < n; ++i) phi_out[i] = kb_phi(y[i], H, beta) / peak;
  if (pred_err) *pred_err = predicted_error(0, c, H, beta);
  if (fit_err) {
    WindowPoly w;
    *fit_err = fit_window(0, H, beta, &w);
  }
  return PAI_OK;
}

pai_status pai_forward_plan(const pai_geometry* g, void* cuda_stream, pai_plan_t* out) {
  if (!g || !out) return PAI_ERR_INVALID_ARG;
  pai_geometry gi = *g;
  if (gi.dim == 2) {
    gi.ny = 1;
    gi.dy = 1.0;
  }
  PAI_TRY(validate(gi));
  if (gi.method != PAI_METHOD_KB && gi.method != PAI_METHOD_TSINC) return PAI_ERR_UNSUPPORTED;
  pai_geometry gb = gi;
  gb.nx = forward_box_extent(gi.nx, gi.dx, gi);
  if (gi.dim == 3) gb.ny = forward_box_extent(gi.ny, gi.dy, gi);
  gb.nz = forward_box_extent(gi.nz, gi.dz, gi);
  if (gb.nx > 16384 || gb.ny > 16384 || gb.nz > 8192) return PAI_ERR_UNSUPPORTED;
  pai_plan_s* P = nullptr;
  PAI_TRY(build_plan(&gb, 1, cuda_stream, &P, true));
  P->qimg = gi;
  const size_t box_img = (size_t)gb.nx * gb.ny * gb.nz, box_dat = (size_t)gb.nx * gb.ny * gb.nt;
  pai_status st = plan_malloc(P, (void**)&P->d_qin, box_img * sizeof(float));
  if (st == PAI_OK) st = plan_malloc(P, (void**)&P->d_qout, box_dat * sizeof(float));
  if (st != PAI_OK) {
    release(P);
    return st == PAI_ERR_CUDA ? PAI_ERR_OOM : st;
  }
  P->ws_bytes = (size_t)P->alloc_used;
  *out = P;
  return PAI_OK;
}

pai_status pai_forward_box(pai_plan_t plan, int* bx, int* by, int* bz) {
  if (!plan || !plan->qmode || !bx || !by || !bz) return PAI_ERR_INVALID_ARG;
  const pai_geometry& g = plan->probs[0].g;
  *bx = g.nx;
  *by = g.dim == 3 ? g.ny : 1;
  *bz = g.nz;
  return PAI_OK;
}

pai_status pai_forward_model(pai_plan_t plan, const float* d_f, float* d_p) {
  if (!plan || !d_f || !d_p) return PAI_ERR_INVALID_ARG;
  if (!plan->qmode) return PAI_ERR_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  const pai_geometry& gi = plan->qimg;
  const pai_geometry& gb = plan->probs[0].g;
  const int by = gb.dim == 3 ? gb.ny : 1, ny = gi.dim == 3 ? gi.ny : 1;
  const long long total = (long long)gb.nx * by * gb.nz;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
  const long long want = (total + 255) / 256;
  const int blocks = (int)std::min<long long>(want, (long long)std::max(sms, 1) * 16);
  pad_box_kernel<<<blocks, 256, 0, plan->stream>>>(d_f, plan->d_qin, gi.nx, ny, gi.nz, by, gb.nz, total);
  pai_status st = cuda_status(cudaGetLastError());
  if (st == PAI_OK) st = run(plan, plan->d_qin, plan->d_qout, true);
  if (st == PAI_OK && plan->d_cut) {
    // the data model g = w_cut * (Q f): the weight applied while the detector rows leave the box
    CutoffLaunch a{plan->d_qout, d_p, plan->d_cut, gi.nx, ny, gi.nt, by, plan->cut_R, gi.dim};
    st = cuda_status(launch_cutoff(a, plan->stream, sms));
    if (st == PAI_OK) plan->own_kernels += 1;
  } else if (st == PAI_OK) {
    // detectors x < nx (and y < ny) of the box data [bx][by][nt]
    const size_t row = (size_t)ny * gi.nt * sizeof(float), pitch = (size_t)by * gi.nt * sizeof(float);
    st = cuda_status(cudaMemcpy2DAsync(d_p, row, plan->d_qout, pitch, row, gi.nx, cudaMemcpyDeviceToDevice,
                                       plan->stream));
  }
  if (st == PAI_OK) plan->own_kernels += 1;  // the pad kernel (the rest is counted by run)
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_cutoff_table(int dim, double eps, double* table, int capacity, int* R) {
  if ((dim != 2 && dim != 3) || !(eps >= 1.0 && eps <= 256.0)) return PAI_ERR_INVALID_ARG;
  const int r = cutoff_radius(eps);
  if (R) *R = r;
  if (!table) return PAI_OK;
  long long n = 1;
  for (int a = 0; a < dim; ++a) n *= r + 1;
  if (capacity < n) return PAI_ERR_INVALID_ARG;
  std::vector<double> w;
  cutoff_table(dim, eps, w);
  std::copy(w.begin(), w.end(), table);
  return PAI_OK;
}

pai_status pai_set_cutoff(pai_plan_t plan, double eps) {
  if (!plan) return PAI_ERR_INVALID_ARG;
  if (plan->probs.size() != 1) return PAI_ERR_UNSUPPORTED;
  const pai_geometry& g = data_geometry(plan);
  if (eps != 0.0) {
    if (!(eps >= 1.0 && eps <= 256.0)) return PAI_ERR_INVALID_ARG;
    const int R = cutoff_radius(eps);
    const int ny = g.dim == 3 ? g.ny : 2 * R;
    if (g.nx < 2 * R || ny < 2 * R || g.nt < 2 * R) return PAI_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  pai_status st = cuda_status(cudaStreamSynchronize(plan->stream));
  if (st == PAI_OK) {
    cudaFree(plan->d_cut);
    plan->d_cut = nullptr;
    plan->cut_R = 0;
    plan->cut_eps = 0.0;
  }
  if (st == PAI_OK && eps != 0.0) {
    std::vector<double> w;
    cutoff_table(g.dim, eps, w);
    std::vector<float> wf(w.begin(), w.end());
    float* d = nullptr;
    st = plan_malloc(plan, (void**)&d, wf.size() * sizeof(float));
    if (st == PAI_OK) st = cuda_status(cudaMemcpy(d, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (st == PAI_OK) {
      plan->d_cut = d;
      plan->cut_R = cutoff_radius(eps);
      plan->cut_eps = eps;
    } else {
      cudaFree(d);
    }
  }
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

pai_status pai_cutoff(pai_plan_t plan, const float* d_in, float* d_out) {
  if (!plan || !d_in || !d_out || !plan->d_cut) return PAI_ERR_INVALID_ARG;
  const pai_geometry& g = data_geometry(plan);
  const int ny = g.dim == 3 ? g.ny : 1;
  const size_t bytes = (size_t)g.nx * ny * g.nt * sizeof(float);
  const char *a = reinterpret_cast<const char*>(d_in), *b = reinterpret_cast<const char*>(d_out);
  if (a != b && a < b + bytes && b < a + bytes) return PAI_ERR_INVALID_ARG;  // partial overlap
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != plan->device) cudaSetDevice(plan->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
  CutoffLaunch la{d_in, d_out, plan->d_cut, g.nx, ny, g.nt, ny, plan->cut_R, g.dim};
  pai_status st = cuda_status(launch_cutoff(la, plan->stream, sms));
  if (st == PAI_OK) plan->own_kernels += 1;
  if (prev != plan->device) cudaSetDevice(prev);
  return st;
}

const char* pai_status_string(pai_status s) {
  switch (s) {
    case PAI_OK: return "success";
    case PAI_ERR_INVALID_ARG: return "invalid argument";
    case PAI_ERR_UNSUPPORTED: return "unsupported configuration";
    case PAI_ERR_OOM: return "out of memory";
    case PAI_ERR_CUDA: return "CUDA error";
    case PAI_ERR_CUFFT: return "cuFFT error";
    case PAI_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
