// pai_noalloc.cu -- pai_spectrum_rows_noalloc: the fused NUFFT row stage
// (the same row kernel pai_spectrum launches) for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are off limits --
// a process whose device memory is already fully reserved by someone else's
// caching allocator or memory pool, or a real-time loop where an allocation
// (which may synchronise the device) is not allowed.  Such a caller passes its
// own input and output buffers; everything else the kernel needs (its
// descriptor, work list, work counter, twiddle table and window / node tables)
// lives in one file-scope static device array of PAI_NOALLOC_SCRATCH_BYTES
// bytes that every GPU which loads the library holds until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.  All calls share the array and it keeps the previous
// call's contents: each call rewrites every byte the kernel reads (the work
// counter included, which must start at zero) with one stream-ordered copy.
// Calls whose work overlaps on the GPU race on the array.
#include <cstring>
#include <mutex>

#include "pai_internal.h"

namespace {

constexpr size_t kScratchBytes = PAI_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* ptr = nullptr;  // device address of g_scratch on that device
};
DeviceScratch g_devices[kMaxDevices];
std::mutex g_mutex;
// Host image of the scratch contents, copied in one transfer per call.
alignas(256) unsigned char g_stage[kScratchBytes];

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" pai_status pai_spectrum_rows_noalloc(const pai_geometry* g_in, const float* d_pt, float* d_fhat,
                                                void* cuda_stream) {
  using namespace pai;
  if (!g_in) return PAI_ERR_INVALID_ARG;
  pai_geometry g = *g_in;
  if (g.dim == 2) {
    g.ny = 1;
    g.dy = 1.0;
  }
  int st = validate_geometry(g);
  if (st != PAI_OK) return (pai_status)st;
  if (g.method != PAI_METHOD_KB) return PAI_ERR_UNSUPPORTED;
  ProblemParams pp;
  st = choose_problem_params(g, pp);
  if (st != PAI_OK) return (pai_status)st;
  const double kPi = 3.14159265358979323846;
  const double alpha_eff = pp.beta * pp.c_eff;
  if (!(alpha_eff > kPi) || !(alpha_eff < kPi * (2 * pp.c_eff - 1))) return PAI_ERR_INVALID_ARG;

  // launch shape: the same rule as a single-problem plan without the tuner
  const int tpr = pp.M / kElemsPerThread;
  int threads = tpr > 512 ? tpr : 512;
  if (threads > 1024) return PAI_ERR_UNSUPPORTED;
  const int rpc = threads / tpr;

  RowProblem rp{};
  fill_row_scalars(g, pp.M, rp);
  rp.rpc = rpc;
  const int rows = rp.rows;
  const int nitems = (rows + rpc - 1) / rpc;

  // scratch layout (256-byte aligned sections)
  size_t off = 0;
  const size_t o_prob = off;  off = align256(off + sizeof(RowProblem));
  const size_t o_items = off; off = align256(off + (size_t)nitems * sizeof(WorkItem));
  const size_t o_count = off; off = align256(off + sizeof(int));
  const size_t o_tw = off;    off = align256(off + (size_t)twiddle_entries(pp.M) * sizeof(float2));
  const size_t o_pre = off;   off = align256(off + (size_t)g.nt * sizeof(float));
  const size_t o_rows = off;  off = align256(off + (size_t)rows * 2 * sizeof(float));
  const size_t o_zt = off;    off = align256(off + (size_t)(g.nz / 2 + 1) * 4 * sizeof(float));
  const size_t used = off;
  if (used > kScratchBytes) return PAI_ERR_UNSUPPORTED;
  // the pointers are checked after the size, so an oversized geometry is
  // rejected on the host whatever the caller passes
  if (!d_pt || !d_fhat) return PAI_ERR_INVALID_ARG;

  WindowPoly poly;
  if (!(fit_window(0, pp.H, pp.beta, &poly) < 1e-6)) return PAI_ERR_UNSUPPORTED;

  std::lock_guard<std::mutex> lock(g_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAI_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PAI_ERR_UNSUPPORTED;
  DeviceScratch& ds = g_devices[dev];
  if (!ds.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return PAI_ERR_CUDA;
    ds.ptr = static_cast<unsigned char*>(p);
    ds.ready = true;
  }
  unsigned char* base = ds.ptr;

  // host image of the scratch
  std::memset(g_stage, 0, used);
  rp.pt = reinterpret_cast<const float2*>(d_pt);
  rp.fh = reinterpret_cast<float2*>(d_fhat);
  rp.prescale = reinterpret_cast<const float*>(base + o_pre);
  rp.rowS = reinterpret_cast<const float2*>(base + o_rows);
  rp.zt = reinterpret_cast<const float4*>(base + o_zt);
  std::memcpy(g_stage + o_prob, &rp, sizeof(rp));
  WorkItem* items = reinterpret_cast<WorkItem*>(g_stage + o_items);
  for (int i = 0; i < nitems; ++i) {
    items[i].problem = 0;
    items[i].row0 = i * rpc;
  }
  *reinterpret_cast<int*>(g_stage + o_count) = 0;  // the work counter starts at zero on every call
  twiddle_table(pp.M, reinterpret_cast<float2*>(g_stage + o_tw));
  fill_row_tables(g, pp.c_eff, pp.H, pp.beta, reinterpret_cast<float*>(g_stage + o_pre),
                  reinterpret_cast<float*>(g_stage + o_rows), reinterpret_cast<float*>(g_stage + o_zt));

  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemcpyAsync(base, g_stage, used, cudaMemcpyHostToDevice, s) != cudaSuccess) return PAI_ERR_CUDA;

  RowLaunch L{};
  L.problems = reinterpret_cast<const RowProblem*>(base + o_prob);
  L.items = reinterpret_cast<const WorkItem*>(base + o_items);
  L.nitems = nitems;
  L.counter = reinterpret_cast<int*>(base + o_count);
  L.tw = reinterpret_cast<const float2*>(base + o_tw);
  L.Mmax = pp.M;
  L.H = pp.H;
  const size_t smem = row_fft_region_bytes(threads, pp.M);
  L.fft_region = (int)(smem / sizeof(float2));
  const int occ = row_kernel_max_ctas_per_sm(0, threads, smem, pp.H);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PAI_ERR_CUDA;
  if (occ < 1) return PAI_ERR_UNSUPPORTED;
  const int ctas = nitems < occ * sms ? nitems : occ * sms;
  if (launch_row_forward(L, poly, threads, ctas, smem, s) != cudaSuccess) return PAI_ERR_CUDA;
  return PAI_OK;
}
