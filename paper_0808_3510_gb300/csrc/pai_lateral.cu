// pai_lateral.cu -- lateral real-to-complex FFT of the detector data
// (Eq. fft-1a) for line detectors whose detector count nx is a power of two.
//
// p[x][n] (FP32, time n fastest) -> pt[k][n] (complex64), k = 0 .. nx/2, the
// unnormalised DFT over x for every time sample n.  The transform runs along
// the slow axis, so each CTA takes a tile of 2*FP consecutive time columns:
//   * the tile is read with full 32-byte sectors (2*FP floats per detector);
//   * columns are paired into FP complex sequences z = p[:, n] + i p[:, n+1]
//     (two real FFTs for the price of one complex FFT);
//   * FP complex FFTs of length nx run in shared memory with the same
//     Stockham passes as the row kernels;
//   * the pairs are separated, P_n[k] = (Z[k] + conj Z[-k]) / 2 and
//     P_{n+1}[k] = (Z[k] - conj Z[-k]) / (2i), and written as 16-byte stores.
#include "pai_row_kernels.cuh"

namespace pai {

// Complex values per FFT slot: padded layout plus a shift of 4 values so the
// FP slots start in different shared-memory banks.
__host__ __device__ inline int lateral_slot(int nx) { return nx + (nx >> 5) + 4; }

template <int FP>
__global__ void __launch_bounds__(1024) lateral_r2c_kernel(const float* __restrict__ p, float2* __restrict__ pt,
                                                           int nx, int mshift, int nt, const float2* __restrict__ tw,
                                                           int twstride) {
  extern __shared__ float2 smem[];
  const int tpr = nx / kElemsPerThread;
  const int S = lateral_slot(nx);
  const int n0 = blockIdx.x * (2 * FP);
  const int T = blockDim.x;
  // load the tile: thread t takes column pair f = t % FP of detectors x = t / FP + i T / FP
  {
    // T / FP = nx / 16 threads per column pair, so each thread loads exactly
    // kElemsPerThread detectors: issue all loads before the shared stores
    const int f = threadIdx.x % FP;
    const int x0 = threadIdx.x / FP;
    const int xs = T / FP;
    const bool live = 2 * f < nt - n0;  // columns left (>= 2, even)
    const float2* src = reinterpret_cast<const float2*>(p + (size_t)x0 * nt + n0) + f;
    float2 z[kElemsPerThread];
#pragma unroll
    for (int i = 0; i < kElemsPerThread; ++i)
      z[i] = live ? __ldg(src + (size_t)i * xs * (nt / 2)) : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < kElemsPerThread; ++i) smem[f * S + PADI(x0 + i * xs)] = z[i];
  }
  __syncthreads();
  {
    const int slot = threadIdx.x / tpr;
    const int lane = threadIdx.x - slot * tpr;
    fft_smem<false, kLayoutFlat>(smem + slot * S, nx, mshift, lane, tpr, tw, twstride);
  }
  // separate the paired columns and store pt[k][n0 + 2f .. n0 + 2f + 1]
  {
    const int f = threadIdx.x % FP;
    const int k0 = threadIdx.x / FP;
    const int ks = T / FP;
    const int half = nx >> 1;
    const float2* Z = smem + f * S;
    if (2 * f < nt - n0) {
      for (int k = k0; k <= half; k += ks) {
        const float2 a = Z[k];
        const float2 b = Z[(nx - k) & (nx - 1)];
        // P_even = (a + conj b)/2, P_odd = (a - conj b)/(2i)
        const float4 o = make_float4(0.5f * (a.x + b.x), 0.5f * (a.y - b.y), 0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
        *reinterpret_cast<float4*>(pt + (size_t)k * nt + n0 + 2 * f) = o;
      }
    }
  }
}

int lateral_pairs_per_cta(int nx) {
  int fp = 4;
  while (fp > 1 && fp * (nx / kElemsPerThread) > 1024) fp >>= 1;
  return fp;
}

size_t lateral_smem_bytes(int nx) { return (size_t)lateral_pairs_per_cta(nx) * lateral_slot(nx) * sizeof(float2); }

bool lateral_supported(int nx, int nt) {
  if (nx < 32 || (nx & (nx - 1)) != 0) return false;
  if ((nx / kElemsPerThread) > 1024) return false;
  if (nt % 2 != 0) return false;
  return lateral_smem_bytes(nx) <= 200 * 1024;
}

template <int FP>
static cudaError_t lat_launch(const float* p, float2* pt, int nx, int nt, const float2* tw, int twstride,
                              cudaStream_t s) {
  const size_t smem = lateral_smem_bytes(nx);
  cudaError_t e = cudaFuncSetAttribute(lateral_r2c_kernel<FP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int mshift = 0;
  while ((1 << mshift) < nx) ++mshift;
  const int threads = FP * (nx / kElemsPerThread);
  const int ctas = (nt + 2 * FP - 1) / (2 * FP);
  lateral_r2c_kernel<FP><<<ctas, threads, smem, s>>>(p, pt, nx, mshift, nt, tw, twstride);
  return cudaGetLastError();
}

// pt[k][n] = sum_x e^{-2 pi i k x / nx} p[x][n], k = 0..nx/2 (complex64, stride nt).
// tw: e^{-2 pi i m / (nx twstride)}, m < nx twstride.
cudaError_t launch_lateral_r2c(const float* p, float2* pt, int nx, int nt, const float2* tw, int twstride,
                               cudaStream_t s) {
  switch (lateral_pairs_per_cta(nx)) {
    case 4: return lat_launch<4>(p, pt, nx, nt, tw, twstride, s);
    case 2: return lat_launch<2>(p, pt, nx, nt, tw, twstride, s);
    default: return lat_launch<1>(p, pt, nx, nt, tw, twstride, s);
  }
}

}  // namespace pai
