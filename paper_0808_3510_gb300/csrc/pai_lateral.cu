// pai_lateral.cu -- FFTs along a strided axis for power-of-two lengths:
// the lateral transforms of Algorithm 2 (Eq. fft-1a forward, the lateral part
// of Eq. fft-1 inverse) and their transposes.
//
// Data are viewed as A[outer][L][C]: the transform runs along the middle axis
// (length L, element stride C) for every contiguous column c < C and every
// outer index.  The axis is the slow one, so each CTA takes a tile of columns:
//   * the tile is read and written in full 32-byte sectors;
//   * FP column FFTs of length L run in shared memory with the same Stockham
//     passes as the row kernels (16 values per thread per pass);
//   * real-to-complex: columns c, c+1 are paired as z = a + i b (two real
//     FFTs for one complex FFT) and separated after the transform,
//     A[k] = (Z[k] + conj Z[-k]) / 2, B[k] = (Z[k] - conj Z[-k]) / (2i);
//   * complex-to-real: the two half spectra are merged as Z = A + i B over the
//     full range (Hermitian extension, imaginary parts of the self-conjugate
//     bins k = 0, L/2 ignored as in any C2R), inverse transformed, and the
//     real / imaginary parts are the two real columns.
// All transforms are unnormalised.
#include "pai_row_kernels.cuh"

namespace pai {

// Complex values per FFT slot: padded layout plus a shift of 4 values so the
// FP slots start in different shared-memory banks.
__host__ __device__ inline int lateral_slot(int L) { return L + (L >> 5) + 4; }

enum : int { kLatR2C = 0, kLatC2R = 1, kLatC2C = 2, kLatC2CInv = 3 };

// The values a thread loads, column elements x0 + i L/16 (i = 0..15), are the
// inputs of butterfly x0 of the first radix-16 Stockham pass (Ns = 1): that
// pass runs on them in registers and writes its outputs 16 x0 + r in the
// padded layout, ready for fft_rest.
template <bool INV>
__device__ __forceinline__ void first_pass_regs(float2* Z, float2 (&z)[kElemsPerThread], int x0) {
  dft_reg<kElemsPerThread, INV>(z);
#pragma unroll
  for (int r = 0; r < kElemsPerThread; ++r) Z[PADI(x0 * kElemsPerThread + r)] = z[r];
}

template <int KIND, int FP>
__global__ void __launch_bounds__(1024) lateral_kernel(const void* vin, void* vout, int L,
                                                       int mshift, int C, long long in_outer, long long out_outer,
                                                       const float2* __restrict__ tw, int twstride) {
  extern __shared__ float2 smem[];
  constexpr bool kInv = (KIND == kLatC2R || KIND == kLatC2CInv);
  const int tpr = L / kElemsPerThread;
  const int S = lateral_slot(L);
  const int T = blockDim.x;
  const int f = threadIdx.x % FP;  // column group of this thread in the load / store phases
  const int x0 = threadIdx.x / FP;
  const int xs = T / FP;           // = L / 16
  const int half = L >> 1;
  // columns handled by this CTA: real kinds take 2 FP real columns, complex kinds FP
  constexpr int CPT = (KIND == kLatC2C || KIND == kLatC2CInv) ? FP : 2 * FP;
  const int c0 = blockIdx.x * CPT;
  const long long ob = blockIdx.y;
  float2* Z = smem + f * S;

  // ---- load -------------------------------------------------------------
  if (KIND == kLatR2C) {
    const float* in = static_cast<const float*>(vin) + ob * in_outer;
    const bool live = c0 + 2 * f < C;  // C even: pairs are whole
    const float2* src = reinterpret_cast<const float2*>(in + (size_t)x0 * C + c0) + f;
    float2 z[kElemsPerThread];
#pragma unroll
    for (int i = 0; i < kElemsPerThread; ++i)
      z[i] = live ? __ldg(src + (size_t)i * xs * (C / 2)) : make_float2(0.f, 0.f);
    first_pass_regs<false>(Z, z, x0);
  } else if (KIND == kLatC2C || KIND == kLatC2CInv) {
    const float2* in = static_cast<const float2*>(vin) + ob * in_outer;
    const bool live = c0 + f < C;
    const float2* src = in + (size_t)x0 * C + c0 + f;
    float2 z[kElemsPerThread];
#pragma unroll
    for (int i = 0; i < kElemsPerThread; ++i)  // plain loads: the C2C may run in place
      z[i] = live ? src[(size_t)i * xs * C] : make_float2(0.f, 0.f);
    first_pass_regs<kInv>(Z, z, x0);
  } else {  // C2R: rows k = 0 .. L/2 of two complex columns per slot
    const float2* in = static_cast<const float2*>(vin) + ob * in_outer;
    const bool live = c0 + 2 * f < C;
    // rows k = x0 + i xs, i = 0 .. 8 (the last only for x0 = 0): loads first
    constexpr int NK = kElemsPerThread / 2 + 1;
    float4 abv[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int k = x0 + i * xs;
      abv[i] = (live && k <= half) ? __ldg(reinterpret_cast<const float4*>(in + (size_t)k * C + c0 + 2 * f))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int k = x0 + i * xs;
      if (k > half) break;
      const float4 ab = abv[i];
      if (k == 0 || k == half) {
        // self-conjugate bins: only the real parts enter a C2R
        Z[PADI(k)] = make_float2(ab.x, ab.z);
      } else {
        // Z[k] = A[k] + i B[k];  Z[L-k] = conj A[k] + i conj B[k]
        Z[PADI(k)] = make_float2(ab.x - ab.w, ab.y + ab.z);
        Z[PADI(L - k)] = make_float2(ab.x + ab.w, ab.z - ab.y);
      }
    }
  }
  __syncthreads();
  {
    const int slot = threadIdx.x / tpr;
    const int lane = threadIdx.x - slot * tpr;
    if (KIND == kLatC2R) fft_smem<kInv, kLayoutFlat>(smem + slot * S, L, mshift, lane, tpr, tw, twstride);
    else fft_rest<kInv, kLayoutFlat>(smem + slot * S, L, mshift, lane, tpr, tw, twstride);
  }

  // ---- store ------------------------------------------------------------
  if (KIND == kLatR2C) {
    float2* out = static_cast<float2*>(vout) + ob * out_outer;
    if (c0 + 2 * f < C) {
      for (int k = x0; k <= half; k += xs) {
        const float2 a = Z[k];
        const float2 b = Z[(L - k) & (L - 1)];
        const float4 o = make_float4(0.5f * (a.x + b.x), 0.5f * (a.y - b.y), 0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
        *reinterpret_cast<float4*>(out + (size_t)k * C + c0 + 2 * f) = o;
      }
    }
  } else if (KIND == kLatC2C || KIND == kLatC2CInv) {
    float2* out = static_cast<float2*>(vout) + ob * out_outer;
    if (c0 + f < C) {
#pragma unroll
      for (int i = 0; i < kElemsPerThread; ++i) {
        const int x = x0 + i * xs;
        out[(size_t)x * C + c0 + f] = Z[x];
      }
    }
  } else {
    float* out = static_cast<float*>(vout) + ob * out_outer;
    if (c0 + 2 * f < C) {
#pragma unroll
      for (int i = 0; i < kElemsPerThread; ++i) {
        const int x = x0 + i * xs;
        *reinterpret_cast<float2*>(out + (size_t)x * C + c0 + 2 * f) = Z[x];
      }
    }
  }
}

int lateral_slots_per_cta(int L) {
  // 8 slots for 256- and 512-point columns (a 256^3 gradient step's four
  // lateral stages gained 22 us over 4; 128-point columns lost with 8)
  int fp = (L >= 256 && L <= 512) ? 8 : 4;
  while (fp > 1 && fp * (L / kElemsPerThread) > 1024) fp >>= 1;
  return fp;
}

size_t lateral_smem_bytes(int L) { return (size_t)lateral_slots_per_cta(L) * lateral_slot(L) * sizeof(float2); }

bool lateral_supported(int L, int C) {
  if (L < 32 || (L & (L - 1)) != 0) return false;
  if ((L / kElemsPerThread) > 1024) return false;
  if (C % 2 != 0) return false;
  return lateral_smem_bytes(L) <= 200 * 1024;
}

template <int KIND, int FP>
static cudaError_t lat_launch(const void* in, void* out, int L, int C, int outer, long long in_outer,
                              long long out_outer, const float2* tw, int twstride, cudaStream_t s) {
  const size_t smem = lateral_smem_bytes(L);
  cudaError_t e =
      cudaFuncSetAttribute(lateral_kernel<KIND, FP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int mshift = 0;
  while ((1 << mshift) < L) ++mshift;
  const int threads = FP * (L / kElemsPerThread);
  constexpr int CPT = (KIND == kLatC2C || KIND == kLatC2CInv) ? FP : 2 * FP;
  dim3 grid((C + CPT - 1) / CPT, outer);
  lateral_kernel<KIND, FP><<<grid, threads, smem, s>>>(in, out, L, mshift, C, in_outer, out_outer, tw, twstride);
  return cudaGetLastError();
}

template <int KIND>
static cudaError_t lat_dispatch(const void* in, void* out, int L, int C, int outer, long long in_outer,
                                long long out_outer, const float2* tw, int twstride, cudaStream_t s) {
  switch (lateral_slots_per_cta(L)) {
    case 8: return lat_launch<KIND, 8>(in, out, L, C, outer, in_outer, out_outer, tw, twstride, s);
    case 4: return lat_launch<KIND, 4>(in, out, L, C, outer, in_outer, out_outer, tw, twstride, s);
    case 2: return lat_launch<KIND, 2>(in, out, L, C, outer, in_outer, out_outer, tw, twstride, s);
    default: return lat_launch<KIND, 1>(in, out, L, C, outer, in_outer, out_outer, tw, twstride, s);
  }
}

// out[o][k][c] = sum_x e^{-2 pi i k x / L} in[o][x][c], k = 0..L/2.
cudaError_t launch_lateral_r2c(const float* in, float2* out, int L, int C, int outer, const float2* tw, int twstride,
                               cudaStream_t s) {
  return lat_dispatch<kLatR2C>(in, out, L, C, outer, (long long)L * C, (long long)(L / 2 + 1) * C, tw, twstride, s);
}

// out[o][x][c] = sum over the Hermitian extension of in[o][k][c] of e^{+2 pi i k x / L} (unnormalised C2R).
cudaError_t launch_lateral_c2r(const float2* in, float* out, int L, int C, int outer, const float2* tw, int twstride,
                               cudaStream_t s) {
  return lat_dispatch<kLatC2R>(in, out, L, C, outer, (long long)(L / 2 + 1) * C, (long long)L * C, tw, twstride, s);
}

// out[o][k][c] = sum_x e^{-+2 pi i k x / L} in[o][x][c]; in place allowed (each CTA owns its columns).
cudaError_t launch_lateral_c2c(const float2* in, float2* out, int L, int C, int outer, bool inverse, const float2* tw,
                               int twstride, cudaStream_t s) {
  if (inverse)
    return lat_dispatch<kLatC2CInv>(in, out, L, C, outer, (long long)L * C, (long long)L * C, tw, twstride, s);
  return lat_dispatch<kLatC2C>(in, out, L, C, outer, (long long)L * C, (long long)L * C, tw, twstride, s);
}

// In-place FFT of contiguous lines (the depth transform of Eq. fft-1 and its
// transpose): line r occupies data[r L .. r L + L).  One row slot of L/16
// threads per line; the first pass reads straight from global memory.
template <bool INV>
__global__ void __launch_bounds__(1024) rows_fft_kernel(float2* data, int L, int mshift, int rows,
                                                        const float2* __restrict__ tw, int twstride) {
  extern __shared__ float2 smem[];
  const int tpr = L / kElemsPerThread;
  const int slot = threadIdx.x / tpr;
  const int lane = threadIdx.x - slot * tpr;
  const int rpc = blockDim.x / tpr;
  const int row = blockIdx.x * rpc + slot;
  const bool valid = row < rows;
  float2* X = smem + slot * lateral_slot(L);
  float2* line = data + (size_t)(valid ? row : 0) * L;
  {
    constexpr int R = 16;
    const int LR = L / R;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = line[lane + r * LR];  // plain loads: the transform is in place
    dft_reg<R, INV>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = lane * R + r;
      X[PADI(idx)] = v[r];
    }
  }
  __syncthreads();
  fft_rest<INV, kLayoutFlat>(X, L, mshift, lane, tpr, tw, twstride);
  if (valid)
    for (int z = lane; z < L; z += tpr) line[z] = X[z];
}

cudaError_t launch_rows_c2c(float2* data, int L, int rows, bool inverse, const float2* tw, int twstride,
                            cudaStream_t s) {
  if (L < 32 || (L & (L - 1)) != 0 || L / kElemsPerThread > 1024) return cudaErrorInvalidValue;
  int mshift = 0;
  while ((1 << mshift) < L) ++mshift;
  const int tpr = L / kElemsPerThread;
  const int threads = tpr > 128 ? tpr : 128;  // (128 measured 1.5 us faster than 256 per 256^3 depth stage)
  const int rpc = threads / tpr;
  const size_t smem = (size_t)rpc * lateral_slot(L) * sizeof(float2);
  const int ctas = (rows + rpc - 1) / rpc;
  cudaError_t e;
  if (inverse) {
    e = cudaFuncSetAttribute(rows_fft_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rows_fft_kernel<true><<<ctas, threads, smem, s>>>(data, L, mshift, rows, tw, twstride);
  } else {
    e = cudaFuncSetAttribute(rows_fft_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rows_fft_kernel<false><<<ctas, threads, smem, s>>>(data, L, mshift, rows, tw, twstride);
  }
  return cudaGetLastError();
}

}  // namespace pai
