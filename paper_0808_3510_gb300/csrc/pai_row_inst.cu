// pai_row_inst.cu -- explicit instantiation of the row kernels for a range of
// half tap counts H, compiled several times with different ranges so the
// instantiations build in parallel.  PAI_HLO / PAI_HHI select the range.
#include "pai_row_kernels.cuh"

#ifndef PAI_HLO
#define PAI_HLO 2
#define PAI_HHI 12
#endif
#define PAI_CAT2(a, b) a##b
#define PAI_CAT(a, b) PAI_CAT2(a, b)
#define PAI_FN(name) PAI_CAT(PAI_CAT(name, _h), PAI_HLO)

namespace pai {

template <int H>
static cudaError_t fwd_h(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                         cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(row_forward_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  row_forward_kernel<H><<<ctas, threads, smem, s>>>(L, w);
  return cudaGetLastError();
}

template <int H>
static cudaError_t adj_h(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                         cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(row_adjoint_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  row_adjoint_kernel<H><<<ctas, threads, smem, s>>>(L, w);
  return cudaGetLastError();
}

template <int H>
static int occ_h(bool adjoint, int threads, size_t smem) {
  int n = 0;
  if (adjoint) {
    if (cudaFuncSetAttribute(row_adjoint_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, row_adjoint_kernel<H>, threads, smem) != cudaSuccess)
      return 0;
  } else {
    if (cudaFuncSetAttribute(row_forward_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, row_forward_kernel<H>, threads, smem) != cudaSuccess)
      return 0;
  }
  return n;
}

#define PAI_ONE(F, HH, ...) \
  if (H == HH && HH >= PAI_HLO && HH <= PAI_HHI) return F<(HH >= PAI_HLO && HH <= PAI_HHI ? HH : PAI_HLO)>(__VA_ARGS__);
#define PAI_ALL(F, ...)                                                                          \
  PAI_ONE(F, 2, __VA_ARGS__) PAI_ONE(F, 3, __VA_ARGS__) PAI_ONE(F, 4, __VA_ARGS__)               \
  PAI_ONE(F, 5, __VA_ARGS__) PAI_ONE(F, 6, __VA_ARGS__) PAI_ONE(F, 7, __VA_ARGS__)               \
  PAI_ONE(F, 8, __VA_ARGS__) PAI_ONE(F, 9, __VA_ARGS__) PAI_ONE(F, 10, __VA_ARGS__)              \
  PAI_ONE(F, 11, __VA_ARGS__) PAI_ONE(F, 12, __VA_ARGS__)

// Returns cudaErrorNotSupported when H is outside this unit's range.
cudaError_t PAI_FN(row_forward)(int H, const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                                cudaStream_t s) {
  PAI_ALL(fwd_h, L, w, threads, ctas, smem, s)
  return cudaErrorNotSupported;
}

cudaError_t PAI_FN(row_adjoint)(int H, const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                                cudaStream_t s) {
  PAI_ALL(adj_h, L, w, threads, ctas, smem, s)
  return cudaErrorNotSupported;
}

int PAI_FN(row_occupancy)(int H, bool adjoint, int threads, size_t smem) {
  PAI_ALL(occ_h, adjoint, threads, smem)
  return -1;
}

}  // namespace pai
