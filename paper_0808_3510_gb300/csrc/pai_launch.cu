// pai_launch.cu -- dispatch of the row kernels to the instantiation units.
#include "pai_internal.h"

namespace pai {

#define PAI_UNIT(lo)                                                                                          \
  cudaError_t row_forward_h##lo(int, const RowLaunch&, const WindowPoly&, int, int, size_t, cudaStream_t, bool); \
  cudaError_t row_adjoint_h##lo(int, const RowLaunch&, const WindowPoly&, int, int, size_t, cudaStream_t, bool); \
  int row_occupancy_h##lo(int, int, int, size_t, bool);
PAI_UNIT(2)
PAI_UNIT(5)
PAI_UNIT(7)
PAI_UNIT(9)

size_t row_fft_region_bytes(int threads, int M) {
  const int tpr = M / kElemsPerThread;
  return (size_t)(threads / tpr) * (size_t)row_slot_stride(M) * sizeof(float2);
}

cudaError_t launch_row_forward(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                               cudaStream_t s, bool zf) {
  const int H = L.H;
  if (H < 5) return row_forward_h2(H, L, w, threads, ctas, smem, s, zf);
  if (H < 7) return row_forward_h5(H, L, w, threads, ctas, smem, s, zf);
  if (H < 9) return row_forward_h7(H, L, w, threads, ctas, smem, s, zf);
  return row_forward_h9(H, L, w, threads, ctas, smem, s, zf);
}

cudaError_t launch_row_adjoint(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                               cudaStream_t s, bool zf) {
  const int H = L.H;
  if (H < 5) return row_adjoint_h2(H, L, w, threads, ctas, smem, s, zf);
  if (H < 7) return row_adjoint_h5(H, L, w, threads, ctas, smem, s, zf);
  if (H < 9) return row_adjoint_h7(H, L, w, threads, ctas, smem, s, zf);
  return row_adjoint_h9(H, L, w, threads, ctas, smem, s, zf);
}

int row_kernel_max_ctas_per_sm(int kind, int threads, size_t smem, int H, bool zf) {
  if (H < 5) return row_occupancy_h2(H, kind, threads, smem, zf);
  if (H < 7) return row_occupancy_h5(H, kind, threads, smem, zf);
  if (H < 9) return row_occupancy_h7(H, kind, threads, smem, zf);
  return row_occupancy_h9(H, kind, threads, smem, zf);
}

}  // namespace pai
