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

template <typename K>
static cudaError_t launch_k(K kernel, const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                           cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<ctas, threads, smem, s>>>(L, w);
  return cudaGetLastError();
}

template <typename K>
static int occ_k(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) return 0;
  return n;
}

template <int H>
static cudaError_t fwd_h(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem, cudaStream_t s,
                         bool zf) {
  if (zf) return launch_k(row_forward_kernel<H, true>, L, w, threads, ctas, smem, s);
  return L.paired ? launch_k(row_forward_kernel<H, false, true>, L, w, threads, ctas, smem, s)
                  : launch_k(row_forward_kernel<H, false>, L, w, threads, ctas, smem, s);
}

template <int H>
static cudaError_t adj_h(const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem, cudaStream_t s,
                         bool zf) {
  if (L.spread_mode == 3)
    return zf ? launch_k(row_adjoint_pairs_kernel<H, true, false>, L, w, threads, ctas, smem, s)
              : launch_k(row_adjoint_pairs_kernel<H, false, false>, L, w, threads, ctas, smem, s);
  if (L.spread_mode == 4)
    return zf ? launch_k(row_adjoint_pairs_kernel<H, true, true>, L, w, threads, ctas, smem, s)
              : launch_k(row_adjoint_pairs_kernel<H, false, true>, L, w, threads, ctas, smem, s);
  return zf ? launch_k(row_adjoint_kernel<H, true>, L, w, threads, ctas, smem, s)
            : launch_k(row_adjoint_kernel<H, false>, L, w, threads, ctas, smem, s);
}

// kind: 0 forward, 1 adjoint, 2 adjoint with the pair spread, 3 forward (paired layout), 4 adjoint with the
// atomic pair spread
template <int H>
static int occ_h(int kind, int threads, size_t smem, bool zf) {
  if (kind == 2)
    return zf ? occ_k(row_adjoint_pairs_kernel<H, true, false>, threads, smem)
              : occ_k(row_adjoint_pairs_kernel<H, false, false>, threads, smem);
  if (kind == 4)
    return zf ? occ_k(row_adjoint_pairs_kernel<H, true, true>, threads, smem)
              : occ_k(row_adjoint_pairs_kernel<H, false, true>, threads, smem);
  if (kind == 3) return occ_k(row_forward_kernel<H, false, true>, threads, smem);
  if (kind == 1)
    return zf ? occ_k(row_adjoint_kernel<H, true>, threads, smem) : occ_k(row_adjoint_kernel<H, false>, threads, smem);
  return zf ? occ_k(row_forward_kernel<H, true>, threads, smem) : occ_k(row_forward_kernel<H, false>, threads, smem);
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
                                cudaStream_t s, bool zf) {
  PAI_ALL(fwd_h, L, w, threads, ctas, smem, s, zf)
  return cudaErrorNotSupported;
}

cudaError_t PAI_FN(row_adjoint)(int H, const RowLaunch& L, const WindowPoly& w, int threads, int ctas, size_t smem,
                                cudaStream_t s, bool zf) {
  PAI_ALL(adj_h, L, w, threads, ctas, smem, s, zf)
  return cudaErrorNotSupported;
}

int PAI_FN(row_occupancy)(int H, int kind, int threads, size_t smem, bool zf) {
  PAI_ALL(occ_h, kind, threads, smem, zf)
  return -1;
}

}  // namespace pai
