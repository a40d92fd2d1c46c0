// The α-scaling, the forward time DFT and Chebyshev step k = 1 in one launch (2D, FP32); the
// body, with its bytes and its tiling, is ends::dft_first_body (cheb_ends.cuh).
#include "cheb_ends.cuh"

namespace aao {

namespace {

template <int ELL>
__global__ void __launch_bounds__(256) k_dft_first(GridDesc g, const double* __restrict__ r,
                                                   const double* __restrict__ rscale, float* __restrict__ bhat,
                                                   float* __restrict__ x2, const float* __restrict__ cx,
                                                   const float* __restrict__ cy, const __grid_constant__ DftArgs<float> da,
                                                   const __grid_constant__ StepArgs<float> sa) {
  extern __shared__ __align__(16) float sb[];
  __shared__ float gs[ELL];
  ends::dft_first_body<ELL>(g, blockIdx.x, blockIdx.y, r, rscale, bhat, x2, cx, cy, da, sa, sb, gs);
}

template <int ELL>
cudaError_t launch_dft_first_ell(const GridDesc& g, const double* r, const double* rscale, float* bhat, float* x2,
                                 const float* cx, const float* cy, const DftArgs<float>& da,
                                 const StepArgs<float>& sa, cudaStream_t s) {
  const size_t smem = sizeof(float) * ends::dft_first_smem_floats(ELL);
  cudaError_t e = cudaFuncSetAttribute(k_dft_first<ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((g.n0 + ends::kFX - 1) / ends::kFX), (unsigned)((g.n1 + ends::kFY - 1) / ends::kFY), 1);
  k_dft_first<ELL><<<grid, dim3(32, ends::kFY, 1), smem, s>>>(g, r, rscale, bhat, x2, cx, cy, da, sa);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dft_first(const GridDesc& g, int ell, const double* r, const double* rscale, float* bhat,
                             float* x2, const float* cx, const float* cy, const DftArgs<float>& da,
                             const StepArgs<float>& sa, cudaStream_t s) {
  if (g.n2 != 1 || g.n0 % 4 != 0 || g.n1 > 65535 * ends::kFY ||
      ((reinterpret_cast<uintptr_t>(bhat) | reinterpret_cast<uintptr_t>(x2) | reinterpret_cast<uintptr_t>(cx) |
        reinterpret_cast<uintptr_t>(cy)) & 15) != 0)
    return cudaErrorInvalidValue;
  switch (ell) {
#define AAO_DF(L) \
  case L:         \
    return launch_dft_first_ell<L>(g, r, rscale, bhat, x2, cx, cy, da, sa, s);
    AAO_DF(4)
    AAO_DF(6)
    AAO_DF(8)
    AAO_DF(10)
    AAO_DF(12)
    AAO_DF(14)
    AAO_DF(16)
#undef AAO_DF
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace aao
