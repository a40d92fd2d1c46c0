// Chebyshev step kernels for 2D grids (instantiations; bodies in cheb_kernels.cuh).
#include "cheb_kernels.cuh"
#include "cheb_pair.cuh"
#include "cheb_quad.cuh"

namespace aao {
template cudaError_t launch_step_dim<float, 2>(const GridDesc&, int, int, int, bool, const float*, const float*,
                                               const float*, const float*, const float*, float*, double*,
                                               const StepArgs<float>&, const IdftArgs<float>&, cudaStream_t);
template cudaError_t launch_step_dim<double, 2>(const GridDesc&, int, int, int, bool, const double*,
                                                const double*, const double*, const double*, const double*,
                                                double*, double*, const StepArgs<double>&,
                                                const IdftArgs<double>&, cudaStream_t);

cudaError_t launch_pair(const GridDesc& g, int ell, int psrc, const float* cx, const float* cy, const float* bhat,
                        const float* xk, const float* xkm1, float* out1, float* out2, const StepArgs<float>& s1,
                        const StepArgs<float>& s2, cudaStream_t s) {
  switch (ell) {
#define AAO_PAIR_CASE(L) \
  case L:                \
    return launch_pair_ell<L>(g, psrc, cx, cy, bhat, xk, xkm1, out1, out2, s1, s2, s);
    AAO_PAIR_CASE(4)
    AAO_PAIR_CASE(6)
    AAO_PAIR_CASE(8)
    AAO_PAIR_CASE(10)
    AAO_PAIR_CASE(12)
    AAO_PAIR_CASE(14)
    AAO_PAIR_CASE(16)
#undef AAO_PAIR_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_quad(const GridDesc& g, int ell, int psrc, const float* cx, const float* cy, const float* bhat,
                        const float* xk, const float* xkm1, float* out3, float* out4, const QuadSteps& qs,
                        cudaStream_t s) {
  switch (ell) {
#define AAO_QUAD_CASE(L) \
  case L:                \
    return launch_quad_ell<L>(g, psrc, cx, cy, bhat, xk, xkm1, out3, out4, qs, s);
    AAO_QUAD_CASE(4)
    AAO_QUAD_CASE(6)
    AAO_QUAD_CASE(8)
    AAO_QUAD_CASE(10)
    AAO_QUAD_CASE(12)
    AAO_QUAD_CASE(14)
    AAO_QUAD_CASE(16)
#undef AAO_QUAD_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace aao
