// Chebyshev step kernels for 2D grids (instantiations; bodies in cheb_kernels.cuh).
#include "cheb_kernels.cuh"

namespace aao {
template cudaError_t launch_step_dim<float, 2>(const GridDesc&, int, int, int, bool, const float*, const float*,
                                               const float*, const float*, const float*, float*, double*,
                                               const StepArgs<float>&, const IdftArgs<float>&, cudaStream_t);
template cudaError_t launch_step_dim<double, 2>(const GridDesc&, int, int, int, bool, const double*,
                                                const double*, const double*, const double*, const double*,
                                                double*, double*, const StepArgs<double>&,
                                                const IdftArgs<double>&, cudaStream_t);
}  // namespace aao
