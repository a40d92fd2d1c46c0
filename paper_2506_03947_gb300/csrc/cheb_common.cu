// Pointwise transform kernels and the dimension dispatch of the Chebyshev steps.
#include "cheb_kernels.cuh"

namespace aao {

#define AAO_EXTERN_STEP(T, D)                                                                              \
  extern template cudaError_t launch_step_dim<T, D>(const GridDesc&, int, int, int, bool, const T*, const T*, \
                                                    const T*, const T*, const T*, T*, double*,             \
                                                    const StepArgs<T>&, const IdftArgs<T>&, cudaStream_t);
AAO_EXTERN_STEP(float, 1)
AAO_EXTERN_STEP(float, 2)
AAO_EXTERN_STEP(float, 3)
AAO_EXTERN_STEP(double, 1)
AAO_EXTERN_STEP(double, 2)
AAO_EXTERN_STEP(double, 3)
#undef AAO_EXTERN_STEP

template <typename T>
cudaError_t launch_step(const GridDesc& g, int dim, int ell, int ksrc, int psrc, bool last, const T* cx, const T* cy,
                        const T* cz, const T* bhat, const T* xk, T* xio, double* z, const StepArgs<T>& sa,
                        const IdftArgs<T>& ia, cudaStream_t s) {
  switch (dim) {
    case 1:
      return launch_step_dim<T, 1>(g, ell, ksrc, psrc, last, cx, cy, cz, bhat, xk, xio, z, sa, ia, s);
    case 2:
      return launch_step_dim<T, 2>(g, ell, ksrc, psrc, last, cx, cy, cz, bhat, xk, xio, z, sa, ia, s);
    case 3:
      return launch_step_dim<T, 3>(g, ell, ksrc, psrc, last, cx, cy, cz, bhat, xk, xio, z, sa, ia, s);
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_dft(const GridDesc& g, int /*dim*/, int ell, const double* r, const double* rscale, T* bhat,
                       const DftArgs<T>& da, cudaStream_t s) {
  const unsigned blocks = (unsigned)((g.N + 255) / 256);
  switch (ell) {
#define AAO_DFT_CASE(L)                                                   \
  case L:                                                                 \
    k_dft<T, L><<<blocks, 256, 0, s>>>(g.N, r, rscale, bhat, da);         \
    break;
    AAO_DFT_CASE(4)
    AAO_DFT_CASE(6)
    AAO_DFT_CASE(8)
    AAO_DFT_CASE(10)
    AAO_DFT_CASE(12)
    AAO_DFT_CASE(14)
    AAO_DFT_CASE(16)
#undef AAO_DFT_CASE
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_direct(const GridDesc& g, int /*dim*/, int ell, const double* r, const double* rscale, double* z,
                          const DftArgs<T>& da, const StepArgs<T>& sa, const IdftArgs<T>& ia, cudaStream_t s) {
  const unsigned blocks = (unsigned)((g.N + 255) / 256);
  switch (ell) {
#define AAO_DIRECT_CASE(L)                                                        \
  case L:                                                                         \
    k_direct<T, L><<<blocks, 256, 0, s>>>(g.N, r, rscale, z, da, sa, ia);         \
    break;
    AAO_DIRECT_CASE(4)
    AAO_DIRECT_CASE(6)
    AAO_DIRECT_CASE(8)
    AAO_DIRECT_CASE(10)
    AAO_DIRECT_CASE(12)
    AAO_DIRECT_CASE(14)
    AAO_DIRECT_CASE(16)
#undef AAO_DIRECT_CASE
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_step<float>(const GridDesc&, int, int, int, int, bool, const float*, const float*,
                                        const float*, const float*, const float*, float*, double*,
                                        const StepArgs<float>&, const IdftArgs<float>&, cudaStream_t);
template cudaError_t launch_step<double>(const GridDesc&, int, int, int, int, bool, const double*, const double*,
                                         const double*, const double*, const double*, double*, double*,
                                         const StepArgs<double>&, const IdftArgs<double>&, cudaStream_t);
template cudaError_t launch_dft<float>(const GridDesc&, int, int, const double*, const double*, float*,
                                       const DftArgs<float>&, cudaStream_t);
template cudaError_t launch_dft<double>(const GridDesc&, int, int, const double*, const double*, double*,
                                        const DftArgs<double>&, cudaStream_t);
template cudaError_t launch_direct<float>(const GridDesc&, int, int, const double*, const double*, double*,
                                          const DftArgs<float>&, const StepArgs<float>&, const IdftArgs<float>&,
                                          cudaStream_t);
template cudaError_t launch_direct<double>(const GridDesc&, int, int, const double*, const double*, double*,
                                           const DftArgs<double>&, const StepArgs<double>&,
                                           const IdftArgs<double>&, cudaStream_t);

}  // namespace aao
