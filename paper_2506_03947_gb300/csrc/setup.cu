// Set-up kernels run once per aao_create: per-cell face coefficients (FP64 and
// FP32 copies), validation of the diffusivities, and the Gershgorin bound of A.
#include "aao_internal.cuh"

namespace aao {

// cx[c] = kappa of the face (c, c+x) or 0 on the last column; likewise cy, cz.
// Each face is owned by its lower cell.  partials[blk] = max over the block of
// S_c = sum of the face diffusivities touching c; bad[0] is set when a face
// value is not finite or not positive.
__global__ void __launch_bounds__(256)
    k_build_coeffs(GridDesc g, const double* __restrict__ kx, const double* __restrict__ ky,
                   const double* __restrict__ kz, double* __restrict__ cx, double* __restrict__ cy,
                   double* __restrict__ cz, float* __restrict__ fx, float* __restrict__ fy, float* __restrict__ fz,
                   double* __restrict__ partials, int* __restrict__ bad) {
  __shared__ double sh[8];
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double smax = 0.0;
  if (c < g.N) {
    const int i = (int)(c % g.n0);
    const int j = (int)((c / g.n0) % g.n1);
    const int k = (int)(c / ((int64_t)g.n0 * g.n1));
    double ex = 0.0, ey = 0.0, ez = 0.0;
    if (i < g.n0 - 1) ex = kx[((int64_t)k * g.n1 + j) * (g.n0 - 1) + i];
    if (j < g.n1 - 1) ey = ky[((int64_t)k * (g.n1 - 1) + j) * g.n0 + i];
    if (k < g.n2 - 1) ez = kz[c];
    int b = 0;
    if (i < g.n0 - 1 && !(ex > 0.0 && isfinite(ex))) b = 1;
    if (j < g.n1 - 1 && !(ey > 0.0 && isfinite(ey))) b = 1;
    if (k < g.n2 - 1 && !(ez > 0.0 && isfinite(ez))) b = 1;
    if (b) atomicOr(bad, 1);
    cx[c] = ex;
    cy[c] = ey;
    cz[c] = ez;
    fx[c] = (float)ex;
    fy[c] = (float)ey;
    fz[c] = (float)ez;
    double wx = 0.0, wy = 0.0, wz = 0.0;
    if (i > 0) wx = kx[((int64_t)k * g.n1 + j) * (g.n0 - 1) + i - 1];
    if (j > 0) wy = ky[((int64_t)k * (g.n1 - 1) + j - 1) * g.n0 + i];
    if (k > 0) wz = kz[c - (int64_t)g.n0 * g.n1];
    smax = ex + ey + ez + wx + wy + wz;
    if (!isfinite(smax)) smax = 0.0;
  }
  // block max (fixed order)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < 8; ++w) m = fmax(m, sh[w]);
    partials[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(256) k_reduce_max(const double* __restrict__ partials, int nb, double* out) {
  __shared__ double sh[8];
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, partials[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < 8; ++w) r = fmax(r, sh[w]);
    *out = r;
  }
}

int build_coeff_blocks(int64_t N) { return (int)((N + 255) / 256); }

cudaError_t launch_build_coeffs(const GridDesc& g, const double* kx, const double* ky, const double* kz,
                                double* cx, double* cy, double* cz, float* fx, float* fy, float* fz,
                                double* partials, int* bad, double* smax_out, cudaStream_t s) {
  const int nb = build_coeff_blocks(g.N);
  k_build_coeffs<<<nb, 256, 0, s>>>(g, kx, ky, kz, cx, cy, cz, fx, fy, fz, partials, bad);
  count_launch();
  k_reduce_max<<<1, 256, 0, s>>>(partials, nb, smax_out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace aao
