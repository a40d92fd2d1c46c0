// Exact (best-case) P_alpha^{-1} for spatially constant face diffusivities, FP64.
//
// Section 2.2: with A = X Phi X^T, Eq. 5 becomes
//   P_alpha^{-1} = (Gamma^{-1} U (x) I)(I (x) X)(I (x) Phi - Lambda (x) I)^{-1}(I (x) X^T)(U* Gamma (x) I).
// For the finite-volume Neumann operator with diffusivity kappa_a on every face of axis a,
// X is the orthonormal DCT-II along each axis and Phi = 1 + sum_a kappa_a 4 sin^2(pi k_a / (2 n_a)).
// The apply is: the time DFT (the path's own kernel), the spatial DCT of every frequency plane
// as batched FP64 GEMMs with the n_a x n_a DCT matrices (cuBLAS: plain dense products), the
// division by (phi - lambda_m) per cell and frequency, the inverse DCT, and the inverse time
// DFT with Gamma^{-1}.  This is the comparison preconditioner of the paper's experiments
// ("best case"), not part of the inner Chebyshev path.
#include <cublas_v2.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "aao_internal.cuh"

namespace aao {

namespace {

// y = v / (phi - lambda_m) on the packed frequency planes (plane 0: m = 0, plane 1: m = ell/2,
// planes 2m, 2m+1: Re, Im of m); phi from the per-axis eigenvalue parts.
__global__ void __launch_bounds__(256)
    k_dct_divide(GridDesc g, int ell, const double* __restrict__ ex, const double* __restrict__ ey,
                 const double* __restrict__ ez, double* __restrict__ v, DctShifts sh) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const int i = (int)(c % g.n0);
  const int64_t r = c / g.n0;
  const int j = (int)(r % g.n1);
  const int k = (int)(r / g.n1);
  const double phi = 1.0 + ex[i] + (ey ? ey[j] : 0.0) + (ez ? ez[k] : 0.0);
  const int64_t N = g.N;
  v[c] = v[c] / (phi - sh.lam_re[0]);
  v[N + c] = v[N + c] / (phi - sh.lam_re[ell / 2]);
  for (int m = 1; m < ell / 2; ++m) {
    const double dr = phi - sh.lam_re[m], di = -sh.lam_im[m];
    const double den = dr * dr + di * di;
    const double vr = v[(int64_t)(2 * m) * N + c], vi = v[(int64_t)(2 * m + 1) * N + c];
    // (vr + i vi) / (dr + i di) = ((vr dr + vi di) + i (vi dr - vr di)) / (dr^2 + di^2)
    v[(int64_t)(2 * m) * N + c] = (vr * dr + vi * di) / den;
    v[(int64_t)(2 * m + 1) * N + c] = (vi * dr - vr * di) / den;
  }
}

// z_t = igamma_t sum_m (Re y_m ci[t][m] - Im y_m si[t][m]) from the packed planes.
__global__ void __launch_bounds__(256)
    k_idft_planes(int64_t N, int ell, const double* __restrict__ y, double* __restrict__ z,
                  const __grid_constant__ IdftArgs<double> ia) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double fre[kMaxF], fim[kMaxF];
  fre[0] = y[c];
  fim[0] = 0.0;
  fre[ell / 2] = y[N + c];
  fim[ell / 2] = 0.0;
  for (int m = 1; m < ell / 2; ++m) {
    fre[m] = y[(int64_t)(2 * m) * N + c];
    fim[m] = y[(int64_t)(2 * m + 1) * N + c];
  }
  for (int t = 0; t < ell; ++t) {
    double acc = 0.0;
    for (int m = 0; m <= ell / 2; ++m) acc += fre[m] * ia.ci[t][m] - fim[m] * ia.si[t][m];
    z[(int64_t)t * N + c] = acc * ia.igamma[t];
  }
}

cudaError_t blas_error(cublasStatus_t st) {
  if (st == CUBLAS_STATUS_SUCCESS) return cudaSuccess;
  if (st == CUBLAS_STATUS_ALLOC_FAILED) return cudaErrorMemoryAllocation;
  return cudaErrorUnknown;
}

}  // namespace

struct DctPlan {
  int dim = 0;
  int n[3] = {1, 1, 1};
  double* C[3] = {nullptr, nullptr, nullptr};   // column-major C[k + n i] = s_k cos(pi k (i + 1/2) / n)
  double* ev[3] = {nullptr, nullptr, nullptr};  // kappa_a 4 sin^2(pi k / (2 n_a))
  double* work = nullptr;                       // ell N
  cublasHandle_t blas = nullptr;
};

void dct_plan_destroy(DctPlan* p) {
  if (!p) return;
  for (int a = 0; a < 3; ++a) {
    if (p->C[a]) cudaFree(p->C[a]);
    if (p->ev[a]) cudaFree(p->ev[a]);
  }
  if (p->work) cudaFree(p->work);
  if (p->blas) cublasDestroy(p->blas);
  delete p;
}

cudaError_t dct_plan_create(DctPlan** out, const GridDesc& g, int dim, int ell, const double kappa[3]) {
  *out = nullptr;
  DctPlan* p = new DctPlan();
  p->dim = dim;
  p->n[0] = g.n0;
  p->n[1] = g.n1;
  p->n[2] = g.n2;
  cudaError_t e = cudaSuccess;
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < dim && e == cudaSuccess; ++a) {
    const int n = p->n[a];
    std::vector<double> C((size_t)n * n), ev(n);
    for (int k = 0; k < n; ++k) {
      const double s = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      for (int i = 0; i < n; ++i) C[(size_t)k + (size_t)n * i] = s * std::cos(pi * k * (i + 0.5) / n);
      const double sn = std::sin(pi * k / (2.0 * n));
      ev[k] = kappa[a] * 4.0 * sn * sn;
    }
    e = cudaMalloc(&p->C[a], sizeof(double) * C.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->C[a], C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->ev[a], sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->ev[a], ev.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->work, sizeof(double) * (size_t)ell * (size_t)g.N);
  if (e == cudaSuccess) e = blas_error(cublasCreate(&p->blas));
  if (e == cudaSuccess) e = blas_error(cublasSetMathMode(p->blas, CUBLAS_DEFAULT_MATH));
  if (e != cudaSuccess) {
    dct_plan_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

// Spatial DCT (inverse = false) or its inverse of every plane of v (ell planes of N), in place,
// through p->work.  Each axis is one strided-batched GEMM with the axis' DCT matrix.
static cudaError_t dct_planes(DctPlan* p, int ell, double* v, bool inverse, cudaStream_t s) {
  const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
  const long long N = (long long)n0 * n1 * n2;
  const double one = 1.0, zero = 0.0;
  cublasStatus_t st = cublasSetStream(p->blas, s);
  double* src = v;
  double* dst = p->work;
  const cublasOperation_t tC = inverse ? CUBLAS_OP_T : CUBLAS_OP_N;   // C or C^T applied from the left
  const cublasOperation_t tCr = inverse ? CUBLAS_OP_N : CUBLAS_OP_T;  // C^T or C applied from the right
  // x: each plane as a column-major n0 x (n1 n2) matrix M, M <- C_x M (or C_x^T M)
  if (st == CUBLAS_STATUS_SUCCESS)
    st = cublasDgemmStridedBatched(p->blas, tC, CUBLAS_OP_N, n0, n1 * n2, n0, &one, p->C[0], n0, 0, src, n0, N,
                                   &zero, dst, n0, N, ell);
  std::swap(src, dst);
  if (p->dim >= 2 && st == CUBLAS_STATUS_SUCCESS) {
    // y: every z-slab as an n0 x n1 matrix, M <- M C_y^T (or M C_y)
    st = cublasDgemmStridedBatched(p->blas, CUBLAS_OP_N, tCr, n0, n1, n1, &one, src, n0, (long long)n0 * n1,
                                   p->C[1], n1, 0, &zero, dst, n0, (long long)n0 * n1, ell * n2);
    std::swap(src, dst);
  }
  if (p->dim == 3 && st == CUBLAS_STATUS_SUCCESS) {
    // z: each plane as an (n0 n1) x n2 matrix, M <- M C_z^T (or M C_z)
    st = cublasDgemmStridedBatched(p->blas, CUBLAS_OP_N, tCr, n0 * n1, n2, n2, &one, src, n0 * n1, N, p->C[2], n2, 0,
                                   &zero, dst, n0 * n1, N, ell);
    std::swap(src, dst);
  }
  if (st != CUBLAS_STATUS_SUCCESS) return blas_error(st);
  if (src != v) return cudaMemcpyAsync(v, src, sizeof(double) * (size_t)ell * N, cudaMemcpyDeviceToDevice, s);
  return cudaSuccess;
}

cudaError_t dct_precond(DctPlan* p, const GridDesc& g, int ell, double* vhat, double* z, const DctShifts& sh,
                        const IdftArgs<double>& ia, cudaStream_t s) {
  cudaError_t e = dct_planes(p, ell, vhat, false, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((g.N + 255) / 256);
  k_dct_divide<<<grid, 256, 0, s>>>(g, ell, p->ev[0], p->dim >= 2 ? p->ev[1] : nullptr,
                                    p->dim == 3 ? p->ev[2] : nullptr, vhat, sh);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = dct_planes(p, ell, vhat, true, s);
  if (e != cudaSuccess) return e;
  k_idft_planes<<<grid, 256, 0, s>>>(g.N, ell, vhat, z, ia);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_idft_planes(int64_t N, int ell, const double* y, double* z, const IdftArgs<double>& ia,
                               cudaStream_t s) {
  k_idft_planes<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, ell, y, z, ia);
  count_launch();
  return cudaGetLastError();
}

// Per-axis minimum and maximum of the interior faces (as ordered bit patterns of positive
// doubles); slots 2a, 2a+1 of mm hold min and max of axis a.
__global__ void k_face_range(GridDesc g, const double* __restrict__ cx, const double* __restrict__ cy,
                             const double* __restrict__ cz, unsigned long long* mm) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const int i = (int)(c % g.n0);
  const int64_t r = c / g.n0;
  const int j = (int)(r % g.n1);
  const int k = (int)(r / g.n1);
  if (i < g.n0 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cx[c]);
    atomicMin(&mm[0], b);
    atomicMax(&mm[1], b);
  }
  if (cy && j < g.n1 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cy[c]);
    atomicMin(&mm[2], b);
    atomicMax(&mm[3], b);
  }
  if (cz && k < g.n2 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cz[c]);
    atomicMin(&mm[4], b);
    atomicMax(&mm[5], b);
  }
}

cudaError_t face_ranges(const GridDesc& g, const double* cx, const double* cy, const double* cz, double out[6],
                        cudaStream_t s) {
  unsigned long long* mm = nullptr;
  cudaError_t e = cudaMalloc(&mm, sizeof(unsigned long long) * 6);
  unsigned long long init[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_face_range<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, cx, cy, cz, mm);
    count_launch();
    e = cudaGetLastError();
  }
  unsigned long long hb[6] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb, mm, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (mm) cudaFree(mm);
  for (int q = 0; q < 6; ++q) {
    const bool none = (q % 2 == 0) ? hb[q] == ~0ull : false;
    double v = 0.0;
    std::memcpy(&v, &hb[q], sizeof(double));
    out[q] = none ? 0.0 : v;
  }
  return e;
}

}  // namespace aao
