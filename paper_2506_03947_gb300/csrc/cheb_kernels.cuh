// Fused Chebyshev kernels of the preconditioner apply (Eq. 5 with inner CI).
//
// One thread owns one grid cell and all ell/2+1 distinct frequencies of it:
// the cell's stencil coefficients are loaded once and reused for every
// frequency plane (Section 2.2: the ell shifted problems of Eq. 7 share A).
// Each step computes, for every frequency m,
//   x_{k+1} = x_k + a_m (x_k - x_{k-1}) + g_m (bhat_m - A x_k + lambda_m x_k)
// which is the three-term form of Chebyshev semi-iteration on
// B_m = A - lambda_m I over the segment of Lemma 2.  The first step takes
// x_1 = bhat/theta and x_0 = 0 without reading x buffers; the last step feeds
// x_p straight into the inverse transform (Eq. 5's Gamma^{-1} U) and writes
// the FP64 result.
#pragma once

#include "aao_internal.cuh"
#include "cheb_v4.cuh"

#include <type_traits>

namespace aao {

// conversions between the Chebyshev field type and FP64 (integer pipe for FP32)
template <typename T>
__device__ __forceinline__ T to_T(double v) {
  if constexpr (std::is_same<T, float>::value) return d2f_rn(v);
  else return v;
}
template <typename T>
__device__ __forceinline__ double from_T(T v) {
  if constexpr (std::is_same<T, float>::value) return f2d_exact(v);
  else return v;
}

template <typename T, int DIM>
struct Stencil {
  T kap[2 * DIM];
  int64_t nb[2 * DIM];
};

// Neighbour indices are clamped to the cell itself at the boundary, where the
// face coefficient is zero (no boundary faces: homogeneous Neumann).
template <typename T, int DIM>
__device__ __forceinline__ void load_stencil(const GridDesc& g, int i, int j, int k, int64_t c,
                                             const T* __restrict__ cx, const T* __restrict__ cy,
                                             const T* __restrict__ cz, Stencil<T, DIM>& s) {
  s.kap[0] = __ldg(cx + c);
  s.kap[1] = (i > 0) ? __ldg(cx + c - 1) : T(0);
  s.nb[0] = (i < g.n0 - 1) ? c + 1 : c;
  s.nb[1] = (i > 0) ? c - 1 : c;
  if constexpr (DIM >= 2) {
    s.kap[2] = __ldg(cy + c);
    s.kap[3] = (j > 0) ? __ldg(cy + c - g.n0) : T(0);
    s.nb[2] = (j < g.n1 - 1) ? c + g.n0 : c;
    s.nb[3] = (j > 0) ? c - g.n0 : c;
  }
  if constexpr (DIM == 3) {
    const int64_t pl = (int64_t)g.n0 * g.n1;
    s.kap[4] = __ldg(cz + c);
    s.kap[5] = (k > 0) ? __ldg(cz + c - pl) : T(0);
    s.nb[4] = (k < g.n2 - 1) ? c + pl : c;
    s.nb[5] = (k > 0) ? c - pl : c;
  }
}

// (A v)_c = v_c + sum_f kappa_f (v_c - v_nbr(f)) on one plane; returns A v and v_c.
template <typename T, int DIM>
__device__ __forceinline__ T apply_A(const T* __restrict__ p, int64_t c, const Stencil<T, DIM>& s,
                                     T& vc) {
  vc = __ldg(p + c);
  T acc = vc;
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) acc += s.kap[q] * (vc - __ldg(p + s.nb[q]));
  return acc;
}

template <typename T, int ELL, int DIM, int KSRC, int PSRC, bool LAST>
__global__ void __launch_bounds__(256)
    k_cheb_step(GridDesc g, const T* __restrict__ cx, const T* __restrict__ cy, const T* __restrict__ cz,
                const T* __restrict__ bhat, const T* __restrict__ xk, T* xio, double* __restrict__ z,
                StepArgs<T> sa, IdftArgs<T> ia) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.n0 || j >= g.n1) return;
  const int64_t N = g.N;
  const int64_t c = i + (int64_t)g.n0 * (j + (int64_t)g.n1 * k);
  Stencil<T, DIM> st;
  load_stencil<T, DIM>(g, i, j, k, c, cx, cy, cz, st);
  const T* src = (KSRC == 0) ? bhat : xk;

  T zt[LAST ? ELL : 1];
  if constexpr (LAST) {
#pragma unroll
    for (int t = 0; t < ELL; ++t) zt[t] = T(0);
  }

  // Real frequencies m = 0 (plane 0) and m = ELL/2 (plane 1).
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = (r == 0) ? 0 : ELL / 2;
    T vc;
    const T Av = apply_A<T, DIM>(src + r * N, c, st, vc);
    const T b = (KSRC == 0) ? vc : __ldg(bhat + r * N + c);
    T x, Ax;
    if constexpr (KSRC == 0) {
      x = vc * sa.it_re[m];
      Ax = Av * sa.it_re[m];
    } else {
      x = vc;
      Ax = Av;
    }
    T xm;
    if constexpr (PSRC == 0) xm = T(0);
    else if constexpr (PSRC == 1) xm = b * sa.it_re[m];
    else xm = xio[r * N + c];
    const T res = b - Ax + sa.lam_re[m] * x;
    const T xn = x + sa.a_re[m] * (x - xm) + sa.g_re[m] * res;
    if constexpr (!LAST) {
      xio[r * N + c] = xn;
    } else {
#pragma unroll
      for (int t = 0; t < ELL; ++t) zt[t] += xn * ia.ci[t][m];
    }
  }

  // Complex frequencies m = 1 .. ELL/2-1 (planes 2m, 2m+1).
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    const int64_t pr = (int64_t)(2 * m) * N, pi = (int64_t)(2 * m + 1) * N;
    T vr, vi;
    const T Ar = apply_A<T, DIM>(src + pr, c, st, vr);
    const T Ai = apply_A<T, DIM>(src + pi, c, st, vi);
    T br, bi;
    if constexpr (KSRC == 0) {
      br = vr;
      bi = vi;
    } else {
      br = __ldg(bhat + pr + c);
      bi = __ldg(bhat + pi + c);
    }
    const T itr = sa.it_re[m], iti = sa.it_im[m];
    T xr, xi, Axr, Axi;
    if constexpr (KSRC == 0) {
      xr = vr * itr - vi * iti;
      xi = vr * iti + vi * itr;
      Axr = Ar * itr - Ai * iti;
      Axi = Ar * iti + Ai * itr;
    } else {
      xr = vr;
      xi = vi;
      Axr = Ar;
      Axi = Ai;
    }
    T mr, mi;
    if constexpr (PSRC == 0) {
      mr = T(0);
      mi = T(0);
    } else if constexpr (PSRC == 1) {
      mr = br * itr - bi * iti;
      mi = br * iti + bi * itr;
    } else {
      mr = xio[pr + c];
      mi = xio[pi + c];
    }
    const T lr = sa.lam_re[m], li = sa.lam_im[m];
    const T rr = br - Axr + (lr * xr - li * xi);
    const T ri = bi - Axi + (lr * xi + li * xr);
    const T dr = xr - mr, di = xi - mi;
    const T ar = sa.a_re[m], ai = sa.a_im[m], gr = sa.g_re[m], gi = sa.g_im[m];
    const T nr = xr + (ar * dr - ai * di) + (gr * rr - gi * ri);
    const T ni = xi + (ar * di + ai * dr) + (gr * ri + gi * rr);
    if constexpr (!LAST) {
      xio[pr + c] = nr;
      xio[pi + c] = ni;
    } else {
#pragma unroll
      for (int t = 0; t < ELL; ++t) zt[t] += nr * ia.ci[t][m] - ni * ia.si[t][m];
    }
  }

  if constexpr (LAST) {
#pragma unroll
    for (int t = 0; t < ELL; ++t) z[(int64_t)t * N + c] = from_T<T>(zt[t] * ia.igamma_T[t]);
  }
}

// Forward transform (Eq. 5's U* Gamma): r (FP64, block-major) -> packed bhat.
// gs[t] = gamma_t * scale in T, formed once per block by the caller.
template <typename T, int ELL>
__device__ __forceinline__ void dft_point(int64_t N, int64_t c, const double* __restrict__ r, const T* gs,
                                          const DftArgs<T>& da, T (&fre)[ELL / 2 + 1],
                                          T (&fim)[ELL / 2 + 1]) {
  // alpha-scaling in T: the mixed path rounds r to FP32 first and scales in FP32
  T s[ELL];
#pragma unroll
  for (int t = 0; t < ELL; ++t) s[t] = to_T<T>(__ldg(r + (int64_t)t * N + c)) * gs[t];
#pragma unroll
  for (int m = 0; m <= ELL / 2; ++m) {
    T re = T(0), im = T(0);
#pragma unroll
    for (int t = 0; t < ELL; ++t) {
      re += s[t] * da.cf[t][m];
      im -= s[t] * da.sf[t][m];
    }
    fre[m] = re;
    fim[m] = im;
  }
}

// Body of one block (cell block cb) of the forward transform; gs is the block's
// shared array of ELL scalings.  Shared by the single-instance and batched kernels.
template <typename T, int ELL>
__device__ __forceinline__ void dft_body(int64_t N, int64_t cb, const double* __restrict__ r,
                                         const double* __restrict__ rscale, T* __restrict__ bhat,
                                         const DftArgs<T>& da, T* gs) {
  if (threadIdx.x < ELL) gs[threadIdx.x] = (T)(da.gamma[threadIdx.x] * (rscale ? *rscale : 1.0));
  __syncthreads();
  const int64_t c = cb * blockDim.x + threadIdx.x;
  if (c >= N) return;
  T fre[ELL / 2 + 1], fim[ELL / 2 + 1];
  dft_point<T, ELL>(N, c, r, gs, da, fre, fim);
  bhat[c] = fre[0];
  bhat[N + c] = fre[ELL / 2];
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    bhat[(int64_t)(2 * m) * N + c] = fre[m];
    bhat[(int64_t)(2 * m + 1) * N + c] = fim[m];
  }
}

template <typename T, int ELL>
__global__ void __launch_bounds__(256)
    k_dft(int64_t N, const double* __restrict__ r, const double* __restrict__ rscale, T* __restrict__ bhat,
          const __grid_constant__ DftArgs<T> da) {
  __shared__ T gs[ELL];
  dft_body<T, ELL>(N, blockIdx.x, r, rscale, bhat, da, gs);
}

// p = 1: z = Gamma^{-1} U (bhat / theta) with no stencil work (x_1 = bhat/theta).
template <typename T, int ELL>
__global__ void __launch_bounds__(256)
    k_direct(int64_t N, const double* __restrict__ r, const double* __restrict__ rscale, double* __restrict__ z,
             DftArgs<T> da, StepArgs<T> sa, IdftArgs<T> ia) {
  __shared__ T gs[ELL];
  __shared__ T ig[ELL];
  if (threadIdx.x < ELL) {
    gs[threadIdx.x] = (T)(da.gamma[threadIdx.x] * (rscale ? *rscale : 1.0));
    ig[threadIdx.x] = (T)ia.igamma[threadIdx.x];
  }
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  T fre[ELL / 2 + 1], fim[ELL / 2 + 1];
  dft_point<T, ELL>(N, c, r, gs, da, fre, fim);
  T zt[ELL];
#pragma unroll
  for (int t = 0; t < ELL; ++t) zt[t] = T(0);
#pragma unroll
  for (int m = 0; m <= ELL / 2; ++m) {
    const T yr = fre[m] * sa.it_re[m] - fim[m] * sa.it_im[m];
    const T yi = fre[m] * sa.it_im[m] + fim[m] * sa.it_re[m];
#pragma unroll
    for (int t = 0; t < ELL; ++t) zt[t] += yr * ia.ci[t][m] - yi * ia.si[t][m];
  }
#pragma unroll
  for (int t = 0; t < ELL; ++t) z[(int64_t)t * N + c] = from_T<T>(zt[t] * ig[t]);
}

// ---- dispatch -------------------------------------------------------------

// FP32 steps on grids whose rows are a multiple of 4 cells use the vectorised
// kernel (16-byte accesses; the inverse-transform output needs a 16-byte
// aligned z as well).
template <int ELL, int DIM>
cudaError_t launch_step_v4(const GridDesc& g, int ksrc, int psrc, bool last, const float* cx, const float* cy,
                           const float* cz, const float* bhat, const float* xk, float* xio, double* z,
                           const StepArgs<float>& sa, const IdftArgs<float>& ia, cudaStream_t s) {
  dim3 block, grid;
  if (DIM == 1) {
    block = dim3(256, 1, 1);
    grid = dim3((unsigned)((g.n0 + 1023) / 1024), 1, 1);
  } else {
    block = dim3(32, 8, 1);
    grid = dim3((unsigned)((g.n0 + 127) / 128), (unsigned)((g.n1 + 7) / 8), (unsigned)g.n2);
  }
  const int mode = ksrc * 100 + psrc * 10 + (last ? 1 : 0);
#define AAO_V4(K, P, LST) \
  k_cheb_step_v4<ELL, DIM, K, P, LST><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia)
  switch (mode) {
    case 0: AAO_V4(0, 0, false); break;
    case 1: AAO_V4(0, 0, true); break;
    case 110: AAO_V4(1, 1, false); break;
    case 111: AAO_V4(1, 1, true); break;
    case 120: AAO_V4(1, 2, false); break;
    case 121: AAO_V4(1, 2, true); break;
    default: return cudaErrorInvalidValue;
  }
#undef AAO_V4
  count_launch();
  return cudaGetLastError();
}

template <typename T, int ELL, int DIM>
cudaError_t launch_step_ell_dim(const GridDesc& g, int ksrc, int psrc, bool last, const T* cx, const T* cy,
                                const T* cz, const T* bhat, const T* xk, T* xio, double* z,
                                const StepArgs<T>& sa, const IdftArgs<T>& ia, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (g.n0 % 4 == 0 && (!last || (reinterpret_cast<uintptr_t>(z) % 16) == 0))
      return launch_step_v4<ELL, DIM>(g, ksrc, psrc, last, cx, cy, cz, bhat, xk, xio, z, sa, ia, s);
  }
  dim3 block, grid;
  if (DIM == 1) {
    block = dim3(256, 1, 1);
    grid = dim3((unsigned)((g.n0 + 255) / 256), 1, 1);
  } else {
    block = dim3(32, 8, 1);
    grid = dim3((unsigned)((g.n0 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)g.n2);
  }
  const int mode = ksrc * 100 + psrc * 10 + (last ? 1 : 0);
  switch (mode) {
    case 0:
      k_cheb_step<T, ELL, DIM, 0, 0, false><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    case 1:
      k_cheb_step<T, ELL, DIM, 0, 0, true><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    case 110:
      k_cheb_step<T, ELL, DIM, 1, 1, false><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    case 111:
      k_cheb_step<T, ELL, DIM, 1, 1, true><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    case 120:
      k_cheb_step<T, ELL, DIM, 1, 2, false><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    case 121:
      k_cheb_step<T, ELL, DIM, 1, 2, true><<<grid, block, 0, s>>>(g, cx, cy, cz, bhat, xk, xio, z, sa, ia);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T, int DIM>
cudaError_t launch_step_dim(const GridDesc& g, int ell, int ksrc, int psrc, bool last, const T* cx, const T* cy,
                            const T* cz, const T* bhat, const T* xk, T* xio, double* z, const StepArgs<T>& sa,
                            const IdftArgs<T>& ia, cudaStream_t s) {
  switch (ell) {
#define AAO_STEP_CASE(L) \
  case L:                \
    return launch_step_ell_dim<T, L, DIM>(g, ksrc, psrc, last, cx, cy, cz, bhat, xk, xio, z, sa, ia, s);
    AAO_STEP_CASE(4)
    AAO_STEP_CASE(6)
    AAO_STEP_CASE(8)
    AAO_STEP_CASE(10)
    AAO_STEP_CASE(12)
    AAO_STEP_CASE(14)
    AAO_STEP_CASE(16)
#undef AAO_STEP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace aao
