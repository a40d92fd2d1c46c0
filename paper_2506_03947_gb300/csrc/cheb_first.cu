// The α-scaling, the forward time DFT and Chebyshev step k = 1 in one launch (2D, FP32).
//
// Eq. 5 applies Γ (the α-scaling) and the time DFT U* to the residual r, then each frequency's
// shifted solve starts from x_1 = b̂/θ and x_0 = 0 (Eq. 7 over Lemma 2's segment).  Step 1 needs
// A x_1 = (A b̂)/θ, i.e. b̂ at the four neighbours of every cell.  A block owns a 128 × 8 tile of
// cells (32 × 8 threads, four consecutive cells along x each): it transforms r on the tile and a
// one-cell ring around it into shared memory (the ring's transform is recomputed by the
// neighbouring blocks as well: (130 × 10)/(128 × 8) = 1.27 transforms per cell), then runs step
// 1 on the tile from shared memory and writes b̂ (needed by every later step) and x_2.
//
// Per cell the launch moves r (8ℓ B) and the two face arrays (8 B) in and b̂ and x_2 (4ℓ B each)
// out: 16ℓ + 8 bytes, against 12ℓ + (8ℓ + 8) for the transform and the first step as two
// launches (b̂ written and read back).  The transform of each cell is the one of the separate
// transform kernel, operation for operation (FP32 rounding of r, FP32 α-scaling, the same
// summation order), so b̂ is bitwise the same; step 1 uses the single-step kernel's formulas.
#include "aao_internal.cuh"
#include "cheb_kernels.cuh"

namespace aao {

namespace {

constexpr int kFX = 128, kFY = 8;            // interior tile
constexpr int kEX = kFX + 2, kEY = kFY + 2;  // with the one-cell ring
constexpr int kPad = 4;    // tile column 0 at shared index kPad (16-byte aligned), the ring's columns at
                           // kPad - 1 and kPad + kFX
constexpr int kRow = 136;  // shared row stride (floats): >= kPad + kFX + 1, a multiple of 4

template <int ELL>
__global__ void __launch_bounds__(256) k_dft_first(GridDesc g, const double* __restrict__ r,
                                                   const double* __restrict__ rscale, float* __restrict__ bhat,
                                                   float* __restrict__ x2, const float* __restrict__ cx,
                                                   const float* __restrict__ cy, const __grid_constant__ DftArgs<float> da,
                                                   const __grid_constant__ StepArgs<float> sa) {
  extern __shared__ __align__(16) float sb[];  // [ELL planes][kEY rows][kRow]
  __shared__ float gs[ELL];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < ELL) gs[tid] = (float)(da.gamma[tid] * (rscale ? *rscale : 1.0));
  __syncthreads();
  const int64_t N = g.N;
  const int gx0 = blockIdx.x * kFX - 1, gy0 = blockIdx.y * kFY - 1;  // grid cell of ring corner (-1, -1)

  // transform of the tile and its ring into shared memory (zero outside the grid)
  for (int q = tid; q < kEX * kEY; q += 256) {
    const int ey = q / kEX, ex = q - ey * kEX;
    const int gx = gx0 + ex, gy = gy0 + ey;
    float fre[ELL / 2 + 1], fim[ELL / 2 + 1];
    if (gx >= 0 && gx < g.n0 && gy >= 0 && gy < g.n1) {
      dft_point<float, ELL>(N, (int64_t)gy * g.n0 + gx, r, gs, da, fre, fim);
    } else {
#pragma unroll
      for (int m = 0; m <= ELL / 2; ++m) fre[m] = fim[m] = 0.f;
    }
    float* o = sb + ey * kRow + kPad - 1 + ex;
    o[0] = fre[0];
    o[kEY * kRow] = fre[ELL / 2];
#pragma unroll
    for (int m = 1; m < ELL / 2; ++m) {
      o[(2 * m) * kEY * kRow] = fre[m];
      o[(2 * m + 1) * kEY * kRow] = fim[m];
    }
  }
  __syncthreads();

  // step 1 on the thread's four cells: x_2 = x_1 + a (x_1 - 0) + g (bhat - A x_1 + lambda x_1)
  const int lane = threadIdx.x;
  const int i0 = blockIdx.x * kFX + 4 * lane, j = blockIdx.y * kFY + threadIdx.y;
  const bool act = i0 < g.n0 && j < g.n1;  // n0 % 4 == 0: all four cells or none
  const int64_t c = (int64_t)j * g.n0 + i0;
  const bool west = i0 > 0, south = j > 0;
  const F4 kE = act ? ld4(cx + c) : zero4();
  float kw0 = __shfl_up_sync(0xffffffffu, kE.v[3], 1);
  if (lane == 0) kw0 = (act && west) ? __ldg(cx + c - 1) : 0.f;
  const F4 kW{{kw0, kE.v[0], kE.v[1], kE.v[2]}};
  const F4 kN = act ? ld4(cy + c) : zero4();
  const F4 kS = (act && south) ? ld4(cy + c - g.n0) : zero4();
  const int srow = (threadIdx.y + 1) * kRow + kPad + 4 * lane;  // first cell of the thread

  // A v on one shared plane: neighbours outside the grid are zero in shared memory and their
  // faces are zero, so the stencil needs no boundary branches
  auto plane = [&](int pl, F4& v, F4& Av) {
    const float* p = sb + pl * kEY * kRow + srow;
    const float4 vc = *reinterpret_cast<const float4*>(p);
    const float4 vn = *reinterpret_cast<const float4*>(p + kRow);
    const float4 vs = *reinterpret_cast<const float4*>(p - kRow);
    float left = __shfl_up_sync(0xffffffffu, vc.w, 1);
    float right = __shfl_down_sync(0xffffffffu, vc.x, 1);
    if (lane == 0) left = p[-1];
    if (lane == 31) right = p[4];
    v = F4{{vc.x, vc.y, vc.z, vc.w}};
    const F4 n{{vn.x, vn.y, vn.z, vn.w}}, sth{{vs.x, vs.y, vs.z, vs.w}};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = v.v[e];
      const float xe = (e < 3) ? v.v[e + 1] : right;
      const float xw = (e > 0) ? v.v[e - 1] : left;
      float acc = x;
      acc += kE.v[e] * (x - xe);
      acc += kW.v[e] * (x - xw);
      acc += kN.v[e] * (x - n.v[e]);
      acc += kS.v[e] * (x - sth.v[e]);
      Av.v[e] = acc;
    }
  };

  // real frequencies m = 0 (plane 0) and m = ELL/2 (plane 1)
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int m = (rr == 0) ? 0 : ELL / 2;
    F4 b, Ab;
    plane(rr, b, Ab);
    F4 xn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = b.v[e] * sa.it_re[m];
      const float Ax = Ab.v[e] * sa.it_re[m];
      const float res = b.v[e] - Ax + sa.lam_re[m] * x;
      xn.v[e] = x + sa.a_re[m] * (x - 0.f) + sa.g_re[m] * res;
    }
    if (act) {
      st4(bhat + rr * N + c, b);
      st4(x2 + rr * N + c, xn);
    }
  }
  // complex frequencies m = 1 .. ELL/2 - 1 (planes 2m, 2m+1)
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    F4 br, bi, Ar, Ai;
    plane(2 * m, br, Ar);
    plane(2 * m + 1, bi, Ai);
    const float itr = sa.it_re[m], iti = sa.it_im[m];
    const float lr = sa.lam_re[m], li = sa.lam_im[m];
    const float ar = sa.a_re[m], ai = sa.a_im[m], gr = sa.g_re[m], gi = sa.g_im[m];
    F4 nr4, ni4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xr = br.v[e] * itr - bi.v[e] * iti;
      const float xi = br.v[e] * iti + bi.v[e] * itr;
      const float Axr = Ar.v[e] * itr - Ai.v[e] * iti;
      const float Axi = Ar.v[e] * iti + Ai.v[e] * itr;
      const float rre = br.v[e] - Axr + (lr * xr - li * xi);
      const float rim = bi.v[e] - Axi + (lr * xi + li * xr);
      const float dr = xr - 0.f, di = xi - 0.f;
      nr4.v[e] = xr + (ar * dr - ai * di) + (gr * rre - gi * rim);
      ni4.v[e] = xi + (ar * di + ai * dr) + (gr * rim + gi * rre);
    }
    if (act) {
      const int64_t pr = (int64_t)(2 * m) * N, pi = (int64_t)(2 * m + 1) * N;
      st4(bhat + pr + c, br);
      st4(bhat + pi + c, bi);
      st4(x2 + pr + c, nr4);
      st4(x2 + pi + c, ni4);
    }
  }
}

template <int ELL>
cudaError_t launch_dft_first_ell(const GridDesc& g, const double* r, const double* rscale, float* bhat, float* x2,
                                 const float* cx, const float* cy, const DftArgs<float>& da,
                                 const StepArgs<float>& sa, cudaStream_t s) {
  const size_t smem = sizeof(float) * ELL * kEY * kRow;
  cudaError_t e = cudaFuncSetAttribute(k_dft_first<ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((g.n0 + kFX - 1) / kFX), (unsigned)((g.n1 + kFY - 1) / kFY), 1);
  k_dft_first<ELL><<<grid, dim3(32, kFY, 1), smem, s>>>(g, r, rscale, bhat, x2, cx, cy, da, sa);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dft_first(const GridDesc& g, int ell, const double* r, const double* rscale, float* bhat,
                             float* x2, const float* cx, const float* cy, const DftArgs<float>& da,
                             const StepArgs<float>& sa, cudaStream_t s) {
  if (g.n2 != 1 || g.n0 % 4 != 0 || g.n1 > 65535 * kFY ||
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
