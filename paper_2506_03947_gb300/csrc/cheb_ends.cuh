// The two ends of the 2D mixed preconditioner apply, as device bodies shared by the
// single-instance kernels and the batched ones:
//  * dft_first_body: the α-scaling, the forward time DFT and Chebyshev step k = 1 (Eq. 5, Eq. 7
//    over Lemma 2's segment) on one 128 × 8 tile.  The block transforms r on the tile and a
//    one-cell ring around it into shared memory (the ring's transform is recomputed by the
//    neighbouring blocks as well: (130 × 10)/(128 × 8) = 1.27 transforms per cell), then runs
//    step 1 from shared memory and writes b̂ (needed by every later step) and x_2.  Per cell it
//    moves r (8ℓ B) and the two face arrays (8 B) in and b̂ and x_2 (4ℓ B each) out: 16ℓ + 8
//    bytes, against 12ℓ + (8ℓ + 8) for the transform and the first step as two launches.  The
//    transform of each cell is the separate transform kernel's, operation for operation (FP32
//    rounding of r, FP32 α-scaling, the same summation order), so b̂ is bitwise the same; step 1
//    uses the single-step kernel's formulas.
//  * idft_pair: z_t = gamma_t^{-1} sum_m (Re x_p(m) ci[t][m] - Im x_p(m) si[t][m]) (Eq. 5's
//    Gamma^{-1} U) for two consecutive cells: the packed frequency planes of x_p in FP32 (plane
//    0 = f_0, plane 1 = f_{ell/2}, planes 2m, 2m+1 = Re, Im f_m), z in FP64 (exact conversions of
//    the FP32 values, block-major like r).  Same summation order as the last-step kernel: f_0,
//    then f_{ell/2}, then m = 1 .. ell/2 - 1.
#pragma once

#include "aao_internal.cuh"
#include "cheb_kernels.cuh"

namespace aao {

namespace ends {

constexpr int kFX = 128, kFY = 8;            // interior tile
constexpr int kEX = kFX + 2, kEY = kFY + 2;  // with the one-cell ring
constexpr int kPad = 4;    // tile column 0 at shared index kPad (16-byte aligned), the ring's columns at
                           // kPad - 1 and kPad + kFX
constexpr int kRow = 136;  // shared row stride (floats): >= kPad + kFX + 1, a multiple of 4

// Dynamic shared memory of dft_first_body, in floats.
constexpr int dft_first_smem_floats(int ell) { return ell * kEY * kRow; }

// One 32 x 8-thread block: tile (bx, by) of grid g.  sb: dft_first_smem_floats(ELL) floats of
// dynamic shared memory, 16-byte aligned; gs: ELL floats of shared memory.
template <int ELL>
__device__ __forceinline__ void dft_first_body(const GridDesc& g, int bx, int by, const double* __restrict__ r,
                                               const double* __restrict__ rscale, float* __restrict__ bhat,
                                               float* __restrict__ x2, const float* __restrict__ cx,
                                               const float* __restrict__ cy, const DftArgs<float>& da,
                                               const StepArgs<float>& sa, float* sb, float* gs) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < ELL) gs[tid] = (float)(da.gamma[tid] * (rscale ? *rscale : 1.0));
  __syncthreads();
  const int64_t N = g.N;
  const int gx0 = bx * kFX - 1, gy0 = by * kFY - 1;  // grid cell of ring corner (-1, -1)

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
  const int i0 = bx * kFX + 4 * lane, j = by * kFY + threadIdx.y;
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

// Two cells c, c + 1 of the inverse transform (all ELL planes of the two cells are loaded
// first: ELL 8-byte loads in flight, then one time block at a time).
template <int ELL>
__device__ __forceinline__ void idft_pair(int64_t N, int64_t c, const float* __restrict__ x, double* __restrict__ z,
                                          const IdftArgs<float>& ia) {
  float2 v[ELL];
#pragma unroll
  for (int pl = 0; pl < ELL; ++pl) v[pl] = __ldcs(reinterpret_cast<const float2*>(x + (int64_t)pl * N + c));
#pragma unroll
  for (int t = 0; t < ELL; ++t) {
    float a0 = 0.f, a1 = 0.f;
    const float c0 = ia.ci[t][0], c1 = ia.ci[t][ELL / 2];
    a0 += v[0].x * c0, a1 += v[0].y * c0;
    a0 += v[1].x * c1, a1 += v[1].y * c1;
#pragma unroll
    for (int m = 1; m < ELL / 2; ++m) {
      const float cr = ia.ci[t][m], si = ia.si[t][m];
      const float2 r = v[2 * m], im = v[2 * m + 1];
      a0 += r.x * cr - im.x * si;
      a1 += r.y * cr - im.y * si;
    }
    const float gmul = ia.igamma_T[t];
    *reinterpret_cast<double2*>(z + (int64_t)t * N + c) = make_double2(f2d_exact(a0 * gmul), f2d_exact(a1 * gmul));
  }
}

}  // namespace ends

}  // namespace aao
