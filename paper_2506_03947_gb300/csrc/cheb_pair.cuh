// Two Chebyshev steps per launch (2D, FP32): temporal blocking of the sweep.
//
// Steps k and k+1 of Chebyshev semi-iteration on every frequency,
//   x_{k+1} = x_k + a_k (x_k - x_{k-1}) + g_k (bhat - A x_k + lambda x_k)
//   x_{k+2} = x_{k+1} + a_{k+1} (x_{k+1} - x_k) + g_{k+1} (bhat - A x_{k+1} + lambda x_{k+1}),
// are fused: each block computes x_{k+1} on its tile plus a one-cell halo,
// keeps it in shared memory, and computes x_{k+2} on the tile from there.  Per
// cell and per pair of steps the launch reads x_k, x_{k-1}, bhat and the face
// coefficients once and writes x_{k+1} and x_{k+2}: (5 ell + 2) * 4 bytes
// instead of 2 (4 ell + 2) * 4 for two single steps.
//
// Tiles overlap: a block is 32 lanes x (TY + 2) rows of warps, each lane owns
// four consecutive cells (16-byte accesses); lanes 0 and 31 and the first and
// last warp rows form the halo, computed for step k only, so the tile's
// interior is 120 x TY cells.  Reads of x_{k-1} and bhat on the halo come
// from neighbouring tiles, so the outputs go to buffers no block reads in the
// same launch.
#pragma once

#include "aao_internal.cuh"
#include "cheb_v4.cuh"

namespace aao {

constexpr int kPairTY = 8;                  // interior rows per tile
constexpr int kPairRows = kPairTY + 2;      // warp rows per block
constexpr int kPairCols = 128;              // cells per warp row (32 lanes x 4)
constexpr int kPairInnerX = kPairCols - 8;  // interior cells per tile along x

template <int ELL>
constexpr size_t pair_smem_bytes() {
  return sizeof(float) * (size_t)ELL * kPairRows * kPairCols;
}

// PSRC: x_{k-1} = bhat/theta (1, step k = 2) or from buffer xkm1 (2).
template <int ELL, int PSRC>
__global__ void __launch_bounds__(32 * kPairRows)
    k_cheb_pair_v4(GridDesc g, const float* __restrict__ cx, const float* __restrict__ cy,
                   const float* __restrict__ bhat, const float* __restrict__ xk, const float* __restrict__ xkm1,
                   float* __restrict__ out1, float* __restrict__ out2, StepArgs<float> s1, StepArgs<float> s2) {
  extern __shared__ float sm[];  // [ELL][kPairRows][kPairCols]: x_{k+1} on tile + halo
  const int lane = threadIdx.x;
  const int r = threadIdx.y;                                       // 0 .. kPairRows-1
  const int i0 = blockIdx.x * kPairInnerX - 4 + 4 * lane;          // first of this lane's four cells
  const int j = blockIdx.y * kPairTY + r - 1;
  const bool rowok = (j >= 0 && j < g.n1);
  const int64_t N = g.N;
  const int64_t c = (int64_t)g.n0 * j + i0;
  Stencil4<2> st;
  st.act = rowok && i0 >= 0 && i0 < g.n0;
  st.west = i0 > 0;
  st.east = i0 + 4 < g.n0;
  st.kE = st.act ? ld4(cx + c) : zero4();
  {
    float kprev = __shfl_up_sync(0xffffffffu, st.kE.v[3], 1);
    if (lane == 0) kprev = (st.act && st.west) ? __ldg(cx + c - 1) : 0.f;
    st.kW = F4{{kprev, st.kE.v[0], st.kE.v[1], st.kE.v[2]}};
  }
  st.oN = (j < g.n1 - 1) ? g.n0 : 0;
  st.oS = (j > 0) ? -(int64_t)g.n0 : 0;
  st.kN = st.act ? ld4(cy + c) : zero4();
  st.kS = (st.act && j > 0) ? ld4(cy + c - g.n0) : zero4();
  st.oU = st.oD = 0;
  const bool inner = (lane >= 1 && lane <= 30) && (r >= 1 && r <= kPairTY) && st.act;
  float* row_sm = sm + (size_t)r * kPairCols + 4 * lane;

  // ---- step k on tile + halo: x_{k+1} into shared memory (and global for the interior)
#pragma unroll
  for (int q = 0; q < 2; ++q) {  // real frequencies: planes 0 and 1
    const int m = (q == 0) ? 0 : ELL / 2;
    F4 vc;
    const F4 Av = apply_A4<2>(xk + q * N, c, lane, st, vc);
    const F4 b = st.act ? ld4(bhat + q * N + c) : zero4();
    F4 xm = zero4();
    if (PSRC == 2 && st.act) xm = ld4(xkm1 + q * N + c);
    F4 xn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float pm = (PSRC == 1) ? b.v[e] * s1.it_re[m] : xm.v[e];
      const float res = b.v[e] - Av.v[e] + s1.lam_re[m] * vc.v[e];
      xn.v[e] = st.act ? vc.v[e] + s1.a_re[m] * (vc.v[e] - pm) + s1.g_re[m] * res : 0.f;
    }
    st4(row_sm + (size_t)q * kPairRows * kPairCols, xn);
    if (inner) st4(out1 + q * N + c, xn);
  }
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    const int64_t pr = (int64_t)(2 * m) * N, pi = (int64_t)(2 * m + 1) * N;
    F4 vr, vi;
    const F4 Ar = apply_A4<2>(xk + pr, c, lane, st, vr);
    const F4 Ai = apply_A4<2>(xk + pi, c, lane, st, vi);
    const F4 br = st.act ? ld4(bhat + pr + c) : zero4();
    const F4 bi = st.act ? ld4(bhat + pi + c) : zero4();
    F4 mr = zero4(), mi = zero4();
    if (PSRC == 2 && st.act) {
      mr = ld4(xkm1 + pr + c);
      mi = ld4(xkm1 + pi + c);
    }
    const float itr = s1.it_re[m], iti = s1.it_im[m], lr = s1.lam_re[m], li = s1.lam_im[m];
    const float ar = s1.a_re[m], ai = s1.a_im[m], gr = s1.g_re[m], gi = s1.g_im[m];
    F4 nr4, ni4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float pr_, pi_;
      if (PSRC == 1) {
        pr_ = br.v[e] * itr - bi.v[e] * iti;
        pi_ = br.v[e] * iti + bi.v[e] * itr;
      } else {
        pr_ = mr.v[e];
        pi_ = mi.v[e];
      }
      const float xr = vr.v[e], xi = vi.v[e];
      const float rr = br.v[e] - Ar.v[e] + (lr * xr - li * xi);
      const float ri = bi.v[e] - Ai.v[e] + (lr * xi + li * xr);
      const float dr = xr - pr_, di = xi - pi_;
      nr4.v[e] = st.act ? xr + (ar * dr - ai * di) + (gr * rr - gi * ri) : 0.f;
      ni4.v[e] = st.act ? xi + (ar * di + ai * dr) + (gr * ri + gi * rr) : 0.f;
    }
    st4(row_sm + (size_t)(2 * m) * kPairRows * kPairCols, nr4);
    st4(row_sm + (size_t)(2 * m + 1) * kPairRows * kPairCols, ni4);
    if (inner) {
      st4(out1 + pr + c, nr4);
      st4(out1 + pi + c, ni4);
    }
  }
  __syncthreads();
  if (!inner) return;  // halo lanes and rows are done (no barrier follows)

  // ---- step k+1 on the interior, x_{k+1} from shared memory
  // Neighbour values outside the grid were stored as 0 and meet zero face coefficients.
  auto apply_sm = [&](int q, F4& vc) {
    const float* rowp = sm + ((size_t)q * kPairRows + r) * kPairCols + 4 * lane;
    const float4 cc = *reinterpret_cast<const float4*>(rowp);
    const float4 nn = *reinterpret_cast<const float4*>(rowp + kPairCols);
    const float4 ss = *reinterpret_cast<const float4*>(rowp - kPairCols);
    const float left = rowp[-1], right = rowp[4];
    vc = F4{{cc.x, cc.y, cc.z, cc.w}};
    const float nv[4] = {nn.x, nn.y, nn.z, nn.w}, sv[4] = {ss.x, ss.y, ss.z, ss.w};
    F4 a;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x = vc.v[e];
      const float xe = (e < 3) ? vc.v[e + 1] : right;
      const float xw = (e > 0) ? vc.v[e - 1] : left;
      float acc = x;
      acc += st.kE.v[e] * (x - xe);
      acc += st.kW.v[e] * (x - xw);
      acc += st.kN.v[e] * (x - nv[e]);
      acc += st.kS.v[e] * (x - sv[e]);
      a.v[e] = acc;
    }
    return a;
  };
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int m = (q == 0) ? 0 : ELL / 2;
    F4 v1;
    const F4 Av = apply_sm(q, v1);
    const F4 b = ld4(bhat + q * N + c);
    const F4 x0 = ld4(xk + q * N + c);
    F4 xn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float res = b.v[e] - Av.v[e] + s2.lam_re[m] * v1.v[e];
      xn.v[e] = v1.v[e] + s2.a_re[m] * (v1.v[e] - x0.v[e]) + s2.g_re[m] * res;
    }
    st4(out2 + q * N + c, xn);
  }
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    const int64_t pr = (int64_t)(2 * m) * N, pi = (int64_t)(2 * m + 1) * N;
    F4 vr, vi;
    const F4 Ar = apply_sm(2 * m, vr);
    const F4 Ai = apply_sm(2 * m + 1, vi);
    const F4 br = ld4(bhat + pr + c), bi = ld4(bhat + pi + c);
    const F4 xr0 = ld4(xk + pr + c), xi0 = ld4(xk + pi + c);
    const float lr = s2.lam_re[m], li = s2.lam_im[m];
    const float ar = s2.a_re[m], ai = s2.a_im[m], gr = s2.g_re[m], gi = s2.g_im[m];
    F4 nr4, ni4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xr = vr.v[e], xi = vi.v[e];
      const float rr = br.v[e] - Ar.v[e] + (lr * xr - li * xi);
      const float ri = bi.v[e] - Ai.v[e] + (lr * xi + li * xr);
      const float dr = xr - xr0.v[e], di = xi - xi0.v[e];
      nr4.v[e] = xr + (ar * dr - ai * di) + (gr * rr - gi * ri);
      ni4.v[e] = xi + (ar * di + ai * dr) + (gr * ri + gi * rr);
    }
    st4(out2 + pr + c, nr4);
    st4(out2 + pi + c, ni4);
  }
}

template <int ELL>
cudaError_t launch_pair_ell(const GridDesc& g, int psrc, const float* cx, const float* cy, const float* bhat,
                            const float* xk, const float* xkm1, float* out1, float* out2, const StepArgs<float>& s1,
                            const StepArgs<float>& s2, cudaStream_t s) {
  const dim3 block(32, kPairRows, 1);
  const dim3 grid((unsigned)((g.n0 + kPairInnerX - 1) / kPairInnerX), (unsigned)((g.n1 + kPairTY - 1) / kPairTY), 1);
  const size_t smem = pair_smem_bytes<ELL>();
  if (psrc == 1) {
    cudaFuncSetAttribute(k_cheb_pair_v4<ELL, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cheb_pair_v4<ELL, 1><<<grid, block, smem, s>>>(g, cx, cy, bhat, xk, xkm1, out1, out2, s1, s2);
  } else {
    cudaFuncSetAttribute(k_cheb_pair_v4<ELL, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cheb_pair_v4<ELL, 2><<<grid, block, smem, s>>>(g, cx, cy, bhat, xk, xkm1, out1, out2, s1, s2);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace aao
