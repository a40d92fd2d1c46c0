// Four Chebyshev steps per launch (2D, FP32): deeper temporal blocking.
//
// Steps k .. k+3 of Chebyshev semi-iteration on every frequency (Eq. 7 over
// Lemma 2's segment),
//   x_{q+1} = x_q + a_q (x_q - x_{q-1}) + g_q (bhat - A x_q + lambda x_q),
// run on a tile held in shared memory.  A block owns an interior tile of
// 120 x TY cells and stages x_k on the tile plus a four-cell halo, x_{k-1}
// and bhat beside it; level q+1 is computed on a region one cell smaller on
// every side than level q, in place over level q-1 (each cell reads level
// q-1 only at itself).  After four levels the interior holds x_{k+4}, the
// other buffer x_{k+3}; both are written out.  Per cell and four steps the
// launch moves (5 ell + 2) * 4 bytes (reads x_k, x_{k-1}, bhat, two face
// arrays; writes two fields) instead of 4 (4 ell + 2) * 4.
//
// Frequencies are processed one plane pair at a time (the two real
// frequencies together, then each complex one), so the staged tile is two
// planes deep; the face coefficients and the diagonal d = 1 + sum kappa of
// A are staged once per block.  Each level forms the residual as
//   b - (A - lambda) x = bhat + sum_f kappa_f x_nbr(f) - (d - lambda) x,
// one multiply-add per term; its rounding (about d u |x|) enters the update
// multiplied by g ~ 2/mu_max, i.e. a few units of roundoff of |x| per step.
#pragma once

#include <type_traits>

#include "aao_internal.cuh"
#include "cheb_v4.cuh"

namespace aao {

constexpr int kQuadS = 4;                      // fused steps (= halo width)
constexpr int kQuadCols = 128;                 // staged cells per row (32 lanes x 4)
constexpr int kQuadPad = 4;                    // zero padding each side of a staged row
constexpr int kQuadStride = kQuadCols + 2 * kQuadPad;
constexpr int kQuadInnerX = kQuadCols - 2 * kQuadS;  // 120
constexpr int kQuadTileTY = 16;                // interior rows of a tile
constexpr int kQuadTileNT = 384;               // threads of a tile block

template <int TY>
__host__ __device__ constexpr int quad_rows() {
  return TY + 2 * kQuadS;
}
// shared memory: two level buffers (2 planes each), cx, cy and the diagonal
template <int TY>
constexpr size_t quad_smem_bytes() {
  return sizeof(float) * (size_t)quad_rows<TY>() * kQuadStride * (2 * 2 + 3);
}

using QuadArgs = QuadSteps;

// PSRC: x_{k-1} = bhat/theta (1, first fused step is k = 2) or read from xkm1 (2).
// NT threads: NT/32 warps, each owning the staged rows warp, warp + NT/32, ...
// (RPW of them) for the whole launch, so bhat of those rows stays in registers.
// The body runs tile (bx, by); it is shared by the single-instance kernel below and the batched
// one, which maps its blocks to (instance, tile) pairs.
template <int ELL, int TY, int PSRC, int NT>
__device__ __forceinline__ void cheb_quad_body(const GridDesc& g, int bx, int by, const float* __restrict__ cx,
                                               const float* __restrict__ cy, const float* __restrict__ bhat,
                                               const float* __restrict__ xk, const float* __restrict__ xkm1,
                                               float* __restrict__ out3, float* __restrict__ out4,
                                               const QuadArgs& qa) {
  constexpr int ROWS = quad_rows<TY>();
  constexpr int PLANE = ROWS * kQuadStride;      // floats per staged plane
  extern __shared__ float sm[];
  float* bufA = sm;                  // [2][ROWS][stride]
  float* bufB = sm + 2 * PLANE;
  float* kxs = sm + 4 * PLANE;       // cx
  float* kys = sm + 5 * PLANE;       // cy
  float* kds = sm + 6 * PLANE;       // diagonal 1 + sum of the four face coefficients
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  constexpr int RPW = (ROWS + NW - 1) / NW;   // staged rows per warp
  F4 hreg[RPW][2];                             // bhat of this thread's rows, current pass
  const int gx0 = bx * kQuadInnerX - kQuadS;   // global x of staged column 0
  const int gy0 = by * TY - kQuadS;            // global y of staged row 0
  const int gx = gx0 + 4 * lane;
  const bool colok = gx >= 0 && gx < g.n0;             // four cells all in or all out (n0 % 4 == 0)
  const int64_t N = g.N;

  // zero the padding columns once (read as neighbours of edge cells that no valid cell uses)
  for (int i = threadIdx.x; i < 8 * ROWS; i += NT) {
    const int row = i >> 3, k = i & 7;
    const int col = (k < 4) ? k : kQuadPad + kQuadCols + (k - 4);
    float* base[7] = {bufA, bufA + PLANE, bufB, bufB + PLANE, kxs, kys, kds};
#pragma unroll
    for (int b = 0; b < 7; ++b) base[b][(size_t)row * kQuadStride + col] = 0.f;
  }
  // stage the face coefficients and the diagonal of the whole staged region (zero outside the grid)
  for (int ly = warp; ly < ROWS; ly += NW) {
    const int gy = gy0 + ly;
    const bool ok = colok && gy >= 0 && gy < g.n1;
    const int64_t c = (int64_t)g.n0 * gy + gx;
    const F4 a = ok ? ld4(cx + c) : zero4();
    const F4 b = ok ? ld4(cy + c) : zero4();
    const F4 bs = (ok && gy > 0) ? ld4(cy + c - g.n0) : zero4();
    float aw = __shfl_up_sync(0xffffffffu, a.v[3], 1);
    if (lane == 0) aw = (ok && gx > 0) ? __ldg(cx + c - 1) : 0.f;
    const float kw[4] = {aw, a.v[0], a.v[1], a.v[2]};
    F4 d;
#pragma unroll
    for (int e = 0; e < 4; ++e) d.v[e] = ok ? 1.f + ((a.v[e] + kw[e]) + (b.v[e] + bs.v[e])) : 0.f;
    st4(kxs + (size_t)ly * kQuadStride + kQuadPad + 4 * lane, a);
    st4(kys + (size_t)ly * kQuadStride + kQuadPad + 4 * lane, b);
    st4(kds + (size_t)ly * kQuadStride + kQuadPad + 4 * lane, d);
  }

  const int npass = ELL / 2;
  for (int pass = 0; pass < npass; ++pass) {
    // The pass body is instantiated for the real pair (pass 0) and for a complex frequency, so
    // the level loop carries no run-time branch on the pass type.
    auto run = [&](auto cplx_c) {
      constexpr bool cplx = decltype(cplx_c)::value;
      // planes of this pass: (0, 1) = the two real frequencies, else (2m, 2m+1) for complex m = pass
      const int p0 = (pass == 0) ? 0 : 2 * pass;
      const int p1 = p0 + 1;
      const int m0 = (pass == 0) ? 0 : pass;      // frequency of plane p0
      const int m1 = (pass == 0) ? ELL / 2 : pass;  // frequency of plane p1
      __syncthreads();  // previous pass finished reading the buffers
      // ---- stage x_k (bufA) and x_{k-1} (bufB) on the staged region; bhat into registers
#pragma unroll
      for (int rr = 0; rr < RPW; ++rr) {
        const int ly = warp + rr * NW;
        if (ly >= ROWS) break;
        const int gy = gy0 + ly;
        const bool ok = colok && gy >= 0 && gy < g.n1;
        const int64_t c = (int64_t)g.n0 * gy + gx;
        const size_t o = (size_t)ly * kQuadStride + kQuadPad + 4 * lane;
        const F4 x0 = ok ? ld4(xk + p0 * N + c) : zero4();
        const F4 x1 = ok ? ld4(xk + p1 * N + c) : zero4();
        const F4 h0 = ok ? ld4(bhat + p0 * N + c) : zero4();
        const F4 h1 = ok ? ld4(bhat + p1 * N + c) : zero4();
        F4 m0v, m1v;
        if (PSRC == 2) {
          m0v = ok ? ld4(xkm1 + p0 * N + c) : zero4();
          m1v = ok ? ld4(xkm1 + p1 * N + c) : zero4();
        } else {
          // x_1 = bhat / theta
          const StepArgs<float>& s0 = qa.s[0];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (cplx) {
              m0v.v[e] = h0.v[e] * s0.it_re[m0] - h1.v[e] * s0.it_im[m0];
              m1v.v[e] = h0.v[e] * s0.it_im[m0] + h1.v[e] * s0.it_re[m0];
            } else {
              m0v.v[e] = h0.v[e] * s0.it_re[m0];
              m1v.v[e] = h1.v[e] * s0.it_re[m1];
            }
          }
        }
        st4(bufA + o, x0);
        st4(bufA + PLANE + o, x1);
        st4(bufB + o, m0v);
        st4(bufB + PLANE + o, m1v);
        hreg[rr][0] = h0;
        hreg[rr][1] = h1;
      }
      // ---- four levels; level q+1 lives where level q-1 was
      float* cur = bufA;   // level q
      float* oth = bufB;   // level q-1, overwritten by level q+1
#pragma unroll
      for (int lv = 0; lv < kQuadS; ++lv) {
        __syncthreads();
        const StepArgs<float>& st = qa.s[lv];
        const int lo = lv + 1;  // valid region of the new level: rows/cols [lo, extent - lo)
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
          const int ly = warp + rr * NW;
          if (ly >= ROWS) break;
          if (ly < lo || ly >= ROWS - lo) continue;
          const size_t o = (size_t)ly * kQuadStride + kQuadPad + 4 * lane;
          // coefficients of the four cells (E: own cx, W: cx of the left cell, N: own cy, S: cy of the row below)
          const float4 kxe = *reinterpret_cast<const float4*>(kxs + o);
          const float kxw = kxs[o - 1];
          const float4 kyn = *reinterpret_cast<const float4*>(kys + o);
          const float4 kys_ = *reinterpret_cast<const float4*>(kys + o - kQuadStride);
          const float4 kdd = *reinterpret_cast<const float4*>(kds + o);
          const float kE[4] = {kxe.x, kxe.y, kxe.z, kxe.w};
          const float kW[4] = {kxw, kxe.x, kxe.y, kxe.z};
          const float kN[4] = {kyn.x, kyn.y, kyn.z, kyn.w};
          const float kS[4] = {kys_.x, kys_.y, kys_.z, kys_.w};
          const float kD[4] = {kdd.x, kdd.y, kdd.z, kdd.w};
          // nb[pl][e] = bhat + sum of kappa * neighbour values; xc = centre; xm = level q-1
          float nb[2][4], xc[2][4], xm[2][4];
#pragma unroll
          for (int pl = 0; pl < 2; ++pl) {
            const float* rp = cur + (size_t)pl * PLANE + o;
            const float4 cc = *reinterpret_cast<const float4*>(rp);
            const float4 nn = *reinterpret_cast<const float4*>(rp + kQuadStride);
            const float4 ss = *reinterpret_cast<const float4*>(rp - kQuadStride);
            const float left = rp[-1], right = rp[4];
            const float c4[4] = {cc.x, cc.y, cc.z, cc.w};
            const float n4[4] = {nn.x, nn.y, nn.z, nn.w};
            const float s4[4] = {ss.x, ss.y, ss.z, ss.w};
            const float4 mm = *reinterpret_cast<const float4*>(oth + (size_t)pl * PLANE + o);
            const float m4[4] = {mm.x, mm.y, mm.z, mm.w};
            const F4& h4v = hreg[rr][pl];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float xe = (e < 3) ? c4[e + 1] : right;
              const float xw = (e > 0) ? c4[e - 1] : left;
              float acc = fmaf(kE[e], xe, h4v.v[e]);
              acc = fmaf(kW[e], xw, acc);
              acc = fmaf(kN[e], n4[e], acc);
              acc = fmaf(kS[e], s4[e], acc);
              nb[pl][e] = acc;
              xc[pl][e] = c4[e];
              xm[pl][e] = m4[e];
            }
          }
          float n0v[4], n1v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (cplx) {
              const float lr = st.lam_re[m0], li = st.lam_im[m0];
              const float ar = st.a_re[m0], ai = st.a_im[m0], gr = st.g_re[m0], gi = st.g_im[m0];
              const float xr = xc[0][e], xi = xc[1][e];
              const float dl = kD[e] - lr;
              // b - (A - lambda) x, real and imaginary parts
              const float rr_ = fmaf(-li, xi, fmaf(-dl, xr, nb[0][e]));
              const float ri = fmaf(li, xr, fmaf(-dl, xi, nb[1][e]));
              const float dr = xr - xm[0][e], di = xi - xm[1][e];
              n0v[e] = fmaf(-gi, ri, fmaf(gr, rr_, fmaf(-ai, di, fmaf(ar, dr, xr))));
              n1v[e] = fmaf(gi, rr_, fmaf(gr, ri, fmaf(ai, dr, fmaf(ar, di, xi))));
            } else {
              const float r0 = fmaf(-(kD[e] - st.lam_re[m0]), xc[0][e], nb[0][e]);
              const float r1 = fmaf(-(kD[e] - st.lam_re[m1]), xc[1][e], nb[1][e]);
              n0v[e] = fmaf(st.g_re[m0], r0, fmaf(st.a_re[m0], xc[0][e] - xm[0][e], xc[0][e]));
              n1v[e] = fmaf(st.g_re[m1], r1, fmaf(st.a_re[m1], xc[1][e] - xm[1][e], xc[1][e]));
            }
          }
          *reinterpret_cast<float4*>(oth + o) = make_float4(n0v[0], n0v[1], n0v[2], n0v[3]);
          *reinterpret_cast<float4*>(oth + PLANE + o) = make_float4(n1v[0], n1v[1], n1v[2], n1v[3]);
        }
        float* t = cur;
        cur = oth;
        oth = t;
      }
      __syncthreads();
      // ---- write the interior: level 4 (cur) -> out4, level 3 (oth) -> out3
      if (lane >= 1 && lane <= 30 && colok) {
        for (int ly = kQuadS + warp; ly < kQuadS + TY; ly += NW) {
          const int gy = gy0 + ly;
          if (gy >= g.n1) break;
          const int64_t c = (int64_t)g.n0 * gy + gx;
          const size_t o = (size_t)ly * kQuadStride + kQuadPad + 4 * lane;
          *reinterpret_cast<float4*>(out4 + p0 * N + c) = *reinterpret_cast<const float4*>(cur + o);
          *reinterpret_cast<float4*>(out4 + p1 * N + c) = *reinterpret_cast<const float4*>(cur + PLANE + o);
          *reinterpret_cast<float4*>(out3 + p0 * N + c) = *reinterpret_cast<const float4*>(oth + o);
          *reinterpret_cast<float4*>(out3 + p1 * N + c) = *reinterpret_cast<const float4*>(oth + PLANE + o);
        }
      }
    };
    if (pass == 0) run(std::false_type{});
    else run(std::true_type{});
  }
}

template <int ELL, int TY, int PSRC, int NT>
__global__ void __launch_bounds__(NT)
    k_cheb_quad(GridDesc g, const float* __restrict__ cx, const float* __restrict__ cy,
                const float* __restrict__ bhat, const float* __restrict__ xk, const float* __restrict__ xkm1,
                float* __restrict__ out3, float* __restrict__ out4, const __grid_constant__ QuadArgs qa) {
  cheb_quad_body<ELL, TY, PSRC, NT>(g, blockIdx.x, blockIdx.y, cx, cy, bhat, xk, xkm1, out3, out4, qa);
}

template <int ELL, int TY, int NT>
cudaError_t launch_quad_cfg(const GridDesc& g, int psrc, const float* cx, const float* cy, const float* bhat,
                            const float* xk, const float* xkm1, float* out3, float* out4, const QuadArgs& qa,
                            cudaStream_t s) {
  const dim3 block(NT, 1, 1);
  const dim3 grid((unsigned)((g.n0 + kQuadInnerX - 1) / kQuadInnerX), (unsigned)((g.n1 + TY - 1) / TY), 1);
  const size_t smem = quad_smem_bytes<TY>();
  cudaError_t e;
  if (psrc == 1) {
    e = cudaFuncSetAttribute(k_cheb_quad<ELL, TY, 1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cheb_quad<ELL, TY, 1, NT><<<grid, block, smem, s>>>(g, cx, cy, bhat, xk, xkm1, out3, out4, qa);
  } else {
    e = cudaFuncSetAttribute(k_cheb_quad<ELL, TY, 2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cheb_quad<ELL, TY, 2, NT><<<grid, block, smem, s>>>(g, cx, cy, bhat, xk, xkm1, out3, out4, qa);
  }
  count_launch();
  return cudaGetLastError();
}

template <int ELL>
cudaError_t launch_quad_ell(const GridDesc& g, int psrc, const float* cx, const float* cy, const float* bhat,
                            const float* xk, const float* xkm1, float* out3, float* out4, const QuadArgs& qa,
                            cudaStream_t s) {
  return launch_quad_cfg<ELL, kQuadTileTY, kQuadTileNT>(g, psrc, cx, cy, bhat, xk, xkm1, out3, out4, qa, s);
}

}  // namespace aao
