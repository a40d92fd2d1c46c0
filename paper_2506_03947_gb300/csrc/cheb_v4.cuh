// Vectorised FP32 Chebyshev step: four consecutive cells along x per thread.
//
// Same arithmetic as k_cheb_step (three-term Chebyshev step on every
// frequency, Eq. 7 over Lemma 2's segment), organised for memory-level
// parallelism on the mixed path: every plane access is one 16-byte load per
// thread (a warp covers 128 consecutive cells of one row), the x-neighbours
// at the ends of a thread's four cells come from the adjacent lanes by warp
// shuffle, and only the two cells at a warp's edges are loaded separately.
// Used when n0 is a multiple of 4 (16-byte aligned rows and planes).
#pragma once

#include "aao_internal.cuh"

namespace aao {

struct F4 {
  float v[4];
};

__device__ __forceinline__ F4 ld4(const float* __restrict__ p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ F4 ld4_rw(const float* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st4(float* p, const F4& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ F4 zero4() { return F4{{0.f, 0.f, 0.f, 0.f}}; }

template <int DIM>
struct Stencil4 {
  F4 kE, kW, kN, kS, kU, kD;   // face coefficients of the four cells
  int64_t oN, oS, oU, oD;      // neighbour offsets (0 where the neighbour does not exist)
  bool act, west, east;        // thread has cells; a cell exists left / right of the four
};

// A v on one plane for the thread's four cells; returns A v and the centre values.
template <int DIM>
__device__ __forceinline__ F4 apply_A4(const float* __restrict__ p, int64_t c, int lane, const Stencil4<DIM>& s,
                                       F4& vc) {
  vc = s.act ? ld4(p + c) : zero4();
  float left = __shfl_up_sync(0xffffffffu, vc.v[3], 1);
  float right = __shfl_down_sync(0xffffffffu, vc.v[0], 1);
  if (lane == 0) left = (s.act && s.west) ? __ldg(p + c - 1) : 0.f;
  if (lane == 31) right = (s.act && s.east) ? __ldg(p + c + 4) : 0.f;
  F4 vn = zero4(), vs = zero4(), vu = zero4(), vd = zero4();
  if (DIM >= 2 && s.act) {
    vn = ld4(p + c + s.oN);
    vs = ld4(p + c + s.oS);
  }
  if (DIM == 3 && s.act) {
    vu = ld4(p + c + s.oU);
    vd = ld4(p + c + s.oD);
  }
  F4 a;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float x = vc.v[e];
    const float xe = (e < 3) ? vc.v[e + 1] : right;
    const float xw = (e > 0) ? vc.v[e - 1] : left;
    float acc = x;
    acc += s.kE.v[e] * (x - xe);
    acc += s.kW.v[e] * (x - xw);
    if (DIM >= 2) {
      acc += s.kN.v[e] * (x - vn.v[e]);
      acc += s.kS.v[e] * (x - vs.v[e]);
    }
    if (DIM == 3) {
      acc += s.kU.v[e] * (x - vu.v[e]);
      acc += s.kD.v[e] * (x - vd.v[e]);
    }
    a.v[e] = acc;
  }
  return a;
}

// The thread's four cells of block (bx, by, bz): their first cell index and the face
// coefficients of the stencil (loaded once; the multi-right-hand-side kernels apply them to
// several fields).  Returns false when the thread's row is outside the grid (uniform across a
// warp, which shares j and k).
template <int DIM>
__device__ __forceinline__ bool make_stencil4(const GridDesc& g, int bx, int by, int bz, const float* __restrict__ cx,
                                              const float* __restrict__ cy, const float* __restrict__ cz,
                                              Stencil4<DIM>& st, int64_t& c) {
  const int lane = threadIdx.x & 31;
  const int i0 = (bx * blockDim.x + threadIdx.x) * 4;
  const int j = by * blockDim.y + threadIdx.y;
  const int k = bz;
  if (j >= g.n1) return false;
  const int64_t pl = (int64_t)g.n0 * g.n1;
  c = (int64_t)g.n0 * (j + (int64_t)g.n1 * k) + i0;
  st.act = i0 < g.n0;
  st.west = i0 > 0;
  st.east = i0 + 4 < g.n0;
  st.kE = st.act ? ld4(cx + c) : zero4();
  {
    float kprev = __shfl_up_sync(0xffffffffu, st.kE.v[3], 1);
    if (lane == 0) kprev = (st.act && st.west) ? __ldg(cx + c - 1) : 0.f;
    st.kW = F4{{kprev, st.kE.v[0], st.kE.v[1], st.kE.v[2]}};
  }
  st.oN = st.oS = st.oU = st.oD = 0;
  if (DIM >= 2) {
    st.oN = (j < g.n1 - 1) ? g.n0 : 0;
    st.oS = (j > 0) ? -(int64_t)g.n0 : 0;
    st.kN = st.act ? ld4(cy + c) : zero4();
    st.kS = (st.act && j > 0) ? ld4(cy + c - g.n0) : zero4();
  }
  if (DIM == 3) {
    st.oU = (k < g.n2 - 1) ? pl : 0;
    st.oD = (k > 0) ? -pl : 0;
    st.kU = st.act ? ld4(cz + c) : zero4();
    st.kD = (st.act && k > 0) ? ld4(cz + c - pl) : zero4();
  }
  return true;
}

// One Chebyshev step of one field set on the thread's four cells (stencil from make_stencil4).
template <int ELL, int DIM, int KSRC, int PSRC, bool LAST>
__device__ __forceinline__ void cheb_step_v4_apply(const GridDesc& g, const Stencil4<DIM>& st, int64_t c,
                                                   const float* __restrict__ bhat, const float* __restrict__ xk,
                                                   float* xio, double* __restrict__ z, const StepArgs<float>& sa,
                                                   const IdftArgs<float>& ia) {
  const int lane = threadIdx.x & 31;
  const int64_t N = g.N;
  const float* src = (KSRC == 0) ? bhat : xk;

  float zt[LAST ? 4 : 1][LAST ? ELL : 1];
  if constexpr (LAST) {
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int t = 0; t < ELL; ++t) zt[e][t] = 0.f;
  }

  // real frequencies: m = 0 (plane 0) and m = ELL/2 (plane 1)
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int m = (r == 0) ? 0 : ELL / 2;
    F4 vc;
    const F4 Av = apply_A4<DIM>(src + r * N, c, lane, st, vc);
    const F4 b = (KSRC == 0) ? vc : (st.act ? ld4(bhat + r * N + c) : zero4());
    const F4 xm = (PSRC == 2 && st.act) ? ld4_rw(xio + r * N + c) : zero4();
    F4 xn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float x, Ax, xmm;
      if (KSRC == 0) {
        x = vc.v[e] * sa.it_re[m];
        Ax = Av.v[e] * sa.it_re[m];
      } else {
        x = vc.v[e];
        Ax = Av.v[e];
      }
      if (PSRC == 0) xmm = 0.f;
      else if (PSRC == 1) xmm = b.v[e] * sa.it_re[m];
      else xmm = xm.v[e];
      const float res = b.v[e] - Ax + sa.lam_re[m] * x;
      xn.v[e] = x + sa.a_re[m] * (x - xmm) + sa.g_re[m] * res;
    }
    if constexpr (!LAST) {
      if (st.act) st4(xio + r * N + c, xn);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < ELL; ++t) zt[e][t] += xn.v[e] * ia.ci[t][m];
    }
  }

  // complex frequencies m = 1 .. ELL/2-1 (planes 2m, 2m+1)
#pragma unroll
  for (int m = 1; m < ELL / 2; ++m) {
    const int64_t pr = (int64_t)(2 * m) * N, pi = (int64_t)(2 * m + 1) * N;
    F4 vr, vi;
    const F4 Ar = apply_A4<DIM>(src + pr, c, lane, st, vr);
    const F4 Ai = apply_A4<DIM>(src + pi, c, lane, st, vi);
    F4 br, bi;
    if (KSRC == 0) {
      br = vr;
      bi = vi;
    } else {
      br = st.act ? ld4(bhat + pr + c) : zero4();
      bi = st.act ? ld4(bhat + pi + c) : zero4();
    }
    F4 mr = zero4(), mi = zero4();
    if (PSRC == 2 && st.act) {
      mr = ld4_rw(xio + pr + c);
      mi = ld4_rw(xio + pi + c);
    }
    const float itr = sa.it_re[m], iti = sa.it_im[m];
    const float lr = sa.lam_re[m], li = sa.lam_im[m];
    const float ar = sa.a_re[m], ai = sa.a_im[m], gr = sa.g_re[m], gi = sa.g_im[m];
    F4 nr4, ni4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float xr, xi, Axr, Axi;
      if (KSRC == 0) {
        xr = vr.v[e] * itr - vi.v[e] * iti;
        xi = vr.v[e] * iti + vi.v[e] * itr;
        Axr = Ar.v[e] * itr - Ai.v[e] * iti;
        Axi = Ar.v[e] * iti + Ai.v[e] * itr;
      } else {
        xr = vr.v[e];
        xi = vi.v[e];
        Axr = Ar.v[e];
        Axi = Ai.v[e];
      }
      float pr_, pi_;
      if (PSRC == 0) {
        pr_ = 0.f;
        pi_ = 0.f;
      } else if (PSRC == 1) {
        pr_ = br.v[e] * itr - bi.v[e] * iti;
        pi_ = br.v[e] * iti + bi.v[e] * itr;
      } else {
        pr_ = mr.v[e];
        pi_ = mi.v[e];
      }
      const float rr = br.v[e] - Axr + (lr * xr - li * xi);
      const float ri = bi.v[e] - Axi + (lr * xi + li * xr);
      const float dr = xr - pr_, di = xi - pi_;
      nr4.v[e] = xr + (ar * dr - ai * di) + (gr * rr - gi * ri);
      ni4.v[e] = xi + (ar * di + ai * dr) + (gr * ri + gi * rr);
    }
    if constexpr (!LAST) {
      if (st.act) {
        st4(xio + pr + c, nr4);
        st4(xio + pi + c, ni4);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int t = 0; t < ELL; ++t) zt[e][t] += nr4.v[e] * ia.ci[t][m] - ni4.v[e] * ia.si[t][m];
    }
  }

  if constexpr (LAST) {
    if (st.act) {
#pragma unroll
      for (int t = 0; t < ELL; ++t) {
        double2* zp = reinterpret_cast<double2*>(z + (int64_t)t * N + c);
        const float gmul = ia.igamma_T[t];
        zp[0] = make_double2(f2d_exact(zt[0][t] * gmul), f2d_exact(zt[1][t] * gmul));
        zp[1] = make_double2(f2d_exact(zt[2][t] * gmul), f2d_exact(zt[3][t] * gmul));
      }
    }
  }
}

// Body of one block (bx, by, bz) of the step; shared by the single-instance and
// the batched kernels.
template <int ELL, int DIM, int KSRC, int PSRC, bool LAST>
__device__ __forceinline__ void cheb_step_v4_body(const GridDesc& g, int bx, int by, int bz,
                                                  const float* __restrict__ cx, const float* __restrict__ cy,
                                                  const float* __restrict__ cz, const float* __restrict__ bhat,
                                                  const float* __restrict__ xk, float* xio,
                                                  double* __restrict__ z, const StepArgs<float>& sa,
                                                  const IdftArgs<float>& ia) {
  Stencil4<DIM> st;
  int64_t c = 0;
  if (!make_stencil4<DIM>(g, bx, by, bz, cx, cy, cz, st, c)) return;
  cheb_step_v4_apply<ELL, DIM, KSRC, PSRC, LAST>(g, st, c, bhat, xk, xio, z, sa, ia);
}

template <int ELL, int DIM, int KSRC, int PSRC, bool LAST>
__global__ void __launch_bounds__(256)
    k_cheb_step_v4(GridDesc g, const float* __restrict__ cx, const float* __restrict__ cy,
                   const float* __restrict__ cz, const float* __restrict__ bhat, const float* __restrict__ xk,
                   float* xio, double* __restrict__ z, const __grid_constant__ StepArgs<float> sa,
                   const __grid_constant__ IdftArgs<float> ia) {
  cheb_step_v4_body<ELL, DIM, KSRC, PSRC, LAST>(g, blockIdx.x, blockIdx.y, blockIdx.z, cx, cy, cz, bhat, xk, xio, z,
                                                sa, ia);
}

}  // namespace aao
