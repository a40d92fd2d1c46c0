// Four Chebyshev steps per launch (2D, FP32), persistent, TMA-fed.
//
// Same arithmetic as the shared-memory tile kernel (cheb_quad.cuh): steps
// k .. k+3 of the Chebyshev semi-iteration (Eq. 7 over Lemma 2's segment) on
// every frequency,
//   x_{q+1} = x_q + a_q (x_q - x_{q-1}) + g_q (bhat - A x_q + lambda x_q),
// with the residual formed as bhat + sum_f kappa_f x_nbr(f) - (d - lambda) x
// (d = 1 + sum of the four face coefficients).
//
// Organisation (one CTA per SM, persistent over tiles):
//  * A tile is 120 x 22 interior cells plus a four-cell halo: 128 x 30 staged
//    cells.  Warp w owns staged rows R*w .. R*w+R-1 and lane l owns columns
//    4l .. 4l+3 of them for the whole tile; the face coefficients and the
//    diagonal of those cells live in registers across all ell/2 passes.
//  * A pass handles one plane pair (the two real frequencies, then each
//    complex one).  Its x_k, x_{k-1} and bhat tiles (three boxes of
//    128 x 30 x 2 floats) arrive by TMA into one of two shared-memory stages;
//    the copy of the next pass (or the next tile's first pass) is issued as
//    soon as the current one has landed, so loads overlap a whole pass of
//    arithmetic.
//  * Each thread keeps its cells' two newest levels and bhat in registers.
//    Only the first and last row of every warp go through shared memory
//    (into the consumed x_{k-1} / bhat boxes of the current stage), so a
//    level costs one barrier and, per warp row pair, two stores and two
//    loads per plane; east/west neighbours come from warp shuffles.
//  * After four levels the interior (lanes 1..30, rows 4..25) holds x_{k+3}
//    and x_{k+4}; both are stored straight from registers.
// Every wait on a TMA transaction is bounded (wait_limit SM clocks, about a
// second by default); on expiry the block records the fault in the caller's device flag,
// waits (with the default bound) for its copies in flight and returns.
#include <cuda.h>

#include "aao_internal.cuh"

namespace aao {

static_assert(sizeof(FieldMap) == sizeof(CUtensorMap), "FieldMap must hold a CUtensorMap");
static_assert(alignof(FieldMap) >= 64, "FieldMap must be 64-byte aligned");

namespace {

constexpr int kS = 4;                   // fused steps = halo width
constexpr int kCols = 128;              // staged columns (32 lanes x 4)
constexpr int kInX = kCols - 2 * kS;    // 120 interior columns
constexpr int kTY = kQuadTmaTY;         // interior rows
constexpr int kRows = kTY + 2 * kS;     // staged rows
constexpr int kPlane = kRows * kCols;   // floats of one staged plane
constexpr int kBox = 2 * kPlane;        // floats of one box (two planes)
constexpr unsigned kBoxBytes = kBox * 4u;
constexpr int kStage = 3 * kBox;        // x_k, x_{k-1}, bhat boxes
constexpr int kCoefRows = kRows + 1;    // face coefficients: the staged rows and the row above them
constexpr int kCoef = kCoefRows * kCols;
constexpr unsigned kCoefBytes = 2u * kCoef * 4u;  // cx and cy boxes
constexpr size_t kSmemBytes = (size_t)2 * kStage * 4 + (size_t)kCoefBytes + 64;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Non-blocking test (try_wait above may suspend the thread for a while in hardware).
__device__ __forceinline__ bool mbar_peek(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of the given parity, for at most `limit` SM clocks (and 2^24 polls);
// a zero limit only tests once, without blocking.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit = kQuadTmaWaitCycles) {
  if (limit <= 0) return mbar_peek(bar, parity);
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_test(bar, parity)) return true;
    if (clock64() - t0 > limit) break;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_box(unsigned dst, const FieldMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const FieldMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <int R>
struct TileCoef {
  float kE[R][4], kN[R][4], kS0[4], kD[R][4];
};

// One level for the warp's R rows: cur (level q) -> prv (level q-1, overwritten by level q+1).
// nS / nN: level q of the rows just above and below the warp's rows.
template <int R, bool CPLX>
__device__ __forceinline__ void quad_level(float (&cur)[R][2][4], float (&prv)[R][2][4], const float (&hh)[R][2][4],
                                           const float (&nS)[2][4], const float (&nN)[2][4], const TileCoef<R>& tc,
                                           const float (&kW0)[R], const StepArgs<float>& st, int m0, int m1) {
  float nb[R][2][4];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      const float left = __shfl_up_sync(0xffffffffu, cur[r][pl][3], 1);
      const float right = __shfl_down_sync(0xffffffffu, cur[r][pl][0], 1);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float xe = (e < 3) ? cur[r][pl][e + 1] : right;
        const float xw = (e > 0) ? cur[r][pl][e - 1] : left;
        const float xn = (r < R - 1) ? cur[r + 1][pl][e] : nN[pl][e];
        const float xs = (r > 0) ? cur[r - 1][pl][e] : nS[pl][e];
        const float kw = (e > 0) ? tc.kE[r][e - 1] : kW0[r];
        const float ks = (r > 0) ? tc.kN[r - 1][e] : tc.kS0[e];
        float acc = fmaf(tc.kE[r][e], xe, hh[r][pl][e]);
        acc = fmaf(kw, xw, acc);
        acc = fmaf(tc.kN[r][e], xn, acc);
        acc = fmaf(ks, xs, acc);
        nb[r][pl][e] = acc;
      }
    }
  }
  if (CPLX) {
    const float lr = st.lam_re[m0], li = st.lam_im[m0];
    const float ar = st.a_re[m0], ai = st.a_im[m0], gr = st.g_re[m0], gi = st.g_im[m0];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float xr = cur[r][0][e], xi = cur[r][1][e];
        const float dl = tc.kD[r][e] - lr;
        const float rr = fmaf(-li, xi, fmaf(-dl, xr, nb[r][0][e]));
        const float ri = fmaf(li, xr, fmaf(-dl, xi, nb[r][1][e]));
        const float dr = xr - prv[r][0][e], di = xi - prv[r][1][e];
        prv[r][0][e] = fmaf(-gi, ri, fmaf(gr, rr, fmaf(-ai, di, fmaf(ar, dr, xr))));
        prv[r][1][e] = fmaf(gi, rr, fmaf(gr, ri, fmaf(ai, dr, fmaf(ar, di, xi))));
      }
    }
  } else {
    const float l0 = st.lam_re[m0], l1 = st.lam_re[m1];
    const float a0 = st.a_re[m0], a1 = st.a_re[m1], g0 = st.g_re[m0], g1 = st.g_re[m1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x0 = cur[r][0][e], x1 = cur[r][1][e];
        const float r0 = fmaf(-(tc.kD[r][e] - l0), x0, nb[r][0][e]);
        const float r1 = fmaf(-(tc.kD[r][e] - l1), x1, nb[r][1][e]);
        prv[r][0][e] = fmaf(g0, r0, fmaf(a0, x0 - prv[r][0][e], x0));
        prv[r][1][e] = fmaf(g1, r1, fmaf(a1, x1 - prv[r][1][e], x1));
      }
    }
  }
}

// Rows just above / below the warp's rows, level q, from a staged box (zero outside the tile).
template <int R>
__device__ __forceinline__ void load_halo_rows(const float* box, int ly0, int lane, float (&nS)[2][4],
                                               float (&nN)[2][4]) {
#pragma unroll
  for (int pl = 0; pl < 2; ++pl) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f), n = s;
    if (ly0 > 0) s = lds4(box + pl * kPlane + (ly0 - 1) * kCols + 4 * lane);
    if (ly0 + R < kRows) n = lds4(box + pl * kPlane + (ly0 + R) * kCols + 4 * lane);
    nS[pl][0] = s.x, nS[pl][1] = s.y, nS[pl][2] = s.z, nS[pl][3] = s.w;
    nN[pl][0] = n.x, nN[pl][1] = n.y, nN[pl][2] = n.z, nN[pl][3] = n.w;
  }
}

// The warp's first and last rows of a new level, for the neighbouring warps.
template <int R>
__device__ __forceinline__ void store_edge_rows(float* box, int ly0, int lane, const float (&v)[R][2][4]) {
#pragma unroll
  for (int pl = 0; pl < 2; ++pl) {
    sts4(box + pl * kPlane + ly0 * kCols + 4 * lane, v[0][pl]);
    if (R > 1) sts4(box + pl * kPlane + (ly0 + R - 1) * kCols + 4 * lane, v[R - 1][pl]);
  }
}

// Thread 0: issue the box copies of iteration it (tile, pass) into stage it & 1.
template <int NPASS, int PSRC>
__device__ __forceinline__ void issue_pass(int it, float* sm, unsigned long long* bars, int ntx, const FieldMap* mxk,
                                           const FieldMap* mxkm1, const FieldMap* mbhat) {
  const int tile = (int)blockIdx.x + (it / NPASS) * (int)gridDim.x;
  const int pass = it % NPASS;
  const int tx = tile % ntx, ty = tile / ntx;
  const int x = tx * kInX - kS, y = ty * kTY - kS, z = (pass == 0) ? 0 : 2 * pass;
  float* st = sm + (it & 1) * kStage;
  const unsigned bar = smem_u32(&bars[it & 1]);
  mbar_arrive_tx(bar, (PSRC == 2 ? 3u : 2u) * kBoxBytes);
  tma_load_box(smem_u32(st), mxk, x, y, z, bar);
  if (PSRC == 2) tma_load_box(smem_u32(st + kBox), mxkm1, x, y, z, bar);
  tma_load_box(smem_u32(st + 2 * kBox), mbhat, x, y, z, bar);
}

// Thread 0: issue the face-coefficient boxes of the block's j-th tile (rows gy0-1 .. gy0+kRows-1).
__device__ __forceinline__ void issue_coef(int j, float* coef, unsigned long long* bars, int ntx, const FieldMap* mcx,
                                           const FieldMap* mcy) {
  const int tile = (int)blockIdx.x + j * (int)gridDim.x;
  const int tx = tile % ntx, ty = tile / ntx;
  const unsigned bar = smem_u32(&bars[2]);
  mbar_arrive_tx(bar, kCoefBytes);
  tma_load_2d(smem_u32(coef), mcx, tx * kInX - kS, ty * kTY - kS - 1, bar);
  tma_load_2d(smem_u32(coef + kCoef), mcy, tx * kInX - kS, ty * kTY - kS - 1, bar);
}

// One pass: the four levels on one plane pair, from the staged boxes to the interior outputs.
// CPLX: the pair is Re/Im of the complex frequency m0 (else the real frequencies m0 and m1);
// the choice is made once per pass, outside the level code.
template <int ELL, int R, int PSRC, bool CPLX>
__device__ __forceinline__ void quad_pass(const float* X, float* M, float* H, int ly0, int lane, const TileCoef<R>& tc,
                                          const float (&kW0)[R], const QuadSteps& qa, int m0, int m1, bool colok,
                                          int gy0, int gx, const GridDesc& g, int p0, float* __restrict__ out3,
                                          float* __restrict__ out4) {
  const int64_t N = g.N;
  float xa[R][2][4], xb[R][2][4], hh[R][2][4];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int o = (ly0 + r) * kCols + 4 * lane;
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      const float4 x = lds4(X + pl * kPlane + o);
      const float4 h = lds4(H + pl * kPlane + o);
      xa[r][pl][0] = x.x, xa[r][pl][1] = x.y, xa[r][pl][2] = x.z, xa[r][pl][3] = x.w;
      hh[r][pl][0] = h.x, hh[r][pl][1] = h.y, hh[r][pl][2] = h.z, hh[r][pl][3] = h.w;
      if (PSRC == 2) {
        const float4 m = lds4(M + pl * kPlane + o);
        xb[r][pl][0] = m.x, xb[r][pl][1] = m.y, xb[r][pl][2] = m.z, xb[r][pl][3] = m.w;
      }
    }
    if (PSRC != 2) {
      // x_1 = bhat / theta (complex division for a complex frequency)
      const StepArgs<float>& s0 = qa.s[0];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float h0 = hh[r][0][e], h1 = hh[r][1][e];
        if (CPLX) {
          xb[r][0][e] = h0 * s0.it_re[m0] - h1 * s0.it_im[m0];
          xb[r][1][e] = h0 * s0.it_im[m0] + h1 * s0.it_re[m0];
        } else {
          xb[r][0][e] = h0 * s0.it_re[m0];
          xb[r][1][e] = h1 * s0.it_re[m1];
        }
      }
    }
  }
  float nS[2][4], nN[2][4];
  // level 0 -> 1 (neighbours from the x_k box), edge rows of level 1 into M
  load_halo_rows<R>(X, ly0, lane, nS, nN);
  quad_level<R, CPLX>(xa, xb, hh, nS, nN, tc, kW0, qa.s[0], m0, m1);
  store_edge_rows<R>(M, ly0, lane, xb);
  __syncthreads();
  // level 1 -> 2, edge rows into H
  load_halo_rows<R>(M, ly0, lane, nS, nN);
  quad_level<R, CPLX>(xb, xa, hh, nS, nN, tc, kW0, qa.s[1], m0, m1);
  store_edge_rows<R>(H, ly0, lane, xa);
  __syncthreads();
  // level 2 -> 3, edge rows into M (level 1 there has been read by everyone)
  load_halo_rows<R>(H, ly0, lane, nS, nN);
  quad_level<R, CPLX>(xa, xb, hh, nS, nN, tc, kW0, qa.s[2], m0, m1);
  store_edge_rows<R>(M, ly0, lane, xb);
  __syncthreads();
  // level 3 -> 4
  load_halo_rows<R>(M, ly0, lane, nS, nN);
  quad_level<R, CPLX>(xb, xa, hh, nS, nN, tc, kW0, qa.s[3], m0, m1);

  // interior: level 4 (xa) -> out4, level 3 (xb) -> out3
  if (lane >= 1 && lane <= 30 && colok) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ly = ly0 + r;
      const int gy = gy0 + ly;
      if (ly < kS || ly >= kS + kTY || gy >= g.n1) continue;
      const int64_t c = (int64_t)g.n0 * gy + gx;
#pragma unroll
      for (int pl = 0; pl < 2; ++pl) {
        const int64_t o = (int64_t)(p0 + pl) * N + c;
        *reinterpret_cast<float4*>(out4 + o) = make_float4(xa[r][pl][0], xa[r][pl][1], xa[r][pl][2], xa[r][pl][3]);
        *reinterpret_cast<float4*>(out3 + o) = make_float4(xb[r][pl][0], xb[r][pl][1], xb[r][pl][2], xb[r][pl][3]);
      }
    }
  }
}

// PSRC: x_{k-1} = bhat/theta (1, first fused step is k = 2) or the staged x_{k-1} box (2).
template <int ELL, int R, int PSRC>
__global__ void __launch_bounds__(32 * kRows / R, 1)
    k_cheb_quad_tma(GridDesc g, int ntx, int ntiles, const __grid_constant__ FieldMap mcx,
                    const __grid_constant__ FieldMap mcy, const __grid_constant__ FieldMap mxk,
                    const __grid_constant__ FieldMap mxkm1, const __grid_constant__ FieldMap mbhat,
                    float* __restrict__ out3, float* __restrict__ out4, QuadSteps qa, long long wait_limit,
                    unsigned* __restrict__ fault) {
  constexpr int NPASS = ELL / 2;
  extern __shared__ __align__(1024) float sm[];
  float* coef = sm + 2 * kStage;  // cx box, then cy box: [kCoefRows][kCols], row j = staged row j - 1
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(coef + 2 * kCoef);  // stage 0, stage 1, coef
  volatile int* s_abort = reinterpret_cast<volatile int*>(bars + 3);
  const int lane = threadIdx.x & 31;
  const int ly0 = (threadIdx.x >> 5) * R;
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int total = my_tiles * NPASS;

  if (threadIdx.x == 0) {
    *s_abort = (smem_u32(sm) & 127u) ? 1 : 0;
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    mbar_init(smem_u32(&bars[2]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  __syncthreads();
  if (*s_abort) {
    if (threadIdx.x == 0) atomicOr(fault, 2u);
    return;
  }

  if (threadIdx.x == 0 && total > 0) {
    issue_pass<NPASS, PSRC>(0, sm, bars, ntx, &mxk, &mxkm1, &mbhat);
    issue_coef(0, coef, bars, ntx, &mcx, &mcy);
  }

  TileCoef<R> tc;
  float kW0[R];
  int it = 0;
  bool coef_wait_failed = false;
  for (; it < total; ++it) {
    const int j = it / NPASS;  // the block's tile counter
    const int tile = (int)blockIdx.x + j * (int)gridDim.x;
    const int pass = it - j * NPASS;
    const int tx = tile % ntx, ty = tile / ntx;
    const int gx = tx * kInX - kS + 4 * lane;
    const int gy0 = ty * kTY - kS;
    const bool colok = gx >= 0 && gx < g.n0;  // the four cells are all in or all out (n0 % 4 == 0)
    if (pass == 0) {
      // Face coefficients of the thread's cells (zero outside the grid, by the TMA fill) and the
      // diagonal d = 1 + sum of the four faces.  Lane 0's west face belongs to staged column 0,
      // whose new levels are never used; it is taken as 0.
      if (!mbar_wait(smem_u32(&bars[2]), (unsigned)j & 1u, wait_limit)) {
        *s_abort = 1;
        coef_wait_failed = true;
      }
      const float* CX = coef;
      const float* CY = coef + kCoef;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 a = lds4(CX + (ly0 + r + 1) * kCols + 4 * lane);
        const float4 b = lds4(CY + (ly0 + r + 1) * kCols + 4 * lane);
        tc.kE[r][0] = a.x, tc.kE[r][1] = a.y, tc.kE[r][2] = a.z, tc.kE[r][3] = a.w;
        tc.kN[r][0] = b.x, tc.kN[r][1] = b.y, tc.kN[r][2] = b.z, tc.kN[r][3] = b.w;
        const float w = __shfl_up_sync(0xffffffffu, a.w, 1);
        kW0[r] = (lane == 0) ? 0.f : w;
        if (r == 0) {
          const float4 sv = lds4(CY + ly0 * kCols + 4 * lane);
          tc.kS0[0] = sv.x, tc.kS0[1] = sv.y, tc.kS0[2] = sv.z, tc.kS0[3] = sv.w;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float kw = (e > 0) ? tc.kE[r][e - 1] : kW0[r];
          const float ks = (r > 0) ? tc.kN[r - 1][e] : tc.kS0[e];
          tc.kD[r][e] = 1.f + ((tc.kE[r][e] + kw) + (tc.kN[r][e] + ks));
        }
      }
    }
    // this iteration's boxes have landed; everyone is done with the other stage
    if (!mbar_wait(smem_u32(&bars[it & 1]), (unsigned)(it >> 1) & 1u, wait_limit)) *s_abort = 1;
    fence_async_smem();
    __syncthreads();
    if (*s_abort) break;
    if (threadIdx.x == 0) {
      if (it + 1 < total) issue_pass<NPASS, PSRC>(it + 1, sm, bars, ntx, &mxk, &mxkm1, &mbhat);
      // everyone has read this tile's coefficients (pass 0, before the barrier above)
      if (pass == 1 && j + 1 < my_tiles) issue_coef(j + 1, coef, bars, ntx, &mcx, &mcy);
    }

    float* X = sm + (it & 1) * kStage;  // x_k box; then the x_{k-1} box (M) and the bhat box (H)
    float* M = X + kBox;
    float* H = M + kBox;

    if (pass == 0)
      quad_pass<ELL, R, PSRC, false>(X, M, H, ly0, lane, tc, kW0, qa, 0, ELL / 2, colok, gy0, gx, g, 0, out3, out4);
    else
      quad_pass<ELL, R, PSRC, true>(X, M, H, ly0, lane, tc, kW0, qa, pass, pass, colok, gy0, gx, g, 2 * pass, out3,
                                    out4);
  }
  if (it < total) {
    // A wait expired: wait (bounded) for the copies in flight, record, return.  In flight are
    // this iteration's stage and, between pass 1 of a tile and pass 0 of the next, the
    // coefficient boxes of the next tile.
    if (threadIdx.x == 0) {
      const int j = it / NPASS, pass = it - j * NPASS;
      mbar_wait(smem_u32(&bars[it & 1]), (unsigned)(it >> 1) & 1u);
      if (pass == 0 && coef_wait_failed) mbar_wait(smem_u32(&bars[2]), (unsigned)j & 1u);
      else if (pass >= 1 && j + 1 < my_tiles) mbar_wait(smem_u32(&bars[2]), (unsigned)(j + 1) & 1u);
      atomicOr(fault, 1u);
    }
  }
}

template <int ELL, int R>
cudaError_t launch_qt(const GridDesc& g, int psrc, const FieldMap& mcx, const FieldMap& mcy, const FieldMap& mxk,
                      const FieldMap& mxkm1, const FieldMap& mbhat, float* out3, float* out4, const QuadSteps& qs,
                      long long wait_limit, unsigned* fault, cudaStream_t s) {
  constexpr int NT = 32 * kRows / R;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ntx = (g.n0 + kInX - 1) / kInX;
  const int nty = (g.n1 + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  const int grid = ntiles < nsm ? ntiles : nsm;
  if (psrc == 1) {
    auto k = k_cheb_quad_tma<ELL, R, 1>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, kSmemBytes, s>>>(g, ntx, ntiles, mcx, mcy, mxk, mxkm1, mbhat, out3, out4, qs, wait_limit, fault);
  } else {
    auto k = k_cheb_quad_tma<ELL, R, 2>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, kSmemBytes, s>>>(g, ntx, ntiles, mcx, mcy, mxk, mxkm1, mbhat, out3, out4, qs, wait_limit, fault);
  }
  count_launch();
  return cudaGetLastError();
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

namespace {

EncodeTiledFn encode_fn(cudaError_t* err) {
  static EncodeTiledFn fn = nullptr;
  *err = cudaSuccess;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    if (q != cudaDriverEntryPointSuccess || !p) {
      *err = cudaErrorNotSupported;
      return nullptr;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// FP32 tensor of rank 2 (n0, n1) or 3 (n0, n1, ell), zero fill outside, no swizzle.
cudaError_t encode(FieldMap* out, const float* base, const GridDesc& g, int rank, int ell, const cuuint32_t* box) {
  cudaError_t e;
  EncodeTiledFn fn = encode_fn(&e);
  if (!fn) return e;
  if (!out || !base || g.n0 % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u)) return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {(cuuint64_t)g.n0, (cuuint64_t)g.n1, (cuuint64_t)ell};
  const cuuint64_t strides[2] = {(cuuint64_t)g.n0 * 4u, (cuuint64_t)g.N * 4u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
                        const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_field_map(FieldMap* out, const float* base, const GridDesc& g, int ell) {
  if (ell < 2) return cudaErrorInvalidValue;
  const cuuint32_t box[3] = {(cuuint32_t)kCols, (cuuint32_t)kRows, 2u};
  return encode(out, base, g, 3, ell, box);
}

cudaError_t encode_coef_map(FieldMap* out, const float* base, const GridDesc& g) {
  const cuuint32_t box[2] = {(cuuint32_t)kCols, (cuuint32_t)kCoefRows};
  return encode(out, base, g, 2, 1, box);
}

cudaError_t launch_quad_tma(const GridDesc& g, int ell, int psrc, const FieldMap& mcx, const FieldMap& mcy,
                            const FieldMap& mxk, const FieldMap& mxkm1, const FieldMap& mbhat, float* out3, float* out4,
                            const QuadSteps& qs, long long wait_limit, unsigned* fault, cudaStream_t s) {
  if (g.n2 != 1 || g.n0 % 4 != 0 || (psrc != 1 && psrc != 2) || wait_limit < 0 || !fault) return cudaErrorInvalidValue;
  switch (ell) {
#define AAO_QT_CASE(L) \
  case L:              \
    return launch_qt<L, kQuadTmaR>(g, psrc, mcx, mcy, mxk, mxkm1, mbhat, out3, out4, qs, wait_limit, fault, s);
    AAO_QT_CASE(4)
    AAO_QT_CASE(6)
    AAO_QT_CASE(8)
    AAO_QT_CASE(10)
    AAO_QT_CASE(12)
    AAO_QT_CASE(14)
    AAO_QT_CASE(16)
#undef AAO_QT_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t quad_tma_fault(unsigned* dev_flag, unsigned* host_flag, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(host_flag, dev_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *host_flag) {
    e = cudaMemsetAsync(dev_flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e;
}

}  // namespace aao
