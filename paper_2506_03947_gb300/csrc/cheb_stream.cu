// S Chebyshev steps per launch (2D, FP32), streamed along y: the warp-strip kernel.
//
// Steps k .. k+S-1 of the Chebyshev semi-iteration (Eq. 7 over Lemma 2's segment) on every
// frequency,
//   x_{q+1} = x_q + a_q (x_q - x_{q-1}) + g_q (bhat - A x_q + lambda x_q),
// with the residual formed as bhat + sum_f kappa_f x_nbr(f) - (d - lambda) x
// (d = 1 + sum of the four face coefficients): the north and south terms first, packed over
// the lane's two cells in FP32x2 operations, then the east and west terms per cell in scalar
// FMAs (their operands straddle the lane's pair; packed, they needed register moves that cost
// more than the scalar FMAs).  The rest of the step is packed.
//
// Organisation:
//  * A unit of work is (plane pair, y segment, x strip).  A strip is 64 staged columns (lane l
//    owns columns 2l, 2l+1), of which the middle 64 - 2S are interior; a segment is H interior
//    rows, streamed from S rows above it to S rows below it.  Units are spread over all warps of
//    a persistent grid (one CTA per SM); warps never wait on one another.
//  * Level 0 (x_k) of stream row t arrives at step t; level j+1 of row t - lag(j+1) is computed
//    at the same step from level j's three rows around it: lag(j) = j in the lockstep schedule,
//    0, 1, 2, 4, 5 in the skewed one (S = 4, level_lag).  Each level's three newest rows live in
//    registers (the step loop is unrolled by 6, a multiple of three, so the rotation is a
//    renaming); level S of row t - lag(S), and level S-1 of the same row, are the outputs.
//  * Inputs stream through per-warp shared-memory rings filled by cp.async, zero-filled
//    outside the grid (the Neumann boundary: faces and values outside are zero).  With S = 4
//    a lane copies 16 bytes, four columns of one plane of a pair (lanes 0-15 the first, 16-31
//    the second; cx and cy likewise), so a row of a pair of arrays is one copy instruction;
//    with S = 2 (strips two columns off a multiple of four) each lane copies its own 8 bytes
//    per array.  Rows are issued D steps ahead; at each step a lane waits for its own copies of
//    the row (cp.async.wait_group) and a warp barrier (__syncwarp) publishes every lane's, and
//    also orders the ring slot's last reads (x_{k-1} of row t-1, read before the barrier)
//    before its refill, so D = 5 rows fit a 6-row ring.  Ring A holds x_k and x_{k-1}, ring B
//    bhat and the two face arrays, 6 rows each.  When a row lands, its bhat and face
//    coefficients (with the diagonal) move into register windows of 6 rows, where all S levels
//    read them; shared memory is read once per value.  The step loop is unrolled by 6, so
//    every ring slot and window row is a compile-time constant.
//  * Per cell and S steps the launch moves (5 ell + 2) * 4 bytes algorithmically (reads x_k,
//    x_{k-1}, bhat, two face arrays; writes two fields); the redundant halo reads are
//    64/(64-2S) across x and (H+2S)/H across y, and mostly hit L2 (neighbouring units run
//    side by side).
// cp.async waits are hardware waits on the thread's own copies and the warp barrier involves
// only the warp's own lanes: nothing here spins, and warps never wait on one another.
#include <type_traits>
#include <utility>

#include "aao_internal.cuh"
#include "batch.cuh"
#include "cheb_ends.cuh"

namespace aao {

namespace {

constexpr int kSW = 64;  // staged columns of a strip

__device__ __forceinline__ void cp8(unsigned dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp16(unsigned dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ float2 lds2(unsigned a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}

// ring B arrays of a row: bhat plane 0, bhat plane 1, kE (cx), kN (cy)
constexpr int kB_H0 = 0, kB_H1 = 1, kB_E = 2, kB_N = 3, kNB = 4;
// Both rings hold 6 rows and the step loop is unrolled by 6 (a multiple of the three
// level-window rows), so every ring slot and window row is a compile-time constant.
constexpr int kRing = 6, kUnroll = 6;

template <int PSRC>
struct StreamGeom {
  static constexpr int NA = (PSRC == 2) ? 4 : 2;  // ring A arrays: x_k planes (+ x_{k-1} planes)
  static constexpr int lane_bytes = (kRing * NA + kRing * kNB) * 8;  // both rings, per lane
};

struct Unit {
  int p0;       // first plane of the pair
  int m0, m1;   // frequencies of the two planes (real pass) or the complex frequency (m0)
  int y0;       // first interior row of the segment
  int gx;       // global column of this lane's first cell
  bool colok;   // this lane's two cells are inside the grid
};

// Packed FP32x2 arithmetic on a lane's two cells (each component rounds as fmaf / a + b).
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Per-level scalars of a pass, hoisted out of the step loop as duplicated pairs.  Real pass:
// (l, a, g) of the two real frequencies; complex pass: (lr, li, ar, ai, gr, gi) of one frequency.
template <int S>
struct PassCoef {
  float2 c[S][6];
};

template <int S, bool CPLX>
__device__ __forceinline__ void load_pass_coef(PassCoef<S>& pc, const StepArgs<float>* steps, int m0, int m1) {
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const StepArgs<float>& st = steps[q];
    if (CPLX) {
      pc.c[q][0] = dup(st.lam_re[m0]), pc.c[q][1] = dup(st.lam_im[m0]);
      pc.c[q][2] = dup(st.a_re[m0]), pc.c[q][3] = dup(st.a_im[m0]);
      pc.c[q][4] = dup(st.g_re[m0]), pc.c[q][5] = dup(st.g_im[m0]);
    } else {
      pc.c[q][0] = dup(st.lam_re[m0]), pc.c[q][1] = dup(st.lam_re[m1]);
      pc.c[q][2] = dup(st.a_re[m0]), pc.c[q][3] = dup(st.a_re[m1]);
      pc.c[q][4] = dup(st.g_re[m0]), pc.c[q][5] = dup(st.g_re[m1]);
    }
  }
}

// Face coefficients of one row for this lane's two cells: east, north and west faces and the
// negated diagonal -d = -(1 + sum of the four faces) (cell 1's west face is cell 0's east face).
struct RowCoef {
  float2 e, n, nd;
  float w0;  // west face of cell 0 (the east face of the lane to the left)
};

// Geometry and fields of one instance's launch.  For a single instance it sits in the kernel's
// __grid_constant__ parameter block, for a batch in a per-warp shared-memory copy; either way
// the pointers and sizes are read where they are used, not held in registers.
struct StreamGeo {
  GridDesc g;
  int npass, ell, H, nseg, nstrip;
  const float* cx;
  const float* cy;
  const float* bhat;
  const float* xk;
  const float* xkm1;
  float* outA;
  float* outB;
};

struct StreamArgs {
  StreamGeo geo;
  FuseSteps fs;
};

// Row lag of level j behind the newest input row: level j of stream row t - lag(j) is computed
// at step t.  Lockstep (SK 0): lag(j) = j, so within a step each level waits for the one below.
// Skewed (SK 1, S = 4): lags 0, 1, 2, 4, 5, so levels 3 and 4 read rows of level 2 computed one
// step earlier, and a step holds two independent chains, (row load, level 1, level 2) and
// (level 3, level 4), at the cost of one more streamed step per unit.
template <int SK>
__device__ __host__ constexpr int level_lag(int j) {
  return SK ? (j <= 2 ? j : j + 1) : j;
}

template <int S, int D, int PSRC, bool CPLX, int SK>
struct StreamUnit {
  static constexpr int NA = StreamGeom<PSRC>::NA;
  static constexpr int LS = level_lag<SK>(S);  // lag of the output level
  static_assert(D + 1 <= kRing && S + 2 <= kRing, "ring or window too shallow");
  static_assert(SK == 0 || S == 4, "the skewed schedule is defined for S = 4");
  static_assert(LS + 1 <= kRing, "face window too shallow");

  const StreamGeo& a;
  unsigned ringA, ringB;  // this warp's rings (shared addresses) plus the lane's 8-byte slot
  unsigned cpA, cpB;      // ... plus the lane's copy slot (S = 4: 16 bytes, lanes 16-31 in the
                          // second array of a pair; S = 2: the lane's own 8 bytes)
  // Copies, S = 4 (the strip starts at a multiple of four columns): lane l moves 16 bytes
  // (columns 4 (l mod 16) .. 4 (l mod 16) + 3 of the strip) of the pair's first plane (l < 16)
  // or second plane (l >= 16), and of cx (l < 16) or cy, and then reads its own two cells,
  // copied by another lane (visible to it after the warp barrier).  S = 2 (strips start two
  // columns off a multiple of four): each lane copies its own two cells, 8 bytes per array.
  // Element offsets of the lane's copy chunk: in the fields (its plane) and in its face array
  // (column 0 when the chunk is outside the grid: such copies read nothing)
  int64_t offf;
  int offc;
  const float* fsrc;  // cx or cy
  int64_t offo;       // element offset of the lane's own first cell in plane p0 (outputs)
  int y0;      // first interior row of the segment (stream row S)
  bool colok, interior_lane;
  int ybase;   // grid row of stream row 0 (y0 - S)
  int nrow;    // n1 when the lane's copy chunk is inside the grid, else 0: stream row u is
               // copied iff (unsigned)(ybase + u) < nrow
  int hout;    // rows of the segment this lane writes (0 for halo lanes and lanes outside)
  PassCoef<S> pc;
  float it[2];            // 1/theta (x_1 = bhat/theta): real (it0, it1), complex (re, im)
  float2 L[S][3][2];      // level windows: L[j][r % 3][plane] = level j of stream row r
  float2 Hw[kRing][2];    // bhat of stream row r in Hw[r % 6][plane]
  RowCoef Cw[kRing];      // face coefficients of stream row r in Cw[r % 6]
  float2 nS6;             // north faces of stream row t - 6 (SK 1: the south faces of level 4's row)
  float2 last[2];         // level S of the step's output row
  float2 pvk[2];          // x_{k-1} of row t - 1 (PSRC 2), read before this step's copies may
                          // reuse its ring slot (D = 5)

  __device__ __forceinline__ unsigned slotA(int row_slot, int arr) const {
    return ringA + (unsigned)((row_slot * NA + arr) * 256);
  }
  __device__ __forceinline__ unsigned slotB(int row_slot, int arr) const {
    return ringB + (unsigned)((row_slot * kNB + arr) * 256);
  }

  // copies of stream row u into ring slot SL of both rings (the two arrays of each pair of
  // slots are adjacent, so one 16-byte copy per lane fills both)
  template <int SL>
  __device__ __forceinline__ void issue(int u) {
    const int y = ybase + u;
    const bool ok = (unsigned)y < (unsigned)nrow;
    const int64_t row = ok ? (int64_t)y * a.g.n0 : 0;
    const int64_t of = offf + row, oc = offc + row;
    if constexpr (S == 4) {
      const unsigned nb = ok ? 16u : 0u;
      cp16(cpA + (unsigned)((SL * NA + 0) * 256), a.xk + of, nb);
      if (PSRC == 2) cp16(cpA + (unsigned)((SL * NA + 2) * 256), a.xkm1 + of, nb);
      cp16(cpB + (unsigned)((SL * kNB + kB_H0) * 256), a.bhat + of, nb);
      cp16(cpB + (unsigned)((SL * kNB + kB_E) * 256), fsrc + oc, nb);
    } else {
      const unsigned nb = ok ? 8u : 0u;
      cp8(cpA + (unsigned)((SL * NA + 0) * 256), a.xk + of, nb);
      cp8(cpA + (unsigned)((SL * NA + 1) * 256), a.xk + a.g.N + of, nb);
      if (PSRC == 2) {
        cp8(cpA + (unsigned)((SL * NA + 2) * 256), a.xkm1 + of, nb);
        cp8(cpA + (unsigned)((SL * NA + 3) * 256), a.xkm1 + a.g.N + of, nb);
      }
      cp8(cpB + (unsigned)((SL * kNB + kB_H0) * 256), a.bhat + of, nb);
      cp8(cpB + (unsigned)((SL * kNB + kB_H1) * 256), a.bhat + a.g.N + of, nb);
      cp8(cpB + (unsigned)((SL * kNB + kB_E) * 256), a.cx + oc, nb);
      cp8(cpB + (unsigned)((SL * kNB + kB_N) * 256), a.cy + oc, nb);
    }
  }

  // step t = 6 b + I of the stream (T: streamed input rows)
  template <int I>
  __device__ __forceinline__ void step(int t, int T) {
    constexpr int PH = I % 3;
    constexpr int SL = I;                        // ring slot and window row of stream row t
    constexpr int SLm = (I + kRing - 1) % kRing;  // ... of row t - 1
    cp_wait<D - 1>();  // row t has landed (this lane's copies); past the last row, stale rows
                       // feed only halo rows that no output depends on
    if (PSRC == 2) {
      pvk[0] = lds2(slotA(SLm, 2));
      pvk[1] = lds2(slotA(SLm, 3));
    }
    __syncwarp();      // row t of every lane has landed; and every lane is done reading the ring
                       // slot (row t + D - 6 <= t - 1) the next copies overwrite
    if (t + D < T) issue<(I + D) % kRing>(t + D);
    cp_commit();
    if (SK) nS6 = Cw[SL].n;  // row t - 6, about to be replaced by row t
    {
      L[0][PH][0] = lds2(slotA(SL, 0));
      L[0][PH][1] = lds2(slotA(SL, 1));
      Hw[SL][0] = lds2(slotB(SL, kB_H0));
      Hw[SL][1] = lds2(slotB(SL, kB_H1));
      // face coefficients of row t; d = 1 + ((kE + kW) + (kN + kS)), kS = kN of row t - 1
      RowCoef& c = Cw[SL];
      c.e = lds2(slotB(SL, kB_E));
      c.n = lds2(slotB(SL, kB_N));
      c.w0 = __shfl_up_sync(0xffffffffu, c.e.y, 1);
      const float2 t3 = f2add(f2add(c.e, make_float2(c.w0, c.e.x)), f2add(c.n, Cw[SLm].n));
      c.nd = f2fma(t3, dup(-1.f), dup(-1.f));  // -(1 + t3), exactly -RN(1 + t3)
    }
    if (SK) {
      // levels 3 and 4 first (they read level 2's rows of earlier steps, and level 1's row
      // t - 4, which level 1 replaces this step), then levels 1 and 2
      level<I, 2>();
      level<I, 3>();
      level<I, 0>();
      level<I, 1>();
    } else {
      levels<I>(std::make_integer_sequence<int, S>{});
    }
    // outputs: level S and level S-1 of stream row t - LS (segment row t - LS - S)
    const int oy = t - LS - S;
    if ((unsigned)oy < (unsigned)hout) {
      constexpr int RS = ((PH - LS) % 3 + 3) % 3;
      const int64_t o = offo + (int64_t)(y0 + oy) * a.g.n0;
      *reinterpret_cast<float2*>(a.outB + o) = last[0];
      *reinterpret_cast<float2*>(a.outB + o + a.g.N) = last[1];
      if (a.outA) {  // null on the sweep's final launch, which keeps x_p alone
        *reinterpret_cast<float2*>(a.outA + o) = L[S - 1][RS][0];
        *reinterpret_cast<float2*>(a.outA + o + a.g.N) = L[S - 1][RS][1];
      }
    }
  }

  template <int I, int... J>
  __device__ __forceinline__ void levels(std::integer_sequence<int, J...>) {
    (level<I, J>(), ...);
  }

  // level j+1 of stream row rho = t - lag(j+1)
  template <int I, int j>
  __device__ __forceinline__ void level() {
    constexpr int LG = level_lag<SK>(j + 1);
    constexpr int RS = ((I - LG) % 3 + 3) % 3;  // rho % 3
    constexpr int RN = (RS + 1) % 3, RSo = (RS + 2) % 3;
    constexpr int W = ((I - LG) % kRing + kRing) % kRing;       // rho % 6
    constexpr int Wm = ((I - LG - 1) % kRing + kRing) % kRing;  // (rho - 1) % 6
    static_assert(j > 0 || LG == 1, "level 1 reads x_{k-1} of row t - 1");
    const RowCoef& cf = Cw[W];
    const float2 kS = (LG + 1 == kRing) ? nS6 : Cw[Wm].n;  // row t - 6 has left the window
    const float2* hh = Hw[W];
    const float2 m1 = dup(-1.f);
    float2 pv[2];
    if (j == 0) {
      if (PSRC == 2) {
        pv[0] = pvk[0];
        pv[1] = pvk[1];
      } else {
        // x_{k-1} = x_1 = bhat / theta
        const float h00 = hh[0].x, h01 = hh[0].y, h10 = hh[1].x, h11 = hh[1].y;
        if (CPLX) {
          pv[0] = make_float2(h00 * it[0] - h10 * it[1], h01 * it[0] - h11 * it[1]);
          pv[1] = make_float2(h00 * it[1] + h10 * it[0], h01 * it[1] + h11 * it[0]);
        } else {
          pv[0] = make_float2(h00 * it[0], h01 * it[0]);
          pv[1] = make_float2(h10 * it[1], h11 * it[1]);
        }
      }
    } else {
      pv[0] = L[j > 0 ? j - 1 : 0][RS][0];
      pv[1] = L[j > 0 ? j - 1 : 0][RS][1];
    }
    // stencil: nb = bhat + kE xE + kW xW + kN xN + kS xS on both planes, both cells at once
    float2 nb[2];
    const float2(&cur)[2] = L[j][RS];
#pragma unroll
    for (int pl = 0; pl < 2; ++pl) {
      const float left = __shfl_up_sync(0xffffffffu, cur[pl].y, 1);
      const float right = __shfl_down_sync(0xffffffffu, cur[pl].x, 1);
      // north and south on both cells packed (their operands are aligned pairs); east and west
      // per cell in scalar FMAs (their operands straddle the lane's pair), written straight into
      // the halves of the result
      const float2 ns = f2fma(kS, L[j][RSo][pl], f2fma(cf.n, L[j][RN][pl], hh[pl]));
      nb[pl].x = fmaf(cf.w0, left, fmaf(cf.e.x, cur[pl].y, ns.x));
      nb[pl].y = fmaf(cf.e.x, cur[pl].x, fmaf(cf.e.y, right, ns.y));
    }
    float2 nw[2];
    const float2* q = pc.c[j];
    if (CPLX) {
      // residual r = nb - (d - lambda) x and x + a (x - x_prev) + g r in complex arithmetic;
      // the products with -li, -ai, -gi are formed as li (-xi), ai (-di), gi (-ri) (same values)
      const float2 xr = cur[0], xi = cur[1];
      const float2 ndl = f2add(cf.nd, q[0]);                 // -(d - lr)
      const float2 rr = f2fma(q[1], neg2(xi), f2fma(ndl, xr, nb[0]));
      const float2 ri = f2fma(q[1], xr, f2fma(ndl, xi, nb[1]));
      const float2 dr = f2fma(pv[0], m1, xr), di = f2fma(pv[1], m1, xi);  // x - x_prev
      nw[0] = f2fma(q[5], neg2(ri), f2fma(q[4], rr, f2fma(q[3], neg2(di), f2fma(q[2], dr, xr))));
      nw[1] = f2fma(q[5], rr, f2fma(q[4], ri, f2fma(q[3], dr, f2fma(q[2], di, xi))));
    } else {
      const float2 x0 = cur[0], x1 = cur[1];
      const float2 q0 = f2fma(f2add(cf.nd, q[0]), x0, nb[0]);  // nb - (d - l0) x0
      const float2 q1 = f2fma(f2add(cf.nd, q[1]), x1, nb[1]);
      nw[0] = f2fma(q[4], q0, f2fma(q[2], f2fma(pv[0], m1, x0), x0));
      nw[1] = f2fma(q[5], q1, f2fma(q[3], f2fma(pv[1], m1, x1), x1));
    }
    if (j + 1 < S) {
      L[(j + 1 < S) ? j + 1 : 0][RS][0] = nw[0];
      L[(j + 1 < S) ? j + 1 : 0][RS][1] = nw[1];
    } else {
      last[0] = nw[0];
      last[1] = nw[1];
    }
  }

  __device__ __forceinline__ void run() {
    const int T = a.H + 2 * S;       // streamed input rows
    const int TS = T + LS - S;       // steps, a multiple of 6
    issue<0>(0);
    cp_commit();
    issue<1>(1);
    cp_commit();
    issue<2>(2);
    cp_commit();
    if (D >= 4) {
      issue<3>(3);
      cp_commit();
    }
    if (D >= 5) {
      issue<4>(4);
      cp_commit();
    }
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int s2 = 0; s2 < 3; ++s2) L[j][s2][0] = L[j][s2][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kRing; ++r) Cw[r].n = make_float2(0.f, 0.f);
    nS6 = make_float2(0.f, 0.f);
    for (int t = 0; t < TS; t += kUnroll) {
      step<0>(t, T);
      step<1>(t + 1, T);
      step<2>(t + 2, T);
      step<3>(t + 3, T);
      step<4>(t + 4, T);
      step<5>(t + 5, T);
    }
    cp_wait<0>();  // (empty groups only by now) the rings are free for the next unit
    __syncwarp();
  }
};

template <int S, int D, int PSRC, bool CPLX, int SK>
__device__ __forceinline__ void stream_unit(const StreamGeo& a, const StepArgs<float>* steps, const Unit& un,
                                            int lane, unsigned ringA, unsigned ringB) {
  StreamUnit<S, D, PSRC, CPLX, SK> su{a};
  su.ringA = ringA + (unsigned)(lane * 8);
  su.ringB = ringB + (unsigned)(lane * 8);
  su.y0 = un.y0;
  su.colok = un.colok;
  su.interior_lane = lane >= S / 2 && lane < 32 - S / 2;
  su.ybase = un.y0 - S;
  su.hout = (su.interior_lane && un.colok) ? min(a.H, a.g.n1 - un.y0) : 0;
  su.offo = (int64_t)un.p0 * a.g.N + (un.colok ? un.gx : 0);
  if constexpr (S == 4) {
    // the lane's copy chunk: columns gc .. gc + 3 (gc and n0 are multiples of 4: the chunk is
    // wholly inside the grid or wholly outside), plane p0 + (lane >= 16)
    const int hi = lane >> 4;
    const int gc = un.gx - 2 * lane + 4 * (lane & 15);
    const bool cok = gc >= 0 && gc < a.g.n0;
    su.cpA = ringA + (unsigned)(lane * 16);
    su.cpB = ringB + (unsigned)(lane * 16);
    su.nrow = cok ? a.g.n1 : 0;
    su.offc = cok ? gc : 0;  // keep every source address inside its array
    su.offf = (int64_t)(un.p0 + hi) * a.g.N + su.offc;
    su.fsrc = hi ? a.cy : a.cx;
  } else {
    su.cpA = su.ringA;
    su.cpB = su.ringB;
    su.nrow = un.colok ? a.g.n1 : 0;
    su.offc = un.colok ? un.gx : 0;
    su.offf = (int64_t)un.p0 * a.g.N + su.offc;
    su.fsrc = a.cx;
  }
  if (CPLX) {
    su.it[0] = steps[0].it_re[un.m0], su.it[1] = steps[0].it_im[un.m0];
  } else {
    su.it[0] = steps[0].it_re[un.m0], su.it[1] = steps[0].it_re[un.m1];
  }
  load_pass_coef<S, CPLX>(su.pc, steps, un.m0, un.m1);
  su.run();
}

// Registers: the four-step kernels at 8 warps use 180-215 per thread (two warps per SM
// sub-partition of 16 K registers); the two-step kernel stays within 128 at 16 warps.
template <int S, int D, int NW, int PSRC, int SK>
__global__ void __launch_bounds__(NW * 32, 1) k_cheb_stream(const __grid_constant__ StreamArgs args) {
  const StreamGeo& a = args.geo;
  using G = StreamGeom<PSRC>;
  extern __shared__ __align__(16) unsigned char smem_stream[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned base = (unsigned)__cvta_generic_to_shared(smem_stream) + (unsigned)(warp * 32 * G::lane_bytes);
  const unsigned ringA = base;
  const unsigned ringB = base + (unsigned)(kRing * G::NA * 32 * 8);
  const int per_pass = a.nseg * a.nstrip;
  const int nunits = a.npass * per_pass;
  const int total_warps = gridDim.x * NW;
  constexpr int IW = kSW - 2 * S;
  // CTA b takes the contiguous chunk [b units / grid, (b + 1) units / grid) of units (strip
  // fastest): every SM gets work, and neighbouring strips, which share halo columns, run on
  // the same SM
  const int u_begin = (int)((int64_t)blockIdx.x * nunits / gridDim.x);
  const int u_end = (int)((int64_t)(blockIdx.x + 1) * nunits / gridDim.x);
  (void)total_warps;
  for (int u = u_begin + warp; u < u_end; u += NW) {
    Unit un;
    const int pass = u / per_pass;
    const int rem = u - pass * per_pass;
    const int seg = rem / a.nstrip;
    const int strip = rem - seg * a.nstrip;
    un.p0 = 2 * pass;
    un.m0 = pass;
    un.m1 = (pass == 0) ? a.ell / 2 : pass;
    un.y0 = seg * a.H;
    un.gx = strip * IW - S + 2 * lane;
    un.colok = un.gx >= 0 && un.gx < a.g.n0;
    if (pass == 0)
      stream_unit<S, D, PSRC, false, SK>(a, args.fs.s, un, lane, ringA, ringB);
    else
      stream_unit<S, D, PSRC, true, SK>(a, args.fs.s, un, lane, ringA, ringB);
  }
}

template <int S, int D, int NW, int SK>
cudaError_t launch_stream_cfg(const GridDesc& g, int ell, int psrc, int H, const float* cx, const float* cy,
                              const float* bhat, const float* xk, const float* xkm1, float* outA, float* outB,
                              const FuseSteps& fs, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  constexpr int IW = kSW - 2 * S;
  const int nstrip = (g.n0 + IW - 1) / IW;
  const int nseg = (g.n1 + H - 1) / H;
  const int units = (ell / 2) * nseg * nstrip;
  const int grid = units < nsm ? units : nsm;
  StreamArgs a;
  a.geo.g = g;
  a.geo.npass = ell / 2;
  a.geo.ell = ell;
  a.geo.H = H;
  a.geo.nseg = nseg;
  a.geo.nstrip = nstrip;
  a.geo.cx = cx;
  a.geo.cy = cy;
  a.geo.bhat = bhat;
  a.geo.xk = xk;
  a.geo.xkm1 = xkm1;
  a.geo.outA = outA;
  a.geo.outB = outB;
  a.fs = fs;
  if (psrc == 1) {
    auto k = k_cheb_stream<S, D, NW, 1, SK>;
    const size_t smem = (size_t)NW * 32 * StreamGeom<1>::lane_bytes;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, s>>>(a);
  } else {
    auto k = k_cheb_stream<S, D, NW, 2, SK>;
    const size_t smem = (size_t)NW * 32 * StreamGeom<2>::lane_bytes;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, s>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// S = 4 launches stream H + 8 rows when that is a multiple of 6 (levels in lockstep), else the
// skewed schedule when H + 9 is (one more step per unit; see level_lag).
static int stream_skew(const StreamConfig& c) { return (c.S == 4 && (c.H + 2 * c.S) % kUnroll != 0) ? 1 : 0; }

bool stream_config_supported(const StreamConfig& c) {
  if ((c.S != 2 && c.S != 4) || c.H < 1 || c.H > 4096) return false;
  const int sk = stream_skew(c);
  if ((c.H + 2 * c.S + (sk ? 1 : 0)) % kUnroll != 0) return false;
  if (c.D < 3 || c.D > 5 || (c.D == 5 && (c.S != 4 || c.NW != 8))) return false;
  if (c.S == 2) return c.NW == 8 || c.NW == 12 || c.NW == 16;
  if (sk) return c.NW == 8;  // 205-215 registers: no room for 12 warps
  return c.NW == 6 || c.NW == 8 || c.NW == 12;
}

cudaError_t launch_stream(const GridDesc& g, int ell, int psrc, const StreamConfig& c, const float* cx,
                          const float* cy, const float* bhat, const float* xk, const float* xkm1, float* outA,
                          float* outB, const FuseSteps& fs, cudaStream_t s) {
  if (g.n2 != 1 || g.n0 % 4 != 0 || (psrc != 1 && psrc != 2) || ell < 4 || ell > kMaxEll || (ell % 2) ||
      !stream_config_supported(c))
    return cudaErrorInvalidValue;
  // the four-step kernel copies 16-byte chunks of every input array
  if (((reinterpret_cast<uintptr_t>(cx) | reinterpret_cast<uintptr_t>(cy) | reinterpret_cast<uintptr_t>(bhat) |
        reinterpret_cast<uintptr_t>(xk) | reinterpret_cast<uintptr_t>(xkm1)) & 15) != 0)
    return cudaErrorInvalidValue;
  const int sk = stream_skew(c);
#define AAO_STREAM_CFG(SS, DD, NN, KK)                                                                         \
  if (c.S == SS && c.D == DD && c.NW == NN && sk == KK)                                                        \
    return launch_stream_cfg<SS, DD, NN, KK>(g, ell, psrc, c.H, cx, cy, bhat, xk, xkm1, outA, outB, fs, s);
  AAO_STREAM_CFG(4, 3, 6, 0)
  AAO_STREAM_CFG(4, 3, 8, 0)
  AAO_STREAM_CFG(4, 4, 6, 0)
  AAO_STREAM_CFG(4, 4, 8, 0)
  AAO_STREAM_CFG(4, 3, 12, 0)
  AAO_STREAM_CFG(4, 4, 12, 0)
  AAO_STREAM_CFG(4, 3, 8, 1)
  AAO_STREAM_CFG(4, 4, 8, 1)
  AAO_STREAM_CFG(4, 5, 8, 1)
  AAO_STREAM_CFG(4, 5, 8, 0)
  AAO_STREAM_CFG(2, 3, 8, 0)
  AAO_STREAM_CFG(2, 3, 12, 0)
  AAO_STREAM_CFG(2, 4, 8, 0)
  AAO_STREAM_CFG(2, 4, 12, 0)
  AAO_STREAM_CFG(2, 3, 16, 0)
  AAO_STREAM_CFG(2, 4, 16, 0)
#undef AAO_STREAM_CFG
  return cudaErrorInvalidValue;
}

// ---- inverse transform of x_p (the sweep's final output) -------------------------------------

namespace {

// Inverse transform of x_p, two cells per thread (ends::idft_pair, cheb_ends.cuh).
template <int ELL>
__global__ void __launch_bounds__(256, 4) k_idft_planes(int64_t N2, int64_t N, const float* __restrict__ x,
                                                        double* __restrict__ z,
                                                        const __grid_constant__ IdftArgs<float> ia) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N2) return;
  ends::idft_pair<ELL>(N, 2 * q, x, z, ia);
}

}  // namespace

cudaError_t launch_idft_planes(const GridDesc& g, int ell, const float* x, double* z, const IdftArgs<float>& ia,
                               cudaStream_t s) {
  if (g.N % 2 != 0 || (reinterpret_cast<uintptr_t>(x) & 7) != 0 || (reinterpret_cast<uintptr_t>(z) & 15) != 0)
    return cudaErrorInvalidValue;
  const int64_t N2 = g.N / 2;
  const unsigned nb = (unsigned)((N2 + 255) / 256);
  switch (ell) {
#define AAO_IDFT(L)                                                  \
  case L:                                                            \
    k_idft_planes<L><<<nb, 256, 0, s>>>(N2, g.N, x, z, ia);          \
    break;
    AAO_IDFT(4)
    AAO_IDFT(6)
    AAO_IDFT(8)
    AAO_IDFT(10)
    AAO_IDFT(12)
    AAO_IDFT(14)
    AAO_IDFT(16)
#undef AAO_IDFT
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}


// ---- batched form: one persistent launch over the units of every member -------------------

namespace {

// Unit u of a batched launch belongs to list entry li with ustart[li] <= u < ustart[li + 1]
// (member uinst[li]); units are taken from a device queue, one ticket per warp and unit.
struct StreamBatchArgs {
  const BInst* I;
  const int* act;
  const int* ustart;
  const int* uinst;
  int cnt;       // list entries
  int total;     // units over all entries
  int H;         // segment height of every member
  int k;         // first fused step: steps k .. k+S-1 of every member
  int cur, prev, o3, o4;  // the members' rotating fields: x_k, x_{k-1} (PSRC 2), outputs
  StreamQueue* queue;
};

__device__ __forceinline__ float* bfield(const BInst& b, int i) {
  return i == 0 ? b.xa : i == 1 ? b.xb : i == 2 ? b.xc : b.xd;
}

template <int S, int D, int NW, int PSRC>
__global__ void __launch_bounds__(NW * 32, 1) kb_cheb_stream(const __grid_constant__ StreamBatchArgs ba) {
  using G = StreamGeom<PSRC>;
  extern __shared__ __align__(16) unsigned char smem_stream[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned base = (unsigned)__cvta_generic_to_shared(smem_stream) + (unsigned)(warp * 32 * G::lane_bytes);
  const unsigned ringA = base;
  const unsigned ringB = base + (unsigned)(kRing * G::NA * 32 * 8);
  // this warp's copy of the current member's geometry, after all warps' rings
  StreamGeo* geo = reinterpret_cast<StreamGeo*>(smem_stream + (size_t)NW * 32 * G::lane_bytes) + warp;
  constexpr int IW = kSW - 2 * S;
  while (true) {
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(&ba.queue->next, 1u);
    const int u = (int)__shfl_sync(0xffffffffu, t, 0);
    if (u >= ba.total) break;
    int lo = 0, hi = ba.cnt;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (ba.ustart[mid] <= u) lo = mid;
      else hi = mid;
    }
    const int inst = ba.uinst[lo];
    if (!ba.act[inst]) continue;
    const BInst& b = ba.I[inst];
    __syncwarp();  // every lane is done with the previous unit's geometry
    if (lane == 0) {
      StreamGeo gg;
      gg.g = b.g;
      gg.ell = b.ell;
      gg.npass = b.ell / 2;
      gg.H = ba.H;
      gg.nseg = (b.g.n1 + ba.H - 1) / ba.H;
      gg.nstrip = (b.g.n0 + IW - 1) / IW;
      gg.cx = b.cx32;
      gg.cy = b.cy32;
      gg.bhat = b.bhat;
      gg.xk = bfield(b, ba.cur);
      gg.xkm1 = (PSRC == 2) ? bfield(b, ba.prev) : nullptr;
      gg.outA = ba.o3 < 0 ? nullptr : bfield(b, ba.o3);
      gg.outB = bfield(b, ba.o4);
      *geo = gg;
    }
    __syncwarp();
    const StreamGeo& a = *geo;
    const int lu = u - ba.ustart[lo];
    const int per_pass = a.nseg * a.nstrip;
    Unit un;
    const int pass = lu / per_pass;
    const int rem = lu - pass * per_pass;
    const int seg = rem / a.nstrip;
    const int strip = rem - seg * a.nstrip;
    un.p0 = 2 * pass;
    un.m0 = pass;
    un.m1 = (pass == 0) ? a.ell / 2 : pass;
    un.y0 = seg * a.H;
    un.gx = strip * IW - S + 2 * lane;
    un.colok = un.gx >= 0 && un.gx < a.g.n0;
    const StepArgs<float>* steps = b.steps + ba.k;
    if (pass == 0)
      stream_unit<S, D, PSRC, false, 0>(a, steps, un, lane, ringA, ringB);
    else
      stream_unit<S, D, PSRC, true, 0>(a, steps, un, lane, ringA, ringB);
  }
  // every warp ends here once, after its ticket past the end: the last one resets the queue
  // for the next launch
  if (lane == 0) {
    const unsigned d = atomicAdd(&ba.queue->done, 1u);
    if (d == gridDim.x * NW - 1) {
      atomicExch(&ba.queue->next, 0u);
      atomicExch(&ba.queue->done, 0u);
    }
  }
}

template <int S, int D, int NW>
cudaError_t launch_batch_stream_cfg(const StreamBatchArgs& ba, int psrc, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int grid = (ba.total + NW - 1) / NW;
  if (grid > nsm) grid = nsm;
  if (grid < 1) grid = 1;
  if (psrc == 1) {
    auto k = kb_cheb_stream<S, D, NW, 1>;
    const size_t smem = (size_t)NW * 32 * StreamGeom<1>::lane_bytes + (size_t)NW * sizeof(StreamGeo);
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, s>>>(ba);
  } else {
    auto k = kb_cheb_stream<S, D, NW, 2>;
    const size_t smem = (size_t)NW * 32 * StreamGeom<2>::lane_bytes + (size_t)NW * sizeof(StreamGeo);
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, s>>>(ba);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int batch_stream_units(const GridDesc& g, int ell, int S, int H) {
  const int IW = kSW - 2 * S;
  return (ell / 2) * ((g.n1 + H - 1) / H) * ((g.n0 + IW - 1) / IW);
}

cudaError_t launch_batch_stream(const BInst* I, const int* act, const WorkList& units, const StreamConfig& c, int k,
                                int psrc, int cur, int prev, int o3, int o4, StreamQueue* queue, cudaStream_t s) {
  if (!stream_config_supported(c) || stream_skew(c) || (psrc != 1 && psrc != 2) || !queue)
    return cudaErrorInvalidValue;  // the batched launch runs the lockstep schedule
  if (units.total == 0) return cudaSuccess;
  StreamBatchArgs ba;
  ba.I = I;
  ba.act = act;
  ba.ustart = units.start;
  ba.uinst = units.inst;
  ba.cnt = units.cnt;
  ba.total = units.total;
  ba.H = c.H;
  ba.k = k;
  ba.cur = cur;
  ba.prev = prev < 0 ? 0 : prev;
  ba.o3 = o3;
  ba.o4 = o4;
  ba.queue = queue;
#define AAO_BSTREAM_CFG(SS, DD, NN) \
  if (c.S == SS && c.D == DD && c.NW == NN) return launch_batch_stream_cfg<SS, DD, NN>(ba, psrc, s);
  AAO_BSTREAM_CFG(4, 3, 8)
  AAO_BSTREAM_CFG(4, 4, 8)
  AAO_BSTREAM_CFG(2, 3, 8)
  AAO_BSTREAM_CFG(2, 4, 8)
#undef AAO_BSTREAM_CFG
  return cudaErrorInvalidValue;
}

}  // namespace aao
