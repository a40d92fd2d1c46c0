// Device bodies of the FP64 kernels of the outer solve, shared by the
// single-instance kernels (krylov.cu) and the batched ones (batch.cu).
// Reductions are deterministic: partial sums per block in a fixed layout,
// summed in a fixed order by a second kernel.
#pragma once

#include "aao_internal.cuh"

namespace aao {

constexpr int kRedThreads = 256;
constexpr int kRedWarps = kRedThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  `sh` holds kRedWarps doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kRedWarps; ++w) t += sh[w];  // fixed order
  return t;
}

constexpr int kDotGroup = 8;  // dot products accumulated per pass over w

// The flat-vector kernels below walk the vectors two doubles at a time
// (16-byte loads) and unroll by two, so each thread keeps several independent
// loads in flight; L (= ell N) is even whenever N is even, and an odd tail is
// handled separately.
__device__ __forceinline__ double2 ld2(const double* __restrict__ p) {
  return __ldg(reinterpret_cast<const double2*>(p));
}

// partials[i*NB + blk] = vscale[i] * sum_{e in block slice} V_i[e] w[e], for i in [i0, i0+G).
// G is the exact number of vectors of this launch: a runtime bound inside the
// unrolled loop would let the compiler turn the guards into selects and issue
// FP64 multiply-adds for all slots, and FP64 arithmetic is this kernel's limit.
template <int DIM, int MODE>
__device__ __forceinline__ void aao_matvec_body(const GridDesc& g, int ell, int bx, int by, int bz, int blk,
                                                const double* __restrict__ cx, const double* __restrict__ cy,
                                                const double* __restrict__ cz, const double* __restrict__ x,
                                                const double* __restrict__ b, double* __restrict__ y,
                                                double* __restrict__ partials) {
  __shared__ double sh[kRedWarps];
  const int i = bx * blockDim.x + threadIdx.x;
  const int j = by * blockDim.y + threadIdx.y;
  const int k = bz;
  double acc2 = 0.0;
  if (i < g.n0 && j < g.n1) {
    const int64_t N = g.N;
    const int64_t c = i + (int64_t)g.n0 * (j + (int64_t)g.n1 * k);
    double kap[2 * DIM];
    int64_t nb[2 * DIM];
    kap[0] = __ldg(cx + c);
    kap[1] = (i > 0) ? __ldg(cx + c - 1) : 0.0;
    nb[0] = (i < g.n0 - 1) ? c + 1 : c;
    nb[1] = (i > 0) ? c - 1 : c;
    if constexpr (DIM >= 2) {
      kap[2] = __ldg(cy + c);
      kap[3] = (j > 0) ? __ldg(cy + c - g.n0) : 0.0;
      nb[2] = (j < g.n1 - 1) ? c + g.n0 : c;
      nb[3] = (j > 0) ? c - g.n0 : c;
    }
    if constexpr (DIM == 3) {
      const int64_t pl = (int64_t)g.n0 * g.n1;
      kap[4] = __ldg(cz + c);
      kap[5] = (k > 0) ? __ldg(cz + c - pl) : 0.0;
      nb[4] = (k < g.n2 - 1) ? c + pl : c;
      nb[5] = (k > 0) ? c - pl : c;
    }
    // diagonal form (1 + sum kappa) x_c - sum kappa x_nbr: the diagonal is formed
    // once per cell and reused for all ell blocks (FP64 arithmetic is the
    // scarce resource here, not bandwidth)
    double diag = 1.0;
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) diag += kap[q];
    double prev = 0.0;
    // two time blocks per iteration (ell is even): their loads are in flight together
#pragma unroll 2
    for (int t = 0; t < ell; ++t) {
      const double* xt = x + (int64_t)t * N;
      const double xc = __ldg(xt + c);
      double a = diag * xc - prev;
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q) a -= kap[q] * __ldg(xt + nb[q]);
      double v = a;
      prev = xc;
      if constexpr (MODE == 1) {
        v = __ldg(b + (int64_t)t * N + c) - v;
        acc2 += v * v;
      }
      y[(int64_t)t * N + c] = v;
    }
  }
  if constexpr (MODE == 1) {
    const double s = block_sum(acc2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blk] = s;
  }
}

// Dot products accumulate as explicit FMA chains: on GB300 the FP64 pipe is the
// limit of these kernels, and a*b + c*d + acc would cost a multiply, an FMA and
// an add instead of two FMAs.
template <int G>
__device__ __forceinline__ void multidot_body(int blk, int nblk, const double* __restrict__ V, int64_t ldv, int i0,
                                              const double* __restrict__ vscale, const double* __restrict__ w,
                                              int64_t L, double* __restrict__ partials) {
  __shared__ double sh[G][kRedWarps];
  double acc[G];
#pragma unroll
  for (int q = 0; q < G; ++q) acc[q] = 0.0;
  const bool vec = ((L | ldv) & 1) == 0 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  const int64_t tid = (int64_t)blk * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)nblk * blockDim.x;
  const double* V0 = V + (int64_t)i0 * ldv;
  if (vec) {
    const int64_t L2 = L / 2;
    int64_t e2 = tid;
    for (; e2 + nthr < L2; e2 += 2 * nthr) {
      const double2 wa = ld2(w + 2 * e2), wb = ld2(w + 2 * (e2 + nthr));
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const double* vq = V0 + (int64_t)q * ldv;
        const double2 va = ld2(vq + 2 * e2), vb = ld2(vq + 2 * (e2 + nthr));
        acc[q] = fma(vb.y, wb.y, fma(vb.x, wb.x, fma(va.y, wa.y, fma(va.x, wa.x, acc[q]))));
      }
    }
    for (; e2 < L2; e2 += nthr) {
      const double2 wa = ld2(w + 2 * e2);
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const double2 va = ld2(V0 + (int64_t)q * ldv + 2 * e2);
        acc[q] = fma(va.y, wa.y, fma(va.x, wa.x, acc[q]));
      }
    }
  } else {
    for (int64_t e = tid; e < L; e += nthr) {
      const double we = __ldg(w + e);
#pragma unroll
      for (int q = 0; q < G; ++q) acc[q] += __ldg(V0 + (int64_t)q * ldv + e) * we;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) sh[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < G) {
    const int q = threadIdx.x;
    double t = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < kRedWarps; ++w2) t += sh[q][w2];
    const double scl = vscale ? vscale[i0 + q] : 1.0;
    partials[(int64_t)(i0 + q) * nblk + blk] = t * scl;
  }
}

__device__ __forceinline__ void orth_update_body(int blk, int nblk, const double* __restrict__ V, int64_t ldv, int nv,
                                                 const double* __restrict__ h, const double* __restrict__ vscale,
                                                 double* __restrict__ w, int64_t L, double* __restrict__ partials) {
  __shared__ double coef[kMaxRestart + 1];
  __shared__ double sh[kRedWarps];
  for (int q = threadIdx.x; q < nv; q += blockDim.x) coef[q] = h[q] * (vscale ? vscale[q] : 1.0);
  __syncthreads();
  double acc2 = 0.0;
  const bool vec = ((L | ldv) & 1) == 0 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  const int64_t tid = (int64_t)blk * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)nblk * blockDim.x;
  if (vec) {
    const int64_t L2 = L / 2;
    for (int64_t e2 = tid; e2 < L2; e2 += nthr) {
      double2 v = *reinterpret_cast<const double2*>(w + 2 * e2);
      int q = 0;
      for (; q + 4 <= nv; q += 4) {
        const double2 a0 = ld2(V + (int64_t)q * ldv + 2 * e2);
        const double2 a1 = ld2(V + (int64_t)(q + 1) * ldv + 2 * e2);
        const double2 a2 = ld2(V + (int64_t)(q + 2) * ldv + 2 * e2);
        const double2 a3 = ld2(V + (int64_t)(q + 3) * ldv + 2 * e2);
        v.x -= coef[q] * a0.x; v.y -= coef[q] * a0.y;
        v.x -= coef[q + 1] * a1.x; v.y -= coef[q + 1] * a1.y;
        v.x -= coef[q + 2] * a2.x; v.y -= coef[q + 2] * a2.y;
        v.x -= coef[q + 3] * a3.x; v.y -= coef[q + 3] * a3.y;
      }
      for (; q < nv; ++q) {
        const double2 a = ld2(V + (int64_t)q * ldv + 2 * e2);
        v.x -= coef[q] * a.x;
        v.y -= coef[q] * a.y;
      }
      *reinterpret_cast<double2*>(w + 2 * e2) = v;
      acc2 = fma(v.y, v.y, fma(v.x, v.x, acc2));
    }
  } else {
    for (int64_t e = tid; e < L; e += nthr) {
      double v = w[e];
      for (int q = 0; q < nv; ++q) v -= coef[q] * __ldg(V + (int64_t)q * ldv + e);
      w[e] = v;
      acc2 += v * v;
    }
  }
  if (partials) {
    const double t = block_sum(acc2, sh);
    if (threadIdx.x == 0) partials[blk] = t;
  }
}


// L2 eviction-priority policies (PTX createpolicy): the vector being orthogonalised is
// re-read by every modified Gram-Schmidt step and is kept (evict_last); the basis
// vectors stream past it (evict_first).
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ double2 ld2_pol(const double* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld2_ro_pol(const double* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st2_pol(double* p, double2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol) : "memory");
}

// One fused step of modified Gram-Schmidt on w (block-major FP64, length L).  MODE:
//   kMgsDot    (first step of a column): partial sums of V_inext . w;
//   kMgsUpdDot (middle steps): w -= (hprev * vscale[iprev]) V_iprev, then V_inext . w;
//   kMgsUpdNrm (last step):    the same update, then w . w.
// Per-block partials go to part[blk]; the last block to finish (ticket on *counter) sums the
// nblk partials in a fixed order and writes *hnext = vscale[inext] * sum (the plain sum for
// w . w), then resets the counter for the next launch.  Every block owns the same element
// slice in every step, so w needs no grid-wide sync.  The mode is a template parameter:
// with runtime branches in the streaming loop the kernel ran at half its bandwidth.
constexpr int kMgsDot = 0, kMgsUpdDot = 1, kMgsUpdNrm = 2;

template <int MODE>
__device__ __forceinline__ void mgs_step_body(int blk, int nblk, const double* __restrict__ V, int64_t ldv, int iprev,
                                              int inext, const double* __restrict__ vscale,
                                              const double* __restrict__ hprev, double* __restrict__ hnext,
                                              double* __restrict__ w, int64_t L, double* __restrict__ part,
                                              unsigned* __restrict__ counter) {
  constexpr bool UPD = MODE != kMgsDot;
  constexpr bool DOT = MODE != kMgsUpdNrm;
  __shared__ double sh[kRedWarps];
  __shared__ int s_last;
  const double coef = UPD ? *hprev * (vscale ? vscale[iprev] : 1.0) : 0.0;
  const double* Vp = V + (int64_t)(UPD ? iprev : 0) * ldv;
  const double* Vn = V + (int64_t)(DOT ? inext : 0) * ldv;
  double acc = 0.0;
  const bool vec = ((L | ldv) & 1) == 0 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  const int64_t tid = (int64_t)blk * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)nblk * blockDim.x;
  if (vec) {
    const uint64_t keep = l2_policy_keep(), stream = l2_policy_stream();
    const int64_t L2 = L / 2;
    double a0 = 0.0, a1 = 0.0;
    // software-pipelined: the loads of the thread's next element pair are issued before the
    // FP64 arithmetic of the current one (the cache-hinted accesses keep their program order),
    // so each warp has a pair's loads in flight while its FMAs wait for the FP64 pipe
    const double2 z2 = make_double2(0.0, 0.0);
    double2 v = z2, a = z2, b = z2;
    int64_t e2 = tid;
    if (e2 < L2) {
      v = ld2_pol(w + 2 * e2, keep);
      if (UPD) a = ld2_ro_pol(Vp + 2 * e2, stream);
      if (DOT) b = ld2_ro_pol(Vn + 2 * e2, stream);
    }
    while (e2 < L2) {
      const int64_t f2 = e2 + nthr;
      double2 vn = z2, an = z2, bn = z2;
      if (f2 < L2) {
        vn = ld2_pol(w + 2 * f2, keep);
        if (UPD) an = ld2_ro_pol(Vp + 2 * f2, stream);
        if (DOT) bn = ld2_ro_pol(Vn + 2 * f2, stream);
      }
      if (UPD) {
        v.x = fma(-coef, a.x, v.x);
        v.y = fma(-coef, a.y, v.y);
        st2_pol(w + 2 * e2, v, keep);
      }
      if (DOT) {
        a0 = fma(b.x, v.x, a0);
        a1 = fma(b.y, v.y, a1);
      } else {
        a0 = fma(v.x, v.x, a0);
        a1 = fma(v.y, v.y, a1);
      }
      v = vn;
      a = an;
      b = bn;
      e2 = f2;
    }
    acc = a0 + a1;
  } else {
    for (int64_t e = tid; e < L; e += nthr) {
      double v = w[e];
      if (UPD) {
        v = fma(-coef, __ldg(Vp + e), v);
        w[e] = v;
      }
      acc = DOT ? fma(__ldg(Vn + e), v, acc) : fma(v, v, acc);
    }
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    part[blk] = t;
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double u = 0.0;
    for (int q = threadIdx.x; q < nblk; q += blockDim.x) u += __ldcg(part + q);
    u = block_sum(u, sh);
    if (threadIdx.x == 0) {
      *hnext = DOT ? u * (vscale ? vscale[inext] : 1.0) : u;
      *counter = 0u;
    }
  }
}

__device__ __forceinline__ void norm2_body(int blk, int nblk, const double* __restrict__ v, int64_t L,
                                           double* __restrict__ partials) {
  __shared__ double sh[kRedWarps];
  double acc2 = 0.0;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  for (int64_t e = (int64_t)blk * blockDim.x + threadIdx.x; e < L; e += stride) {
    const double a = __ldg(v + e);
    acc2 += a * a;
  }
  const double t = block_sum(acc2, sh);
  if (threadIdx.x == 0) partials[blk] = t;
}

// out (+)= sum_b partials[b], fixed summation order.
__device__ __forceinline__ void reduce_body(const double* __restrict__ partials, int nb, double* __restrict__ out,
                                            int accumulate) {
  __shared__ double sh[kRedWarps];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += partials[b];
  const double t = block_sum(a, sh);
  if (threadIdx.x == 0) *out = accumulate ? *out + t : t;
}

// Column j of the Hessenberg matrix: H[i][j] = h1[i] + h2[i] (i <= j), H[j+1][j] = sqrt(nrm2);
// apply the stored rotations, build the new one, update g, and record the
// relative residual estimate |g[j+1]| / bnorm.  vscale[j+1] = 1/H[j+1][j].
// bnorm <= 0: ||b|| is read from sc[bnorm()] (so a captured step serves any right-hand side).
__device__ __forceinline__ void givens_body(double* sc, int j, int m, double bnorm) {
  const ScLayout L{m};
  if (!(bnorm > 0.0)) bnorm = sc[L.bnorm()];
  for (int i = 0; i <= j; ++i) sc[L.H(i, j)] = sc[L.h1(i)] + sc[L.h2(i)];
  const double hn = sqrt(sc[L.nrm2()]);
  sc[L.hnext()] = hn;
  sc[L.vscale(j + 1)] = (hn > 0.0) ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double a = sc[L.H(i, j)], b = sc[L.H(i + 1, j)];
    sc[L.H(i, j)] = sc[L.cs(i)] * a + sc[L.sn(i)] * b;
    sc[L.H(i + 1, j)] = -sc[L.sn(i)] * a + sc[L.cs(i)] * b;
  }
  const double hjj = sc[L.H(j, j)];
  const double r = hypot(hjj, hn);
  double c = 1.0, s = 0.0;
  if (r != 0.0) {
    c = hjj / r;
    s = hn / r;
  }
  sc[L.cs(j)] = c;
  sc[L.sn(j)] = s;
  sc[L.H(j, j)] = r;
  sc[L.H(j + 1, j)] = 0.0;
  const double gj = sc[L.gv(j)];
  sc[L.gv(j + 1)] = -s * gj;
  sc[L.gv(j)] = c * gj;
  sc[L.est()] = fabs(sc[L.gv(j + 1)]) / bnorm;
}

__device__ __forceinline__ void backsolve_body(double* sc, int k, int m) {
  const ScLayout L{m};
  for (int i = k - 1; i >= 0; --i) {
    double v = sc[L.gv(i)];
    for (int q = i + 1; q < k; ++q) v -= sc[L.H(i, q)] * sc[L.y(q)];
    sc[L.y(i)] = v / sc[L.H(i, i)];
  }
}

__device__ __forceinline__ void xupdate_body(int blk, int nblk, const double* __restrict__ Z, int64_t ldz, int k,
                                             const double* __restrict__ y, double* __restrict__ x, int64_t L) {
  __shared__ double coef[kMaxRestart];
  for (int q = threadIdx.x; q < k; q += blockDim.x) coef[q] = y[q];
  __syncthreads();
  const int64_t stride = (int64_t)nblk * blockDim.x;
  const bool vec = ((L | ldz) & 1) == 0 && ((reinterpret_cast<uintptr_t>(Z) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
  if (vec) {
    // 16-byte elements, four basis vectors loaded together; the sum runs in the order q = 0 .. k-1
    for (int64_t e2 = (int64_t)blk * blockDim.x + threadIdx.x; e2 < L / 2; e2 += stride) {
      double2 v = *reinterpret_cast<const double2*>(x + 2 * e2);
      int q = 0;
      for (; q + 4 <= k; q += 4) {
        const double2 z0 = ld2(Z + (int64_t)q * ldz + 2 * e2), z1 = ld2(Z + (int64_t)(q + 1) * ldz + 2 * e2);
        const double2 z2 = ld2(Z + (int64_t)(q + 2) * ldz + 2 * e2), z3 = ld2(Z + (int64_t)(q + 3) * ldz + 2 * e2);
        v.x = fma(coef[q + 3], z3.x, fma(coef[q + 2], z2.x, fma(coef[q + 1], z1.x, fma(coef[q], z0.x, v.x))));
        v.y = fma(coef[q + 3], z3.y, fma(coef[q + 2], z2.y, fma(coef[q + 1], z1.y, fma(coef[q], z0.y, v.y))));
      }
      for (; q < k; ++q) {
        const double2 z = ld2(Z + (int64_t)q * ldz + 2 * e2);
        v.x = fma(coef[q], z.x, v.x);
        v.y = fma(coef[q], z.y, v.y);
      }
      *reinterpret_cast<double2*>(x + 2 * e2) = v;
    }
    return;
  }
  for (int64_t e = (int64_t)blk * blockDim.x + threadIdx.x; e < L; e += stride) {
    double v = x[e];
    for (int q = 0; q < k; ++q) v = fma(coef[q], __ldg(Z + (int64_t)q * ldz + e), v);
    x[e] = v;
  }
}

// Start of a cycle: beta = sqrt(nrm2); g = (beta, 0, ..); vscale[0] = 1/beta.
__device__ __forceinline__ void cycle_init_body(double* sc, int m) {
  const ScLayout L{m};
  const double beta = sqrt(sc[L.nrm2()]);
  for (int i = 0; i <= m; ++i) sc[L.gv(i)] = 0.0;
  for (int i = 0; i <= m; ++i) sc[L.h2(i)] = 0.0;   // the single-pass orthogonalisations leave h2 at zero
  sc[L.gv(0)] = beta;
  sc[L.vscale(0)] = (beta > 0.0) ? 1.0 / beta : 0.0;
}

}  // namespace aao
