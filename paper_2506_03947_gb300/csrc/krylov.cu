// FP64 kernels of the outer solve: the all-at-once matvec (Eq. 1), the
// Gram-Schmidt reductions and updates of FGMRES, Givens rotations, the
// triangular solve and the solution update.
//
// Reductions are deterministic: every flat-vector reduction uses a block count
// that depends on the vector length only, writes one partial sum per block,
// and a second kernel adds the partials in a fixed order.
#include "krylov_bodies.cuh"

#include <atomic>

namespace aao {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_add(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---- script-A matvec --------------------------------------------------------

// y_t = A x_t - x_{t-1} (MODE 0) or y_t = b_t - (A x_t - x_{t-1}) (MODE 1), for all
// t at one cell per thread; A = I + K with per-cell face coefficients.  MODE 1
// also writes one partial sum of y^2 per block.
template <int DIM, int MODE>
__global__ void __launch_bounds__(256)
    k_aao_matvec(GridDesc g, int ell, const double* __restrict__ cx, const double* __restrict__ cy,
                 const double* __restrict__ cz, const double* __restrict__ x, const double* __restrict__ b,
                 double* __restrict__ y, double* __restrict__ partials) {
  aao_matvec_body<DIM, MODE>(g, ell, blockIdx.x, blockIdx.y, blockIdx.z,
                             blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z), cx, cy, cz, x, b, y,
                             partials);
}

cudaError_t launch_aao_matvec(const GridDesc& g, int dim, int ell, const double* cx, const double* cy,
                              const double* cz, const double* x, const double* b, double* y, double* partials,
                              int* nblocks_out, cudaStream_t s) {
  dim3 block, grid;
  if (dim == 1) {
    block = dim3(256, 1, 1);
    grid = dim3((unsigned)((g.n0 + 255) / 256), 1, 1);
  } else {
    block = dim3(32, 8, 1);
    grid = dim3((unsigned)((g.n0 + 31) / 32), (unsigned)((g.n1 + 7) / 8), (unsigned)g.n2);
  }
  if (nblocks_out) *nblocks_out = (int)(grid.x * grid.y * grid.z);
  const int mode = (b != nullptr) ? 1 : 0;
#define AAO_MV(D, M) k_aao_matvec<D, M><<<grid, block, 0, s>>>(g, ell, cx, cy, cz, x, b, y, partials)
  switch (dim * 10 + mode) {
    case 10: AAO_MV(1, 0); break;
    case 11: AAO_MV(1, 1); break;
    case 20: AAO_MV(2, 0); break;
    case 21: AAO_MV(2, 1); break;
    case 30: AAO_MV(3, 0); break;
    case 31: AAO_MV(3, 1); break;
    default: return cudaErrorInvalidValue;
  }
#undef AAO_MV
  count_launch();
  return cudaGetLastError();
}

// ---- flat-vector reductions ---------------------------------------------------

int reduction_blocks(int64_t L) {
  // about 8 elements per thread at least, at most 1216 blocks (8 per SM on 152 SMs)
  int64_t nb = (L + (int64_t)kRedThreads * 8 - 1) / ((int64_t)kRedThreads * 8);
  if (nb < 1) nb = 1;
  if (nb > 1216) nb = 1216;
  return (int)nb;
}

// partials[i*NB + blk] = vscale[i] * sum_{e in block slice} V_i[e] w[e], for i in [i0, i0+G).
// G is the exact number of vectors of this launch: a runtime bound inside the
// unrolled loop would let the compiler turn the guards into selects and issue
// FP64 multiply-adds for all slots, and FP64 arithmetic is this kernel's limit.
template <int G>
__global__ void __launch_bounds__(kRedThreads)
    k_multidot(const double* __restrict__ V, int64_t ldv, int i0, const double* __restrict__ vscale,
               const double* __restrict__ w, int64_t L, double* __restrict__ partials) {
  multidot_body<G>(blockIdx.x, gridDim.x, V, ldv, i0, vscale, w, L, partials);
}

cudaError_t launch_multidot(const double* V, int64_t ldv, int nv, const double* vscale, const double* w,
                            int64_t L, double* partials, cudaStream_t s) {
  const int nb = reduction_blocks(L);
  for (int i0 = 0; i0 < nv; i0 += kDotGroup) {
    const int g = (nv - i0 < kDotGroup) ? nv - i0 : kDotGroup;
    switch (g) {
#define AAO_MD(G) \
  case G:         \
    k_multidot<G><<<nb, kRedThreads, 0, s>>>(V, ldv, i0, vscale, w, L, partials); \
    break;
      AAO_MD(1)
      AAO_MD(2)
      AAO_MD(3)
      AAO_MD(4)
      AAO_MD(5)
      AAO_MD(6)
      AAO_MD(7)
      AAO_MD(8)
#undef AAO_MD
      default:
        return cudaErrorInvalidValue;
    }
    count_launch();
  }
  return cudaGetLastError();
}

// w[e] -= sum_i h[i] vscale[i] V_i[e]; optional per-block partial sums of the new w^2.
__global__ void __launch_bounds__(kRedThreads)
    k_orth_update(const double* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ h,
                  const double* __restrict__ vscale, double* __restrict__ w, int64_t L,
                  double* __restrict__ partials) {
  orth_update_body(blockIdx.x, gridDim.x, V, ldv, nv, h, vscale, w, L, partials);
}

cudaError_t launch_orth_update(const double* V, int64_t ldv, int nv, const double* h, const double* vscale,
                               double* w, int64_t L, double* partials_norm, cudaStream_t s) {
  const int nb = reduction_blocks(L);
  k_orth_update<<<nb, kRedThreads, 0, s>>>(V, ldv, nv, h, vscale, w, L, partials_norm);
  count_launch();
  return cudaGetLastError();
}

template <int MODE>
__global__ void __launch_bounds__(kRedThreads)
    k_mgs_step(const double* __restrict__ V, int64_t ldv, int iprev, int inext, const double* __restrict__ vscale,
               const double* __restrict__ hprev, double* __restrict__ hnext, double* __restrict__ w, int64_t L,
               double* __restrict__ part, unsigned* __restrict__ counter) {
  mgs_step_body<MODE>(blockIdx.x, gridDim.x, V, ldv, iprev, inext, vscale, hprev, hnext, w, L, part, counter);
}

// Blocks of the modified Gram-Schmidt steps: four per SM (measured on GB300: the fused
// update + dot pass streams at 5.7 TB/s with four 256-thread blocks per SM and at 5.0 TB/s
// with eight; more blocks also lengthen the last block's sum of the partials), at most
// reduction_blocks(L).
int mgs_blocks(int64_t L) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm <= 0) {
      cudaGetLastError();
      nsm = 152;
    }
  }
  const int nb = reduction_blocks(L);
  return nb < 4 * nsm ? nb : 4 * nsm;
}

cudaError_t launch_mgs_step(const double* V, int64_t ldv, int iprev, int inext, const double* vscale,
                            const double* hprev, double* hnext, double* w, int64_t L, double* part,
                            unsigned* counter, cudaStream_t s) {
  const int nb = mgs_blocks(L);
  if (iprev < 0)
    k_mgs_step<kMgsDot><<<nb, kRedThreads, 0, s>>>(V, ldv, iprev, inext, vscale, hprev, hnext, w, L, part, counter);
  else if (inext >= 0)
    k_mgs_step<kMgsUpdDot><<<nb, kRedThreads, 0, s>>>(V, ldv, iprev, inext, vscale, hprev, hnext, w, L, part, counter);
  else
    k_mgs_step<kMgsUpdNrm><<<nb, kRedThreads, 0, s>>>(V, ldv, iprev, inext, vscale, hprev, hnext, w, L, part, counter);
  count_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
    k_norm2_partials(const double* __restrict__ v, int64_t L, double* __restrict__ partials) {
  norm2_body(blockIdx.x, gridDim.x, v, L, partials);
}

cudaError_t launch_norm2_partials(const double* v, int64_t L, double* partials, cudaStream_t s) {
  k_norm2_partials<<<reduction_blocks(L), kRedThreads, 0, s>>>(v, L, partials);
  count_launch();
  return cudaGetLastError();
}

// out[i] (+)= sum_b partials[i*nb + b]: one block per i, fixed summation order.
__global__ void __launch_bounds__(kRedThreads)
    k_reduce(const double* __restrict__ partials, int nb, double* __restrict__ out, int accumulate) {
  reduce_body(partials + (int64_t)blockIdx.x * nb, nb, out + blockIdx.x, accumulate);
}

cudaError_t launch_reduce(const double* partials, int nv, int nb, double* out, int accumulate, cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  k_reduce<<<nv, kRedThreads, 0, s>>>(partials, nb, out, accumulate);
  count_launch();
  return cudaGetLastError();
}

// ---- small dense FGMRES steps (one thread; sizes <= kMaxRestart) ---------------

__global__ void k_givens(double* sc, int j, int m, double bnorm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  givens_body(sc, j, m, bnorm);
}

cudaError_t launch_givens(double* sc, int j, int m, double bnorm, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(sc, j, m, bnorm);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_backsolve(double* sc, int k, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  backsolve_body(sc, k, m);
}

cudaError_t launch_backsolve(double* sc, int k, int m, cudaStream_t s) {
  k_backsolve<<<1, 32, 0, s>>>(sc, k, m);
  count_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
    k_xupdate(const double* __restrict__ Z, int64_t ldz, int k, const double* __restrict__ y,
              double* __restrict__ x, int64_t L) {
  xupdate_body(blockIdx.x, gridDim.x, Z, ldz, k, y, x, L);
}

cudaError_t launch_xupdate(const double* Z, int64_t ldz, int k, const double* y, double* x, int64_t L,
                           cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_xupdate<<<reduction_blocks(L), kRedThreads, 0, s>>>(Z, ldz, k, y, x, L);
  count_launch();
  return cudaGetLastError();
}

// Outer Chebyshev step (the paper's outer solver): d = c1 d + c2 z, then x += d.
__global__ void __launch_bounds__(kRedThreads)
    k_ci_update(double* __restrict__ d, const double* __restrict__ z, double* __restrict__ x, double c1, double c2,
                int64_t L) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += stride) {
    const double dn = fma(c2, __ldg(z + e), c1 * d[e]);
    d[e] = dn;
    x[e] += dn;
  }
}

cudaError_t launch_ci_update(double* d, const double* z, double* x, double c1, double c2, int64_t L, cudaStream_t s) {
  k_ci_update<<<reduction_blocks(L), kRedThreads, 0, s>>>(d, z, x, c1, c2, L);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_cycle_init(double* sc, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cycle_init_body(sc, m);
}

cudaError_t launch_cycle_init(double* sc, int m, cudaStream_t s) {
  k_cycle_init<<<1, 32, 0, s>>>(sc, m);
  count_launch();
  return cudaGetLastError();
}

}  // namespace aao
