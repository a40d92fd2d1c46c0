// Batched kernels: one launch runs a phase of the solve for many instances.
//
// Each launch covers a static work list: the blocks of every listed instance,
// numbered consecutively (prefix offsets start[]); a block finds its instance
// by binary search and runs the same device body as the single-instance
// kernel on its own block coordinates.  Instances whose active flag is 0
// (converged, or finished with their Krylov cycle) exit at once, so the
// launch geometry never changes and a whole Arnoldi step can be captured in a
// CUDA graph.  The Chebyshev kernels are templated on ell, so their lists are
// split by ell; the FP64 kernels take ell at run time.
#include "batch.cuh"
#include "cheb_ends.cuh"
#include "cheb_kernels.cuh"
#include "cheb_quad.cuh"
#include "krylov_bodies.cuh"

namespace aao {

__device__ __forceinline__ int wl_find(const WorkList& wl, int b) {
  int lo = 0, hi = wl.cnt;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (wl.start[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---- preconditioner: forward transform and Chebyshev steps (FP32, 2D, v4) ----

template <int ELL>
__global__ void __launch_bounds__(256) kb_dft(const BInst* __restrict__ I, const int* __restrict__ act, WorkList wl,
                                               int j) {
  __shared__ float gs[ELL];
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  dft_body<float, ELL>(b.g.N, blockIdx.x - wl.start[li], b.V + (int64_t)j * b.L, b.sc + L.vscale(j), b.bhat, *b.da,
                       gs);
}

// Member-local block lb of the single-step kernels (32 x 8 threads, four cells per thread along
// x) as block coordinates (bx, by, bz) of the member's grid.
__device__ __forceinline__ void step_block(const GridDesc& g, int lb, int& bx, int& by, int& bz) {
  const int gx = (g.n0 + 127) / 128, gy = (g.n1 + 7) / 8;
  bx = lb % gx;
  by = (lb / gx) % gy;
  bz = lb / (gx * gy);
}

// The transform and step 1 of every member of one ell in one launch (ends::dft_first_body on
// the same 128 x 8 tiles as the single steps; 2D): bhat and x_2 into field 0.
template <int ELL>
__global__ void __launch_bounds__(256) kb_dft_first(const BInst* __restrict__ I, const int* __restrict__ act,
                                                     WorkList wl, int j) {
  extern __shared__ __align__(16) float sb_first[];
  __shared__ float gs[ELL];
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;  // the whole block: before any barrier
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  int bx, by, bz;
  step_block(b.g, blockIdx.x - wl.start[li], bx, by, bz);
  ends::dft_first_body<ELL>(b.g, bx, by, b.V + (int64_t)j * b.L, b.sc + L.vscale(j), b.bhat, b.xa, b.cx32, b.cy32,
                            *b.da, b.steps[1], sb_first, gs);
}

// Step k = 1 from x_1 = bhat/theta (x_0 = 0): x_2 into field 0.
template <int ELL, int DIM>
__global__ void __launch_bounds__(256) kb_step_first(const BInst* __restrict__ I, const int* __restrict__ act,
                                                      WorkList wl, int j) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  int bx, by, bz;
  step_block(b.g, blockIdx.x - wl.start[li], bx, by, bz);
  cheb_step_v4_body<ELL, DIM, 0, 0, false>(b.g, bx, by, bz, b.cx32, b.cy32, b.cz32, b.bhat, nullptr, b.xa,
                                           nullptr, b.steps[1], *b.ia);
}

__device__ __forceinline__ float* field(const BInst& b, int i) {
  return i == 0 ? b.xa : i == 1 ? b.xb : i == 2 ? b.xc : b.xd;
}

// z = Z_j = Gamma^{-1} U x_p for every member of one ell (ends::idft_pair), x_p in field fld;
// member-local block lb covers cells [1024 lb, 1024 lb + 1024) (the list gives a member at least
// N / 1024 blocks: its 128 x 8 tiles).
template <int ELL>
__global__ void __launch_bounds__(256) kb_idft(const BInst* __restrict__ I, const int* __restrict__ act, WorkList wl,
                                                int j, int fld) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const int64_t base = (int64_t)(blockIdx.x - wl.start[li]) * 1024;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t c = base + 512 * h + 2 * threadIdx.x;
    if (c < b.g.N)
      ends::idft_pair<ELL>(b.g.N, c, field(b, fld), b.Z + (int64_t)j * b.L, *b.ia);
  }
}

// Steps k .. k+3 from x_k = field cur and x_{k-1} = field prev (PSRC 2) or bhat/theta (PSRC 1),
// writing x_{k+3} to field o3 and x_{k+4} to field o4; one block per (instance, tile).
template <int ELL, int PSRC>
__global__ void __launch_bounds__(kQuadTileNT, 2) kb_quad(const BInst* __restrict__ I, const int* __restrict__ act,
                                                        WorkList wl, int k, int cur, int prev, int o3, int o4) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const int lb = blockIdx.x - wl.start[li];
  const GridDesc g = b.g;
  const int tx = (g.n0 + kQuadInnerX - 1) / kQuadInnerX;
  static_assert(sizeof(QuadArgs) == 4 * sizeof(StepArgs<float>), "four consecutive step tables");
  cheb_quad_body<ELL, kQuadTileTY, PSRC, kQuadTileNT>(g, lb % tx, lb / tx, b.cx32, b.cy32, b.bhat, field(b, cur),
                                                      PSRC == 2 ? field(b, prev) : nullptr, field(b, o3),
                                                      field(b, o4), *reinterpret_cast<const QuadArgs*>(b.steps + k));
}

// One step k from x_k = field cur; x_{k-1} = field io (PSRC 2, overwritten by x_{k+1}) or
// bhat/theta (PSRC 1, x_{k+1} into field io).
template <int ELL, int DIM, int PSRC>
__global__ void __launch_bounds__(256) kb_step_f(const BInst* __restrict__ I, const int* __restrict__ act,
                                                  WorkList wl, int k, int j, int cur, int io) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  int bx, by, bz;
  step_block(b.g, blockIdx.x - wl.start[li], bx, by, bz);
  cheb_step_v4_body<ELL, DIM, 1, PSRC, false>(b.g, bx, by, bz, b.cx32, b.cy32, b.cz32, b.bhat, field(b, cur),
                                              field(b, io), nullptr, b.steps[k], *b.ia);
}

// Members that share one grid and its face coefficients (right-hand sides of one operator):
// one block per tile of that grid; the tile's stencil is loaded once and applied to every
// active member's fields.  KSRC 0: step k = 1 from x_1 = bhat/theta into field 0.
template <int ELL, int DIM, int KSRC, int PSRC>
__global__ void __launch_bounds__(256) kb_step_shared(const BInst* __restrict__ I, const int* __restrict__ act, int M,
                                                       int k, int j, int cur, int io) {
  const BInst& b0 = I[0];
  int bx, by, bz;
  step_block(b0.g, blockIdx.x, bx, by, bz);
  Stencil4<DIM> st;
  int64_t c = 0;
  if (!make_stencil4<DIM>(b0.g, bx, by, bz, b0.cx32, b0.cy32, b0.cz32, st, c)) return;
  for (int r = 0; r < M; ++r) {
    if (!act[r]) continue;
    const BInst& b = I[r];
    const float* xk = (KSRC == 0) ? nullptr : field(b, cur);
    float* xio = (KSRC == 0) ? b.xa : field(b, io);
    cheb_step_v4_apply<ELL, DIM, KSRC, PSRC, false>(b.g, st, c, b.bhat, xk, xio, nullptr, b.steps[KSRC == 0 ? 1 : k],
                                                    *b.ia);
  }
}

// ---- FP64 outer solve ----------------------------------------------------------

// mode 0: V_{j+1} = script-A Z_j; mode 1: V_0 = b - script-A x with norm partials
template <int MODE, int DIM>
__global__ void __launch_bounds__(256) kb_matvec(const BInst* __restrict__ I, const int* __restrict__ act, WorkList wl,
                                                  int j) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const int lb = blockIdx.x - wl.start[li];
  const int gx = (b.g.n0 + 31) / 32, gy = (b.g.n1 + 7) / 8;
  const int bx = lb % gx, by = (lb / gx) % gy, bz = lb / (gx * gy);
  if (MODE == 0)
    aao_matvec_body<DIM, 0>(b.g, b.ell, bx, by, bz, lb, b.cx64, b.cy64, b.cz64, b.Z + (int64_t)j * b.L, nullptr,
                            b.V + (int64_t)(j + 1) * b.L, nullptr);
  else
    aao_matvec_body<DIM, 1>(b.g, b.ell, bx, by, bz, lb, b.cx64, b.cy64, b.cz64, b.x, b.b, b.V, b.partials);
}

template <int G>
__global__ void __launch_bounds__(kRedThreads) kb_multidot(const BInst* __restrict__ I, const int* __restrict__ act,
                                                            WorkList wl, int j, int i0) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  multidot_body<G>(blockIdx.x - wl.start[li], b.nbred, b.V, b.L, i0, b.sc + L.vscale(0), b.V + (int64_t)(j + 1) * b.L,
                   b.L, b.partials);
}

__global__ void __launch_bounds__(kRedThreads) kb_orth_update(const BInst* __restrict__ I, const int* __restrict__ act,
                                                               WorkList wl, int j, int second) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  orth_update_body(blockIdx.x - wl.start[li], b.nbred, b.V, b.L, j + 1, b.sc + (second ? L.h2(0) : L.h1(0)),
                   b.sc + L.vscale(0), b.V + (int64_t)(j + 1) * b.L, b.L,
                   second ? b.partials + (int64_t)(b.m + 1) * b.nbred : nullptr);
}

// Step i of modified Gram-Schmidt on w = V_{j+1} (MODE as in mgs_step_body).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) kb_mgs_step(const BInst* __restrict__ I, const int* __restrict__ act,
                                                            WorkList wl, int j, int iprev, int inext) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  double* hnext = (MODE == kMgsUpdNrm) ? b.sc + L.nrm2() : b.sc + L.h1(inext);
  const double* hprev = (MODE == kMgsDot) ? nullptr : b.sc + L.h1(iprev);
  mgs_step_body<MODE>(blockIdx.x - wl.start[li], b.nbmgs, b.V, b.L, iprev, inext, b.sc + L.vscale(0), hprev, hnext,
                      b.V + (int64_t)(j + 1) * b.L, b.L, b.partials, b.counter);
}

__global__ void __launch_bounds__(kRedThreads) kb_norm2(const BInst* __restrict__ I, const int* __restrict__ act,
                                                         WorkList wl) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  norm2_body(blockIdx.x - wl.start[li], b.nbred, b.b, b.L, b.partials);
}

// grid (nout, instances of wl): what = 0 -> h1[i], 1 -> h2[i] from the multi-dot
// partials; 2 -> nrm2 from the update's norm partials; 3 -> nrm2 from the residual
// matvec partials; 4 -> nrm2 from kb_norm2's partials.
__global__ void __launch_bounds__(kRedThreads) kb_reduce(const BInst* __restrict__ I, const int* __restrict__ act,
                                                          WorkList wl, int what) {
  const int inst = wl.inst[blockIdx.y];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  const int i = blockIdx.x;
  if (what <= 1) {
    reduce_body(b.partials + (int64_t)i * b.nbred, b.nbred, b.sc + (what == 0 ? L.h1(i) : L.h2(i)), 0);
  } else if (i == 0) {
    const double* src = (what == 2) ? b.partials + (int64_t)(b.m + 1) * b.nbred : b.partials;
    const int nb = (what == 3) ? b.nbmv : b.nbred;
    reduce_body(src, nb, b.sc + L.nrm2(), 0);
  }
}

// one block per instance, thread 0: op 0 givens(j), 1 cycle_init, 2 backsolve(kvec),
// 3 gather (est, hnext) -> out[2 inst], 4 gather sqrt(nrm2) -> out[2 inst] and store it as bnorm,
// 5 gather sqrt(nrm2) -> out[2 inst]
__global__ void kb_small(const BInst* __restrict__ I, const int* __restrict__ act, WorkList wl, int op, int j,
                         const int* __restrict__ kvec, double* __restrict__ out) {
  const int inst = wl.inst[blockIdx.x];
  if (threadIdx.x != 0 || !act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  switch (op) {
    case 0: givens_body(b.sc, j, b.m, b.sc[L.bnorm()]); break;
    case 1: cycle_init_body(b.sc, b.m); break;
    case 2: backsolve_body(b.sc, kvec[inst], b.m); break;
    case 3:
      out[2 * inst] = b.sc[L.est()];
      out[2 * inst + 1] = b.sc[L.hnext()];
      break;
    case 4:
      b.sc[L.bnorm()] = sqrt(b.sc[L.nrm2()]);
      out[2 * inst] = b.sc[L.bnorm()];
      break;
    case 5: out[2 * inst] = sqrt(b.sc[L.nrm2()]); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kRedThreads) kb_xupdate(const BInst* __restrict__ I, const int* __restrict__ act,
                                                           WorkList wl, const int* __restrict__ kvec) {
  const int li = wl_find(wl, blockIdx.x);
  const int inst = wl.inst[li];
  if (!act[inst]) return;
  const BInst& b = I[inst];
  const ScLayout L{b.m};
  xupdate_body(blockIdx.x - wl.start[li], b.nbred, b.Z, b.L, kvec[inst], b.sc + L.y(0), b.x, b.L);
}

// ---- launchers -------------------------------------------------------------------

#define AAO_BCHECK()        \
  do {                      \
    count_launch();         \
    cudaError_t e_ = cudaGetLastError(); \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

int batch_quad_tiles(const GridDesc& g) {
  return ((g.n0 + kQuadInnerX - 1) / kQuadInnerX) * ((g.n1 + kQuadTileTY - 1) / kQuadTileTY);
}

template <int ELL>
cudaError_t batch_precond_ell(const BInst* I, const int* act, const WorkList& wdft, const WorkList& wstep,
                              const WorkList& wquad, int p, int j, cudaStream_t s) {
  if (wdft.cnt == 0) return cudaSuccess;
  if (p < 2) return cudaErrorInvalidValue;  // the batch runs p >= 2
  kb_dft<ELL><<<wdft.total, 256, 0, s>>>(I, act, wdft, j);
  AAO_BCHECK();
  const dim3 blk(32, 8, 1);
  // k = 1: x_1 = bhat/theta, x_0 = 0 -> x_2 in field 0
  kb_step_first<ELL, 2><<<wstep.total, blk, 0, s>>>(I, act, wstep, j);
  AAO_BCHECK();
  // Four-step launches while steps k .. k+3 all come before the last step; the four fields
  // rotate so that a launch never writes a field it reads (same schedule as the single solver).
  const size_t qsmem = quad_smem_bytes<kQuadTileTY>();
  int cur = 0, prev = -1, k = 2;
  while (k + 3 <= p - 2) {
    int o[2], n = 0;
    for (int f = 0; f < 4 && n < 2; ++f)
      if (f != cur && f != prev) o[n++] = f;
    if (prev < 0) {
      const cudaError_t ea = cudaFuncSetAttribute(kb_quad<ELL, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)qsmem);
      if (ea != cudaSuccess) return ea;
      kb_quad<ELL, 1><<<wquad.total, kQuadTileNT, qsmem, s>>>(I, act, wquad, k, cur, 0, o[0], o[1]);
    } else {
      const cudaError_t ea = cudaFuncSetAttribute(kb_quad<ELL, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)qsmem);
      if (ea != cudaSuccess) return ea;
      kb_quad<ELL, 2><<<wquad.total, kQuadTileNT, qsmem, s>>>(I, act, wquad, k, cur, prev, o[0], o[1]);
    }
    AAO_BCHECK();
    prev = o[0];
    cur = o[1];
    k += 4;
  }
  // single steps up to p - 1, x_{k+1} over x_{k-1}; then z = Gamma^{-1} U x_p into Z_j
  for (; k <= p - 1; ++k) {
    int dst = prev;
    if (dst < 0) dst = (cur == 0) ? 1 : 0;
    if (prev < 0) kb_step_f<ELL, 2, 1><<<wstep.total, blk, 0, s>>>(I, act, wstep, k, j, cur, dst);
    else kb_step_f<ELL, 2, 2><<<wstep.total, blk, 0, s>>>(I, act, wstep, k, j, cur, dst);
    AAO_BCHECK();
    prev = cur;
    cur = dst;
  }
  kb_idft<ELL><<<wstep.total, 256, 0, s>>>(I, act, wstep, j, cur);
  AAO_BCHECK();
  return cudaSuccess;
}

template <int ELL, int DIM>
cudaError_t batch_precond_head_ell(const BInst* I, const int* act, const SharedSteps& sh, const WorkList& wdft,
                                   const WorkList& wstep, int p, int j, cudaStream_t s) {
  if (wdft.cnt == 0) return cudaSuccess;
  if (p < 3) return cudaErrorInvalidValue;  // the split schedule needs a step before the last one
  kb_dft<ELL><<<wdft.total, 256, 0, s>>>(I, act, wdft, j);
  AAO_BCHECK();
  const dim3 blk(32, 8, 1);
  if (sh.on) kb_step_shared<ELL, DIM, 0, 0><<<sh.ntiles, blk, 0, s>>>(I, act, sh.M, 1, j, 0, 0);
  else kb_step_first<ELL, DIM><<<wstep.total, blk, 0, s>>>(I, act, wstep, j);  // x_2 into field 0
  AAO_BCHECK();
  return cudaSuccess;
}

template <int ELL, int DIM>
cudaError_t batch_steps_mid_ell(const BInst* I, const int* act, const SharedSteps& sh, const WorkList& wstep, int p,
                                int j, int k, int* curp, int* prevp, cudaStream_t s) {
  if (!sh.on && wstep.cnt == 0) return cudaSuccess;
  const dim3 blk(32, 8, 1);
  const unsigned nb = sh.on ? (unsigned)sh.ntiles : (unsigned)wstep.total;
  int cur = *curp, prev = *prevp;
  for (; k <= p - 2; ++k) {
    int dst = prev;
    if (dst < 0) dst = (cur == 0) ? 1 : 0;
    if (sh.on) {
      if (prev < 0) kb_step_shared<ELL, DIM, 1, 1><<<nb, blk, 0, s>>>(I, act, sh.M, k, j, cur, dst);
      else kb_step_shared<ELL, DIM, 1, 2><<<nb, blk, 0, s>>>(I, act, sh.M, k, j, cur, dst);
    } else {
      if (prev < 0) kb_step_f<ELL, DIM, 1><<<nb, blk, 0, s>>>(I, act, wstep, k, j, cur, dst);
      else kb_step_f<ELL, DIM, 2><<<nb, blk, 0, s>>>(I, act, wstep, k, j, cur, dst);
    }
    AAO_BCHECK();
    prev = cur;
    cur = dst;
  }
  *curp = cur;
  *prevp = prev;
  return cudaSuccess;
}

cudaError_t batch_precond_head(const BInst* I, const int* act, int ell, int dim, const SharedSteps& sh,
                               const WorkList& wdft, const WorkList& wstep, int p, int j, cudaStream_t s) {
  switch (ell * 10 + dim) {
#define AAO_BH(L)                                                                         \
  case L * 10 + 2: return batch_precond_head_ell<L, 2>(I, act, sh, wdft, wstep, p, j, s); \
  case L * 10 + 3: return batch_precond_head_ell<L, 3>(I, act, sh, wdft, wstep, p, j, s);
    AAO_BH(4)
    AAO_BH(6)
    AAO_BH(8)
    AAO_BH(10)
    AAO_BH(12)
    AAO_BH(14)
    AAO_BH(16)
#undef AAO_BH
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_dft_first(const BInst* I, const int* act, int ell, const WorkList& wstep, int j, cudaStream_t s) {
  if (wstep.cnt == 0) return cudaSuccess;
  switch (ell) {
#define AAO_BDF(L)                                                                                         \
  case L: {                                                                                                \
    const int smem = (int)(sizeof(float) * ends::dft_first_smem_floats(L));                              \
    const cudaError_t e = cudaFuncSetAttribute(kb_dft_first<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (e != cudaSuccess) return e;                                                                        \
    kb_dft_first<L><<<wstep.total, dim3(32, 8, 1), smem, s>>>(I, act, wstep, j);                          \
    break;                                                                                                 \
  }
    AAO_BDF(4)
    AAO_BDF(6)
    AAO_BDF(8)
    AAO_BDF(10)
    AAO_BDF(12)
    AAO_BDF(14)
    AAO_BDF(16)
#undef AAO_BDF
    default:
      return cudaErrorInvalidValue;
  }
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_idft(const BInst* I, const int* act, int ell, const WorkList& wstep, int j, int fld,
                       cudaStream_t s) {
  if (wstep.cnt == 0) return cudaSuccess;
  switch (ell) {
#define AAO_BID(L) \
  case L:          \
    kb_idft<L><<<wstep.total, 256, 0, s>>>(I, act, wstep, j, fld); \
    break;
    AAO_BID(4)
    AAO_BID(6)
    AAO_BID(8)
    AAO_BID(10)
    AAO_BID(12)
    AAO_BID(14)
    AAO_BID(16)
#undef AAO_BID
    default:
      return cudaErrorInvalidValue;
  }
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_steps_mid(const BInst* I, const int* act, int ell, int dim, const SharedSteps& sh,
                            const WorkList& wstep, int p, int j, int kf, int* cur, int* prev, cudaStream_t s) {
  switch (ell * 10 + dim) {
#define AAO_BM(L)                                                                               \
  case L * 10 + 2: return batch_steps_mid_ell<L, 2>(I, act, sh, wstep, p, j, kf, cur, prev, s); \
  case L * 10 + 3: return batch_steps_mid_ell<L, 3>(I, act, sh, wstep, p, j, kf, cur, prev, s);
    AAO_BM(4)
    AAO_BM(6)
    AAO_BM(8)
    AAO_BM(10)
    AAO_BM(12)
    AAO_BM(14)
    AAO_BM(16)
#undef AAO_BM
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_precond(const BInst* I, const int* act, int ell, const WorkList& wdft, const WorkList& wstep,
                          const WorkList& wquad, int p, int j, cudaStream_t s) {
  switch (ell) {
    case 4: return batch_precond_ell<4>(I, act, wdft, wstep, wquad, p, j, s);
    case 6: return batch_precond_ell<6>(I, act, wdft, wstep, wquad, p, j, s);
    case 8: return batch_precond_ell<8>(I, act, wdft, wstep, wquad, p, j, s);
    case 10: return batch_precond_ell<10>(I, act, wdft, wstep, wquad, p, j, s);
    case 12: return batch_precond_ell<12>(I, act, wdft, wstep, wquad, p, j, s);
    case 14: return batch_precond_ell<14>(I, act, wdft, wstep, wquad, p, j, s);
    case 16: return batch_precond_ell<16>(I, act, wdft, wstep, wquad, p, j, s);
    default: return cudaErrorInvalidValue;
  }
}

int batch_step_blocks(const GridDesc& g) { return ((g.n0 + 127) / 128) * ((g.n1 + 7) / 8) * g.n2; }

int batch_matvec_blocks(const GridDesc& g) { return ((g.n0 + 31) / 32) * ((g.n1 + 7) / 8) * g.n2; }

cudaError_t batch_matvec(const BInst* I, const int* act, const WorkList& wmv, int mode, int j, int dim,
                         cudaStream_t s) {
  const dim3 blk(32, 8, 1);
  if (dim == 3) {
    if (mode == 0) kb_matvec<0, 3><<<wmv.total, blk, 0, s>>>(I, act, wmv, j);
    else kb_matvec<1, 3><<<wmv.total, blk, 0, s>>>(I, act, wmv, j);
  } else {
    if (mode == 0) kb_matvec<0, 2><<<wmv.total, blk, 0, s>>>(I, act, wmv, j);
    else kb_matvec<1, 2><<<wmv.total, blk, 0, s>>>(I, act, wmv, j);
  }
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_gram_schmidt(const BInst* I, const int* act, const WorkList& wred, const WorkList& wone, int j,
                               cudaStream_t s) {
  const int nv = j + 1;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i0 = 0; i0 < nv; i0 += kDotGroup) {
      const int g = (nv - i0 < kDotGroup) ? nv - i0 : kDotGroup;
      switch (g) {
#define AAO_BMD(G) \
  case G: kb_multidot<G><<<wred.total, kRedThreads, 0, s>>>(I, act, wred, j, i0); break;
        AAO_BMD(1)
        AAO_BMD(2)
        AAO_BMD(3)
        AAO_BMD(4)
        AAO_BMD(5)
        AAO_BMD(6)
        AAO_BMD(7)
        AAO_BMD(8)
#undef AAO_BMD
        default: return cudaErrorInvalidValue;
      }
      AAO_BCHECK();
    }
    kb_reduce<<<dim3(nv, wone.cnt, 1), kRedThreads, 0, s>>>(I, act, wone, pass);
    AAO_BCHECK();
    kb_orth_update<<<wred.total, kRedThreads, 0, s>>>(I, act, wred, j, pass);
    AAO_BCHECK();
  }
  kb_reduce<<<dim3(1, wone.cnt, 1), kRedThreads, 0, s>>>(I, act, wone, 2);
  AAO_BCHECK();
  return cudaSuccess;
}

// At least 16 K elements (64 per thread) per block: with the reduction lists' ~2 K the fixed
// cost of a block (last-block ticket, block sums) rivalled its streaming work.
int batch_mgs_blocks(int64_t L) {
  const int64_t per_block = (int64_t)kRedThreads * 64;
  int64_t nb = (L + per_block - 1) / per_block;
  const int64_t cap = reduction_blocks(L);
  if (nb > cap) nb = cap;
  return nb < 1 ? 1 : (int)nb;
}

cudaError_t batch_mgs(const BInst* I, const int* act, const WorkList& wmgs, int j, cudaStream_t s) {
  kb_mgs_step<kMgsDot><<<wmgs.total, kRedThreads, 0, s>>>(I, act, wmgs, j, -1, 0);
  AAO_BCHECK();
  for (int i = 1; i <= j; ++i) {
    kb_mgs_step<kMgsUpdDot><<<wmgs.total, kRedThreads, 0, s>>>(I, act, wmgs, j, i - 1, i);
    AAO_BCHECK();
  }
  kb_mgs_step<kMgsUpdNrm><<<wmgs.total, kRedThreads, 0, s>>>(I, act, wmgs, j, j, -1);
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_reduce(const BInst* I, const int* act, const WorkList& wone, int what, cudaStream_t s) {
  kb_reduce<<<dim3(1, wone.cnt, 1), kRedThreads, 0, s>>>(I, act, wone, what);
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_small(const BInst* I, const int* act, const WorkList& wone, int op, int j, const int* kvec,
                        double* out, cudaStream_t s) {
  kb_small<<<wone.cnt, 32, 0, s>>>(I, act, wone, op, j, kvec, out);
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_norm2_b(const BInst* I, const int* act, const WorkList& wred, cudaStream_t s) {
  kb_norm2<<<wred.total, kRedThreads, 0, s>>>(I, act, wred);
  AAO_BCHECK();
  return cudaSuccess;
}

cudaError_t batch_xupdate(const BInst* I, const int* act, const WorkList& wred, const int* kvec, cudaStream_t s) {
  kb_xupdate<<<wred.total, kRedThreads, 0, s>>>(I, act, wred, kvec);
  AAO_BCHECK();
  return cudaSuccess;
}

}  // namespace aao
