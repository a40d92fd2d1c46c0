// Declarations of the batched launchers (batch.cu) used by the host driver.
#pragma once

#include "aao_internal.cuh"

namespace aao {

// Blocks of the listed instances, numbered consecutively: instance inst[i] owns
// blocks [start[i], start[i+1]); total = start[cnt].  Device arrays.
struct WorkList {
  const int* start;
  const int* inst;
  int cnt;
  int total;
};

// Everything a batched kernel needs about one instance (device array, one entry per member).
struct BInst {
  GridDesc g;
  int ell, m, nbred, nbmv, nbmgs;  // reduction, matvec and modified Gram-Schmidt blocks
  int64_t L;
  const float *cx32, *cy32, *cz32;
  const double *cx64, *cy64, *cz64;
  float *bhat, *xa, *xb, *xc, *xd;  // transformed rhs and the four rotating Chebyshev fields
  double *V, *Z, *sc, *partials;
  unsigned* counter;             // the member's last-block ticket (modified Gram-Schmidt)
  const StepArgs<float>* steps;  // p entries
  const DftArgs<float>* da;
  const IdftArgs<float>* ia;
  const double* b;
  double* x;
};

// Tiles (blocks) of the four-step kernel for one grid.
int batch_quad_tiles(const GridDesc& g);
// P_NC^{-1} of Arnoldi step j for the members of one ell: transform, step 1, four-step
// launches (shared-memory tile kernel; list wquad) while they fit before the last step, single
// steps for the rest (list wstep), the last step fused with the inverse transform into Z_j.
cudaError_t batch_precond(const BInst* I, const int* act, int ell, const WorkList& wdft, const WorkList& wstep,
                          const WorkList& wquad, int p, int j, cudaStream_t s);
cudaError_t batch_matvec(const BInst* I, const int* act, const WorkList& wmv, int mode, int j, int dim,
                         cudaStream_t s);
cudaError_t batch_gram_schmidt(const BInst* I, const int* act, const WorkList& wred, const WorkList& wone, int j,
                               cudaStream_t s);
// Modified Gram-Schmidt of Arnoldi step j: j + 2 fused launches over the list (one per basis
// vector, as in the single-instance solver), each writing h_i (or ||w||^2) from its last block.
// List wmgs gives instance i batch_mgs_blocks(L_i) blocks.
int batch_mgs_blocks(int64_t L);
cudaError_t batch_mgs(const BInst* I, const int* act, const WorkList& wmgs, int j, cudaStream_t s);
cudaError_t batch_reduce(const BInst* I, const int* act, const WorkList& wone, int what, cudaStream_t s);
cudaError_t batch_small(const BInst* I, const int* act, const WorkList& wone, int op, int j, const int* kvec,
                        double* out, cudaStream_t s);
cudaError_t batch_norm2_b(const BInst* I, const int* act, const WorkList& wred, cudaStream_t s);
cudaError_t batch_xupdate(const BInst* I, const int* act, const WorkList& wred, const int* kvec, cudaStream_t s);

// The single-step sweep of P_NC^{-1} for Arnoldi step j, per ell: batch_precond_head (the
// transform and step 1: bhat, and x_2 into field 0), batch_steps_mid (steps), and batch_idft
// (the inverse transform of x_p, below).
// dim: 2 or 3 (every member).  shared: every member has the same grid and face coefficients
// (right-hand sides of one operator); the step kernels then take one block per tile of that
// grid, load the tile's stencil once and apply it to every active member (M members,
// ntiles = the tile count of the grid), and wstep serves only the inverse transform.
struct SharedSteps {
  bool on;
  int M;
  int ntiles;
};
cudaError_t batch_precond_head(const BInst* I, const int* act, int ell, int dim, const SharedSteps& sh,
                               const WorkList& wdft, const WorkList& wstep, int p, int j, cudaStream_t s);
// Single steps k = kf .. p-2 (pass p + 1 to run through step p - 1, whose output is x_p), with
// x_k in field *cur and x_{k-1} in field *prev (-1: bhat/theta) at kf; each writes x_{k+1} over
// x_{k-1}.  On return *cur and *prev name the fields of the newest two iterates.
cudaError_t batch_steps_mid(const BInst* I, const int* act, int ell, int dim, const SharedSteps& sh,
                            const WorkList& wstep, int p, int j, int kf, int* cur, int* prev, cudaStream_t s);
// The ends of the sweep (members of one ell; list wstep: the 128 x 8 (x 1) tiles of each
// member): the transform with step 1 (2D members: bhat and x_2 into field 0), and the inverse
// transform of x_p (field fld) into Z_j (2D and 3D members, 1024 cells per block).
cudaError_t batch_dft_first(const BInst* I, const int* act, int ell, const WorkList& wstep, int j, cudaStream_t s);
cudaError_t batch_idft(const BInst* I, const int* act, int ell, const WorkList& wstep, int j, int fld,
                       cudaStream_t s);
// Blocks of the single-step kernels (32 x 8 threads, four cells each along x) for one grid.
int batch_step_blocks(const GridDesc& g);
// Blocks of the matvec kernel (32 x 8 threads, one cell each) for one grid.
int batch_matvec_blocks(const GridDesc& g);

// Device work queue of a batched warp-strip launch: tickets are taken from next; each warp
// adds one to done when it leaves, and the last one resets both (zero between launches).
struct StreamQueue {
  unsigned next, done;
};
// Units (plane pair x segment x strip) of one member for halo depth S and segment height H.
int batch_stream_units(const GridDesc& g, int ell, int S, int H);
// One launch of S fused steps k .. k+S-1 over the units of every active member (list units:
// member inst[i] owns units [start[i], start[i+1])), persistent over a device queue; the fields
// are the members' rotating buffers (0..3): x_k = cur, x_{k-1} = prev (psrc 2) or bhat/theta
// (psrc 1), outputs x_{k+S-1} -> o3 (o3 < 0: not written, the sweep's final launch) and
// x_{k+S} -> o4.
cudaError_t launch_batch_stream(const BInst* I, const int* act, const WorkList& units, const StreamConfig& c, int k,
                                int psrc, int cur, int prev, int o3, int o4, StreamQueue* queue, cudaStream_t s);

}  // namespace aao
