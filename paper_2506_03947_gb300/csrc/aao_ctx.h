// The handle behind aao_handle, and the few host helpers the library's translation units share
// (the C ABI is declared in include/aao.h).  Private to libaao.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "aao.h"
#include "aao_internal.cuh"

struct aao_multi;  // right-hand-side views of a handle and their batch (multi.cu)

struct aao_ctx {
  int dim = 0;
  int64_t n[3] = {1, 1, 1};
  int64_t N = 0, L = 0;
  int ell = 0;
  double alpha = 0.0;
  int prec = AAO_MIXED;
  int p = 20;                    // Chebyshev steps run per apply (max over frequencies)
  int palloc[aao::kMaxF] = {};   // per-frequency steps m = 0..ell/2 (NC2); all == p for NC1
  bool nc2 = false;
  int m = 64;
  int orth = AAO_ORTH_MGS;
  double mu_min = 1.0, mu_max = 0.0;
  cudaStream_t stream = nullptr;
  aao::GridDesc g{};

  double *cx64 = nullptr, *cy64 = nullptr, *cz64 = nullptr;
  float *cx32 = nullptr, *cy32 = nullptr, *cz32 = nullptr;
  void *bhat = nullptr, *xa = nullptr, *xb = nullptr;  // Chebyshev fields (float or double)
  void *xc = nullptr, *xd = nullptr;                   // extra fields for fused step pairs (2D mixed)
  bool pairs = false;                                  // fused two-step kernels in use
  aao::FieldMap fmap[7];                               // TMA descriptors of xa, xb, xc, xd, bhat, cx32, cy32
  bool tma = false;                                    // descriptors built: persistent four-step kernel usable
  int step_kernel = AAO_STEP_AUTO;                     // aao_set_step_kernel
  aao::StreamConfig scfg{};                            // warp-strip kernel configuration
  aao::StreamConfig tail{};  // the two-step final launch of a sweep whose remaining step count is 2 mod 4
  int auto_kind = AAO_STEP_TMA;                        // the kernel AAO_STEP_AUTO selects
  bool owns_coeffs = true;                             // false for a view sharing another handle's operator
  aao_multi* multi = nullptr;                          // cached views of aao_solve_multi
  bool multi_prof = false;  // aao_multi_profile_enable: event timing of the sweeps of aao_solve_multi
  bool tuned = false;                                  // kernel and configuration from the autotuner
  bool tma_used = false;                               // TMA kernel launched since the last fault check
  long long wait_limit = aao::kQuadTmaWaitCycles;      // bound of the TMA waits (aao_set_wait_limit)

  // CUDA graphs of Arnoldi step j (preconditioner, script-A product, Gram-Schmidt, Givens,
  // read-back of the residual estimate), captured on first use and replayed; dropped when
  // the tables, the step kernel or the wait limit change.
  int pmode = AAO_PRECOND_NC;     // aao_set_precond_mode
  aao::DctPlan* dct = nullptr;    // best-case P_alpha (AAO_PRECOND_EXACT_DCT)
  aao::SpPlan* sp = nullptr;      // P_SP (AAO_PRECOND_SP)
  std::vector<cudaGraphExec_t> step_graphs;
  cudaStream_t gstream = nullptr;  // non-blocking stream the graphs are captured on and run on
  cudaEvent_t gevent = nullptr;    // orders gstream after the caller's stream
  std::vector<long long> step_graph_launches;
  std::vector<char> step_graph_tma;
  double *V = nullptr, *Z = nullptr;                   // Krylov bases, (m+1) and m vectors of L
  double* sc = nullptr;                                // small scalars, ScLayout
  unsigned* counter = nullptr;                         // last-block ticket of the MGS steps (0 at rest)
  unsigned* tma_fault = nullptr;                       // the TMA kernel's fault word (device, 0 at rest)
  double* partials = nullptr;                          // reduction partials
  int64_t part_cap = 0;
  double *stage_a = nullptr, *stage_b = nullptr;       // staging for host pointers (L each)
  double* pinned = nullptr;                            // pinned host scalars

  std::vector<aao::StepArgs<float>> steps32;    // index k = 0 .. p-1 (0 holds 1/theta for p = 1)
  std::vector<aao::StepArgs<double>> steps64;
  aao::DftArgs<float> dft32{};
  aao::DftArgs<double> dft64{};
  aao::IdftArgs<float> idft32{};
  aao::IdftArgs<double> idft64{};

  aao_stats stats{};
  std::string err;

  // event timing of kernel classes (aao_profile_*)
  struct Pending {
    int cls;
    int e0;
    int launches;
    double bytes;
  };
  bool prof = false;
  std::vector<cudaEvent_t> events;
  std::vector<Pending> pending;
  aao_profile profacc{};
};

// Message of the last failed create (handles and batches), shared by the entry points.
extern std::string g_create_error;

namespace aao {
// Record a formatted message on h (or as the create error when h is NULL); returns code.
int handle_fail(aao_ctx* h, int code, const char* fmt, ...);
// Device memory of the current device (or managed memory): used in place at the boundary.
bool is_device_ptr(const void* p);
// Device memory of another GPU: refused at the boundary.
bool is_other_device_ptr(const void* p);
// z = P^{-1} r on the handle's stream (r scaled by *rscale when rscale is not NULL).
int handle_precond(aao_ctx* h, const double* r, const double* rscale, double* z);
// Drop the captured Arnoldi-step graphs (after a change of kernels or tables).
void handle_reset_graphs(aao_ctx* h);
// Read and clear the persistent TMA kernel's fault flag (synchronises the stream).
int handle_check_tma(aao_ctx* h);
// The staging buffers for host pointers (ell N doubles each), allocated on first use.
int handle_ensure_stage(aao_ctx* h);
// The fused-sweep kernel the handle runs (AAO_STEP_AUTO resolved).
inline int effective_step_kernel(const aao_ctx* h) {
  return h->step_kernel == AAO_STEP_AUTO ? h->auto_kind : h->step_kernel;
}
// Warp-strip configurations used without a cache entry (tune.cu): the fused sweep (S = 4) and
// its two-step final launch (S = 2).
StreamConfig default_stream_config(const GridDesc& g, int ell);
StreamConfig default_tail_config(const GridDesc& g, int ell);
// Configuration (S, D, NW) with the smallest segment height that puts all units of one launch
// into `waves` rounds over the device's warps (skew 1: a height for the skewed schedule).
StreamConfig wave_stream_config(const GridDesc& g, int ell, int S, int D, int NW, int waves, int skew);
// Apply the tune cache's entry for h, if a cache is configured and holds one (tune.cu).
void apply_tune_cache(aao_ctx* h);
// Release the views of aao_solve_multi (multi.cu).
void multi_destroy(aao_multi* m);
}  // namespace aao
