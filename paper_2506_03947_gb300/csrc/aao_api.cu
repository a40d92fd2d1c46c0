// Host side of libaao: the C ABI declared in include/aao.h.
//
// aao_create builds the scalar set-up of the method on the host in FP64
// (shifts lambda_j and scalings of Section 2.2, Chebyshev coefficients for the
// segment of Lemma 2) and everything O(N) on the device.  The solve loop is
// driven from the host: per Arnoldi step it launches the preconditioner
// kernels, the script-A matvec and the Gram-Schmidt kernels, and reads back
// one 16-byte residual estimate to decide whether to stop.
#include "aao.h"
#include "aao_internal.cuh"
#include "batch.cuh"
#include "host_tables.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <type_traits>
#include <vector>

namespace aao {
long long launch_count();
void count_launch_add(long long n);
cudaError_t launch_build_coeffs(const GridDesc& g, const double* kx, const double* ky, const double* kz,
                                double* cx, double* cy, double* cz, float* fx, float* fy, float* fz,
                                double* partials, int* bad, double* smax_out, cudaStream_t s);
int build_coeff_blocks(int64_t N);
}  // namespace aao

using aao::DftArgs;
using aao::GridDesc;
using aao::IdftArgs;
using aao::ScLayout;
using aao::StepArgs;

#include "aao_ctx.h"

std::string g_create_error;

namespace {

int fail(aao_ctx* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

#define AAO_CK(h, call)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail((h), e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
  } while (0)

// Pointer kinds at the boundary: device memory of the current device (or managed memory) is
// used in place; host memory is staged.  Another GPU's memory is neither: the kernels run on the
// current device and cannot reach it without peer access, so it is refused.
enum PtrKind { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };

PtrKind ptr_kind(const void* p) {
  if (!p) return kPtrHost;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPtrHost;
  }
  if (a.type == cudaMemoryTypeManaged) return kPtrDevice;
  if (a.type != cudaMemoryTypeDevice) return kPtrHost;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return kPtrOtherDevice;
  }
  return a.device == dev ? kPtrDevice : kPtrOtherDevice;
}

bool is_device_ptr(const void* p) { return ptr_kind(p) == kPtrDevice; }

bool is_other_device_ptr(const void* p) { return ptr_kind(p) == kPtrOtherDevice; }

// ---- profiling: events around timed launches -------------------------------

int prof_begin(aao_ctx* h, int cls, double bytes, int launches = 1) {
  if (!h->prof) return -1;
  const int idx = (int)h->pending.size();
  const int e0 = 2 * idx;
  while ((int)h->events.size() < e0 + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->events.push_back(e);
  }
  if (cudaEventRecord(h->events[e0], h->stream) != cudaSuccess) return -1;
  h->pending.push_back({cls, e0, launches, bytes});
  return idx;
}

void prof_end(aao_ctx* h, int idx) {
  if (idx < 0) return;
  cudaEventRecord(h->events[h->pending[idx].e0 + 1], h->stream);
}

// The stream must be synchronised: every recorded pair has completed.
void prof_resolve(aao_ctx* h) {
  for (const auto& p : h->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->events[p.e0], h->events[p.e0 + 1]) == cudaSuccess) {
      h->profacc.ms[p.cls] += ms;
      h->profacc.launches[p.cls] += p.launches;
      h->profacc.bytes[p.cls] += p.bytes;
    }
  }
  h->pending.clear();
}

// Chebyshev and transform tables for the current p (host FP64, Section 2.2 and
// Lemma 2; host_tables.h), with their FP32 copies.
void reset_graphs(aao_ctx* h);

void build_tables(aao_ctx* h) {
  reset_graphs(h);
  const int p = std::max(h->p, 1);
  aao::ChebTables tb;
  aao::cheb_tables_init(tb, h->ell, h->alpha, h->mu_min, h->mu_max);
  h->steps32.assign(p, StepArgs<float>{});
  h->steps64.assign(p, StepArgs<double>{});
  for (int k = 0; k < p; ++k) {
    aao::cheb_tables_step(tb, k, h->nc2 ? h->palloc : nullptr, h->steps64[k]);
    h->steps32[k] = aao::narrow_step(h->steps64[k]);
  }
  aao::transform_tables(h->ell, h->alpha, h->dft64, h->idft64);
  aao::narrow_transforms(h->dft64, h->idft64, h->dft32, h->idft32);
}

template <typename T>
int precond_impl(aao_ctx* h, const double* r, const double* rscale, double* z, const std::vector<StepArgs<T>>& st,
                 const DftArgs<T>& da, const IdftArgs<T>& ia, const T* cx, const T* cy, const T* cz) {
  const int p = h->p;
  cudaStream_t s = h->stream;
  T* bhat = (T*)h->bhat;
  T* xa = (T*)h->xa;
  T* xb = (T*)h->xb;
  const double N = (double)h->N, ell = (double)h->ell, Ts = (double)sizeof(T), dim = (double)h->dim;
  if (p == 1) {
    const int pi = prof_begin(h, AAO_PROF_STEP_LAST, N * 16.0 * ell);
    AAO_CK(h, aao::launch_direct<T>(h->g, h->dim, h->ell, r, rscale, z, da, st[0], ia, s));
    prof_end(h, pi);
    return AAO_OK;
  }
  int pi = prof_begin(h, AAO_PROF_DFT, N * (8.0 * ell + ell * Ts));
  AAO_CK(h, aao::launch_dft<T>(h->g, h->dim, h->ell, r, rscale, bhat, da, s));
  prof_end(h, pi);
  // algorithmic bytes of one step: x_k (or bhat) read, bhat read when x_k is a
  // buffer, x_{k-1} read when buffered, coefficients, and x_{k+1} or z written
  auto step_bytes = [&](int ksrc, int psrc, bool last) {
    double b = ell * Ts + (ksrc == 1 ? ell * Ts : 0.0) + (psrc == 2 ? ell * Ts : 0.0) + dim * Ts;
    b += last ? 8.0 * ell : ell * Ts;
    return N * b;
  };
  auto step_class = [](int ksrc, int psrc, bool last) {
    if (last) return AAO_PROF_STEP_LAST;
    if (ksrc == 0) return AAO_PROF_STEP_FIRST;
    if (psrc == 1) return AAO_PROF_STEP_SECOND;
    return AAO_PROF_STEP_MID;
  };
  // In FP32 with an even cell count the last step runs as a middle step (x_p into the buffer of
  // x_{p-2}) and the inverse transform is a launch of its own (k_idft_planes): the fused last
  // step holds the ell time blocks of z in registers beside the stencil and runs far below the
  // bandwidth of the two launches that replace it.
  const bool split = std::is_same<T, float>::value && h->N % 2 == 0 && (reinterpret_cast<uintptr_t>(z) & 15) == 0;
  const int fused_last = split ? p : p - 1;  // the step that writes z itself (none when split)
  // k = 1: x_1 = bhat/theta, x_0 = 0 -> x_2 in xa (or z)
  pi = prof_begin(h, step_class(0, 0, fused_last == 1), step_bytes(0, 0, fused_last == 1));
  AAO_CK(h, aao::launch_step<T>(h->g, h->dim, h->ell, 0, 0, fused_last == 1, cx, cy, cz, bhat, nullptr, xa, z, st[1],
                                ia, s));
  prof_end(h, pi);
  T* xp = xa;  // x_p when split
  if (p >= 3) {
    // k = 2: x_2 from xa, x_1 = bhat/theta -> x_3 in xb (or z)
    pi = prof_begin(h, step_class(1, 1, fused_last == 2), step_bytes(1, 1, fused_last == 2));
    AAO_CK(h, aao::launch_step<T>(h->g, h->dim, h->ell, 1, 1, fused_last == 2, cx, cy, cz, bhat, xa, xb, z, st[2], ia,
                                  s));
    prof_end(h, pi);
    xp = xb;
  }
  for (int k = 3; k <= p - 1; ++k) {
    // x_k in `cur`, x_{k-1} in `prev`; x_{k+1} overwrites x_{k-1} (or goes to z)
    T* cur = (k % 2 == 1) ? xb : xa;
    T* prev = (k % 2 == 1) ? xa : xb;
    const bool last = (k == fused_last);
    pi = prof_begin(h, step_class(1, 2, last), step_bytes(1, 2, last));
    AAO_CK(h, aao::launch_step<T>(h->g, h->dim, h->ell, 1, 2, last, cx, cy, cz, bhat, cur, prev, z, st[k], ia, s));
    prof_end(h, pi);
    xp = prev;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (split) {
      // z = Gamma^{-1} U x_p
      pi = prof_begin(h, AAO_PROF_STEP_LAST, N * (4.0 * ell + 8.0 * ell));
      AAO_CK(h, aao::launch_idft_planes(h->g, h->ell, xp, z, ia, s));
      prof_end(h, pi);
    }
  }
  return AAO_OK;
}

// Mixed 2D schedule with fused steps: the transform and k = 1 in one launch, then
//  * warp strips (AAO_STEP_STREAM): S-step launches up to and including the last step, whose
//    output x_p goes through a separate inverse transform (see the branch below);
//  * TMA and tile kernels: four-step launches while all four come before the last step, pairs,
//    at most one single step, then the last step fused with the inverse transform.
// Four field buffers rotate so that a launch never writes a buffer it (or a neighbouring tile)
// reads.
int precond_pairs(aao_ctx* h, const double* r, const double* rscale, double* z) {
  const int p = h->p;
  cudaStream_t s = h->stream;
  const auto& st = h->steps32;
  const auto& ia = h->idft32;
  float* bhat = (float*)h->bhat;
  float* X[4] = {(float*)h->xa, (float*)h->xb, (float*)h->xc, (float*)h->xd};
  const float *cx = h->cx32, *cy = h->cy32, *cz = h->cz32;
  const double N = (double)h->N, ell = (double)h->ell;
  int pi = -1;
  if (p == 2) {
    pi = prof_begin(h, AAO_PROF_DFT, N * (8.0 * ell + 4.0 * ell));
    AAO_CK(h, aao::launch_dft<float>(h->g, h->dim, h->ell, r, rscale, bhat, h->dft32, s));
    prof_end(h, pi);
    pi = prof_begin(h, AAO_PROF_STEP_LAST, N * (4.0 * ell + 8.0 + 8.0 * ell));
    AAO_CK(h, aao::launch_step<float>(h->g, h->dim, h->ell, 0, 0, true, cx, cy, cz, bhat, nullptr, X[0], z, st[1], ia,
                                      s));
    prof_end(h, pi);
    return AAO_OK;
  }
  // the transform and step 1 in one launch: r read, bhat and x_2 (field 0) written
  pi = prof_begin(h, AAO_PROF_STEP_FIRST, N * (16.0 * ell + 8.0));
  AAO_CK(h, aao::launch_dft_first(h->g, h->ell, r, rscale, bhat, X[0], cx, cy, h->dft32, st[1], s));
  prof_end(h, pi);
  int cur = 0, prev = -1;  // prev = -1: x_{k-1} = x_1 = bhat/theta (not stored)
  int k = 2;
  const int kind = aao::effective_step_kernel(h);
  if (kind == AAO_STEP_STREAM && p - 2 >= 2) {
    // Steps 2 .. p-1 by warp-strip launches (S steps each, streamed along y): one single step
    // first when their count is odd, launches of the handle's S, one two-step launch for a
    // remainder of two.  The final launch keeps x_p alone and the inverse transform reads it.
    int R = p - 2;
    if (R % 2 == 1) {
      const int dst = 1;  // x_3 (x_2 is in field 0, x_1 = bhat/theta)
      pi = prof_begin(h, AAO_PROF_STEP_SECOND, N * (3.0 * 4.0 * ell + 8.0));
      AAO_CK(h, aao::launch_step<float>(h->g, h->dim, h->ell, 1, 1, false, cx, cy, cz, bhat, X[cur], X[dst], z, st[k],
                                        ia, s));
      prof_end(h, pi);
      prev = cur;
      cur = dst;
      ++k;
      --R;
    }
    // The warp-strip launches run back to back: one event span over all of them, whose
    // average is the per-launch time (events between them would add gaps of their own).
    const int span = prof_begin(h, AAO_PROF_STEP_QUAD, 0.0, 0);
    while (R > 0) {
      const bool four = h->scfg.S == 4 && R >= 4;
      const aao::StreamConfig& c = (four || h->scfg.S == 2) ? h->scfg : h->tail;
      const int S = c.S;
      const bool fin = (R == S);
      int o[2], n = 0;
      for (int b = 0; b < 4 && n < 2; ++b)
        if (b != cur && b != prev) o[n++] = b;
      aao::FuseSteps fs;
      for (int q = 0; q < S; ++q) fs.s[q] = st[k + q];
      const double sets = (prev < 0 ? 2.0 : 3.0) + (fin ? 1.0 : 2.0);
      if (span >= 0) {
        h->pending[span].bytes += N * (sets * 4.0 * ell + 8.0);
        h->pending[span].launches += 1;
      }
      AAO_CK(h, aao::launch_stream(h->g, h->ell, prev < 0 ? 1 : 2, c, cx, cy, bhat, X[cur],
                                   prev < 0 ? nullptr : X[prev], fin ? nullptr : X[o[0]], fin ? X[o[0]] : X[o[1]],
                                   fs, s));
      if (fin) {
        cur = o[0];
      } else {
        prev = o[0];
        cur = o[1];
      }
      k += S;
      R -= S;
    }
    prof_end(h, span);
    // z = Gamma^{-1} U x_p
    pi = prof_begin(h, AAO_PROF_STEP_LAST, N * (4.0 * ell + 8.0 * ell));
    AAO_CK(h, aao::launch_idft_planes(h->g, h->ell, X[cur], z, ia, s));
    prof_end(h, pi);
    return AAO_OK;
  }
  while (k + 3 <= p - 2 && kind != AAO_STEP_STREAM) {
    int o[2], n = 0;
    for (int b = 0; b < 4 && n < 2; ++b)
      if (b != cur && b != prev) o[n++] = b;
    aao::QuadSteps qs;
    for (int q = 0; q < 4; ++q) qs.s[q] = st[k + q];
    pi = prof_begin(h, AAO_PROF_STEP_QUAD, N * ((prev < 0 ? 4.0 : 5.0) * 4.0 * ell + 8.0));
    if (h->tma && kind == AAO_STEP_TMA) {
      AAO_CK(h, aao::launch_quad_tma(h->g, h->ell, prev < 0 ? 1 : 2, h->fmap[5], h->fmap[6], h->fmap[cur],
                                     h->fmap[prev < 0 ? cur : prev], h->fmap[4], X[o[0]], X[o[1]], qs,
                                     h->wait_limit, h->tma_fault, s));
      h->tma_used = true;
    } else {
      AAO_CK(h, aao::launch_quad(h->g, h->ell, prev < 0 ? 1 : 2, cx, cy, bhat, X[cur], prev < 0 ? nullptr : X[prev],
                                 X[o[0]], X[o[1]], qs, s));
    }
    prof_end(h, pi);
    prev = o[0];
    cur = o[1];
    k += 4;
  }
  while (k + 1 <= p - 2) {
    int o[2], n = 0;
    for (int b = 0; b < 4 && n < 2; ++b)
      if (b != cur && b != prev) o[n++] = b;
    pi = prof_begin(h, AAO_PROF_STEP_PAIR, N * ((prev < 0 ? 4.0 : 5.0) * 4.0 * ell + 8.0));
    AAO_CK(h, aao::launch_pair(h->g, h->ell, prev < 0 ? 1 : 2, cx, cy, bhat, X[cur], prev < 0 ? nullptr : X[prev],
                               X[o[0]], X[o[1]], st[k], st[k + 1], s));
    prof_end(h, pi);
    prev = o[0];
    cur = o[1];
    k += 2;
  }
  if (k <= p - 2) {
    int dst = prev;
    if (dst < 0)
      for (int b = 0; b < 4; ++b)
        if (b != cur) {
          dst = b;
          break;
        }
    const int psrc = prev < 0 ? 1 : 2;
    pi = prof_begin(h, psrc == 1 ? AAO_PROF_STEP_SECOND : AAO_PROF_STEP_MID,
                    N * ((psrc == 1 ? 3.0 : 4.0) * 4.0 * ell + 8.0));
    AAO_CK(h, aao::launch_step<float>(h->g, h->dim, h->ell, 1, psrc, false, cx, cy, cz, bhat, X[cur], X[dst], z, st[k],
                                      ia, s));
    prof_end(h, pi);
    prev = cur;
    cur = dst;
    k += 1;
  }
  const int psrc = prev < 0 ? 1 : 2;
  pi = prof_begin(h, AAO_PROF_STEP_LAST, N * ((psrc == 1 ? 2.0 : 3.0) * 4.0 * ell + 8.0 + 8.0 * ell));
  AAO_CK(h, aao::launch_step<float>(h->g, h->dim, h->ell, 1, psrc, true, cx, cy, cz, bhat, X[cur],
                                    prev < 0 ? X[cur] : X[prev], z, st[k], ia, s));
  prof_end(h, pi);
  return AAO_OK;
}

// Read (and clear) the device flag the persistent four-step kernel raises
// when one of its bounded TMA waits expires; synchronises the stream.
int check_tma(aao_ctx* h) {
  if (!h->tma_used) return AAO_OK;
  h->tma_used = false;
  unsigned flag = 0;
  AAO_CK(h, aao::quad_tma_fault(h->tma_fault, &flag, h->stream));
  if (flag & 2u) return fail(h, AAO_ECUDA, "four-step TMA kernel: shared-memory base not 128-byte aligned");
  if (flag) return fail(h, AAO_ETIMEOUT, "four-step TMA kernel: a bounded TMA wait expired");
  return AAO_OK;
}

// Best-case P_alpha^{-1} (constant diffusivities, FP64): time DFT, then dct_precond.
int precond_dct(aao_ctx* h, const double* r, const double* rscale, double* z) {
  AAO_CK(h, aao::launch_dft<double>(h->g, h->dim, h->ell, r, rscale, (double*)h->bhat, h->dft64, h->stream));
  aao::DctShifts sh{};
  for (int m = 0; m <= h->ell / 2; ++m) {
    sh.lam_re[m] = h->steps64[0].lam_re[m];
    sh.lam_im[m] = h->steps64[0].lam_im[m];
  }
  AAO_CK(h, aao::dct_precond(h->dct, h->g, h->ell, (double*)h->bhat, z, sh, h->idft64, h->stream));
  return AAO_OK;
}

// P_SP^{-1} (Section 4): time DFT, then the fixed-iteration real Krylov solves (sp_precond).
int precond_sp(aao_ctx* h, const double* r, const double* rscale, double* z) {
  AAO_CK(h, aao::launch_dft<double>(h->g, h->dim, h->ell, r, rscale, (double*)h->bhat, h->dft64, h->stream));
  aao::DctShifts sh{};
  for (int m = 0; m <= h->ell / 2; ++m) {
    sh.lam_re[m] = h->steps64[0].lam_re[m];
    sh.lam_im[m] = h->steps64[0].lam_im[m];
  }
  AAO_CK(h, aao::sp_precond(h->sp, h->g, h->ell, h->p, (double*)h->bhat, (double*)h->xa, z, sh, h->idft64,
                            h->stream));
  return AAO_OK;
}

int precond(aao_ctx* h, const double* r, const double* rscale, double* z) {
  if (h->pmode == AAO_PRECOND_EXACT_DCT) return precond_dct(h, r, rscale, z);
  if (h->pmode == AAO_PRECOND_SP) return precond_sp(h, r, rscale, z);
  if (h->pairs && h->p >= 3) return precond_pairs(h, r, rscale, z);
  if (h->prec == AAO_MIXED)
    return precond_impl<float>(h, r, rscale, z, h->steps32, h->dft32, h->idft32, h->cx32, h->cy32, h->cz32);
  return precond_impl<double>(h, r, rscale, z, h->steps64, h->dft64, h->idft64, h->cx64, h->cy64, h->cz64);
}

int matvec(aao_ctx* h, const double* x, const double* b, double* y, int* nblocks) {
  const double bytes = (double)h->N * (16.0 * h->ell + 8.0 * h->dim + (b ? 8.0 * h->ell : 0.0));
  const int pi = prof_begin(h, AAO_PROF_MATVEC, bytes);
  AAO_CK(h, aao::launch_aao_matvec(h->g, h->dim, h->ell, h->cx64, h->cy64, h->cz64, x, b, y, h->partials, nblocks,
                                   h->stream));
  prof_end(h, pi);
  return AAO_OK;
}

int read_scalars(aao_ctx* h, int offset, int count, double* out) {
  AAO_CK(h, cudaMemcpyAsync(h->pinned, h->sc + offset, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < count; ++i) out[i] = h->pinned[i];
  prof_resolve(h);
  return AAO_OK;
}

int ensure_stage(aao_ctx* h) {
  if (!h->stage_a) AAO_CK(h, cudaMalloc(&h->stage_a, sizeof(double) * h->L));
  if (!h->stage_b) AAO_CK(h, cudaMalloc(&h->stage_b, sizeof(double) * h->L));
  return AAO_OK;
}

// explicit ||b - script-A x||^2 into sc[nrm2] with r written to `r`; returns its value.
int residual(aao_ctx* h, const double* b, const double* x, double* r, double* rn2) {
  int nb = 0;
  int rc = matvec(h, x, b, r, &nb);
  if (rc) return rc;
  const ScLayout Lsc{h->m};
  AAO_CK(h, aao::launch_reduce(h->partials, 1, nb, h->sc + Lsc.nrm2(), 0, h->stream));
  return read_scalars(h, Lsc.nrm2(), 1, rn2);
}

// Orthogonalise w = V_{j+1} against V_0 .. V_j (Arnoldi step j): the coefficients
// go to h1 (and h2 for the second classical pass), ||w||^2 of the result to nrm2.
int orthogonalize(aao_ctx* h, int j, double* w) {
  const ScLayout Lsc{h->m};
  const int64_t L = h->L;
  cudaStream_t s = h->stream;
  const int nv = j + 1;
  const int nb = aao::reduction_blocks(L);
  double* normpart = h->partials + (int64_t)(h->m + 1) * nb;
  if (h->orth == AAO_ORTH_MGS) {
    // modified Gram-Schmidt, one fused kernel per basis vector: step i subtracts the
    // projection on V_{i-1} and forms V_i . w; its last block writes h_i.  Bytes: the first
    // step reads V_0 and w, the middle ones read V_{i-1}, V_i, w and write w, the last
    // reads V_j and w and writes w (and forms ||w||^2).
    const double bytes = 8.0 * (double)L * (2.0 + 4.0 * (nv - 1) + 3.0);
    const int pi = prof_begin(h, AAO_PROF_ORTH, bytes, nv + 1);
    const double* vs = h->sc + Lsc.vscale(0);
    AAO_CK(h, aao::launch_mgs_step(h->V, L, -1, 0, vs, nullptr, h->sc + Lsc.h1(0), w, L, h->partials, h->counter,
                                   s));
    for (int i = 1; i < nv; ++i)
      AAO_CK(h, aao::launch_mgs_step(h->V, L, i - 1, i, vs, h->sc + Lsc.h1(i - 1), h->sc + Lsc.h1(i), w, L,
                                     h->partials, h->counter, s));
    AAO_CK(h, aao::launch_mgs_step(h->V, L, nv - 1, -1, vs, h->sc + Lsc.h1(nv - 1), h->sc + Lsc.nrm2(), w, L,
                                   h->partials, h->counter, s));
    prof_end(h, pi);
    return AAO_OK;
  }
  // classical Gram-Schmidt (once, or twice for CGS2): algorithmic bytes = each V_i read
  // once per pass plus w
  const int ndot = (nv + 7) / 8;
  const double dot_bytes = 8.0 * (double)L * (nv + ndot);
  const double upd_bytes = 8.0 * (double)L * (nv + 2);
  const bool reorth = h->orth == AAO_ORTH_CGS2;
  const int passes = reorth ? 2 : 1;
  const int pi = prof_begin(h, AAO_PROF_ORTH, passes * (dot_bytes + upd_bytes), passes * (ndot + 2) + 1);
  AAO_CK(h, aao::launch_multidot(h->V, L, nv, h->sc + Lsc.vscale(0), w, L, h->partials, s));
  AAO_CK(h, aao::launch_reduce(h->partials, nv, nb, h->sc + Lsc.h1(0), 0, s));
  if (reorth) {
    AAO_CK(h, aao::launch_orth_update(h->V, L, nv, h->sc + Lsc.h1(0), h->sc + Lsc.vscale(0), w, L, nullptr, s));
    AAO_CK(h, aao::launch_multidot(h->V, L, nv, h->sc + Lsc.vscale(0), w, L, h->partials, s));
    AAO_CK(h, aao::launch_reduce(h->partials, nv, nb, h->sc + Lsc.h2(0), 0, s));
    AAO_CK(h, aao::launch_orth_update(h->V, L, nv, h->sc + Lsc.h2(0), h->sc + Lsc.vscale(0), w, L, normpart, s));
  } else {
    AAO_CK(h, cudaMemsetAsync(h->sc + Lsc.h2(0), 0, sizeof(double) * nv, s));
    AAO_CK(h, aao::launch_orth_update(h->V, L, nv, h->sc + Lsc.h1(0), h->sc + Lsc.vscale(0), w, L, normpart, s));
  }
  AAO_CK(h, aao::launch_reduce(normpart, 1, nb, h->sc + Lsc.nrm2(), 0, s));
  prof_end(h, pi);
  return AAO_OK;
}

// x_zero: x holds x_0 = 0 on entry, so the first residual is b itself (no script-A product).
void reset_graphs(aao_ctx* h) {
  for (cudaGraphExec_t g : h->step_graphs)
    if (g) cudaGraphExecDestroy(g);
  h->step_graphs.clear();
  h->step_graph_launches.clear();
  h->step_graph_tma.clear();
}

// Arnoldi step j in stream order; ends with the 16-byte copy of (estimate, h_{j+1,j}) to
// pinned memory.  Givens reads ||b|| from sc[bnorm] (set at the start of the solve).
int arnoldi_step_launches(aao_ctx* h, int j) {
  const ScLayout Lsc{h->m};
  const int64_t L = h->L;
  double* Vj = h->V + (int64_t)j * L;
  double* Zj = h->Z + (int64_t)j * L;
  double* w = h->V + (int64_t)(j + 1) * L;
  int rc = precond(h, Vj, h->sc + Lsc.vscale(j), Zj);
  if (rc) return rc;
  rc = matvec(h, Zj, nullptr, w, nullptr);
  if (rc) return rc;
  rc = orthogonalize(h, j, w);
  if (rc) return rc;
  AAO_CK(h, aao::launch_givens(h->sc, j, h->m, -1.0, h->stream));
  AAO_CK(h, cudaMemcpyAsync(h->pinned, h->sc + Lsc.est(), sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
  return AAO_OK;
}

// Run Arnoldi step j (through its CUDA graph unless the event profiler is on) and read back
// eh = (residual estimate, h_{j+1,j}).
int arnoldi_step(aao_ctx* h, int j, double* eh) {
  if (h->prof || h->pmode != AAO_PRECOND_NC) {
    const int rc = arnoldi_step_launches(h, j);
    if (rc) return rc;
  } else {
    // The caller's stream may be the legacy default stream, which cannot be captured: the
    // step is captured on, and replayed on, the handle's own stream, ordered after the
    // caller's stream by an event (the host synchronises after every step).
    if (!h->gstream) AAO_CK(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    if (!h->gevent) AAO_CK(h, cudaEventCreateWithFlags(&h->gevent, cudaEventDisableTiming));
    AAO_CK(h, cudaEventRecord(h->gevent, h->stream));
    AAO_CK(h, cudaStreamWaitEvent(h->gstream, h->gevent, 0));
    if ((int)h->step_graphs.size() <= j) {
      h->step_graphs.resize(j + 1, nullptr);
      h->step_graph_launches.resize(j + 1, 0);
      h->step_graph_tma.resize(j + 1, 0);
    }
    if (!h->step_graphs[j]) {
      const long long c0 = aao::launch_count();
      const bool tma0 = h->tma_used;
      h->tma_used = false;
      AAO_CK(h, cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
      cudaStream_t user = h->stream;
      h->stream = h->gstream;  // the launchers use the handle's stream
      const int rc = arnoldi_step_launches(h, j);
      h->stream = user;
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(h->gstream, &graph);
      const bool tma_in = h->tma_used;
      h->tma_used = tma0;
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      AAO_CK(h, ec);
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      AAO_CK(h, ei);
      h->step_graphs[j] = exec;
      h->step_graph_launches[j] = aao::launch_count() - c0;
      h->step_graph_tma[j] = tma_in ? 1 : 0;
      aao::count_launch_add(-h->step_graph_launches[j]);  // captured, not run: counted at each replay
    }
    AAO_CK(h, cudaGraphLaunch(h->step_graphs[j], h->gstream));
    aao::count_launch_add(h->step_graph_launches[j]);
    if (h->step_graph_tma[j]) h->tma_used = true;
    AAO_CK(h, cudaStreamSynchronize(h->gstream));
  }
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  eh[0] = h->pinned[0];
  eh[1] = h->pinned[1];
  prof_resolve(h);
  return AAO_OK;
}

int solve_impl(aao_ctx* h, const double* b, double* x, double tol, int max_outer, int fixed, bool x_zero) {
  const ScLayout Lsc{h->m};
  const int64_t L = h->L;
  cudaStream_t s = h->stream;
  aao_stats& st = h->stats;
  std::memset(&st, 0, sizeof(st));
  st.mu_min = h->mu_min;
  st.mu_max = h->mu_max;
  int64_t inner_total = (int64_t)h->ell * h->p;  // A-matvecs of one preconditioner apply (Table 1)
  if (h->nc2) {
    inner_total = 0;
    for (int j = 0; j < h->ell; ++j) {
      const int mm = (j <= h->ell / 2) ? j : h->ell - j;  // conjugate shifts share a budget
      inner_total += h->palloc[mm];
    }
  }
  if (h->pmode == AAO_PRECOND_EXACT_DCT) inner_total = 0;  // no products with A inside the exact P_alpha
  const int64_t per_outer = inner_total + h->ell;

  // ||b||
  AAO_CK(h, aao::launch_norm2_partials(b, L, h->partials, s));
  AAO_CK(h, aao::launch_reduce(h->partials, 1, aao::reduction_blocks(L), h->sc + Lsc.nrm2(), 0, s));
  double bn2 = 0.0;
  int rc = read_scalars(h, Lsc.nrm2(), 1, &bn2);
  if (rc) return rc;
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) return fail(h, AAO_ENUMERIC, "||b|| is not finite");
  if (bnorm == 0.0) {
    AAO_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * L, s));
    AAO_CK(h, cudaStreamSynchronize(s));
    st.converged = 1;
    return AAO_OK;
  }
  h->pinned[2] = bnorm;  // for the Givens steps (the stream is idle: read_scalars synchronised)
  AAO_CK(h, cudaMemcpyAsync(h->sc + Lsc.bnorm(), h->pinned + 2, sizeof(double), cudaMemcpyHostToDevice, s));
  int total = 0;
  const int m = fixed ? fixed : h->m;
  while (true) {
    double rn2 = 0.0;
    if (x_zero && st.cycles == 0) {
      // r_0 = b; sc[nrm2] still holds ||b||^2 from above for the cycle initialisation
      AAO_CK(h, cudaMemcpyAsync(h->V, b, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
      rn2 = bn2;
    } else {
      rc = residual(h, b, x, h->V, &rn2);
      if (rc) return rc;
      st.a_matvecs += h->ell;
    }
    const double rel = std::sqrt(rn2) / bnorm;
    st.resid_explicit = rel;
    if (!std::isfinite(rel)) return fail(h, AAO_ENUMERIC, "residual is not finite");
    if (fixed && st.cycles > 0) {
      st.converged = rel < tol;
      return AAO_OK;
    }
    if (!fixed && rel < tol) {
      st.converged = 1;
      return AAO_OK;
    }
    if (total >= max_outer) return fail(h, AAO_ENOTCONV, "no convergence in %d outer iterations (rel. residual %.3e)",
                                        total, rel);
    AAO_CK(h, aao::launch_cycle_init(h->sc, h->m, s));
    st.cycles++;
    const double beta = std::sqrt(rn2);
    int k = 0;
    for (int j = 0; j < m && total < max_outer; ++j) {
      double eh[2];
      rc = arnoldi_step(h, j, eh);
      if (rc) return rc;
      k = j + 1;
      total++;
      st.outer_its = total;
      st.a_matvecs += per_outer;
      st.resid_est = eh[0];
      if (st.n_hist < AAO_MAX_HIST) st.hist[st.n_hist++] = eh[0];
      if (!std::isfinite(eh[0]) || !std::isfinite(eh[1]))
        return fail(h, AAO_ENUMERIC, "non-finite value in Arnoldi step %d", total);
      const bool breakdown = eh[1] <= 1e-14 * beta;
      if (breakdown) break;
      if (!fixed && eh[0] < tol) break;
    }
    AAO_CK(h, aao::launch_backsolve(h->sc, k, h->m, s));
    AAO_CK(h, aao::launch_xupdate(h->Z, L, k, h->sc + Lsc.y(0), x, L, s));
  }
}

// Outer Chebyshev semi-iteration on P^{-1} script-A x = P^{-1} b over [l_min, l_max]
// (Section 5 with Corollary 1's interval), residual updated as r -= script-A d.
int solve_ci_impl(aao_ctx* h, const double* b, double* x, double tol, int max_its, double l_min, double l_max,
                  int fixed) {
  const ScLayout Lsc{h->m};
  const int64_t L = h->L;
  cudaStream_t s = h->stream;
  aao_stats& st = h->stats;
  std::memset(&st, 0, sizeof(st));
  st.mu_min = h->mu_min;
  st.mu_max = h->mu_max;
  int64_t inner_total = (int64_t)h->ell * h->p;
  if (h->nc2) {
    inner_total = 0;
    for (int j = 0; j < h->ell; ++j) inner_total += h->palloc[(j <= h->ell / 2) ? j : h->ell - j];
  }
  AAO_CK(h, aao::launch_norm2_partials(b, L, h->partials, s));
  AAO_CK(h, aao::launch_reduce(h->partials, 1, aao::reduction_blocks(L), h->sc + Lsc.nrm2(), 0, s));
  double bn2 = 0.0;
  int rc = read_scalars(h, Lsc.nrm2(), 1, &bn2);
  if (rc) return rc;
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) return fail(h, AAO_ENUMERIC, "||b|| is not finite");
  if (bnorm == 0.0) {
    AAO_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * L, s));
    AAO_CK(h, cudaStreamSynchronize(s));
    st.converged = 1;
    return AAO_OK;
  }
  double* r = h->V;
  double* r2 = h->V + L;
  double* z = h->Z;
  double* d = h->Z + L;
  const double theta = 0.5 * (l_max + l_min), delta = 0.5 * (l_max - l_min);
  const double sigma1 = delta > 0.0 ? theta / delta : 0.0;
  double rho = delta > 0.0 ? 1.0 / sigma1 : 0.0;
  double rn2 = 0.0;
  rc = residual(h, b, x, r, &rn2);  // r = b - script-A x
  if (rc) return rc;
  st.a_matvecs += h->ell;
  rc = precond(h, r, nullptr, z);
  if (rc) return rc;
  double c1 = 0.0, c2 = 1.0 / theta;
  const int nmax = fixed ? fixed : max_its;
  for (int it = 0; it < nmax; ++it) {
    AAO_CK(h, aao::launch_ci_update(d, z, x, c1, c2, L, s));  // d_k, x_{k+1} = x_k + d_k
    rc = residual(h, r, d, r2, &rn2);                           // r_{k+1} = r_k - script-A d_k
    if (rc) return rc;
    std::swap(r, r2);
    st.outer_its = it + 1;
    st.a_matvecs += h->ell + inner_total;
    const double rel = std::sqrt(rn2) / bnorm;
    st.resid_est = rel;
    if (st.n_hist < AAO_MAX_HIST) st.hist[st.n_hist++] = rel;
    if (!std::isfinite(rel)) return fail(h, AAO_ENUMERIC, "outer Chebyshev residual is not finite");
    if (!fixed && rel < tol) break;
    if (it + 1 == nmax) break;
    rc = precond(h, r, nullptr, z);
    if (rc) return rc;
    if (delta > 0.0) {
      const double rho_next = 1.0 / (2.0 * sigma1 - rho);
      c1 = rho_next * rho;
      c2 = 2.0 * rho_next / delta;
      rho = rho_next;
    } else {
      c1 = 0.0;
      c2 = 1.0 / theta;
    }
  }
  // explicit residual of the final iterate
  rc = residual(h, b, x, r2, &rn2);
  if (rc) return rc;
  st.a_matvecs += h->ell;
  st.resid_explicit = std::sqrt(rn2) / bnorm;
  st.converged = st.resid_explicit < tol;
  if (!fixed && !st.converged)
    return fail(h, AAO_ENOTCONV, "outer Chebyshev: no convergence in %d iterations (rel. residual %.3e)",
                st.outer_its, st.resid_explicit);
  return AAO_OK;
}

}  // namespace

namespace aao {
int handle_fail(aao_ctx* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}
bool is_device_ptr(const void* p) { return ::is_device_ptr(p); }
bool is_other_device_ptr(const void* p) { return ::is_other_device_ptr(p); }
int handle_precond(aao_ctx* h, const double* r, const double* rscale, double* z) {
  return ::precond(h, r, rscale, z);
}
void handle_reset_graphs(aao_ctx* h) { ::reset_graphs(h); }
int handle_check_tma(aao_ctx* h) { return ::check_tma(h); }
int handle_ensure_stage(aao_ctx* h) { return ::ensure_stage(h); }
}  // namespace aao


extern "C" {

void aao_default_options(aao_options* opt) {
  if (!opt) return;
  opt->prec = AAO_MIXED;
  opt->inner_its = 20;
  opt->restart = 64;
  opt->orth = AAO_ORTH_MGS;
  opt->mu_max_override = 0.0;
  opt->stream = nullptr;
}

const char* aao_last_create_error(void) { return g_create_error.c_str(); }

const char* aao_last_error(aao_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t aao_kernel_launch_count(void) { return (int64_t)aao::launch_count(); }

void aao_destroy(aao_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->multi) aao::multi_destroy(h->multi);
  h->multi = nullptr;
  if (!h->owns_coeffs) {
    // a view: the face arrays belong to the handle it was made from
    h->cx64 = h->cy64 = h->cz64 = nullptr;
    h->cx32 = h->cy32 = h->cz32 = nullptr;
  }
  void* dev[] = {h->cx64, h->cy64, h->cz64, h->cx32, h->cy32, h->cz32, h->bhat, h->xa, h->xb, h->xc,
                 h->xd,   h->V,    h->Z,    h->sc,   h->partials, h->stage_a, h->stage_b, h->counter,
                 h->tma_fault};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  reset_graphs(h);
  if (h->dct) aao::dct_plan_destroy(h->dct);
  if (h->sp) aao::sp_plan_destroy(h->sp);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->gevent) cudaEventDestroy(h->gevent);
  delete h;
}

int aao_create(aao_handle* out, int dim, const int64_t n[3], const double* kx, const double* ky, const double* kz,
               int ell, double alpha, const aao_options* opt_in) {
  if (!out) return fail(nullptr, AAO_EINVAL, "aao_create: handle pointer is NULL");
  *out = nullptr;
  aao_options opt;
  aao_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (dim < 1 || dim > 3) return fail(nullptr, AAO_EINVAL, "dim must be 1, 2 or 3 (got %d)", dim);
  if (!n) return fail(nullptr, AAO_EINVAL, "n is NULL");
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1) return fail(nullptr, AAO_EINVAL, "n[%d] = %lld must be >= 1", d, (long long)n[d]);
    if (d >= dim && n[d] != 1) return fail(nullptr, AAO_EINVAL, "n[%d] must be 1 for dim = %d", d, dim);
  }
  if (n[0] > 2000000000LL || n[1] > 8LL * 65535 || n[2] > 65535)
    return fail(nullptr, AAO_EINVAL, "grid too large (n0 <= 2e9, n1 <= 524280, n2 <= 65535)");
  {
    // N, ell N and the Krylov bases' byte counts must not wrap: N <= 2^36 cells
    int64_t nn = 0;
    if (__builtin_mul_overflow(n[0], n[1], &nn) || __builtin_mul_overflow(nn, n[2], &nn) || nn > (1LL << 36))
      return fail(nullptr, AAO_EINVAL, "grid too large: n0 * n1 * n2 must be at most 2^36 cells");
  }
  if (n[0] > 1 && !kx) return fail(nullptr, AAO_EINVAL, "kx is NULL but n0 > 1");
  if (n[1] > 1 && !ky) return fail(nullptr, AAO_EINVAL, "ky is NULL but n1 > 1");
  if (n[2] > 1 && !kz) return fail(nullptr, AAO_EINVAL, "kz is NULL but n2 > 1");
  if (ell < 4 || ell > AAO_MAX_ELL || (ell % 2) != 0)
    return fail(nullptr, AAO_EINVAL, "ell must be even and in [4, %d] (got %d)", AAO_MAX_ELL, ell);
  if (!(alpha > 0.0 && alpha < 1.0))
    return fail(nullptr, AAO_EINVAL, "alpha must satisfy 0 < alpha < mu_min^ell = 1 (got %g)", alpha);
  if (opt.prec != AAO_FP64 && opt.prec != AAO_MIXED) return fail(nullptr, AAO_EINVAL, "bad precision mode %d", opt.prec);
  if (opt.inner_its < 1 || opt.inner_its > 100000) return fail(nullptr, AAO_EINVAL, "inner_its must be in [1, 100000]");
  if (opt.orth != AAO_ORTH_CGS && opt.orth != AAO_ORTH_CGS2 && opt.orth != AAO_ORTH_MGS)
    return fail(nullptr, AAO_EINVAL, "bad orthogonalisation mode %d", opt.orth);
  if (opt.restart < 1 || opt.restart > AAO_MAX_RESTART)
    return fail(nullptr, AAO_EINVAL, "restart must be in [1, %d]", AAO_MAX_RESTART);
  if (!(opt.mu_max_override >= 0.0) || !std::isfinite(opt.mu_max_override))
    return fail(nullptr, AAO_EINVAL, "mu_max_override must be finite and >= 0");
  if (opt.mu_max_override > 0.0 && opt.mu_max_override <= 1.0)
    return fail(nullptr, AAO_EINVAL, "mu_max_override must exceed mu_min = 1");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, AAO_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(ce));
  }

  aao_ctx* h = new aao_ctx();
  h->dim = dim;
  for (int d = 0; d < 3; ++d) h->n[d] = n[d];
  h->N = n[0] * n[1] * n[2];
  h->ell = ell;
  h->L = (int64_t)ell * h->N;
  h->alpha = alpha;
  h->prec = opt.prec;
  h->p = opt.inner_its;
  h->m = opt.restart;
  h->orth = opt.orth;
  h->stream = (cudaStream_t)opt.stream;
  h->g.n0 = (int)n[0];
  h->g.n1 = (int)n[1];
  h->g.n2 = (int)n[2];
  h->g.N = h->N;

  auto bail = [&](int code) {
    g_create_error = h->err;
    aao_destroy(h);
    return code;
  };
#define AAO_CK_CREATE(call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      fail(h, e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
      return bail(e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA);                         \
    }                                                                                                \
  } while (0)

  const int64_t N = h->N;
  const int64_t nfx = n[2] * n[1] * (n[0] - 1), nfy = n[2] * (n[1] - 1) * n[0], nfz = (n[2] - 1) * n[1] * n[0];
  AAO_CK_CREATE(cudaMalloc(&h->cx64, sizeof(double) * N));
  AAO_CK_CREATE(cudaMalloc(&h->cy64, sizeof(double) * N));
  AAO_CK_CREATE(cudaMalloc(&h->cz64, sizeof(double) * N));
  AAO_CK_CREATE(cudaMalloc(&h->cx32, sizeof(float) * N));
  AAO_CK_CREATE(cudaMalloc(&h->cy32, sizeof(float) * N));
  AAO_CK_CREATE(cudaMalloc(&h->cz32, sizeof(float) * N));
  const int nbred = aao::reduction_blocks(h->L);
  const int nbmv = (int)(((n[0] + 31) / 32) * ((n[1] + 7) / 8) * n[2]) + (int)((n[0] + 255) / 256);
  const int nbcf = aao::build_coeff_blocks(N);
  h->part_cap = std::max<int64_t>({(int64_t)(h->m + 2) * nbred, (int64_t)nbmv, (int64_t)nbcf}) + 64;
  AAO_CK_CREATE(cudaMalloc(&h->partials, sizeof(double) * h->part_cap));
  const ScLayout Lsc{h->m};
  AAO_CK_CREATE(cudaMalloc(&h->sc, sizeof(double) * Lsc.size()));
  AAO_CK_CREATE(cudaMemset(h->sc, 0, sizeof(double) * Lsc.size()));
  AAO_CK_CREATE(cudaMalloc(&h->counter, sizeof(unsigned)));
  AAO_CK_CREATE(cudaMemset(h->counter, 0, sizeof(unsigned)));
  AAO_CK_CREATE(cudaMalloc(&h->tma_fault, sizeof(unsigned)));
  AAO_CK_CREATE(cudaMemset(h->tma_fault, 0, sizeof(unsigned)));
  AAO_CK_CREATE(cudaMallocHost(&h->pinned, sizeof(double) * 16));

  // face arrays: device pointers are used in place, host arrays are staged
  const double* fk[3] = {kx, ky, kz};
  const int64_t fn[3] = {nfx, nfy, nfz};
  double* tmp[3] = {nullptr, nullptr, nullptr};
  const double* dk[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < 3; ++d) {
    if (fn[d] == 0) continue;
    if (is_other_device_ptr(fk[d])) {
      for (double* t : tmp)
        if (t) cudaFree(t);
      fail(h, AAO_EINVAL, "face array %d must be host memory or memory of the current device", d);
      return bail(AAO_EINVAL);
    }
    if (is_device_ptr(fk[d])) {
      dk[d] = fk[d];
    } else {
      cudaError_t e = cudaMalloc(&tmp[d], sizeof(double) * fn[d]);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp[d], fk[d], sizeof(double) * fn[d], cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) {
        for (double* t : tmp)
          if (t) cudaFree(t);
        fail(h, AAO_ECUDA, "staging face array %d: %s", d, cudaGetErrorString(e));
        return bail(e == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA);
      }
      dk[d] = tmp[d];
    }
  }
  int* bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, sizeof(int) * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int) * 2, h->stream);
  if (e == cudaSuccess)
    e = aao::launch_build_coeffs(h->g, dk[0], dk[1], dk[2], h->cx64, h->cy64, h->cz64, h->cx32, h->cy32, h->cz32,
                                 h->partials, bad, h->sc + Lsc.nrm2(), h->stream);
  int hbad[2] = {0, 0};
  double smax = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hbad, bad, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&smax, h->sc + Lsc.nrm2(), sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  for (double* t : tmp)
    if (t) cudaFree(t);
  if (bad) cudaFree(bad);
  if (e != cudaSuccess) {
    fail(h, AAO_ECUDA, "coefficient set-up: %s", cudaGetErrorString(e));
    return bail(AAO_ECUDA);
  }
  if (hbad[0]) {
    fail(h, AAO_EINVAL, "face diffusivities must be finite and > 0");
    return bail(AAO_EINVAL);
  }
  h->mu_min = 1.0;  // K annihilates constants and is PSD: lambda_min(I + K) = 1
  h->mu_max = opt.mu_max_override > 0.0 ? opt.mu_max_override : 1.0 + 2.0 * smax;  // Gershgorin
  if (!(h->mu_max >= h->mu_min)) h->mu_max = h->mu_min;

  const size_t fsz = (h->prec == AAO_MIXED) ? sizeof(float) : sizeof(double);
  AAO_CK_CREATE(cudaMalloc(&h->bhat, fsz * h->L));
  AAO_CK_CREATE(cudaMalloc(&h->xa, fsz * h->L));
  AAO_CK_CREATE(cudaMalloc(&h->xb, fsz * h->L));
  h->pairs = (h->prec == AAO_MIXED && dim == 2 && n[0] % 4 == 0);
  if (h->pairs) {
    AAO_CK_CREATE(cudaMalloc(&h->xc, fsz * h->L));
    AAO_CK_CREATE(cudaMalloc(&h->xd, fsz * h->L));
    // TMA descriptors for the persistent four-step kernel; without them the
    // shared-memory tile kernel runs the same steps.
    const float* fields[5] = {(const float*)h->xa, (const float*)h->xb, (const float*)h->xc, (const float*)h->xd,
                              (const float*)h->bhat};
    bool ok = true;
    for (int i = 0; i < 5 && ok; ++i) ok = aao::encode_field_map(&h->fmap[i], fields[i], h->g, ell) == cudaSuccess;
    if (ok) ok = aao::encode_coef_map(&h->fmap[5], h->cx32, h->g) == cudaSuccess;
    if (ok) ok = aao::encode_coef_map(&h->fmap[6], h->cy32, h->g) == cudaSuccess;
    cudaGetLastError();
    h->tma = ok;
    // the default fused-sweep kernel: warp strips with a configuration sized to the device,
    // unless the tune cache holds an entry for this grid
    h->auto_kind = AAO_STEP_STREAM;
    h->scfg = aao::default_stream_config(h->g, ell);
    h->tail = aao::default_tail_config(h->g, ell);
    aao::apply_tune_cache(h);
  }
  AAO_CK_CREATE(cudaMalloc(&h->V, sizeof(double) * h->L * (h->m + 1)));
  AAO_CK_CREATE(cudaMalloc(&h->Z, sizeof(double) * h->L * h->m));
  build_tables(h);
  *out = h;
#undef AAO_CK_CREATE
  return AAO_OK;
}

int aao_get_bounds(aao_handle h, double* mu_min, double* mu_max) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (mu_min) *mu_min = h->mu_min;
  if (mu_max) *mu_max = h->mu_max;
  return AAO_OK;
}

// A double array must be 8-byte aligned: the kernels read and write it element by element at
// least.  (Outputs written two doubles at a time are staged when not 16-byte aligned.)
static bool misaligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) != 0; }

int aao_matvec(aao_handle h, const double* x, double* y) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (!x || !y || x == y) return fail(h, AAO_EINVAL, "aao_matvec: x and y must be distinct non-NULL pointers");
  if (misaligned8(x) || misaligned8(y)) return fail(h, AAO_EINVAL, "aao_matvec: x and y must be 8-byte aligned");
  h->err.clear();
  if (is_other_device_ptr(x) || is_other_device_ptr(y))
    return fail(h, AAO_EINVAL, "aao_matvec: x and y must be host memory or memory of the current device");
  const bool hx = !is_device_ptr(x), hy = !is_device_ptr(y);
  int rc = (hx || hy) ? ensure_stage(h) : AAO_OK;
  if (rc) return rc;
  const double* dx = x;
  double* dy = y;
  if (hx) {
    AAO_CK(h, cudaMemcpyAsync(h->stage_a, x, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
    dx = h->stage_a;
  }
  if (hy) dy = h->stage_b;
  rc = matvec(h, dx, nullptr, dy, nullptr);
  if (rc) return rc;
  if (hy) AAO_CK(h, cudaMemcpyAsync(y, dy, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream));
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  return AAO_OK;
}

int aao_precond_apply(aao_handle h, const double* r, double* z) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (!r || !z || r == z) return fail(h, AAO_EINVAL, "aao_precond_apply: r and z must be distinct non-NULL pointers");
  if (misaligned8(r) || misaligned8(z))
    return fail(h, AAO_EINVAL, "aao_precond_apply: r and z must be 8-byte aligned");
  h->err.clear();
  if (is_other_device_ptr(r) || is_other_device_ptr(z))
    return fail(h, AAO_EINVAL, "aao_precond_apply: r and z must be host memory or memory of the current device");
  // z is written two doubles at a time by the inverse transforms: a device z that is not
  // 16-byte aligned is staged like host memory and copied on the device afterwards
  const bool zdev = is_device_ptr(z);
  const bool hr = !is_device_ptr(r), hz = !zdev || (reinterpret_cast<uintptr_t>(z) & 15) != 0;
  int rc = (hr || hz) ? ensure_stage(h) : AAO_OK;
  if (rc) return rc;
  const double* dr = r;
  double* dz = z;
  if (hr) {
    AAO_CK(h, cudaMemcpyAsync(h->stage_a, r, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
    dr = h->stage_a;
  }
  if (hz) dz = h->stage_b;
  rc = precond(h, dr, nullptr, dz);
  if (rc == AAO_OK) rc = check_tma(h);
  if (rc) return rc;
  if (hz)
    AAO_CK(h, cudaMemcpyAsync(z, dz, sizeof(double) * h->L, zdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream));
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  return AAO_OK;
}

static int solve_entry(aao_handle h, const double* b, double* x, double tol, int max_outer, int inner_its,
                       int use_x0, int fixed) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  h->err.clear();
  if (!b || !x || b == x) return fail(h, AAO_EINVAL, "b and x must be distinct non-NULL pointers");
  if (misaligned8(b) || misaligned8(x)) return fail(h, AAO_EINVAL, "b and x must be 8-byte aligned");
  if (!fixed && !(tol > 0.0 && tol < 1.0)) return fail(h, AAO_EINVAL, "tol must be in (0, 1)");
  if (max_outer < 1) return fail(h, AAO_EINVAL, "max_outer must be >= 1");
  if (fixed && fixed > h->m) return fail(h, AAO_EINVAL, "fixed step count %d exceeds restart %d", fixed, h->m);
  if (inner_its < 0 || inner_its > 100000) return fail(h, AAO_EINVAL, "inner_its must be in [0, 100000]");
  if (inner_its > 0 && (inner_its != h->p || h->nc2)) {
    h->p = inner_its;
    h->nc2 = false;
    build_tables(h);
  }
  if (is_other_device_ptr(b) || is_other_device_ptr(x))
    return fail(h, AAO_EINVAL, "b and x must be host memory or memory of the current device");
  const bool hb = !is_device_ptr(b), hx = !is_device_ptr(x);
  int rc = (hb || hx) ? ensure_stage(h) : AAO_OK;
  if (rc) return rc;
  const double* db = b;
  double* dx = x;
  if (hb) {
    AAO_CK(h, cudaMemcpyAsync(h->stage_a, b, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
    db = h->stage_a;
  }
  if (hx) {
    dx = h->stage_b;
    if (use_x0) AAO_CK(h, cudaMemcpyAsync(dx, x, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
  }
  if (!use_x0) AAO_CK(h, cudaMemsetAsync(dx, 0, sizeof(double) * h->L, h->stream));
  rc = solve_impl(h, db, dx, fixed ? 1.0 : tol, fixed ? fixed : max_outer, fixed, !use_x0);
  if (rc == AAO_OK || rc == AAO_ENOTCONV) {
    const int rt = check_tma(h);
    if (rt) return rt;
  }
  if (hx && (rc == AAO_OK || rc == AAO_ENOTCONV)) {
    cudaError_t e = cudaMemcpyAsync(x, dx, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, AAO_ECUDA, "copy of x to host: %s", cudaGetErrorString(e));
  }
  if (rc == AAO_OK || rc == AAO_ENOTCONV) AAO_CK(h, cudaStreamSynchronize(h->stream));
  return rc;
}

int aao_solve(aao_handle h, const double* b, double* x, double tol, int max_outer, int inner_its, int use_x0) {
  return solve_entry(h, b, x, tol, max_outer, inner_its, use_x0, 0);
}

int aao_solve_fixed(aao_handle h, const double* b, double* x, int k, int inner_its) {
  if (k < 1) return fail(h, AAO_EINVAL, "k must be >= 1");
  return solve_entry(h, b, x, 0.5, k, inner_its, 0, k);
}

int aao_profile_enable(aao_handle h, int on) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  h->pending.clear();
  h->profacc = aao_profile{};
  h->prof = on != 0;
  return AAO_OK;
}

int aao_profile_get(aao_handle h, aao_profile* out) {
  if (!h || !out) return fail(h, AAO_EINVAL, "NULL argument");
  AAO_CK(h, cudaStreamSynchronize(h->stream));
  prof_resolve(h);
  *out = h->profacc;
  return AAO_OK;
}

int aao_set_inner_alloc(aao_handle h, const int32_t* p, int ell) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (!p || ell != h->ell) return fail(h, AAO_EINVAL, "p must hold ell = %d counts", h->ell);
  int pmax = 0;
  for (int j = 0; j < ell; ++j) {
    if (p[j] < 0 || p[j] > 100000) return fail(h, AAO_EINVAL, "step counts must be in [0, 100000]");
    if (j > 0 && p[j] != p[ell - j])
      return fail(h, AAO_EINVAL, "conjugate shifts need equal counts: p[%d] = %d but p[%d] = %d", j, p[j], ell - j,
                  p[ell - j]);
    pmax = std::max(pmax, (int)p[j]);
  }
  if (pmax < 1) return fail(h, AAO_EINVAL, "at least one frequency needs a step");
  for (int m = 0; m <= ell / 2; ++m) h->palloc[m] = p[m];
  h->nc2 = true;
  h->p = pmax;
  build_tables(h);
  return AAO_OK;
}

int aao_set_step_kernel(aao_handle h, int kind) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (kind != AAO_STEP_AUTO && kind != AAO_STEP_TILE && kind != AAO_STEP_TMA && kind != AAO_STEP_STREAM)
    return fail(h, AAO_EINVAL, "unknown step kernel %d", kind);
  if (kind == AAO_STEP_STREAM && !h->pairs)
    return fail(h, AAO_EINVAL, "the warp-strip kernel needs the 2D mixed path with n0 %% 4 == 0");
  if (kind == AAO_STEP_TMA && !h->tma)
    return fail(h, AAO_EINVAL, "the persistent TMA kernel needs the 2D mixed path with n0 %% 4 == 0 and TMA descriptors");
  if (kind == AAO_STEP_TILE && !h->pairs)
    return fail(h, AAO_EINVAL, "the fused tile kernels need the 2D mixed path with n0 %% 4 == 0");
  h->step_kernel = kind;
  reset_graphs(h);
  return AAO_OK;
}

int aao_set_precond_mode(aao_handle h, int mode) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (mode == AAO_PRECOND_NC) {
    h->pmode = mode;
    reset_graphs(h);
    return AAO_OK;
  }
  if (mode == AAO_PRECOND_SP) {
    if (h->prec != AAO_FP64) return fail(h, AAO_EINVAL, "P_SP is applied in FP64: create the handle with AAO_FP64");
    if (!h->sp) AAO_CK(h, aao::sp_plan_create(&h->sp, h->g, h->dim, h->cx64, h->cy64, h->cz64, h->stream));
    h->pmode = mode;
    reset_graphs(h);
    return AAO_OK;
  }
  if (mode != AAO_PRECOND_EXACT_DCT) return fail(h, AAO_EINVAL, "unknown preconditioner mode %d", mode);
  if (h->prec != AAO_FP64) return fail(h, AAO_EINVAL, "the best-case P_alpha is applied in FP64: create the handle with AAO_FP64");
  if (!h->dct) {
    double mm[6] = {0, 0, 0, 0, 0, 0};
    AAO_CK(h, aao::face_ranges(h->g, h->cx64, h->dim >= 2 ? h->cy64 : nullptr, h->dim == 3 ? h->cz64 : nullptr, mm,
                               h->stream));
    double kap[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < h->dim; ++a) {
      const double lo = mm[2 * a], hi = mm[2 * a + 1];
      if (hi > 0.0 && !(hi - lo <= 1e-12 * hi))
        return fail(h, AAO_EINVAL, "the best-case P_alpha needs one diffusivity per axis (axis %d has %.17g .. %.17g)",
                    a, lo, hi);
      kap[a] = hi;
    }
    AAO_CK(h, aao::dct_plan_create(&h->dct, h->g, h->dim, h->ell, kap));
  }
  h->pmode = mode;
  reset_graphs(h);
  return AAO_OK;
}

int aao_set_wait_limit(aao_handle h, int64_t cycles) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  if (cycles < 0) return fail(h, AAO_EINVAL, "wait limit must be >= 0 SM clocks");
  h->wait_limit = cycles;
  reset_graphs(h);
  return AAO_OK;
}

int aao_set_stream_config(aao_handle h, int S, int H, int D, int NW) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  aao::StreamConfig c;
  c.S = S;
  c.H = H;
  c.D = D;
  c.NW = NW;
  if (!aao::stream_config_supported(c))
    return fail(h, AAO_EINVAL, "unsupported warp-strip configuration S=%d H=%d D=%d NW=%d", S, H, D, NW);
  h->scfg = c;
  reset_graphs(h);
  return AAO_OK;
}

int aao_set_stream_tail(aao_handle h, int H, int D, int NW) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  aao::StreamConfig c;
  c.S = 2;
  c.H = H;
  c.D = D;
  c.NW = NW;
  if (!aao::stream_config_supported(c))
    return fail(h, AAO_EINVAL, "unsupported two-step configuration H=%d D=%d NW=%d", H, D, NW);
  h->tail = c;
  reset_graphs(h);
  return AAO_OK;
}

int aao_get_stream_tail(aao_handle h, int32_t out[3]) {
  if (!h || !out) return fail(h, AAO_EINVAL, "NULL argument");
  out[0] = h->tail.H;
  out[1] = h->tail.D;
  out[2] = h->tail.NW;
  return AAO_OK;
}

int aao_get_stream_config(aao_handle h, int32_t out[4]) {
  if (!h || !out) return fail(h, AAO_EINVAL, "NULL argument");
  out[0] = h->scfg.S;
  out[1] = h->scfg.H;
  out[2] = h->scfg.D;
  out[3] = h->scfg.NW;
  return AAO_OK;
}

int aao_get_step_kernel(aao_handle h) {
  if (!h) return -1;
  if (!h->pairs) return AAO_STEP_AUTO;
  const int k = aao::effective_step_kernel(h);
  if (k == AAO_STEP_TMA && !h->tma) return AAO_STEP_TILE;
  return k;
}

int aao_assign_iterations(int ell, int64_t nx, double mu_max, double mu_min, double alpha, double eta, int32_t* out) {
  if (ell < 2 || (ell % 2) || nx < 1 || !(mu_max > mu_min) || !(alpha > 0.0) || !(eta > 0.0) || !out ||
      !(std::pow(alpha, 1.0 / ell) < mu_min))
    return AAO_EINVAL;
  using cd = std::complex<double>;
  const double pi = 3.14159265358979323846;
  const double root = std::pow(alpha, 1.0 / ell);
  std::vector<double> r(ell);
  double sig1 = 0.0, sum = 0.0;
  for (int j = 0; j < ell; ++j) {
    const cd lam = root * std::exp(cd(0.0, -2.0 * pi * j / ell));
    // sigma_j of Theorem 4: condition number of Re(B_j) on [mu_min, mu_max]
    const double kap = (mu_max - lam.real()) / (mu_min - lam.real());
    const double sig = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    if (j == 0) sig1 = sig;
    r[j] = std::log(sig1) / std::log(sig);
    sum += r[j];
  }
  for (int j = 0; j < ell; ++j) out[j] = (int32_t)std::floor(r[j] / sum * (double)ell * (double)nx * eta);
  return AAO_OK;
}

int aao_solve_ci(aao_handle h, const double* b, double* x, double tol, int max_outer, int inner_its, int use_x0,
                 double l_min, double l_max, int fixed_its) {
  if (!h) return fail(nullptr, AAO_EINVAL, "NULL handle");
  h->err.clear();
  if (!b || !x || b == x) return fail(h, AAO_EINVAL, "b and x must be distinct non-NULL pointers");
  if (misaligned8(b) || misaligned8(x)) return fail(h, AAO_EINVAL, "b and x must be 8-byte aligned");
  if (!fixed_its && !(tol > 0.0 && tol < 1.0)) return fail(h, AAO_EINVAL, "tol must be in (0, 1)");
  if (max_outer < 1 && !fixed_its) return fail(h, AAO_EINVAL, "max_outer must be >= 1");
  if (fixed_its < 0) return fail(h, AAO_EINVAL, "fixed_its must be >= 0");
  if (h->m < 2) return fail(h, AAO_EINVAL, "the outer Chebyshev solve needs restart >= 2 (workspace)");
  if (l_min <= 0.0 && l_max <= 0.0) {
    // Corollary 1: [1, mu_N^ell / (mu_N^ell - alpha)]
    const double mell = std::pow(h->mu_min, h->ell);
    l_min = 1.0;
    l_max = mell / (mell - h->alpha);
  }
  if (!(l_min > 0.0 && l_max >= l_min && std::isfinite(l_max)))
    return fail(h, AAO_EINVAL, "need 0 < l_min <= l_max");
  if (inner_its < 0 || inner_its > 100000) return fail(h, AAO_EINVAL, "inner_its must be in [0, 100000]");
  if (inner_its > 0 && (inner_its != h->p || h->nc2)) {
    h->p = inner_its;
    h->nc2 = false;
    build_tables(h);
  }
  if (is_other_device_ptr(b) || is_other_device_ptr(x))
    return fail(h, AAO_EINVAL, "b and x must be host memory or memory of the current device");
  const bool hb = !is_device_ptr(b), hx = !is_device_ptr(x);
  int rc = (hb || hx) ? ensure_stage(h) : AAO_OK;
  if (rc) return rc;
  const double* db = b;
  double* dx = x;
  if (hb) {
    AAO_CK(h, cudaMemcpyAsync(h->stage_a, b, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
    db = h->stage_a;
  }
  if (hx) {
    dx = h->stage_b;
    if (use_x0) AAO_CK(h, cudaMemcpyAsync(dx, x, sizeof(double) * h->L, cudaMemcpyHostToDevice, h->stream));
  }
  if (!use_x0) AAO_CK(h, cudaMemsetAsync(dx, 0, sizeof(double) * h->L, h->stream));
  rc = solve_ci_impl(h, db, dx, tol, max_outer, l_min, l_max, fixed_its);
  if (rc == AAO_OK || rc == AAO_ENOTCONV) {
    const int rt = check_tma(h);
    if (rt) return rt;
  }
  if (hx && (rc == AAO_OK || rc == AAO_ENOTCONV)) {
    cudaError_t e = cudaMemcpyAsync(x, dx, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, AAO_ECUDA, "copy of x to host: %s", cudaGetErrorString(e));
  }
  if (rc == AAO_OK || rc == AAO_ENOTCONV) AAO_CK(h, cudaStreamSynchronize(h->stream));
  return rc;
}

int aao_get_stats(aao_handle h, aao_stats* s) {
  if (!h || !s) return fail(h, AAO_EINVAL, "NULL argument");
  *s = h->stats;
  return AAO_OK;
}

}  // extern "C"
