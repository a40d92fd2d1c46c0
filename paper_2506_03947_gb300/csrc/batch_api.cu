// Batched solve: many handles' solves in lockstep (aao_batch_* in include/aao.h).
//
// Every phase of an Arnoldi step (preconditioner, script-A product, Gram-Schmidt, Givens) runs
// as one launch over all active members, from static work lists, and each step is captured once
// as a CUDA graph and replayed.  The kernels are in batch.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "aao_ctx.h"
#include "batch.cuh"

namespace aao {
long long launch_count();
void count_launch_add(long long n);
}  // namespace aao

using aao::is_device_ptr;

// Batch sweep without fused launches: one Chebyshev step per launch (3D members).
constexpr int kSweepSingle = -1;

// ---- batched solve -----------------------------------------------------------------

struct aao_batch_ctx {
  int M = 0, p = 0, m = 0;
  bool mgs = true;  // modified Gram-Schmidt when every member uses it, else CGS2
  std::vector<aao_ctx*> mem;
  cudaStream_t stream = nullptr;
  bool use_graphs = true;
  std::vector<aao::BInst> hI;
  aao::BInst* dI = nullptr;
  int* dact = nullptr;
  int* dkvec = nullptr;
  double* dout = nullptr;
  double* hout = nullptr;  // pinned, 2M
  std::vector<void*> owned;
  std::vector<std::pair<int, aao::WorkList>> wdft, wstep, wquad;  // per ell
  aao::WorkList wmv{}, wred{}, wone{}, wmgs{};
  // fused sweeps: one warp-strip launch over the units of all members (any ell), from a device
  // queue (sweep = AAO_STEP_STREAM), or the shared-memory tile kernel per ell (AAO_STEP_TILE)
  int sweep = AAO_STEP_STREAM;  // AAO_STEP_STREAM, AAO_STEP_TILE or kSweepSingle
  int dim = 2;                  // every member's
  aao::SharedSteps shared{false, 0, 0};  // right-hand sides of one operator
  aao::StreamConfig scfg{};
  aao::WorkList wunits{};
  // the two-step final launch of a sweep whose remaining step count is 2 mod 4 (S = 2, the
  // sweep's D, NW = 8, segment height H - 2) and its units
  aao::StreamConfig tail{};
  aao::WorkList wunits2{};
  aao::StreamQueue* queue = nullptr;
  std::vector<int> hact;  // host copy of the active flags
  // event timing of the Chebyshev sweeps (aao_batch_profile_enable; graphs are not used
  // meanwhile): each fused launch, or the middle single steps of each ell group, is one span
  bool prof = false;
  std::vector<cudaEvent_t> events;
  std::vector<double> pend_bytes;
  std::vector<int> pend_launches;
  double prof_ms = 0.0, prof_bytes = 0.0;
  long long prof_launches = 0;
  std::vector<cudaGraphExec_t> graphs;
  std::vector<long long> graph_launches;
  std::vector<aao_stats> stats;
  std::string err;
};

namespace {

int bfail(aao_batch_ctx* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  else g_create_error = buf;
  return code;
}

#define AAO_BCK(b, call)                                                                                  \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess)                                                                                \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA, "%s: %s (%s:%d)", #call, \
                   cudaGetErrorString(e_), __FILE__, __LINE__);                                           \
  } while (0)

int make_worklist(aao_batch_ctx* B, const std::vector<int>& inst, const std::vector<int>& blocks, aao::WorkList* out) {
  std::vector<int> start(inst.size() + 1, 0);
  for (size_t i = 0; i < inst.size(); ++i) start[i + 1] = start[i] + blocks[i];
  int* ds = nullptr;
  int* di = nullptr;
  AAO_BCK(B, cudaMalloc(&ds, sizeof(int) * start.size()));
  B->owned.push_back(ds);
  AAO_BCK(B, cudaMalloc(&di, sizeof(int) * std::max<size_t>(1, inst.size())));
  B->owned.push_back(di);
  AAO_BCK(B, cudaMemcpy(ds, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
  if (!inst.empty()) AAO_BCK(B, cudaMemcpy(di, inst.data(), sizeof(int) * inst.size(), cudaMemcpyHostToDevice));
  out->start = ds;
  out->inst = di;
  out->cnt = (int)inst.size();
  out->total = start.back();
  return AAO_OK;
}

// The two-step tail configuration of a four-step sweep configuration, and its unit list.
int set_tail(aao_batch_ctx* B, const aao::StreamConfig& c) {
  aao::StreamConfig t = c;
  t.S = 2;
  t.H = c.H - 2;  // H + 8 a multiple of 6 <=> (H - 2) + 4 a multiple of 6
  t.NW = 8;
  if (!aao::stream_config_supported(t)) return bfail(B, AAO_EINVAL, "no two-step configuration for H=%d", c.H);
  std::vector<int> all(B->M), nunits(B->M);
  for (int i = 0; i < B->M; ++i) {
    all[i] = i;
    nunits[i] = aao::batch_stream_units(B->hI[i].g, B->hI[i].ell, 2, t.H);
  }
  aao::WorkList wl{};
  const int rc = make_worklist(B, all, nunits, &wl);
  if (rc) return rc;
  B->wunits2 = wl;
  B->tail = t;
  return AAO_OK;
}

// Phases of Arnoldi step j for every active instance, in stream order.
// Algorithmic bytes of one fused launch over the active members: x_k, x_{k-1} (psrc 2), bhat
// and two face arrays read, two fields written, 4-byte values.
// fin: the sweep's final launch, which writes x_p alone.
double fused_bytes(const aao_batch_ctx* B, int psrc, bool fin = false) {
  const double sets = (psrc == 1 ? 2.0 : 3.0) + (fin ? 1.0 : 2.0);
  double t = 0.0;
  for (int i = 0; i < B->M; ++i)
    if (B->hact.empty() || B->hact[i]) t += (double)B->hI[i].g.N * (sets * 4.0 * B->hI[i].ell + 8.0);
  return t;
}


// Algorithmic bytes of one single-step launch over the active members of the group with this
// ell: x_k, x_{k-1} (psrc 2) and bhat read, x_{k+1} written, 4-byte values; the dim face arrays
// once for the group when the members share them, else once per member.
double single_bytes(const aao_batch_ctx* B, int ell, int psrc) {
  double t = 0.0, faces = 0.0;
  for (int i = 0; i < B->M; ++i)
    if ((B->hact.empty() || B->hact[i]) && B->hI[i].ell == ell) {
      const double n = (double)B->hI[i].g.N;
      t += n * (psrc == 1 ? 3.0 : 4.0) * 4.0 * ell;
      const double f = n * 4.0 * B->dim;
      faces = B->shared.on ? f : faces + f;
    }
  return t + faces;
}

// Record the start of a profiled span of `launches` launches carrying `bytes`; returns its slot
// (-1 if profiling is off, -2 on a CUDA error).
int prof_begin(aao_batch_ctx* B, double bytes, int launches) {
  if (!B->prof) return -1;
  const int ev = (int)B->pend_bytes.size();
  while ((int)B->events.size() < 2 * ev + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -2;
    B->events.push_back(e);
  }
  if (cudaEventRecord(B->events[2 * ev], B->stream) != cudaSuccess) return -2;
  B->pend_bytes.push_back(bytes);
  B->pend_launches.push_back(launches);
  return ev;
}

int batch_precond_stream(aao_batch_ctx* B, int j) {
  cudaStream_t s = B->stream;
  // the transform and step 1 of each ell group in one launch each (bhat and x_2 in field 0)
  for (size_t g = 0; g < B->wstep.size(); ++g)
    AAO_BCK(B, aao::batch_dft_first(B->dI, B->dact, B->wstep[g].first, B->wstep[g].second, j, s));
  // steps 2 .. p-1 as in the single solver: step 2 alone when their count is odd, four-step
  // launches, a two-step launch for a remainder of two; the final launch writes x_p alone.  The
  // four fields rotate so that a launch never writes a field it reads.
  int cur = 0, prev = -1, k = 2, R = B->p - 2;
  if (R % 2 == 1) {
    for (size_t g = 0; g < B->wstep.size(); ++g) {
      int c = 0, pv = -1;  // one single step: the middle-step loop over k = 2 .. (k + 2) - 2
      AAO_BCK(B, aao::batch_steps_mid(B->dI, B->dact, B->wstep[g].first, B->dim, B->shared, B->wstep[g].second, k + 2,
                                      j, k, &c, &pv, s));
      cur = c;
      prev = pv;
    }
    ++k;
    --R;
  }
  // the fused launches run back to back: one event span over all of them (events between them
  // would add gaps of their own)
  const int ev = prof_begin(B, 0.0, 0);
  if (ev == -2) return bfail(B, AAO_ECUDA, "profiling events could not be created or recorded");
  while (R > 0) {
    const int S = R >= 4 ? 4 : 2;
    const bool fin = (R == S);
    const aao::StreamConfig& c = (S == 4) ? B->scfg : B->tail;
    const aao::WorkList& units = (S == 4) ? B->wunits : B->wunits2;
    int o[2], n = 0;
    for (int f = 0; f < 4 && n < 2; ++f)
      if (f != cur && f != prev) o[n++] = f;
    const int psrc = prev < 0 ? 1 : 2;
    if (ev >= 0) {
      B->pend_bytes[ev] += fused_bytes(B, psrc, fin);
      B->pend_launches[ev] += 1;
    }
    AAO_BCK(B, aao::launch_batch_stream(B->dI, B->dact, units, c, k, psrc, cur, prev, fin ? -1 : o[0],
                                        fin ? o[0] : o[1], B->queue, s));
    if (fin) {
      cur = o[0];
    } else {
      prev = o[0];
      cur = o[1];
    }
    k += S;
    R -= S;
  }
  if (ev >= 0) AAO_BCK(B, cudaEventRecord(B->events[2 * ev + 1], s));
  // z = Gamma^{-1} U x_p into Z_j, per ell group
  for (size_t g = 0; g < B->wstep.size(); ++g)
    AAO_BCK(B, aao::batch_idft(B->dI, B->dact, B->wstep[g].first, B->wstep[g].second, j, cur, s));
  return AAO_OK;
}

// Resolve the recorded fused-launch events (the stream has been synchronised).
void batch_prof_resolve(aao_batch_ctx* B) {
  for (size_t i = 0; i < B->pend_bytes.size(); ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, B->events[2 * i], B->events[2 * i + 1]) == cudaSuccess) {
      B->prof_ms += ms;
      B->prof_bytes += B->pend_bytes[i];
      B->prof_launches += B->pend_launches[i];
    }
  }
  B->pend_bytes.clear();
  B->pend_launches.clear();
}

int batch_step_launches(aao_batch_ctx* B, int j) {
  cudaStream_t s = B->stream;
  if (B->sweep == AAO_STEP_STREAM) {
    const int rc = batch_precond_stream(B, j);
    if (rc) return rc;
  } else if (B->sweep == kSweepSingle) {
    // one Chebyshev step per launch: transform and step 1, then steps 2 .. p-1
    for (size_t g = 0; g < B->wdft.size(); ++g)
      AAO_BCK(B, aao::batch_precond_head(B->dI, B->dact, B->wdft[g].first, B->dim, B->shared, B->wdft[g].second,
                                         B->wstep[g].second, B->p, j, s));
    for (size_t g = 0; g < B->wstep.size(); ++g) {
      const int ell = B->wstep[g].first;
      int cur = 0, prev = -1;
      // steps 2 .. p-1 as middle steps (the last one writes x_p), profiled as one timed span of
      // p-2 launches; then z = Gamma^{-1} U x_p by the inverse-transform launch of the group.  A
      // last step with the inverse transform fused (its z time blocks held in registers beside
      // the stencil) runs far below the bandwidth of these two launches.
      double bytes = 0.0;
      if (B->prof)
        for (int k = 2; k <= B->p - 1; ++k) bytes += single_bytes(B, ell, k == 2 ? 1 : 2);
      const int ev = prof_begin(B, bytes, B->p - 2);
      if (ev == -2) return bfail(B, AAO_ECUDA, "profiling events could not be created or recorded");
      AAO_BCK(B, aao::batch_steps_mid(B->dI, B->dact, ell, B->dim, B->shared, B->wstep[g].second, B->p + 1, j, 2, &cur,
                                      &prev, s));
      if (ev >= 0) AAO_BCK(B, cudaEventRecord(B->events[2 * ev + 1], s));
      AAO_BCK(B, aao::batch_idft(B->dI, B->dact, ell, B->wstep[g].second, j, cur, s));
    }
  } else {
    for (size_t g = 0; g < B->wdft.size(); ++g)
      AAO_BCK(B, aao::batch_precond(B->dI, B->dact, B->wdft[g].first, B->wdft[g].second, B->wstep[g].second,
                                    B->wquad[g].second, B->p, j, s));
  }
  AAO_BCK(B, aao::batch_matvec(B->dI, B->dact, B->wmv, 0, j, B->dim, s));
  if (B->mgs) AAO_BCK(B, aao::batch_mgs(B->dI, B->dact, B->wmgs, j, s));
  else AAO_BCK(B, aao::batch_gram_schmidt(B->dI, B->dact, B->wred, B->wone, j, s));
  AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 0, j, B->dkvec, B->dout, s));
  AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 3, j, B->dkvec, B->dout, s));
  return AAO_OK;
}

int batch_run_step(aao_batch_ctx* B, int j) {
  if (!B->use_graphs || B->prof) return batch_step_launches(B, j);
  if ((int)B->graphs.size() <= j) {
    B->graphs.resize(j + 1, nullptr);
    B->graph_launches.resize(j + 1, 0);
  }
  if (!B->graphs[j]) {
    const long long c0 = aao::launch_count();
    AAO_BCK(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_step_launches(B, j);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(B->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    AAO_BCK(B, ec);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    AAO_BCK(B, ei);
    B->graphs[j] = exec;
    B->graph_launches[j] = aao::launch_count() - c0;
    aao::count_launch_add(-B->graph_launches[j]);  // captured, not run: counted at each replay
  }
  AAO_BCK(B, cudaGraphLaunch(B->graphs[j], B->stream));
  aao::count_launch_add(B->graph_launches[j]);
  return AAO_OK;
}

int batch_read(aao_batch_ctx* B) {
  AAO_BCK(B, cudaMemcpyAsync(B->hout, B->dout, sizeof(double) * 2 * B->M, cudaMemcpyDeviceToHost, B->stream));
  AAO_BCK(B, cudaStreamSynchronize(B->stream));
  batch_prof_resolve(B);
  return AAO_OK;
}

int batch_set_active(aao_batch_ctx* B, const std::vector<int>& act) {
  B->hact = act;
  AAO_BCK(B, cudaMemcpyAsync(B->dact, act.data(), sizeof(int) * B->M, cudaMemcpyHostToDevice, B->stream));
  AAO_BCK(B, cudaStreamSynchronize(B->stream));  // act is a host temporary
  return AAO_OK;
}

}  // namespace

extern "C" {

void aao_batch_destroy(aao_batch hb) {
  if (!hb) return;
  if (hb->stream) cudaStreamSynchronize(hb->stream);
  for (cudaGraphExec_t g : hb->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (void* p : hb->owned) cudaFree(p);
  if (hb->dI) cudaFree(hb->dI);
  if (hb->dact) cudaFree(hb->dact);
  if (hb->dkvec) cudaFree(hb->dkvec);
  if (hb->dout) cudaFree(hb->dout);
  if (hb->hout) cudaFreeHost(hb->hout);
  if (hb->queue) cudaFree(hb->queue);
  for (cudaEvent_t e : hb->events) cudaEventDestroy(e);
  if (hb->stream) cudaStreamDestroy(hb->stream);
  delete hb;
}

int aao_batch_create(aao_batch* out, int count, const aao_handle* members, int use_graphs) {
  if (!out) return bfail(nullptr, AAO_EINVAL, "aao_batch_create: out is NULL");
  *out = nullptr;
  if (count < 1 || !members) return bfail(nullptr, AAO_EINVAL, "need at least one member handle");
  for (int i = 0; i < count; ++i) {
    const aao_ctx* h = members[i];
    if (!h) return bfail(nullptr, AAO_EINVAL, "member %d is NULL", i);
    if (h->prec != AAO_MIXED || (h->dim != 2 && h->dim != 3) || h->n[0] % 4 != 0)
      return bfail(nullptr, AAO_EINVAL, "member %d: the batch runs mixed-precision 2D or 3D grids with n0 %% 4 == 0", i);
    if (h->dim != members[0]->dim) return bfail(nullptr, AAO_EINVAL, "members must share the grid dimension");
    if (h->dim == 3 && h->p < 3) return bfail(nullptr, AAO_EINVAL, "member %d: 3D batches need inner_its >= 3", i);
    if (h->p < 2) return bfail(nullptr, AAO_EINVAL, "member %d: the batch needs inner_its >= 2", i);
    if (h->p != members[0]->p || h->m != members[0]->m)
      return bfail(nullptr, AAO_EINVAL, "members must share inner_its and restart (member %d differs)", i);
    if (h->m < 2) return bfail(nullptr, AAO_EINVAL, "restart must be >= 2");
  }
  aao_batch_ctx* B = new aao_batch_ctx();
  B->M = count;
  B->p = members[0]->p;
  B->m = members[0]->m;
  B->use_graphs = use_graphs != 0;
  auto bail = [&](int code) {
    g_create_error = B->err;
    aao_batch_destroy(B);
    return code;
  };
#define AAO_BCK_CREATE(call)               \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) {               \
      bfail(B, e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
      return bail(e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA); \
    }                                      \
  } while (0)
  AAO_BCK_CREATE(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
  B->hI.resize(count);
  std::vector<int> all(count), bdft(count), bstep(count), bquad(count), bmv(count), bred(count), bmgs(count),
      bone(count, 1);
  std::vector<int> ells;
  for (int i = 0; i < count; ++i) {
    aao_ctx* h = members[i];
    B->mem.push_back(h);
    aao::BInst& bi = B->hI[i];
    bi.g = h->g;
    bi.ell = h->ell;
    bi.m = h->m;
    bi.L = h->L;
    bi.nbred = aao::reduction_blocks(h->L);
    bi.nbmgs = aao::batch_mgs_blocks(h->L);
    bi.nbmv = aao::batch_matvec_blocks(h->g);
    bi.cx32 = h->cx32;
    bi.cy32 = h->cy32;
    bi.cz32 = h->cz32;
    bi.cx64 = h->cx64;
    bi.cy64 = h->cy64;
    bi.cz64 = h->cz64;
    bi.bhat = (float*)h->bhat;
    bi.xa = (float*)h->xa;
    bi.xb = (float*)h->xb;
    bi.xc = (float*)h->xc;
    bi.xd = (float*)h->xd;
    bi.V = h->V;
    bi.Z = h->Z;
    bi.sc = h->sc;
    bi.partials = h->partials;
    bi.counter = h->counter;
    if (h->orth != AAO_ORTH_MGS) B->mgs = false;
    void* dsteps = nullptr;
    AAO_BCK_CREATE(cudaMalloc(&dsteps, sizeof(aao::StepArgs<float>) * h->steps32.size()));
    B->owned.push_back(dsteps);
    AAO_BCK_CREATE(cudaMemcpy(dsteps, h->steps32.data(), sizeof(aao::StepArgs<float>) * h->steps32.size(),
                              cudaMemcpyHostToDevice));
    void* dda = nullptr;
    void* dia = nullptr;
    AAO_BCK_CREATE(cudaMalloc(&dda, sizeof(aao::DftArgs<float>)));
    B->owned.push_back(dda);
    AAO_BCK_CREATE(cudaMalloc(&dia, sizeof(aao::IdftArgs<float>)));
    B->owned.push_back(dia);
    AAO_BCK_CREATE(cudaMemcpy(dda, &h->dft32, sizeof(aao::DftArgs<float>), cudaMemcpyHostToDevice));
    AAO_BCK_CREATE(cudaMemcpy(dia, &h->idft32, sizeof(aao::IdftArgs<float>), cudaMemcpyHostToDevice));
    bi.steps = (const aao::StepArgs<float>*)dsteps;
    bi.da = (const aao::DftArgs<float>*)dda;
    bi.ia = (const aao::IdftArgs<float>*)dia;
    bi.b = nullptr;
    bi.x = nullptr;
    all[i] = i;
    bdft[i] = (int)((h->N + 255) / 256);
    bstep[i] = aao::batch_step_blocks(h->g);
    bquad[i] = aao::batch_quad_tiles(h->g);
    bmv[i] = bi.nbmv;
    bred[i] = bi.nbred;
    bmgs[i] = bi.nbmgs;
    if (std::find(ells.begin(), ells.end(), h->ell) == ells.end()) ells.push_back(h->ell);
  }
  for (int ell : ells) {
    std::vector<int> inst, nd, ns, nq;
    for (int i = 0; i < count; ++i)
      if (members[i]->ell == ell) {
        inst.push_back(i);
        nd.push_back(bdft[i]);
        ns.push_back(bstep[i]);
        nq.push_back(bquad[i]);
      }
    aao::WorkList wd, ws, wq;
    if (make_worklist(B, inst, nd, &wd) || make_worklist(B, inst, ns, &ws) || make_worklist(B, inst, nq, &wq))
      return bail(AAO_ECUDA);
    B->wdft.push_back({ell, wd});
    B->wstep.push_back({ell, ws});
    B->wquad.push_back({ell, wq});
  }
  // warp-strip units of every member (any ell) for the fused sweeps: segments of 64 rows
  B->scfg.S = 4;
  B->scfg.H = 64;
  B->scfg.D = 3;
  B->scfg.NW = 8;
  B->dim = members[0]->dim;
  if (B->p < 7) B->sweep = AAO_STEP_TILE;  // no step of the fused form would fit
  if (B->dim == 3) B->sweep = kSweepSingle;  // the fused kernels are 2D
  {
    // right-hand sides of one operator: same grid, same face arrays (and the same step tables)
    bool same = true;
    for (int i = 1; i < count && same; ++i) {
      const aao_ctx* a = members[i];
      const aao_ctx* b0 = members[0];
      same = a->g.n0 == b0->g.n0 && a->g.n1 == b0->g.n1 && a->g.n2 == b0->g.n2 && a->cx32 == b0->cx32 &&
             a->cy32 == b0->cy32 && a->cz32 == b0->cz32 && a->ell == b0->ell && a->alpha == b0->alpha &&
             a->mu_max == b0->mu_max;
    }
    B->shared.on = same && count > 1;
    B->shared.M = count;
    B->shared.ntiles = aao::batch_step_blocks(members[0]->g);
  }
  {
    std::vector<int> nunits(count);
    for (int i = 0; i < count; ++i) nunits[i] = aao::batch_stream_units(members[i]->g, members[i]->ell, 4, B->scfg.H);
    if (make_worklist(B, all, nunits, &B->wunits)) return bail(AAO_ECUDA);
    if (set_tail(B, B->scfg)) return bail(AAO_ECUDA);
  }
  AAO_BCK_CREATE(cudaMalloc(&B->queue, sizeof(aao::StreamQueue)));
  AAO_BCK_CREATE(cudaMemset(B->queue, 0, sizeof(aao::StreamQueue)));
  if (make_worklist(B, all, bmv, &B->wmv) || make_worklist(B, all, bred, &B->wred) ||
      make_worklist(B, all, bmgs, &B->wmgs) || make_worklist(B, all, bone, &B->wone))
    return bail(AAO_ECUDA);
  AAO_BCK_CREATE(cudaMalloc(&B->dI, sizeof(aao::BInst) * count));
  AAO_BCK_CREATE(cudaMalloc(&B->dact, sizeof(int) * count));
  AAO_BCK_CREATE(cudaMalloc(&B->dkvec, sizeof(int) * count));
  AAO_BCK_CREATE(cudaMalloc(&B->dout, sizeof(double) * 2 * count));
  AAO_BCK_CREATE(cudaMallocHost(&B->hout, sizeof(double) * 2 * count));
  B->stats.assign(count, aao_stats{});
  *out = B;
#undef AAO_BCK_CREATE
  return AAO_OK;
}

int aao_batch_solve(aao_batch B, const double* const* b, double* const* x, double tol, int max_outer) {
  if (!B) return bfail(nullptr, AAO_EINVAL, "NULL batch");
  B->err.clear();
  if (!b || !x) return bfail(B, AAO_EINVAL, "b and x must be arrays of M device pointers");
  if (!(tol > 0.0 && tol < 1.0) || max_outer < 1) return bfail(B, AAO_EINVAL, "need 0 < tol < 1 and max_outer >= 1");
  const int M = B->M;
  for (int i = 0; i < M; ++i) {
    if (!is_device_ptr(b[i]) || !is_device_ptr(x[i]) || b[i] == x[i])
      return bfail(B, AAO_EINVAL, "instance %d: b and x must be distinct device pointers", i);
    if (((reinterpret_cast<uintptr_t>(b[i]) | reinterpret_cast<uintptr_t>(x[i])) & 7) != 0)
      return bfail(B, AAO_EINVAL, "instance %d: b and x must be 8-byte aligned", i);
    B->hI[i].b = b[i];
    B->hI[i].x = x[i];
  }
  AAO_BCK(B, cudaDeviceSynchronize());  // inputs may come from any stream
  AAO_BCK(B, cudaMemcpyAsync(B->dI, B->hI.data(), sizeof(aao::BInst) * M, cudaMemcpyHostToDevice, B->stream));
  for (int i = 0; i < M; ++i) {
    AAO_BCK(B, cudaMemsetAsync(x[i], 0, sizeof(double) * B->hI[i].L, B->stream));
    B->stats[i] = aao_stats{};
    B->stats[i].mu_min = B->mem[i]->mu_min;
    B->stats[i].mu_max = B->mem[i]->mu_max;
  }
  std::vector<int> act(M, 1), done(M, 0), kvec(M, 0), total(M, 0);
  std::vector<double> bnorm(M, 0.0), beta(M, 0.0);
  int rc = batch_set_active(B, act);
  if (rc) return rc;
  AAO_BCK(B, aao::batch_norm2_b(B->dI, B->dact, B->wred, B->stream));
  AAO_BCK(B, aao::batch_reduce(B->dI, B->dact, B->wone, 4, B->stream));
  AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 4, 0, B->dkvec, B->dout, B->stream));
  if ((rc = batch_read(B))) return rc;
  for (int i = 0; i < M; ++i) {
    bnorm[i] = B->hout[2 * i];
    if (!std::isfinite(bnorm[i])) return bfail(B, AAO_ENUMERIC, "instance %d: ||b|| is not finite", i);
    if (bnorm[i] == 0.0) {
      done[i] = 1;
      B->stats[i].converged = 1;
    }
  }
  while (true) {
    // explicit residuals of the instances still running
    for (int i = 0; i < M; ++i) act[i] = !done[i];
    if (std::none_of(act.begin(), act.end(), [](int v) { return v; })) break;
    if ((rc = batch_set_active(B, act))) return rc;
    AAO_BCK(B, aao::batch_matvec(B->dI, B->dact, B->wmv, 1, 0, B->dim, B->stream));
    AAO_BCK(B, aao::batch_reduce(B->dI, B->dact, B->wone, 3, B->stream));
    AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 5, 0, B->dkvec, B->dout, B->stream));
    if ((rc = batch_read(B))) return rc;
    for (int i = 0; i < M; ++i) {
      if (!act[i]) continue;
      const double rn = B->hout[2 * i];
      const double rel = rn / bnorm[i];
      B->stats[i].resid_explicit = rel;
      B->stats[i].a_matvecs += B->hI[i].ell;
      if (!std::isfinite(rel)) return bfail(B, AAO_ENUMERIC, "instance %d: residual is not finite", i);
      if (rel < tol) {
        done[i] = 1;
        B->stats[i].converged = 1;
        act[i] = 0;
      } else if (total[i] >= max_outer) {
        done[i] = 1;
        act[i] = 0;
      } else {
        beta[i] = rn;
        B->stats[i].cycles++;
      }
    }
    if (std::none_of(act.begin(), act.end(), [](int v) { return v; })) break;
    if ((rc = batch_set_active(B, act))) return rc;
    AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 1, 0, B->dkvec, B->dout, B->stream));
    std::vector<int> part = act;
    std::fill(kvec.begin(), kvec.end(), 0);
    for (int j = 0; j < B->m; ++j) {
      if ((rc = batch_run_step(B, j))) return rc;
      if ((rc = batch_read(B))) return rc;
      bool changed = false;
      for (int i = 0; i < M; ++i) {
        if (!act[i]) continue;
        const double est = B->hout[2 * i], hn = B->hout[2 * i + 1];
        total[i]++;
        kvec[i] = j + 1;
        aao_stats& st = B->stats[i];
        st.outer_its = total[i];
        st.resid_est = est;
        st.a_matvecs += (int64_t)B->hI[i].ell * (B->p + 1);
        if (st.n_hist < AAO_MAX_HIST) st.hist[st.n_hist++] = est;
        if (!std::isfinite(est) || !std::isfinite(hn))
          return bfail(B, AAO_ENUMERIC, "instance %d: non-finite value in Arnoldi step %d", i, total[i]);
        if (est < tol || hn <= 1e-14 * beta[i] || total[i] >= max_outer) {
          act[i] = 0;
          changed = true;
        }
      }
      if (std::none_of(act.begin(), act.end(), [](int v) { return v; })) break;
      if (changed && (rc = batch_set_active(B, act))) return rc;
    }
    // solution update of this cycle's participants
    if ((rc = batch_set_active(B, part))) return rc;
    AAO_BCK(B, cudaMemcpyAsync(B->dkvec, kvec.data(), sizeof(int) * M, cudaMemcpyHostToDevice, B->stream));
    AAO_BCK(B, aao::batch_small(B->dI, B->dact, B->wone, 2, 0, B->dkvec, B->dout, B->stream));
    AAO_BCK(B, aao::batch_xupdate(B->dI, B->dact, B->wred, B->dkvec, B->stream));
    AAO_BCK(B, cudaStreamSynchronize(B->stream));  // kvec is a host temporary
  }
  AAO_BCK(B, cudaStreamSynchronize(B->stream));
  int nconv = 0;
  for (int i = 0; i < M; ++i) nconv += B->stats[i].converged;
  if (nconv < M) return bfail(B, AAO_ENOTCONV, "%d of %d instances did not converge in %d iterations", M - nconv, M,
                              max_outer);
  return AAO_OK;
}

int aao_batch_get_stats(aao_batch B, int i, aao_stats* s) {
  if (!B || !s || i < 0 || i >= B->M) return bfail(B, AAO_EINVAL, "bad batch stats request");
  *s = B->stats[i];
  return AAO_OK;
}

const char* aao_batch_last_error(aao_batch B) { return B ? B->err.c_str() : g_create_error.c_str(); }

int aao_batch_set_sweep(aao_batch B, int kind, int S, int H, int D, int NW) {
  if (!B) return bfail(nullptr, AAO_EINVAL, "NULL batch");
  if (B->dim == 3 && kind != AAO_STEP_AUTO)
    return bfail(B, AAO_EINVAL, "3D batches run single steps only (AAO_STEP_AUTO)");
  if (kind == AAO_STEP_AUTO) {
    if (B->p < 3) return bfail(B, AAO_EINVAL, "single-step sweeps need inner_its >= 3");
    B->sweep = kSweepSingle;
  } else if (kind == AAO_STEP_TILE) {
    B->sweep = kind;
  } else if (kind == AAO_STEP_STREAM) {
    aao::StreamConfig c;
    c.S = S;
    c.H = H;
    c.D = D;
    c.NW = NW;
    if (!aao::stream_config_supported(c) || S != 4 || NW != 8 || D > 4 || (H + 8) % 6 != 0)
      return bfail(B, AAO_EINVAL,
                   "the batched warp-strip launch runs S = 4, D 3 or 4, NW = 8 and the lockstep schedule, H + 8 "
                   "a multiple of 6 (got S=%d H=%d D=%d NW=%d)",
                   S, H, D, NW);
    if (B->p - 2 < S + 1) return bfail(B, AAO_EINVAL, "inner_its %d leaves no fused launch", B->p);
    std::vector<int> all(B->M), nunits(B->M);
    for (int i = 0; i < B->M; ++i) {
      all[i] = i;
      nunits[i] = aao::batch_stream_units(B->hI[i].g, B->hI[i].ell, S, H);
    }
    aao::WorkList wl{};
    const int rc = make_worklist(B, all, nunits, &wl);
    if (rc) return rc;
    const int rt = set_tail(B, c);
    if (rt) return rt;
    B->wunits = wl;
    B->scfg = c;
    B->sweep = kind;
  } else {
    return bfail(B, AAO_EINVAL, "unknown sweep kind %d", kind);
  }
  for (cudaGraphExec_t g : B->graphs)
    if (g) cudaGraphExecDestroy(g);
  B->graphs.clear();
  B->graph_launches.clear();
  return AAO_OK;
}

int aao_batch_profile_enable(aao_batch B, int on) {
  if (!B) return bfail(nullptr, AAO_EINVAL, "NULL batch");
  AAO_BCK(B, cudaStreamSynchronize(B->stream));
  B->pend_bytes.clear();
  B->pend_launches.clear();
  B->prof_ms = B->prof_bytes = 0.0;
  B->prof_launches = 0;
  B->prof = on != 0;
  return AAO_OK;
}

int aao_batch_get_profile(aao_batch B, int64_t* launches, double* ms, double* bytes) {
  if (!B) return bfail(nullptr, AAO_EINVAL, "NULL batch");
  AAO_BCK(B, cudaStreamSynchronize(B->stream));
  batch_prof_resolve(B);
  if (launches) *launches = B->prof_launches;
  if (ms) *ms = B->prof_ms;
  if (bytes) *bytes = B->prof_bytes;
  return AAO_OK;
}

}  // extern "C"
