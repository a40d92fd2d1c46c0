// Several right-hand sides of one operator, solved together (aao_solve_multi in include/aao.h).
//
// Each right-hand side gets a view of the handle: its own Chebyshev fields and Krylov spaces,
// the handle's face coefficients, grid, shifts and step tables.  The views run as one batch
// (batch_api.cu): every phase of an Arnoldi step is one launch over all right-hand sides, and
// because the views share the operator the Chebyshev step kernels load each tile's stencil
// (the face coefficients and the diagonal) once and apply it to every active right-hand side.
// The views are kept on the handle and reused while the number of right-hand sides, p and
// the tables stay the same.
#include <cstring>
#include <vector>

#include "aao_ctx.h"

struct aao_multi {
  int nrhs = 0, p = 0;
  const void* tables = nullptr;  // identity of the handle's step tables when the views were made
  std::vector<aao_ctx*> views;
  aao_batch batch = nullptr;
};

namespace aao {

void multi_destroy(aao_multi* m) {
  if (!m) return;
  if (m->batch) aao_batch_destroy(m->batch);
  for (aao_ctx* v : m->views) aao_destroy(v);
  delete m;
}

namespace {

// A view of h: copies of its scalars and tables, h's face arrays, fresh fields and Krylov spaces.
cudaError_t make_view(const aao_ctx* h, aao_ctx** out) {
  aao_ctx* v = new aao_ctx();
  v->dim = h->dim;
  for (int d = 0; d < 3; ++d) v->n[d] = h->n[d];
  v->N = h->N;
  v->L = h->L;
  v->ell = h->ell;
  v->alpha = h->alpha;
  v->prec = h->prec;
  v->p = h->p;
  std::memcpy(v->palloc, h->palloc, sizeof(v->palloc));
  v->nc2 = h->nc2;
  v->m = h->m;
  v->orth = h->orth;
  v->mu_min = h->mu_min;
  v->mu_max = h->mu_max;
  v->stream = h->stream;
  v->g = h->g;
  v->owns_coeffs = false;
  v->cx64 = h->cx64;
  v->cy64 = h->cy64;
  v->cz64 = h->cz64;
  v->cx32 = h->cx32;
  v->cy32 = h->cy32;
  v->cz32 = h->cz32;
  v->pairs = h->pairs;
  v->tma = false;
  v->scfg = h->scfg;
  v->tail = h->tail;
  v->auto_kind = h->auto_kind;
  v->steps32 = h->steps32;
  v->steps64 = h->steps64;
  v->dft32 = h->dft32;
  v->dft64 = h->dft64;
  v->idft32 = h->idft32;
  v->idft64 = h->idft64;
  v->part_cap = h->part_cap;
  const ScLayout Lsc{v->m};
  const size_t fsz = (v->prec == AAO_MIXED) ? sizeof(float) : sizeof(double);
  cudaError_t e = cudaMalloc(&v->partials, sizeof(double) * v->part_cap);
  if (e == cudaSuccess) e = cudaMalloc(&v->sc, sizeof(double) * Lsc.size());
  if (e == cudaSuccess) e = cudaMemset(v->sc, 0, sizeof(double) * Lsc.size());
  if (e == cudaSuccess) e = cudaMalloc(&v->counter, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(v->counter, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&v->tma_fault, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(v->tma_fault, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&v->pinned, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&v->bhat, fsz * v->L);
  if (e == cudaSuccess) e = cudaMalloc(&v->xa, fsz * v->L);
  if (e == cudaSuccess) e = cudaMalloc(&v->xb, fsz * v->L);
  if (e == cudaSuccess && v->pairs) e = cudaMalloc(&v->xc, fsz * v->L);
  if (e == cudaSuccess && v->pairs) e = cudaMalloc(&v->xd, fsz * v->L);
  if (e == cudaSuccess) e = cudaMalloc(&v->V, sizeof(double) * v->L * (v->m + 1));
  if (e == cudaSuccess) e = cudaMalloc(&v->Z, sizeof(double) * v->L * v->m);
  if (e != cudaSuccess) {
    aao_destroy(v);
    return e;
  }
  *out = v;
  return cudaSuccess;
}

}  // namespace

}  // namespace aao

extern "C" {

int aao_solve_multi(aao_handle h, int nrhs, const double* const* b, double* const* x, double tol, int max_outer) {
  using aao::handle_fail;
  if (!h) return handle_fail(nullptr, AAO_EINVAL, "NULL handle");
  h->err.clear();
  if (nrhs < 1 || nrhs > 256) return handle_fail(h, AAO_EINVAL, "nrhs must be in [1, 256]");
  if (!b || !x) return handle_fail(h, AAO_EINVAL, "b and x must be arrays of nrhs device pointers");
  if (h->prec != AAO_MIXED || (h->dim != 2 && h->dim != 3) || h->n[0] % 4 != 0)
    return handle_fail(h, AAO_EINVAL, "the multi-right-hand-side solve runs mixed-precision 2D or 3D grids with "
                                      "n0 %% 4 == 0");
  if (h->pmode != AAO_PRECOND_NC) return handle_fail(h, AAO_EINVAL, "the multi-right-hand-side solve runs P_NC");
  if (h->p < 3 || h->m < 2) return handle_fail(h, AAO_EINVAL, "the multi-right-hand-side solve needs inner_its >= 3 "
                                                              "and restart >= 2");
  if (h->nc2) return handle_fail(h, AAO_EINVAL, "per-frequency budgets are not run by the multi-right-hand-side solve");
  if (!(tol > 0.0 && tol < 1.0) || max_outer < 1)
    return handle_fail(h, AAO_EINVAL, "need 0 < tol < 1 and max_outer >= 1");
  for (int i = 0; i < nrhs; ++i)
    if (!aao::is_device_ptr(b[i]) || !aao::is_device_ptr(x[i]) || b[i] == x[i])
      return handle_fail(h, AAO_EINVAL, "right-hand side %d: b and x must be distinct device pointers", i);
  aao_multi* m = h->multi;
  if (m && (m->nrhs != nrhs || m->p != h->p || m->tables != (const void*)h->steps32.data())) {
    aao::multi_destroy(m);
    m = h->multi = nullptr;
  }
  if (!m) {
    m = new aao_multi();
    m->nrhs = nrhs;
    m->p = h->p;
    m->tables = h->steps32.data();
    for (int i = 0; i < nrhs; ++i) {
      aao_ctx* v = nullptr;
      const cudaError_t e = aao::make_view(h, &v);
      if (e != cudaSuccess) {
        aao::multi_destroy(m);
        return handle_fail(h, e == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA,
                           "workspace of right-hand side %d: %s", i, cudaGetErrorString(e));
      }
      m->views.push_back(v);
    }
    const int rc = aao_batch_create(&m->batch, nrhs, m->views.data(), 1);
    if (rc != AAO_OK) {
      const std::string msg = aao_last_create_error();
      aao::multi_destroy(m);
      return handle_fail(h, rc, "%s", msg.c_str());
    }
    if (h->multi_prof) {
      const int rp = aao_batch_profile_enable(m->batch, 1);
      if (rp != AAO_OK) {
        const std::string msg = aao_batch_last_error(m->batch);
        aao::multi_destroy(m);
        return handle_fail(h, rp, "%s", msg.c_str());
      }
    }
    h->multi = m;
  }
  const int rc = aao_batch_solve(m->batch, b, x, tol, max_outer);
  if (rc != AAO_OK) handle_fail(h, rc, "%s", aao_batch_last_error(m->batch));
  return rc;
}

int aao_multi_get_stats(aao_handle h, int i, aao_stats* s) {
  if (!h || !s) return aao::handle_fail(h, AAO_EINVAL, "NULL argument");
  if (!h->multi || i < 0 || i >= h->multi->nrhs)
    return aao::handle_fail(h, AAO_EINVAL, "no multi-right-hand-side solve with right-hand side %d", i);
  return aao_batch_get_stats(h->multi->batch, i, s);
}

int aao_multi_profile_enable(aao_handle h, int on) {
  if (!h) return aao::handle_fail(nullptr, AAO_EINVAL, "NULL handle");
  h->multi_prof = on != 0;
  if (!h->multi) return AAO_OK;
  const int rc = aao_batch_profile_enable(h->multi->batch, on);
  if (rc != AAO_OK) return aao::handle_fail(h, rc, "%s", aao_batch_last_error(h->multi->batch));
  return AAO_OK;
}

int aao_multi_get_profile(aao_handle h, int64_t* launches, double* ms, double* bytes) {
  if (!h) return aao::handle_fail(nullptr, AAO_EINVAL, "NULL handle");
  if (!h->multi) {
    if (launches) *launches = 0;
    if (ms) *ms = 0.0;
    if (bytes) *bytes = 0.0;
    return AAO_OK;
  }
  const int rc = aao_batch_get_profile(h->multi->batch, launches, ms, bytes);
  if (rc != AAO_OK) return aao::handle_fail(h, rc, "%s", aao_batch_last_error(h->multi->batch));
  return AAO_OK;
}

}  // extern "C"
