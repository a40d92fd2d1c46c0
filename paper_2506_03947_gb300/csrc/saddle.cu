// P_SP (Section 4): Eq. 5 with every shifted solve replaced by a fixed number of Krylov steps
// in real arithmetic, FP64, 1D, 2D and 3D grids.
//   * real shifts (frequencies 0 and ell/2): preconditioned CG on B = A - lambda I;
//   * complex shifts: MINRES on the saddle-point system S = [[Phi, Psi], [Psi, -Phi]]
//     (Phi = Im(lambda') I > 0, Psi = A - Re(lambda') I, lambda' the shift with positive
//     imaginary part: (A - lambda) x = b  <=>  (A - conj lambda) conj x = conj b), with the
//     block-diagonal preconditioner P_D = diag(Phi + Psi, Phi + Psi) (Section 4's theorem).
// The SPD blocks are applied by one V-cycle of an aggregation multigrid (the paper uses an
// algebraic multigrid, HSL_MI20, as a black box): 2 x 2 (3D: 2 x 2 x 2) aggregates, Galerkin coarse operators
// with piecewise-constant prolongation (for B = (1 + c) I + K every level is (1 + c) W + K_H,
// W the aggregate sizes, K_H with summed crossing face diffusivities), weighted Jacobi
// (omega 2/3, two sweeps before and after the coarse correction), 16 sweeps on the coarsest
// level (every side <= 4 cells).  One hierarchy serves every shift.
#include <cmath>
#include <vector>

#include "aao_internal.cuh"

namespace aao {

namespace {

constexpr double kOmega = 2.0 / 3.0;
constexpr int kNu = 2;
constexpr int kNuCoarse = 16;
constexpr int kCoarsest = 4;

struct Lvl {
  int m0, m1, m2;
  const double* w;   // cell weights (nullptr on the finest level: all 1)
  const double* kx;  // face to +x of every cell (0 on the last column)
  const double* ky;  // face to +y (0 on the last row); nullptr for 1D
  const double* kz;  // face to +z (0 on the last plane); nullptr for 1D and 2D
  __host__ __device__ int64_t n() const { return (int64_t)m0 * m1 * m2; }
};

// (i, j, k) of cell q of a level
__device__ __forceinline__ void cell_ijk(const Lvl& L, int64_t q, int& i, int& j, int& k) {
  const int64_t pl = (int64_t)L.m0 * L.m1;
  k = (int)(q / pl);
  const int64_t r = q - (int64_t)k * pl;
  j = (int)(r / L.m0);
  i = (int)(r - (int64_t)j * L.m0);
}

// Up to two planes (the u and v blocks of one saddle system, or one CG vector) per launch,
// each with its own shift c: B_c x = (1 + c) W x + K x.
struct Shifts {
  double c[2];
};

__device__ __forceinline__ double lvl_Bx(const Lvl& L, double c, const double* x, int i, int j, int k, double xc,
                                         double* diag) {
  const int64_t pl = (int64_t)L.m0 * L.m1;
  const int64_t q = (int64_t)k * pl + (int64_t)j * L.m0 + i;
  const double w = L.w ? L.w[q] : 1.0;
  double y = (1.0 + c) * w * xc;
  double d = (1.0 + c) * w;
  if (i < L.m0 - 1) {
    const double f = L.kx[q];
    y += f * (xc - x[q + 1]);
    d += f;
  }
  if (i > 0) {
    const double f = L.kx[q - 1];
    y += f * (xc - x[q - 1]);
    d += f;
  }
  if (L.ky) {
    if (j < L.m1 - 1) {
      const double f = L.ky[q];
      y += f * (xc - x[q + L.m0]);
      d += f;
    }
    if (j > 0) {
      const double f = L.ky[q - L.m0];
      y += f * (xc - x[q - L.m0]);
      d += f;
    }
  }
  if (L.kz) {
    if (k < L.m2 - 1) {
      const double f = L.kz[q];
      y += f * (xc - x[q + pl]);
      d += f;
    }
    if (k > 0) {
      const double f = L.kz[q - pl];
      y += f * (xc - x[q - pl]);
      d += f;
    }
  }
  if (diag) *diag = d;
  return y;
}

// mode 0: y = B x;  1: y = b - B x;  2 (Jacobi): y = first ? omega b / D : x + omega (b - B x) / D
__global__ void __launch_bounds__(256)
    k_lvl(Lvl L, Shifts sh, int mode, int first, const double* __restrict__ b, const double* __restrict__ x,
          double* __restrict__ y) {
  const int64_t n = L.n();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int p = blockIdx.y;
  const double c = sh.c[p];
  const double* xp = x ? x + p * n : nullptr;
  int i, j, k;
  cell_ijk(L, q, i, j, k);
  if (mode == 2 && first) {
    double d;
    lvl_Bx(L, c, b + p * n, i, j, k, 0.0, &d);  // diagonal only (x = 0)
    y[p * n + q] = kOmega * b[p * n + q] / d;
    return;
  }
  double d;
  const double bx = lvl_Bx(L, c, xp, i, j, k, xp[q], &d);
  if (mode == 0) y[p * n + q] = bx;
  else if (mode == 1) y[p * n + q] = b[p * n + q] - bx;
  else y[p * n + q] = xp[q] + kOmega * (b[p * n + q] - bx) / d;
}

// coarse b = sum of the fine residual over each aggregate (2 x 2 x 2 cells, fewer at the far
// edges and along axes of length 1); planes along blockIdx.y
__global__ void __launch_bounds__(256)
    k_restrict(Lvl f, Lvl c, const double* __restrict__ r, double* __restrict__ bc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c.n()) return;
  const int p = blockIdx.y;
  int I, J, K;
  cell_ijk(c, q, I, J, K);
  const double* rp = r + (int64_t)p * f.n();
  double s = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
        if (i < f.m0 && j < f.m1 && k < f.m2) s += rp[((int64_t)k * f.m1 + j) * f.m0 + i];
      }
  bc[(int64_t)p * c.n() + q] = s;
}

// fine x += coarse x of its aggregate
__global__ void __launch_bounds__(256)
    k_prolong_add(Lvl f, Lvl c, const double* __restrict__ xc, double* __restrict__ x) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f.n()) return;
  const int p = blockIdx.y;
  int i, j, k;
  cell_ijk(f, q, i, j, k);
  x[(int64_t)p * f.n() + q] += xc[(int64_t)p * c.n() + ((int64_t)(k / 2) * c.m1 + j / 2) * c.m0 + i / 2];
}

// coarse weights and faces of the Galerkin product (sums over aggregates / crossing faces, in
// the fine cells' order)
__global__ void __launch_bounds__(256)
    k_coarsen(Lvl f, Lvl c, double* __restrict__ w, double* __restrict__ kx, double* __restrict__ ky,
              double* __restrict__ kz) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= c.n()) return;
  int I, J, K;
  cell_ijk(c, q, I, J, K);
  auto fidx = [&](int i, int j, int k) { return ((int64_t)k * f.m1 + j) * f.m0 + i; };
  double ws = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
        if (i < f.m0 && j < f.m1 && k < f.m2) ws += f.w ? f.w[fidx(i, j, k)] : 1.0;
      }
  if (I < c.m0 - 1) {
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj) {
        const int j = 2 * J + dj, k = 2 * K + dk;
        if (j < f.m1 && k < f.m2) sx += f.kx[fidx(2 * I + 1, j, k)];
      }
  }
  if (f.ky && J < c.m1 - 1) {
    for (int dk = 0; dk < 2; ++dk)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, k = 2 * K + dk;
        if (i < f.m0 && k < f.m2) sy += f.ky[fidx(i, 2 * J + 1, k)];
      }
  }
  if (f.kz && K < c.m2 - 1) {
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj;
        if (i < f.m0 && j < f.m1) sz += f.kz[fidx(i, j, 2 * K + 1)];
      }
  }
  w[q] = ws;
  kx[q] = sx;
  if (ky) ky[q] = sy;
  if (kz) kz[q] = sz;
}

// y = a[s] x + b[s] y + c[s] z over planes grouped by sub-problem (plane p belongs to s = p / pps);
// elementwise, so y may be the same array as x
struct Coef3 {
  double a[2], b[2], c[2];
};
__global__ void __launch_bounds__(256)
    k_lin3(int64_t n, int pps, Coef3 k, const double* x, double* y, const double* z) {  // y may alias x
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int p = blockIdx.y;
  const int s = p / pps;
  const int64_t o = (int64_t)p * n + q;
  double v = k.a[s] * x[o];
  if (k.b[s] != 0.0) v += k.b[s] * y[o];
  if (z && k.c[s] != 0.0) v += k.c[s] * z[o];
  y[o] = v;
}

// su = phi zu + Psi zv, sv = Psi zu - phi zv, Psi = A - re I (finest level)
__global__ void __launch_bounds__(256)
    k_saddle(Lvl L, double phi, double re, const double* __restrict__ zu, const double* __restrict__ zv,
             double* __restrict__ su, double* __restrict__ sv) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L.n()) return;
  int i, j, k;
  cell_ijk(L, q, i, j, k);
  const double pu = lvl_Bx(L, -re, zu, i, j, k, zu[q], nullptr);
  const double pv = lvl_Bx(L, -re, zv, i, j, k, zv[q], nullptr);
  su[q] = phi * zu[q] + pv;
  sv[q] = pu - phi * zv[q];
}

// per-block partial sums of sum_p <a_p, b_p> over np planes of length n
__global__ void __launch_bounds__(256)
    k_dot(int64_t n, int np, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int p = 0; p < np; ++p)
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
      acc = fma(a[(int64_t)p * n + q], b[(int64_t)p * n + q], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct SpPlan {
  std::vector<Lvl> lv;
  std::vector<double*> owned;             // coarse-level arrays
  std::vector<double*> xa, xb, bb, rr;    // per level: two iterate buffers, right side, residual (2 planes)
  int64_t N = 0;
  double* vec = nullptr;                  // Krylov vectors, 16 x 2N
  double* part = nullptr;                 // dot partials
  double* red = nullptr;                  // reduced dots
  double* hred = nullptr;                 // pinned copy
  int nb = 0;
  long long a_products = 0;               // A applications of the last apply
};

void sp_plan_destroy(SpPlan* p) {
  if (!p) return;
  for (double* d : p->owned) cudaFree(d);
  for (auto* v : {&p->xa, &p->xb, &p->bb, &p->rr})
    for (double* d : *v) cudaFree(d);
  if (p->vec) cudaFree(p->vec);
  if (p->part) cudaFree(p->part);
  if (p->red) cudaFree(p->red);
  if (p->hred) cudaFreeHost(p->hred);
  delete p;
}

cudaError_t sp_plan_create(SpPlan** out, const GridDesc& g, int dim, const double* cx, const double* cy,
                           const double* cz, cudaStream_t s) {
  *out = nullptr;
  if (dim < 1 || dim > 3 || (dim < 3 && g.n2 != 1) || (dim == 3 && !cz)) return cudaErrorInvalidValue;
  SpPlan* p = new SpPlan();
  p->N = g.N;
  cudaError_t e = cudaSuccess;
  p->lv.push_back(Lvl{g.n0, g.n1, g.n2, nullptr, cx, dim >= 2 ? cy : nullptr, dim == 3 ? cz : nullptr});
  while (e == cudaSuccess &&
         (p->lv.back().m0 > kCoarsest || p->lv.back().m1 > kCoarsest || p->lv.back().m2 > kCoarsest)) {
    const Lvl f = p->lv.back();
    Lvl c{(f.m0 + 1) / 2, (f.m1 + 1) / 2, (f.m2 + 1) / 2, nullptr, nullptr, nullptr, nullptr};
    const int64_t nc = c.n();
    double *w = nullptr, *kx = nullptr, *ky = nullptr, *kz = nullptr;
    e = cudaMalloc(&w, sizeof(double) * nc);
    if (e == cudaSuccess) e = cudaMalloc(&kx, sizeof(double) * nc);
    if (e == cudaSuccess && f.ky) e = cudaMalloc(&ky, sizeof(double) * nc);
    if (e == cudaSuccess && f.kz) e = cudaMalloc(&kz, sizeof(double) * nc);
    for (double* d : {w, kx, ky, kz})
      if (d) p->owned.push_back(d);
    if (e != cudaSuccess) break;
    k_coarsen<<<blocks_for(nc), 256, 0, s>>>(f, c, w, kx, ky, kz);
    count_launch();
    e = cudaGetLastError();
    c.w = w;
    c.kx = kx;
    c.ky = ky;
    c.kz = kz;
    p->lv.push_back(c);
  }
  for (size_t q = 0; q < p->lv.size() && e == cudaSuccess; ++q) {
    const int64_t n = 2 * p->lv[q].n();
    double *a = nullptr, *b = nullptr, *bb = nullptr, *r = nullptr;
    e = cudaMalloc(&a, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bb, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&r, sizeof(double) * n);
    p->xa.push_back(a);
    p->xb.push_back(b);
    p->bb.push_back(bb);
    p->rr.push_back(r);
  }
  p->nb = (int)std::min<int64_t>(1024, (g.N + 255) / 256);
  if (e == cudaSuccess) e = cudaMalloc(&p->vec, sizeof(double) * 16 * 2 * g.N);
  if (e == cudaSuccess) e = cudaMalloc(&p->part, sizeof(double) * p->nb);
  if (e == cudaSuccess) e = cudaMalloc(&p->red, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&p->hred, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    sp_plan_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

namespace {

// x (level 0, np planes) = V-cycle of B_{sh} applied to b; np <= 2
cudaError_t vcycle(SpPlan* P, const Shifts& sh, int np, const double* b, double* x, cudaStream_t s) {
  const int nl = (int)P->lv.size();
  // descend: each level's right side is in bb[q] (level 0: b), smoothed iterate in xa[q]
  const double* bq = b;
  for (int q = 0; q < nl; ++q) {
    const Lvl& L = P->lv[q];
    const int64_t n = L.n();
    const dim3 grid(blocks_for(n), np);
    const int sweeps = (q == nl - 1) ? kNuCoarse : kNu;
    double* cur = P->xa[q];
    double* oth = P->xb[q];
    k_lvl<<<grid, 256, 0, s>>>(L, sh, 2, 1, bq, nullptr, cur);
    count_launch();
    for (int it = 1; it < sweeps; ++it) {
      k_lvl<<<grid, 256, 0, s>>>(L, sh, 2, 0, bq, cur, oth);
      count_launch();
      std::swap(cur, oth);
    }
    if (cur != P->xa[q]) std::swap(P->xa[q], P->xb[q]);
    if (q == nl - 1) break;
    k_lvl<<<grid, 256, 0, s>>>(L, sh, 1, 0, bq, P->xa[q], P->rr[q]);
    count_launch();
    const Lvl& C = P->lv[q + 1];
    k_restrict<<<dim3(blocks_for(C.n()), np), 256, 0, s>>>(L, C, P->rr[q], P->bb[q + 1]);
    count_launch();
    bq = P->bb[q + 1];
  }
  // ascend: correct and post-smooth
  for (int q = nl - 2; q >= 0; --q) {
    const Lvl& L = P->lv[q];
    const Lvl& C = P->lv[q + 1];
    const int64_t n = L.n();
    const dim3 grid(blocks_for(n), np);
    const double* bl = (q == 0) ? b : P->bb[q];
    k_prolong_add<<<grid, 256, 0, s>>>(L, C, P->xa[q + 1], P->xa[q]);
    count_launch();
    // post-smoothing: ping-pong between xa[q] and xb[q]; the finest level's last sweep writes x
    double* cur = P->xa[q];
    for (int it = 0; it < kNu; ++it) {
      double* dst = (q == 0 && it == kNu - 1) ? x : (cur == P->xa[q] ? P->xb[q] : P->xa[q]);
      k_lvl<<<grid, 256, 0, s>>>(L, sh, 2, 0, bl, cur, dst);
      count_launch();
      cur = dst;
    }
    if (q > 0 && cur != P->xa[q]) std::swap(P->xa[q], P->xb[q]);
  }
  if (nl == 1) return cudaMemcpyAsync(x, P->xa[0], sizeof(double) * np * P->N, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// sum over np planes of <a, b> into the pinned host value (synchronises s)
cudaError_t dot(SpPlan* P, int np, const double* a, const double* b, double* out, cudaStream_t s) {
  k_dot<<<P->nb, 256, 0, s>>>(P->N, np, a, b, P->part);
  count_launch();
  cudaError_t e = launch_reduce(P->part, 1, P->nb, P->red, 0, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->hred, P->red, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *out = P->hred[0];
  return e;
}

cudaError_t lin3(SpPlan* P, int np, double a, double b, double c, const double* x, double* y, const double* z,
                 cudaStream_t s) {
  Coef3 k{{a, a}, {b, b}, {c, c}};
  k_lin3<<<dim3(blocks_for(P->N), np), 256, 0, s>>>(P->N, np, k, x, y, z);
  count_launch();
  return cudaGetLastError();
}

#define SP_CK(call)                       \
  do {                                    \
    const cudaError_t e_ = (call);        \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

// iters steps of CG on B_c x = b (one plane), x_0 = 0, preconditioner: one V-cycle
cudaError_t pcg(SpPlan* P, double c, const double* b, double* x, int iters, cudaStream_t s) {
  const int64_t N = P->N;
  double *r = P->vec, *z = r + N, *p = z + N, *q = p + N;
  const Shifts sh{{c, c}};
  const Lvl& L0 = P->lv[0];
  SP_CK(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
  SP_CK(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  SP_CK(vcycle(P, sh, 1, r, z, s));
  SP_CK(cudaMemcpyAsync(p, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double rz = 0.0;
  SP_CK(dot(P, 1, r, z, &rz, s));
  for (int k = 0; k < iters; ++k) {
    if (rz == 0.0) break;
    k_lvl<<<dim3(blocks_for(N), 1), 256, 0, s>>>(L0, sh, 0, 0, nullptr, p, q);
    count_launch();
    P->a_products++;
    double pq = 0.0;
    SP_CK(dot(P, 1, p, q, &pq, s));
    const double a = rz / pq;
    SP_CK(lin3(P, 1, a, 1.0, 0.0, p, x, nullptr, s));   // x += a p
    SP_CK(lin3(P, 1, -a, 1.0, 0.0, q, r, nullptr, s));  // r -= a q
    if (k == iters - 1) break;
    SP_CK(vcycle(P, sh, 1, r, z, s));
    double rzn = 0.0;
    SP_CK(dot(P, 1, r, z, &rzn, s));
    SP_CK(lin3(P, 1, 1.0, rzn / rz, 0.0, z, p, nullptr, s));  // p = z + beta p
    rz = rzn;
  }
  return cudaSuccess;
}

// iters steps of preconditioned MINRES on S [u; v] = [fu; fv] (two planes f), x_0 = 0;
// S with Phi = phi I, Psi = A - re I; P_D blocks by one V-cycle of B_c, c = phi - re.
cudaError_t minres(SpPlan* P, double phi, double re, const double* f, double* x, int iters, cudaStream_t s) {
  const int64_t N = P->N, N2 = 2 * N;
  double* b = P->vec;
  double *vold = b, *v = b + N2, *vn = v + N2, *z = vn + N2, *zn = z + N2, *w = zn + N2, *wold = w + N2,
         *wn = wold + N2, *sz = wn + N2;
  const Shifts sh{{phi - re, phi - re}};
  const Lvl& L0 = P->lv[0];
  SP_CK(cudaMemsetAsync(x, 0, sizeof(double) * N2, s));
  SP_CK(cudaMemsetAsync(vold, 0, sizeof(double) * N2, s));
  SP_CK(cudaMemsetAsync(w, 0, sizeof(double) * N2, s));
  SP_CK(cudaMemsetAsync(wold, 0, sizeof(double) * N2, s));
  SP_CK(cudaMemcpyAsync(v, f, sizeof(double) * N2, cudaMemcpyDeviceToDevice, s));
  SP_CK(vcycle(P, sh, 2, v, z, s));
  double g2 = 0.0;
  SP_CK(dot(P, 2, z, v, &g2, s));
  double gamma = std::sqrt(std::max(g2, 0.0)), gamma_old = 1.0, eta = gamma;
  double s_old = 0.0, sn = 0.0, c_old = 1.0, cn = 1.0;
  for (int k = 0; k < iters; ++k) {
    if (gamma == 0.0) break;
    SP_CK(lin3(P, 2, 1.0 / gamma, 0.0, 0.0, z, z, nullptr, s));  // z /= gamma
    k_saddle<<<blocks_for(N), 256, 0, s>>>(L0, phi, re, z, z + N, sz, sz + N);
    count_launch();
    P->a_products += 2;
    double delta = 0.0;
    SP_CK(dot(P, 2, sz, z, &delta, s));
    // vn = sz - (delta/gamma) v - (gamma/gamma_old) vold
    SP_CK(cudaMemcpyAsync(vn, sz, sizeof(double) * N2, cudaMemcpyDeviceToDevice, s));
    SP_CK(lin3(P, 2, -delta / gamma, 1.0, -gamma / gamma_old, v, vn, vold, s));
    SP_CK(vcycle(P, sh, 2, vn, zn, s));
    double gn2 = 0.0;
    SP_CK(dot(P, 2, zn, vn, &gn2, s));
    const double gamma_n = std::sqrt(std::max(gn2, 0.0));
    const double a0 = cn * delta - c_old * sn * gamma;
    const double a1 = std::hypot(a0, gamma_n);
    const double a2 = sn * delta + c_old * cn * gamma;
    const double a3 = s_old * gamma;
    const double c_n = a0 / a1, s_n = gamma_n / a1;
    // wn = (z - a3 wold - a2 w) / a1; x += c_n eta wn
    SP_CK(cudaMemcpyAsync(wn, z, sizeof(double) * N2, cudaMemcpyDeviceToDevice, s));
    SP_CK(lin3(P, 2, -a3 / a1, 1.0 / a1, -a2 / a1, wold, wn, w, s));
    SP_CK(lin3(P, 2, c_n * eta, 1.0, 0.0, wn, x, nullptr, s));
    eta = -s_n * eta;
    std::swap(vold, v);  // vold <- v, v <- vn (vn's buffer becomes free)
    std::swap(v, vn);
    std::swap(z, zn);
    gamma_old = gamma;
    gamma = gamma_n;
    std::swap(wold, w);  // wold <- w, w <- wn
    std::swap(w, wn);
    c_old = cn;
    cn = c_n;
    s_old = sn;
    sn = s_n;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t sp_precond(SpPlan* P, const GridDesc& g, int ell, int iters, double* vhat, double* y, double* z,
                       const DctShifts& sh, const IdftArgs<double>& ia, cudaStream_t s) {
  const int64_t N = g.N;
  P->a_products = 0;
  double* f = P->vec + 12 * 2 * N;   // saddle right side (two planes)
  double* xs = f + 2 * N;            // saddle solution (two planes)
  // real shifts: frequency 0 (plane 0) and ell/2 (plane 1)
  SP_CK(pcg(P, -sh.lam_re[0], vhat, y, iters, s));
  SP_CK(pcg(P, -sh.lam_re[ell / 2], vhat + N, y + N, iters, s));
  for (int m = 1; m < ell / 2; ++m) {
    const double* br = vhat + (int64_t)(2 * m) * N;
    const double* bi = br + N;
    const double lr = sh.lam_re[m], li = sh.lam_im[m];
    const bool conj = li < 0.0;
    // lambda' = conj(lambda) when Im lambda < 0, b' = conj(b): right side [-Im b'; Re b']
    SP_CK(cudaMemcpyAsync(f + N, br, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));  // Re b' = Re b
    SP_CK(cudaMemcpyAsync(f, bi, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    if (!conj) SP_CK(lin3(P, 1, -1.0, 0.0, 0.0, f, f, nullptr, s));  // -Im b' = -Im b
    SP_CK(minres(P, std::fabs(li), lr, f, xs, iters, s));
    // [u; v] = [Re x'; -Im x']: x = conj(x') = u + i v when conjugated, else u - i v
    double* yr = y + (int64_t)(2 * m) * N;
    SP_CK(cudaMemcpyAsync(yr, xs, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    SP_CK(cudaMemcpyAsync(yr + N, xs + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    if (!conj) SP_CK(lin3(P, 1, -1.0, 0.0, 0.0, yr + N, yr + N, nullptr, s));
  }
  return launch_idft_planes(N, ell, y, z, ia, s);
}

long long sp_last_products(const SpPlan* P) { return P ? P->a_products : 0; }

}  // namespace aao
