// Exact (best-case) P_alpha^{-1} for spatially constant face diffusivities, FP64.
//
// Section 2.2: with A = X Phi X^T, Eq. 5 becomes
//   P_alpha^{-1} = (Gamma^{-1} U (x) I)(I (x) X)(I (x) Phi - Lambda (x) I)^{-1}(I (x) X^T)(U* Gamma (x) I).
// For the finite-volume Neumann operator with diffusivity kappa_a on every face of axis a,
// X is the orthonormal DCT-II along each axis and Phi = 1 + sum_a kappa_a 4 sin^2(pi k_a / (2 n_a)).
// The apply is: the time DFT (the path's own kernel), the spatial DCT of every frequency plane
// (each of the ell packed planes is a real field: the transform acts on Re and Im parts alike),
// the division by (phi - lambda_m) per cell and frequency, the inverse DCT, and the inverse
// time DFT with Gamma^{-1}.  This is the comparison preconditioner of the paper's experiments
// ("best case"), not part of the inner Chebyshev path.
//
// The spatial transforms are this library's kernels, one launch per axis, in place: a block
// loads a few whole lines of the axis into shared memory and transforms them.
//  * Power-of-two lengths: the orthonormal DCT-II of a real line x through one complex FFT of
//    the same length (Makhoul, IEEE Trans. ASSP 28(1), 1980): v = (x_0, x_2, ..., x_3, x_1)
//    (even entries, then odd entries reversed), V = FFT(v), y_k = c_k Re(e^{-i pi k/(2n)} V_k),
//    c_0 = sqrt(1/n), c_k = sqrt(2/n).  The inverse (DCT-III) builds
//    V_k = e^{i pi k/(2n)} (y_k/c_k - i y_{n-k}/c_{n-k}) (y_n = 0), v = IFFT(V) (real) and undoes
//    the reordering.  The FFT is radix-2 in shared memory with FP64 twiddles from the host.
//    O(n log n) per line instead of the O(n^2) of a dense product.
//  * Other lengths: the direct sums y_k = sum_j C_kj x_j (inverse: x_j = sum_k C_kj y_k) with the
//    orthonormal DCT-II matrix C_kj = c_k cos(pi k (2j + 1)/(2n)) from the host.
#include <cmath>
#include <cstring>
#include <vector>

#include "aao_internal.cuh"

namespace aao {

namespace {

// y = v / (phi - lambda_m) on the packed frequency planes (plane 0: m = 0, plane 1: m = ell/2,
// planes 2m, 2m+1: Re, Im of m); phi from the per-axis eigenvalue parts.
__global__ void __launch_bounds__(256)
    k_dct_divide(GridDesc g, int ell, const double* __restrict__ ex, const double* __restrict__ ey,
                 const double* __restrict__ ez, double* __restrict__ v, DctShifts sh) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const int i = (int)(c % g.n0);
  const int64_t r = c / g.n0;
  const int j = (int)(r % g.n1);
  const int k = (int)(r / g.n1);
  const double phi = 1.0 + ex[i] + (ey ? ey[j] : 0.0) + (ez ? ez[k] : 0.0);
  const int64_t N = g.N;
  v[c] = v[c] / (phi - sh.lam_re[0]);
  v[N + c] = v[N + c] / (phi - sh.lam_re[ell / 2]);
  for (int m = 1; m < ell / 2; ++m) {
    const double dr = phi - sh.lam_re[m], di = -sh.lam_im[m];
    const double den = dr * dr + di * di;
    const double vr = v[(int64_t)(2 * m) * N + c], vi = v[(int64_t)(2 * m + 1) * N + c];
    // (vr + i vi) / (dr + i di) = ((vr dr + vi di) + i (vi dr - vr di)) / (dr^2 + di^2)
    v[(int64_t)(2 * m) * N + c] = (vr * dr + vi * di) / den;
    v[(int64_t)(2 * m + 1) * N + c] = (vi * dr - vr * di) / den;
  }
}

// z_t = igamma_t sum_m (Re y_m ci[t][m] - Im y_m si[t][m]) from the packed planes.
__global__ void __launch_bounds__(256)
    k_idft_planes(int64_t N, int ell, const double* __restrict__ y, double* __restrict__ z,
                  const __grid_constant__ IdftArgs<double> ia) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double fre[kMaxF], fim[kMaxF];
  fre[0] = y[c];
  fim[0] = 0.0;
  fre[ell / 2] = y[N + c];
  fim[ell / 2] = 0.0;
  for (int m = 1; m < ell / 2; ++m) {
    fre[m] = y[(int64_t)(2 * m) * N + c];
    fim[m] = y[(int64_t)(2 * m + 1) * N + c];
  }
  for (int t = 0; t < ell; ++t) {
    double acc = 0.0;
    for (int m = 0; m <= ell / 2; ++m) acc += fre[m] * ia.ci[t][m] - fim[m] * ia.si[t][m];
    z[(int64_t)t * N + c] = acc * ia.igamma[t];
  }
}

}  // namespace

namespace {

// Lines of one axis: a field of `planes` planes of N values, each plane seen as
// [outer][n][inner] (x: inner 1, y: inner n0, z: inner n0 n1); line (p, o, i) has its values at
// p N + o n inner + i + j inner, j < n.  A block takes `per` lines with consecutive (p, o, i),
// i fastest, so that for inner > 1 the block's loads of one j are contiguous.
struct AxisLines {
  int n, inner, outer, per;
  int64_t N;
  int64_t total;  // planes * outer * inner lines
};

__device__ __forceinline__ int64_t line_base(const AxisLines& a, int64_t l) {
  const int64_t i = l % a.inner;
  const int64_t r = l / a.inner;
  const int64_t o = r % a.outer;
  const int64_t p = r / a.outer;
  return p * a.N + o * (int64_t)a.n * a.inner + i;
}

__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// Orthonormal DCT-II (INV = false) or DCT-III (INV = true) of the block's lines, power-of-two n.
// Shared memory: per line n complex values (the FFT) and n reals (the input line).
// tw[k] = exp(-2 pi i k / n), k < n/2; rot[k] = exp(-i pi k / (2n)), k < n.
template <bool INV>
__global__ void __launch_bounds__(256) k_dct_axis_fft(double* __restrict__ v, AxisLines a, int bits,
                                                      const double2* __restrict__ tw,
                                                      const double2* __restrict__ rot) {
  extern __shared__ double2 dsm[];
  const int n = a.n, per = a.per;
  double2* buf = dsm;                                                  // [per][n]
  double* lin = reinterpret_cast<double*>(dsm + (size_t)per * n);      // [per][n]
  const int64_t l0 = (int64_t)blockIdx.x * per;
  const int nl = (int)((a.total - l0) < per ? (a.total - l0) : per);
  const double sq1 = sqrt(1.0 / n), sq2 = sqrt(2.0 / n);
  // load the lines (j outer, line inner: contiguous when inner > 1)
  for (int idx = threadIdx.x; idx < per * n; idx += blockDim.x) {
    const int ll = (a.inner > 1) ? idx % per : idx / n;
    const int j = (a.inner > 1) ? idx / per : idx % n;
    if (ll < nl) lin[ll * n + j] = v[line_base(a, l0 + ll) + (int64_t)j * a.inner];
  }
  __syncthreads();
  // FFT input in bit-reversed order
  for (int idx = threadIdx.x; idx < per * n; idx += blockDim.x) {
    const int ll = idx / n, k = idx % n;
    if (ll >= nl) continue;
    const double* x = lin + ll * n;
    double2 val;
    if (!INV) {
      // v_k: even entries, then odd entries reversed
      const double xv = (k < n / 2) ? x[2 * k] : x[2 * (n - 1 - k) + 1];
      val = make_double2(xv, 0.0);
    } else {
      // V_k = e^{i pi k/(2n)} (Y_k - i Y_{n-k}),  Y_k = y_k / c_k,  Y_n = 0
      const double yk = x[k] / (k == 0 ? sq1 : sq2);
      const double ynk = (k == 0) ? 0.0 : x[n - k] / sq2;
      const double2 r = rot[k];  // e^{-i pi k/(2n)}: use its conjugate
      const double cr = r.x, ci = -r.y;
      // (cr + i ci)(yk - i ynk)
      val = make_double2(cr * yk + ci * ynk, ci * yk - cr * ynk);
    }
    buf[ll * n + bitrev((unsigned)k, bits)] = val;
  }
  __syncthreads();
  // radix-2 stages
  for (int s = 1; s <= bits; ++s) {
    const int half = 1 << (s - 1);
    const int stride = n >> s;  // twiddle index step
    for (int idx = threadIdx.x; idx < per * (n / 2); idx += blockDim.x) {
      const int ll = idx / (n / 2), b = idx % (n / 2);
      if (ll >= nl) continue;
      const int grp = b / half, pos = b % half;
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      double2 w = tw[pos * stride];
      if (INV) w.y = -w.y;
      double2* line = buf + ll * n;
      const double2 u = line[i0], t = line[i1];
      const double2 wt = make_double2(w.x * t.x - w.y * t.y, w.x * t.y + w.y * t.x);
      line[i0] = make_double2(u.x + wt.x, u.y + wt.y);
      line[i1] = make_double2(u.x - wt.x, u.y - wt.y);
    }
    __syncthreads();
  }
  // outputs
  for (int idx = threadIdx.x; idx < per * n; idx += blockDim.x) {
    const int ll = (a.inner > 1) ? idx % per : idx / n;
    const int j = (a.inner > 1) ? idx / per : idx % n;
    if (ll >= nl) continue;
    const double2* V = buf + ll * n;
    double out;
    if (!INV) {
      // y_j = c_j Re(e^{-i pi j/(2n)} V_j)
      const double2 r = rot[j];
      out = (j == 0 ? sq1 : sq2) * (r.x * V[j].x - r.y * V[j].y);
    } else {
      // x_{2m} = v_m, x_{2m+1} = v_{n-1-m}, v = IFFT(V) = (1/n) sum_k V_k e^{+2 pi i m k/n}
      const int m = (j % 2 == 0) ? j / 2 : n - 1 - j / 2;
      out = V[m].x / n;
    }
    v[line_base(a, l0 + ll) + (int64_t)j * a.inner] = out;
  }
}

// Direct sums for any n: y_k = sum_j C_kj x_j (INV = false) or x_j = sum_k C_kj y_k (INV = true),
// C row-major n x n (C[k n + j]).
template <bool INV>
__global__ void __launch_bounds__(256) k_dct_axis_direct(double* __restrict__ v, AxisLines a,
                                                         const double* __restrict__ C) {
  extern __shared__ double2 dsm[];
  double* lin = reinterpret_cast<double*>(dsm);  // [per][n]
  const int n = a.n, per = a.per;
  const int64_t l0 = (int64_t)blockIdx.x * per;
  const int nl = (int)((a.total - l0) < per ? (a.total - l0) : per);
  for (int idx = threadIdx.x; idx < per * n; idx += blockDim.x) {
    const int ll = (a.inner > 1) ? idx % per : idx / n;
    const int j = (a.inner > 1) ? idx / per : idx % n;
    if (ll < nl) lin[ll * n + j] = v[line_base(a, l0 + ll) + (int64_t)j * a.inner];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < per * n; idx += blockDim.x) {
    const int ll = (a.inner > 1) ? idx % per : idx / n;
    const int k = (a.inner > 1) ? idx / per : idx % n;
    if (ll >= nl) continue;
    const double* x = lin + ll * n;
    double acc = 0.0;
    if (!INV)
      for (int j = 0; j < n; ++j) acc = fma(C[(int64_t)k * n + j], x[j], acc);
    else
      for (int j = 0; j < n; ++j) acc = fma(C[(int64_t)j * n + k], x[j], acc);
    v[line_base(a, l0 + ll) + (int64_t)k * a.inner] = acc;
  }
}

}  // namespace

struct DctPlan {
  int dim = 0;
  int n[3] = {1, 1, 1};
  int bits[3] = {0, 0, 0};                      // log2 n for power-of-two axes, else 0
  double2* tw[3] = {nullptr, nullptr, nullptr};   // exp(-2 pi i k/n), k < n/2
  double2* rot[3] = {nullptr, nullptr, nullptr};  // exp(-i pi k/(2n)), k < n
  double* C[3] = {nullptr, nullptr, nullptr};     // row-major DCT-II matrix (other lengths)
  double* ev[3] = {nullptr, nullptr, nullptr};    // kappa_a 4 sin^2(pi k / (2 n_a))
};

void dct_plan_destroy(DctPlan* p) {
  if (!p) return;
  for (int a = 0; a < 3; ++a) {
    if (p->tw[a]) cudaFree(p->tw[a]);
    if (p->rot[a]) cudaFree(p->rot[a]);
    if (p->C[a]) cudaFree(p->C[a]);
    if (p->ev[a]) cudaFree(p->ev[a]);
  }
  delete p;
}

cudaError_t dct_plan_create(DctPlan** out, const GridDesc& g, int dim, int ell, const double kappa[3]) {
  (void)ell;
  *out = nullptr;
  DctPlan* p = new DctPlan();
  p->dim = dim;
  p->n[0] = g.n0;
  p->n[1] = g.n1;
  p->n[2] = g.n2;
  cudaError_t e = cudaSuccess;
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < dim && e == cudaSuccess; ++a) {
    const int n = p->n[a];
    std::vector<double> ev(n);
    for (int k = 0; k < n; ++k) {
      const double sn = std::sin(pi * k / (2.0 * n));
      ev[k] = kappa[a] * 4.0 * sn * sn;
    }
    e = cudaMalloc(&p->ev[a], sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->ev[a], ev.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    const bool pow2 = n >= 2 && (n & (n - 1)) == 0 && n <= 4096;
    if (pow2) {
      int b = 0;
      while ((1 << b) < n) ++b;
      p->bits[a] = b;
      std::vector<double2> tw(n / 2), rot(n);
      for (int k = 0; k < n / 2; ++k) tw[k] = make_double2(std::cos(2.0 * pi * k / n), -std::sin(2.0 * pi * k / n));
      for (int k = 0; k < n; ++k) rot[k] = make_double2(std::cos(pi * k / (2.0 * n)), -std::sin(pi * k / (2.0 * n)));
      if (e == cudaSuccess) e = cudaMalloc(&p->tw[a], sizeof(double2) * tw.size());
      if (e == cudaSuccess) e = cudaMemcpy(p->tw[a], tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMalloc(&p->rot[a], sizeof(double2) * rot.size());
      if (e == cudaSuccess) e = cudaMemcpy(p->rot[a], rot.data(), sizeof(double2) * rot.size(), cudaMemcpyHostToDevice);
    } else {
      std::vector<double> C((size_t)n * n);
      for (int k = 0; k < n; ++k) {
        const double c = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
        for (int j = 0; j < n; ++j) C[(size_t)k * n + j] = c * std::cos(pi * k * (2.0 * j + 1.0) / (2.0 * n));
      }
      if (e == cudaSuccess) e = cudaMalloc(&p->C[a], sizeof(double) * C.size());
      if (e == cudaSuccess) e = cudaMemcpy(p->C[a], C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) {
    dct_plan_destroy(p);
    return e;
  }
  *out = p;
  return cudaSuccess;
}

// Spatial DCT (inverse = false) or its inverse of every plane of v (ell planes of N), in place,
// one launch per axis.
static cudaError_t dct_planes(DctPlan* p, int ell, double* v, bool inverse, cudaStream_t s) {
  const int64_t N = (int64_t)p->n[0] * p->n[1] * p->n[2];
  for (int a = 0; a < p->dim; ++a) {
    AxisLines al;
    al.n = p->n[a];
    al.inner = (a == 0) ? 1 : (a == 1 ? p->n[0] : p->n[0] * p->n[1]);
    al.outer = (a == 0) ? p->n[1] * p->n[2] : (a == 1 ? p->n[2] : 1);
    al.N = N;
    al.total = (int64_t)ell * al.outer * al.inner;
    const bool fft = p->bits[a] > 0;
    const size_t per_line = fft ? (size_t)al.n * (sizeof(double2) + sizeof(double)) : (size_t)al.n * sizeof(double);
    int per = (int)(96 * 1024 / per_line);
    if (per < 1) per = 1;
    if (per > 32) per = 32;
    if ((int64_t)per > al.total) per = (int)al.total;
    al.per = per;
    const size_t smem = per_line * per;
    const unsigned grid = (unsigned)((al.total + per - 1) / per);
    cudaError_t e;
    if (fft) {
      auto k = inverse ? k_dct_axis_fft<true> : k_dct_axis_fft<false>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, 256, smem, s>>>(v, al, p->bits[a], p->tw[a], p->rot[a]);
    } else {
      auto k = inverse ? k_dct_axis_direct<true> : k_dct_axis_direct<false>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, 256, smem, s>>>(v, al, p->C[a]);
    }
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t dct_precond(DctPlan* p, const GridDesc& g, int ell, double* vhat, double* z, const DctShifts& sh,
                        const IdftArgs<double>& ia, cudaStream_t s) {
  cudaError_t e = dct_planes(p, ell, vhat, false, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((g.N + 255) / 256);
  k_dct_divide<<<grid, 256, 0, s>>>(g, ell, p->ev[0], p->dim >= 2 ? p->ev[1] : nullptr,
                                    p->dim == 3 ? p->ev[2] : nullptr, vhat, sh);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = dct_planes(p, ell, vhat, true, s);
  if (e != cudaSuccess) return e;
  k_idft_planes<<<grid, 256, 0, s>>>(g.N, ell, vhat, z, ia);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_idft_planes(int64_t N, int ell, const double* y, double* z, const IdftArgs<double>& ia,
                               cudaStream_t s) {
  k_idft_planes<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, ell, y, z, ia);
  count_launch();
  return cudaGetLastError();
}

// Per-axis minimum and maximum of the interior faces (as ordered bit patterns of positive
// doubles); slots 2a, 2a+1 of mm hold min and max of axis a.
__global__ void k_face_range(GridDesc g, const double* __restrict__ cx, const double* __restrict__ cy,
                             const double* __restrict__ cz, unsigned long long* mm) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  const int i = (int)(c % g.n0);
  const int64_t r = c / g.n0;
  const int j = (int)(r % g.n1);
  const int k = (int)(r / g.n1);
  if (i < g.n0 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cx[c]);
    atomicMin(&mm[0], b);
    atomicMax(&mm[1], b);
  }
  if (cy && j < g.n1 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cy[c]);
    atomicMin(&mm[2], b);
    atomicMax(&mm[3], b);
  }
  if (cz && k < g.n2 - 1) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(cz[c]);
    atomicMin(&mm[4], b);
    atomicMax(&mm[5], b);
  }
}

cudaError_t face_ranges(const GridDesc& g, const double* cx, const double* cy, const double* cz, double out[6],
                        cudaStream_t s) {
  unsigned long long* mm = nullptr;
  cudaError_t e = cudaMalloc(&mm, sizeof(unsigned long long) * 6);
  unsigned long long init[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_face_range<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, cx, cy, cz, mm);
    count_launch();
    e = cudaGetLastError();
  }
  unsigned long long hb[6] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb, mm, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (mm) cudaFree(mm);
  for (int q = 0; q < 6; ++q) {
    const bool none = (q % 2 == 0) ? hb[q] == ~0ull : false;
    double v = 0.0;
    std::memcpy(&v, &hb[q], sizeof(double));
    out[q] = none ? 0.0 : v;
  }
  return e;
}

}  // namespace aao
