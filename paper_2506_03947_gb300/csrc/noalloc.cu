// aao_precond_apply_noalloc: the preconditioner apply for callers that must
// not allocate device memory.
//
// Who needs it: an application whose device memory is owned entirely by its
// own pool (a framework's caching allocator, or a fixed memory budget in a
// GPU shared by several services) cannot let a library call cudaMalloc behind
// its back, and a latency-bound caller cannot afford the device-wide
// synchronisation that cudaMalloc/cudaFree may imply.  aao_create allocates a
// workspace, so such callers cannot hold a handle at all.  This entry point
// needs no handle and performs no allocation: every temporary it needs (the
// per-cell face coefficients, the three Chebyshev field buffers and the
// reduction partials of the Gershgorin bound) lives in one fixed array
// declared below, which every GPU that loads the library keeps until the
// process exits.
//
// The kernels are the same ones the handle path launches; only where their
// temporaries live differs.
#include "aao.h"
#include "aao_internal.cuh"

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

namespace aao {
cudaError_t launch_build_coeffs(const GridDesc& g, const double* kx, const double* ky, const double* kz,
                                double* cx, double* cy, double* cz, float* fx, float* fy, float* fz,
                                double* partials, int* bad, double* smax_out, cudaStream_t s);
int build_coeff_blocks(int64_t N);
}  // namespace aao

// The scratch: 16 MiB per device.  Its size bounds the problems this entry
// point accepts (see aao.h).  In host code the name is only a stand-in for
// the device symbol; its device address comes from cudaGetSymbolAddress.
static constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

int say(char* buf, int len, int code, const char* fmt, ...) {
  if (buf && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, (size_t)len, fmt, ap);
    va_end(ap);
  }
  return code;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch on the current device; looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Same shift, scaling and transform tables as the handle path, for one step at
// a time (no heap use): lambda_m = alpha^{1/ell} exp(-2 pi i m/ell),
// theta_m = (mu_max + mu_min)/2 - lambda_m, delta = (mu_max - mu_min)/2.
struct Tables {
  int ell, F;
  double delta;
  std::complex<double> lam[aao::kMaxF], theta[aao::kMaxF], rho_prev[aao::kMaxF];
};

void tables_init(Tables& tb, int ell, double alpha, double mu_min, double mu_max) {
  using cd = std::complex<double>;
  const double pi = 3.14159265358979323846;
  tb.ell = ell;
  tb.F = ell / 2 + 1;
  tb.delta = 0.5 * (mu_max - mu_min);
  const double root = std::pow(alpha, 1.0 / ell);
  for (int m = 0; m < tb.F; ++m) {
    tb.lam[m] = root * std::exp(cd(0.0, -2.0 * pi * m / ell));
    if (m == 0 || 2 * m == ell) tb.lam[m] = cd(tb.lam[m].real(), 0.0);
    tb.theta[m] = 0.5 * (mu_max + mu_min) - tb.lam[m];
    tb.rho_prev[m] = tb.delta / tb.theta[m];
  }
}

// Coefficients of step k; must be called for k = 0, 1, 2, ... in order.
template <typename T>
void tables_step(Tables& tb, int k, aao::StepArgs<T>& s) {
  using cd = std::complex<double>;
  s = aao::StepArgs<T>{};
  for (int m = 0; m < tb.F; ++m) {
    cd a(0.0, 0.0), gk(0.0, 0.0);
    if (k >= 1 && tb.delta == 0.0) {
      gk = 1.0 / tb.theta[m];
    } else if (k >= 1) {
      const cd rho = 1.0 / (2.0 * tb.theta[m] / tb.delta - tb.rho_prev[m]);
      a = rho * tb.rho_prev[m];
      gk = 2.0 * rho / tb.delta;
      tb.rho_prev[m] = rho;
    }
    const cd it = 1.0 / tb.theta[m];
    s.lam_re[m] = (T)tb.lam[m].real();
    s.lam_im[m] = (T)tb.lam[m].imag();
    s.a_re[m] = (T)a.real();
    s.a_im[m] = (T)a.imag();
    s.g_re[m] = (T)gk.real();
    s.g_im[m] = (T)gk.imag();
    s.it_re[m] = (T)it.real();
    s.it_im[m] = (T)it.imag();
  }
}

template <typename T>
void transform_tables(int ell, double alpha, aao::DftArgs<T>& da, aao::IdftArgs<T>& ia) {
  const double pi = 3.14159265358979323846;
  const double isq = 1.0 / std::sqrt((double)ell);
  da = aao::DftArgs<T>{};
  ia = aao::IdftArgs<T>{};
  for (int t = 0; t < ell; ++t) {
    da.gamma[t] = std::pow(alpha, (double)t / ell);
    ia.igamma[t] = std::pow(alpha, -(double)t / ell);
    ia.igamma_T[t] = (T)ia.igamma[t];
    for (int m = 0; m <= ell / 2; ++m) {
      const double ang = 2.0 * pi * (double)((t * m) % ell) / ell;
      da.cf[t][m] = (T)(std::cos(ang) * isq);
      da.sf[t][m] = (T)(std::sin(ang) * isq);
      if (m == 0) {
        ia.ci[t][m] = (T)isq;
      } else if (2 * m == ell) {
        ia.ci[t][m] = (T)((t % 2 == 0) ? isq : -isq);
      } else {
        ia.ci[t][m] = (T)(2.0 * std::cos(ang) * isq);
        ia.si[t][m] = (T)(2.0 * std::sin(ang) * isq);
      }
    }
  }
}

template <typename T>
cudaError_t run_apply(const aao::GridDesc& g, int dim, int ell, double alpha, int p, double mu_min, double mu_max,
                      const T* cx, const T* cy, const T* cz, T* bhat, T* xa, T* xb, const double* r, double* z,
                      cudaStream_t s) {
  Tables tb;
  tables_init(tb, ell, alpha, mu_min, mu_max);
  aao::DftArgs<T> da;
  aao::IdftArgs<T> ia;
  transform_tables<T>(ell, alpha, da, ia);
  aao::StepArgs<T> st;
  tables_step<T>(tb, 0, st);
  cudaError_t e;
  if (p == 1) return aao::launch_direct<T>(g, dim, ell, r, nullptr, z, da, st, ia, s);
  if ((e = aao::launch_dft<T>(g, dim, ell, r, nullptr, bhat, da, s)) != cudaSuccess) return e;
  tables_step<T>(tb, 1, st);
  if ((e = aao::launch_step<T>(g, dim, ell, 0, 0, p == 2, cx, cy, cz, bhat, nullptr, xa, z, st, ia, s)) != cudaSuccess)
    return e;
  if (p >= 3) {
    tables_step<T>(tb, 2, st);
    if ((e = aao::launch_step<T>(g, dim, ell, 1, 1, p == 3, cx, cy, cz, bhat, xa, xb, z, st, ia, s)) != cudaSuccess)
      return e;
  }
  for (int k = 3; k <= p - 1; ++k) {
    tables_step<T>(tb, k, st);
    T* cur = (k % 2 == 1) ? xb : xa;
    T* prev = (k % 2 == 1) ? xa : xb;
    if ((e = aao::launch_step<T>(g, dim, ell, 1, 2, k == p - 1, cx, cy, cz, bhat, cur, prev, z, st, ia, s)) !=
        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" int aao_precond_apply_noalloc(int dim, const int64_t n[3], const double* kx, const double* ky,
                                         const double* kz, int ell, double alpha, int prec, int inner_its,
                                         double mu_max, const double* r, double* z, void* stream, char* err,
                                         int err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (dim < 1 || dim > 3 || !n) return say(err, err_len, AAO_EINVAL, "dim must be 1, 2 or 3 and n non-NULL");
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1) return say(err, err_len, AAO_EINVAL, "n[%d] must be >= 1", d);
    if (d >= dim && n[d] != 1) return say(err, err_len, AAO_EINVAL, "n[%d] must be 1 for dim = %d", d, dim);
  }
  if (n[0] > 2000000000LL || n[1] > 8LL * 65535 || n[2] > 65535)
    return say(err, err_len, AAO_EINVAL, "grid too large");
  if (ell < 4 || ell > AAO_MAX_ELL || ell % 2)
    return say(err, err_len, AAO_EINVAL, "ell must be even and in [4, %d]", AAO_MAX_ELL);
  if (!(alpha > 0.0 && alpha < 1.0)) return say(err, err_len, AAO_EINVAL, "alpha must satisfy 0 < alpha < 1");
  if (prec != AAO_FP64 && prec != AAO_MIXED) return say(err, err_len, AAO_EINVAL, "bad precision mode");
  if (inner_its < 1 || inner_its > 100000) return say(err, err_len, AAO_EINVAL, "inner_its must be in [1, 100000]");
  if (!(mu_max >= 0.0) || !std::isfinite(mu_max) || (mu_max > 0.0 && mu_max <= 1.0))
    return say(err, err_len, AAO_EINVAL, "mu_max must be 0 (Gershgorin bound) or > 1");
  const double* fk[3] = {kx, ky, kz};
  for (int d = 0; d < 3; ++d)
    if (n[d] > 1 && !on_device(fk[d]))
      return say(err, err_len, AAO_EINVAL, "face array %d must be a device pointer", d);
  if (!on_device(r) || !on_device(z) || r == z)
    return say(err, err_len, AAO_EINVAL, "r and z must be distinct device pointers");

  const int64_t N = n[0] * n[1] * n[2];
  const int64_t L = (int64_t)ell * N;
  const size_t Ts = (prec == AAO_MIXED) ? sizeof(float) : sizeof(double);
  const int nb = aao::build_coeff_blocks(N);
  // layout of the scratch: FP64 coefficients, FP32 coefficients, partials, flag, fields
  const size_t off_c64 = 0;
  const size_t off_c32 = off_c64 + 3 * align256(sizeof(double) * (size_t)N);
  const size_t off_part = off_c32 + 3 * align256(sizeof(float) * (size_t)N);
  const size_t off_flag = off_part + align256(sizeof(double) * ((size_t)nb + 1));
  const size_t off_field = off_flag + 256;
  const size_t need = off_field + 3 * align256(Ts * (size_t)L);
  if (need > kNoallocScratchBytes)
    return say(err, err_len, AAO_EINVAL,
               "problem needs %zu bytes of scratch (ell*N = %lld, %s); the allocation-free entry point holds "
               "%zu bytes",
               need, (long long)L, prec == AAO_MIXED ? "mixed" : "fp64", kNoallocScratchBytes);

  void* base_v = nullptr;
  cudaError_t e = scratch_address(&base_v);
  if (e != cudaSuccess) return say(err, err_len, AAO_ECUDA, "scratch address: %s", cudaGetErrorString(e));
  unsigned char* base = (unsigned char*)base_v;
  cudaStream_t s = (cudaStream_t)stream;
  double* c64[3];
  float* c32[3];
  for (int d = 0; d < 3; ++d) {
    c64[d] = (double*)(base + off_c64 + d * align256(sizeof(double) * (size_t)N));
    c32[d] = (float*)(base + off_c32 + d * align256(sizeof(float) * (size_t)N));
  }
  double* partials = (double*)(base + off_part);
  double* smax_dev = partials + nb;
  int* bad = (int*)(base + off_flag);
  unsigned char* fields = base + off_field;

  aao::GridDesc g;
  g.n0 = (int)n[0];
  g.n1 = (int)n[1];
  g.n2 = (int)n[2];
  g.N = N;
  // the flag must start at zero on every call (the scratch keeps the last call's contents)
  e = cudaMemsetAsync(bad, 0, sizeof(int) * 2, s);
  if (e == cudaSuccess)
    e = aao::launch_build_coeffs(g, kx, ky, kz, c64[0], c64[1], c64[2], c32[0], c32[1], c32[2], partials, bad,
                                 smax_dev, s);
  int hbad[2] = {0, 0};
  double smax = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hbad, bad, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&smax, smax_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(err, err_len, AAO_ECUDA, "coefficient set-up: %s", cudaGetErrorString(e));
  if (hbad[0]) return say(err, err_len, AAO_EINVAL, "face diffusivities must be finite and > 0");
  const double mu_min = 1.0;
  double mmax = mu_max > 0.0 ? mu_max : 1.0 + 2.0 * smax;
  if (!(mmax >= mu_min)) mmax = mu_min;

  if (prec == AAO_MIXED) {
    float* f0 = (float*)fields;
    float* f1 = (float*)(fields + align256(Ts * (size_t)L));
    float* f2 = (float*)(fields + 2 * align256(Ts * (size_t)L));
    e = run_apply<float>(g, dim, ell, alpha, inner_its, mu_min, mmax, c32[0], c32[1], c32[2], f0, f1, f2, r, z, s);
  } else {
    double* f0 = (double*)fields;
    double* f1 = (double*)(fields + align256(Ts * (size_t)L));
    double* f2 = (double*)(fields + 2 * align256(Ts * (size_t)L));
    e = run_apply<double>(g, dim, ell, alpha, inner_its, mu_min, mmax, c64[0], c64[1], c64[2], f0, f1, f2, r, z, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(err, err_len, AAO_ECUDA, "preconditioner kernels: %s", cudaGetErrorString(e));
  return AAO_OK;
}
