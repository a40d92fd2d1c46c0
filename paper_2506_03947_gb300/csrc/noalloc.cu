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
// It runs the method's steps one Chebyshev step per launch (the transform, the
// single-step sweep kernels and the sweep fused with the inverse transform).  A
// handle fuses several steps per launch on 2D grids in mixed precision, so the
// two results agree to rounding, not bit for bit.
#include "aao.h"
#include "aao_internal.cuh"
#include "host_tables.h"

#include <cmath>
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

// Device memory of the current device, or managed memory.  Memory of another GPU is refused:
// the kernels run on the current device, and without peer access its addresses are not
// reachable from there.
bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
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

// The shift, scaling and transform tables come from the same host builder as the handle
// path's (host_tables.h), one step at a time.
template <typename T>
struct Narrow;
template <>
struct Narrow<double> {
  static const aao::StepArgs<double>& step(const aao::StepArgs<double>& s) { return s; }
  static void transforms(const aao::DftArgs<double>& da, const aao::IdftArgs<double>& ia, aao::DftArgs<double>& oa,
                         aao::IdftArgs<double>& oi) {
    oa = da;
    oi = ia;
  }
};
template <>
struct Narrow<float> {
  static aao::StepArgs<float> step(const aao::StepArgs<double>& s) { return aao::narrow_step(s); }
  static void transforms(const aao::DftArgs<double>& da, const aao::IdftArgs<double>& ia, aao::DftArgs<float>& oa,
                         aao::IdftArgs<float>& oi) {
    aao::narrow_transforms(da, ia, oa, oi);
  }
};

template <typename T>
cudaError_t run_apply(const aao::GridDesc& g, int dim, int ell, double alpha, int p, double mu_min, double mu_max,
                      const T* cx, const T* cy, const T* cz, T* bhat, T* xa, T* xb, const double* r, double* z,
                      cudaStream_t s) {
  aao::ChebTables tb;
  aao::cheb_tables_init(tb, ell, alpha, mu_min, mu_max);
  aao::DftArgs<double> da64;
  aao::IdftArgs<double> ia64;
  aao::transform_tables(ell, alpha, da64, ia64);
  aao::DftArgs<T> da;
  aao::IdftArgs<T> ia;
  Narrow<T>::transforms(da64, ia64, da, ia);
  aao::StepArgs<double> s64;
  auto step = [&](int k) {
    aao::cheb_tables_step(tb, k, nullptr, s64);
    return Narrow<T>::step(s64);
  };
  cudaError_t e;
  aao::StepArgs<T> st = step(0);
  if (p == 1) return aao::launch_direct<T>(g, dim, ell, r, nullptr, z, da, st, ia, s);
  if ((e = aao::launch_dft<T>(g, dim, ell, r, nullptr, bhat, da, s)) != cudaSuccess) return e;
  st = step(1);
  if ((e = aao::launch_step<T>(g, dim, ell, 0, 0, p == 2, cx, cy, cz, bhat, nullptr, xa, z, st, ia, s)) != cudaSuccess)
    return e;
  if (p >= 3) {
    st = step(2);
    if ((e = aao::launch_step<T>(g, dim, ell, 1, 1, p == 3, cx, cy, cz, bhat, xa, xb, z, st, ia, s)) != cudaSuccess)
      return e;
  }
  for (int k = 3; k <= p - 1; ++k) {
    st = step(k);
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
  // N within the array before any size arithmetic (no product below can wrap)
  int64_t N = 0;
  if (__builtin_mul_overflow(n[0], n[1], &N) || __builtin_mul_overflow(N, n[2], &N) ||
      N > (int64_t)(kNoallocScratchBytes / sizeof(float)))
    return say(err, err_len, AAO_EINVAL,
               "problem needs more scratch than the %zu bytes the allocation-free entry point holds "
               "(n = %lld x %lld x %lld)",
               kNoallocScratchBytes, (long long)n[0], (long long)n[1], (long long)n[2]);
  const double* fk[3] = {kx, ky, kz};
  for (int d = 0; d < 3; ++d)
    if (n[d] > 1 && !on_device(fk[d]))
      return say(err, err_len, AAO_EINVAL, "face array %d must be a device pointer on the current device", d);
  if (!on_device(r) || !on_device(z) || r == z)
    return say(err, err_len, AAO_EINVAL, "r and z must be distinct device pointers on the current device");
  // r is read element by element; z is written two doubles at a time by the inverse transform
  if ((reinterpret_cast<uintptr_t>(r) & 7) != 0 || (reinterpret_cast<uintptr_t>(z) & 15) != 0)
    return say(err, err_len, AAO_EINVAL, "r must be 8-byte and z 16-byte aligned");

  const int64_t L = (int64_t)ell * N;
  const size_t Ts = (prec == AAO_MIXED) ? sizeof(float) : sizeof(double);
  const size_t To = (prec == AAO_MIXED) ? sizeof(double) : sizeof(float);
  const int nb = aao::build_coeff_blocks(N);
  // layout of the scratch: the coefficients of the path's precision, partials, flag, fields.
  // The set-up kernel also writes the other precision's copy; that copy is dead before the
  // first field is written, so it sits at the start of the field region.
  const size_t off_cu = 0;
  const size_t off_part = off_cu + 3 * align256(Ts * (size_t)N);
  const size_t off_flag = off_part + align256(sizeof(double) * ((size_t)nb + 1));
  const size_t off_field = off_flag + 256;
  const size_t field_bytes = 3 * align256(Ts * (size_t)L);
  const size_t other_bytes = 3 * align256(To * (size_t)N);
  const size_t need = off_field + (field_bytes > other_bytes ? field_bytes : other_bytes);
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
  const size_t off_c64 = (prec == AAO_MIXED) ? off_field : off_cu;
  const size_t off_c32 = (prec == AAO_MIXED) ? off_cu : off_field;
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
