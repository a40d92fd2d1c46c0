// Internal declarations shared by the CUDA translation units of libaao.
//
// Device data layouts:
//  * FP64 block vectors (b, x, Krylov V and Z): ell planes of N doubles
//    ("block-major", Eq. 1), cell c = i + n0*(j + n1*k).
//  * Chebyshev fields (bhat, x_k, x_{k-1}): ell planes of N values of type T
//    (float in the mixed path, double in the FP64 path).  The ell/2+1
//    frequencies that are distinct for real input pack into exactly ell
//    planes: plane 0 = Re f_0, plane 1 = Re f_{ell/2}, planes 2m and 2m+1 =
//    Re and Im of f_m for m = 1 .. ell/2-1 (f_0 and f_{ell/2} are real).
//  * Face diffusivities per cell: cx[c] = kappa of the face between c and its
//    +x neighbour (0 on the last column), likewise cy, cz.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aao {

constexpr int kMaxEll = 16;
constexpr int kMaxF = kMaxEll / 2 + 1;
constexpr int kMaxRestart = 64;

struct GridDesc {
  int n0, n1, n2;
  int64_t N;
};

// Coefficients of one Chebyshev step k (producing x_{k+1}) for every
// frequency m = 0 .. ell/2 (indexing: m, not the packed plane):
//   x_{k+1} = x_k + a (x_k - x_{k-1}) + g (bhat - A x_k + lambda x_k)
// with a = rho_k rho_{k-1}, g = 2 rho_k / delta, and itheta = 1/theta (x_1 = bhat/theta).
template <typename T>
struct StepArgs {
  T lam_re[kMaxF], lam_im[kMaxF];
  T a_re[kMaxF], a_im[kMaxF];
  T g_re[kMaxF], g_im[kMaxF];
  T it_re[kMaxF], it_im[kMaxF];
};

// Forward transform: s_t = gamma_t * scale * r_t (FP64), then
//   Re f_m = sum_t s_t cf[t][m],  Im f_m = -sum_t s_t sf[t][m]
// with cf = cos(2 pi t m/ell)/sqrt(ell), sf = sin(2 pi t m/ell)/sqrt(ell).
template <typename T>
struct DftArgs {
  double gamma[kMaxEll];
  T cf[kMaxEll][kMaxF];
  T sf[kMaxEll][kMaxF];
};

// Inverse transform of the ell/2+1 distinct frequencies y_m (real signal):
//   z_t = igamma_t * sum_m (Re y_m ci[t][m] - Im y_m si[t][m])
// with ci[t][0] = 1/sqrt(ell), ci[t][ell/2] = (-1)^t/sqrt(ell),
// ci[t][m] = 2 cos(2 pi t m/ell)/sqrt(ell), si[t][m] = 2 sin(.)/sqrt(ell).
template <typename T>
struct IdftArgs {
  double igamma[kMaxEll];
  T igamma_T[kMaxEll];   // igamma rounded to T on the host
  T ci[kMaxEll][kMaxF];
  T si[kMaxEll][kMaxF];
};

// Modes of the Chebyshev step kernel.
//  KSRC: where x_k comes from: 0 = x_1 = bhat/theta (step k = 1), 1 = buffer.
//  PSRC: where x_{k-1} comes from: 0 = zero (k = 1), 1 = bhat/theta (k = 2), 2 = buffer.
//  LAST: write x_{k+1} to the field buffer (false) or inverse-transform it to z (true).

// Launchers (one per precision; dispatch on ell and dim inside).  All return
// cudaSuccess or the launch error.  Every launch adds 1 to the launch counter.
template <typename T>
cudaError_t launch_dft(const GridDesc& g, int dim, int ell, const double* r, const double* rscale,
                       T* bhat, const DftArgs<T>& da, cudaStream_t s);
template <typename T>
cudaError_t launch_direct(const GridDesc& g, int dim, int ell, const double* r, const double* rscale,
                          double* z, const DftArgs<T>& da, const StepArgs<T>& sa,
                          const IdftArgs<T>& ia, cudaStream_t s);
template <typename T>
cudaError_t launch_step(const GridDesc& g, int dim, int ell, int ksrc, int psrc, bool last,
                        const T* cx, const T* cy, const T* cz, const T* bhat, const T* xk, T* xio,
                        double* z, const StepArgs<T>& sa, const IdftArgs<T>& ia, cudaStream_t s);

// Two fused FP32 steps (k, k+1) on a 2D grid with n0 % 4 == 0 (cheb_d2.cu):
// reads xk, xkm1 (or bhat/theta when psrc == 1) and bhat; writes x_{k+1} to
// out1 and x_{k+2} to out2, which must differ from every input.
cudaError_t launch_pair(const GridDesc& g, int ell, int psrc, const float* cx, const float* cy, const float* bhat,
                        const float* xk, const float* xkm1, float* out1, float* out2, const StepArgs<float>& s1,
                        const StepArgs<float>& s2, cudaStream_t s);

// Four fused FP32 steps (k .. k+3) on a 2D grid with n0 % 4 == 0 (cheb_d2.cu):
// reads xk, xkm1 (or bhat/theta when psrc == 1) and bhat; writes x_{k+3} to
// out3 and x_{k+4} to out4, which must differ from every input.  s[q] holds
// the coefficients of step k + q.
struct QuadSteps {
  StepArgs<float> s[4];
};
cudaError_t launch_quad(const GridDesc& g, int ell, int psrc, const float* cx, const float* cy, const float* bhat,
                        const float* xk, const float* xkm1, float* out3, float* out4, const QuadSteps& qs,
                        cudaStream_t s);

// Persistent TMA-fed variant of the four-step kernel (cheb_quad_tma.cu):
// tiles of 120 x kQuadTmaTY interior cells, kQuadTmaR staged rows per warp.
// Its x_k, x_{k-1} and bhat arrive through TMA descriptors of the ell-plane
// FP32 fields (3D: n0, n1, ell; box 128 x (kQuadTmaTY + 8) x 2).  22 rows give
// 15 warps per CTA (123 registers, 216 KB of shared memory) and, on a 1024^2 grid,
// 423 tiles, i.e. three rounds over 152 SMs; 16 rows gave 12 warps and 576 tiles
// in four rounds (7 % slower), 24 rows 16 warps at the shared-memory limit (12 % slower).
constexpr int kQuadTmaTY = 22;
constexpr int kQuadTmaR = 2;
constexpr long long kQuadTmaWaitCycles = 2000000000ll;  // bound of one TMA wait (~1 s at 2 GHz)
struct alignas(64) FieldMap {
  unsigned long long opaque[16];  // a CUtensorMap
};
// Encode the descriptor of one field (base: ell planes of N floats, 16-byte aligned).
cudaError_t encode_field_map(FieldMap* out, const float* base, const GridDesc& g, int ell);
// Descriptor of one FP32 face-coefficient array (N floats; box 128 x (kQuadTmaTY + 9)).
cudaError_t encode_coef_map(FieldMap* out, const float* base, const GridDesc& g);
// Same contract as launch_quad; the face arrays cx, cy and the fields xk, xkm1
// (psrc == 2 only) and bhat are given by their descriptors.
// wait_limit: bound of each TMA wait in SM clocks (kQuadTmaWaitCycles normally).
cudaError_t launch_quad_tma(const GridDesc& g, int ell, int psrc, const FieldMap& mcx, const FieldMap& mcy,
                            const FieldMap& mxk, const FieldMap& mxkm1, const FieldMap& mbhat, float* out3,
                            float* out4, const QuadSteps& qs, long long wait_limit, unsigned* fault,
                            cudaStream_t s);
// fault: a device word of the caller (one per handle) in which the kernel ORs 1 when one of
// its bounded waits expired and 2 when its shared-memory base was misaligned.
// Read the caller's fault word into *host_flag and clear it; synchronises s.
cudaError_t quad_tma_fault(unsigned* dev_flag, unsigned* host_flag, cudaStream_t s);

// Warp-strip variant streamed along y (cheb_stream.cu): S fused steps per launch
// (k .. k+S-1), same contract as launch_quad with S in place of 4: reads xk, xkm1 (or
// bhat/theta when psrc == 1) and bhat; writes x_{k+S-1} to outA and x_{k+S} to outB, which
// must differ from every input; fs.s[q] holds the coefficients of step k + q.
// A warp owns a 64-column strip (64 - 2S interior columns) of an H-row segment and streams
// it from S rows above to S rows below; inputs arrive through per-lane cp.async rings issued
// D rows ahead; NW warps per CTA, one CTA per SM.
constexpr int kMaxFuse = 8;
struct FuseSteps {
  StepArgs<float> s[kMaxFuse];
};
struct StreamConfig {
  int S = 4;    // fused steps (halo width)
  int H = 88;   // interior rows of a segment; H + 2S must be a multiple of 6
  int D = 4;    // rows in flight ahead of the one being consumed
  int NW = 8;   // warps per CTA
};
bool stream_config_supported(const StreamConfig& c);
cudaError_t launch_stream(const GridDesc& g, int ell, int psrc, const StreamConfig& c, const float* cx,
                          const float* cy, const float* bhat, const float* xk, const float* xkm1, float* outA,
                          float* outB, const FuseSteps& fs, cudaStream_t s);
// Transform and Chebyshev step k = 1 in one launch (2D, n0 % 4 == 0, FP32): writes bhat and
// x_2 (16-byte aligned bhat, x2, cx, cy).
cudaError_t launch_dft_first(const GridDesc& g, int ell, const double* r, const double* rscale, float* bhat,
                             float* x2, const float* cx, const float* cy, const DftArgs<float>& da,
                             const StepArgs<float>& sa, cudaStream_t s);
// z = Gamma^{-1} U x_p from the packed FP32 planes of x_p (2 cells per thread; N even, x 8-byte
// and z 16-byte aligned).
cudaError_t launch_idft_planes(const GridDesc& g, int ell, const float* x, double* z, const IdftArgs<float>& ia,
                               cudaStream_t s);

// Best-case P_alpha^{-1} for spatially constant diffusivities (dct.cu): spatial DCT-II of the
// frequency planes, division by (phi - lambda_m), inverse DCT, inverse time DFT (Section 2.2).
struct DctShifts {
  double lam_re[kMaxF], lam_im[kMaxF];
};
struct DctPlan;
// kappa[a]: the (constant) face diffusivity of axis a (0 for a missing axis).
cudaError_t dct_plan_create(DctPlan** out, const GridDesc& g, int dim, int ell, const double kappa[3]);
void dct_plan_destroy(DctPlan* p);
// vhat: the ell packed frequency planes of the time DFT (overwritten); z: ell planes of N.
cudaError_t dct_precond(DctPlan* p, const GridDesc& g, int ell, double* vhat, double* z, const DctShifts& sh,
                        const IdftArgs<double>& ia, cudaStream_t s);
// Per-axis (min, max) of the interior faces of cx, cy, cz (cy/cz may be null); synchronises s.
cudaError_t face_ranges(const GridDesc& g, const double* cx, const double* cy, const double* cz, double out[6],
                        cudaStream_t s);

// Inverse time DFT of ell packed frequency planes y into z (ell planes), with Gamma^{-1}.
cudaError_t launch_idft_planes(int64_t N, int ell, const double* y, double* z, const IdftArgs<double>& ia,
                               cudaStream_t s);

// P_SP (saddle.cu): fixed-iteration PCG on the real shifts and block-diagonally preconditioned
// MINRES on the saddle-point systems of the complex ones, with one aggregation-multigrid
// V-cycle per preconditioner block (Section 4).  1D/2D/3D, FP64.
struct SpPlan;
cudaError_t sp_plan_create(SpPlan** out, const GridDesc& g, int dim, const double* cx, const double* cy,
                           const double* cz, cudaStream_t s);
void sp_plan_destroy(SpPlan* p);
// vhat: packed frequency planes of the time DFT; y: ell planes of work space; z: result.
cudaError_t sp_precond(SpPlan* p, const GridDesc& g, int ell, int iters, double* vhat, double* y, double* z,
                       const DctShifts& sh, const IdftArgs<double>& ia, cudaStream_t s);
long long sp_last_products(const SpPlan* p);

// FP64 Krylov kernels (krylov.cu).
// y = script-A x (mode 0) or y = b - script-A x with per-block partial sums of y^2 (mode 1).
cudaError_t launch_aao_matvec(const GridDesc& g, int dim, int ell, const double* cx, const double* cy,
                              const double* cz, const double* x, const double* b, double* y,
                              double* partials, int* nblocks_out, cudaStream_t s);
// Number of blocks the flat-vector reductions use for length L (depends on L only).
int reduction_blocks(int64_t L);
// partials[i*NB + blk] = vscale[i] * sum over the block's slice of V_i . w, i < nv.
cudaError_t launch_multidot(const double* V, int64_t ldv, int nv, const double* vscale, const double* w,
                            int64_t L, double* partials, cudaStream_t s);
// w -= sum_i (h[i] * vscale[i]) V_i for i < nv; optional per-block partial sums of w^2.
cudaError_t launch_orth_update(const double* V, int64_t ldv, int nv, const double* h, const double* vscale,
                               double* w, int64_t L, double* partials_norm, cudaStream_t s);
// One fused modified Gram-Schmidt step (see mgs_step_body): with iprev >= 0,
// w -= (*hprev) vscale[iprev] V_iprev; then *hnext = vscale[inext] * V_inext . w
// (inext >= 0) or w . w (inext < 0), summed by the last block to finish over
// mgs_blocks(L) partials in part.  counter: one unsigned, zero between launches.
int mgs_blocks(int64_t L);
cudaError_t launch_mgs_step(const double* V, int64_t ldv, int iprev, int inext, const double* vscale,
                            const double* hprev, double* hnext, double* w, int64_t L, double* part,
                            unsigned* counter, cudaStream_t s);
// partial sums of v^2 per block.
cudaError_t launch_norm2_partials(const double* v, int64_t L, double* partials, cudaStream_t s);
// out[i] (+)= sum_b partials[i*NB + b] for i < nv, fixed order (deterministic).
cudaError_t launch_reduce(const double* partials, int nv, int nb, double* out, int accumulate,
                          cudaStream_t s);
// One Arnoldi column: combine h1 + h2, the new norm, rotations, residual estimate.
cudaError_t launch_givens(double* sc, int j, int m, double bnorm, cudaStream_t s);
// y = R^{-1} g for the first k columns; x += sum y_i Z_i.
cudaError_t launch_backsolve(double* sc, int k, int m, cudaStream_t s);
cudaError_t launch_xupdate(const double* Z, int64_t ldz, int k, const double* y, double* x, int64_t L,
                           cudaStream_t s);
// d = c1 d + c2 z; x += d (outer Chebyshev iteration).
cudaError_t launch_ci_update(double* d, const double* z, double* x, double c1, double c2, int64_t L, cudaStream_t s);
// Starting vector of a cycle: sc[vscale 0] = 1/sqrt(nrm2), g[0] = sqrt(nrm2), clears H/g.
cudaError_t launch_cycle_init(double* sc, int m, cudaStream_t s);

// Layout of the small FP64 scalar block `sc` (device), m = restart length.
struct ScLayout {
  int m;
  __host__ __device__ int H(int i, int j) const { return i * m + j; }          // (m+1) x m
  __host__ __device__ int cs(int i) const { return (m + 1) * m + i; }
  __host__ __device__ int sn(int i) const { return (m + 1) * m + m + i; }
  __host__ __device__ int gv(int i) const { return (m + 1) * m + 2 * m + i; }  // m+1
  __host__ __device__ int y(int i) const { return (m + 1) * m + 3 * m + 1 + i; }
  __host__ __device__ int vscale(int i) const { return (m + 1) * m + 4 * m + 1 + i; }  // m+1
  __host__ __device__ int h1(int i) const { return (m + 1) * m + 5 * m + 2 + i; }      // m+1
  __host__ __device__ int h2(int i) const { return (m + 1) * m + 6 * m + 3 + i; }      // m+1
  __host__ __device__ int nrm2() const { return (m + 1) * m + 7 * m + 4; }
  __host__ __device__ int est() const { return (m + 1) * m + 7 * m + 5; }
  __host__ __device__ int hnext() const { return (m + 1) * m + 7 * m + 6; }
  __host__ __device__ int bnorm() const { return (m + 1) * m + 7 * m + 7; }
  __host__ __device__ int size() const { return (m + 1) * m + 7 * m + 8; }
};

void count_launch();

// IEEE binary64 -> binary32 with round-to-nearest-even, on the integer pipe.
// GB300 issues FP64<->FP32 conversions on its (narrow) FP64 pipe; the mixed
// path converts every residual value once per preconditioner apply.  Results
// below the FP32 normal range become signed zero and results above it
// infinity (NaN also becomes infinity); the scaled residuals here are far
// from both limits.
__device__ __forceinline__ float d2f_rn(double d) {
  const int hi = __double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned sign = (unsigned)hi & 0x80000000u;
  const int fe = ((hi >> 20) & 0x7ff) - 896;
  const unsigned m = (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u) || (rem == 0x10000000u && (m & 1u));
  unsigned bits = ((unsigned)fe << 23) + m + up;
  bits = (fe <= 0) ? 0u : bits;
  bits = (fe >= 255) ? 0x7f800000u : bits;
  return __uint_as_float(sign | bits);
}

// IEEE binary32 -> binary64 (exact) on the integer pipe; FP32 subnormals
// become signed zero, infinities and NaNs keep their class.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  const unsigned eo = (e == 0u) ? 0u : ((e == 255u) ? 0x7ffu : e + 896u);
  const unsigned mm = (e == 0u) ? 0u : m;
  const unsigned hi = sign | (eo << 20) | (mm >> 3);
  const unsigned lo = mm << 29;
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace aao
