// Host-side scalar set-up of the preconditioner (FP64), shared by the handle
// path (aao_api.cu) and the allocation-free entry point (noalloc.cu).
//
// Section 2.2 and Lemma 2: the shifts lambda_m = alpha^{1/ell} exp(-2 pi i m/ell)
// (paired with the forward transform exp(-2 pi i t m/ell)), the Chebyshev segment
// of B_m = A - lambda_m I with centre theta_m = (mu_max + mu_min)/2 - lambda_m and
// half-width delta = (mu_max - mu_min)/2, and the three-term coefficients
// rho_0 = delta/theta, rho_k = 1/(2 theta/delta - rho_{k-1}),
// a_k = rho_k rho_{k-1}, g_k = 2 rho_k/delta.  Eq. 5: Gamma = diag(alpha^{t/ell})
// and the length-ell transforms.  No heap use: one step is produced at a time.
#pragma once

#include <cmath>
#include <complex>

#include "aao_internal.cuh"

namespace aao {

struct ChebTables {
  int ell = 0, F = 0;
  double delta = 0.0;
  std::complex<double> lam[kMaxF], theta[kMaxF], rho_prev[kMaxF];
};

inline void cheb_tables_init(ChebTables& tb, int ell, double alpha, double mu_min, double mu_max) {
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

// Coefficients of step k (producing x_{k+1}); call for k = 0, 1, 2, ... in order.
// palloc (nullable): per-frequency step budgets m = 0 .. ell/2 (Algorithm 1); a
// frequency past its budget keeps its iterate (a = g = 0), a zero budget gives
// y_m = 0 (1/theta = 0).  The single-point segment delta = 0 (one cell, A = I)
// takes the delta -> 0 limit of the recurrence, the exact solve: a = 0, g = 1/theta.
inline void cheb_tables_step(ChebTables& tb, int k, const int* palloc, StepArgs<double>& s) {
  using cd = std::complex<double>;
  s = StepArgs<double>{};
  for (int m = 0; m < tb.F; ++m) {
    cd a(0.0, 0.0), gk(0.0, 0.0);
    const bool spent = palloc && k >= 1 && k >= palloc[m];
    if (spent) {
    } else if (k >= 1 && tb.delta == 0.0) {
      gk = 1.0 / tb.theta[m];
    } else if (k >= 1) {
      const cd rho = 1.0 / (2.0 * tb.theta[m] / tb.delta - tb.rho_prev[m]);
      a = rho * tb.rho_prev[m];
      gk = 2.0 * rho / tb.delta;
      tb.rho_prev[m] = rho;
    }
    const cd it = (palloc && palloc[m] == 0) ? cd(0.0, 0.0) : 1.0 / tb.theta[m];
    s.lam_re[m] = tb.lam[m].real();
    s.lam_im[m] = tb.lam[m].imag();
    s.a_re[m] = a.real();
    s.a_im[m] = a.imag();
    s.g_re[m] = gk.real();
    s.g_im[m] = gk.imag();
    s.it_re[m] = it.real();
    s.it_im[m] = it.imag();
  }
}

// The FP32 copy of a step's coefficients (each value rounded once from FP64).
inline StepArgs<float> narrow_step(const StepArgs<double>& s) {
  StepArgs<float> f{};
  for (int m = 0; m < kMaxF; ++m) {
    f.lam_re[m] = (float)s.lam_re[m];
    f.lam_im[m] = (float)s.lam_im[m];
    f.a_re[m] = (float)s.a_re[m];
    f.a_im[m] = (float)s.a_im[m];
    f.g_re[m] = (float)s.g_re[m];
    f.g_im[m] = (float)s.g_im[m];
    f.it_re[m] = (float)s.it_re[m];
    f.it_im[m] = (float)s.it_im[m];
  }
  return f;
}

// Forward and inverse transform tables (Eq. 5) in FP64; see DftArgs / IdftArgs.
inline void transform_tables(int ell, double alpha, DftArgs<double>& da, IdftArgs<double>& ia) {
  const double pi = 3.14159265358979323846;
  const double isq = 1.0 / std::sqrt((double)ell);
  da = DftArgs<double>{};
  ia = IdftArgs<double>{};
  for (int t = 0; t < ell; ++t) {
    da.gamma[t] = std::pow(alpha, (double)t / ell);
    ia.igamma[t] = std::pow(alpha, -(double)t / ell);
    ia.igamma_T[t] = ia.igamma[t];
    for (int m = 0; m <= ell / 2; ++m) {
      const double ang = 2.0 * pi * (double)((t * m) % ell) / ell;
      da.cf[t][m] = std::cos(ang) * isq;
      da.sf[t][m] = std::sin(ang) * isq;
      if (m == 0) {
        ia.ci[t][m] = isq;
      } else if (2 * m == ell) {
        ia.ci[t][m] = (t % 2 == 0) ? isq : -isq;
      } else {
        ia.ci[t][m] = 2.0 * std::cos(ang) * isq;
        ia.si[t][m] = 2.0 * std::sin(ang) * isq;
      }
    }
  }
}

// FP32 transform tables: twiddles rounded once from FP64; gamma and 1/gamma stay FP64
// (the mixed transforms scale in FP64), igamma_T holds 1/gamma rounded to FP32.
inline void narrow_transforms(const DftArgs<double>& da, const IdftArgs<double>& ia, DftArgs<float>& fa,
                              IdftArgs<float>& fi) {
  fa = DftArgs<float>{};
  fi = IdftArgs<float>{};
  for (int t = 0; t < kMaxEll; ++t) {
    fa.gamma[t] = da.gamma[t];
    fi.igamma[t] = ia.igamma[t];
    fi.igamma_T[t] = (float)ia.igamma[t];
    for (int m = 0; m < kMaxF; ++m) {
      fa.cf[t][m] = (float)da.cf[t][m];
      fa.sf[t][m] = (float)da.sf[t][m];
      fi.ci[t][m] = (float)ia.ci[t][m];
      fi.si[t][m] = (float)ia.si[t][m];
    }
  }
}

}  // namespace aao
