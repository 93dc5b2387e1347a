// Host-side set-up of the RBSOG + RBL library (runs once per rbsog_set_system):
//   - the SOG parameters of Sec. 2.1: nominal weights w_m = sqrt(2) ln b /
//     (sqrt(pi) b^m s) of Eq. (far), the narrowest weight w_0 fixed by
//     N(r_c) = 0 and the bandwidth s by N'(r_c) = 0 (C^1 cutoff at r_c = r_shell);
//   - the exact sampler of P(k) = k^2 Fhat(k) / S (Eq. (Pk)) written as a mixture
//     over (Gaussian g, axis d) of separable lattice Gaussians, with 64-bit
//     fixed-point CDFs and S in closed form;
//   - the FP32 cubic tables of the SOG sums used by the mixed-precision pair
//     kernel.
#include "setup.h"

#include <algorithm>
#include <cmath>

namespace rb {

static double pow_int(double b, int m) {
  double r = 1.0;
  for (int k = 0; k < m; k++) r *= b;
  return r;
}

void sog_fill(double b, int M, double s, double w0, SogParams &out) {
  out.b = b;
  out.M = M;
  out.s = s;
  out.w.assign(M + 1, 0.0);
  out.a.assign(M + 1, 0.0);
  const double c = std::sqrt(2.0) * std::log(b) / std::sqrt(M_PI);
  for (int m = 0; m <= M; m++) {
    const double bm = pow_int(b, m) * s;
    out.a[m] = bm * bm;
    out.w[m] = c / bm;
  }
  out.w[0] = w0;
}

// w_0 from value continuity N(r_c) = 0 at bandwidth s.
static double w0_for(double b, int M, double rc, double s) {
  SogParams p;
  sog_fill(b, M, s, 0.0, p);
  double tail = 0.0;
  for (int m = M; m >= 1; m--) tail += p.w[m] * std::exp(-rc * rc / (2.0 * p.a[m]));
  return std::exp(rc * rc / (2.0 * s * s)) * (1.0 / rc - tail);
}

// N'(r_c) = -1/r_c^2 + sum_m w_m (r_c / a_m) e^{-r_c^2 / (2 a_m)}
static double dN_rc(double b, int M, double rc, double s) {
  SogParams p;
  sog_fill(b, M, s, w0_for(b, M, rc, s), p);
  double g = 0.0;
  for (int m = M; m >= 0; m--) g += p.w[m] / p.a[m] * std::exp(-rc * rc / (2.0 * p.a[m]));
  return rc * g - 1.0 / (rc * rc);
}

int sog_solve(double b, int M, double rc, SogParams &out) {
  // log-spaced scan of s over [r_c/6, r_c/2]; refine each sign change by
  // bisection to the last representable bit; keep the root whose w_0 is
  // closest to its nominal value.
  const int NS = 3000;
  const double lo = std::log(rc / 6.0), hi = std::log(rc / 2.0);
  double best = -1.0, best_dev = 1e300;
  double sp = std::exp(lo), fp = dN_rc(b, M, rc, sp);
  for (int k = 1; k <= NS; k++) {
    const double sk = std::exp(lo + (hi - lo) * k / NS);
    const double fk = dN_rc(b, M, rc, sk);
    if ((fp < 0.0) != (fk < 0.0) || fk == 0.0) {
      double a = sp, c = sk, fa = fp;
      while (true) {
        const double mid = 0.5 * (a + c);
        if (!(mid > a && mid < c)) break;
        const double fm = dN_rc(b, M, rc, mid);
        if (fm == 0.0) { a = c = mid; break; }
        if ((fm < 0.0) == (fa < 0.0)) { a = mid; fa = fm; } else { c = mid; }
      }
      const double sr = 0.5 * (a + c);
      const double nominal = std::sqrt(2.0) * std::log(b) / (std::sqrt(M_PI) * sr);
      const double dev = std::fabs(w0_for(b, M, rc, sr) / nominal - 1.0);
      if (dev < best_dev) { best_dev = dev; best = sr; }
    }
    sp = sk;
    fp = fk;
  }
  if (best < 0.0) return RBSOG_E_NO_SOG_ROOT;
  sog_fill(b, M, best, w0_for(b, M, rc, best), out);
  return RBSOG_OK;
}

// ---------------------------------------------------------------------------
static unsigned long long to_fixed(double cum, double tot) {
  const double two64 = 18446744073709551616.0;
  const double x = std::floor(cum / tot * two64);
  if (x >= two64) return ~0ull;
  if (x <= 0.0) return 0ull;
  return (unsigned long long)x;
}

void sampler_build(const SogParams &sog, const double L[3], Sampler &T) {
  const int G = sog.M + 1;
  T.nmax.assign(3 * G, 0);
  T.off0.assign(3 * G, 0);
  T.off2.assign(3 * G, 0);
  T.cdf.clear();
  T.cmix.assign(3 * G, 0ull);
  std::vector<double> Z(3 * G, 0.0);
  const double cut = 60.0;  // Gaussian factors below e^-60 carry no 64-bit CDF mass
  for (int g = 0; g < G; g++) {
    const double a = sog.a[g];
    const double cg = std::pow(2.0 * M_PI, 1.5) * sog.w[g] * a * std::sqrt(a);  // (2pi)^{3/2} w_g b^{3g} s^3
    double T0[3], T2[3];
    for (int d = 0; d < 3; d++) {
      const double kap = 2.0 * M_PI / L[d];
      int nm = (int)std::ceil(std::sqrt(2.0 * cut / a) / kap);
      nm = std::max(nm, 1);
      const int len = 2 * nm + 1;
      std::vector<double> e0(len), e2(len);
      double s0 = 0.0, s2 = 0.0;
      for (int q = 0; q < len; q++) {
        const double k = kap * (double)(q - nm);
        e0[q] = std::exp(-0.5 * a * k * k);
        e2[q] = k * k * e0[q];
        s0 += e0[q];
        s2 += e2[q];
      }
      T0[d] = s0;
      T2[d] = s2;
      T.nmax[3 * g + d] = nm;
      T.off0[3 * g + d] = (int)T.cdf.size();
      double r = 0.0;
      for (int q = 0; q < len; q++) { r += e0[q]; T.cdf.push_back(to_fixed(r, s0)); }
      T.off2[3 * g + d] = (int)T.cdf.size();
      r = 0.0;
      for (int q = 0; q < len; q++) { r += e2[q]; T.cdf.push_back(s2 > 0.0 ? to_fixed(r, s2) : ~0ull); }
    }
    Z[3 * g + 0] = cg * T2[0] * T0[1] * T0[2];
    Z[3 * g + 1] = cg * T0[0] * T2[1] * T0[2];
    Z[3 * g + 2] = cg * T0[0] * T0[1] * T2[2];
  }
  double tot = 0.0;
  for (double z : Z) tot += z;
  double r = 0.0;
  for (int q = 0; q < 3 * G; q++) { r += Z[q]; T.cmix[q] = to_fixed(r, tot); }
  T.S = tot;
}

// ---------------------------------------------------------------------------
// Cubic Hermite tables on x = r^2 in [0, r_shell^2] of
//   G(x) = sum_m w_m / a_m e^{-x/(2 a_m)}  (force of the SOG part, Eq. (Fshort))
//   F(x) = sum_m w_m e^{-x/(2 a_m)}        (potential of the far part, Eq. (far))
// Interval i holds (c0, c1, c2, c3) of c0 + c1 f + c2 f^2 + c3 f^3, f in [0, 1).
void sog_tables(const SogParams &sog, double rs2, int nt, std::vector<float> &gt,
                std::vector<float> &ft) {
  const double h = rs2 / nt;
  auto eval = [&](double x, double &G, double &dG, double &F, double &dF) {
    G = dG = F = dF = 0.0;
    for (int m = sog.M; m >= 0; m--) {
      const double e = std::exp(-x / (2.0 * sog.a[m]));
      G += sog.w[m] / sog.a[m] * e;
      dG -= sog.w[m] / (2.0 * sog.a[m] * sog.a[m]) * e;
      F += sog.w[m] * e;
      dF -= sog.w[m] / (2.0 * sog.a[m]) * e;
    }
  };
  gt.assign(4 * nt, 0.0f);
  ft.assign(4 * nt, 0.0f);
  for (int i = 0; i < nt; i++) {
    double G0, dG0, F0, dF0, G1, dG1, F1, dF1;
    eval(h * i, G0, dG0, F0, dF0);
    eval(h * (i + 1), G1, dG1, F1, dF1);
    auto herm = [&](double y0, double d0, double y1, double d1, float *c) {
      c[0] = (float)y0;
      c[1] = (float)(h * d0);
      c[2] = (float)(3.0 * (y1 - y0) - h * (2.0 * d0 + d1));
      c[3] = (float)(2.0 * (y0 - y1) + h * (d0 + d1));
    };
    herm(G0, dG0, G1, dG1, &gt[4 * i]);
    herm(F0, dF0, F1, dF1, &ft[4 * i]);
  }
}

int cell_count(double L, double r_out) {
  const double w = 0.5 * r_out * (1.0 + 1.0 / 4096.0);
  const int c = (int)std::floor(L / w);
  return c < 1 ? 1 : c;
}

}  // namespace rb
