// Host-side set-up routines (SOG solve, P(k) sampler tables, FP32 SOG tables,
// cell grid) of the RBSOG + RBL library.
#pragma once

#include <vector>

#include "rbsog.h"

namespace rb {

struct SogParams {
  double b = 0, s = 0;
  int M = 0;
  std::vector<double> w;  // w_m, w_0 modified
  std::vector<double> a;  // a_m = (b^m s)^2
};

struct Sampler {
  std::vector<int> nmax, off0, off2;     // per (g, d), index 3 g + d
  std::vector<unsigned long long> cdf;   // flat 1-D CDFs (plain, then k^2-weighted)
  std::vector<unsigned long long> cmix;  // mixture CDF over (g, d)
  double S = 0;                          // sum_{k != 0} k^2 Fhat(k)
};

// Weights and widths for given (b, M, s) with the given w_0.
void sog_fill(double b, int M, double s, double w0, SogParams &out);
// Solve s and w_0 for C^1 continuity at r_c; RBSOG_E_NO_SOG_ROOT if none.
int sog_solve(double b, int M, double rc, SogParams &out);
void sampler_build(const SogParams &sog, const double L[3], Sampler &T);
void sog_tables(const SogParams &sog, double rs2, int nt, std::vector<float> &gt,
                std::vector<float> &ft);
// Cells per axis: max(1, floor(L / (r_out/2 (1 + 2^-12)))), r_out the outer
// list radius (r_shell, or r_shell + skin for kept lists).
int cell_count(double L, double r_out);

}  // namespace rb
