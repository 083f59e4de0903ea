// Host-side check of the double-float arithmetic used for complex128 states:
// prints the worst relative errors against IEEE double on seeded random inputs.
#include <cmath>
#include <cstdio>
#include <random>

#include "df64.cuh"

using sv::df;

static double rel(double got, double want, double scale) { return std::fabs(got - want) / scale; }

int main() {
  std::mt19937_64 rng(2403);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-30, 4);  // amplitude / matrix-entry magnitudes
  double e_conv = 0, e_add = 0, e_mul = 0, e_fma = 0, e_rot = 0;
  for (int i = 0; i < 200000; ++i) {
    const double a = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), ex(rng)) * (u(rng) < 0 ? -1 : 1);
    const double b = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), ex(rng)) * (u(rng) < 0 ? -1 : 1);
    const double c = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), ex(rng)) * (u(rng) < 0 ? -1 : 1);
    const df A(a), B(b), C(c);
    e_conv = std::fmax(e_conv, rel((double)A, a, std::fabs(a)));
    e_add = std::fmax(e_add, rel((double)(A + B), a + b, std::fmax(std::fabs(a), std::fabs(b))));
    e_mul = std::fmax(e_mul, rel((double)(A * B), a * b, std::fabs(a * b)));
    e_fma = std::fmax(e_fma, rel((double)fma(A, B, C), std::fma(a, b, c), std::fmax(std::fabs(a * b), std::fabs(c))));
    // a real 2x2 rotation on a complex pair, as in the RY / Givens blocks
    const double th = u(rng) * 3.0, co = std::cos(th), si = std::sin(th);
    const double ar = u(rng), ai = u(rng), br = u(rng), bi = u(rng);
    const df CO(co), SI(si), NS(-si);
    const df r0 = fma(CO, df(ar), NS * df(br)), r1 = fma(SI, df(ar), CO * df(br));
    const df i0 = fma(CO, df(ai), NS * df(bi));
    e_rot = std::fmax(e_rot, std::fmax(rel((double)r0, co * ar - si * br, 1.0),
                                       std::fmax(rel((double)r1, si * ar + co * br, 1.0),
                                                 rel((double)i0, co * ai - si * bi, 1.0))));
  }
  // conversions down to 2^-100 keep ~48 bits
  for (int i = 0; i < 100000; ++i) {
    const double a = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), -std::uniform_int_distribution<int>(0, 99)(rng));
    e_conv = std::fmax(e_conv, rel((double)df(a), a, a));
  }
  // exact float -> double re-encoding, subnormals included
  for (int i = 0; i < 100000; ++i) {
    const float f = std::ldexp((float)u(rng), -std::uniform_int_distribution<int>(0, 149)(rng));
    if (sv::df_f2d_exact(f) != (double)f) e_conv = 1.0;
  }
  // lean stream conversions: amplitudes down to 2^-70 keep ~47 bits; below
  // 2^-126 they become zero
  double e_fast = 0;
  for (int i = 0; i < 200000; ++i) {
    const double a = std::ldexp(0.5 + 0.5 * std::fabs(u(rng)), -std::uniform_int_distribution<int>(-4, 70)(rng)) *
                     (u(rng) < 0 ? -1 : 1);
    const df F = sv::df_split_fast(a);
    e_fast = std::fmax(e_fast, rel(sv::df_join_fast(F), a, std::fabs(a)));
    e_fast = std::fmax(e_fast, rel((double)F, a, std::fabs(a)));
    if (std::fabs(F.l) > 0.5f * std::ldexp(1.0f, std::ilogb(F.h) - 23)) e_fast = 1.0;  // canonical pair
  }
  if (sv::df_join_fast(sv::df_split_fast(std::ldexp(1.0, -130))) != 0.0) e_fast = 1.0;
  if (sv::df_join_fast(sv::df_split_fast(0.0)) != 0.0) e_fast = 1.0;
  const double z = (double)df(0.0), nz = (double)df(-0.0);
  std::printf("conv %.3e add %.3e mul %.3e fma %.3e rot %.3e fastconv %.3e zero %g %g\n", e_conv, e_add, e_mul,
              e_fma, e_rot, e_fast, z, nz);
  return 0;
}
