// Host-side check of the lattice index arithmetic the kernels use
// (su3_device.cuh): multiply-shift division, site coordinates of a half
// index, and the neighbour half indices by additive offsets, against plain
// integer division and coordinate arithmetic with explicit periodic wrap.
// Compiled with nvcc and run on the CPU; launches nothing on a GPU.
#include <cstdio>
#include <cstdlib>

#include "su3_device.cuh"

using namespace su3dev;

static int failures = 0;

static void expect(bool ok, const char* what, long long a, long long b, long long c) {
  if (!ok && failures++ < 20) std::printf("FAIL %s (%lld %lld %lld)\n", what, a, b, c);
}

static void check_division() {
  const unsigned ds[] = {1, 2, 3, 5, 6, 7, 12, 16, 31, 32, 33, 48, 64, 100, 1000, 4096, 65535, 65536, 65537,
                         1u << 20, (1u << 20) + 1, 1000003, 1u << 30, (1u << 30) + 1, 2147483647u};
  for (unsigned d : ds) {
    const Divisor dv = make_divisor(d);
    const long long ns[] = {0, 1, (long long)d - 1, d, (long long)d + 1, 2147483647LL, 2147483646LL,
                            (2147483647LL / d) * d, (2147483647LL / d) * d - 1, 123456789};
    for (long long n : ns) {
      if (n < 0 || n > 2147483647LL) continue;
      expect(udiv((int)n, dv) == (int)(n / d), "udiv", n, d, udiv((int)n, dv));
    }
    for (long long n = 0; n < 200000; n += 7) expect(udiv((int)n, dv) == (int)(n / d), "udiv", n, d, 0);
  }
  for (unsigned d = 1; d <= 5000; ++d) {
    const Divisor dv = make_divisor(d);
    for (long long n = 2147483647LL; n > 2147483647LL - 3 * (long long)d; --n)
      expect(udiv((int)n, dv) == (int)(n / d), "udiv top", n, d, 0);
  }
}

static int half_of(const int L[4], const int x[4]) { return (x[0] >> 1) + (L[0] / 2) * (x[1] + L[1] * (x[2] + L[2] * x[3])); }

static void check_lattice(int L0, int L1, int L2, int L3) {
  const Geometry g = make_geometry(L0, L1, L2, L3);
  const int L[4] = {L0, L1, L2, L3};
  for (int p = 0; p < 2; ++p)
    for (int h = 0; h < g.Vh; ++h) {
      const Site st = site_of(g, h, p);
      const int x[4] = {st.x0, st.x1, st.x2, st.x3};
      bool in = true;
      for (int d = 0; d < 4; ++d) in = in && x[d] >= 0 && x[d] < L[d];
      expect(in, "coordinates in range", h, p, 0);
      if (!in) continue;
      expect(((x[0] + x[1] + x[2] + x[3]) & 1) == p, "parity", h, p, 0);
      const int s = x[0] + L0 * (x[1] + L1 * (x[2] + L2 * x[3]));
      expect(canon(g, st) == s && s / 2 == h, "canonical index", h, p, s);
      for (int nu = 0; nu < 4; ++nu) {
        for (int dd = -1; dd <= 1; dd += 2) {
          int y[4] = {x[0], x[1], x[2], x[3]};
          y[nu] = (y[nu] + dd + L[nu]) % L[nu];
          expect(nb_half(g, st, nu, dd) == half_of(L, y), "nb_half", h, nu, dd);
        }
        for (int rho = 0; rho < 4; ++rho) {
          if (rho == nu) continue;
          int y[4] = {x[0], x[1], x[2], x[3]};
          y[nu] = (y[nu] + 1) % L[nu];
          y[rho] = (y[rho] - 1 + L[rho]) % L[rho];
          expect(nb_half2(g, st, nu, rho) == half_of(L, y), "nb_half2", h, nu, rho);
        }
      }
    }
}

int main() {
  check_division();
  const int dims[][4] = {{2, 2, 2, 2}, {4, 4, 4, 4}, {2, 4, 6, 8}, {6, 2, 4, 2}, {10, 14, 6, 12},
                         {8, 8, 8, 16}, {12, 12, 12, 12}, {32, 32, 32, 32}, {64, 2, 2, 2}, {2, 2, 2, 64}};
  for (const auto& d : dims) check_lattice(d[0], d[1], d[2], d[3]);
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("index arithmetic ok\n");
  return 0;
}
