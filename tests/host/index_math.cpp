// Host checks of the index arithmetic the box-mesh kernels rely on (built and run by
// tests/test_host_index_math.py with the host compiler):
//  * hx_fastdiv_init: n / d = (n m) >> s for every dividend below 2^31,
//  * hx_eline: both E-vector layouts are bijections onto [0, E n^3), the element-major one
//    equal to e n^3 + l, the line layout placing an element row's x-lines side by side.
#include <cstdio>
#include <random>
#include <vector>

#include "hx_internal.h"

static int fails = 0;
#define CHECK(c, ...)                 \
  do {                                \
    if (!(c)) {                       \
      if (fails < 20) {               \
        std::printf("FAIL: " __VA_ARGS__); \
        std::printf("\n");            \
      }                               \
      ++fails;                        \
    }                                 \
  } while (0)

static void check_div(int d, std::mt19937_64& rng) {
  unsigned m;
  int s;
  hx_fastdiv_init(d, &m, &s);
  auto q = [&](long long n) { return (long long)(((unsigned long long)(unsigned)n * m) >> s); };
  std::uniform_int_distribution<long long> u(0, (1LL << 31) - 1);
  for (int t = 0; t < 2000; ++t) {
    const long long n = u(rng);
    CHECK(q(n) == n / d, "d=%d n=%lld", d, n);
  }
  // around multiples of d and at the top of the range
  for (long long k = 0; k < 64; ++k)
    for (long long n : {k * d - 1, k * d, k * d + 1})
      if (n >= 0 && n < (1LL << 31)) CHECK(q(n) == n / d, "d=%d n=%lld", d, n);
  const long long top = (1LL << 31) - 1, kt = top / d;
  for (long long n = top - 64; n <= top; ++n)
    if (n >= 0) CHECK(q(n) == n / d, "d=%d n=%lld", d, n);
  for (long long k = kt - 2; k <= kt; ++k)  // the largest multiples of d below 2^31
    for (long long n : {k * d - 1, k * d, k * d + 1})
      if (n >= 0 && n <= top) CHECK(q(n) == n / d, "d=%d n=%lld", d, n);
}

static void check_layout(int nx, int ny, int nz, int n) {
  const long long E = (long long)nx * ny * nz, n3 = (long long)n * n * n;
  for (int which = 0; which < 2; ++which) {
    const HxELayout L = which ? hx_elayout_rows(nx) : HxELayout{0, 0u, 0};
    std::vector<char> seen(E * n3, 0);
    for (long long e = 0; e < E; ++e)
      for (int r = 0; r < n * n; ++r) {
        const long long base = hx_eline(L, e, r, n);
        for (int i = 0; i < n; ++i) {
          const long long pos = base + i;
          CHECK(pos >= 0 && pos < E * n3, "layout %d: position %lld out of range", which, pos);
          if (pos < 0 || pos >= E * n3) continue;
          CHECK(!seen[pos], "layout %d: position %lld twice", which, pos);
          seen[pos] = 1;
          if (!which) CHECK(pos == e * n3 + r * n + i, "element-major position of e=%lld", e);
          if (which) {
            // element (ex, row) line r: ((row n^2 + r) nx + ex) n + i
            const long long row = e / nx, ex = e % nx;
            CHECK(pos == ((row * n * n + r) * nx + ex) * n + i, "line-layout position of e=%lld", e);
          }
        }
      }
  }
}

int main() {
  std::mt19937_64 rng(20191003);
  for (int d = 1; d <= 3000; ++d) check_div(d, rng);
  std::uniform_int_distribution<int> big(3001, (1 << 30));
  for (int t = 0; t < 300; ++t) check_div(big(rng), rng);
  check_div((1 << 30) + 12345, rng);
  check_div(2147483647, rng);
  const int grids[][4] = {{1, 1, 1, 2}, {3, 2, 2, 2}, {4, 3, 1, 5}, {5, 1, 2, 4}, {2, 3, 4, 9}, {7, 2, 3, 3}};
  for (const auto& g : grids) check_layout(g[0], g[1], g[2], g[3]);
  const HxGridAsm ga = hx_grid_asm(4, 96, 96, 96, 385, 385);
  CHECK(ga.p == 4 && ga.nx == 96 && ga.gx == 385 && ga.gy == 385, "grid descriptor");
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("OK\n");
  return 0;
}
