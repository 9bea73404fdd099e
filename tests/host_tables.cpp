// Host test of the library's geometry and tally-axis classification (mc_tables.h): the first-guess
// rules of the tally axes and the box-cell entries of cells.  Built with the host C++ compiler by
// tests/test_host_tables.py; prints "ok" and exits 0 when every check holds.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "mc_tables.h"

using mcgb::bin_guess_params;
using mcgb::box_cell_entry;

static int failures = 0;
#define CHECK(c)                                                        \
  do {                                                                  \
    if (!(c)) {                                                         \
      std::printf("FAILED line %d: %s\n", __LINE__, #c);                \
      ++failures;                                                       \
    }                                                                   \
  } while (0)

// the bin by plain bisection: e[i] <= x < e[i+1]
static int bisect(const std::vector<float>& e, float x) {
  const int n = (int)e.size() - 1;
  if (!(x >= e[0])) return -1;
  if (!(x < e[n])) return n;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (e[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// the guess of a classified axis, in float as the walk forms it (the log through the host's log2f)
static int guess(int kind, float a, float b, const std::vector<float>& e, float x) {
  if (kind == 1) return (int)std::floor((x - a) * b);
  return x < e[1] ? 0 : 1 + (int)std::floor(std::log2(x * a) * b);
}

// every guess of `kind` within one bin of the bisection's bin, over random points of the axis
static void check_axis(const std::vector<float>& e, int want_kind, bool log_points, unsigned seed) {
  int kind;
  float a, b;
  bin_guess_params(e, kind, a, b);
  CHECK(kind == want_kind);
  if (kind == 0) return;
  std::mt19937 rng(seed);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  const int n = (int)e.size() - 1;
  for (int t = 0; t < 200000; ++t) {
    double xd;
    if (log_points) xd = (t % 10 == 0) ? e[1] * u(rng) : e[1] * std::pow((double)e[n] / e[1], u(rng));
    else xd = e[0] + (e[n] - e[0]) * u(rng);
    const float x = (float)xd;
    const int want = bisect(e, x);
    if (want < 0 || want >= n) continue;
    const int g = guess(kind, a, b, e, x);
    if (std::abs(g - want) > 1) {
      std::printf("axis kind %d: x = %.9g guess %d bin %d\n", kind, x, g, want);
      ++failures;
      return;
    }
  }
  // the edges themselves: a point on an edge belongs to the bin above it
  for (int k = 0; k < n; ++k) CHECK(std::abs(guess(kind, a, b, e, e[k]) - bisect(e, e[k])) <= 1);
}

static mc_cell cell(std::initializer_list<std::pair<int, int>> hs) {
  mc_cell c = {};
  for (const auto& h : hs) {
    c.surface[c.n_halfspaces] = h.first;
    c.sense[c.n_halfspaces] = h.second;
    ++c.n_halfspaces;
  }
  return c;
}

int main() {
  // equal spacing: the lattice mesh (34 bins over 17 x 1.26 cm) and a slab's 50 bins from -2
  std::vector<float> lat(35), slab(51), sq(41), lg(51), pure(21), small(4);
  for (int k = 0; k <= 34; ++k) lat[k] = (float)(21.42 * k / 34);
  for (int k = 0; k <= 50; ++k) slab[k] = (float)(-2.0 + 5.0 * k / 50);
  check_axis(lat, 1, false, 1);
  check_axis(slab, 1, false, 2);
  // log-spaced time bins after a first bin [0, 1e-9], and log spacing from the first edge on
  lg[0] = 0.0f;
  for (int k = 1; k <= 50; ++k) lg[k] = (float)std::pow(10.0, -9.0 + 6.0 * (k - 1) / 49);
  for (int k = 0; k <= 20; ++k) pure[k] = (float)std::pow(10.0, -3.0 + 4.0 * k / 20);
  check_axis(lg, 2, true, 3);
  check_axis(pure, 2, true, 4);
  // irregular spacing and too few bins: bisection
  for (int k = 0; k <= 40; ++k) sq[k] = (float)(k * k + 0.5 * k);
  for (int k = 0; k <= 3; ++k) small[k] = (float)k;
  check_axis(sq, 0, false, 5);
  check_axis(small, 0, false, 6);

  // surfaces: planes x = 0, x = 1, y = 0, y = 1, z = 0, z = 1, a z-cylinder, a second plane x = 0.5
  mc_surface s[8] = {};
  const int kinds[8] = {MC_SURF_PX, MC_SURF_PX, MC_SURF_PY, MC_SURF_PY, MC_SURF_PZ, MC_SURF_PZ, MC_SURF_CZ, MC_SURF_PX};
  for (int i = 0; i < 8; ++i) s[i].kind = kinds[i];
  int b[7];
  // a cube listed as x >= 0, x <= 1, y >= 0, y <= 1, z >= 0, z <= 1 (sense +1: positive side)
  const mc_cell cube = cell({{0, 1}, {1, -1}, {2, 1}, {3, -1}, {4, 1}, {5, -1}});
  box_cell_entry(cube, s, b);
  CHECK(b[0] == 1);
  for (int ax = 0; ax < 3; ++ax) {
    CHECK(b[1 + 2 * ax] == ((2 * ax) | ((2 * ax) << 16)));              // lower plane, list position 2 ax
    CHECK(b[2 + 2 * ax] == ((2 * ax + 1) | ((2 * ax + 1) << 16)));      // upper plane
  }
  // the same box listed in another order keeps each plane's own list position
  const mc_cell cube2 = cell({{5, -1}, {0, 1}, {3, -1}, {1, -1}, {2, 1}, {4, 1}});
  box_cell_entry(cube2, s, b);
  CHECK(b[0] == 1 && b[1] == (0 | (1 << 16)) && b[2] == (1 | (3 << 16)) && b[6] == (5 | (0 << 16)));
  // a slab between two x planes: y and z unbounded
  box_cell_entry(cell({{0, 1}, {1, -1}}), s, b);
  CHECK(b[0] == 1 && b[3] == -1 && b[4] == -1 && b[5] == -1 && b[6] == -1);
  // a cylinder among the halfspaces, and two lower x planes: not boxes
  box_cell_entry(cell({{0, 1}, {1, -1}, {6, -1}}), s, b);
  CHECK(b[0] == 0);
  box_cell_entry(cell({{0, 1}, {7, 1}, {1, -1}}), s, b);
  CHECK(b[0] == 0);

  if (failures) return 1;
  std::printf("ok\n");
  return 0;
}
