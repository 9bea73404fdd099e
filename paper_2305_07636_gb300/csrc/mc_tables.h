// Host-side classification of the problem's geometry and tally axes for the walk's shortcuts:
// plain C++ (no CUDA), so that it is compiled into the library and, on its own, into a host test.
// Not part of the ABI.
#pragma once
#include <cmath>
#include <vector>

#include "../../include/mc.h"

namespace mcgb {

// First-guess parameters of a bin search over float edges e[0..n] (the device's bin_find): kind 1
// for equal spacing (bin floor((x - a) b)), kind 2 for geometric spacing from edge 1 on, as in
// log-spaced time bins after a first bin [0, e1] (bin 1 + floor(log2(x a) b)), kind 0 otherwise
// (bisection).  The device corrects every guess against the edges, so only the search's cost
// depends on these numbers.
inline void bin_guess_params(const std::vector<float>& e, int& kind, float& a, float& b) {
  kind = 0;
  a = b = 0.0f;
  const int n = (int)e.size() - 1;
  if (n < 4) return;
  const double w = (double)e[n] - (double)e[0];
  bool lin = w > 0.0;
  for (int k = 1; k < n && lin; ++k)
    lin = std::fabs((double)e[k] - ((double)e[0] + w * k / n)) <= 1e-3 * w / n;
  if (lin) {
    kind = 1;
    a = e[0];
    b = (float)(n / w);
    return;
  }
  if (!(e[1] > 0.0f) || !(e[n] > e[1])) return;
  const double r = std::log2((double)e[n] / (double)e[1]) / (n - 1);
  bool geo = r > 0.0;
  for (int k = 2; k < n && geo; ++k)
    geo = std::fabs(std::log2((double)e[k] / (double)e[1]) - r * (k - 1)) <= 1e-3 * r;
  if (geo) {
    kind = 2;
    a = (float)(1.0 / (double)e[1]);
    b = (float)(1.0 / r);
  }
}

// The box-cell entry of a cell (7 ints): b[0] = 1 when the cell is bounded by axis-aligned planes
// only, at most one lower and one upper plane per axis; then per axis its lower and upper plane as
// surface | (position in the cell's halfspace list << 16), or -1.  A halfspace of sense +1 keeps
// the side where the plane's function is positive, so its plane bounds the cell from below.
inline void box_cell_entry(const mc_cell& C, const mc_surface* surfaces, int b[7]) {
  for (int i = 0; i < 7; ++i) b[i] = -1;
  b[0] = 1;
  for (int i = 0; i < C.n_halfspaces; ++i) {
    const int s = C.surface[i], k = surfaces[s].kind;
    if (k != MC_SURF_PX && k != MC_SURF_PY && k != MC_SURF_PZ) {
      b[0] = 0;
      return;
    }
    int& slot = b[1 + 2 * k + (C.sense[i] > 0 ? 0 : 1)];
    if (slot != -1) {
      b[0] = 0;
      return;
    }
    slot = s | (i << 16);
  }
}

}  // namespace mcgb
