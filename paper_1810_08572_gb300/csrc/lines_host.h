// Host part of the line preconditioner (la.cuh, lines.cu): the chains of
// strongly coupled cells and their storage layout.  Plain C++ (no CUDA), so
// that the layout can be checked without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

namespace fvs {

struct LineLayout {
  int64_t nlines = 0, ngroups = 0, padded = 0;
  int max_len = 0;
  std::vector<int64_t> goff;   // [ngroups + 1] first entry of each group of 32 lines
  std::vector<int32_t> llen;   // [ngroups * 32] length of each line (0: no line)
  std::vector<int32_t> cell;   // [padded] cell at entry goff[g] + 32 * position + lane (-1: padding)
  std::vector<int8_t> sprev, snext;   // slot of the previous / next cell of the line in the cell's row (-1: none)
};

// Chains from an n-row slot-major ELL operator (entry k of row i at
// k * n + i, w slots): every row keeps its two largest off-diagonal
// magnitudes (the first slot wins a tie), the second only if it is at least
// `strong` times the first (so that the chains of a thin direction do not
// join at their ends through a weak coupling); i and j are joined where
// each chose the other, so every cell has at most two partners and the
// chains are paths and cycles.  Paths are walked from an end, cycles from
// their first cell; a walk longer than max_line starts a new line.  Lines
// are sorted by decreasing length and stored 32 to a group, each group
// padded to its longest line, position-major inside the group.
inline void build_line_layout(const int32_t* col, const double* val, int64_t n, int w, int max_line,
                              LineLayout& L, double strong = 0.25) {
  L = LineLayout();
  if (n <= 0) return;
  auto at = [&](int k, int64_t i) { return (size_t)k * (size_t)n + (size_t)i; };
  std::vector<int32_t> best((size_t)2 * n, -1);
  for (int64_t i = 0; i < n; ++i) {
    double m0 = 0.0, m1 = 0.0;
    int32_t b0 = -1, b1 = -1;
    for (int k = 0; k < w; ++k) {
      const int32_t j = col[at(k, i)];
      if (j < 0 || j >= n || j == i) continue;
      const double a = std::fabs(val[at(k, i)]);
      if (!(a > 0.0)) continue;
      if (a > m0) {
        if (j != b0) {
          m1 = m0;
          b1 = b0;
        }
        m0 = a;
        b0 = j;
      } else if (a > m1 && j != b0) {
        m1 = a;
        b1 = j;
      }
    }
    best[2 * i] = b0;
    best[2 * i + 1] = (m1 >= strong * m0) ? b1 : -1;
  }
  auto chose = [&](int32_t j, int64_t i) { return best[2 * j] == i || best[2 * j + 1] == i; };
  std::vector<int32_t> nb((size_t)2 * n, -1);
  for (int64_t i = 0; i < n; ++i) {
    int q = 0;
    for (int t = 0; t < 2; ++t) {
      const int32_t j = best[2 * i + t];
      if (j >= 0 && chose(j, i)) nb[2 * i + q++] = j;
    }
  }
  std::vector<uint8_t> seen((size_t)n, 0);
  std::vector<int32_t> order;
  order.reserve((size_t)n);
  std::vector<int64_t> start;
  auto walk = [&](int64_t i0) {
    int64_t prev = -1, cur = i0;
    start.push_back((int64_t)order.size());
    int len = 0;
    while (cur >= 0 && !seen[cur]) {
      if (len == max_line) {
        start.push_back((int64_t)order.size());
        len = 0;
      }
      seen[cur] = 1;
      order.push_back((int32_t)cur);
      ++len;
      int64_t next = -1;
      for (int t = 0; t < 2; ++t) {
        const int32_t j = nb[2 * cur + t];
        if (j >= 0 && j != prev && !seen[j]) {
          next = j;
          break;
        }
      }
      prev = cur;
      cur = next;
    }
  };
  for (int64_t i = 0; i < n; ++i)
    if (!seen[i] && (nb[2 * i] < 0 || nb[2 * i + 1] < 0)) walk(i);
  for (int64_t i = 0; i < n; ++i)
    if (!seen[i]) walk(i);
  start.push_back((int64_t)order.size());
  L.nlines = (int64_t)start.size() - 1;

  std::vector<int64_t> ids((size_t)L.nlines);
  std::iota(ids.begin(), ids.end(), 0);
  auto length = [&](int64_t q) { return start[q + 1] - start[q]; };
  std::stable_sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b) { return length(a) > length(b); });
  L.ngroups = (L.nlines + 31) / 32;
  L.goff.assign((size_t)L.ngroups + 1, 0);
  L.llen.assign((size_t)L.ngroups * 32, 0);
  for (int64_t g = 0; g < L.ngroups; ++g) {
    const int lg = (int)length(ids[g * 32]);
    L.max_len = std::max(L.max_len, lg);
    L.goff[g + 1] = L.goff[g] + (int64_t)lg * 32;
  }
  L.padded = L.goff[L.ngroups];
  L.cell.assign((size_t)L.padded, -1);
  L.sprev.assign((size_t)L.padded, -1);
  L.snext.assign((size_t)L.padded, -1);
  auto slot_of = [&](int32_t c, int32_t j) -> int8_t {
    for (int k = 0; k < w; ++k)
      if (col[at(k, c)] == j) return (int8_t)k;
    return -1;
  };
  for (int64_t q = 0; q < L.nlines; ++q) {
    const int64_t line = ids[q], g = q / 32;
    const int lane = (int)(q % 32);
    const int len = (int)length(line);
    L.llen[q] = len;
    for (int pos = 0; pos < len; ++pos) {
      const int64_t idx = L.goff[g] + (int64_t)pos * 32 + lane;
      const int32_t c = order[start[line] + pos];
      L.cell[idx] = c;
      if (pos > 0) L.sprev[idx] = slot_of(c, order[start[line] + pos - 1]);
      if (pos + 1 < len) L.snext[idx] = slot_of(c, order[start[line] + pos + 1]);
    }
  }
}

}  // namespace fvs
