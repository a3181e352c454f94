// Test shim: exposes the host layout of the line preconditioner
// (paper_1810_08572_gb300/csrc/lines_host.h) to ctypes, without CUDA.
#include "../paper_1810_08572_gb300/csrc/lines_host.h"

extern "C" {

// sizes[0..3] = nlines, ngroups, padded, max_len.  The arrays are filled
// only when cap_groups >= ngroups and cap_padded >= padded.
int line_layout(const int32_t* col, const double* val, int64_t n, int w, int max_line, int64_t* sizes,
                int64_t cap_groups, int64_t cap_padded, int64_t* goff, int32_t* llen, int32_t* cell, int8_t* sprev,
                int8_t* snext) {
  fvs::LineLayout L;
  fvs::build_line_layout(col, val, n, w, max_line, L);
  sizes[0] = L.nlines;
  sizes[1] = L.ngroups;
  sizes[2] = L.padded;
  sizes[3] = L.max_len;
  if (cap_groups < L.ngroups || cap_padded < L.padded) return 1;
  for (int64_t g = 0; g <= L.ngroups; ++g) goff[g] = L.goff[g];
  for (int64_t t = 0; t < L.ngroups * 32; ++t) llen[t] = L.llen[t];
  for (int64_t e = 0; e < L.padded; ++e) {
    cell[e] = L.cell[e];
    sprev[e] = L.sprev[e];
    snext[e] = L.snext[e];
  }
  return 0;
}
}
