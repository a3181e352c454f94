#pragma once
#include "common.cuh"

namespace fvs {
struct ScanWork {
  DBuf<int32_t> bsum;
  DBuf<int32_t> total;   // [1] sum of all inputs (device)
  fvs_status ensure(int64_t n);
};
// out[i] = sum_{j<i} in[j]; the grand total lands in w.total[0].
fvs_status exclusive_scan(cudaStream_t s, ScanWork& w, int64_t n, const int32_t* in, int32_t* out);
}  // namespace fvs
