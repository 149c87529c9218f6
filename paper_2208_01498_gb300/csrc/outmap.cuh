// Output layout map of a GEMM node: where element C[b][m][n] is stored in
// the layout its consumer reads (see GemmDesc::c_pos).
#pragma once
#include <cstdint>

#include "tnc_kernels.h"

namespace tnc {

// output offset of bits v placed at positions pos[0..n)
__device__ __forceinline__ uint64_t scatter_bits(uint64_t v, const int8_t* pos, int n) {
  uint64_t r = 0;
  for (int i = 0; i < n; ++i) r |= ((v >> i) & 1) << pos[i];
  return r;
}

// element offset of C[b][m][n] in the consumer's layout
struct OutMap {
  int ident, nN, nM, nB;
  int8_t pos[kMaxRank];
  __device__ __forceinline__ uint64_t row(int64_t b, int64_t m, int64_t M, int64_t N) const {
    if (ident) return ((uint64_t)b * M + m) * N;
    return scatter_bits(m, pos + nN, nM) | scatter_bits(b, pos + nN + nM, nB);
  }
  __device__ __forceinline__ uint64_t col(int64_t n) const {
    if (ident) return n;
    return scatter_bits(n, pos, nN);
  }
};

inline OutMap out_map(const GemmDesc& d) {
  OutMap o;
  o.ident = d.c_ident;
  o.nN = d.nN, o.nM = d.nM, o.nB = d.nB;
  for (int i = 0; i < kMaxRank; ++i) o.pos[i] = d.c_pos[i];
  return o;
}

}  // namespace tnc
