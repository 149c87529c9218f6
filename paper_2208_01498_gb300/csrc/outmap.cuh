// Output layout map of a GEMM node: where element C[b][m][n] is stored in
// the layout its consumer reads (see GemmDesc::c_pos).
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "tnc_kernels.h"

namespace tnc {

// output offset of bits v placed at positions pos[0..n)
__device__ __forceinline__ uint64_t scatter_bits(uint64_t v, const int8_t* pos, int n) {
  uint64_t r = 0;
  for (int i = 0; i < n; ++i) r |= ((v >> i) & 1) << pos[i];
  return r;
}

// one value of a hi/lo plane pair: hi = x rounded (bf16 or tf32), lo = the
// remainder rounded again
__device__ __forceinline__ void put_split(void* base, uint64_t plane, uint64_t idx, float x, int tf32) {
  if (tf32) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - __uint_as_float(h)));
    ((uint32_t*)base)[idx] = h;
    ((uint32_t*)base)[plane + idx] = l;
  } else {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    ((__nv_bfloat16*)base)[idx] = h;
    ((__nv_bfloat16*)base)[plane + idx] = l;
  }
}

// element offset of C[b][m][n] in the consumer's layout, and its store in
// the consumer's operand format
struct OutMap {
  int ident, nN, nM, nB;
  int fmt, kbits, tf32;
  uint64_t plane;
  int8_t pos[kMaxRank];
  __device__ __forceinline__ void store(void* base, uint64_t e, float2 v) const {
    if (fmt == 0) {
      ((float2*)base)[e] = v;
    } else if (fmt == 1) {
      put_split(base, plane, 2 * e, v.x, tf32);
      put_split(base, plane, 2 * e + 1, v.y, tf32);
    } else {
      const uint64_t bn = e >> kbits, k = e & (((uint64_t)1 << kbits) - 1);
      const uint64_t i0 = (bn << (kbits + 2)) + 2 * k, i1 = i0 + ((uint64_t)2 << kbits);
      put_split(base, plane, i0, v.x, tf32);
      put_split(base, plane, i0 + 1, -v.y, tf32);
      put_split(base, plane, i1, v.y, tf32);
      put_split(base, plane, i1 + 1, v.x, tf32);
    }
  }
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
  o.fmt = d.c_fmt, o.kbits = d.c_kbits, o.tf32 = d.c_tf32, o.plane = d.c_plane;
  for (int i = 0; i < kMaxRank; ++i) o.pos[i] = d.c_pos[i];
  return o;
}

}  // namespace tnc
