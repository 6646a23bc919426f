// Warp-level tensor-core helpers shared by the tensor-core detection kernels (Algorithm 1)
// and the tensor-core unfolded TASER kernels: mma.sync m16n8k16 with BF16 or FP16
// operands and FP32 accumulation, operand packing, and the tile bookkeeping of the
// triangular product L~ T^ (one warp per instance, L~ held in the accumulator layout).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace taser {

template <bool FP16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (FP16) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
  }
}

template <bool FP16>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if constexpr (FP16) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// The packed f32x2 operations (common.cuh) handle the two columns (2tq, 2tq + 1) an
// accumulator register pair holds with one instruction.
// acc[e], acc[e + 1] = f(acc[e], acc[e + 1]) for a packed operation f.
#define TASER_PAIR_APPLY(arr, e, expr)          \
  do {                                          \
    const uint64_t _x = f2pack(arr[e], arr[e + 1]); \
    const uint64_t _y = (expr);                 \
    f2unpack(_y, arr[e], arr[e + 1]);           \
  } while (0)

// BF16 split x = hi + lo of a float pair (hi = bf16(x), lo = bf16(x - hi)): the products
// hi hi' + hi lo' + lo hi' carry about 2^-16 relative error, where a single BF16 product
// carries 2^-8.  Used only by the objective monitor, whatever the path's precision.
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  hi = pack2<false>(x0, x1);
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
  lo = pack2<false>(x0 - h0, x1 - h1);
}

// Tile bookkeeping for bucket NB (16 or 32).
template <int NB>
struct TcCfg {
  static constexpr int KT = NB / 16;     // k-tiles over the variable columns
  static constexpr int NT = NB / 8;      // n-tiles over the variable columns
  static constexpr int MT = KT + 1;      // m-tiles; the last holds row NB only
  static constexpr int NV = 2 * NT;      // column-sum values per lane before reduction
  static constexpr int WARPS = 4;
  __host__ __device__ static constexpr bool has_tile(int M, int n) {
    return M == MT - 1 ? true : n <= 2 * M + 1;
  }
  __host__ __device__ static constexpr int kmax(int M) { return M == MT - 1 ? KT - 1 : M; }
};

}  // namespace taser
