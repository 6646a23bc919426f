// Internal helpers shared by the libtaser kernels (device side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "taser.h"

#define TASER_FULL_MASK 0xffffffffu

namespace taser {

// Bucket of variable columns used by the detection and spectral kernels: a problem
// of size N (N-1 variable columns plus the augmented last index) runs in the bucket
// NB >= N-1, NB in {8, 16, 32, 64}.  Real index r < N-1 maps to bucket index r, the
// last real index N-1 maps to bucket index NB; bucket indices N-1..NB-1 are padding
// with zero T~ rows/columns and zero D, which leaves the real entries unchanged.
__host__ __device__ inline int bucket_of(int N) {
  const int nv = N - 1;
  return nv <= 8 ? 8 : nv <= 16 ? 16 : nv <= 32 ? 32 : 64;
}

// Bucket index -> real index (or -1 for padding).
__device__ __forceinline__ int bucket_to_real(int i, int N, int NB) {
  return i < N - 1 ? i : (i == NB ? N - 1 : -1);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(TASER_FULL_MASK, v, o);
  return v;
}

}  // namespace taser
