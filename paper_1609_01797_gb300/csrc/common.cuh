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

// One detection problem as the iteration kernels see it.
struct Job {
  const float* T;      // T~, N x N row-major
  const float* D;      // D, N
  const float* tau;    // step size (one float)
  float* L;            // L~ output (N x N) or nullptr
  int8_t* s;           // decisions (N - 1)
  uint32_t* flag;      // flag word or nullptr
  int N;
  int t_max;
};

__device__ __forceinline__ Job dense_job(int64_t inst, int N, int t_max, const float* Tt, const float* Dg,
                                         const float* tau, float* L, int8_t* s, uint32_t* flags) {
  Job j;
  j.T = Tt + inst * (int64_t)N * N;
  j.D = Dg + inst * (int64_t)N;
  j.tau = tau + inst;
  j.L = L != nullptr ? L + inst * (int64_t)N * N : nullptr;
  j.s = s + inst * (int64_t)(N - 1);
  j.flag = flags != nullptr ? flags + inst : nullptr;
  j.N = N;
  j.t_max = t_max;
  return j;
}

__device__ __forceinline__ Job item_job(const taser_item& it, int64_t idx, const float* T_pool, const float* D_pool,
                                        const float* tau, float* L_pool, int8_t* s_pool, uint32_t* flags) {
  Job j;
  j.T = T_pool + it.t_off;
  j.D = D_pool + it.d_off;
  j.tau = tau + idx;
  j.L = (L_pool != nullptr && it.l_off >= 0) ? L_pool + it.l_off : nullptr;
  j.s = s_pool + it.s_off;
  j.flag = flags != nullptr ? flags + idx : nullptr;
  j.N = it.N;
  j.t_max = it.t_max;
  return j;
}

// Work queue of one size bucket, filled on the device: item indices
// list[meta[b] .. meta[b] + meta[4 + b]), popped through the atomic counter meta[8 + b].
struct Queue {
  const taser_item* items;
  const int* list;
  int* meta;
  int b;
  __device__ __forceinline__ int count() const { return *((volatile const int*)meta + 4 + b); }
  __device__ __forceinline__ int pop(int k) const { return atomicAdd(meta + 8 + b, k); }
  __device__ __forceinline__ int item_at(int pos) const { return list[meta[b] + pos]; }
};

// Packed FP32 pairs for the f32x2 FMA/multiply instructions: a pair lives in one 64-bit
// register, and each half of a result is the IEEE result of the scalar operation.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(TASER_FULL_MASK, v, o);
  return v;
}

}  // namespace taser
