// Internal helpers shared by the libtaser kernels (device side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "taser.h"

#define TASER_FULL_MASK 0xffffffffu

// Bounds-checked debug build (compiled with -DTASER_DEBUG, libtaser_debug.so).
//   TASER_IN(i, n)   is true when 0 <= i < n.  Otherwise it counts a failure, records the
//                    first failing translation unit, line and index, and is false, so that
//                    the access it guards is skipped.  Nothing traps or waits.
//   TASER_FINITE(v)  counts a non-finite output value.
// Each translation unit has its own counters (TASER_TU numbers it); the host collects them
// through taser_debug_report.  In release builds TASER_IN is the constant true and
// TASER_FINITE nothing, so the compiler removes every check.
#ifndef TASER_TU
#define TASER_TU 0
#endif
#ifdef TASER_DEBUG
namespace taser {
namespace dbg {
struct Word {
  unsigned long long fails;      // failed index checks
  unsigned long long first;      // TU << 56 | line << 32 | (index & 0xffffffff) of the first
  unsigned long long nonfinite;  // non-finite output values
};
static __device__ Word word;
static __device__ __noinline__ void record(int line, long long idx) {
  const unsigned long long prior = atomicAdd(&word.fails, 1ull);
  if (prior == 0ull)
    word.first = ((unsigned long long)TASER_TU << 56) | ((unsigned long long)(line & 0xffffff) << 32) |
                 ((unsigned long long)idx & 0xffffffffull);
}
static __device__ __forceinline__ bool in(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  record(line, i);
  return false;
}
static __device__ __forceinline__ void finite(float v) {
  if (!isfinite(v)) atomicAdd(&word.nonfinite, 1ull);
}
}  // namespace dbg
}  // namespace taser
#define TASER_IN(i, n) (taser::dbg::in((long long)(i), (long long)(n), __LINE__))
#define TASER_FINITE(v) taser::dbg::finite(v)
// Host: copies this translation unit's counters into out[3] and clears them.
#define TASER_DEBUG_COLLECTOR(name)                                                        \
  namespace taser {                                                                        \
  namespace dbg {                                                                          \
  cudaError_t take_##name(unsigned long long* out) {                                       \
    Word w{};                                                                              \
    cudaError_t e = cudaMemcpyFromSymbol(&w, word, sizeof(Word));                          \
    if (e != cudaSuccess) return e;                                                        \
    out[0] += w.fails;                                                                     \
    if (out[1] == 0ull) out[1] = w.first;                                                  \
    out[2] += w.nonfinite;                                                                 \
    const Word zero{};                                                                     \
    return cudaMemcpyToSymbol(word, &zero, sizeof(Word));                                  \
  }                                                                                        \
  }                                                                                        \
  }
#else
#define TASER_IN(i, n) true
#define TASER_FINITE(v) ((void)0)
#define TASER_DEBUG_COLLECTOR(name)
#endif
// Guards that vanish from release builds token for token, so that a kernel's release code
// keeps its exact shape: TASER_CHECKED(c) stmt is `if (c) stmt` in the debug build and
// `stmt` otherwise; `cond TASER_AND(c)` is `cond && (c)` in the debug build and `cond`
// otherwise.  (Checks folded in as constants changed the release code generation of two
// kernels measurably, 8-9%.)
#ifdef TASER_DEBUG
#define TASER_CHECKED(c) if (c)
#define TASER_AND(c) &&(c)
#else
#define TASER_CHECKED(c)
#define TASER_AND(c)
#endif

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
  // The pools' extents are not passed in: a debug build checks that the offsets are
  // non-negative (the instance's own indices are checked where they are used).
  (void)(TASER_IN(it.t_off, INT64_MAX) && TASER_IN(it.d_off, INT64_MAX) && TASER_IN(it.s_off, INT64_MAX) &&
         TASER_IN(it.l_off + 1, INT64_MAX));
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
  int64_t n;   // items of the call (the length of list and items)
  __device__ __forceinline__ int count() const { return *((volatile const int*)meta + 4 + b); }
  __device__ __forceinline__ int pop(int k) const { return atomicAdd(meta + 8 + b, k); }
  __device__ __forceinline__ int item_at(int pos) const {
    const int at = meta[b] + pos;
    const int idx = TASER_IN(at, n) ? list[at] : 0;
    return TASER_IN(idx, n) ? idx : 0;
  }
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
