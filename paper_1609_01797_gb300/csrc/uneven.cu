// Uneven batches (problems of different N and t_max in one call): a size-bucketed work
// queue built on the device and one persistent, queue-fed kernel per bucket.  The whole
// sequence is stream-ordered without host synchronisation, so it can be captured in a
// CUDA graph and replayed with a single launch.
#include "common.cuh"

namespace taser {

cudaError_t detect_fp32_queue(int nb, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, int literal, float* L_pool, int8_t* s_pool, uint32_t* flags,
                              cudaStream_t st);
cudaError_t detect_tc_queue(int nb, bool fp16, const Queue& q, int blocks_per_sm, int pop, const float* T_pool,
                            const float* D_pool, const float* tau, int literal, float* L_pool, int8_t* s_pool,
                            uint32_t* flags, cudaStream_t st);

constexpr int kClasses = 64;               // t_max classes per bucket (64 = 64 and more)
constexpr int kKeys = 4 * kClasses;
constexpr int kMetaInts = 16;              // start[4], count[4], head[4], spare
static_assert(kMetaInts * sizeof(int) <= 256, "the queue metadata lives in the 256 bytes after the item list");

__device__ __forceinline__ int bucket_index(int N) {
  const int nv = N - 1;
  return nv <= 8 ? 0 : nv <= 16 ? 1 : nv <= 32 ? 2 : 3;
}

// Counting sort of the item indices by (bucket, t_max descending): the longest items of a
// bucket come first, which balances the persistent kernels' tails.  One block.
__global__ void __launch_bounds__(1024)
bucketize_kernel(int n, const taser_item* __restrict__ items, int* __restrict__ list, int* __restrict__ meta,
                 uint32_t* __restrict__ flags) {
  __shared__ int hist[kKeys];
  __shared__ int offs[kKeys];
  const int tid = threadIdx.x;
  for (int k = tid; k < kKeys; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const taser_item it = items[i];
    if (it.N >= 2 && it.N <= TASER_MAX_N && it.t_max >= 1) {
      const int key = bucket_index(it.N) * kClasses + (kClasses - min(it.t_max, kClasses));
      atomicAdd(&hist[key], 1);
    } else if (flags != nullptr) {
      flags[i] |= TASER_FLAG_BAD_ITEM;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int k = 0; k < kKeys; ++k) {
      offs[k] = run;
      run += hist[k];
    }
    for (int b = 0; b < 4; ++b) {
      int cnt = 0;
      for (int k = 0; k < kClasses; ++k) cnt += hist[b * kClasses + k];
      meta[b] = offs[b * kClasses];
      meta[4 + b] = cnt;
      meta[8 + b] = 0;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const taser_item it = items[i];
    if (it.N >= 2 && it.N <= TASER_MAX_N && it.t_max >= 1) {
      const int key = bucket_index(it.N) * kClasses + (kClasses - min(it.t_max, kClasses));
      list[atomicAdd(&offs[key], 1)] = i;
    }
  }
}

size_t uneven_workspace_bytes(int64_t n_items) {
  const size_t list = ((size_t)n_items * sizeof(int) + 255) & ~size_t(255);
  return list + 256;
}

cudaError_t detect_fx14_queue(int nb, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, float* L_pool, int8_t* s_pool, uint32_t* flags, cudaStream_t st);

cudaError_t detect_uneven(int64_t n_items, const taser_item* items, const float* T_pool, const float* D_pool,
                          const float* tau, int precision, int literal, float* L_pool, int8_t* s_pool,
                          uint32_t* flags, void* workspace, const taser_uneven_tuning* tuning, cudaStream_t st) {
  int* list = static_cast<int*>(workspace);
  int* meta = reinterpret_cast<int*>(static_cast<char*>(workspace) +
                                     (((size_t)n_items * sizeof(int) + 255) & ~size_t(255)));
  bucketize_kernel<<<1, 1024, 0, st>>>((int)n_items, items, list, meta, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int order[4] = {3, 2, 1, 0};        // the heaviest bucket first
  for (int oi = 0; oi < 4; ++oi) {
    const int b = order[oi];
    const int nb = 8 << b;
    Queue q;
    q.items = items;
    q.list = list;
    q.meta = meta;
    q.b = b;
    const int bps = tuning != nullptr ? tuning->blocks_per_sm[b] : 0;
    const int pop = tuning != nullptr ? tuning->pop[b] : 1;
    if (precision == TASER_FIXED14) {
      e = detect_fx14_queue(nb, q, bps, T_pool, D_pool, tau, L_pool, s_pool, flags, st);
    } else if (precision != TASER_FP32 && nb >= 16) {
      e = detect_tc_queue(nb, precision == TASER_FP16_TC, q, bps, pop, T_pool, D_pool, tau, literal, L_pool, s_pool,
                          flags, st);
    } else {
      e = detect_fp32_queue(nb, q, bps, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace taser
