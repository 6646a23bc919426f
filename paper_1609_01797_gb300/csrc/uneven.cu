// Uneven batches (problems of different N and t_max in one call): a size-bucketed work
// queue built on the device and one persistent, queue-fed kernel per bucket.  The whole
// sequence is stream-ordered without host synchronisation, so it can be captured in a
// CUDA graph and replayed with a single launch.
#include "common.cuh"

namespace taser {

cudaError_t detect_fp32_queue(int nb, const Queue& q, int blocks_per_sm, int rounds, const float* T_pool,
                              const float* D_pool, const float* tau, int literal, float* L_pool, int8_t* s_pool,
                              uint32_t* flags, cudaStream_t st);
cudaError_t detect_tc_queue(int nb, bool fp16, const Queue& q, int blocks_per_sm, int pop, const float* T_pool,
                            const float* D_pool, const float* tau, int literal, float* L_pool, int8_t* s_pool,
                            uint32_t* flags, cudaStream_t st);

constexpr int kClasses = 64;               // t_max classes per bucket (64 = 64 and more)
// Items per queue pop when no tuning is given, per bucket N <= 9 / 17 / 33 / 65.
constexpr int kTcPopDefault[4] = {1, 4, 2, 1};
constexpr int kFp32PopDefault[4] = {4, 2, 1, 1};   // one warp-load
constexpr int kKeys = 4 * kClasses;
constexpr int kMetaInts = 16;              // start[4], count[4], head[4], spare
static_assert(kMetaInts * sizeof(int) <= 256, "the queue metadata lives in the 256 bytes after the item list");

__device__ __forceinline__ int bucket_index(int N) {
  const int nv = N - 1;
  return nv <= 8 ? 0 : nv <= 16 ? 1 : nv <= 32 ? 2 : 3;
}

// Counting sort of the item indices by (bucket, t_max descending): the longest items of a
// bucket come first, which balances the persistent kernels' tails.  Three grid-wide passes:
// per-block histograms added into a global one, an exclusive scan (one block), and a
// scatter in which each block reserves one range per key with a single global atomic.
__device__ __forceinline__ int item_key(const taser_item& it) {
  return bucket_index(it.N) * kClasses + (kClasses - min(it.t_max, kClasses));
}
// The bounds-checked debug build also rejects (and counts) negative pool offsets; the
// release build takes the offsets as given.
__device__ __forceinline__ bool item_ok(const taser_item& it) {
  return it.N >= 2 && it.N <= TASER_MAX_N && it.t_max >= 1 && TASER_IN(it.t_off, INT64_MAX) &&
         TASER_IN(it.d_off, INT64_MAX) && TASER_IN(it.s_off, INT64_MAX) && TASER_IN(it.l_off + 1, INT64_MAX);
}

constexpr int kSortThreads = 256;
constexpr int kSortItemsPerBlock = 4096;

__global__ void __launch_bounds__(kSortThreads)
bucket_hist_kernel(int n, const taser_item* __restrict__ items, int* __restrict__ ghist,
                   uint32_t* __restrict__ flags) {
  __shared__ int hist[kKeys];
  for (int k = threadIdx.x; k < kKeys; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const int i0 = blockIdx.x * kSortItemsPerBlock, i1 = min(n, i0 + kSortItemsPerBlock);
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const taser_item it = items[i];
    if (item_ok(it)) {
      if (TASER_IN(item_key(it), kKeys)) atomicAdd(&hist[item_key(it)], 1);
    } else if (flags != nullptr) {
      flags[i] |= TASER_FLAG_BAD_ITEM;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kKeys; k += blockDim.x)
    if (hist[k] != 0) atomicAdd(&ghist[k], hist[k]);
}

// One block of kKeys threads: goffs = exclusive scan of ghist; queue metadata per bucket.
__global__ void __launch_bounds__(kKeys)
bucket_scan_kernel(const int* __restrict__ ghist, int* __restrict__ goffs, int* __restrict__ meta) {
  __shared__ int sc[kKeys];
  const int k = threadIdx.x;
  sc[k] = ghist[k];
  __syncthreads();
  for (int o = 1; o < kKeys; o <<= 1) {     // inclusive Hillis-Steele scan
    const int v = k >= o ? sc[k - o] : 0;
    __syncthreads();
    sc[k] += v;
    __syncthreads();
  }
  const int excl = sc[k] - ghist[k];
  goffs[k] = excl;
  if (k % kClasses == 0) {
    const int b = k / kClasses;
    meta[b] = excl;
    meta[4 + b] = sc[k + kClasses - 1] - excl;
    meta[8 + b] = 0;
  }
}

__global__ void __launch_bounds__(kSortThreads)
bucket_scatter_kernel(int n, const taser_item* __restrict__ items, int* __restrict__ goffs,
                      int* __restrict__ list) {
  __shared__ int hist[kKeys];
  __shared__ int base[kKeys];
  for (int k = threadIdx.x; k < kKeys; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const int i0 = blockIdx.x * kSortItemsPerBlock, i1 = min(n, i0 + kSortItemsPerBlock);
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const taser_item it = items[i];
    if (item_ok(it) && TASER_IN(item_key(it), kKeys)) atomicAdd(&hist[item_key(it)], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kKeys; k += blockDim.x) {
    base[k] = hist[k] != 0 ? atomicAdd(&goffs[k], hist[k]) : 0;
    hist[k] = 0;
  }
  __syncthreads();
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const taser_item it = items[i];
    if (item_ok(it)) {
      const int key = item_key(it);
      if (!TASER_IN(key, kKeys)) continue;
      const int at = base[key] + atomicAdd(&hist[key], 1);
      if (TASER_IN(at, n)) list[at] = i;
    }
  }
}

// Workspace: [list: n_items ints, 256-byte aligned] [meta: 256 bytes] [histogram: kKeys ints]
// [running offsets: kKeys ints].
size_t uneven_workspace_bytes(int64_t n_items) {
  const size_t list = ((size_t)n_items * sizeof(int) + 255) & ~size_t(255);
  return list + 256 + 2 * kKeys * sizeof(int);
}

cudaError_t detect_fx14_queue(int nb, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, float* L_pool, int8_t* s_pool, uint32_t* flags, cudaStream_t st);

namespace {
// Streams (per host thread and device) on which the bucket kernels run after the sort: the
// N <= 65 bucket, the longest, on a high-priority stream; the other three back to back on
// a low-priority one, so their blocks take the SMs that the heavy kernel's blocks free in
// its tail.  Forked from and joined back into the caller's stream with events, which a
// CUDA graph capture records as a branch.  Created on first use and kept.
struct BucketLanes {
  cudaStream_t hi = nullptr, lo = nullptr;
  cudaEvent_t fork = nullptr, join_hi = nullptr, join_lo = nullptr;
};
cudaError_t bucket_lanes(BucketLanes*& out) {
  thread_local BucketLanes lanes[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  BucketLanes& b = lanes[dev];
  if (b.hi == nullptr) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.hi, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.lo, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_hi, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_lo, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      b = BucketLanes{};
      return e;
    }
  }
  out = &b;
  return cudaSuccess;
}
}  // namespace

cudaError_t detect_uneven(int64_t n_items, const taser_item* items, const float* T_pool, const float* D_pool,
                          const float* tau, int precision, int literal, float* L_pool, int8_t* s_pool,
                          uint32_t* flags, void* workspace, const taser_uneven_tuning* tuning, cudaStream_t st) {
  int* list = static_cast<int*>(workspace);
  int* meta = reinterpret_cast<int*>(static_cast<char*>(workspace) +
                                     (((size_t)n_items * sizeof(int) + 255) & ~size_t(255)));
  int* ghist = meta + 256 / sizeof(int);
  int* goffs = ghist + kKeys;
  cudaError_t e = cudaMemsetAsync(ghist, 0, kKeys * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int sort_blocks = (int)((n_items + kSortItemsPerBlock - 1) / kSortItemsPerBlock);
  if (sort_blocks > 0)
    bucket_hist_kernel<<<sort_blocks, kSortThreads, 0, st>>>((int)n_items, items, ghist, flags);
  bucket_scan_kernel<<<1, kKeys, 0, st>>>(ghist, goffs, meta);
  if (sort_blocks > 0)
    bucket_scatter_kernel<<<sort_blocks, kSortThreads, 0, st>>>((int)n_items, items, goffs, list);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BucketLanes* lanes = nullptr;
  e = bucket_lanes(lanes);
  if (e == cudaSuccess) e = cudaEventRecord(lanes->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lanes->hi, lanes->fork, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lanes->lo, lanes->fork, 0);
  if (e != cudaSuccess) return e;
  const int order[4] = {3, 2, 1, 0};        // the heaviest bucket first
  // A failed bucket launch stops the loop but the side streams are still joined back
  // into `st` below, so a stream capture in progress stays joined and reports the launch
  // error instead of an unjoined-capture error.
  cudaError_t launch_err = cudaSuccess;
  for (int oi = 0; oi < 4 && launch_err == cudaSuccess; ++oi) {
    const int b = order[oi];
    const cudaStream_t bs = b == 3 ? lanes->hi : lanes->lo;
    const int nb = 8 << b;
    Queue q;
    q.items = items;
    q.list = list;
    q.meta = meta;
    q.b = b;
    q.n = n_items;
    const int bps = tuning != nullptr ? tuning->blocks_per_sm[b] : 0;
    const bool tc = precision != TASER_FP32 && precision != TASER_FIXED14 && nb >= 16;
    // Default items per pop (measured on the 200,000-item batch): the short tensor-core
    // jobs take 4 (N <= 17) or 2 (N <= 33) items per atomic; on the FP32 path larger pops
    // than one warp-load gained nothing.
    const int pop_default = tc ? kTcPopDefault[b] : kFp32PopDefault[b];
    const int pop = tuning != nullptr && tuning->pop[b] > 0 ? tuning->pop[b] : pop_default;
    if (precision == TASER_FIXED14) {
      e = detect_fx14_queue(nb, q, bps, T_pool, D_pool, tau, L_pool, s_pool, flags, bs);
    } else if (tc) {
      e = detect_tc_queue(nb, precision == TASER_FP16_TC, q, bps, pop, T_pool, D_pool, tau, literal, L_pool, s_pool,
                          flags, bs);
    } else {
      // FP32: whole warp-loads per pop (4 / 2 / 1 / 1 items at N <= 9 / 17 / 33 / 65).
      const int per_load = nb <= 8 ? 4 : (nb == 16 ? 2 : 1);
      e = detect_fp32_queue(nb, q, bps, (pop + per_load - 1) / per_load, T_pool, D_pool, tau, literal, L_pool,
                            s_pool, flags, bs);
    }
    launch_err = e;
  }
  e = cudaEventRecord(lanes->join_hi, lanes->hi);
  if (e == cudaSuccess) e = cudaEventRecord(lanes->join_lo, lanes->lo);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, lanes->join_hi, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, lanes->join_lo, 0);
  return launch_err != cudaSuccess ? launch_err : e;
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(uneven)
