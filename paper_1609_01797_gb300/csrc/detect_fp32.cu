// FP32 TASER iterations (Algorithm 1) on the CUDA cores.
//
// Mapping: lane j of an instance owns variable column j of L~ and V.  Column j of
// T^ = -2 tau T~ (negated so every product is one FMA) lives in registers for all
// t_max iterations, as packed pairs (T^_kj, T^_k+1,j); the rows of L~(t-1) are broadcast
// from shared memory, and one LDS.128 feeds two packed f32x2 FMAs, which keep the even-
// and odd-k partial sums of the row.  The stored L~ is zero above the diagonal and in the
// row padding, so the last float4 of a row needs no masking.  Column norms of the prox
// (Sec. III-C) are then lane-local sums.
// Buckets: NB = 8 / 16 -> 4 / 2 instances per warp, NB = 32 -> one instance per warp,
// NB = 64 -> two warps per instance (the second warp skips rows < 32, all above its
// columns).  L~ never leaves the SM between iterations.
//
// The per-instance body (fp32_run) serves the dense kernel (instances at a fixed stride)
// and the queue-fed persistent kernel of uneven batches; the instances sharing a warp
// may have different t_max, so each emits its outputs at its own last iteration.
#include "common.cuh"

namespace taser {


template <int NB>
struct Fp32Cfg {
  static constexpr int G = NB < 32 ? NB : 32;        // lanes of one instance in a warp
  static constexpr int IPW = 32 / G;                 // instances per warp
  static constexpr int WPI = NB > 32 ? NB / 32 : 1;  // warps per instance
  static constexpr int S = NB + 4;                   // smem row stride (floats), 16B rows
  static constexpr int INST_FLOATS = (NB + 1) * S + 4;
  static constexpr int WARPS = 4;                    // warps per CTA
  static constexpr int IPC = WARPS * IPW / WPI;      // instances per CTA
  static constexpr int SMEM_BYTES = IPC * INST_FLOATS * 4;
};

template <int NB>
__device__ __forceinline__ void sync_instance(int bar_id) {
  if constexpr (NB > 32) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(64) : "memory");
  } else {
    __syncwarp();
  }
}

// Runs Algorithm 1 for `jb` (inactive lanes compute on zeros and write nothing).
// t_loop: iterations the warp executes (the largest t_max among its instances).  MIXED:
// instances sharing the warp may have different t_max, so outputs are emitted inside the
// loop at each instance's own last iteration; otherwise once after the loop.
// MON: objective monitoring (taser_detect_monitored).  f(L~) = Tr(L~ T~ L~^T) equals
// sum_{i >= k} L~_ik (L~ T~)_ik, and the gradient step computes exactly that lower part:
// V = L~ - 2 tau tril(L~ T~), so f(L~(t)) = sum L~(t)_ik (L~(t)_ik - V(t+1)_ik) / (2 tau),
// accumulated from the iteration's own FP32 values (no extra product).  One more product
// after the last iteration gives f(L~(t_max)); its V is discarded.
template <int NB, bool MIXED, bool MON = false>
__device__ __forceinline__ void fp32_run(const Job& jb, bool active, int t_loop, float* Ls, float* xs, int j,
                                         int lane, int warp, int bar_id, int literal, double* obj = nullptr,
                                         float ascent_tol = 0.f) {
  using C = Fp32Cfg<NB>;
  const int colbase = NB > 32 ? (warp % C::WPI) * 32 : 0;  // warp-uniform
  const unsigned gmask = C::G == 32 ? TASER_FULL_MASK : (((1u << C::G) - 1u) << ((lane / C::G) * C::G));
  const int N = active ? jb.N : NB + 1;
  const int jr = j < N - 1 ? j : -1;                         // real column (variable)
  const float tau = active ? *jb.tau : 0.f;
  const float m2tau = -2.f * tau;

  // Column j of T^ = -2 tau T~ (T~ symmetric: T~[k][j] read row by row, coalesced), as
  // pairs (k, k + 1); pairs past k = NB are zero.
  constexpr int NP2 = NB / 2 + 2;
  uint64_t tn2[NP2];
  float tNB = 0.f;
#pragma unroll
  for (int p = 0; p < NP2; ++p) {
    float v2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * p + h;
      float v = 0.f;
      if (k <= NB) {
        const int kr = bucket_to_real(k, N, NB);
        if (active && jr >= 0 && kr >= 0 && TASER_IN(kr * N + jr, N * N)) v = jb.T[(int64_t)kr * N + jr];
      }
      v2[h] = m2tau * v;
      if (k == NB) tNB = v2[h];
    }
    tn2[p] = f2pack(v2[0], v2[1]);
  }
  const float Dj = (active && jr >= 0 && TASER_IN(jr, N)) ? jb.D[jr] : 0.f;
  const float DN = active ? jb.D[N - 1] : 0.f;
  const float tnNN = m2tau * (active ? jb.T[(int64_t)(N - 1) * N + (N - 1)] : 0.f);

  // L~(0) = D (Algorithm 1 initialisation).
  for (int idx = j; idx < C::INST_FLOATS; idx += (NB <= 32 ? C::G : 64)) Ls[idx] = 0.f;
  sync_instance<NB>(bar_id);
  if (TASER_IN(j * C::S + j, C::INST_FLOATS)) Ls[j * C::S + j] = Dj;
  if (j == 0) Ls[NB * C::S + NB] = DN;
  float l[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) l[i] = (i == j) ? Dj : 0.f;
  float LNN = DN;
  uint32_t fl = 0;
  sync_instance<NB>(bar_id);

  // Outputs of this instance (its lanes call this together).
  auto emit = [&]() {
    uint32_t f = fl;
    if constexpr (NB <= 32) {
#pragma unroll
      for (int o = C::G / 2; o > 0; o >>= 1) f |= __shfl_xor_sync(gmask, f, o);
      if (j == 0 && jb.flag != nullptr && f) *jb.flag |= f;
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f |= __shfl_xor_sync(TASER_FULL_MASK, f, o);
      if (lane == 0 && jb.flag != nullptr && f) atomicOr(jb.flag, f);
    }
    // Decisions s_k = sign(L~_{N,k}) (sign(0) = +1), times sign(L~_NN) in literal mode.
    if (jr >= 0 && TASER_IN(jr, N - 1)) {
      float r = l[NB];
      TASER_FINITE(r);
      if (literal && LNN < 0.f) r = -r;
      jb.s[jr] = (r >= 0.f) ? int8_t(1) : int8_t(-1);
    }
    if (jb.L != nullptr) {
#pragma unroll
      for (int i = 0; i <= NB; ++i) {
        const int ir = bucket_to_real(i, N, NB);
        if (ir < 0) continue;
        if (jr >= 0 && TASER_IN(ir * N + jr, N * N)) {
          jb.L[(int64_t)ir * N + jr] = l[i];
          TASER_FINITE(l[i]);
        }
        if (j == 0 && TASER_IN(ir * N + N - 1, N * N)) jb.L[(int64_t)ir * N + (N - 1)] = (ir == N - 1) ? LNN : 0.f;
      }
    }
  };

  double f_prev = 0.0;
  for (int t = 0; t < t_loop + (MON ? 1 : 0); ++t) {
    const bool last_pass = MON && t == t_loop;   // only f(L~(t_max)); L~ stays as it is
    // Partial of V_NN = L~_NN (1 - 2 tau T~_NN) - 2 tau sum_k L~_Nk T~_kN from L~(t-1).
    float part = l[NB] * tNB;
#pragma unroll
    for (int o = C::G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(TASER_FULL_MASK, part, o);
    float fterm = 0.f;   // MON: this lane's sum of L~_ij (L~_ij - V_ij)

    // V = L~ - tril(2 tau L~ T~): row i needs L~_ik, k <= i only (triangular skip).
#pragma unroll
    for (int i = 0; i <= NB; ++i) {
      if (NB > 32 && i < 32 && colbase != 0) {
        l[i] = 0.f;  // rows above every column of this warp
        continue;
      }
      uint64_t acc2 = f2pack(l[i], 0.f);
      const float* row = Ls + i * C::S;
#pragma unroll
      for (int k4 = 0; k4 <= i; k4 += 4) {
        const float4 q = *reinterpret_cast<const float4*>(row + k4);
        acc2 = f2fma(f2pack(q.x, q.y), tn2[k4 / 2], acc2);
        if (k4 + 2 <= i) acc2 = f2fma(f2pack(q.z, q.w), tn2[k4 / 2 + 1], acc2);
      }
      float a0, a1;
      f2unpack(acc2, a0, a1);
      const float v = (i >= j) ? a0 + a1 : 0.f;
      if constexpr (MON) {
        fterm = fmaf(l[i], l[i] - v, fterm);
        if (!last_pass) l[i] = v;
      } else {
        l[i] = v;  // l now holds column j of V
      }
    }
    if constexpr (MON) {
#pragma unroll
      for (int o = C::G / 2; o > 0; o >>= 1) fterm += __shfl_xor_sync(TASER_FULL_MASK, fterm, o);
      if constexpr (NB > 32) {
        if (lane == 0) xs[2 + warp % C::WPI] = fterm;
      }
    }
    if constexpr (NB > 32) {
      if (lane == 0) xs[warp % C::WPI] = part;
    }
    sync_instance<NB>(bar_id);  // every lane has finished reading L~(t-1)
    if constexpr (NB > 32) part = xs[0] + xs[1];
    const float vnn = fmaf(LNN, tnNN, LNN) + part;
    if constexpr (MON) {
      if constexpr (NB > 32) fterm = xs[2] + xs[3];
      fterm = fmaf(LNN, LNN - vnn, fterm);
      // f in FP64 from the FP32 sum; ascent when f(L~(t)) > f(L~(t-1)) + tol |f(L~(t-1))|.
      const double f = tau > 0.f ? (double)fterm / (2.0 * (double)tau) : 0.0;
      if (t > 0 && f > f_prev + (double)ascent_tol * fabs(f_prev)) fl |= TASER_FLAG_ASCENT;
      f_prev = f;
      if (active && obj != nullptr && j == 0 && colbase == 0 && TASER_IN(t, t_loop + 1)) obj[t] = f;
      if (last_pass) {
        if constexpr (NB > 32) sync_instance<NB>(bar_id);   // xs is read before it is reused
        break;
      }
    }
    if (vnn <= 0.f) fl |= TASER_FLAG_LNN_SIGN;
    if (literal) LNN = vnn >= 0.f ? DN : -DN;

    // prox: column j rescaled to norm D_jj.
    float n2 = 0.f;
#pragma unroll
    for (int i = 0; i <= NB; ++i) {
      if (NB > 32 && i < 32 && colbase != 0) continue;
      n2 = fmaf(l[i], l[i], n2);
    }
    float sc = 0.f;
    if (n2 > 0.f) {
      sc = Dj * rsqrtf(n2);
    } else if (jr >= 0) {
      fl |= TASER_FLAG_ZERO_COLUMN;
    }
#pragma unroll
    for (int i = 0; i <= NB; ++i) {
      if (NB > 32 && i < 32 && colbase != 0) continue;
      l[i] *= sc;
      if (TASER_IN(i * C::S + j, C::INST_FLOATS)) Ls[i * C::S + j] = l[i];
    }
    if (literal && j == 0) Ls[NB * C::S + NB] = LNN;
    sync_instance<NB>(bar_id);

    if constexpr (MIXED) {
      if (t + 1 == (active ? jb.t_max : -1)) emit();
    }
  }
  if constexpr (!MIXED) {
    if (active) emit();
  }
}

template <int NB>
__device__ __forceinline__ void fp32_lane_layout(int warp, int lane, int& local_inst, int& j) {
  using C = Fp32Cfg<NB>;
  if constexpr (NB <= 32) {
    local_inst = warp * C::IPW + lane / C::G;
    j = lane % C::G;
  } else {
    local_inst = warp / C::WPI;
    j = (warp % C::WPI) * 32 + lane;
  }
}

template <int NB, bool MON = false>
__global__ void __launch_bounds__(128, NB == 32 ? 3 : 1)
detect_fp32_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                   const float* __restrict__ tau_g, int t_max, int literal, float* __restrict__ Lout,
                   int8_t* __restrict__ s_hat, uint32_t* __restrict__ flags, double* __restrict__ obj,
                   float ascent_tol) {
  using C = Fp32Cfg<NB>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int local_inst, j;
  fp32_lane_layout<NB>(warp, lane, local_inst, j);
  const int64_t inst = (int64_t)blockIdx.x * C::IPC + local_inst;
  const bool active = inst < batch;
  float* Ls = smem + local_inst * C::INST_FLOATS;
  if (!TASER_IN(local_inst, C::IPC)) return;
  const Job jb = dense_job(active ? inst : 0, N, t_max, Tt, Dg, tau_g, Lout, s_hat, flags);
  double* ob = (MON && obj != nullptr) ? obj + (active ? inst : 0) * (int64_t)(t_max + 1) : nullptr;
  fp32_run<NB, false, MON>(jb, active, t_max, Ls, Ls + (NB + 1) * C::S, j, lane, warp, 1 + local_inst, literal, ob,
                           ascent_tol);
}

// Persistent, queue-fed: each warp (each warp pair for NB = 64) pops the next items of
// its bucket until the queue is empty, `rounds` warp-loads per pop (one atomic per
// rounds x IPW items: short jobs would otherwise queue on the counter).
template <int NB>
__global__ void __launch_bounds__(128, NB == 32 ? 3 : 1)
detect_fp32_queue_kernel(Queue q, int rounds, const float* __restrict__ T_pool, const float* __restrict__ D_pool,
                         const float* __restrict__ tau, int literal, float* __restrict__ L_pool,
                         int8_t* __restrict__ s_pool, uint32_t* __restrict__ flags) {
  using C = Fp32Cfg<NB>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int local_inst, j;
  fp32_lane_layout<NB>(warp, lane, local_inst, j);
  float* Ls = smem + local_inst * C::INST_FLOATS;
  float* xs = Ls + (NB + 1) * C::S;
  int* pop_slot = reinterpret_cast<int*>(xs + 2);
  const int count = q.count();
  for (;;) {
    constexpr int PER_ROUND = NB <= 32 ? C::IPW : 1;            // items of one warp-load
    int base;
    if constexpr (NB <= 32) {
      base = 0;
      if (lane == 0) base = q.pop(PER_ROUND * rounds);
      base = __shfl_sync(TASER_FULL_MASK, base, 0);
    } else {
      if ((warp % C::WPI) == 0 && lane == 0) *pop_slot = q.pop(rounds);
      sync_instance<NB>(1 + local_inst);
      base = *pop_slot;
      sync_instance<NB>(1 + local_inst);
    }
    if (base >= count) break;                                   // uniform per warp (pair)
    for (int r = 0; r < rounds; ++r) {
      const int b0 = base + r * PER_ROUND;
      if (b0 >= count) break;                                   // uniform per warp (pair)
      const int pos = NB <= 32 ? b0 + (lane / C::G) : b0;
      const bool active = pos < count;
      const int idx = active ? q.item_at(pos) : 0;
      const taser_item it = q.items[idx];
      const Job jb = item_job(it, idx, T_pool, D_pool, tau, L_pool, s_pool, flags);
      int t_loop = active ? jb.t_max : 0;
      if constexpr (NB <= 32) t_loop = __reduce_max_sync(TASER_FULL_MASK, t_loop);
      fp32_run<NB, (Fp32Cfg<NB>::IPW > 1)>(jb, active, t_loop, Ls, xs, j, lane, warp, 1 + local_inst, literal);
      sync_instance<NB>(1 + local_inst);
    }
  }
}

template <int NB, bool MON>
static cudaError_t launch_fp32(int64_t batch, int N, const float* Tt, const float* D, const float* tau,
                               int t_max, int literal, float* L, int8_t* s, uint32_t* flags, double* obj,
                               float ascent_tol, cudaStream_t st) {
  using C = Fp32Cfg<NB>;
  const int64_t blocks = (batch + C::IPC - 1) / C::IPC;
  if (C::SMEM_BYTES > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(detect_fp32_kernel<NB, MON>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  detect_fp32_kernel<NB, MON><<<(unsigned)blocks, 128, C::SMEM_BYTES, st>>>(batch, N, Tt, D, tau, t_max, literal,
                                                                           L, s, flags, obj, ascent_tol);
  return cudaGetLastError();
}

cudaError_t detect_fp32(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                        int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 8: return launch_fp32<8, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, nullptr, 0.f, st);
    case 16: return launch_fp32<16, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, nullptr, 0.f, st);
    case 32: return launch_fp32<32, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, nullptr, 0.f, st);
    default: return launch_fp32<64, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, nullptr, 0.f, st);
  }
}

// taser_detect_monitored on the FP32 kernel: f(L~(t)) per iteration and the ascent flag.
cudaError_t detect_fp32_monitored(int64_t batch, int N, const float* Tt, const float* D, const float* tau,
                                  int t_max, int literal, float ascent_tol, double* obj, float* L, int8_t* s,
                                  uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 8: return launch_fp32<8, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, obj, ascent_tol, st);
    case 16: return launch_fp32<16, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, obj, ascent_tol, st);
    case 32: return launch_fp32<32, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, obj, ascent_tol, st);
    default: return launch_fp32<64, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, obj, ascent_tol, st);
  }
}

// Queue-fed launch for bucket NB with `blocks` persistent blocks.
template <int NB>
static cudaError_t launch_fp32_queue(const Queue& q, int blocks_per_sm, int rounds, const float* T_pool,
                                     const float* D_pool, const float* tau, int literal, float* L_pool,
                                     int8_t* s_pool, uint32_t* flags, cudaStream_t st) {
  using C = Fp32Cfg<NB>;
  const size_t smem = C::SMEM_BYTES;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(detect_fp32_queue_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_fp32_queue_kernel<NB>, 128, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  detect_fp32_queue_kernel<NB><<<sms * per_sm, 128, smem, st>>>(q, rounds > 0 ? rounds : 1, T_pool, D_pool, tau,
                                                               literal, L_pool, s_pool, flags);
  return cudaGetLastError();
}

cudaError_t detect_fp32_queue(int nb, const Queue& q, int blocks_per_sm, int rounds, const float* T_pool,
                              const float* D_pool, const float* tau, int literal, float* L_pool, int8_t* s_pool,
                              uint32_t* flags, cudaStream_t st) {
  switch (nb) {
    case 8:
      return launch_fp32_queue<8>(q, blocks_per_sm, rounds, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
    case 16:
      return launch_fp32_queue<16>(q, blocks_per_sm, rounds, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
    case 32:
      return launch_fp32_queue<32>(q, blocks_per_sm, rounds, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
    default:
      return launch_fp32_queue<64>(q, blocks_per_sm, rounds, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
  }
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(detect_fp32)
