// FP32 TASER iterations (Algorithm 1) on the CUDA cores.
//
// Mapping: lane j of an instance owns variable column j of L~ and V.  Column j of
// T^ = -2 tau T~ (negated so every product is one FFMA) lives in registers for all
// t_max iterations; the rows of L~(t-1) are broadcast from shared memory (one LDS.128
// feeds four FFMAs).  Column norms of the prox (Sec. III-C) are then lane-local sums.
// Buckets: NB = 8 / 16 -> 4 / 2 instances per warp, NB = 32 -> one instance per warp,
// NB = 64 -> two warps per instance (the second warp skips rows < 32, all above its
// columns).  L~ never leaves the SM between iterations.
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

template <int NB>
__global__ void __launch_bounds__(128)
detect_fp32_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                   const float* __restrict__ tau_g, int t_max, int literal, float* __restrict__ Lout,
                   int8_t* __restrict__ s_hat, uint32_t* __restrict__ flags) {
  using C = Fp32Cfg<NB>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int local_inst, j;
  if constexpr (NB <= 32) {
    local_inst = warp * C::IPW + lane / C::G;
    j = lane % C::G;
  } else {
    local_inst = warp / C::WPI;
    j = (warp % C::WPI) * 32 + lane;
  }
  const int colbase = NB > 32 ? (warp % C::WPI) * 32 : 0;  // warp-uniform
  const int64_t inst = (int64_t)blockIdx.x * C::IPC + local_inst;
  const bool active = inst < batch;
  float* Ls = smem + local_inst * C::INST_FLOATS;
  float* xs = Ls + (NB + 1) * C::S;                         // cross-warp partial sums
  const int bar_id = 1 + local_inst;

  const int jr = j < N - 1 ? j : -1;                        // real column (variable)
  const float* T = Tt + (active ? inst : 0) * (int64_t)N * N;
  const float tau = active ? tau_g[inst] : 0.f;
  const float m2tau = -2.f * tau;

  // Column j of T^ = -2 tau T~ (T~ symmetric: T~[k][j] read row by row, coalesced).
  float tn[NB + 1];
#pragma unroll
  for (int k = 0; k <= NB; ++k) {
    const int kr = bucket_to_real(k, N, NB);
    float v = 0.f;
    if (active && jr >= 0 && kr >= 0) v = T[(int64_t)kr * N + jr];
    tn[k] = m2tau * v;
  }
  const float Dj = (active && jr >= 0) ? Dg[inst * N + jr] : 0.f;
  const float DN = active ? Dg[inst * N + N - 1] : 0.f;
  const float tnNN = m2tau * (active ? T[(int64_t)(N - 1) * N + (N - 1)] : 0.f);

  // L~(0) = D (Algorithm 1 initialisation).
  for (int idx = j; idx < C::INST_FLOATS; idx += (NB <= 32 ? C::G : 64)) Ls[idx] = 0.f;
  sync_instance<NB>(bar_id);
  Ls[j * C::S + j] = Dj;
  if (j == 0) Ls[NB * C::S + NB] = DN;
  float l[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) l[i] = (i == j) ? Dj : 0.f;
  float LNN = DN;
  uint32_t fl = 0;
  sync_instance<NB>(bar_id);

  for (int t = 0; t < t_max; ++t) {
    // Partial of V_NN = L~_NN (1 - 2 tau T~_NN) - 2 tau sum_k L~_Nk T~_kN from L~(t-1).
    float part = l[NB] * tn[NB];
#pragma unroll
    for (int o = C::G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(TASER_FULL_MASK, part, o);

    // V = L~ - tril(2 tau L~ T~): row i needs L~_ik, k <= i only (triangular skip).
#pragma unroll
    for (int i = 0; i <= NB; ++i) {
      if (NB > 32 && i < 32 && colbase != 0) {
        l[i] = 0.f;  // rows above every column of this warp
        continue;
      }
      float acc = l[i];
      const float* row = Ls + i * C::S;
#pragma unroll
      for (int k4 = 0; k4 <= i; k4 += 4) {
        const float4 q = *reinterpret_cast<const float4*>(row + k4);
        acc = fmaf(q.x, tn[k4], acc);
        if (k4 + 1 <= i) acc = fmaf(q.y, tn[k4 + 1], acc);
        if (k4 + 2 <= i) acc = fmaf(q.z, tn[k4 + 2], acc);
        if (k4 + 3 <= i) acc = fmaf(q.w, tn[k4 + 3], acc);
      }
      l[i] = (i >= j) ? acc : 0.f;  // l now holds column j of V
    }
    if constexpr (NB > 32) {
      if (lane == 0) xs[warp % C::WPI] = part;
    }
    sync_instance<NB>(bar_id);  // every lane has finished reading L~(t-1)
    if constexpr (NB > 32) part = xs[0] + xs[1];
    const float vnn = fmaf(LNN, tnNN, LNN) + part;
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
      Ls[i * C::S + j] = l[i];
    }
    if (literal && j == 0) Ls[NB * C::S + NB] = LNN;
    sync_instance<NB>(bar_id);
  }

  // OR the flags of the instance's lanes (all lanes still present for the shuffles).
  if constexpr (NB <= 32) {
#pragma unroll
    for (int o = C::G / 2; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  }
  if (!active) return;
  if (flags != nullptr && fl) {
    if constexpr (NB <= 32) {
      if (j == 0) flags[inst] |= fl;
    } else {
      if (lane == 0) atomicOr(&flags[inst], fl);
    }
  }
  // Decisions s_k = sign(L~_{N,k}) (sign(0) = +1), times sign(L~_NN) in literal mode.
  if (jr >= 0) {
    float r = l[NB];
    if (literal && LNN < 0.f) r = -r;
    s_hat[inst * (N - 1) + jr] = (r >= 0.f) ? int8_t(1) : int8_t(-1);
  }
  if (Lout != nullptr) {
    float* Lo = Lout + inst * (int64_t)N * N;
#pragma unroll
    for (int i = 0; i <= NB; ++i) {
      const int ir = bucket_to_real(i, N, NB);
      if (ir < 0) continue;
      if (jr >= 0) Lo[(int64_t)ir * N + jr] = l[i];
      if (j == 0) Lo[(int64_t)ir * N + (N - 1)] = (ir == N - 1) ? LNN : 0.f;
    }
  }
}

template <int NB>
static cudaError_t launch_fp32(int64_t batch, int N, const float* Tt, const float* D, const float* tau,
                               int t_max, int literal, float* L, int8_t* s, uint32_t* flags,
                               cudaStream_t st) {
  using C = Fp32Cfg<NB>;
  const int64_t blocks = (batch + C::IPC - 1) / C::IPC;
  if (C::SMEM_BYTES > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(detect_fp32_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  detect_fp32_kernel<NB><<<(unsigned)blocks, 128, C::SMEM_BYTES, st>>>(batch, N, Tt, D, tau, t_max, literal,
                                                                      L, s, flags);
  return cudaGetLastError();
}

cudaError_t detect_fp32(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                        int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 8: return launch_fp32<8>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    case 16: return launch_fp32<16>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    case 32: return launch_fp32<32>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    default: return launch_fp32<64>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
  }
}

}  // namespace taser
