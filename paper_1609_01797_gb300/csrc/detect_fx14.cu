// Fixed-point TASER: the 14-bit datapath of the paper's VLSI designs (Sec. IV-B operation
// modes, Sec. IV-D fixed-point parameters and inverse square-root LUT), computed exactly
// in integer arithmetic.
//
// Formats (two's complement, saturating to [-2^13, 2^13 - 1]):
//   L~, V rows < N: 8 fraction bits;  row N: 7;  L~_NN (constant register): 5;
//   T^ = 2 tau T~: 12 fraction bits (|T^_ij| <= 2 alpha < 2);  D_j: 8, D_N: 5.
// Rounding to a narrower format is round-half-up: (a + 2^(k-1)) >> k, arithmetic shift.
// The MAC accumulates exactly (row i < N at 20 fraction bits, row N at 19); the squared
// column norm is exact (16 fraction bits); its inverse square root comes from a LUT of
// 2^11 entries (13 fraction bits) indexed by the top 11 bits of the norm after an even
// normalisation x = m 4^e, m in [1, 4); the scale D_j * LUT keeps its power-of-two part
// as a shift and each PE rounds V_ij * scale once.  Only the constant-L~_NN mode exists.
//
// One warp per instance, lane j owns column j (and j + 32 at N > 33).  Its column of T^
// lives in registers; L~ lives in shared memory, one int per entry, and its rows are
// broadcast to the lanes (one LDS.128 feeds four IMADs).  Products are below 2^26, so
// 16 of them (four partial sums of four) are summed in int32 before each 64-bit
// accumulate: exact for every input.
#include <math.h>

#include "common.cuh"

namespace taser {

template <int NB>
struct FxCfg {
  static constexpr int CPL = NB == 64 ? 2 : 1;     // columns per lane
  static constexpr int KC = NB >= 16 ? 16 : NB;    // products summed in int32 per chunk
  static constexpr int NCH = NB / KC;
  static constexpr int SLOT = (NB + 1) * NB;       // ints per warp: NB rows + row N
  static constexpr int WARPS = 4;
};

constexpr int kFxLutEntries = 2048;
constexpr int kFxLutInts = kFxLutEntries / 2;      // uint16 entries

// floor(x * scale + 1/2) as a 14-bit code (scale a power of two, so x * scale is exact and
// the + 1/2 is exact below 2^23; larger magnitudes saturate either way).  NaN -> 0.
__device__ __forceinline__ int fx_quant(float x, float scale, bool& sat) {
  const float v = floorf(__fadd_rn(__fmul_rn(x, scale), 0.5f));
  if (isnan(v)) {
    sat = true;
    return 0;
  }
  if (v < -8192.f) {
    sat = true;
    return -8192;
  }
  if (v > 8191.f) {
    sat = true;
    return 8191;
  }
  return (int)v;
}

__device__ __forceinline__ int fx_sat(long long a, bool& sat) {
  if (a < -8192) {
    sat = true;
    return -8192;
  }
  if (a > 8191) {
    sat = true;
    return 8191;
  }
  return (int)a;
}

__device__ __forceinline__ long long fx_round_shift(long long a, int k) { return (a + (1ll << (k - 1))) >> k; }

// Algorithm 1 on one instance.  Lq: this warp's (NB + 1) x NB ints; lut: 2048 uint16.
template <int NB>
__device__ __forceinline__ void fx_run(const Job& jb, int* Lq, const unsigned short* lut, int lane) {
  using C = FxCfg<NB>;
  constexpr int CPL = C::CPL, KC = C::KC, NCH = C::NCH;
  const int N = jb.N, nv = N - 1;
  const float* T = jb.T;
  const float tau2 = __fadd_rn(*jb.tau, *jb.tau);
  bool sat = false;
  uint32_t fl = 0;

  // Quantised inputs: this lane's columns of T^ (bucket rows), T^_{N,j}, T^_{j,N} and D_j.
  int tc[CPL][NB], tNj[CPL], tjN[CPL], dq[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = lane + 32 * c;
    const bool real = j < nv;
#pragma unroll
    for (int k = 0; k < NB; ++k)
      tc[c][k] = (real && k < nv && TASER_IN(k * N + j, N * N))
                     ? fx_quant(__fmul_rn(tau2, T[(int64_t)k * N + j]), 4096.f, sat)
                     : 0;
    const bool ok = real && TASER_IN(nv * N + j, N * N) && TASER_IN(j * N + nv, N * N) && TASER_IN(j, N);
    tNj[c] = ok ? fx_quant(__fmul_rn(tau2, T[(int64_t)nv * N + j]), 4096.f, sat) : 0;
    tjN[c] = ok ? fx_quant(__fmul_rn(tau2, T[(int64_t)j * N + nv]), 4096.f, sat) : 0;
    dq[c] = ok ? fx_quant(jb.D[j], 256.f, sat) : 0;
  }
  const int tNN = fx_quant(__fmul_rn(tau2, T[(int64_t)nv * N + nv]), 4096.f, sat);
  const int lnn = fx_quant(jb.D[nv], 32.f, sat);

  // L~(0) = D: diagonal codes, zero elsewhere (row N starts at zero).
  int* rowN = Lq + NB * NB;
  for (int i = lane; i < C::SLOT; i += 32) Lq[i] = 0;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = lane + 32 * c;
    if (j < nv && TASER_IN(j * NB + j, NB * NB)) Lq[j * NB + j] = dq[c];
  }
  __syncwarp();

  // acc[c] += sum over the KC columns k of chunk ch of L~_ik T^_kj, with four independent
  // int32 partial sums (each at most 4 products below 2^26: exact) for instruction-level
  // parallelism, then one 64-bit accumulate.
  auto chunk_mac = [&](const int* lrow, int ch, long long (&acc)[CPL]) {
    int p0[CPL], p1[CPL], p2[CPL], p3[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) p0[c] = p1[c] = p2[c] = p3[c] = 0;
#pragma unroll
    for (int kk = 0; kk < KC; kk += 4) {
      const int4 l4 = *reinterpret_cast<const int4*>(lrow + kk);
      const int k0 = ch * KC + kk;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        p0[c] += l4.x * tc[c][k0];
        p1[c] += l4.y * tc[c][k0 + 1];
        p2[c] += l4.z * tc[c][k0 + 2];
        p3[c] += l4.w * tc[c][k0 + 3];
      }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc[c] += (long long)((p0[c] + p1[c]) + (p2[c] + p3[c]));
  };

  for (int t = 0; t < jb.t_max; ++t) {
    long long x[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) x[c] = 0;

    // Gradient step, rows i < N: V_ij = round((L~_ij 2^12 - sum_k<=i L~_ik T^_kj) / 2^12).
    for (int i = 0; i < nv; ++i) {
      int* row = Lq + i * NB;
      long long acc[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[c] = 0;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        if (ch * KC > i) break;                    // L~_ik = 0 for k > i
        chunk_mac(row + ch * KC, ch, acc);
      }
      int v[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;             // j <= i < nv <= NB: inside the row
        v[c] = j <= i ? fx_sat(fx_round_shift(((long long)row[j] << 12) - acc[c], 12), sat) : 0;
      }
      __syncwarp();                                // every lane has read row i
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;
        if (j <= i && TASER_IN(i * NB + j, NB * NB)) {
          row[j] = v[c];
          x[c] += (long long)(v[c] * v[c]);
        }
      }
    }

    // Row N: 19 fraction bits; the L~_NN (5-bit) product is aligned by 2 bits.
    {
      long long acc[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[c] = 0;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) chunk_mac(rowN + ch * KC, ch, acc);
      // V_NN (for the flag only): L~_NN 2^14 - sum_k L~_Nk T^_kN - (L~_NN T^_NN) 2^2.
      long long part = 0;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;
        if (j < nv) part += (long long)(rowN[j] * tjN[c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(TASER_FULL_MASK, part, o);
      const long long vnn = ((long long)lnn << 14) - part - ((long long)(lnn * tNN) << 2);
      if (vnn <= 0) fl |= TASER_FLAG_LNN_SIGN;
      int v[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;
        v[c] = 0;
        if (j < nv) {
          const long long a = ((long long)rowN[j] << 12) - acc[c] - ((long long)(lnn * tNj[c]) << 2);
          v[c] = fx_sat(fx_round_shift(a, 12), sat);
        }
      }
      __syncwarp();
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lane + 32 * c;
        if (j < nv) {
          rowN[j] = v[c];
          x[c] += 4ll * (long long)(v[c] * v[c]);   // 7 -> 8 fraction bits before squaring
        }
      }
    }

    // Prox: scale unit (LUT inverse square root times D_j), then each PE rescales.
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = lane + 32 * c;
      if (j >= nv) continue;
      int cs = 0, sh = 13;
      if (x[c] > 0) {
        const unsigned long long ux = (unsigned long long)x[c];
        const int e = (63 - __clzll(x[c])) & ~1;
        const unsigned long long idx = e >= 9 ? (ux >> (e - 9)) : (ux << (9 - e));
        cs = TASER_IN(idx, 2048) ? dq[c] * (int)lut[idx] : 0;
        sh = 13 + (e >> 1);
      } else {
        fl |= TASER_FLAG_ZERO_COLUMN;
      }
      for (int i = j; i < nv; ++i) {
        if (!TASER_IN(i * NB + j, NB * NB)) continue;
        int* p = Lq + i * NB + j;
        *p = fx_sat(fx_round_shift((long long)(*p) * cs, sh), sat);
      }
      rowN[j] = fx_sat(fx_round_shift((long long)rowN[j] * cs, sh), sat);
    }
    __syncwarp();
  }

  // Outputs: flags, decisions sign(L~_N,j) (sign(0) = +1), L~ as reals.
  if (sat) fl |= TASER_FLAG_SATURATED;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  if (lane == 0 && jb.flag != nullptr && fl) atomicOr(jb.flag, fl);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = lane + 32 * c;
    if (j < nv && TASER_IN(j, N - 1)) jb.s[j] = rowN[j] >= 0 ? int8_t(1) : int8_t(-1);
  }
  if (jb.L != nullptr) {
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N, cc = e - r * N;
      float val = 0.f;
      if (cc <= r) {
        if (r == nv) val = cc == nv ? (float)lnn * (1.f / 32.f) : (float)rowN[cc] * (1.f / 128.f);
        else val = TASER_IN(r * NB + cc, NB * NB) ? (float)Lq[r * NB + cc] * (1.f / 256.f) : 0.f;
      }
      jb.L[e] = val;
    }
  }
  __syncwarp();
}

// Persistent kernel: dense instances at a fixed stride, or items popped from a bucket queue.
template <int NB, bool QUEUE>
__global__ void __launch_bounds__(128, NB == 64 ? 1 : 4)
detect_fx14_kernel(int64_t batch, int N, int t_max, const float* __restrict__ Tt, const float* __restrict__ Dg,
                   const float* __restrict__ tau, float* __restrict__ L, int8_t* __restrict__ s,
                   uint32_t* __restrict__ flags, Queue q, const float* __restrict__ T_pool,
                   const float* __restrict__ D_pool, float* __restrict__ L_pool, int8_t* __restrict__ s_pool) {
  using C = FxCfg<NB>;
  extern __shared__ __align__(16) int fsm[];
  unsigned short* lut = reinterpret_cast<unsigned short*>(fsm);
  // LUT[i] = round(2^13 / sqrt((i + 1/2) / 512)) for i in [512, 2048), IEEE double steps.
  for (int i = threadIdx.x; i < kFxLutEntries; i += blockDim.x)
    lut[i] = i < 512 ? (unsigned short)0 : (unsigned short)floor(8192.0 / sqrt((i + 0.5) / 512.0) + 0.5);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* Lq = fsm + kFxLutInts + warp * C::SLOT;
  const int64_t stride = (int64_t)gridDim.x * C::WARPS;
  for (int64_t k = 0;; ++k) {
    Job jb;
    if constexpr (QUEUE) {
      int pos = 0;
      if (lane == 0) pos = q.pop(1);
      pos = __shfl_sync(TASER_FULL_MASK, pos, 0);
      if (pos >= q.count()) break;
      const int idx = q.item_at(pos);
      jb = item_job(q.items[idx], idx, T_pool, D_pool, tau, L_pool, s_pool, flags);
    } else {
      const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp + k * stride;
      if (inst >= batch) break;
      jb = dense_job(inst, N, t_max, Tt, Dg, tau, L, s, flags);
    }
    fx_run<NB>(jb, Lq, lut, lane);
  }
}

template <int NB, bool QUEUE>
static cudaError_t launch_fx14(int64_t batch, int N, int t_max, const float* Tt, const float* D, const float* tau,
                               float* L, int8_t* s, uint32_t* flags, const Queue& q, int blocks_per_sm,
                               const float* T_pool, const float* D_pool, float* L_pool, int8_t* s_pool,
                               cudaStream_t st) {
  using C = FxCfg<NB>;
  const size_t smem = (size_t)(kFxLutInts + C::WARPS * C::SLOT) * sizeof(int);
  auto kern = detect_fx14_kernel<NB, QUEUE>;
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, 32 * C::WARPS, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  int64_t blocks = (int64_t)sms * per_sm;
  if (!QUEUE) {
    const int64_t need = (batch + C::WARPS - 1) / C::WARPS;
    if (need < blocks) blocks = need;
  }
  kern<<<(unsigned)blocks, 32 * C::WARPS, smem, st>>>(batch, N, t_max, Tt, D, tau, L, s, flags, q, T_pool, D_pool,
                                                    L_pool, s_pool);
  return cudaGetLastError();
}

cudaError_t detect_fx14(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max, float* L,
                        int8_t* s, uint32_t* flags, cudaStream_t st) {
  const Queue q{};
  switch (bucket_of(N)) {
    case 8:
      return launch_fx14<8, false>(batch, N, t_max, Tt, D, tau, L, s, flags, q, 0, nullptr, nullptr, nullptr,
                                   nullptr, st);
    case 16:
      return launch_fx14<16, false>(batch, N, t_max, Tt, D, tau, L, s, flags, q, 0, nullptr, nullptr, nullptr,
                                    nullptr, st);
    case 32:
      return launch_fx14<32, false>(batch, N, t_max, Tt, D, tau, L, s, flags, q, 0, nullptr, nullptr, nullptr,
                                    nullptr, st);
    default:
      return launch_fx14<64, false>(batch, N, t_max, Tt, D, tau, L, s, flags, q, 0, nullptr, nullptr, nullptr,
                                    nullptr, st);
  }
}

cudaError_t detect_fx14_queue(int nb, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, float* L_pool, int8_t* s_pool, uint32_t* flags, cudaStream_t st) {
  switch (nb) {
    case 8:
      return launch_fx14<8, true>(0, 0, 0, nullptr, nullptr, tau, nullptr, nullptr, flags, q, blocks_per_sm, T_pool,
                                  D_pool, L_pool, s_pool, st);
    case 16:
      return launch_fx14<16, true>(0, 0, 0, nullptr, nullptr, tau, nullptr, nullptr, flags, q, blocks_per_sm, T_pool,
                                   D_pool, L_pool, s_pool, st);
    case 32:
      return launch_fx14<32, true>(0, 0, 0, nullptr, nullptr, tau, nullptr, nullptr, flags, q, blocks_per_sm, T_pool,
                                   D_pool, L_pool, s_pool, st);
    default:
      return launch_fx14<64, true>(0, 0, 0, nullptr, nullptr, tau, nullptr, nullptr, flags, q, blocks_per_sm, T_pool,
                                   D_pool, L_pool, s_pool, st);
  }
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(detect_fx14)
