// Tensor-core TASER iterations for 34 <= N <= 65 (bucket of 64 variable columns).
//
// Same arithmetic as detect_tc.cu (mma.m16n8k16 with BF16/FP16 operands and FP32
// accumulation, FP32 master L~ in the accumulator layout, FP32 prox) with two warps per
// instance.  Row blocks of 16 are split for balance: warp 0 owns blocks 0 and 3, warp 1
// blocks 1 and 2 (2 + 32 and 8 + 18 mma per iteration), and each warp owns half of the
// augmented row 64 (n-tiles 0..3 or 4..7, 16 mma each).  Per iteration the warps exchange
// through shared memory (double-buffered by iteration parity, two pair barriers):
//   1. their half of row 64 as packed A-operand pairs (the row-64 tile needs all k-tiles),
//      and their part of V_NN's partial sum;
//   2. their partial column sums of squares.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"

namespace taser {

template <bool FP16>
__device__ __forceinline__ uint32_t pack2_64(float lo, float hi) {
  if constexpr (FP16) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
  }
}

template <bool FP16>
__device__ __forceinline__ void mma64(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
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

// (v[e], v[e + 1]) *= sc2, as one packed multiply.
__device__ __forceinline__ void p2scale(float* v, uint64_t sc2) {
  f2unpack(f2mul(f2pack(v[0], v[1]), sc2), v[0], v[1]);
}

// Shared exchange area of one instance (floats): [parity][ row64 A pairs (32 u32) |
// V_NN partial (1) | pad | column partial sums [2 warps][64] ], then the queue pop slot.
constexpr int X64_ROW = 0, X64_VNN = 32, X64_COL = 36, X64_PAR = 36 + 128;
constexpr int X64_INST = 2 * X64_PAR + 8;   // + pop slot

__device__ __forceinline__ void pair_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// ROLE 0: row blocks 0 and 3, row-64 n-tiles 0..3.  ROLE 1: blocks 1 and 2, n-tiles 4..7.
template <bool FP16, int ROLE>
__device__ __forceinline__ void tc64_run(const Job& jb, float* X, int lane, int bar, int literal) {
  constexpr int MLO = ROLE ? 1 : 0, MHI = ROLE ? 2 : 3;
  constexpr int NLO = 2 * MLO + 2, NHI = 2 * MHI + 2;   // n-tiles of the two row blocks
  constexpr int RN0 = 4 * ROLE;                          // first n-tile of this warp's row-64 half
  const int g = lane >> 2, tq = lane & 3;
  const int N = jb.N;
  const float* T = jb.T;
  const float m2tau = -2.f * (*jb.tau);
#ifdef TASER_DEBUG
  auto tval = [&](int k, int n) -> float {
    return (k < N - 1 && n < N - 1 && TASER_IN(k * N + n, N * N)) ? m2tau * T[(int64_t)k * N + n] : 0.f;
  };
#else
  // (The release code keeps this kernel's original shape: folding in the debug build's
  // checks, even as constants, was measured 8.5% slower at N = 65.)
  auto tval = [&](int k, int n) -> float { return (k < N - 1 && n < N - 1) ? m2tau * T[(int64_t)k * N + n] : 0.f; };
#endif
  auto needB = [](int kt, int n) -> bool {
    return (kt <= MLO && n < NLO) || (kt <= MHI && n < NHI) || (n >= RN0 && n < RN0 + 4);
  };
  uint32_t bf[4][8][2];
#pragma unroll
  for (int kt = 0; kt < 4; ++kt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      if (!needB(kt, nt)) continue;
      const int k0 = 16 * kt + 2 * tq, n = 8 * nt + g;
      bf[kt][nt][0] = pack2_64<FP16>(tval(k0, n), tval(k0 + 1, n));
      bf[kt][nt][1] = pack2_64<FP16>(tval(k0 + 8, n), tval(k0 + 9, n));
    }
  // Row N of T^ at this warp's row-64 columns c = 8 (RN0 + n) + 2tq + p.
  float tN[4][2];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int c = 8 * (RN0 + n) + 2 * tq + p;
      tN[n][p] = (g == 0 && c < N - 1) ? m2tau * T[(int64_t)(N - 1) * N + c] : 0.f;
    }
  uint64_t tN2[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) tN2[n] = f2pack(tN[n][0], tN[n][1]);
  const float tnNN = m2tau * T[(int64_t)(N - 1) * N + (N - 1)];
  const float DN = jb.D[N - 1];
  // Column scales are owned per lane for columns 8g + 2tq + p (after the reduction).
  float Down[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int c = 8 * g + 2 * tq + p;
    Down[p] = c < N - 1 ? jb.D[c] : 0.f;
  }
  float lo[NLO][4], hi[NHI][4], rw[4][4];
#pragma unroll
  for (int n = 0; n < NLO; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 16 * MLO + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
      lo[n][e] = (r == c && r < N - 1) ? jb.D[r] : 0.f;
    }
#pragma unroll
  for (int n = 0; n < NHI; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 16 * MHI + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
      hi[n][e] = (r == c && r < N - 1) ? jb.D[r] : 0.f;
    }
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) rw[n][e] = 0.f;   // L~(0) row N: zeros (and L~_NN = D_N)
  float LNN = DN;
  uint32_t fl = 0;

  for (int t = 0; t < jb.t_max; ++t) {
    float* XP = X + (t & 1) * X64_PAR;
    // --- exchange 1: this warp's half of row 64 (A pairs, lanes g == 0) and V_NN partial
    uint64_t part2 = 0ull;
#pragma unroll
    for (int n = 0; n < 4; ++n) part2 = f2fma(f2pack(rw[n][0], rw[n][1]), tN2[n], part2);
    float part, part_hi;
    f2unpack(part2, part, part_hi);
    part += part_hi;
    part += __shfl_xor_sync(TASER_FULL_MASK, part, 1);
    part += __shfl_xor_sync(TASER_FULL_MASK, part, 2);
    uint32_t* rowA = reinterpret_cast<uint32_t*>(XP + X64_ROW);
    if (g == 0) {
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {          // this warp's k-tiles 2 ROLE + kk
        const int kt = 2 * ROLE + kk;
        rowA[(kt * 4 + tq) * 2 + 0] = pack2_64<FP16>(rw[2 * kk][0], rw[2 * kk][1]);
        rowA[(kt * 4 + tq) * 2 + 1] = pack2_64<FP16>(rw[2 * kk + 1][0], rw[2 * kk + 1][1]);
      }
      if (tq == 0) XP[X64_VNN + ROLE * 2] = part;
    }
    pair_bar(bar);
    const float vpart = XP[X64_VNN] + XP[X64_VNN + 2];
    // --- products: V = L~ - L~ T^ for the owned row blocks and the row-64 half
    auto block_mma = [&](auto& acc, auto mtag) {
      constexpr int M = decltype(mtag)::value;
      constexpr int NT = 2 * M + 2;
      uint32_t a[4][4];
#pragma unroll
      for (int kt = 0; kt <= M; ++kt) {
        a[kt][0] = pack2_64<FP16>(acc[2 * kt][0], acc[2 * kt][1]);
        a[kt][1] = pack2_64<FP16>(acc[2 * kt][2], acc[2 * kt][3]);
        a[kt][2] = pack2_64<FP16>(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
        a[kt][3] = pack2_64<FP16>(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
      }
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int kt = 0; kt <= M; ++kt) mma64<FP16>(acc[n], a[kt], bf[kt][n]);
#pragma unroll
      for (int n = 2 * M; n <= 2 * M + 1; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 16 * M + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
          if (c > r) acc[n][e] = 0.f;
        }
    };
    block_mma(lo, std::integral_constant<int, MLO>{});
    block_mma(hi, std::integral_constant<int, MHI>{});
    {
      uint32_t a[4][4];
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        a[kt][0] = g == 0 ? rowA[(kt * 4 + tq) * 2 + 0] : 0u;
        a[kt][2] = g == 0 ? rowA[(kt * 4 + tq) * 2 + 1] : 0u;
        a[kt][1] = 0u;
        a[kt][3] = 0u;
      }
      const uint64_t lnn2 = f2pack(LNN, LNN);
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        // k = N term in FP32 (tN is 0 for g != 0)
        f2unpack(f2fma(lnn2, tN2[n], f2pack(rw[n][0], rw[n][1])), rw[n][0], rw[n][1]);
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma64<FP16>(rw[n], a[kt], bf[kt][RN0 + n]);
      }
    }
    const float vnn = fmaf(LNN, tnNN, LNN) + vpart;
    if (vnn <= 0.f) fl |= TASER_FLAG_LNN_SIGN;
    if (literal) LNN = vnn >= 0.f ? DN : -DN;
    // --- column sums of squares: 16 partials per lane (n-tile, parity) over owned rows
    float s[16];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      uint64_t v2 = 0ull;
      auto sq = [&](float a, float b) {
        const uint64_t x = f2pack(a, b);
        v2 = f2fma(x, x, v2);
      };
      if (n < NLO) {
        sq(lo[n][2], lo[n][3]);
        sq(lo[n][0], lo[n][1]);
      }
      if (n < NHI) {
        sq(hi[n][2], hi[n][3]);
        sq(hi[n][0], hi[n][1]);
      }
      if (n >= RN0 && n < RN0 + 4) sq(rw[n - RN0][0], rw[n - RN0][1]);
      f2unpack(v2, s[2 * n], s[2 * n + 1]);
    }
    // transpose-reduce over g: lane ends with columns 8g + 2tq + {0, 1}
#pragma unroll
    for (int step = 0; step < 3; ++step) {
      const int m = 16 >> step;
      const int h = 8 >> step;
      const bool up = (lane & m) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const float send = up ? s[i] : s[i + h];
        const float keep = up ? s[i + h] : s[i];
        s[i] = keep + __shfl_xor_sync(TASER_FULL_MASK, send, m);
      }
    }
    float* col = XP + X64_COL;
#pragma unroll
    for (int p = 0; p < 2; ++p) col[ROLE * 64 + 8 * g + 2 * tq + p] = s[p];
    pair_bar(bar);
    float sc_own[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int c = 8 * g + 2 * tq + p;
      const float tot = col[c] + col[64 + c];
      sc_own[p] = 0.f;
      if (tot > 0.f) {
        sc_own[p] = Down[p] * rsqrtf(tot);
      } else if (c < N - 1) {
        fl |= TASER_FLAG_ZERO_COLUMN;
      }
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const uint64_t sc2 = f2pack(__shfl_sync(TASER_FULL_MASK, sc_own[0], 4 * n + tq),
                                  __shfl_sync(TASER_FULL_MASK, sc_own[1], 4 * n + tq));
      if (n < NLO) {
        p2scale(&lo[n][0], sc2);
        p2scale(&lo[n][2], sc2);
      }
      if (n < NHI) {
        p2scale(&hi[n][0], sc2);
        p2scale(&hi[n][2], sc2);
      }
      if (n >= RN0 && n < RN0 + 4) p2scale(&rw[n - RN0][0], sc2);
    }
  }

  // Outputs.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  if (lane == 0 && jb.flag != nullptr && fl) atomicOr(jb.flag, fl);
  if (g == 0) {
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int c = 8 * (RN0 + n) + 2 * tq + p;
#ifdef TASER_DEBUG
        if (c < N - 1 && TASER_IN(c, N - 1)) {
          TASER_FINITE(rw[n][p]);
#else
        if (c < N - 1) {
#endif
          float r = rw[n][p];
          if (literal && LNN < 0.f) r = -r;
          jb.s[c] = r >= 0.f ? int8_t(1) : int8_t(-1);
        }
      }
  }
  if (jb.L != nullptr) {
    float* Lo = jb.L;
    auto put = [&](auto& acc, auto mtag, int nmax) {
      constexpr int M = decltype(mtag)::value;
#pragma unroll
      for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 16 * M + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
#ifdef TASER_DEBUG
          if (r >= N - 1 || c >= N - 1 || !TASER_IN(r * N + c, N * N)) continue;
          Lo[(int64_t)r * N + c] = n < nmax ? acc[n < nmax ? n : 0][e] : 0.f;
          TASER_FINITE(Lo[(int64_t)r * N + c]);
#else
          if (r >= N - 1 || c >= N - 1) continue;
          Lo[(int64_t)r * N + c] = n < nmax ? acc[n < nmax ? n : 0][e] : 0.f;
#endif
        }
    };
    put(lo, std::integral_constant<int, MLO>{}, NLO);
    put(hi, std::integral_constant<int, MHI>{}, NHI);
    if (g == 0) {
#pragma unroll
      for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int c = 8 * (RN0 + n) + 2 * tq + p;
#ifdef TASER_DEBUG
          if (c < N - 1 && TASER_IN((N - 1) * N + c, N * N)) Lo[(int64_t)(N - 1) * N + c] = rw[n][p];
#else
          if (c < N - 1) Lo[(int64_t)(N - 1) * N + c] = rw[n][p];
#endif
        }
    }
    if (ROLE == 0)
#ifdef TASER_DEBUG
      for (int rr = lane; rr < N; rr += 32)
        if (TASER_IN(rr * N + N - 1, N * N)) Lo[(int64_t)rr * N + (N - 1)] = rr == N - 1 ? LNN : 0.f;
#else
      for (int rr = lane; rr < N; rr += 32) Lo[(int64_t)rr * N + (N - 1)] = rr == N - 1 ? LNN : 0.f;
#endif
  }
}

// Per warp pair in dynamic shared memory: the exchange area, two staging slots for T~, D
// and tau (the current job and the prefetched next one) and the two jobs' records.
constexpr int SLOT64 = 65 * 65 + 65 + 1 + 3;               // 4,294 floats: N^2 + N + 1, padded
constexpr int REC64 = 16;                                 // floats per job record
constexpr int ITEM64 = 10;                                // floats per prefetched taser_item
constexpr int PAIR64 = X64_INST + 2 * SLOT64 + 2 * REC64 + 4 * ITEM64 + 8;
static_assert(X64_INST % 4 == 0 && SLOT64 % 2 == 0 && PAIR64 % 4 == 0, "16-byte aligned slots and records");

struct JobRec64 {   // outputs and sizes of a staged job (56 bytes)
  float* L;
  int8_t* s;
  uint32_t* flag;
  int N, t_max;
};
static_assert(sizeof(JobRec64) <= REC64 * sizeof(float), "job record fits its slot");
static_assert(sizeof(taser_item) == ITEM64 * sizeof(float) && sizeof(taser_item) % 8 == 0, "item copied 8 bytes at a time");

__device__ __forceinline__ void cp_async4_64(float* smem_dst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}

// Two warps per instance, two instances per block.  Pair p of P takes jobs p, p + P,
// p + 2P, ... of its source: the dense batch, or the bucket's list of item indices, which
// the bucketing kernel sorted by t_max (longest first), so the strided split is balanced.
// While a pair iterates on one job, both warps prefetch the next job's T~, D and tau into
// the other slot with cp.async; for a bucket list, thread 0 also prefetches, when a job is
// taken, the list entry four jobs and the item record two jobs after it (each lands in a
// commit group that is complete before it is read), so no global load sits between jobs.
// `from_list` repeats QUEUE at run time: the queue-fed instantiation then keeps both job
// sources in its code, and measured 20% faster (its iteration loop is compiled with more
// registers) than with the source fixed at compile time; the dense instantiation does not
// need it.
template <bool FP16, bool QUEUE>
__global__ void __launch_bounds__(128)
detect_tc64_kernel(bool from_list, int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                   const float* __restrict__ tau, int t_max, float* __restrict__ L, int8_t* __restrict__ s,
                   uint32_t* __restrict__ flags, Queue q, const float* __restrict__ T_pool,
                   const float* __restrict__ D_pool, float* __restrict__ L_pool, int8_t* __restrict__ s_pool,
                   int literal) {
  extern __shared__ __align__(16) float xsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp >> 1, role = warp & 1;
  float* X = xsm + pair * PAIR64;
  float* slots = X + X64_INST;
  JobRec64* recs = reinterpret_cast<JobRec64*>(slots + 2 * SLOT64);
  // Descriptor prefetch rings (bucket lists): item records [4] and list entries [8].
  taser_item* litem = reinterpret_cast<taser_item*>(recs + 2);
  int* lidx = reinterpret_cast<int*>(litem + 4);
  const int bar = 1 + pair;
  const int tid = role * 32 + lane;                     // thread index within the pair
  const int64_t stride = (int64_t)gridDim.x * 2, gp = (int64_t)blockIdx.x * 2 + pair;
  const int64_t count = (QUEUE && from_list) ? (int64_t)q.count() : batch;
  const int lbase = (QUEUE && from_list) ? q.meta[q.b] : 0;
  int64_t k = 0;                                        // jobs acquired so far

  auto valid = [&](int64_t kk) { return gp + kk * stride < count; };
#ifdef TASER_DEBUG
  auto list_at = [&](int64_t kk) {
    const int64_t at = lbase + (gp + kk * stride);
    return q.list + (TASER_IN(at, q.n) ? at : 0);
  };
#else
  auto list_at = [&](int64_t kk) { return q.list + lbase + (gp + kk * stride); };
#endif
  // Thread 0: item record of job kk (its list entry is already in the ring), 8 bytes at a time.
  auto fetch_item = [&](int64_t kk) {
#ifdef TASER_DEBUG
    const float* src = reinterpret_cast<const float*>(q.items + (TASER_IN(lidx[kk & 7], q.n) ? lidx[kk & 7] : 0));
#else
    const float* src = reinterpret_cast<const float*>(q.items + lidx[kk & 7]);
#endif
    float* dst = reinterpret_cast<float*>(litem + (kk & 3));
#pragma unroll
    for (int h = 0; h < (int)(sizeof(taser_item) / 8); ++h) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst + 2 * h);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + 2 * h) : "memory");
    }
  };
  // Next job of this pair (the same answer in both warps).  For a bucket list, the job's
  // descriptors are in the rings; the prefetches for later jobs join the next commit group.
  auto acquire = [&](Job& jb) -> bool {
    const int64_t kk = k++;
    if (!valid(kk)) return false;
    if (QUEUE && from_list) {
      if (tid == 0) {
        if (valid(kk + 2)) fetch_item(kk + 2);
        if (valid(kk + 4)) cp_async4_64(reinterpret_cast<float*>(lidx + ((kk + 4) & 7)),
                                        reinterpret_cast<const float*>(list_at(kk + 4)));
      }
      jb = item_job(litem[kk & 3], lidx[kk & 7], T_pool, D_pool, tau, L_pool, s_pool, flags);
    } else {
      jb = dense_job(gp + kk * stride, N, t_max, Tt, Dg, tau, L, s, flags);
    }
    return true;
  };
  // Both warps copy a share of the job's T~ (N x N), D (N) and tau into slot `w`; thread 0
  // records its outputs and sizes.
  auto stage = [&](const Job& jb, int w) {
    float* S = slots + w * SLOT64;
    const int nn = jb.N * jb.N;
#ifdef TASER_DEBUG
    for (int i = tid; i < nn; i += 64)
      if (TASER_IN(i, SLOT64)) cp_async4_64(S + i, jb.T + i);
    for (int i = tid; i < jb.N; i += 64)
      if (TASER_IN(nn + i, SLOT64)) cp_async4_64(S + nn + i, jb.D + i);
    if (tid == 0) {
      if (TASER_IN(nn + jb.N, SLOT64)) cp_async4_64(S + nn + jb.N, jb.tau);
#else
    for (int i = tid; i < nn; i += 64) cp_async4_64(S + i, jb.T + i);
    for (int i = tid; i < jb.N; i += 64) cp_async4_64(S + nn + i, jb.D + i);
    if (tid == 0) {
      cp_async4_64(S + nn + jb.N, jb.tau);
#endif
      recs[w] = JobRec64{jb.L, jb.s, jb.flag, jb.N, jb.t_max};
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (QUEUE && from_list) {   // the first four list entries and two items, loaded directly
    if (tid == 0) {
      for (int64_t j = 0; j < 4 && valid(j); ++j) lidx[j] = *list_at(j);
      for (int64_t j = 0; j < 2 && valid(j); ++j) litem[j] = q.items[lidx[j]];
    }
    pair_bar(bar);
  }
  int cur = 0;
  bool have;
  {
    Job j0;
    have = acquire(j0);
    if (have) stage(j0, 0);
  }
  while (have) {
    bool have_next;
    {
      Job jn;
      have_next = acquire(jn);
      if (have_next) stage(jn, cur ^ 1);
    }
    if (have_next) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    pair_bar(bar);                                      // the current slot is complete in both warps
    const JobRec64 r = recs[cur];
    const float* S = slots + cur * SLOT64;
    Job jb;
    jb.T = S;
    jb.D = S + r.N * r.N;
    jb.tau = S + r.N * r.N + r.N;
    jb.L = r.L;
    jb.s = r.s;
    jb.flag = r.flag;
    jb.N = r.N;
    jb.t_max = r.t_max;
    if (role == 0) tc64_run<FP16, 0>(jb, X, lane, bar, literal);
    else tc64_run<FP16, 1>(jb, X, lane, bar, literal);
    pair_bar(bar);                                      // both warps are done with the slot and record
    cur ^= 1;
    have = have_next;
  }
}

template <bool FP16, bool QUEUE>
static cudaError_t launch_tc64(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                               int literal, float* L, int8_t* s, uint32_t* flags, const Queue& q, int blocks_per_sm,
                               const float* T_pool, const float* D_pool, float* L_pool, int8_t* s_pool,
                               cudaStream_t st) {
  const size_t smem = (size_t)2 * PAIR64 * sizeof(float);
  auto kern = detect_tc64_kernel<FP16, QUEUE>;
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, 128, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  int64_t blocks = (int64_t)sms * per_sm;
  if (!QUEUE) {
    const int64_t need = (batch + 1) / 2;
    if (need < blocks) blocks = need;
  }
  kern<<<(unsigned)blocks, 128, smem, st>>>(QUEUE, batch, N, Tt, D, tau, t_max, L, s, flags, q, T_pool, D_pool, L_pool,
                                            s_pool, literal);
  return cudaGetLastError();
}

cudaError_t detect_tc64(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                        int literal, bool fp16, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  Queue q{};
  return fp16 ? launch_tc64<true, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, q, 0, nullptr, nullptr,
                                         nullptr, nullptr, st)
              : launch_tc64<false, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, q, 0, nullptr, nullptr,
                                          nullptr, nullptr, st);
}

cudaError_t detect_tc64_queue(bool fp16, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, int literal, float* L_pool, int8_t* s_pool, uint32_t* flags,
                              cudaStream_t st) {
  return fp16 ? launch_tc64<true, true>(0, 0, nullptr, nullptr, tau, 0, literal, nullptr, nullptr, flags, q,
                                        blocks_per_sm, T_pool, D_pool, L_pool, s_pool, st)
              : launch_tc64<false, true>(0, 0, nullptr, nullptr, tau, 0, literal, nullptr, nullptr, flags, q,
                                         blocks_per_sm, T_pool, D_pool, L_pool, s_pool, st);
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(detect_tc64)
