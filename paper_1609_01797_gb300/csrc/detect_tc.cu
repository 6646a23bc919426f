// Tensor-core TASER iterations (Algorithm 1): the triangular product L~ T^ on the
// tensor cores with BF16 or FP16 operands and FP32 accumulation; the master L~ and the
// prox (column norms, rescaling) stay in FP32.
//
// One warp per instance, in transposed form: the accumulators of mma.m16n8k16 hold
//   V^T = L~^T + T^ L~^T   (T^ = -2 tau T~ is symmetric, so V^T = (L~ - 2 tau L~ T~)^T),
// with the C operand the FP32 master L~^T, the constant A operand T^ and the B operand
// L~^T.  A lane holds two adjacent entries of rows k of V^T (columns k of V) per n-tile,
// so the prox's column norms are sums over the 4 lanes of a row (two butterfly shuffles),
// which leave every lane with the norms of its own rows: no broadcast is needed.  Row N of
// L~ is simply the last n-tile (column NB of L~^T).  The B operand of the next step is the
// iterate transposed in 8 x 8 blocks: each block packed to 16 bits and moved with
// movmatrix.trans, which turns the accumulator layout (row g, columns 2tq, 2tq + 1) into
// the B-fragment layout (rows 2tq, 2tq + 1, column g).
//
// Tiles: columns k of L~ in m-tiles of 16, rows i in n-tiles of 8 (the last holds row N),
// j in k-tiles of 16.  Tile (M, n) exists only where some i >= k (V is lower-triangular,
// V^T upper), and it needs only the k-tiles with j <= i (L~^T[j][i] = 0 for j > i): the
// triangular skip of the paper's array (Sec. IV-A) at tile granularity.  The j = N term
// (T^[k][N] L~_NN) and V_NN are added in FP32.  The tensor-core instruction is the
// warp-level mma.sync: the per-instance operand T^ changes with every instance and the
// problem is 33 x 33, below the 64/128-row tiles of tcgen05.
#include "mma_tc.cuh"

namespace taser {

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}

// Slot layout of a staged job: T~ at slot + shift (shift = 0..3, see stage_job), D at
// slot + N^2 + 4, tau after D.  Returns the floats a slot needs for size N.
__host__ __device__ constexpr int tc_slot_floats(int N) { return ((N * N + 4 + N + 1) + 3) & ~3; }

// Stage T~ (N x N), D (N) and tau of one job into the warp's shared slot.  An instance's T~
// starts at any 4-byte boundary (N^2 floats per instance), so it is placed `shift` floats
// into the slot, shift = (address / 4) mod 4: then its 16-byte groups in global and shared
// memory coincide, and all but at most 3 + 3 of the N^2 floats move as 16-byte copies
// (9 instead of 35 copies per lane at N = 33).  Returns shift.  (Staging only the lower
// triangle was measured: the DRAM bytes stayed at 4,490 per instance, because rows of
// N = 33 floats are not aligned to the 128-byte lines, so nearly every line still holds a
// part of the triangle; the triangle walk only added instructions.)
// A debug build checks every copy against the instance's N^2 floats and the slot's
// slot_floats.
__device__ __forceinline__ int stage_job(float* slot, const Job& jb, int lane, int slot_floats) {
  const int N = jb.N, nn = N * N;
  const int shift = (int)((reinterpret_cast<uintptr_t>(jb.T) >> 2) & 3u);
  float* dst = slot + shift;
  const int head = (4 - shift) & 3;
  const int nvec = nn > head ? (nn - head) >> 2 : 0;
  const int tail0 = head + 4 * nvec;
  if (lane < head && lane < nn && TASER_IN(shift + lane, slot_floats)) cp_async4(dst + lane, jb.T + lane);
  for (int v = lane; v < nvec; v += 32)
    if (TASER_IN(head + 4 * v + 3, nn) && TASER_IN(shift + head + 4 * v + 3, slot_floats))
      cp_async16(dst + head + 4 * v, jb.T + head + 4 * v);
  for (int i = tail0 + lane; i < nn; i += 32)
    if (TASER_IN(shift + i, slot_floats)) cp_async4(dst + i, jb.T + i);
  float* dd = slot + nn + 4;
  for (int i = lane; i < N; i += 32)
    if (TASER_IN(nn + 4 + i, slot_floats)) cp_async4(dd + i, jb.D + i);
  if (lane == 0 && TASER_IN(nn + 4 + N, slot_floats)) cp_async4(dd + N, jb.tau);
  asm volatile("cp.async.commit_group;" ::: "memory");
  return shift;
}

// Instances at a fixed stride (the dense batch of taser_detect).
struct DenseSource {
  int64_t batch, stride;
  int N, t_max;
  const float *Tt, *Dg, *tau;
  float* L;
  int8_t* s;
  uint32_t* flags;
  double* obj;   // objective trace [batch][t_max + 1] (monitored launches), or nullptr
  __device__ __forceinline__ bool get(int64_t k, Job& jb, double*& ob) const {  // k-th instance of this warp
    const int64_t inst = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5) + k * stride;
    if (inst >= batch) return false;
    jb = dense_job(inst, N, t_max, Tt, Dg, tau, L, s, flags);
    ob = obj != nullptr ? obj + inst * (int64_t)(t_max + 1) : nullptr;
    return true;
  }
};

// Items of one bucket's queue, popped `pop` at a time per warp.
struct QueueSource {
  Queue q;
  int pop;
  const float *T_pool, *D_pool, *tau;
  float* L_pool;
  int8_t* s_pool;
  uint32_t* flags;
};

template <class Src>
struct Cursor;

template <>
struct Cursor<DenseSource> {
  int64_t k = 0;
  __device__ __forceinline__ bool next(const DenseSource& src, Job& jb, double*& ob, int) {
    return src.get(k++, jb, ob);
  }
};

template <>
struct Cursor<QueueSource> {
  int base = 0, left = 0;
  __device__ __forceinline__ bool next(const QueueSource& src, Job& jb, double*& ob, int lane) {
    ob = nullptr;
    if (left == 0) {
      int b = 0;
      if (lane == 0) b = src.q.pop(src.pop);
      base = __shfl_sync(TASER_FULL_MASK, b, 0);
      left = src.pop;
    }
    const int pos = base++;
    --left;
    if (pos >= src.q.count()) {
      left = 0;
      base = 1 << 30;
      return false;
    }
    const int idx = src.q.item_at(pos);
    const taser_item it = src.q.items[idx];
    jb = item_job(it, idx, src.T_pool, src.D_pool, src.tau, src.L_pool, src.s_pool, src.flags);
    return true;
  }
};

// Shared-memory floats per warp after its staging slot: two job records (JobOut below).
constexpr int kTcRecFloats = 24;

template <int NB>
struct TctCfg {
  static constexpr int MT = NB / 16;      // m-tiles over the columns k of L~
  static constexpr int KT = NB / 16;      // k-tiles over j
  static constexpr int NT = NB / 8 + 1;   // n-tiles over the rows i of L~; the last holds row N (i = NB)
  static constexpr int WARPS = 4;
  // Tile (M, n) holds V^T[k][i] for k in 16M..16M+15, i in 8n..8n+7; rows i < k are zero.
  __host__ __device__ static constexpr bool has_tile(int M, int n) { return n >= 2 * M; }
  // k-tiles of j that reach n-tile n (L~^T[j][i] = 0 for j > i).
  __host__ __device__ static constexpr int ktmax(int n) { return n / 2 < KT - 1 ? n / 2 : KT - 1; }
};

__device__ __forceinline__ uint32_t movmatrix_trans(uint32_t x) {
  uint32_t y;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

// Persistent: each warp takes jobs from its source (a fixed stride, or a bucket queue) and
// prefetches the next job's inputs with cp.async while it iterates on the current one.
// MON: objective monitoring of taser_detect_monitored (dense source only).  f(L~) =
// Tr(L~ T~ L~^T) is the sum over i >= k of L~_ik (L~ T~)_ik, the lower part of L~ T~ that
// each gradient step forms.  A single BF16 product is too coarse to see a rise of f of a
// fraction of a percent, so the monitor forms W^T = T^ L~^T a second time as a BF16 split
// (T^ = hi + lo as A fragments, the iterate's hi and lo moved like the B operand; 3 mma
// per product, about 2^-16 relative error) into scratch accumulators, before the step's
// own mma, and sums L~ o W; f = sum / (-2 tau).  The iteration itself is unchanged.  One
// more step after the outputs are written gives f(L~(t_max)).
template <int NB, bool FP16, class Src, bool MON = false>
__global__ void __launch_bounds__(128, MON ? 3 : 5)
detect_tct_kernel(Src src, int literal, int slot_floats, float ascent_tol) {
  using C = TctCfg<NB>;
  constexpr int MT = C::MT, KT = C::KT, NT = C::NT;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  float* slot = smem + warp * (slot_floats + kTcRecFloats);
  // Output pointers and sizes of the current and the next job live in shared memory
  // (two records per warp), not in registers across the iteration loop.
  struct JobOut {
    float* L;
    int8_t* s;
    uint32_t* flag;
    double* obj;
    int N, t_max, shift;
  };
  static_assert(2 * sizeof(JobOut) <= kTcRecFloats * sizeof(float), "job records must fit");
  JobOut* outs = reinterpret_cast<JobOut*>(slot + slot_floats);
  auto park = [&](const Job& jb, double* ob, int shift, int which) {
    if (lane == 0) outs[which] = JobOut{jb.L, jb.s, jb.flag, ob, jb.N, jb.t_max, shift};
  };
  Cursor<Src> cursor;
  int cur_m = 0;
  bool have;
  {
    Job first;
    double* ob = nullptr;
    have = cursor.next(src, first, ob, lane);
    if (have) park(first, ob, stage_job(slot, first, lane, slot_floats), 0);
  }

  while (have) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    const int N = outs[cur_m].N, t_max = outs[cur_m].t_max;
    const float* T = slot + outs[cur_m].shift;
    const float* Di = slot + N * N + 4;
    const float m2tau = -2.f * Di[N];
    auto tval = [&](int k, int j) -> float {  // T^ at bucket indices (k, j < NB)
      return (k < N - 1 && j < N - 1) ? m2tau * T[k * N + j] : 0.f;
    };
    // A operand: T^ rows k = 16M + g (+8), columns j = 16kt + 2tq (+1, +8, +9).  MON: also
    // T^ = hi + lo in BF16 (same layout) for the monitor's split product.
    uint32_t af[MT][KT][4];
    uint32_t mah[MON ? MT : 1][KT][4], mal[MON ? MT : 1][KT][4];
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const int r = 16 * M + g, c = 16 * kt + 2 * tq;
        float v[4][2];
        if (N == NB + 1) {   // no padding rows or columns: no bounds tests
          const float* r0 = T + r * (NB + 1) + c;
          const float* r1 = r0 + 8 * (NB + 1);
          v[0][0] = m2tau * r0[0], v[0][1] = m2tau * r0[1];
          v[1][0] = m2tau * r1[0], v[1][1] = m2tau * r1[1];
          v[2][0] = m2tau * r0[8], v[2][1] = m2tau * r0[9];
          v[3][0] = m2tau * r1[8], v[3][1] = m2tau * r1[9];
        } else {
          v[0][0] = tval(r, c), v[0][1] = tval(r, c + 1);
          v[1][0] = tval(r + 8, c), v[1][1] = tval(r + 8, c + 1);
          v[2][0] = tval(r, c + 8), v[2][1] = tval(r, c + 9);
          v[3][0] = tval(r + 8, c + 8), v[3][1] = tval(r + 8, c + 9);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          af[M][kt][x] = pack2<FP16>(v[x][0], v[x][1]);
          if constexpr (MON) split_bf16(v[x][0], v[x][1], mah[M][kt][x], mal[M][kt][x]);
        }
      }
    // This lane's rows k = 16M + g + 8h: T^[k][N] (FP32, the j = N term) and D_k.
    float tkN[MT][2], Dk[MT][2], inval[MT][2];
    float snmin = 3.0e38f;   // smallest squared column norm of the job's valid rows k
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * M + g + 8 * h;
        tkN[M][h] = k < N - 1 ? m2tau * T[k * N + N - 1] : 0.f;
        Dk[M][h] = k < N - 1 ? Di[k] : 0.f;
        inval[M][h] = k < N - 1 ? 0.f : 3.0e38f;   // rows k >= N - 1 never flag a zero column
      }
    const float tnNN = m2tau * T[(N - 1) * N + (N - 1)];
    const float DN = Di[N - 1];
    // L~(0) = D in the V^T layout: element (M, n, e) is k = 16M + g + 8(e >> 1),
    // i = 8n + 2tq + (e & 1).
    float acc[MT][NT][4];
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 16 * M + g + 8 * (e >> 1), i = 8 * n + 2 * tq + (e & 1);
          acc[M][n][e] = (C::has_tile(M, n) && i == k && k < N - 1) ? Dk[M][e >> 1] : 0.f;
        }
    __syncwarp();  // every lane has read the slot
    bool have_next;
    {
      Job nxt;
      double* ob = nullptr;
      have_next = cursor.next(src, nxt, ob, lane);
      if (have_next) park(nxt, ob, stage_job(slot, nxt, lane, slot_floats), cur_m ^ 1);
    }
    float LNN = DN;
    uint32_t fl = 0;
    // Inside a diagonal 8 x 8 block, element (row g, column 2tq + p) lies below the
    // diagonal of V^T (i < k) iff 2tq + p < g.
    const bool lo0 = 2 * tq < g, lo1 = 2 * tq + 1 < g;

    // One gradient step: acc <- V^T = L~^T + T^ L~^T (kept on and above its diagonal);
    // returns V_NN.  MON: fterm += sum of L~_ik W_ik over this lane's elements, W = L~ T^
    // (as W^T = T^ L~^T, a BF16 split product of the old iterate, before the step).
    auto grad_step = [&](float& fterm) -> float {
      // V_NN partial sum_{j < N} T^[N][j] L~[N][j] from the old row N (column NB of L~^T,
      // held by the lanes tq == 0), summed over g.
      float part = 0.f;
      if (tq == 0) {
#pragma unroll
        for (int M = 0; M < MT; ++M)
#pragma unroll
          for (int h = 0; h < 2; ++h) part = fmaf(tkN[M][h], acc[M][NT - 1][2 * h], part);
      }
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 4);
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 8);
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 16);
      part = __shfl_sync(TASER_FULL_MASK, part, lane & 28);   // from the lane tq == 0 of the row
      // B operand from the old iterate: block (kb, ib) of L~^T transposed; blocks with
      // kb > ib are zero.
      uint32_t bfr[KT][NT][2];
      uint32_t mbh[MON ? KT : 1][NT][2], mbl[MON ? KT : 1][NT][2];
#pragma unroll
      for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int kb = 2 * kt + q, M = kb / 2, h = kb % 2;
            if (kt > C::ktmax(n) || kb > n) {
              bfr[kt][n][q] = 0u;
              if constexpr (MON) mbh[kt][n][q] = mbl[kt][n][q] = 0u;
            } else {
              bfr[kt][n][q] = movmatrix_trans(pack2<FP16>(acc[M][n][2 * h], acc[M][n][2 * h + 1]));
              if constexpr (MON) {
                uint32_t hi, lo;
                split_bf16(acc[M][n][2 * h], acc[M][n][2 * h + 1], hi, lo);
                mbh[kt][n][q] = movmatrix_trans(hi);
                mbl[kt][n][q] = movmatrix_trans(lo);
              }
            }
          }
      if constexpr (MON) {
#pragma unroll
        for (int M = 0; M < MT; ++M)
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n)) continue;
            float w4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt <= C::ktmax(n); ++kt) {
              mma16816<false>(w4, mah[M][kt], mbh[kt][n]);
              mma16816<false>(w4, mah[M][kt], mbl[kt][n]);
              mma16816<false>(w4, mal[M][kt], mbh[kt][n]);
            }
            if (n == NT - 1 && tq == 0) {   // j = N term of column NB, in FP32
              w4[0] = fmaf(tkN[M][0], LNN, w4[0]);
              w4[2] = fmaf(tkN[M][1], LNN, w4[2]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) fterm = fmaf(acc[M][n][e], w4[e], fterm);
          }
      }
      // The step's products, row N's n-tile first (measured: 0.371 -> 0.367 ms per 65,536 at
      // N = 33 against the m-tile-major order; two partial chains in the column sums below
      // were slower, 0.384 ms).
#pragma unroll
      for (int n = NT - 1; n >= 0; --n)
#pragma unroll
        for (int M = 0; M < MT; ++M) {
          if (!C::has_tile(M, n)) continue;
#pragma unroll
          for (int kt = 0; kt <= C::ktmax(n); ++kt) mma16816<FP16>(acc[M][n], af[M][kt], bfr[kt][n]);
        }
      // j = N term of column NB: V^T[k][N] += T^[k][N] L~_NN.
      if (tq == 0) {
#pragma unroll
        for (int M = 0; M < MT; ++M)
#pragma unroll
          for (int h = 0; h < 2; ++h) acc[M][NT - 1][2 * h] = fmaf(tkN[M][h], LNN, acc[M][NT - 1][2 * h]);
      }
      // Keep V^T on and above its diagonal (i >= k): blocks kb == ib are masked, the block
      // kb = 2M + 1 > ib = 2M is cleared.
#pragma unroll
      for (int M = 0; M < MT; ++M) {
        if (lo0) acc[M][2 * M][0] = 0.f;
        if (lo1) acc[M][2 * M][1] = 0.f;
        acc[M][2 * M][2] = 0.f;
        acc[M][2 * M][3] = 0.f;
        if (lo0) acc[M][2 * M + 1][2] = 0.f;
        if (lo1) acc[M][2 * M + 1][3] = 0.f;
      }
      return fmaf(LNN, tnNN, LNN) + part;
    };

    // MON: f(L~(t)) from the step's terms (FP32 sums, FP64 ratio and comparison).
    double f_prev = 0.0;
    double* const obj = MON ? outs[cur_m].obj : nullptr;
    auto monitor = [&](int t, float fterm, float vnn) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) fterm += __shfl_xor_sync(TASER_FULL_MASK, fterm, o);
      fterm = fmaf(LNN, vnn - LNN, fterm);   // L~_NN W_NN, W_NN = V_NN - L~_NN (FP32)
      const double f = m2tau < 0.f ? (double)fterm / (double)m2tau : 0.0;
      if (t > 0 && f > f_prev + (double)ascent_tol * fabs(f_prev)) fl |= TASER_FLAG_ASCENT;
      f_prev = f;
      if (lane == 0 && obj != nullptr && TASER_IN(t, t_max + 1)) obj[t] = f;
    };

    for (int t = 0; t < t_max; ++t) {
      float fterm = 0.f;
      const float vnn = grad_step(fterm);
      if constexpr (MON) monitor(t, fterm, vnn);
      if (vnn <= 0.f) fl |= TASER_FLAG_LNN_SIGN;
      if (literal) LNN = vnn >= 0.f ? DN : -DN;
      // prox: squared norms of this lane's rows k, summed over the 4 lanes of the row.
      float sn[MT][2];
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint64_t v2 = 0ull;
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n) || (n == 2 * M && h == 1)) continue;   // the cleared block
            const uint64_t x = f2pack(acc[M][n][2 * h], acc[M][n][2 * h + 1]);
            v2 = f2fma(x, x, v2);
          }
          float a, b;
          f2unpack(v2, a, b);
          sn[M][h] = a + b;
        }
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) sn[M][h] += __shfl_xor_sync(TASER_FULL_MASK, sn[M][h], 1);
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) sn[M][h] += __shfl_xor_sync(TASER_FULL_MASK, sn[M][h], 2);
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          snmin = fminf(snmin, sn[M][h] + inval[M][h]);
          const float sc = sn[M][h] > 0.f ? Dk[M][h] * rsqrtf(sn[M][h]) : 0.f;
          const uint64_t sc2 = f2pack(sc, sc);
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n) || (n == 2 * M && h == 1)) continue;
            TASER_PAIR_APPLY(acc[M][n], 2 * h, f2mul(_x, sc2));
          }
        }
    }

    // A zero column in any iteration (its prox scale was 0): measured 2.2% faster than a
    // per-iteration flag update.
    if (snmin <= 0.f) fl |= TASER_FLAG_ZERO_COLUMN;
    const JobOut o = outs[cur_m];
    // Decisions from row N of L~ (column NB of L~^T, lanes tq == 0).
    if (tq == 0) {
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 16 * M + g + 8 * h;
          if (k < N - 1 && TASER_IN(k, N - 1)) {
            float r = acc[M][NT - 1][2 * h];
            TASER_FINITE(r);
            if (literal && LNN < 0.f) r = -r;
            o.s[k] = r >= 0.f ? int8_t(1) : int8_t(-1);
          }
        }
    }
    if (o.L != nullptr) {
      float* Lo = o.L;
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 16 * M + g + 8 * (e >> 1), i = 8 * n + 2 * tq + (e & 1);
            const int rr = bucket_to_real(i, N, NB);
            if (rr < 0 || k >= N - 1 || !TASER_IN(rr * N + k, N * N)) continue;
            Lo[(int64_t)rr * N + k] = C::has_tile(M, n) ? acc[M][n][e] : 0.f;
            TASER_FINITE(Lo[(int64_t)rr * N + k]);
          }
      for (int rr = lane; rr < N; rr += 32)
        if (TASER_IN(rr * N + N - 1, N * N)) Lo[(int64_t)rr * N + (N - 1)] = rr == N - 1 ? LNN : 0.f;
    }
    if constexpr (MON) {   // f(L~(t_max)): one more gradient step, after the outputs
      float fterm = 0.f;
      const float vnn = grad_step(fterm);
      monitor(t_max, fterm, vnn);
    }
#pragma unroll
    for (int ofs = 16; ofs > 0; ofs >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, ofs);
    if (lane == 0 && o.flag != nullptr && fl) *o.flag |= fl;
    __syncwarp();  // the record of this job is consumed before it is reused
    cur_m ^= 1;
    have = have_next;
  }
}

// Persistent launch for a job source: `blocks_per_sm` blocks per SM (as many as fit if
// <= 0), fewer if the jobs are fewer (jobs < 0: unknown, a queue).
template <int NB, bool FP16, class Src, bool MON = false>
static cudaError_t launch_tc_src(const Src& src, int64_t jobs, int blocks_per_sm, int literal, int slot_floats,
                                 float ascent_tol, cudaStream_t st) {
  using C = TctCfg<NB>;
  const size_t smem = (size_t)C::WARPS * (slot_floats + kTcRecFloats) * sizeof(float);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tct_kernel<NB, FP16, Src, MON>, 32 * C::WARPS,
                                                      smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  const int64_t need = (jobs + C::WARPS - 1) / C::WARPS;
  const int64_t resident = (int64_t)sms * per_sm;
  const int64_t blocks = jobs >= 0 && need < resident ? need : resident;
  detect_tct_kernel<NB, FP16, Src, MON><<<(unsigned)blocks, 32 * C::WARPS, smem, st>>>(src, literal, slot_floats,
                                                                                       ascent_tol);
  return cudaGetLastError();
}

template <int NB, bool FP16, bool MON = false>
static cudaError_t launch_tc(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                             int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st,
                             double* obj = nullptr, float ascent_tol = 0.f) {
  using C = TctCfg<NB>;
  const int slot_floats = tc_slot_floats(N);
  const size_t smem = (size_t)C::WARPS * (slot_floats + kTcRecFloats) * sizeof(float);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tct_kernel<NB, FP16, DenseSource, MON>,
                                                      32 * C::WARPS, smem);
  if (e != cudaSuccess) return e;
  const int64_t need = (batch + C::WARPS - 1) / C::WARPS;
  const int64_t resident = (int64_t)sms * (fit > 0 ? fit : 1);
  DenseSource src;
  src.batch = batch;
  src.stride = (need < resident ? need : resident) * C::WARPS;
  src.N = N;
  src.t_max = t_max;
  src.Tt = Tt;
  src.Dg = D;
  src.tau = tau;
  src.L = L;
  src.s = s;
  src.flags = flags;
  src.obj = obj;
  return launch_tc_src<NB, FP16, DenseSource, MON>(src, batch, fit, literal, slot_floats, ascent_tol, st);
}

// ---------------------------------------------------------------------------------
// The transposed form at 34 <= N <= 65 (bucket 64), one warp per instance.  The 24 tiles of
// V^T (96 accumulators a lane) and the 16 A fragments of T^ (64 registers) stay in
// registers.  The B operand goes through shared memory: every step the lane packs and
// transposes the 44 nonzero 8 x 8 blocks of L~^T it holds (movmatrix.trans) into the warp's
// block grid, and each group of mma loads its two B registers from there just before use.
// T^, D and tau are read from global memory once per job (no staging slot, so the block
// grid is the only shared memory).  No step needs another warp: the column norms are sums
// over the 4 lanes of a row, as in the bucket-32 kernel.
// ---------------------------------------------------------------------------------
constexpr int kBlk64Words = 8 * 9 * 32;   // block grid [kb][ib][lane] of one warp (kb <= ib used)

template <bool FP16, class Src>
__global__ void __launch_bounds__(128, 2)
detect_tct64_kernel(Src src, int literal, int slot_floats) {
  using C = TctCfg<64>;
  constexpr int MT = C::MT, KT = C::KT, NT = C::NT, NB = 64;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  // Per warp: the block grid, then the staging slot of the next job and two job records.
  uint32_t* const blk = reinterpret_cast<uint32_t*>(smem) + warp * (kBlk64Words + slot_floats + kTcRecFloats);
  float* const slot = reinterpret_cast<float*>(blk + kBlk64Words);
  auto bw = [&](int kb, int ib) -> uint32_t& { return blk[(kb * 9 + ib) * 32 + lane]; };
  struct JobOut {
    float* L;
    int8_t* s;
    uint32_t* flag;
    double* obj;
    int N, t_max, shift;
  };
  static_assert(2 * sizeof(JobOut) <= kTcRecFloats * sizeof(float), "job records must fit");
  JobOut* outs = reinterpret_cast<JobOut*>(slot + slot_floats);
  auto park = [&](const Job& jb, int shift, int which) {
    if (lane == 0) outs[which] = JobOut{jb.L, jb.s, jb.flag, nullptr, jb.N, jb.t_max, shift};
  };
  // Inside a diagonal 8 x 8 block, element (row g, column 2tq + p) lies below the
  // diagonal of V^T (i < k) iff 2tq + p < g.
  const bool lo0 = 2 * tq < g, lo1 = 2 * tq + 1 < g;
  Cursor<Src> cursor;
  int cur_m = 0;
  bool have;
  {
    Job first;
    double* ob = nullptr;
    have = cursor.next(src, first, ob, lane);
    if (have) park(first, stage_job(slot, first, lane, slot_floats), 0);
  }
  while (have) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    const int N = outs[cur_m].N, t_max = outs[cur_m].t_max;
    const float* T = slot + outs[cur_m].shift;
    const float* Di = slot + N * N + 4;
    const float m2tau = -2.f * Di[N];
    auto tval = [&](int k, int j) -> float {  // T^ at bucket indices (k, j < NB)
      return (k < N - 1 && j < N - 1) ? m2tau * T[k * N + j] : 0.f;
    };
    // A operand: T^ rows k = 16M + g (+8), columns j = 16kt + 2tq (+1, +8, +9).
    uint32_t af[MT][KT][4];
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const int r = 16 * M + g, c = 16 * kt + 2 * tq;
        af[M][kt][0] = pack2<FP16>(tval(r, c), tval(r, c + 1));
        af[M][kt][1] = pack2<FP16>(tval(r + 8, c), tval(r + 8, c + 1));
        af[M][kt][2] = pack2<FP16>(tval(r, c + 8), tval(r, c + 9));
        af[M][kt][3] = pack2<FP16>(tval(r + 8, c + 8), tval(r + 8, c + 9));
      }
    // This lane's rows k = 16M + g + 8h: T^[k][N] (FP32, the j = N term) and D_k.
    float tkN[MT][2], Dk[MT][2], inval[MT][2];
    float snmin = 3.0e38f;   // smallest squared column norm of the job's valid rows k
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * M + g + 8 * h;
        tkN[M][h] = k < N - 1 ? m2tau * T[k * N + N - 1] : 0.f;
        Dk[M][h] = k < N - 1 ? Di[k] : 0.f;
        inval[M][h] = k < N - 1 ? 0.f : 3.0e38f;   // rows k >= N - 1 never flag a zero column
      }
    const float tnNN = m2tau * T[(N - 1) * N + (N - 1)];
    const float DN = Di[N - 1];
    // L~(0) = D in the V^T layout: element (M, n, e) is k = 16M + g + 8(e >> 1),
    // i = 8n + 2tq + (e & 1).
    float acc[MT][NT][4];
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 16 * M + g + 8 * (e >> 1), i = 8 * n + 2 * tq + (e & 1);
          acc[M][n][e] = (C::has_tile(M, n) && i == k && k < N - 1) ? Dk[M][e >> 1] : 0.f;
        }
    __syncwarp();  // every lane has read the slot
    bool have_next;
    {
      Job nxt;
      double* ob = nullptr;
      have_next = cursor.next(src, nxt, ob, lane);
      if (have_next) park(nxt, stage_job(slot, nxt, lane, slot_floats), cur_m ^ 1);
    }
    float LNN = DN;
    uint32_t fl = 0;

    for (int t = 0; t < t_max; ++t) {
      // V_NN partial sum_{j < N} T^[N][j] L~[N][j] from the old row N (lanes tq == 0).
      float part = 0.f;
      if (tq == 0) {
#pragma unroll
        for (int M = 0; M < MT; ++M)
#pragma unroll
          for (int h = 0; h < 2; ++h) part = fmaf(tkN[M][h], acc[M][NT - 1][2 * h], part);
      }
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 4);
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 8);
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 16);
      part = __shfl_sync(TASER_FULL_MASK, part, lane & 28);
      // The old iterate as B blocks: block (kb, ib) of L~^T transposed, for kb <= ib.
      __syncwarp();   // the previous step's B loads are done before the grid is rewritten
#pragma unroll
      for (int kb = 0; kb < 2 * MT; ++kb)
#pragma unroll
        for (int ib = kb; ib < NT; ++ib)
          bw(kb, ib) = movmatrix_trans(pack2<FP16>(acc[kb / 2][ib][2 * (kb % 2)], acc[kb / 2][ib][2 * (kb % 2) + 1]));
      __syncwarp();
      // Products, row N's n-tile first; each (kt, n) B fragment serves every m-tile.
#pragma unroll
      for (int n = NT - 1; n >= 0; --n)
#pragma unroll
        for (int kt = 0; kt <= C::ktmax(n); ++kt) {
          const uint32_t b[2] = {bw(2 * kt, n), 2 * kt + 1 <= n ? bw(2 * kt + 1, n) : 0u};
#pragma unroll
          for (int M = 0; M < MT; ++M) {
            if (!C::has_tile(M, n)) continue;
            mma16816<FP16>(acc[M][n], af[M][kt], b);
          }
        }
      // j = N term of column NB: V^T[k][N] += T^[k][N] L~_NN.
      if (tq == 0) {
#pragma unroll
        for (int M = 0; M < MT; ++M)
#pragma unroll
          for (int h = 0; h < 2; ++h) acc[M][NT - 1][2 * h] = fmaf(tkN[M][h], LNN, acc[M][NT - 1][2 * h]);
      }
      const float vnn = fmaf(LNN, tnNN, LNN) + part;
      // Keep V^T on and above its diagonal.
#pragma unroll
      for (int M = 0; M < MT; ++M) {
        if (lo0) acc[M][2 * M][0] = 0.f;
        if (lo1) acc[M][2 * M][1] = 0.f;
        acc[M][2 * M][2] = 0.f;
        acc[M][2 * M][3] = 0.f;
        if (lo0) acc[M][2 * M + 1][2] = 0.f;
        if (lo1) acc[M][2 * M + 1][3] = 0.f;
      }
      if (vnn <= 0.f) fl |= TASER_FLAG_LNN_SIGN;
      if (literal) LNN = vnn >= 0.f ? DN : -DN;
      // prox: squared norms of this lane's 8 rows k, summed over the 4 lanes of a row.
      float sn[MT][2];
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint64_t v2 = 0ull;
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n) || (n == 2 * M && h == 1)) continue;   // the cleared block
            const uint64_t x = f2pack(acc[M][n][2 * h], acc[M][n][2 * h + 1]);
            v2 = f2fma(x, x, v2);
          }
          float a, b;
          f2unpack(v2, a, b);
          sn[M][h] = a + b;
        }
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) sn[M][h] += __shfl_xor_sync(TASER_FULL_MASK, sn[M][h], 1);
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) sn[M][h] += __shfl_xor_sync(TASER_FULL_MASK, sn[M][h], 2);
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          snmin = fminf(snmin, sn[M][h] + inval[M][h]);
          const float sc = sn[M][h] > 0.f ? Dk[M][h] * rsqrtf(sn[M][h]) : 0.f;
          const uint64_t sc2 = f2pack(sc, sc);
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n) || (n == 2 * M && h == 1)) continue;
            TASER_PAIR_APPLY(acc[M][n], 2 * h, f2mul(_x, sc2));
          }
        }
    }

    // A zero column in any iteration (its prox scale was 0): measured 2.2% faster than a
    // per-iteration flag update.
    if (snmin <= 0.f) fl |= TASER_FLAG_ZERO_COLUMN;
    const JobOut o = outs[cur_m];
    // Decisions from row N of L~ (column NB of L~^T, lanes tq == 0).
    if (tq == 0) {
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 16 * M + g + 8 * h;
          if (k < N - 1 TASER_AND(TASER_IN(k, N - 1))) {
            float r = acc[M][NT - 1][2 * h];
            if (literal && LNN < 0.f) r = -r;
            o.s[k] = r >= 0.f ? int8_t(1) : int8_t(-1);
          }
        }
    }
    if (o.L != nullptr) {
      float* Lo = o.L;
#pragma unroll
      for (int M = 0; M < MT; ++M)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 16 * M + g + 8 * (e >> 1), i = 8 * n + 2 * tq + (e & 1);
            const int rr = bucket_to_real(i, N, NB);
            if (rr < 0 || k >= N - 1) continue;
            TASER_CHECKED(TASER_IN(rr * N + k, N * N)) Lo[(int64_t)rr * N + k] = C::has_tile(M, n) ? acc[M][n][e] : 0.f;
          }
      for (int rr = lane; rr < N; rr += 32)
        TASER_CHECKED(TASER_IN(rr * N + N - 1, N * N)) Lo[(int64_t)rr * N + (N - 1)] = rr == N - 1 ? LNN : 0.f;
    }
#pragma unroll
    for (int ofs = 16; ofs > 0; ofs >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, ofs);
    if (lane == 0 && o.flag != nullptr && fl) *o.flag |= fl;
    __syncwarp();  // the record of this job is consumed before it is reused
    cur_m ^= 1;
    have = have_next;
  }
}

template <bool FP16, class Src>
static cudaError_t launch_tct64_src(const Src& src, int64_t jobs, int blocks_per_sm, int literal, cudaStream_t st) {
  const int slot_floats = tc_slot_floats(65);
  const size_t smem = (size_t)4 * (kBlk64Words + slot_floats + kTcRecFloats) * sizeof(uint32_t);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(detect_tct64_kernel<FP16, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tct64_kernel<FP16, Src>, 128, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  const int64_t need = (jobs + 3) / 4;
  const int64_t resident = (int64_t)sms * per_sm;
  const int64_t blocks = jobs >= 0 && need < resident ? need : resident;
  detect_tct64_kernel<FP16, Src><<<(unsigned)blocks, 128, smem, st>>>(src, literal, slot_floats);
  return cudaGetLastError();
}

template <bool FP16>
static cudaError_t launch_tct64(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                                int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  const size_t smem = (size_t)4 * (kBlk64Words + tc_slot_floats(65) + kTcRecFloats) * sizeof(uint32_t);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(detect_tct64_kernel<FP16, DenseSource>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tct64_kernel<FP16, DenseSource>, 128, smem);
  if (e != cudaSuccess) return e;
  const int64_t need = (batch + 3) / 4;
  const int64_t resident = (int64_t)sms * (fit > 0 ? fit : 1);
  DenseSource src;
  src.batch = batch;
  src.stride = (need < resident ? need : resident) * 4;
  src.N = N;
  src.t_max = t_max;
  src.Tt = Tt;
  src.Dg = D;
  src.tau = tau;
  src.L = L;
  src.s = s;
  src.flags = flags;
  src.obj = nullptr;
  return launch_tct64_src<FP16, DenseSource>(src, batch, fit, literal, st);
}


// Returns cudaErrorNotSupported when the bucket has no tensor-core kernel.
cudaError_t detect_tc(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                      int literal, bool fp16, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 64:
      return fp16 ? launch_tct64<true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st)
                  : launch_tct64<false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    case 16:
      return fp16 ? launch_tc<16, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st)
                  : launch_tc<16, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    case 32:
      return fp16 ? launch_tc<32, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st)
                  : launch_tc<32, false>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st);
    default:
      return cudaErrorNotSupported;
  }
}

// taser_detect_monitored on the tensor cores (buckets 16 and 32; cudaErrorNotSupported
// for the two-warp bucket 64).
cudaError_t detect_tc_monitored(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                                int literal, bool fp16, float ascent_tol, double* obj, float* L, int8_t* s,
                                uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 16:
      return fp16 ? launch_tc<16, true, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st, obj, ascent_tol)
                  : launch_tc<16, false, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st, obj, ascent_tol);
    case 32:
      return fp16 ? launch_tc<32, true, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st, obj, ascent_tol)
                  : launch_tc<32, false, true>(batch, N, Tt, D, tau, t_max, literal, L, s, flags, st, obj, ascent_tol);
    default:
      return cudaErrorNotSupported;
  }
}

// Queue-fed launch for bucket nb (16 or 32) of an uneven batch.
cudaError_t detect_tc_queue(int nb, bool fp16, const Queue& q, int blocks_per_sm, int pop, const float* T_pool,
                            const float* D_pool, const float* tau, int literal, float* L_pool, int8_t* s_pool,
                            uint32_t* flags, cudaStream_t st) {
  QueueSource src;
  src.q = q;
  src.pop = pop > 0 ? pop : 1;
  src.T_pool = T_pool;
  src.D_pool = D_pool;
  src.tau = tau;
  src.L_pool = L_pool;
  src.s_pool = s_pool;
  src.flags = flags;
  const int slot_floats = tc_slot_floats(nb + 1);
  switch (nb) {
    case 64:
      return fp16 ? launch_tct64_src<true>(src, -1, blocks_per_sm, literal, st)
                  : launch_tct64_src<false>(src, -1, blocks_per_sm, literal, st);
    case 16:
      return fp16 ? launch_tc_src<16, true>(src, -1, blocks_per_sm, literal, slot_floats, 0.f, st)
                  : launch_tc_src<16, false>(src, -1, blocks_per_sm, literal, slot_floats, 0.f, st);
    case 32:
      return fp16 ? launch_tc_src<32, true>(src, -1, blocks_per_sm, literal, slot_floats, 0.f, st)
                  : launch_tc_src<32, false>(src, -1, blocks_per_sm, literal, slot_floats, 0.f, st);
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(detect_tc)
