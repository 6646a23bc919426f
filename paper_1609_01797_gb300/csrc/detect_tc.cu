// Tensor-core TASER iterations (Algorithm 1): the triangular product L~ T^ on the
// tensor cores with BF16 or FP16 operands and FP32 accumulation; the master L~ and the
// prox (column norms, rescaling) stay in FP32.
//
// One warp per instance.  L~ is kept in registers in the accumulator layout of
// mma.m16n8k16: an accumulator pair of n-tiles (2k, 2k+1) is exactly the A operand of
// k-tile k, so the next iteration's A operand is a register conversion, no shuffle or
// shared-memory round trip.  The C operand is the FP32 master L~ and B = -2 tau T~, so
// one mma gives V = L~ - L~ T^ directly.
//
// Tiles: rows are split into m-tiles of 16, variable columns into n-tiles of 8 and
// k-tiles of 16.  Row block M (< NB/16) needs k-tiles 0..M and n-tiles 0..2M+1 only (L~
// is lower-triangular, V is kept on and below the diagonal): the triangular skip of the
// paper's array (Sec. IV-A) at tile granularity.  The augmented last row NB is one more
// m-tile whose only live row is row NB; its L~_NN T^_{N,c} term is added in FP32.
// The tensor-core instruction is the warp-level mma.sync: the per-instance operand B
// changes with every instance and M is 33 rows, below the 64/128-row tiles of tcgen05.
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

// Persistent: each warp takes jobs from its source (a fixed stride, or a bucket queue) and
// prefetches the next job's inputs with cp.async while it iterates on the current one.
// MON: objective monitoring of taser_detect_monitored (dense source only).  f(L~) =
// Tr(L~ T~ L~^T) is the sum over i >= k of L~_ik (L~ T~)_ik, the lower part of L~ T~ that
// each gradient step forms.  A single BF16 product is too coarse to see a rise of f of a
// fraction of a percent, so the monitor forms W = L~ T^ (T^ = -2 tau T~) tile by tile a
// second time as a BF16 split (3 mma per product, about 2^-16 relative error) into
// scratch accumulators, before the tile's own mma, and sums L~ o W; f = sum / (-2 tau).
// The iteration itself is unchanged.  One more step after the outputs are written gives
// f(L~(t_max)).
template <int NB, bool FP16, class Src, bool MON = false>
__global__ void __launch_bounds__(128, MON ? 3 : 4)
detect_tc_kernel(Src src, int literal, int slot_floats, float ascent_tol) {
  using C = TcCfg<NB>;
  constexpr int KT = C::KT, NT = C::NT, MT = C::MT;
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
    if (have) {
      const int shift = stage_job(slot, first, lane, slot_floats);
      park(first, ob, shift, 0);
    }
  }

  while (have) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    const int N = outs[cur_m].N, t_max = outs[cur_m].t_max;
    const float* T = slot + outs[cur_m].shift;
    const float* Di = slot + N * N + 4;
    const float m2tau = -2.f * Di[N];
    auto tval = [&](int k, int n) -> float {  // -2 tau T~ at bucket indices (k, n < NB)
      return (k < N - 1 && n < N - 1) ? m2tau * T[k * N + n] : 0.f;
    };
    // B operand: B[k][n] = -2 tau T~[k][n]; lane holds rows 2tq..2tq+1 and +8, column g.
    // A problem that fills the bucket (N = NB + 1, e.g. QPSK 128x16 at N = 33) has no padding
    // rows or columns, so its values need no bounds test.
    uint32_t bf[KT][NT][2];
    if (N == NB + 1) {
#pragma unroll
      for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int k0 = 16 * kt + 2 * tq, n = 8 * nt + g;
          const float* c0 = T + k0 * (NB + 1) + n;
          if (!TASER_IN((k0 + 9) * (NB + 1) + n, N * N)) {
            bf[kt][nt][0] = bf[kt][nt][1] = 0u;
            continue;
          }
          bf[kt][nt][0] = pack2<FP16>(m2tau * c0[0], m2tau * c0[NB + 1]);
          bf[kt][nt][1] = pack2<FP16>(m2tau * c0[8 * (NB + 1)], m2tau * c0[9 * (NB + 1)]);
        }
    } else {
#pragma unroll
      for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int k0 = 16 * kt + 2 * tq, n = 8 * nt + g;
          bf[kt][nt][0] = pack2<FP16>(tval(k0, n), tval(k0 + 1, n));
          bf[kt][nt][1] = pack2<FP16>(tval(k0 + 8, n), tval(k0 + 9, n));
        }
    }
    // MON: T^ = hi + lo in BF16 (B layout of bf).
    uint32_t mbh[MON ? KT : 1][NT][2], mbl[MON ? KT : 1][NT][2];
    if constexpr (MON) {
#pragma unroll
      for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int k0 = 16 * kt + 2 * tq, n = 8 * nt + g;
          split_bf16(tval(k0, n), tval(k0 + 1, n), mbh[kt][nt][0], mbl[kt][nt][0]);
          split_bf16(tval(k0 + 8, n), tval(k0 + 9, n), mbh[kt][nt][1], mbl[kt][nt][1]);
        }
    }
    // Row N of T^ at this lane's accumulator columns c = 8n + 2tq + p (FP32).
    float tN[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int c = 8 * nt + 2 * tq + p;
        tN[nt][p] = (g == 0 && c < N - 1 && TASER_IN((N - 1) * N + c, N * N)) ? m2tau * T[(N - 1) * N + c] : 0.f;
      }
    uint64_t tN2[NT];   // packed pairs (zero off the lanes g == 0 that hold row N)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) tN2[nt] = f2pack(tN[nt][0], tN[nt][1]);
    auto tN2f = [&](int n, int p) -> float { return tN[n][p]; };
    const float tnNN = m2tau * T[(N - 1) * N + (N - 1)];
    const float DN = Di[N - 1];
    // After the column-sum reduction this lane owns column cown.
    const int own_idx = NT == 4 ? g : (g >> 1);
    const int cown = 8 * (own_idx >> 1) + 2 * tq + (own_idx & 1);
    const float Down = cown < N - 1 ? Di[cown] : 0.f;
    // L~(0) = D in accumulator layout: element (M, n, e) is row 16M + g + 8(e >> 1),
    // column 8n + 2tq + (e & 1).
    float acc[MT][NT][4];
#pragma unroll
    for (int M = 0; M < MT; ++M)
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 16 * M + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
          acc[M][n][e] = (M < MT - 1 && r == c && r < N - 1) ? Di[r] : 0.f;
        }
    __syncwarp();  // every lane has read the slot
    bool have_next;
    {
      Job nxt;
      double* ob = nullptr;
      have_next = cursor.next(src, nxt, ob, lane);
      if (have_next) {
        const int shift = stage_job(slot, nxt, lane, slot_floats);
        park(nxt, ob, shift, cur_m ^ 1);
      }
    }
    float LNN = DN;
    uint32_t fl = 0;
    // Inside a diagonal 16 x 16 block the element (row g + 8h, column 2tq + p + 8h') lies
    // above the diagonal iff h' > h, or h' == h and 2tq + p > g.
    const bool up0 = 2 * tq > g, up1 = 2 * tq + 1 > g;
    const int src_row0 = 4 * (2 * tq) + (g != 0), src_row1 = 4 * (2 * tq + 1) + (g != 0);

    // One gradient step: acc <- V = L~ - tril(2 tau L~ T~) (kept lower-triangular);
    // returns V_NN.  MON: fterm += sum of L~_ik W_ik over this lane's elements, W = L~ T^.
    auto grad_step = [&](float& fterm) -> float {
      // V_NN partial from row N of L~(t-1) (lanes g == 0 hold it), FP32.
      uint64_t part2 = 0ull;
#pragma unroll
      for (int n = 0; n < NT; ++n) part2 = f2fma(f2pack(acc[MT - 1][n][0], acc[MT - 1][n][1]), tN2[n], part2);
      float part, part_hi;
      f2unpack(part2, part, part_hi);
      part += part_hi;
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 1);
      part += __shfl_xor_sync(TASER_FULL_MASK, part, 2);
      part = __shfl_sync(TASER_FULL_MASK, part, 0);

#pragma unroll
      for (int M = 0; M < MT; ++M) {
        // A operand of row block M from the FP32 master (old L~).  The last row block
        // holds row N only (its rows g + 8 are identically zero).
        uint32_t a[KT][4];
#pragma unroll
        for (int kt = 0; kt <= C::kmax(M); ++kt) {
          a[kt][0] = pack2<FP16>(acc[M][2 * kt][0], acc[M][2 * kt][1]);
          a[kt][2] = pack2<FP16>(acc[M][2 * kt + 1][0], acc[M][2 * kt + 1][1]);
          if (M < MT - 1) {
            a[kt][1] = pack2<FP16>(acc[M][2 * kt][2], acc[M][2 * kt][3]);
            a[kt][3] = pack2<FP16>(acc[M][2 * kt + 1][2], acc[M][2 * kt + 1][3]);
          } else {
            a[kt][1] = 0u;
            a[kt][3] = 0u;
          }
        }
        if constexpr (MON) {
          // W = L~ T^ of this row block as a BF16 split, dotted with L~ (the old values:
          // every tile's own mma comes later).  Row N: the transposed product T^ l_N^T, whose
          // columns are moved into the accumulator layout, plus L~_NN T^_{N,c} in FP32.
          uint32_t ah[KT][4], al[KT][4];
#pragma unroll
          for (int kt = 0; kt <= C::kmax(M); ++kt) {
            split_bf16(acc[M][2 * kt][0], acc[M][2 * kt][1], ah[kt][0], al[kt][0]);
            split_bf16(acc[M][2 * kt + 1][0], acc[M][2 * kt + 1][1], ah[kt][2], al[kt][2]);
            if (M < MT - 1) {
              split_bf16(acc[M][2 * kt][2], acc[M][2 * kt][3], ah[kt][1], al[kt][1]);
              split_bf16(acc[M][2 * kt + 1][2], acc[M][2 * kt + 1][3], ah[kt][3], al[kt][3]);
            } else {
              ah[kt][1] = ah[kt][3] = al[kt][1] = al[kt][3] = 0u;
            }
          }
          if (M < MT - 1) {
#pragma unroll
            for (int n = 0; n < NT; ++n) {
              if (!C::has_tile(M, n)) continue;
              float w4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
              for (int kt = 0; kt <= C::kmax(M); ++kt) {
                mma16816<false>(w4, ah[kt], mbh[kt][n]);
                mma16816<false>(w4, ah[kt], mbl[kt][n]);
                mma16816<false>(w4, al[kt], mbh[kt][n]);
              }
#pragma unroll
              for (int e = 0; e < 4; ++e) fterm = fmaf(acc[M][n][e], w4[e], fterm);
            }
          } else {
            float d[KT][4];
#pragma unroll
            for (int mt = 0; mt < KT; ++mt) {
#pragma unroll
              for (int e = 0; e < 4; ++e) d[mt][e] = 0.f;
#pragma unroll
              for (int kt = 0; kt < KT; ++kt) {
                const uint32_t th[4] = {mbh[kt][2 * mt][0], mbh[kt][2 * mt + 1][0], mbh[kt][2 * mt][1],
                                        mbh[kt][2 * mt + 1][1]};
                const uint32_t tl[4] = {mbl[kt][2 * mt][0], mbl[kt][2 * mt + 1][0], mbl[kt][2 * mt][1],
                                        mbl[kt][2 * mt + 1][1]};
                const uint32_t bh2[2] = {ah[kt][0], ah[kt][2]}, bl2[2] = {al[kt][0], al[kt][2]};
                mma16816<false>(d[mt], th, bh2);
                mma16816<false>(d[mt], tl, bh2);
                mma16816<false>(d[mt], th, bl2);
              }
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
              const float v0 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], src_row0);
              const float v1 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], src_row1);
              fterm = fmaf(acc[M][n][0], fmaf(LNN, tN2f(n, 0), v0), fterm);
              fterm = fmaf(acc[M][n][1], fmaf(LNN, tN2f(n, 1), v1), fterm);
            }
          }
        }
        if (M == MT - 1) {
          // k = N term of row N in FP32: L~_NN T^_{N,c}.
          const uint64_t lnn2 = f2pack(LNN, LNN);
#pragma unroll
          for (int n = 0; n < NT; ++n) TASER_PAIR_APPLY(acc[M][n], 0, f2fma(lnn2, tN2[n], _x));
        }
        if (M == MT - 1 && KT >= 2) {
          // Row N as the transposed product T^ L~_N^T (T^ symmetric): KT m-tiles of output
          // columns against KT k-tiles, KT^2 mma instead of the KT NT of a 16-row tile with
          // one live row (4 instead of 8 at NB = 32; at NB = 16 the saved mma costs more in
          // shuffles than it gains, measured).  The A fragments of T^ are the B fragments
          // already held; the B operand is the packed row N (column 0; rows g != 0 of the
          // row-N tile are zero).
          float d[KT][4];
#pragma unroll
          for (int mt = 0; mt < KT; ++mt) {
#pragma unroll
            for (int e = 0; e < 4; ++e) d[mt][e] = 0.f;
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) {
              const uint32_t at[4] = {bf[kt][2 * mt][0], bf[kt][2 * mt + 1][0], bf[kt][2 * mt][1],
                                      bf[kt][2 * mt + 1][1]};
              const uint32_t bt[2] = {a[kt][0], a[kt][2]};
              mma16816<FP16>(d[mt], at, bt);
            }
          }
          // Column c = 8n + 2tq + p of row N sits in D column 0 at lane 4 (c mod 8), element
          // 2 (n mod 2) of m-tile n / 2; lanes g != 0 read a lane with tq = 1 (D column 2,
          // zero), so their row-N tile stays zero.
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            const float v0 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], src_row0);
            const float v1 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], src_row1);
            TASER_PAIR_APPLY(acc[M][n], 0, f2fma(f2pack(1.f, 1.f), f2pack(v0, v1), _x));
          }
        } else {
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            if (!C::has_tile(M, n)) continue;
#pragma unroll
            for (int kt = 0; kt <= C::kmax(M); ++kt) {
              if (M == MT - 1) mma16816_top<FP16>(acc[M][n], a[kt], bf[kt][n]);
              else mma16816<FP16>(acc[M][n], a[kt], bf[kt][n]);
            }
          }
        }
      }
      // Keep V lower-triangular inside the diagonal blocks: the rows g of n-tile 2M + 1
      // are above the diagonal on every lane.
#pragma unroll
      for (int M = 0; M < MT - 1; ++M) {
        if (up0) acc[M][2 * M][0] = 0.f;
        if (up1) acc[M][2 * M][1] = 0.f;
        acc[M][2 * M + 1][0] = 0.f;
        acc[M][2 * M + 1][1] = 0.f;
        if (up0) acc[M][2 * M + 1][2] = 0.f;
        if (up1) acc[M][2 * M + 1][3] = 0.f;
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

      // prox: column sums of squares, reduced over the 8 lanes sharing tq.
      float s[C::NV];
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        uint64_t v2 = 0ull;
#pragma unroll
        for (int M = 0; M < MT; ++M) {
          if (!C::has_tile(M, n)) continue;
          if (!(M < MT - 1 && n == 2 * M + 1)) {   // rows g of n-tile 2M + 1 are zero
            const uint64_t x01 = f2pack(acc[M][n][0], acc[M][n][1]);
            v2 = f2fma(x01, x01, v2);
          }
          if (M < MT - 1) {
            const uint64_t x23 = f2pack(acc[M][n][2], acc[M][n][3]);
            v2 = f2fma(x23, x23, v2);
          }
        }
        f2unpack(v2, s[2 * n], s[2 * n + 1]);
      }
      // Transpose-reduce over lane bits 4, 3, 2 (each step halves the values a lane keeps),
      // then a shuffle broadcast of the scales.  (An exchange of the partials and scales
      // through shared memory was measured at bucket 32, together with the triangle
      // staging above: 4,890 instead of 4,182 warp instructions per instance, 0.440 instead
      // of 0.391 ms per 65,536; the FMA-pipe count rose by 18 per iteration, the register
      // moves that assemble the 16-byte stores and the addressing.)
      {
        int len = C::NV;
#pragma unroll
        for (int m = 16; m >= 4; m >>= 1) {
          const bool up = (lane & m) != 0;
          if (len > 1) {
            const int h = len >> 1;
#pragma unroll
            for (int i = 0; i < C::NV / 2; ++i) {
              if (i >= h) break;
              const float send = up ? s[i] : s[i + h];
              const float keep = up ? s[i + h] : s[i];
              s[i] = keep + __shfl_xor_sync(TASER_FULL_MASK, send, m);
            }
            len = h;
          } else {
            s[0] += __shfl_xor_sync(TASER_FULL_MASK, s[0], m);
          }
        }
      }
      float sc_own = 0.f;
      if (s[0] > 0.f) {
        sc_own = Down * rsqrtf(s[0]);
      } else if (cown < N - 1) {
        fl |= TASER_FLAG_ZERO_COLUMN;
      }
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        float sc[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int idx = 2 * n + p;
          sc[p] = __shfl_sync(TASER_FULL_MASK, sc_own, 4 * (NT == 4 ? idx : 2 * idx) + tq);
        }
        const uint64_t sc2 = f2pack(sc[0], sc[1]);
#pragma unroll
        for (int M = 0; M < MT; ++M) {
          if (!C::has_tile(M, n)) continue;
          if (!(M < MT - 1 && n == 2 * M + 1)) TASER_PAIR_APPLY(acc[M][n], 0, f2mul(_x, sc2));
          if (M < MT - 1) TASER_PAIR_APPLY(acc[M][n], 2, f2mul(_x, sc2));
        }
      }
    }

    const JobOut o = outs[cur_m];

    // Decisions from row N (lanes g == 0).
    if (g == 0) {
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int c = 8 * n + 2 * tq + p;
          if (c < N - 1 && TASER_IN(c, N - 1)) {
            float r = acc[MT - 1][n][p];
            TASER_FINITE(r);
            if (literal && LNN < 0.f) r = -r;
            o.s[c] = r >= 0.f ? int8_t(1) : int8_t(-1);
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
            if (M == MT - 1 && e >= 2) continue;
            const int r = 16 * M + g + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
            const int rr = bucket_to_real(r, N, NB);
            if (rr < 0 || c >= N - 1 || !TASER_IN(rr * N + c, N * N)) continue;
            Lo[(int64_t)rr * N + c] = C::has_tile(M, n) ? acc[M][n][e] : 0.f;
            TASER_FINITE(Lo[(int64_t)rr * N + c]);
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

template <int NB, bool FP16, class Src, bool MON = false>
static cudaError_t launch_tc_src(const Src& src, int64_t jobs, int blocks_per_sm, int literal, int slot_floats,
                                 float ascent_tol, cudaStream_t st) {
  using C = TcCfg<NB>;
  const size_t smem = (size_t)C::WARPS * (slot_floats + kTcRecFloats) * sizeof(float);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tc_kernel<NB, FP16, Src, MON>, 32 * C::WARPS,
                                                      smem);
  if (e != cudaSuccess) return e;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : (fit > 0 ? fit : 1);
  const int64_t need = (jobs + C::WARPS - 1) / C::WARPS;
  const int64_t resident = (int64_t)sms * per_sm;
  const int64_t blocks = jobs >= 0 && need < resident ? need : resident;
  detect_tc_kernel<NB, FP16, Src, MON><<<(unsigned)blocks, 32 * C::WARPS, smem, st>>>(src, literal, slot_floats,
                                                                                      ascent_tol);
  return cudaGetLastError();
}

template <int NB, bool FP16, bool MON = false>
static cudaError_t launch_tc(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                             int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st,
                             double* obj = nullptr, float ascent_tol = 0.f) {
  using C = TcCfg<NB>;
  const int slot_floats = tc_slot_floats(N);
  int dev = 0, sms = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, detect_tc_kernel<NB, FP16, DenseSource, MON>,
                                                      32 * C::WARPS,
                                                      (size_t)C::WARPS * (slot_floats + kTcRecFloats) * sizeof(float));
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

cudaError_t detect_tc64(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                        int literal, bool fp16, float* L, int8_t* s, uint32_t* flags, cudaStream_t st);
cudaError_t detect_tc64_queue(bool fp16, const Queue& q, int blocks_per_sm, const float* T_pool, const float* D_pool,
                              const float* tau, int literal, float* L_pool, int8_t* s_pool, uint32_t* flags,
                              cudaStream_t st);

// Returns cudaErrorNotSupported when the bucket has no tensor-core kernel.
cudaError_t detect_tc(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                      int literal, bool fp16, float* L, int8_t* s, uint32_t* flags, cudaStream_t st) {
  switch (bucket_of(N)) {
    case 64:
      return detect_tc64(batch, N, Tt, D, tau, t_max, literal, fp16, L, s, flags, st);
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
      return detect_tc64_queue(fp16, q, blocks_per_sm, T_pool, D_pool, tau, literal, L_pool, s_pool, flags, st);
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
