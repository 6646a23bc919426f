// Unfolded TASER on the tensor cores: Algorithm 1 with a learnable step per iteration,
// tau_t = alpha_t / ||T~||_2 (mode "fixed", L~_NN = D_NN), its forward with checkpoints
// and the hand-written adjoint, with the triangular products L~ T~ (forward) and
// Vbar T~ (adjoint) on mma.sync m16n8k16 with BF16 or FP16 operands and FP32
// accumulation.  The master iterates, the prox and its Jacobian stay FP32.  The same
// equations as the FP32 unfolded kernels (unfolded.cu):
//   V_t = L~(t-1) - tau_t tril(2 L~(t-1) T~),  L~(t) = prox(V_t),  soft x_k = L~_N,k / D_k;
//   adjoint of one step, given Lbar = dloss/dL~(t) and G = tril(2 L~(t-1) T~) = (L~ - V)/tau:
//     Vbar_.k = (D_k / ||V_.k||) (Lbar_.k - u_k (u_k . Lbar_.k)),  u_k = V_.k / ||V_.k||, k < N,
//     dloss/dtau_t = -<Vbar, G>,   dloss/dL~(t-1) = tril(Vbar - tau_t Vbar (2 T~)).
//
// Bucket 32 only (18 <= N <= 33, the tensor-core bucket of the detector); one warp per
// instance with L~ in the accumulator layout of the detector's tensor-core kernel.  The
// per-iteration step enters through the A operand: A = bf16(-2 tau_t L~), B = bf16(T~),
// C = L~, so one mma gives V.  Column reductions (norms, and the four column sums of the
// adjoint) meet in shared memory.  The adjoint recomputes each segment of c iterations
// from its checkpoint and keeps the iterates in shared memory in the lanes' own layout.
#include "mma_tc.cuh"

namespace taser {

namespace {

constexpr int kNB = 32;
using UTC = TcCfg<kNB>;
constexpr int kKT = UTC::KT, kNT = UTC::NT, kMT = UTC::MT;
// Live accumulator elements per lane: the 2 full row blocks (all n-tiles, zero where a
// tile lies above the diagonal) and the two live values of each row-N tile.
constexpr int kNE = (kMT - 1) * kNT * 4 + kNT * 2;   // 40
// Column-reduction scratch: for each of the 8 lanes g, NQ rows of 36 floats (the 8 column
// partials of lane (g, tq) at tq * 8 + (2n + p)), row groups g spaced by NQ * 36 (+ 4 for
// even NQ) floats so that a 16-byte store of every lane of a quarter-warp hits distinct
// banks; then 2 x 32 per-column scalars.
__host__ __device__ constexpr int kRedRows(int nq) { return nq * 36 + ((nq & 1) ? 0 : 4); }
constexpr int kRedFloats = 8 * kRedRows(4) + 64;
constexpr int kSlotFloats = ((33 * 33 + 33 + 1) + 3) & ~3;    // T~, D, spare (staging)

struct LaneGeom {
  int lane, g, tq;
  bool up0, up1;            // above the diagonal inside a diagonal block (rows g)
  int src_row0, src_row1;   // source lanes of the row-N columns of the transposed product
  int cown;                 // the column a lane owns after a reduction: 8(g/2) + 2tq + g%2
  __device__ LaneGeom(int l) : lane(l), g(l >> 2), tq(l & 3) {
    up0 = 2 * tq > g;
    up1 = 2 * tq + 1 > g;
    src_row0 = 4 * (2 * tq) + (g != 0);
    src_row1 = 4 * (2 * tq + 1) + (g != 0);
    cown = 8 * (g >> 1) + 2 * tq + (g & 1);
  }
};

using Acc = float[kMT][kNT][4];

// Flat index of a live element (M, n, e) in an iterate stored in the lanes' layout.
__device__ __forceinline__ constexpr int flat(int M, int n, int e) {
  return M < kMT - 1 ? (M * kNT + n) * 4 + e : (kMT - 1) * kNT * 4 + n * 2 + e;
}

// Stage the lower triangle of T~ (symmetric; N x N row-major places) and D into `slot`.
__device__ __forceinline__ void stage_T(float* slot, const float* T, const float* D, int N, int lane) {
  const int ntri = N * (N + 1) / 2;
  int i = 0, j = lane;
  while (j > i) {
    j -= i + 1;
    ++i;
  }
  for (int e = lane; e < ntri; e += 32) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(slot + i * N + j);
    TASER_CHECKED(TASER_IN(i * N + j, N * N) && TASER_IN(j, i + 1))
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(T + i * N + j) : "memory");
    j += 32;
    while (j > i) {
      j -= i + 1;
      ++i;
    }
  }
  for (int k = lane; k < N; k += 32) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(slot + N * N + k);
    TASER_CHECKED(TASER_IN(N * N + k, kSlotFloats))
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(D + k) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
}

// B fragments of T~ (unscaled) and row N of T~ at the lane's accumulator columns.
template <bool FP16>
__device__ __forceinline__ void load_B(const float* slot, int N, const LaneGeom& L, uint32_t (&bf)[kKT][kNT][2],
                                       uint64_t (&tN2)[kNT]) {
  auto tv = [&](int k, int n) -> float {
    const int hi = k >= n ? k : n, lo = k >= n ? n : k;
    return (k < N - 1 && n < N - 1) ? slot[hi * N + lo] : 0.f;
  };
#pragma unroll
  for (int kt = 0; kt < kKT; ++kt)
#pragma unroll
    for (int nt = 0; nt < kNT; ++nt) {
      const int k0 = 16 * kt + 2 * L.tq, n = 8 * nt + L.g;
      bf[kt][nt][0] = pack2<FP16>(tv(k0, n), tv(k0 + 1, n));
      bf[kt][nt][1] = pack2<FP16>(tv(k0 + 8, n), tv(k0 + 9, n));
    }
#pragma unroll
  for (int nt = 0; nt < kNT; ++nt) {
    float t2[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int c = 8 * nt + 2 * L.tq + p;
      t2[p] = (L.g == 0 && c < N - 1) ? slot[(N - 1) * N + c] : 0.f;
    }
    tN2[nt] = f2pack(t2[0], t2[1]);
  }
}

// X <- tril(X + s X T~) with the products in BF16/FP16 (A = s X, B = T~, C = X), X
// lower-triangular over the variable rows plus row N.  lnn is X_NN (its product with row
// N of T~ is added in FP32).  Row N runs as the transposed product T~ (s x_N)^T.
template <bool FP16>
__device__ __forceinline__ void tc_step(Acc& acc, const uint32_t (&bf)[kKT][kNT][2], const uint64_t (&tN2)[kNT],
                                        float s, float lnn, const LaneGeom& L) {
  const uint64_t s2 = f2pack(s, s);
#pragma unroll
  for (int M = 0; M < kMT; ++M) {
    uint32_t a[kKT][4];
#pragma unroll
    for (int kt = 0; kt <= UTC::kmax(M); ++kt) {
      float x0, x1, x2, x3;
      f2unpack(f2mul(f2pack(acc[M][2 * kt][0], acc[M][2 * kt][1]), s2), x0, x1);
      f2unpack(f2mul(f2pack(acc[M][2 * kt + 1][0], acc[M][2 * kt + 1][1]), s2), x2, x3);
      a[kt][0] = pack2<FP16>(x0, x1);
      a[kt][2] = pack2<FP16>(x2, x3);
      if (M < kMT - 1) {
        f2unpack(f2mul(f2pack(acc[M][2 * kt][2], acc[M][2 * kt][3]), s2), x0, x1);
        f2unpack(f2mul(f2pack(acc[M][2 * kt + 1][2], acc[M][2 * kt + 1][3]), s2), x2, x3);
        a[kt][1] = pack2<FP16>(x0, x1);
        a[kt][3] = pack2<FP16>(x2, x3);
      } else {
        a[kt][1] = 0u;
        a[kt][3] = 0u;
      }
    }
    if (M == kMT - 1) {
      const float sl = s * lnn;
      const uint64_t lnn2 = f2pack(sl, sl);
#pragma unroll
      for (int n = 0; n < kNT; ++n) TASER_PAIR_APPLY(acc[M][n], 0, f2fma(lnn2, tN2[n], _x));
      float d[kKT][4];
#pragma unroll
      for (int mt = 0; mt < kKT; ++mt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) d[mt][e] = 0.f;
#pragma unroll
        for (int kt = 0; kt < kKT; ++kt) {
          const uint32_t at[4] = {bf[kt][2 * mt][0], bf[kt][2 * mt + 1][0], bf[kt][2 * mt][1], bf[kt][2 * mt + 1][1]};
          const uint32_t bt[2] = {a[kt][0], a[kt][2]};
          mma16816<FP16>(d[mt], at, bt);
        }
      }
#pragma unroll
      for (int n = 0; n < kNT; ++n) {
        const float v0 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], L.src_row0);
        const float v1 = __shfl_sync(TASER_FULL_MASK, d[n >> 1][2 * (n & 1)], L.src_row1);
        TASER_PAIR_APPLY(acc[M][n], 0, f2fma(f2pack(1.f, 1.f), f2pack(v0, v1), _x));
      }
    } else {
#pragma unroll
      for (int n = 0; n < kNT; ++n) {
        if (!UTC::has_tile(M, n)) continue;
#pragma unroll
        for (int kt = 0; kt <= UTC::kmax(M); ++kt) mma16816<FP16>(acc[M][n], a[kt], bf[kt][n]);
      }
    }
  }
#pragma unroll
  for (int M = 0; M < kMT - 1; ++M) {
    if (L.up0) acc[M][2 * M][0] = 0.f;
    if (L.up1) acc[M][2 * M][1] = 0.f;
    acc[M][2 * M + 1][0] = 0.f;
    acc[M][2 * M + 1][1] = 0.f;
    if (L.up0) acc[M][2 * M + 1][2] = 0.f;
    if (L.up1) acc[M][2 * M + 1][3] = 0.f;
  }
}

// Calls f(M, n, e) for every live element of a lane (rows g of n-tile 2M + 1, always
// above the diagonal, are skipped).
template <class F>
__device__ __forceinline__ void for_live(F&& f) {
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n) {
      if (!UTC::has_tile(M, n)) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (M == kMT - 1 && e >= 2) continue;
        if (M < kMT - 1 && n == 2 * M + 1 && e < 2) continue;
        f(M, n, e);
      }
    }
}

// Column sums of NQ per-lane partial arrays (part[q][2n + p] for the lane's columns);
// returns the totals of the column the lane owns (L.cown).
template <int NQ>
__device__ __forceinline__ void col_reduce(float* red, const float (&part)[NQ][2 * kNT], float (&tot)[NQ],
                                           const LaneGeom& L) {
  constexpr int RS = kRedRows(NQ);
  float* w = red + L.g * RS + L.tq * 8;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    *reinterpret_cast<float4*>(w + q * 36) = make_float4(part[q][0], part[q][1], part[q][2], part[q][3]);
    *reinterpret_cast<float4*>(w + q * 36 + 4) = make_float4(part[q][4], part[q][5], part[q][6], part[q][7]);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float acc = red[q * 36 + L.tq * 8 + L.g];
#pragma unroll
    for (int r = 1; r < 8; ++r) acc += red[r * RS + q * 36 + L.tq * 8 + L.g];
    tot[q] = acc;
  }
  __syncwarp();
}

// Per-column scalars from their owner lanes to every lane holding that column: out[q][2n + p].
template <int NS>
__device__ __forceinline__ void col_bcast(float* sc, const float (&own)[NS], float (&out)[NS][2 * kNT],
                                          const LaneGeom& L) {
#pragma unroll
  for (int q = 0; q < NS; ++q) sc[q * 32 + L.tq * 8 + L.g] = own[q];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const float4 a = *reinterpret_cast<const float4*>(sc + q * 32 + L.tq * 8);
    const float4 b = *reinterpret_cast<const float4*>(sc + q * 32 + L.tq * 8 + 4);
    out[q][0] = a.x; out[q][1] = a.y; out[q][2] = a.z; out[q][3] = a.w;
    out[q][4] = b.x; out[q][5] = b.y; out[q][6] = b.z; out[q][7] = b.w;
  }
  __syncwarp();
}

// prox (Sec. III-C): every variable column rescaled to norm D_k (Down = D of L.cown).
__device__ __forceinline__ void tc_prox(Acc& acc, float* red, float Down, const LaneGeom& L) {
  float part[1][2 * kNT];
#pragma unroll
  for (int i = 0; i < 2 * kNT; ++i) part[0][i] = 0.f;
  for_live([&](int M, int n, int e) { part[0][2 * n + (e & 1)] = fmaf(acc[M][n][e], acc[M][n][e], part[0][2 * n + (e & 1)]); });
  float tot[1];
  col_reduce<1>(red, part, tot, L);
  float own[1] = {tot[0] > 0.f ? Down * rsqrtf(tot[0]) : 0.f};
  float sc[1][2 * kNT];
  col_bcast<1>(red + 8 * kRedRows(4), own, sc, L);
  for_live([&](int M, int n, int e) { acc[M][n][e] *= sc[0][2 * n + (e & 1)]; });
}

__device__ __forceinline__ void init_diag(Acc& acc, const float* Dsl, int N, const LaneGeom& L) {
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 16 * M + L.g + 8 * (e >> 1), c = 8 * n + 2 * L.tq + (e & 1);
        acc[M][n][e] = (M < kMT - 1 && r == c && r < N - 1) ? Dsl[r] : 0.f;
      }
}

// L~ in real indices, full N x N with zeros above the diagonal (the checkpoint layout).
__device__ __forceinline__ void store_full(float* out, const Acc& acc, int N, float LNN, const LaneGeom& L) {
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (M == kMT - 1 && e >= 2) continue;
        const int r = 16 * M + L.g + 8 * (e >> 1), c = 8 * n + 2 * L.tq + (e & 1);
        const int rr = bucket_to_real(r, N, kNB);
        if (rr < 0 || c >= N - 1) continue;
        const bool zero = !UTC::has_tile(M, n) || (M < kMT - 1 && n == 2 * M + 1 && e < 2);
        TASER_CHECKED(TASER_IN(rr * N + c, N * N)) out[(int64_t)rr * N + c] = zero ? 0.f : acc[M][n][e];
      }
  for (int rr = L.lane; rr < N; rr += 32) TASER_CHECKED(TASER_IN(rr * N + N - 1, N * N)) out[(int64_t)rr * N + (N - 1)] = rr == N - 1 ? LNN : 0.f;
}

__device__ __forceinline__ void load_full(const float* in, Acc& acc, int N, const LaneGeom& L) {
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 16 * M + L.g + 8 * (e >> 1), c = 8 * n + 2 * L.tq + (e & 1);
        const int rr = bucket_to_real(r, N, kNB);
        const bool live = UTC::has_tile(M, n) && !(M == kMT - 1 && e >= 2) &&
                          !(M < kMT - 1 && n == 2 * M + 1 && e < 2);
        acc[M][n][e] = (live && rr >= 0 && c < N - 1 TASER_AND(TASER_IN(rr * N + c, N * N))) ? in[(int64_t)rr * N + c] : 0.f;
      }
}

// Iterates of a segment in shared memory, in the lanes' own layout (10 x 16 bytes per lane).
__device__ __forceinline__ void put_iter(float* it, const Acc& acc, int lane) {
  float v[kNE];
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (!(M == kMT - 1 && e >= 2)) v[flat(M, n, e)] = acc[M][n][e];
#pragma unroll
  for (int q = 0; q < kNE / 4; ++q)
    *reinterpret_cast<float4*>(it + (q * 32 + lane) * 4) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void get_iter(const float* it, Acc& acc, int lane) {
  float v[kNE];
#pragma unroll
  for (int q = 0; q < kNE / 4; ++q) {
    const float4 x = *reinterpret_cast<const float4*>(it + (q * 32 + lane) * 4);
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[M][n][e] = (M == kMT - 1 && e >= 2) ? 0.f : v[flat(M, n, e)];
}

}  // namespace

template <bool FP16>
__global__ void __launch_bounds__(128, 4)
unfolded_tc_forward_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                           const float* __restrict__ inv_norm, const float* __restrict__ alpha_t, int t_max, int c,
                           float* __restrict__ ckpt, float* __restrict__ soft, int8_t* __restrict__ s_hat) {
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5;
  const LaneGeom L(threadIdx.x & 31);
  const int64_t inst = (int64_t)blockIdx.x * 4 + warp;
  if (inst >= batch) return;
  float* slot = smem + warp * (kSlotFloats + kRedFloats);
  float* red = slot + kSlotFloats;
  stage_T(slot, Tt + inst * (int64_t)N * N, Dg + inst * (int64_t)N, N, L.lane);
  uint32_t bf[kKT][kNT][2];
  uint64_t tN2[kNT];
  load_B<FP16>(slot, N, L, bf, tN2);
  const float* Dsl = slot + N * N;
  const float DN = Dsl[N - 1];
  const float Down = L.cown < N - 1 ? Dsl[L.cown] : 0.f;
  Acc acc;
  init_diag(acc, Dsl, N, L);
  float Drow[kNT][2];   // D of the row-N columns (lanes g == 0), for the soft output
#pragma unroll
  for (int n = 0; n < kNT; ++n)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int cc = 8 * n + 2 * L.tq + p;
      Drow[n][p] = cc < N - 1 ? Dsl[cc] : 0.f;
    }
  __syncwarp();
  const float inv = inv_norm[inst];
  const int n_ckpt = (t_max + c - 1) / c;
  for (int t = 0; t < t_max; ++t) {
    if (t % c == 0 && ckpt != nullptr TASER_AND(TASER_IN(inst * n_ckpt + t / c, batch * n_ckpt))) store_full(ckpt + (inst * n_ckpt + t / c) * (int64_t)N * N, acc, N, DN, L);
    tc_step<FP16>(acc, bf, tN2, -2.f * alpha_t[t] * inv, DN, L);
    tc_prox(acc, red, Down, L);
  }
  if (L.g == 0) {
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int cc = 8 * n + 2 * L.tq + p;
        if (cc < N - 1 TASER_AND(TASER_IN(inst * (N - 1) + cc, batch * (N - 1)))) {
          const float x = acc[kMT - 1][n][p];
          soft[inst * (N - 1) + cc] = Drow[n][p] > 0.f ? x / Drow[n][p] : 0.f;
          if (s_hat != nullptr) s_hat[inst * (N - 1) + cc] = x >= 0.f ? int8_t(1) : int8_t(-1);
        }
      }
  }
}

template <bool FP16>
__global__ void __launch_bounds__(32, 8)
unfolded_tc_backward_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                            const float* __restrict__ inv_norm, const float* __restrict__ alpha_t, int t_max, int c,
                            const float* __restrict__ ckpt, const float* __restrict__ grad_soft,
                            float* __restrict__ grad_tau) {
  extern __shared__ __align__(16) float smem[];
  const LaneGeom L(threadIdx.x & 31);
  const int64_t inst = blockIdx.x;
  if (inst >= batch) return;
  float* its = smem;                                  // c iterates of kNE x 32 floats
  float* red = smem + (size_t)c * kNE * 32;
  // T~ and D are staged in the iterate area before any iterate is written.
  stage_T(its, Tt + inst * (int64_t)N * N, Dg + inst * (int64_t)N, N, L.lane);
  uint32_t bf[kKT][kNT][2];
  uint64_t tN2[kNT];
  load_B<FP16>(its, N, L, bf, tN2);
  const float DN = its[N * N + N - 1];
  const float Down = L.cown < N - 1 ? its[N * N + L.cown] : 0.f;
  Acc lbar;
#pragma unroll
  for (int M = 0; M < kMT; ++M)
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) lbar[M][n][e] = 0.f;
  if (L.g == 0) {   // Lbar(t_max): the last row only, dloss/dL~_N,k = dloss/dx_k / D_k
#pragma unroll
    for (int n = 0; n < kNT; ++n)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int cc = 8 * n + 2 * L.tq + p;
        const float Dc = cc < N - 1 ? its[N * N + cc] : 0.f;
        lbar[kMT - 1][n][p] = Dc > 0.f TASER_AND(TASER_IN(inst * (N - 1) + cc, batch * (N - 1))) ? grad_soft[inst * (N - 1) + cc] / Dc : 0.f;
      }
  }
  // The adjoint is linear in Lbar, so it runs on Lbar 2^-e with e the exponent of the
  // instance's largest |Lbar| (exact), and dloss/dtau_t is scaled back by 2^e.  Loss
  // gradients of a mean over a batch are tiny (~1e-6 here), and s Vbar, the A operand of
  // the adjoint's product, would sink below FP16's normal range (6e-5) and lose its bits.
  float amax = 0.f;
#pragma unroll
  for (int n = 0; n < kNT; ++n) amax = fmaxf(amax, fmaxf(fabsf(lbar[kMT - 1][n][0]), fabsf(lbar[kMT - 1][n][1])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TASER_FULL_MASK, amax, o));
  int gexp = 0;
  if (amax > 0.f && isfinite(amax)) frexpf(amax, &gexp);
  gexp = max(-120, min(120, gexp));
  const float gdown = ldexpf(1.f, -gexp), gup = ldexpf(1.f, gexp);
#pragma unroll
  for (int n = 0; n < kNT; ++n) {
    lbar[kMT - 1][n][0] *= gdown;
    lbar[kMT - 1][n][1] *= gdown;
  }
  __syncwarp();   // the staged T~ and D are read before the iterates overwrite them
  const float inv = inv_norm[inst];
  const int n_ckpt = (t_max + c - 1) / c;
  for (int kc = n_ckpt - 1; kc >= 0; --kc) {
    const int t0 = kc * c, t1 = min(t0 + c, t_max);
    Acc acc;
    TASER_CHECKED(TASER_IN(inst * n_ckpt + kc, batch * n_ckpt)) load_full(ckpt + (inst * n_ckpt + kc) * (int64_t)N * N, acc, N, L);
    put_iter(its, acc, L.lane);
    for (int s = t0 + 1; s < t1; ++s) {   // recompute L~(t0+1) .. L~(t1-1)
      tc_step<FP16>(acc, bf, tN2, -2.f * alpha_t[s - 1] * inv, DN, L);
      tc_prox(acc, red, Down, L);
      TASER_CHECKED(TASER_IN(s - t0, c)) put_iter(its + (size_t)(s - t0) * kNE * 32, acc, L.lane);
    }
    for (int s = t1; s > t0; --s) {       // step s maps L~(s-1) -> L~(s) with tau_s
      const float tau = alpha_t[s - 1] * inv;
      Acc lp, v;
      TASER_CHECKED(TASER_IN(s - 1 - t0, c)) get_iter(its + (size_t)(s - 1 - t0) * kNE * 32, lp, L.lane);
#pragma unroll
      for (int M = 0; M < kMT; ++M)
#pragma unroll
        for (int n = 0; n < kNT; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) v[M][n][e] = lp[M][n][e];
      tc_step<FP16>(v, bf, tN2, -2.f * tau, DN, L);
      // Column sums: ||V||^2, V.Lbar, Lbar.L~, V.L~ (G = (L~ - V) / tau).
      float part[4][2 * kNT];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 2 * kNT; ++i) part[q][i] = 0.f;
      for_live([&](int M, int n, int e) {
        const int i = 2 * n + (e & 1);
        const float x = v[M][n][e], b = lbar[M][n][e], l = lp[M][n][e];
        part[0][i] = fmaf(x, x, part[0][i]);
        part[1][i] = fmaf(x, b, part[1][i]);
        part[2][i] = fmaf(b, l, part[2][i]);
        part[3][i] = fmaf(x, l, part[3][i]);
      });
      float tot[4];
      col_reduce<4>(red, part, tot, L);
      const bool col = L.cown < N - 1 && tot[0] > 0.f;
      const float rn = col ? rsqrtf(tot[0]) : 0.f;
      const float proj = rn * tot[1];
      const float fa = Down * rn;                     // Vbar = fa Lbar - fb V on this column
      const float fb = fa * rn * proj;
      const float tb = (fa * (tot[2] - tot[1]) - fb * (tot[3] - tot[0])) / tau;   // <Vbar, G>
      const float taubar = -warp_sum(tb) * gup;
      if (L.lane == 0 TASER_AND(TASER_IN(inst * t_max + (s - 1), batch * t_max))) grad_tau[inst * t_max + (s - 1)] = taubar;
      float own[2] = {fa, fb};
      float ab[2][2 * kNT];
      col_bcast<2>(red + 8 * kRedRows(4), own, ab, L);
      for_live([&](int M, int n, int e) {
        const int i = 2 * n + (e & 1);
        lbar[M][n][e] = fmaf(ab[0][i], lbar[M][n][e], -ab[1][i] * v[M][n][e]);
      });
      // Lbar(s-1) = tril(Vbar - 2 tau Vbar T~); column N of Vbar is zero (L~_NN is fixed).
      tc_step<FP16>(lbar, bf, tN2, -2.f * tau, 0.f, L);
    }
  }
}

// Shared memory of the tensor-core adjoint for checkpoint spacing c (bytes).
size_t unfolded_tc_backward_smem(int c) {
  const size_t its = (size_t)c * kNE * 32;
  return ((its > (size_t)kSlotFloats ? its : (size_t)kSlotFloats) + kRedFloats) * sizeof(float);
}

cudaError_t unfolded_tc(bool backward, bool fp16, int64_t batch, int N, const float* Tt, const float* D,
                        const float* inv_norm, const float* alpha_t, int t_max, int c, float* ckpt, float* soft,
                        int8_t* s_hat, const float* grad_soft, float* grad_tau, cudaStream_t st) {
  if (bucket_of(N) != kNB) return cudaErrorNotSupported;
  if (!backward) {
    const size_t smem = 4 * (size_t)(kSlotFloats + kRedFloats) * sizeof(float);
    const int64_t blocks = (batch + 3) / 4;
    if (fp16) {
      unfolded_tc_forward_kernel<true><<<(unsigned)blocks, 128, smem, st>>>(batch, N, Tt, D, inv_norm, alpha_t,
                                                                            t_max, c, ckpt, soft, s_hat);
    } else {
      unfolded_tc_forward_kernel<false><<<(unsigned)blocks, 128, smem, st>>>(batch, N, Tt, D, inv_norm, alpha_t,
                                                                             t_max, c, ckpt, soft, s_hat);
    }
    return cudaGetLastError();
  }
  const size_t smem = unfolded_tc_backward_smem(c);
  cudaError_t e = fp16 ? cudaFuncSetAttribute(unfolded_tc_backward_kernel<true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                       : cudaFuncSetAttribute(unfolded_tc_backward_kernel<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (fp16) {
    unfolded_tc_backward_kernel<true><<<(unsigned)batch, 32, smem, st>>>(batch, N, Tt, D, inv_norm, alpha_t, t_max,
                                                                         c, ckpt, grad_soft, grad_tau);
  } else {
    unfolded_tc_backward_kernel<false><<<(unsigned)batch, 32, smem, st>>>(batch, N, Tt, D, inv_norm, alpha_t, t_max,
                                                                          c, ckpt, grad_soft, grad_tau);
  }
  return cudaGetLastError();
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(unfolded_tc)
