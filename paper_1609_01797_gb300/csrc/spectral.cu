// ||T~||_2 and the step size tau = alpha / ||T~||_2 (Sec. III-B; inputs of Algorithm 1).
//
// ||T~||_2 of a symmetric matrix is its largest |eigenvalue|.  A power iteration is not
// used: on MU-MIMO matrices the two largest eigenvalues are often close and hundreds of
// steps still leave errors of 1e-3.  Instead each T~ is reduced to tridiagonal form with
// Householder reflections (FP32, backward stable), and the extreme eigenvalues of the
// tridiagonal matrix are found by Sturm-count multisection.  When T~ is known to be
// semidefinite (MU-MIMO: T = A^T A; JED: T = -A^T A) only that end is searched; otherwise
// lambda_max(T~) and lambda_max(-T~) are bracketed side by side.
//
// Layout: T~ is embedded in an (NV+1) x (NV+1) matrix with zero padding (zero rows and
// columns add zero eigenvalues, which do not change ||T~||_2 since ||T~||_2 >= 0).  The
// first reflection eliminates column 0, leaving an NV x NV trailing matrix whose columns
// 1..NV live in lane registers:
//  - spectral_fold_kernel (real, NV <= 32) and spectral_herm_fold_kernel (QPSK complex
//    form, NV <= 16): NV / 2 lanes per instance, two columns per lane (c and NV + 1 - c),
//    several instances per warp;
//  - spectral_kernel (real, NV = 64) and spectral_herm_kernel (complex, NV = 32): one warp
//    per instance, column c in lane (c - 1) mod 32.
#include <type_traits>

#include "common.cuh"

namespace taser {

template <int NV>
struct SpecCfg {
  static constexpr int S = NV > 32 ? NV / 32 : 1;  // columns per lane
  static constexpr int NP = NV + 1;                // padded order
  static constexpr int VB = ((NP + 3) / 4) * 4;    // padded vector length (16B rows)
  static constexpr int WARPS = 4;
  static constexpr int WARP_FLOATS = 2 * VB + 2 * VB;  // x, w, d, e
};

// Householder steps per compiled block: the real kernel's steps are longer, the complex
// one's shorter (measured: 2 beats 1, whose fully unrolled body misses the instruction
// cache, and 4).
constexpr int KBLK = 4;
constexpr int KBLK_HERM = 2;

// Calls f(std::integral_constant<int, KB>) for KB = 0, BLK, 2 BLK, ... < NV - 1.
template <int NV, int BLK, int KB = 0, typename F>
__device__ __forceinline__ void static_for_blocks(F&& f) {
  if constexpr (KB < NV - 1) {
    f(std::integral_constant<int, KB>{});
    static_for_blocks<NV, BLK, KB + BLK>(f);
  }
}

// Exponent e with 2^e <= m < 2^(e+1), clamped to [-126, 126] (0 for zero or non-finite m):
// the matrix is scaled by 2^-e (exact, both factors normal floats) so its largest entry
// lies in [1, 4) and tiny reflector norms are judged against that scale; ||T~|| is scaled
// back by 2^e.
__device__ __forceinline__ int scale_exponent(float m) {
  if (!(m > 0.f) || !(m <= 3.0e38f)) return 0;
  const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// An int known at compile time, usable where a runtime int is expected.
template <int V>
struct SpecInt {
  __host__ __device__ constexpr operator int() const { return V; }
};

// Below this squared norm (relative to the scaled matrix, largest entry about 1) the
// column is already eliminated: the rest is rounding residue far under FP32's resolution.
constexpr float kTinyNorm2 = 0x1p-100f;

// Sturm count: number of eigenvalues of the tridiagonal (sg*d, e) below sigma, as the
// number of negative pivots q_j of the LDL^T factorisation of (sg*T - sigma I).  No pivot
// guard sits in the recurrence: IEEE infinities carry a zero pivot through (Demmel, Dhillon
// and Ren, 1995).  A pivot +0 yields -inf next (counted), -0 yields +inf, and the pivot
// after an infinite one is finite again.  This needs e2 > 0 throughout (0 * inf would be a
// NaN), so callers floor the squared off-diagonals at kTinyNorm2.  The count reads the sign
// bit, so -0 counts as negative and +0 does not, matching the infinities they produce.
template <int NP>
__device__ __forceinline__ int sturm_count(const float (&d)[NP], const float (&e2)[NP], float sg, float sigma) {
  float q = sg * d[0] - sigma;
  int cnt = (int)(__float_as_uint(q) >> 31);
#pragma unroll
  for (int j = 1; j < NP; ++j) {
    q = (sg * d[j] - sigma) - __fdividef(e2[j - 1], q);
    cnt += (int)(__float_as_uint(q) >> 31);
  }
  return cnt;
}

// sign_hint: +1 -> T~ is positive semidefinite (||T~|| = lambda_max), -1 -> negative
// semidefinite (||T~|| = lambda_max(-T~)), 0 -> unknown (both ends are searched).
template <int NV>
__global__ void __launch_bounds__(128)
spectral_kernel(int64_t batch, int N, const float* __restrict__ Tt, float alpha, int sign_hint,
                float* __restrict__ tau, float* __restrict__ nrm_out) {
  using C = SpecCfg<NV>;
  constexpr int S = C::S, NP = C::NP, VB = C::VB;
  __shared__ __align__(16) float sm[C::WARPS * C::WARP_FLOATS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp;
  if (inst >= batch) return;
  float* xb = sm + warp * C::WARP_FLOATS;
  float* wb = xb + VB;
  float* db = wb + VB;
  float* eb = db + VB;

  const float* T = Tt + inst * (int64_t)N * N;
  // col[s][r] = A[r][c_s], c_s = lane + 1 + 32 s.
  float col[S][NP];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int c = lane + 1 + 32 * s;
#pragma unroll
    for (int r = 0; r < NP; ++r)
      col[s][r] = (r < N && c < N && TASER_IN(inst * N * N + r * N + c, batch * N * N)) ? T[(int64_t)r * N + c]
                                                                                        : 0.f;
  }
  float d0 = TASER_IN(inst * N * N, batch * N * N) ? T[0] : 0.f;
  float amax = fabsf(d0);
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int r = 0; r < NP; ++r) amax = fmaxf(amax, fabsf(col[s][r]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TASER_FULL_MASK, amax, o));
  const int ex = scale_exponent(amax);
  {
    const float sc = pow2f(-ex);
    d0 *= sc;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int r = 0; r < NP; ++r) col[s][r] *= sc;
  }
  for (int i = lane; i < VB; i += 32) {
    xb[i] = 0.f;
    wb[i] = 0.f;
  }
  __syncwarp();

  // Householder steps k = 0 .. NV-2 in blocks of KBLK: each block body is compiled once
  // with its trailing range starting at KB + 1 (entries j <= k inside the block are zero
  // in the published vector), which keeps the code inside the instruction cache.  Row k of
  // the lane's columns is picked by a short select chain over the block's rows.
  if (lane == 0) db[0] = d0;
  static_for_blocks<NV, KBLK>([&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    constexpr int KE = (KB + KBLK < NV - 1) ? KB + KBLK : NV - 1;   // k in [KB, KE)
#pragma unroll 1
    for (int k = KB; k < KE; ++k) {
      // x = column k below the diagonal: x_c = A[c][k] = A[k][c] sits in the owner of column
      // c.  The reflector H = I - beta v v^T with v = x - ah e_{k+1}, ah = -sign(x_{k+1}) ||x||,
      // maps x to ah e_{k+1}; v is published (zero for rows <= k).
      float ck[S];
      float sig2 = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int c = lane + 1 + 32 * s;
        float v = 0.f;
#pragma unroll
        for (int r = KB; r < KE; ++r) v = (r == k) ? col[s][r] : v;
        ck[s] = v;
        if (c > k && c <= NV) sig2 = fmaf(v, v, sig2);
      }
      sig2 = warp_sum(sig2);
      // x_{k+1} from the owner of column k + 1 (lane k mod 32, column slot k / 32).
      float xs = ck[0];
#pragma unroll
      for (int s = 1; s < S; ++s) xs = (k / 32 == s) ? ck[s] : xs;
      const float x1 = __shfl_sync(TASER_FULL_MASK, xs, k & 31);
      // Reflector scalars from a reciprocal square root (a few ulp; the reflection stays
      // orthogonal to that order, below the FP32 rounding of the updates).  A column with
      // ||x||^2 under kTinyNorm2 is left as it is (beta = 0).
      const bool refl = sig2 >= kTinyNorm2;
      const float sig = refl ? sig2 * rsqrtf(sig2) : 0.f;
      const float ah = x1 >= 0.f ? -sig : sig;             // new subdiagonal entry
      const float vv2 = 2.f * (sig2 + sig * fabsf(x1));    // ||v||^2
      const float beta = refl ? __fdividef(2.f, vv2) : 0.f;
      float vi[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int c = lane + 1 + 32 * s;
        const bool live = c > k && c <= NV;
        vi[s] = live ? (c == k + 1 ? ck[s] - ah : ck[s]) : 0.f;
        if (c <= NV && TASER_IN(c, VB)) xb[c] = vi[s];
        if (c == k && TASER_IN(k, VB)) db[k] = ck[s];
      }
      __syncwarp();
      float x[VB];
#pragma unroll
      for (int j4 = (KB + 1) & ~3; j4 < VB; j4 += 4) {
        const float4 q = *reinterpret_cast<const float4*>(xb + j4);
        x[j4] = q.x; x[j4 + 1] = q.y; x[j4 + 2] = q.z; x[j4 + 3] = q.w;
      }
      // p_i = beta sum_j A[j][i] v_j for this lane's columns i > k.
      float p[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        float acc = 0.f;
#pragma unroll
        for (int j = KB + 1; j < NP; ++j) acc = fmaf(col[s][j], x[j], acc);
        const int c = lane + 1 + 32 * s;
        p[s] = (c > k && c <= NV) ? beta * acc : 0.f;
      }
      float kk = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) kk = fmaf(vi[s], p[s], kk);
      kk = 0.5f * beta * warp_sum(kk);
      float w[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int c = lane + 1 + 32 * s;
        w[s] = fmaf(-kk, vi[s], p[s]);
        if (c <= NV && TASER_IN(c, VB)) wb[c] = w[s];
      }
      if (lane == 0 && TASER_IN(k, VB)) eb[k] = ah;
      __syncwarp();
      float wv[VB];
#pragma unroll
      for (int j4 = (KB + 1) & ~3; j4 < VB; j4 += 4) {
        const float4 q = *reinterpret_cast<const float4*>(wb + j4);
        wv[j4] = q.x; wv[j4 + 1] = q.y; wv[j4 + 2] = q.z; wv[j4 + 3] = q.w;
      }
      // A <- A - v w^T - w v^T on the trailing block.
#pragma unroll
      for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int j = KB + 1; j < NP; ++j) col[s][j] = fmaf(-x[j], w[s], fmaf(-wv[j], vi[s], col[s][j]));
      }
      __syncwarp();
    }
  });
  // Trailing 2 x 2 block: d_{NV-1}, e_{NV-1}, d_NV.
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int c = lane + 1 + 32 * s;
    if (c == NV - 1) {
      db[NV - 1] = col[s][NV - 1];
      eb[NV - 1] = col[s][NV];
    }
    if (c == NV) db[NV] = col[s][NV];
  }
  __syncwarp();
  float d[NP], e2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d[j] = db[j];
    e2[j] = j < NV ? eb[j] * eb[j] : 0.f;
  }

  // Sturm multisection.  Two-sided (hint 0): lanes 0..15 bracket lambda_max(A), lanes
  // 16..31 lambda_max(-A), 17 parts per round.  One-sided: all lanes, 33 parts.
  const bool two = sign_hint == 0;
  const float sg = two ? (lane < 16 ? 1.f : -1.f) : (sign_hint > 0 ? 1.f : -1.f);
  const int l = two ? (lane & 15) : lane;
  const int parts = two ? 17 : 33;
  const int rounds = two ? 7 : 5;   // 17^7 > 4e8, 33^5 > 3.9e7
  float lo = -3.0e38f, hi = -3.0e38f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float dj = sg * d[j];
    const float r = (j > 0 ? sqrtf(e2[j - 1]) : 0.f) + sqrtf(e2[j]);
    lo = fmaxf(lo, dj);
    hi = fmaxf(hi, dj + r);
  }
  // The Sturm count needs e2 > 0; the floor comes after the bracket, which it must not
  // widen (the zero matrix keeps the norm 0).
#pragma unroll
  for (int j = 0; j < NP; ++j) e2[j] = fmaxf(e2[j], kTinyNorm2);
  const float inv_parts = 1.f / (float)parts;
#pragma unroll 1
  for (int round = 0; round < rounds; ++round) {
    const float step = (hi - lo) * inv_parts;
    const float sigma = fmaf(step, (float)(l + 1), lo);
    const int cnt = sturm_count<NP>(d, e2, sg, sigma);
    const unsigned ball = __ballot_sync(TASER_FULL_MASK, cnt == NP);
    const unsigned half = two ? (lane < 16 ? (ball & 0xffffu) : (ball >> 16)) : ball;
    if (half == 0u) {
      lo = fmaf(step, (float)(parts - 1), lo);
    } else {
      const int f = __ffs(half) - 1;
      const float nhi = fmaf(step, (float)(f + 1), lo);
      const float nlo = f == 0 ? lo : fmaf(step, (float)f, lo);
      lo = nlo;
      hi = nhi;
    }
  }
  float nrm = 0.5f * (lo + hi);
  if (two) nrm = fmaxf(nrm, __shfl_xor_sync(TASER_FULL_MASK, nrm, 16));
  nrm *= pow2f(ex);
  if (lane == 0 && TASER_IN(inst, batch)) {
    tau[inst] = nrm > 0.f ? alpha / nrm : 0.f;
    if (nrm_out != nullptr) nrm_out[inst] = nrm;
    TASER_FINITE(nrm);
  }
}

// ---------------------------------------------------------------------------------
// QPSK: ||T~||_2 from the complex Hermitian form.
//
// For QPSK, T~ (N = 2U + 1) is the real form [[Re M, -Im M], [Im M, Re M]] of the
// preconditioned complex Gram M~ of [H / sqrt2, -y] ((U+1) x (U+1), Hermitian) with the
// row and column of the imaginary part of the augmented coordinate deleted.  Every
// eigenvalue of M~ appears twice in its real form, so by Cauchy interlacing the largest
// and smallest eigenvalues of T~ are those of M~, and ||T~||_2 = ||M~||_2.  M~ is read
// from T~:  M~_ab = T~_ab + i T~_{U+a,b},  M~_{a,N} = T~_{a,2U} + i T~_{U+a,2U}.
// Tridiagonalising the (U+1) complex matrix costs about 2.5x fewer flops and half the
// sequential steps of the real (2U+1) one.  The one-column layout below (one lane per
// trailing column) serves UV = 32; UV = 8 and 16 use the folded layout further down (two
// columns per lane).
// ---------------------------------------------------------------------------------
template <int UV>
struct HermCfg {
  static constexpr int G = UV;                 // lanes per instance (columns 1..UV)
  static constexpr int IPW = 32 / UV;          // instances per warp
  static constexpr int NP = UV + 1;            // padded complex order; aug at index UV
  static constexpr int VB = (NP + 1) & ~1;     // complex vector length (16B pairs)
  static constexpr int WARPS = 4;
  static constexpr int IPC = WARPS * IPW;
  static constexpr int INST_FLOATS = 8 * VB + 2 * VB;  // xd, wd ({re, re, im, im}), db, eb2
  // Multisection rounds: the bracket shrinks by (UV + 1)^ROUNDS.  For positive semidefinite
  // M~ the initial bracket is at most 2 lambda_max wide (|e_j| <= max d), so UV = 16 with 5
  // rounds (17^5 = 1.4e6) leaves at most 7e-7 relative, about the Householder error (measured
  // 7.2e-7 at most against FP64 over 65,536 QPSK 128x16 matrices).
  static constexpr int ROUNDS = UV == 32 ? 5 : (UV == 16 ? 5 : 8);
};

__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

// The complex multiply-adds of the reduction and of the rank-2 update run as packed f32x2
// operations (common.cuh) on {re, im} against duplicated pairs {v, v} read from shared
// memory.
template <int UV, bool NEG>
__global__ void __launch_bounds__(128)
spectral_herm_kernel(int64_t batch, int U, const float* __restrict__ Tt, float alpha, float* __restrict__ tau,
                     float* __restrict__ nrm_out) {
  using C = HermCfg<UV>;
  constexpr int NP = C::NP, VB = C::VB, G = C::G;
  __shared__ __align__(16) float sm[C::IPC * C::INST_FLOATS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int local = warp * C::IPW + grp;
  const int64_t inst = (int64_t)blockIdx.x * C::IPC + local;
  const bool active = inst < batch;
  // x and w of the current reflection as duplicated pairs {re, re, im, im} (one LDS.128
  // gives both pair operands of a complex multiply-add).
  float4* xd = reinterpret_cast<float4*>(sm + local * C::INST_FLOATS);
  float4* wd = xd + VB;
  float* db = reinterpret_cast<float*>(wd + VB);
  float* eb2 = db + VB;
  // col[j] = M~[j][c], c = gl + 1; index UV is the augmented coordinate.  A problem that
  // fills the bucket (U = UV, e.g. QPSK 128x16) reads with compile-time sizes (addresses
  // are a base plus immediates).
  const int c = gl + 1;
  float2 col[NP];
  float m00 = 0.f;
  auto load = [&](auto u_c) {
    const int Uc = u_c, N = 2 * Uc + 1;
    const float* T = Tt + (active ? inst : 0) * (int64_t)N * N;
    // NEG reads the negative semidefinite JED form as its (positive semidefinite) negation;
    // the norm is the same.
    auto t = [&](int a, int b) -> float {
      const float v = active && TASER_IN(inst * N * N + a * N + b, batch * N * N) ? T[a * N + b] : 0.f;
      return NEG ? -v : v;
    };
    const bool cu = c < UV && c < Uc, ca = c == UV;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const bool ju = j < UV && j < Uc, ja = j == UV;
      float2 v = make_float2(0.f, 0.f);
      if (ju && cu) v = make_float2(t(j, c), t(Uc + j, c));
      else if (ju && ca) v = make_float2(t(j, 2 * Uc), t(Uc + j, 2 * Uc));
      else if (ja && cu) v = make_float2(t(c, 2 * Uc), -t(Uc + c, 2 * Uc));
      else if (ja && ca) v = make_float2(t(2 * Uc, 2 * Uc), 0.f);
      col[j] = v;
    }
    m00 = Uc >= 1 ? t(0, 0) : 0.f;
  };
  if (U == UV) load(SpecInt<UV>{});
  else load(U);
  float amax = fabsf(m00);
#pragma unroll
  for (int j = 0; j < NP; ++j) amax = fmaxf(amax, fmaxf(fabsf(col[j].x), fabsf(col[j].y)));
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TASER_FULL_MASK, amax, o));
  const int ex = scale_exponent(amax);
  {
    const float sc = pow2f(-ex);
    m00 *= sc;
#pragma unroll
    for (int j = 0; j < NP; ++j) col[j] = make_float2(col[j].x * sc, col[j].y * sc);
  }
  for (int i = gl; i < VB; i += G) {
    xd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    wd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (gl == 0) db[0] = m00;
  __syncwarp();

  static_for_blocks<UV, KBLK_HERM>([&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    constexpr int KE = (KB + KBLK_HERM < UV - 1) ? KB + KBLK_HERM : UV - 1;   // k in [KB, KE)
#pragma unroll 1
    for (int k = KB; k < KE; ++k) {
      // x = column k below the diagonal: lane c holds x_c = M[c][k] = conj(M[k][c]) in its
      // own column.  The reflector H = I - beta v v^H with v = x - alpha e_{k+1},
      // alpha = -e^{i theta} sigma (theta = arg x_{k+1}, sigma = ||x||) maps x to alpha e_{k+1}.
      float2 ck = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = KB; r < KE; ++r) ck = (r == k) ? col[r] : ck;
      const bool live = c > k;
      const float2 xc = make_float2(ck.x, -ck.y);
      float sig2 = live ? fmaf(ck.x, ck.x, ck.y * ck.y) : 0.f;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sig2 += __shfl_xor_sync(TASER_FULL_MASK, sig2, o);
      const int src = grp * G + k;                                   // lane of column k + 1
      const float2 x1 = make_float2(__shfl_sync(TASER_FULL_MASK, xc.x, src), __shfl_sync(TASER_FULL_MASK, xc.y, src));
      // Reflector scalars from reciprocal square roots (a few ulp; the reflection stays
      // orthogonal to that order, below the FP32 rounding of the updates).  A column with
      // ||x||^2 under kTinyNorm2 is left as it is (beta = 0); an x_{k+1} that small takes
      // the phase 1, and ||v||^2 then uses Re(conj(e^{i theta}) x_{k+1}) = Re x_{k+1}.
      const bool refl = sig2 >= kTinyNorm2;
      const float sig = refl ? sig2 * rsqrtf(sig2) : 0.f;
      const float n1 = fmaf(x1.x, x1.x, x1.y * x1.y);
      const bool big1 = n1 >= kTinyNorm2;
      const float r1 = big1 ? rsqrtf(n1) : 0.f;
      const float2 ph = big1 ? make_float2(x1.x * r1, x1.y * r1) : make_float2(1.f, 0.f);
      const float ax1 = big1 ? n1 * r1 : x1.x;                                   // Re(conj(ph) x_{k+1})
      const float2 v1 = make_float2(fmaf(ph.x, sig, x1.x), fmaf(ph.y, sig, x1.y));   // x_{k+1} - alpha
      const float vv2 = 2.f * sig * (sig + ax1);                                 // ||v||^2
      const float beta = refl ? __fdividef(2.f, vv2) : 0.f;
      // Publish v (zero for rows <= k) as duplicated pairs.
      const float2 vc = live ? (c == k + 1 ? v1 : xc) : make_float2(0.f, 0.f);
      if (TASER_IN(c, VB)) xd[c] = make_float4(vc.x, vc.x, vc.y, vc.y);
      if (c == k && TASER_IN(k, VB)) db[k] = ck.x;
      __syncwarp();
      // p_c = beta sum_j conj(M[j][c]) v_j in one pass over j:
      //   A = sum {Re M, Im M} {Re v, Re v},  Bs = sum {Re M, Im M} {Im v, Im v},
      //   conj(M) v = (A.re + Bs.im, Bs.re - A.im).
      uint64_t A = 0ull, Bs = 0ull;
#pragma unroll
      for (int j = KB + 1; j < NP; ++j) {
        const float4 q = xd[j];
        const uint64_t X1 = f2pack(q.x, q.y), X2 = f2pack(q.z, q.w);
        const uint64_t Mj = f2pack(col[j].x, col[j].y);
        A = f2fma(Mj, X1, A);
        Bs = f2fma(Mj, X2, Bs);
      }
      float ax, ay, bx, by;
      f2unpack(A, ax, ay);
      f2unpack(Bs, bx, by);
      const float2 p = live ? make_float2(beta * (ax + by), beta * (bx - ay)) : make_float2(0.f, 0.f);
      float kk = fmaf(vc.x, p.x, vc.y * p.y);                       // Re(conj(v_c) p_c)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) kk += __shfl_xor_sync(TASER_FULL_MASK, kk, o);
      kk *= 0.5f * beta;
      const float2 w = make_float2(fmaf(-kk, vc.x, p.x), fmaf(-kk, vc.y, p.y));
      if (TASER_IN(c, VB)) wd[c] = make_float4(w.x, w.x, w.y, w.y);
      if (c == k + 1 && TASER_IN(k, VB)) eb2[k] = sig2;                               // |alpha|^2
      __syncwarp();
      // M[j][c] -= v_j conj(w_c) + w_j conj(v_c), as four pair FMAs per row:
      //   v conj(w) = {Re v, Re v}{Re w, -Im w} + {Im v, Im v}{Im w, Re w}.
      const uint64_t nWa = f2pack(-w.x, w.y), nWb = f2pack(-w.y, -w.x);
      const uint64_t nVa = f2pack(-vc.x, vc.y), nVb = f2pack(-vc.y, -vc.x);
#pragma unroll
      for (int j = KB + 1; j < NP; ++j) {
        const float4 q = xd[j], u = wd[j];
        uint64_t Mj = f2pack(col[j].x, col[j].y);
        Mj = f2fma(f2pack(q.x, q.y), nWa, Mj);
        Mj = f2fma(f2pack(q.z, q.w), nWb, Mj);
        Mj = f2fma(f2pack(u.x, u.y), nVa, Mj);
        Mj = f2fma(f2pack(u.z, u.w), nVb, Mj);
        f2unpack(Mj, col[j].x, col[j].y);
      }
      __syncwarp();
    }
  });
  // Trailing 2 x 2 block.
  if (c == UV - 1) {
    db[UV - 1] = col[UV - 1].x;
    eb2[UV - 1] = fmaf(col[UV].x, col[UV].x, col[UV].y * col[UV].y);
  }
  if (c == UV) db[UV] = col[UV].x;
  __syncwarp();
  float d[NP], e2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d[j] = db[j];
    e2[j] = j < UV ? eb2[j] : 0.f;
  }
  // One-sided multisection for lambda_max (M~ is positive semidefinite), G + 1 parts.
  float lo = -3.0e38f, hi = -3.0e38f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float r = (j > 0 ? sqrtf(e2[j - 1]) : 0.f) + sqrtf(e2[j]);
    lo = fmaxf(lo, d[j]);
    hi = fmaxf(hi, d[j] + r);
  }
  // The Sturm count needs e2 > 0; the floor comes after the bracket, which it must not
  // widen (the zero matrix keeps the norm 0).
#pragma unroll
  for (int j = 0; j < NP; ++j) e2[j] = fmaxf(e2[j], kTinyNorm2);
  const float inv_parts = 1.f / (float)(G + 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
#pragma unroll 1
  for (int round = 0; round < C::ROUNDS; ++round) {
    const float step = (hi - lo) * inv_parts;
    const float sigma = fmaf(step, (float)(gl + 1), lo);
    const int cnt = sturm_count<NP>(d, e2, 1.f, sigma);
    const unsigned ball = __ballot_sync(TASER_FULL_MASK, cnt == NP);
    const unsigned mine = (ball >> (grp * G)) & gmask;
    if (mine == 0u) {
      lo = fmaf(step, (float)G, lo);
    } else {
      const int f = __ffs(mine) - 1;
      const float nhi = fmaf(step, (float)(f + 1), lo);
      const float nlo = f == 0 ? lo : fmaf(step, (float)f, lo);
      lo = nlo;
      hi = nhi;
    }
  }
  const float nrm = 0.5f * (lo + hi) * pow2f(ex);
  if (active && gl == 0 && TASER_IN(inst, batch)) {
    tau[inst] = nrm > 0.f ? alpha / nrm : 0.f;
    if (nrm_out != nullptr) nrm_out[inst] = nrm;
    TASER_FINITE(nrm);
  }
}

// Folded layout of the complex Householder for UV = 8 and 16: G = UV / 2 lanes per
// instance (four instances per warp at UV = 16, eight at UV = 8).  Lane gl holds two
// columns, ca = gl + 1 (1..UV/2) and cb = UV - gl (UV/2 + 1..UV).  The per-step scalar work
// (reductions, reflector scalars, selects) is then shared by twice as many instances as in
// the one-column layout, and one shared-memory read of v and w serves both columns.  From
// step UV/2 on every ca column is finished, and those blocks drop it at compile time.  The
// multisection evaluates one point per lane, G + 1 parts per round.  Measured at QPSK
// 128x16: 0.183 -> 0.135 ms per 65,536 matrices (128 registers, 4 blocks per SM; at 3
// blocks and 138 registers 0.150 ms; with 5 blocks and spills 0.155 ms; Householder blocks
// of 1 or 4 steps 0.158 and 0.144 ms).
template <int UV>
struct HermFoldCfg {
  static constexpr int HALF = UV / 2;
  static constexpr int G = HALF;               // lanes per instance
  static constexpr int IPW = 32 / G;           // instances per warp
  static constexpr int NP = UV + 1;
  static constexpr int VB = (NP + 1) & ~1;
  static constexpr int WARPS = 4;
  static constexpr int IPC = WARPS * IPW;
  static constexpr int INST_FLOATS = 8 * VB + 2 * VB;  // xd, wd ({re, re, im, im}), db, eb2
  // One point a lane, G + 1 parts per round: 9^7 = 4.8e6 at UV = 16, 5^12 = 2.4e8 at UV = 8.
  static constexpr int ROUNDS = UV == 16 ? 7 : 12;
};

template <int UV, bool NEG>
__global__ void __launch_bounds__(128, 4)
spectral_herm_fold_kernel(int64_t batch, int U, const float* __restrict__ Tt, float alpha, float* __restrict__ tau,
                          float* __restrict__ nrm_out) {
  using C = HermFoldCfg<UV>;
  constexpr int NP = C::NP, VB = C::VB, G = C::G, HALF = C::HALF;
  static_assert(HALF % KBLK_HERM == 0, "a Householder block must not straddle step UV / 2");
  static_assert(HALF >= 2, "the trailing 2 x 2 block sits in the cb columns");
  __shared__ __align__(16) float sm[C::IPC * C::INST_FLOATS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int local = warp * C::IPW + grp;
  const int64_t inst = (int64_t)blockIdx.x * C::IPC + local;
  const bool active = inst < batch;
  float4* xd = reinterpret_cast<float4*>(sm + local * C::INST_FLOATS);
  float4* wd = xd + VB;
  float* db = reinterpret_cast<float*>(wd + VB);
  float* eb2 = db + VB;
  const int ca = gl + 1, cb = UV - gl;
  float2 colA[NP], colB[NP];
  float m00 = 0.f;
  auto load = [&](auto u_c) {
    const int Uc = u_c, N = 2 * Uc + 1;
    const float* T = Tt + (active ? inst : 0) * (int64_t)N * N;
    auto t = [&](int a, int b) -> float {
      const float v = active && TASER_IN(inst * N * N + a * N + b, batch * N * N) ? T[a * N + b] : 0.f;
      return NEG ? -v : v;
    };
    // M~[j][c] as in the one-column layout: users below min(UV, Uc), the augmented
    // coordinate at index UV.
    auto entry = [&](int j, int c) -> float2 {
      const bool ju = j < UV && j < Uc, ja = j == UV;
      const bool cu = c < UV && c < Uc, cx = c == UV;
      if (ju && cu) return make_float2(t(j, c), t(Uc + j, c));
      if (ju && cx) return make_float2(t(j, 2 * Uc), t(Uc + j, 2 * Uc));
      if (ja && cu) return make_float2(t(c, 2 * Uc), -t(Uc + c, 2 * Uc));
      if (ja && cx) return make_float2(t(2 * Uc, 2 * Uc), 0.f);
      return make_float2(0.f, 0.f);
    };
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      colA[j] = entry(j, ca);
      colB[j] = entry(j, cb);
    }
    m00 = Uc >= 1 ? t(0, 0) : 0.f;
  };
  if (U == UV) load(SpecInt<UV>{});
  else load(U);
  float amax = fabsf(m00);
#pragma unroll
  for (int j = 0; j < NP; ++j)
    amax = fmaxf(fmaxf(amax, fmaxf(fabsf(colA[j].x), fabsf(colA[j].y))),
                 fmaxf(fabsf(colB[j].x), fabsf(colB[j].y)));
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TASER_FULL_MASK, amax, o));
  const int ex = scale_exponent(amax);
  {
    const float sc = pow2f(-ex);
    m00 *= sc;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      colA[j] = make_float2(colA[j].x * sc, colA[j].y * sc);
      colB[j] = make_float2(colB[j].x * sc, colB[j].y * sc);
    }
  }
  for (int i = gl; i < VB; i += G) {
    xd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    wd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (gl == 0) db[0] = m00;
  __syncwarp();

  static_for_blocks<UV, KBLK_HERM>([&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    constexpr int KE = (KB + KBLK_HERM < UV - 1) ? KB + KBLK_HERM : UV - 1;   // k in [KB, KE)
    constexpr bool LIVE_A = KB < HALF;   // k < UV / 2 throughout the block: some ca > k
#pragma unroll 1
    for (int k = KB; k < KE; ++k) {
      // Row k of both columns: x_c = conj(M[k][c]) for c > k.  ckA also gives the diagonal
      // M[k][k] when ca == k (k <= UV / 2).
      float2 ckA = make_float2(0.f, 0.f), ckB = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = KB; r < KE; ++r) {
        ckA = (r == k) ? colA[r] : ckA;
        ckB = (r == k) ? colB[r] : ckB;
      }
      const bool liveA = LIVE_A && ca > k, liveB = cb > k;
      const float2 xcA = make_float2(ckA.x, -ckA.y), xcB = make_float2(ckB.x, -ckB.y);
      float sig2 = (liveA ? fmaf(ckA.x, ckA.x, ckA.y * ckA.y) : 0.f) + (liveB ? fmaf(ckB.x, ckB.x, ckB.y * ckB.y) : 0.f);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sig2 += __shfl_xor_sync(TASER_FULL_MASK, sig2, o);
      // x_{k+1}: column k + 1 is ca of lane k (k + 1 <= UV / 2) or cb of lane UV - 1 - k.
      const bool x1_in_a = k + 1 <= HALF;
      const int src = grp * G + (x1_in_a ? k : UV - 1 - k);
      const float sx = x1_in_a ? xcA.x : xcB.x, sy = x1_in_a ? xcA.y : xcB.y;
      const float2 x1 = make_float2(__shfl_sync(TASER_FULL_MASK, sx, src), __shfl_sync(TASER_FULL_MASK, sy, src));
      const bool refl = sig2 >= kTinyNorm2;
      const float sig = refl ? sig2 * rsqrtf(sig2) : 0.f;
      const float n1 = fmaf(x1.x, x1.x, x1.y * x1.y);
      const bool big1 = n1 >= kTinyNorm2;
      const float r1 = big1 ? rsqrtf(n1) : 0.f;
      const float2 ph = big1 ? make_float2(x1.x * r1, x1.y * r1) : make_float2(1.f, 0.f);
      const float ax1 = big1 ? n1 * r1 : x1.x;
      const float2 v1 = make_float2(fmaf(ph.x, sig, x1.x), fmaf(ph.y, sig, x1.y));
      const float vv2 = 2.f * sig * (sig + ax1);
      const float beta = refl ? __fdividef(2.f, vv2) : 0.f;
      const float2 vcA = liveA ? (ca == k + 1 ? v1 : xcA) : make_float2(0.f, 0.f);
      const float2 vcB = liveB ? (cb == k + 1 ? v1 : xcB) : make_float2(0.f, 0.f);
      if (LIVE_A && TASER_IN(ca, VB)) xd[ca] = make_float4(vcA.x, vcA.x, vcA.y, vcA.y);
      if (TASER_IN(cb, VB)) xd[cb] = make_float4(vcB.x, vcB.x, vcB.y, vcB.y);
      if (ca == k && TASER_IN(k, VB)) db[k] = ckA.x;
      if (cb == k && TASER_IN(k, VB)) db[k] = ckB.x;
      __syncwarp();
      uint64_t AA = 0ull, AB = 0ull, BA = 0ull, BB = 0ull;
#pragma unroll
      for (int j = KB + 1; j < NP; ++j) {
        const float4 q = xd[j];
        const uint64_t X1 = f2pack(q.x, q.y), X2 = f2pack(q.z, q.w);
        if constexpr (LIVE_A) {
          const uint64_t Ma = f2pack(colA[j].x, colA[j].y);
          AA = f2fma(Ma, X1, AA);
          AB = f2fma(Ma, X2, AB);
        }
        const uint64_t Mb = f2pack(colB[j].x, colB[j].y);
        BA = f2fma(Mb, X1, BA);
        BB = f2fma(Mb, X2, BB);
      }
      float2 pA = make_float2(0.f, 0.f), pB;
      if constexpr (LIVE_A) {
        float ax, ay, bx, by;
        f2unpack(AA, ax, ay);
        f2unpack(AB, bx, by);
        pA = liveA ? make_float2(beta * (ax + by), beta * (bx - ay)) : make_float2(0.f, 0.f);
      }
      {
        float ax, ay, bx, by;
        f2unpack(BA, ax, ay);
        f2unpack(BB, bx, by);
        pB = liveB ? make_float2(beta * (ax + by), beta * (bx - ay)) : make_float2(0.f, 0.f);
      }
      float kk = fmaf(vcA.x, pA.x, vcA.y * pA.y) + fmaf(vcB.x, pB.x, vcB.y * pB.y);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) kk += __shfl_xor_sync(TASER_FULL_MASK, kk, o);
      kk *= 0.5f * beta;
      const float2 wA = make_float2(fmaf(-kk, vcA.x, pA.x), fmaf(-kk, vcA.y, pA.y));
      const float2 wB = make_float2(fmaf(-kk, vcB.x, pB.x), fmaf(-kk, vcB.y, pB.y));
      if (LIVE_A && TASER_IN(ca, VB)) wd[ca] = make_float4(wA.x, wA.x, wA.y, wA.y);
      if (TASER_IN(cb, VB)) wd[cb] = make_float4(wB.x, wB.x, wB.y, wB.y);
      if (gl == 0 && TASER_IN(k, VB)) eb2[k] = sig2;                                  // |alpha|^2
      __syncwarp();
      const uint64_t nWaA = f2pack(-wA.x, wA.y), nWbA = f2pack(-wA.y, -wA.x);
      const uint64_t nVaA = f2pack(-vcA.x, vcA.y), nVbA = f2pack(-vcA.y, -vcA.x);
      const uint64_t nWaB = f2pack(-wB.x, wB.y), nWbB = f2pack(-wB.y, -wB.x);
      const uint64_t nVaB = f2pack(-vcB.x, vcB.y), nVbB = f2pack(-vcB.y, -vcB.x);
#pragma unroll
      for (int j = KB + 1; j < NP; ++j) {
        const float4 q = xd[j], u = wd[j];
        const uint64_t Q1 = f2pack(q.x, q.y), Q2 = f2pack(q.z, q.w), U1 = f2pack(u.x, u.y), U2 = f2pack(u.z, u.w);
        if constexpr (LIVE_A) {
          uint64_t Ma = f2pack(colA[j].x, colA[j].y);
          Ma = f2fma(Q1, nWaA, Ma);
          Ma = f2fma(Q2, nWbA, Ma);
          Ma = f2fma(U1, nVaA, Ma);
          Ma = f2fma(U2, nVbA, Ma);
          f2unpack(Ma, colA[j].x, colA[j].y);
        }
        uint64_t Mb = f2pack(colB[j].x, colB[j].y);
        Mb = f2fma(Q1, nWaB, Mb);
        Mb = f2fma(Q2, nWbB, Mb);
        Mb = f2fma(U1, nVaB, Mb);
        Mb = f2fma(U2, nVbB, Mb);
        f2unpack(Mb, colB[j].x, colB[j].y);
      }
      __syncwarp();
    }
  });
  // Trailing 2 x 2 block: columns UV - 1 and UV are cb of lanes 1 and 0.
  if (cb == UV - 1) {
    db[UV - 1] = colB[UV - 1].x;
    eb2[UV - 1] = fmaf(colB[UV].x, colB[UV].x, colB[UV].y * colB[UV].y);
  }
  if (cb == UV) db[UV] = colB[UV].x;
  __syncwarp();
  float d[NP], e2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d[j] = db[j];
    e2[j] = j < UV ? eb2[j] : 0.f;
  }
  float lo = -3.0e38f, hi = -3.0e38f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float r = (j > 0 ? sqrtf(e2[j - 1]) : 0.f) + sqrtf(e2[j]);
    lo = fmaxf(lo, d[j]);
    hi = fmaxf(hi, d[j] + r);
  }
  // The Sturm count needs e2 > 0; the floor comes after the bracket, which it must not
  // widen (the zero matrix keeps the norm 0).
#pragma unroll
  for (int j = 0; j < NP; ++j) e2[j] = fmaxf(e2[j], kTinyNorm2);
  // One-sided multisection, G + 1 parts: lane gl evaluates the point sigma = lo + (gl + 1) step.
  // (Two points a lane over UV + 1 parts, 5 rounds, were 1.5% slower at UV = 16.)
  const float inv_parts = 1.f / (float)(G + 1);
  const unsigned gmask = (1u << G) - 1u;
#pragma unroll 1
  for (int round = 0; round < C::ROUNDS; ++round) {
    const float step = (hi - lo) * inv_parts;
    const float sigma = fmaf(step, (float)(gl + 1), lo);
    const int cnt = sturm_count<NP>(d, e2, 1.f, sigma);
    const unsigned mine = (__ballot_sync(TASER_FULL_MASK, cnt == NP) >> (grp * G)) & gmask;
    const int f = mine ? __ffs(mine) - 1 : G;   // first point at or above lambda_max
    if (f == G) {
      lo = fmaf(step, (float)G, lo);
    } else {
      const float nhi = fmaf(step, (float)(f + 1), lo);
      const float nlo = f == 0 ? lo : fmaf(step, (float)f, lo);
      lo = nlo;
      hi = nhi;
    }
  }
  const float nrm = 0.5f * (lo + hi) * pow2f(ex);
  if (active && gl == 0 && TASER_IN(inst, batch)) {
    tau[inst] = nrm > 0.f ? alpha / nrm : 0.f;
    if (nrm_out != nullptr) nrm_out[inst] = nrm;
    TASER_FINITE(nrm);
  }
}

template <int UV>
static cudaError_t launch_herm(int64_t batch, int U, const float* Tt, bool neg, float alpha, float* tau,
                               float* nrm, cudaStream_t st) {
  if constexpr (UV <= 16) {
    const int64_t blocks = (batch + HermFoldCfg<UV>::IPC - 1) / HermFoldCfg<UV>::IPC;
    if (neg) spectral_herm_fold_kernel<UV, true><<<(unsigned)blocks, 128, 0, st>>>(batch, U, Tt, alpha, tau, nrm);
    else spectral_herm_fold_kernel<UV, false><<<(unsigned)blocks, 128, 0, st>>>(batch, U, Tt, alpha, tau, nrm);
  } else {
    // UV = 32: two columns a lane would need about 130 registers for the matrix alone.
    const int64_t blocks = (batch + HermCfg<UV>::IPC - 1) / HermCfg<UV>::IPC;
    if (neg) spectral_herm_kernel<UV, true><<<(unsigned)blocks, 128, 0, st>>>(batch, U, Tt, alpha, tau, nrm);
    else spectral_herm_kernel<UV, false><<<(unsigned)blocks, 128, 0, st>>>(batch, U, Tt, alpha, tau, nrm);
  }
  return cudaGetLastError();
}

// ||T~||_2 of QPSK matrices (N = 2U + 1) through the complex form; U <= 32.  sign = +1 for
// a positive semidefinite T~ (MIMO), -1 for a negative semidefinite one (JED).
cudaError_t spectral_qpsk(int64_t batch, int U, const float* Tt, int sign, float alpha, float* tau, float* nrm,
                          cudaStream_t st) {
  const bool neg = sign < 0;
  if (U + 1 <= 9) return launch_herm<8>(batch, U, Tt, neg, alpha, tau, nrm, st);
  if (U + 1 <= 17) return launch_herm<16>(batch, U, Tt, neg, alpha, tau, nrm, st);
  return launch_herm<32>(batch, U, Tt, neg, alpha, tau, nrm, st);
}

// Folded layout of the real Householder for NV = 8, 16 and 32: G = NV / 2 lanes per
// instance (two instances per warp at NV = 32, four at 16, eight at 8).  Lane gl holds
// columns ca = gl + 1 and cb = NV - gl as one packed pair (A[j][ca], A[j][cb]); v and w are
// published as duplicated pairs (x_j, x_j), so one packed multiply-add per row serves both
// columns of the reduction p = beta A v and two serve their rank-2 update.  A finished
// column (c <= k) has v_c = w_c = 0 and its updates add zero.
// The multisection keeps the one-column kernel's structure: one-sided, each lane evaluates
// two of NV points (NV + 1 parts); two-sided, one point on each side (G + 1 parts a side).
// Measured per 131,072 JED BPSK matrices (B = 16): K = 16 0.394 -> 0.189 ms, K = 32 0.988 ->
// 0.939 ms; per 65,536 BPSK 32x8 0.095 -> 0.029 ms.  At NV = 32 the 128-register bound
// spills a little and is still faster than 152 registers at 3 blocks per SM.
template <int NV>
struct SpecFoldCfg {
  static constexpr int HALF = NV / 2;
  static constexpr int G = HALF;                  // lanes per instance
  static constexpr int IPW = 32 / G;              // instances per warp
  static constexpr int NP = NV + 1;               // padded order
  static constexpr int VB = ((NP + 3) / 4) * 4;   // pair vectors padded to 16-byte pairs of rows
  static constexpr int WARPS = 4;
  static constexpr int IPC = WARPS * IPW;
  static constexpr int INST_FLOATS = 2 * VB + 2 * VB + 2 * VB;   // xd, wd (pairs), d, e
  // Resolution (parts^rounds) of the one-sided search: 33^5 = 3.9e7, 17^6 = 2.4e7,
  // 9^8 = 4.3e7; of the two-sided one: 17^7 = 4.1e8, 9^9 = 3.9e8, 5^12 = 2.4e8.
  static constexpr int ROUNDS1 = NV == 32 ? 5 : (NV == 16 ? 6 : 8);
  static constexpr int ROUNDS2 = NV == 32 ? 7 : (NV == 16 ? 9 : 12);
};

template <int NV>
__global__ void __launch_bounds__(128, 4)
spectral_fold_kernel(int64_t batch, int N, const float* __restrict__ Tt, float alpha, int sign_hint,
                     float* __restrict__ tau, float* __restrict__ nrm_out) {
  using C = SpecFoldCfg<NV>;
  constexpr int NP = C::NP, VB = C::VB, G = C::G, HALF = C::HALF;
  __shared__ __align__(16) float sm[C::IPC * C::INST_FLOATS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane % G;
  const int local = warp * C::IPW + grp;
  const int64_t inst = (int64_t)blockIdx.x * C::IPC + local;
  const bool active = inst < batch;
  float2* xd = reinterpret_cast<float2*>(sm + local * C::INST_FLOATS);
  float2* wd = xd + VB;
  float* db = reinterpret_cast<float*>(wd + VB);
  float* eb = db + VB;
  const int ca = gl + 1, cb = NV - gl;
  const float* T = Tt + (active ? inst : 0) * (int64_t)N * N;
  auto a_rc = [&](int r, int c) -> float {
    return active && r < N && c < N && TASER_IN(inst * N * N + r * N + c, batch * N * N) ? T[(int64_t)r * N + c] : 0.f;
  };
  uint64_t cab[NP];
  float amax;
  float d0 = a_rc(0, 0);
  {
    float ma = fabsf(d0);
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      const float x = a_rc(r, ca), y = a_rc(r, cb);
      ma = fmaxf(ma, fmaxf(fabsf(x), fabsf(y)));
      cab[r] = f2pack(x, y);
    }
    amax = ma;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(TASER_FULL_MASK, amax, o));
  const int ex = scale_exponent(amax);
  {
    const float sc = pow2f(-ex);
    const uint64_t sc2 = f2pack(sc, sc);
    d0 *= sc;
#pragma unroll
    for (int r = 0; r < NP; ++r) cab[r] = f2mul(cab[r], sc2);
  }
  for (int i = gl; i < VB; i += G) {
    xd[i] = make_float2(0.f, 0.f);
    wd[i] = make_float2(0.f, 0.f);
  }
  if (gl == 0) db[0] = d0;
  __syncwarp();

  static_for_blocks<NV, KBLK>([&](auto kb) {
    constexpr int KB = decltype(kb)::value;
    constexpr int KE = (KB + KBLK < NV - 1) ? KB + KBLK : NV - 1;   // k in [KB, KE)
    constexpr int J0 = (KB + 1) & ~1;                                 // rows read in pairs
#pragma unroll 1
    for (int k = KB; k < KE; ++k) {
      // Row k of both columns: x_c = A[k][c] for c > k (A symmetric).
      uint64_t ckp = 0ull;
#pragma unroll
      for (int r = KB; r < KE; ++r) ckp = (r == k) ? cab[r] : ckp;
      float ckA, ckB;
      f2unpack(ckp, ckA, ckB);
      const bool liveA = ca > k, liveB = cb > k;
      float sig2 = (liveA ? ckA * ckA : 0.f) + (liveB ? ckB * ckB : 0.f);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sig2 += __shfl_xor_sync(TASER_FULL_MASK, sig2, o);
      // x_{k+1}: column k + 1 is ca of lane k (k + 1 <= NV / 2) or cb of lane NV - 1 - k.
      const bool x1_in_a = k + 1 <= HALF;
      const float x1 = __shfl_sync(TASER_FULL_MASK, x1_in_a ? ckA : ckB, grp * G + (x1_in_a ? k : NV - 1 - k));
      // Reflector H = I - beta v v^T, v = x - ah e_{k+1}, ah = -sign(x_{k+1}) ||x||.
      const bool refl = sig2 >= kTinyNorm2;
      const float sig = refl ? sig2 * rsqrtf(sig2) : 0.f;
      const float ah = x1 >= 0.f ? -sig : sig;
      const float vv2 = 2.f * (sig2 + sig * fabsf(x1));
      const float beta = refl ? __fdividef(2.f, vv2) : 0.f;
      const float vA = liveA ? (ca == k + 1 ? ckA - ah : ckA) : 0.f;
      const float vB = liveB ? (cb == k + 1 ? ckB - ah : ckB) : 0.f;
      if (TASER_IN(ca, VB)) xd[ca] = make_float2(vA, vA);
      if (TASER_IN(cb, VB)) xd[cb] = make_float2(vB, vB);
      if (ca == k && TASER_IN(k, VB)) db[k] = ckA;
      if (cb == k && TASER_IN(k, VB)) db[k] = ckB;
      __syncwarp();
      // (p_ca, p_cb) = beta sum_j (A[j][ca], A[j][cb]) v_j.
      uint64_t acc = 0ull;
#pragma unroll
      for (int j = J0; j < NP; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(xd + j);   // rows j, j + 1
        acc = f2fma(cab[j], f2pack(q.x, q.y), acc);
        if (j + 1 < NP) acc = f2fma(cab[j + 1], f2pack(q.z, q.w), acc);
      }
      float pA, pB;
      f2unpack(acc, pA, pB);
      pA = liveA ? beta * pA : 0.f;
      pB = liveB ? beta * pB : 0.f;
      float kk = fmaf(vA, pA, vB * pB);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) kk += __shfl_xor_sync(TASER_FULL_MASK, kk, o);
      kk *= 0.5f * beta;
      const float wA = fmaf(-kk, vA, pA), wB = fmaf(-kk, vB, pB);
      if (TASER_IN(ca, VB)) wd[ca] = make_float2(wA, wA);
      if (TASER_IN(cb, VB)) wd[cb] = make_float2(wB, wB);
      if (gl == 0 && TASER_IN(k, VB)) eb[k] = ah;
      __syncwarp();
      // A <- A - v w^T - w v^T on the lane's two columns.
      const uint64_t nw = f2pack(-wA, -wB), nv = f2pack(-vA, -vB);
#pragma unroll
      for (int j = J0; j < NP; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(xd + j);
        const float4 u = *reinterpret_cast<const float4*>(wd + j);
        cab[j] = f2fma(f2pack(q.x, q.y), nw, f2fma(f2pack(u.x, u.y), nv, cab[j]));
        if (j + 1 < NP) cab[j + 1] = f2fma(f2pack(q.z, q.w), nw, f2fma(f2pack(u.z, u.w), nv, cab[j + 1]));
      }
      __syncwarp();
    }
  });
  // Trailing 2 x 2 block: columns NV - 1 and NV are cb of lanes 1 and 0.
  {
    float bl, bn, al_unused;
    f2unpack(cab[NV - 1], al_unused, bl);
    float an_unused;
    f2unpack(cab[NV], an_unused, bn);
    (void)al_unused;
    (void)an_unused;
    if (cb == NV - 1) {
      db[NV - 1] = bl;
      eb[NV - 1] = bn;
    }
    if (cb == NV) db[NV] = bn;
  }
  __syncwarp();
  float d[NP], e2[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    d[j] = db[j];
    e2[j] = j < NV ? eb[j] * eb[j] : 0.f;
  }
  // Multisection.  One-sided: sg = the hint's sign, points 2 gl and 2 gl + 1 of NV.
  // Two-sided (hint 0): the point gl of lambda_max(A) and the point gl of lambda_max(-A).
  const bool two = sign_hint == 0;
  const float sg0 = two ? 1.f : (sign_hint > 0 ? 1.f : -1.f);
  const float sg1 = two ? -1.f : sg0;
  const int parts = two ? G + 1 : NV + 1;
  const int rounds = two ? C::ROUNDS2 : C::ROUNDS1;
  // Bracket per side: [max sg d_j, max (sg d_j + |e_{j-1}| + |e_j|)].
  float lo0 = -3.0e38f, hi0 = -3.0e38f, lo1 = -3.0e38f, hi1 = -3.0e38f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float r = (j > 0 ? sqrtf(e2[j - 1]) : 0.f) + sqrtf(e2[j]);
    lo0 = fmaxf(lo0, sg0 * d[j]);
    hi0 = fmaxf(hi0, sg0 * d[j] + r);
    lo1 = fmaxf(lo1, sg1 * d[j]);
    hi1 = fmaxf(hi1, sg1 * d[j] + r);
  }
  // The Sturm count needs e2 > 0; the floor comes after the bracket, which it must not
  // widen (the zero matrix keeps the norm 0).
#pragma unroll
  for (int j = 0; j < NP; ++j) e2[j] = fmaxf(e2[j], kTinyNorm2);
  const float inv_parts = 1.f / (float)parts;
  const unsigned gmask = (1u << G) - 1u;
  // index of the point of lane gl on each side: one-sided 2 gl and 2 gl + 1, two-sided gl
  const int p0 = two ? gl : 2 * gl, p1 = two ? gl : 2 * gl + 1;
#pragma unroll 1
  for (int round = 0; round < rounds; ++round) {
    const float st0 = (hi0 - lo0) * inv_parts, st1 = (hi1 - lo1) * inv_parts;
    const float s0 = fmaf(st0, (float)(p0 + 1), lo0);
    const float s1 = two ? fmaf(st1, (float)(p1 + 1), lo1) : fmaf(st0, (float)(p1 + 1), lo0);
    const int c0 = sturm_count<NP>(d, e2, sg0, s0);
    const int c1 = sturm_count<NP>(d, e2, sg1, s1);
    const unsigned m0 = (__ballot_sync(TASER_FULL_MASK, c0 == NP) >> (grp * G)) & gmask;
    const unsigned m1 = (__ballot_sync(TASER_FULL_MASK, c1 == NP) >> (grp * G)) & gmask;
    if (two) {
      // each side: first of its G points at or above its lambda_max
      if (m0 == 0u) {
        lo0 = fmaf(st0, (float)G, lo0);
      } else {
        const int f = __ffs(m0) - 1;
        const float nhi = fmaf(st0, (float)(f + 1), lo0);
        lo0 = f == 0 ? lo0 : fmaf(st0, (float)f, lo0);
        hi0 = nhi;
      }
      if (m1 == 0u) {
        lo1 = fmaf(st1, (float)G, lo1);
      } else {
        const int f = __ffs(m1) - 1;
        const float nhi = fmaf(st1, (float)(f + 1), lo1);
        lo1 = f == 0 ? lo1 : fmaf(st1, (float)f, lo1);
        hi1 = nhi;
      }
    } else {
      // one side, points interleaved over the lanes: p = 2 gl (m0) and 2 gl + 1 (m1)
      const int f0 = m0 ? 2 * (__ffs(m0) - 1) : 2 * G;
      const int f1 = m1 ? 2 * (__ffs(m1) - 1) + 1 : 2 * G;
      const int f = min(f0, f1);
      if (f == 2 * G) {
        lo0 = fmaf(st0, (float)(2 * G), lo0);
      } else {
        const float nhi = fmaf(st0, (float)(f + 1), lo0);
        lo0 = f == 0 ? lo0 : fmaf(st0, (float)f, lo0);
        hi0 = nhi;
      }
    }
  }
  float nrm = 0.5f * (lo0 + hi0);
  if (two) nrm = fmaxf(nrm, 0.5f * (lo1 + hi1));
  nrm *= pow2f(ex);
  if (active && gl == 0 && TASER_IN(inst, batch)) {
    tau[inst] = nrm > 0.f ? alpha / nrm : 0.f;
    if (nrm_out != nullptr) nrm_out[inst] = nrm;
    TASER_FINITE(nrm);
  }
}

template <int NV>
static cudaError_t launch_spectral(int64_t batch, int N, const float* Tt, float alpha, int hint, float* tau,
                                   float* nrm, cudaStream_t st) {
  if constexpr (NV <= 32) {
    const int64_t blocks = (batch + SpecFoldCfg<NV>::IPC - 1) / SpecFoldCfg<NV>::IPC;
    spectral_fold_kernel<NV><<<(unsigned)blocks, 128, 0, st>>>(batch, N, Tt, alpha, hint, tau, nrm);
  } else {
    // NV = 64: two columns a lane already (S = 2); a fold would need 4.
    const int64_t blocks = (batch + SpecCfg<NV>::WARPS - 1) / SpecCfg<NV>::WARPS;
    spectral_kernel<NV><<<(unsigned)blocks, 32 * SpecCfg<NV>::WARPS, 0, st>>>(batch, N, Tt, alpha, hint, tau, nrm);
  }
  return cudaGetLastError();
}

cudaError_t spectral(int64_t batch, int N, const float* Tt, float alpha, int hint, float* tau, float* nrm,
                     cudaStream_t st) {
  switch (bucket_of(N)) {
    case 8: return launch_spectral<8>(batch, N, Tt, alpha, hint, tau, nrm, st);
    case 16: return launch_spectral<16>(batch, N, Tt, alpha, hint, tau, nrm, st);
    case 32: return launch_spectral<32>(batch, N, Tt, alpha, hint, tau, nrm, st);
    default: return launch_spectral<64>(batch, N, Tt, alpha, hint, tau, nrm, st);
  }
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(spectral)
