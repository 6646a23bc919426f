// ||T~||_2 and the step size tau = alpha / ||T~||_2 (Sec. III-B; inputs of Algorithm 1).
//
// ||T~||_2 of a symmetric matrix is its largest |eigenvalue|.  A power iteration is not
// used: on MU-MIMO matrices the two largest eigenvalues are often close and hundreds of
// steps still leave errors of 1e-3.  Instead each warp reduces one T~ to tridiagonal form
// with Householder reflections (FP32, backward stable) and then finds the extreme
// eigenvalues of the tridiagonal matrix by Sturm-count multisection: lanes 0..15 bracket
// lambda_max(T~), lanes 16..31 bracket lambda_max(-T~), each round splitting the bracket
// into 17 parts.
//
// Layout: T~ is embedded in an (NV+1) x (NV+1) matrix with zero padding (zero rows and
// columns add zero eigenvalues, which do not change ||T~||_2 since ||T~||_2 >= 0).  The
// first reflection eliminates column 0, leaving an NV x NV trailing matrix whose column
// c (1..NV) lives in the registers of lane (c-1) mod 32.
#include "common.cuh"

namespace taser {

template <int NV>
struct SpecCfg {
  static constexpr int S = NV > 32 ? NV / 32 : 1;  // columns per lane
  static constexpr int NP = NV + 1;                // padded order
  static constexpr int VB = ((NP + 3) / 4) * 4;    // padded vector length (16B rows)
  static constexpr int WARPS = 4;
  static constexpr int WARP_FLOATS = 2 * VB + 2 * VB;  // x, w, d, e
  static constexpr int ROUNDS = 7;                 // 17^7 > 4e8: ~fp32 resolution
};

template <int NV>
__global__ void __launch_bounds__(128)
spectral_kernel(int64_t batch, int N, const float* __restrict__ Tt, float alpha, float* __restrict__ tau,
                float* __restrict__ nrm_out) {
  using C = SpecCfg<NV>;
  constexpr int S = C::S, NP = C::NP;
  __shared__ __align__(16) float sm[C::WARPS * C::WARP_FLOATS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp;
  if (inst >= batch) return;
  float* xb = sm + warp * C::WARP_FLOATS;
  float* wb = xb + C::VB;
  float* db = wb + C::VB;
  float* eb = db + C::VB;

  const float* T = Tt + inst * (int64_t)N * N;
  // col[s][r] = A[r][c_s], c_s = lane + 1 + 32 s.
  float col[S][NP];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int c = lane + 1 + 32 * s;
#pragma unroll
    for (int r = 0; r < NP; ++r) col[s][r] = (r < N && c < N) ? T[(int64_t)r * N + c] : 0.f;
  }
  const float d0 = T[0];
  for (int i = lane; i < C::VB; i += 32) {
    xb[i] = 0.f;
    wb[i] = 0.f;
  }
  __syncwarp();

#pragma unroll
  for (int k = 0; k + 2 <= NV; ++k) {
    // Publish column k on and below the diagonal: xb[j] = A[j][k] = A[k][j], j >= k.
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int c = lane + 1 + 32 * s;
      if (c <= NV) xb[c] = (c >= k) ? col[s][k] : 0.f;
    }
    if (lane == 0) xb[0] = (k == 0) ? d0 : 0.f;
    __syncwarp();
    const float dk = xb[k];
    const float x1 = xb[k + 1];
    float sig2 = 0.f;
#pragma unroll
    for (int j = k + 1; j < NP; ++j) sig2 = fmaf(xb[j], xb[j], sig2);
    const float sig = sqrtf(sig2);
    const float ah = x1 >= 0.f ? -sig : sig;             // new subdiagonal entry
    const float vv2 = 2.f * (sig2 + sig * fabsf(x1));    // ||v||^2, v = x - ah e_{k+1}
    const float beta = vv2 > 0.f ? 2.f / vv2 : 0.f;
    const float v1 = x1 - ah;
    // p_i = beta sum_j A[j][i] v_j for this lane's columns i > k.
    float p[S], vi[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int c = lane + 1 + 32 * s;
      float acc = col[s][k + 1] * v1;
#pragma unroll
      for (int j = k + 2; j < NP; ++j) acc = fmaf(col[s][j], xb[j], acc);
      const bool live = c > k && c <= NV;
      p[s] = live ? beta * acc : 0.f;
      vi[s] = live ? (c == k + 1 ? v1 : xb[c]) : 0.f;
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
      if (c <= NV) wb[c] = w[s];
    }
    if (lane == 0) {
      db[k] = dk;
      eb[k] = ah;
    }
    __syncwarp();
    // A <- A - v w^T - w v^T on the trailing block (rows j > k of this lane's columns).
#pragma unroll
    for (int s = 0; s < S; ++s) {
      col[s][k + 1] = fmaf(-v1, w[s], fmaf(-wb[k + 1], vi[s], col[s][k + 1]));
#pragma unroll
      for (int j = k + 2; j < NP; ++j) col[s][j] = fmaf(-xb[j], w[s], fmaf(-wb[j], vi[s], col[s][j]));
    }
    __syncwarp();
  }
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

  // Sturm multisection on the tridiagonal (d, e): half 0 -> lambda_max(A), half 1 ->
  // lambda_max(-A).
  const float sg = lane < 16 ? 1.f : -1.f;
  const int l = lane & 15;
  float lo = -3.0e38f, hi = -3.0e38f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float dj = sg * db[j];
    const float r = (j > 0 ? fabsf(eb[j - 1]) : 0.f) + (j < NV ? fabsf(eb[j]) : 0.f);
    lo = fmaxf(lo, dj);
    hi = fmaxf(hi, dj + r);
  }
  const float pivmin = 1e-30f;
#pragma unroll 1
  for (int round = 0; round < C::ROUNDS; ++round) {
    const float step = (hi - lo) * (1.f / 17.f);
    const float sigma = fmaf(step, (float)(l + 1), lo);
    float q = sg * db[0] - sigma;
    int cnt = q < 0.f;
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      if (fabsf(q) < pivmin) q = -pivmin;
      q = (sg * db[j] - sigma) - __fdividef(eb[j - 1] * eb[j - 1], q);
      cnt += q < 0.f;
    }
    const unsigned ball = __ballot_sync(TASER_FULL_MASK, cnt == NP);
    const unsigned half = lane < 16 ? (ball & 0xffffu) : (ball >> 16);
    if (half == 0u) {
      lo = fmaf(step, 16.f, lo);
    } else {
      const int f = __ffs(half) - 1;
      const float nhi = fmaf(step, (float)(f + 1), lo);
      const float nlo = f == 0 ? lo : fmaf(step, (float)f, lo);
      lo = nlo;
      hi = nhi;
    }
  }
  const float lam = 0.5f * (lo + hi);
  const float nrm = fmaxf(lam, __shfl_xor_sync(TASER_FULL_MASK, lam, 16));
  if (lane == 0) {
    tau[inst] = nrm > 0.f ? alpha / nrm : 0.f;
    if (nrm_out != nullptr) nrm_out[inst] = nrm;
  }
}

template <int NV>
static cudaError_t launch_spectral(int64_t batch, int N, const float* Tt, float alpha, float* tau, float* nrm,
                                   cudaStream_t st) {
  const int64_t blocks = (batch + SpecCfg<NV>::WARPS - 1) / SpecCfg<NV>::WARPS;
  spectral_kernel<NV><<<(unsigned)blocks, 32 * SpecCfg<NV>::WARPS, 0, st>>>(batch, N, Tt, alpha, tau, nrm);
  return cudaGetLastError();
}

cudaError_t spectral(int64_t batch, int N, const float* Tt, float alpha, float* tau, float* nrm,
                     cudaStream_t st) {
  switch (bucket_of(N)) {
    case 8: return launch_spectral<8>(batch, N, Tt, alpha, tau, nrm, st);
    case 16: return launch_spectral<16>(batch, N, Tt, alpha, tau, nrm, st);
    case 32: return launch_spectral<32>(batch, N, Tt, alpha, tau, nrm, st);
    default: return launch_spectral<64>(batch, N, Tt, alpha, tau, nrm, st);
  }
}

}  // namespace taser
